// Type-3 target side (arXiv:2010.05978 Sec. 3.2, eq. nufft3 and step 3):
// for each scattered target, interpolate the FFT of the deconvolved spread
// grid with the exponential-of-semicircle kernel (the inner type-2 NUFFT),
// divide by the kernel's Fourier transform at the target's frequency (the
// type-3 deconvolution), and apply the post-phase exp(-i s.C) of the node
// centring together with the target chirp and 1/(i lz):
//   u_k = 1/(i lz) exp(i pi |xi_k|^2 / lz - 2 pi i xi_k.C / lz) v'_k,
// optionally u^oc = 1 - u^ap (eq. bab).  Phases in FP64 with reduction.
#include "dfloat.cuh"
#include "spread.cuh"

namespace fres {

namespace {

constexpr double kTwoPiHi = 6.28318530717958623199592693709;
constexpr double kTwoPiLo = 2.44929359829470635445e-16;
constexpr double kInvTwoPi = 0.159154943091895335768883763373;

__device__ __forceinline__ double reduce_phase(double ph) {
    double n = rint(ph * kInvTwoPi);
    ph = fma(-n, kTwoPiHi, ph);
    return fma(-n, kTwoPiLo, ph);
}

// psihat(t) for |t| <= t_max from its even Chebyshev series
// sum_k a_k T_{2k}(t / t_max) = sum_k a_k T_k(2 (t/t_max)^2 - 1), by Clenshaw.
template <typename T>
__device__ __forceinline__ T kernel_ft_cheb(T t, const T* a, int n, T inv_tmax) {
    const T x = t * inv_tmax;
    const T y = (T)2 * x * x - (T)1;
    T b1 = 0, b2 = 0;
    for (int k = n - 1; k >= 1; --k) {
        const T b0 = (T)2 * y * b1 - b2 + a[k];
        b2 = b1;
        b1 = b0;
    }
    return y * b1 - b2 + a[0];
}

// Bin of a target: the 16 x 16 block of the FFT grid holding its frequency.
__device__ __forceinline__ int target_bin(double xi, double eta, const InterpParams& ip) {
    double tau1 = (xi - ip.xi_c) * ip.K1, tau2 = (eta - ip.eta_c) * ip.K2;
    if (!(fabs(tau1) <= ip.nfft1) || !(fabs(tau2) <= ip.nfft2)) return 0;
    int c1 = (int)floor(tau1), c2 = (int)floor(tau2);
    if (c1 < 0) c1 += ip.nfft1;
    if (c2 < 0) c2 += ip.nfft2;
    c1 = min(c1, ip.nfft1 - 1);
    c2 = min(c2, ip.nfft2 - 1);
    return (c2 >> 4) * ip.nbin1 + (c1 >> 4);
}

__global__ void k_target_count(const double* __restrict__ targets, long long M, InterpParams ip,
                               int* __restrict__ counts) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        atomicAdd(&counts[target_bin(t.x, t.y, ip)], 1);
    }
}

// One block: exclusive scan of the bin counts into cursors; resets counts.
__global__ void k_target_scan(int nbins, int* counts, int* cursor) {
    __shared__ long long s[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (nbins + nt - 1) / nt;
    const int lo = min(t * per, nbins), hi = min(lo + per, nbins);
    long long sum = 0;
    for (int i = lo; i < hi; ++i) sum += counts[i];
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        long long a = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    long long run = s[t] - sum;
    for (int i = lo; i < hi; ++i) {
        const int c = counts[i];
        cursor[i] = (int)run;
        run += c;
        counts[i] = 0;
    }
}

__global__ void k_target_scatter(const double* __restrict__ targets, long long M, InterpParams ip,
                                 int* __restrict__ cursor, int* __restrict__ perm) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        const int pos = atomicAdd(&cursor[target_bin(t.x, t.y, ip)], 1);
        if (pos >= 0 && pos < M) perm[pos] = (int)k;
    }
}

// Targets are visited in bin order (perm) when a permutation is given, so a
// warp's targets share grid cells in L1; results go to the caller's order.
template <typename T, int W>
__global__ void __launch_bounds__(256)
k_interp(const double* __restrict__ targets, long long M, const cx_t<T>* __restrict__ F,
         InterpParams ip, T beta, const double* __restrict__ cheb, int ncheb,
         cx_t<T>* __restrict__ out, unsigned* __restrict__ status, const HornerTab hz,
         const int* __restrict__ perm) {
    __shared__ T s_a[kMaxCheb];
    for (int i = threadIdx.x; i < ncheb; i += blockDim.x) s_a[i] = (T)cheb[i];
    __syncthreads();
    const T inv_tmax = (T)ip.inv_tmax;
    for (long long kk = blockIdx.x * (long long)blockDim.x + threadIdx.x; kk < M;
         kk += (long long)gridDim.x * blockDim.x) {
        const long long k = perm ? (long long)perm[kk] : kk;
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        int s1, s2;
        T f1, f2, targ1, targ2, phr;
        if constexpr (std::is_same<T, float>::value) {
            // FP32 fast mode: double-float coordinates and phase (no FP64 arithmetic)
            const dflt xi = df_from_double(t.x), eta = df_from_double(t.y);
            if (!(xi.hi >= ip.boxf[0] && xi.hi <= ip.boxf[1] && eta.hi >= ip.boxf[2] &&
                  eta.hi <= ip.boxf[3]))
                atomicOr(status, kStatusTargetOutside);
            dflt g1 = df_add(df_mul(xi, dflt{ip.dK1[0], ip.dK1[1]}), dflt{ip.dG1[0], ip.dG1[1]});
            dflt g2 = df_add(df_mul(eta, dflt{ip.dK2[0], ip.dK2[1]}), dflt{ip.dG2[0], ip.dG2[1]});
            if (!(fabsf(g1.hi) <= (float)ip.nfft1) || !(fabsf(g2.hi) <= (float)ip.nfft2)) {
                atomicOr(status, kStatusNonFinite);
                g1 = g2 = dflt{0.0f, 0.0f};
            }
            int c1, c2;
            df_floor_split(g1, &c1, &f1);
            df_floor_split(g2, &c2, &f2);
            s1 = c1 + 1;
            s2 = c2 + 1;
            // tau = g - (nfft/2 - w/2), exactly in double-float, then scaled
            targ1 = df_add(g1, dflt{-(0.5f * ip.nfft1 - 0.5f * W), 0.0f}).hi * ip.shK1;
            targ2 = df_add(g2, dflt{-(0.5f * ip.nfft2 - 0.5f * W), 0.0f}).hi * ip.shK2;
            const dflt kq = {ip.dkq[0], ip.dkq[1]};
            const dflt q1 = df_mul(xi, df_add(df_mul(kq, xi), dflt{ip.dp1[0], ip.dp1[1]}));
            const dflt q2 = df_mul(eta, df_add(df_mul(kq, eta), dflt{ip.dp2[0], ip.dp2[1]}));
            phr = df_reduce_2pi(df_add(q1, q2));
        } else {
            const double xi = t.x, eta = t.y;
            if (!(xi >= ip.box[0] && xi <= ip.box[1] && eta >= ip.box[2] && eta <= ip.box[3]))
                atomicOr(status, kStatusTargetOutside);
            const double d1 = xi - ip.xi_c, d2 = eta - ip.eta_c;
            double tau1 = d1 * ip.K1, tau2 = d2 * ip.K2;
            if (!isfinite(tau1) || !isfinite(tau2) || fabs(tau1) > ip.nfft1 ||
                fabs(tau2) > ip.nfft2) {
                atomicOr(status, kStatusNonFinite);
                tau1 = tau2 = 0.0;
            }
            const double gs1 = tau1 + 0.5 * ip.nfft1 - 0.5 * W;
            const double gs2 = tau2 + 0.5 * ip.nfft2 - 0.5 * W;
            const double fl1 = floor(gs1), fl2 = floor(gs2);
            f1 = (T)(gs1 - fl1);
            f2 = (T)(gs2 - fl2);
            s1 = (int)fl1 + 1;
            s2 = (int)fl2 + 1;
            targ1 = (T)(d1 * ip.sh1);
            targ2 = (T)(d2 * ip.sh2);
            phr = (T)reduce_phase(ip.kq * (xi * xi + eta * eta) + ip.p1 * xi + ip.p2 * eta);
        }
        // F is stored fftshifted, so a target's support never wraps; targets
        // of the plan's box sit in the middle half of the grid.
        const int lim1 = ip.nfft1 - W - 2, lim2 = ip.nfft2 - W;
        if (s1 < 0 || s1 > lim1 || s2 < 0 || s2 > lim2) {
            atomicOr(status, kStatusTargetOutside);
            s1 = min(max(s1, 0), lim1);
            s2 = min(max(s2, 0), lim2);
        }
        T kx[W], ky[W];
        kernel_values<T, W>(f1, beta, hz, kx);
        kernel_values<T, W>(f2, beta, hz, ky);
        T gr = 0, gi = 0;
        if constexpr (std::is_same<T, float>::value && (W % 2 == 0)) {
            // W + 2 cells from the even cell at or below s1, as W/2 + 1
            // aligned 16-byte loads; the weights are shifted by s1's parity.
            const int odd = s1 & 1;
            float kk[W + 2];
#pragma unroll
            for (int i = 0; i < W + 2; ++i) {
                const float lo = (i < W) ? kx[i] : 0.0f;
                const float hi = (i >= 1 && i <= W) ? kx[i - 1] : 0.0f;
                kk[i] = odd ? hi : lo;
            }
            const float4* base =
                reinterpret_cast<const float4*>(F + (long long)s2 * ip.nfft1 + (s1 - odd));
            const int row4 = ip.nfft1 / 2;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float4* row = base + (long long)b * row4;
                float rr = 0.0f, ri = 0.0f;
#pragma unroll
                for (int q = 0; q < W / 2 + 1; ++q) {
                    const float4 v = __ldg(row + q);
                    rr = fmaf(kk[2 * q], v.x, fmaf(kk[2 * q + 1], v.z, rr));
                    ri = fmaf(kk[2 * q], v.y, fmaf(kk[2 * q + 1], v.w, ri));
                }
                gr = fmaf(ky[b], rr, gr);
                gi = fmaf(ky[b], ri, gi);
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const cx_t<T>* row = F + (long long)(s2 + b) * ip.nfft1 + s1;
                T rr = 0, ri = 0;
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    const cx_t<T> v = __ldg(&row[a]);
                    rr += kx[a] * v.x;
                    ri += kx[a] * v.y;
                }
                gr += ky[b] * rr;
                gi += ky[b] * ri;
            }
        }
        const T dec = kernel_ft_cheb<T>(targ1, s_a, ncheb, inv_tmax) *
                      kernel_ft_cheb<T>(targ2, s_a, ncheb, inv_tmax);
        T sn, cs;
        if constexpr (std::is_same<T, float>::value) {
            sincosf(phr, &sn, &cs);
        } else {
            sincos(phr, &sn, &cs);
        }
        // (cs + i sn) (gr + i gi) / dec * (-i / lz)
        const T sc = (T)ip.inv_lz / dec;
        const T pr = cs * gr - sn * gi, pi = cs * gi + sn * gr;
        T ur = pi * sc, ui = -pr * sc;
        if (ip.occulter) {
            ur = (T)1 - ur;
            ui = -ui;
        }
        cx_t<T> o;
        o.x = ur;
        o.y = ui;
        out[k] = o;
    }
}

// Chebyshev samples of psihat on [0, t_max]: s_i = psihat(t_max cos(pi (i + 1/2) / (2n)))
// for i < n (the even half of a 2n-point Chebyshev grid).
__global__ void k_cheb_samples(int n, double tmax, int w, double beta, const double* gq_t,
                               const double* gq_w, int q, double* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = cos(kPi * (i + 0.5) / (2.0 * n));
    out[i] = kernel_ft<double>(tmax * x, w, beta, gq_t, gq_w, q);
}

}  // namespace

void launch_cheb_samples(int n, double tmax, int w, double beta, const double* gq_t,
                         const double* gq_w, int q, double* out, cudaStream_t st) {
    k_cheb_samples<<<(n + 63) / 64, 64, 0, st>>>(n, tmax, w, beta, gq_t, gq_w, q, out);
}

void launch_target_sort(const double* targets, long long M, const InterpParams& ip, int* counts,
                        int* cursor, int* perm, cudaStream_t st) {
    if (M <= 0) return;
    long long nb = (M + 255) / 256;
    int blocks = (int)(nb < 152LL * 16 ? nb : 152LL * 16);
    k_target_count<<<blocks, 256, 0, st>>>(targets, M, ip, counts);
    k_target_scan<<<1, 1024, 0, st>>>(ip.nbin1 * ip.nbin2, counts, cursor);
    k_target_scatter<<<blocks, 256, 0, st>>>(targets, M, ip, cursor, perm);
}

template <typename T>
void launch_interp_w(const double* targets, long long M, const cx_t<T>* F, const InterpParams& ip,
                     const KernelShape& ks, const double* cheb, int ncheb,
                     void* out, unsigned* status, const int* perm, cudaStream_t st) {
    if (M <= 0) return;
    long long nb = (M + 255) / 256;
    int blocks = (int)(nb < 152LL * 32 ? nb : 152LL * 32);
    T beta = (T)ks.beta;
#define FRES_INTERP_CASE(WW)                                                                   \
    case WW:                                                                                   \
        k_interp<T, WW><<<blocks, 256, 0, st>>>(targets, M, F, ip, beta, cheb, ncheb,         \
                                                (cx_t<T>*)out, status, ks.horner, perm);       \
        break;
    switch (ks.w) {
        FRES_INTERP_CASE(2) FRES_INTERP_CASE(3) FRES_INTERP_CASE(4) FRES_INTERP_CASE(5)
        FRES_INTERP_CASE(6) FRES_INTERP_CASE(7) FRES_INTERP_CASE(8) FRES_INTERP_CASE(9)
        FRES_INTERP_CASE(10) FRES_INTERP_CASE(11) FRES_INTERP_CASE(12) FRES_INTERP_CASE(13)
        FRES_INTERP_CASE(14) FRES_INTERP_CASE(15) FRES_INTERP_CASE(16)
        default: break;
    }
#undef FRES_INTERP_CASE
}

template void launch_interp_w<float>(const double*, long long, const float2*, const InterpParams&,
                                     const KernelShape&, const double*, int, void*, unsigned*,
                                     const int*, cudaStream_t);
template void launch_interp_w<double>(const double*, long long, const double2*,
                                      const InterpParams&, const KernelShape&, const double*, int,
                                      void*, unsigned*, const int*, cudaStream_t);

}  // namespace fres
