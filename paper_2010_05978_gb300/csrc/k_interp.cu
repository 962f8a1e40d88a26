// Type-3 target side (arXiv:2010.05978 Sec. 3.2, eq. nufft3 and step 3):
// for each scattered target, interpolate the FFT of the deconvolved spread
// grid with the exponential-of-semicircle kernel (the inner type-2 NUFFT),
// divide by the kernel's Fourier transform at the target's frequency (the
// type-3 deconvolution), and apply the post-phase exp(-i s.C) of the node
// centring together with the target chirp and 1/(i lz):
//   u_k = 1/(i lz) exp(i pi |xi_k|^2 / lz - 2 pi i xi_k.C / lz) v'_k,
// optionally u^oc = 1 - u^ap (eq. bab).
//
// The FFT grid F is stored fftshifted, so a target's w x w support never
// wraps.  FP32 fast mode: target coordinates, the box check and the phase are
// double-float (no FP64 arithmetic); for large target sets the targets are
// first bucketed by the 16 x 16 block of F holding their support, and each
// block's (16 + w)^2 patch of F is interpolated from shared memory.  FP64
// mode: FP64 coordinates and phase, gathers straight from global memory.
#include <type_traits>

#include "dfloat.cuh"
#include "spread.cuh"

namespace fres {

namespace {

constexpr int kBin = kTargetBin;    // target bins: kBin x kBin cells of F

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

// Support start (s1, s2) and fractional offsets of a target in the
// fftshifted FFT grid, FP32 fast mode (double-float), plus the argument of
// the kernel transform per dimension.  Out-of-box targets are flagged and
// clamped so every access stays inside F.
template <int W>
__device__ __forceinline__ void geom_f32(const double2 t, const InterpParams& ip, unsigned* status,
                                         dflt& xi, dflt& eta, int& s1, int& s2, float& f1,
                                         float& f2, float& targ1, float& targ2) {
    xi = df_from_double(t.x);
    eta = df_from_double(t.y);
    bool bad = !(xi.hi >= ip.boxf[0] && xi.hi <= ip.boxf[1] && eta.hi >= ip.boxf[2] &&
                 eta.hi <= ip.boxf[3]);
    dflt g1 = df_add(df_mul(xi, dflt{ip.dK1[0], ip.dK1[1]}), dflt{ip.dG1[0], ip.dG1[1]});
    dflt g2 = df_add(df_mul(eta, dflt{ip.dK2[0], ip.dK2[1]}), dflt{ip.dG2[0], ip.dG2[1]});
    if (!(fabsf(g1.hi) <= (float)ip.nfft1) || !(fabsf(g2.hi) <= (float)ip.nfft2)) {
        bad = true;
        g1 = g2 = dflt{0.0f, 0.0f};
    }
    int c1, c2;
    df_floor_split(g1, &c1, &f1);
    df_floor_split(g2, &c2, &f2);
    s1 = c1 + 1;
    s2 = c2 + 1;
    const int lim1 = ip.nfft1 - W - 2, lim2 = ip.nfft2 - W;
    if (s1 < 0 || s1 > lim1 || s2 < 0 || s2 > lim2) {
        bad = true;
        s1 = min(max(s1, 0), lim1);
        s2 = min(max(s2, 0), lim2);
    }
    if (bad && status) atomicOr(status, kStatusTargetOutside);
    // tau = g - (nfft/2 - w/2), exactly in double-float, then scaled
    targ1 = df_add(g1, dflt{-(0.5f * ip.nfft1 - 0.5f * W), 0.0f}).hi * ip.shK1;
    targ2 = df_add(g2, dflt{-(0.5f * ip.nfft2 - 0.5f * W), 0.0f}).hi * ip.shK2;
}

// Chirp and post-phase xi (kq xi + p1) + eta (kq eta + p2), reduced mod 2 pi.
__device__ __forceinline__ float phase_f32(dflt xi, dflt eta, const InterpParams& ip) {
    const dflt kq = {ip.dkq[0], ip.dkq[1]};
    const dflt q1 = df_mul(xi, df_add(df_mul(kq, xi), dflt{ip.dp1[0], ip.dp1[1]}));
    const dflt q2 = df_mul(eta, df_add(df_mul(kq, eta), dflt{ip.dp2[0], ip.dp2[1]}));
    return df_reduce_2pi(df_add(q1, q2));
}

// u = (cs + i sn) g / dec * (-i / lz), then Babinet if requested.
template <typename T>
__device__ __forceinline__ cx_t<T> epilogue(T gr, T gi, T dec, T sn, T cs, const InterpParams& ip) {
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
    return o;
}

// ------------------------------------------------------------------ generic kernel
// One thread per target, gathers from global memory (FP64 mode, and FP32
// mode for small target sets).
template <typename T, int W>
__global__ void __launch_bounds__(256)
k_interp(const double* __restrict__ targets, long long M, const cx_t<T>* __restrict__ F,
         InterpParams ip, T beta, const double* __restrict__ cheb, int ncheb,
         cx_t<T>* __restrict__ out, unsigned* __restrict__ status, const horner_t<T> hz) {
    __shared__ T s_a[kMaxCheb];
    for (int i = threadIdx.x; i < ncheb; i += blockDim.x) s_a[i] = (T)cheb[i];
    __syncthreads();
    const T inv_tmax = (T)ip.inv_tmax;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        int s1, s2;
        T f1, f2, targ1, targ2, phr;
        if constexpr (std::is_same<T, float>::value) {
            dflt xi, eta;
            geom_f32<W>(t, ip, status, xi, eta, s1, s2, f1, f2, targ1, targ2);
            phr = phase_f32(xi, eta, ip);
        } else {
            const double xi = t.x, eta = t.y;
            bool bad = !(xi >= ip.box[0] && xi <= ip.box[1] && eta >= ip.box[2] && eta <= ip.box[3]);
            const double d1 = xi - ip.xi_c, d2 = eta - ip.eta_c;
            double tau1 = d1 * ip.K1, tau2 = d2 * ip.K2;
            if (!isfinite(tau1) || !isfinite(tau2) || fabs(tau1) > ip.nfft1 ||
                fabs(tau2) > ip.nfft2) {
                bad = true;
                tau1 = tau2 = 0.0;
            }
            const double gs1 = tau1 + 0.5 * ip.nfft1 - 0.5 * W;
            const double gs2 = tau2 + 0.5 * ip.nfft2 - 0.5 * W;
            const double fl1 = floor(gs1), fl2 = floor(gs2);
            f1 = (T)(gs1 - fl1);
            f2 = (T)(gs2 - fl2);
            s1 = (int)fl1 + 1;
            s2 = (int)fl2 + 1;
            const int lim1 = ip.nfft1 - W - 2, lim2 = ip.nfft2 - W;
            if (s1 < 0 || s1 > lim1 || s2 < 0 || s2 > lim2) {
                bad = true;
                s1 = min(max(s1, 0), lim1);
                s2 = min(max(s2, 0), lim2);
            }
            if (bad) atomicOr(status, kStatusTargetOutside);
            targ1 = (T)(d1 * ip.sh1);
            targ2 = (T)(d2 * ip.sh2);
            phr = (T)reduce_phase(ip.kq * (xi * xi + eta * eta) + ip.p1 * xi + ip.p2 * eta);
        }
        T kx[W], ky[W];
        kernel_values<T, W>(f1, beta, hz, kx);
        kernel_values<T, W>(f2, beta, hz, ky);
        T gr = 0, gi = 0;
        if constexpr (std::is_same<T, float>::value && (W % 2 == 0)) {
            // W + 2 cells from the even cell at or below s1, as W/2 + 1
            // aligned 16-byte loads (nfft1 is even; s1 <= nfft1 - W - 2 keeps
            // the last load inside the row); weights shifted by s1's parity.
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
        if constexpr (std::is_same<T, float>::value) sincosf(phr, &sn, &cs);
        else sincos(phr, &sn, &cs);
        out[k] = epilogue<T>(gr, gi, dec, sn, cs, ip);
    }
}

// ------------------------------------------------------------------ cooperative FP32 kernel
// FP32 direct gathers, cooperatively: a warp takes 32 targets; each lane
// first does its own target's geometry, phase and kernel values (into shared
// memory), then LP lanes at a time gather one target's w x w support a row
// per instruction (LP consecutive cells: one or two cache lines, instead of
// one line per lane), reduce across the LP lanes and hand the sum to the
// target's lane for the deconvolution and epilogue.  Random targets make the
// per-lane pattern L1-bound (one wavefront per lane per load); this one needs
// a fraction of the wavefronts.
template <int W>
__global__ void __launch_bounds__(256)
k_interp_coop(const double* __restrict__ targets, long long M, const float2* __restrict__ F,
              InterpParams ip, const double* __restrict__ cheb, int ncheb,
              float2* __restrict__ out, unsigned* __restrict__ status, const HornerTab hz,
              float beta) {
    constexpr int LP = W <= 8 ? 8 : 16;   // lanes per target in the gather
    constexpr int TG = 32 / LP;           // targets per gather step
    __shared__ float s_a[kMaxCheb];
    __shared__ __align__(16) float s_kx[8][32][LP];
    __shared__ __align__(16) float s_ky[8][32][LP];
    __shared__ int2 s_s[8][32];
    for (int i = threadIdx.x; i < ncheb; i += blockDim.x) s_a[i] = (float)cheb[i];
    __syncthreads();
    const float inv_tmax = (float)ip.inv_tmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = lane % LP, sub = lane / LP;
    for (long long base = ((long long)blockIdx.x * 8 + warp) * 32; base < M;
         base += (long long)gridDim.x * 8 * 32) {
        const long long k = base + lane;
        const bool on = k < M;
        int s1 = 0, s2 = 0;
        float f1 = 0.0f, f2 = 0.0f, targ1 = 0.0f, targ2 = 0.0f, phr = 0.0f;
        if (on) {
            const double2 t = reinterpret_cast<const double2*>(targets)[k];
            dflt xi, eta;
            geom_f32<W>(t, ip, status, xi, eta, s1, s2, f1, f2, targ1, targ2);
            phr = phase_f32(xi, eta, ip);
        }
        float kx[W], ky[W];
        kernel_values<float, W>(f1, beta, hz, kx);
        kernel_values<float, W>(f2, beta, hz, ky);
        // a lane's row of LP slots as 16-byte stores (scalar stores of rows LP
        // floats apart would be LP/4-way bank conflicted)
#pragma unroll
        for (int q = 0; q < LP; q += 4) {
            float4 vx, vy;
            vx.x = q < W ? kx[q] : 0.0f;
            vx.y = q + 1 < W ? kx[q + 1] : 0.0f;
            vx.z = q + 2 < W ? kx[q + 2] : 0.0f;
            vx.w = q + 3 < W ? kx[q + 3] : 0.0f;
            vy.x = q < W ? ky[q] : 0.0f;
            vy.y = q + 1 < W ? ky[q + 1] : 0.0f;
            vy.z = q + 2 < W ? ky[q + 2] : 0.0f;
            vy.w = q + 3 < W ? ky[q + 3] : 0.0f;
            *reinterpret_cast<float4*>(&s_kx[warp][lane][q]) = vx;
            *reinterpret_cast<float4*>(&s_ky[warp][lane][q]) = vy;
        }
        s_s[warp][lane] = make_int2(s1, s2);
        __syncwarp();
        float gr = 0.0f, gi = 0.0f;
#pragma unroll 1
        for (int g = 0; g < 32 / TG; ++g) {
            const int j = g * TG + sub;
            const int2 sj = s_s[warp][j];
            float rr = 0.0f, ri = 0.0f;
            if (a < W) {
                const float kxa = s_kx[warp][j][a];
                const float2* col = F + (long long)sj.y * ip.nfft1 + sj.x + a;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const float2 v = __ldg(col + (long long)b * ip.nfft1);
                    const float wgt = s_ky[warp][j][b] * kxa;
                    rr = fmaf(wgt, v.x, rr);
                    ri = fmaf(wgt, v.y, ri);
                }
            }
#pragma unroll
            for (int o = LP / 2; o > 0; o >>= 1) {
                rr += __shfl_xor_sync(0xffffffffu, rr, o);
                ri += __shfl_xor_sync(0xffffffffu, ri, o);
            }
            // lanes g TG .. g TG + TG - 1 own this step's targets: sum from lane (l - g TG) LP
            const int src = ((lane - g * TG) * LP) & 31;
            const float vr = __shfl_sync(0xffffffffu, rr, src);
            const float vi = __shfl_sync(0xffffffffu, ri, src);
            if (lane >= g * TG && lane < (g + 1) * TG) {
                gr = vr;
                gi = vi;
            }
        }
        __syncwarp();   // the next 32 targets overwrite the shared tables
        if (on) {
            const float dec = kernel_ft_cheb<float>(targ1, s_a, ncheb, inv_tmax) *
                              kernel_ft_cheb<float>(targ2, s_a, ncheb, inv_tmax);
            float sn, cs;
            sincosf(phr, &sn, &cs);
            out[k] = epilogue<float>(gr, gi, dec, sn, cs, ip);
        }
    }
}

// ------------------------------------------------------------------ binned FP32 path
template <int W>
__device__ __forceinline__ int target_bin(const double2 t, const InterpParams& ip) {
    dflt xi, eta;
    int s1, s2;
    float f1, f2, a1, a2;
    geom_f32<W>(t, ip, nullptr, xi, eta, s1, s2, f1, f2, a1, a2);
    return (s2 / kBin) * ip.nbin1 + (s1 / kBin);
}

template <int W>
__global__ void k_target_count(const double* __restrict__ targets, long long M, InterpParams ip,
                               int* __restrict__ counts) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        atomicAdd(&counts[target_bin<W>(t, ip)], 1);
    }
}

// One block: exclusive scan of the bin counts (staged in shared memory) into
// bin starts and scatter cursors; clears the counts.
__global__ void k_target_scan(int nbins, int* __restrict__ counts, int* __restrict__ start,
                              int* __restrict__ cursor) {
    __shared__ long long s[1024];
    extern __shared__ int s_cnt[];
    const int t = threadIdx.x, nt = blockDim.x;
    for (int i = t; i < nbins; i += nt) {
        s_cnt[i] = counts[i];
        counts[i] = 0;
    }
    __syncthreads();
    const int per = (nbins + nt - 1) / nt;
    const int lo = min(t * per, nbins), hi = min(lo + per, nbins);
    long long sum = 0;
    for (int i = lo; i < hi; ++i) sum += s_cnt[i];
    s[t] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const long long a = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    long long run = s[t] - sum;
    for (int i = lo; i < hi; ++i) {
        const int c = s_cnt[i];
        s_cnt[i] = (int)run;
        run += c;
    }
    __syncthreads();
    for (int i = t; i < nbins; i += nt) {
        start[i] = s_cnt[i];
        cursor[i] = s_cnt[i];
    }
}

// Multi-block exclusive scan of the bin counts for large FFT grids: chunk
// sums, one block scanning the chunk sums, then each chunk's own scan from
// its offset (into bin starts and scatter cursors; counts cleared).
__global__ void k_bin_chunk_sums(int nbins, const int* __restrict__ counts, int* __restrict__ partial) {
    __shared__ int s[32];
    const int b0 = blockIdx.x * kBinChunk;
    int sum = 0;
    for (int i = b0 + threadIdx.x; i < min(b0 + kBinChunk, nbins); i += blockDim.x) sum += counts[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (int)(blockDim.x >> 5) ? s[threadIdx.x] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_bin_chunk_scan(int nchunks, int* __restrict__ partial) {
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int i = 0; i < nchunks; ++i) {
        const int c = partial[i];
        partial[i] = run;
        run += c;
    }
}

__global__ void k_bin_chunk_write(int nbins, int* __restrict__ counts, const int* __restrict__ partial,
                                  int* __restrict__ start, int* __restrict__ cursor) {
    __shared__ int s[kBinChunk];
    __shared__ int w[32];
    const int b0 = blockIdx.x * kBinChunk, n = min(kBinChunk, nbins - b0);
    const int per = kBinChunk / blockDim.x;          // contiguous bins per thread
    const int lo = threadIdx.x * per;
    int sum = 0;
    for (int i = 0; i < per; ++i) {
        const int v = lo + i < n ? counts[b0 + lo + i] : 0;
        s[lo + i] = v;
        sum += v;
    }
    // exclusive scan of the per-thread sums (warp shuffles, then warp totals)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) w[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int v = lane < (int)(blockDim.x >> 5) ? w[lane] : 0;
        int vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        w[lane] = vi - v;
    }
    __syncthreads();
    int run = partial[blockIdx.x] + w[wid] + inc - sum;
    for (int i = 0; i < per && lo + i < n; ++i) {
        const int b = b0 + lo + i;
        start[b] = run;
        cursor[b] = run;
        counts[b] = 0;
        run += s[lo + i];
    }
}

template <int W>
__global__ void k_target_scatter(const double* __restrict__ targets, long long M, InterpParams ip,
                                 int* __restrict__ cursor, int* __restrict__ perm) {
    // four targets per thread and pass: four atomics in flight at once
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M; k += 4 * stride) {
        int pos[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long ku = k + u * stride;
            pos[u] = -1;
            if (ku < M) {
                const double2 t = reinterpret_cast<const double2*>(targets)[ku];
                pos[u] = atomicAdd(&cursor[target_bin<W>(t, ip)], 1);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (pos[u] >= 0 && pos[u] < M) perm[pos[u]] = (int)(k + u * stride);
    }
}

// Binned interpolation: a block takes bins dynamically (work[0]); it copies
// the bin's (kBin + w) x (kBin + w) patch of F to shared memory and interpolates
// the bin's targets from it, writing each result to the target's own index.
template <int W>
__global__ void __launch_bounds__(128)
k_interp_binned(const double* __restrict__ targets, long long M, const float2* __restrict__ F,
                InterpParams ip, const double* __restrict__ cheb, int ncheb,
                float2* __restrict__ out, unsigned* __restrict__ status, const HornerTab hz,
                const int* __restrict__ perm, const int* __restrict__ bin_start, int nbins,
                int* __restrict__ work, float beta) {
    constexpr int P = kBin + W;          // patch edge
    constexpr int PS = P + 1;            // patch row stride (float2)
    __shared__ float2 patch[P * PS];
    __shared__ float s_a[kMaxCheb];
    // bins are claimed kClaim at a time (one atomic per claim; most bins of a
    // large grid hold no targets and cost only a bounds check), their starts
    // loaded together
    constexpr int kClaim = 16;
    __shared__ int s_b;
    __shared__ int s_start[kClaim + 1];
    for (int i = threadIdx.x; i < ncheb; i += blockDim.x) s_a[i] = (float)cheb[i];
    const float inv_tmax = (float)ip.inv_tmax;
    for (int b = nbins, b0 = nbins, b_end = nbins;; ++b) {
        if (b >= b_end) {
            __syncthreads();
            if (threadIdx.x == 0) s_b = atomicAdd(&work[0], kClaim);
            __syncthreads();
            b = b0 = s_b;
            if (b >= nbins) break;
            b_end = min(b + kClaim, nbins);
            if (threadIdx.x <= b_end - b0)
                s_start[threadIdx.x] = b0 + (int)threadIdx.x < nbins ? bin_start[b0 + threadIdx.x] : (int)M;
            __syncthreads();
        }
        const int beg = s_start[b - b0];
        const int end = s_start[b - b0 + 1];
        if (beg >= end) continue;
        // the first two targets of this thread: perm entries two steps
        // ahead, target coordinates one step ahead, so a target's loads are
        // in flight while the previous one (or the patch copy) is worked on
        const int bs = blockDim.x;
        int i = beg + threadIdx.x;
        int k0 = i < end ? __ldg(&perm[i]) : -1;
        int k1 = i + bs < end ? __ldg(&perm[i + bs]) : -1;
        double2 t0 = k0 >= 0 ? __ldg(&reinterpret_cast<const double2*>(targets)[k0])
                             : make_double2(0.0, 0.0);
        __syncthreads();   // the previous bin's targets are done with the patch
        const int ox = (b % ip.nbin1) * kBin, oy = (b / ip.nbin1) * kBin;
        for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
            const int r = e / P, c = e % P;
            const int gy = oy + r, gx = ox + c;
            float2 v = make_float2(0.0f, 0.0f);
            if (gy < ip.nfft2 && gx < ip.nfft1) v = __ldg(&F[(long long)gy * ip.nfft1 + gx]);
            patch[r * PS + c] = v;
        }
        __syncthreads();
        for (; i < end; i += bs) {
            const int k = k0;
            const double2 t = t0;
            k0 = k1;
            if (k1 >= 0) t0 = __ldg(&reinterpret_cast<const double2*>(targets)[k1]);
            k1 = i + 2 * bs < end ? __ldg(&perm[i + 2 * bs]) : -1;
            dflt xi, eta;
            int s1, s2;
            float f1, f2, targ1, targ2;
            geom_f32<W>(t, ip, status, xi, eta, s1, s2, f1, f2, targ1, targ2);
            const int x = s1 - ox, y = s2 - oy;   // in [0, 16) by construction of the bins
            float kx[W], ky[W];
            kernel_values<float, W>(f1, beta, hz, kx);
            kernel_values<float, W>(f2, beta, hz, ky);
            float gr = 0.0f, gi = 0.0f;
            if ((unsigned)x < (unsigned)kBin && (unsigned)y < (unsigned)kBin) {
#pragma unroll
                for (int bb = 0; bb < W; ++bb) {
                    const float2* row = patch + (y + bb) * PS + x;
                    float rr = 0.0f, ri = 0.0f;
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const float2 v = row[a];
                        rr = fmaf(kx[a], v.x, rr);
                        ri = fmaf(kx[a], v.y, ri);
                    }
                    gr = fmaf(ky[bb], rr, gr);
                    gi = fmaf(ky[bb], ri, gi);
                }
            } else if (status) {
                atomicOr(status, kStatusNonFinite);   // bin / geometry mismatch: cannot happen
            }
            const float dec = kernel_ft_cheb<float>(targ1, s_a, ncheb, inv_tmax) *
                              kernel_ft_cheb<float>(targ2, s_a, ncheb, inv_tmax);
            float sn, cs;
            sincosf(phase_f32(xi, eta, ip), &sn, &cs);
            out[k] = epilogue<float>(gr, gi, dec, sn, cs, ip);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&work[1], 1) == (int)gridDim.x - 1) {
            work[0] = 0;
            work[1] = 0;
        }
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

inline int nblk(long long n, int b, int cap) {
    long long g = (n + b - 1) / b;
    return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace

void launch_cheb_samples(int n, double tmax, int w, double beta, const double* gq_t,
                         const double* gq_w, int q, double* out, cudaStream_t st) {
    k_cheb_samples<<<(n + 63) / 64, 64, 0, st>>>(n, tmax, w, beta, gq_t, gq_w, q, out);
}

void launch_target_sort(const double* targets, long long M, const InterpParams& ip, int w,
                        const T3Sort* sort, cudaStream_t st) {
    if (M <= 0) return;
    const int nbins = ip.nbin1 * ip.nbin2;
    const int gb = nblk(M, 256, 152 * 16);
    if (nbins <= kBinScanStaged) {
        const size_t dyn = sizeof(int) * (size_t)nbins;
        cudaFuncSetAttribute(k_target_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    }
    auto scan = [&]() {
        if (nbins <= kBinScanStaged) {
            k_target_scan<<<1, 1024, sizeof(int) * (size_t)nbins, st>>>(nbins, sort->counts,
                                                                        sort->start, sort->cursor);
        } else {
            const int nchunks = (nbins + kBinChunk - 1) / kBinChunk;
            k_bin_chunk_sums<<<nchunks, 256, 0, st>>>(nbins, sort->counts, sort->partial);
            k_bin_chunk_scan<<<1, 32, 0, st>>>(nchunks, sort->partial);
            k_bin_chunk_write<<<nchunks, 256, 0, st>>>(nbins, sort->counts, sort->partial,
                                                       sort->start, sort->cursor);
        }
    };
#define FRES_SORT_CASE(WW)                                                                     \
    case WW:                                                                                   \
        k_target_count<WW><<<gb, 256, 0, st>>>(targets, M, ip, sort->counts);                  \
        scan();                                                                                \
        k_target_scatter<WW><<<gb, 256, 0, st>>>(targets, M, ip, sort->cursor, sort->perm);    \
        return;
    switch (w) {
        FRES_SORT_CASE(4) FRES_SORT_CASE(5) FRES_SORT_CASE(6) FRES_SORT_CASE(7)
        FRES_SORT_CASE(8) FRES_SORT_CASE(9) FRES_SORT_CASE(10)
        default: break;
    }
#undef FRES_SORT_CASE
}

template <typename T>
void launch_interp_w(const double* targets, long long M, const cx_t<T>* F, const InterpParams& ip,
                     const KernelShape& ks, const double* cheb, int ncheb, void* out,
                     unsigned* status, const T3Sort* sort, cudaStream_t st) {
    if (M <= 0) return;
    T beta = (T)ks.beta;
    if constexpr (std::is_same<T, float>::value) {
        if (sort) {   // binned path: interpolate each bin's targets from its patch
            const int nbins = ip.nbin1 * ip.nbin2;
#define FRES_BINNED_CASE(WW)                                                                   \
    case WW:                                                                                   \
        k_interp_binned<WW><<<152 * 8, 128, 0, st>>>(targets, M, F, ip, cheb, ncheb,           \
                                                      (float2*)out, status, ks.horner,         \
                                                      sort->perm, sort->start, nbins,          \
                                                      sort->work, beta);                       \
        return;
            switch (ks.w) {
                FRES_BINNED_CASE(4) FRES_BINNED_CASE(5) FRES_BINNED_CASE(6) FRES_BINNED_CASE(7)
                FRES_BINNED_CASE(8) FRES_BINNED_CASE(9) FRES_BINNED_CASE(10)
                default: break;   // other widths: generic kernel below
            }
#undef FRES_BINNED_CASE
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (ks.w <= 12 && ks.horner.deg >= 0) {   // FP32: cooperative gathers
            const int cb = nblk(M, 256, 152 * 16);
#define FRES_COOP_CASE(WW)                                                                     \
    case WW:                                                                                   \
        k_interp_coop<WW><<<cb, 256, 0, st>>>(targets, M, F, ip, cheb, ncheb, (float2*)out,     \
                                              status, ks.horner, beta);                        \
        return;
            switch (ks.w) {
                FRES_COOP_CASE(2) FRES_COOP_CASE(3) FRES_COOP_CASE(4) FRES_COOP_CASE(5)
                FRES_COOP_CASE(6) FRES_COOP_CASE(7) FRES_COOP_CASE(8) FRES_COOP_CASE(9)
                FRES_COOP_CASE(10) FRES_COOP_CASE(11) FRES_COOP_CASE(12)
                default: break;
            }
#undef FRES_COOP_CASE
        }
    }
    const int blocks = nblk(M, 256, 152 * 32);
#define FRES_INTERP_CASE(WW)                                                                   \
    case WW:                                                                                   \
        k_interp<T, WW><<<blocks, 256, 0, st>>>(targets, M, F, ip, beta, cheb, ncheb,         \
                                                (cx_t<T>*)out, status, horner_of<T>(ks));      \
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

bool interp_binned_width(int w) { return w >= 4 && w <= 10; }

template void launch_interp_w<float>(const double*, long long, const float2*, const InterpParams&,
                                     const KernelShape&, const double*, int, void*, unsigned*,
                                     const T3Sort*, cudaStream_t);
template void launch_interp_w<double>(const double*, long long, const double2*,
                                      const InterpParams&, const KernelShape&, const double*, int,
                                      void*, unsigned*, const T3Sort*, cudaStream_t);

}  // namespace fres

