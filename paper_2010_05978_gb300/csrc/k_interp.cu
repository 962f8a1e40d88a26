// Type-3 target side (arXiv:2010.05978 Sec. 3.2, eq. nufft3 and step 3):
// for each scattered target, interpolate the FFT of the deconvolved spread
// grid with the exponential-of-semicircle kernel (the inner type-2 NUFFT),
// divide by the kernel's Fourier transform at the target's frequency (the
// type-3 deconvolution), and apply the post-phase exp(-i s.C) of the node
// centring together with the target chirp and 1/(i lz):
//   u_k = 1/(i lz) exp(i pi |xi_k|^2 / lz - 2 pi i xi_k.C / lz) v'_k,
// optionally u^oc = 1 - u^ap (eq. bab).  Phases in FP64 with reduction.
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

template <typename T, int W>
__global__ void __launch_bounds__(256)
k_interp(const double* __restrict__ targets, long long M, const cx_t<T>* __restrict__ F,
         InterpParams ip, T beta, const double* __restrict__ gq_t,
         const double* __restrict__ gq_w, int q, cx_t<T>* __restrict__ out,
         unsigned* __restrict__ status) {
    __shared__ T s_gt[64], s_gw[64];
    for (int i = threadIdx.x; i < q && i < 64; i += blockDim.x) {
        s_gt[i] = (T)gq_t[i];
        s_gw[i] = (T)gq_w[i];
    }
    __syncthreads();
    const T half_w = (T)(0.5 * W), two_over_w = (T)(2.0 / W);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M;
         k += (long long)gridDim.x * blockDim.x) {
        const double2 t = reinterpret_cast<const double2*>(targets)[k];
        const double xi = t.x, eta = t.y;
        if (!(xi >= ip.box[0] && xi <= ip.box[1] && eta >= ip.box[2] && eta <= ip.box[3]))
            atomicOr(status, kStatusTargetOutside);
        const double d1 = xi - ip.xi_c, d2 = eta - ip.eta_c;
        double tau1 = d1 * ip.K1, tau2 = d2 * ip.K2;
        if (!isfinite(tau1) || !isfinite(tau2) || fabs(tau1) > ip.nfft1 || fabs(tau2) > ip.nfft2) {
            atomicOr(status, kStatusNonFinite);
            tau1 = tau2 = 0.0;
        }
        const double gs1 = tau1 - 0.5 * W, gs2 = tau2 - 0.5 * W;
        const double fl1 = floor(gs1), fl2 = floor(gs2);
        const T f1 = (T)(gs1 - fl1), f2 = (T)(gs2 - fl2);
        int s1 = (int)fl1 + 1, s2 = (int)fl2 + 1;
        if (s1 < 0) s1 += ip.nfft1;
        if (s2 < 0) s2 += ip.nfft2;
        T kx[W], ky[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            kx[a] = es_kernel<T>(((T)(a + 1) - half_w - f1) * two_over_w, beta);
            ky[a] = es_kernel<T>(((T)(a + 1) - half_w - f2) * two_over_w, beta);
        }
        T gr = 0, gi = 0;
#pragma unroll
        for (int b = 0; b < W; ++b) {
            int yy = s2 + b;
            if (yy >= ip.nfft2) yy -= ip.nfft2;
            const cx_t<T>* row = F + (long long)yy * ip.nfft1;
            T rr = 0, ri = 0;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                int xx = s1 + a;
                if (xx >= ip.nfft1) xx -= ip.nfft1;
                const cx_t<T> v = __ldg(&row[xx]);
                rr += kx[a] * v.x;
                ri += kx[a] * v.y;
            }
            gr += ky[b] * rr;
            gi += ky[b] * ri;
        }
        const T dec = kernel_ft<T>((T)(d1 * ip.sh1), W, beta, s_gt, s_gw, q) *
                      kernel_ft<T>((T)(d2 * ip.sh2), W, beta, s_gt, s_gw, q);
        const double ph = reduce_phase(ip.kq * (xi * xi + eta * eta) + ip.p1 * xi + ip.p2 * eta);
        T sn, cs;
        if (sizeof(T) == 8) {
            double s_, c_;
            sincos(ph, &s_, &c_);
            sn = (T)s_;
            cs = (T)c_;
        } else {
            float s_, c_;
            sincosf((float)ph, &s_, &c_);
            sn = (T)s_;
            cs = (T)c_;
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

}  // namespace

template <typename T>
void launch_interp_w(const double* targets, long long M, const cx_t<T>* F, const InterpParams& ip,
                     const KernelShape& ks, const double* gq_t, const double* gq_w, int q,
                     void* out, unsigned* status, cudaStream_t st) {
    if (M <= 0) return;
    long long nb = (M + 255) / 256;
    int blocks = (int)(nb < 152LL * 32 ? nb : 152LL * 32);
    T beta = (T)ks.beta;
#define FRES_INTERP_CASE(WW)                                                                   \
    case WW:                                                                                   \
        k_interp<T, WW><<<blocks, 256, 0, st>>>(targets, M, F, ip, beta, gq_t, gq_w, q,       \
                                                (cx_t<T>*)out, status);                        \
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
                                     const KernelShape&, const double*, const double*, int, void*,
                                     unsigned*, cudaStream_t);
template void launch_interp_w<double>(const double*, long long, const double2*,
                                      const InterpParams&, const KernelShape&, const double*,
                                      const double*, int, void*, unsigned*, cudaStream_t);

}  // namespace fres
