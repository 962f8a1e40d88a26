// Reverse-mode derivative of a type-1 evaluation with respect to the petal
// profiles of its starshade families (the design problem behind Sec. 4.2 of
// arXiv:2010.05978: A(r) sets the petal widths).
//
// For a real loss L with dL = Re sum_k conj(gamma_k) du_k (u the plan's
// output), write the computed field as u_k = sum_j c_j E_kj with
// E_kj = ax[k1] ay[k2] sum_l exp(-2 pi i k.l / nf) psi(l - g_j) (spreading,
// FFT, output tables).  Then
//   F_j = sum_k conj(gamma_k) E_kj = sum_l psi(l - g_j) btilde_l,
//   btilde = FFT(conj(gamma) ax ay placed at k mod nf)        (a type-2 NUFFT)
// and, with c_j = w_j exp(i phi_j),
//   dL = Re sum_j [F_j dc_j + c_j (dF_j/dg1 dg1 + dF_j/dg2 dg2)],
//   dc = e^{i phi} (dw + i w dphi),  dphi = (2 kq x - a1) dx + (2 kq y - a2) dy,
//   dg1 = U1 dx, dg2 = U2 dy (U = nf h / lz grid cells per unit length).
// A petal node (k, i, l) at radius r_l and angle theta = A_l t_i + 2 pi k / Np
// has w = r_l what_l A_l omegahat_i, so dw/dA_l = r_l what_l omegahat_i and
// d(x, y)/dA_l = r_l t_i (-sin theta, cos theta); dL/dA_l sums its nodes, and
// the profile parameters follow from dA_l/dparam (petal.cuh).
// A node (i, l) of a Fourier boundary family (boundary rule on Gauss-Legendre
// panels, dilation rule of eqs. aqnod/aqwei about c) sits at
// x = c + alpha_l r_i (cos t_i, sin t_i) with weight
// w = alpha_l wtilde_l ((X_i - cx) V_i - (Y_i - cy) W_i) = alpha_l wtilde_l what_i r_i^2
// (the tangent terms r'(t_i) cancel in the cross product), so
// dL/dr_i = sum_l alpha_l (cos t_i dL/dx + sin t_i dL/dy) + 2 alpha_l wtilde_l what_i r_i dL/dw,
// and dL/dp = sum_i dL/dr_i dr_i/dp for the coefficients p = (r0, a_k, b_k) of
// r(t) = r0 + sum_k (a_k cos kt + b_k sin kt).  Both are the exact derivative
// of the discrete map the plan computes.
#include <type_traits>

#include "internal.cuh"
#include "petal.cuh"
#include "spread.cuh"

namespace fres {

namespace {

// btilde input: sgn conj(gamma) ax ay (sgn = -1 for occulter output, whose
// derivative is minus that of the aperture field).
template <typename T>
__global__ void k_adj_prologue(const cx_t<T>* __restrict__ gamma, const cx_t<T>* __restrict__ ax,
                               const cx_t<T>* __restrict__ ay, cx_t<T>* __restrict__ out, int n1,
                               int n2, int B, T sgn) {
    const long long per = (long long)n1 * n2, total = per * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const long long r = e - b * per;
        const int k2 = (int)(r / n1), k1 = (int)(r - (long long)k2 * n1);
        const cx_t<T> g = gamma[e], x = ax[(long long)b * n1 + k1], y = ay[(long long)b * n2 + k2];
        const T pr = x.x * y.x - x.y * y.y, pi = x.x * y.y + x.y * y.x;   // ax ay
        cx_t<T> o;
        o.x = sgn * (g.x * pr + g.y * pi);    // conj(g) (ax ay)
        o.y = sgn * (g.x * pi - g.y * pr);
        out[e] = o;
    }
}

// dL/dw, dL/dx, dL/dy of a node with strength w e^{i phi}: F and dF/dg by
// kernel and kernel-derivative interpolation of btilde (stored fftshifted:
// natural cell l at (l + nf/2) mod nf), FP64 throughout.
template <typename T, int W>
__device__ __forceinline__ void node_derivs(const ChirpParams& cp, double x, double y, double w,
                                            const cx_t<T>* __restrict__ G, int nf1, int nf2,
                                            double beta, double* dLdw, double* dLdx,
                                            double* dLdy) {
    // chirp phase and (shifted, folded) grid coordinates, as the forward pass
    double sp, cph;
    sincos(reduce_phase(cp.kq * (x * x + y * y) - cp.a1 * x - cp.a2 * y + cp.a0), &sp, &cph);
    double g1 = x * cp.u1, g2 = y * cp.u2;
    g1 = (g1 - floor(g1)) * cp.nf1 + cp.sh1;
    g2 = (g2 - floor(g2)) * cp.nf2 + cp.sh2;
    if (g1 >= cp.nf1) g1 -= cp.nf1;
    if (g2 >= cp.nf2) g2 -= cp.nf2;
    const double gs1 = g1 - 0.5 * W, gs2 = g2 - 0.5 * W;
    const double fl1 = floor(gs1), fl2 = floor(gs2);
    const int s1 = (int)fl1 + 1, s2 = (int)fl2 + 1;
    const double fr1 = gs1 - fl1, fr2 = gs2 - fl2;
    // psi(l - g) and d/dg psi(l - g) = -psi'(l - g) at the W cells per dimension
    double p1[W], d1[W], p2[W], d2[W];
#pragma unroll
    for (int a = 0; a < W; ++a) {
        const double z1 = ((double)(a + 1) - 0.5 * W - fr1) * (2.0 / W);
        const double z2 = ((double)(a + 1) - 0.5 * W - fr2) * (2.0 / W);
        const double r1 = 1.0 - z1 * z1, r2 = 1.0 - z2 * z2;
        p1[a] = r1 > 0.0 ? exp(beta * (sqrt(r1) - 1.0)) : 0.0;
        p2[a] = r2 > 0.0 ? exp(beta * (sqrt(r2) - 1.0)) : 0.0;
        // psi'(u) = psi * beta * (-z / sqrt(1 - z^2)) * (2 / W); d/dg = -psi'
        d1[a] = r1 > 0.0 ? p1[a] * beta * z1 / sqrt(r1) * (2.0 / W) : 0.0;
        d2[a] = r2 > 0.0 ? p2[a] * beta * z2 / sqrt(r2) * (2.0 / W) : 0.0;
    }
    double Fr = 0, Fi = 0, G1r = 0, G1i = 0, G2r = 0, G2i = 0;
    for (int b = 0; b < W; ++b) {
        int row = s2 + b + nf2 / 2;
        row -= (row >= nf2) ? nf2 : 0;
        row -= (row >= nf2) ? nf2 : 0;
        const cx_t<T>* R = G + (long long)row * nf1;
        double rr = 0, ri = 0, drr = 0, dri = 0;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            int col = s1 + a + nf1 / 2;
            col -= (col >= nf1) ? nf1 : 0;
            col -= (col >= nf1) ? nf1 : 0;
            const cx_t<T> val = R[col];
            rr += p1[a] * (double)val.x;
            ri += p1[a] * (double)val.y;
            drr += d1[a] * (double)val.x;
            dri += d1[a] * (double)val.y;
        }
        Fr += p2[b] * rr;
        Fi += p2[b] * ri;
        G1r += p2[b] * drr;
        G1i += p2[b] * dri;
        G2r += d2[b] * rr;
        G2i += d2[b] * ri;
    }
    // e^{i phi} F and c dF/dg with c = w e^{i phi}
    const double eFr = cph * Fr - sp * Fi, eFi = cph * Fi + sp * Fr;
    const double U1 = cp.nf1 * cp.u1, U2 = cp.nf2 * cp.u2;
    *dLdw = eFr;
    // Re(i w eF dphi/dx + w e^{i phi} dF/dg1 U1)
    *dLdx = -w * eFi * (2.0 * cp.kq * x - cp.a1) + w * U1 * (cph * G1r - sp * G1i);
    *dLdy = -w * eFi * (2.0 * cp.kq * y - cp.a2) + w * U2 * (cph * G2r - sp * G2i);
}

__device__ __forceinline__ int family_of_block(const FamTable& ft) {
    int a = 0, b = ft.nfam - 1;
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (ft.blk0[mid] <= (int)blockIdx.x) a = mid;
        else b = mid - 1;
    }
    return a;
}

// Boundary parameter t_i and weight what_i of boundary node i of a Fourier
// family: Gauss-Legendre panels (the periodic trapezoid rule, eq. ptr, for a
// starshade's disc).
__device__ __forceinline__ void fourier_t(const FamilyDev& f, long long i, double* t,
                                          double* what) {
    const int q = (int)(i / f.p), s = (int)(i - (long long)q * f.p);
    const double hP = kTwoPi / f.n_panels;
    *t = f.ptr ? (q + 1) * hP : (q + f.gl_p_t[s]) * hP;
    *what = f.ptr ? hP : f.gl_p_w[s] * hP;
}

// One thread per node of the families the gradient is taken for (other
// families' blocks exit).  mode 0: PETALS families, contribution to dL/dA_l;
// mode 1: Fourier boundary families (not a starshade's internal disc),
// contribution to dL/dr_i.
template <typename T, int W>
__global__ void __launch_bounds__(kNodeThreads)
k_adj_nodes(FamTable ft, const cx_t<T>* __restrict__ bt, int nf1, int nf2, double beta,
            double* __restrict__ contrib, int mode) {
    __shared__ int s_fi;
    if (threadIdx.x == 0) s_fi = family_of_block(ft);
    __syncthreads();
    const FamilyDev& f = ft.fams[s_fi];
    if (mode == 0 && f.kind != FRESNEL_FAMILY_PETALS) return;
    if (mode == 1 && (f.kind != FRESNEL_FAMILY_FOURIER || f.ptr)) return;
    const ChirpParams& cp = ft.cps[f.prob];
    const long long j = (long long)(blockIdx.x - ft.blk0[s_fi]) * blockDim.x + threadIdx.x;
    if (j >= f.n_nodes) return;
    const cx_t<T>* G = bt + (long long)f.prob * nf1 * nf2;
    double dLdw, dLdx, dLdy;
    if (mode == 1) {
        const long long i = j / f.m;
        const int l = (int)(j - i * f.m);
        const double a = f.gl_m_a[l], aw = f.gl_m_aw[l];
        const double x = f.cx + a * f.bx[i], y = f.cy + a * f.by[i], w = aw * f.bc[i];
        node_derivs<T, W>(cp, x, y, w, G, nf1, nf2, beta, &dLdw, &dLdx, &dLdy);
        double t, what, st, ct;
        fourier_t(f, i, &t, &what);
        sincos(t, &st, &ct);
        const double r = f.bx[i] * ct + f.by[i] * st;
        contrib[f.offset + j] = a * (ct * dLdx + st * dLdy) + 2.0 * aw * what * r * dLdw;
        return;
    }
    const long long k = j / f.n_bdry, q = j - k * f.n_bdry;
    const int i = (int)(q / f.m), l = (int)(q - (long long)i * f.m);
    const double u = f.bx[q], v = f.by[q];
    const double cr = f.rot[2 * k], sr = f.rot[2 * k + 1];
    const double dx0 = u * cr - v * sr, dy0 = u * sr + v * cr;   // x - c
    const double x = f.cx + dx0, y = f.cy + dy0, w = f.bc[q];
    node_derivs<T, W>(cp, x, y, w, G, nf1, nf2, beta, &dLdw, &dLdx, &dLdy);
    // chain to A_l: dw/dA = r what omegahat, d(x,y)/dA = r t (-sin, cos) = t (-(y-cy), x-cx)
    const double span = f.pR - f.pa, wedge = kTwoPi / f.n_panels;
    const double r = f.pa + span * f.gl_m_a[l];
    const double dwdA = r * (span * f.gl_m_aw[l]) * (wedge * f.gl_p_w[i]);
    const double t = -0.5 * wedge + wedge * f.gl_p_t[i];
    contrib[f.offset + j] = dLdw * dwdA + t * (-dy0 * dLdx + dx0 * dLdy);
}

// Fourier families (list sf): dL/dr_i = sum over radii of the node
// contributions, one warp per boundary node, into rbuf[bofs[f] + i].
__global__ void k_adj_rsum(const FamilyDev* __restrict__ fams, const int* __restrict__ sf, int nsf,
                           const long long* __restrict__ bofs, const double* __restrict__ contrib,
                           double* __restrict__ rbuf) {
    const int lane = threadIdx.x & 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    long long base = 0;
    for (int fi = 0; fi < nsf; ++fi) {
        const FamilyDev& f = fams[sf[fi]];
        if (wid < base + f.n_bdry) {
            const long long i = wid - base;
            double s = 0.0;
            for (int l = lane; l < f.m; l += 32) s += contrib[f.offset + i * f.m + l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) rbuf[bofs[fi] + i] = s;
            return;
        }
        base += f.n_bdry;
    }
}

// One block per (Fourier family, coefficient): dL/dp = sum_i dL/dr_i dr_i/dp
// with dr/dr0 = 1, dr/da_k = cos k t, dr/db_k = sin k t (fixed-order block sum).
__global__ void k_adj_modes(const FamilyDev* __restrict__ fams, const int* __restrict__ sf,
                            const long long* __restrict__ bofs, const long long* __restrict__ gofs,
                            const double* __restrict__ rbuf, double* __restrict__ grad) {
    __shared__ double s_part[32];
    const int fi = blockIdx.y, kk = blockIdx.x;
    const FamilyDev& f = fams[sf[fi]];
    if (kk > 2 * f.K) return;
    const int k = (kk + 1) / 2;
    double s = 0.0;
    for (long long i = threadIdx.x; i < f.n_bdry; i += blockDim.x) {
        double t, what;
        fourier_t(f, i, &t, &what);
        const double phi = kk == 0 ? 1.0 : (kk % 2 == 1 ? cos(k * t) : sin(k * t));
        s += rbuf[bofs[fi] + i] * phi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_part[w];
        grad[gofs[fi] + kk] = tot;
    }
}

// One block per PETALS family (list pf): dL/dA_l = sum over petals and angles
// of the node contributions (one warp per l), then the profile parameters,
// added by one thread in increasing l (a fixed order: the gradient repeats
// bit for bit), kL radii at a time.
__global__ void k_adj_reduce(const FamilyDev* __restrict__ fams, const int* __restrict__ pf,
                             const long long* __restrict__ gofs,
                             const double* __restrict__ contrib, double* __restrict__ grad) {
    constexpr int kL = 1024;
    __shared__ double s_l[kL];
    const FamilyDev& f = fams[pf[blockIdx.x]];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long nki = (long long)f.n_panels * f.p;      // nodes per radius
    for (int l0 = 0; l0 < f.m; l0 += kL) {
        const int l1 = min(l0 + kL, f.m);
        for (int l = l0 + warp; l < l1; l += nw) {
            double s = 0.0;
            for (long long e = lane; e < nki; e += 32) s += contrib[f.offset + e * f.m + l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) s_l[l - l0] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int l = l0; l < l1; ++l) {
                const double r = f.pa + (f.pR - f.pa) * f.gl_m_a[l];
                int idx[4];
                double val[4];
                const int cnt = petal_profile_grad(f, l, r, idx, val);
                for (int q = 0; q < cnt; ++q) grad[gofs[blockIdx.x] + idx[q]] += s_l[l - l0] * val[q];
            }
        }
        __syncthreads();
    }
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

template <typename T>
void launch_adj_prologue(const void* gamma, const void* ax, const void* ay, void* out, int n1,
                         int n2, int B, int occulter, cudaStream_t st) {
    const long long total = (long long)n1 * n2 * B;
    const int blocks = (int)std::min<long long>(nblk(total, 256), 152 * 16);
    k_adj_prologue<T><<<blocks, 256, 0, st>>>((const cx_t<T>*)gamma, (const cx_t<T>*)ax,
                                              (const cx_t<T>*)ay, (cx_t<T>*)out, n1, n2, B,
                                              occulter ? (T)-1 : (T)1);
}
template void launch_adj_prologue<float>(const void*, const void*, const void*, void*, int, int,
                                         int, int, cudaStream_t);
template void launch_adj_prologue<double>(const void*, const void*, const void*, void*, int, int,
                                          int, int, cudaStream_t);

template <typename T>
void launch_adj_nodes(const FamTable& ft, int nblocks, const void* bt, int nf1, int nf2,
                      const KernelShape& ks, double* contrib, int mode, cudaStream_t st) {
#define FRES_ADJ_CASE(WW)                                                                     \
    case WW:                                                                                  \
        k_adj_nodes<T, WW><<<nblocks, kNodeThreads, 0, st>>>(ft, (const cx_t<T>*)bt, nf1, nf2, \
                                                            ks.beta, contrib, mode);          \
        break;
    switch (ks.w) {
        FRES_ADJ_CASE(2) FRES_ADJ_CASE(3) FRES_ADJ_CASE(4) FRES_ADJ_CASE(5) FRES_ADJ_CASE(6)
        FRES_ADJ_CASE(7) FRES_ADJ_CASE(8) FRES_ADJ_CASE(9) FRES_ADJ_CASE(10) FRES_ADJ_CASE(11)
        FRES_ADJ_CASE(12) FRES_ADJ_CASE(13) FRES_ADJ_CASE(14) FRES_ADJ_CASE(15) FRES_ADJ_CASE(16)
        default: break;
    }
#undef FRES_ADJ_CASE
}
template void launch_adj_nodes<float>(const FamTable&, int, const void*, int, int,
                                      const KernelShape&, double*, int, cudaStream_t);
template void launch_adj_nodes<double>(const FamTable&, int, const void*, int, int,
                                       const KernelShape&, double*, int, cudaStream_t);

void launch_adj_reduce(const FamilyDev* fams, const int* pf, const long long* gofs, int npf,
                       const double* contrib, double* grad, cudaStream_t st) {
    if (npf > 0) k_adj_reduce<<<npf, 256, 0, st>>>(fams, pf, gofs, contrib, grad);
}

void launch_adj_shape_reduce(const FamilyDev* fams, const int* sf, int nsf, int max_params,
                             long long n_bdry_total, const long long* bofs, const long long* gofs,
                             const double* contrib, double* rbuf, double* grad, cudaStream_t st) {
    if (nsf <= 0) return;
    const long long threads = 32 * n_bdry_total;
    k_adj_rsum<<<(int)((threads + 255) / 256), 256, 0, st>>>(fams, sf, nsf, bofs, contrib, rbuf);
    k_adj_modes<<<dim3(max_params, nsf), 256, 0, st>>>(fams, sf, bofs, gofs, rbuf, grad);
}

}  // namespace fres
