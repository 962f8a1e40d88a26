// Node-side kernels: Gauss-Legendre rules, boundary line rules, the areal
// dilation rule with the chirp (Sec. 3.2 step 1), grid coordinates and the
// counting sort of nodes into spreading tiles; plus the small plan-time tables
// (FFT twiddles, deconvolution and output-chirp factors).
// Paper: arXiv:2010.05978, Secs. 3.2-3.3 and 4.1 (eqs. split, aqnod, aqwei, vliq1).
#include "dfloat.cuh"
#include "internal.cuh"
#include "petal.cuh"

namespace fres {

namespace {

__device__ __forceinline__ void agg_count(int key, int* counts) {
    unsigned mask = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    if (key >= 0 && lane == __ffs(mask) - 1) atomicAdd(&counts[key], __popc(mask));
}

__device__ __forceinline__ int agg_reserve(int key, int* cursor) {
    unsigned mask = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (key >= 0 && lane == leader) base = atomicAdd(&cursor[key], __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// ------------------------------------------------------------------ source screens
// s(x, y) = A(x, y) exp(i k OPD(x, y)) (Sec. 5: the strength of each areal
// node times the source term), A and OPD by Catmull-Rom interpolation of
// their samples: cubic convolution with the weights, for the fraction t of
// the cell, -t(1-t)^2/2, (2 - 5t^2 + 3t^3)/2, t(1 + 4t - 3t^2)/2, -t^2(1-t)/2
// on samples -1, 0, 1, 2.  The stencil stays inside the samples (cells 1 ..
// n - 3; nodes beyond take the nearest interior value).
template <typename T>
__device__ __forceinline__ void cr_weights(T t, T w[4]) {
    const T t2 = t * t, t3 = t2 * t;
    w[0] = (T)0.5 * (-t3 + (T)2 * t2 - t);
    w[1] = (T)0.5 * ((T)3 * t3 - (T)5 * t2 + (T)2);
    w[2] = (T)0.5 * ((T)-3 * t3 + (T)4 * t2 + t);
    w[3] = (T)0.5 * (t3 - t2);
}

template <typename T>
__device__ __forceinline__ T cr_interp(const T* __restrict__ a, int n1, int i1, int i2,
                                       const T wx[4], const T wy[4]) {
    T s = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const T* row = a + (long long)(i2 - 1 + b) * n1 + (i1 - 1);
        const T r = wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2] + wx[3] * row[3];
        s += wy[b] * r;
    }
    return s;
}

template <typename T>
__device__ __forceinline__ void apply_screen(const ScreenDev& sc, double k, T x, T y, T& cre,
                                             T& cim) {
    T u = (x - (T)sc.x0) * (T)sc.ihx, v = (y - (T)sc.y0) * (T)sc.ihy;
    u = u < (T)1 ? (T)1 : (u > (T)(sc.n1 - 2) ? (T)(sc.n1 - 2) : u);
    v = v < (T)1 ? (T)1 : (v > (T)(sc.n2 - 2) ? (T)(sc.n2 - 2) : v);
    if (!(u == u) || !(v == v)) u = v = (T)1;   // non-finite node: flagged elsewhere
    const int i1 = min((int)u, sc.n1 - 3), i2 = min((int)v, sc.n2 - 3);
    T wx[4], wy[4];
    cr_weights<T>(u - (T)i1, wx);
    cr_weights<T>(v - (T)i2, wy);
    const T A = sc.amp ? cr_interp<T>((const T*)sc.amp, sc.n1, i1, i2, wx, wy) : (T)1;
    T sr = A, si = (T)0;
    if (sc.opd) {
        const T ph = (T)k * cr_interp<T>((const T*)sc.opd, sc.n1, i1, i2, wx, wy);
        T sn, cs;
        if constexpr (sizeof(T) == 4) sincosf(ph, &sn, &cs);
        else sincos(ph, &sn, &cs);
        sr = A * cs;
        si = A * sn;
    }
    const T r = cre * sr - cim * si, im = cre * si + cim * sr;
    cre = r;
    cim = im;
}

// Up to four tiles touched by a node whose support starts at (s1, s2).
__device__ __forceinline__ void node_tiles(int s1, int s2, const ChirpParams& cp, int key[4]) {
    int e1 = s1 + cp.w - 1; if (e1 >= cp.nf1) e1 -= cp.nf1;
    int e2 = s2 + cp.w - 1; if (e2 >= cp.nf2) e2 -= cp.nf2;
    int ta = s1 / kTile, tb = e1 / kTile;
    int sa = s2 / kTile, sb = e2 / kTile;
    const int b = cp.tile_base;
    key[0] = b + sa * cp.ntx + ta;
    key[1] = (tb != ta) ? b + sa * cp.ntx + tb : -1;
    key[2] = (sb != sa) ? b + sb * cp.ntx + ta : -1;
    key[3] = (tb != ta && sb != sa) ? b + sb * cp.ntx + tb : -1;
}

// ------------------------------------------------------------------ Gauss-Legendre
// Roots of P_n by Newton's method on the three-term recurrence
// (j + 1) P_{j+1} = (2j + 1) x P_j - j P_{j-1}, from Tricomi's asymptotic
// estimate of each root; the weights 2 / ((1 - x^2) P_n'(x)^2); both mapped
// from (-1, 1) to (0, 1), ascending.  The roots are symmetric (x_{n-1-i} =
// -x_i): thread i < ceil(n/2) finds root i and writes both.  The recurrence
// divides by j + 1 through a per-block table of reciprocals (FP64 division is
// many times the cost of a multiply).
template <bool kTable>
__device__ __forceinline__ void legendre_pn(int n, double x, const double* inv, double* pn,
                                            double* pn1) {
    double p0 = 1.0, p1 = x;
    for (int j = 1; j < n; ++j) {
        const double q = (2.0 * j + 1.0) * x * p1 - j * p0;
        const double p2 = kTable ? q * inv[j + 1] : q / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

// kTable: the reciprocals 1/j (j <= n) in dynamic shared memory (n small
// enough); otherwise the recurrence divides.
template <bool kTable>
__global__ void k_gauss_legendre(int n, double* t01, double* w01) {
    extern __shared__ double s_inv[];   // s_inv[j] = 1 / j, j = 1 .. n
    if (kTable) {
        for (int j = threadIdx.x; j <= n; j += blockDim.x) s_inv[j] = j > 0 ? 1.0 / j : 0.0;
        __syncthreads();
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int half = (n + 1) / 2;
    if (i >= half) return;
    const double nn = (double)n;
    double x = (1.0 - (nn - 1.0) / (8.0 * nn * nn * nn)) * cos(kPi * (i + 0.75) / (nn + 0.5));
    if (2 * i + 1 == n) x = 0.0;   // odd n: the middle root
    double pn, pn1;
    int converged = 0;
    for (int it = 0; it < 100 && converged < 2; ++it) {
        legendre_pn<kTable>(n, x, s_inv, &pn, &pn1);
        const double dp = nn * (x * pn - pn1) / (x * x - 1.0);
        const double dx = pn / dp;
        x -= dx;
        if (fabs(dx) < 1e-15) ++converged;
    }
    legendre_pn<kTable>(n, x, s_inv, &pn, &pn1);
    const double dp = nn * (x * pn - pn1) / (x * x - 1.0);
    const double w = 1.0 / ((1.0 - x * x) * dp * dp);
    t01[i] = 0.5 * (1.0 - x);
    w01[i] = w;
    if (n - 1 - i != i) {
        t01[n - 1 - i] = 0.5 * (1.0 + x);
        w01[n - 1 - i] = w;
    }
}

// ------------------------------------------------------------------ boundary line rules
// Fourier star, Sec. 4.1: X(t) = r cos t, Y(t) = r sin t about the centre,
// r = r0 + sum (a_k cos kt + b_k sin kt); panel q of n_panels equal t-panels
// carries p Gauss-Legendre nodes: W = what X'(t), V = what Y'(t) (eq. vliq1).
// Stored relative to the centre: bx = X - cx, by = Y - cy, bc = bx V - by W.
__device__ __forceinline__ void split_store(float* dst, double v) {
    const float hi = (float)v;
    dst[0] = hi;
    dst[1] = (float)(v - (double)hi);
}

// Spoke coefficients of boundary node i for the FP32 fast mode (see
// k_nodes_count_df): A1 = 2 kq c.b - a.b, A2 = kq |b|^2, and the per-unit-alpha
// grid-coordinate slopes G1.  Computed once per boundary node in FP64.
__device__ __forceinline__ void store_spoke(const FamilyDev& f, const ChirpParams& cp, long long i,
                                            double bx, double by, double bc) {
    if (!f.spoke) return;
    float* s = f.spoke + 8 * i;
    split_store(s + 0, 2.0 * cp.kq * (f.cx * bx + f.cy * by) - cp.a1 * bx - cp.a2 * by);
    split_store(s + 2, cp.kq * (bx * bx + by * by));
    if (!cp.type3) {
        split_store(s + 4, (double)cp.nf1 * cp.u1 * bx);
        split_store(s + 6, (double)cp.nf2 * cp.u2 * by);
    } else {
        split_store(s + 4, bx * cp.inv_h1);
        split_store(s + 6, by * cp.inv_h2);
    }
    f.bcf[i] = (float)bc;
}

__global__ void k_boundary_fourier(FamilyDev f, ChirpParams cp) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= f.n_bdry) return;
    int q = (int)(i / f.p), s = (int)(i % f.p);
    double hP = kTwoPi / f.n_panels;
    // GL panels, or the periodic trapezoid rule t_q = 2 pi (q+1)/n (eq. ptr)
    double t = f.ptr ? (q + 1) * hP : (q + f.gl_p_t[s]) * hP;
    double what = f.ptr ? hP : f.gl_p_w[s] * hP;
    double st, ct;
    sincos(t, &st, &ct);
    double r = f.params[0], dr = 0.0;
    double ck = 1.0, sk = 0.0;
    for (int k = 1; k <= f.K; ++k) {
        double c2 = ck * ct - sk * st;
        sk = sk * ct + ck * st;
        ck = c2;
        double a = f.params[2 * k - 1], b = f.params[2 * k];
        r += a * ck + b * sk;
        dr += k * (b * ck - a * sk);
    }
    double X = r * ct, Y = r * st;
    double W = what * (dr * ct - r * st);
    double V = what * (dr * st + r * ct);
    f.bx[i] = X;
    f.by[i] = Y;
    if (f.bw) {
        f.bw[i] = W;
        f.bv[i] = V;
    }
    f.bc[i] = X * V - Y * W;
    store_spoke(f, cp, i, X, Y, X * V - Y * W);
}

// Explicit vector line rule: params = [X.., Y.., W.., V..].
__global__ void k_boundary_line(FamilyDev f, ChirpParams cp) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long n = f.n_bdry;
    if (i >= n) return;
    double X = f.params[i] - f.cx, Y = f.params[n + i] - f.cy;
    double W = f.params[2 * n + i], V = f.params[3 * n + i];
    f.bx[i] = X;
    f.by[i] = Y;
    if (f.bw) {
        f.bw[i] = W;
        f.bv[i] = V;
    }
    f.bc[i] = X * V - Y * W;
    store_spoke(f, cp, i, X, Y, X * V - Y * W);
}

// ------------------------------------------------------------------ starshade petals
// Tables of the first petal (centred on angle 0) for index i*m + l:
// r_l = a + (R-a) rho_l and what_l = (R-a) rhow_l from the m-point rule on
// (0,1); t_i = -pi/Np + (2 pi/Np) tau_i, omegahat_i = (2 pi/Np) tauw_i from
// the p-point rule; u, v = r_l (cos, sin)(A(r_l) t_i), w = r_l what_l A omegahat_i.
// Also the petal rotations cos, sin(2 pi k / Np).
__global__ void k_petal_tables(FamilyDev f) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q < f.n_panels) {
        double s, c;
        sincospi(2.0 * (double)q / f.n_panels, &s, &c);
        f.rot[2 * q] = c;
        f.rot[2 * q + 1] = s;
    }
    if (q >= f.n_bdry) return;
    const int i = (int)(q / f.m), l = (int)(q - (long long)i * f.m);
    const double span = f.pR - f.pa, wedge = kTwoPi / f.n_panels;
    const double r = f.pa + span * f.gl_m_a[l];
    const double A = petal_profile(f, l, r);
    const double t = -0.5 * wedge + wedge * f.gl_p_t[i];
    double s, c;
    sincos(A * t, &s, &c);
    f.bx[q] = r * c;
    f.by[q] = r * s;
    f.bc[q] = r * (span * f.gl_m_aw[l]) * A * (wedge * f.gl_p_w[i]);
}

// ------------------------------------------------------------------ FP32 fast mode nodes
// Double-float form of the dilation rule for one spoke (boundary node i):
// with x = c + alpha b, the chirp phase kq |x|^2 - a.x + a0 equals
// A0 + alpha (A1 + alpha A2) and the grid coordinate (minus w/2) equals
// G0 + alpha G1, so a node costs a few double-float operations and no FP64.
// Common tail of the double-float node paths: fold (type 1), split into
// support start and fraction, bounds, record and tile keys.
__device__ __forceinline__ void finish_df(dflt v1, dflt v2, float cre, float cim,
                                          const ChirpParams& cp, NodeRec<float>* out,
                                          unsigned* status, int key[4]) {
    NodeRec<float> r;
    r.cre = cre;
    r.cim = cim;
    if (!cp.type3) {   // fold into [0, nf): the type-1 grid is periodic (Sec. 3.3)
        const float q1 = floorf(v1.hi / (float)cp.nf1), q2 = floorf(v2.hi / (float)cp.nf2);
        v1 = df_add(v1, dflt{-q1 * (float)cp.nf1, 0.0f});
        v2 = df_add(v2, dflt{-q2 * (float)cp.nf2, 0.0f});
    }
    int c1, c2;
    df_floor_split(v1, &c1, &r.f1);
    df_floor_split(v2, &c2, &r.f2);
    int s1 = c1 + 1, s2 = c2 + 1;
    if (!(v1.hi == v1.hi) || !(v2.hi == v2.hi)) {
        atomicOr(status, kStatusNonFinite);
        s1 = s2 = 0;
        r.cre = r.cim = 0.0f;
    }
    if (!cp.type3) {
        s1 = ((s1 % cp.nf1) + cp.nf1) % cp.nf1;
        s2 = ((s2 % cp.nf2) + cp.nf2) % cp.nf2;
    } else if (s1 < 0 || s2 < 0 || s1 + cp.w > cp.nf1 || s2 + cp.w > cp.nf2) {
        atomicOr(status, kStatusNodeOutside);
        s1 = min(max(s1, 0), cp.nf1 - cp.w);
        s2 = min(max(s2, 0), cp.nf2 - cp.w);
    }
    r.s1 = s1;
    r.s2 = s2;
    *out = r;
    node_tiles(s1, s2, cp, key);
}

__device__ __forceinline__ void node_df(const FamilyDev& f, const ChirpParams& cp, long long j,
                                        NodeRec<float>* rec, unsigned* status, int key[4],
                                        const ScreenDev& scr) {
    // j < 2^30 (plan limit): 32-bit division
    const unsigned i = (unsigned)j / (unsigned)f.m;
    const int l = (int)((unsigned)j - i * (unsigned)f.m);
    const float4 sA = reinterpret_cast<const float4*>(f.spoke)[2 * i];
    const float4 sG = reinterpret_cast<const float4*>(f.spoke)[2 * i + 1];
    const float2 a2 = reinterpret_cast<const float2*>(f.adf)[l];
    const dflt al = {a2.x, a2.y};
    dflt ph = df_mul(al, dflt{sA.z, sA.w});
    ph = df_add(ph, dflt{sA.x, sA.y});
    ph = df_mul(al, ph);
    ph = df_add(ph, dflt{f.A0[0], f.A0[1]});
    const float phr = df_reduce_2pi(ph);
    const float w = f.awf[l] * f.bcf[i];
    float sn, cs;
    sincosf(phr, &sn, &cs);
    dflt v1 = df_add(df_mul(al, dflt{sG.x, sG.y}), dflt{f.G0x[0], f.G0x[1]});
    dflt v2 = df_add(df_mul(al, dflt{sG.z, sG.w}), dflt{f.G0y[0], f.G0y[1]});
    float cre = w * cs, cim = w * sn;
    if (scr.n1) {   // the node itself, c + alpha (X_i - c), in FP32
        const float x = (float)f.cx + al.hi * (float)f.bx[i];
        const float y = (float)f.cy + al.hi * (float)f.by[i];
        apply_screen<float>(scr, cp.screen_k, x, y, cre, cim);
    }
    finish_df(v1, v2, cre, cim, cp, rec + f.offset + j, status, key);
}

// Starshade petals in the double-float form: node (k, i, l) is table entry
// (i, l) of petal 0 rotated to petal k, whose rotation is folded into the
// per-petal slopes (Sec. 4.2 nodes; no FP64 per node).
__device__ __forceinline__ void node_petal_df(const FamilyDev& f, const ChirpParams& cp,
                                              long long j, NodeRec<float>* rec, unsigned* status,
                                              int key[4], const ScreenDev& scr) {
    const unsigned k = (unsigned)j / (unsigned)f.n_bdry;   // j < 2^30
    const unsigned q = (unsigned)j - k * (unsigned)f.n_bdry;
    const float4 t0 = reinterpret_cast<const float4*>(f.ptab)[2 * q];
    const float4 t1 = reinterpret_cast<const float4*>(f.ptab)[2 * q + 1];
    const dflt u = {t0.x, t0.y}, v = {t0.z, t0.w};
    const float* K = f.pk + kPetalK * k;   // slopes, then the petal's own A0, G0x, G0y
    dflt ph = df_add(df_mul(u, dflt{K[0], K[1]}), df_mul(v, dflt{K[2], K[3]}));
    ph = df_add(ph, df_add(dflt{t1.x, t1.y}, dflt{K[12], K[13]}));
    const float phr = df_reduce_2pi(ph);
    float sn, cs;
    sincosf(phr, &sn, &cs);
    dflt v1 = df_add(df_add(df_mul(u, dflt{K[4], K[5]}), df_mul(v, dflt{K[6], K[7]})),
                     dflt{K[14], K[15]});
    dflt v2 = df_add(df_add(df_mul(u, dflt{K[8], K[9]}), df_mul(v, dflt{K[10], K[11]})),
                     dflt{K[16], K[17]});
    float cre = t1.z * cs, cim = t1.z * sn;
    if (scr.n1) {   // the node itself: petal 0's (u, v) moved to petal k, in FP32
        const float c = (float)f.rot[2 * k], sr = (float)f.rot[2 * k + 1];
        float x = (float)f.cx + (u.hi * c - v.hi * sr);
        float y = (float)f.cy + (u.hi * sr + v.hi * c);
        if (f.shift) {
            x += (float)f.shift[2 * k];
            y += (float)f.shift[2 * k + 1];
        }
        apply_screen<float>(scr, cp.screen_k, x, y, cre, cim);
    }
    finish_df(v1, v2, cre, cim, cp, rec + f.offset + j, status, key);
}

// Double-float table of a triangle family (FP32 fast mode), from its FP64
// vertices: v0 + c, v1 - v0, v2 - v1 as (hi, lo) pairs and the FP32 cross
// product (v1 - v0) x (v2 - v1).
__global__ void k_tri_df_tables(FamilyDev f) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= f.n_panels) return;
    const double* v = f.params + 6 * t;
    const double d1x = v[2] - v[0], d1y = v[3] - v[1], ex = v[4] - v[2], ey = v[5] - v[3];
    float* o = f.tdf + 16 * t;
    split_store(o + 0, f.cx + v[0]);
    split_store(o + 2, f.cy + v[1]);
    split_store(o + 4, d1x);
    split_store(o + 6, d1y);
    split_store(o + 8, ex);
    split_store(o + 10, ey);
    o[12] = (float)(d1x * ey - d1y * ex);
    o[13] = o[14] = o[15] = 0.0f;
}

// Double-float table of a petal family (FP32 fast mode), from its FP64 table.
__global__ void k_petal_df_tables(FamilyDev f, ChirpParams cp) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= f.n_bdry) return;
    const double u = f.bx[q], v = f.by[q];
    const double R = reduce_phase(cp.kq * (u * u + v * v));
    float* t = f.ptab + 8 * q;
    split_store(t + 0, u);
    split_store(t + 2, v);
    split_store(t + 4, R);
    t[6] = (float)f.bc[q];
    t[7] = 0.0f;
}

// Triangle-union nodes in the double-float form (FP32 fast mode, no FP64
// per node): x = v0 + alpha_l ((v1 - v0) + s_i (v2 - v1)) with s = alpha the
// family's Gauss rule on (0, 1), w = alpha_l what_l what_i (v1 - v0) x (v2 - v1)
// (Sec. 4.3 with eqs. aqnod, aqwei), then the chirp phase and the grid
// coordinate from the family's double-float constants.
__device__ __forceinline__ void node_tri_df(const FamilyDev& f, const ChirpParams& cp, long long j,
                                            NodeRec<float>* rec, unsigned* status, int key[4],
                                            const ScreenDev& scr) {
    const unsigned pp = (unsigned)(f.p * f.p);                     // j < 2^30
    const unsigned t = (unsigned)j / pp, q = (unsigned)j - t * pp;
    const unsigned i = q / (unsigned)f.p, l = q - i * (unsigned)f.p;
    const float4* T = reinterpret_cast<const float4*>(f.tdf) + 4 * (size_t)t;
    const float4 A = T[0], B = T[1], C = T[2];
    const float cross = T[3].x;
    const float2 s2 = reinterpret_cast<const float2*>(f.adf)[i];
    const float2 a2 = reinterpret_cast<const float2*>(f.adf)[l];
    const dflt s = {s2.x, s2.y}, a = {a2.x, a2.y};
    const dflt rx = df_add(dflt{B.x, B.y}, df_mul(s, dflt{C.x, C.y}));
    const dflt ry = df_add(dflt{B.z, B.w}, df_mul(s, dflt{C.z, C.w}));
    const dflt x = df_add(dflt{A.x, A.y}, df_mul(a, rx));
    const dflt y = df_add(dflt{A.z, A.w}, df_mul(a, ry));
    const float w = f.awf[l] * f.wpf[i] * cross;
    dflt ph = df_mul(dflt{f.tk[0], f.tk[1]}, df_add(df_mul(x, x), df_mul(y, y)));
    ph = df_add(ph, df_mul(dflt{f.tk[2], f.tk[3]}, x));
    ph = df_add(ph, df_mul(dflt{f.tk[4], f.tk[5]}, y));
    ph = df_add(ph, dflt{f.A0[0], f.A0[1]});
    float sn, cs;
    sincosf(df_reduce_2pi(ph), &sn, &cs);
    float cre = w * cs, cim = w * sn;
    if (scr.n1) apply_screen<float>(scr, cp.screen_k, x.hi, y.hi, cre, cim);
    const dflt v1 = df_add(df_mul(x, dflt{f.tk[6], f.tk[7]}), dflt{f.G0x[0], f.G0x[1]});
    const dflt v2 = df_add(df_mul(y, dflt{f.tk[8], f.tk[9]}), dflt{f.G0y[0], f.G0y[1]});
    finish_df(v1, v2, cre, cim, cp, rec + f.offset + j, status, key);
}

template <typename T>
__device__ __forceinline__ void node_generic(const FamilyDev& f, const ChirpParams& cp, long long j,
                                             NodeRec<T>* rec, double* dx, double* dy, double* dw,
                                             unsigned* status, int key[4], const ScreenDev& scr) {
    double x, y, w;
    if (f.kind == FRESNEL_FAMILY_NODES) {
        x = f.params[j];
        y = f.params[f.n_nodes + j];
        w = f.params[2 * f.n_nodes + j];
    } else if (f.kind == FRESNEL_FAMILY_TRIANGLES) {
        // triangle t, edge node i on v1 -> v2, radius l about v0 (Sec. 4.3):
        // x = v0 + alpha_l (X_i - v0), w = alpha_l what_l what_i (v1 - v0) x (v2 - v1)
        const unsigned pp = (unsigned)(f.p * f.p);                 // j < 2^30
        const unsigned t = (unsigned)j / pp, q = (unsigned)j - t * pp;
        const unsigned i = q / (unsigned)f.p, l = q - i * (unsigned)f.p;
        const double* v = f.params + 6 * (size_t)t;
        const double d1x = v[2] - v[0], d1y = v[3] - v[1];         // v1 - v0
        const double ex = v[4] - v[2], ey = v[5] - v[3];           // v2 - v1
        const double s = f.gl_m_a[i], a = f.gl_m_a[l];
        x = f.cx + v[0] + a * (d1x + s * ex);
        y = f.cy + v[1] + a * (d1y + s * ey);
        w = f.gl_m_aw[l] * f.gl_p_w[i] * (d1x * ey - d1y * ex);
    } else if (f.kind == FRESNEL_FAMILY_PETALS) {
        // node (k, i, l) = petal 0's node (i, l) rotated by 2 pi k / Np
        const unsigned k = (unsigned)j / (unsigned)f.n_bdry;   // j < 2^30
        const unsigned q = (unsigned)j - k * (unsigned)f.n_bdry;
        const double u = f.bx[q], v = f.by[q];
        const double c = f.rot[2 * k], s = f.rot[2 * k + 1];
        x = f.cx + (u * c - v * s);
        y = f.cy + (u * s + v * c);
        if (f.shift) {   // a rigidly moved petal (rotation folded into rot)
            x += f.shift[2 * k];
            y += f.shift[2 * k + 1];
        }
        w = f.bc[q];
    } else {
        const unsigned i = (unsigned)j / (unsigned)f.m;   // j < 2^30
        const int l = (int)((unsigned)j - i * (unsigned)f.m);
        double a = f.gl_m_a[l];
        x = f.cx + a * f.bx[i];
        y = f.cy + a * f.by[i];
        w = f.gl_m_aw[l] * f.bc[i];
    }
    long long g = f.offset + j;
    if (dx) {
        dx[g] = x;
        dy[g] = y;
        dw[g] = w;
    }
    double ph = reduce_phase(cp.kq * (x * x + y * y) - cp.a1 * x - cp.a2 * y + cp.a0);
    NodeRec<T> r;
    if (sizeof(T) == 8) {
        double sn, cs;
        sincos(ph, &sn, &cs);
        r.cre = (T)(w * cs);
        r.cim = (T)(w * sn);
    } else {
        float sn, cs;
        sincosf((float)ph, &sn, &cs);
        r.cre = (T)((float)w * cs);
        r.cim = (T)((float)w * sn);
    }
    if (scr.n1) apply_screen<T>(scr, cp.screen_k, (T)x, (T)y, r.cre, r.cim);
    double g1, g2;
    if (!cp.type3) {
        double u = x * cp.u1;
        u -= floor(u);
        g1 = u * cp.nf1 + cp.sh1;
        if (g1 >= cp.nf1) g1 -= cp.nf1;
        double v = y * cp.u2;
        v -= floor(v);
        g2 = v * cp.nf2 + cp.sh2;
        if (g2 >= cp.nf2) g2 -= cp.nf2;
    } else {
        g1 = (x - cp.C1) * cp.inv_h1 + 0.5 * cp.nf1;
        g2 = (y - cp.C2) * cp.inv_h2 + 0.5 * cp.nf2;
    }
    if (!isfinite(g1) || !isfinite(g2)) {
        atomicOr(status, kStatusNonFinite);
        g1 = g2 = 0.0;
        r.cre = r.cim = (T)0;
    }
    double gs1 = g1 - 0.5 * cp.w, gs2 = g2 - 0.5 * cp.w;
    double fl1 = floor(gs1), fl2 = floor(gs2);
    int s1 = (int)fl1 + 1, s2 = (int)fl2 + 1;
    r.f1 = (T)(gs1 - fl1);
    r.f2 = (T)(gs2 - fl2);
    if (!cp.type3) {
        if (s1 < 0) s1 += cp.nf1;
        if (s1 >= cp.nf1) s1 -= cp.nf1;
        if (s2 < 0) s2 += cp.nf2;
        if (s2 >= cp.nf2) s2 -= cp.nf2;
    } else if (s1 < 0 || s2 < 0 || s1 + cp.w > cp.nf1 || s2 + cp.w > cp.nf2) {
        atomicOr(status, kStatusNodeOutside);
        s1 = min(max(s1, 0), cp.nf1 - cp.w);
        s2 = min(max(s2, 0), cp.nf2 - cp.w);
    }
    r.s1 = s1;
    r.s2 = s2;
    rec[g] = r;
    node_tiles(s1, s2, cp, key);
}

// Block -> family (binary search over the block starts), then the family
// and its problem's chirp parameters are copied into shared memory.
struct FamSmem {
    FamilyDev f;
    ChirpParams cp;
    int fi, b0, prob;   // family, its first block, its problem
};

__device__ __forceinline__ void load_family(const FamTable& ft, FamSmem& sm) {
    if (threadIdx.x == 0) {
        int a = 0, b = ft.nfam - 1;
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (ft.blk0[mid] <= (int)blockIdx.x) a = mid;
            else b = mid - 1;
        }
        sm.fi = a;
        sm.b0 = ft.blk0[a];
        sm.prob = ft.fams[a].prob;
    }
    __syncthreads();
    // both records in one pass (the family's words, then its problem's)
    static_assert(sizeof(FamilyDev) % 4 == 0 && sizeof(ChirpParams) % 4 == 0, "word copy");
    constexpr int nf = (int)(sizeof(FamilyDev) / 4), nc = (int)(sizeof(ChirpParams) / 4);
    const int* src = reinterpret_cast<const int*>(ft.fams + sm.fi);
    const int* src2 = reinterpret_cast<const int*>(ft.cps + sm.prob);
    int* dst = reinterpret_cast<int*>(&sm.f);
    int* dst2 = reinterpret_cast<int*>(&sm.cp);
    for (int i = threadIdx.x; i < nf + nc; i += blockDim.x) {
        if (i < nf) dst[i] = src[i];
        else dst2[i - nf] = src2[i - nf];
    }
    __syncthreads();
}

// ------------------------------------------------------------------ nodes + chirp + count
// Dilation rule (eqs. aqnod, aqwei): x = c + alpha_l (X_i - c),
// w = alpha_l wtilde_l ((X_i-cx) V_i - (Y_i-cy) W_i), node j = i*m + l; the
// starshade petals (Sec. 4.2) from their tables; explicit nodes as given.
// Strength (Sec. 3.2 step 1, with the optional pre-phase of Sec. 3.3):
// c = w exp(i [pi |x|^2 / lz - a1 x - a2 y + a0]), phase reduced mod 2 pi
// before the sine/cosine.  Grid coordinate: type 1 g = frac(x h / lz) nf (the
// folded x~ of Sec. 3.3 scaled to grid points); type 3 g = (x - C)/h_s + nf/2.
// FP32 fast mode runs the dilation families in the double-float spoke form
// (no FP64 per node); FP64 per node otherwise.  One launch covers every
// family of every problem of the plan.
template <typename T>
__global__ void __launch_bounds__(kNodeThreads)
k_nodes(FamTable ft, NodeRec<T>* rec, int* counts, double* dx, double* dy, double* dw,
        unsigned* status) {
    __shared__ __align__(16) FamSmem sm;
    load_family(ft, sm);
    const FamilyDev& f = sm.f;
    const long long j = (long long)(blockIdx.x - sm.b0) * blockDim.x + threadIdx.x;
    int key[4] = {-1, -1, -1, -1};
    if (j < f.n_nodes) {
        if constexpr (sizeof(T) == 4) {
            if (f.spoke && !dx)
                node_df(f, sm.cp, j, reinterpret_cast<NodeRec<float>*>(rec), status, key, ft.scr);
            else if (f.ptab && !dx)
                node_petal_df(f, sm.cp, j, reinterpret_cast<NodeRec<float>*>(rec), status, key,
                              ft.scr);
            else if (f.tdf && !dx)
                node_tri_df(f, sm.cp, j, reinterpret_cast<NodeRec<float>*>(rec), status, key,
                            ft.scr);
            else
                node_generic<T>(f, sm.cp, j, rec, dx, dy, dw, status, key, ft.scr);
        } else {
            node_generic<T>(f, sm.cp, j, rec, dx, dy, dw, status, key, ft.scr);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) agg_count(key[k], counts);
}

// Scatter of a plan's records (families as in k_nodes) to every tile their
// support touches.
template <typename T>
__global__ void __launch_bounds__(kNodeThreads)
k_scatter_fams(FamTable ft, const NodeRec<T>* rec, int* cursor, NodeRec<T>* sorted,
               long long cap, unsigned* status) {
    __shared__ __align__(16) FamSmem sm;
    load_family(ft, sm);
    const FamilyDev& f = sm.f;
    const long long j = (long long)(blockIdx.x - sm.b0) * blockDim.x + threadIdx.x;
    int key[4] = {-1, -1, -1, -1};
    NodeRec<T> r;
    if (j < f.n_nodes) {
        r = rec[f.offset + j];
        node_tiles(r.s1, r.s2, sm.cp, key);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int pos = agg_reserve(key[k], cursor);
        if (key[k] >= 0) {
            if (pos >= 0 && pos < cap) sorted[pos] = r;
            else atomicOr(status, kStatusOverflow);
        }
    }
}

// Records for the standalone spreader (fresnel_spread): points given directly
// by periodic grid coordinates (g1, g2) and FP32 strengths.
__global__ void k_records_from_coords(long long n, const double* __restrict__ g1,
                                      const double* __restrict__ g2,
                                      const float2* __restrict__ c, ChirpParams cp,
                                      NodeRec<float>* __restrict__ rec, int* __restrict__ counts,
                                      unsigned* __restrict__ status) {
    long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int key[4] = {-1, -1, -1, -1};
    if (j < n) {
        double a = g1[j] - 0.5 * cp.w, b = g2[j] - 0.5 * cp.w;
        NodeRec<float> r;
        float2 cj = c[j];
        if (!isfinite(a) || !isfinite(b)) {
            atomicOr(status, kStatusNonFinite);
            a = b = 0.0;
            cj = make_float2(0.0f, 0.0f);
        }
        a -= cp.nf1 * floor(a / cp.nf1);
        b -= cp.nf2 * floor(b / cp.nf2);
        const double fa = floor(a), fb = floor(b);
        r.f1 = (float)(a - fa);
        r.f2 = (float)(b - fb);
        r.s1 = (((int)fa + 1) % cp.nf1 + cp.nf1) % cp.nf1;
        r.s2 = (((int)fb + 1) % cp.nf2 + cp.nf2) % cp.nf2;
        r.cre = cj.x;
        r.cim = cj.y;
        rec[j] = r;
        node_tiles(r.s1, r.s2, cp, key);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) agg_count(key[k], counts);
}

// Scatter each record to every tile its support touches (positions reserved
// with warp-aggregated atomics on per-tile cursors set by the scan).
template <typename T>
__global__ void k_scatter(long long n, ChirpParams cp, const NodeRec<T>* rec, int* cursor,
                          NodeRec<T>* sorted, long long cap, unsigned* status) {
    long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int key[4] = {-1, -1, -1, -1};
    NodeRec<T> r;
    if (j < n) {
        r = rec[j];
        node_tiles(r.s1, r.s2, cp, key);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int pos = agg_reserve(key[k], cursor);
        if (key[k] >= 0) {
            if (pos >= 0 && pos < cap) sorted[pos] = r;
            else atomicOr(status, kStatusNodeOutside);
        }
    }
}

// ------------------------------------------------------------------ scan -> chunks
// One block: exclusive scan of per-tile record counts.  A tile with more than
// chunk_cap records becomes ceil(count / cap) chunks and is listed in
// split_tiles; every other tile (empty ones too: they write zeros, so the grid
// needs no separate clearing) is one chunk.  Chunks of split tiles are placed
// first, the unsplit tiles after them.  Resets counts for the next pass.
// When the counts fit in shared memory (staged = 1) they are first copied in
// one coalesced burst and the global copy is cleared at once, so the block
// pays one memory round trip instead of one per tile it owns.
__global__ void k_scan_chunks(int ntiles, int* __restrict__ counts, int* __restrict__ cursor,
                              Chunk* __restrict__ chunks, int* __restrict__ n_meta,
                              int* __restrict__ split_tiles, int chunk_cap, int max_chunks,
                              int max_split, int staged) {
    __shared__ long long s_rec[1024], s_sc[1024], s_ns[1024], s_st[1024];
    extern __shared__ int s_counts[];
    int t = threadIdx.x, nt = blockDim.x;
    const int* cnt = counts;
    if (staged) {
        for (int i = t; i < ntiles; i += nt) {
            s_counts[i] = counts[i];
            counts[i] = 0;
        }
        __syncthreads();
        cnt = s_counts;
    }
    int per = (ntiles + nt - 1) / nt;
    int lo = min(t * per, ntiles), hi = min(lo + per, ntiles);
    long long rsum = 0, sc = 0, ns = 0, stl = 0;
    for (int i = lo; i < hi; ++i) {
        int c = cnt[i];
        rsum += c;
        if (c > chunk_cap) {
            sc += (c + chunk_cap - 1) / chunk_cap;
            ++stl;
        } else {
            ++ns;
        }
    }
    s_rec[t] = rsum;
    s_sc[t] = sc;
    s_ns[t] = ns;
    s_st[t] = stl;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {   // Hillis-Steele inclusive scans
        long long a = 0, b = 0, c = 0, d = 0;
        if (t >= off) { a = s_rec[t - off]; b = s_sc[t - off]; c = s_ns[t - off]; d = s_st[t - off]; }
        __syncthreads();
        s_rec[t] += a; s_sc[t] += b; s_ns[t] += c; s_st[t] += d;
        __syncthreads();
    }
    const long long total_split_chunks = s_sc[nt - 1];
    // staged: per split tile (in order) its first chunk, record offset and count
    int* s_cstart = s_counts + ntiles;
    int* s_sroff = s_cstart + ntiles + 1;
    int* s_scnt = s_sroff + ntiles;
    long long roff = s_rec[t] - rsum, scoff = s_sc[t] - sc, nsoff = s_ns[t] - ns, stoff = s_st[t] - stl;
    for (int i = lo; i < hi; ++i) {
        int c = cnt[i];
        cursor[i] = (int)roff;
        if (c > chunk_cap) {
            int nch = (c + chunk_cap - 1) / chunk_cap;
            if (staged) {   // chunks written below, in parallel over the block
                s_cstart[stoff] = (int)scoff;
                s_sroff[stoff] = (int)roff;
                s_scnt[stoff] = c;
            } else {
                for (int k = 0; k < nch; ++k) {
                    long long ci = scoff + k;
                    if (ci < max_chunks) {
                        Chunk ch;
                        ch.tile = i;
                        ch.begin = (int)(roff + (long long)k * chunk_cap);
                        ch.end = (int)min(roff + (long long)(k + 1) * chunk_cap, roff + c);
                        ch.split = stoff < max_split ? split_code((int)stoff, k == 0) : 1;
                        chunks[ci] = ch;
                    }
                }
            }
            scoff += nch;
            if (stoff < max_split) split_tiles[stoff] = i;
            ++stoff;
        } else {
            long long ci = total_split_chunks + nsoff;
            if (ci < max_chunks) {
                Chunk ch;
                ch.tile = i;
                ch.begin = (int)roff;
                ch.end = (int)(roff + c);
                ch.split = 0;
                chunks[ci] = ch;
            }
            ++nsoff;
        }
        roff += c;
        if (!staged) counts[i] = 0;
    }
    if (staged) {
        const int nsplit = (int)s_st[nt - 1];
        if (t == 0) s_cstart[nsplit] = (int)total_split_chunks;
        __syncthreads();
        // chunk ci of the split tiles: find its tile by binary search
        for (long long ci = t; ci < total_split_chunks && ci < max_chunks; ci += nt) {
            int a = 0, b = nsplit - 1;
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (s_cstart[mid] <= ci) a = mid;
                else b = mid - 1;
            }
            const int k = (int)(ci - s_cstart[a]);
            const long long r0 = s_sroff[a], c = s_scnt[a];
            Chunk ch;
            ch.tile = split_tiles[a];
            ch.begin = (int)(r0 + (long long)k * chunk_cap);
            ch.end = (int)min(r0 + (long long)(k + 1) * chunk_cap, r0 + c);
            ch.split = a < max_split ? split_code(a, k == 0) : 1;
            chunks[ci] = ch;
        }
    }
    if (t == nt - 1) {
        n_meta[0] = (int)min(total_split_chunks + s_ns[t], (long long)max_chunks);
        n_meta[1] = (int)min(s_st[t], (long long)max_split);
    }
}

// Batched plans: block b scans problem b's tiles [b ntiles, (b+1) ntiles).
// Cursors are absolute positions from rec_off[b]; split tiles (count > cap)
// give ceil(count / cap) chunks in the problem's split-chunk region, every
// other tile one chunk in its plain region, split tiles are listed in its
// split-tile region.  The regions were sized at plan time from the same
// deterministic counts; unused entries are padded (empty split-flagged
// chunks add nothing, split-tile entries -1 are skipped) and a count beyond
// a region sets kStatusOverflow (the entries beyond it are dropped).
// Clears the counts.
__global__ void __launch_bounds__(1024)
k_scan_problems(int ntiles, int* __restrict__ counts, int* __restrict__ cursor,
                Chunk* __restrict__ chunks, int* __restrict__ split_tiles, ScanLayout L,
                int chunk_cap, int staged, unsigned* __restrict__ status) {
    __shared__ long long s_rec[1024], s_sc[1024], s_ns[1024], s_st[1024];
    extern __shared__ int s_counts[];
    const int t = threadIdx.x, nt = blockDim.x, b = blockIdx.x;
    const int base = b * ntiles;
    int* cnt_g = counts + base;
    int* cur = cursor + base;
    const int sc0 = L.sc_off[b], sc1 = L.sc_off[b + 1];
    const int pl0 = L.pl_off[b], pl1 = L.pl_off[b + 1];
    const int st0 = L.st_off[b], st1 = L.st_off[b + 1];
    const long long r0 = L.rec_off[b], r1 = L.rec_off[b + 1];
    const int* cnt = cnt_g;
    __shared__ int s_live[kMaxTileRows];
    if (staged) {
        for (int i = t; i < ntiles; i += nt) {
            s_counts[i] = cnt_g[i];
            cnt_g[i] = 0;
        }
        cnt = s_counts;
    }
    // tile rows holding records (all rows live when no live map is kept)
    for (int r = t; r < L.nty && r < kMaxTileRows; r += nt) s_live[r] = L.live ? 0 : 1;
    __syncthreads();
    if (L.live) {
        for (int i = t; i < ntiles; i += nt)
            if (cnt[i] > 0) s_live[i / L.ntx] = 1;
        __syncthreads();
        for (int r = t; r < L.nty; r += nt) L.live[b * L.nty + r] = s_live[r];
    }
    const int per = (ntiles + nt - 1) / nt;
    const int lo = min(t * per, ntiles), hi = min(lo + per, ntiles);
    long long rsum = 0, sc = 0, ns = 0, stl = 0;
    for (int i = lo; i < hi; ++i) {
        const int c = cnt[i];
        rsum += c;
        if (c > chunk_cap) {
            sc += (c + chunk_cap - 1) / chunk_cap;
            ++stl;
        } else if (!L.live || s_live[i / L.ntx]) {
            ++ns;
        }
    }
    {   // inclusive block scans of the four sums: warp shuffles, then warp totals
        __shared__ long long w_tot[4][32];
        const int lane = t & 31, wid = t >> 5, nwarp = (nt + 31) >> 5;
        auto wscan = [&](long long v) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            return v;
        };
        long long inc[4] = {wscan(rsum), wscan(sc), wscan(ns), wscan(stl)};
        if (lane == 31)
            for (int q = 0; q < 4; ++q) w_tot[q][wid] = inc[q];
        __syncthreads();
        if (wid == 0)
            for (int q = 0; q < 4; ++q) {
                const long long v = lane < nwarp ? w_tot[q][lane] : 0;
                w_tot[q][lane] = wscan(v) - v;
            }
        __syncthreads();
        s_rec[t] = inc[0] + w_tot[0][wid];
        s_sc[t] = inc[1] + w_tot[1][wid];
        s_ns[t] = inc[2] + w_tot[2][wid];
        s_st[t] = inc[3] + w_tot[3][wid];
        __syncthreads();
    }
    const long long TS = s_sc[nt - 1], NS = s_ns[nt - 1], TST = s_st[nt - 1], RT = s_rec[nt - 1];
    if (t == 0 && (TS > sc1 - sc0 || NS > pl1 - pl0 || TST > st1 - st0 || RT > r1 - r0))
        atomicOr(status, kStatusOverflow);
    int* s_cstart = s_counts + ntiles;
    int* s_sroff = s_cstart + ntiles + 1;
    int* s_scnt = s_sroff + ntiles;
    long long roff = s_rec[t] - rsum, scoff = s_sc[t] - sc, nsoff = s_ns[t] - ns, stoff = s_st[t] - stl;
    for (int i = lo; i < hi; ++i) {
        const int c = cnt[i];
        cur[i] = (int)(r0 + roff);
        if (c > chunk_cap) {
            const int nch = (c + chunk_cap - 1) / chunk_cap;
            if (staged) {   // chunks written below, in parallel over the block
                s_cstart[stoff] = (int)scoff;
                s_sroff[stoff] = (int)roff;
                s_scnt[stoff] = c;
            } else {
                for (int k = 0; k < nch; ++k) {
                    const long long ci = sc0 + scoff + k;
                    if (ci < sc1) {
                        Chunk ch;
                        ch.tile = base + i;
                        ch.begin = (int)(r0 + roff + (long long)k * chunk_cap);
                        ch.end = (int)(r0 + min(roff + (long long)(k + 1) * chunk_cap, roff + c));
                        ch.split = st0 + stoff < st1 ? split_code((int)(st0 + stoff), k == 0) : 1;
                        chunks[ci] = ch;
                    }
                }
            }
            scoff += nch;
            if (st0 + stoff < st1) split_tiles[st0 + stoff] = base + i;
            ++stoff;
        } else if (!L.live || s_live[i / L.ntx]) {
            const long long ci = pl0 + nsoff;
            if (ci < pl1) {
                Chunk ch;
                ch.tile = base + i;
                ch.begin = (int)(r0 + roff);
                ch.end = (int)(r0 + roff + c);
                ch.split = 0;
                chunks[ci] = ch;
            }
            ++nsoff;
        }
        roff += c;
        if (!staged) cnt_g[i] = 0;
    }
    if (staged) {
        const int nsplit = (int)TST;
        if (t == 0) s_cstart[nsplit] = (int)TS;
        __syncthreads();
        for (long long ci = t; ci < TS && sc0 + ci < sc1; ci += nt) {
            int a = 0, bb = nsplit - 1;
            while (a < bb) {
                const int mid = (a + bb + 1) >> 1;
                if (s_cstart[mid] <= ci) a = mid;
                else bb = mid - 1;
            }
            if (st0 + a >= st1) continue;   // region overflow (already flagged)
            const int k = (int)(ci - s_cstart[a]);
            const long long ro = s_sroff[a], c = s_scnt[a];
            Chunk ch;
            ch.tile = split_tiles[st0 + a];
            ch.begin = (int)(r0 + ro + (long long)k * chunk_cap);
            ch.end = (int)(r0 + min(ro + (long long)(k + 1) * chunk_cap, ro + c));
            ch.split = split_code(st0 + a, k == 0);
            chunks[sc0 + ci] = ch;
        }
    }
    // padding of unused region entries
    for (long long ci = sc0 + TS + t; ci < sc1; ci += nt) chunks[ci] = Chunk{base, 0, 0, 1};
    for (long long ci = pl0 + NS + t; ci < pl1; ci += nt) chunks[ci] = Chunk{base, 0, 0, 1};
    for (long long i = st0 + TST + t; i < st1; i += nt) split_tiles[i] = -1;
}

// ------------------------------------------------------------------ plan-time tables
__global__ void k_twiddles(int n, void* table, int is_double) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s, c;
    sincospi(-2.0 * j / n, &s, &c);
    if (is_double) ((double2*)table)[j] = make_double2(c, s);
    else ((float2*)table)[j] = make_float2((float)c, (float)s);
}

// Output factors of the type-1 path (Sec. 3.3 step 3 and the deconvolution):
// A[k'] = exp(i pi xi^2 / lz) / psihat(2 pi k / nf) [* 1/(i lz)],
// xi = x0 + k h, k = k' - floor(n/2).  FP64, phase reduced mod 2 pi.
__global__ void k_t1_tables(int n, int nf, double h, double x0, double lz, int w, double beta,
                            int with_ilz, int shift, void* table, int is_double,
                            const double* gq_t, const double* gq_w, int q) {
    int kp = blockIdx.x * blockDim.x + threadIdx.x;
    if (kp >= n) return;
    int k = kp - n / 2;
    double xi = x0 + k * h;
    double ph = reduce_phase(kPi * xi * xi / lz);
    double s, c;
    sincos(ph, &s, &c);
    // undo the spreading shift: exp(2 pi i k shift / nf), argument exact mod nf
    long long m = ((long long)k * shift) % nf;
    if (m < 0) m += nf;
    double ss, cs;
    sincospi(2.0 * (double)m / nf, &ss, &cs);
    const double c2 = c * cs - s * ss, s2 = s * cs + c * ss;
    c = c2;
    s = s2;
    double inv = 1.0 / kernel_ft(kTwoPi * k / nf, w, beta, gq_t, gq_w, q);
    double re = c * inv, im = s * inv;
    if (with_ilz) {   // times 1/(i lz) = -i / lz
        double r2 = im / lz, i2 = -re / lz;
        re = r2;
        im = i2;
    }
    if (is_double) ((double2*)table)[kp] = make_double2(re, im);
    else ((float2*)table)[kp] = make_float2((float)re, (float)im);
}

// Type-3 inner type-2 deconvolution: 1 / psihat(2 pi l / nfft), l = i - ng/2.
__global__ void k_t3_deconv(int ng, int nfft, int w, double beta, void* table, int is_double,
                            const double* gq_t, const double* gq_w, int q) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    int l = i - ng / 2;
    double v = 1.0 / kernel_ft(kTwoPi * l / nfft, w, beta, gq_t, gq_w, q);
    if (is_double) ((double*)table)[i] = v;
    else ((float*)table)[i] = (float)v;
}

inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_gauss_legendre(int n, double* t01, double* w01, cudaStream_t st) {
    const size_t dyn = sizeof(double) * ((size_t)n + 1);
    const int blocks = nblk((n + 1) / 2, 64);
    if (dyn <= 48 * 1024) {
        k_gauss_legendre<true><<<blocks, 64, dyn, st>>>(n, t01, w01);
    } else {
        k_gauss_legendre<false><<<blocks, 64, 0, st>>>(n, t01, w01);
    }
}

void launch_boundary(const FamilyDev& f, const ChirpParams& cp, cudaStream_t st) {
    if (f.kind == FRESNEL_FAMILY_FOURIER)
        k_boundary_fourier<<<nblk(f.n_bdry, 128), 128, 0, st>>>(f, cp);
    else if (f.kind == FRESNEL_FAMILY_LINE_RULE)
        k_boundary_line<<<nblk(f.n_bdry, 128), 128, 0, st>>>(f, cp);
    else if (f.kind == FRESNEL_FAMILY_PETALS && !f.ptab)
        k_petal_tables<<<nblk(std::max<long long>(f.n_bdry, f.n_panels), 128), 128, 0, st>>>(f);
    else if (f.kind == FRESNEL_FAMILY_PETALS)
        k_petal_df_tables<<<nblk(f.n_bdry, 128), 128, 0, st>>>(f, cp);
    else if (f.kind == FRESNEL_FAMILY_TRIANGLES && f.tdf)
        k_tri_df_tables<<<nblk(f.n_panels, 128), 128, 0, st>>>(f);
}

template <typename T>
void launch_nodes(const FamTable& ft, int nblocks, NodeRec<T>* rec, int* counts, double* dx,
                  double* dy, double* dw, unsigned* status, cudaStream_t st) {
    if (nblocks <= 0) return;
    k_nodes<T><<<nblocks, kNodeThreads, 0, st>>>(ft, rec, counts, dx, dy, dw, status);
}
template void launch_nodes<float>(const FamTable&, int, NodeRec<float>*, int*, double*, double*,
                                  double*, unsigned*, cudaStream_t);
template void launch_nodes<double>(const FamTable&, int, NodeRec<double>*, int*, double*,
                                   double*, double*, unsigned*, cudaStream_t);

template <typename T>
void launch_scatter_fams(const FamTable& ft, int nblocks, const NodeRec<T>* rec, int* cursor,
                         NodeRec<T>* sorted, long long cap, unsigned* status, cudaStream_t st) {
    if (nblocks <= 0) return;
    k_scatter_fams<T><<<nblocks, kNodeThreads, 0, st>>>(ft, rec, cursor, sorted, cap, status);
}
template void launch_scatter_fams<float>(const FamTable&, int, const NodeRec<float>*, int*,
                                         NodeRec<float>*, long long, unsigned*, cudaStream_t);
template void launch_scatter_fams<double>(const FamTable&, int, const NodeRec<double>*, int*,
                                          NodeRec<double>*, long long, unsigned*, cudaStream_t);

void launch_scan_problems(int B, int ntiles, int* counts, int* cursor, Chunk* chunks,
                          int* split_tiles, const ScanLayout& L, int chunk_cap, unsigned* status,
                          cudaStream_t st) {
    const size_t dyn = sizeof(int) * (4 * (size_t)ntiles + 1);
    const int staged = dyn <= 160 * 1024 ? 1 : 0;
    if (staged)
        cudaFuncSetAttribute(k_scan_problems, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
    k_scan_problems<<<B, 1024, staged ? dyn : 0, st>>>(ntiles, counts, cursor, chunks,
                                                       split_tiles, L, chunk_cap, staged, status);
}

template <typename T>
void launch_scatter(long long n, const ChirpParams& cp, const NodeRec<T>* rec, int* cursor,
                    NodeRec<T>* sorted, long long cap, unsigned* status, cudaStream_t st) {
    if (n <= 0) return;
    k_scatter<T><<<nblk(n, 256), 256, 0, st>>>(n, cp, rec, cursor, sorted, cap, status);
}
template void launch_scatter<float>(long long, const ChirpParams&, const NodeRec<float>*, int*,
                                    NodeRec<float>*, long long, unsigned*, cudaStream_t);
template void launch_scatter<double>(long long, const ChirpParams&, const NodeRec<double>*, int*,
                                     NodeRec<double>*, long long, unsigned*, cudaStream_t);

void launch_records_from_coords(long long n, const double* g1, const double* g2, const float2* c,
                                const ChirpParams& cp, NodeRec<float>* rec, int* counts,
                                unsigned* status, cudaStream_t st) {
    if (n <= 0) return;
    k_records_from_coords<<<nblk(n, 256), 256, 0, st>>>(n, g1, g2, c, cp, rec, counts, status);
}

void launch_scan_chunks(int ntiles, int* counts, int* cursor, Chunk* chunks, int* n_meta,
                        int* split_tiles, int chunk_cap, int max_chunks, int max_split,
                        cudaStream_t st) {
    // counts staged in shared memory when they fit next to the static arrays
    const size_t dyn = sizeof(int) * (4 * (size_t)ntiles + 1);   // counts + split-tile tables
    const int staged = dyn <= 160 * 1024 ? 1 : 0;
    if (staged)
        cudaFuncSetAttribute(k_scan_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
    k_scan_chunks<<<1, 1024, staged ? dyn : 0, st>>>(ntiles, counts, cursor, chunks, n_meta,
                                                     split_tiles, chunk_cap, max_chunks,
                                                     max_split, staged);
}

void launch_twiddles(int n, void* table, int is_double, cudaStream_t st) {
    k_twiddles<<<nblk(n, 256), 256, 0, st>>>(n, table, is_double);
}

void launch_t1_tables(int n, int nf, double h, double x0, double lz, int w, double beta,
                      int with_ilz, int shift, void* table, int is_double, const double* gq_t,
                      const double* gq_w, int q, cudaStream_t st) {
    k_t1_tables<<<nblk(n, 128), 128, 0, st>>>(n, nf, h, x0, lz, w, beta, with_ilz, shift, table,
                                              is_double, gq_t, gq_w, q);
}

void launch_t3_deconv(int ng, int nfft, int w, double beta, void* table, int is_double,
                      const double* gq_t, const double* gq_w, int q, cudaStream_t st) {
    k_t3_deconv<<<nblk(ng, 128), 128, 0, st>>>(ng, nfft, w, beta, table, is_double, gq_t,
                                               gq_w, q);
}

}  // namespace fres
