// Hand-written 2D FFT for the NUFFT fine grid: batched 1D mixed-radix
// (4, 2, 3, 5) Stockham transforms held in shared memory, one pass along rows
// (contiguous) and one along columns (a CTA takes C adjacent columns so global
// accesses stay coalesced).  Forward sign e^{-2 pi i k l / n}, unnormalised.
//
// The FFT is the middle step of the type-1 and type-3 NUFFTs used by the
// paper's fast algorithm (arXiv:2010.05978, Secs. 3.2-3.3; "under the hood the
// NUFFT uses FFTs", Sec. 4.1).  Both passes are pruned to what the path needs:
// the type-1 row pass keeps only the n1 wanted modes; the type-1 column pass
// keeps n2 modes and applies the fused output epilogue (deconvolution, target
// chirp, 1/(i lz), Babinet); the type-3 passes read only the nonzero central
// block of the zero-padded grid and fuse the inner type-2 deconvolution.
//
// Each Stockham stage with radix r and p = product of earlier radices maps
// butterfly i (k = i mod p) from inputs x[i + q n/r] (twiddled by
// w_n^{q k n/(p r)}) to outputs y[(i - k) r + k + t p]; stages ping-pong
// between two shared-memory buffers with one barrier each.  The first stage
// reads its inputs straight from global memory and the last writes its
// outputs straight to global memory (through the pruning and the epilogue),
// so a transform makes no separate staging passes.
#include "internal.cuh"

namespace fres {

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftBlocksPerSm = 3;
constexpr long long kFftSmemTarget = 76 * 1024;   // three blocks per SM

template <typename T> struct Ops {
    using C = cx_t<T>;
    static __device__ __forceinline__ C mk(T a, T b) { C c; c.x = a; c.y = b; return c; }
    static __device__ __forceinline__ C add(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ C sub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
    static __device__ __forceinline__ C mul(C a, C b) {
        return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    static __device__ __forceinline__ C scale(C a, T s) { return mk(a.x * s, a.y * s); }
    static __device__ __forceinline__ C mul_negi(C a) { return mk(a.y, -a.x); }   // -i a
};

// In-register DFTs y_t = sum_q u_q e^{-2 pi i q t / R}.  Radix 8 is two
// radix-4 halves joined by w_8^k; radix 16 is 4 x 4 with w_16^{n2 k1}
// twiddles between the two radix-4 layers (Cooley-Tukey in registers).
template <typename T, int R> struct Dft;
template <typename T> struct Dft<T, 2> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        y[0] = Ops<T>::add(u[0], u[1]);
        y[1] = Ops<T>::sub(u[0], u[1]);
    }
};
template <typename T> struct Dft<T, 4> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        using O = Ops<T>;
        C t0 = O::add(u[0], u[2]), t1 = O::sub(u[0], u[2]);
        C t2 = O::add(u[1], u[3]), t3 = O::mul_negi(O::sub(u[1], u[3]));
        y[0] = O::add(t0, t2);
        y[2] = O::sub(t0, t2);
        y[1] = O::add(t1, t3);
        y[3] = O::sub(t1, t3);
    }
};
template <typename T> struct Dft<T, 3> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        using O = Ops<T>;
        const T c3 = (T)-0.5, s3 = (T)0.86602540378443864676372317075294;
        C s = O::add(u[1], u[2]), d = O::sub(u[1], u[2]);
        C a = O::add(u[0], O::scale(s, c3));
        C b = O::mul_negi(O::scale(d, s3));   // -i s3 (u1 - u2)
        y[0] = O::add(u[0], s);
        y[1] = O::add(a, b);
        y[2] = O::sub(a, b);
    }
};
template <typename T> struct Dft<T, 5> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        using O = Ops<T>;
        const T c1 = (T)0.30901699437494742410229341718282;   // cos(2 pi/5)
        const T s1 = (T)0.95105651629515357211643933337938;   // sin(2 pi/5)
        const T c2 = (T)-0.80901699437494742410229341718282;  // cos(4 pi/5)
        const T s2 = (T)0.58778525229247312916870595463907;   // sin(4 pi/5)
        C a14 = O::add(u[1], u[4]), d14 = O::sub(u[1], u[4]);
        C a23 = O::add(u[2], u[3]), d23 = O::sub(u[2], u[3]);
        C r1 = O::add(u[0], O::add(O::scale(a14, c1), O::scale(a23, c2)));
        C r2 = O::add(u[0], O::add(O::scale(a14, c2), O::scale(a23, c1)));
        C i1 = O::mul_negi(O::add(O::scale(d14, s1), O::scale(d23, s2)));
        C i2 = O::mul_negi(O::sub(O::scale(d14, s2), O::scale(d23, s1)));
        y[0] = O::add(u[0], O::add(a14, a23));
        y[1] = O::add(r1, i1);
        y[4] = O::sub(r1, i1);
        y[2] = O::add(r2, i2);
        y[3] = O::sub(r2, i2);
    }
};
template <typename T> struct Dft<T, 8> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        using O = Ops<T>;
        const T r = (T)0.70710678118654752440084436210485;   // 1/sqrt(2)
        C e[4] = {u[0], u[2], u[4], u[6]}, o[4] = {u[1], u[3], u[5], u[7]}, a[4], b[4];
        Dft<T, 4>::run(e, a);
        Dft<T, 4>::run(o, b);
        // w8^1 = (1 - i)/sqrt2, w8^2 = -i, w8^3 = -(1 + i)/sqrt2
        b[1] = O::mk(r * (b[1].x + b[1].y), r * (b[1].y - b[1].x));
        b[2] = O::mul_negi(b[2]);
        b[3] = O::mk(r * (b[3].y - b[3].x), -r * (b[3].x + b[3].y));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            y[k] = O::add(a[k], b[k]);
            y[k + 4] = O::sub(a[k], b[k]);
        }
    }
};
template <typename T> struct Dft<T, 16> {
    using C = cx_t<T>;
    static __device__ __forceinline__ void run(const C* u, C* y) {
        using O = Ops<T>;
        // cos / sin of 2 pi j / 16, j = 0..9
        const T cs[10] = {(T)1, (T)0.92387953251128675612818318939679,
                          (T)0.70710678118654752440084436210485,
                          (T)0.38268343236508977172845998403040, (T)0,
                          (T)-0.38268343236508977172845998403040,
                          (T)-0.70710678118654752440084436210485,
                          (T)-0.92387953251128675612818318939679, (T)-1,
                          (T)-0.92387953251128675612818318939679};
        const T sn[10] = {(T)0, (T)0.38268343236508977172845998403040,
                          (T)0.70710678118654752440084436210485,
                          (T)0.92387953251128675612818318939679, (T)1,
                          (T)0.92387953251128675612818318939679,
                          (T)0.70710678118654752440084436210485,
                          (T)0.38268343236508977172845998403040, (T)0,
                          (T)-0.38268343236508977172845998403040};
        C A[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            C v[4] = {u[n2], u[4 + n2], u[8 + n2], u[12 + n2]};
            Dft<T, 4>::run(v, A[n2]);
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) {
                const int j = n2 * k1;
                if (j > 0) A[n2][k1] = O::mul(A[n2][k1], O::mk(cs[j], -sn[j]));
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C v[4] = {A[0][k1], A[1][k1], A[2][k1], A[3][k1]}, d[4];
            Dft<T, 4>::run(v, d);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = d[k2];
        }
    }
};

// Shared-memory element index with one padding slot per 16 elements, so the
// stride-R writes of the early Stockham stages spread over all banks.
__host__ __device__ __forceinline__ int pad(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4) + 1; }

template <typename T> __host__ __device__ constexpr int emax() { return 8; }

// A stage whose inputs come from global memory (FIRST: load(e) for natural
// input index e, always p = 1) and/or whose outputs go straight to global
// memory (LAST: store(k, value) for natural output index k); otherwise as
// stage().  Fusing the first and last stages with the loads and stores saves
// two shared-memory round trips and two barriers per transform.
template <typename T, int R, int NCOL, bool FIRST, bool LAST, class Load, class Store>
__device__ __forceinline__ void stage_io(const cx_t<T>* __restrict__ src, cx_t<T>* __restrict__ dst,
                                         int n, int p, unsigned pmagic,
                                         const cx_t<T>* __restrict__ tw, Load& load, Store& store) {
    using O = Ops<T>;
    using C = cx_t<T>;
    const int nb = n / R;
    const int items = nb * NCOL;
    const int twstep = n / (p * R);
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
        const int c = w & (NCOL - 1), i = w / NCOL;
        const int k = (FIRST || p == 1) ? 0 : i - (int)__umulhi((unsigned)i, pmagic) * p;
        const int kt = k * twstep;
        C u[R], y[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if constexpr (FIRST) {
                u[q] = load(i + q * nb);
            } else {
                u[q] = src[pad(i + q * nb) * NCOL + c];
                if (q > 0 && k > 0) u[q] = O::mul(u[q], __ldg(&tw[q * kt]));
            }
        }
        Dft<T, R>::run(u, y);
        const int j = (i - k) * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if constexpr (LAST) store(j + t * p, y[t]);
            else dst[pad(j + t * p) * NCOL + c] = y[t];
        }
    }
    __syncthreads();
}

template <typename T, int NCOL, bool FIRST, bool LAST, class Load, class Store>
__device__ __forceinline__ void stage_dispatch(int r, const cx_t<T>* src, cx_t<T>* dst, int n, int p,
                                               unsigned mg, const cx_t<T>* tw, Load& load,
                                               Store& store) {
    switch (r) {
        case 16:
            if constexpr (sizeof(T) == 4)
                stage_io<T, 16, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store);
            break;
        case 8: stage_io<T, 8, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store); break;
        case 4: stage_io<T, 4, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store); break;
        case 2: stage_io<T, 2, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store); break;
        case 3: stage_io<T, 3, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store); break;
        case 5: stage_io<T, 5, NCOL, FIRST, LAST>(src, dst, n, p, mg, tw, load, store); break;
    }
}

// The whole transform with the first stage reading load(e) and the last
// writing store(k, v) (natural indices); A and B are the shared ping-pong
// buffers.  Every thread of the block must call it (it holds barriers).
template <typename T, int NCOL, class Load, class Store>
__device__ void fft_fused(cx_t<T>* A, cx_t<T>* B, const FftPlan& fp, const cx_t<T>* tw, Load& load,
                          Store& store) {
    const int S = fp.nstages;
    if (S == 1) {
        stage_dispatch<T, NCOL, true, true>(fp.radix[0], A, B, fp.n, 1, 0u, tw, load, store);
        return;
    }
    stage_dispatch<T, NCOL, true, false>(fp.radix[0], A, A, fp.n, 1, 0u, tw, load, store);
    for (int s = 1; s < S - 1; ++s) {
        stage_dispatch<T, NCOL, false, false>(fp.radix[s], A, B, fp.n, fp.p[s], fp.pmagic[s], tw,
                                              load, store);
        cx_t<T>* t = A;
        A = B;
        B = t;
    }
    stage_dispatch<T, NCOL, false, true>(fp.radix[S - 1], A, B, fp.n, fp.p[S - 1],
                                         fp.pmagic[S - 1], tw, load, store);
}

// Natural input index e of a length-n transform whose len inputs hold modes
// i - len/2 (centred) or index i itself: the input index, or -1 (zero).
__device__ __forceinline__ int in_src(int e, int len, int n, int centered) {
    if (!centered) return e < len ? e : -1;
    const int hi = len - len / 2;
    if (e < hi) return e + len / 2;
    if (e >= n - len / 2) return e - n + len / 2;
    return -1;
}
// Kept output slot of natural output index k (centred order over len), or -1.
__device__ __forceinline__ int out_slot(int k, int len, int n) {
    if (k < len - len / 2) return k + len / 2;
    if (k >= n - len / 2) return k - n + len / 2;
    return -1;
}



template <typename T>
__global__ void __launch_bounds__(kFftThreads, kFftBlocksPerSm)
k_fft_rows(FftPlan fp, RowPassArgs a) {
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* S = (C*)smem_raw;
    C* S2 = S + padded_len(fp.n);
    const int n = fp.n;
    const C* tw = (const C*)a.twiddle;
    const T* dcol = (const T*)a.deconv_col;
    // rows of dead tile rows are zero in and out of the transform: skipped,
    // through the plan's list of live rows when it has one, else by the rows'
    // live flags
    auto next_live = [&](int r) {
        if (a.live)
            while (r < a.nrows && !a.live[(r / a.batch_rows) * a.nty + (r % a.batch_rows) / kTile])
                r += gridDim.x;
        return r;
    };
    auto transform = [&](int row) {
        const C* in = (const C*)a.in + (long long)row * a.in_stride;
        C* out = (C*)a.out + (long long)row * a.out_stride;
        const T rowf = a.deconv_row ? ((const T*)a.deconv_row)[row] : (T)1;
        auto load = [&](int e) {
            const int i = in_src(e, a.in_len, n, a.centered_in);
            if (i < 0) return Ops<T>::mk(0, 0);
            C v = in[i];
            if (a.centered_in) v = Ops<T>::scale(v, rowf * (dcol ? dcol[i] : (T)1));
            return v;
        };
        auto store = [&](int k, C v) {
            const int kp = out_slot(k, a.out_len, n);
            if (kp >= 0) out[kp] = v;
        };
        fft_fused<T, 1>(S, S2, fp, tw, load, store);
    };
    if (a.row_list) {
        for (int i = blockIdx.x; i < a.nlist; i += gridDim.x) transform(a.row_list[i]);
    } else {
        for (int row = next_live(blockIdx.x); row < a.nrows; row = next_live(row + gridDim.x))
            transform(row);
    }
}

template <typename T, int NCOL, int MODE>
__global__ void __launch_bounds__(kFftThreads, kFftBlocksPerSm)
k_fft_cols(FftPlan fp, ColPassArgs a) {
    using C = cx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned s_live[kMaxTileRows / 32];
    C* S = (C*)smem_raw;
    C* S2 = S + padded_len(fp.n) * NCOL;
    const int n = fp.n;
    const C* tw = (const C*)a.twiddle;
    const int ngroups = (a.ncols + NCOL - 1) / NCOL;
    const int nouter = MODE == kFftPlain ? max(a.batch, 1) : a.nouter;
    const int total = ngroups * nouter;            // (outer index, column group) work items
    const int c = threadIdx.x & (NCOL - 1);        // this thread's column in every group
    for (int gg = blockIdx.x; gg < total; gg += gridDim.x) {
        const int o = gg / ngroups, col = (gg - o * ngroups) * NCOL + c;
        const bool on = col < a.ncols;
        if constexpr (MODE == kFftPlain) {
            const int bi = o;
            const C* in = (const C*)a.in + (long long)bi * a.in_bstride + col;
            C* out = (C*)a.out + (long long)bi * a.out_bstride + col;
            if (a.live) {   // live tile rows of this transform as a bit mask
                for (int t = threadIdx.x; t < kMaxTileRows / 32; t += blockDim.x) s_live[t] = 0u;
                __syncthreads();
                for (int t = threadIdx.x; t < a.nty; t += blockDim.x)
                    if (a.live[(long long)bi * a.nty + t]) atomicOr(&s_live[t >> 5], 1u << (t & 31));
                __syncthreads();
            }
            C axc = Ops<T>::mk(1, 0);
            const C* ay = nullptr;
            if (a.ax && on) {
                axc = ((const C*)a.ax)[(long long)bi * a.ncols + col];
                ay = (const C*)a.ay + (long long)bi * a.out_len;
            }
            auto load = [&](int e) {
                const int i = in_src(e, a.in_len, n, a.centered_in);
                if (i < 0 || !on) return Ops<T>::mk(0, 0);
                if (a.live) {
                    const int tr = i / kTile;
                    if (!((s_live[tr >> 5] >> (tr & 31)) & 1u)) return Ops<T>::mk(0, 0);
                }
                return in[(long long)i * a.ncols];
            };
            auto store = [&](int k, C v) {
                const int kp = out_slot(k, a.out_len, n);
                if (kp < 0 || !on) return;
                if (ay) {
                    v = Ops<T>::mul(Ops<T>::mul(v, axc), __ldg(&ay[kp]));
                    if (a.occulter) v = Ops<T>::mk((T)1 - v.x, -v.y);
                }
                out[(long long)kp * a.ncols] = v;
            };
            fft_fused<T, NCOL>(S, S2, fp, tw, load, store);
        } else if constexpr (MODE == kFftRowStep1) {
            // grid row o viewed as fa x fb (element e = fb a + b at column b = col)
            const C* in = (const C*)a.in + (long long)o * a.in_stride;
            C* out = (C*)a.out + (long long)o * a.fN + col;
            const T rowf = a.deconv_row ? ((const T*)a.deconv_row)[o] : (T)1;
            const T* dcol = (const T*)a.deconv_col;
            auto load = [&](int ea) {
                if (!on) return Ops<T>::mk(0, 0);
                const int i = in_src(a.fb * ea + col, a.in_len, a.fN, a.centered_in);
                if (i < 0) return Ops<T>::mk(0, 0);
                C v = in[i];
                if (a.centered_in) v = Ops<T>::scale(v, rowf * (dcol ? dcol[i] : (T)1));
                return v;
            };
            auto store = [&](int k1, C v) {
                if (on) out[(long long)k1 * a.fb] = v;
            };
            fft_fused<T, NCOL>(S, S2, fp, tw, load, store);
        } else if constexpr (MODE == kFftColStep1) {
            // outer index o = b: rows e = fb a + b of the grid columns
            const C* in = (const C*)a.in + col;
            C* out = (C*)a.out + (long long)o * a.ncols + col;
            auto load = [&](int ea) {
                if (!on) return Ops<T>::mk(0, 0);
                const int i = in_src(a.fb * ea + o, a.in_len, a.fN, a.centered_in);
                if (i < 0) return Ops<T>::mk(0, 0);
                return in[(long long)i * a.ncols];
            };
            auto store = [&](int k1, C v) {
                if (on) out[(long long)k1 * a.fb * a.ncols] = v;
            };
            fft_fused<T, NCOL>(S, S2, fp, tw, load, store);
        } else if constexpr (MODE == kFftRowStep2) {
            // transform (l = o, k1 = col): scratch row (o fa + k1), b contiguous
            const C* in = (const C*)a.in + ((long long)o * a.fa + col) * a.fb;
            C* out = (C*)a.out + (long long)o * a.out_stride;
            const C* twN = (const C*)a.twN;
            auto load = [&](int b) {
                if (!on) return Ops<T>::mk(0, 0);
                return Ops<T>::mul(in[b], __ldg(&twN[b * col]));
            };
            auto store = [&](int k2, C v) {
                const int kp = out_slot(col + a.fa * k2, a.out_len, a.fN);
                if (kp >= 0 && on) out[kp] = v;
            };
            fft_fused<T, NCOL>(S, S2, fp, tw, load, store);
        } else {   // kFftColStep2: outer index o = k1
            const C* in = (const C*)a.in + (long long)o * a.fb * a.ncols + col;
            C* out = (C*)a.out + col;
            const C* twN = (const C*)a.twN;
            C axc = Ops<T>::mk(1, 0);
            if (a.ax && on) axc = ((const C*)a.ax)[col];
            auto load = [&](int b) {
                if (!on) return Ops<T>::mk(0, 0);
                return Ops<T>::mul(in[(long long)b * a.ncols], __ldg(&twN[b * o]));
            };
            auto store = [&](int k2, C v) {
                const int kp = out_slot(o + a.fa * k2, a.out_len, a.fN);
                if (kp < 0 || !on) return;
                if (a.ax) {
                    v = Ops<T>::mul(Ops<T>::mul(v, axc), __ldg(&((const C*)a.ay)[kp]));
                    if (a.occulter) v = Ops<T>::mk((T)1 - v.x, -v.y);
                }
                out[(long long)kp * a.ncols] = v;
            };
            fft_fused<T, NCOL>(S, S2, fp, tw, load, store);
        }
    }
}

int threads_for(int elems, int em) {
    int t = (elems + em - 1) / em;
    t = (t + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > kFftThreads) t = kFftThreads;
    return t;
}

}  // namespace

FftPlan make_fft_plan(int n, int max_radix) {
    FftPlan fp{};
    fp.n = n;
    int m = n;
    if (max_radix >= 16)
        while (m % 16 == 0) { fp.radix[fp.nstages++] = 16; m /= 16; }
    if (max_radix >= 8)
        while (m % 8 == 0) { fp.radix[fp.nstages++] = 8; m /= 8; }
    while (m % 4 == 0) { fp.radix[fp.nstages++] = 4; m /= 4; }
    while (m % 2 == 0) { fp.radix[fp.nstages++] = 2; m /= 2; }
    while (m % 3 == 0) { fp.radix[fp.nstages++] = 3; m /= 3; }
    while (m % 5 == 0) { fp.radix[fp.nstages++] = 5; m /= 5; }
    if (m != 1) fp.nstages = -1;
    long long p = 1;
    for (int s = 0; s < fp.nstages; ++s) {
        fp.p[s] = (int)p;
        fp.pmagic[s] = p == 1 ? 0u : (unsigned)(((1ULL << 32) + (unsigned long long)p - 1) / p);
        p *= fp.radix[s];
    }
    return fp;
}

// Largest column batch (power of two, <= 8) whose two n x C ping-pong buffers
// fit in shared memory; 0 if n itself does not.
bool fft_supported(int n, int is_double, int* max_cols) {
    FftPlan fp = make_fft_plan(n, 4);
    if (fp.nstages < 0 || n < 2) return false;
    const long long smem_cap = 227 * 1024;
    const int esz = is_double ? 16 : 8;
    int c = 8;
    while (c > 0 && 2LL * padded_len(n) * c * esz > smem_cap) c >>= 1;
    if (max_cols) *max_cols = c;
    return c > 0;
}

template <typename T>
void launch_fft_rows(const FftPlan& fp, const RowPassArgs& a, cudaStream_t st) {
    const size_t smem = 2 * (size_t)padded_len(fp.n) * sizeof(cx_t<T>);
    // one thread per butterfly of the leading (largest) radix: a radix-16
    // plan gets n/16 threads, all busy in its radix-16 stages, and more rows
    // resident per SM
    const int threads = threads_for(fp.n, fp.radix[0] > emax<T>() ? fp.radix[0] : emax<T>());
    const int nwork = a.row_list ? a.nlist : a.nrows;
    int blocks = nwork < 152 * 16 ? nwork : 152 * 16;
    if (blocks < 1) blocks = 1;
    cudaFuncSetAttribute(k_fft_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fft_rows<T><<<blocks, threads, smem, st>>>(fp, a);
}

template <typename T, int MODE>
void launch_cols_mode(const FftPlan& fp, const ColPassArgs& a, int cmax, cudaStream_t st) {
    const size_t smem = 2 * (size_t)padded_len(fp.n) * cmax * sizeof(cx_t<T>);
    const int threads = threads_for(fp.n * cmax, emax<T>());
    const int nouter = MODE == kFftPlain ? (a.batch > 1 ? a.batch : 1) : a.nouter;
    const long long work = (long long)((a.ncols + cmax - 1) / cmax) * nouter;
    int blocks = work < 152 * 16 ? (int)work : 152 * 16;
    if (blocks < 1) blocks = 1;
#define FRES_COLS(NC)                                                                          \
    case NC:                                                                                   \
        cudaFuncSetAttribute(k_fft_cols<T, NC, MODE>,                                          \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
        k_fft_cols<T, NC, MODE><<<blocks, threads, smem, st>>>(fp, a);                         \
        break;
    switch (cmax) {
        FRES_COLS(1) FRES_COLS(2) FRES_COLS(4) FRES_COLS(8)
        default: break;
    }
#undef FRES_COLS
}

template <typename T>
void launch_fft_cols(const FftPlan& fp, const ColPassArgs& a, cudaStream_t st) {
    int cmax = 0;
    fft_supported(fp.n, sizeof(T) == 8, &cmax);
    // fewer columns per block when that keeps three blocks per SM
    while (cmax > 1 && 2LL * padded_len(fp.n) * cmax * (long long)sizeof(cx_t<T>) > kFftSmemTarget)
        cmax >>= 1;
    switch (a.mode) {
        case kFftRowStep1: launch_cols_mode<T, kFftRowStep1>(fp, a, cmax, st); break;
        case kFftColStep1: launch_cols_mode<T, kFftColStep1>(fp, a, cmax, st); break;
        case kFftColStep2: launch_cols_mode<T, kFftColStep2>(fp, a, cmax, st); break;
        case kFftRowStep2: launch_cols_mode<T, kFftRowStep2>(fp, a, cmax, st); break;
        default: launch_cols_mode<T, kFftPlain>(fp, a, cmax, st); break;
    }
}

// n = fa * fb with both factors single-pass lengths, fa the divisor closest
// to sqrt(n) from below that works.
bool fft_split(int n, int is_double, int* fa, int* fb) {
    int best = 0;
    for (int d = 2; (long long)d * d <= n; ++d) {
        if (n % d) continue;
        if (make_fft_plan(d, 4).nstages < 0 || make_fft_plan(n / d, 4).nstages < 0) continue;
        if (fft_supported(d, is_double, nullptr) && fft_supported(n / d, is_double, nullptr)) best = d;
    }
    if (!best) return false;
    *fa = best;
    *fb = n / best;
    return true;
}

template void launch_fft_rows<float>(const FftPlan&, const RowPassArgs&, cudaStream_t);
template void launch_fft_rows<double>(const FftPlan&, const RowPassArgs&, cudaStream_t);
template void launch_fft_cols<float>(const FftPlan&, const ColPassArgs&, cudaStream_t);
template void launch_fft_cols<double>(const FftPlan&, const ColPassArgs&, cudaStream_t);

// ------------------------------------------------------------------ direct column DFT
// When only a narrow band of the type-1 grid's rows holds nodes (a starshade
// a few grid cells across on a pupil-sized grid), the column transform of the
// kept outputs is a small dense product: for problem b, kept output slot kp
// (natural index k) and column c,
//   out[kp][c] = sum_{r live} w_n^{k r} in[r][c],
// i.e. (n_out x R) x (R x ncols) with R live rows.  A block takes 64
// columns and up to four 64-output tiles; it stages 32 (FP64: 16) live rows
// at a time of the input (once for all its tiles when they fit one chunk)
// and of the twiddle matrix (from the exact n-point table, index k r mod n:
// a mask for power-of-two n) in shared memory, and each thread accumulates a 4 x 4 tile (outputs
// ty + 16 i, columns tx + 16 j: conflict-free shared reads, coalesced stores)
// before the output epilogue of the FFT path.
namespace {

constexpr int kDftTile = 64;

template <typename T>
__global__ void __launch_bounds__(256)
k_col_dft(ColPassArgs a, int n, unsigned nmask, unsigned* __restrict__ status) {
    using C = cx_t<T>;
    using O = Ops<T>;
    constexpr int kDftChunk = sizeof(T) == 4 ? 32 : 16;   // live rows staged at a time
    __shared__ C sX[kDftChunk][kDftTile];
    __shared__ C sW[kDftChunk][kDftTile];
    __shared__ int s_rows[kDftMaxRows];
    __shared__ int s_nt;
    const int b = blockIdx.z;
    const int c0 = blockIdx.x * kDftTile;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // the problem's live tile rows in increasing order (one warp, ballots):
    // a fixed summation order, so the outputs repeat bit for bit
    if (tid < 32) {
        int cnt = 0;
        for (int t0 = 0; t0 < a.nty; t0 += 32) {
            const int t = t0 + tid;
            const bool on = t < a.nty && a.live[(long long)b * a.nty + t] != 0;
            const unsigned m = __ballot_sync(0xffffffffu, on);
            const int q = cnt + __popc(m & ((1u << tid) - 1u));
            if (on && q < kDftMaxRows / kTile)
                for (int i = 0; i < kTile; ++i) s_rows[q * kTile + i] = t * kTile + i;
            cnt += __popc(m);
        }
        if (tid == 0) s_nt = cnt;
    }
    __syncthreads();
    int R = s_nt * kTile;
    if (R > kDftMaxRows) {
        if (tid == 0) atomicOr(status, kStatusOverflow);
        R = kDftMaxRows;
    }
    const int len = a.out_len;
    const C* in = (const C*)a.in + (long long)b * a.in_bstride;
    const C* tw = (const C*)a.twiddle;
    C* out = (C*)a.out + (long long)b * a.out_bstride;
    const C* ax = a.ax ? (const C*)a.ax + (long long)b * a.ncols : nullptr;
    const C* ay = a.ax ? (const C*)a.ay + (long long)b * len : nullptr;
    // live rows fitting one chunk are staged once for all the block's output tiles
    const bool one = R <= kDftChunk;
    auto stage_x = [&](int r0, int rc) {
        for (int e = tid; e < kDftChunk * kDftTile; e += blockDim.x) {
            const int r = e / kDftTile, c = e % kDftTile, col = c0 + c;
            C x = O::mk(0, 0);
            if (r < rc && col < a.ncols) x = in[(long long)s_rows[r0 + r] * a.ncols + col];
            sX[r][c] = x;
        }
    };
    if (one) stage_x(0, R);
    const int nkt = (len + kDftTile - 1) / kDftTile;
    for (int kt = blockIdx.y; kt < nkt; kt += gridDim.y) {
        const int k0 = kt * kDftTile;
        C acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = O::mk(0, 0);
        for (int r0 = 0; r0 < R; r0 += kDftChunk) {
            const int rc = min(kDftChunk, R - r0);
            __syncthreads();   // the previous tile's or chunk's values are consumed
            if (!one) stage_x(r0, rc);
            for (int e = tid; e < kDftChunk * kDftTile; e += blockDim.x) {
                // twiddle row r, output kk = c
                const int r = e / kDftTile, c = e % kDftTile, kp = k0 + c;
                C w = O::mk(0, 0);
                if (r < rc && kp < len) {
                    const unsigned k = kp >= len / 2 ? kp - len / 2 : kp - len / 2 + n;
                    const unsigned kr = k * (unsigned)s_rows[r0 + r];   // < 2^26
                    w = __ldg(&tw[nmask ? (kr & nmask) : kr % (unsigned)n]);
                }
                sW[r][c] = w;
            }
            __syncthreads();
            for (int r = 0; r < rc; ++r) {
                C w[4], x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) w[i] = sW[r][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = sX[r][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[i][j].x = fma(w[i].x, x[j].x, fma(-w[i].y, x[j].y, acc[i][j].x));
                        acc[i][j].y = fma(w[i].x, x[j].y, fma(w[i].y, x[j].x, acc[i][j].y));
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kp = k0 + ty + 16 * i;
            if (kp >= len) continue;
            const C yv = ay ? __ldg(&ay[kp]) : O::mk(1, 0);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = c0 + tx + 16 * j;
                if (col >= a.ncols) continue;
                C v = acc[i][j];
                if (ax) {
                    v = O::mul(O::mul(v, __ldg(&ax[col])), yv);
                    if (a.occulter) v = O::mk((T)1 - v.x, -v.y);
                }
                out[(long long)kp * a.ncols + col] = v;
            }
        }
    }
}

// In-register 32-point DFT, y_t = sum_q u_q e^{-2 pi i q t / 32}, in place:
// q = 4 m + q2, t = t1 + 8 t2 (Cooley-Tukey): 8-point DFTs over m, twiddles
// w_32^{q2 t1}, then 4-point DFTs over q2.
template <typename T>
__device__ __forceinline__ void dft32(cx_t<T>* y) {
    using C = cx_t<T>;
    using O = Ops<T>;
    // cos (2 pi j / 32), j = 0..8; sin (2 pi j / 32) = cos (2 pi (8 - j) / 32)
    const T c[9] = {(T)1, (T)0.98078528040323044912618223613424,
                    (T)0.92387953251128675612818318939679,
                    (T)0.83146961230254523707878837761791,
                    (T)0.70710678118654752440084436210485,
                    (T)0.55557023301960222474283081394853,
                    (T)0.38268343236508977172845998403040,
                    (T)0.19509032201612826784828486847702, (T)0};
    C A[4][8];
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
        C v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = y[4 * m + q2];
        Dft<T, 8>::run(v, A[q2]);
#pragma unroll
        for (int t1 = 1; t1 < 8; ++t1) {
            const int j = q2 * t1;   // < 32: w_32^j = (cos, -sin) of 2 pi j / 32
            if (j == 0) continue;
            const int jq = j & 7, quad = j >> 3;   // j = 8 quad + jq
            // (cos, sin) of 2 pi j / 32 from the first quadrant
            T cs = c[jq], sn = c[8 - jq];
            if (quad == 1) { const T t = cs; cs = -sn; sn = t; }
            else if (quad == 2) { cs = -cs; sn = -sn; }
            else if (quad == 3) { const T t = cs; cs = sn; sn = -t; }
            A[q2][t1] = O::mul(A[q2][t1], O::mk(cs, -sn));
        }
    }
#pragma unroll
    for (int t1 = 0; t1 < 8; ++t1) {
        C v[4] = {A[0][t1], A[1][t1], A[2][t1], A[3][t1]}, d[4];
        Dft<T, 4>::run(v, d);
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) y[t1 + 8 * t2] = d[t2];
    }
}

// Type-1 column pass over one live tile row by a pruned FFT.  A problem
// whose nodes occupy the 32 grid rows row0 .. row0 + 31 has, for the
// natural output index k = P a + b (P = n / 32, a < 32, b < P),
//   sum_j w_n^{k (row0 + j)} x_j = w_n^{k row0} sum_j w_32^{a j} (w_n^{b j} x_j):
// a 32-point DFT per b of the inputs twiddled by w_n^{b j}, about 30
// operations per output instead of the direct sum's 32 multiply-adds, then
// the epilogue (ax[c] folded into the staged inputs, ay[k] and Babinet).
// A warp takes 32 adjacent columns and one b; the block's 8 warps (8 b)
// share the staged 32 x 32 input block.  Stores: each output row segment of
// a warp is 32 adjacent columns.
template <typename T>
__global__ void __launch_bounds__(256)
k_col_pfft(ColPassArgs a, int n, unsigned nmask, unsigned* __restrict__ status) {
    using C = cx_t<T>;
    using O = Ops<T>;
    __shared__ C xs[kTile][kTile + 1];
    __shared__ int s_nt, s_row0;
    const int pb = blockIdx.z, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.x * kTile, col = c0 + lane;
    const int P = n / kTile;
    const int bb = blockIdx.y * 8 + warp;   // this warp's b
    const int len = a.out_len;
    if (tid == 0) {
        s_nt = 0;
        s_row0 = 0;
    }
    __syncthreads();
    for (int t = tid; t < a.nty; t += blockDim.x)
        if (a.live[(long long)pb * a.nty + t]) {
            atomicAdd(&s_nt, 1);
            s_row0 = t * kTile;
        }
    __syncthreads();
    const int nt = s_nt, row0 = s_row0;
    const C* in = (const C*)a.in + (long long)pb * a.in_bstride;
    C* out = (C*)a.out + (long long)pb * a.out_bstride;
    const C* tw = (const C*)a.twiddle;
    const C* ax = a.ax ? (const C*)a.ax + (long long)pb * a.ncols : nullptr;
    const C* ay = a.ax ? (const C*)a.ay + (long long)pb * len : nullptr;
    const bool bab = ay && a.occulter;
    if (nt != 1) {   // no nodes: u^ap = 0 (u^oc = 1); several live tile rows: flagged
        if (nt > 1 && tid == 0) atomicOr(status, kStatusOverflow);
        if (nt == 0 && bb < P && col < a.ncols)
            for (int aa = 0; aa < kTile; ++aa) {
                const int kp = out_slot(P * aa + bb, len, n);
                if (kp >= 0) out[(long long)kp * a.ncols + col] = O::mk(bab ? (T)1 : (T)0, 0);
            }
        return;
    }
    for (int e = tid; e < kTile * kTile; e += blockDim.x) {
        const int r = e / kTile, cc = e % kTile, cg = c0 + cc;
        C x = O::mk(0, 0);
        if (cg < a.ncols) {
            x = in[(long long)(row0 + r) * a.ncols + cg];
            if (ax) x = O::mul(x, ax[cg]);
        }
        xs[r][cc] = x;
    }
    __syncthreads();
    if (bb >= P || col >= a.ncols) return;
    C y[kTile];
#pragma unroll
    for (int j = 0; j < kTile; ++j) {
        const C x = xs[j][lane];
        y[j] = j == 0 ? x : O::mul(x, __ldg(&tw[bb * j]));   // bb j < n
    }
    dft32<T>(y);
#pragma unroll
    for (int aa = 0; aa < kTile; ++aa) {
        const int k = P * aa + bb;
        const int kp = out_slot(k, len, n);
        if (kp >= 0) {
            const unsigned kr = (unsigned)k * (unsigned)row0;   // < n^2 <= 2^30
            C v = O::mul(y[aa], __ldg(&tw[nmask ? (kr & nmask) : kr % (unsigned)n]));
            if (ay) {
                v = O::mul(v, __ldg(&ay[kp]));
                if (a.occulter) v = O::mk((T)1 - v.x, -v.y);
            }
            out[(long long)kp * a.ncols + col] = v;
        }
    }
}

}  // namespace

template <typename T>
void launch_col_dft(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st) {
    // each block takes up to four 64-output tiles of its 64 columns
    const int nkt = (a.out_len + kDftTile - 1) / kDftTile;
    const dim3 grid((a.ncols + kDftTile - 1) / kDftTile, (nkt + 3) / 4, a.batch > 1 ? a.batch : 1);
    // power-of-two n: the index reduction is a mask instead of a division
    const unsigned nmask = (n & (n - 1)) == 0 ? (unsigned)(n - 1) : 0u;
    k_col_dft<T><<<grid, 256, 0, st>>>(a, n, nmask, status);
}
template void launch_col_dft<float>(const ColPassArgs&, int, unsigned*, cudaStream_t);
template void launch_col_dft<double>(const ColPassArgs&, int, unsigned*, cudaStream_t);

bool col_pfft_supported(int n, int live_rows) {
    return live_rows == kTile && n % kTile == 0 && n <= 32768;
}

void launch_col_pfft_d(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st) {
    const int P = n / kTile;
    const dim3 grid((a.ncols + kTile - 1) / kTile, (P + 7) / 8, a.batch > 1 ? a.batch : 1);
    const unsigned nmask = (n & (n - 1)) == 0 ? (unsigned)(n - 1) : 0u;
    k_col_pfft<double><<<grid, 256, 0, st>>>(a, n, nmask, status);
}

}  // namespace fres
