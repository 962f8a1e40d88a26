// Type-1 column pass over a narrow live band on the tensor cores (FP32 fast
// mode).  When a problem's nodes occupy one tile row of the spreading grid
// (a starshade at a few Fresnel numbers: one live tile row of a 1024^2 grid),
// the column transform of the NUFFT of Sec. 3.3 reduces to a dense complex
// product over those R = 32 live rows (see k_col_dft in k_fft.cu):
//   out[kp][c] = sum_{r live} w_n^{k r} in[r][c],   k the natural index of slot kp,
// then the output epilogue out[kp][c] ax[c] ay[kp] (deconvolution, target
// chirp) and Babinet.  The product is linear, so the column factor ax[c]
// scales the staged input block and the output factor ay[kp] the staged
// twiddles: the epilogue is left with Babinet and the store.
//
// It runs transposed, out^T = in^T W^T, so that a tensor-memory lane is a
// column c and an accumulator column an output kp: in the epilogue the 32
// threads of a warp hold 32 consecutive columns of one output row, and every
// store is a coalesced 256-byte row segment.  In real form, with W = Wr + i Wi
// and X = Xr + i Xi,
//   Re = Xr Wr - Xi Wi,  Im = Xi Wr + Xr Wi,
// products of a (128 columns x 32 rows) input block by (32 rows x 32 outputs)
// twiddle blocks, as tcgen05 MMAs of kind::tf32 with FP32 accumulators in
// tensor memory.  FP32 accuracy comes from splitting both operands into TF32
// high and low parts and summing hi.hi + hi.lo + lo.hi (the dropped lo.lo
// term is ~2^-22 of the product); the Xi Wi product uses the instruction's
// negate-A flag.
//
// One CTA (8 warps, two per SM) per (problem, 128 columns, 16 chunks of outputs).
// The input block is staged once in shared memory (no-swizzle K-major layout
// of the MMA descriptors: 8-row x 16-byte core matrices); the twiddle blocks
// of successive 32-output chunks and their accumulators are double-buffered,
// so a ninth warp issues chunk i's 48 MMAs (committed to an mbarrier) while
// the other eight read chunk i - 1's accumulators with tcgen05.ld and store
// its outputs; one barrier per chunk.  Every wait is bounded: on giving up
// the CTA flags kStatusTimeout, stops, frees its tensor memory and returns.
#include "internal.cuh"

namespace fres {

namespace {

constexpr int kTcM = 128;            // columns per CTA (TMEM lanes), MMA M
constexpr int kTcN = 32;             // outputs per chunk (accumulator columns), MMA N
constexpr int kTcR = 32;             // live rows (one tile row)
constexpr int kTcK = 2 * kTcR;       // real K: [Xr | Xi] against [Wr | Wi]
constexpr int kTcThreads = 288;     // 8 staging / epilogue warps and an MMA-issuing warp
constexpr int kTcWork = 256;        // threads of the staging / epilogue warps
constexpr int kTcCols = 4 * kTcN;    // TMEM: 2 buffers x (Re, Im) x kTcN columns
constexpr int kTcChunksPerCta = 16;  // output chunks of one CTA (512 outputs: the whole column)
constexpr long long kTcMaxPolls = 1LL << 24;   // ~1 s of 64 ns back-offs

struct TcSmem {
    float x_hi[kTcM * kTcK];         // input block, 32 KB each (cm_index layout)
    float x_lo[kTcM * kTcK];
    float w_hi[2][kTcN * kTcK];      // twiddle chunks, 8 KB each, double-buffered
    float w_lo[2][kTcN * kTcK];
    unsigned long long mbar[2];
    unsigned tmem_base;
    int ok;
    int nt;
    int row0;
};

// Float index of element (row, k) of a K-major operand with kTcK columns:
// core matrices of 8 rows x 4 elements (128 contiguous bytes), K-adjacent
// core matrices 128 B apart, 8-row groups kTcK / 4 x 128 B apart.
__device__ __forceinline__ int cm_index(int row, int k) {
    return ((row >> 3) * (kTcK / 4) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (K)
// byte offset 128, stride (8-row group) byte offset kTcK / 4 * 128, all in
// 16-byte units; version 1 at bit 46.
__device__ __forceinline__ unsigned long long smem_desc(const float* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned long long d = (unsigned long long)((a & 0x3FFFFu) >> 4);
    d |= (unsigned long long)(128u >> 4) << 16;
    d |= (unsigned long long)((kTcK / 4 * 128u) >> 4) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor of kind::tf32: F32 accumulator, TF32 A and B, both
// K-major, M = kTcM, N = kTcN, optionally A negated.
__host__ __device__ constexpr unsigned tc_idesc(bool neg_a) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((unsigned)(kTcN >> 3) << 17) | ((unsigned)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    unsigned h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hi));
    lo = __uint_as_float(l);
}

__device__ __forceinline__ void split4(const float* v, float4& hi, float4& lo) {
    split_tf32(v[0], hi.x, lo.x);
    split_tf32(v[1], hi.y, lo.y);
    split_tf32(v[2], hi.z, lo.z);
    split_tf32(v[3], hi.w, lo.w);
}

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long a,
                                         unsigned long long b, unsigned idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned phase) {
    for (long long i = 0; i < kTcMaxPolls; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(addr), "r"(phase)
            : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Twiddle chunk starting at output slot kp0 into buffer q: W(m, j) = Wr,
// W(m, kTcR + j) = Wi for output kp0 + m and live row row0 + j, each times
// the output's epilogue factor ay[kp0 + m] (zero past the kept outputs).  Thread t: output m = t % 32, rows 4 (t / 32) .. + 3.
__device__ __forceinline__ void stage_twiddles(TcSmem& sm, int q, int kp0, int len, int n,
                                               unsigned nmask, int row0,
                                               const float2* __restrict__ tw,
                                               const float2* __restrict__ ay) {
    const int m = threadIdx.x & (kTcN - 1), j0 = (threadIdx.x / kTcN) * 4;
    const int kp = kp0 + m;
    unsigned kn = 0;
    if (kp < len) kn = kp >= len / 2 ? kp - len / 2 : kp - len / 2 + n;
    const float2 yv = (ay && kp < len) ? __ldg(&ay[kp]) : make_float2(1.0f, 0.0f);
    {
        const int j = j0;
        float wr[4], wi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 w = make_float2(0.0f, 0.0f);
            if (kp < len) {
                const unsigned kr = kn * (unsigned)(row0 + j + u);   // < 2^26
                w = __ldg(&tw[nmask ? (kr & nmask) : kr % (unsigned)n]);
            }
            wr[u] = w.x * yv.x - w.y * yv.y;
            wi[u] = w.x * yv.y + w.y * yv.x;
        }
        float4 h, l;
        split4(wr, h, l);
        *reinterpret_cast<float4*>(&sm.w_hi[q][cm_index(m, j)]) = h;
        *reinterpret_cast<float4*>(&sm.w_lo[q][cm_index(m, j)]) = l;
        split4(wi, h, l);
        *reinterpret_cast<float4*>(&sm.w_hi[q][cm_index(m, kTcR + j)]) = h;
        *reinterpret_cast<float4*>(&sm.w_lo[q][cm_index(m, kTcR + j)]) = l;
    }
}

// One thread issues a chunk's 48 MMAs into accumulator buffer q and commits
// them.  Descriptors advance by adding 16-byte units to the start address.
__device__ __forceinline__ void issue_chunk(TcSmem& sm, int q, unsigned tmem) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    constexpr int kSteps = kTcR / 8;   // 8-deep K steps per half
    constexpr unsigned long long kStep = 2 * 32 * 4 / 16;          // one K step: 256 B
    constexpr unsigned long long kHalf = kSteps * kStep;            // the imaginary half
    const unsigned id_pos = tc_idesc(false), id_neg = tc_idesc(true);
    const unsigned d_re = tmem + q * 2 * kTcN, d_im = d_re + kTcN;
    const unsigned long long xh = smem_desc(sm.x_hi), xl = smem_desc(sm.x_lo);
    const unsigned long long wh = smem_desc(sm.w_hi[q]), wl = smem_desc(sm.w_lo[q]);
#pragma unroll
    for (int s = 0; s < kSteps; ++s) {
        // K step s of the real half (Xr, Wr) and of the imaginary half (Xi, Wi)
        const unsigned long long o1 = s * kStep, o2 = kHalf + s * kStep;
        const int first = s == 0 ? 0 : 1;
        // Re = Xr Wr - Xi Wi
        mma_tf32(d_re, xh + o1, wh + o1, id_pos, first);
        mma_tf32(d_re, xh + o1, wl + o1, id_pos, 1);
        mma_tf32(d_re, xl + o1, wh + o1, id_pos, 1);
        mma_tf32(d_re, xh + o2, wh + o2, id_neg, 1);
        mma_tf32(d_re, xh + o2, wl + o2, id_neg, 1);
        mma_tf32(d_re, xl + o2, wh + o2, id_neg, 1);
        // Im = Xi Wr + Xr Wi
        mma_tf32(d_im, xh + o2, wh + o1, id_pos, first);
        mma_tf32(d_im, xh + o2, wl + o1, id_pos, 1);
        mma_tf32(d_im, xl + o2, wh + o1, id_pos, 1);
        mma_tf32(d_im, xh + o1, wh + o2, id_pos, 1);
        mma_tf32(d_im, xh + o1, wl + o2, id_pos, 1);
        mma_tf32(d_im, xl + o1, wh + o2, id_pos, 1);
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            (unsigned)__cvta_generic_to_shared(&sm.mbar[q]))
        : "memory");
}

__global__ void __launch_bounds__(kTcThreads)
k_col_dft_tc(ColPassArgs a, int n, unsigned nmask, unsigned* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& sm = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, c0 = blockIdx.x * kTcM;
    const int len = a.out_len;
    const int nchunks = (len + kTcN - 1) / kTcN;
    const int ch0 = blockIdx.y * kTcChunksPerCta;
    const int ch1 = min(ch0 + kTcChunksPerCta, nchunks);
    if (tid == 0) {
        sm.nt = 0;
        sm.ok = 1;
        sm.row0 = 0;
        for (int q = 0; q < 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                             (unsigned)__cvta_generic_to_shared(&sm.mbar[q]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // tensor memory for the two accumulator buffers
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(&sm.tmem_base)),
                     "r"((unsigned)kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the problem's live tile row (the plan routes here only problems with
    // one; more is flagged and leaves the outputs unwritten)
    for (int t = tid; t < a.nty; t += blockDim.x)
        if (a.live[(long long)b * a.nty + t]) {
            atomicAdd(&sm.nt, 1);
            sm.row0 = t * kTile;
        }
    __syncthreads();
    const unsigned tmem = sm.tmem_base;
    const int nt = sm.nt, row0 = sm.row0;
    if (nt > 1 && tid == 0) atomicOr(status, kStatusOverflow);
    const float2* tw = (const float2*)a.twiddle;
    const float2* ax = a.ax ? (const float2*)a.ax + (long long)b * a.ncols : nullptr;
    const float2* ay = a.ax ? (const float2*)a.ay + (long long)b * len : nullptr;
    float2* out = (float2*)a.out + (long long)b * a.out_bstride;
    // epilogue geometry: warp w holds TMEM lanes (columns) 32 (w % 4) + lane
    // and outputs 16 (w / 4) .. + 15 of each chunk
    const int col = c0 + 32 * (warp & 3) + lane;
    const int mh = 16 * (warp >> 2);
    const unsigned tlane = (unsigned)(32 * (warp & 3)) << 16;
    if (nt == 0 && tid < kTcWork) {   // no nodes in this problem: u^ap = 0 (u^oc = 1)
        if (col < a.ncols)
            for (int kp = ch0 * kTcN + mh; kp < min(ch1 * kTcN, len); kp += kTcN)
                for (int j = 0; j < 16 && kp + j < len; ++j)
                    out[(long long)(kp + j) * a.ncols + col] =
                        make_float2(ay && a.occulter ? 1.0f : 0.0f, 0.0f);
    }
    unsigned phase0 = 0u, phase1 = 0u;        // the mbarriers' current phases
    int ok = 1;
    if (nt == 1 && ch0 < ch1) {
        // ---- input block: X(c, j) = Xr, X(c, kTcR + j) = Xi (column c's live rows)
        if (tid < kTcWork) {
            const float2* in = (const float2*)a.in + (long long)b * a.in_bstride;
            const int c = tid & (kTcM - 1), j0 = (tid >> 7) * (kTcR / 2);
            // the column factor ax[c] of the epilogue, folded into the input
            const float2 xs = (ax && c0 + c < a.ncols) ? __ldg(&ax[c0 + c])
                                                       : make_float2(1.0f, 0.0f);
            for (int j = j0; j < j0 + kTcR / 2; j += 4) {
                float xr[4], xi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float2 x = make_float2(0.0f, 0.0f);
                    if (c0 + c < a.ncols) x = in[(long long)(row0 + j + u) * a.ncols + c0 + c];
                    xr[u] = x.x * xs.x - x.y * xs.y;
                    xi[u] = x.x * xs.y + x.y * xs.x;
                }
                float4 h, l;
                split4(xr, h, l);
                *reinterpret_cast<float4*>(&sm.x_hi[cm_index(c, j)]) = h;
                *reinterpret_cast<float4*>(&sm.x_lo[cm_index(c, j)]) = l;
                split4(xi, h, l);
                *reinterpret_cast<float4*>(&sm.x_hi[cm_index(c, kTcR + j)]) = h;
                *reinterpret_cast<float4*>(&sm.x_lo[cm_index(c, kTcR + j)]) = l;
            }
        }
        for (int ch = ch0; ch <= ch1; ++ch) {
            const int q = (ch - ch0) & 1;
            if (ch < ch1 && tid < kTcWork)
                stage_twiddles(sm, q, ch * kTcN, len, n, nmask, row0, tw, ay);
            // staged operands visible to the tensor cores; the accumulator reads of
            // the previous epilogue done; every thread's wait succeeded so far
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            ok = __syncthreads_and(ok);
            if (!ok) break;
            if (ch < ch1 && tid == kTcWork) issue_chunk(sm, q, tmem);
            if (ch > ch0 && tid < kTcWork) {   // epilogue of chunk ch - 1 while chunk ch runs
                const int qp = q ^ 1;
                const unsigned ph = qp ? phase1 : phase0;
                ok = mbar_wait((unsigned)__cvta_generic_to_shared(&sm.mbar[qp]), ph) ? 1 : 0;
                if (qp) phase1 ^= 1u;
                else phase0 ^= 1u;
                if (!__all_sync(0xffffffffu, ok)) {   // warp-uniform before tcgen05.ld
                    if (lane == 0) atomicOr(status, kStatusTimeout);
                    ok = 0;
                    continue;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int kp0 = (ch - 1) * kTcN + mh;
                const unsigned tb = tmem + tlane + qp * 2 * kTcN + mh;
                float re[16], im[16];
                tmem_ld16(tb, re);
                tmem_ld16(tb + kTcN, im);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (col < a.ncols) {
                    // the epilogue's factors are in the operands: only Babinet remains
                    const bool bab = ay && a.occulter;
                    float2* o = out + (long long)kp0 * a.ncols + col;
                    const int jn = min(16, len - kp0);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j < jn)
                            o[(long long)j * a.ncols] =
                                bab ? make_float2(1.0f - re[j], -im[j]) : make_float2(re[j], im[j]);
                    }
                }
            }
        }
    }
    // after giving up: wait (bounded again) for the batches still in flight
    // before the tensor memory is freed
    if (!ok) {
        mbar_wait((unsigned)__cvta_generic_to_shared(&sm.mbar[0]), phase0);
        mbar_wait((unsigned)__cvta_generic_to_shared(&sm.mbar[1]), phase1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((unsigned)kTcCols)
                     : "memory");
    }
}

}  // namespace

bool col_dft_tc_supported(const ColPassArgs& a, int live_rows) {
    // one live tile row, 16-byte aligned column blocks of the input
    return live_rows == kTcR && a.ncols > 0 && a.out_len > 0;
}

void launch_col_dft_tc(const ColPassArgs& a, int n, unsigned* status, cudaStream_t st) {
    const size_t smem = sizeof(TcSmem);
    cudaFuncSetAttribute(k_col_dft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int nchunks = (a.out_len + kTcN - 1) / kTcN;
    const dim3 grid((a.ncols + kTcM - 1) / kTcM, (nchunks + kTcChunksPerCta - 1) / kTcChunksPerCta,
                    a.batch > 1 ? a.batch : 1);
    const unsigned nmask = (n & (n - 1)) == 0 ? (unsigned)(n - 1) : 0u;
    k_col_dft_tc<<<grid, kTcThreads, smem, st>>>(a, n, nmask, status);
}

}  // namespace fres
