// Exponential-of-semicircle spreading of the strengths onto the fine grid:
//   b[l1, l2] = sum_j c_j psi(l1 - g1_j) psi(l2 - g2_j),
//   psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)) for |u| < w/2,
// the first stage of the type-1 (Sec. 3.3) and type-3 (Sec. 3.2, eq. nufft3)
// NUFFTs of arXiv:2010.05978 (the paper uses them as a library, FINUFFT).
//
// Owner-computes tiles: every 32 x 32 tile of the grid is produced by one
// work item.  Nodes whose support straddles tiles were duplicated into each
// touched tile by the binning, so each work item adds only inside its own
// tile and writes it back with one coalesced store per grid point: no grid
// clearing pass.  Tiles holding more than the chunk cap of records (the
// dilation rule's spokes all meet at the centre, so a few tiles can hold
// tens of thousands) are split into chunks that run in parallel; such a tile
// is cleared first and its chunks add their nonzero cells with global atomic
// adds.  Work items are handed out dynamically, split chunks first.  A split
// tile's first chunk clears the tile and then raises its ready flag; the
// tile's other chunks build their private sums first and wait for the flag
// (a bounded wait: on giving up they skip their addition and flag
// kStatusTimeout) only before adding.  The first chunk is claimed before the
// others, so its block is running and the wait ends.
//
// Inside a chunk there are no atomics either: each warp owns a private copy
// of the tile in shared memory.  A warp stages 32 records at a time (one per
// lane: support offsets, the w kernel values along x, and c times the w
// kernel values along y), then walks them one by one with its lanes mapped
// onto the w x w support cells, so every lane updates a distinct cell
// (read-modify-write, no conflicts between lanes).  The warps' tiles are
// summed once per chunk.  Dense clusters of nodes (the dilation rule's
// spokes meet at the centre) therefore cost the same as sparse ones.
#pragma once
#include <type_traits>

#include "internal.cuh"

namespace fres {

template <typename T> __device__ __forceinline__ T es_kernel(T z, T beta);
template <> __device__ __forceinline__ float es_kernel<float>(float z, float beta) {
    float a = 1.0f - z * z;
    return a > 0.0f ? expf(beta * (sqrtf(a) - 1.0f)) : 0.0f;
}
template <> __device__ __forceinline__ double es_kernel<double>(double z, double beta) {
    double a = 1.0 - z * z;
    return a > 0.0 ? exp(beta * (sqrt(a) - 1.0)) : 0.0;
}

// The w kernel values of a node with fractional offset f: cell s + a sits at
// offset (a + 1 - w/2 - f) from the node.  The plan's piecewise polynomials
// when present (FP32 and FP64 tables), else exp/sqrt.
template <typename T, int W>
__device__ __forceinline__ void kernel_values(T f, T beta, const horner_t<T>& hz, T* out) {
    if (hz.deg >= 0) {
        horner_eval<W>(hz, f, out);
        return;
    }
    const T half_w = (T)(0.5 * W), two_over_w = (T)(2.0 / W);
#pragma unroll
    for (int a = 0; a < W; ++a) out[a] = es_kernel<T>(((T)(a + 1) - half_w - f) * two_over_w, beta);
}

constexpr int kSpreadWarps = 4;
constexpr int kTileStride = 40;   // float2 row stride: rows land on disjoint bank halves

// Lane -> support cell map of a staged record: column a = lane % W and rows
// b0 + p RPW (p < NPASS), b0 = lane / W.  A record's c ky values are staged
// in the order slot = (b % RPW) NPASS + b / RPW, so each lane's NPASS values
// are adjacent, in rows of CS slots.  FP32 with NPASS even reads them as
// 16-byte pairs: CS = 2 mod 4 keeps the pairs aligned and the staging stores
// at two-way bank conflicts.  Otherwise CS is odd (conflict-free stores).
template <typename T, int W>
struct LaneMap {
    static constexpr int RPW = 32 / W < W ? 32 / W : W;   // rows covered per pass
    static constexpr int NPASS = (W + RPW - 1) / RPW;
    static constexpr bool kPairs = std::is_same<T, float>::value && NPASS % 2 == 0;
    static constexpr int CS = kPairs ? (RPW * NPASS % 4 == 0 ? RPW * NPASS + 2 : RPW * NPASS)
                                     : (RPW * NPASS) | 1;
};

template <typename T, int W>
struct SpreadSmem {
    cx_t<T> tile[kSpreadWarps][kTile * kTileStride];
    cx_t<T> cky[kSpreadWarps][32][LaneMap<T, W>::CS];
    T kx[kSpreadWarps][32][W + 1];
    int dxy[kSpreadWarps][32][2];
    int s_ci;
    int s_ok;
};

// Tile ids are global over the problems of a batched plan: problem
// tile / ntiles, whose grid starts nf1 * nf2 cells after the previous one's.
template <typename T>
__device__ __forceinline__ cx_t<T>* tile_origin(cx_t<T>* grid, int tile, int nf1, int nf2,
                                                int ntx, int ntiles) {
    const int prob = tile / ntiles, lt = tile - prob * ntiles;
    return grid + (long long)prob * nf1 * nf2 + (long long)((lt / ntx) * kTile) * nf1 +
           (lt % ntx) * kTile;
}

// Thread 0 waits for a split tile's ready flag: at most max_spin polls
// (< 0: none), 256 ns apart.  Returns true once the flag is up; on giving up
// flags kStatusTimeout and returns false.
__device__ __forceinline__ bool wait_ready(const int* ready, long long max_spin,
                                           unsigned* status) {
    for (long long it = 0; it < max_spin; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ready) : "memory");
        if (v) return true;
        __nanosleep(256);
    }
    if (status) atomicOr(status, kStatusTimeout);
    return false;
}

// A lane's NPASS staged values (adjacent slots): 16-byte loads where the
// pairs are aligned (FP32, NPASS even: CS and the slot offset b0 NPASS even).
template <typename T, int NPASS>
__device__ __forceinline__ void load_pass_values(const cx_t<T>* src, cx_t<T>* v) {
    if constexpr (std::is_same<T, float>::value && NPASS % 2 == 0) {
#pragma unroll
        for (int k = 0; k < NPASS; k += 2) {
            const float4 q = *reinterpret_cast<const float4*>(src + k);
            v[k] = make_float2(q.x, q.y);
            v[k + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NPASS; ++k) v[k] = src[k];
    }
}

// Chunks are taken dynamically from work[0]; the last block to finish puts
// both counters back to zero for the next launch.
template <typename T, int W>
__global__ void __launch_bounds__(kSpreadWarps * 32)
k_spread(const NodeRec<T>* __restrict__ sorted, const Chunk* __restrict__ chunks,
         const int* __restrict__ n_meta, cx_t<T>* __restrict__ grid, int* __restrict__ work,
         int* __restrict__ ready, int max_split, long long max_spin, unsigned* __restrict__ status,
         int nf1, int nf2, int ntx, int ntiles, T beta, const horner_t<T> hz) {
    constexpr int TT = kTile * kTile;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SpreadSmem<T, W>& sm = *reinterpret_cast<SpreadSmem<T, W>*>(smem_raw);
    constexpr int RPW = LaneMap<T, W>::RPW, NPASS = LaneMap<T, W>::NPASS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    cx_t<T>* my = sm.tile[warp];
    const int n_chunks = n_meta[0];
    for (;;) {
        if (threadIdx.x == 0) sm.s_ci = atomicAdd(&work[0], 1);
        __syncthreads();
        const int ci = sm.s_ci;
        if (ci >= n_chunks) break;
        const Chunk ch = chunks[ci];
        // padding chunks (split 1) hold no records and add nothing
        const int sidx = ch.split >= 2 ? (ch.split >> 1) - 1 : -1;
        cx_t<T>* dst = tile_origin<T>(grid, ch.tile, nf1, nf2, ntx, ntiles);
        if (sidx >= 0 && (ch.split & 1)) {   // a split tile's first chunk: clear it, raise the flag
            for (int e = threadIdx.x; e < TT; e += blockDim.x) {
                cx_t<T> z;
                z.x = (T)0;
                z.y = (T)0;
                dst[(long long)(e / kTile) * nf1 + e % kTile] = z;
            }
            __syncthreads();
            if (threadIdx.x == 0 && sidx < max_split) {
                __threadfence();
                asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(ready + sidx), "r"(1)
                             : "memory");
            }
        }
        const int lt = ch.tile % ntiles;
        const int tx0 = (lt % ntx) * kTile;
        const int ty0 = (lt / ntx) * kTile;
        for (int e = lane; e < TT; e += 32) {
            cx_t<T> z;
            z.x = (T)0;
            z.y = (T)0;
            my[(e / kTile) * kTileStride + (e % kTile)] = z;
        }
        __syncwarp();
        for (int base = ch.begin + warp * 32; base < ch.end; base += kSpreadWarps * 32) {
            const int k = base + lane;
            const int cnt = min(32, ch.end - base);
            if (lane < cnt) {
                const NodeRec<T> r = sorted[k];
                int dx = r.s1 - tx0;
                if (dx >= kTile) dx -= nf1;
                int dy = r.s2 - ty0;
                if (dy >= kTile) dy -= nf2;
                sm.dxy[warp][lane][0] = dx;
                sm.dxy[warp][lane][1] = dy;
                T kxv[W], kyv[W];
                kernel_values<T, W>(r.f1, beta, hz, kxv);
                kernel_values<T, W>(r.f2, beta, hz, kyv);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    sm.kx[warp][lane][a] = kxv[a];
                    cx_t<T> v;
                    v.x = r.cre * kyv[a];
                    v.y = r.cim * kyv[a];
                    sm.cky[warp][lane][(a % RPW) * NPASS + a / RPW] = v;
                }
                sm.kx[warp][lane][W] = (T)0;
            }
            __syncwarp();
            const int a = lane % W, b0 = lane / W;
            const bool lane_on = lane < RPW * W;
            for (int j = 0; j < cnt; ++j) {
                const int dx = sm.dxy[warp][j][0], dy = sm.dxy[warp][j][1];
                const int x = dx + a;
                if (lane_on && (unsigned)x < (unsigned)kTile) {
                    const T kxv = sm.kx[warp][j][a];
                    cx_t<T> cv[NPASS];
                    load_pass_values<T, NPASS>(&sm.cky[warp][j][b0 * NPASS], cv);
#pragma unroll
                    for (int k = 0; k < NPASS; ++k) {
                        const int b = b0 + k * RPW;
                        const int y = dy + b;
                        if (b < W && (unsigned)y < (unsigned)kTile) {
                            const cx_t<T> c = cv[k];
                            cx_t<T>& cell = my[y * kTileStride + x];
                            cx_t<T> o = cell;
                            o.x += c.x * kxv;
                            o.y += c.y * kxv;
                            cell = o;
                        }
                    }
                }
                __syncwarp();
            }
        }
        // a split tile's later chunks add only once its first chunk cleared it
        if (threadIdx.x == 0) {
            sm.s_ok = 1;
            if (sidx >= 0 && !(ch.split & 1))
                sm.s_ok = sidx < max_split ? (wait_ready(ready + sidx, max_spin, status) ? 1 : 0)
                                           : 0;
        }
        __syncthreads();
        if (!sm.s_ok) continue;   // gave up (flagged): the tile misses this chunk
        // sum the warps' tiles (fixed order); store, or add into a shared tile
        for (int e = threadIdx.x; e < TT; e += blockDim.x) {
            const int rr = e / kTile, cc = e % kTile;
            cx_t<T> s = sm.tile[0][rr * kTileStride + cc];
#pragma unroll
            for (int v = 1; v < kSpreadWarps; ++v) {
                const cx_t<T> t = sm.tile[v][rr * kTileStride + cc];
                s.x += t.x;
                s.y += t.y;
            }
            cx_t<T>* g = dst + (long long)rr * nf1 + cc;
            if (!ch.split) {
                *g = s;
            } else if (s.x != (T)0 || s.y != (T)0) {
                atomicAdd(&g->x, s.x);
                atomicAdd(&g->y, s.y);
            }
        }
        __syncthreads();
    }
    // the last block to finish puts the counters and the ready flags back to zero
    if (threadIdx.x == 0) {
        __threadfence();
        sm.s_ok = atomicAdd(&work[1], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (sm.s_ok) {
        for (int i = threadIdx.x; i < max_split; i += blockDim.x) ready[i] = 0;
        if (threadIdx.x == 0) {
            work[0] = 0;
            work[1] = 0;
        }
    }
}

// ------------------------------------------------------------------ deterministic mode
// Exact fixed-point accumulation.  Every contribution v (one component of
// c_j psi psi, rounded once in T) is scaled by 2^S and held as H 2^40 + L with
// integers H = rint(2^(S-40) v) and L = rint(2^S v - H 2^40): the difference
// is exact in T, so L only rounds 2^S v to an integer.  Sums of integers do
// not depend on the order of the additions (two's-complement adds wrap
// associatively), so neither the order of the records within a tile (it
// follows the scatter's atomic reservations) nor the order in which a split
// tile's chunks finish changes a bit of the grid.  S is fixed per evaluation
// from B = 2 T_max c_max (T_max: records of the fullest tile; c_max: the
// largest strength component, a maximum, which no order changes):
// 2^S B <= 2^100, so |sum H| < 2^61 and, with T_max < 2^23, |sum L| < 2^62.
// The resolution 2^-S <= B 2^-99 lies far below either precision's rounding.

template <typename T>
struct DetScale {
    T a, b;       // 2^S = a b (each factor inside T's range)
    double inv;   // 2^-S
};

// c_max from the partial maxima (+inf marks a non-finite strength) and the
// scale; flags kStatusNonFinite (scale 1) or kStatusOverflow (B > 2^350).
template <typename T>
__device__ __forceinline__ DetScale<T> det_scale(double cmax, int tmax, unsigned* status,
                                                 bool report) {
    int S = 0;
    if (!(cmax < INFINITY)) {
        if (report && status) atomicOr(status, kStatusNonFinite);
    } else if (cmax > 0.0) {
        int e;
        frexp(2.0 * (double)max(tmax, 1) * cmax, &e);   // B < 2^e
        S = 100 - e;
        if (S < -250) {
            if (report && status) atomicOr(status, kStatusOverflow);
            S = -250;
        }
        S = min(S, 250);
    }
    DetScale<T> d;
    d.a = (T)ldexp(1.0, S / 2);
    d.b = (T)ldexp(1.0, S - S / 2);
    d.inv = ldexp(1.0, -S);
    return d;
}

__device__ __forceinline__ long long det_to_ll(float v) { return __float2ll_rn(v); }
__device__ __forceinline__ long long det_to_ll(double v) { return __double2ll_rn(v); }

// (H, L) of one contribution
template <typename T>
__device__ __forceinline__ void det_split(T v, const DetScale<T>& sc, long long& h, long long& l) {
    const T x = (v * sc.a) * sc.b;
    const T hh = rint(x * (T)9.094947017729282379150390625e-13);   // 2^-40
    h = det_to_ll(hh);
    l = det_to_ll(x - hh * (T)1099511627776.0);                    // 2^40
}

template <typename T>
__device__ __forceinline__ T det_value(long long h, long long l, double inv) {
    return (T)(((double)h * 1099511627776.0 + (double)l) * inv);
}

// Block maximum of |cre|, |cim| over the records into part[blockIdx.x]
// (+inf where a strength is not finite).
template <typename T>
__global__ void __launch_bounds__(256)
k_det_cmax(const NodeRec<T>* __restrict__ rec, long long n, double* __restrict__ part) {
    __shared__ double s[8];
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = fabs((double)rec[i].cre), b = fabs((double)rec[i].cim);
        m = (a < INFINITY && b < INFINITY) ? fmax(m, fmax(a, b)) : INFINITY;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s[w]);
        part[blockIdx.x] = m;
    }
}

// max over the kDetPartials partial maxima, by one block (every block
// computes the same value)
__device__ __forceinline__ double det_block_cmax(const double* __restrict__ part, double* s_red) {
    double m = 0.0;
    for (int i = threadIdx.x; i < kDetPartials; i += blockDim.x) m = fmax(m, part[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_red[w]);
    __syncthreads();
    return m;
}

template <typename T, int W>
struct DetSmem {
    unsigned long long acc[kTile * kTile * 4];   // per cell: re H, re L, im H, im L
    cx_t<T> cky[kSpreadWarps][32][LaneMap<T, W>::CS];
    T kx[kSpreadWarps][32][W + 1];
    int dxy[kSpreadWarps][32][2];
    double red[kSpreadWarps];
    int s_ci;
    int s_last;
};

// The deterministic spreading pass: one fixed-point tile per block (shared
// 64-bit atomic adds: warps may meet on a cell), chunks claimed dynamically
// as in k_spread.  A plain tile is converted and stored; a split tile's
// chunks add their nonzero cells into its fixed-point accumulator in global
// memory (64-bit atomic adds), which k_spread_det_finish converts.  No chunk
// waits on another.
template <typename T, int W>
__global__ void __launch_bounds__(kSpreadWarps * 32)
k_spread_det(const NodeRec<T>* __restrict__ sorted, const Chunk* __restrict__ chunks,
             const int* __restrict__ n_meta, cx_t<T>* __restrict__ grid, int* __restrict__ work,
             unsigned long long* __restrict__ split_acc, int max_split,
             const double* __restrict__ det_part, int tmax, unsigned* __restrict__ status,
             int nf1, int nf2, int ntx, int ntiles, T beta, const horner_t<T> hz) {
    constexpr int TT = kTile * kTile;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DetSmem<T, W>& sm = *reinterpret_cast<DetSmem<T, W>*>(smem_raw);
    constexpr int RPW = LaneMap<T, W>::RPW, NPASS = LaneMap<T, W>::NPASS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DetScale<T> sc =
        det_scale<T>(det_block_cmax(det_part, sm.red), tmax, status, blockIdx.x == 0 && threadIdx.x == 0);
    const int n_chunks = n_meta[0];
    for (;;) {
        if (threadIdx.x == 0) sm.s_ci = atomicAdd(&work[0], 1);
        __syncthreads();
        const int ci = sm.s_ci;
        if (ci >= n_chunks) break;
        const Chunk ch = chunks[ci];
        if (ch.split == 1) {   // padding: no records
            __syncthreads();
            continue;
        }
        const int sidx = ch.split >= 2 ? (ch.split >> 1) - 1 : -1;
        const int lt = ch.tile % ntiles;
        const int tx0 = (lt % ntx) * kTile;
        const int ty0 = (lt / ntx) * kTile;
        for (int e = threadIdx.x; e < TT * 4; e += blockDim.x) sm.acc[e] = 0ull;
        __syncthreads();
        for (int base = ch.begin + warp * 32; base < ch.end; base += kSpreadWarps * 32) {
            const int k = base + lane;
            const int cnt = min(32, ch.end - base);
            if (lane < cnt) {
                const NodeRec<T> r = sorted[k];
                int dx = r.s1 - tx0;
                if (dx >= kTile) dx -= nf1;
                int dy = r.s2 - ty0;
                if (dy >= kTile) dy -= nf2;
                sm.dxy[warp][lane][0] = dx;
                sm.dxy[warp][lane][1] = dy;
                T kxv[W], kyv[W];
                kernel_values<T, W>(r.f1, beta, hz, kxv);
                kernel_values<T, W>(r.f2, beta, hz, kyv);
#pragma unroll
                for (int a = 0; a < W; ++a) {
                    sm.kx[warp][lane][a] = kxv[a];
                    cx_t<T> v;
                    v.x = r.cre * kyv[a];
                    v.y = r.cim * kyv[a];
                    sm.cky[warp][lane][(a % RPW) * NPASS + a / RPW] = v;
                }
                sm.kx[warp][lane][W] = (T)0;
            }
            __syncwarp();
            const int a = lane % W, b0 = lane / W;
            const bool lane_on = lane < RPW * W;
            for (int j = 0; j < cnt; ++j) {
                const int dx = sm.dxy[warp][j][0], dy = sm.dxy[warp][j][1];
                const int x = dx + a;
                if (lane_on && (unsigned)x < (unsigned)kTile) {
                    const T kxv = sm.kx[warp][j][a];
#pragma unroll
                    for (int q = 0; q < NPASS; ++q) {
                        const int b = b0 + q * RPW;
                        const int y = dy + b;
                        if (b < W && (unsigned)y < (unsigned)kTile) {
                            const cx_t<T> c = sm.cky[warp][j][b0 * NPASS + q];
                            long long h, l;
                            unsigned long long* cell = sm.acc + (y * kTile + x) * 4;
                            det_split<T>(c.x * kxv, sc, h, l);
                            atomicAdd(cell, (unsigned long long)h);
                            atomicAdd(cell + 1, (unsigned long long)l);
                            det_split<T>(c.y * kxv, sc, h, l);
                            atomicAdd(cell + 2, (unsigned long long)h);
                            atomicAdd(cell + 3, (unsigned long long)l);
                        }
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (sidx < 0) {
            cx_t<T>* dst = tile_origin<T>(grid, ch.tile, nf1, nf2, ntx, ntiles);
            for (int e = threadIdx.x; e < TT; e += blockDim.x) {
                const unsigned long long* c = sm.acc + e * 4;
                cx_t<T> v;
                v.x = det_value<T>((long long)c[0], (long long)c[1], sc.inv);
                v.y = det_value<T>((long long)c[2], (long long)c[3], sc.inv);
                dst[(long long)(e / kTile) * nf1 + e % kTile] = v;
            }
        } else if (sidx < max_split) {
            unsigned long long* g = split_acc + (size_t)sidx * TT * 4;
            for (int e = threadIdx.x; e < TT * 4; e += blockDim.x)
                if (sm.acc[e]) atomicAdd(g + e, sm.acc[e]);
        } else if (threadIdx.x == 0 && status) {
            atomicOr(status, kStatusOverflow);   // no accumulator for this split tile
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        sm.s_last = atomicAdd(&work[1], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (sm.s_last && threadIdx.x == 0) {
        work[0] = 0;
        work[1] = 0;
    }
}

// Split tiles: fixed-point accumulator -> grid tile, then the accumulator
// back to zero for the next evaluation.  Block s takes split tiles s,
// s + gridDim.x, ... (split_tiles[s] < 0: unused slot).
template <typename T>
__global__ void __launch_bounds__(256)
k_spread_det_finish(const int* __restrict__ split_tiles, int max_split,
                    unsigned long long* __restrict__ split_acc, const double* __restrict__ det_part,
                    int tmax, cx_t<T>* __restrict__ grid, int nf1, int nf2, int ntx, int ntiles) {
    constexpr int TT = kTile * kTile;
    __shared__ double red[8];
    const DetScale<T> sc = det_scale<T>(det_block_cmax(det_part, red), tmax, nullptr, false);
    for (int s = blockIdx.x; s < max_split; s += gridDim.x) {
        const int tile = split_tiles[s];
        if (tile < 0) continue;
        cx_t<T>* dst = tile_origin<T>(grid, tile, nf1, nf2, ntx, ntiles);
        unsigned long long* g = split_acc + (size_t)s * TT * 4;
        for (int e = threadIdx.x; e < TT; e += blockDim.x) {
            const unsigned long long* c = g + e * 4;
            cx_t<T> v;
            v.x = det_value<T>((long long)c[0], (long long)c[1], sc.inv);
            v.y = det_value<T>((long long)c[2], (long long)c[3], sc.inv);
            dst[(long long)(e / kTile) * nf1 + e % kTile] = v;
            g[e * 4] = g[e * 4 + 1] = g[e * 4 + 2] = g[e * 4 + 3] = 0ull;
        }
    }
}

template <typename T, int W>
void launch_spread_det_w(const NodeRec<T>* sorted, long long n_records, const Chunk* chunks,
                         const int* n_meta, int max_chunks, const int* split_tiles, int max_split,
                         unsigned long long* split_acc, double* det_part, int tmax,
                         cx_t<T>* grid, int* work, unsigned* status, int nf1, int nf2, int ntx,
                         int ntiles, T beta, const horner_t<T>& hz, cudaStream_t st) {
    k_det_cmax<T><<<kDetPartials, 256, 0, st>>>(sorted, n_records, det_part);
    const size_t smem = sizeof(DetSmem<T, W>);
    cudaFuncSetAttribute(k_spread_det<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_det<T, W>, kSpreadWarps * 32,
                                                  smem);
    int g = 152 * (per_sm < 1 ? 1 : per_sm);
    if (g > max_chunks) g = max_chunks;
    if (g < 1) g = 1;
    k_spread_det<T, W><<<g, kSpreadWarps * 32, smem, st>>>(sorted, chunks, n_meta, grid, work,
                                                           split_acc, max_split, det_part, tmax,
                                                           status, nf1, nf2, ntx, ntiles, beta,
                                                           hz);
    if (max_split > 0)
        k_spread_det_finish<T><<<max_split < 152 * 4 ? max_split : 152 * 4, 256, 0, st>>>(
            split_tiles, max_split, split_acc, det_part, tmax, grid, nf1, nf2, ntx, ntiles);
}

template <typename T>
void launch_spread_det_impl(const NodeRec<T>* sorted, long long n_records, const Chunk* chunks,
                            const int* n_meta, int max_chunks, const int* split_tiles,
                            int max_split, unsigned long long* split_acc, double* det_part,
                            int tmax, cx_t<T>* grid, int* work, unsigned* status, int nf1,
                            int nf2, int ntx, int ntiles, const KernelShape& ks, cudaStream_t st) {
    T beta = (T)ks.beta;
#define FRES_DET_CASE(WW)                                                                     \
    case WW:                                                                                  \
        launch_spread_det_w<T, WW>(sorted, n_records, chunks, n_meta, max_chunks, split_tiles, \
                                   max_split, split_acc, det_part, tmax, grid, work, status,  \
                                   nf1, nf2, ntx, ntiles, beta, horner_of<T>(ks), st);        \
        break;
    switch (ks.w) {
        FRES_DET_CASE(2) FRES_DET_CASE(3) FRES_DET_CASE(4) FRES_DET_CASE(5)
        FRES_DET_CASE(6) FRES_DET_CASE(7) FRES_DET_CASE(8) FRES_DET_CASE(9)
        FRES_DET_CASE(10) FRES_DET_CASE(11) FRES_DET_CASE(12) FRES_DET_CASE(13)
        FRES_DET_CASE(14) FRES_DET_CASE(15) FRES_DET_CASE(16)
        default: break;
    }
#undef FRES_DET_CASE
}

template <typename T, int W>
void launch_spread_w(const NodeRec<T>* sorted, const Chunk* chunks, const int* n_meta,
                     int max_chunks, int* ready, int max_split, long long max_spin,
                     cx_t<T>* grid, int* work, unsigned* status, int nf1, int nf2, int ntx,
                     int ntiles, T beta, const horner_t<T>& hz, int nblocks, cudaStream_t st) {
    const size_t smem = sizeof(SpreadSmem<T, W>);
    cudaFuncSetAttribute(k_spread<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread<T, W>, kSpreadWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int g = 152 * per_sm;
    if (nblocks > 0 && nblocks < g) g = nblocks;
    if (g > max_chunks) g = max_chunks;
    if (g < 1) g = 1;
    k_spread<T, W><<<g, kSpreadWarps * 32, smem, st>>>(sorted, chunks, n_meta, grid, work,
                                                       ready, max_split, max_spin, status, nf1,
                                                       nf2, ntx, ntiles, beta, hz);
}

template <typename T>
void launch_spread_impl(const NodeRec<T>* sorted, const Chunk* chunks, const int* n_meta,
                        int max_chunks, int* ready, int max_split, long long max_spin,
                        cx_t<T>* grid, int* work, unsigned* status, int nf1, int nf2, int ntx,
                        int ntiles, const KernelShape& ks, int nblocks, cudaStream_t st) {
    T beta = (T)ks.beta;
#define FRES_SPREAD_CASE(WW)                                                                  \
    case WW:                                                                                  \
        launch_spread_w<T, WW>(sorted, chunks, n_meta, max_chunks, ready, max_split,         \
                               max_spin, grid, work, status, nf1, nf2, ntx, ntiles, beta,    \
                               horner_of<T>(ks), nblocks, st);                               \
        break;
    switch (ks.w) {
        FRES_SPREAD_CASE(2) FRES_SPREAD_CASE(3) FRES_SPREAD_CASE(4) FRES_SPREAD_CASE(5)
        FRES_SPREAD_CASE(6) FRES_SPREAD_CASE(7) FRES_SPREAD_CASE(8) FRES_SPREAD_CASE(9)
        FRES_SPREAD_CASE(10) FRES_SPREAD_CASE(11) FRES_SPREAD_CASE(12) FRES_SPREAD_CASE(13)
        FRES_SPREAD_CASE(14) FRES_SPREAD_CASE(15) FRES_SPREAD_CASE(16)
        default: break;
    }
#undef FRES_SPREAD_CASE
}

}  // namespace fres
