// Exponential-of-semicircle spreading of the strengths onto the fine grid:
//   b[l1, l2] = sum_j c_j psi(l1 - g1_j) psi(l2 - g2_j),
//   psi(u) = exp(beta (sqrt(1 - (2u/w)^2) - 1)) for |u| < w/2,
// the first stage of the type-1 (Sec. 3.3) and type-3 (Sec. 3.2, eq. nufft3)
// NUFFTs of arXiv:2010.05978 (the paper uses them as a library, FINUFFT).
//
// Owner-computes tiles: every 32 x 32 tile of the grid is produced by one
// work item (or, for tiles holding more than the chunk cap of node records,
// several chunks whose partial tiles are summed in a fixed order by the last
// chunk to finish).  Nodes whose support straddles tiles were duplicated into
// each touched tile by the binning, so each chunk adds only inside its own
// tile: accumulation is in shared memory, write-back is one coalesced store
// per grid point, and no global atomics or grid clearing are needed.
#pragma once
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

template <typename T, int W>
__global__ void __launch_bounds__(256)
k_spread(const NodeRec<T>* __restrict__ sorted, const Chunk* __restrict__ chunks,
         const int* __restrict__ n_chunks_p, cx_t<T>* __restrict__ grid,
         cx_t<T>* __restrict__ partials, int* __restrict__ tile_counters, int nf1, int nf2,
         int ntx, T beta) {
    constexpr int TT = kTile * kTile;
    __shared__ cx_t<T> tile[TT];
    __shared__ int s_last;
    const int n_chunks = *n_chunks_p;
    const T half_w = (T)(0.5 * W);
    const T two_over_w = (T)(2.0 / W);
    for (int ci = blockIdx.x; ci < n_chunks; ci += gridDim.x) {
        const Chunk ch = chunks[ci];
        const int tx0 = (ch.tile % ntx) * kTile;
        const int ty0 = (ch.tile / ntx) * kTile;
        for (int e = threadIdx.x; e < TT; e += blockDim.x) {
            tile[e].x = (T)0;
            tile[e].y = (T)0;
        }
        __syncthreads();
        for (int k = ch.begin + threadIdx.x; k < ch.end; k += blockDim.x) {
            const NodeRec<T> r = sorted[k];
            int dx = r.s1 - tx0;
            if (dx >= kTile) dx -= nf1;
            int dy = r.s2 - ty0;
            if (dy >= kTile) dy -= nf2;
            T kx[W], ky[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                // cell s + a sits at offset (a + 1 - w/2 - f) from the node
                kx[a] = es_kernel<T>(((T)(a + 1) - half_w - r.f1) * two_over_w, beta);
                ky[a] = es_kernel<T>(((T)(a + 1) - half_w - r.f2) * two_over_w, beta);
            }
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const int yy = dy + b;
                if (yy >= 0 && yy < kTile) {
                    const T vr = r.cre * ky[b], vi = r.cim * ky[b];
#pragma unroll
                    for (int a = 0; a < W; ++a) {
                        const int xx = dx + a;
                        if (xx >= 0 && xx < kTile) {
                            atomicAdd(&tile[yy * kTile + xx].x, vr * kx[a]);
                            atomicAdd(&tile[yy * kTile + xx].y, vi * kx[a]);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (ch.slot < 0) {
            for (int e = threadIdx.x; e < TT; e += blockDim.x) {
                const int rr = e / kTile, cc = e % kTile;
                grid[(long long)(ty0 + rr) * nf1 + tx0 + cc] = tile[e];
            }
        } else {
            cx_t<T>* mine = partials + (long long)ch.slot * TT;
            for (int e = threadIdx.x; e < TT; e += blockDim.x) mine[e] = tile[e];
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                s_last = (atomicAdd(&tile_counters[ch.tile], 1) == ch.nchunks - 1);
            __syncthreads();
            if (s_last) {
                __threadfence();
                for (int e = threadIdx.x; e < TT; e += blockDim.x) {
                    T sr = (T)0, si = (T)0;
                    for (int s = 0; s < ch.nchunks; ++s) {
                        const cx_t<T> v = __ldcg(&partials[(long long)(ch.first_slot + s) * TT + e]);
                        sr += v.x;
                        si += v.y;
                    }
                    const int rr = e / kTile, cc = e % kTile;
                    cx_t<T> o;
                    o.x = sr;
                    o.y = si;
                    grid[(long long)(ty0 + rr) * nf1 + tx0 + cc] = o;
                }
                if (threadIdx.x == 0) tile_counters[ch.tile] = 0;
            }
        }
        __syncthreads();
    }
}

template <typename T>
void launch_spread_impl(const NodeRec<T>* sorted, const Chunk* chunks, const int* n_chunks,
                        int max_chunks, cx_t<T>* grid, cx_t<T>* partials, int* tile_counters,
                        int nf1, int nf2, int ntx, const KernelShape& ks, int nblocks,
                        cudaStream_t st) {
    int g = nblocks < max_chunks ? nblocks : max_chunks;
    if (g < 1) g = 1;
    T beta = (T)ks.beta;
#define FRES_SPREAD_CASE(WW)                                                                  \
    case WW:                                                                                  \
        k_spread<T, WW><<<g, 256, 0, st>>>(sorted, chunks, n_chunks, grid, partials,          \
                                           tile_counters, nf1, nf2, ntx, beta);               \
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
