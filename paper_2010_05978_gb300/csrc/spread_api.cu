// fresnel_spread: the exponential-of-semicircle spreading step of the NUFFT
// (the first stage of the type-1 / type-3 transforms behind the fast
// algorithm of arXiv:2010.05978, Secs. 3.2-3.3) as a standalone call, for
// points given directly by periodic grid coordinates.  Same kernels as the
// plan path: records + tile counts -> scan -> scatter -> split-tile clearing
// -> owner-computes tile spreading.
#include <cmath>
#include <string>

#include "internal.cuh"

using namespace fres;

namespace {

struct SpreadScratch {
    NodeRec<float>* rec;
    NodeRec<float>* sorted;
    int* counts;
    int* cursor;
    Chunk* chunks;
    int* split_tiles;
    int* n_meta;
    int* work;
    unsigned* status;
    int* ready;
};

// Upper bounds that hold for any input: every point touches at most four
// tiles; every tile is one chunk plus one per chunk_cap records when split.
constexpr int kStandaloneChunkCap = 512;

long long max_records(long long n) { return 4 * n; }
long long max_chunks(long long n, int ntiles) {
    return ntiles + max_records(n) / kStandaloneChunkCap + 1;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the scratch pieces inside one block of memory.
size_t scratch_layout(long long n, int ntiles, size_t off[10]) {
    size_t o = 0;
    off[0] = o; o = align256(o + sizeof(NodeRec<float>) * (size_t)std::max(1LL, n));
    off[1] = o; o = align256(o + sizeof(NodeRec<float>) * (size_t)std::max(1LL, max_records(n)));
    off[2] = o; o = align256(o + sizeof(int) * (size_t)ntiles);
    off[3] = o; o = align256(o + sizeof(int) * (size_t)ntiles);
    off[4] = o; o = align256(o + sizeof(Chunk) * (size_t)max_chunks(n, ntiles));
    off[5] = o; o = align256(o + sizeof(int) * (size_t)ntiles);
    off[6] = o; o = align256(o + 2 * sizeof(int));
    off[7] = o; o = align256(o + 2 * sizeof(int));
    off[8] = o; o = align256(o + sizeof(unsigned));
    off[9] = o; o = align256(o + sizeof(int) * (size_t)ntiles);
    return o;
}

SpreadScratch carve(unsigned char* base, const size_t off[10]) {
    SpreadScratch s;
    s.rec = (NodeRec<float>*)(base + off[0]);
    s.sorted = (NodeRec<float>*)(base + off[1]);
    s.counts = (int*)(base + off[2]);
    s.cursor = (int*)(base + off[3]);
    s.chunks = (Chunk*)(base + off[4]);
    s.split_tiles = (int*)(base + off[5]);
    s.n_meta = (int*)(base + off[6]);
    s.work = (int*)(base + off[7]);
    s.status = (unsigned*)(base + off[8]);
    s.ready = (int*)(base + off[9]);
    return s;
}

}  // namespace

// Validation shared with the allocation-free variant.
fresnel_status fres_spread_check(const double* g1, const double* g2, const void* c, long long n,
                                 int nf1, int nf2, int w, double beta, void* grid) {
    if (n < 0) return fres_fail(FRESNEL_ERR_ARG, "N must be >= 0");
    if (n > 0 && (!g1 || !g2 || !c)) return fres_fail(FRESNEL_ERR_ARG, "point arrays are NULL");
    if (!grid) return fres_fail(FRESNEL_ERR_ARG, "grid is NULL");
    if (w < 2 || w > kMaxW) return fres_fail(FRESNEL_ERR_ARG, "w must lie in [2, 16]");
    if (!(beta > 0) || !std::isfinite(beta)) return fres_fail(FRESNEL_ERR_ARG, "beta must be > 0");
    if (nf1 < 64 || nf2 < 64 || nf1 % kTile || nf2 % kTile)
        return fres_fail(FRESNEL_ERR_ARG, "nf1, nf2 must be multiples of 32 and >= 64");
    if (n > (1LL << 28)) return fres_fail(FRESNEL_ERR_UNSUPPORTED, "more than 2^28 points");
    return FRESNEL_OK;
}

// Runs the spreading pipeline with scratch already in place.  counts, work
// and the split tiles' ready flags must be zero on entry (all are left zero).
fresnel_status fres_spread_run(const double* g1, const double* g2, const void* c, long long n,
                               int nf1, int nf2, int w, double beta, void* grid,
                               unsigned char* scratch, cudaStream_t st) {
    const int ntx = nf1 / kTile, nty = nf2 / kTile, ntiles = ntx * nty;
    size_t off[10];
    scratch_layout(n, ntiles, off);
    SpreadScratch s = carve(scratch, off);
    ChirpParams cp{};
    cp.w = w;
    cp.nf1 = nf1;
    cp.nf2 = nf2;
    cp.ntx = ntx;
    cp.nty = nty;
    KernelShape ks{};
    ks.w = w;
    ks.beta = beta;
    ks.betaf = (float)beta;
    ks.horner.deg = -1;   // exact exp/sqrt kernel values
    const int mch = (int)max_chunks(n, ntiles);
    launch_records_from_coords(n, g1, g2, (const float2*)c, cp, s.rec, s.counts, s.status, st);
    launch_scan_chunks(ntiles, s.counts, s.cursor, s.chunks, s.n_meta, s.split_tiles,
                       kStandaloneChunkCap, mch, ntiles, st);
    launch_scatter<float>(n, cp, s.rec, s.cursor, s.sorted, max_records(n), s.status, st);
    launch_spread<float>(s.sorted, s.chunks, s.n_meta, mch, s.ready, ntiles, kDefaultMaxSpin,
                         (float2*)grid, s.work, s.status, nf1, nf2, ntx, ntiles, ks, 0, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("spread launch: ") + cudaGetErrorString(e));
    return FRESNEL_OK;
}

size_t fres_spread_scratch_bytes(long long n, int nf1, int nf2) {
    size_t off[10];
    return scratch_layout(n, (nf1 / kTile) * (nf2 / kTile), off);
}

size_t fres_spread_zero_offsets(long long n, int nf1, int nf2, size_t* counts_off,
                                size_t* work_off, size_t* status_off, size_t* ready_off) {
    size_t off[10];
    size_t total = scratch_layout(n, (nf1 / kTile) * (nf2 / kTile), off);
    *counts_off = off[2];
    *work_off = off[7];
    *status_off = off[8];
    *ready_off = off[9];
    return total;
}

extern "C" fresnel_status fresnel_spread(const double* d_g1, const double* d_g2, const void* d_c,
                                         long long N, int nf1, int nf2, int w, double beta,
                                         void* d_grid, void* cuda_stream) {
    fresnel_status s = fres_spread_check(d_g1, d_g2, d_c, N, nf1, nf2, w, beta, d_grid);
    if (s != FRESNEL_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    size_t counts_off, work_off, status_off, ready_off;
    const size_t bytes = fres_spread_zero_offsets(N, nf1, nf2, &counts_off, &work_off, &status_off,
                                                  &ready_off);
    const int ntiles = (nf1 / kTile) * (nf2 / kTile);
    unsigned char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fres_fail(FRESNEL_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(scratch + counts_off, 0, sizeof(int) * ntiles, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + work_off, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + status_off, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + ready_off, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(scratch, st);
        cudaStreamSynchronize(st);
        return fres_fail(FRESNEL_ERR_CUDA, std::string("fresnel_spread: clearing the scratch: ") +
                                               cudaGetErrorString(e));
    }
    s = fres_spread_run(d_g1, d_g2, d_c, N, nf1, nf2, w, beta, d_grid, scratch, st);
    unsigned h = 0;
    cudaMemcpyAsync(&h, scratch + status_off, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    e = cudaStreamSynchronize(st);
    if (s != FRESNEL_OK) return s;
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("fresnel_spread: ") + cudaGetErrorString(e));
    if (h & kStatusTimeout)
        return fres_fail(FRESNEL_ERR_TIMEOUT, "fresnel_spread: a split tile's chunk gave up waiting");
    if (h) return fres_fail(FRESNEL_ERR_DEVICE, "fresnel_spread: non-finite coordinate");
    return FRESNEL_OK;
}
