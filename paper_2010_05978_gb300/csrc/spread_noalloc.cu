// fresnel_spread_noalloc: fresnel_spread for callers that cannot allocate
// device memory -- code running inside another framework that owns the
// device's memory pool and forbids allocations behind its back, or embedded
// callers (plugins, real-time loops) that may not allocate after start-up.  The scratch the spreading kernels need (node
// records, tile counts and cursors, work-item lists, counters) lives in one
// file-scope static device array of fixed size; the caller still passes the
// points, strengths and output grid.
#include <mutex>
#include <string>

#include "internal.cuh"

// Scratch shared by every call on a device (kept until the process exits).
static __device__ __align__(256) unsigned char g_spread_scratch[FRESNEL_SPREAD_NOALLOC_SCRATCH_BYTES];

// Host code must not use g_spread_scratch as a device address: its name on
// the host is a stand-in.  The device address is looked up once per device
// (with that device current) and kept for the life of the process; after a
// cudaDeviceReset the module may load at another address, so the cached
// address is then stale and the call must not be used again.
static std::mutex g_scratch_mutex;
static unsigned char* g_scratch_ptr[64] = {};

fresnel_status fres_spread_check(const double* g1, const double* g2, const void* c, long long n,
                                 int nf1, int nf2, int w, double beta, void* grid);
fresnel_status fres_spread_run(const double* g1, const double* g2, const void* c, long long n,
                               int nf1, int nf2, int w, double beta, void* grid,
                               unsigned char* scratch, cudaStream_t st);
size_t fres_spread_zero_offsets(long long n, int nf1, int nf2, size_t* counts_off,
                                size_t* work_off, size_t* status_off, size_t* ready_off);

static fresnel_status scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fres_fail(FRESNEL_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spread_scratch);
        if (e != cudaSuccess || !p)
            return fres_fail(FRESNEL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e));
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return FRESNEL_OK;
}

extern "C" fresnel_status fresnel_spread_noalloc(const double* d_g1, const double* d_g2,
                                                 const void* d_c, long long N, int nf1, int nf2,
                                                 int w, double beta, void* d_grid,
                                                 void* cuda_stream) {
    fresnel_status s = fres_spread_check(d_g1, d_g2, d_c, N, nf1, nf2, w, beta, d_grid);
    if (s != FRESNEL_OK) return s;
    if (N > FRESNEL_SPREAD_NOALLOC_MAX_POINTS)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED,
                         "fresnel_spread_noalloc: N exceeds FRESNEL_SPREAD_NOALLOC_MAX_POINTS (" +
                             std::to_string(FRESNEL_SPREAD_NOALLOC_MAX_POINTS) + ")");
    if ((long long)nf1 * nf2 > FRESNEL_SPREAD_NOALLOC_MAX_GRID)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED,
                         "fresnel_spread_noalloc: nf1 * nf2 exceeds FRESNEL_SPREAD_NOALLOC_MAX_GRID (" +
                             std::to_string(FRESNEL_SPREAD_NOALLOC_MAX_GRID) + ")");
    size_t counts_off, work_off, status_off, ready_off;
    const size_t bytes = fres_spread_zero_offsets(N, nf1, nf2, &counts_off, &work_off, &status_off,
                                                  &ready_off);
    if (bytes > (size_t)FRESNEL_SPREAD_NOALLOC_SCRATCH_BYTES)
        return fres_fail(FRESNEL_ERR_UNSUPPORTED, "fresnel_spread_noalloc: scratch too small");
    unsigned char* scratch = nullptr;
    s = scratch_address(&scratch);
    if (s != FRESNEL_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The array keeps the previous call's contents: clear what must start at zero.
    const int ntiles = (nf1 / 32) * (nf2 / 32);
    cudaError_t e = cudaMemsetAsync(scratch + counts_off, 0, sizeof(int) * ntiles, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + work_off, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + status_off, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + ready_off, 0, sizeof(int) * ntiles, st);
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("fresnel_spread_noalloc: clearing the "
                                                       "scratch: ") + cudaGetErrorString(e));
    s = fres_spread_run(d_g1, d_g2, d_c, N, nf1, nf2, w, beta, d_grid, scratch, st);
    if (s != FRESNEL_OK) return s;
    unsigned h = 0;
    e = cudaMemcpyAsync(&h, scratch + status_off, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return fres_fail(FRESNEL_ERR_CUDA, std::string("fresnel_spread_noalloc: ") +
                                               cudaGetErrorString(e));
    if (h & fres::kStatusTimeout)
        return fres_fail(FRESNEL_ERR_TIMEOUT, "fresnel_spread_noalloc: a split tile's chunk gave up waiting");
    if (h) return fres_fail(FRESNEL_ERR_DEVICE, "fresnel_spread_noalloc: non-finite coordinate");
    return FRESNEL_OK;
}
