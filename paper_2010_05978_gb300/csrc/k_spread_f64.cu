// FP64 instantiation of the spreading kernel (see spread.cuh).
#include "spread.cuh"
namespace fres {
template <>
void launch_spread<double>(const NodeRec<double>* sorted, const Chunk* chunks, const int* n_chunks,
                           int max_chunks, double2* grid, double2* partials, int* tile_counters,
                           int nf1, int nf2, int ntx, const KernelShape& ks, int nblocks,
                           cudaStream_t st) {
    launch_spread_impl<double>(sorted, chunks, n_chunks, max_chunks, grid, partials,
                               tile_counters, nf1, nf2, ntx, ks, nblocks, st);
}
}  // namespace fres
