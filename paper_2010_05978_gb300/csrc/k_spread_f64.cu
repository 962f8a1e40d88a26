// FP64 instantiation of the spreading kernel (see spread.cuh).
#include "spread.cuh"
namespace fres {
template <>
void launch_spread<double>(const NodeRec<double>* sorted, const Chunk* chunks, const int* n_meta,
                        int max_chunks, const int* split_tiles, int max_split, double2* grid,
                        int* work, int nf1, int nf2, int ntx, int ntiles, const KernelShape& ks,
                        int nblocks, cudaStream_t st) {
    launch_spread_impl<double>(sorted, chunks, n_meta, max_chunks, split_tiles, max_split, grid, work,
                           nf1, nf2, ntx, ntiles, ks, nblocks, st);
}
}  // namespace fres
