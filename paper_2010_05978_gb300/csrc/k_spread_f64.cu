// FP64 instantiation of the spreading kernel (see spread.cuh).
#include "spread.cuh"
namespace fres {
template <>
void launch_spread<double>(const NodeRec<double>* sorted, const Chunk* chunks, const int* n_meta,
                        int max_chunks, int* ready, int max_split, long long max_spin, double2* grid,
                        int* work, unsigned* status, int nf1, int nf2, int ntx, int ntiles,
                        const KernelShape& ks, int nblocks, cudaStream_t st) {
    launch_spread_impl<double>(sorted, chunks, n_meta, max_chunks, ready, max_split, max_spin, grid,
                           work, status, nf1, nf2, ntx, ntiles, ks, nblocks, st);
}
template <>
void launch_spread_det<double>(const NodeRec<double>* sorted, long long n_records, const Chunk* chunks,
                            const int* n_meta, int max_chunks, const int* split_tiles,
                            int max_split, unsigned long long* split_acc, double* det_part,
                            int tmax, cx_t<double>* grid, int* work, unsigned* status, int nf1,
                            int nf2, int ntx, int ntiles, const KernelShape& ks, cudaStream_t st) {
    launch_spread_det_impl<double>(sorted, n_records, chunks, n_meta, max_chunks, split_tiles,
                               max_split, split_acc, det_part, tmax, grid, work, status, nf1, nf2,
                               ntx, ntiles, ks, st);
}
}  // namespace fres
