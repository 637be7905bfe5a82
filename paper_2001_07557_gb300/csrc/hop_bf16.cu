// hop_bf16.cu -- Wilson hop kernels with BF16 storage (one translation unit per
// precision): the shared-memory staged kernel of hop_async.cuh, and, when the
// handle selects it, the tensor-core kernel of hop_mma.cuh for 8 or more
// right-hand sides.
#include "hop_async.cuh"
#include "hop_mma.cuh"

namespace lq {
LQ_INDEX_FAULTS_READER(index_faults_bf16)
cudaError_t launch_hop_bf16(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    (void)block;
    if (hop_mma_applies(a, r12, epi)) return launch_hop_mma<LQ_BF16>(a, dag, epi, st);
    return launch_hop_async<LQ_BF16>(a, r12, dag, epi, st);
}
cudaError_t launch_hop_batch_bf16(const HopArgs* args, const int* lat_off, int nlat, bool r12, bool dag, int epi,
                                 int grid, cudaStream_t st, int* occ) {
    return launch_hop_batch_prec<LQ_BF16>(args, lat_off, nlat, r12, dag, epi, grid, st, occ);
}
}  // namespace lq
