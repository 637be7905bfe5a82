// hop_f32.cu -- Wilson hop kernels with F32 storage (one translation unit per
// precision): the shared-memory staged kernel of hop_async.cuh, and for a
// launch of several right-hand sides (or domain-wall slices) the kernel of
// hop_shared.cuh, whose blocks share each link between them.
#include "hop_async.cuh"
#include "hop_shared.cuh"

namespace lq {
LQ_INDEX_FAULTS_READER(index_faults_f32)
cudaError_t launch_hop_f32(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    (void)block;
    if (hop_shared_applies(a)) return launch_hop_shared<LQ_F32>(a, r12, dag, epi, st);
    return launch_hop_async<LQ_F32>(a, r12, dag, epi, st);
}
cudaError_t launch_hop_batch_f32(const HopArgs* args, const int* lat_off, int nlat, bool r12, bool dag, int epi,
                                 int grid, cudaStream_t st, int* occ) {
    return launch_hop_batch_prec<LQ_F32>(args, lat_off, nlat, r12, dag, epi, grid, st, occ);
}
}  // namespace lq
