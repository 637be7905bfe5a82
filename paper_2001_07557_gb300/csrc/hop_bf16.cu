// hop_bf16.cu -- Wilson hop kernels with BF16 storage (one translation unit per
// precision): the shared-memory staged kernel of hop_async.cuh.
#include "hop_async.cuh"

namespace lq {
cudaError_t launch_hop_bf16(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    (void)block;
    return launch_hop_async<LQ_BF16>(a, r12, dag, epi, st);
}
}  // namespace lq
