// hop_bf16.cu -- Wilson hop kernels with BF16 storage (one translation unit per precision).
#include "hop.cuh"

namespace lq {
cudaError_t launch_hop_bf16(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    return launch_hop_prec<LQ_BF16>(a, r12, dag, epi, block, st);
}
}  // namespace lq
