// hop_f64.cu -- Wilson hop kernels with F64 storage (one translation unit per precision).
#include "hop.cuh"

namespace lq {
LQ_INDEX_FAULTS_READER(index_faults_f64)
cudaError_t launch_hop_f64(const HopArgs& a, bool r12, bool dag, int epi, int block, cudaStream_t st) {
    return launch_hop_prec<LQ_F64>(a, r12, dag, epi, block, st);
}
}  // namespace lq
