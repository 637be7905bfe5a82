// cg.cu -- conjugate-gradient solvers on the normal equations.
#include "handle.h"

extern "C" {

int cg_solve(lq_handle* h, void* x, const void* b, const lq_cg_params* cp, lq_cg_stats* stats, void* stream) {
    (void)h; (void)x; (void)b; (void)cp; (void)stats; (void)stream;
    return LQ_ERR_ARG;
}

int lq_batch_cg_solve(lq_handle** hs, int nlat, void** xs, const void** bs, const lq_cg_params* cp,
                      lq_cg_stats* stats, void* stream) {
    (void)hs; (void)nlat; (void)xs; (void)bs; (void)cp; (void)stats; (void)stream;
    return LQ_ERR_ARG;
}

}  // extern "C"
