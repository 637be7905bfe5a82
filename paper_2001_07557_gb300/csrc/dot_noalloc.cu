// dot_noalloc.cu -- lq_dot_noalloc: the FP64 complex inner product of lq_dot,
// for callers that must not allocate device memory.
//
// lq_dot keeps its reduction partials in handle workspace that it grows with
// cudaMalloc on first use.  Some callers cannot allow that: code that owns
// the whole device memory budget through its own pool allocator, latency-
// critical loops where cudaMalloc / cudaFree would synchronise the device, and
// code that runs while a stream is being captured, where an allocation call
// is an error.  This entry point runs the same reduction kernel with its
// scratch in a fixed, file-scope device array instead, and calls no
// allocating routine.
#include <mutex>

#include "blas.h"
#include "handle.h"

namespace {

constexpr int kMaxDevices = 64;
// partials: 2 doubles per block per right-hand side; then one ticket per right-hand side
constexpr size_t kPartialBytes = sizeof(double) * 2 * (size_t)lq::kMaxGrid * LQ_DOT_NOALLOC_MAX_RHS;
constexpr size_t kScratchBytes = kPartialBytes + 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_dot_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_dot_scratch on the current device (host code may not
// use the symbol itself: on the host it only names a stand-in).
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return LQ_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dot_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LQ_ERR_CUDA;
        }
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[device]);
    return LQ_OK;
}

}  // namespace

using namespace lq;

extern "C" int lq_dot_noalloc(lq_handle* h, double* result, const void* a, const void* b, int fmt, int subset,
                              int nrhs, int five_d, void* stream) {
    if (!h || !result || !a || !b || !valid_fmt(fmt)) return LQ_ERR_ARG;
    if (subset < LQ_FULL || subset > LQ_ODD) return LQ_ERR_ARG;
    if (!aligned16(a) || !aligned16(b) || (reinterpret_cast<uintptr_t>(result) & 7u)) return LQ_ERR_LAYOUT;
    long nsites;
    if (five_d) {
        if (h->p.Ls < 1) return LQ_ERR_ARG;
        nrhs = 1;
        nsites = 2L * h->g.Vh * h->p.Ls;
    } else {
        if (nrhs < 1) return LQ_ERR_ARG;
        nsites = (subset == LQ_FULL ? 2L : 1L) * h->g.Vh;
    }
    if (nrhs > LQ_DOT_NOALLOC_MAX_RHS) return LQ_ERR_ARG;  // the static scratch holds at most this many
    DeviceGuard dg(h->device);
    // the result and both fields must be memory the device can address (a plain host
    // pointer would be dereferenced by the kernel)
    if (!device_accessible(result) || !device_accessible(a) || !device_accessible(b)) return LQ_ERR_LAYOUT;
    unsigned char* scratch;
    int rc = scratch_address(h->device, &scratch);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* partial = reinterpret_cast<double*>(scratch);
    unsigned* tickets = reinterpret_cast<unsigned*>(scratch + kPartialBytes);
    // the array keeps the previous call's contents: the tickets must start at zero
    if (cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nrhs, st) != cudaSuccess) return LQ_ERR_CUDA;
    const bool native = (fmt & LQ_NATIVE) != 0;
    const int prec = fmt & 0xF;
    const size_t site_bytes = native ? (size_t)spinor_site_bytes(prec) : (size_t)24 * (prec == LQ_F64 ? 8 : 4);
    return status_of(launch_cdot(fmt, a, b, site_bytes * nsites, nsites, h->g.Vh, nrhs, partial, tickets, result, st));
}
