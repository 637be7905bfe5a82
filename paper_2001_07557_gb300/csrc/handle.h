// handle.h -- the opaque lq_handle and the host-side helpers shared by the
// C ABI translation units (apply calls, solvers).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "lqcd.h"
#include "lqcd_kernels.h"

struct lq_handle {
    lq_params p;
    lq::Geom g;
    int device;
    int U_prec;       // precision of the saved site-major gauge copy
    void* U_sm;       // device copy of the site-major gauge field (source for every packing)
    void* links[4][2];  // native links per [precision][compress12], packed on first use
    struct Buf {
        void* ptr;
        size_t bytes;
    } ws[26];         // workspace buffers, grown on demand
    int hop_block[4]; // threads per block of the hop kernels, per precision
    int hop_kernel;   // LQ_HOP_CUDA_CORES (default) or LQ_HOP_TENSOR_CORES (lq_set_hop_kernel)
    const int* skip;  // per-rhs early-exit flags the solvers hand to the hop launches (else null)
    int skip_stride;
    // fused |K p|^2 for the next operator output (the K of K^dag K), else null
    double* red_partial;
    unsigned* red_ticket;
    lq::CgScalars* red_st;
    cudaStream_t solver_stream;  // private non-blocking stream the solvers capture into graphs
    void* pinned;                // pinned host buffer the solvers poll their scalars into
    size_t pinned_bytes;
    // executable CG iteration graphs kept across solves, one per solver shape
    // (key: operator, search-direction and residual precisions, right-hand
    // sides); each solve captures afresh and updates the kept graph's parameters
    struct GraphSlot {
        int key[4];
        cudaGraphExec_t exec;
    } graphs[6];
    int graph_next;  // slot the next new shape replaces
};

namespace lq {

// workspace slots: conversions 0-2; solver vectors 3-7 (inner CG), 8-12 (FP64
// residuals), 13-15 (defect-correction vectors), 16-17 (block CG), 20-23 (FP32
// middle level of the three-precision solve); 18 lq_dot partials; 19 solver scalars
enum { WS_IN = 0, WS_OUT = 1, WS_TMP = 2, WS_CG0 = 3, WS_DOT = 18, WS_CTL = 19, WS_MOB = 24 /* 24, 25 */ };

inline int status_of(cudaError_t e) { return e == cudaSuccess ? LQ_OK : LQ_ERR_CUDA; }

// An executable graph for `graph`, the capture of a solver shape `key`: the
// handle's kept graph of that shape with its parameters updated from `graph`
// (cudaGraphExecUpdate), or a new instantiation stored in a slot.  The handle
// owns the result; the caller still destroys `graph`.
int cached_graph_exec(lq_handle* h, const int key[4], cudaGraph_t graph, cudaGraphExec_t* exec);

// Make sure workspace k holds at least `bytes`; returns LQ_OK / LQ_ERR_NOMEM.
int ensure_ws(lq_handle* h, int k, size_t bytes, void** out);

// Native links of a precision (packed from the saved gauge copy on first use).
int get_links(lq_handle* h, int prec, const char** links, size_t* link_block, cudaStream_t st);

// Links of this precision stored as 2 rows?  FP64 hops are bound by FP64
// arithmetic, so FP64 always keeps all 3 rows (rebuilding row 3 costs FMAs).
inline bool link_r12(const lq_handle* h, int prec) { return h->p.compress12 != 0 && prec != LQ_F64; }

// Bytes of one native parity block of one field.
inline size_t native_block_bytes(const lq_handle* h, int prec) {
    return (size_t)spinor_site_bytes(prec) * (size_t)h->g.Vh;
}

// Native-layout hop/operator launches used by the apply calls and the solvers.
// All fields are native, of precision prec.  nrhs fields back to back.
int native_wilson_full(lq_handle* h, int prec, char* out, const char* in, int nrhs, bool dag, cudaStream_t st);
int native_wilson_block(lq_handle* h, int prec, char* out, const char* in, int out_parity, int nrhs, bool dag,
                        double c_hop, cudaStream_t st);
int native_wilson_schur(lq_handle* h, int prec, char* out, const char* in, char* tmp, int nrhs, bool dag,
                        cudaStream_t st);
int native_dwf(lq_handle* h, int prec, char* out, const char* in, bool dag, cudaStream_t st);
// Even-odd domain wall (FP64/FP32).  Half fields: Ls even (or odd) blocks
// back to back; full fields: Ls slices of two blocks.  tmp holds Ls blocks.
int native_dwf_schur(lq_handle* h, int prec, char* out_e, const char* in_e, char* tmp, bool dag, cudaStream_t st);
int native_dwf_prepare(lq_handle* h, int prec, char* bhat_e, const char* eta, char* tmp, cudaStream_t st);
int native_dwf_reconstruct(lq_handle* h, int prec, char* psi, const char* x_e, const char* eta, cudaStream_t st);

// Launch descriptors of the Wilson operator pieces (links packed on demand).
int prep_wilson_full(lq_handle* h, int prec, char* out, const char* in, int nrhs, HopArgs* a, cudaStream_t st);
int prep_wilson_block(lq_handle* h, int prec, char* out, const char* in, int out_parity, int nrhs, double c_hop,
                      HopArgs* a, cudaStream_t st);
int prep_wilson_schur2(lq_handle* h, int prec, char* out, const char* tmp, const char* in, int nrhs, HopArgs* a,
                       cudaStream_t st);

// ---------------------------------------------------------- argument checks

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

inline bool valid_fmt(int fmt) {
    const int prec = fmt & 0xF;
    const bool native = (fmt & LQ_NATIVE) != 0;
    if ((fmt & ~(0xF | LQ_NATIVE)) != 0) return false;
    if (prec < LQ_F64 || prec > LQ_BF16) return false;
    if (!native && prec > LQ_F32) return false;
    return true;
}

inline size_t field_bytes(const lq_handle* h, int fmt, int subset, int nrhs) {
    const int prec = fmt & 0xF;
    const bool native = (fmt & LQ_NATIVE) != 0;
    const size_t sites = (subset == LQ_FULL ? 2 : 1) * (size_t)h->g.Vh;
    if (native) return sites * (size_t)spinor_site_bytes(prec) * nrhs;
    return sites * 24 * (prec == LQ_F64 ? 8 : 4) * nrhs;
}

// Can kernels on the current device dereference p?  Device and managed memory,
// and pinned host memory mapped into the unified address space, can; other
// host memory only where the device reads pageable memory (coherent host link).
inline bool device_accessible(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return true;
    if (at.type == cudaMemoryTypeHost) return at.devicePointer == p;
    int dev = 0, pageable = 0;
    return cudaGetDevice(&dev) == cudaSuccess &&
           cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess && pageable;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace lq
