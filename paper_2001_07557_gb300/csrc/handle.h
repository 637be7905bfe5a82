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
    } ws[8];          // workspace buffers, grown on demand
    int hop_block[4]; // threads per block of the hop kernels, per precision
};

namespace lq {

enum { WS_IN = 0, WS_OUT = 1, WS_TMP = 2, WS_CG0 = 3 };

inline int status_of(cudaError_t e) { return e == cudaSuccess ? LQ_OK : LQ_ERR_CUDA; }

// Make sure workspace k holds at least `bytes`; returns LQ_OK / LQ_ERR_NOMEM.
int ensure_ws(lq_handle* h, int k, size_t bytes, void** out);

// Native links of a precision (packed from the saved gauge copy on first use).
int get_links(lq_handle* h, int prec, const char** links, size_t* link_block, cudaStream_t st);

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

}  // namespace lq
