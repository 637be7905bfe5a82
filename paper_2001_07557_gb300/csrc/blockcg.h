// blockcg.h -- block CG inner solver (FP32 block vectors, FP64 N x N algebra).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace lq {

constexpr int kMaxBlockRhs = 16;

// The operator the block CG iterates, A = K^dag K, for all N columns at once
// and in two stages on the solver's stream: apply(ctx, out, in, 0) leaves
// K in in kimage (same column layout and stride as in), apply(ctx, out, in, 1)
// writes out = K^dag kimage.  P^dag A P = (K P)^dag (K P) is formed as the
// Gram of K P with itself, which reads N columns instead of 2N and is
// Hermitian positive semidefinite by construction; it runs on a second stream
// while the second stage runs.
struct BlockCgOps {
    void* ctx;
    int (*apply)(void* ctx, char* out, const char* in, int stage);
    const char* kimage;
};

// Bytes of device scratch block_cg needs for N columns over nsites sites.
inline size_t block_cg_scratch_bytes(int N) {
    return sizeof(double2) * ((size_t)152 * 4 * N * N + (size_t)N * N) + sizeof(float2) * N * N + 256;
}

// Block CG on A X = B from X = 0 for N columns of FP32 native fields, each
// `stride` bytes (a multiple of 16) holding nsites sites.  R, P, Q are
// scratch fields of the same shape; ws: block_cg_scratch_bytes(N) device
// bytes; hostbuf: N*N pinned double2.  Stops when every column's residual is
// below tol times its start, when the block loses rank, or after maxiter.
// LQ_ERR_ARG if N is outside 1..kMaxBlockRhs, stride is not a multiple of 16
// or ops.kimage is null.
int block_cg(const BlockCgOps& ops, char* X, const char* B, char* R, char* P, char* Q, size_t stride, long nsites,
             int N, double tol, int maxiter, void* ws, double2* hostbuf, cudaStream_t s, int* iters);

}  // namespace lq
