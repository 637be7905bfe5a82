// blockcg.cu -- block conjugate gradient (O'Leary 1980) for N right-hand
// sides that share one operator A = K^dag K.
//
//   R = B - A X,  P = R
//   repeat:  Q = A P                      (one multi-RHS operator launch set)
//            Delta = P^dag Q,  rho = R^dag R          (N x N, FP64 sums)
//            alpha = Delta^{-1} rho
//            X += P alpha,  R -= Q alpha
//            beta = rho^{-1} (R^dag R)_new,  P = R + P beta
//
// The block vectors live in FP32 storage (FP32 arithmetic); the N x N Gram
// matrices are summed in FP64 on the device (per-thread FP64 accumulators,
// per-block partials, a fixed-order second pass) and the N x N algebra
// (Cholesky solves) runs in FP64 on the host.  As a mixed-precision solver
// the block CG is the inner solve of the FP64 defect-correction loop in
// cg.cu: it stops when every column's residual has dropped by the inner
// tolerance, or when Delta stops being numerically positive definite (the
// block has lost rank), and the FP64 outer loop restarts from the true
// residual.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "blas.h"
#include "blockcg.h"

namespace lq {

namespace {

constexpr int kGT = 128;  // threads per block of the block kernels

// G[i][j] partials: sum over the block's sites of <A_i(x), B_j(x)>.
// grid = (site blocks, N); thread = (site, i); the N B-spinors of a site are
// re-read from L1 by the N threads that share the site.
template <int P>
__global__ void __launch_bounds__(kGT) gram_partial_kernel(const char* A, const char* B, size_t stride, long nsites,
                                                           int Vh, int N, double2* partial) {
    const int i = blockIdx.y;
    double2 acc[kMaxBlockRhs];
#pragma unroll
    for (int j = 0; j < kMaxBlockRhs; ++j) acc[j] = make_double2(0.0, 0.0);
    for (long s = (long)blockIdx.x * kGT + threadIdx.x; s < nsites; s += (long)gridDim.x * kGT) {
        const int bk = (int)(s / Vh), x = (int)(s - (long)bk * Vh);
        const size_t blk = (size_t)bk * spinor_site_bytes(P) * Vh;
        cplx<float> a[12];
        load_spinor<P, float>(A + (size_t)i * stride + blk, Vh, x, a);
#pragma unroll
        for (int j = 0; j < kMaxBlockRhs; ++j) {
            if (j < N) {
                cplx<float> b[12];
                load_spinor<P, float>(B + (size_t)j * stride + blk, Vh, x, b);
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    re = fmaf(a[k].re, b[k].re, re);
                    re = fmaf(a[k].im, b[k].im, re);
                    im = fmaf(a[k].re, b[k].im, im);
                    im = fmaf(-a[k].im, b[k].re, im);
                }
                acc[j].x += re;
                acc[j].y += im;
            }
        }
    }
    // block reduction of the N accumulators: warps, then shared memory
    __shared__ double2 red[kGT / 32][kMaxBlockRhs];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxBlockRhs; ++j) {
        if (j < N) {
            double x = acc[j].x, y = acc[j].y;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                y += __shfl_xor_sync(0xffffffffu, y, o);
            }
            if (lane == 0) red[w][j] = make_double2(x, y);
        }
    }
    __syncthreads();
    if (threadIdx.x < N) {
        const int j = threadIdx.x;
        double2 t = make_double2(0.0, 0.0);
        for (int q = 0; q < kGT / 32; ++q) {
            t.x += red[q][j].x;
            t.y += red[q][j].y;
        }
        partial[((size_t)blockIdx.x * N + i) * N + j] = t;
    }
}

// G = sum over blocks of the partials (fixed order); one thread per entry.
__global__ void gram_final_kernel(const double2* partial, int nblk, int N, double2* G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * N) return;
    double2 t = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) {
        const double2 v = partial[(size_t)b * N * N + e];
        t.x += v.x;
        t.y += v.y;
    }
    G[e] = t;
}

// Y_j = cy * Y_j + sum_k M[k][j] X_k  and, if X2/Y2 are given, Y2_j = Y2_j + sum_k M2[k][j] X2_k
// with the same matrix (M2 = -M handled by sign2).  thread = (site, j).
template <int P>
__global__ void __launch_bounds__(kGT) block_axpy_kernel(char* Y, const char* X, float cy, char* Y2, const char* X2,
                                                         float sign2, const float2* M, size_t stride, long nsites,
                                                         int Vh, int N) {
    const int j = blockIdx.y;
    __shared__ float2 m[kMaxBlockRhs];
    if (threadIdx.x < N) m[threadIdx.x] = M[threadIdx.x * N + j];
    __syncthreads();
    for (long s = (long)blockIdx.x * kGT + threadIdx.x; s < nsites; s += (long)gridDim.x * kGT) {
        const int bk = (int)(s / Vh), x = (int)(s - (long)bk * Vh);
        const size_t blk = (size_t)bk * spinor_site_bytes(P) * Vh;
        cplx<float> y[12], y2[12];
        if (cy != 0.f) {
            load_spinor<P, float>(Y + (size_t)j * stride + blk, Vh, x, y);
#pragma unroll
            for (int c = 0; c < 12; ++c) y[c] = {cy * y[c].re, cy * y[c].im};
        } else {
#pragma unroll
            for (int c = 0; c < 12; ++c) y[c] = {0.f, 0.f};
        }
        if (Y2) load_spinor<P, float>(Y2 + (size_t)j * stride + blk, Vh, x, y2);
        for (int k = 0; k < N; ++k) {
            const float2 mk = m[k];
            cplx<float> v[12];
            load_spinor<P, float>(X + (size_t)k * stride + blk, Vh, x, v);
#pragma unroll
            for (int c = 0; c < 12; ++c) cmac(y[c], cplx<float>{mk.x, mk.y}, v[c]);
            if (Y2) {
                load_spinor<P, float>(X2 + (size_t)k * stride + blk, Vh, x, v);
                const cplx<float> m2 = {sign2 * mk.x, sign2 * mk.y};
#pragma unroll
                for (int c = 0; c < 12; ++c) cmac(y2[c], m2, v[c]);
            }
        }
        store_spinor<P, float>(Y + (size_t)j * stride + blk, Vh, x, y);
        if (Y2) store_spinor<P, float>(Y2 + (size_t)j * stride + blk, Vh, x, y2);
    }
}

int block_grid(long nsites) {
    const long want = (nsites + kGT - 1) / kGT;
    return (int)std::min<long>(want, 152L * 4);
}

using cd = std::complex<double>;

// Solve H Z = Y for Hermitian positive definite H (N x N, row-major) by
// Cholesky; Y and Z are N x N.  Returns false if H is not numerically
// positive definite (pivot <= eps * largest diagonal).
bool chol_solve(const std::vector<cd>& H, const std::vector<cd>& Y, std::vector<cd>& Z, int N) {
    std::vector<cd> L(N * N, 0.0);
    double dmax = 0;
    for (int i = 0; i < N; ++i) dmax = std::max(dmax, H[i * N + i].real());
    for (int j = 0; j < N; ++j) {
        double d = H[j * N + j].real();
        for (int k = 0; k < j; ++k) d -= std::norm(L[j * N + k]);
        if (!(d > 1e-13 * dmax)) return false;
        const double ljj = std::sqrt(d);
        L[j * N + j] = ljj;
        for (int i = j + 1; i < N; ++i) {
            cd s = H[i * N + j];
            for (int k = 0; k < j; ++k) s -= L[i * N + k] * std::conj(L[j * N + k]);
            L[i * N + j] = s / ljj;
        }
    }
    Z = Y;
    for (int c = 0; c < N; ++c) {  // forward: L w = y ; back: L^dag z = w
        for (int i = 0; i < N; ++i) {
            cd s = Z[i * N + c];
            for (int k = 0; k < i; ++k) s -= L[i * N + k] * Z[k * N + c];
            Z[i * N + c] = s / L[i * N + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            cd s = Z[i * N + c];
            for (int k = i + 1; k < N; ++k) s -= std::conj(L[k * N + i]) * Z[k * N + c];
            Z[i * N + c] = s / L[i * N + i];
        }
    }
    return true;
}

}  // namespace

int block_cg(const BlockCgOps& ops, char* X, const char* Bv, char* R, char* Pa, char* Pb, char* Q, size_t stride,
             long nsites, int Vh, int N, double tol, int maxiter, void* ws, double2* hostbuf, cudaStream_t s,
             int* iters) {
    if (N < 1 || N > kMaxBlockRhs) return LQ_ERR_ARG;
    const int nblk = block_grid(nsites);
    double2* partial = static_cast<double2*>(ws);
    double2* Gd = partial + (size_t)nblk * N * N;
    float2* Md = reinterpret_cast<float2*>(Gd + N * N);
    auto gram = [&](const char* A, const char* Bm, std::vector<cd>& G) -> int {
        dim3 grid(nblk, N);
        gram_partial_kernel<LQ_F32><<<grid, kGT, 0, s>>>(A, Bm, stride, nsites, Vh, N, partial);
        gram_final_kernel<<<(N * N + 127) / 128, 128, 0, s>>>(partial, nblk, N, Gd);
        if (cudaMemcpyAsync(hostbuf, Gd, sizeof(double2) * N * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LQ_ERR_CUDA;
        G.resize(N * N);
        for (int e = 0; e < N * N; ++e) G[e] = cd(hostbuf[e].x, hostbuf[e].y);
        return LQ_OK;
    };
    auto upload = [&](const std::vector<cd>& M) -> int {
        float2* hf = reinterpret_cast<float2*>(hostbuf);
        for (int e = 0; e < N * N; ++e) hf[e] = make_float2((float)M[e].real(), (float)M[e].imag());
        return cudaMemcpyAsync(Md, hf, sizeof(float2) * N * N, cudaMemcpyHostToDevice, s) == cudaSuccess
                   ? LQ_OK : LQ_ERR_CUDA;
    };
    auto axpy = [&](char* Y, const char* Xv, float cy, char* Y2, const char* X2, float sign2) -> int {
        dim3 grid(nblk, N);
        block_axpy_kernel<LQ_F32><<<grid, kGT, 0, s>>>(Y, Xv, cy, Y2, X2, sign2, Md, stride, nsites, Vh, N);
        return cudaGetLastError() == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
    };

    // X = 0, R = B, P = R
    if (cudaMemsetAsync(X, 0, stride * N, s) != cudaSuccess ||
        cudaMemcpyAsync(R, Bv, stride * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(Pa, Bv, stride * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LQ_ERR_CUDA;
    std::vector<cd> rho, rho0, delta, alpha, beta, rhonew;
    int rc = gram(R, R, rho);
    if (rc) return rc;
    rho0 = rho;
    char* P = Pa;
    char* Pn = Pb;
    int it = 0;
    for (; it < maxiter; ++it) {
        bool done = true;
        for (int j = 0; j < N; ++j) done = done && rho[j * N + j].real() <= tol * tol * rho0[j * N + j].real();
        if (done) break;
        if ((rc = ops.apply(ops.ctx, Q, P))) return rc;
        if ((rc = gram(P, Q, delta))) return rc;
        if (!chol_solve(delta, rho, alpha, N)) break;  // block lost rank: hand back to the outer loop
        if ((rc = upload(alpha))) return rc;
        // X += P alpha ; R -= Q alpha
        if ((rc = axpy(X, P, 1.f, R, Q, -1.f))) return rc;
        if ((rc = gram(R, R, rhonew))) return rc;
        if (!chol_solve(rho, rhonew, beta, N)) {
            ++it;
            break;
        }
        if ((rc = upload(beta))) return rc;
        // Pn = R + P beta  (R enters with coefficient 1 through the identity trick below)
        if (cudaMemcpyAsync(Pn, R, stride * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return LQ_ERR_CUDA;
        if ((rc = axpy(Pn, P, 1.f, nullptr, nullptr, 0.f))) return rc;
        std::swap(P, Pn);
        rho = rhonew;
    }
    *iters = it;
    return cudaGetLastError() == cudaSuccess ? LQ_OK : LQ_ERR_CUDA;
}

}  // namespace lq
