// Least squares with a QRDM factorization, and FP64 iterative refinement.
//
// Given A Pi = Q R from qrdm_factor (reflectors below the diagonal, htau,
// permutation) and a rank r, the basic solution of min ||A x - b|| is
//   x = Pi [R11^{-1} (Q^T b)_{1:r}; 0]
// (Q^T b by the stored reflectors H_1..H_r, R11 the leading r x r block).
// Refinement (for a factorization computed in reduced precision): with the
// original FP64 matrix, r_k = b - A x_k in FP64, x_{k+1} = x_k + basic(r_k).
// The paper stops at the factorization; the solve is this library's.
//
// Kernels: one CTA per right-hand side column keeps that column in shared
// memory for the reflector sweep and the back substitution (rows m <= 24576);
// the FP64 residual is a column-oriented GEMV over row tiles.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/qrdm.h"

namespace qrdm {
void set_last_cuda_error(int e);
namespace {

constexpr int LS_THREADS = 512;
constexpr int LS_MAX_ROWS = 24576;  // a column of B in shared memory (192 KB)

__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += red[q];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// y := Q^T b for column c (Q = H_0 ... H_{k-1}, H_j = I - htau_j v_j v_j^T,
// v_j(j) = 1, v_j(i) = QR(i, j) for i > j), then the back substitution
// R11 z = y_{0:r}, written to Z (r x nrhs).
__global__ void __launch_bounds__(LS_THREADS) k_ls_basic(const double* __restrict__ QR, int64_t m, int64_t ldq,
                                                          const double* __restrict__ htau, int64_t r,
                                                          const double* __restrict__ B, int64_t ldb,
                                                          double* __restrict__ Z, int64_t ldz) {
  extern __shared__ double s_y[];  // m
  __shared__ double s_red[33];
  const int64_t c = blockIdx.x;
  const double* b = B + c * ldb;
  for (int64_t i = threadIdx.x; i < m; i += LS_THREADS) s_y[i] = b[i];
  __syncthreads();
  for (int64_t j = 0; j < r; ++j) {
    const double ht = htau[j];
    if (ht == 0.0) continue;  // uniform
    const double* v = QR + j * ldq;
    double d = 0.0;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += LS_THREADS) d = fma(v[i], s_y[i], d);
    d = block_sum(d, s_red) + s_y[j];
    const double w = ht * d;
    if (threadIdx.x == 0) s_y[j] -= w;
    for (int64_t i = j + 1 + threadIdx.x; i < m; i += LS_THREADS) s_y[i] = fma(-w, v[i], s_y[i]);
    __syncthreads();
  }
  // back substitution, column-oriented: z_i = y_i / R_ii, then y_{0:i} -= R_{0:i,i} z_i
  for (int64_t i = r - 1; i >= 0; --i) {
    if (threadIdx.x == 0) s_y[i] = s_y[i] / QR[i * ldq + i];
    __syncthreads();
    const double zi = s_y[i];
    const double* col = QR + i * ldq;
    for (int64_t t = threadIdx.x; t < i; t += LS_THREADS) s_y[t] = fma(-col[t], zi, s_y[t]);
    __syncthreads();
  }
  double* z = Z + c * ldz;
  for (int64_t i = threadIdx.x; i < r; i += LS_THREADS) z[i] = s_y[i];
}

// X[perm[i], c] (+)= Z[i, c] for i < r (x = Pi [z; 0]); set: zero X first
__global__ void k_ls_scatter(const int32_t* __restrict__ perm, int64_t n, int64_t r, const double* __restrict__ Z,
                             int64_t ldz, double* __restrict__ X, int64_t ldx, int64_t nrhs, int accumulate) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * nrhs) return;
  const int64_t i = e % n, c = e / n;
  const double add = (i < r) ? Z[c * ldz + i] : 0.0;
  double* x = X + c * ldx + perm[i];
  *x = accumulate ? *x + add : add;
}

// R = B - A X (FP64), rows split over CTAs; each thread owns rows and walks the
// columns of A in order (coalesced reads, a fixed summation order)
__global__ void k_ls_residual(const double* __restrict__ A, int64_t m, int64_t n, int64_t lda,
                              const double* __restrict__ X, int64_t ldx, const double* __restrict__ B, int64_t ldb,
                              double* __restrict__ Rr, int64_t ldr, int64_t nrhs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t c = blockIdx.y;
  if (i >= m || c >= nrhs) return;
  const double* x = X + c * ldx;
  double acc = 0.0;
  for (int64_t j = 0; j < n; ++j) acc = fma(A[j * lda + i], x[j], acc);
  Rr[c * ldr + i] = B[c * ldb + i] - acc;
}

// column 2-norms of an m x nrhs block into out[nrhs] (one CTA per column)
__global__ void __launch_bounds__(LS_THREADS) k_ls_colnorm(const double* __restrict__ V, int64_t m, int64_t ld,
                                                            double* __restrict__ out) {
  __shared__ double s_red[33];
  const double* v = V + (int64_t)blockIdx.x * ld;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += LS_THREADS) s = fma(v[i], v[i], s);
  s = block_sum(s, s_red);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s);
}

size_t ls_work_doubles(int64_t m, int64_t r, int64_t nrhs) { return (size_t)(m + r + 1) * (size_t)nrhs; }

}  // namespace
}  // namespace qrdm

using namespace qrdm;

extern "C" {

int qrdm_ls_workspace_size(int64_t m, int64_t n, int64_t rank, int64_t nrhs, size_t* bytes) {
  if (m < 0 || m > LS_MAX_ROWS) return -1;
  if (n < 0 || n > INT32_MAX) return -2;
  if (rank < 0 || rank > (m < n ? m : n)) return -3;
  if (nrhs < 0 || nrhs > 65535) return -4;
  if (!bytes) return -5;
  *bytes = ls_work_doubles(m, rank, nrhs) * sizeof(double);
  return 0;
}

int qrdm_ls_solve(const double* dA, int64_t lda, const double* dQR, int64_t ldqr, int64_t m, int64_t n,
                  const double* d_htau, const int32_t* d_perm, int64_t rank, const double* dB, int64_t ldb,
                  int64_t nrhs, double* dX, int64_t ldx, int32_t refine, double* h_resid, void* d_work,
                  size_t work_bytes, void* stream) {
  if (refine > 0 && !dA) return -1;
  if (refine > 0 && lda < (m > 1 ? m : 1)) return -2;
  if (!dQR && m > 0 && n > 0) return -3;
  if (ldqr < (m > 1 ? m : 1)) return -4;
  if (m < 0 || m > LS_MAX_ROWS) return -5;
  if (n < 0 || n > INT32_MAX) return -6;
  if (!d_htau && rank > 0) return -7;
  if (!d_perm && n > 0) return -8;
  if (rank < 0 || rank > (m < n ? m : n)) return -9;
  if (!dB && m > 0 && nrhs > 0) return -10;
  if (ldb < (m > 1 ? m : 1)) return -11;
  if (nrhs < 0 || nrhs > 65535) return -12;
  if (!dX && n > 0 && nrhs > 0) return -13;
  if (ldx < (n > 1 ? n : 1)) return -14;
  if (refine < 0 || refine > 100) return -15;
  if (n == 0 || nrhs == 0) return 0;
  const size_t need = ls_work_doubles(m, rank, nrhs) * sizeof(double);
  if (!d_work || work_bytes < need || ((uintptr_t)d_work % 16) != 0) return QRDM_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  double* Z = (double*)d_work;                      // rank x nrhs
  double* Rr = Z + (size_t)rank * (size_t)nrhs;     // m x nrhs residuals
  double* Nr = Rr + (size_t)m * (size_t)nrhs;       // nrhs residual norms
  const int64_t ldz = rank > 0 ? rank : 1;
  const size_t smem = (size_t)(m > 0 ? m : 1) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_ls_basic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  auto basic = [&](const double* rhs, int64_t ldr, int accumulate) -> cudaError_t {
    if (rank > 0) k_ls_basic<<<(unsigned)nrhs, LS_THREADS, smem, s>>>(dQR, m, ldqr, d_htau, rank, rhs, ldr, Z, ldz);
    const int64_t tot = n * nrhs;
    k_ls_scatter<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_perm, n, rank, Z, ldz, dX, ldx, nrhs, accumulate);
    return cudaGetLastError();
  };
  auto residual = [&](int it) -> cudaError_t {
    dim3 g((unsigned)((m + 255) / 256), (unsigned)nrhs);
    k_ls_residual<<<g, 256, 0, s>>>(dA, m, n, lda, dX, ldx, dB, ldb, Rr, m > 0 ? m : 1, nrhs);
    cudaError_t ee = cudaGetLastError();
    if (ee == cudaSuccess && h_resid) {
      k_ls_colnorm<<<(unsigned)nrhs, LS_THREADS, 0, s>>>(Rr, m, m > 0 ? m : 1, Nr);
      ee = cudaMemcpyAsync(h_resid + (size_t)it * (size_t)nrhs, Nr, sizeof(double) * (size_t)nrhs,
                           cudaMemcpyDeviceToHost, s);
      if (ee == cudaSuccess) ee = cudaStreamSynchronize(s);
    }
    return ee;
  };
  if (e == cudaSuccess) e = basic(dB, ldb, 0);
  for (int it = 0; it < refine && e == cudaSuccess; ++it) {
    e = residual(it);
    if (e == cudaSuccess) e = basic(Rr, m > 0 ? m : 1, 1);
  }
  if (e == cudaSuccess && h_resid && dA) e = residual(refine);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

}  // extern "C"
