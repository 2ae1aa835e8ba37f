// Blocked QR with column pivoting, lazy updates (Quintana-Orti, Sun and
// Bischof; the scheme of LAPACK's xGEQP3/xLAQPS), as a GPU comparator for
// QRDM.  The paper measures QRDM against xGEQP3 (Sec. 5); this is the same
// algorithm written for GB300, not a library call.
//
// Per block of nb columns (F is n x nb):
//   for each column k = k0 + j of the block:
//     p = argmax_{i >= k} vn1_i (ties to the lowest position); swap k <-> p
//     lazy update of the pivot column only: a_k -= A[:, k0:k] F[k, 0:j]^T
//     Householder reflector v_k, htau_k of a_k (rows k..m-1)
//     F[:, j] = htau_k A^T v_k - htau_k F[:, 0:j] (A[:, k0:k]^T v_k)
//     pivot row: A[k, k+1:] -= A[k, k0:k+1] F[k+1:, 0:j+1]^T
//     downdate vn1 from the updated row; a column whose downdate cancels
//     (t (vn1/vn2)^2 <= sqrt(eps)) ends the block after this column
//   trailing update A[kend:, kend:] -= V F[kend:, :]^T, then the marked
//   columns' norms are recomputed exactly.
// One cooperative persistent kernel: every CTA computes the argmax and the
// reflector scalars redundantly; rows are split over all threads for the
// pivot column, columns over warps for the F column, the row update, the
// downdate and the trailing update.  Two bounded grid barriers per column.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/qrdm.h"

namespace qrdm {
void set_last_cuda_error(int e);
namespace {

constexpr int QT = 256;            // threads per CTA
constexpr int QW = QT / 32;
constexpr int QP3_NB_MAX = 32;     // block size cap (one lane per block column)
constexpr int QV_ROWS = 128;       // rows of V staged per pass of the trailing update
constexpr double QEPS = 2.220446049250313080847e-16;
constexpr long long QSPIN_NS = 2000000000LL;  // global-timer nanoseconds before a barrier wait gives up (2 s)

struct alignas(128) Qp3State {
  unsigned int gbar;
  int32_t abort_flag;
  int32_t diag_code;
  int32_t diag_cta;
  int64_t diag_k;
  int64_t rank, rank_colmax;
  double anorm;
  int32_t nonfinite;
  int32_t stop;     // 1 + index of the last block in which a norm must be recomputed (never reset)
  int64_t ksteps;   // columns factored
  int64_t blocks;
};

struct Qp3Params {
  double* A;
  int64_t m, n, lda, kmin;
  int32_t nb;
  double eps1;
  double* htau;
  int32_t* perm;
  Qp3State* st;
  double* vn1;   // [n] partial norms
  double* vn2;   // [n] norms at the last exact computation
  double* F;     // [nb][n]
  double* part;  // [grid][nb + 2] partial sums of the pivot column
  int32_t* mark; // [n] recompute marks
};

__device__ __forceinline__ bool qbetter(double va, int64_t pa, double vb, int64_t pb) {
  return va > vb || (va == vb && pa < pb);
}

__device__ bool qbarrier(Qp3State* st, unsigned int target, int64_t k) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* ctr = &st->gbar;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    unsigned int cur = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(ctr) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (*(volatile int32_t*)&st->abort_flag) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if ((long long)(t - t0) > QSPIN_NS) {
        if (atomicExch(&st->abort_flag, 1) == 0) {
          st->diag_code = 1;
          st->diag_cta = (int)blockIdx.x;
          st->diag_k = k;
        }
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
  return *(volatile int32_t*)&st->abort_flag == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_qp3_state_init(Qp3Params P) {
  Qp3State* st = P.st;
  st->gbar = 0u;
  st->abort_flag = 0;
  st->diag_code = 0;
  st->diag_cta = -1;
  st->diag_k = -1;
  st->rank = -1;
  st->rank_colmax = -1;
  st->anorm = 0.0;
  st->nonfinite = 0;
  st->stop = 0;
  st->ksteps = 0;
  st->blocks = 0;
}

__global__ void __launch_bounds__(QT) k_qp3(Qp3Params P) {
  Qp3State* st = P.st;
  __shared__ double s_red[QW][QP3_NB_MAX + 2];
  __shared__ double s_fp[QP3_NB_MAX];   // F row of the pivot column
  __shared__ double s_y[QP3_NB_MAX];    // y_c = v_c^T v_k (c < j)
  __shared__ double s_vk[QP3_NB_MAX];   // A[k, k0 + c] (c < j), the block reflectors at row k
  __shared__ double s_sc[6];
  __shared__ int64_t s_pos[QW];
  __shared__ double s_val[QW];
  __shared__ double s_f[QW][QP3_NB_MAX];  // F row of each warp's column (trailing update)
  extern __shared__ double s_v[];       // QV_ROWS x nb staged V for the trailing update
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int G = gridDim.x, cta = blockIdx.x;
  const int64_t m = P.m, n = P.n, lda = P.lda, kmin = P.kmin;
  double* A = P.A;
  const int64_t gthreads = (int64_t)G * QT, gtid = (int64_t)cta * QT + tid;
  const int64_t gwarps = (int64_t)G * QW, gwarp = (int64_t)cta * QW + wp;
  unsigned int bar = 0;
  const double sqeps = sqrt(QEPS);

  // ---- initial norms (columns over warps), identity permutation
  double amax = 0.0;
  int bad = 0;
  for (int64_t j = gwarp; j < n; j += gwarps) {
    const double* a = A + j * lda;
    double s = 0.0;
    for (int64_t i = lane; i < m; i += 32) s = fma(a[i], a[i], s);
    s = warp_sum(s);
    const double nr = sqrt(s);
    if (lane == 0) {
      P.vn1[j] = nr;
      P.vn2[j] = nr;
      P.mark[j] = 0;
      P.perm[j] = (int32_t)j;
    }
    if (!isfinite(nr)) bad = 1;
    amax = fmax(amax, nr);
  }
  for (int64_t i = gtid; i < kmin; i += gthreads) P.htau[i] = 0.0;
  if (lane == 0) {
    if (bad) atomicExch(&st->nonfinite, 1);
    // norms are non-negative: their bit patterns order like the values
    atomicMax((unsigned long long*)&st->anorm, (unsigned long long)__double_as_longlong(amax));
  }
  bar += G;
  if (!qbarrier(st, bar, -1)) return;
  if (*(volatile int32_t*)&st->nonfinite) return;
  const double anorm = *(volatile double*)&st->anorm;

  int64_t k = 0;
  int32_t blk = 0;
  while (k < kmin) {
    ++blk;
    const int64_t k0 = k;
    const int kbmax = (int)min((int64_t)P.nb, kmin - k0);
    int j = 0;
    bool stop = false;
    for (; j < kbmax && !stop; ++j) {
      k = k0 + j;
      // ---- argmax of vn1 over [k, n), every CTA (same data, same result)
      double bv = -1.0;
      int64_t bp = INT64_MAX;
      for (int64_t i = k + tid; i < n; i += QT) {
        const double x = P.vn1[i];
        if (qbetter(x, i, bv, bp)) {
          bv = x;
          bp = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (qbetter(ov, op, bv, bp)) {
          bv = ov;
          bp = op;
        }
      }
      if (lane == 0) {
        s_val[wp] = bv;
        s_pos[wp] = bp;
      }
      __syncthreads();
      if (tid == 0) {
        for (int q = 1; q < QW; ++q)
          if (qbetter(s_val[q], s_pos[q], s_val[0], s_pos[0])) {
            s_val[0] = s_val[q];
            s_pos[0] = s_pos[q];
          }
      }
      __syncthreads();
      const double mu = s_val[0];
      const int64_t p = s_pos[0];
      if (cta == 0 && tid == 0) {
        // the stopping criterion of Sec. 3.4 (recorded; column pivoting goes on)
        if (st->rank_colmax < 0 && mu <= P.eps1 * anorm) st->rank_colmax = k;
        if (st->rank < 0 && sqrt((double)(n - k)) * mu <= P.eps1 * anorm) st->rank = k;
        if (p != k) {
          const int32_t t = P.perm[k];
          P.perm[k] = P.perm[p];
          P.perm[p] = t;
        }
      }
      if (tid < j) {
        s_fp[tid] = P.F[(int64_t)tid * n + p];
        s_vk[tid] = 0.0;
      }
      __syncthreads();
      // ---- rows over all threads: finish the previous column (scale its
      // reflector, store beta), swap k <-> p, lazy update of the pivot column,
      // partial sums of |x|^2 (rows > k) and A[r, k0+c] x_r (c < j, rows > k)
      double ps[QP3_NB_MAX + 1];
#pragma unroll
      for (int c = 0; c <= QP3_NB_MAX; ++c) ps[c] = 0.0;
      for (int64_t r = gtid; r < m; r += gthreads) {
        if (j > 0) {
          const int64_t kp = k - 1;
          if (r > kp && s_sc[3] != 0.0) A[kp * lda + r] *= s_sc[2];
          if (r == kp) A[kp * lda + r] = s_sc[0];
        }
        if (p != k) {
          const double t = A[k * lda + r];
          A[k * lda + r] = A[p * lda + r];
          A[p * lda + r] = t;
        }
        if (r >= k) {
          double x = A[k * lda + r];
          for (int c = 0; c < j; ++c) x = fma(-A[(k0 + c) * lda + r], s_fp[c], x);
          A[k * lda + r] = x;
          if (r > k) {
            ps[0] = fma(x, x, ps[0]);
            for (int c = 0; c < j; ++c) ps[1 + c] = fma(A[(k0 + c) * lda + r], x, ps[1 + c]);
          }
        }
      }
      // only warps holding rows in (k, m) have non-zero partial sums
      const int64_t w0 = gtid - lane;  // first row of this warp (one row per thread when m <= grid threads)
      bool live = false;
      for (int64_t rb = w0; rb < m; rb += gthreads) live |= (rb + 31 > k);
      if (live) {
        for (int c = 0; c <= j; ++c) {
          const double v = warp_sum(ps[c]);
          if (lane == 0) s_red[wp][c] = v;
        }
      } else if (lane <= j) {
        s_red[wp][lane] = 0.0;
      }
      __syncthreads();
      if (tid <= j) {
        double s = 0.0;
        for (int q = 0; q < QW; ++q) s += s_red[q][tid];
        P.part[(int64_t)cta * (QP3_NB_MAX + 2) + tid] = s;
      }
      bar += G;
      if (!qbarrier(st, bar, k)) return;
      // ---- reflector scalars, every CTA (partials summed in CTA order)
      if (tid <= j) {
        double s = 0.0;
        for (int q = 0; q < G; ++q) s += P.part[(int64_t)q * (QP3_NB_MAX + 2) + tid];
        if (tid == 0)
          s_sc[5] = s;
        else
          s_y[tid - 1] = s;
      }
      if (tid < j) s_vk[tid] = A[(k0 + tid) * lda + k];
      __syncthreads();
      if (tid == 0) {
        const double alpha = A[k * lda + k], s2 = s_sc[5];
        if (s2 == 0.0) {
          s_sc[0] = alpha;  // beta
          s_sc[1] = 0.0;    // htau
          s_sc[2] = 0.0;    // 1 / (alpha - beta)
        } else {
          const double nrm = sqrt(alpha * alpha + s2);
          const double beta = (alpha >= 0.0) ? -nrm : nrm;
          s_sc[0] = beta;
          s_sc[1] = (beta - alpha) / beta;
          s_sc[2] = 1.0 / (alpha - beta);
        }
        s_sc[3] = (s2 == 0.0) ? 0.0 : 1.0;
      }
      __syncthreads();
      const double ht = s_sc[1], rden = s_sc[2];
      if (cta == 0 && tid == 0) P.htau[k] = ht;
      // y_c = v_c^T v_k = A[k, k0+c] + rden sum_{r>k} A[r, k0+c] x_r
      if (tid < j) s_y[tid] = s_vk[tid] + rden * s_y[tid];
      __syncthreads();
      // ---- columns over warps: F column, pivot-row update, downdate
      for (int64_t i = k + 1 + gwarp; i < n; i += gwarps) {
        double* a = A + i * lda;
        if (i == p) {
          // the column that moved from k to p keeps its F row and its norms
          if (lane < j) P.F[(int64_t)lane * n + p] = P.F[(int64_t)lane * n + k];
          if (lane == 0) {
            P.vn1[p] = P.vn1[k];
            P.vn2[p] = P.vn2[k];
            P.mark[p] = P.mark[k];
          }
          __syncwarp();
        }
        double g = 0.0;
        const double* xk = A + k * lda;
        for (int64_t r = k + 1 + lane; r < m; r += 32) g = fma(a[r], xk[r], g);
        g = warp_sum(g);
        double corr = 0.0;
        const double fic = (lane < j) ? P.F[(int64_t)lane * n + i] : 0.0;
        if (lane < j) corr = fic * s_y[lane];
        corr = warp_sum(corr);
        const double aki = a[k];
        const double fij = ht * (aki + rden * g) - ht * corr;
        if (lane == 0) P.F[(int64_t)j * n + i] = fij;
        // pivot row: A[k, i] -= sum_{c<j} A[k, k0+c] F[i, c] + 1 * F[i, j]
        double ru = (lane < j) ? s_vk[lane] * fic : 0.0;
        ru = warp_sum(ru);
        const double akn = aki - ru - fij;
        if (lane == 0) {
          a[k] = akn;
          // downdate of the partial norm from the updated pivot-row entry
          const double u = P.vn1[i];
          if (u != 0.0) {
            const double x = akn / u;
            double t = 1.0 - x * x;
            if (t < 0.0) t = 0.0;
            const double ratio = u / P.vn2[i];
            if (t * ratio * ratio <= sqeps) {
              P.mark[i] = 1;
              atomicMax(&st->stop, blk);
            } else {
              P.vn1[i] = u * sqrt(t);
            }
          }
        }
      }
      bar += G;
      if (!qbarrier(st, bar, k)) return;
      stop = *(volatile int32_t*)&st->stop == blk;
    }
    // ---- block end: kb columns factored
    const int kb = j;
    const int64_t kend = k0 + kb;
    const int64_t kl = kend - 1;
    for (int64_t r = gtid; r < m; r += gthreads) {  // the last column's reflector
      if (r > kl && s_sc[3] != 0.0) A[kl * lda + r] *= s_sc[2];
      if (r == kl) A[kl * lda + r] = s_sc[0];
    }
    if (cta == 0 && tid == 0) {
      st->ksteps = kend;
      st->blocks += 1;
    }
    bar += G;
    if (!qbarrier(st, bar, kend)) return;
    // trailing update A[kend:, kend:] -= V F[kend:, 0:kb]^T, rows staged in
    // shared memory in passes, columns over warps; then exact norms of the
    // marked columns
    const int64_t mr = m - kend;
    if (kend < n && mr > 0) {
      for (int64_t rs = 0; rs < mr; rs += QV_ROWS) {
        const int rows = (int)min((int64_t)QV_ROWS, mr - rs);
        __syncthreads();
        for (int e = tid; e < rows * kb; e += QT) {
          const int rr = e % rows, c = e / rows;
          s_v[rr * (QP3_NB_MAX + 1) + c] = A[(k0 + c) * lda + kend + rs + rr];
        }
        __syncthreads();
        for (int64_t i = kend + gwarp; i < n; i += gwarps) {
          if (lane < kb) s_f[wp][lane] = P.F[(int64_t)lane * n + i];
          __syncwarp();
          const double* fr = s_f[wp];
          double* a = A + i * lda + kend + rs;
          for (int rr = lane; rr < rows; rr += 32) {
            const double* vr = s_v + rr * (QP3_NB_MAX + 1);
            double d = 0.0;
            for (int c = 0; c < kb; ++c) d = fma(vr[c], fr[c], d);
            a[rr] -= d;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    for (int64_t i = kend + gwarp; i < n; i += gwarps) {
      if (P.mark[i]) {
        const double* a = A + i * lda;
        double s = 0.0;
        for (int64_t r = kend + lane; r < m; r += 32) s = fma(a[r], a[r], s);
        s = warp_sum(s);
        if (lane == 0) {
          const double nr = sqrt(s);
          P.vn1[i] = nr;
          P.vn2[i] = nr;
          P.mark[i] = 0;
        }
      }
    }
    bar += G;
    if (!qbarrier(st, bar, kend)) return;
    k = kend;
  }
}

struct Qp3Layout {
  size_t st, vn1, vn2, F, part, mark, total;
};

size_t qup(size_t x) { return (x + 255) / 256 * 256; }

Qp3Layout qp3_layout(int64_t n, int nb, int grid) {
  Qp3Layout L;
  size_t o = 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  L.st = o;
  o = qup(o + sizeof(Qp3State));
  L.vn1 = o;
  o = qup(o + nn * sizeof(double));
  L.vn2 = o;
  o = qup(o + nn * sizeof(double));
  L.F = o;
  o = qup(o + nn * (size_t)nb * sizeof(double));
  L.part = o;
  o = qup(o + (size_t)grid * (QP3_NB_MAX + 2) * sizeof(double));
  L.mark = o;
  o = qup(o + nn * sizeof(int32_t));
  L.total = o;
  return L;
}

constexpr int QP3_GRID_MAX_PER_SM = 2;

int qp3_grid(int* grid) {
  int dev = 0, sms = 0, coop = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const size_t smem = (size_t)QV_ROWS * (QP3_NB_MAX + 1) * sizeof(double);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_qp3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_qp3, QT, smem);
  if (e != cudaSuccess) return (int)e;
  if (!coop || nb < 1) return -1;
  *grid = sms * (nb < QP3_GRID_MAX_PER_SM ? nb : QP3_GRID_MAX_PER_SM);
  return 0;
}

}  // namespace
}  // namespace qrdm

using namespace qrdm;

extern "C" {

int qrdm_qp3_workspace_size(int64_t m, int64_t n, int32_t nb, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > INT32_MAX) return -2;
  if (nb < 1 || nb > QP3_NB_MAX) return -3;
  if (!bytes) return -4;
  int grid = 0;
  const int e = qp3_grid(&grid);
  if (e > 0) {
    set_last_cuda_error(e);
    return QRDM_ERR_CUDA;
  }
  if (e < 0) return QRDM_ERR_UNSUPPORTED;
  *bytes = qp3_layout(n, nb, grid).total;
  return 0;
}

int qrdm_qp3_factor(double* dA, int64_t m, int64_t n, int64_t lda, int32_t nb, double* d_htau, int32_t* d_perm,
                    qrdm_info* info, int32_t eps1_mode, void* d_work, size_t work_bytes, void* stream) {
  if (m < 0) return -1;
  if (n < 0 || n > INT32_MAX) return -2;
  if (!dA && m > 0 && n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (nb < 1 || nb > QP3_NB_MAX) return -5;
  const int64_t kmin = m < n ? m : n;
  if (!d_htau && kmin > 0) return -6;
  if (!d_perm && n > 0) return -7;
  if (!info) return -8;
  if (eps1_mode != 0 && eps1_mode != 1) return -9;
  memset(info, 0, sizeof(*info));
  cudaStream_t s = (cudaStream_t)stream;
  if (kmin == 0) {
    if (n > 0) {
      int32_t* h = new int32_t[(size_t)n];
      for (int64_t j = 0; j < n; ++j) h[j] = (int32_t)j;
      cudaError_t e = cudaMemcpyAsync(d_perm, h, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      delete[] h;
      if (e != cudaSuccess) {
        set_last_cuda_error((int)e);
        return QRDM_ERR_CUDA;
      }
    }
    return 0;
  }
  int grid = 0;
  const int ge = qp3_grid(&grid);
  if (ge > 0) {
    set_last_cuda_error(ge);
    info->cuda_error = ge;
    return QRDM_ERR_CUDA;
  }
  if (ge < 0) return QRDM_ERR_UNSUPPORTED;
  const Qp3Layout L = qp3_layout(n, nb, grid);
  if (!d_work) return -10;
  if (work_bytes < L.total || ((uintptr_t)d_work % 256) != 0) return QRDM_ERR_WORKSPACE;
  char* w = (char*)d_work;
  Qp3Params P;
  memset(&P, 0, sizeof(P));
  P.A = dA;
  P.m = m;
  P.n = n;
  P.lda = lda;
  P.kmin = kmin;
  P.nb = nb;
  P.eps1 = (eps1_mode == 1) ? QEPS * sqrt((double)n) : QEPS * (double)n;
  P.htau = d_htau;
  P.perm = d_perm;
  P.st = (Qp3State*)(w + L.st);
  P.vn1 = (double*)(w + L.vn1);
  P.vn2 = (double*)(w + L.vn2);
  P.F = (double*)(w + L.F);
  P.part = (double*)(w + L.part);
  P.mark = (int32_t*)(w + L.mark);
  k_qp3_state_init<<<1, 1, 0, s>>>(P);
  cudaError_t e = cudaGetLastError();
  const size_t smem = (size_t)QV_ROWS * (QP3_NB_MAX + 1) * sizeof(double);
  void* args[] = {(void*)&P};
  if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((void*)k_qp3, dim3(grid), dim3(QT), args, smem, s);
  Qp3State hs;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, P.st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    info->cuda_error = (int32_t)e;
    return QRDM_ERR_CUDA;
  }
  if (hs.nonfinite) return QRDM_ERR_NONFINITE;
  if (hs.abort_flag) {
    info->fail_code = hs.diag_code;
    info->fail_cta = hs.diag_cta;
    info->fail_step = hs.diag_k;
    info->fail_ns = hs.diag_k;
    return hs.diag_code == 1 ? QRDM_ERR_TIMEOUT : QRDM_ERR_INTERNAL;
  }
  info->rank = hs.rank >= 0 ? hs.rank : kmin;
  info->rank_colmax = hs.rank_colmax >= 0 ? hs.rank_colmax : kmin;
  info->nsteps = hs.blocks;
  info->launches = 2;
  return 0;
}

}  // extern "C"
