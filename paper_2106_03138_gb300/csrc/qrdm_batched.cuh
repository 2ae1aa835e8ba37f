// Batched QRDM: many independent matrices in one persistent launch.
//
// Each CTA factors whole matrices, one at a time, taken from a work queue
// (an atomic counter over a host-chosen order, largest first).  Every phase
// of Alg. 4 runs inside the CTA with block barriers only, so no CTA ever
// waits on another and there is no cross-CTA wait to bound.  The decisions,
// the sub-panel blocking and the block reflector updates are those of the
// single-matrix path.  FP64 throughout.
//
// Tunables (picked per batch by the host autotuner): CTAs per SM, rows of V
// staged per pass (the shared-memory tile height) and lanes per column in
// the block-reflector phases (LPC, a template parameter).
#pragma once

#include "qrdm_kernels.cuh"

namespace qrdm {

constexpr int BT = 256;      // threads per CTA
constexpr int BW = BT / 32;  // warps per CTA
constexpr int G_ROWS = 64;   // rows of the gathered columns staged per Gram pass
constexpr int LDV = PB + 1;  // staged V row stride (odd: conflict-free 8-byte reads)

// dynamic shared memory of k_batched: packed Gram matrix, then one staging buffer
__host__ __device__ constexpr int64_t batched_gram_doubles(int kmax) {
  return ((int64_t)kmax * (kmax + 1) / 2 + 1) & ~1ll;
}
__host__ __device__ constexpr int64_t batched_buf_doubles(int kmax, int rows_pp) {
  return (int64_t)kmax * (G_ROWS + 1) > (int64_t)rows_pp * LDV ? (int64_t)kmax * (G_ROWS + 1)
                                                                 : (int64_t)rows_pp * LDV;
}
__host__ __device__ constexpr int64_t batched_smem_bytes(int kmax, int rows_pp) {
  return (batched_gram_doubles(kmax) + batched_buf_doubles(kmax, rows_pp)) * (int64_t)sizeof(double);
}
// per-CTA global scratch: u, uref, mark (nmax each) and W (PB x nmax)
__host__ __device__ constexpr int64_t batched_scratch_doubles(int64_t nmax) { return nmax * (3 + PB); }

struct BatchDesc {
  double* A;
  double* htau;
  int32_t* perm;
  int64_t m, n, lda;
  StepRecord* trace;  // optional step trace (nullptr: none)
  int32_t* traceJ;    // trace_cap x kmax original column indices of J
  int64_t trace_cap;
  float* feat_log;    // optional [log_cap][POL_NFEAT] policy features per step
  double* act_log;    // optional [log_cap][2] (tau_s, delta_s) per step
  int64_t log_cap;
};

struct BatchParams {
  const BatchDesc* desc;  // [count]
  const int32_t* order;   // [count] processing order (largest first)
  int64_t count;
  double tau, delta;
  int32_t kmax, eps1_mode, stop_at_rank, check_last, no_break, sdd;
  int32_t rows_pp;        // rows of V staged per pass
  int32_t pad0;
  int32_t* next;          // work counter (zeroed before the launch)
  double* scratch;        // per CTA, batched_scratch_doubles(nmax)
  int64_t nmax;
  int64_t* rank;          // [count]
  int64_t* rank_colmax;   // [count]
  int32_t* status;        // [count] 0 ok, 1 non-finite input
  int64_t* steps;         // [count]
  unsigned long long* phase_clk;  // optional: SM cycles per phase, then the sum and max of CTA active cycles
  PolicyParams pol;               // learned (tau, delta) (pol.active = 0: fixed)
};

// Non-negative doubles order like their bit patterns read as int64, so the
// argmax compares run on the integer pipe (the FP64 pipe is the scarce one).
__device__ __forceinline__ long long okey(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool kbetter(long long ka, int64_t pa, long long kb, int64_t pb) {
  return ka > kb || (ka == kb && pa < pb);
}

// argmax of u[j] over j in [lo, hi), j != skip, mark[j] == 0 (when mark) and
// u[j] >= thr (thr_key < 0: no threshold); ties to the lowest position
// (reading R15).  pos = -1 when nothing qualifies.  Uniform result.
__device__ __forceinline__ void b_argmax(const double* u, const double* mark, int64_t lo, int64_t hi,
                                         long long thr_key, int64_t skip, long long* s_k, int64_t* s_p,
                                         double* mu, int64_t* pos) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long bk = -1;
  int64_t bp = INT64_MAX;
  for (int64_t j = lo + threadIdx.x; j < hi; j += BT) {
    const long long x = okey(u[j]);
    if (j == skip || x < thr_key || (mark && mark[j] != 0.0)) continue;
    if (kbetter(x, j, bk, bp)) {
      bk = x;
      bp = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
    if (kbetter(ok, op, bk, bp)) {
      bk = ok;
      bp = op;
    }
  }
  if (lane == 0) {
    s_k[w] = bk;
    s_p[w] = bp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < BW; ++q)
      if (kbetter(s_k[q], s_p[q], s_k[0], s_p[0])) {
        s_k[0] = s_k[q];
        s_p[0] = s_p[q];
      }
  }
  __syncthreads();
  *mu = (s_k[0] < 0) ? -1.0 : __longlong_as_double(s_k[0]);
  *pos = (s_p[0] == INT64_MAX) ? -1 : s_p[0];
  __syncthreads();
}

// Block reflector of one sub-panel (lj <= NT reflectors, V below the diagonal
// of columns r0..r0+lj-1 from row r0) on columns c0..c0+n2-1, rows r0..m-1:
// A -= V (T^T (V^T A)) (Sec. 3.2, compact WY).  LPC lanes share a column;
// NT (1, 2, 4, 8 or 16) is lj rounded up, so small blocks do no padded FMAs.
template <int LPC, int NT>
__device__ __forceinline__ void b_reflect(double* A, int64_t lda, int64_t m, int64_t r0, int64_t c0, int64_t n2, int lj,
                                       int rows_pp, int64_t nmax, double* s_dyn, double (*s_T)[PB], double* Wb) {
  constexpr int CPW = 32 / LPC;  // columns per warp
  constexpr int LD = NT + 1;     // staged V row stride
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int sub = lane / LPC, lr = lane % LPC;
  const int64_t mr = m - r0;
  // W = V^T A (lj x n2), accumulated over row passes in Wb
  for (int64_t rs = 0; rs < mr; rs += rows_pp) {
    const int rows = (int)min((int64_t)rows_pp, mr - rs);
    __syncthreads();
    for (int e = tid; e < rows * NT; e += BT) {
      const int rr = e % rows, t = e / rows;
      s_dyn[rr * LD + t] = (t < lj) ? vget(A, lda, r0, rs + rr, t) : 0.0;
    }
    __syncthreads();
    for (int64_t cg0 = (int64_t)wp * CPW; cg0 < n2; cg0 += (int64_t)BW * CPW) {
      const int64_t c = cg0 + sub;
      double acc[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) acc[t] = 0.0;
      if (c < n2) {
        const double* a = A + (c0 + c) * lda + r0 + rs;
        for (int r = lr; r < rows; r += LPC) {
          const double xv = a[r];
          const double* vr = s_dyn + r * LD;
#pragma unroll
          for (int t = 0; t < NT; ++t) acc[t] = fma(vr[t], xv, acc[t]);
        }
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
      }
      if (c < n2) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          if (t % LPC == lr && t < lj) {
            double* wt = Wb + (int64_t)t * nmax + c;
            *wt = (rs == 0) ? acc[t] : *wt + acc[t];
          }
        }
      }
    }
  }
  __syncthreads();
  // W = T^T W, column by column
  if (NT > 1) {
    for (int64_t c = tid; c < n2; c += BT) {
      double wv[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) wv[t] = (t < lj) ? Wb[(int64_t)t * nmax + c] : 0.0;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (t < lj) {
          double s = 0.0;
#pragma unroll
          for (int qq = 0; qq <= t; ++qq) s = fma(s_T[qq][t], wv[qq], s);
          Wb[(int64_t)t * nmax + c] = s;
        }
      }
    }
  }
  const double t00 = s_T[0][0];  // NT == 1: T^T W is a scaling, folded into the update
  // A -= V W
  for (int64_t rs = 0; rs < mr; rs += rows_pp) {
    const int rows = (int)min((int64_t)rows_pp, mr - rs);
    __syncthreads();
    if (mr > rows_pp) {  // V of this pass (a single pass keeps the staged V)
      for (int e = tid; e < rows * NT; e += BT) {
        const int rr = e % rows, t = e / rows;
        s_dyn[rr * LD + t] = (t < lj) ? vget(A, lda, r0, rs + rr, t) : 0.0;
      }
      __syncthreads();
    }
    for (int64_t cg0 = (int64_t)wp * CPW; cg0 < n2; cg0 += (int64_t)BW * CPW) {
      const int64_t c = cg0 + sub;
      if (c >= n2) continue;
      double wv[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) wv[t] = (t < lj) ? Wb[(int64_t)t * nmax + c] : 0.0;
      if (NT == 1) wv[0] *= t00;
      double* a = A + (c0 + c) * lda + r0 + rs;
      int r = lr;
      for (; r + LPC < rows; r += 2 * LPC) {
        const double* v0 = s_dyn + r * LD;
        const double* v1 = v0 + LPC * LD;
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          d0 = fma(v0[t], wv[t], d0);
          d1 = fma(v1[t], wv[t], d1);
        }
        a[r] -= d0;
        a[r + LPC] -= d1;
      }
      if (r < rows) {
        const double* v0 = s_dyn + r * LD;
        double d0 = 0.0;
#pragma unroll
        for (int t = 0; t < NT; ++t) d0 = fma(v0[t], wv[t], d0);
        a[r] -= d0;
      }
    }
  }
  __syncthreads();
}

template <int LPC>
__device__ __noinline__ void b_reflect_any(double* A, int64_t lda, int64_t m, int64_t r0, int64_t c0, int64_t n2,
                                              int lj, int rows_pp, int64_t nmax, double* s_dyn, double (*s_T)[PB],
                                              double* Wb) {
  if (lj <= 1)
    b_reflect<LPC, 1>(A, lda, m, r0, c0, n2, lj, rows_pp, nmax, s_dyn, s_T, Wb);
  else if (lj <= 2)
    b_reflect<LPC, 2>(A, lda, m, r0, c0, n2, lj, rows_pp, nmax, s_dyn, s_T, Wb);
  else if (lj <= 4)
    b_reflect<LPC, 4>(A, lda, m, r0, c0, n2, lj, rows_pp, nmax, s_dyn, s_T, Wb);
  else if (lj <= 8)
    b_reflect<LPC, 8>(A, lda, m, r0, c0, n2, lj, rows_pp, nmax, s_dyn, s_T, Wb);
  else
    b_reflect<LPC, 16>(A, lda, m, r0, c0, n2, lj, rows_pp, nmax, s_dyn, s_T, Wb);
}

// per-phase SM clock accounting (profile runs only)
enum BatchPhase { BP_INIT = 0, BP_SELECT, BP_GRAM, BP_PICK, BP_SWAP, BP_PANEL, BP_REFLECT, BP_DOWNDATE, BP_N };

template <int LPC>
__global__ void __launch_bounds__(BT, 2) k_batched(BatchParams B) {
  extern __shared__ double s_shm[];
  double* s_g = s_shm;                                   // packed upper Gram matrix
  double* s_dyn = s_shm + batched_gram_doubles(B.kmax);  // staging: Gram rows or V rows
  __shared__ long long s_k[BW];
  __shared__ int64_t s_p[BW];
  __shared__ double s_v[BW];
  __shared__ double s_rd[KMAX];     // reciprocal column norms of the gathered columns
  __shared__ int32_t s_cols[KMAX];  // candidate positions (j* first)
  __shared__ int32_t s_J[KMAX];     // picked candidates (indices into s_cols)
  __shared__ int64_t s_sel[KMAX];   // current positions of the picked columns
  __shared__ double s_tot[2 * PB];
  __shared__ double s_T[PB][PB];
  __shared__ double s_y[PB];
  __shared__ double s_sc[8];
  __shared__ int s_i[2];
  __shared__ PolicyCarry s_pc;
  __shared__ float s_feat[POL_NFEAT];
  __shared__ int s_pcnt[8 * BW];
  __shared__ float s_h[2 * POL_HIDDEN];
  __shared__ double s_pout[2];
  __shared__ double s_minb;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  double* u = B.scratch + (int64_t)blockIdx.x * batched_scratch_doubles(B.nmax);
  double* uref = u + B.nmax;
  double* mark = uref + B.nmax;
  double* Wb = mark + B.nmax;  // [PB][nmax]
  const double sqeps = sqrt(EPS);
  // phase accounting (thread 0 at block-uniform points; profile runs only)
  __shared__ unsigned long long s_pacc[BP_N];
  if (tid < BP_N) s_pacc[tid] = 0;
  long long tclk = clock64();
  const long long tstart = tclk;
  const bool prof = (B.phase_clk != nullptr) && tid == 0;
#define QRDM_BPHASE(ph)                     \
  do {                                      \
    if (prof) {                             \
      const long long now_ = clock64();     \
      s_pacc[ph] += (unsigned long long)(now_ - tclk); \
      tclk = now_;                          \
    }                                       \
  } while (0)

  for (;;) {
    if (tid == 0) s_i[0] = atomicAdd(B.next, 1);
    __syncthreads();
    const int64_t qi = s_i[0];
    __syncthreads();
    if (qi >= B.count) break;
    const int32_t mi = B.order[qi];
    const BatchDesc D = B.desc[mi];
    if (tid == 0) {
      s_pc.prev_l = 0.0f;
      s_pc.prev_k = 0.0f;
      s_pc.cos_mean = 0.0f;
      s_pc.cos_max = 0.0f;
      s_pc.prev_tau = 0.0f;
      s_pc.off = 0;
      s_pc.prev_learned = 0;
      s_pc.prev_minb = INFINITY;
    }
    double* A = D.A;
    const int64_t m = D.m, n = D.n, lda = D.lda, kmin = m < n ? m : n;
    // ---- a1: column norms, identity permutation, zero htau
    double amax = 0.0;
    bool finite = true;
    for (int64_t j = wp; j < n; j += BW) {
      const double* a = A + j * lda;
      double s = 0.0;
      for (int64_t i = lane; i < m; i += 32) s = fma(a[i], a[i], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double nr = sqrt(s);
      if (lane == 0) {
        u[j] = nr;
        uref[j] = nr;
        mark[j] = 0.0;
        D.perm[j] = (int32_t)j;
      }
      if (!isfinite(nr)) finite = false;
      if (nr > amax) amax = nr;
    }
    for (int64_t i = tid; i < kmin; i += BT) D.htau[i] = 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) s_v[wp] = amax;
    const int fin_all = __syncthreads_and(finite ? 1 : 0);
    if (tid == 0) {
      double a = 0.0;
      for (int q = 0; q < BW; ++q) a = fmax(a, s_v[q]);
      s_sc[7] = a;
    }
    __syncthreads();
    const double anorm = s_sc[7];
    __syncthreads();
    if (!fin_all) {
      if (tid == 0) {
        B.status[mi] = 1;
        B.rank[mi] = -1;
        B.rank_colmax[mi] = -1;
        B.steps[mi] = 0;
      }
      continue;
    }
    QRDM_BPHASE(BP_INIT);
    const double eps1 = (B.eps1_mode == 1) ? EPS * sqrt((double)n) : EPS * (double)n;
    int64_t rank = -1, rank_cm = -1, step = 0, ns = 0;
    int dm_on = 1;
    while (ns < kmin) {
      // ---- a2/a3: argmax (Alg. 1), stopping test (Sec. 3.4), DM safeguard (Sec. 4)
      double mu;
      int64_t jstar;
      b_argmax(u, nullptr, ns, n, -1, -1, s_k, s_p, &mu, &jstar);
      const int64_t nrem = n - ns;
      if (rank_cm < 0 && mu <= eps1 * anorm) rank_cm = ns;
      if (rank < 0 && sqrt((double)nrem) * mu <= eps1 * anorm) {
        rank = ns;
        dm_on = 0;
        if (B.stop_at_rank) break;
      }
      int kcap = dm_on ? B.kmax : 1;
      if (kcap > kmin - ns) kcap = (int)(kmin - ns);
      // (tau_s, delta_s) of this step: fixed, or from the learned policy
      double tau_s = B.tau, delta_s = B.delta;
      bool learned = false;
      if (B.pol.active && dm_on) {
        // guard: every pivot the previous (learned) step accepted must be at
        // least rho_min times the largest partial norm left after it
        if (tid == 0 && s_pc.prev_learned && s_pc.prev_minb < B.pol.rho_min * mu) s_pc.off = 1;
        pol_features<BT>(u, ns, n, jstar, mu, anorm, s_pc, s_feat, s_pcnt);
        if (D.feat_log && step < D.log_cap && tid < POL_NFEAT) D.feat_log[step * POL_NFEAT + tid] = s_feat[tid];
        if (B.pol.w && !s_pc.off) {
          pol_mlp<BT>(B.pol, s_feat, s_h, s_pout);
          tau_s = s_pout[0];
          delta_s = s_pout[1];
          learned = true;
        }
      }
      if (D.act_log && step < D.log_cap && tid == 0) {
        D.act_log[2 * step] = tau_s;
        D.act_log[2 * step + 1] = delta_s;
      }
      if (tid == 0) s_minb = INFINITY;
      // candidate set (eq. def_candidate_set): the kcap-1 largest u_j >= tau mu,
      // j != j*, by (u desc, position asc) (readings R1, R2, R4)
      const double thr = tau_s * mu;
      const long long thr_key = okey(thr);
      if (tid == 0) s_cols[0] = (int32_t)jstar;
      int nc = 0;
      for (int c = 1; c < kcap; ++c) {
        double cv;
        int64_t cp;
        b_argmax(u, mark, ns, n, thr_key, jstar, s_k, s_p, &cv, &cp);
        if (cp < 0) break;
        if (tid == 0) {
          s_cols[c] = (int32_t)cp;
          mark[cp] = 1.0;
        }
        ++nc;
        __syncthreads();
      }
      int ncand_all = nc;
      if (D.trace && step < D.trace_cap && nc == kcap - 1 && kcap > 1) {
        // the trace records the uncapped count: count the rest
        int cnt = 0;
        for (int64_t j = ns + tid; j < n; j += BT)
          if (j != jstar && mark[j] == 0.0 && okey(u[j]) >= thr_key) ++cnt;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) s_k[wp] = cnt;
        __syncthreads();
        if (tid == 0) {
          long long t = 0;
          for (int q = 0; q < BW; ++q) t += s_k[q];
          s_i[1] = (int)t;
        }
        __syncthreads();
        ncand_all += s_i[1];
        __syncthreads();
      }
      __syncthreads();
      for (int c = 1 + tid; c <= nc; c += BT) mark[s_cols[c]] = 0.0;  // reset the marks
      const int kc = nc + 1;
      QRDM_BPHASE(BP_SELECT);
      // ---- a4: Gram matrix of the kc gathered columns over rows ns..m-1
      //          (Sec. 4, option (ii): Gram, then diagonal scaling)
      const int np = kc * (kc + 1) / 2;
      int k = 1;
      if (kc > 1) {
        for (int e = tid; e < np; e += BT) s_g[e] = 0.0;
        constexpr int LDS = G_ROWS + 1;
        for (int64_t g0 = ns; g0 < m; g0 += G_ROWS) {
          const int rows = (int)min((int64_t)G_ROWS, m - g0);
          __syncthreads();
          for (int e = tid; e < kc * G_ROWS; e += BT) {
            const int a = e / G_ROWS, i = e % G_ROWS;
            s_dyn[a * LDS + i] = (i < rows) ? A[(int64_t)s_cols[a] * lda + g0 + i] : 0.0;
          }
          __syncthreads();
          for (int e = tid; e < np; e += BT) {
            int b = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            while (b * (b + 1) / 2 > e) --b;
            while ((b + 1) * (b + 2) / 2 <= e) ++b;
            const int a = e - b * (b + 1) / 2;
            const double* xa = s_dyn + a * LDS;
            const double* xb = s_dyn + b * LDS;
            double s = s_g[e];
            for (int i = 0; i < rows; ++i) s = fma(xa[i], xb[i], s);
            s_g[e] = s;
          }
        }
        __syncthreads();
        QRDM_BPHASE(BP_GRAM);
        for (int a = tid; a < kc; a += BT) {
          const double d = sqrt(s_g[tri(a, a)]);
          s_rd[a] = (d > 0.0) ? 1.0 / d : 0.0;
        }
        __syncthreads();
        // ---- a5: greedy DM pick (Alg. 1 loop), strict |theta| < delta (R5, R6)
        if (wp == 0) {
          double dlt = delta_s;
          if (B.sdd) {
            const double dm = tau_s * tau_s / (double)((kc - 1) > 1 ? (kc - 1) : 1);
            if (dm < dlt) dlt = dm;
          }
          if (B.pol.active) {
            // |theta(j*, i)| statistics over the candidates (a feature of the next step)
            double cs = 0.0, cm = 0.0;
            for (int a = 1 + lane; a < kc; a += 32) {
              const double rr = s_rd[0] * s_rd[a];
              const double th = (rr > 0.0) ? fabs(s_g[tri(0, a)]) * rr : 1.0;
              cs += th;
              cm = fmax(cm, th);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              cs += __shfl_xor_sync(0xffffffffu, cs, o);
              cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
            }
            if (lane == 0) {
              s_pc.cos_mean = (float)(cs / (double)(kc - 1));
              s_pc.cos_max = (float)cm;
            }
          }
          int kk = 1;
          if (lane == 0) s_J[0] = 0;
          __syncwarp();
          for (int a = 1; a < kc; ++a) {
            bool ok = true;
            for (int b = lane; b < kk; b += 32) {
              const int jb = s_J[b];
              const double rr = s_rd[a] * s_rd[jb];
              const double th = (rr > 0.0) ? fabs(s_g[tri(jb, a)]) * rr : 1.0;
              if (!(th < dlt)) ok = false;
            }
            if (__all_sync(0xffffffffu, ok)) {
              if (lane == 0) s_J[kk] = a;
              ++kk;
            }
            __syncwarp();
          }
          if (lane == 0) s_i[0] = kk;
        }
        __syncthreads();
        k = s_i[0];
      } else {
        if (tid == 0) s_J[0] = 0;
      }
      __syncthreads();
      QRDM_BPHASE(BP_PICK);
      // ---- a6: pairwise swaps n_s + t <-> current position of J_t (Sec. 4, R14).
      // Thread 0 resolves the swap partners first (index work only); then every
      // thread performs the whole swap sequence on the rows it owns, so the
      // sequence needs no barrier between swaps.
      if (tid == 0) {
        for (int t = 0; t < k; ++t) s_sel[t] = s_cols[s_J[t]];
        for (int t = 0; t < k; ++t) {
          const int64_t q = ns + t, p = s_sel[t];
          if (p == q) continue;
          for (int t2 = t + 1; t2 < k; ++t2)
            if (s_sel[t2] == q) s_sel[t2] = p;
          double x = u[q];
          u[q] = u[p];
          u[p] = x;
          x = uref[q];
          uref[q] = uref[p];
          uref[p] = x;
          const int32_t pt = D.perm[q];
          D.perm[q] = D.perm[p];
          D.perm[p] = pt;
        }
      }
      __syncthreads();
      for (int t = 0; t < k; ++t) {
        const int64_t q = ns + t, p = s_sel[t];
        if (p == q) continue;
        double* cq = A + q * lda;
        double* cp = A + p * lda;
        for (int64_t i = tid; i < m; i += BT) {
          const double a = cq[i];
          cq[i] = cp[i];
          cp[i] = a;
        }
      }
      __syncthreads();
      if (D.trace && step < D.trace_cap) {
        if (tid == 0) {
          StepRecord* r = D.trace + step;
          r->ns = ns;
          r->jstar = jstar;
          r->ncand_all = ncand_all;
          r->ncand = nc;
          r->k = k;
          r->dm_on = dm_on;
          r->mu = mu;
          r->eps_s = tau_s * mu;
          r->nrecomp = 0;
        }
        if (D.traceJ)
          for (int t = tid; t < B.kmax; t += BT) D.traceJ[step * B.kmax + t] = (t < k) ? D.perm[ns + t] : -1;
      }
      QRDM_BPHASE(BP_SWAP);
      // ---- a7/a8/a9: sub-panels of PB columns (Alg. 4 panel with its break
      //      test, R10, R11), each followed by its block reflector
      const double eps_s = tau_s * mu;
      if (B.pol.active && kc == 1 && tid == 0) {
        s_pc.cos_mean = 0.0f;
        s_pc.cos_max = 0.0f;
      }
      int lacc = 0;
      bool broke = false;
      for (int jb = 0; jb < k && !broke; jb += PB) {
        const int w = min(PB, k - jb);
        const int64_t r0 = ns + jb;
        int lj = w;
        for (int l = 0; l < w; ++l) {
          const int64_t p = r0 + l;
          const double* x = A + p * lda;
          // x^T [sub-panel column] over rows > p, and the pivot-row values
          for (int t = wp; t < w; t += BW) {
            const double* ct = A + (r0 + t) * lda;
            double acc = 0.0, acc1 = 0.0;
            int64_t i = p + 1 + lane;
            for (; i + 32 < m; i += 64) {
              acc = fma(x[i], ct[i], acc);
              acc1 = fma(x[i + 32], ct[i + 32], acc1);
            }
            if (i < m) acc = fma(x[i], ct[i], acc);
            acc += acc1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
              s_tot[t] = acc;
              s_tot[PB + t] = ct[p];
            }
          }
          __syncthreads();
          const int lg = jb + l;
          if (tid == 0) {
            const double alpha = s_tot[PB + l], s2 = s_tot[l];
            const double nrm = sqrt(alpha * alpha + s2);
            const bool check = (lg >= 1) && !B.no_break && (B.check_last ? (lg < k) : (lg + 1 < k));
            s_sc[4] = (check && nrm < eps_s) ? 1.0 : 0.0;
            if (s2 == 0.0) {  // H = I: beta = alpha, htau = 0
              s_sc[0] = alpha;
              s_sc[1] = 0.0;
              s_sc[2] = 0.0;
            } else {
              const double beta = (alpha >= 0.0) ? -nrm : nrm;
              s_sc[0] = beta;
              s_sc[1] = (beta - alpha) / beta;
              s_sc[2] = 1.0 / (alpha - beta);
            }
          }
          __syncthreads();
          if (s_sc[4] != 0.0) {
            lj = l;
            broke = true;
            break;
          }
          const double beta = s_sc[0], ht = s_sc[1], rden = s_sc[2];
          if (tid == 0) s_minb = fmin(s_minb, fabs(beta));
          // column l of T (forward columnwise compact WY): y_r = v_r^T v_l
          if (tid < l) s_y[tid] = s_tot[PB + tid] + s_tot[tid] * rden;
          __syncthreads();
          if (tid < l) {
            double sacc = 0.0;
            for (int qq = tid; qq < l; ++qq) sacc += s_T[tid][qq] * s_y[qq];
            s_T[tid][l] = (ht == 0.0) ? 0.0 : -ht * sacc;
          }
          if (tid == 0) {
            s_T[l][l] = ht;
            D.htau[p] = ht;
          }
          // H_p on the sub-panel columns right of p
          if (ht != 0.0) {
            for (int t = l + 1 + wp; t < w; t += BW) {
              double* ct = A + (r0 + t) * lda;
              const double hw = ht * (s_tot[PB + t] + s_tot[t] * rden);
              const double hwr = hw * rden;
              for (int64_t i = p + 1 + lane; i < m; i += 32) ct[i] = fma(-hwr, x[i], ct[i]);
              if (lane == 0) ct[p] -= hw;
            }
          }
          __syncthreads();
          double* xc = A + p * lda;
          if (ht != 0.0)
            for (int64_t i = p + 1 + tid; i < m; i += BT) xc[i] = xc[i] * rden;
          if (tid == 0) xc[p] = beta;
          __syncthreads();
        }
        lacc += lj;
        QRDM_BPHASE(BP_PANEL);
        const int64_t c0 = ns + jb + w;
        const int64_t n2 = n - c0;
        if (lj > 0 && n2 > 0)
          b_reflect_any<LPC>(A, lda, m, r0, c0, n2, lj, B.rows_pp, B.nmax, s_dyn, s_T, Wb);
        QRDM_BPHASE(BP_REFLECT);
      }
      if (D.trace && step < D.trace_cap && tid == 0) D.trace[step].l = lacc;
      // ---- a10: partial norm update (Sec. 3.2 block form; R8, R9, R16).
      // 8 lanes per column, 4 columns per warp: every FP64 warp instruction
      // costs the FP64 pipe the same whatever its active lanes.
      const int64_t nsn = ns + lacc;
      int nrec = 0;
      {
        const int sub = lane >> 3, l8 = lane & 7;
        for (int64_t jg = ns + (int64_t)wp * 4; jg < n; jg += (int64_t)BW * 4) {
          const int64_t j = jg + sub;
          int mode = 0;  // 0: nothing, 1: factored (u = 0), 2: downdate, 3: recompute
          double uj = 0.0;
          if (j < n) {
            if (j < nsn) {
              mode = 1;
            } else if (j < ns + k) {
              mode = 3;
            } else {
              uj = u[j];
              mode = (uj == 0.0) ? 0 : 2;
            }
          }
          const double* a = A + (j < n ? j : 0) * lda;
          double q = 0.0;
          if (mode == 2)
            for (int64_t r = ns + l8; r < nsn; r += 8) {
              const double xv = a[r] / uj;
              q = fma(xv, xv, q);
            }
          q += __shfl_xor_sync(0xffffffffu, q, 4);
          q += __shfl_xor_sync(0xffffffffu, q, 2);
          q += __shfl_xor_sync(0xffffffffu, q, 1);
          double t = 0.0;
          if (mode == 2) {
            t = 1.0 - q;
            if (t < 0.0) t = 0.0;
            const double ratio = uj / uref[j];
            if (t * ratio * ratio <= sqeps) mode = 3;
          }
          double sq = 0.0;
          if (mode == 3)
            for (int64_t r = nsn + l8; r < m; r += 8) sq = fma(a[r], a[r], sq);
          sq += __shfl_xor_sync(0xffffffffu, sq, 4);
          sq += __shfl_xor_sync(0xffffffffu, sq, 2);
          sq += __shfl_xor_sync(0xffffffffu, sq, 1);
          if (l8 == 0) {
            if (mode == 1) {
              u[j] = 0.0;
            } else if (mode == 3) {
              const double nr = sqrt(sq);
              u[j] = nr;
              uref[j] = nr;
              ++nrec;
            } else if (mode == 2) {
              u[j] = uj * sqrt(t);
            }
          }
        }
      }
      nrec = __reduce_add_sync(0xffffffffu, nrec);
      if (D.trace && step < D.trace_cap && lane == 0 && nrec)
        atomicAdd((unsigned long long*)&D.trace[step].nrecomp, (unsigned long long)nrec);
      if (B.pol.active && dm_on && tid == 0) {
        s_pc.prev_learned = learned ? 1 : 0;
        s_pc.prev_minb = s_minb;
        s_pc.prev_l = (float)lacc;
        s_pc.prev_k = (float)k;
        s_pc.prev_tau = (float)tau_s;
      }
      __syncthreads();
      QRDM_BPHASE(BP_DOWNDATE);
      ns = nsn;
      ++step;
      if (lacc == 0) break;  // cannot happen: the first panel column is never tested
    }
    if (tid == 0) {
      B.rank[mi] = (rank >= 0) ? rank : (ns >= kmin ? kmin : ns);
      B.rank_colmax[mi] = (rank_cm >= 0) ? rank_cm : (ns >= kmin ? kmin : ns);
      B.status[mi] = 0;
      B.steps[mi] = step;
    }
    __syncthreads();
  }
  if (prof) {
#pragma unroll
    for (int q = 0; q < BP_N; ++q)
      if (s_pacc[q]) atomicAdd(B.phase_clk + q, s_pacc[q]);
    const unsigned long long act = (unsigned long long)(clock64() - tstart);
    atomicAdd(B.phase_clk + BP_N, act);
    atomicMax(B.phase_clk + BP_N + 1, act);
  }
#undef QRDM_BPHASE
}

}  // namespace qrdm
