// QRDM block-step kernels for GB300 (sm_103a), FP64.
//
// One block step of QRDM2 (Algorithm 4) runs as the kernel sequence
//   k_select -> k_gram -> k_gram_reduce -> k_pick -> k_permute -> k_panel
//   -> k_trail_w -> k_trail_wreduce -> k_trail_update -> k_downdate
// All kernels read the step state (n_s, k, l, ...) from device memory, so the
// host never needs the values to launch them; grids are fixed and CTAs loop
// over the work units of the current step.
//
// FP64 on GB300 issues about 2 FMA per clock per SM (1.2 TFLOP/s for the
// chip), so every FP64-heavy phase is spread over all SMs; HBM traffic is a
// secondary concern for this precision.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "qrdm_policy.cuh"

namespace cg = cooperative_groups;

namespace qrdm {

constexpr int KMAX = 128;          // largest supported k_max
constexpr int PB = 16;             // sub-panel width of the blocked panel
constexpr double EPS = 2.220446049250313080847e-16;  // 2^-52
constexpr int PANEL_THREADS = 256;
constexpr int GEMM_THREADS = 256;

// Step state, one per factorization, in the workspace.
struct alignas(128) DevState {
  int64_t ns;       // columns factored (n_s)
  int64_t step;     // block steps started
  int64_t rank;     // -1 until the Sec. 3.4 criterion holds
  int64_t rank_colmax;
  int64_t jstar;    // position of the largest partial norm
  int64_t ncand_all;
  double mu;        // largest partial norm at step start
  double eps_s;     // tau * mu
  double anorm;     // max_j ||a_j||
  unsigned long long anorm_bits;
  int32_t done;     // 1 once the factorization is finished
  int32_t dm_on;    // DM pivoting on (1) or single-column pivoting (0)
  int32_t kc;       // 1 + |I|: columns in the cosine matrix
  int32_t k;        // |J|
  int32_t l;        // reflectors accepted by the panel
  int32_t npairs;   // column moves of the permutation
  int32_t nonfinite;
  int32_t pbreak;   // 1 once the panel's break test fired in this step
  int32_t cur_lj;   // reflectors accepted by the current sub-panel (0: inactive)
  int32_t pad[3];
  // per sub-panel of the current step: reflectors accepted, and whether
  // another sub-panel follows; the trailing kernels of sub-panel j read these,
  // not the fields above, because sub-panel j + 1 may run beside them
  int32_t sub_l[KMAX / PB];
  int32_t sub_next[KMAX / PB];
  double flops[24]; // algorithmic flops per kernel id (profile)
  // grid barrier of the fused single-column kernel and its diagnostics
  unsigned int gbar;     // arrivals (monotonic within one launch)
  int32_t abort_flag;    // set when a bounded wait gave up or a check failed; every kernel then stops
  int32_t diag_code;     // where (QRDM_FAIL_* of the C header): 1 grid barrier wait, 2 pivot index out
                         // of range, 4 tensor-core mbarrier wait, 8 checked-path index check
  int32_t diag_cta;
  int64_t diag_step;
  int64_t diag_ns;
  int64_t diag_value;
  // learned (tau, delta): the values of the current step and the carry
  double tau_s, delta_s;
  double pol_minb;     // smallest accepted |R_ii| of the current step
  PolicyCarry pc;
  int32_t pol_learned; // 1: the current step used the MLP's (tau, delta)
};

struct StepRecord {  // layout of qrdm_step_record
  int64_t ns, jstar, ncand_all, ncand, k, l, dm_on, nrecomp;
  double mu, eps_s;
};

struct Params {
  double* A;
  int64_t m, n, lda, kmin;
  double tau, delta, eps1;
  double sqeps_dd;       // recompute threshold of the norm downdate: sqrt(unit roundoff of the trailing update)
  int32_t kmax, stop_at_rank, check_last, no_break, sdd, max_steps;
  double* htau;
  int32_t* perm;
  // workspace
  DevState* st;
  double* u;       // [n] partial norms
  double* uref;    // [n] norms at the last exact computation
  int32_t* cols;   // [KMAX] positions: j* then the sorted candidates
  int32_t* mdst;   // [2*KMAX] permutation moves: column mdst[e] <- column msrc[e]
  int32_t* msrc;
  double* Gp;      // [gram_chunks][kmax*kmax] partial Gram matrices (packed upper)
  double* G;       // [kmax*kmax] packed upper Gram matrix
  double* T;       // [KMAX*KMAX] compact-WY T, column-major, ld KMAX
  double* Wp;      // [wchunks][kmax][n] partial V^T A22
  double* W;       // [kmax][n] T^T V^T A22
  int32_t gram_chunks;  // CTAs of k_gram (= partial Gram matrices)
  int32_t gram_rows;    // rows of one chunk of the Gram kernel in use (GRAM_ROWS_CC, or GRAM_ROWS on tcgen05)
  int32_t wchunks;      // most row chunks of the W phase
  int32_t w_units;      // target work units of the W phase (same in k_trail_w and k_trail_wreduce)
  int32_t mixed;        // 1: FP32-class trailing update and Gram (geometry of k_trail_w32)
  int32_t merged;       // 1: sub-panel updates stop at the panel's end; one merged trailing update per step
  float* Wt;            // tensor-core forms: V^T A22 of row segment s at Wt + (s + 1) n 64, [column][64] (aliases Wp)
  int32_t tc_nseg;      // merged form: most row segments of the W GEMM
  unsigned char* tc_vw; // tensor-core forms: V's operand image for the W pass
  unsigned char* tc_vu; // V's operand image for the update
  unsigned char* tc_wi; // W's operand image for the update
  int32_t tc_al;        // 1: A and lda allow 16-byte loads from an even row (the W pass starts its rows there)
  int32_t tcu_tma;      // 1: the update streams A by tensor copies from that even row (V's update image shifted too)
  int32_t sel_stage;    // 1: k_select's dynamic shared memory holds u[ns..n)
  int32_t checked;      // 1: range-check every device-derived index before use (opts.checked)
  int32_t test_fault;   // test hook of opts.test_fault (0: none)
  int64_t wait_ns;      // limit of every bounded device-side wait, in global-timer nanoseconds
  // optional trace
  StepRecord* trace;
  int32_t* traceJ;
  int64_t trace_cap;
  PolicyParams pol;  // learned (tau, delta) and feature logging (pol.active = 0: off)
};

// kernel ids (same numbering as QRDM_K_* in the C header)
enum KernelId {
  KID_COLNORM = 0, KID_SELECT, KID_GRAM, KID_GRAM_REDUCE, KID_PICK, KID_PERMUTE, KID_PANEL, KID_TRAIL_W,
  KID_TRAIL_WREDUCE, KID_TRAIL_UPDATE, KID_DOWNDATE, KID_STEP_END, KID_QRP_TAIL, KID_WY_T, KID_TC_VIMG, KID_TC_WSUM,
  KID_TC_W, KID_TC_UPDATE
};

__device__ __forceinline__ void add_flops(DevState* st, int kid, double f) { atomicAdd(&st->flops[kid], f); }

// failure codes of DevState::diag_code (same values as QRDM_FAIL_* in the C header)
constexpr int FAIL_GRID_BARRIER = 1;
constexpr int FAIL_PIVOT_RANGE = 2;
constexpr int FAIL_MMA_WAIT = 4;
constexpr int FAIL_CHECK = 8;

// The GPU's global timer in nanoseconds: the clock of every bounded wait, so
// that a limit means the same time at any SM clock.
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Record the first failure of a factorization (later ones keep the first
// record) and raise the abort flag that every kernel observes.
__device__ __forceinline__ void record_fail(DevState* st, int code, int who, int64_t step, int64_t ns,
                                            int64_t value) {
  if (atomicExch(&st->abort_flag, 1) == 0) {
    st->diag_code = code;
    st->diag_cta = who;
    st->diag_step = step;
    st->diag_ns = ns;
    st->diag_value = value;
    __threadfence();
  }
}

// A checked-path index check: true when lo <= v < hi; otherwise the failure is
// recorded (kernel id `kid`, the bad value) and the caller skips the access.
__device__ __forceinline__ bool in_range(const Params& P, int kid, int64_t v, int64_t lo, int64_t hi) {
  if (v >= lo && v < hi) return true;
  record_fail(P.st, FAIL_CHECK, kid, P.st->step, P.st->ns, v);
  return false;
}

// FP64 <-> FP32 by integer operations on the IEEE-754 fields.  GB300 executes
// F2F conversions that involve FP64 on its narrow FP64 pipe (about 2 per clock
// per SM), which would bound the streaming FP32-class kernels; the integer
// pipe is far wider.  Finite inputs only (the matrix is checked on entry).
//   to FP32: the magnitude's exponent|mantissa field is rounded to 23 mantissa
//   bits by adding half a unit of the last kept bit (round to nearest, ties
//   away from zero; a carry moves into the exponent as it should), then the
//   exponent is rebiased; magnitudes below 2^-126 flush to a signed zero.
//   to FP64: exact; FP32 subnormals (never produced with flushing) map to zero.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const long long em = (long long)((mag + (1ull << 28)) >> 29) - ((long long)(1023 - 127) << 23);
  unsigned bits = sign | (unsigned)em;
  bits = (em < (1ll << 23)) ? sign : bits;  // biased FP32 exponent <= 0: flush to signed zero
  bits = (em >= (255ll << 23)) ? (sign | 0x7F800000u) : bits;
  return __uint_as_float(bits);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned mant = b & 0x7FFFFFu;
  unsigned hi = sign | ((e + (1023u - 127u)) << 20) | (mant >> 3);
  unsigned lo = mant << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// sum_{q < cnt} p[q * stride], added in q order from 0.0 (so bit for bit the
// plain loop) with the loads issued eight at a time: the partial sums these
// reductions read sit in L2, and a loop that waits for each load in turn is
// latency-bound
__device__ __forceinline__ double sum_strided(const double* p, int64_t stride, int64_t cnt) {
  double s = 0.0;
  int64_t q = 0;
  for (; q + 8 <= cnt; q += 8) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = p[(q + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
  }
  for (; q < cnt; ++q) s += p[q * stride];
  return s;
}

// operand load in a kernel's compute type
__device__ __forceinline__ double to_tc(double x, double) { return x; }
__device__ __forceinline__ float to_tc(double x, float) { return f64_to_f32_rn(x); }

// multiply-add in the compute type of a kernel (FP64, or FP32 in the
// mixed-precision form)
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// ---------------------------------------------------------------------------
// a1: column norms u_j = ||a_j||, uref = u, perm = identity, anorm = max u.
// One warp per column, lanes stride the rows (coalesced).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_colnorm_init(Params P) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = warp; j < P.n; j += nwarps) {
    const double* a = P.A + j * P.lda;
    double s = 0.0;
    for (int64_t i = lane; i < P.m; i += 32) {
      double x = a[i];
      s = fma(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      double nr = sqrt(s);
      P.u[j] = nr;
      P.uref[j] = nr;
      P.perm[j] = (int32_t)j;
      if (j == 0) add_flops(P.st, KID_COLNORM, 2.0 * (double)P.m * (double)P.n);
      if (!isfinite(nr)) {
        P.st->nonfinite = 1;
      } else {
        atomicMax(&P.st->anorm_bits, (unsigned long long)__double_as_longlong(nr));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Block-wide helpers (1024-thread select kernel).
// ---------------------------------------------------------------------------
struct ArgMax {
  double v;
  int64_t p;
};
// The partial norms are non-negative, and non-negative doubles order like
// their bit patterns read as int64: the selection compares keys on the
// integer pipe (a warp-wide FP64 compare takes the FP64 pipe as long as an
// FMA).  Larger value first, ties to the lower position.
__device__ __forceinline__ long long ukey(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool kbetter_u(long long ka, int64_t pa, long long kb, int64_t pb) {
  return ka > kb || (ka == kb && pa < pb);
}

// ---------------------------------------------------------------------------
// a2/a3: stopping test, argmax, candidate set (one CTA of 1024 threads).
// Also advances n_s by the previous step's l.
// ---------------------------------------------------------------------------
constexpr int SEL_THREADS = 1024;
constexpr int SEL_STAGE_MAX = 24576;  // most partial norms k_select stages in shared memory (192 KB)

__device__ int block_sum_int(int v, int* red) {
  // red: >= 32 ints of shared memory
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int t = 0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Given a 256-bin histogram in shared memory, find the digit d (scanning from
// the top when `desc`, else from the bottom) holding the krem-th element;
// returns d and writes the count of elements strictly before bin d to *before.
__device__ int hist_pick(const int* hist, int krem, bool desc, int* s_out) {
  // executed by warp 0
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    // each lane owns 8 consecutive bins in scan order
    int c[8];
    int tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int bin = desc ? 255 - (lane * 8 + q) : lane * 8 + q;
      c[q] = hist[bin];
      tot += c[q];
    }
    // exclusive scan of tot across lanes
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int excl = incl - tot;
    bool mine = (excl < krem) && (krem <= incl);
    unsigned b = __ballot_sync(0xffffffffu, mine);
    int owner = __ffs(b) - 1;
    if (lane == owner) {
      int run = excl;
      for (int q = 0; q < 8; ++q) {
        if (run + c[q] >= krem) {
          int bin = desc ? 255 - (lane * 8 + q) : lane * 8 + q;
          s_out[0] = bin;
          s_out[1] = run;
          break;
        }
        run += c[q];
      }
    }
  }
  __syncthreads();
  return s_out[0];
}

__global__ void __launch_bounds__(SEL_THREADS) k_select(Params P) {
  DevState* st = P.st;
  __shared__ long long s_k[32];
  __shared__ int64_t s_p[32];
  __shared__ int s_red[40];
  __shared__ int s_hist[256];
  __shared__ int s_pick[2];
  __shared__ int s_ctl[8];
  __shared__ double s_ctld[4];
  __shared__ int s_list[KMAX];
  __shared__ long long s_lk[KMAX];
  __shared__ int s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  if (tid == 0) {
    int go = 1;
    if (st->done) go = 0;
    if (go && *(volatile int32_t*)&st->abort_flag) {
      st->done = 1;
      go = 0;
    }
    if (go && (st->ns >= P.kmin || (P.max_steps > 0 && st->step >= P.max_steps))) {
      st->done = 1;
      go = 0;
    }
    if (go) {
      st->l = 0;
      st->pbreak = 0;
      st->cur_lj = 0;
      for (int q = 0; q < KMAX / PB; ++q) {
        st->sub_l[q] = 0;
        st->sub_next[q] = 0;
      }
    }
    s_ctl[0] = go;
  }
  __syncthreads();
  if (!s_ctl[0]) return;
  const int64_t ns = st->ns, n = P.n;
  // the partial norms u[ns..n) in shared memory when the launch gave room
  // for them (P.sel_stage): the argmax, the count, every radix pass and the
  // gather read them there
  extern __shared__ double s_u[];
  const bool staged = P.sel_stage != 0;
  if (staged) {
    for (int64_t j = ns + tid; j < n; j += SEL_THREADS) s_u[j - ns] = P.u[j];
    __syncthreads();
  }
  const double* uu = staged ? s_u - ns : P.u;  // uu[j] = u[j] for j >= ns

  // argmax over u[ns..n), ties to the lowest position (integer keys)
  long long bk = -1;
  int64_t bp = INT64_MAX;
  for (int64_t j = ns + tid; j < n; j += SEL_THREADS) {
    const long long x = ukey(uu[j]);
    if (kbetter_u(x, j, bk, bp)) {
      bk = x;
      bp = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
    if (kbetter_u(ok, op, bk, bp)) {
      bk = ok;
      bp = op;
    }
  }
  if (lane == 0) {
    s_k[w] = bk;
    s_p[w] = bp;
  }
  __syncthreads();
  if (w == 0) {
    bk = s_k[lane];
    bp = s_p[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
      if (kbetter_u(ok, op, bk, bp)) {
        bk = ok;
        bp = op;
      }
    }
    if (lane == 0) {
      const double mu = __longlong_as_double(bk);
      const int64_t jstar = bp;
      const int64_t nrem = n - ns;
      const double anorm = __longlong_as_double((long long)st->anorm_bits);
      st->anorm = anorm;
      const double rhs = P.eps1 * anorm;
      if (st->rank_colmax < 0 && mu <= rhs) st->rank_colmax = ns;
      int stop = 0;
      if (st->rank < 0 && sqrt((double)nrem) * mu <= rhs) {
        st->rank = ns;
        st->dm_on = 0;
        if (P.stop_at_rank) stop = 1;
      }
      if (P.checked && !stop && !in_range(P, KID_SELECT, jstar, ns, n)) stop = 1;
      if (stop) {
        st->done = 1;
      } else {
        st->mu = mu;
        st->jstar = jstar;
        int64_t kcap = st->dm_on ? P.kmax : 1;
        if (kcap > P.kmin - ns) kcap = P.kmin - ns;
        s_ctl[2] = (int)kcap;
        s_ctl[3] = st->dm_on;
        s_ctld[1] = mu;
        s_ctld[2] = anorm;
        const int64_t rec = st->step;
        if (P.trace && rec < P.trace_cap) {
          StepRecord* r = P.trace + rec;
          r->ns = ns;
          r->jstar = jstar;
          r->dm_on = st->dm_on;
          r->mu = mu;
          r->nrecomp = 0;
        }
        P.cols[0] = (int32_t)jstar;
      }
      s_ctl[1] = stop;
      s_p[0] = jstar;
    }
  }
  __syncthreads();
  if (s_ctl[1]) return;
  const int64_t jstar = s_p[0];
  const int K = s_ctl[2] - 1;  // candidates to keep
  {
    // (tau_s, delta_s) of this step: fixed, or from the learned policy
    __shared__ float s_feat[POL_NFEAT];
    __shared__ int s_pcnt[8 * (SEL_THREADS / 32)];
    __shared__ float s_h[2 * POL_HIDDEN];
    __shared__ double s_pout[2];
    const double mu = s_ctld[1];
    if (tid == 0) {
      s_pout[0] = P.tau;
      s_pout[1] = P.delta;
    }
    int learned = 0;
    if (P.pol.active && s_ctl[3]) {
      if (tid == 0 && st->pc.prev_learned && st->pc.prev_minb < P.pol.rho_min * mu) st->pc.off = 1;
      __syncthreads();
      const PolicyCarry pc = st->pc;
      pol_features<SEL_THREADS>(P.u, ns, n, jstar, mu, s_ctld[2], pc, s_feat, s_pcnt);
      const int64_t rec = st->step;
      if (P.pol.feat_log && rec < P.pol.log_cap && tid < POL_NFEAT) P.pol.feat_log[rec * POL_NFEAT + tid] = s_feat[tid];
      if (P.pol.w && !pc.off) {
        pol_mlp<SEL_THREADS>(P.pol, s_feat, s_h, s_pout);
        learned = 1;
      }
    }
    __syncthreads();
    if (tid == 0) {
      const double tau_s = s_pout[0], delta_s = s_pout[1];
      st->tau_s = tau_s;
      st->delta_s = delta_s;
      st->pol_learned = learned;
      st->pol_minb = INFINITY;
      st->eps_s = tau_s * mu;
      s_ctld[0] = tau_s * mu;
      const int64_t rec = st->step;
      if (P.trace && rec < P.trace_cap) P.trace[rec].eps_s = tau_s * mu;
      if (P.pol.act_log && rec < P.pol.log_cap) {
        P.pol.act_log[2 * rec] = tau_s;
        P.pol.act_log[2 * rec + 1] = delta_s;
      }
    }
    __syncthreads();
  }
  const double thr = s_ctld[0];
  const long long tk = ukey(thr);  // u >= thr exactly when ukey(u) >= tk (both non-negative)

  // count candidates
  int c = 0;
  if (K > 0) {
    for (int64_t j = ns + tid; j < n; j += SEL_THREADS)
      if (j != jstar && ukey(uu[j]) >= tk) ++c;
  }
  const int ncand_all = (K > 0) ? block_sum_int(c, s_red) : 0;
  const int keep = ncand_all < K ? ncand_all : K;

  // threshold key: select the keep-th largest (u desc) key, then positions
  unsigned long long tkey = 0;  // take keys > tkey, and keys == tkey with pos <= tpos
  int64_t tpos = INT64_MAX;
  if (keep > 0 && ncand_all > keep) {
    unsigned long long prefix = 0, pmask = 0;
    int krem = keep;
    for (int shift = 56; shift >= 0; shift -= 8) {
      for (int b = tid; b < 256; b += SEL_THREADS) s_hist[b] = 0;
      __syncthreads();
      for (int64_t j = ns + tid; j < n; j += SEL_THREADS) {
        const long long kx = ukey(uu[j]);
        if (j != jstar && kx >= tk) {
          const unsigned long long key = (unsigned long long)kx;
          if ((key & pmask) == prefix) atomicAdd(&s_hist[(key >> shift) & 255], 1);
        }
      }
      __syncthreads();
      int d = hist_pick(s_hist, krem, true, s_pick);
      krem -= s_pick[1];
      prefix |= ((unsigned long long)d) << shift;
      pmask |= 255ull << shift;
      __syncthreads();
    }
    tkey = prefix;
    // krem = how many with key == tkey to take (lowest positions first)
    int neq = 0;
    for (int64_t j = ns + tid; j < n; j += SEL_THREADS) {
      const long long kx = ukey(uu[j]);
      if (j != jstar && kx >= tk && (unsigned long long)kx == tkey) ++neq;
    }
    neq = block_sum_int(neq, s_red);
    if (neq > krem) {
      // krem-th smallest position among the ties (positions < 2^31)
      uint32_t pprefix = 0, ppmask = 0;
      int prem = krem;
      for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += SEL_THREADS) s_hist[b] = 0;
        __syncthreads();
        for (int64_t j = ns + tid; j < n; j += SEL_THREADS) {
          const long long kx = ukey(uu[j]);
          if (j != jstar && kx >= tk && (unsigned long long)kx == tkey) {
            uint32_t pk = (uint32_t)j;
            if ((pk & ppmask) == pprefix) atomicAdd(&s_hist[(pk >> shift) & 255], 1);
          }
        }
        __syncthreads();
        int d = hist_pick(s_hist, prem, false, s_pick);
        prem -= s_pick[1];
        pprefix |= ((uint32_t)d) << shift;
        ppmask |= 255u << shift;
        __syncthreads();
      }
      tpos = (int64_t)pprefix;
    }
  } else if (keep > 0) {
    tkey = 0;  // take every candidate
    tpos = INT64_MAX;
  }

  // gather the kept candidates
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  if (keep > 0) {
    const bool all = (ncand_all <= keep);
    for (int64_t j = ns + tid; j < n; j += SEL_THREADS) {
      const long long kx = ukey(uu[j]);
      if (j == jstar || kx < tk) continue;
      const unsigned long long key = (unsigned long long)kx;
      bool take = all || key > tkey || (key == tkey && j <= tpos);
      if (take) {
        int slot = atomicAdd(&s_cnt, 1);
        if (slot < KMAX) {
          s_list[slot] = (int)j;
          s_lk[slot] = kx;
        }
      }
    }
  }
  __syncthreads();
  const int got = s_cnt;
  // order by (u desc, position asc): rank counting
  if (tid < got && got <= KMAX) {
    const long long xk = s_lk[tid];
    const int xp = s_list[tid];
    int r = 0;
    for (int b = 0; b < got; ++b) {
      if (kbetter_u(s_lk[b], s_list[b], xk, xp)) ++r;
    }
    if (!P.checked || (in_range(P, KID_SELECT, xp, ns, n) && in_range(P, KID_SELECT, 1 + r, 1, P.kmax)))
      P.cols[1 + r] = xp;
  }
  if (tid == 0) {
    int bad = (got != keep);
    st->kc = 1 + keep;
    st->ncand_all = ncand_all;
    if (bad) {
      st->nonfinite = 2;  // internal inconsistency
      st->done = 1;
    }
    const int64_t rec = st->step;
    if (P.trace && rec < P.trace_cap) {
      P.trace[rec].ncand_all = ncand_all;
      P.trace[rec].ncand = keep;
    }
  }
}

// ---------------------------------------------------------------------------
// a4: Gram matrix of the kc = 1 + |I| gathered columns over rows n_s..m-1.
// Each CTA owns row chunks (grid-stride) and writes a partial upper triangle;
// k_gram_reduce sums the partials in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int GRAM_ROWS = 64;     // rows of one chunk of the tensor-core Gram (whole K atoms)
constexpr int GRAM_ROWS_CC = 16;  // rows of one chunk of the CUDA-core Gram: enough chunks for every SM

template <typename TC>
__device__ __forceinline__ void gram_body(Params& P) {
  DevState* st = P.st;
  if (st->done) return;
  const int kc = st->kc;
  if (kc <= 1) return;
  const int64_t ns = st->ns, m = P.m;
  const int64_t mr = m - ns;
  extern __shared__ double smg_raw[];
  TC* smg = reinterpret_cast<TC*>(smg_raw);  // [kc][GRAM_ROWS_CC + 1]
  const int LDS = GRAM_ROWS_CC + 1;
  const int npairs = kc * (kc + 1) / 2;
  TC acc[(KMAX * (KMAX + 1) / 2 + 255) / 256];
  const int nper = (npairs + blockDim.x - 1) / blockDim.x;
  for (int q = 0; q < nper; ++q) acc[q] = (TC)0;
  const int64_t nchunks = (mr + GRAM_ROWS_CC - 1) / GRAM_ROWS_CC;
  // chunk c of this CTA: c = blockIdx.x, blockIdx.x + gridDim.x, ...
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t r0 = ns + c * GRAM_ROWS_CC;
    const int rows = (int)min((int64_t)GRAM_ROWS_CC, m - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * GRAM_ROWS_CC; e += blockDim.x) {
      int a = e / GRAM_ROWS_CC, i = e % GRAM_ROWS_CC;
      double x = 0.0;
      if (i < rows) x = P.A[(int64_t)P.cols[a] * P.lda + r0 + i];
      smg[a * LDS + i] = to_tc(x, (TC)0);
    }
    __syncthreads();
    for (int q = 0; q < nper; ++q) {
      int e = threadIdx.x + q * blockDim.x;
      if (e >= npairs) break;
      // e -> (a, b) with a <= b, column-major upper triangle enumeration
      int b = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);  // FP32 estimate, corrected below
      while ((b + 1) * (b + 2) / 2 <= e) ++b;
      while (b * (b + 1) / 2 > e) --b;
      int a = e - b * (b + 1) / 2;
      const TC* xa = smg + a * LDS;
      const TC* xb = smg + b * LDS;
      TC s = acc[q];
      for (int i = 0; i < rows; ++i) s = fmat(xa[i], xb[i], s);
      acc[q] = s;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(P.st, KID_GRAM, (double)mr * kc * (kc + 1.0));
  double* out = P.Gp + (int64_t)blockIdx.x * P.kmax * P.kmax;
  for (int q = 0; q < nper; ++q) {
    int e = threadIdx.x + q * blockDim.x;
    if (e < npairs) out[e] = (double)acc[q];
  }
}

__global__ void __launch_bounds__(256) k_gram(Params P) { gram_body<double>(P); }
// mixed-precision form: the candidate Gram matrix in FP32, partials summed in FP64
__global__ void __launch_bounds__(256) k_gram32(Params P) { gram_body<float>(P); }

// G = sum of the Gram kernel's partials: 8 threads per entry each add a
// contiguous eighth of the partials (in order), then the eight sums are added
// in order, so the result is fixed while eight times as many loads are in
// flight (the partials sit in L2)
constexpr int GRED_ENTRIES = 32;  // entries per CTA of k_gram_reduce (256 threads)
__global__ void __launch_bounds__(256) k_gram_reduce(Params P) {
  const DevState* st = P.st;
  if (st->done) return;
  const int kc = st->kc;
  if (kc <= 1) return;
  const int npairs = kc * (kc + 1) / 2;
  const int64_t mr = P.m - st->ns;
  const int64_t nchunks = (mr + P.gram_rows - 1) / P.gram_rows;  // the Gram kernel's row chunks
  const int nparts = (int)min((int64_t)P.gram_chunks, nchunks);
  __shared__ double s_part[GRED_ENTRIES][9];
  const int le = threadIdx.x >> 3, h = threadIdx.x & 7;
  const int per = (nparts + 7) / 8;
  for (int e0 = blockIdx.x * GRED_ENTRIES; e0 < npairs; e0 += gridDim.x * GRED_ENTRIES) {
    const int e = e0 + le;
    const int c0 = h * per, c1 = min(nparts, c0 + per);
    const int64_t stride = (int64_t)P.kmax * P.kmax;
    s_part[le][h] = (e < npairs && c1 > c0) ? sum_strided(P.Gp + (int64_t)c0 * stride + e, stride, c1 - c0) : 0.0;
    __syncthreads();
    if (h == 0 && e < npairs) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += s_part[le][q];
      P.G[e] = t;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a5/a6: greedy DM pick (Alg. 1 loop) and the pairwise-swap permutation.
// One CTA; warp 0 does the sequential parts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tri(int a, int b) {  // packed upper index, a <= b
  return b * (b + 1) / 2 + a;
}

__global__ void __launch_bounds__(256) k_pick(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  constexpr int KW = KMAX / 32;  // 32-bit words of a row of the compatibility matrix
  __shared__ double s_d[KMAX];   // reciprocal column norms 1/sqrt(G_aa)
  __shared__ int s_col[KMAX];    // positions of the kc gathered columns
  __shared__ int s_J[KMAX];
  __shared__ uint32_t s_cmp[KMAX][KW];  // bit b of row a (b < a): |theta(a, b)| < delta
  __shared__ uint32_t s_jm[KW];         // the accepted set J as a bit set
  __shared__ int s_k, s_np, s_nm;
  __shared__ int s_pos[2 * KMAX];  // positions the swaps touch (entry t < k: ns + t)
  __shared__ int s_eid[KMAX];      // entry holding J_t's position at the step start
  __shared__ int s_cid[2 * KMAX];  // entry e now holds the column that started at entry s_cid[e]
  __shared__ int s_inv[2 * KMAX];  // inverse of s_cid
  __shared__ double s_mv[2 * KMAX][2];
  __shared__ int s_mvp[2 * KMAX];
  extern __shared__ double s_g[];  // packed upper Gram matrix, kc*(kc+1)/2
  const int kc = st->kc;
  const int64_t ns = st->ns;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  constexpr int NW = 256 / 32;

  if (kc > 1)
    for (int e = tid; e < kc * (kc + 1) / 2; e += blockDim.x) s_g[e] = P.G[e];
  for (int a = tid; a < kc; a += blockDim.x) s_col[a] = P.cols[a];
  __syncthreads();
  for (int a = tid; a < kc; a += blockDim.x) {
    const double d = (kc > 1) ? sqrt(s_g[tri(a, a)]) : 1.0;
    s_d[a] = (d > 0.0) ? 1.0 / d : 0.0;  // reciprocal norm; 0 marks a zero column
  }
  __syncthreads();
  const double tau_s = st->tau_s;
  double dlt = st->delta_s;
  if (P.sdd && kc > 1) {
    const double dm = tau_s * tau_s / (double)((kc - 1) > 1 ? (kc - 1) : 1);
    if (dm < dlt) dlt = dm;
  }
  if (P.pol.active && wp == 0) {
    // |theta(j*, i)| statistics over the candidates (a feature of the next step)
    double cs = 0.0, cm = 0.0;
    for (int a = 1 + lane; a < kc; a += 32) {
      const double rr = s_d[0] * s_d[a];
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
      st->pc.cos_mean = (kc > 1) ? (float)(cs / (double)(kc - 1)) : 0.0f;
      st->pc.cos_max = (float)cm;
    }
  }
  // the cosine test of every candidate pair at once: |theta_ab| = |G_ab| /
  // (||c_a|| ||c_b||) < delta, a zero column counting as |theta| = 1; warp w
  // takes rows a = w, w + 8, ..., lane b mod 32 of each word
  for (int a = wp; a < kc; a += NW) {
    const double ra = s_d[a];
    for (int q = 0; q < KW && 32 * q < a; ++q) {
      const int b = 32 * q + lane;
      bool ok = false;
      if (b < a) {
        const double rr = ra * s_d[b];
        const double th = (rr > 0.0) ? fabs(s_g[tri(b, a)]) * rr : 1.0;
        ok = th < dlt;
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, ok);
      if (lane == 0) s_cmp[a][q] = bal;
    }
  }
  __syncthreads();
  // greedy DM pick (Alg. 1 loop): candidates in order, a accepted when its
  // test passes against every accepted b (all of them before a)
  if (tid == 0) {
    for (int q = 0; q < KW; ++q) s_jm[q] = 0u;
    s_jm[0] = 1u;
    s_J[0] = 0;
    int k = 1;
    for (int a = 1; a < kc; ++a) {
      uint32_t bad = 0u;
      for (int q = 0; 32 * q < a; ++q) bad |= s_jm[q] & ~s_cmp[a][q];
      if (bad == 0u) {
        s_jm[a >> 5] |= 1u << (a & 31);
        s_J[k++] = a;
      }
    }
    s_k = k;
  }
  __syncthreads();
  const int k = s_k;
  // the positions the pairwise swaps touch: ns + t for t < k, then the
  // positions of the J_t outside the block, in t order (warp 0)
  if (wp == 0) {
    int napp = 0;
    for (int t0 = 0; t0 < k; t0 += 32) {
      const int t = t0 + lane;
      const int pj = (t < k) ? s_col[s_J[t]] : 0;
      const bool app = (t < k) && pj >= ns + k;
      const uint32_t bal = __ballot_sync(0xffffffffu, app);
      const int r = napp + __popc(bal & ((1u << lane) - 1u));
      if (t < k) {
        s_pos[t] = (int)(ns + t);
        if (app) {
          s_pos[k + r] = pj;
          s_eid[t] = k + r;
        } else {
          s_eid[t] = (int)(pj - ns);
        }
      }
      napp += __popc(bal);
    }
    if (lane == 0) s_np = k + napp;
  }
  __syncthreads();
  const int np = s_np;
  for (int e = tid; e < np; e += blockDim.x) {
    s_cid[e] = e;
    s_inv[e] = e;
  }
  __syncthreads();
  // permutation by pairwise swaps (Sec. 4): position ns + t <-> the current
  // position of J_t, simulated on the entries with the inverse map
  if (tid == 0) {
    for (int t = 0; t < k; ++t) {
      const int e = s_inv[s_eid[t]];
      if (e != t) {
        const int ct = s_cid[t], ce = s_cid[e];
        s_cid[t] = ce;
        s_cid[e] = ct;
        s_inv[ce] = t;
        s_inv[ct] = e;
      }
    }
  }
  __syncthreads();
  // the moves, in entry order: the column that started at s_pos[s_cid[e]] goes to s_pos[e]
  if (wp == 0) {
    int nm = 0;
    for (int e0 = 0; e0 < np; e0 += 32) {
      const int e = e0 + lane;
      const int src = (e < np) ? s_pos[s_cid[e]] : 0;
      const bool mv = (e < np) && src != s_pos[e];
      const uint32_t bal = __ballot_sync(0xffffffffu, mv);
      if (mv) {
        const int r = nm + __popc(bal & ((1u << lane) - 1u));
        P.mdst[r] = s_pos[e];
        P.msrc[r] = src;
        s_mvp[r] = e;
      }
      nm += __popc(bal);
    }
    if (lane == 0) s_nm = nm;
  }
  __syncthreads();
  if (tid == 0) {
    int nm = s_nm;
    if (P.checked) {
      if (P.test_fault == 2 && st->step == 0) {
        // test hook: a destination one past the last column (refused below)
        if (nm == 0) {
          P.msrc[0] = (int32_t)ns;
          s_mvp[0] = 0;
          nm = 1;
        }
        P.mdst[0] = (int32_t)P.n;
      }
      bool ok = in_range(P, KID_PICK, k, 1, kc + 1) && in_range(P, KID_PICK, nm, 0, 2 * KMAX + 1);
      for (int e = 0; ok && e < nm; ++e)
        ok = in_range(P, KID_PICK, P.mdst[e], ns, P.n) && in_range(P, KID_PICK, P.msrc[e], ns, P.n) &&
             in_range(P, KID_PICK, s_mvp[e], 0, np);
      if (!ok) nm = 0;  // no move is made; the factorization stops at this step's end
    }
    st->npairs = nm;
    st->k = k;
    s_nm = nm;
  }
  __syncthreads();
  const int nm = s_nm;
  for (int qq = tid; qq < nm; qq += blockDim.x) {
    const int src = P.msrc[qq];
    s_mv[qq][0] = P.u[src];
    s_mv[qq][1] = P.uref[src];
    s_mvp[qq] = P.perm[src];
  }
  __syncthreads();
  for (int qq = tid; qq < nm; qq += blockDim.x) {
    const int dst = P.mdst[qq];
    P.u[dst] = s_mv[qq][0];
    P.uref[dst] = s_mv[qq][1];
    P.perm[dst] = s_mvp[qq];
  }
  __syncthreads();
  if (P.trace && st->step < P.trace_cap) {
    if (tid == 0) P.trace[st->step].k = k;
    if (P.traceJ) {
      for (int t = tid; t < P.kmax; t += blockDim.x)
        P.traceJ[st->step * P.kmax + t] = (t < k) ? P.perm[ns + t] : -1;
    }
  }
}

// ---------------------------------------------------------------------------
// a6: apply the column moves to A (whole columns, rows 0..m-1).  Each CTA
// stages 32 rows of every moved column in shared memory, then writes them to
// their destinations, so overlapping sources and destinations are safe.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_permute(Params P) {
  const DevState* st = P.st;
  if (st->done) return;
  const int nm = st->npairs;
  if (nm == 0) return;
  extern __shared__ double s[];  // [2*kmax][33]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < P.m; r0 += (int64_t)gridDim.x * 32) {
    const int64_t i = r0 + lane;
    __syncthreads();
    for (int e = w; e < nm; e += nw) {
      const int64_t src = P.msrc[e];
      const bool ok = !P.checked || (src >= 0 && src < P.n);
      s[e * 33 + lane] = (i < P.m && ok) ? P.A[src * P.lda + i] : 0.0;
    }
    __syncthreads();
    for (int e = w; e < nm; e += nw) {
      const int64_t dst = P.mdst[e];
      if (P.checked && !(dst >= 0 && dst < P.n)) {
        if (lane == 0 && r0 == (int64_t)blockIdx.x * 32) record_fail(P.st, FAIL_CHECK, KID_PERMUTE, P.st->step, P.st->ns, dst);
        continue;
      }
      if (i < P.m) P.A[dst * P.lda + i] = s[e * 33 + lane];
    }
  }
}

// ---------------------------------------------------------------------------
// a7/a8: the Householder panel, blocked.  The k panel columns are factored in
// sub-panels of PB columns; k_panel(j) factors sub-panel j on one thread-block
// cluster, applying the break test of Alg. 4 with the panel-wide column index,
// and builds the sub-panel's compact-WY T_j.  The trailing kernels then apply
// (I - V_j T_j V_j^T)^T to every column right of the sub-panel (the rest of the
// panel and the trailing matrix), which is right-looking blocked QR.
//
// CTA r of the cluster owns a contiguous slice of the rows and only touches
// those rows.  Per reflector there is one cluster barrier: every CTA reduces
// x^T [sub-panel] over its rows (x = current column below the pivot), plus
// the pivot-row values, into a partial vector in its shared memory; after the
// barrier each CTA gathers all partials (distributed shared memory) and sums
// them in the same order, so all CTAs derive identical scalars and take the
// same break decision.
// ---------------------------------------------------------------------------
constexpr int MAX_CLUSTER = 16;
constexpr int PANEL_SMEM_MAX = 200 * 1024;  // sub-panel slice held in shared memory up to this size

// Element (i, t) of the sub-panel: absolute row i, sub-panel column t.  With
// SMEM the CTA's rows [rb, re) live in shared memory (column stride lds).
template <bool SMEM>
struct PanelView {
  double* base;  // SMEM: shared slice; else: A
  int64_t ld;    // SMEM: lds; else: lda
  int64_t rb;    // SMEM: first row held; else: 0
  int64_t c0;    // first column (absolute) of the sub-panel
  __device__ __forceinline__ double& at(int64_t i, int t) const {
    return SMEM ? base[(int64_t)t * ld + (i - rb)] : base[(c0 + t) * ld + i];
  }
};

template <bool SMEM>
__device__ __forceinline__ void panel_body(Params& P, int j) {
  cg::cluster_group cluster = cg::this_cluster();
  DevState* st = P.st;
  if (st->done) return;  // uniform across the cluster
  const int k = st->k;
  // checked path: the block size and its columns and rows (values fixed for
  // the launch, so every CTA of the cluster takes the same decision)
  if (P.checked && !(in_range(P, KID_PANEL, k, 1, P.kmax + 1) && in_range(P, KID_PANEL, st->ns + k, 1, P.n + 1) &&
                     in_range(P, KID_PANEL, st->ns, 0, P.m)))
    return;
  const int jb = j * PB;
  const int crank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  if (jb >= k || st->pbreak) {  // sub-panel beyond the panel, or the panel stopped
    if (crank == 0 && tid == 0) {
      st->cur_lj = 0;
      st->sub_l[j] = 0;
      st->sub_next[j] = 0;
    }
    return;
  }
  const int cs = (int)cluster.num_blocks();
  const int w = min(PB, k - jb);
  const int64_t m = P.m, lda = P.lda;
  const int64_t r0 = st->ns + jb;  // the sub-panel's first row and first column
  const int64_t mr = m - r0;
  const int64_t rpc = (mr + cs - 1) / cs;
  const int64_t rb = r0 + (int64_t)crank * rpc;
  const int64_t re = min(m, rb + rpc);
  __shared__ double s_slot[2][2 * PB];
  __shared__ double s_tot[2 * PB];
  __shared__ double s_y[PB];
  __shared__ double s_T[PB][PB];
  __shared__ double s_sc[8];
  __shared__ double s_rden[PB], s_beta[PB];  // per reflector: 1 / (alpha - beta) and beta (applied at the end)
  extern __shared__ double s_pan[];  // SMEM: [PB][lds]
  const int lane = tid & 31, wp = tid >> 5;
  const int nw = PANEL_THREADS / 32;
  double* A = P.A;
  PanelView<SMEM> V;
  if (SMEM) {
    const int64_t lds = ((m + cs - 1) / cs) | 1;  // odd stride: spreads columns over banks
    V.base = s_pan;
    V.ld = lds;
    V.rb = rb;
    V.c0 = r0;
    // this CTA's rows of the sub-panel, columns in rows (coalesced)
    for (int t = wp; t < w; t += nw) {
      const double* src = A + (r0 + t) * lda;
      for (int64_t i = rb + lane; i < re; i += 32) V.at(i, t) = src[i];
    }
    __syncthreads();
  } else {
    V.base = A;
    V.ld = lda;
    V.rb = 0;
    V.c0 = r0;
  }
  const double eps_s = st->eps_s;
  // The FP32-class form applies each sub-panel with the panel's compact-WY T;
  // every other form gets W = T^T V^T A by forward substitution with V^T V,
  // which its W pass computes on all SMs, so the panel skips T and the dot
  // products it would need (v_t^T v_l, t < l).
  const bool keep_t = P.mixed != 0;
  int lacc = w;
  bool broke = false;
  // On this GPU a warp-wide FP64 instruction holds the SM's narrow FP64 pipe
  // as long as an FMA of 32 lanes, whatever its lanes add: the per-reflector
  // reductions and scalars below are laid out to issue few of them.
  int64_t flops = 0;       // thread 0: flops of this launch (integer pipe)
  double minb = INFINITY;  // thread 0: smallest accepted |R_ii| (the learned policy's guard)
  __shared__ double s_hw[PB], s_hwr[PB];  // reflector l's coefficients of the columns t > l it updates
  __shared__ int s_brk, s_app;             // reflector l: the break test fired / H_l is not the identity
  for (int l = 0; l < w; ++l) {
    const int64_t p = r0 + l;  // pivot row and column
    double* slot = s_slot[l & 1];
    const int64_t i0 = max(rb, p + 1);
    const bool own_p = (p >= rb && p < re);
    const int lo = keep_t ? 0 : l;  // first column whose dot product this reflector needs
    // partial dot products x_l^T x_t over this CTA's rows below the pivot
    // (t = l: the squared tail norm), and the pivot-row entries.  Warp wp
    // takes columns t1 = lo + wp and t2 = t1 + 8; a pair shares the first
    // level of its lane tree (lanes 0-15 keep t1, 16-31 keep t2), the same
    // xor 16, 8, 4, 2, 1 tree as one column alone
    {
      const int t1 = lo + wp, t2 = t1 + nw;
      if (t1 < w) {
        const bool two = t2 < w;
        double a1 = 0.0, a2 = 0.0;
        for (int64_t i = i0 + lane; i < re; i += 32) {
          const double xl = V.at(i, l);
          a1 = fma(xl, V.at(i, t1), a1);
          if (two) a2 = fma(xl, V.at(i, t2), a2);
        }
        double r;
        if (two) {
          const bool up = lane >= 16;
          r = (up ? a2 : a1) + __shfl_xor_sync(0xffffffffu, up ? a1 : a2, 16);
        } else {
          r = a1 + __shfl_xor_sync(0xffffffffu, a1, 16);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) {
          slot[t1] = r;
          slot[PB + t1] = own_p ? V.at(p, t1) : 0.0;
        }
        if (two && lane == 16) {
          slot[t2] = r;
          slot[PB + t2] = own_p ? V.at(p, t2) : 0.0;
        }
      }
    }
    cluster.sync();
    // cluster-wide sums of the dot products in warp 0: lanes L and L + 16
    // read CTA L mod 16's partials of the even and odd columns, and a
    // transposed lane tree adds them (each level keeps half of a lane's
    // values; the lane pairs are the xor 8, 4, 2, 1 tree of every value, the
    // same in every CTA, so all CTAs get the same bits).  The pivot-row
    // entries come straight from the CTA holding the pivot row (warp 1).
    {
      const int nv = w - lo;
      if (wp == 0) {
        const int c = lane & 15, h = lane >> 4;
        double v[8];
        if (c < cs) {
          const double* rem = cluster.map_shared_rank(&s_slot[l & 1][0], c);
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = (2 * i + h < nv) ? rem[lo + 2 * i + h] : 0.0;
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.0;
        }
        bool up = (c & 8) != 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          v[i] = (up ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, up ? v[i] : v[i + 4], 8);
        up = (c & 4) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i)
          v[i] = (up ? v[i + 2] : v[i]) + __shfl_xor_sync(0xffffffffu, up ? v[i] : v[i + 2], 4);
        up = (c & 2) != 0;
        v[0] = (up ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, up ? v[0] : v[1], 2);
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
        const int e = 2 * (c >> 1) + h;  // the column this lane pair now holds
        if ((c & 1) == 0 && e < nv) s_tot[lo + e] = v[0];
      } else if (wp == 1) {
        const int own = (int)((p - r0) / rpc);
        if (lane < nv) s_tot[PB + lo + lane] = cluster.map_shared_rank(&s_slot[l & 1][0], own)[PB + lo + lane];
      }
    }
    __syncthreads();
    // the reflector's scalars in warp 0: beta from the norm, then the two
    // quotients htau = (beta - alpha) / beta and 1 / (alpha - beta) at once in
    // lanes 0 and 1 (FP64 division is a long instruction sequence here), then
    // the coefficients of the columns it updates, lane t for column t
    const int lg = jb + l;  // column index within the whole panel
    if (wp == 0) {
      const double alpha = s_tot[PB + l];
      const double s2 = s_tot[l];
      const double nrm = sqrt(alpha * alpha + s2);
      const double beta = (s2 == 0.0) ? alpha : ((alpha >= 0.0) ? -nrm : nrm);
      const double num = (lane == 0) ? (beta - alpha) : 1.0;
      const double den = (lane == 0) ? beta : (alpha - beta);
      const double qv = num / den;
      const double q0 = __shfl_sync(0xffffffffu, qv, 0);
      const double q1 = __shfl_sync(0xffffffffu, qv, 1);
      const double ht = (s2 == 0.0) ? 0.0 : q0;    // htau (a zero tail: H = I)
      const double rden = (s2 == 0.0) ? 0.0 : q1;  // 1 / (alpha - beta)
      if (lane > l && lane < w) {
        // v_i = x_i / (alpha - beta) below the pivot folded into the scale of x_l
        const double hw = ht * (s_tot[PB + lane] + s_tot[lane] * rden);
        s_hw[lane] = hw;
        s_hwr[lane] = hw * rden;
      }
      if (lane == 0) {
        const bool check = (lg >= 1) && !P.no_break && (P.check_last ? (lg < k) : (lg + 1 < k));
        s_brk = (check && nrm < eps_s) ? 1 : 0;
        s_app = (s2 == 0.0) ? 0 : 1;
        s_sc[0] = beta;
        s_sc[1] = ht;
        s_sc[2] = rden;
      }
    }
    __syncthreads();
    if (tid == 0) flops += 2 * (m - p - 1) * (int64_t)(w - lo);
    if (s_brk) {  // break test of Alg. 4 (identical in every CTA)
      lacc = l;
      broke = true;
      break;
    }
    const double ht = s_sc[1], rden = s_sc[2];
    if (tid == 0) {
      const double beta = s_sc[0];
      minb = fmin(minb, fabs(beta));
      s_rden[l] = s_app ? rden : 1.0;  // v_l = x_l / (alpha - beta) below the pivot
      s_beta[l] = beta;
      if (crank == 0) P.htau[p] = ht;
    }
    if (keep_t && crank == 0) {
      // compact-WY T_j column l: y_t = v_t^T v_l for t < l, from the unscaled
      // x_t (v_t = x_t / (alpha_t - beta_t) below its pivot, scaled at the end)
      if (tid < l) s_y[tid] = s_rden[tid] * (s_tot[PB + tid] + s_tot[tid] * rden);
      __syncthreads();
      if (tid < l) {
        double sacc = 0.0;
        for (int q = tid; q < l; ++q) sacc += s_T[tid][q] * s_y[q];
        s_T[tid][l] = (ht == 0.0) ? 0.0 : -ht * sacc;
      }
      if (tid == 0) s_T[l][l] = ht;
    }
    // apply H_l to the rest of the sub-panel (own rows); x_l stays unscaled
    if (s_app) {
      for (int t = l + 1 + wp; t < w; t += nw) {
        const double hw = s_hw[t], hwr = s_hwr[t];
        for (int64_t i = i0 + lane; i < re; i += 32) V.at(i, t) = fma(-hwr, V.at(i, l), V.at(i, t));
        if (own_p && lane == 0) V.at(p, t) -= hw;
      }
      if (tid == 0) flops += 2 * (m - p) * (int64_t)(w - l - 1);
    }
    __syncthreads();
  }
  // the accepted columns become v_t below the pivot and beta_t on it
  for (int t = wp; t < lacc; t += nw) {
    const int64_t pt = r0 + t;
    const double sc = s_rden[t];
    for (int64_t i = max(rb, pt + 1) + lane; i < re; i += 32) V.at(i, t) = V.at(i, t) * sc;
    if (pt >= rb && pt < re && lane == 0) V.at(pt, t) = s_beta[t];
  }
  __syncthreads();
  if (SMEM) {  // write the slice back
    for (int t = wp; t < w; t += nw) {
      double* dst = A + (r0 + t) * lda;
      for (int64_t i = rb + lane; i < re; i += 32) dst[i] = V.at(i, t);
    }
  }
  cluster.sync();  // every gather of this CTA's shared memory is done
  if (crank == 0) {
    if (keep_t)
      for (int e = tid; e < lacc * lacc; e += PANEL_THREADS) {
        const int r = e % lacc, c = e / lacc;
        P.T[(int64_t)c * KMAX + r] = (r <= c) ? s_T[r][c] : 0.0;
      }
    if (tid == 0) {
      st->cur_lj = lacc;
      st->sub_l[j] = lacc;
      st->sub_next[j] = (!broke && jb + PB < k) ? 1 : 0;
      st->l += lacc;
      if (lacc > 0) st->pol_minb = fmin(st->pol_minb, minb);
      if (broke) st->pbreak = 1;
      if (P.trace && st->step < P.trace_cap) P.trace[st->step].l = st->l;
      add_flops(st, KID_PANEL, (double)flops);
    }
  }
}

// the sub-panel slice in shared memory (when it fits) or in global memory
__global__ void __launch_bounds__(PANEL_THREADS) k_panel(Params P, int j) { panel_body<true>(P, j); }
__global__ void __launch_bounds__(PANEL_THREADS) k_panel_g(Params P, int j) { panel_body<false>(P, j); }

// ---------------------------------------------------------------------------
// a9: block reflector application after sub-panel j:
//   A[r0:m, c0:n] -= V_j (T_j^T (V_j^T A[r0:m, c0:n])),
// r0 = n_s + j PB (the sub-panel's first row and column), c0 = the first
// column right of the sub-panel, l = reflectors the sub-panel accepted.
// V_j (mr x l) is unit lower trapezoidal, stored below the diagonal of the
// sub-panel columns.  Three kernels: partial W = V^T A over row chunks,
// W = T^T sum(partials), A -= V W.  FFMA64 throughout.
// ---------------------------------------------------------------------------
struct SubGeom {
  int64_t r0, c0;
  int l;
};

// last column (exclusive) a sub-panel's block reflector reaches: the whole
// trailing matrix, or only the rest of the panel when the trailing block gets
// one merged update per step
// (j < 0: the merged update itself, all of the step's reflectors on the
// trailing block)
__device__ __forceinline__ int64_t trail_end(const Params& P, const DevState* st, int j) {
  return (P.merged && j >= 0) ? min(P.n, st->ns + (int64_t)st->k) : P.n;
}

__device__ __forceinline__ SubGeom sub_geom(const DevState* st, int j) {
  SubGeom g;
  const int k = st->k;
  if (j < 0) {
    g.r0 = st->ns;
    g.c0 = st->ns + k;
    g.l = st->l;
    return g;
  }
  g.r0 = st->ns + (int64_t)j * PB;
  g.c0 = st->ns + min((j + 1) * PB, k);
  g.l = st->sub_l[j];
  return g;
}
constexpr int TW_COLS = 32;   // columns per W work unit
constexpr int TW_SUB = 32;    // rows staged per pass
constexpr int TU_ROWS = 64;   // update tile rows
constexpr int TU_COLS = 64;   // update tile cols
constexpr int TU_KC = 32;     // reflectors per staged chunk

__device__ __forceinline__ double vget(const double* A, int64_t lda, int64_t ns, int64_t r, int t) {
  // V(r, t), r relative to ns
  if (r < t) return 0.0;
  if (r == t) return 1.0;
  return A[(ns + t) * lda + ns + r];
}

// number of row chunks for the W phase (same on every CTA)
__device__ __forceinline__ int64_t wchunk_rows(int64_t mr, int64_t ncoltiles, int wchunks, int target_units) {
  int64_t want = (target_units + ncoltiles - 1) / ncoltiles;
  if (want > wchunks) want = wchunks;
  if (want < 1) want = 1;
  int64_t rows = (mr + want - 1) / want;
  rows = (rows + TW_SUB - 1) / TW_SUB * TW_SUB;
  if (rows < TW_SUB) rows = TW_SUB;
  return rows;
}

// Thread layout of the W phase: TG reflector groups x (256/TG) columns; each
// thread accumulates NQ = ceil(l/TG) reflectors of one column, so no FMA slot
// is wasted on reflectors past l (a predicated-off FFMA64 still costs issue).
__device__ __forceinline__ int w_tg(int l) { return l >= 8 ? 8 : (l >= 4 ? 4 : (l >= 2 ? 2 : 1)); }

struct WGeom {
  int64_t nct, rows_per, nrc;
  int cols;
  // partial W of row chunk q, reflector t, column c at Wp[q qstride + t tstride + c - cofs]
  int64_t qstride, tstride, cofs;
  bool narrow;  // the packed 64-column layout of a merged form's panel columns
};

// Columns of a sub-panel's W pass (j >= 0, every form but the FP32-class
// one): first the sub-panel's own l accepted columns, read as V (so their
// partials sum to S = V^T V, which replaces the compact-WY T), then the
// columns it updates, [c0, cend).  Logical column c maps to a matrix column.
struct WCols {
  int64_t r0, c0;  // first sub-panel column, first updated column
  int ns;          // S columns in front (0: none)
  __device__ __forceinline__ int64_t phys(int64_t c) const { return c < ns ? r0 + c : c0 + (c - ns); }
};

__device__ __forceinline__ bool w_has_s(const Params& P, int j) { return j >= 0 && !P.mixed; }

// sub-panel updates of the merged form reach at most 64 columns (the rest of
// the panel): more row chunks keep the SMs busy, their partials packed 64
// columns wide so that up to wchunks * n / 64 of them fit the buffer
constexpr int NARROW_WCHUNKS = 128;
constexpr int NARROW_COLS = 64;

// Row chunks of k_trail_w32: passes of at least S32_ROWS rows (one staged V
// block per pass), at most wchunks of them.
__device__ __forceinline__ int64_t w32_rows_per(const Params& P, int64_t mr);

// n2: columns of the pass; narrow_c0 >= 0: the pass covers matrix columns
// [narrow_c0, narrow_c0 + span) of a merged form's panel, packed 64 wide
__device__ __forceinline__ WGeom w_geom(const Params& P, int l, int64_t n2, int64_t mr, int64_t narrow_c0 = -1,
                                        int64_t span = 0) {
  WGeom g;
  g.qstride = (int64_t)P.kmax * P.n;
  g.tstride = P.n;
  g.cofs = 0;
  g.narrow = false;
  if (P.mixed) {
    g.cols = 0;
    g.nct = 0;
    g.rows_per = w32_rows_per(P, mr);
    g.nrc = (mr + g.rows_per - 1) / g.rows_per;
    return g;
  }
  g.cols = GEMM_THREADS / w_tg(l);
  g.nct = (n2 + g.cols - 1) / g.cols;
  int cap = P.wchunks;
  const int64_t fit = (int64_t)P.wchunks * P.n / NARROW_COLS;  // packed chunks the buffer holds
  if (narrow_c0 >= 0 && span <= NARROW_COLS && fit >= 1) {
    cap = (int)min((int64_t)NARROW_WCHUNKS, fit);
    g.qstride = (int64_t)P.kmax * NARROW_COLS;
    g.tstride = NARROW_COLS;
    g.cofs = narrow_c0;
    g.narrow = true;
  }
  g.rows_per = wchunk_rows(mr, g.nct, cap, P.w_units);
  g.nrc = (mr + g.rows_per - 1) / g.rows_per;
  return g;
}

template <int TG, int NQ, typename TC>
__device__ __forceinline__ void trail_w_body(const Params& P, double* smem, int l, int64_t ns, const WCols& wc,
                                             int64_t mr, const WGeom& g, int64_t ncol_all) {
  constexpr int COLS = GEMM_THREADS / TG;
  constexpr int LDA_S = COLS + 1;
  constexpr int LDV_S = KMAX + 1;
  TC* s_a = reinterpret_cast<TC*>(smem);  // [TW_SUB][COLS + 1]
  TC* s_v = s_a + TW_SUB * LDA_S;         // [TW_SUB][KMAX + 1]
  const int64_t lda = P.lda;
  const int tid = threadIdx.x;
  const int c = tid % COLS, tg = tid / COLS;
  const int64_t units = g.nct * g.nrc;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t ct = u % g.nct, rc = u / g.nct;
    const int64_t cbase = ct * COLS;  // logical
    const int ncols = (int)min((int64_t)COLS, ncol_all - cbase);
    const int64_t rbeg = rc * g.rows_per, rend = min(mr, rbeg + g.rows_per);
    TC acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = (TC)0;
    // Software pipeline (l >= 4, TG >= 4): the elements of pass r0 + TW_SUB
    // are loaded into registers while pass r0 is computed from shared memory,
    // so the global load latency hides behind the FMAs (each thread holds AE
    // elements of A and VE of V).  Tiny blocks (TG < 4) stage directly.
    constexpr bool PIPE = TG >= 4 && NQ <= 4;  // the sub-panel updates (l <= 16)
    constexpr int AE = PIPE ? TW_SUB * COLS / GEMM_THREADS : 1;                          // 32 / TG
    constexpr int VE = PIPE ? (TW_SUB * TG * NQ + GEMM_THREADS - 1) / GEMM_THREADS : 1;  // l <= TG NQ
    double ra[AE], rv[VE];
    auto load_pass = [&](int64_t p0) {
      const int prow = (int)min((int64_t)TW_SUB, rend - p0);
#pragma unroll
      for (int k = 0; k < AE; ++k) {
        const int e = tid + k * GEMM_THREADS;
        const int cc = e / TW_SUB, rr = e % TW_SUB;
        double v = 0.0;
        if (rr < prow && cc < ncols) {
          const int64_t cl = cbase + cc;
          v = (cl < wc.ns) ? vget(P.A, lda, ns, p0 + rr, (int)cl) : P.A[wc.phys(cl) * lda + ns + p0 + rr];
        }
        ra[k] = v;
      }
#pragma unroll
      for (int k = 0; k < VE; ++k) {
        const int e = tid + k * GEMM_THREADS;
        const int t = e / TW_SUB, rr = e % TW_SUB;
        rv[k] = (t < l && rr < prow) ? vget(P.A, lda, ns, p0 + rr, t) : 0.0;
      }
    };
    if (PIPE) load_pass(rbeg);
    for (int64_t r0 = rbeg; r0 < rend; r0 += TW_SUB) {
      const int rows = (int)min((int64_t)TW_SUB, rend - r0);
      __syncthreads();  // the previous pass is done with shared memory
      if (PIPE) {
#pragma unroll
        for (int k = 0; k < AE; ++k) {
          const int e = tid + k * GEMM_THREADS;
          s_a[(e % TW_SUB) * LDA_S + e / TW_SUB] = (TC)ra[k];
        }
#pragma unroll
        for (int k = 0; k < VE; ++k) {
          const int e = tid + k * GEMM_THREADS;
          if (e / TW_SUB < l) s_v[(e % TW_SUB) * LDV_S + e / TW_SUB] = (TC)rv[k];
        }
      } else {
        for (int e = tid; e < TW_SUB * COLS; e += GEMM_THREADS) {
          const int cc = e / TW_SUB, rr = e % TW_SUB;
          double v = 0.0;
          if (rr < rows && cc < ncols) {
            const int64_t cl = cbase + cc;
            v = (cl < wc.ns) ? vget(P.A, lda, ns, r0 + rr, (int)cl) : P.A[wc.phys(cl) * lda + ns + r0 + rr];
          }
          s_a[rr * LDA_S + cc] = (TC)v;
        }
        for (int e = tid; e < TW_SUB * l; e += GEMM_THREADS) {
          const int t = e / TW_SUB, rr = e % TW_SUB;
          s_v[rr * LDV_S + t] = (TC)((rr < rows) ? vget(P.A, lda, ns, r0 + rr, t) : 0.0);
        }
      }
      __syncthreads();
      if (PIPE && r0 + TW_SUB < rend) load_pass(r0 + TW_SUB);
      for (int rr = 0; rr < rows; ++rr) {
        const TC a = s_a[rr * LDA_S + c];
        const TC* vr = s_v + rr * LDV_S + tg;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          if (q < NQ - 1 || tg + q * TG < l) acc[q] = fmat(vr[q * TG], a, acc[q]);
        }
      }
    }
    if (c < ncols) {
      double* out = P.Wp + rc * g.qstride;
      const int64_t pc = wc.phys(cbase + c) - g.cofs;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int t = tg + q * TG;
        if (t < l) out[(int64_t)t * g.tstride + pc] = (double)acc[q];
      }
    }
  }
}

constexpr int TRAIL_W_SMEM = (TW_SUB * (GEMM_THREADS + 1) + TW_SUB * (KMAX + 1)) * (int)sizeof(double);

template <typename TC>
__device__ __forceinline__ void trail_w_kernel(Params& P, int j) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t ns = sg.r0;  // base row/column of V
  const int64_t j0 = sg.c0;
  const int64_t cend = trail_end(P, st, j);
  const int64_t n2 = cend - j0, mr = P.m - ns;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  WCols wc;
  wc.r0 = ns;
  wc.c0 = j0;
  wc.ns = w_has_s(P, j) ? l : 0;
  const int64_t ncol_all = wc.ns + n2;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TRAIL_W, 2.0 * (double)mr * (double)ncol_all * l);
  extern __shared__ double smw[];
  const WGeom g = w_geom(P, l, ncol_all, mr, (P.merged && j >= 0) ? ns : -1, cend - ns);
  const int tg = w_tg(l);
  const int nq = (l + tg - 1) / tg;
  if (tg == 1) {
    trail_w_body<1, 1, TC>(P, smw, l, ns, wc, mr, g, ncol_all);
  } else if (tg == 2) {
    if (nq == 1) trail_w_body<2, 1, TC>(P, smw, l, ns, wc, mr, g, ncol_all);
    else trail_w_body<2, 2, TC>(P, smw, l, ns, wc, mr, g, ncol_all);
  } else if (tg == 4) {
    if (nq == 1) trail_w_body<4, 1, TC>(P, smw, l, ns, wc, mr, g, ncol_all);
    else trail_w_body<4, 2, TC>(P, smw, l, ns, wc, mr, g, ncol_all);
  } else {
    switch (nq) {
      case 1: trail_w_body<8, 1, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 2: trail_w_body<8, 2, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 3: trail_w_body<8, 3, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 4: trail_w_body<8, 4, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 5: trail_w_body<8, 5, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 6: trail_w_body<8, 6, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 7: trail_w_body<8, 7, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 8: trail_w_body<8, 8, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 9: trail_w_body<8, 9, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 10: trail_w_body<8, 10, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 11: trail_w_body<8, 11, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 12: trail_w_body<8, 12, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 13: trail_w_body<8, 13, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 14: trail_w_body<8, 14, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      case 15: trail_w_body<8, 15, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
      default: trail_w_body<8, 16, TC>(P, smw, l, ns, wc, mr, g, ncol_all); break;
    }
  }
}

__global__ void __launch_bounds__(GEMM_THREADS) k_trail_w(Params P, int j) { trail_w_kernel<double>(P, j); }

// The narrow sub-panel updates of the merged forms split their W pass into
// up to NARROW_WCHUNKS row chunks (so that every SM works on a 64-column
// span): their partials are first summed into chunk 0 by many CTAs, 8
// threads per entry each adding a contiguous eighth of the chunks in order,
// then the eight sums in order (a fixed result), and k_trail_wreduce reads
// one chunk.  Entry (t, pc): reflector t, packed column pc of the span.
constexpr int WPRE_MIN_CHUNKS = 24;  // fewer row chunks are summed by k_trail_wreduce itself
__device__ __forceinline__ bool wpre_used(const Params& P, const WGeom& g, int j) {
  return P.merged && j >= 0 && g.narrow && g.nrc >= WPRE_MIN_CHUNKS;
}

__global__ void __launch_bounds__(256) k_trail_wpresum(Params P, int j) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t cend = trail_end(P, st, j);
  const int64_t n2 = cend - sg.c0, mr = P.m - sg.r0;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  const WGeom g = w_geom(P, l, l + n2, mr, sg.r0, cend - sg.r0);
  if (!wpre_used(P, g, j)) return;
  const int64_t span = cend - sg.r0;
  const int64_t nent = (int64_t)l * span;
  __shared__ double s_part[32][9];
  const int le = threadIdx.x >> 3, h = threadIdx.x & 7;
  const int64_t per = (g.nrc + 7) / 8;
  for (int64_t e0 = (int64_t)blockIdx.x * 32; e0 < nent; e0 += (int64_t)gridDim.x * 32) {
    const int64_t e = e0 + le;
    const int64_t t = e / span, pc = e % span;
    const int64_t c0 = h * per, c1 = min(g.nrc, c0 + per);
    double* base = P.Wp + t * g.tstride + pc;
    s_part[le][h] = (e < nent && c1 > c0) ? sum_strided(base + c0 * g.qstride, g.qstride, c1 - c0) : 0.0;
    __syncthreads();
    if (h == 0 && e < nent) {
      double v = 0.0;
      for (int q = 0; q < 8; ++q) v += s_part[le][q];
      base[0] = v;  // chunk 0
    }
    __syncthreads();
  }
}

// W = T^T sum(partials), the partials of k_trail_w's row chunks.  For a
// sub-panel (j >= 0, every form but the FP32-class one) T is not formed:
// with S = V^T V from the W pass, T^-1 = strict_upper(S) + diag(1/htau)
// (Schreiber & Van Loan's compact WY in the inverse form of Puglisi), so
// W solves (T^-1)^T W = V^T A by forward substitution,
//   W_t = htau_t (P_t - sum_{q<t} S_qt W_q),
// which a zero htau_t (H_t = I) turns into W_t = 0 as T's zero column would.
__global__ void __launch_bounds__(GEMM_THREADS) k_trail_wreduce(Params P, int j) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t j0 = sg.c0;
  const int64_t cend = trail_end(P, st, j);
  const int64_t n2 = cend - j0, mr = P.m - sg.r0;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  const bool use_s = w_has_s(P, j);
  const int nsx = use_s ? l : 0;
  const int64_t nct = (n2 + TW_COLS - 1) / TW_COLS;
  // the row chunks of k_trail_w (k_trail_w32 in the FP32-class form)
  const WGeom g = w_geom(P, l, nsx + n2, mr, (P.merged && j >= 0) ? sg.r0 : -1, cend - sg.r0);
  const int64_t nrc = wpre_used(P, g, j) ? 1 : g.nrc;  // k_trail_wpresum summed them into chunk 0
  if (blockIdx.x == 0 && threadIdx.x == 0)
    add_flops(st, KID_TRAIL_WREDUCE, (double)n2 * l * ((double)(nrc - 1) + (l + 1.0)));
  __shared__ double s_w[KMAX][TW_COLS + 1];
  __shared__ double s_S[PB][PB + 1];
  __shared__ double s_tau[PB];
  const int tid = threadIdx.x;
  const int c = tid % TW_COLS, tg = tid / TW_COLS, TG = GEMM_THREADS / TW_COLS;
  if (use_s) {  // S_qt = v_q^T v_t (q < t < l <= PB) and htau, once per CTA
    for (int e = tid; e < l * l; e += GEMM_THREADS) {
      const int q = e / l, t = e % l;
      s_S[q][t] = (q < t) ? sum_strided(P.Wp + (int64_t)q * g.tstride + sg.r0 + t - g.cofs, g.qstride, nrc) : 0.0;
    }
    if (tid < l) s_tau[tid] = P.htau[sg.r0 + tid];
  }
  for (int64_t ct = blockIdx.x; ct < nct; ct += gridDim.x) {
    const int64_t cbase = j0 + ct * TW_COLS;
    const bool ok = (cbase + c) < cend;
    __syncthreads();
    for (int t = tg; t < l; t += TG) {
      s_w[t][c] = ok ? sum_strided(P.Wp + (int64_t)t * g.tstride + cbase + c - g.cofs, g.qstride, nrc) : 0.0;
    }
    __syncthreads();
    if (use_s) {
      if (tg == 0) {  // one thread per column, t ascending
        for (int t = 0; t < l; ++t) {
          double sv = s_w[t][c];
          for (int q = 0; q < t; ++q) sv = fma(-s_S[q][t], s_w[q][c], sv);
          sv *= s_tau[t];
          s_w[t][c] = sv;
          if (ok) P.W[(int64_t)t * P.n + cbase + c] = sv;
        }
      }
    } else {
      for (int t = tg; t < l; t += TG) {
        // (T^T W)_t = sum_{q <= t} T(q, t) W_q
        double sv = 0.0;
        const double* Tc = P.T + (int64_t)t * KMAX;
        for (int q = 0; q <= t; ++q) sv = fma(Tc[q], s_w[q][c], sv);
        if (ok) P.W[(int64_t)t * P.n + cbase + c] = sv;
      }
    }
  }
}

// part (sub-panels, j >= 0): 0 every column right of the sub-panel; 1 only
// the next sub-panel's columns (what its panel needs first); 2 the others.
// Parts 1 and 2 together make part 0, so part 2 may run beside the next
// sub-panel's panel.
__device__ __forceinline__ void update_range(const Params& P, const DevState* st, int j, int part, int64_t* c0,
                                             int64_t* cend) {
  const SubGeom sg = sub_geom(st, j);
  *c0 = sg.c0;
  *cend = trail_end(P, st, j);
  if (part == 0 || j < 0) return;
  // the next sub-panel's columns, when one follows
  const int64_t split = st->sub_next[j] ? min(*cend, st->ns + min((int64_t)(j + 2) * PB, (int64_t)st->k)) : *c0;
  if (part == 1) *cend = split;
  else *c0 = split;
}

// A[rows, cols] -= V W in tiles of TU_ROWS x TCN (TCN = 64 or 32), 16 x 16
// threads with 4 x (TCN / 16) outputs each, reflectors staged TU_KC at a time
template <typename TC, int TCN>
__device__ __forceinline__ void trail_update_tiles(Params& P, int l, int64_t ns, int64_t j0, int64_t cend,
                                                   int64_t mr, TC (*s_v)[TU_ROWS], TC (*s_w)[TU_COLS]) {
  constexpr int NJ = TCN / 16;
  const int64_t lda = P.lda;
  const int64_t n2 = cend - j0;
  const int64_t nrt = (mr + TU_ROWS - 1) / TU_ROWS;
  const int64_t nct = (n2 + TCN - 1) / TCN;
  const int64_t units = nrt * nct;
  const int tid = threadIdx.x;
  const int tr = tid % 16, tc = tid / 16;  // 16 x 16 threads
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t rt = u % nrt, ct = u / nrt;
    const int64_t rbase = rt * TU_ROWS;  // relative to ns
    const int64_t cbase = j0 + ct * TCN;
    TC acc[4][NJ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) acc[i][jj] = (TC)0;
    for (int t0 = 0; t0 < l; t0 += TU_KC) {
      const int kcnt = min(TU_KC, l - t0);
      __syncthreads();
      for (int e = tid; e < TU_KC * TU_ROWS; e += GEMM_THREADS) {
        int t = e / TU_ROWS, r = e % TU_ROWS;
        double v = 0.0;
        if (t < kcnt && rbase + r < mr) v = vget(P.A, lda, ns, rbase + r, t0 + t);
        s_v[t][r] = (TC)v;
      }
      for (int e = tid; e < TU_KC * TCN; e += GEMM_THREADS) {
        int t = e / TCN, c = e % TCN;
        double v = 0.0;
        if (t < kcnt && cbase + c < cend) v = P.W[(int64_t)(t0 + t) * P.n + cbase + c];
        s_w[t][c] = (TC)v;
      }
      __syncthreads();
      for (int t = 0; t < kcnt; ++t) {
        TC vv[4], ww[NJ];
#pragma unroll
        for (int i = 0; i < 4; ++i) vv[i] = s_v[t][tr + 16 * i];
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) ww[jj] = s_w[t][tc + 16 * jj];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < NJ; ++jj) acc[i][jj] = fmat(vv[i], ww[jj], acc[i][jj]);
      }
    }
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const int64_t col = cbase + tc + 16 * jj;
      if (col >= cend) continue;
      double* a = P.A + col * lda + ns;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t r = rbase + tr + 16 * i;
        if (r < mr) a[r] -= (double)acc[i][jj];
      }
    }
  }
}

template <typename TC>
__device__ __forceinline__ void trail_update_kernel(Params& P, int j, int part) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t ns = sg.r0, m = P.m;
  int64_t j0, cend;
  update_range(P, st, j, part, &j0, &cend);
  const int64_t n2 = cend - j0, mr = m - ns;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TRAIL_UPDATE, 2.0 * (double)mr * (double)n2 * l);
  __shared__ TC s_v[TU_KC][TU_ROWS];
  __shared__ TC s_w[TU_KC][TU_COLS];
  // tiles 32 columns wide when 64-wide ones would not fill one wave (the
  // narrow updates of the panel's own columns): twice the CTAs, less of each
  // tile past the last column; every element is summed in the same order
  const int64_t nrt = (mr + TU_ROWS - 1) / TU_ROWS;
  if (nrt * ((n2 + 63) / 64) < (int64_t)gridDim.x)
    trail_update_tiles<TC, 32>(P, l, ns, j0, cend, mr, s_v, s_w);
  else
    trail_update_tiles<TC, 64>(P, l, ns, j0, cend, mr, s_v, s_w);
}

__global__ void __launch_bounds__(GEMM_THREADS) k_trail_update(Params P, int j, int part) {
  trail_update_kernel<double>(P, j, part);
}

// ---------------------------------------------------------------------------
// a9, FP32-class form.  With l <= PB = 16 reflectors per pass the update moves
// 8 (W) + 16 (update) bytes of FP64 per element for 4 l flops: HBM-bound on
// FP32 CUDA cores, so the kernels are built for streaming, not for tensor
// cores: one warp per column, lanes stride the rows (coalesced 8-byte loads,
// several in flight per lane), V staged in shared memory as FP32 rows of PB,
// products and sums in FP32, the result written back in FP64.
// ---------------------------------------------------------------------------
constexpr int S32_ROWS = 1024;  // rows of V staged per pass

__device__ __forceinline__ int64_t w32_rows_per(const Params& P, int64_t mr) {
  int64_t r = (mr + P.wchunks - 1) / P.wchunks;
  r = (r + 31) / 32 * 32;
  return r < S32_ROWS ? S32_ROWS : r;
}
constexpr int S32_COLS = 64;    // columns per work unit (8 warps x 8 columns)
constexpr int S32_SMEM = S32_ROWS * PB * (int)sizeof(float);

// V rows [rs, rs + rows) of the sub-panel as FP32, row-major with PB columns
__device__ __forceinline__ void stage_v32(const Params& P, float* s_v, int64_t base, int64_t rs, int rows, int l) {
  for (int e = threadIdx.x; e < rows * PB; e += GEMM_THREADS) {
    const int rr = e % rows, t = e / rows;  // consecutive threads: consecutive rows of one column
    float v = 0.f;
    if (t < l) v = f64_to_f32_rn(vget(P.A, P.lda, base, rs + rr, t));
    s_v[rr * PB + t] = v;
  }
}

constexpr int W32_CPW = 4;                     // columns per warp in k_trail_w32
constexpr int W32_COLS = 8 * W32_CPW;          // columns per work unit

__global__ void __launch_bounds__(GEMM_THREADS, 2) k_trail_w32(Params P, int j) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t base = sg.r0, j0 = sg.c0;
  const int64_t n2 = P.n - j0, mr = P.m - base;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TRAIL_W, 2.0 * (double)mr * (double)n2 * l);
  extern __shared__ float s32[];
  float* s_v = s32;  // [S32_ROWS][PB]
  const WGeom g = w_geom(P, l, n2, mr);  // row chunks shared with k_trail_wreduce
  const int64_t ncb = (n2 + W32_COLS - 1) / W32_COLS;
  const int64_t units = g.nrc * ncb;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  // contiguous unit ranges per CTA: consecutive units share a row chunk
  const int64_t ub = units * blockIdx.x / gridDim.x, ue = units * (blockIdx.x + 1) / gridDim.x;
  int64_t staged_rs = -1;  // first row of the V block now in shared memory
  for (int64_t u = ub; u < ue; ++u) {
    const int64_t rc = u / ncb, cb = u % ncb;
    const int64_t rbeg = rc * g.rows_per, rend = min(mr, rbeg + g.rows_per);
    const int64_t col0 = j0 + cb * W32_COLS + wp * W32_CPW;
    int ncol = (int)min((int64_t)W32_CPW, P.n - col0);
    if (ncol < 0) ncol = 0;
    const double* a[W32_CPW];
#pragma unroll
    for (int c = 0; c < W32_CPW; ++c) a[c] = P.A + (col0 + (c < ncol ? c : 0)) * P.lda + base;
    float acc[W32_CPW][PB];
#pragma unroll
    for (int c = 0; c < W32_CPW; ++c)
#pragma unroll
      for (int t = 0; t < PB; ++t) acc[c][t] = 0.f;
    for (int64_t rs = rbeg; rs < rend; rs += S32_ROWS) {
      const int rows = (int)min((int64_t)S32_ROWS, rend - rs);
      if (rs != staged_rs) {  // uniform across the CTA; consecutive units share a pass
        __syncthreads();
        stage_v32(P, s_v, base, rs, rows, l);
        __syncthreads();
        staged_rs = rs;
      }
      if (ncol > 0) {
        // rows outer, two rows per lane per pass: W32_CPW x 2 loads in flight
        for (int r = lane; r < rows; r += 64) {
          const bool two = (r + 32 < rows);
          double x0[W32_CPW], x1[W32_CPW];
#pragma unroll
          for (int c = 0; c < W32_CPW; ++c) {
            x0[c] = a[c][rs + r];
            x1[c] = two ? a[c][rs + r + 32] : 0.0;
          }
          float y0[W32_CPW], y1[W32_CPW];
#pragma unroll
          for (int c = 0; c < W32_CPW; ++c) {
            y0[c] = f64_to_f32_rn(x0[c]);
            y1[c] = f64_to_f32_rn(x1[c]);
          }
          const float4* v0 = reinterpret_cast<const float4*>(s_v + r * PB);
          const float4* v1 = reinterpret_cast<const float4*>(s_v + (two ? r + 32 : r) * PB);
#pragma unroll
          for (int q = 0; q < PB / 4; ++q) {
            const float4 p0 = v0[q];
            const float4 p1 = two ? v1[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < W32_CPW; ++c) {
              acc[c][4 * q + 0] = fmaf(p1.x, y1[c], fmaf(p0.x, y0[c], acc[c][4 * q + 0]));
              acc[c][4 * q + 1] = fmaf(p1.y, y1[c], fmaf(p0.y, y0[c], acc[c][4 * q + 1]));
              acc[c][4 * q + 2] = fmaf(p1.z, y1[c], fmaf(p0.z, y0[c], acc[c][4 * q + 2]));
              acc[c][4 * q + 3] = fmaf(p1.w, y1[c], fmaf(p0.w, y0[c], acc[c][4 * q + 3]));
            }
          }
        }
      }
    }
    // reduce over lanes and store this row chunk's partial W (FP64)
    double* out = P.Wp + rc * (int64_t)P.kmax * P.n;
#pragma unroll
    for (int c = 0; c < W32_CPW; ++c) {
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        float v = acc[c][t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && t < l && c < ncol) out[(int64_t)t * P.n + col0 + c] = (double)v;
      }
    }
  }
}

__global__ void __launch_bounds__(GEMM_THREADS, 2) k_trail_update32(Params P, int j) {
  DevState* st = P.st;
  if (st->done) return;
  const SubGeom sg = sub_geom(st, j);
  const int l = sg.l;
  const int64_t base = sg.r0, j0 = sg.c0;
  const int64_t n2 = P.n - j0, mr = P.m - base;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TRAIL_UPDATE, 2.0 * (double)mr * (double)n2 * l);
  extern __shared__ float s32[];
  float* s_v = s32;  // [S32_ROWS][PB]
  const int64_t nrb = (mr + S32_ROWS - 1) / S32_ROWS;
  const int64_t ncb = (n2 + W32_COLS - 1) / W32_COLS;
  const int64_t units = nrb * ncb;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t ub = units * blockIdx.x / gridDim.x, ue = units * (blockIdx.x + 1) / gridDim.x;
  int64_t staged_rb = -1;
  for (int64_t u = ub; u < ue; ++u) {
    const int64_t rb = u / ncb, cb = u % ncb;
    const int64_t rs = rb * S32_ROWS;
    const int rows = (int)min((int64_t)S32_ROWS, mr - rs);
    if (rb != staged_rb) {  // uniform across the CTA
      __syncthreads();
      stage_v32(P, s_v, base, rs, rows, l);
      __syncthreads();
      staged_rb = rb;
    }
    const int64_t col0 = j0 + cb * W32_COLS + wp * W32_CPW;
    int ncol = (int)min((int64_t)W32_CPW, P.n - col0);
    if (ncol <= 0) continue;
    // this warp's W columns (FP32, in registers)
    float wv[W32_CPW][PB];
#pragma unroll
    for (int c = 0; c < W32_CPW; ++c)
#pragma unroll
      for (int t = 0; t < PB; ++t)
        wv[c][t] = (t < l && c < ncol) ? f64_to_f32_rn(P.W[(int64_t)t * P.n + col0 + c]) : 0.f;
    double* a[W32_CPW];
#pragma unroll
    for (int c = 0; c < W32_CPW; ++c) a[c] = P.A + (col0 + (c < ncol ? c : 0)) * P.lda + base + rs;
    for (int r = lane; r < rows; r += 64) {  // two rows per lane: 8 loads in flight
      const bool two = (r + 32 < rows);
      double x0[W32_CPW], x1[W32_CPW];
#pragma unroll
      for (int c = 0; c < W32_CPW; ++c) {
        x0[c] = (c < ncol) ? a[c][r] : 0.0;
        x1[c] = (two && c < ncol) ? a[c][r + 32] : 0.0;
      }
      float d0[W32_CPW], d1[W32_CPW];
#pragma unroll
      for (int c = 0; c < W32_CPW; ++c) d0[c] = d1[c] = 0.f;
      const float4* v0 = reinterpret_cast<const float4*>(s_v + r * PB);
      const float4* v1 = reinterpret_cast<const float4*>(s_v + (two ? r + 32 : r) * PB);
#pragma unroll
      for (int q = 0; q < PB / 4; ++q) {
        const float4 p0 = v0[q], p1 = v1[q];
#pragma unroll
        for (int c = 0; c < W32_CPW; ++c) {
          d0[c] = fmaf(p0.x, wv[c][4 * q + 0], d0[c]);
          d0[c] = fmaf(p0.y, wv[c][4 * q + 1], d0[c]);
          d0[c] = fmaf(p0.z, wv[c][4 * q + 2], d0[c]);
          d0[c] = fmaf(p0.w, wv[c][4 * q + 3], d0[c]);
          d1[c] = fmaf(p1.x, wv[c][4 * q + 0], d1[c]);
          d1[c] = fmaf(p1.y, wv[c][4 * q + 1], d1[c]);
          d1[c] = fmaf(p1.z, wv[c][4 * q + 2], d1[c]);
          d1[c] = fmaf(p1.w, wv[c][4 * q + 3], d1[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < W32_CPW; ++c) {
        if (c < ncol) {
          a[c][r] = x0[c] - f32_to_f64(d0[c]);
          if (two) a[c][r + 32] = x1[c] - f32_to_f64(d1[c]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// a10/a11: partial norm update.  One warp per column j >= ns + l:
//   rejected panel columns (ns+l <= j < ns+k): recompute;
//   trailing columns: block downdate over rows ns..ns+l-1, recompute when
//   t (u/uref)^2 <= sqrt(u_upd), u_upd the unit roundoff of the trailing
//   update (eps in the FP64 forms).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_downdate(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l, k = st->k;
  const int64_t ns = st->ns, m = P.m, lda = P.lda;
  const int64_t nsn = ns + l;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const double sqeps = P.sqeps_dd;
  int nrec = 0;
  for (int64_t j = ns + gw; j < P.n; j += nwarps) {
    const double* a = P.A + j * lda;
    if (j < nsn) {
      if (lane == 0) P.u[j] = 0.0;
      continue;
    }
    bool recompute = (j < ns + k);
    double uj = P.u[j];
    double t = 0.0;
    if (!recompute) {
      if (uj == 0.0) continue;
      double q = 0.0;
      for (int64_t r = ns + lane; r < nsn; r += 32) {
        double x = a[r] / uj;
        q = fma(x, x, q);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      t = 1.0 - q;
      if (t < 0.0) t = 0.0;
      double ratio = uj / P.uref[j];
      double test = t * ratio * ratio;
      recompute = (test <= sqeps);
    }
    if (recompute) {
      double s = 0.0;
      for (int64_t r = nsn + lane; r < m; r += 32) s = fma(a[r], a[r], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        double nr = sqrt(s);
        P.u[j] = nr;
        P.uref[j] = nr;
        ++nrec;
      }
    } else if (lane == 0) {
      P.u[j] = uj * sqrt(t);
    }
  }
  if (lane == 0 && nrec && P.trace && st->step < P.trace_cap)
    atomicAdd((unsigned long long*)&P.trace[st->step].nrecomp, (unsigned long long)nrec);
  if (lane == 0 && nrec) add_flops(st, KID_DOWNDATE, 2.0 * (double)(m - nsn) * nrec);
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_DOWNDATE, 3.0 * (double)l * (double)(P.n - ns - k));
}

// ---------------------------------------------------------------------------
// Single-column pivoting steps (k = 1: every step once DM is off, or
// k_max = 1 throughout) fused into one cooperative persistent kernel.  Per
// step every CTA computes the argmax and the reflector redundantly (same data,
// same order, so the same result), then CTA (c mod G) owns trailing position c:
// it applies H to that column and updates its partial norm.  Two grid barriers
// per step: after all CTAs have read the pivot column, and after all updates.
// ---------------------------------------------------------------------------
constexpr int QRP_THREADS = 256;
constexpr int QRP_OWN_MAX = 512;  // trailing columns one CTA of the single-column kernel owns, at most

// Grid-wide barrier for a cooperative launch: arrival counter with release,
// polling with acquire, bounded by limit_ns of the global timer.  Returns
// false (and raises the abort flag) when the wait gave up or another CTA's
// did; every CTA then leaves its loop.
__device__ __forceinline__ bool grid_barrier(DevState* st, unsigned int target, int64_t step, int64_t ns,
                                             int64_t limit_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* ctr = &st->gbar;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
    const unsigned long long t0 = gtimer_ns();
    unsigned int cur = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(ctr) : "memory");
      if ((int)(cur - target) >= 0) break;
      if (*(volatile int32_t*)&st->abort_flag) break;
      if ((int64_t)(gtimer_ns() - t0) > limit_ns) {
        record_fail(st, FAIL_GRID_BARRIER, (int)blockIdx.x, step, ns, (int64_t)cur);
        break;
      }
      __nanosleep(64);
    }
  }
  __syncthreads();
  return *(volatile int32_t*)&st->abort_flag == 0;
}

__device__ __forceinline__ void qrp_block_argmax(const double* u, int64_t ns, int64_t n, double* s_v, int64_t* s_p,
                                                 double* mu_out, int64_t* j_out) {
  // integer keys of the non-negative partial norms (the compares stay off the FP64 pipe);
  // s_v holds the keys' bit patterns
  long long* s_k = reinterpret_cast<long long*>(s_v);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  long long bk = -1;
  int64_t bp = INT64_MAX;
  for (int64_t j = ns + tid; j < n; j += QRP_THREADS) {
    const long long x = ukey(u[j]);
    if (kbetter_u(x, j, bk, bp)) {
      bk = x;
      bp = j;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
    const int64_t op = __shfl_xor_sync(0xffffffffu, bp, o);
    if (kbetter_u(ok, op, bk, bp)) {
      bk = ok;
      bp = op;
    }
  }
  if (lane == 0) {
    s_k[w] = bk;
    s_p[w] = bp;
  }
  __syncthreads();
  if (tid == 0) {
    bk = s_k[0];
    bp = s_p[0];
    for (int q = 1; q < QRP_THREADS / 32; ++q)
      if (kbetter_u(s_k[q], s_p[q], bk, bp)) {
        bk = s_k[q];
        bp = s_p[q];
      }
    s_k[QRP_THREADS / 32] = bk;
    s_p[QRP_THREADS / 32] = bp;
  }
  __syncthreads();
  *mu_out = __longlong_as_double(s_k[QRP_THREADS / 32]);
  *j_out = s_p[QRP_THREADS / 32];
  __syncthreads();
}

__global__ void __launch_bounds__(QRP_THREADS, 1) k_qrp_tail(Params P) {
  DevState* st = P.st;
  extern __shared__ double s_x[];  // pivot column rows ns..m-1
  __shared__ double s_v[QRP_THREADS / 32 + 1];
  __shared__ int64_t s_p[QRP_THREADS / 32 + 1];
  __shared__ double s_sc[8];
  __shared__ double s_red[QRP_THREADS / 32];
  __shared__ double s_rr[QRP_OWN_MAX];  // the updated row-ns entries of this CTA's columns
  __shared__ int s_rrec[QRP_OWN_MAX];   // 1: the column's norm is recomputed exactly
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int G = (int)gridDim.x, cta = (int)blockIdx.x;
  const int64_t m = P.m, n = P.n, lda = P.lda, kmin = P.kmin;
  double* A = P.A;
  const double sqeps = sqrt(EPS);
  if (st->done) return;  // uniform: read before any CTA writes it
  int64_t ns = st->ns, step = st->step;
  int dm_on = st->dm_on;
  int64_t rank = st->rank, rank_cm = st->rank_colmax;
  const double anorm = __longlong_as_double((long long)st->anorm_bits);
  const double rhs = P.eps1 * anorm;
  double flops = 0.0;
  unsigned int bar = 0;  // barriers passed in this launch
  bar += G;
  // every CTA has read the state (test hook 1: one arrival more than the grid
  // makes, so that this wait runs out)
  if (!grid_barrier(st, bar + (P.test_fault == 1 ? 1u : 0u), step, ns, P.wait_ns)) goto out;
  for (;;) {
    if (ns >= kmin || (P.max_steps > 0 && step >= P.max_steps)) break;
    double mu;
    int64_t jstar;
    qrp_block_argmax(P.u, ns, n, s_v, s_p, &mu, &jstar);
    if (jstar < ns || jstar >= n) {  // identical in every CTA
      if (cta == 0 && tid == 0) record_fail(st, FAIL_PIVOT_RANGE, 0, step, ns, jstar);
      break;
    }
    // stopping test (Sec. 3.4) and the DM safeguard, identical in every CTA
    const int64_t nrem = n - ns;
    if (rank_cm < 0 && mu <= rhs) rank_cm = ns;
    bool stop = false;
    if (rank < 0 && sqrt((double)nrem) * mu <= rhs) {
      rank = ns;
      dm_on = 0;
      if (P.stop_at_rank) stop = true;
    }
    if (stop) break;
    // pivot column into shared memory, its tail norm and the reflector
    const int64_t mr = m - ns;
    const double* xc = A + jstar * lda + ns;
    double part = 0.0;
    for (int64_t i = tid; i < mr; i += QRP_THREADS) {
      const double v = xc[i];
      s_x[i] = v;
      if (i > 0) part = fma(v, v, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_red[wp] = part;
    __syncthreads();
    if (wp == 0) {  // warp 0: beta, then the two quotients at once in lanes 0 and 1
      double s2 = 0.0;
      for (int q = 0; q < QRP_THREADS / 32; ++q) s2 += s_red[q];
      const double alpha = s_x[0];
      const double nrm = sqrt(alpha * alpha + s2);
      const double beta = (s2 == 0.0) ? alpha : ((alpha >= 0.0) ? -nrm : nrm);
      const double qv = ((lane == 0) ? (beta - alpha) : 1.0) / ((lane == 0) ? beta : (alpha - beta));
      const double q1 = __shfl_sync(0xffffffffu, qv, 1);
      if (lane == 0) {
        s_sc[0] = beta;
        s_sc[1] = (s2 == 0.0) ? 0.0 : qv;
        s_sc[2] = (s2 == 0.0) ? 0.0 : q1;
      }
    }
    __syncthreads();
    const double beta = s_sc[0], ht = s_sc[1], rden = s_sc[2];
    const bool app = ht != 0.0;
    // v = x / (alpha - beta) below the pivot, formed once per CTA in shared
    // memory: the owner writes it back, every CTA's updates use it
    if (app)
      for (int64_t i = 1 + tid; i < mr; i += QRP_THREADS) s_x[i] *= rden;
    bar += G;
    if (!grid_barrier(st, bar, step, ns, P.wait_ns)) break;  // all CTAs have read column jstar
    // the owner of position jstar moves the columns: ns <- pivot (R part, beta,
    // v), jstar <- old column ns; it also swaps u, uref and perm
    if ((int)(jstar % G) == cta) {
      double* cn = A + ns * lda;
      double* cj = A + jstar * lda;
      if (jstar != ns) {
        for (int64_t i = tid; i < ns; i += QRP_THREADS) {
          const double a = cj[i], b = cn[i];
          cn[i] = a;
          cj[i] = b;
        }
        for (int64_t i = ns + tid; i < m; i += QRP_THREADS) cj[i] = cn[i];
      }
      __syncthreads();
      for (int64_t i = ns + 1 + tid; i < m; i += QRP_THREADS) cn[i] = s_x[i - ns];
      if (tid == 0) {
        cn[ns] = beta;
        if (jstar != ns) {
          double t = P.u[ns];
          P.u[ns] = P.u[jstar];
          P.u[jstar] = t;
          t = P.uref[ns];
          P.uref[ns] = P.uref[jstar];
          P.uref[jstar] = t;
          const int32_t pt = P.perm[ns];
          P.perm[ns] = P.perm[jstar];
          P.perm[jstar] = pt;
        }
        P.htau[ns] = ht;
        P.u[ns] = 0.0;
        if (P.trace && step < P.trace_cap) {
          StepRecord* r = P.trace + step;
          r->ns = ns;
          r->jstar = jstar;
          r->ncand_all = 0;
          r->ncand = 0;
          r->k = 1;
          r->l = 1;
          r->dm_on = dm_on;
          r->mu = mu;
          r->eps_s = P.tau * mu;
          if (P.traceJ) {
            P.traceJ[step * P.kmax] = P.perm[ns];
            for (int t2 = 1; t2 < P.kmax; ++t2) P.traceJ[step * P.kmax + t2] = -1;
          }
        }
      }
      __syncthreads();
    }
    // every CTA: apply H to its trailing positions (one warp per column),
    // then the partial norms of all of them at once (block downdate with
    // recomputation, l = 1: one thread per column for the scalar part, so its
    // divisions and square root issue once per 32 columns, then one warp per
    // column that needs the exact norm)
    int nrec = 0;
    {
      // first position > ns owned by this CTA, and how many it owns
      const int64_t c_first = ns + 1 + ((cta - (int)((ns + 1) % G)) % G + G) % G;
      const int nown = (c_first < n) ? (int)((n - 1 - c_first) / G + 1) : 0;
      for (int q = wp; q < nown; q += QRP_THREADS / 32) {
        double* ac = A + (c_first + (int64_t)q * G) * lda;
        if (app) {
          double wsum = 0.0;
          for (int64_t i = ns + 1 + lane; i < m; i += 32) wsum = fma(s_x[i - ns], ac[i], wsum);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
          wsum += ac[ns];
          const double hw = ht * wsum;
          for (int64_t i = ns + 1 + lane; i < m; i += 32) ac[i] = fma(-hw, s_x[i - ns], ac[i]);
          __syncwarp();
          if (lane == 0) ac[ns] -= hw;
        }
        if (lane == 0) s_rr[q] = ac[ns];
        __syncwarp();
      }
      __syncthreads();
      for (int q = tid; q < nown; q += QRP_THREADS) {
        const int64_t c = c_first + (int64_t)q * G;
        const double uc = P.u[c];
        int rec = 0;
        if (uc != 0.0) {
          const double x = s_rr[q] / uc;
          double t = 1.0 - x * x;
          if (t < 0.0) t = 0.0;
          const double ratio = uc / P.uref[c];
          if (t * ratio * ratio <= sqeps)
            rec = 1;
          else
            P.u[c] = uc * sqrt(t);
        }
        s_rrec[q] = rec;
      }
      __syncthreads();
      for (int q = wp; q < nown; q += QRP_THREADS / 32) {
        if (!s_rrec[q]) continue;
        const int64_t c = c_first + (int64_t)q * G;
        const double* ac = A + c * lda;
        double sq = 0.0;
        for (int64_t i = ns + 1 + lane; i < m; i += 32) sq = fma(ac[i], ac[i], sq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (lane == 0) {
          const double nr = sqrt(sq);
          P.u[c] = nr;
          P.uref[c] = nr;
          ++nrec;
        }
      }
    }
    if (lane == 0 && nrec && P.trace && step < P.trace_cap)
      atomicAdd((unsigned long long*)&P.trace[step].nrecomp, (unsigned long long)nrec);
    flops += 4.0 * (double)mr * (double)(n - ns - 1) / G + 2.0 * (double)mr;
    bar += G;
    if (!grid_barrier(st, bar, step, ns, P.wait_ns)) break;  // all columns and partial norms updated
    ++ns;
    ++step;
  }
out:
  if (cta == 0 && tid == 0) {
    st->ns = ns;
    st->step = step;
    st->dm_on = dm_on;
    st->rank = rank;
    st->rank_colmax = rank_cm;
    st->k = 1;
    st->l = 0;
    st->done = 1;
  }
  if (tid == 0) add_flops(st, KID_QRP_TAIL, flops);
}

// a11: end of a block step, n_s += l.  Runs after every other kernel of the
// step, so all of them saw the same n_s.
__global__ void k_step_end(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  if (*(volatile int32_t*)&st->abort_flag) {  // a wait gave up or a check tripped in this step
    st->done = 1;
    return;
  }
  if (P.checked && !(in_range(P, KID_STEP_END, st->l, 1, (int64_t)st->k + 1) &&
                     in_range(P, KID_STEP_END, st->ns + st->l, 1, P.kmin + 1))) {
    st->done = 1;
    return;
  }
  if (P.pol.active && st->dm_on) {
    // carry for the next step's features and for the guard of the learned
    // (tau, delta), checked at the next step's start against its mu
    st->pc.prev_learned = st->pol_learned;
    st->pc.prev_minb = st->pol_minb;
    st->pc.prev_l = (float)st->l;
    st->pc.prev_k = (float)st->k;
    st->pc.prev_tau = (float)st->tau_s;
  }
  st->ns += st->l;
  st->step += 1;
}

__global__ void k_state_init(Params P) {
  DevState* st = P.st;
  st->ns = 0;
  st->step = 0;
  st->rank = -1;
  st->rank_colmax = -1;
  st->anorm_bits = 0ull;
  st->done = 0;
  st->dm_on = 1;
  st->nonfinite = 0;
  st->k = 0;
  st->l = 0;
  st->kc = 0;
  st->npairs = 0;
  st->pbreak = 0;
  st->cur_lj = 0;
  for (int q = 0; q < KMAX / PB; ++q) {
    st->sub_l[q] = 0;
    st->sub_next[q] = 0;
  }
  for (int i = 0; i < 24; ++i) st->flops[i] = 0.0;
  st->gbar = 0u;
  st->abort_flag = 0;
  st->diag_code = 0;
  st->diag_cta = -1;
  st->diag_step = -1;
  st->diag_ns = -1;
  st->diag_value = 0;
  st->tau_s = P.tau;
  st->delta_s = P.delta;
  st->pol_minb = INFINITY;
  st->pc.prev_l = 0.0f;
  st->pc.prev_k = 0.0f;
  st->pc.cos_mean = 0.0f;
  st->pc.cos_max = 0.0f;
  st->pc.prev_tau = 0.0f;
  st->pc.off = 0;
  st->pc.prev_learned = 0;
  st->pc.prev_minb = INFINITY;
  st->pol_learned = 0;
}

}  // namespace qrdm
