// Learned per-step (tau, delta): the features of a block step and the small
// MLP that maps them to (tau_s, delta_s).  The paper fixes (tau, delta) for a
// whole factorization and studies the choice empirically (Sec. 5, parameter
// study); predicting them per step is this library's addition.
//
// Features (POL_NFEAT = 16), taken at the start of a DM step, after the
// argmax mu = u_{j*}:
//   f0..f7  min(#{j >= n_s, j != j*: u_j >= t_b mu}, 128) / 128 for
//           t_b = 0.95, 0.9, 0.75, 0.6, 0.45, 0.3, 0.15, 0.05 (the candidate
//           counts the DM threshold of Alg. 1 would give at those tau)
//   f8      (n - n_s) / n, f9 log2(n - n_s) / 16
//   f10     log10(mu / max_j ||a_j||) / 16
//   f11     l of the previous step / 64 (clipped at 1), f12 its l / k
//   f13/f14 mean and max |theta(j*, i)| over the previous step's candidates
//   f15     tau used by the previous step
// (first step: f11 = 0, f12 = 1, f13 = f14 = 0, f15 = 0).
//
// MLP: 16 -> 64 -> 64 -> 2, ReLU, BF16 weights, FP32 accumulation;
// tau = tau_lo + (tau_hi - tau_lo) sigmoid(o_0), delta likewise from o_1.
// Weight blob (BF16, row-major): W1[16][64], b1[64], W2[64][64], b2[64],
// W3[64][2], b3[2].
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace qrdm {

constexpr int POL_NFEAT = 16;
constexpr int POL_HIDDEN = 64;
constexpr int POL_NOUT = 2;
constexpr int POL_OFF_W1 = 0;
constexpr int POL_OFF_B1 = POL_OFF_W1 + POL_NFEAT * POL_HIDDEN;
constexpr int POL_OFF_W2 = POL_OFF_B1 + POL_HIDDEN;
constexpr int POL_OFF_B2 = POL_OFF_W2 + POL_HIDDEN * POL_HIDDEN;
constexpr int POL_OFF_W3 = POL_OFF_B2 + POL_HIDDEN;
constexpr int POL_OFF_B3 = POL_OFF_W3 + POL_HIDDEN * POL_NOUT;
constexpr int POL_NPARAM = POL_OFF_B3 + POL_NOUT;  // 5378

// Device view of the policy (built from qrdm_policy on the host).
struct PolicyParams {
  const __nv_bfloat16* w;  // nullptr: features only (fixed tau, delta)
  float* feat_log;         // optional [cap][POL_NFEAT] per-step features
  double* act_log;         // optional [cap][2] (tau_s, delta_s) used per step
  int64_t log_cap;
  double tau_lo, tau_hi, delta_lo, delta_hi;
  double rho_min;          // guard: accepted |R_ii| of a learned step >= rho_min * (largest partial norm after it)
  int32_t active;          // 1: a policy object was passed
  int32_t pad;
};

// Per-factorization memory of the previous step, carried between steps.
struct PolicyCarry {
  float prev_l, prev_k, cos_mean, cos_max, prev_tau;
  int32_t off;           // 1 once the guard fired: fixed (tau, delta) from then on
  int32_t prev_learned;  // the previous step used the MLP's (tau, delta)
  int32_t pad;
  double prev_minb;      // smallest |R_ii| the previous step accepted
};

__device__ __forceinline__ long long pol_key(double x) { return __double_as_longlong(x); }

// Block-wide features into s_feat[POL_NFEAT] (every thread of the block
// calls it; NT threads).  s_cnt: int scratch of 8 * (NT / 32) entries.
template <int NT>
__device__ __noinline__ void pol_features(const double* u, int64_t ns, int64_t n, int64_t jstar, double mu, double anorm,
                             const PolicyCarry& pc, float* s_feat, int* s_cnt) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float thresh[8] = {0.95f, 0.9f, 0.75f, 0.6f, 0.45f, 0.3f, 0.15f, 0.05f};
  long long tk[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) tk[b] = pol_key((double)thresh[b] * mu);
  int c[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) c[b] = 0;
  for (int64_t j = ns + tid; j < n; j += NT) {
    if (j == jstar) continue;
    const long long x = pol_key(u[j]);
#pragma unroll
    for (int b = 0; b < 8; ++b) c[b] += (x >= tk[b]) ? 1 : 0;
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    int v = __reduce_add_sync(0xffffffffu, c[b]);
    if (lane == 0) s_cnt[b * NW + w] = v;
  }
  __syncthreads();
  if (tid < 8) {
    int t = 0;
    for (int q = 0; q < NW; ++q) t += s_cnt[tid * NW + q];
    s_feat[tid] = (float)(t < 128 ? t : 128) / 128.0f;
  }
  if (tid == 0) {
    const double nrem = (double)(n - ns);
    s_feat[8] = (float)(nrem / (double)(n > 0 ? n : 1));
    s_feat[9] = log2f((float)nrem) / 16.0f;
    const float r = (anorm > 0.0 && mu > 0.0) ? (float)(mu / anorm) : 1e-30f;
    s_feat[10] = log10f(fmaxf(r, 1e-30f)) / 16.0f;
    s_feat[11] = fminf(pc.prev_l / 64.0f, 1.0f);
    s_feat[12] = pc.prev_k > 0.0f ? pc.prev_l / pc.prev_k : 1.0f;
    s_feat[13] = pc.cos_mean;
    s_feat[14] = pc.cos_max;
    s_feat[15] = pc.prev_tau;
  }
  __syncthreads();
}

__device__ __forceinline__ float pol_sigmoid(float x) { return 1.0f / (1.0f + __expf(-x)); }

// MLP forward on s_feat (block of NT >= POL_HIDDEN threads); out[0..1] =
// (tau, delta).  s_h: float scratch of 2 * POL_HIDDEN.
template <int NT>
__device__ __noinline__ void pol_mlp(const PolicyParams& pp, const float* s_feat, float* s_h, double* s_out) {
  static_assert(NT >= POL_HIDDEN, "block too small for the MLP");
  const int tid = threadIdx.x;
  const __nv_bfloat16* W = pp.w;
  if (tid < POL_HIDDEN) {
    float a = __bfloat162float(W[POL_OFF_B1 + tid]);
#pragma unroll
    for (int i = 0; i < POL_NFEAT; ++i) a = fmaf(s_feat[i], __bfloat162float(W[POL_OFF_W1 + i * POL_HIDDEN + tid]), a);
    s_h[tid] = fmaxf(a, 0.0f);
  }
  __syncthreads();
  if (tid < POL_HIDDEN) {
    float a = __bfloat162float(W[POL_OFF_B2 + tid]);
    for (int i = 0; i < POL_HIDDEN; ++i) a = fmaf(s_h[i], __bfloat162float(W[POL_OFF_W2 + i * POL_HIDDEN + tid]), a);
    s_h[POL_HIDDEN + tid] = fmaxf(a, 0.0f);
  }
  __syncthreads();
  if (tid < 32) {
    float a0 = 0.0f, a1 = 0.0f;
    for (int i = tid; i < POL_HIDDEN; i += 32) {
      const float h = s_h[POL_HIDDEN + i];
      a0 = fmaf(h, __bfloat162float(W[POL_OFF_W3 + i * POL_NOUT + 0]), a0);
      a1 = fmaf(h, __bfloat162float(W[POL_OFF_W3 + i * POL_NOUT + 1]), a1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (tid == 0) {
      a0 += __bfloat162float(W[POL_OFF_B3 + 0]);
      a1 += __bfloat162float(W[POL_OFF_B3 + 1]);
      s_out[0] = pp.tau_lo + (pp.tau_hi - pp.tau_lo) * (double)pol_sigmoid(a0);
      s_out[1] = pp.delta_lo + (pp.delta_hi - pp.delta_lo) * (double)pol_sigmoid(a1);
    }
  }
  __syncthreads();
}

}  // namespace qrdm
