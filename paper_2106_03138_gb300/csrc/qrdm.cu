// C ABI of the GB300 QRDM library: argument checks, workspace layout, and the
// host loop that enqueues one block step (Algorithm 4) at a time.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/qrdm.h"
#include "qrdm_kernels.cuh"

using namespace qrdm;

namespace {

thread_local int g_last_cuda = 0;

constexpr int GRAM_CHUNKS_MAX = 256;
constexpr int QRP_SMEM_MAX = 200 * 1024;  // pivot column of the fused single-column kernel
constexpr int WCHUNKS = 16;
constexpr size_t ALIGN = 256;

static_assert(sizeof(StepRecord) == sizeof(qrdm_step_record), "trace record layout");

size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  size_t st, u, uref, cols, mdst, msrc, Gp, G, T, Wp, W, total;
};

Layout make_layout(int64_t m, int64_t n, int kmax) {
  (void)m;
  Layout L;
  size_t off = 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t kk = (size_t)kmax * (size_t)kmax;
  L.st = off;
  off = up(off + sizeof(DevState));
  L.u = off;
  off = up(off + nn * sizeof(double));
  L.uref = off;
  off = up(off + nn * sizeof(double));
  L.cols = off;
  off = up(off + KMAX * sizeof(int32_t));
  L.mdst = off;
  off = up(off + 2 * KMAX * sizeof(int32_t));
  L.msrc = off;
  off = up(off + 2 * KMAX * sizeof(int32_t));
  L.Gp = off;
  off = up(off + (size_t)GRAM_CHUNKS_MAX * kk * sizeof(double));
  L.G = off;
  off = up(off + kk * sizeof(double));
  L.T = off;
  off = up(off + (size_t)KMAX * KMAX * sizeof(double));
  L.Wp = off;
  off = up(off + (size_t)WCHUNKS * kmax * nn * sizeof(double));
  L.W = off;
  off = up(off + (size_t)kmax * nn * sizeof(double));
  L.total = off;
  return L;
}

struct DeviceConfig {
  int device = -1;
  int sms = 0;
  int cluster = 0;  // panel cluster size
  int coop = 0;     // cooperative launch supported
  int qrp_grid = 0; // CTAs of the fused single-column kernel (one per SM)
  bool ok = false;
  cudaEvent_t ev[2 * QRDM_NKERNELS] = {};  // profile events, created on first use
  bool have_events = false;
};

thread_local DeviceConfig g_cfg;
thread_local std::vector<cudaEvent_t> g_events;

int configure(DeviceConfig* cfg) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (g_cfg.ok && g_cfg.device == dev) {
    *cfg = g_cfg;
    return 0;
  }
  DeviceConfig c;
  c.device = dev;
  e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int perm_smem = (int)(2 * KMAX * 33 * sizeof(double));
  const int gram_smem = (int)(KMAX * (GRAM_ROWS + 1) * sizeof(double));
  if ((e = cudaFuncSetAttribute(k_trail_w, cudaFuncAttributeMaxDynamicSharedMemorySize, TRAIL_W_SMEM)) != cudaSuccess)
    return (int)e;
  if ((e = cudaFuncSetAttribute(k_trail_w32, cudaFuncAttributeMaxDynamicSharedMemorySize, S32_SMEM)) != cudaSuccess)
    return (int)e;
  if ((e = cudaFuncSetAttribute(k_trail_update32, cudaFuncAttributeMaxDynamicSharedMemorySize, S32_SMEM)) !=
      cudaSuccess)
    return (int)e;
  if ((e = cudaFuncSetAttribute(k_gram32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(KMAX * (GRAM_ROWS + 1) * sizeof(double)))) != cudaSuccess)
    return (int)e;
  const int pick_smem_max = (int)(KMAX * (KMAX + 1) / 2 * sizeof(double));
  if ((e = cudaFuncSetAttribute(k_pick, cudaFuncAttributeMaxDynamicSharedMemorySize, pick_smem_max)) != cudaSuccess)
    return (int)e;
  if ((e = cudaFuncSetAttribute(k_permute, cudaFuncAttributeMaxDynamicSharedMemorySize, perm_smem)) != cudaSuccess)
    return (int)e;
  if ((e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, gram_smem)) != cudaSuccess)
    return (int)e;
  // panel cluster: 16 CTAs when the device allows it, else 8
  c.cluster = 8;
  if ((e = cudaFuncSetAttribute(k_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_MAX)) !=
      cudaSuccess)
    return (int)e;
  if (cudaFuncSetAttribute(k_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(k_panel_g, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t lc = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.gridDim = dim3(16);
    lc.blockDim = dim3(PANEL_THREADS);
    lc.dynamicSmemBytes = PANEL_SMEM_MAX;
    lc.attrs = at;
    lc.numAttrs = 1;
    int ncl = 0, ncl_g = 0;
    lc.dynamicSmemBytes = PANEL_SMEM_MAX;
    const bool ok_s = cudaOccupancyMaxActiveClusters(&ncl, (void*)k_panel, &lc) == cudaSuccess && ncl >= 1;
    lc.dynamicSmemBytes = 0;
    const bool ok_g = cudaOccupancyMaxActiveClusters(&ncl_g, (void*)k_panel_g, &lc) == cudaSuccess && ncl_g >= 1;
    if (ok_s && ok_g) c.cluster = 16;
  }
  cudaGetLastError();  // clear a refused non-portable query
  e = cudaDeviceGetAttribute(&c.coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess) return (int)e;
  if ((e = cudaFuncSetAttribute(k_qrp_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, QRP_SMEM_MAX)) !=
      cudaSuccess)
    return (int)e;
  {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qrp_tail, QRP_THREADS, QRP_SMEM_MAX);
    if (e != cudaSuccess) return (int)e;
    c.qrp_grid = (c.coop && per_sm >= 1) ? c.sms : 0;
  }
  c.ok = true;
  g_cfg = c;
  *cfg = c;
  return 0;
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      g_last_cuda = (int)e_;                      \
      info->cuda_error = (int32_t)e_;             \
      return QRDM_ERR_CUDA;                       \
    }                                             \
  } while (0)

}  // namespace

extern "C" {

int qrdm_version(void) { return 100; }

int qrdm_last_cuda_error(void) { return g_last_cuda; }

const char* qrdm_strerror(int code) {
  switch (code) {
    case QRDM_OK:
      return "success";
    case QRDM_ERR_CUDA:
      return "a CUDA runtime call failed";
    case QRDM_ERR_NONFINITE:
      return "the matrix holds a NaN or an infinity";
    case QRDM_ERR_WORKSPACE:
      return "workspace missing, too small or not 256-byte aligned";
    case QRDM_ERR_UNSUPPORTED:
      return "unsupported device or option";
    case QRDM_ERR_INTERNAL:
      return "internal consistency check failed";
    default:
      return code < 0 ? "invalid argument" : "unknown error";
  }
}

int qrdm_workspace_size(int64_t m, int64_t n, int32_t k_max, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > INT32_MAX) return -2;
  if (k_max < 1 || k_max > QRDM_KMAX_LIMIT) return -3;
  if (!bytes) return -4;
  *bytes = make_layout(m, n, k_max).total;
  return 0;
}

int qrdm_factor(double* dA, int64_t m, int64_t n, int64_t lda, double tau, double delta, int32_t k_max,
                double* d_htau, int32_t* d_perm, qrdm_info* info, const qrdm_opts* opts, void* d_work,
                size_t work_bytes, void* stream_, qrdm_step_record* d_trace, int32_t* d_trace_J, int64_t trace_cap) {
  if (m < 0) return -1;
  if (n < 0 || n > INT32_MAX) return -2;
  if (!dA && m > 0 && n > 0) return -3;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (!(tau > 0.0 && tau <= 1.0)) return -5;
  if (!(delta >= 0.0 && delta <= 1.0)) return -6;
  if (k_max < 1 || k_max > QRDM_KMAX_LIMIT) return -7;
  const int64_t kmin = m < n ? m : n;
  if (!d_htau && kmin > 0) return -8;
  if (!d_perm && n > 0) return -9;
  if (!info) return -10;
  memset(info, 0, sizeof(*info));
  qrdm_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.eps1_mode != 0 && o.eps1_mode != 1) return -11;
  if (o.precision != 0 && o.precision != 1) return -11;
  cudaStream_t stream = (cudaStream_t)stream_;

  if (n == 0 || m == 0) {
    // nothing to factor; the permutation is the identity
    if (n > 0) {
      // identity permutation via a tiny host copy
      int32_t* h = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      if (!h) return QRDM_ERR_INTERNAL;
      for (int64_t j = 0; j < n; ++j) h[j] = (int32_t)j;
      cudaError_t e = cudaMemcpyAsync(d_perm, h, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      free(h);
      if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        info->cuda_error = (int32_t)e;
        return QRDM_ERR_CUDA;
      }
    }
    info->rank = 0;
    info->rank_colmax = 0;
    return QRDM_OK;
  }

  const Layout L = make_layout(m, n, k_max);
  if (!d_work) return -12;
  if (work_bytes < L.total || ((uintptr_t)d_work % ALIGN) != 0) return QRDM_ERR_WORKSPACE;

  DeviceConfig cfg;
  {
    int e = configure(&cfg);
    if (e) {
      g_last_cuda = e;
      info->cuda_error = e;
      return QRDM_ERR_CUDA;
    }
  }

  char* w = (char*)d_work;
  Params P;
  memset(&P, 0, sizeof(P));
  P.A = dA;
  P.m = m;
  P.n = n;
  P.lda = lda;
  P.kmin = kmin;
  P.tau = tau;
  P.delta = delta;
  P.eps1 = (o.eps1_mode == 1) ? EPS * sqrt((double)n) : EPS * (double)n;
  if (o.precision == 1) {
    // FP32-class updates leave roundoff of about 2^-24 ||A|| in the trailing
    // block; the rank threshold must sit above it
    const double e32 = 8.0 * 5.9604644775390625e-8 * sqrt((double)n);
    if (e32 > P.eps1) P.eps1 = e32;
  }
  const bool mixed = (o.precision == 1);
  P.mixed = mixed ? 1 : 0;
  P.kmax = k_max;
  P.stop_at_rank = o.stop_at_rank;
  P.check_last = o.check_last;
  P.no_break = o.no_break;
  P.sdd = o.sdd;
  P.max_steps = o.max_steps;
  P.htau = d_htau;
  P.perm = d_perm;
  P.st = (DevState*)(w + L.st);
  P.u = (double*)(w + L.u);
  P.uref = (double*)(w + L.uref);
  P.cols = (int32_t*)(w + L.cols);
  P.mdst = (int32_t*)(w + L.mdst);
  P.msrc = (int32_t*)(w + L.msrc);
  P.Gp = (double*)(w + L.Gp);
  P.G = (double*)(w + L.G);
  P.T = (double*)(w + L.T);
  P.Wp = (double*)(w + L.Wp);
  P.W = (double*)(w + L.W);
  const int sms = cfg.sms;
  P.gram_chunks = sms < GRAM_CHUNKS_MAX ? sms : GRAM_CHUNKS_MAX;
  P.wchunks = WCHUNKS;
  const int gemm_grid = 2 * sms;
  P.w_units = 4 * gemm_grid;
  P.trace = (StepRecord*)d_trace;
  P.traceJ = d_trace_J;
  P.trace_cap = d_trace ? trace_cap : 0;

  CK(cudaMemsetAsync(d_htau, 0, sizeof(double) * (size_t)kmin, stream));
  if (d_trace && trace_cap > 0) CK(cudaMemsetAsync(d_trace, 0, sizeof(qrdm_step_record) * (size_t)trace_cap, stream));
  if (d_trace_J && trace_cap > 0)
    CK(cudaMemsetAsync(d_trace_J, 0xff, sizeof(int32_t) * (size_t)trace_cap * (size_t)k_max, stream));
  k_state_init<<<1, 1, 0, stream>>>(P);
  if (o.profile && !g_cfg.have_events) {
    for (int i = 0; i < 2 * QRDM_NKERNELS; ++i) CK(cudaEventCreate(&g_cfg.ev[i]));
    g_cfg.have_events = true;
  }
  if (o.profile) CK(cudaEventRecord(g_cfg.ev[2 * QRDM_K_COLNORM], stream));
  {
    int64_t g = (n + 7) / 8;
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    k_colnorm_init<<<(unsigned)g, 256, 0, stream>>>(P);
  }
  CK(cudaGetLastError());
  if (o.profile) CK(cudaEventRecord(g_cfg.ev[2 * QRDM_K_COLNORM + 1], stream));
  DevState hs;
  CK(cudaMemcpyAsync(&hs, P.st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  if (hs.nonfinite) return QRDM_ERR_NONFINITE;
  if (o.profile) {
    float msk = 0.f;
    CK(cudaEventElapsedTime(&msk, g_cfg.ev[2 * QRDM_K_COLNORM], g_cfg.ev[2 * QRDM_K_COLNORM + 1]));
    o.profile->ms[QRDM_K_COLNORM] += msk;
    o.profile->launches[QRDM_K_COLNORM] += 1;
  }

  const int perm_smem = (int)(2 * k_max * 33 * sizeof(double));
  const int gram_smem = (int)(k_max * (GRAM_ROWS + 1) * sizeof(double));
  const int pick_smem = (int)((k_max * (k_max + 1) / 2) * sizeof(double));
  unsigned perm_grid = (unsigned)((m + 31) / 32);
  if (perm_grid > (unsigned)(4 * sms)) perm_grid = 4 * sms;
  unsigned dd_grid = (unsigned)((n + 7) / 8);
  if (dd_grid > (unsigned)(8 * sms)) dd_grid = 8 * sms;
  const unsigned gred_grid = (unsigned)((k_max * (k_max + 1) / 2 + 255) / 256);

  cudaLaunchConfig_t pc = {};
  cudaLaunchAttribute pat[1];
  pat[0].id = cudaLaunchAttributeClusterDimension;
  pat[0].val.clusterDim.x = cfg.cluster;
  pat[0].val.clusterDim.y = 1;
  pat[0].val.clusterDim.z = 1;
  pc.gridDim = dim3(cfg.cluster);
  pc.blockDim = dim3(PANEL_THREADS);
  // each CTA holds ceil(m / cluster) rows of up to PB columns in shared memory
  const int64_t panel_lds = ((m + cfg.cluster - 1) / cfg.cluster) | 1;
  const int64_t panel_smem = (int64_t)PB * panel_lds * (int64_t)sizeof(double);
  const bool panel_in_smem = panel_smem <= PANEL_SMEM_MAX;
  pc.dynamicSmemBytes = panel_in_smem ? (size_t)panel_smem : 0;
  pc.stream = stream;
  pc.attrs = pat;
  pc.numAttrs = 1;

  qrdm_profile* prof = o.profile;
  const int nsub_full = (k_max + PB - 1) / PB;
  // events for profiling: two pools (the previous batch is read while the
  // next one runs), each with a start/end pair per launch
  constexpr int MAX_BATCH = 16;
  const int per_step = 7 + 4 * nsub_full;
  const int pool = MAX_BATCH * per_step;
  if (prof && (int)g_events.size() < 2 * 2 * pool) {
    while ((int)g_events.size() < 2 * 2 * pool) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      g_events.push_back(e);
    }
  }
  int64_t launches = 2;
  struct Rec {
    int kid;
    int ev;
  };
  std::vector<Rec> recs[2];
  int cur = 0;
  auto run = [&](int kid, auto&& launch) -> cudaError_t {
    int evi = -1;
    if (prof) {
      evi = 2 * pool * cur + 2 * (int)recs[cur].size();
      cudaError_t e = cudaEventRecord(g_events[evi], stream);
      if (e != cudaSuccess) return e;
    }
    launch();
    ++launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && prof) {
      e = cudaEventRecord(g_events[evi + 1], stream);
      recs[cur].push_back({kid, evi});
    }
    return e;
  };
  auto harvest = [&](int which) -> cudaError_t {
    for (const Rec& r : recs[which]) {
      float msk = 0.f;
      cudaError_t e = cudaEventElapsedTime(&msk, g_events[r.ev], g_events[r.ev + 1]);
      if (e != cudaSuccess) return e;
      prof->ms[r.kid] += msk;
      prof->launches[r.kid] += 1;
    }
    recs[which].clear();
    return cudaSuccess;
  };
  auto enqueue_step = [&](int nsub) -> cudaError_t {
    cudaError_t e;
    if ((e = run(QRDM_K_SELECT, [&] { k_select<<<1, SEL_THREADS, 0, stream>>>(P); })) != cudaSuccess) return e;
    if ((e = run(QRDM_K_GRAM, [&] {
           if (mixed)
             k_gram32<<<P.gram_chunks, 256, gram_smem, stream>>>(P);
           else
             k_gram<<<P.gram_chunks, 256, gram_smem, stream>>>(P);
         })) != cudaSuccess)
      return e;
    if ((e = run(QRDM_K_GRAM_REDUCE, [&] { k_gram_reduce<<<gred_grid, 256, 0, stream>>>(P); })) != cudaSuccess)
      return e;
    if ((e = run(QRDM_K_PICK, [&] { k_pick<<<1, 256, pick_smem, stream>>>(P); })) != cudaSuccess) return e;
    if ((e = run(QRDM_K_PERMUTE, [&] { k_permute<<<perm_grid, 256, perm_smem, stream>>>(P); })) != cudaSuccess)
      return e;
    for (int j = 0; j < nsub; ++j) {
      if ((e = run(QRDM_K_PANEL, [&] {
             if (panel_in_smem)
               cudaLaunchKernelEx(&pc, k_panel, P, j);
             else
               cudaLaunchKernelEx(&pc, k_panel_g, P, j);
           })) != cudaSuccess)
        return e;
      if ((e = run(QRDM_K_TRAIL_W, [&] {
             if (mixed)
               k_trail_w32<<<gemm_grid, GEMM_THREADS, S32_SMEM, stream>>>(P, j);
             else
               k_trail_w<<<gemm_grid, GEMM_THREADS, TRAIL_W_SMEM, stream>>>(P, j);
           })) != cudaSuccess)
        return e;
      if ((e = run(QRDM_K_TRAIL_WREDUCE, [&] { k_trail_wreduce<<<sms, GEMM_THREADS, 0, stream>>>(P, j); })) !=
          cudaSuccess)
        return e;
      if ((e = run(QRDM_K_TRAIL_UPDATE, [&] {
             if (mixed)
               k_trail_update32<<<gemm_grid, GEMM_THREADS, S32_SMEM, stream>>>(P, j);
             else
               k_trail_update<<<gemm_grid, GEMM_THREADS, 0, stream>>>(P, j);
           })) != cudaSuccess)
        return e;
    }
    if ((e = run(QRDM_K_DOWNDATE, [&] { k_downdate<<<dd_grid, 256, 0, stream>>>(P); })) != cudaSuccess) return e;
    return run(QRDM_K_STEP_END, [&] { k_step_end<<<1, 1, 0, stream>>>(P); });
  };

  // Single-column steps (DM off, or k_max = 1) run fused in one cooperative
  // kernel when the pivot column fits in shared memory.
  const bool qrp_fused = cfg.qrp_grid > 0 && (int64_t)m * (int64_t)sizeof(double) <= QRP_SMEM_MAX;
  auto launch_qrp = [&]() -> cudaError_t {
    void* args[] = {(void*)&P};
    const size_t smem = (size_t)m * sizeof(double);
    return run(QRDM_K_QRP_TAIL, [&] {
      cudaLaunchCooperativeKernel((void*)k_qrp_tail, dim3(cfg.qrp_grid), dim3(QRP_THREADS), args, smem, stream);
    });
  };

  // Steps are enqueued in batches; the state is read back once per batch.
  // Kernels of steps past the end return at once (the state says done).
  int64_t iters = 0, last_ns = 0;
  int batch = 1;
  bool dm_off = (k_max == 1);
  for (;;) {
    const int nsub = dm_off ? 1 : nsub_full;
    if (dm_off && qrp_fused) {
      if (getenv("QRDM_DEBUG"))
        fprintf(stderr, "qrdm: fused single-column kernel from ns=%lld step=%lld (grid %d, smem %lld)\n",
                (long long)hs.ns, (long long)hs.step, cfg.qrp_grid, (long long)(m * 8));
      CK(launch_qrp());
    } else {
      for (int b = 0; b < batch; ++b) CK(enqueue_step(nsub));
    }
    iters += batch;
    if (prof) CK(harvest(cur ^ 1));
    CK(cudaMemcpyAsync(&hs, P.st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (prof) cur ^= 1;
    if (hs.done || iters > kmin + 2) break;
    dm_off = (hs.dm_on == 0);
    // next batch: about half the steps the recent progress says remain
    const int64_t adv = hs.ns - last_ns;
    last_ns = hs.ns;
    const double per = adv > 0 ? (double)adv / batch : 1.0;
    int64_t guess = (int64_t)((double)(kmin - hs.ns) / per / 2.0);
    batch = (int)(guess < 1 ? 1 : (guess > MAX_BATCH ? MAX_BATCH : guess));
  }
  if (prof) {
    CK(harvest(cur ^ 1));
    for (int i = 0; i < QRDM_NKERNELS; ++i) prof->flops[i] += hs.flops[i];
  }
  info->launches = launches;
  if (!hs.done || hs.nonfinite) {
    if (getenv("QRDM_DEBUG"))
      fprintf(stderr,
              "qrdm: internal error: done=%d flag=%d diag_code=%d cta=%d step=%lld ns=%lld value=%lld gbar=%u\n",
              hs.done, hs.nonfinite, hs.diag_code, hs.diag_cta, (long long)hs.diag_step, (long long)hs.diag_ns,
              (long long)hs.diag_value, hs.gbar);
    return QRDM_ERR_INTERNAL;
  }
  info->rank = hs.rank >= 0 ? hs.rank : (hs.ns >= kmin ? kmin : hs.ns);
  info->rank_colmax = hs.rank_colmax >= 0 ? hs.rank_colmax : (hs.ns >= kmin ? kmin : hs.ns);
  info->nsteps = hs.step;
  return QRDM_OK;
}

}  // extern "C"
