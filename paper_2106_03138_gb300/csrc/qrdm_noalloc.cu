// qrdm_factor_noalloc: the factorization for callers that cannot allocate
// device memory.  Its workspace is a fixed array in this library's device
// image (QRDM_NOALLOC_SCRATCH_BYTES, 32 MiB), held on every GPU that loads
// the library until the process exits.  All calls share that array.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/qrdm.h"

namespace qrdm {
// qrdm_factor with every launch on the caller's stream (no second stream or
// events are created: this entry point creates nothing)
int factor_impl(double* dA, int64_t m, int64_t n, int64_t lda, double tau, double delta, int32_t k_max,
                double* d_htau, int32_t* d_perm, qrdm_info* info, const qrdm_opts* opts, void* d_work,
                size_t work_bytes, void* stream, qrdm_step_record* d_trace, int32_t* d_trace_J, int64_t trace_cap,
                bool allow_side);
}  // namespace qrdm

namespace {

// The shared scratch.  In host code `g_scratch` only names the symbol; its
// device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_scratch[QRDM_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_ptr[MAX_DEVICES] = {};

// Device address of the scratch on the current device, looked up once.
int scratch_address(void** out, int* cuda_err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *cuda_err = (int)e;
    return QRDM_ERR_CUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) return QRDM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      *cuda_err = (int)e;
      return QRDM_ERR_CUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return QRDM_OK;
}

}  // namespace

extern "C" int qrdm_factor_noalloc(double* dA, int64_t m, int64_t n, int64_t lda, double tau, double delta,
                                   int32_t k_max, double* d_htau, int32_t* d_perm, qrdm_info* info,
                                   const qrdm_opts* opts, void* stream, qrdm_step_record* d_trace,
                                   int32_t* d_trace_J, int64_t trace_cap) {
  if (opts && opts->profile) return QRDM_ERR_UNSUPPORTED;  // profiling creates CUDA events
  if (m == 0 || n == 0)  // nothing to factor: qrdm_factor checks every argument and needs no workspace
    return qrdm::factor_impl(dA, m, n, lda, tau, delta, k_max, d_htau, d_perm, info, opts, nullptr, 0, stream,
                             d_trace, d_trace_J, trace_cap, false);
  size_t need = 0;
  if (m >= 0 && n >= 0 && n <= INT32_MAX && k_max >= 1 && k_max <= QRDM_KMAX_LIMIT) {
    if (qrdm_workspace_size(m, n, k_max, &need) == 0 && need > (size_t)QRDM_NOALLOC_SCRATCH_BYTES)
      return QRDM_ERR_WORKSPACE;  // this shape needs more than the fixed scratch holds
  }
  void* scratch = nullptr;
  int cuda_err = 0;
  int rc = scratch_address(&scratch, &cuda_err);
  if (rc != QRDM_OK) {
    if (info) info->cuda_error = cuda_err;
    return rc;
  }
  // qrdm_factor validates every argument and re-initializes the whole step
  // state in the workspace, so the previous call's contents do not matter.
  return qrdm::factor_impl(dA, m, n, lda, tau, delta, k_max, d_htau, d_perm, info, opts, scratch,
                           (size_t)QRDM_NOALLOC_SCRATCH_BYTES, stream, d_trace, d_trace_J, trace_cap, false);
}
