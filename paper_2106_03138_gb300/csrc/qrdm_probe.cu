// qrdm_fp64_probe: the FP64 arithmetic rates of this GPU, measured with the
// two instruction forms an FP64 kernel can use, so that the FP64 kernels'
// roofline has a measured denominator beside the one derived from the unit
// count and the clock.  Not part of the factorization.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qrdm.h"

namespace {

constexpr int PROBE_THREADS = 256;

// FFMA64: eight independent multiply-add chains per thread.  The values stay
// finite and the sum is stored, so nothing is optimized away.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(double* out, int iters) {
  const double b = 0.999999999, c = 1e-12;
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

// DMMA: mma.sync m8n8k4 FP64 (512 flops per warp instruction), four
// independent accumulators per warp.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dmma(double* out, int iters) {
  const double av = 1.0 + 1e-6 * threadIdx.x, bv = 0.999999 - 1e-7 * threadIdx.x;
  double d[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) d[k][0] = d[k][1] = 1e-3 * k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[k][0]), "+d"(d[k][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1];
  out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" int qrdm_fp64_probe(int32_t which, int32_t blocks, int32_t iters, void* d_out, size_t out_bytes,
                               double* flops, float* ms, void* stream_) {
  if (which != 0 && which != 1) return -1;
  if (blocks < 1) return -2;
  if (iters < 1) return -3;
  if (!d_out || out_bytes < (size_t)blocks * PROBE_THREADS * sizeof(double)) return -4;
  if (!flops) return -6;
  if (!ms) return -7;
  cudaStream_t s = (cudaStream_t)stream_;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    if (which == 0)
      k_probe_ffma<<<blocks, PROBE_THREADS, 0, s>>>((double*)d_out, iters);
    else
      k_probe_dmma<<<blocks, PROBE_THREADS, 0, s>>>((double*)d_out, iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return QRDM_ERR_CUDA;
  const double threads = (double)blocks * PROBE_THREADS;
  *flops = (which == 0) ? 2.0 * 8.0 * threads * iters : 512.0 * 4.0 * (threads / 32.0) * iters;
  return 0;
}
