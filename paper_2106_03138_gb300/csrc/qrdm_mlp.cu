// Training of the learned (tau, delta) policy: the 16 -> 64 -> 64 -> 2 MLP of
// qrdm_policy.cuh, with FP32 master weights, BF16 working weights (what the
// factorization reads) and FP32 accumulation.  Loss, per minibatch of B
// samples with targets t in [0, 1]^2 (normalized tau, delta):
//   L = (1/B) sum_b sum_o (y_bo - t_bo)^2 / 2,   y = sigmoid(o).
// Every kernel is deterministic: each output element is one thread's
// in-order sum (no atomics).  Minibatches are drawn with a counter-based hash
// (splitmix64 of seed, step, row), so a run is reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/qrdm.h"
#include "qrdm_policy.cuh"

namespace qrdm {
void set_last_cuda_error(int e);
namespace {

constexpr int F = POL_NFEAT, H = POL_HIDDEN, O = POL_NOUT, NP = POL_NPARAM;
static_assert(NP == QRDM_POLICY_NPARAM, "parameter count");
static_assert(F == QRDM_POLICY_NFEAT && H == QRDM_POLICY_HIDDEN, "layer sizes");

__device__ __forceinline__ float w16(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// splitmix64 (Steele, Lea, Flood 2014), a counter-based generator
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// minibatch gather: row b of the batch is sample hash(seed, step, b) mod n
__global__ void k_mlp_gather(const float* __restrict__ X, const float* __restrict__ T, int64_t nsamples, int64_t batch,
                             uint64_t seed, int64_t step, float* __restrict__ xb, float* __restrict__ tb) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const uint64_t h = mix64(seed ^ mix64((uint64_t)step * 0x100000001B3ull + (uint64_t)b));
  const int64_t i = (int64_t)(h % (uint64_t)nsamples);
  for (int f = 0; f < F; ++f) xb[b * F + f] = X[i * F + f];
  for (int o = 0; o < O; ++o) tb[b * O + o] = T[i * O + o];
}

// forward: a1 = x W1 + b1, h1 = relu(a1), a2 = h1 W2 + b2, h2 = relu(a2),
// o = h2 W3 + b3, y = sigmoid(o).  One thread per (sample, unit).
__global__ void k_mlp_l1(const __nv_bfloat16* __restrict__ w, const float* __restrict__ x, int64_t batch,
                         float* __restrict__ h1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * H) return;
  const int64_t b = e / H;
  const int j = (int)(e % H);
  float a = w16(w, POL_OFF_B1 + j);
  for (int i = 0; i < F; ++i) a = fmaf(x[b * F + i], w16(w, POL_OFF_W1 + i * H + j), a);
  h1[e] = fmaxf(a, 0.0f);
}

__global__ void k_mlp_l2(const __nv_bfloat16* __restrict__ w, const float* __restrict__ h1, int64_t batch,
                         float* __restrict__ h2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * H) return;
  const int64_t b = e / H;
  const int j = (int)(e % H);
  float a = w16(w, POL_OFF_B2 + j);
  for (int i = 0; i < H; ++i) a = fmaf(h1[b * H + i], w16(w, POL_OFF_W2 + i * H + j), a);
  h2[e] = fmaxf(a, 0.0f);
}

__global__ void k_mlp_l3(const __nv_bfloat16* __restrict__ w, const float* __restrict__ h2, int64_t batch,
                         float* __restrict__ y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * O) return;
  const int64_t b = e / O;
  const int o = (int)(e % O);
  float a = 0.0f;
  for (int i = 0; i < H; ++i) a = fmaf(h2[b * H + i], w16(w, POL_OFF_W3 + i * O + o), a);
  a += w16(w, POL_OFF_B3 + o);
  y[e] = 1.0f / (1.0f + expf(-a));
}

// backward, deltas: d3 = (y - t) y (1 - y) / B; d2 = (d3 W3^T) [a2 > 0];
// d1 = (d2 W2^T) [a1 > 0]   (h > 0 exactly when a > 0)
__global__ void k_mlp_d3(const float* __restrict__ y, const float* __restrict__ t, int64_t batch,
                         float* __restrict__ d3) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * O) return;
  const float yv = y[e];
  d3[e] = (yv - t[e]) * yv * (1.0f - yv) / (float)batch;
}

__global__ void k_mlp_d2(const __nv_bfloat16* __restrict__ w, const float* __restrict__ d3,
                         const float* __restrict__ h2, int64_t batch, float* __restrict__ d2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * H) return;
  const int64_t b = e / H;
  const int i = (int)(e % H);
  float s = 0.0f;
  for (int o = 0; o < O; ++o) s = fmaf(w16(w, POL_OFF_W3 + i * O + o), d3[b * O + o], s);
  d2[e] = (h2[e] > 0.0f) ? s : 0.0f;
}

__global__ void k_mlp_d1(const __nv_bfloat16* __restrict__ w, const float* __restrict__ d2,
                         const float* __restrict__ h1, int64_t batch, float* __restrict__ d1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * H) return;
  const int64_t b = e / H;
  const int i = (int)(e % H);
  float s = 0.0f;
  for (int j = 0; j < H; ++j) s = fmaf(w16(w, POL_OFF_W2 + i * H + j), d2[b * H + j], s);
  d1[e] = (h1[e] > 0.0f) ? s : 0.0f;
}

// weight gradients: one thread per parameter, a sum over the batch in order.
// Layer (in, delta): W[i][j] += sum_b in[b][i] delta[b][j], bias[j] += sum_b delta[b][j]
__device__ __forceinline__ float layer_grad(const float* in, int nin, const float* d, int nout, int64_t batch, int i,
                                            int j) {
  float s = 0.0f;
  if (i < 0) {
    for (int64_t b = 0; b < batch; ++b) s += d[b * nout + j];
  } else {
    for (int64_t b = 0; b < batch; ++b) s = fmaf(in[b * nin + i], d[b * nout + j], s);
  }
  return s;
}

__global__ void k_mlp_wgrad(const float* __restrict__ x, const float* __restrict__ h1, const float* __restrict__ h2,
                            const float* __restrict__ d1, const float* __restrict__ d2, const float* __restrict__ d3,
                            int64_t batch, float* __restrict__ g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  float v;
  if (p < POL_OFF_B1) {
    v = layer_grad(x, F, d1, H, batch, p / H, p % H);
  } else if (p < POL_OFF_W2) {
    v = layer_grad(nullptr, 0, d1, H, batch, -1, p - POL_OFF_B1);
  } else if (p < POL_OFF_B2) {
    const int q = p - POL_OFF_W2;
    v = layer_grad(h1, H, d2, H, batch, q / H, q % H);
  } else if (p < POL_OFF_W3) {
    v = layer_grad(nullptr, 0, d2, H, batch, -1, p - POL_OFF_B2);
  } else if (p < POL_OFF_B3) {
    const int q = p - POL_OFF_W3;
    v = layer_grad(h2, H, d3, O, batch, q / O, q % O);
  } else {
    v = layer_grad(nullptr, 0, d3, O, batch, -1, p - POL_OFF_B3);
  }
  g[p] = v;
}

// loss = (1/B) sum (y - t)^2 / 2, one CTA, fixed order
__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ t, int64_t batch,
                           float* __restrict__ loss) {
  __shared__ float s[256];
  float a = 0.0f;
  for (int64_t e = threadIdx.x; e < batch * O; e += 256) {
    const float d = y[e] - t[e];
    a = fmaf(d, d, a);
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5f * s[0] / (float)batch;
}

// Adam (Kingma & Ba 2015) with decoupled weight decay on the FP32 master
// weights (biases not decayed); refreshes the BF16 working copy.
__global__ void k_mlp_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ w16o, const float* __restrict__ g,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float wd, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const bool bias = (p >= POL_OFF_B1 && p < POL_OFF_W2) || (p >= POL_OFF_B2 && p < POL_OFF_W3) || p >= POL_OFF_B3;
  float wp = w[p];
  wp -= lr * ((mp / c1) / (sqrtf(vp / c2) + eps) + (bias ? 0.0f : wd * wp));
  w[p] = wp;
  w16o[p] = __float2bfloat16_rn(wp);
}

// He-uniform initialization from the counter-based hash; biases zero
__global__ void k_mlp_init(float* __restrict__ w, __nv_bfloat16* __restrict__ w16o, uint64_t seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  int fan_in = 0;
  if (p < POL_OFF_B1)
    fan_in = F;
  else if (p >= POL_OFF_W2 && p < POL_OFF_B2)
    fan_in = H;
  else if (p >= POL_OFF_W3 && p < POL_OFF_B3)
    fan_in = H;
  float val = 0.0f;
  if (fan_in) {
    const uint64_t h = mix64(seed ^ mix64((uint64_t)p));
    const float u01 = (float)((h >> 40) & 0xFFFFFFull) / 16777216.0f;  // [0, 1)
    const float lim = sqrtf(6.0f / (float)fan_in);
    val = (2.0f * u01 - 1.0f) * lim;
  }
  w[p] = val;
  w16o[p] = __float2bfloat16_rn(val);
}

__global__ void k_mlp_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16o) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) w16o[p] = __float2bfloat16_rn(w[p]);
}

unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// activations and deltas of a batch in one float workspace
struct Acts {
  float *xb, *tb, *h1, *h2, *y, *d1, *d2, *d3, *g, *loss;
};
size_t acts_floats(int64_t batch) { return (size_t)batch * (F + O + 4 * H + 2 * O) + NP + 4; }
Acts acts(float* w, int64_t batch) {
  Acts a;
  a.xb = w;
  a.tb = a.xb + batch * F;
  a.h1 = a.tb + batch * O;
  a.h2 = a.h1 + batch * H;
  a.y = a.h2 + batch * H;
  a.d1 = a.y + batch * O;
  a.d2 = a.d1 + batch * H;
  a.d3 = a.d2 + batch * H;
  a.g = a.d3 + batch * O;
  a.loss = a.g + NP;
  return a;
}

cudaError_t forward(const __nv_bfloat16* w, const float* x, int64_t batch, float* h1, float* h2, float* y,
                    cudaStream_t s) {
  k_mlp_l1<<<nblk(batch * H, 256), 256, 0, s>>>(w, x, batch, h1);
  k_mlp_l2<<<nblk(batch * H, 256), 256, 0, s>>>(w, h1, batch, h2);
  k_mlp_l3<<<nblk(batch * O, 256), 256, 0, s>>>(w, h2, batch, y);
  return cudaGetLastError();
}

cudaError_t backward(const __nv_bfloat16* w, const float* x, const float* t, int64_t batch, const Acts& a,
                     cudaStream_t s) {
  k_mlp_d3<<<nblk(batch * O, 256), 256, 0, s>>>(a.y, t, batch, a.d3);
  k_mlp_d2<<<nblk(batch * H, 256), 256, 0, s>>>(w, a.d3, a.h2, batch, a.d2);
  k_mlp_d1<<<nblk(batch * H, 256), 256, 0, s>>>(w, a.d2, a.h1, batch, a.d1);
  k_mlp_wgrad<<<nblk(NP, 128), 128, 0, s>>>(x, a.h1, a.h2, a.d1, a.d2, a.d3, batch, a.g);
  k_mlp_loss<<<1, 256, 0, s>>>(a.y, t, batch, a.loss);
  return cudaGetLastError();
}

}  // namespace
}  // namespace qrdm

using namespace qrdm;

extern "C" {

int qrdm_mlp_workspace_size(int64_t batch, size_t* bytes) {
  if (batch < 1 || batch > (1 << 24)) return -1;
  if (!bytes) return -2;
  *bytes = acts_floats(batch) * sizeof(float);
  return 0;
}

int qrdm_mlp_init(float* d_w32, void* d_w16, uint64_t seed, void* stream) {
  if (!d_w32) return -1;
  if (!d_w16) return -2;
  k_mlp_init<<<nblk(NP, 256), 256, 0, (cudaStream_t)stream>>>(d_w32, (__nv_bfloat16*)d_w16, seed);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

int qrdm_mlp_to_bf16(const float* d_w32, void* d_w16, void* stream) {
  if (!d_w32) return -1;
  if (!d_w16) return -2;
  k_mlp_to_bf16<<<nblk(NP, 256), 256, 0, (cudaStream_t)stream>>>(d_w32, (__nv_bfloat16*)d_w16);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

int qrdm_mlp_forward(const void* d_w16, const float* d_x, int64_t batch, float* d_y, float* d_work,
                     size_t work_bytes, void* stream) {
  if (!d_w16) return -1;
  if (!d_x) return -2;
  if (batch < 1 || batch > (1 << 24)) return -3;
  if (!d_y) return -4;
  if (!d_work || work_bytes < acts_floats(batch) * sizeof(float)) return QRDM_ERR_WORKSPACE;
  const Acts a = acts(d_work, batch);
  const cudaError_t e = forward((const __nv_bfloat16*)d_w16, d_x, batch, a.h1, a.h2, d_y, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

int qrdm_mlp_loss_grad(const void* d_w16, const float* d_x, const float* d_t, int64_t batch, float* d_grad,
                       float* d_loss, float* d_work, size_t work_bytes, void* stream) {
  if (!d_w16) return -1;
  if (!d_x) return -2;
  if (!d_t) return -3;
  if (batch < 1 || batch > (1 << 24)) return -4;
  if (!d_grad) return -5;
  if (!d_loss) return -6;
  if (!d_work || work_bytes < acts_floats(batch) * sizeof(float)) return QRDM_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const __nv_bfloat16* w = (const __nv_bfloat16*)d_w16;
  const Acts a = acts(d_work, batch);
  cudaError_t e = forward(w, d_x, batch, a.h1, a.h2, a.y, s);
  if (e == cudaSuccess) e = backward(w, d_x, d_t, batch, a, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_grad, a.g, sizeof(float) * NP, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_loss, a.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

int qrdm_mlp_adam_step(float* d_w32, void* d_w16, const float* d_grad, float* d_m, float* d_v, int64_t t, float lr,
                       float beta1, float beta2, float eps, float weight_decay, void* stream) {
  if (!d_w32) return -1;
  if (!d_w16) return -2;
  if (!d_grad) return -3;
  if (!d_m) return -4;
  if (!d_v) return -5;
  if (t < 1) return -6;
  if (!(lr > 0.0f)) return -7;
  if (!(beta1 >= 0.0f && beta1 < 1.0f)) return -8;
  if (!(beta2 >= 0.0f && beta2 < 1.0f)) return -9;
  if (!(eps > 0.0f)) return -10;
  if (!(weight_decay >= 0.0f)) return -11;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  k_mlp_adam<<<nblk(NP, 256), 256, 0, (cudaStream_t)stream>>>(d_w32, (__nv_bfloat16*)d_w16, d_grad, d_m, d_v, lr,
                                                               beta1, beta2, eps, weight_decay, c1, c2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_cuda_error((int)e);
    return QRDM_ERR_CUDA;
  }
  return 0;
}

int qrdm_mlp_train(float* d_w32, void* d_w16, float* d_adam, const float* d_x, const float* d_t, int64_t nsamples,
                   int64_t batch, int64_t steps, float lr, float weight_decay, uint64_t seed, float* d_loss_log,
                   float* d_work, size_t work_bytes, void* stream) {
  if (!d_w32) return -1;
  if (!d_w16) return -2;
  if (!d_adam) return -3;
  if (!d_x) return -4;
  if (!d_t) return -5;
  if (nsamples < 1) return -6;
  if (batch < 1 || batch > (1 << 24)) return -7;
  if (steps < 0) return -8;
  if (!(lr > 0.0f)) return -9;
  if (!(weight_decay >= 0.0f)) return -10;
  if (!d_work || work_bytes < acts_floats(batch) * sizeof(float)) return QRDM_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const Acts a = acts(d_work, batch);
  float* m = d_adam;
  float* v = d_adam + NP;
  __nv_bfloat16* w16o = (__nv_bfloat16*)d_w16;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t it = 0; it < steps; ++it) {
    k_mlp_gather<<<nblk(batch, 256), 256, 0, s>>>(d_x, d_t, nsamples, batch, seed, it, a.xb, a.tb);
    cudaError_t e = forward(w16o, a.xb, batch, a.h1, a.h2, a.y, s);
    if (e == cudaSuccess) e = backward(w16o, a.xb, a.tb, batch, a, s);
    if (e == cudaSuccess && d_loss_log)
      e = cudaMemcpyAsync(d_loss_log + it, a.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      set_last_cuda_error((int)e);
      return QRDM_ERR_CUDA;
    }
    const float c1 = 1.0f - powf(b1, (float)(it + 1)), c2 = 1.0f - powf(b2, (float)(it + 1));
    k_mlp_adam<<<nblk(NP, 256), 256, 0, s>>>(d_w32, w16o, a.g, m, v, lr, b1, b2, eps, weight_decay, c1, c2);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_cuda_error((int)e);
      return QRDM_ERR_CUDA;
    }
  }
  return 0;
}

}  // extern "C"
