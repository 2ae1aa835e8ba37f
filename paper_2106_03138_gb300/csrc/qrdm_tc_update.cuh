// a9, tensor-core forms (opts.precision = 2: split-BF16x3, 3: 3xTF32).
//
// The panel's sub-panels update only the remaining panel columns (FP64);
// the trailing block A22 = A[ns:, ns+k:] then receives one merged update with
// all l reflectors of the step (l <= 64), as in Alg. 4:
//   T   = the l x l compact-WY factor of the step (k_tc_vtv + k_tc_tbuild),
//   W   = T^T V^T A22          (k_tc_w over row segments, tcgen05; k_tc_wsum),
//   A22 = A22 - V W                                (k_tc_update, tcgen05).
// One pass over A22 for W and one for the update instead of one pair per
// sub-panel: the form is HBM-bound, and the merge divides its traffic by the
// number of sub-panels.  Operands are converted on load: FP64 -> FP32 (round
// to nearest, integer pipe) -> x = hi + lo with hi, lo BF16 (precision 2) or
// TF32 (precision 3); each product uses hi*hi + hi*lo + lo*hi (lo*lo dropped:
// about 2^-17 relative for BF16, 2^-21 for TF32), FP32 accumulation in TMEM.
// A stays FP64 in HBM.
#pragma once

#include "qrdm_kernels.cuh"
#include "qrdm_tc.cuh"

namespace qrdm {

constexpr int TC_THREADS = 256;
constexpr int TCW_COLS = 128;   // columns per CTA of the W GEMM (its M)
constexpr int TCU_ROWS = 128;   // rows per CTA of the update (its M)
constexpr int TCU_COLS = 256;   // columns per CTA of the update (its N)
constexpr int TC_LMAX = 64;     // reflectors per merged update (K of the update, N of the W GEMM)
constexpr long long TC_WAIT = 2000000000LL;  // clock cycles before an MMA wait gives up (about 1 s)
constexpr int TCW_TILE_A = TCW_COLS * 128;   // bytes of one A tile (128 rows x one 128-byte atom of K)
constexpr int TCW_TILE_V = TC_LMAX * 128;    // bytes of one V tile (64 rows x one atom of K)
constexpr int TCW_STAGE = 2 * TCW_TILE_A + 2 * TCW_TILE_V;
constexpr int TCW_SMEM = 1024 + 2 * TCW_STAGE + 64;

// operand format: 1 BF16 (kind::f16), 2 TF32 (kind::tf32); K of one 128-byte atom
template <int FMT>
struct TcFmt {
  static constexpr int ESZ = (FMT == 1) ? 2 : 4;
  static constexpr int KA = 128 / ESZ;        // elements of K per atom
  static constexpr int NA = TC_LMAX / KA;     // atoms for the 64 reflectors of the update
};
template <int FMT>
constexpr int tcu_smem() {
  return 1024 + 2 * TCU_ROWS * 128 * TcFmt<FMT>::NA + 2 * TCU_COLS * 128 * TcFmt<FMT>::NA + 64;
}
constexpr int TCV_ROWS_MIN = 128;  // rows per CTA of k_tc_vtv (at least)
constexpr int TCV_CHUNKS = 64;     // at most this many row chunks (partial V^T V in the Gram partials buffer)

template <int FMT>
__device__ __forceinline__ void tc_put(unsigned char* hi, unsigned char* lo, uint32_t off, float x) {
  if (FMT == 1) {
    __nv_bfloat16 h, l;
    tc::split_bf16(x, &h, &l);
    *reinterpret_cast<__nv_bfloat16*>(hi + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + off) = l;
  } else {
    const float h = tc::tf32_rna(x);
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = tc::tf32_rna(x - h);
  }
}

template <int FMT>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (FMT == 1)
    tc::mma_bf16(d, a, b, idesc, acc);
  else
    tc::mma_tf32(d, a, b, idesc, acc);
}

// the step's reflectors V^T V (pairs i < j, unit diagonal convention): partial
// sums over row chunks, one chunk per CTA, into Gp[chunk][pair index]
__global__ void __launch_bounds__(TC_THREADS) k_tc_vtv(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 1 || st->k >= P.n - ns || mr <= 0) return;
  __shared__ double s_v[64][TC_LMAX + 1];
  const int64_t per = max((int64_t)TCV_ROWS_MIN, (mr + TCV_CHUNKS - 1) / TCV_CHUNKS);
  const int64_t nch = (mr + per - 1) / per;
  const int tid = threadIdx.x;
  const int npair = l * (l - 1) / 2;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int64_t rb = ch * per, re = min(mr, rb + per);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int64_t r0 = rb; r0 < re; r0 += 64) {
      const int rows = (int)min((int64_t)64, re - r0);
      __syncthreads();
      for (int e = tid; e < 64 * l; e += TC_THREADS) {
        const int t = e / 64, rr = e % 64;
        s_v[rr][t] = (rr < rows) ? vget(P.A, P.lda, ns, r0 + rr, t) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = tid + q * TC_THREADS;
        if (e < npair) {
          int j = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);  // e -> (i < j)
          while (j * (j - 1) / 2 > e) --j;
          while ((j + 1) * j / 2 <= e) ++j;
          const int i = e - j * (j - 1) / 2;
          double s = acc[q];
          for (int rr = 0; rr < rows; ++rr) s = fma(s_v[rr][i], s_v[rr][j], s);
          acc[q] = s;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * TC_THREADS;
      if (e < npair) P.Gp[ch * (int64_t)P.kmax * P.kmax + e] = acc[q];
    }
  }
}

// T (l x l, forward columnwise): T_jj = htau_j, T[0:j, j] = -htau_j T[0:j, 0:j] S[0:j, j]
// with S = V^T V summed from the partials; one CTA; T into P.T (column-major, ld KMAX)
__global__ void __launch_bounds__(TC_THREADS) k_tc_tbuild(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 0 || st->k >= P.n - ns || mr <= 0) return;
  __shared__ double s_t[TC_LMAX][TC_LMAX + 1];
  double* S = P.G;  // V^T V (row i, column j at i * kmax + j); the step's Gram is no longer needed
  const int64_t per = max((int64_t)TCV_ROWS_MIN, (mr + TCV_CHUNKS - 1) / TCV_CHUNKS);
  const int64_t nch = (mr + per - 1) / per;
  const int tid = threadIdx.x;
  const int npair = l * (l - 1) / 2;
  for (int e = tid; e < npair; e += TC_THREADS) {
    int j = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);
    while (j * (j - 1) / 2 > e) --j;
    while ((j + 1) * j / 2 <= e) ++j;
    const int i = e - j * (j - 1) / 2;
    double s = 0.0;
    for (int64_t c = 0; c < nch; ++c) s += P.Gp[c * (int64_t)P.kmax * P.kmax + e];
    S[(int64_t)i * P.kmax + j] = s;
  }
  for (int e = tid; e < TC_LMAX * TC_LMAX; e += TC_THREADS) s_t[e / TC_LMAX][e % TC_LMAX] = 0.0;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    const double ht = P.htau[ns + j];
    if (tid < j) {
      double s = 0.0;
      for (int q = tid; q < j; ++q) s = fma(s_t[tid][q], S[(int64_t)q * P.kmax + j], s);
      s_t[tid][j] = -ht * s;
    }
    if (tid == 0) s_t[j][j] = ht;
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += TC_THREADS) {
    const int r = e % l, c = e / l;
    P.T[(int64_t)c * KMAX + r] = (r <= c) ? s_t[r][c] : 0.0;
  }
}

// Split over rows (split-K): segment s of the rows gets its own CTAs, so that
// a narrow trailing block still fills the SMs; the segments' partial sums are
// added in FP64.
constexpr int TC_SEG_ROWS_MIN = 512;
constexpr int TC_SEG_ALIGN = 64;  // segment rows are a multiple of every format's K atom
__device__ __forceinline__ void tc_segments(int64_t mr, int nseg_max, int ka, int64_t* nseg, int64_t* seg_rows) {
  int64_t ns_ = (mr + TC_SEG_ROWS_MIN - 1) / TC_SEG_ROWS_MIN;
  if (ns_ > nseg_max) ns_ = nseg_max;
  if (ns_ < 1) ns_ = 1;
  int64_t sr = (mr + ns_ - 1) / ns_;
  sr = (sr + ka - 1) / ka * ka;
  *nseg = (mr + sr - 1) / sr;
  *seg_rows = sr;
}

// partial V^T A22 over one row segment for 128 trailing columns: D (columns x
// 64 reflectors) in TMEM, stages of one K atom of rows, double-buffered; every
// thread issues its stage's global loads before converting them.  The tensor
// core's FP32 accumulation does not round to nearest, so its error grows with
// the number of MMAs summed into one accumulator: each chunk of rows gets its
// own accumulator (two alternate in TMEM), which the warps add into FP32
// registers (round to nearest) once the chunk's MMAs are done, while the next
// chunk's MMAs run.  Raw sums to Wpart[segment][column][64].
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS) k_tc_w(Params P) {
  constexpr int ESZ = TcFmt<FMT>::ESZ, KA = TcFmt<FMT>::KA;
  constexpr int NLA = TCW_COLS * KA / TC_THREADS;  // A elements per thread and stage
  constexpr int NLV = TC_LMAX * KA / TC_THREADS;   // V elements per thread and stage
  constexpr int HALF = TC_LMAX / 2;                // reflector sums each thread keeps
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, j0 = ns + st->k;
  const int64_t n2 = P.n - j0, mr = P.m - ns, lda = P.lda;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  const int64_t c0 = j0 + (int64_t)blockIdx.x * TCW_COLS;
  int64_t nseg, seg_rows;
  tc_segments(mr, P.tc_nseg, TC_SEG_ALIGN, &nseg, &seg_rows);
  const int64_t seg = blockIdx.y;
  if (c0 >= P.n || seg >= nseg) return;
  if (blockIdx.x == 0 && seg == 0 && threadIdx.x == 0)
    add_flops(st, KID_TRAIL_W, 2.0 * (double)mr * (double)n2 * l);
  const int64_t rbeg = seg * seg_rows, rend = min(mr, rbeg + seg_rows);
  extern __shared__ unsigned char tcw_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcw_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* stg[2] = {base, base + TCW_STAGE};
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 2 * TCW_STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (wp == 0) tc::tmem_alloc(tslot, 2 * TC_LMAX);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    *s_fail = 0;
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  // this thread's TMEM view: lanes of its warp quarter, its half of the reflectors
  const uint32_t tview = taddr + ((uint32_t)((wp & 3) * 32) << 16) + (uint32_t)((wp >> 2) * HALF);
  float wsum[HALF];
#pragma unroll
  for (int t = 0; t < HALF; ++t) wsum[t] = 0.0f;
  const uint32_t idesc = tc::idesc_f32acc(TCW_COLS, TC_LMAX, FMT);
  const int64_t nchunks = (rend - rbeg + KA - 1) / KA;
  for (int64_t i = 0; i < nchunks; ++i) {
    const int s = (int)(i & 1);
    const int64_t r0 = rbeg + i * KA;  // relative to ns
    double xa[NLA], xv[NLV];
#pragma unroll
    for (int q = 0; q < NLA; ++q) {
      const int e = tid + q * TC_THREADS;
      const int c = e / KA, kk = e % KA;
      const int64_t col = c0 + c, rr = r0 + kk;
      xa[q] = (col < P.n && rr < rend) ? P.A[col * lda + ns + rr] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < NLV; ++q) {
      const int e = tid + q * TC_THREADS;
      const int t = e / KA, kk = e % KA;
      const int64_t rr = r0 + kk;
      xv[q] = (t < l && rr < rend) ? vget(P.A, lda, ns, rr, t) : 0.0;
    }
    if (i >= 2) {  // the MMAs of chunk i - 2 have finished with this stage and accumulator
      if (tid == 0 && !tc::mbar_wait(&bar[s], (uint32_t)(((i >> 1) - 1) & 1), TC_WAIT)) *s_fail = 1;
      __syncthreads();
      if (*s_fail) break;
      tc::fence_after_sync();
#pragma unroll
      for (int q = 0; q < HALF / 16; ++q) {
        float g[16];
        tc::tmem_ld16(tview + (uint32_t)(s * TC_LMAX + q * 16), g);
#pragma unroll
        for (int v = 0; v < 16; ++v) wsum[q * 16 + v] += g[v];
      }
    }
    unsigned char* aH = stg[s];
    unsigned char* aL = aH + TCW_TILE_A;
    unsigned char* vH = aL + TCW_TILE_A;
    unsigned char* vL = vH + TCW_TILE_V;
#pragma unroll
    for (int q = 0; q < NLA; ++q) {
      const int e = tid + q * TC_THREADS;
      tc_put<FMT>(aH, aL, tc::sw128_off_e<ESZ>(e / KA, e % KA), f64_to_f32_rn(xa[q]));
    }
#pragma unroll
    for (int q = 0; q < NLV; ++q) {
      const int e = tid + q * TC_THREADS;
      tc_put<FMT>(vH, vL, tc::sw128_off_e<ESZ>(e / KA, e % KA), f64_to_f32_rn(xv[q]));
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_h = tc::smem_u32(aH), a_l = tc::smem_u32(aL), v_h = tc::smem_u32(vH), v_l = tc::smem_u32(vL);
      const uint32_t d = taddr + (uint32_t)(s * TC_LMAX);
      // the small cross terms first: the truncation of each MMA's sum is then
      // at the scale of the full sum only for the hi*hi terms
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(d, tc::sw128_desc(a_h + o), tc::sw128_desc(v_l + o), idesc, kk > 0 ? 1u : 0u);
        tc_mma<FMT>(d, tc::sw128_desc(a_l + o), tc::sw128_desc(v_h + o), idesc, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(d, tc::sw128_desc(a_h + o), tc::sw128_desc(v_h + o), idesc, 1u);
      }
      tc::mma_commit(&bar[s]);
    }
  }
  // the last one or two chunks are still in their accumulators; the commit of
  // the last chunk covers every MMA issued before it
  const int64_t last = nchunks - 1;
  if (tid == 0 && !*s_fail && !tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), TC_WAIT)) *s_fail = 1;
  __syncthreads();
  tc::fence_after_sync();
  if (*s_fail) {
    if (tid == 0 && atomicExch(&st->abort_flag, 1) == 0) st->diag_code = 4;
  } else {
    for (int64_t i = max((int64_t)0, last - 1); i <= last; ++i) {
#pragma unroll
      for (int q = 0; q < HALF / 16; ++q) {
        float g[16];
        tc::tmem_ld16(tview + (uint32_t)((int)(i & 1) * TC_LMAX + q * 16), g);
#pragma unroll
        for (int v = 0; v < 16; ++v) wsum[q * 16 + v] += g[v];
      }
    }
    // thread = trailing column (TMEM lane) and one half of its reflector sums
    const int64_t col = c0 + (wp & 3) * 32 + lane;
    if (col < P.n) {
      float4* o4 = reinterpret_cast<float4*>(P.Wt + ((seg + 1) * P.n + col) * TC_LMAX + (wp >> 2) * HALF);
#pragma unroll
      for (int v = 0; v < HALF / 4; ++v)
        o4[v] = make_float4(wsum[4 * v], wsum[4 * v + 1], wsum[4 * v + 2], wsum[4 * v + 3]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wp == 0) tc::tmem_dealloc(taddr, 2 * TC_LMAX);
}

// W = T^T (sum of the segments' V^T A22) per trailing column: one warp per
// column; lanes t and t + 32 sum their reflector's segments in FP64, then
// apply T (upper, from P.T) in FP32 and write Wt[col][64].
__global__ void __launch_bounds__(TC_THREADS) k_tc_wsum(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, j0 = ns + st->k;
  const int64_t n2 = P.n - j0, mr = P.m - ns;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  __shared__ float s_T[TC_LMAX][TC_LMAX + 1];
  __shared__ float s_g[TC_THREADS / 32][TC_LMAX];
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < TC_LMAX * TC_LMAX; e += TC_THREADS) {
    const int q = e / TC_LMAX, t = e % TC_LMAX;
    s_T[q][t] = (q < l && t < l && q <= t) ? (float)P.T[(int64_t)t * KMAX + q] : 0.0f;
  }
  __syncthreads();
  int64_t nseg, seg_rows;
  tc_segments(mr, P.tc_nseg, TC_SEG_ALIGN, &nseg, &seg_rows);
  (void)seg_rows;
  const int64_t gw = (int64_t)blockIdx.x * (TC_THREADS / 32) + wp;
  const int64_t nwarps = (int64_t)gridDim.x * (TC_THREADS / 32);
  for (int64_t c = gw; c < n2; c += nwarps) {
    const int64_t col = j0 + c;
    double g0 = 0.0, g1 = 0.0;
    for (int64_t sg = 0; sg < nseg; ++sg) {
      const float* part = P.Wt + ((sg + 1) * P.n + col) * TC_LMAX;
      g0 += (double)part[lane];
      g1 += (double)part[lane + 32];
    }
    s_g[wp][lane] = (float)g0;
    s_g[wp][lane + 32] = (float)g1;
    __syncwarp();
    float w0 = 0.0f, w1 = 0.0f;
    for (int q = 0; q <= lane; ++q) w0 = fmaf(s_T[q][lane], s_g[wp][q], w0);
    for (int q = 0; q <= lane + 32; ++q) w1 = fmaf(s_T[q][lane + 32], s_g[wp][q], w1);
    P.Wt[col * TC_LMAX + lane] = w0;
    P.Wt[col * TC_LMAX + lane + 32] = w1;
    __syncwarp();
  }
}

// A22 tile (128 rows x 256 columns) -= V (rows x l) W (l x columns), K = 64
// reflectors in NA atoms
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS) k_tc_update(Params P) {
  constexpr int ESZ = TcFmt<FMT>::ESZ, KA = TcFmt<FMT>::KA, NA = TcFmt<FMT>::NA;
  constexpr int TV = TCU_ROWS * 128;  // bytes of one atom of the V tile
  constexpr int TW = TCU_COLS * 128;  // bytes of one atom of the W tile
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, j0 = ns + st->k;
  const int64_t n2 = P.n - j0, mr = P.m - ns, lda = P.lda;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  const int64_t r0 = (int64_t)blockIdx.x * TCU_ROWS;
  const int64_t cb = j0 + (int64_t)blockIdx.y * TCU_COLS;
  if (r0 >= mr || cb >= P.n) return;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    add_flops(st, KID_TRAIL_UPDATE, 2.0 * (double)mr * (double)n2 * l);
  extern __shared__ unsigned char tcu_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcu_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* vH = base;
  unsigned char* vL = vH + NA * TV;
  unsigned char* wH = vL + NA * TV;
  unsigned char* wL = wH + NA * TW;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wL + NA * TW);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (wp == 0) tc::tmem_alloc(tslot, TCU_COLS);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    *s_fail = 0;
  }
  for (int e = tid; e < TCU_ROWS * 64; e += TC_THREADS) {
    const int t = e >> 7, r = e & 127;
    const int64_t rr = r0 + r;
    const double v = (t < l && rr < mr) ? vget(P.A, lda, ns, rr, t) : 0.0;
    tc_put<FMT>(vH, vL, (t / KA) * TV + tc::sw128_off_e<ESZ>(r, t % KA), f64_to_f32_rn(v));
  }
  for (int e = tid; e < TCU_COLS * 64; e += TC_THREADS) {
    const int c = e >> 6, t = e & 63;
    const int64_t col = cb + c;
    const float w = (col < P.n && t < l) ? P.Wt[col * TC_LMAX + t] : 0.0f;
    tc_put<FMT>(wH, wL, (t / KA) * TW + tc::sw128_off_e<ESZ>(c, t % KA), w);
  }
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_f32acc(TCU_ROWS, TCU_COLS, FMT);
    // cross terms first, then hi*hi (only those truncate at the scale of the sum)
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const uint32_t v_h = tc::smem_u32(vH + a * TV), v_l = tc::smem_u32(vL + a * TV);
      const uint32_t w_h = tc::smem_u32(wH + a * TW), w_l = tc::smem_u32(wL + a * TW);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(taddr, tc::sw128_desc(v_h + o), tc::sw128_desc(w_l + o), idesc, (a > 0 || kk > 0) ? 1u : 0u);
        tc_mma<FMT>(taddr, tc::sw128_desc(v_l + o), tc::sw128_desc(w_h + o), idesc, 1u);
      }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const uint32_t v_h = tc::smem_u32(vH + a * TV), w_h = tc::smem_u32(wH + a * TW);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(taddr, tc::sw128_desc(v_h + o), tc::sw128_desc(w_h + o), idesc, 1u);
      }
    }
    tc::mma_commit(bar);
    if (!tc::mbar_wait(bar, 0u, TC_WAIT)) *s_fail = 1;
  }
  __syncthreads();
  tc::fence_after_sync();
  if (*s_fail) {
    if (tid == 0 && atomicExch(&st->abort_flag, 1) == 0) st->diag_code = 4;
  } else {
    // thread = row (TMEM lane of its quarter); warps w and w + 4 split the columns
    const int q4 = wp & 3, half = wp >> 2;
    const int64_t rr = r0 + q4 * 32 + lane;
    double* a = P.A + ns + rr;
    for (int cc = half * (TCU_COLS / 2); cc < (half + 1) * (TCU_COLS / 2); cc += 16) {
      float v[16];
      tc::tmem_ld16(taddr + ((uint32_t)(q4 * 32) << 16) + cc, v);
      if (rr < mr) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int64_t col = cb + cc + i;
          if (col < P.n) a[col * lda] -= (double)v[i];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wp == 0) tc::tmem_dealloc(taddr, TCU_COLS);
}

}  // namespace qrdm
