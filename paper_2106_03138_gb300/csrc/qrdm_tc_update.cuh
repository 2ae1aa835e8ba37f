// a9, tensor-core forms (opts.precision = 2: split-BF16x3, 3: 3xTF32).
//
// The panel's sub-panels update only the remaining panel columns (FP64);
// the trailing block A22 = A[ns:, ns+k:] then receives one merged update with
// all l reflectors of the step (l <= 64), as in Alg. 4:
//   T   = the l x l compact-WY factor of the step (k_tc_vtv + k_tc_tbuild),
//   V   -> hi/lo operand images in global memory (k_tc_vimg),
//   W   = T^T V^T A22   (k_tc_w over row segments, tcgen05; k_tc_wsum, which
//                        also writes W's hi/lo operand image),
//   A22 = A22 - V W                                (k_tc_update, tcgen05).
// One pass over A22 for W and one for the update instead of one pair per
// sub-panel: the form is HBM-bound, and the merge divides its traffic by the
// number of sub-panels.  Operands are split on load: FP64 -> FP32 (round to
// nearest, integer pipe) -> x = hi + lo with hi, lo BF16 (precision 2) or
// TF32 (precision 3); each product uses hi*hi + hi*lo + lo*hi (lo*lo
// dropped), exact to 3 * 2^-16 relative for BF16 and about 2^-20 for TF32 at
// worst (2^-18.6 and 2^-24 typical); FP32 accumulation in TMEM.
// A stays FP64 in HBM.  V and W, small and read by many CTAs, are split once
// per step into images laid out exactly as the MMA's shared-memory tiles
// (K-major, 128-byte swizzle), which the kernels copy without conversion.
// The candidate Gram matrix of the DM selection (a3) runs on the tensor cores
// with the same split (k_tc_gram).  Where many MMAs add into one result (the
// W pass and the Gram, K = rows), each K atom gets its own TMEM accumulator,
// summed in FP32 registers with round-to-nearest: the tensor core's own FP32
// accumulation truncates.
#pragma once

#include <cuda.h>

#include "qrdm_kernels.cuh"
#include "qrdm_tc.cuh"

namespace qrdm {

constexpr int TC_THREADS = 256;
constexpr int TCW_COLS = 128;   // columns per CTA of the W GEMM (its M)
constexpr int TCU_ROWS = 128;   // rows of one update tile (its M)
constexpr int TCU_COLS = 128;   // columns of one update tile (its N)
constexpr int TC_LMAX = 64;     // reflectors per merged update (K of the update, N of the W GEMM)
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
// V hi/lo for one row block, W hi/lo for two column tiles (double-buffered)
template <int FMT>
constexpr int tcu_smem() {
  return 1024 + 6 * 128 * 128 * TcFmt<FMT>::NA + 64;
}
constexpr int TCV_ROWS_MIN = 128;  // rows per CTA of k_tc_vtv (at least)
constexpr int TCV_CHUNKS = 128;    // at most this many row chunks (partial V^T V in the Gram partials buffer)
constexpr int TC_ATOM = 128 * 128;  // bytes of one K atom of a 128-row operand tile
constexpr int TC_NSEG_MAX = 16;     // most row segments of the W pass (FP32 partials n x 64 each)

// bytes of one operand image over `rows` rows (or columns), either format:
// V for the W pass (per K chunk: 64 reflector rows x 128 B, hi then lo), V for
// the update (per 128-row block: NA atoms hi, NA atoms lo) and W for the
// update (per 128-column tile, the same) all fit in 512 B per row, padded
__host__ __device__ constexpr size_t tc_img_bytes(int64_t rows) { return (size_t)(rows + 256) * 512; }

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
// sums over row chunks, one chunk per CTA, into Gp[chunk][pair index].  R is
// the arithmetic within a chunk: FP64 for the exact merged form, FP32 for the
// tensor-core forms (whose T is applied in FP32); chunks are added in FP64.
template <typename R>
__global__ void __launch_bounds__(TC_THREADS) k_tc_vtv(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 1 || st->k >= P.n - ns || mr <= 0) return;
  __shared__ R s_v[64][TC_LMAX + 1];
  const int64_t per = max((int64_t)TCV_ROWS_MIN, (mr + TCV_CHUNKS - 1) / TCV_CHUNKS);
  const int64_t nch = (mr + per - 1) / per;
  const int tid = threadIdx.x;
  const int npair = l * (l - 1) / 2;
  // this thread's pairs e = tid + 256 q -> (i < j)
  int pi[8], pj[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + q * TC_THREADS;
    int j = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);
    while (j * (j - 1) / 2 > e) --j;
    while ((j + 1) * j / 2 <= e) ++j;
    pj[q] = j;
    pi[q] = e - j * (j - 1) / 2;
  }
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int64_t rb = ch * per, re = min(mr, rb + per);
    R acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = (R)0;
    for (int64_t r0 = rb; r0 < re; r0 += 64) {
      const int rows = (int)min((int64_t)64, re - r0);
      __syncthreads();
      for (int e = tid; e < 64 * l; e += TC_THREADS) {
        const int t = e / 64, rr = e % 64;
        const double v = (rr < rows) ? vget(P.A, P.lda, ns, r0 + rr, t) : 0.0;
        s_v[rr][t] = (sizeof(R) == 4) ? (R)f64_to_f32_rn(v) : (R)v;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (tid + q * TC_THREADS < npair) {
          R x = acc[q];
          for (int rr = 0; rr < rows; ++rr) x = fmat(s_v[rr][pi[q]], s_v[rr][pj[q]], x);
          acc[q] = x;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + q * TC_THREADS;
      if (e < npair) P.Gp[ch * (int64_t)P.kmax * P.kmax + e] = (sizeof(R) == 4) ? f32_to_f64((float)acc[q]) : (double)acc[q];
    }
  }
}

// T (l x l, forward columnwise): T_jj = htau_j, T[0:j, j] = -htau_j T[0:j, 0:j] S[0:j, j]
// with S = V^T V summed from the chunk partials (chunk-outer, so that each
// thread's loads are independent; the order of the sum is the chunk order);
// S and T in shared memory; one CTA; T into P.T (column-major, ld KMAX)
constexpr int TCB_SMEM = 2 * TC_LMAX * (TC_LMAX + 1) * (int)sizeof(double);
__global__ void __launch_bounds__(TC_THREADS) k_tc_tbuild(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 0 || st->k >= P.n - ns || mr <= 0) return;
  extern __shared__ double tb_smem[];
  double (*s_t)[TC_LMAX + 1] = reinterpret_cast<double (*)[TC_LMAX + 1]>(tb_smem);
  double (*s_s)[TC_LMAX + 1] = reinterpret_cast<double (*)[TC_LMAX + 1]>(tb_smem + TC_LMAX * (TC_LMAX + 1));
  const int64_t per = max((int64_t)TCV_ROWS_MIN, (mr + TCV_CHUNKS - 1) / TCV_CHUNKS);
  const int64_t nch = (mr + per - 1) / per;
  const int tid = threadIdx.x;
  const int npair = l * (l - 1) / 2;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  if (l > 1) {
    for (int64_t c = 0; c < nch; ++c) {
      const double* g = P.Gp + c * (int64_t)P.kmax * P.kmax;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = tid + q * TC_THREADS;
        if (e < npair) acc[q] += g[e];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + q * TC_THREADS;
    if (e < npair) {
      int j = (int)((sqrtf(8.0f * (float)e + 1.0f) + 1.0f) * 0.5f);
      while (j * (j - 1) / 2 > e) --j;
      while ((j + 1) * j / 2 <= e) ++j;
      s_s[e - j * (j - 1) / 2][j] = acc[q];
    }
  }
  for (int e = tid; e < TC_LMAX * TC_LMAX; e += TC_THREADS) s_t[e / TC_LMAX][e % TC_LMAX] = 0.0;
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    const double ht = P.htau[ns + j];
    if (tid < j) {
      double x = 0.0;
      for (int q = tid; q < j; ++q) x = fma(s_t[tid][q], s_s[q][j], x);
      s_t[tid][j] = -ht * x;
    }
    if (tid == 0) s_t[j][j] = ht;
    __syncthreads();
  }
  for (int e = tid; e < l * l; e += TC_THREADS) {
    const int r = e % l, c = e / l;
    P.T[(int64_t)c * KMAX + r] = (r <= c) ? s_t[r][c] : 0.0;
  }
}

// S = V^T V of the step (pairs i < j), the chunk partials of k_tc_vtv summed
// in FP64 in chunk order, into P.G (packed, pair e = j (j - 1) / 2 + i): the
// tensor-core forms apply the step's block reflector through S (k_tc_wsum)
// instead of forming T.
__global__ void __launch_bounds__(TC_THREADS) k_tc_sred(Params P) {
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 1 || st->k >= P.n - ns || mr <= 0) return;
  const int64_t per = max((int64_t)TCV_ROWS_MIN, (mr + TCV_CHUNKS - 1) / TCV_CHUNKS);
  const int64_t nch = (mr + per - 1) / per;
  const int npair = l * (l - 1) / 2;
  for (int e = blockIdx.x * TC_THREADS + threadIdx.x; e < npair; e += gridDim.x * TC_THREADS) {
    P.G[e] = sum_strided(P.Gp + e, (int64_t)P.kmax * P.kmax, nch);
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

// The W pass reads A22 in 16-byte units when it can: with an even lda and a
// 16-byte-aligned A, its rows start at the even row ns - o (o = ns mod 2);
// row ns - 1 meets a zero row of V's image, so it adds nothing.
__device__ __forceinline__ int tc_shift(const Params& P, int64_t ns) { return (P.tc_al && (ns & 1)) ? 1 : 0; }

// V's operand images, one element per thread (rows padded with zeros to the
// next 128): Vw for the W pass (chunk of KA rows: reflector t is the tile's
// row, the chunk's rows its K) and Vu for the update (block of 128 rows: row
// r is the tile's row, the reflectors its K, in NA atoms; shifted by o rows
// like Vw when the update streams A by tensor copies)
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS) k_tc_vimg(Params P) {
  constexpr int ESZ = TcFmt<FMT>::ESZ, KA = TcFmt<FMT>::KA, NA = TcFmt<FMT>::NA;
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, mr = P.m - ns;
  if (l <= 0 || st->k >= P.n - ns || mr <= 0) return;
  const int o = tc_shift(P, ns);  // Vw row r holds V row r - o
  const int64_t pad = (mr + o + 127) / 128 * 128;
  const int64_t total = pad * TC_LMAX;
  for (int64_t e = (int64_t)blockIdx.x * TC_THREADS + threadIdx.x; e < total; e += (int64_t)gridDim.x * TC_THREADS) {
    const int t = (int)(e / pad);
    const int64_t r = e % pad;
    const double v0 = (t < l && r < mr) ? vget(P.A, P.lda, ns, r, t) : 0.0;
    const double vw = (o == 0) ? v0 : ((t < l && r >= 1 && r - 1 < mr) ? vget(P.A, P.lda, ns, r - 1, t) : 0.0);
    const double vu = P.tcu_tma ? vw : v0;  // the streamed update's tiles start at the same even row
    unsigned char* w = P.tc_vw + (r / KA) * (2 * TC_LMAX * 128);
    tc_put<FMT>(w, w + TC_LMAX * 128, tc::sw128_off_e<ESZ>(t, (int)(r % KA)), f64_to_f32_rn(vw));
    unsigned char* u = P.tc_vu + (r / 128) * (2 * NA * TC_ATOM) + (t / KA) * TC_ATOM;
    tc_put<FMT>(u, u + NA * TC_ATOM, tc::sw128_off_e<ESZ>((int)(r % 128), t % KA), f64_to_f32_rn(vu));
  }
}

// FP32 x[0..EPC) -> one 16-byte chunk of hi and one of lo (EPC = 8 BF16 or
// 4 TF32 elements)
template <int FMT>
__device__ __forceinline__ void tc_split16(const float* x, uint4* hi, uint4* lo) {
  if (FMT == 1) {
    uint32_t h[4], w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
      const float2 hf = __bfloat1622float2(hb);
      const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
      h[i] = *reinterpret_cast<const uint32_t*>(&hb);
      w[i] = *reinterpret_cast<const uint32_t*>(&lb);
    }
    *hi = make_uint4(h[0], h[1], h[2], h[3]);
    *lo = make_uint4(w[0], w[1], w[2], w[3]);
  } else {
    float h[4], w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = tc::tf32_rna(x[i]);
      w[i] = tc::tf32_rna(x[i] - h[i]);
    }
    *hi = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
    *lo = make_uint4(__float_as_uint(w[0]), __float_as_uint(w[1]), __float_as_uint(w[2]), __float_as_uint(w[3]));
  }
}

// partial V^T A22 over one row segment for 128 trailing columns: D (columns x
// 64 reflectors) in TMEM, stages of one K atom of rows, double-buffered in
// shared memory.  Thread = (column, 16-byte chunk of the atom) for 2 columns
// 64 apart: it loads the chunk's EPC doubles of each column with plain
// pointer offsets (the loads of chunk i + 1 are issued before chunk i is
// converted, so two chunks are in flight), splits them and stores one
// 16-byte hi and lo chunk each; V's chunk comes from its image (16-byte
// copies).  The tensor core's FP32 accumulation does not round to nearest, so
// its error grows with the number of MMAs summed into one accumulator: each
// chunk of rows gets its own accumulator (two alternate in TMEM), which the
// warps add into FP32 registers (round to nearest) once the chunk's MMAs are
// done, while the next chunk's MMAs run.  Raw sums to
// Wpart[segment][column][64].
constexpr int TCW_THREADS = 512;

template <int FMT>
struct TcwLoad {
  static constexpr int ESZ = TcFmt<FMT>::ESZ, EPC = 16 / ESZ;
  static constexpr int UPT = TCW_COLS * 8 / TCW_THREADS;           // (column, chunk) units per thread
  static constexpr int VPT = 2 * TCW_TILE_V / 16 / TCW_THREADS;    // 16-byte pieces of V per thread
  double a[UPT][EPC];
  uint4 v[VPT];
};

// issue the global loads of chunk i (rows r0 .. r0 + KA relative to ns)
template <int FMT>
__device__ __forceinline__ void tcw_load(TcwLoad<FMT>& L, const double* const* colp, const bool* colok, int64_t i,
                                         int64_t r0, int64_t rend, int kg, const uint4* vsrc, int tid, bool al) {
  constexpr int KA = TcFmt<FMT>::KA, EPC = TcwLoad<FMT>::EPC;
  const bool full = r0 + KA <= rend;
  if (full && al) {  // 16-byte loads: the unit starts at an even row of an aligned column
#pragma unroll
    for (int q = 0; q < TcwLoad<FMT>::UPT; ++q) {
      const double2* src = reinterpret_cast<const double2*>(colp[q] + i * KA);
#pragma unroll
      for (int e = 0; e < EPC / 2; ++e) {
        const double2 d = colok[q] ? src[e] : make_double2(0.0, 0.0);
        L.a[q][2 * e] = d.x;
        L.a[q][2 * e + 1] = d.y;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < TcwLoad<FMT>::UPT; ++q) {
      const double* src = colp[q] + i * KA;
#pragma unroll
      for (int e = 0; e < EPC; ++e) L.a[q][e] = (colok[q] && (full || r0 + kg * EPC + e < rend)) ? src[e] : 0.0;
    }
  }
#pragma unroll
  for (int q = 0; q < TcwLoad<FMT>::VPT; ++q) L.v[q] = vsrc[i * (2 * TCW_TILE_V / 16) + tid + q * TCW_THREADS];
}

template <int FMT>
__device__ __forceinline__ void tcw_store(const TcwLoad<FMT>& L, unsigned char* stage, uint32_t a_off, int tid) {
  constexpr int EPC = TcwLoad<FMT>::EPC;
  unsigned char* aH = stage;
  unsigned char* aL = aH + TCW_TILE_A;
  unsigned char* vH = aL + TCW_TILE_A;  // V hi then lo, as in the image
#pragma unroll
  for (int q = 0; q < TcwLoad<FMT>::UPT; ++q) {
    float f[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) f[e] = f64_to_f32_rn(L.a[q][e]);
    uint4 h, w;
    tc_split16<FMT>(f, &h, &w);
    *reinterpret_cast<uint4*>(aH + a_off + q * (TCW_THREADS / 8) * 128) = h;
    *reinterpret_cast<uint4*>(aL + a_off + q * (TCW_THREADS / 8) * 128) = w;
  }
#pragma unroll
  for (int q = 0; q < TcwLoad<FMT>::VPT; ++q) reinterpret_cast<uint4*>(vH)[tid + q * TCW_THREADS] = L.v[q];
}

template <int FMT>
__global__ void __launch_bounds__(TCW_THREADS, 1) k_tc_w(Params P) {
  constexpr int KA = TcFmt<FMT>::KA;
  constexpr int EPC = TcwLoad<FMT>::EPC, UPT = TcwLoad<FMT>::UPT;
  constexpr int NWQ = TCW_THREADS / 128;       // warps per TMEM lane quarter
  constexpr int PART = TC_LMAX / NWQ;          // reflector sums each thread keeps
  static_assert(KA == 8 * EPC, "an atom row is 8 chunks of 16 bytes");
  static_assert(PART % 16 == 0, "TMEM loads of 16 columns");
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t j0 = st->ns + st->k, n2 = P.n - j0, lda = P.lda;
  if (l <= 0 || n2 <= 0 || P.m - st->ns <= 0) return;
  // rows from the even row ns - o (see tc_shift); row 0 meets V's zero row
  const int o = tc_shift(P, st->ns);
  const int64_t ns = st->ns - o, mr = P.m - ns;
  const int64_t c0 = j0 + (int64_t)blockIdx.x * TCW_COLS;
  int64_t nseg, seg_rows;
  tc_segments(mr, P.tc_nseg, TC_SEG_ALIGN, &nseg, &seg_rows);
  const int64_t seg = blockIdx.y;
  if (c0 >= P.n || seg >= nseg) return;
  if (blockIdx.x == 0 && seg == 0 && threadIdx.x == 0)
    add_flops(st, KID_TC_W, 2.0 * (double)(mr - o) * (double)n2 * l);
  const int64_t rbeg = seg * seg_rows, rend = min(mr, rbeg + seg_rows);
  const bool al = P.tc_al != 0;
  extern __shared__ unsigned char tcw_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcw_raw + 1023) & ~(uintptr_t)1023);
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
  // this thread's TMEM view: lanes of its warp quarter, its part of the reflectors
  const uint32_t tview = taddr + ((uint32_t)((wp & 3) * 32) << 16) + (uint32_t)((wp >> 2) * PART);
  float wsum[PART];
#pragma unroll
  for (int t = 0; t < PART; ++t) wsum[t] = 0.0f;
  // A units: column cq + (TCW_THREADS / 8) q of the tile, 16-byte chunk kg of the atom row
  const int kg = tid & 7, cq = tid >> 3;
  const double* colp[UPT];
  bool colok[UPT];
#pragma unroll
  for (int q = 0; q < UPT; ++q) {
    const int64_t col = c0 + cq + (TCW_THREADS / 8) * q;
    colok[q] = col < P.n;
    colp[q] = P.A + (colok[q] ? col : c0) * lda + ns + rbeg + kg * EPC;
  }
  const uint32_t a_off = (uint32_t)(cq * 128 + ((kg ^ (cq & 7)) << 4));
  const uint4* vsrc = reinterpret_cast<const uint4*>(P.tc_vw + (rbeg / KA) * (2 * TCW_TILE_V));
  const uint32_t idesc = tc::idesc_f32acc(TCW_COLS, TC_LMAX, FMT);
  const int64_t nchunks = (rend - rbeg + KA - 1) / KA;
  int64_t issued = -1;
  TcwLoad<FMT> buf[2];
  tcw_load<FMT>(buf[0], colp, colok, 0, rbeg, rend, kg, vsrc, tid, al);
  // one chunk per step; the loop body is unrolled twice so that the two load
  // buffers are named registers
  for (int64_t i0 = 0; i0 < nchunks; i0 += 2) {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      const int64_t i = i0 + par;
      if (i < nchunks) {
        const int s = par;  // = i & 1
        if (i + 1 < nchunks)
          tcw_load<FMT>(buf[1 - par], colp, colok, i + 1, rbeg + (i + 1) * KA, rend, kg, vsrc, tid, al);
        if (i >= 2) {  // the MMAs of chunk i - 2 have finished with this stage and accumulator
          if (tid == 0 && !tc::mbar_wait(&bar[s], (uint32_t)(((i >> 1) - 1) & 1), P.wait_ns)) *s_fail = 1;
          __syncthreads();
          if (*s_fail) break;
          tc::fence_after_sync();
#pragma unroll
          for (int q = 0; q < PART / 16; ++q) {
            float g[16];
            tc::tmem_ld16(tview + (uint32_t)(s * TC_LMAX + q * 16), g);
#pragma unroll
            for (int v = 0; v < 16; ++v) wsum[q * 16 + v] += g[v];
          }
        }
        unsigned char* stage = base + s * TCW_STAGE;
        tcw_store<FMT>(buf[par], stage, a_off, tid);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after_sync();
          const uint32_t a_h = tc::smem_u32(stage), a_l = a_h + TCW_TILE_A;
          const uint32_t v_h = a_l + TCW_TILE_A, v_l = v_h + TCW_TILE_V;
          const uint32_t d = taddr + (uint32_t)(s * TC_LMAX);
          // the small cross terms first: the truncation of each MMA's sum is
          // then at the scale of the full sum only for the hi*hi terms
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
        issued = i;
      }
    }
    if (*s_fail) break;
  }
  // the last one or two chunks are still in their accumulators; the commit of
  // the last chunk covers every MMA issued before it
  const int64_t last = nchunks - 1;
  if (tid == 0 && !*s_fail && !tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), P.wait_ns)) *s_fail = 1;
  __syncthreads();
  tc::fence_after_sync();
  if (*s_fail) {
    // leave no MMA writing TMEM behind: a bounded wait for the last one issued
    if (tid == 0 && issued >= 0) (void)tc::mbar_wait(&bar[issued & 1], (uint32_t)((issued >> 1) & 1), P.wait_ns);
    if (tid == 0) record_fail(st, FAIL_MMA_WAIT, (int)blockIdx.x, st->step, st->ns, KID_TC_W);
  } else {
    for (int64_t i = max((int64_t)0, last - 1); i <= last; ++i) {
#pragma unroll
      for (int q = 0; q < PART / 16; ++q) {
        float g[16];
        tc::tmem_ld16(tview + (uint32_t)((int)(i & 1) * TC_LMAX + q * 16), g);
#pragma unroll
        for (int v = 0; v < 16; ++v) wsum[q * 16 + v] += g[v];
      }
    }
    // thread = trailing column (TMEM lane) and one part of its reflector sums
    const int64_t col = c0 + (wp & 3) * 32 + lane;
    if (col < P.n) {
      float4* o4 = reinterpret_cast<float4*>(P.Wt + ((seg + 1) * P.n + col) * TC_LMAX + (wp >> 2) * PART);
#pragma unroll
      for (int v = 0; v < PART / 4; ++v)
        o4[v] = make_float4(wsum[4 * v], wsum[4 * v + 1], wsum[4 * v + 2], wsum[4 * v + 3]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wp == 0) tc::tmem_dealloc(taddr, 2 * TC_LMAX);
}

// The W pass with TMA (when A is 16-byte aligned and lda even, P.tc_al),
// warp-specialized.  The FP64 rows of each K chunk arrive by tiled tensor
// copies of 32 rows x 128 columns (32 KB) into a ring of NST boxes, filled as
// soon as the converters release a box, so NST - 1 boxes stay in flight while
// one is converted.  Warps 0-7 convert: 8 lanes per column read 16-byte
// pieces (two rows) side by side and write each pair of rows' hi and lo parts
// straight into the split operand tile (two BF16 in 4 bytes, or two TF32 in
// 8); they also add each finished chunk's accumulator into FP32 registers
// (warp w: TMEM lanes 32 (w mod 4) .. + 31, the tile's columns, and 32 of
// the 64 reflectors).  Warp 8 (one thread) issues the tensor copies, V's
// chunk (one bulk copy from its image), and the MMAs.  Two split stages and
// two accumulators alternate, and the MMAs, their order and the chunk order
// of the sums are those of k_tc_w.
template <int FMT>
struct TcwTma {
  static constexpr int KA = TcFmt<FMT>::KA;
  static constexpr int BOXR = 32;                        // rows of one tensor copy
  static constexpr int BPC = KA / BOXR;                  // boxes per K chunk (2 BF16, 1 TF32)
  static constexpr int NST = 4;                          // FP64 boxes in the ring
  static constexpr int BOX = BOXR * TCW_COLS * 8;        // 32 KB
  static constexpr int THREADS = 288;                    // 8 converter warps and the copy / MMA warp
  static constexpr int SMEM = 1024 + 2 * TCW_STAGE + NST * BOX + 256;
};

template <int FMT>
__global__ void __launch_bounds__(TcwTma<FMT>::THREADS, 1)
    k_tc_w_tma(const __grid_constant__ CUtensorMap tmA, Params P) {
  using G = TcwTma<FMT>;
  constexpr int KA = G::KA, NST = G::NST, BPC = G::BPC, ESZ = TcFmt<FMT>::ESZ;
  constexpr int PART = TC_LMAX / 2;  // reflector sums each converter thread keeps
  static_assert(KA % G::BOXR == 0 && PART % 16 == 0, "whole boxes per chunk, TMEM loads of 16 columns");
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t j0 = st->ns + st->k, n2 = P.n - j0;
  if (l <= 0 || n2 <= 0 || P.m - st->ns <= 0) return;
  const int o = tc_shift(P, st->ns);
  const int64_t ns = st->ns - o, mr = P.m - ns;
  const int64_t c0 = j0 + (int64_t)blockIdx.x * TCW_COLS;
  int64_t nseg, seg_rows;
  tc_segments(mr, P.tc_nseg, TC_SEG_ALIGN, &nseg, &seg_rows);
  const int64_t seg = blockIdx.y;
  if (c0 >= P.n || seg >= nseg) return;
  if (blockIdx.x == 0 && seg == 0 && threadIdx.x == 0)
    add_flops(st, KID_TC_W, 2.0 * (double)(mr - o) * (double)n2 * l);
  const int64_t rbeg = seg * seg_rows, rend = min(mr, rbeg + seg_rows);
  const int64_t nchunks = (rend - rbeg + KA - 1) / KA, nbox = nchunks * BPC;
  extern __shared__ unsigned char tcwt_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcwt_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = base + 2 * TCW_STAGE;  // FP64 boxes
  uint64_t* bar = reinterpret_cast<uint64_t*>(ring + NST * G::BOX);
  uint64_t* b_mma = bar;              // [2] MMAs of split stage / accumulator s done
  uint64_t* b_vt = bar + 2;           // [2] V's chunk landed in split stage s
  uint64_t* b_conv = bar + 4;         // [2] A's chunk converted into split stage s (8 arrivals)
  uint64_t* b_acc = bar + 6;          // [2] accumulator s read (8 arrivals)
  uint64_t* b_full = bar + 8;         // [NST] box landed
  uint64_t* b_free = bar + 8 + NST;   // [NST] box converted (8 arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 8 + 2 * NST);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (wp == 8) tc::tmem_alloc(tslot, 2 * TC_LMAX);
  if (tid == 256) {
    for (int b = 0; b < 8 + 2 * NST; ++b) tc::mbar_init(&bar[b], 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&b_conv[b], 8);
      tc::mbar_init(&b_acc[b], 8);
    }
    for (int b = 0; b < NST; ++b) tc::mbar_init(&b_free[b], 8);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  const unsigned char* vimg = P.tc_vw + (rbeg / KA) * (2 * TCW_TILE_V);
  const long long lim = P.wait_ns;
  int64_t loads = 0, v_iss = 0, v_wait = 0, mma_iss = -1;  // thread 256: copies and MMAs issued / waited
  if (wp == 8) {
    if (lane == 0) {
      bool ok = true;
      auto issue_box = [&](int64_t bx) {
        const int f = (int)(bx % NST);
        tc::mbar_expect_tx(&b_full[f], G::BOX);
        tc::tma_load_2d(ring + f * G::BOX, &tmA, (int32_t)(ns + rbeg + bx * G::BOXR), (int32_t)c0, &b_full[f]);
        loads = bx + 1;
      };
      auto issue_v = [&](int64_t i) {  // V's chunk i into split stage i & 1 (after its A tiles)
        unsigned char* vH = base + (i & 1) * TCW_STAGE + 2 * TCW_TILE_A;
        tc::mbar_expect_tx(&b_vt[i & 1], 2 * TCW_TILE_V);
        tc::bulk_g2s(vH, vimg + i * (2 * TCW_TILE_V), 2 * TCW_TILE_V, &b_vt[i & 1]);
        v_iss = i + 1;
      };
      for (int64_t bx = 0; bx < NST && bx < nbox; ++bx) issue_box(bx);
      issue_v(0);
      if (nchunks > 1) issue_v(1);
      const uint32_t idesc = tc::idesc_f32acc(TCW_COLS, TC_LMAX, FMT);
      for (int64_t i = 0; ok && i < nchunks; ++i) {
        const int s = (int)(i & 1);
        // the chunk's boxes are converted: the ring takes the boxes NST ahead
        for (int b = 0; ok && b < BPC; ++b) {
          const int64_t bx = i * BPC + b;
          if (*s_fail || !tc::mbar_wait(&b_free[bx % NST], (uint32_t)((bx / NST) & 1), lim)) {
            ok = false;
            break;
          }
          if (bx + NST < nbox) issue_box(bx + NST);
        }
        if (!ok) break;
        // split stage s holds chunk i (A converted, V landed) and accumulator s was read
        if (!tc::mbar_wait(&b_conv[s], (uint32_t)((i >> 1) & 1), lim) ||
            !tc::mbar_wait(&b_vt[s], (uint32_t)((i >> 1) & 1), lim) ||
            (i >= 2 && !tc::mbar_wait(&b_acc[s], (uint32_t)(((i - 2) >> 1) & 1), lim))) {
          ok = false;
          break;
        }
        v_wait = i + 1;
        tc::fence_after_sync();
        unsigned char* stage = base + s * TCW_STAGE;
        const uint32_t a_h = tc::smem_u32(stage), a_l = a_h + TCW_TILE_A;
        const uint32_t v_h = a_l + TCW_TILE_A, v_l = v_h + TCW_TILE_V;
        const uint32_t d = taddr + (uint32_t)(s * TC_LMAX);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t oo = kk * 32;
          tc_mma<FMT>(d, tc::sw128_desc(a_h + oo), tc::sw128_desc(v_l + oo), idesc, kk > 0 ? 1u : 0u);
          tc_mma<FMT>(d, tc::sw128_desc(a_l + oo), tc::sw128_desc(v_h + oo), idesc, 1u);
        }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t oo = kk * 32;
          tc_mma<FMT>(d, tc::sw128_desc(a_h + oo), tc::sw128_desc(v_h + oo), idesc, 1u);
        }
        tc::mma_commit(&b_mma[s]);
        mma_iss = i;
        // split stage s^1 takes chunk i + 1's V once chunk i - 1's MMAs are done
        if (i >= 1 && i + 1 < nchunks) {
          if (!tc::mbar_wait(&b_mma[s ^ 1], (uint32_t)(((i - 1) >> 1) & 1), lim)) {
            ok = false;
            break;
          }
          issue_v(i + 1);
        }
      }
      if (!ok) *s_fail = 1;
    }
    __syncwarp();
  } else {
    const uint32_t tview = taddr + ((uint32_t)((wp & 3) * 32) << 16) + (uint32_t)((wp >> 2) * PART);
    float wsum[PART];
#pragma unroll
    for (int t = 0; t < PART; ++t) wsum[t] = 0.0f;
    const int j = tid & 7, cq = tid >> 3;  // lane j of the 8 of columns cq + 32 u
    bool ok = true;
    auto add_acc = [&](int64_t i) {  // chunk i's accumulator into the sums (its MMAs are done)
#pragma unroll
      for (int q = 0; q < PART / 16; ++q) {
        float g[16];
        tc::tmem_ld16(tview + (uint32_t)((int)(i & 1) * TC_LMAX + q * 16), g);
#pragma unroll
        for (int v = 0; v < 16; ++v) wsum[q * 16 + v] += g[v];
      }
    };
    for (int64_t i = 0; ok && i < nchunks; ++i) {
      const int s = (int)(i & 1);
      if (i >= 2) {
        // chunk i - 2 has left split stage s: add its accumulator, free both
        if (*s_fail || !tc::mbar_wait(&b_mma[s], (uint32_t)(((i - 2) >> 1) & 1), P.wait_ns)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        add_acc(i - 2);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&b_acc[s]);
      }
      unsigned char* aH = base + s * TCW_STAGE;
      unsigned char* aL = aH + TCW_TILE_A;
      for (int b = 0; b < BPC; ++b) {
        const int64_t bx = i * BPC + b;
        const int f = (int)(bx % NST);
        if (*s_fail || !tc::mbar_wait(&b_full[f], (uint32_t)((bx / NST) & 1), P.wait_ns)) {
          ok = false;
          break;
        }
        const unsigned char* src = ring + f * G::BOX;
        // the box into registers first, so the ring gets it back before the conversion
        constexpr int NPC = G::BOXR / 16;  // 16-byte pieces per lane and column
        double2 dd_all[TCW_COLS / 32][NPC];
#pragma unroll
        for (int u = 0; u < TCW_COLS / 32; ++u)
#pragma unroll
          for (int e = 0; e < NPC; ++e)
            dd_all[u][e] = *reinterpret_cast<const double2*>(src + (size_t)(cq + 32 * u) * (G::BOXR * 8) + (e * 8 + j) * 16);
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&b_free[f]);  // the box's reads are done
#pragma unroll
        for (int u = 0; u < TCW_COLS / 32; ++u) {
          const int c = cq + 32 * u;
#pragma unroll
          for (int e = 0; e < NPC; ++e) {
            const int h = e * 8 + j;  // 16-byte piece: rows 2h, 2h + 1 of the box, column c
            const double2 dd = dd_all[u][e];
            const float x0 = f64_to_f32_rn(dd.x), x1 = f64_to_f32_rn(dd.y);
            const uint32_t off = tc::sw128_off_e<ESZ>(c, b * G::BOXR + 2 * h);
            if (FMT == 1) {
              __nv_bfloat16 h0, l0, h1, l1;
              tc::split_bf16(x0, &h0, &l0);
              tc::split_bf16(x1, &h1, &l1);
              __nv_bfloat162 hh, ll;
              hh.x = h0;
              hh.y = h1;
              ll.x = l0;
              ll.y = l1;
              *reinterpret_cast<__nv_bfloat162*>(aH + off) = hh;
              *reinterpret_cast<__nv_bfloat162*>(aL + off) = ll;
            } else {
              const float h0 = tc::tf32_rna(x0), h1 = tc::tf32_rna(x1);
              *reinterpret_cast<float2*>(aH + off) = make_float2(h0, h1);
              *reinterpret_cast<float2*>(aL + off) = make_float2(tc::tf32_rna(x0 - h0), tc::tf32_rna(x1 - h1));
            }
          }
        }
      }
      if (!ok) break;
      tc::fence_proxy_async_smem();  // the split tile is read by the tensor core
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&b_conv[s]);
    }
    // the last two chunks' accumulators
    for (int64_t i = (nchunks > 2 ? nchunks - 2 : 0); ok && i < nchunks; ++i) {
      if (*s_fail || !tc::mbar_wait(&b_mma[i & 1], (uint32_t)((i >> 1) & 1), P.wait_ns)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      add_acc(i);
    }
    if (!ok) *s_fail = 1;
    if (ok) {
      const int64_t col = c0 + (wp & 3) * 32 + lane;
      if (col < P.n) {
        float4* o4 = reinterpret_cast<float4*>(P.Wt + ((seg + 1) * P.n + col) * TC_LMAX + (wp >> 2) * PART);
#pragma unroll
        for (int v = 0; v < PART / 4; ++v)
          o4[v] = make_float4(wsum[4 * v], wsum[4 * v + 1], wsum[4 * v + 2], wsum[4 * v + 3]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (tid == 256 && *s_fail) {
    // leave no copy or MMA in flight: bounded waits for the last of each
    if (mma_iss >= 0) (void)tc::mbar_wait(&b_mma[mma_iss & 1], (uint32_t)((mma_iss >> 1) & 1), lim);
    for (int64_t i = v_wait; i < v_iss; ++i)
      if (!tc::mbar_wait(&b_vt[i & 1], (uint32_t)((i >> 1) & 1), lim)) break;
    for (int64_t bx = (loads > NST ? loads - NST : 0); bx < loads; ++bx)
      if (!tc::mbar_wait(&b_full[bx % NST], (uint32_t)((bx / NST) & 1), lim)) break;
    record_fail(st, FAIL_MMA_WAIT, (int)blockIdx.x, st->step, st->ns, KID_TC_W);
  }
  __syncwarp();
  if (wp == 8) tc::tmem_dealloc(taddr, 2 * TC_LMAX);
}

// The candidate Gram matrix G = C^T C of the tensor-core forms (C: the kc <=
// 64 candidate columns of rows ns..m-1, gathered through P.cols).  CTA c
// takes the 64-row chunks c, c + gridDim.x, ... as the FP64/FP32 Gram kernels
// do, so k_gram_reduce sums the same partials.  Per K atom of rows the
// candidates are split into one hi/lo tile (candidate a = tile row a, rows of
// A along K); the tile is both operands: D (128 x 64) += X X^T, of which rows
// and columns a, b < kc are used.  As in the W pass, each atom has its own
// TMEM accumulator (two alternate) that the warps add into FP32 registers.
constexpr int TCG_TILE = 128 * 128;  // bytes of one operand tile (128 rows x one atom)
constexpr int TCG_SMEM = 1024 + 2 * 2 * TCG_TILE + 64;

template <int FMT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gram(Params P) {
  constexpr int ESZ = TcFmt<FMT>::ESZ, KA = TcFmt<FMT>::KA;
  constexpr int EPC = 16 / ESZ;
  constexpr int SUB = GRAM_ROWS / KA;  // K atoms per 64-row chunk
  static_assert(GRAM_ROWS % KA == 0, "chunks of whole atoms");
  DevState* st = P.st;
  if (st->done) return;
  const int kc = st->kc;
  if (kc <= 1) return;
  const int64_t ns = st->ns, m = P.m, mr = m - ns, lda = P.lda;
  const int64_t nchunks = (mr + GRAM_ROWS - 1) / GRAM_ROWS;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(P.st, KID_GRAM, (double)mr * kc * (kc + 1.0));
  if ((int64_t)blockIdx.x >= nchunks) return;
  const int64_t my_chunks = (nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x;
  const int64_t nsteps = my_chunks * SUB;
  extern __shared__ unsigned char tcg_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcg_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 4 * TCG_TILE);
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
  const bool drains = (wp & 3) < 2;  // TMEM lanes 0..63 hold the candidates' rows of D
  const uint32_t tview = taddr + ((uint32_t)((wp & 3) * 32) << 16) + (uint32_t)((wp >> 2) * 32);
  float gsum[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) gsum[t] = 0.0f;
  // units: candidate a = (tid >> 3) + 32 q (q = 0, 1), 16-byte chunk kg of the atom row
  const int kg = tid & 7;
  int64_t colb[2];
  bool aok[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a = (tid >> 3) + 32 * q;
    aok[q] = a < kc;
    colb[q] = aok[q] ? (int64_t)P.cols[a] * lda : 0;
  }
  const uint32_t idesc = tc::idesc_f32acc(128, TC_LMAX, FMT);
  int64_t issued = -1;
  for (int64_t i = 0; i < nsteps; ++i) {
    const int s = (int)(i & 1);
    const int64_t chunk = blockIdx.x + (i / SUB) * gridDim.x;
    const int64_t r0 = ns + chunk * GRAM_ROWS + (i % SUB) * KA;  // absolute first row of the atom
    double xa[2][EPC];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int64_t r = r0 + kg * EPC + e;
        xa[q][e] = (aok[q] && r < m) ? P.A[colb[q] + r] : 0.0;
      }
    }
    if (i >= 2) {  // the MMAs of step i - 2 have finished with this stage and accumulator
      if (tid == 0 && !tc::mbar_wait(&bar[s], (uint32_t)(((i >> 1) - 1) & 1), P.wait_ns)) *s_fail = 1;
      __syncthreads();
      if (*s_fail) break;
      tc::fence_after_sync();
      if (drains) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float g[16];
          tc::tmem_ld16(tview + (uint32_t)(s * TC_LMAX + q * 16), g);
#pragma unroll
          for (int v = 0; v < 16; ++v) gsum[q * 16 + v] += g[v];
        }
      }
    }
    unsigned char* xH = base + s * 2 * TCG_TILE;
    unsigned char* xL = xH + TCG_TILE;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int a = (tid >> 3) + 32 * q;
      float f[EPC];
#pragma unroll
      for (int e = 0; e < EPC; ++e) f[e] = f64_to_f32_rn(xa[q][e]);
      uint4 h, w;
      tc_split16<FMT>(f, &h, &w);
      const uint32_t off = (uint32_t)(a * 128 + ((kg ^ (a & 7)) << 4));
      *reinterpret_cast<uint4*>(xH + off) = h;
      *reinterpret_cast<uint4*>(xL + off) = w;
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t x_h = tc::smem_u32(xH), x_l = x_h + TCG_TILE;
      const uint32_t d = taddr + (uint32_t)(s * TC_LMAX);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(d, tc::sw128_desc(x_h + o), tc::sw128_desc(x_l + o), idesc, kk > 0 ? 1u : 0u);
        tc_mma<FMT>(d, tc::sw128_desc(x_l + o), tc::sw128_desc(x_h + o), idesc, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t o = kk * 32;
        tc_mma<FMT>(d, tc::sw128_desc(x_h + o), tc::sw128_desc(x_h + o), idesc, 1u);
      }
      tc::mma_commit(&bar[s]);
    }
    issued = i;
  }
  const int64_t last = nsteps - 1;
  if (tid == 0 && !*s_fail && !tc::mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1), P.wait_ns)) *s_fail = 1;
  __syncthreads();
  tc::fence_after_sync();
  if (*s_fail) {
    if (tid == 0 && issued >= 0) (void)tc::mbar_wait(&bar[issued & 1], (uint32_t)((issued >> 1) & 1), P.wait_ns);
    if (tid == 0) record_fail(st, FAIL_MMA_WAIT, (int)blockIdx.x, st->step, st->ns, KID_GRAM);
  } else if (drains) {
    for (int64_t i = max((int64_t)0, last - 1); i <= last; ++i) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float g[16];
        tc::tmem_ld16(tview + (uint32_t)((int)(i & 1) * TC_LMAX + q * 16), g);
#pragma unroll
        for (int v = 0; v < 16; ++v) gsum[q * 16 + v] += g[v];
      }
    }
    // thread = candidate a, columns b of its half: the upper triangle a <= b < kc
    const int a = (wp & 3) * 32 + lane;
    double* out = P.Gp + (int64_t)blockIdx.x * P.kmax * P.kmax;
#pragma unroll
    for (int v = 0; v < 32; ++v) {
      const int b = (wp >> 2) * 32 + v;
      if (a <= b && b < kc) out[b * (b + 1) / 2 + a] = f32_to_f64(gsum[v]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wp == 0) tc::tmem_dealloc(taddr, 2 * TC_LMAX);
}

// W = T^T (sum of the segments' V^T A22) per trailing column: one warp per
// column; lanes t and t + 32 sum their reflector's segments in FP64 into
// P_t.  T is not formed: with S = V^T V (k_tc_sred), T^-1 = strict_upper(S) +
// diag(1/htau), so W solves (T^-1)^T W = P by forward substitution,
// W_t = htau_t (P_t - sum_{q<t} S_qt W_q), right-looking across the lanes in
// FP32 (W_t from its lane by a shuffle, then every later lane subtracts its
// S_tu W_t); then W's hi/lo operand image for the update is written
// (128-column tiles from column ns + k; padding columns of the last tile are
// zero).
template <int FMT>
__global__ void __launch_bounds__(TC_THREADS) k_tc_wsum(Params P) {
  constexpr int ESZ = TcFmt<FMT>::ESZ, KA = TcFmt<FMT>::KA, NA = TcFmt<FMT>::NA;
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, j0 = ns + st->k;
  const int64_t n2 = P.n - j0, mr = P.m - ns;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  __shared__ float s_S[TC_LMAX][TC_LMAX + 1];  // S_qt, q < t
  __shared__ float s_tau[TC_LMAX];
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < TC_LMAX * TC_LMAX; e += TC_THREADS) {
    const int q = e / TC_LMAX, t = e % TC_LMAX;
    s_S[q][t] = (q < t && t < l) ? (float)P.G[t * (t - 1) / 2 + q] : 0.0f;
  }
  if (tid < TC_LMAX) s_tau[tid] = (tid < l) ? (float)P.htau[st->ns + tid] : 0.0f;
  __syncthreads();
  int64_t nseg, seg_rows;
  tc_segments(mr + tc_shift(P, ns), P.tc_nseg, TC_SEG_ALIGN, &nseg, &seg_rows);  // the W pass's segments
  (void)seg_rows;
  const int64_t gw = (int64_t)blockIdx.x * (TC_THREADS / 32) + wp;
  const int64_t nwarps = (int64_t)gridDim.x * (TC_THREADS / 32);
  const int64_t npad = (n2 + TCU_COLS - 1) / TCU_COLS * TCU_COLS;
  for (int64_t c = gw; c < npad; c += nwarps) {
    float w0 = 0.0f, w1 = 0.0f;
    if (c < n2) {
      const int64_t col = j0 + c;
      // the segments' partials, loaded all at once (nseg <= TC_NSEG_MAX), added in segment order
      float x0[TC_NSEG_MAX], x1[TC_NSEG_MAX];
#pragma unroll
      for (int sg = 0; sg < TC_NSEG_MAX; ++sg) {
        const float* part = P.Wt + ((sg + 1) * P.n + col) * TC_LMAX;
        x0[sg] = (sg < nseg) ? part[lane] : 0.0f;
        x1[sg] = (sg < nseg) ? part[lane + 32] : 0.0f;
      }
      double g0 = 0.0, g1 = 0.0;
#pragma unroll
      for (int sg = 0; sg < TC_NSEG_MAX; ++sg) {
        if (sg < nseg) {
          g0 += (double)x0[sg];
          g1 += (double)x1[sg];
        }
      }
      float p0 = (float)g0, p1 = (float)g1;  // P_lane, P_{lane + 32}
      for (int t = 0; t < l; ++t) {
        const float pt = __shfl_sync(0xffffffffu, t < 32 ? p0 : p1, t & 31);
        const float wt = s_tau[t] * pt;
        if (lane > t) p0 = fmaf(-s_S[t][lane], wt, p0);
        if (lane + 32 > t) p1 = fmaf(-s_S[t][lane + 32], wt, p1);
        if (lane == (t & 31)) {
          if (t < 32) p0 = wt;
          else p1 = wt;
        }
      }
      w0 = (lane < l) ? p0 : 0.0f;
      w1 = (lane + 32 < l) ? p1 : 0.0f;
    }
    unsigned char* img = P.tc_wi + (c / TCU_COLS) * (2 * NA * TC_ATOM);
    const int cc = (int)(c % TCU_COLS);
    tc_put<FMT>(img + (lane / KA) * TC_ATOM, img + (NA + lane / KA) * TC_ATOM,
                tc::sw128_off_e<ESZ>(cc, lane % KA), w0);
    tc_put<FMT>(img + ((lane + 32) / KA) * TC_ATOM, img + (NA + (lane + 32) / KA) * TC_ATOM,
                tc::sw128_off_e<ESZ>(cc, (lane + 32) % KA), w1);
  }
}

// A22 -= V W in tiles of 128 rows x 128 columns, K = 64 reflectors in NA
// atoms.  Persistent: CTA b takes a contiguous, balanced range of tiles in
// row-block-major order.  Thread 0 brings the operands in with bulk copies
// from their images (V once per row block; W per tile into one of two
// buffers, two tiles ahead) and issues the MMAs into one of two TMEM
// accumulators (2 x 128 columns); meanwhile all warps stream the previous
// tile through HBM (load A, subtract, store), 32 loads per thread in flight.
// threads of k_tc_update: the BF16 form fits two CTAs of 8 warps per SM; the
// 3xTF32 form's operand buffers allow one CTA per SM, which gets 16 warps so
// that as many loads of A stay in flight
template <int FMT>
__host__ __device__ constexpr int tcu_threads() {
  return FMT == 1 ? 256 : 512;
}

template <int FMT>
__global__ void __launch_bounds__(tcu_threads<FMT>(), FMT == 1 ? 2 : 1) k_tc_update(Params P) {
  constexpr int NA = TcFmt<FMT>::NA;
  constexpr int NT = tcu_threads<FMT>();
  constexpr int CPW = TCU_COLS / (NT / 128);  // columns of a tile per warp (its lane quarter's rows)
  constexpr int OPB = 2 * NA * TC_ATOM;  // bytes of one operand tile, hi and lo
  static_assert(TCU_ROWS == 128 && TCU_COLS == 128, "tiles of 128 rows / columns");
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t ns = st->ns, j0 = ns + st->k;
  const int64_t n2 = P.n - j0, mr = P.m - ns, lda = P.lda;
  if (l <= 0 || n2 <= 0 || mr <= 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TC_UPDATE, 2.0 * (double)mr * (double)n2 * l);
  const int64_t nct = (n2 + TCU_COLS - 1) / TCU_COLS;
  const int64_t ntiles = ((mr + TCU_ROWS - 1) / TCU_ROWS) * nct;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;
  extern __shared__ unsigned char tcu_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcu_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* vbuf = base;        // hi atoms, then lo atoms
  unsigned char* wbuf = base + OPB;  // two buffers of OPB bytes
  // [0,1] MMA done, [2,3] W landed, [4] V landed, [5] never arrived on (test hook 3)
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + 3 * OPB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 6);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  const int64_t nloc = t1 - t0;
  if (wp == 0) tc::tmem_alloc(tslot, 2 * TCU_COLS);
  // copies issued / phases waited, per barrier (thread 0): a failed run still
  // waits for every copy it started before the CTA's shared memory goes away
  uint32_t w_iss[2] = {0u, 0u}, w_done[2] = {0u, 0u}, v_iss = 0u, v_done = 0u;
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < 6; ++b) tc::mbar_init(&bar[b], 1);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // V for the first row block, W for the first two tiles
    tc::mbar_expect_tx(&bar[4], OPB);
    tc::bulk_g2s(vbuf, P.tc_vu + (t0 / nct) * OPB, OPB, &bar[4]);
    ++v_iss;
    for (int64_t i = 0; i < 2 && i < nloc; ++i) {
      tc::mbar_expect_tx(&bar[2 + i], OPB);
      tc::bulk_g2s(wbuf + i * OPB, P.tc_wi + ((t0 + i) % nct) * OPB, OPB, &bar[2 + i]);
      ++w_iss[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  const uint32_t idesc = tc::idesc_f32acc(TCU_ROWS, TCU_COLS, FMT);
  const int q4 = wp & 3, part = wp >> 2;  // TMEM lane quarter and column part of this warp
  int64_t cur_rb = -1, issued = -1;
  for (int64_t i = 0; i <= nloc; ++i) {
    if (i < nloc) {
      const int64_t rb = (t0 + i) / nct;
      if (tid == 0) {
        bool ok = true;
        if (rb != cur_rb && i > 0) {  // a new row block: the MMAs issued so far still read V
          ok = tc::mbar_wait(&bar[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), P.wait_ns);
          if (ok) {
            tc::mbar_expect_tx(&bar[4], OPB);
            tc::bulk_g2s(vbuf, P.tc_vu + rb * OPB, OPB, &bar[4]);
            ++v_iss;
          }
        }
        if (ok && rb != cur_rb) {
          ok = tc::mbar_wait(&bar[4], v_done & 1u, P.wait_ns);
          if (ok) ++v_done;
        }
        if (ok) {
          ok = tc::mbar_wait(&bar[2 + (i & 1)], (uint32_t)((i >> 1) & 1), P.wait_ns);
          if (ok) ++w_done[i & 1];
        }
        // test hook 3: a wait nothing completes, before the first MMA (the
        // copies already issued drain in the give-up path below)
        if (ok && i == 0 && P.test_fault == 3) ok = tc::mbar_wait(&bar[5], 0u, P.wait_ns);
        if (ok) {
          tc::fence_after_sync();
          const uint32_t d = taddr + (uint32_t)((i & 1) * TCU_COLS);
          const uint32_t vh = tc::smem_u32(vbuf), vl = vh + NA * TC_ATOM;
          const uint32_t wh = tc::smem_u32(wbuf + (i & 1) * OPB), wl = wh + NA * TC_ATOM;
          // cross terms first, then hi*hi (only those truncate at the scale of the sum)
#pragma unroll
          for (int a = 0; a < NA; ++a) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t o = a * TC_ATOM + kk * 32;
              tc_mma<FMT>(d, tc::sw128_desc(vh + o), tc::sw128_desc(wl + o), idesc, (a > 0 || kk > 0) ? 1u : 0u);
              tc_mma<FMT>(d, tc::sw128_desc(vl + o), tc::sw128_desc(wh + o), idesc, 1u);
            }
          }
#pragma unroll
          for (int a = 0; a < NA; ++a) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t o = a * TC_ATOM + kk * 32;
              tc_mma<FMT>(d, tc::sw128_desc(vh + o), tc::sw128_desc(wh + o), idesc, 1u);
            }
          }
          tc::mma_commit(&bar[i & 1]);
          issued = i;
        } else {
          *s_fail = 1;
        }
      }
      cur_rb = rb;
    }
    if (i >= 1) {  // epilogue of tile i - 1
      const int64_t pi = i - 1, t = t0 + pi, rb = t / nct, ct = t % nct;
      const int64_t rr = rb * TCU_ROWS + q4 * 32 + lane;
      const bool rok = rr < mr;
      double* arow = P.A + ns + rr;
      const int64_t cb0 = j0 + ct * TCU_COLS + part * CPW;
      // A of the first 32 columns does not depend on the MMAs: its loads go
      // out before the wait for them
      double x[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) x[u] = (rok && cb0 + u < P.n) ? arow[(cb0 + u) * lda] : 0.0;
      if (tid == 0 && !*s_fail) {
        if (!tc::mbar_wait(&bar[pi & 1], (uint32_t)((pi >> 1) & 1), P.wait_ns)) {
          *s_fail = 1;
        } else if (pi + 2 < nloc) {  // its W buffer is free: the tile two ahead
          tc::mbar_expect_tx(&bar[2 + (pi & 1)], OPB);
          tc::bulk_g2s(wbuf + (pi & 1) * OPB, P.tc_wi + ((t + 2) % nct) * OPB, OPB, &bar[2 + (pi & 1)]);
          ++w_iss[pi & 1];
        }
      }
      __syncthreads();
      if (*s_fail) break;
      tc::fence_after_sync();
      const uint32_t tb = taddr + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((pi & 1) * TCU_COLS + part * CPW);
#pragma unroll 1
      for (int c = 0; c < CPW; c += 32) {
        const int64_t cb = cb0 + c;
        if (c > 0) {
#pragma unroll
          for (int u = 0; u < 32; ++u) x[u] = (rok && cb + u < P.n) ? arow[(cb + u) * lda] : 0.0;
        }
        float v[32];
        tc::tmem_ld16(tb + c, v);
        tc::tmem_ld16(tb + c + 16, v + 16);
        // FP32 -> FP64 on the integer pipe (exact): GB300's FP64 pipe, about
        // two operations per clock per SM, is left the subtraction alone
#pragma unroll
        for (int u = 0; u < 32; ++u)
          if (rok && cb + u < P.n) arow[(cb + u) * lda] = x[u] - f32_to_f64(v[u]);
      }
      tc::fence_before_sync();
    }
    __syncthreads();  // the epilogue has read its accumulator before the next MMAs reuse it
    if (*s_fail) break;
  }
  if (*s_fail) {
    // leave no copy or MMA in flight behind: bounded waits for the last ones
    if (tid == 0) {
      if (issued >= 0) (void)tc::mbar_wait(&bar[issued & 1], (uint32_t)((issued >> 1) & 1), P.wait_ns);
      for (int b = 0; b < 2; ++b)
        for (; w_done[b] < w_iss[b]; ++w_done[b])
          if (!tc::mbar_wait(&bar[2 + b], w_done[b] & 1u, P.wait_ns)) break;
      for (; v_done < v_iss; ++v_done)
        if (!tc::mbar_wait(&bar[4], v_done & 1u, P.wait_ns)) break;
    }
    if (tid == 0) record_fail(st, FAIL_MMA_WAIT, (int)blockIdx.x, st->step, st->ns, KID_TC_UPDATE);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (wp == 0) tc::tmem_dealloc(taddr, 2 * TCU_COLS);
}


// The update with A streamed by tensor copies (TMA), when A is 16-byte
// aligned with an even lda (P.tc_al): the tiles of k_tc_update start at the
// even row ns - o (o = ns mod 2; V's image then holds a zero row on top, so
// row ns - 1 is rewritten with its own bits), and each tile passes through
// shared memory in four sub-tiles of 32 columns (32 KB of FP64).  A ring of
// NS stages: a tiled tensor copy brings a sub-tile in, the epilogue warps
// subtract the accumulator in place, a tiled tensor copy writes it back, and
// the stage takes the sub-tile NS ahead.  Loads and stores need no thread and
// no load-queue slot, so the ring keeps NS - 1 sub-tiles in flight while one
// is converted.  Warp 8 issues every copy and MMA (one thread); warps 0-7 are
// the epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (the tile's
// rows) and 16 of each sub-tile's columns.  One CTA per SM (persistent, the
// same balanced tile ranges as k_tc_update); the BF16 form double-buffers W,
// the 3xTF32 form (operand tiles twice as large) has one W buffer, reloaded
// as soon as the tile's MMAs are done.
template <int FMT>
struct TcuTma {
  static constexpr int NA = TcFmt<FMT>::NA;
  static constexpr int OPB = 2 * NA * TC_ATOM;  // one operand tile, hi and lo
  static constexpr int NWB = (FMT == 1) ? 2 : 1;  // W buffers
  static constexpr int NS = (FMT == 1) ? 4 : 3;   // FP64 sub-tile stages
  static constexpr int SUBC = 32;                 // columns of a sub-tile
  static constexpr int NSUB = TCU_COLS / SUBC;
  static constexpr int STAGE = TCU_ROWS * SUBC * 8;
  static constexpr int THREADS = 288;  // 8 epilogue warps and the copy / MMA warp
  static constexpr int SMEM = 1024 + (1 + NWB) * OPB + NS * STAGE + 256;
};

template <int FMT>
__global__ void __launch_bounds__(TcuTma<FMT>::THREADS, 1)
    k_tc_update_tma(const __grid_constant__ CUtensorMap tmU, Params P) {
  using G = TcuTma<FMT>;
  constexpr int NA = G::NA, OPB = G::OPB, NWB = G::NWB, NS = G::NS, NSUB = G::NSUB;
  static_assert(TCU_ROWS == 128 && TCU_COLS == 128, "tiles of 128 rows / columns");
  DevState* st = P.st;
  if (st->done) return;
  const int l = st->l;
  const int64_t j0 = st->ns + st->k, n2 = P.n - j0;
  if (l <= 0 || n2 <= 0 || P.m - st->ns <= 0) return;
  const int o = tc_shift(P, st->ns);
  const int64_t r0 = st->ns - o, mr = P.m - r0;  // tile rows start at the even row r0
  if (blockIdx.x == 0 && threadIdx.x == 0) add_flops(st, KID_TC_UPDATE, 2.0 * (double)(mr - o) * (double)n2 * l);
  const int64_t nct = (n2 + TCU_COLS - 1) / TCU_COLS;
  const int64_t ntiles = ((mr + TCU_ROWS - 1) / TCU_ROWS) * nct;
  const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
  if (t0 >= t1) return;
  const int64_t nloc = t1 - t0, nsub = nloc * NSUB;
  extern __shared__ unsigned char tcut_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tcut_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* vbuf = base;                      // V hi atoms, then lo atoms
  unsigned char* wbuf = base + OPB;                // NWB buffers of W
  unsigned char* ring = base + (1 + NWB) * OPB;    // NS FP64 stages
  uint64_t* bar = reinterpret_cast<uint64_t*>(ring + NS * G::STAGE);
  uint64_t* b_mma = bar;             // [2] MMAs of accumulator 0 / 1 done
  uint64_t* b_w = bar + 2;           // [NWB] W landed
  uint64_t* b_v = bar + 4;           // V landed
  uint64_t* b_hook = bar + 5;        // never arrived on (test hook 3)
  uint64_t* b_full = bar + 6;        // [NS] sub-tile landed
  uint64_t* b_done = bar + 6 + NS;   // [NS] sub-tile subtracted (8 arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 6 + 2 * NS);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  if (wp == 8) tc::tmem_alloc(tslot, 2 * TCU_COLS);
  if (tid == 256) {
    for (int b = 0; b < 6 + NS; ++b) tc::mbar_init(&bar[b], 1);
    for (int b = 0; b < NS; ++b) tc::mbar_init(&b_done[b], 8);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *tslot;
  if (wp == 8) {
    if (lane == 0) {
      const long long lim = P.wait_ns;
      auto rb_of = [&](int64_t i) { return (t0 + i) / nct; };
      auto ct_of = [&](int64_t i) { return (t0 + i) % nct; };
      auto sx = [&](int64_t g) { return (int32_t)(r0 + rb_of(g / NSUB) * TCU_ROWS); };
      auto sy = [&](int64_t g) { return (int32_t)(j0 + ct_of(g / NSUB) * TCU_COLS + (g % NSUB) * G::SUBC); };
      int64_t loads = 0, w_iss = 0, w_wait = 0, mma_iss = -1, cur_rb = -1;
      uint32_t v_iss = 0, v_wait = 0;
      bool ok = true;
      auto issue_w = [&](int64_t i) {
        tc::mbar_expect_tx(&b_w[i % NWB], OPB);
        tc::bulk_g2s(wbuf + (i % NWB) * OPB, P.tc_wi + ct_of(i) * OPB, OPB, &b_w[i % NWB]);
        w_iss = i + 1;
      };
      auto issue_load = [&](int64_t g) {
        const int s = (int)(g % NS);
        tc::mbar_expect_tx(&b_full[s], G::STAGE);
        tc::tma_load_2d(ring + s * G::STAGE, &tmU, sx(g), sy(g), &b_full[s]);
        loads = g + 1;
      };
      // MMAs of tile i into accumulator i & 1 (its previous tile's epilogue is done)
      auto issue_mma = [&](int64_t i) -> bool {
        const int64_t rb = rb_of(i);
        if (rb != cur_rb) {  // a new row block: the MMAs issued so far still read V
          if (i > 0 && !tc::mbar_wait(&b_mma[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), lim)) return false;
          tc::mbar_expect_tx(b_v, OPB);
          tc::bulk_g2s(vbuf, P.tc_vu + rb * OPB, OPB, b_v);
          ++v_iss;
          if (!tc::mbar_wait(b_v, v_wait & 1u, lim)) return false;
          ++v_wait;
          cur_rb = rb;
        }
        if (!tc::mbar_wait(&b_w[i % NWB], (uint32_t)((i / NWB) & 1), lim)) return false;
        w_wait = i + 1;
        if (i == 0 && P.test_fault == 3 && !tc::mbar_wait(b_hook, 0u, lim)) return false;
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_f32acc(TCU_ROWS, TCU_COLS, FMT);
        const uint32_t d = taddr + (uint32_t)((i & 1) * TCU_COLS);
        const uint32_t vh = tc::smem_u32(vbuf), vl = vh + NA * TC_ATOM;
        const uint32_t wh = tc::smem_u32(wbuf + (i % NWB) * OPB), wl = wh + NA * TC_ATOM;
        // cross terms first, then hi*hi (only those truncate at the scale of the sum)
#pragma unroll
        for (int a = 0; a < NA; ++a) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t off = a * TC_ATOM + kk * 32;
            tc_mma<FMT>(d, tc::sw128_desc(vh + off), tc::sw128_desc(wl + off), idesc, (a > 0 || kk > 0) ? 1u : 0u);
            tc_mma<FMT>(d, tc::sw128_desc(vl + off), tc::sw128_desc(wh + off), idesc, 1u);
          }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t off = a * TC_ATOM + kk * 32;
            tc_mma<FMT>(d, tc::sw128_desc(vh + off), tc::sw128_desc(wh + off), idesc, 1u);
          }
        }
        tc::mma_commit(&b_mma[i & 1]);
        mma_iss = i;
        return true;
      };
      issue_w(0);
      if (NWB == 2 && nloc > 1) issue_w(1);
      for (int64_t g = 0; g < NS && g < nsub; ++g) issue_load(g);
      ok = issue_mma(0);
      if (ok && NWB == 1 && nloc > 1) {  // the one W buffer is free once tile 0's MMAs are done
        ok = tc::mbar_wait(&b_mma[0], 0u, lim);
        if (ok) issue_w(1);
      }
      for (int64_t g = 0; ok && g < nsub; ++g) {
        const int s = (int)(g % NS);
        const int64_t i = g / NSUB;
        const int sub = (int)(g % NSUB);
        if (*s_fail || !tc::mbar_wait(&b_done[s], (uint32_t)((g / NS) & 1), lim)) {
          ok = false;
          break;
        }
        // (a sub-tile wholly right of the last column was loaded as zeros and is not stored)
        if (sy(g) < P.n) tc::tma_store_2d(&tmU, sx(g), sy(g), ring + s * G::STAGE);
        tc::bulk_commit();
        if (sub == 0 && i + 1 < nloc) {
          // tile i's epilogue has begun, so its MMAs are done: W buffer (i mod 2)
          // takes tile i + 2 (BF16 form), and tile i + 1's MMAs go out
          if (NWB == 2 && i + 2 < nloc) issue_w(i + 2);
          if (!(ok = issue_mma(i + 1))) break;
        }
        if (NWB == 1 && sub == 1 && i + 2 < nloc) {
          if (!(ok = tc::mbar_wait(&b_mma[(i + 1) & 1], (uint32_t)(((i + 1) >> 1) & 1), lim))) break;
          issue_w(i + 2);
        }
        if (g + NS < nsub) {  // the stage takes the sub-tile NS ahead once the store has read it
          tc::bulk_wait_read_all();
          issue_load(g + NS);
        }
      }
      tc::bulk_wait_all();
      if (!ok) {
        *s_fail = 1;
        // leave no copy or MMA in flight: bounded waits for the last of each
        if (mma_iss >= 0) (void)tc::mbar_wait(&b_mma[mma_iss & 1], (uint32_t)((mma_iss >> 1) & 1), lim);
        for (int64_t i = w_wait; i < w_iss; ++i)
          if (!tc::mbar_wait(&b_w[i % NWB], (uint32_t)((i / NWB) & 1), lim)) break;
        if (v_wait < v_iss) (void)tc::mbar_wait(b_v, v_wait & 1u, lim);
        for (int64_t g = (loads > NS ? loads - NS : 0); g < loads; ++g)
          if (!tc::mbar_wait(&b_full[g % NS], (uint32_t)((g / NS) & 1), lim)) break;
        record_fail(st, FAIL_MMA_WAIT, (int)blockIdx.x, st->step, st->ns, KID_TC_UPDATE);
      }
    }
    __syncwarp();
  } else {
    const int q4 = wp & 3, half = wp >> 2;
    const int row = q4 * 32 + lane;  // the tile's row this thread subtracts
    for (int64_t i = 0; i < nloc && !*s_fail; ++i) {
      if (!tc::mbar_wait(&b_mma[i & 1], (uint32_t)((i >> 1) & 1), P.wait_ns)) {
        *s_fail = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t tb = taddr + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((i & 1) * TCU_COLS + half * 16);
      for (int sub = 0; sub < NSUB; ++sub) {
        const int64_t g = i * NSUB + sub;
        const int s = (int)(g % NS);
        float v[16];
        tc::tmem_ld16(tb + (uint32_t)(sub * G::SUBC), v);
        if (!tc::mbar_wait(&b_full[s], (uint32_t)((g / NS) & 1), P.wait_ns)) *s_fail = 1;
        if (*s_fail) break;
        double* col = reinterpret_cast<double*>(ring + s * G::STAGE) + (half * 16) * TCU_ROWS + row;
        // FP32 -> FP64 on the integer pipe (exact); the FP64 pipe does the subtraction
#pragma unroll
        for (int u = 0; u < 16; ++u) col[u * TCU_ROWS] = col[u * TCU_ROWS] - f32_to_f64(v[u]);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&b_done[s]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (wp == 8) tc::tmem_dealloc(taddr, 2 * TCU_COLS);
}

}  // namespace qrdm
