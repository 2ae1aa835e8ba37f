/*
 * qrdm.h -- C ABI of the GB300 QRDM library (libqrdm.so).
 *
 * QRDM is Householder QR with Deviation Maximization column pivoting
 * (Dessole & Marcuzzi, "Deviation Maximization for Rank-Revealing QR
 * Factorizations", 2021): A Pi = Q R, where each block step picks up to
 * k_max well-separated, large-norm columns at once (Algorithm 1), moves them
 * to the front, factors them as a Householder panel that stops early when a
 * column turns out dependent (Algorithm 4), and updates the trailing matrix
 * with one compact-WY block reflector (Sec. 3.2).
 *
 * Every step runs on the GPU as hand-written sm_103a CUDA kernels.  The
 * library allocates no device memory: the caller passes the matrix, the
 * outputs and one workspace buffer sized by qrdm_workspace_size().  All
 * pointers named d_* are device pointers; all others are host pointers.
 * Calls are ordered on the given CUDA stream.  The factorization is driven
 * from the host; qrdm_factor() returns after the stream has completed the
 * work (it synchronizes on `stream` while stepping).
 *
 * Errors: 0 on success; -i when the i-th argument is invalid (LAPACK
 * convention: nothing is read or written); a positive QRDM_ERR_* code
 * otherwise.  On QRDM_ERR_NONFINITE the matrix has not been modified.
 */
#ifndef QRDM_H
#define QRDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QRDM_OK 0
#define QRDM_ERR_CUDA 1      /* a CUDA runtime call failed (qrdm_last_cuda_error() has it) */
#define QRDM_ERR_NONFINITE 2 /* A holds a NaN or an infinity; A is left unmodified */
#define QRDM_ERR_WORKSPACE 3 /* workspace too small or misaligned (256-byte alignment) */
#define QRDM_ERR_UNSUPPORTED 4 /* the device or an option is not supported */
#define QRDM_ERR_INTERNAL 5  /* an internal consistency check failed on the device */
#define QRDM_ERR_TIMEOUT 6   /* a bounded device-side wait gave up (qrdm_info.fail_* say where); A is
                                partially factored, the context stays usable */
#define QRDM_ERR_CHECKED 7   /* with opts.checked: a device-side index check tripped; the access was
                                skipped, the factorization abandoned, A is partially factored */

/* Where a device-side wait or check gave up (qrdm_info.fail_code). */
#define QRDM_FAIL_NONE 0
#define QRDM_FAIL_GRID_BARRIER 1 /* grid barrier of a cooperative kernel: fail_value = arrivals seen */
#define QRDM_FAIL_PIVOT_RANGE 2  /* a pivot position outside [n_s, n): fail_value = the position */
#define QRDM_FAIL_MMA_WAIT 4     /* an mbarrier wait of a tensor-core kernel: fail_value = kernel id */
#define QRDM_FAIL_CHECK 8        /* a checked-path index check: fail_value = the bad index, fail_cta = kernel id */

#define QRDM_KMAX_LIMIT 128 /* largest supported k_max */

/* Kernel ids of qrdm_profile, in launch order within a block step. */
#define QRDM_K_COLNORM 0       /* a1: initial column norms */
#define QRDM_K_SELECT 1        /* a2/a3: stopping test, argmax, candidate set */
#define QRDM_K_GRAM 2          /* a4: candidate Gram matrix, partial sums */
#define QRDM_K_GRAM_REDUCE 3   /* a4: sum of the partial Gram matrices */
#define QRDM_K_PICK 4          /* a5/a6: DM greedy pick, swap sequence */
#define QRDM_K_PERMUTE 5       /* a6: column moves */
#define QRDM_K_PANEL 6         /* a7/a8: Householder panel with break test, T */
#define QRDM_K_TRAIL_W 7       /* a9: W = V^T A22 (partial) */
#define QRDM_K_TRAIL_WREDUCE 8 /* a9: W = T^T sum(partials) (with the pre-sum of many row chunks) */
#define QRDM_K_TRAIL_UPDATE 9  /* a9: A22 -= V W */
#define QRDM_K_DOWNDATE 10     /* a10: partial norm update */
#define QRDM_K_STEP_END 11     /* a11: n_s += l */
#define QRDM_K_QRP_TAIL 12     /* a2..a11 fused for single-column steps (DM off or k_max = 1) */
#define QRDM_K_WY_T 13         /* a8, merged forms: V^T V of the step and its compact-WY T */
#define QRDM_K_TC_VIMG 14      /* a9, tensor-core forms: V's operand images */
#define QRDM_K_TC_WSUM 15      /* a9, tensor-core forms: W = T^T (sum of segments) and W's image */
#define QRDM_K_TC_W 16         /* a9, tensor-core forms: the merged W = V^T A22 (tcgen05) */
#define QRDM_K_TC_UPDATE 17    /* a9, tensor-core forms: the merged A22 -= V W (tcgen05) */
#define QRDM_NKERNELS 18

/* Optional per-kernel timing (host struct, filled when opts->profile is set):
   every launch is bracketed by CUDA events on the caller's stream (and the
   FP64 form's look-ahead, which runs part of each trailing update on a second
   stream beside the next panel, is off, so that each kernel's time is its
   own); ms[] sums
   the device time per kernel, flops[] the algorithmic FP64 flops its
   launches performed (for the trailing update 4 m' n'' l + 2 l^2 n''), and
   launches[] counts them.  Values accumulate across calls; zero the struct to
   reset it. */
typedef struct qrdm_profile {
  double ms[24];
  double flops[24];
  int64_t launches[24];
} qrdm_profile;

/* Options; a NULL pointer means all zero (the defaults). */
typedef struct qrdm_opts {
  /* eps1 in the stopping criterion sqrt(n - n_s) max||c_i|| <= eps1 max||a_i||
     (Sec. 3.4, eq. practical stopping criterion): 0 -> eps*n (default, the
     paper's preferred choice), 1 -> eps*sqrt(n); eps = 2^-52. */
  int32_t eps1_mode;
  /* 0 (default): factor all min(m,n) columns; once the criterion holds, DM is
     switched off and single-column pivoting finishes (Sec. 4, DM safeguard).
     1: stop at the numerical rank; rows >= rank of the trailing block are
     left unreduced and htau[i] = 0 for i >= rank. */
  int32_t stop_at_rank;
  /* 1: the panel break test (Algorithm 4) also checks the last panel column;
     0 (default): the literal test, applied while l+1 < k_s (1-based). */
  int32_t check_last;
  /* 1: no break test at all (Algorithm 3). */
  int32_t no_break;
  /* 1: use delta_s = min(delta, tau^2 / max(1,|I|)) per step (eq. delta_max),
     which makes every DM block satisfy Lemma 1. */
  int32_t sdd;
  /* > 0: stop after this many block steps (partial factorization). */
  int32_t max_steps;
  /* 0 (default): everything in FP64.  1: FP32-class mixed precision: the
     trailing update and the candidate Gram matrix convert their FP64
     operands to FP32 on load and accumulate in FP32 (A stays FP64 and is
     updated in FP64); reflectors, panel, partial norms, recomputation and the
     rank decision stay FP64.  The stopping criterion then uses
     eps1 = max(eps1, 8 * 2^-24 * sqrt(n)), since FP32 updates leave roundoff
     of about 2^-24 ||A|| in the trailing block.
     2: split-BF16x3 on the tensor cores (tcgen05, FP32 accumulation in
     TMEM): the panel's sub-panels update only the rest of the panel (FP64),
     then the trailing block gets one merged update per step with all l
     reflectors, W = T^T V^T A22 and A22 -= V W, operands converted on load
     (FP64 -> FP32 -> hi + lo BF16; hi*hi + hi*lo + lo*hi).  Requires
     k_max <= 64 (QRDM_ERR_UNSUPPORTED otherwise); eps1 = max(eps1,
     2^-16 * sqrt(n)).  The candidate Gram matrix is computed on the tensor
     cores with the same split (partials per 64-row chunk summed in FP64).
     3: as 2 with 3xTF32 (kind::tf32; hi, lo TF32, rounded to nearest): an
     FP32-class form on the tensor cores: a product is exact to about 2^-20
     relative at worst (2^-24 typical), split-BF16x3 to 3 * 2^-16;
     eps1 = max(eps1, 8 * 2^-21 * sqrt(n)).
     In 2 and 3 each chunk of 64 rows of the W product has its own TMEM
     accumulator, summed in FP32 registers with round-to-nearest.
     4: the merged structure of 2 and 3 entirely in FP64 on the CUDA cores
     (the same results as 0 up to rounding order; k_max <= 64).
     In 1, 2 and 3 the partial-norm downdate recomputes a norm once
     t (u/uref)^2 <= sqrt(u_upd), with u_upd = 2^-24, 2^-16 and 2^-21, the
     unit roundoff of that form's trailing update, instead of sqrt(eps).
     Any other value: -11. */
  int32_t precision;
  /* 1: the checked path.  Every index the kernels derive on the device
     (argmax and candidate positions, the column moves of the permutation,
     the block and panel sizes, the step advance) is range-checked before it
     is used; a check that trips records itself in a device status word,
     skips the access and ends the factorization with QRDM_ERR_CHECKED (no
     trap, no assert: the context stays usable).  Results are identical to
     checked = 0.  Stands in for a memory checker. */
  int32_t checked;
  /* host, optional: per-kernel event timing (see qrdm_profile). */
  qrdm_profile* profile;
  /* host, optional: learned per-step (tau, delta) and feature logging (see
     qrdm_policy); NULL: tau and delta fixed for the whole factorization. */
  const struct qrdm_policy* policy;
  /* Limit of every device-side wait (the grid barriers of the cooperative
     single-column kernel, the mbarrier waits of the tensor-core kernels), in
     microseconds of the GPU's global timer; 0: 2 s.  A wait that runs out
     sets an abort flag that every CTA of the factorization observes, waits
     (bounded) for its own copies and MMAs in flight, frees its tensor
     memory, and the call returns QRDM_ERR_TIMEOUT.  Negative: -11. */
  int64_t wait_limit_us;
  /* Test hook, 0 in normal use.  1: the first grid barrier of the
     cooperative single-column kernel waits for one arrival more than the
     grid makes (a wait nothing completes; QRDM_ERR_TIMEOUT).  2 (needs
     checked = 1): the first column-move list gets a destination one past
     the last column, which the checked path must refuse (QRDM_ERR_CHECKED).
     3 (precision 2 or 3): the first tile of the tensor-core update waits
     on an mbarrier nothing arrives on (QRDM_ERR_TIMEOUT after its in-flight
     copies drained and its tensor memory was freed).  Other values: -11. */
  int32_t test_fault;
  int32_t reserved2;
} qrdm_opts;

/*
 * Learned per-step (tau, delta).  The paper fixes tau and delta for a whole
 * factorization and studies their choice empirically (Sec. 5); this library
 * can instead pick them per DM step with a small MLP over features of the
 * step.  Features (QRDM_POLICY_NFEAT = 16 floats, at the start of a DM step,
 * after mu = max u):
 *   0..7  min(#{j >= n_s, j != j*: u_j >= t mu}, 128) / 128 for
 *         t = 0.95, 0.9, 0.75, 0.6, 0.45, 0.3, 0.15, 0.05;
 *   8     (n - n_s) / n;   9  log2(n - n_s) / 16;
 *   10    log10(mu / max_j ||a_j||) / 16;
 *   11    l of the previous step / 64 (at most 1);   12  its l / k;
 *   13,14 mean and max |theta(j*, i)| over the previous step's candidates;
 *   15    tau of the previous step (0, 1, 0, 0, 0 for the first step).
 * MLP 16 -> 64 -> 64 -> 2 with ReLU, BF16 weights, FP32 accumulation;
 * tau_s = tau_lo + (tau_hi - tau_lo) sigmoid(o_0), delta_s likewise from o_1.
 * Weights: QRDM_POLICY_NPARAM bf16 values, row-major W1[16][64], b1[64],
 * W2[64][64], b2[64], W3[64][2], b3[2] (qrdm_mlp_* train them).
 * Guard (a check of the column-pivoting order): at the start of each DM step,
 * if the previous step used the MLP and accepted a pivot |R_ii| smaller than
 * rho_min times the largest partial norm now left (mu of this step), the
 * policy is switched off and the fixed (tau, delta) of the call finish the
 * factorization.  Single-column steps (after the stopping criterion) ignore
 * the policy.
 * With d_weights == NULL nothing is predicted: tau and delta stay fixed and
 * only the logs are written (training data from plain runs).
 */
#define QRDM_POLICY_NFEAT 16
#define QRDM_POLICY_HIDDEN 64
#define QRDM_POLICY_NPARAM 5378

typedef struct qrdm_policy {
  const void* d_weights; /* device bf16 weights, or NULL */
  float* d_feat_log;     /* device, optional: log_cap x 16 features per block step (qrdm_factor only) */
  double* d_act_log;     /* device, optional: log_cap x 2 (tau_s, delta_s) per block step (qrdm_factor only) */
  int64_t log_cap;
  double tau_lo, tau_hi;     /* 0 < tau_lo <= tau_hi <= 1 */
  double delta_lo, delta_hi; /* 0 <= delta_lo <= delta_hi <= 1 */
  double rho_min;            /* >= 0 */
} qrdm_policy;

/* Host-side results of one factorization. */
typedef struct qrdm_info {
  int64_t rank;        /* n_s at which the criterion of Sec. 3.4 first held (min(m,n) if never) */
  int64_t rank_colmax; /* same test without the sqrt(n - n_s) factor */
  int64_t nsteps;      /* block steps executed */
  int64_t launches;    /* kernels this call launched */
  int32_t cuda_error;  /* cudaError_t of the failing call when QRDM_ERR_CUDA */
  int32_t fail_code;   /* QRDM_FAIL_*: where a device-side wait or check gave up (0: none) */
  int32_t fail_cta;    /* CTA that recorded it (QRDM_FAIL_CHECK: the kernel id, QRDM_K_*) */
  int32_t reserved;
  int64_t fail_step;   /* block step at which it happened */
  int64_t fail_ns;     /* n_s at that step */
  int64_t fail_value;  /* code-specific value (see QRDM_FAIL_*) */
} qrdm_info;

/* One record per block step, written on the device when a trace is requested. */
typedef struct qrdm_step_record {
  int64_t ns;        /* columns factored before the step */
  int64_t jstar;     /* current position of the largest partial norm */
  int64_t ncand_all; /* candidates u_i >= tau*mu before the k_max - 1 cap */
  int64_t ncand;     /* |I| after the cap */
  int64_t k;         /* |J|: columns picked by DM */
  int64_t l;         /* reflectors accepted by the panel */
  int64_t dm_on;     /* 1 while DM pivoting is on */
  int64_t nrecomp;   /* partial norms recomputed in the norm update */
  double mu;         /* largest partial norm at step start */
  double eps_s;      /* panel break threshold tau*mu (eq. lenght_check) */
} qrdm_step_record;

/*
 * Bytes of device workspace qrdm_factor() needs for an m x n matrix and this
 * k_max (1 <= k_max <= QRDM_KMAX_LIMIT).  Returns 0 or -i.
 */
int qrdm_workspace_size(int64_t m, int64_t n, int32_t k_max, size_t* bytes);

/*
 * Factor A Pi = Q R in place (QRDM2, Algorithm 4 of the paper, with DM of
 * Algorithm 1 and the Sec. 4 choices).
 *
 *   dA      device, m x n, column-major, leading dimension lda >= max(1,m);
 *           on return R is in the upper triangle and the Householder vectors
 *           v_i (v_i(i) = 1 implicit) below the diagonal, as in LAPACK dgeqp3.
 *   tau     candidate threshold, 0 < tau <= 1 (eq. def_candidate_set).
 *   delta   cosine bound, 0 <= delta <= 1 (strict test |theta| < delta).
 *   k_max   block cap: |J| <= k_max, 1 <= k_max <= QRDM_KMAX_LIMIT; k_max = 1
 *           is QR with column pivoting (Algorithm 2).
 *   d_htau  device, min(m,n) doubles: Q = H_1 ... H_min(m,n),
 *           H_i = I - htau_i v_i v_i^T.
 *   d_perm  device, n int32: column i of A Pi is column d_perm[i] of A (0-based).
 *   info    host, required: rank, rank_colmax, steps.
 *   opts    host, may be NULL.
 *   d_work  device workspace of at least qrdm_workspace_size() bytes,
 *           256-byte aligned; its contents on entry are ignored.
 *   stream  cudaStream_t (NULL: the legacy default stream).
 *   d_trace, d_trace_J, trace_cap: optional (NULL/0) device step trace:
 *           trace_cap records and trace_cap*k_max int32 original column
 *           indices of J per step (-1 padded).
 *
 * Error behaviour: -1..-7 for invalid m, n, dA, lda, tau, delta, k_max; -8/-9
 * for NULL d_htau/d_perm when needed, -10 for NULL info, -11 for invalid
 * opts, -12 for a NULL workspace when one is needed.  m = 0 or n = 0 returns
 * 0 with rank 0 (after the same argument and option checks).
 * QRDM_ERR_TIMEOUT / QRDM_ERR_CHECKED / QRDM_ERR_INTERNAL fill info's fail_*
 * fields; the CUDA context stays usable and the next call starts afresh.
 */
int qrdm_factor(double* dA, int64_t m, int64_t n, int64_t lda, double tau, double delta, int32_t k_max,
                double* d_htau, int32_t* d_perm, qrdm_info* info, const qrdm_opts* opts, void* d_work,
                size_t work_bytes, void* stream, qrdm_step_record* d_trace, int32_t* d_trace_J, int64_t trace_cap);

/*
 * Size of the fixed device scratch used by qrdm_factor_noalloc: 32 MiB.
 * A shape fits when qrdm_workspace_size(m, n, k_max) is at most this, e.g.
 * 4096 x 4096 with k_max <= 32 or 2048 x 2048 with k_max <= 64.
 */
#define QRDM_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * qrdm_factor for callers that cannot allocate device memory: code running
 * under an allocator that owns the whole device (a framework's caching
 * pool, a fixed-footprint service), a real-time loop that must not call
 * cudaMalloc or cudaFree because they may synchronize the device, or a
 * caller with no spare buffer to offer as workspace.  The paper has no
 * counterpart; this is a property of the library.
 *
 * Like qrdm_factor it drives the factorization from the host: it copies the
 * step state to the host and synchronizes `stream` several times per
 * factorization, so it blocks the calling thread, cannot be captured into a
 * CUDA graph and must not be called from a stream callback.
 *
 * Same arguments, outputs and error codes as qrdm_factor() minus d_work and
 * work_bytes.  The workspace is one array of QRDM_NOALLOC_SCRATCH_BYTES in
 * the library's device image; every GPU that loads the library holds it
 * until the process exits, and the call itself allocates nothing.
 *
 *   - Shapes whose workspace exceeds the scratch are rejected with
 *     QRDM_ERR_WORKSPACE before anything is touched.
 *   - The first call on a device looks up the scratch's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     process.
 *   - All calls share the one scratch.  Each call re-initializes every part
 *     of it that it reads, so earlier contents do not matter, but calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on it:
 *     serialize them.
 *   - opts->profile must be NULL (profiling creates CUDA events):
 *     QRDM_ERR_UNSUPPORTED otherwise.
 */
int qrdm_factor_noalloc(double* dA, int64_t m, int64_t n, int64_t lda, double tau, double delta, int32_t k_max,
                        double* d_htau, int32_t* d_perm, qrdm_info* info, const qrdm_opts* opts, void* stream,
                        qrdm_step_record* d_trace, int32_t* d_trace_J, int64_t trace_cap);

/*
 * Batched QRDM: many independent matrices factored by one persistent kernel.
 * Each CTA factors whole matrices taken from a work queue, largest first
 * (geqrf flop count), so no CTA ever waits on another.  Every matrix gets the
 * QRDM2 of qrdm_factor (Algorithm 4 with the DM selection of Algorithm 1 and
 * Sec. 4, the Sec. 3.4 stopping criterion), in FP64, with the same readings;
 * only the summation order inside a CTA differs.  The paper factors one
 * matrix at a time; the batched form, its plan object, the CUDA-graph launch
 * and the autotuner have no counterpart in it.
 *
 * Use:
 *   qrdm_batch_plan_create     validates the matrix list (host array, copied),
 *                              orders it, picks a default tuning;
 *   qrdm_batch_workspace_size  device bytes the plan needs;
 *   qrdm_batch_bind            attaches a workspace and uploads the matrix
 *                              descriptors (synchronizes `stream`);
 *   qrdm_batch_autotune        optional: times every feasible tuning on the
 *                              plan's own matrices, restores them, keeps the
 *                              fastest (allocates a device backup of all
 *                              matrices for its duration);
 *   qrdm_factor_batched        enqueues the factorization on `stream` (a
 *                              counter reset and one kernel launch; no host
 *                              synchronization, so it may be captured);
 *   qrdm_factor_batched_graph  the same through a CUDA graph that the plan
 *                              captures on first use and replays afterwards
 *                              (recaptured when tau, delta, opts, the tuning
 *                              or the workspace change);
 *   qrdm_batch_results         rank, rank_colmax, status (0 ok, 1 non-finite
 *                              input: that matrix is left unmodified and its
 *                              ranks are -1) and block steps per matrix, in
 *                              the caller's order, copied to host arrays
 *                              (NULL: skipped; synchronizes `stream`);
 *   qrdm_batch_plan_destroy.
 * Each matrix is factored in place like qrdm_factor: R and the reflectors in
 * dA, htau in d_htau (min(m, n)), the 0-based int32 permutation in d_perm
 * (n).  Matrices must not overlap.  An optional per-matrix step trace
 * (d_trace, d_trace_J, trace_cap) is written as in qrdm_factor.  opts may be
 * NULL; eps1_mode, stop_at_rank, check_last, no_break and sdd are honoured,
 * max_steps and wait_limit_us are ignored (no CTA ever waits on another),
 * precision, checked and test_fault must be 0 (QRDM_ERR_UNSUPPORTED
 * otherwise).  opts->policy applies to every matrix (its d_weights, ranges and
 * rho_min; the per-matrix logs come from qrdm_batch_matrix).  A profile
 * (qrdm_factor_batched only; it then times the launch
 * with events and synchronizes `stream`) receives, added to its contents:
 * ms[0..7] the kernel time split by the CTAs' clock shares of the phases
 * norms, argmax and candidates, Gram, DM pick, swaps, panel, block
 * reflector, norm downdate; ms[8] the kernel time; flops[0] the load balance
 * (mean over CTAs of their active time divided by the largest); launches[0]
 * one per call.  One plan serves one device and one host
 * thread at a time.
 * Errors: -i for an invalid i-th argument (-2 from qrdm_batch_plan_create
 * for any invalid matrix entry), QRDM_ERR_WORKSPACE for a missing, small or
 * misaligned workspace, QRDM_ERR_UNSUPPORTED for a tuning whose CTAs do not
 * fit on an SM, QRDM_ERR_CUDA.
 */
#define QRDM_BATCH_MAX_CTAS_PER_SM 2

typedef struct qrdm_batch_plan qrdm_batch_plan; /* opaque host object */

typedef struct qrdm_batch_matrix {
  double* dA;      /* device, m x n column-major, leading dimension lda >= max(1, m) */
  int64_t m, n, lda;
  double* d_htau;  /* device, min(m, n) doubles */
  int32_t* d_perm; /* device, n int32 */
  qrdm_step_record* d_trace; /* optional device trace, trace_cap records (NULL/0: none) */
  int32_t* d_trace_J;        /* optional, trace_cap * k_max int32 */
  int64_t trace_cap;
  float* d_feat_log;         /* optional, log_cap x 16 policy features per block step */
  double* d_act_log;         /* optional, log_cap x 2 (tau_s, delta_s) per block step */
  int64_t log_cap;
} qrdm_batch_matrix;

typedef struct qrdm_batch_tuning {
  int32_t ctas_per_sm;   /* resident CTAs per SM, 1..QRDM_BATCH_MAX_CTAS_PER_SM */
  int32_t rows_per_pass; /* rows of V staged in shared memory per pass, 64..1024, multiple of 64 */
  int32_t lanes_per_col; /* lanes sharing one column in the block reflector phases: 4 or 8 */
  int32_t reserved;
} qrdm_batch_tuning;

int qrdm_batch_plan_create(int64_t count, const qrdm_batch_matrix* h_mats, int32_t k_max, qrdm_batch_plan** plan);
void qrdm_batch_plan_destroy(qrdm_batch_plan* plan);
int qrdm_batch_workspace_size(const qrdm_batch_plan* plan, size_t* bytes);
int qrdm_batch_bind(qrdm_batch_plan* plan, void* d_work, size_t work_bytes, void* stream);
int qrdm_batch_get_tuning(const qrdm_batch_plan* plan, qrdm_batch_tuning* tuning);
int qrdm_batch_set_tuning(qrdm_batch_plan* plan, const qrdm_batch_tuning* tuning);
int qrdm_batch_autotune(qrdm_batch_plan* plan, double tau, double delta, const qrdm_opts* opts, void* stream,
                        qrdm_batch_tuning* best, double* best_ms);
int qrdm_factor_batched(qrdm_batch_plan* plan, double tau, double delta, const qrdm_opts* opts, void* stream);
int qrdm_factor_batched_graph(qrdm_batch_plan* plan, double tau, double delta, const qrdm_opts* opts, void* stream);
int qrdm_batch_results(const qrdm_batch_plan* plan, int64_t* h_rank, int64_t* h_rank_colmax, int32_t* h_status,
                       int64_t* h_steps, void* stream);

/*
 * Training of the learned (tau, delta) policy (qrdm_policy): the MLP's
 * forward pass, its loss gradient, Adam, and a minibatch training loop, all
 * on the device.  FP32 master weights d_w32 (QRDM_POLICY_NPARAM floats) and
 * BF16 working weights d_w16 (QRDM_POLICY_NPARAM bf16, what the forward pass
 * and the factorization read).  Inputs x: batch x 16 features (row-major),
 * targets t: batch x 2 in [0, 1] (the normalized tau and delta), outputs
 * y = sigmoid(o): batch x 2.  Loss L = (1/B) sum_b sum_o (y_bo - t_bo)^2 / 2.
 * The gradient is taken with respect to the BF16 weights (the master weights
 * receive it unchanged).  Every kernel is deterministic (fixed summation
 * order, no atomics); minibatch row b of step s is sample
 * splitmix64(seed, s, b) mod nsamples.  The paper has no learned component.
 *   qrdm_mlp_workspace_size  float workspace bytes for a batch;
 *   qrdm_mlp_init            He-uniform weights from the seed, zero biases,
 *                            and the BF16 copy;
 *   qrdm_mlp_to_bf16         refresh the BF16 copy from the master weights;
 *   qrdm_mlp_forward         y for a batch;
 *   qrdm_mlp_loss_grad       L (1 float) and dL/dw (QRDM_POLICY_NPARAM floats);
 *   qrdm_mlp_adam_step       one Adam step (Kingma & Ba; decoupled weight
 *                            decay, none on biases), step counter t >= 1;
 *   qrdm_mlp_train           `steps` minibatches of `batch` samples from
 *                            (d_x, d_t) with Adam (beta1 0.9, beta2 0.999,
 *                            eps 1e-8); d_adam holds 2 x QRDM_POLICY_NPARAM
 *                            floats (zero them before the first call);
 *                            d_loss_log (optional) receives each step's loss.
 * All pointers are device memory; calls enqueue on `stream` and return.
 * Errors: -i for an invalid i-th argument, QRDM_ERR_WORKSPACE, QRDM_ERR_CUDA.
 */
int qrdm_mlp_workspace_size(int64_t batch, size_t* bytes);
int qrdm_mlp_init(float* d_w32, void* d_w16, uint64_t seed, void* stream);
int qrdm_mlp_to_bf16(const float* d_w32, void* d_w16, void* stream);
int qrdm_mlp_forward(const void* d_w16, const float* d_x, int64_t batch, float* d_y, float* d_work,
                     size_t work_bytes, void* stream);
int qrdm_mlp_loss_grad(const void* d_w16, const float* d_x, const float* d_t, int64_t batch, float* d_grad,
                       float* d_loss, float* d_work, size_t work_bytes, void* stream);
int qrdm_mlp_adam_step(float* d_w32, void* d_w16, const float* d_grad, float* d_m, float* d_v, int64_t t, float lr,
                       float beta1, float beta2, float eps, float weight_decay, void* stream);
int qrdm_mlp_train(float* d_w32, void* d_w16, float* d_adam, const float* d_x, const float* d_t, int64_t nsamples,
                   int64_t batch, int64_t steps, float lr, float weight_decay, uint64_t seed, float* d_loss_log,
                   float* d_work, size_t work_bytes, void* stream);

/*
 * Least squares with a QRDM factorization (the paper stops at the
 * factorization; the solve is this library's).  With A Pi = Q R from
 * qrdm_factor (dQR, d_htau, d_perm as it returned them) and a rank r (e.g.
 * info.rank or rank_colmax), the basic solution of min ||A x - b|| is
 *   x = Pi [R11^{-1} (Q^T b)_{1:r}; 0],
 * Q^T b by the stored reflectors H_1..H_r, R11 the leading r x r block of R.
 * refine > 0 iterations of FP64 refinement use the original matrix dA
 * (unchanged copy, FP64): r_k = b - A x_k, x_{k+1} = x_k + basic(r_k).  This
 * recovers FP64 accuracy from a factorization computed in reduced precision
 * (opts.precision = 1, 2 or 3) when the system is compatible (b in the range of A)
 * or its residual is small; for other systems the fixed point satisfies
 * Q1^T (b - A x) = 0 with the computed Q1.
 * Arguments: dA/lda (may be NULL when refine = 0), dQR/ldqr, m, n, d_htau,
 * d_perm, rank, dB/ldb (m x nrhs, read only), dX/ldx (n x nrhs, written),
 * refine (0..100); h_resid (host, optional): (refine + 1) x nrhs residual
 * 2-norms ||b - A x_k|| per column, before each correction and after the
 * last (needs dA; synchronizes the stream per iteration).  Device workspace
 * of qrdm_ls_workspace_size bytes, 16-byte aligned.  m <= 24576 (a column of
 * b is kept in shared memory).
 * Errors: -i for an invalid i-th argument, QRDM_ERR_WORKSPACE, QRDM_ERR_CUDA.
 */
int qrdm_ls_workspace_size(int64_t m, int64_t n, int64_t rank, int64_t nrhs, size_t* bytes);
int qrdm_ls_solve(const double* dA, int64_t lda, const double* dQR, int64_t ldqr, int64_t m, int64_t n,
                  const double* d_htau, const int32_t* d_perm, int64_t rank, const double* dB, int64_t ldb,
                  int64_t nrhs, double* dX, int64_t ldx, int32_t refine, double* h_resid, void* d_work,
                  size_t work_bytes, void* stream);

/*
 * Comparator: blocked QR with column pivoting with lazy updates (the scheme
 * of LAPACK's xGEQP3 / xLAQPS by Quintana-Orti, Sun and Bischof, which the
 * paper measures QRDM against in Sec. 5), written for this GPU as one
 * cooperative persistent kernel.  Pivots are the largest partial norm
 * (ties to the lowest position), so the permutation is that of qrdm_factor
 * with k_max = 1; the block size nb (1..32) only changes how the trailing
 * update is applied (F accumulates nb columns, then one blocked update).
 * A partial norm whose downdate cancels (t (vn1/vn2)^2 <= sqrt(eps)) ends
 * the block early and is recomputed exactly after its update.
 * Outputs as qrdm_factor (R and reflectors in dA, htau, 0-based int32
 * permutation, info.rank / rank_colmax from the Sec. 3.4 criterion with
 * eps1_mode, info.nsteps = blocks).  Workspace: qrdm_qp3_workspace_size
 * bytes, 256-byte aligned.  Synchronizes the stream.
 * Errors: -i for an invalid i-th argument, QRDM_ERR_WORKSPACE,
 * QRDM_ERR_NONFINITE (A left unmodified), QRDM_ERR_UNSUPPORTED (no
 * cooperative launch), QRDM_ERR_TIMEOUT (a grid barrier wait gave up after 2 s; info.fail_*),
 * QRDM_ERR_CUDA.
 */
int qrdm_qp3_workspace_size(int64_t m, int64_t n, int32_t nb, size_t* bytes);
int qrdm_qp3_factor(double* dA, int64_t m, int64_t n, int64_t lda, int32_t nb, double* d_htau, int32_t* d_perm,
                    qrdm_info* info, int32_t eps1_mode, void* d_work, size_t work_bytes, void* stream);

/*
 * FP64 rate probe (not part of the factorization): times one launch of
 * `blocks` x 256 threads that run `iters` rounds of FP64 arithmetic, so that
 * the FP64 kernels' roofline can be read against a measured rate.
 *   which 0: FFMA64, eight independent fma chains per thread (16 flops per
 *            thread and round);
 *   which 1: DMMA, mma.sync m8n8k4 FP64 with four independent accumulators
 *            per warp (2048 flops per warp and round).
 * d_out: device scratch of blocks x 256 doubles (the chains' sums land
 * there); *flops (host) the flops performed, *ms (host) the launch's time by
 * CUDA events on `stream`.  Synchronizes the stream.  Errors: -i for an
 * invalid i-th argument, QRDM_ERR_CUDA.
 */
int qrdm_fp64_probe(int32_t which, int32_t blocks, int32_t iters, void* d_out, size_t out_bytes, double* flops,
                    float* ms, void* stream);

/* Static description of an error code. */
const char* qrdm_strerror(int code);

/* cudaError_t of the last failing CUDA call in this thread (0 if none). */
int qrdm_last_cuda_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int qrdm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QRDM_H */
