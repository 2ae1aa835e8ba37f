/*
 * QRDM oracle: a plain, slow, single-threaded FP64 restatement of QR with
 * Deviation Maximization pivoting (Dessole & Marcuzzi, "Deviation
 * Maximization for Rank-Revealing QR Factorizations", 2021).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library; the two are compared on the same
 * seeded inputs.
 *
 * What it follows, step by step (0-based indices in the code):
 *   - Algorithm 4 (QRDM2): the block loop, the panel with its break check,
 *     compact WY, the trailing update and the norm update.
 *   - Algorithm 1 (DM): argmax, candidate set, cosine matrix, greedy pick.
 *   - Sec. 4: candidates sorted by partial norm and capped (eq.
 *     candidate_set_limited_by_kDM); cosine matrix by option (ii), Gram then
 *     diagonal scaling; DM switched off once column norms reach roundoff
 *     level (eq. column_norm_bound_DM); pivots applied as pairwise swaps.
 *   - Sec. 3.4: the practical stopping criterion (eq. practical stopping
 *     criterion) with eps1 = eps*n or eps*sqrt(n).
 *   - Sec. 3.1 / 3.2: the partial column norm downdate, in block form, with
 *     recomputation when cancellation makes it unreliable (the paper cites
 *     Drmac & Bujanovic 2008 for the robust form; see READINGS).
 *   - Sec. 3.2: compact WY, I - V T V^T = H_1 ... H_l (Schreiber & Van Loan).
 *
 * READINGS where the paper is silent, ambiguous or garbled:
 *   R1  u holds norms (not squared norms); the candidate test is
 *       u_i >= tau * max u (Sec. 2, eq. def_candidate_set).
 *   R2  k_max caps |J|, so |I| <= k_max - 1; k_max = 1 is column pivoting.
 *   R3  Theta is formed over {j*} and I (Alg. 1 forms it over I but compares
 *       candidates with j*).
 *   R4  candidates are visited by decreasing u, ties by lower position.
 *   R5  the cosine test is strict (|theta| < delta); the candidate test is
 *       non-strict; the break test is strict.
 *   R6  D = diag(sqrt(G_aa)) from the Gram diagonal; a zero column gets
 *       |theta| = 1 (never accepted).
 *   R7  DM acts on trailing columns n_s+1..n (1-based).
 *   R8  the block downdate subtracts only the rows eliminated in this step.
 *   R9  robust downdate: t = max(0, 1 - sum_r (r_rj/u_j)^2); if
 *       t * (u_j/uref_j)^2 <= sqrt(eps) the norm is recomputed from the
 *       trailing column and uref_j reset, else u_j *= sqrt(t).
 *   R10 the break test is literal (checked only while l+1 < k_s, 1-based),
 *       optionally also for the last panel column (check_last).
 *   R11 eps_s = tau * mu, mu the largest partial norm at step start.
 *   R12 "O(eps)" in the DM safeguard is the stopping criterion itself: once
 *       it holds DM is off and single-column pivoting finishes the work.
 *   R13 eps = 2^-52.
 *   R14 pairwise swaps use the selected column's current position.
 *   R15 argmax ties go to the lowest position.
 *   R16 rejected panel columns keep the l accepted reflectors and get their
 *       partial norm recomputed.
 *   Householder: beta = -sign(alpha) ||x||, htau = (beta - alpha) / beta,
 *   v = x / (alpha - beta), v_0 = 1; a zero tail gives htau = 0, beta = alpha.
 *
 * Compiled with -O2 -ffp-contract=off: every operation rounds once.
 *
 * PINS (tests/test_oracle_pins.py): closed-form reflectors and T, exact
 * hand-derived DM decisions and equality edges, brute-force column pivoting
 * at k_max = 1, A Pi = Q R to roundoff, exact ranks, the stopping test and
 * the DM safeguard on exact diagonals, the partial norms within the
 * downdate bound of the true norms, the SDD threshold, the paper's SDD
 * lemmas and worst-case theorems, exhaustive subset search, and invariances
 * (exact power-of-two scaling, column permutations, a left orthogonal
 * factor).  tests/test_oracle_bruteforce.py compares every decision with a
 * brute-force QRDM2 (exact norms, unblocked reflectors) on small matrices.
 * Parity unpinned: the
 * permutation on Kahan matrices, whose columns all have unit norm in exact
 * arithmetic, so that every pivot decision there is a rounding tie; those
 * runs are checked through invariants only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OQ_EPS 2.220446049250313080847e-16 /* 2^-52 */

/* one record per block step (see oracle.py for the field meanings) */
typedef struct {
  int64_t ns;        /* columns factored before this step */
  int64_t jstar;     /* current position of the argmax column */
  int64_t ncand_all; /* candidates before the cap */
  int64_t ncand;     /* |I| after the cap */
  int64_t k;         /* |J| */
  int64_t l;         /* reflectors accepted */
  int64_t dm_on;     /* 1 while DM pivoting is on */
  int64_t nrecomp;   /* partial norms recomputed in the norm update */
  double mu;         /* largest partial norm at step start */
  double eps_s;      /* break threshold tau * mu */
  /* decision margins, each divided by the comparison's uncertainty
     (a value below 1 marks a decision that rounding could flip) */
  double s_argmax, s_cand, s_order, s_cos, s_break, s_stop, s_recomp;
  /* raw relative margins */
  double g_argmax, g_cand, g_cos, g_break, g_stop;
} oq_step;

#define A_(i, j) A[(size_t)(j) * (size_t)lda + (size_t)(i)]

static double sumsq(const double* x, int64_t len) {
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s += x[i] * x[i];
  return s;
}

/* Householder reflector on x[0..len): H = I - htau v v^T, H x = beta e_1.
   On return x[0] = beta and x[1..len) holds v's tail (v_0 = 1 implicit). */
void oq_house(int64_t len, double* x, double* beta, double* htau) {
  double alpha = x[0];
  double s2 = sumsq(x + 1, len - 1);
  if (s2 == 0.0) {
    *beta = alpha;
    *htau = 0.0;
    return;
  }
  double nrm = sqrt(alpha * alpha + s2);
  double b = (alpha >= 0.0) ? -nrm : nrm;
  *htau = (b - alpha) / b;
  double den = alpha - b;
  for (int64_t i = 1; i < len; ++i) x[i] = x[i] / den;
  x[0] = b;
  *beta = b;
}

/* Compact WY (forward, columnwise): T upper l x l with
   H_1 H_2 ... H_l = I - V T V^T.  V is mr x l, unit lower trapezoidal,
   stored below its diagonal (entries on and above the diagonal are not read). */
void oq_larft(int64_t mr, int64_t l, const double* V, int64_t ldv, const double* htau, double* T, int64_t ldt) {
  for (int64_t i = 0; i < l; ++i) {
    for (int64_t r = 0; r < l; ++r) T[i * ldt + r] = 0.0;
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)(l > 0 ? l : 1));
  for (int64_t i = 0; i < l; ++i) {
    /* y_r = v_r^T v_i for r < i; v_r has 1 at row r, v_i has 1 at row i, zeros above */
    for (int64_t r = 0; r < i; ++r) {
      double s = V[r * ldv + i]; /* row i of v_r times v_i's unit entry */
      for (int64_t q = i + 1; q < mr; ++q) s += V[r * ldv + q] * V[i * ldv + q];
      y[r] = s;
    }
    /* T[0:i, i] = -htau_i * T[0:i, 0:i] * y */
    for (int64_t r = 0; r < i; ++r) {
      double s = 0.0;
      for (int64_t q = r; q < i; ++q) s += T[q * ldt + r] * y[q];
      T[i * ldt + r] = -htau[i] * s;
    }
    T[i * ldt + i] = htau[i];
  }
  free(y);
}

/* Gram G = C^T C and cosine matrix Theta = D^-1 G D^-1 of the columns
   cols[0..kc) of A, rows r0..m-1 (Sec. 2 definition, Sec. 4 option (ii)).
   G and Theta are kc x kc, column-major, both triangles filled. */
void oq_cosine(int64_t m, int64_t r0, const double* A, int64_t lda, int64_t kc, const int64_t* cols, double* G,
               double* Theta) {
  for (int64_t a = 0; a < kc; ++a) {
    for (int64_t b = a; b < kc; ++b) {
      double s = 0.0;
      const double* ca = A + (size_t)cols[a] * (size_t)lda;
      const double* cb = A + (size_t)cols[b] * (size_t)lda;
      for (int64_t i = r0; i < m; ++i) s += ca[i] * cb[i];
      G[b * kc + a] = s;
      G[a * kc + b] = s;
    }
  }
  for (int64_t a = 0; a < kc; ++a) {
    for (int64_t b = 0; b < kc; ++b) {
      double d = sqrt(G[a * kc + a]) * sqrt(G[b * kc + b]);
      Theta[b * kc + a] = (d > 0.0) ? G[b * kc + a] / d : (a == b ? 1.0 : 1.0);
    }
  }
}

/* relative uncertainty of a partial norm u_j when two correct FP64 programs
   compute it with different rounding: absolute error ~ c_err eps anorm in the
   trailing entries, amplified by uref/u through the downdate. */
static double u_unc(double cerr, double anorm, double u, double uref) {
  if (u <= 0.0) return INFINITY;
  double amp = (uref > u) ? uref / u : 1.0;
  return 1e-12 + cerr * OQ_EPS * anorm * amp / u;
}

static int cmp_desc(double ua, int64_t pa, double ub, int64_t pb) {
  /* 1 if (ua, pa) sorts before (ub, pb): larger u first, then lower position */
  if (ua > ub) return 1;
  if (ua < ub) return 0;
  return pa < pb;
}

/*
 * Factor A (m x n, column-major, leading dimension lda) in place:
 *   A Pi = Q R, R in the upper triangle, reflector tails below the diagonal,
 *   htau[min(m,n)], perm[n] (perm[i] = original index of column i of A Pi).
 * Options:
 *   eps1_mode 0: eps1 = eps*n, 1: eps1 = eps*sqrt(n)  (Sec. 3.4)
 *   stop_at_rank: stop when the criterion first holds (R22 left unreduced)
 *   check_last: break test also on the last panel column (R10)
 *   no_break: Algorithm 3 (no break test)
 *   sdd: per-step delta_s = min(delta, tau^2 / max(1, |I|)) (eq. delta_max)
 *   max_steps: stop after this many block steps (<= 0: no limit)
 *   tau_sched, delta_sched, sched_len (oq_qrdm_sched only): the (tau, delta)
 *   of block step s is (tau_sched[s], delta_sched[s]) for s < sched_len,
 *   else (tau, delta) (a per-step schedule, e.g. one a learned policy chose)
 * Outputs: rank (criterion eq. practical stopping criterion), rank_colmax
 *   (the same test without the sqrt(n - n_s) factor), u_out/uref_out (n, may
 *   be NULL), trace (trace_cap records, may be NULL), Jout (trace_cap*k_max
 *   original column indices of J per step), nsteps.  With stop_at_rank, a
 *   stop by the criterion also writes the stopping test's record (k = -1)
 *   at trace[nsteps] when trace_cap > nsteps.
 * Returns 0, or -i for an invalid i-th argument, or 1 for non-finite input.
 */
int oq_qrdm_sched(int64_t m, int64_t n, double* A, int64_t lda, double tau, double delta, int64_t kmax,
                  int64_t eps1_mode, int64_t stop_at_rank, int64_t check_last, int64_t no_break, int64_t sdd,
                  int64_t max_steps, double* htau, int64_t* perm, int64_t* rank_out, int64_t* rank_colmax_out,
                  double* u_out, double* uref_out, oq_step* trace, int64_t trace_cap, int64_t* Jout,
                  int64_t* nsteps_out, const double* tau_sched, const double* delta_sched, int64_t sched_len) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (!(tau > 0.0 && tau <= 1.0)) return -5;
  if (!(delta >= 0.0 && delta <= 1.0)) return -6;
  if (kmax < 1) return -7;

  const int64_t kmin = m < n ? m : n;
  for (int64_t j = 0; j < n; ++j) perm[j] = j;
  for (int64_t i = 0; i < kmin; ++i) htau[i] = 0.0;
  *rank_out = -1;
  *rank_colmax_out = -1;
  if (nsteps_out) *nsteps_out = 0;

  double* u = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* uref = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double anorm = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double s = sumsq(&A_(0, j), m);
    if (!isfinite(s)) {
      free(u);
      free(uref);
      return 1;
    }
    u[j] = sqrt(s);
    uref[j] = u[j];
    if (u[j] > anorm) anorm = u[j];
  }
  const double eps1 = (eps1_mode == 1) ? OQ_EPS * sqrt((double)n) : OQ_EPS * (double)n;
  const double cerr = sqrt((double)(m > 1 ? m : 1) * (double)(n > 1 ? n : 1));
  const double sqeps = sqrt(OQ_EPS);

  int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)(kmax + 1));
  int64_t* Jloc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(kmax + 1));
  int64_t* selpos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(kmax + 1));
  double* G = (double*)malloc(sizeof(double) * (size_t)(kmax * kmax + 1));
  double* Th = (double*)malloc(sizeof(double) * (size_t)(kmax * kmax + 1));
  double* T = (double*)malloc(sizeof(double) * (size_t)(kmax * kmax + 1));
  double* W = (double*)malloc(sizeof(double) * (size_t)(kmax * (n > 0 ? n : 1) + 1));

  int dm_on = 1;
  int64_t ns = 0, step = 0;
  while (ns < kmin) {
    if (max_steps > 0 && step >= max_steps) break;
    const int in_sched = (tau_sched && delta_sched && step < sched_len);
    const double tau_s = in_sched ? tau_sched[step] : tau;
    const double delta_s = in_sched ? delta_sched[step] : delta;
    oq_step rec;
    memset(&rec, 0, sizeof(rec));
    rec.ns = ns;
    rec.s_argmax = rec.s_cand = rec.s_order = rec.s_cos = rec.s_break = rec.s_stop = rec.s_recomp = INFINITY;
    rec.g_argmax = rec.g_cand = rec.g_cos = rec.g_break = rec.g_stop = INFINITY;

    /* ---- a2/a3: argmax of the partial norms (Alg. 1, first line) ---- */
    int64_t jstar = ns;
    double mu = u[ns];
    for (int64_t j = ns + 1; j < n; ++j) {
      if (u[j] > mu) {
        mu = u[j];
        jstar = j;
      }
    }
    {
      /* margin to the runner-up */
      double second = -1.0;
      int64_t js2 = -1;
      for (int64_t j = ns; j < n; ++j) {
        if (j != jstar && u[j] > second) {
          second = u[j];
          js2 = j;
        }
      }
      if (js2 >= 0 && mu > 0.0) {
        double g = (mu - second) / mu;
        double tol = u_unc(cerr, anorm, mu, uref[jstar]) + u_unc(cerr, anorm, second, uref[js2]);
        rec.g_argmax = g;
        rec.s_argmax = g / tol;
      }
    }
    const int64_t nrem = n - ns;
    /* ---- a2: stopping criterion (Sec. 3.4) and DM safeguard (Sec. 4) ---- */
    if (*rank_colmax_out < 0 && mu <= eps1 * anorm) *rank_colmax_out = ns;
    {
      double lhs = sqrt((double)nrem) * mu, rhs = eps1 * anorm;
      if (rhs > 0.0 && *rank_out < 0) {
        double g = fabs(lhs - rhs) / rhs;
        double tol = sqrt((double)nrem) * mu * u_unc(cerr, anorm, mu, uref[jstar]) / rhs;
        rec.g_stop = g;
        rec.s_stop = (tol > 0.0) ? g / tol : INFINITY;
      }
      if (*rank_out < 0 && lhs <= rhs) {
        *rank_out = ns;
        dm_on = 0;
        if (stop_at_rank) {
          /* the stopping test's own record (its margin s_stop), k = -1, kept
             past the nsteps executed steps */
          rec.k = -1;
          rec.mu = mu;
          rec.jstar = jstar;
          if (trace && step < trace_cap) trace[step] = rec;
          break;
        }
      }
    }
    rec.dm_on = dm_on;
    rec.mu = mu;
    rec.jstar = jstar;
    int64_t kcap = dm_on ? kmax : 1;
    if (kcap > kmin - ns) kcap = kmin - ns;

    /* ---- a3: candidate set I (eq. def_candidate_set), sorted, capped ---- */
    int64_t nc = 0;
    if (kcap > 1) {
      const double thr = tau_s * mu;
      for (int64_t j = ns; j < n; ++j) {
        if (j == jstar) continue;
        if (mu > 0.0) {
          double g = fabs(u[j] - thr) / thr;
          double tol = u_unc(cerr, anorm, u[j], uref[j]) + u_unc(cerr, anorm, mu, uref[jstar]);
          if (g < rec.g_cand) rec.g_cand = g;
          if (g / tol < rec.s_cand) rec.s_cand = g / tol;
        }
        if (u[j] >= thr) cand[nc++] = j;
      }
      /* insertion sort by (u desc, position asc) */
      for (int64_t a = 1; a < nc; ++a) {
        int64_t x = cand[a];
        int64_t b = a - 1;
        while (b >= 0 && cmp_desc(u[x], x, u[cand[b]], cand[b])) {
          cand[b + 1] = cand[b];
          --b;
        }
        cand[b + 1] = x;
      }
      /* order margins among kept candidates and at the cap boundary */
      int64_t keep = nc < kcap - 1 ? nc : kcap - 1;
      int64_t last = (nc > keep) ? keep : keep - 1;
      for (int64_t a = 0; a < last; ++a) {
        int64_t p = cand[a], q = cand[a + 1];
        double g = (u[p] - u[q]) / u[p];
        double tol = u_unc(cerr, anorm, u[p], uref[p]) + u_unc(cerr, anorm, u[q], uref[q]);
        if (g / tol < rec.s_order) rec.s_order = g / tol;
      }
    }
    rec.ncand_all = nc;
    if (nc > kcap - 1) nc = kcap - 1;
    if (nc < 0) nc = 0;
    rec.ncand = nc;

    /* ---- a4/a5: cosine matrix and greedy DM pick (Alg. 1 loop) ---- */
    int64_t k = 1;
    Jloc[0] = 0;
    cols[0] = jstar;
    for (int64_t a = 0; a < nc; ++a) cols[a + 1] = cand[a];
    const int64_t kc = nc + 1;
    if (nc > 0) {
      oq_cosine(m, ns, A, lda, kc, cols, G, Th);
      double dlt = delta_s;
      if (sdd) {
        double dm = tau_s * tau_s / (double)(nc > 1 ? nc : 1);
        if (dm < dlt) dlt = dm;
      }
      for (int64_t a = 1; a < kc; ++a) {
        double worst = 0.0;
        int ok = 1;
        for (int64_t b = 0; b < k; ++b) {
          double th = fabs(Th[Jloc[b] * kc + a]);
          if (G[a * kc + a] <= 0.0 || G[Jloc[b] * kc + Jloc[b]] <= 0.0) th = 1.0;
          if (th > worst) worst = th;
          if (!(th < dlt)) ok = 0;
        }
        /* margin of this candidate's decision; cosine uncertainty from the
           trailing entries' absolute error relative to the column norms */
        double na = sqrt(G[a * kc + a]);
        double g = fabs(worst - dlt);
        double tol = 1e-12 + cerr * OQ_EPS * anorm * (1.0 / (na > 0 ? na : 1e-300) + 1.0 / (mu > 0 ? mu : 1e-300));
        if (g < rec.g_cos) rec.g_cos = g;
        if (g / tol < rec.s_cos) rec.s_cos = g / tol;
        if (ok) Jloc[k++] = a;
      }
    }
    rec.k = k;

    /* ---- a6: pairwise swaps (Sec. 4, last paragraph) ---- */
    for (int64_t t = 0; t < k; ++t) selpos[t] = cols[Jloc[t]];
    for (int64_t t = 0; t < k; ++t) {
      int64_t q = ns + t, p = selpos[t];
      if (p != q) {
        double* cq = &A_(0, q);
        double* cp = &A_(0, p);
        for (int64_t i = 0; i < m; ++i) {
          double tmp = cq[i];
          cq[i] = cp[i];
          cp[i] = tmp;
        }
        double tu = u[q];
        u[q] = u[p];
        u[p] = tu;
        tu = uref[q];
        uref[q] = uref[p];
        uref[p] = tu;
        int64_t tp = perm[q];
        perm[q] = perm[p];
        perm[p] = tp;
        for (int64_t t2 = t + 1; t2 < k; ++t2)
          if (selpos[t2] == q) selpos[t2] = p;
      }
    }
    if (Jout && trace && step < trace_cap) {
      for (int64_t t = 0; t < kmax; ++t) Jout[step * kmax + t] = (t < k) ? perm[ns + t] : -1;
    }

    /* ---- a7: panel with break check (Alg. 4 inner loop) ---- */
    const double eps_s = tau_s * mu;
    rec.eps_s = eps_s;
    int64_t lacc = k;
    for (int64_t l = 0; l < k; ++l) {
      const int64_t col = ns + l;
      int check = (l >= 1) && !no_break && (check_last ? (l < k) : (l + 1 < k));
      if (check) {
        double nrm = sqrt(sumsq(&A_(col, col), m - col));
        if (eps_s > 0.0) {
          double g = fabs(nrm - eps_s) / eps_s;
          double tol = 1e-12 + 2.0 * cerr * OQ_EPS * anorm / eps_s;
          if (g < rec.g_break) rec.g_break = g;
          if (g / tol < rec.s_break) rec.s_break = g / tol;
        }
        if (nrm < eps_s) {
          lacc = l;
          break;
        }
      }
      double beta, ht;
      oq_house(m - col, &A_(col, col), &beta, &ht);
      htau[col] = ht;
      /* apply H = I - ht v v^T to the remaining panel columns */
      for (int64_t j = col + 1; j < ns + k; ++j) {
        double w = A_(col, j);
        for (int64_t i = col + 1; i < m; ++i) w += A_(i, col) * A_(i, j);
        A_(col, j) -= ht * w;
        for (int64_t i = col + 1; i < m; ++i) A_(i, j) -= ht * w * A_(i, col);
      }
    }
    rec.l = lacc;

    /* ---- a8/a9: compact WY and trailing update (Alg. 4) ---- */
    const int64_t mr = m - ns;
    const int64_t j0 = ns + k;
    const int64_t n2 = n - j0;
    if (lacc > 0 && n2 > 0 && mr > 0) {
      oq_larft(mr, lacc, &A_(ns, ns), lda, &htau[ns], T, kmax);
      /* the three loops below treat each trailing column on its own, in the
         same order whether or not the OpenMP build spreads the columns over
         threads, so both builds give identical bits */
      /* W = V^T A22  (lacc x n2) */
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < n2; ++j) {
        const double* a = &A_(ns, j0 + j);
        for (int64_t t = 0; t < lacc; ++t) {
          const double* v = &A_(ns, ns + t);
          double s = a[t]; /* v_t has a unit entry at row t and zeros above */
          for (int64_t i = t + 1; i < mr; ++i) s += v[i] * a[i];
          W[j * kmax + t] = s;
        }
      }
      /* W = T^T W, in place: entry t needs entries q <= t, so t descends */
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < n2; ++j) {
        for (int64_t t = lacc - 1; t >= 0; --t) {
          double s = 0.0;
          for (int64_t q = 0; q <= t; ++q) s += T[t * kmax + q] * W[j * kmax + q];
          W[j * kmax + t] = s;
        }
      }
      /* A22 -= V W */
#pragma omp parallel for schedule(static)
      for (int64_t j = 0; j < n2; ++j) {
        double* a = &A_(ns, j0 + j);
        for (int64_t t = 0; t < lacc; ++t) {
          const double* v = &A_(ns, ns + t);
          double w = W[j * kmax + t];
          a[t] -= w;
          for (int64_t i = t + 1; i < mr; ++i) a[i] -= v[i] * w;
        }
      }
    }

    /* ---- a10: partial norm update (Sec. 3.2 block form, R8/R9/R16) ---- */
    const int64_t nsn = ns + lacc;
    int64_t nrec = 0;
    double s_recomp = rec.s_recomp;
    /* each column on its own; the count and the smallest margin do not
       depend on the order in which columns are visited */
#pragma omp parallel for schedule(static) reduction(+ : nrec) reduction(min : s_recomp)
    for (int64_t j = j0; j < n; ++j) {
      if (u[j] == 0.0) continue;
      double q = 0.0;
      for (int64_t r = ns; r < nsn; ++r) {
        double x = A_(r, j) / u[j];
        q += x * x;
      }
      double t = 1.0 - q;
      if (t < 0.0) t = 0.0;
      double ratio = u[j] / uref[j];
      double test = t * ratio * ratio;
      {
        double g = fabs(test - sqeps) / sqeps;
        /* t is known to about c eps (uref/u)^2 */
        double amp = uref[j] / u[j];
        double tol = 1e-12 + cerr * OQ_EPS * amp * amp / sqeps;
        if (g / tol < s_recomp) s_recomp = g / tol;
      }
      if (test <= sqeps) {
        u[j] = (nsn < m) ? sqrt(sumsq(&A_(nsn, j), m - nsn)) : 0.0;
        uref[j] = u[j];
        ++nrec;
      } else {
        u[j] = u[j] * sqrt(t);
      }
    }
    rec.s_recomp = s_recomp;
    for (int64_t j = nsn; j < j0; ++j) {
      u[j] = (nsn < m) ? sqrt(sumsq(&A_(nsn, j), m - nsn)) : 0.0;
      uref[j] = u[j];
      ++nrec;
    }
    rec.nrecomp = nrec;
    for (int64_t j = ns; j < nsn; ++j) u[j] = 0.0; /* factored columns (eq. after Alg. 3) */

    if (trace && step < trace_cap) trace[step] = rec;
    ++step;
    ns = nsn;
    if (lacc == 0) break; /* cannot happen: l >= 1 always (the first column is never tested) */
  }
  if (*rank_out < 0) *rank_out = (ns >= kmin) ? kmin : ns;
  if (*rank_colmax_out < 0) *rank_colmax_out = (ns >= kmin) ? kmin : ns;
  if (u_out)
    for (int64_t j = 0; j < n; ++j) u_out[j] = u[j];
  if (uref_out)
    for (int64_t j = 0; j < n; ++j) uref_out[j] = uref[j];
  if (nsteps_out) *nsteps_out = step;
  free(u);
  free(uref);
  free(cand);
  free(cols);
  free(Jloc);
  free(selpos);
  free(G);
  free(Th);
  free(T);
  free(W);
  return 0;
}

int64_t oq_step_size(void) { return (int64_t)sizeof(oq_step); }

int oq_qrdm(int64_t m, int64_t n, double* A, int64_t lda, double tau, double delta, int64_t kmax, int64_t eps1_mode,
            int64_t stop_at_rank, int64_t check_last, int64_t no_break, int64_t sdd, int64_t max_steps, double* htau,
            int64_t* perm, int64_t* rank_out, int64_t* rank_colmax_out, double* u_out, double* uref_out,
            oq_step* trace, int64_t trace_cap, int64_t* Jout, int64_t* nsteps_out) {
  return oq_qrdm_sched(m, n, A, lda, tau, delta, kmax, eps1_mode, stop_at_rank, check_last, no_break, sdd, max_steps,
                       htau, perm, rank_out, rank_colmax_out, u_out, uref_out, trace, trace_cap, Jout, nsteps_out,
                       NULL, NULL, 0);
}
