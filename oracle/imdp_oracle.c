/*
 * Plain CPU FP64 oracle for robust value iteration on Interval Markov Decision
 * Processes (IMDPs), written from arXiv 2401.04068 (IntervalMDP.jl).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this code. The CUDA library never calls
 * it, and the two share no code.
 *
 * What it computes, in the paper's order and notation:
 *   - IMDP M = (S, A, P_up, P_lo) with per-(s,a,s') interval bounds; a column
 *     (s,a) is feasible iff sum P_lo <= 1 <= sum P_up and P_lo <= P_up
 *     (Sec. 2, definition of an IMDP and of Gamma_{s,a}).
 *   - Value iteration, Eq. 2:  V_0 = 1_G,
 *       V_k(s) = 1_G(s) + 1_{S\G}(s) opt^pi_a opt^eta_{p in Gamma_{s,a}} sum_s' V_{k-1}(s') p(s').
 *   - The inner problem of Eq. 3 by O-maximization (Sec. 4): order the
 *     destinations by V (ascending for a pessimistic adversary, i.e. give the
 *     least mass to high values; descending for an optimistic one), start from
 *     p = lower, rem = 1 - sum(lower), and walk the ordering giving each state
 *     its full gap (upper - lower) until rem is used up (the sequential
 *     procedure of Sec. 4).
 *   - Returns (V, k, residual) as value_iteration does (Sec. 3.2), and the
 *     control-synthesis policy (Sec. 3.2): an |S| x K time-dependent matrix for
 *     a finite horizon, a stationary |S| vector for an infinite one.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - ties in V are ordered by state index (stable); the value is invariant.
 *   - the first (lowest local index) action attaining the optimum is the policy.
 *   - policy column t (time t from the start) is the argmax of iteration K - t.
 *   - reward: V_0 = r, V_k = r + gamma * opt opt sum V_{k-1} p (Sec. 3.2 says it
 *     "follows similarly"; the recursion is not printed).
 *   - reach-avoid (only in the JSON schema of Appendix A): avoid states fixed
 *     at 0, reach states fixed at 1.
 *   - infinite horizon stops after the first iteration with max|V_k - V_{k-1}| < eps.
 *   - rem = 1 - sum(lower) is summed sequentially in storage order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_EINFEASIBLE = 2, OR_ENOMEM = 3, OR_ENOCONV = 4 };
enum { OR_REACH = 0, OR_REACH_AVOID = 1, OR_REWARD = 2 };

typedef struct {
  int32_t n_states;
  int32_t n_cols;
  const int32_t* stateptr; /* n_states + 1: columns of state s are [stateptr[s], stateptr[s+1]) */
  const int32_t* colptr;   /* n_cols + 1: entries of column j are [colptr[j], colptr[j+1]) */
  const int32_t* rowval;   /* destination state of each entry, strictly increasing per column */
  const double* lower;     /* P_lo per entry */
  const double* upper;     /* P_up per entry */
} oracle_imdp;

typedef struct {
  int32_t property;      /* OR_REACH, OR_REACH_AVOID, OR_REWARD */
  int32_t infinite_time; /* 0: fixed horizon; 1: until max|residual| < eps */
  int32_t horizon;       /* K for a finite horizon; iteration cap for an infinite one */
  double eps;
  int32_t pessimistic;   /* opt^eta = min when 1, max when 0 */
  int32_t maximize;      /* opt^pi = max when 1, min when 0 */
  const int32_t* reach;  int32_t n_reach;
  const int32_t* avoid;  int32_t n_avoid;
  const double* reward;  /* n_states, OR_REWARD only */
  double discount;       /* OR_REWARD only */
} oracle_spec;

/* Feasibility of every column (Sec. 2) and structural sanity of the CSC arrays
 * (Sec. 3.1 and Appendix A: stateptr maps states to column ranges). */
int oracle_validate(const oracle_imdp* m, double tol) {
  if (!m || m->n_states <= 0 || m->n_cols < m->n_states) return OR_EINVAL;
  if (m->stateptr[0] != 0 || m->stateptr[m->n_states] != m->n_cols) return OR_EINVAL;
  for (int32_t s = 0; s < m->n_states; ++s)
    if (m->stateptr[s + 1] <= m->stateptr[s]) return OR_EINVAL; /* every state has an action */
  if (m->colptr[0] != 0) return OR_EINVAL;
  for (int32_t j = 0; j < m->n_cols; ++j) {
    int32_t a = m->colptr[j], b = m->colptr[j + 1];
    if (b < a) return OR_EINVAL;
    double slo = 0.0, sup = 0.0;
    for (int32_t i = a; i < b; ++i) {
      if (m->rowval[i] < 0 || m->rowval[i] >= m->n_states) return OR_EINVAL;
      if (i > a && m->rowval[i] <= m->rowval[i - 1]) return OR_EINVAL;
      double lo = m->lower[i], up = m->upper[i];
      if (!(lo >= 0.0) || !(up <= 1.0) || !(lo <= up)) return OR_EINFEASIBLE;
      slo += lo;
      sup += up;
    }
    if (slo > 1.0 + tol || sup < 1.0 - tol) return OR_EINFEASIBLE;
  }
  return OR_OK;
}

typedef struct { double v; int32_t state; int32_t local; } ord_item;

static int cmp_ascending(const void* x, const void* y) {
  const ord_item* a = (const ord_item*)x; const ord_item* b = (const ord_item*)y;
  if (a->v < b->v) return -1;
  if (a->v > b->v) return 1;
  return (a->state > b->state) - (a->state < b->state);
}
static int cmp_descending(const void* x, const void* y) {
  const ord_item* a = (const ord_item*)x; const ord_item* b = (const ord_item*)y;
  if (a->v > b->v) return -1;
  if (a->v < b->v) return 1;
  return (a->state > b->state) - (a->state < b->state);
}

/* O-maximization for one column (Sec. 4, sequential procedure). The ordering
 * phase sorts the destinations by V; the assignment phase starts from the lower
 * bounds and hands out the remaining mass gap by gap along the ordering.
 * Writes p (length k) and returns sum_i V[row_i] p_i. */
double oracle_omax_column(int32_t k, const int32_t* rows, const double* lo, const double* up,
                          const double* V, int32_t pessimistic, ord_item* scratch, double* p) {
  double rem = 1.0;
  for (int32_t i = 0; i < k; ++i) { p[i] = lo[i]; rem -= lo[i]; }
  for (int32_t i = 0; i < k; ++i) { scratch[i].v = V[rows[i]]; scratch[i].state = rows[i]; scratch[i].local = i; }
  qsort(scratch, (size_t)k, sizeof(ord_item), pessimistic ? cmp_ascending : cmp_descending);
  for (int32_t t = 0; t < k; ++t) {
    int32_t o = scratch[t].local;
    double gap = up[o] - lo[o];
    if (gap < rem) {
      p[o] += gap;
      rem -= gap;
    } else {
      p[o] += rem;
      break;
    }
  }
  double q = 0.0;
  for (int32_t i = 0; i < k; ++i) q += V[rows[i]] * p[i];
  return q;
}

/* Python-facing helper: O-maximization of one column with caller-provided V
 * over the column's own entries (V_local[i] is the value of destination i). */
double oracle_omax_local(int32_t k, const double* v_local, const double* lo, const double* up,
                         int32_t pessimistic, double* p) {
  int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
  ord_item* scratch = (ord_item*)malloc(sizeof(ord_item) * (size_t)(k > 0 ? k : 1));
  if (!rows || !scratch) { free(rows); free(scratch); return NAN; }
  for (int32_t i = 0; i < k; ++i) rows[i] = i;
  double q = oracle_omax_column(k, rows, lo, up, v_local, pessimistic, scratch, p);
  free(rows); free(scratch);
  return q;
}

/* One Bellman update (Eq. 2 / Eq. 3) for all states. Returns max |V_new - V_old|.
 * best_action (nullable) receives the local index of the chosen action, -1 for
 * states held fixed (reach or avoid targets). */
static double bellman_sweep(const oracle_imdp* m, const oracle_spec* sp, const uint8_t* fixed,
                            const double* fixed_val, const double* Vold, double* Vnew,
                            int32_t* best_action, int32_t n_threads) {
  double maxres = 0.0;
  int32_t kmax = 0;
  for (int32_t j = 0; j < m->n_cols; ++j) {
    int32_t k = m->colptr[j + 1] - m->colptr[j];
    if (k > kmax) kmax = k;
  }
  (void)n_threads;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads > 0 ? n_threads : 1) reduction(max : maxres)
#endif
  {
    ord_item* scratch = (ord_item*)malloc(sizeof(ord_item) * (size_t)(kmax > 0 ? kmax : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(kmax > 0 ? kmax : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (int32_t s = 0; s < m->n_states; ++s) {
      double v;
      int32_t best = -1;
      if (fixed[s]) {
        v = fixed_val[s];
      } else {
        double opt = 0.0;
        for (int32_t j = m->stateptr[s]; j < m->stateptr[s + 1]; ++j) {
          int32_t a = m->colptr[j], k = m->colptr[j + 1] - a;
          double q = oracle_omax_column(k, m->rowval + a, m->lower + a, m->upper + a, Vold,
                                        sp->pessimistic, scratch, p);
          int better = (best < 0) || (sp->maximize ? (q > opt) : (q < opt));
          if (better) { opt = q; best = j - m->stateptr[s]; }
        }
        v = (sp->property == OR_REWARD) ? sp->reward[s] + sp->discount * opt : opt;
      }
      Vnew[s] = v;
      if (best_action) best_action[s] = best;
      double r = fabs(v - Vold[s]);
      if (r > maxres) maxres = r;
    }
    free(scratch);
    free(p);
  }
  return maxres;
}

/* value_iteration (Sec. 3.2) with optional control synthesis.
 *   V_out        n_states: V_k after the last iteration
 *   k_out        iterations performed
 *   residual_out n_states (nullable): V_k - V_{k-1} of the last iteration (zeros if k = 0)
 *   policy_out   (nullable) finite horizon: K x n_states, entry [t*n + s] = action at time t
 *                (argmax of iteration K - t); infinite horizon: n_states (last iteration).
 */
int oracle_value_iteration(const oracle_imdp* m, const oracle_spec* sp, double* V_out, int32_t* k_out,
                           double* residual_out, int32_t* policy_out, int32_t n_threads) {
  if (!m || !sp || !V_out) return OR_EINVAL;
  int32_t n = m->n_states;
  if (sp->horizon < 0) return OR_EINVAL;
  if (sp->infinite_time && !(sp->eps > 0.0)) return OR_EINVAL;
  /* discount in (0, 1] for a finite horizon, (0, 1) for an infinite one (Sec. 3.2) */
  if (sp->property == OR_REWARD &&
      (!sp->reward || !(sp->discount > 0.0) || !(sp->discount <= 1.0) ||
       (sp->infinite_time && !(sp->discount < 1.0))))
    return OR_EINVAL;
  uint8_t* fixed = (uint8_t*)calloc((size_t)n, 1);
  double* fixed_val = (double*)calloc((size_t)n, sizeof(double));
  double* Va = (double*)malloc(sizeof(double) * (size_t)n);
  double* Vb = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* act = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!fixed || !fixed_val || !Va || !Vb || !act) {
    free(fixed); free(fixed_val); free(Va); free(Vb); free(act);
    return OR_ENOMEM;
  }
  int status = OR_OK;
  if (sp->property == OR_REACH || sp->property == OR_REACH_AVOID) {
    for (int32_t i = 0; i < sp->n_reach; ++i) {
      int32_t s = sp->reach[i];
      if (s < 0 || s >= n) { status = OR_EINVAL; goto done; }
      fixed[s] = 1; fixed_val[s] = 1.0;
    }
    if (sp->property == OR_REACH_AVOID) {
      for (int32_t i = 0; i < sp->n_avoid; ++i) {
        int32_t s = sp->avoid[i];
        if (s < 0 || s >= n) { status = OR_EINVAL; goto done; }
        if (fixed[s] == 1) { status = OR_EINVAL; goto done; } /* in both sets */
        fixed[s] = 2; fixed_val[s] = 0.0;
      }
    }
    for (int32_t s = 0; s < n; ++s) Va[s] = fixed_val[s]; /* V_0 = 1_G */
  } else if (sp->property == OR_REWARD) {
    for (int32_t s = 0; s < n; ++s) Va[s] = sp->reward[s]; /* V_0 = r */
  } else {
    status = OR_EINVAL;
    goto done;
  }

  {
    int32_t K = sp->horizon;
    int32_t k = 0;
    double* Vold = Va;
    double* Vnew = Vb;
    if (!sp->infinite_time) {
      for (k = 1; k <= K; ++k) {
        bellman_sweep(m, sp, fixed, fixed_val, Vold, Vnew, act, n_threads);
        if (policy_out) {
          int32_t t = K - k;
          for (int32_t s = 0; s < n; ++s) policy_out[(size_t)t * n + s] = act[s];
        }
        double* tmp = Vold; Vold = Vnew; Vnew = tmp;
      }
      k = K;
    } else {
      int32_t cap = K > 0 ? K : 1000000;
      int converged = 0;
      for (k = 1; k <= cap; ++k) {
        double r = bellman_sweep(m, sp, fixed, fixed_val, Vold, Vnew, act, n_threads);
        double* tmp = Vold; Vold = Vnew; Vnew = tmp;
        if (r < sp->eps) { converged = 1; break; }
      }
      if (!converged) { k = cap; status = OR_ENOCONV; }
      if (policy_out) for (int32_t s = 0; s < n; ++s) policy_out[s] = act[s];
    }
    /* Vold holds V_k, Vnew holds V_{k-1} (when k >= 1). */
    for (int32_t s = 0; s < n; ++s) V_out[s] = Vold[s];
    if (residual_out)
      for (int32_t s = 0; s < n; ++s) residual_out[s] = (k >= 1) ? Vold[s] - Vnew[s] : 0.0;
    if (k_out) *k_out = k;
  }
done:
  free(fixed); free(fixed_val); free(Va); free(Vb); free(act);
  return status;
}

int oracle_has_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}
