/*
 * lhdm_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * nonnegative least-squares method of "The Lawson-Hanson Algorithm with
 * Deviation Maximization: Finite Convergence and Sparse Recovery"
 * (Dessole, Dell'Orto, Marcuzzi, 2021).
 *
 * TEST INFRASTRUCTURE.  This file is the independent checker of the CUDA
 * path.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path, and the CUDA path never calls it.
 *
 * What it computes (paper section 2):
 *   min ||A x - b||_2  s.t.  x >= 0                    (problem (1))
 * by Algorithm 1 (LH) when k_max == 1 and by Algorithm 3 (LHDM) otherwise,
 * with Algorithm 2 (DM) for the column selection, Algorithm 4 (Updating,
 * Householder) to append columns and Algorithm 5 (Downdating, Givens) to
 * delete them.  The orthogonal transformations are applied to the whole
 * matrix [A | b] (the first of the two variants named at the end of
 * section 4.1), so the working copy W always equals Q^T A Pi and holds R, B
 * and C of section 2.1 explicitly.
 *
 * Readings where the paper is silent or garbled (all shared with the CUDA
 * path; the exact list lives with the project documentation):
 *  - Z_0 = {1..n}; the LH dual update uses the residual r, not b.
 *  - house(): v = x + sign(x_0)||x|| e_0 with sign(0) = +1,
 *    beta = 2 / v^T v, R diagonal = -sign(x_0)||x||.
 *  - stop when Z is empty or max over eligible Z of w <= tol_w,
 *    tol_w = 10 eps max(m,n) max_j ||a_j|| ||b|| unless given.
 *  - argmax ties: lowest column index.
 *  - DM candidates pass BOTH thresholds, maxima over the eligible part of Z,
 *    sorted by w descending (index ascending), first k_max-1 kept, so
 *    |J| <= k_max; cosines of the projected columns C = W[nP:m, .];
 *    greedy acceptance |theta| < delta strictly, in sorted order.
 *  - delta <= tau2/(k_max-1) is not enforced.
 *  - feasibility drop removes the last appended column by re-applying its
 *    reflector (an involution) to the trailing rows.
 *  - inner loop: i* = argmin of alpha (lowest index on exact ties),
 *    x_{i*} := 0 exactly, Q = {i*} U {i in P : x_i <= 0}; positions deleted
 *    together, column-major bottom-up Givens (Algorithm 5).
 *  - columns with trailing norm u_i <= 100 eps ||a_i|| are ineligible for the
 *    step (rank guard, n > m); a J column whose trailing norm falls below the
 *    same bound after the earlier J reflectors ends J there.
 *  - max_outer (default 3n) caps the outer loop.
 *  - positivity trick ([A -A], section 3.2): the twin of a passive column is
 *    not in Z (its projection is zero in exact arithmetic).  Sign flip
 *    (section 4.2): every passive column with y < 0 is replaced by its twin,
 *    whose R column is the negated one (so y changes sign there and nowhere
 *    else) and whose previous iterate is 0 (it was in Z); an exact zero of y
 *    left after the flips goes through the ordinary inner step.
 *
 * Parity: pinned (see the not-gpu tests): KKT, brute-force enumeration,
 * scipy's nnls, closed forms, exact recovery, hand-built DM cases, the
 * tau1 = 1 / tau2 <= 1/2 no-drop theorem, fresh-QR agreement of the
 * updated/downdated R, and the residual identity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG 1
#define ORC_ERR_MAX_ITER 2
#define ORC_ERR_NONFINITE 4
#define ORC_ERR_ALLOC 7

static const double ORC_EPS = 2.220446049250313e-16; /* 2^-52 */

typedef struct {
  double tau1, tau2, delta;
  int k_max;
  double tol_w;   /* < 0: default */
  int max_outer;  /* <= 0: 3n */
  int twin_n;     /* > 0: the matrix is [A  -A] (section 3.2, the positivity
                     trick) with n = 2 twin_n; column j's twin is j +- twin_n */
  int sign_flip;  /* with twin_n: the sign flip of section 4.2 replaces the
                     inner loop's downdate for negative y (Algorithm LH's
                     inner loop otherwise) */
} orc_params;

typedef struct {
  int status, n_outer, n_inner, n_drop, n_passive, rank_limited, n_flip;
  double resid_norm, max_wZ, tol_w;
} orc_info;

/* ------------------------------------------------------------------------ */
/* State of the partial QR factorisation  Q^T [A | b] Pi  (section 2.1).     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, n;
  double* W;      /* m x n, column-major, ld = m: Q^T A (R, B, C blocks)   */
  double* bt;     /* m: Q^T b                                              */
  int nP;         /* |P|                                                   */
  int* order;     /* ordered passive set = QR column order                 */
  int* pos;       /* pos[i] = position of column i in order, or -1 (in Z)  */
  /* reflectors of the current append, kept so a feasibility drop can undo */
  double* hv;     /* m x kcap, reflector t stored in rows [hrow[t], m)     */
  double* hbeta;
  int* hrow;
  int nh, kcap;
} orc_state;

static double col_dot(const double* a, const double* b, int len) {
  double s = 0.0;
  for (int i = 0; i < len; ++i) s += a[i] * b[i];
  return s;
}

static void state_free(orc_state* s) {
  if (!s) return;
  free(s->W); free(s->bt); free(s->order); free(s->pos);
  free(s->hv); free(s->hbeta); free(s->hrow);
  free(s);
}

static orc_state* state_new(int m, int n, const double* A, int lda,
                            const double* b, int kcap) {
  orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->m = m; s->n = n; s->kcap = kcap < 1 ? 1 : kcap;
  s->W = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  s->bt = (double*)malloc(sizeof(double) * (size_t)m);
  s->order = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  s->pos = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  s->hv = (double*)malloc(sizeof(double) * (size_t)m * (size_t)s->kcap);
  s->hbeta = (double*)malloc(sizeof(double) * (size_t)s->kcap);
  s->hrow = (int*)malloc(sizeof(int) * (size_t)s->kcap);
  if (!s->W || !s->bt || !s->order || !s->pos || !s->hv || !s->hbeta || !s->hrow) {
    state_free(s);
    return NULL;
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) s->W[i + (size_t)j * m] = A[i + (size_t)j * lda];
  for (int i = 0; i < m; ++i) s->bt[i] = b[i];
  for (int j = 0; j < n; ++j) { s->order[j] = -1; s->pos[j] = -1; }
  s->nP = 0; s->nh = 0;
  return s;
}

/* H = I - beta v v^T applied to rows [r0, m) of vector y (v indexed from r0). */
static void apply_reflector(double* y, const double* v, double beta, int r0, int m) {
  double d = 0.0;
  for (int i = r0; i < m; ++i) d += v[i - r0] * y[i];
  d *= beta;
  for (int i = r0; i < m; ++i) y[i] -= d * v[i - r0];
}

/*
 * Algorithm 4 (Updating), one column at a time: house() on the trailing part
 * of column c, applied to every column still in Z and to Q^T b.  The new R
 * column is [W(0:nP-1, c); -sign(x_0)||x||].  Returns 0, or 1 if the trailing
 * norm is not above the rank bound (column left untouched).
 */
static int state_append_one(orc_state* s, int c, double rank_bound) {
  const int m = s->m, r0 = s->nP;
  double* x = s->W + (size_t)c * m;
  double alpha = sqrt(col_dot(x + r0, x + r0, m - r0));
  if (!(alpha > rank_bound) || r0 >= m) return 1;
  if (s->nh >= s->kcap) return 1;
  double* v = s->hv + (size_t)s->nh * m;
  const double x0 = x[r0];
  const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
  for (int i = r0; i < m; ++i) v[i - r0] = x[i];
  v[0] = x0 + sg * alpha;
  const double beta = 2.0 / col_dot(v, v, m - r0);
  for (int j = 0; j < s->n; ++j) {
    if (s->pos[j] >= 0 || j == c) continue;
    apply_reflector(s->W + (size_t)j * m, v, beta, r0, m);
  }
  apply_reflector(s->bt, v, beta, r0, m);
  x[r0] = -sg * alpha;
  for (int i = r0 + 1; i < m; ++i) x[i] = 0.0;
  s->hbeta[s->nh] = beta;
  s->hrow[s->nh] = r0;
  s->nh++;
  s->order[s->nP] = c;
  s->pos[c] = s->nP;
  s->nP++;
  return 0;
}

/*
 * Feasibility drop (Algorithm 3, the loop that ensures a feasible descent
 * direction): remove the LAST column of R.  Its reflector is re-applied to
 * the trailing rows of every Z column, of the dropped column and of Q^T b,
 * which restores them (H is an involution).
 */
static void state_drop_last(orc_state* s) {
  const int m = s->m;
  const int c = s->order[s->nP - 1];
  const int t = s->nh - 1;
  const double* v = s->hv + (size_t)t * m;
  const int r0 = s->hrow[t];
  s->nP--;
  s->order[s->nP] = -1;
  s->pos[c] = -1;
  for (int j = 0; j < s->n; ++j) {
    if (s->pos[j] >= 0) continue;
    apply_reflector(s->W + (size_t)j * m, v, s->hbeta[t], r0, m);
  }
  apply_reflector(s->bt, v, s->hbeta[t], r0, m);
  s->nh--;
}

/* Rotation acting on rows (i-1, i) of every column of W and of Q^T b. */
static void rotate_rows(orc_state* s, int i, double cs, double sn) {
  const int m = s->m;
  for (int j = 0; j < s->n; ++j) {
    double* w = s->W + (size_t)j * m;
    const double top = w[i - 1], bot = w[i];
    w[i - 1] = cs * top + sn * bot;
    w[i] = -sn * top + cs * bot;
  }
  const double top = s->bt[i - 1], bot = s->bt[i];
  s->bt[i - 1] = cs * top + sn * bot;
  s->bt[i] = -sn * top + cs * bot;
}

/*
 * Algorithm 5 (Downdating): delete the R columns at the given positions
 * (strictly ascending) and restore triangular form column by column,
 * annihilating each column's subdiagonal entries from the bottom up with
 * Givens rotations on adjacent rows, applied to the whole of W and Q^T b.
 */
static int state_delete(orc_state* s, int nq, const int* qpos) {
  const int m = s->m;
  for (int t = 0; t < nq; ++t) {
    if (qpos[t] < 0 || qpos[t] >= s->nP) return ORC_ERR_INVALID_ARG;
    if (t > 0 && qpos[t] <= qpos[t - 1]) return ORC_ERR_INVALID_ARG;
  }
  if (nq == 0) return ORC_OK;
  int* keep_old = (int*)malloc(sizeof(int) * (size_t)s->nP);
  if (!keep_old) return ORC_ERR_ALLOC;
  int nk = 0, t = 0;
  for (int p = 0; p < s->nP; ++p) {
    if (t < nq && qpos[t] == p) {
      s->pos[s->order[p]] = -1;
      ++t;
      continue;
    }
    keep_old[nk++] = p;
  }
  int* new_order = (int*)malloc(sizeof(int) * (size_t)(nk > 0 ? nk : 1));
  if (!new_order) { free(keep_old); return ORC_ERR_ALLOC; }
  for (int c = 0; c < nk; ++c) new_order[c] = s->order[keep_old[c]];
  for (int c = 0; c < nk; ++c) {
    double* col = s->W + (size_t)new_order[c] * m;
    for (int i = keep_old[c]; i > c; --i) {
      const double a = col[i - 1], bb = col[i];
      const double r = sqrt(a * a + bb * bb);
      double cs = 1.0, sn = 0.0;
      if (r != 0.0) { cs = a / r; sn = bb / r; }
      rotate_rows(s, i, cs, sn);
      col[i - 1] = r;
      col[i] = 0.0;
    }
  }
  for (int p = 0; p < s->nP; ++p) s->order[p] = -1;
  for (int c = 0; c < nk; ++c) { s->order[c] = new_order[c]; s->pos[new_order[c]] = c; }
  s->nP = nk;
  free(keep_old); free(new_order);
  return ORC_OK;
}

/* Back substitution R y_P = (Q^T b)_{1:nP}; y in column-index space, y_Z = 0. */
static void state_solve(const orc_state* s, double* y) {
  const int m = s->m;
  for (int j = 0; j < s->n; ++j) y[j] = 0.0;
  for (int k = s->nP - 1; k >= 0; --k) {
    double acc = s->bt[k];
    for (int l = k + 1; l < s->nP; ++l) acc -= s->W[k + (size_t)s->order[l] * m] * y[s->order[l]];
    y[s->order[k]] = acc / s->W[k + (size_t)s->order[k] * m];
  }
}

/*
 * Sign flip (section 4.2) at position p of the positivity-trick matrix
 * [A -A]: column k = order[p] is replaced by its twin kb, whose R column is
 * the negated R column of k (Q is unchanged, since Q^T(-a_k) = -Q^T a_k);
 * k returns to Z with W(:, k) = Q^T a_k = [R column; 0], as held.
 */
static void state_flip(orc_state* s, int p, int twin_n) {
  const int m = s->m;
  const int k = s->order[p];
  const int kb = k < twin_n ? k + twin_n : k - twin_n;
  const double* wk = s->W + (size_t)k * m;
  double* wb = s->W + (size_t)kb * m;
  for (int i = 0; i < m; ++i) wb[i] = (i < s->nP) ? -wk[i] : 0.0;
  s->order[p] = kb;
  s->pos[kb] = p;
  s->pos[k] = -1;
}

/*
 * Algorithm 2 (Deviation Maximization) on the columns cols[0..ncols) of a
 * column-major matrix C (ld ldc), using rows [row0, row0+L).  w and u are
 * indexed by the entries of cols.  Writes the ordered J (entries of cols)
 * and returns |J| (0 when no column is given).
 */
static int dm_select_core(int L, int row0, int ncols, const int* cols,
                          const double* C, int ldc, const double* w,
                          const double* u, double tau1, double tau2,
                          double delta, int k_max, int* J) {
  if (ncols <= 0 || k_max < 1) return 0;
  /* j in argmax u_1 (lowest index on ties) */
  int j = -1;
  double wmax = 0.0, umax = 0.0;
  for (int t = 0; t < ncols; ++t) {
    const int c = cols[t];
    if (j < 0 || w[c] > wmax || (w[c] == wmax && c < j)) { j = c; wmax = w[c]; }
    if (t == 0 || u[c] > umax) umax = u[c];
  }
  J[0] = j;
  if (k_max == 1) return 1;
  /* candidate set I: both thresholds (l = 1: w, l = 2: u), i != j */
  int* I = (int*)malloc(sizeof(int) * (size_t)ncols);
  if (!I) return 1;
  int nI = 0;
  for (int t = 0; t < ncols; ++t) {
    const int c = cols[t];
    if (c == j) continue;
    if (w[c] >= tau1 * wmax && u[c] >= tau2 * umax) I[nI++] = c;
  }
  /* order by w descending, index ascending (insertion sort, plain) */
  for (int a = 1; a < nI; ++a) {
    const int c = I[a];
    int b = a - 1;
    while (b >= 0 && (w[I[b]] < w[c] || (w[I[b]] == w[c] && I[b] > c))) {
      I[b + 1] = I[b];
      --b;
    }
    I[b + 1] = c;
  }
  if (nI > k_max - 1) nI = k_max - 1;
  /* cosine matrix of the columns {j} U I (section 2.2, Theta = D^-1 C^T C D^-1) */
  const int K = nI + 1;
  int* Kc = (int*)malloc(sizeof(int) * (size_t)K);
  double* G = (double*)malloc(sizeof(double) * (size_t)K * (size_t)K);
  double* d = (double*)malloc(sizeof(double) * (size_t)K);
  if (!Kc || !G || !d) { free(I); free(Kc); free(G); free(d); return 1; }
  Kc[0] = j;
  for (int a = 0; a < nI; ++a) Kc[a + 1] = I[a];
  for (int a = 0; a < K; ++a)
    for (int b = 0; b < K; ++b)
      G[a + (size_t)b * K] = col_dot(C + (size_t)Kc[a] * ldc + row0, C + (size_t)Kc[b] * ldc + row0, L);
  for (int a = 0; a < K; ++a) d[a] = sqrt(G[a + (size_t)a * K]);
  /* greedy: accept candidate a when |theta(a, l)| < delta for every l in J */
  int nJ = 1;
  int* Jpos = (int*)malloc(sizeof(int) * (size_t)K);
  if (!Jpos) { free(I); free(Kc); free(G); free(d); return 1; }
  Jpos[0] = 0;
  for (int a = 1; a < K; ++a) {
    int ok = 1;
    for (int t = 0; t < nJ; ++t) {
      const int l = Jpos[t];
      const double theta = G[a + (size_t)l * K] / (d[a] * d[l]);
      if (!(fabs(theta) < delta)) { ok = 0; break; }
    }
    if (ok) { Jpos[nJ] = a; J[nJ] = Kc[a]; ++nJ; }
  }
  free(I); free(Kc); free(G); free(d); free(Jpos);
  return nJ;
}

/* With the positivity trick, is column j's twin passive? */
static int twin_passive(const orc_state* s, int j, int twin_n) {
  if (twin_n <= 0) return 0;
  const int jb = j < twin_n ? j + twin_n : j - twin_n;
  return s->pos[jb] >= 0;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                    */
/* ------------------------------------------------------------------------ */

/* Algorithm 2 alone, on an explicit matrix C (L x ncols, ld ldc); every column
 * is a candidate.  Returns |J|; J receives column indices of C. */
int orc_dm_select(int L, int ncols, const double* C, int ldc, const double* w,
                  const double* u, double tau1, double tau2, double delta,
                  int k_max, int* J) {
  if (L < 0 || ncols < 0 || ldc < L || k_max < 1) return -1;
  int* cols = (int*)malloc(sizeof(int) * (size_t)(ncols > 0 ? ncols : 1));
  if (!cols) return -1;
  for (int t = 0; t < ncols; ++t) cols[t] = t;
  const int r = dm_select_core(L, 0, ncols, cols, C, ldc, w, u, tau1, tau2, delta, k_max, J);
  free(cols);
  return r;
}

/* QR-modification primitives exposed for the update/downdate tests. */
void* orc_state_new(int m, int n, const double* A, int lda, const double* b, int kcap) {
  if (m < 1 || n < 1 || lda < m) return NULL;
  return state_new(m, n, A, lda, b, kcap);
}
void orc_state_free(void* s) { state_free((orc_state*)s); }
/* Appends the columns in order (Algorithm 4); returns how many were appended. */
int orc_state_append(void* sv, int k, const int* cols) {
  orc_state* s = (orc_state*)sv;
  s->nh = 0;
  int done = 0;
  for (int t = 0; t < k; ++t) {
    if (cols[t] < 0 || cols[t] >= s->n || s->pos[cols[t]] >= 0) break;
    if (state_append_one(s, cols[t], 0.0)) break;
    ++done;
  }
  return done;
}
int orc_state_drop_last(void* sv) {
  orc_state* s = (orc_state*)sv;
  if (s->nP < 1 || s->nh < 1) return ORC_ERR_INVALID_ARG;
  state_drop_last(s);
  return ORC_OK;
}
int orc_state_delete(void* sv, int nq, const int* qpos) {
  return state_delete((orc_state*)sv, nq, qpos);
}
/* nP, order[nP], R (nP x nP col-major, ld nP), bt[m], W[m x n] (any may be NULL) */
int orc_state_get(void* sv, int* nP, int* order, double* R, double* bt, double* W) {
  orc_state* s = (orc_state*)sv;
  const int m = s->m;
  if (nP) *nP = s->nP;
  if (order) for (int k = 0; k < s->nP; ++k) order[k] = s->order[k];
  if (R)
    for (int k = 0; k < s->nP; ++k)
      for (int i = 0; i < s->nP; ++i)
        R[i + (size_t)k * s->nP] = (i <= k) ? s->W[i + (size_t)s->order[k] * m] : 0.0;
  if (bt) for (int i = 0; i < m; ++i) bt[i] = s->bt[i];
  if (W) memcpy(W, s->W, sizeof(double) * (size_t)m * (size_t)s->n);
  return ORC_OK;
}

/*
 * The solver: Algorithm 3 (LHDM); k_max == 1 gives Algorithm 1 (LH), since
 * DM then returns J = {argmax w}.
 *
 * x[n]          out: solution.
 * p_order[n]    out: ordered passive set (QR column order), -1 padded.
 * info          out.
 * trace         optional (trace_cap rows): per outer step
 *               trace_i[6*s + 0..5] = |J| from DM, |J| kept, inner steps,
 *               nP after the step, columns removed by the inner loop, and
 *               the column j chosen first (the LH argmax);
 *               trace_d[2*s] = ||b - A x|| after the step, trace_d[2*s+1] =
 *               the step's decision margin: the smallest relative distance
 *               of a comparison from flipping (gap between the two largest
 *               eligible w, and |y_i| / max|y|, |x_i| / max|x| over every
 *               sign test of the feasibility and inner loops).
 * R_out         optional: final R (nP x nP, col-major, ld nP), in p_order.
 * Returns info->status.
 */
int orc_nnls(int m, int n, const double* A, int lda, const double* b,
             const orc_params* prm, double* x, int* p_order, orc_info* info,
             int trace_cap, int* trace_i, double* trace_d, double* R_out) {
  orc_info inf;
  memset(&inf, 0, sizeof(inf));
  if (m < 0 || n < 0 || lda < (m > 1 ? m : 1) || !prm || prm->k_max < 1 ||
      (n > 0 && (!x || !p_order)) || (m > 0 && !b) || (m > 0 && n > 0 && !A)) {
    inf.status = ORC_ERR_INVALID_ARG;
    if (info) *info = inf;
    return inf.status;
  }
  if (m == 0 || n == 0) {
    /* empty problem: x = 0 is optimal (every w_i is zero) */
    for (int j = 0; j < n; ++j) { x[j] = 0.0; p_order[j] = -1; }
    if (m > 0) inf.resid_norm = sqrt(col_dot(b, b, m));
    inf.max_wZ = n > 0 ? 0.0 : -INFINITY;
    if (info) *info = inf;
    return inf.status;
  }
  for (int j = 0; j < n; ++j) { x[j] = 0.0; p_order[j] = -1; }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i)
      if (!isfinite(A[i + (size_t)j * lda])) inf.status = ORC_ERR_NONFINITE;
  for (int i = 0; i < m; ++i)
    if (!isfinite(b[i])) inf.status = ORC_ERR_NONFINITE;
  if (inf.status) { if (info) *info = inf; return inf.status; }

  const int k_max = prm->k_max;
  const int twin_n = prm->twin_n;
  if (twin_n < 0 || (twin_n > 0 && n != 2 * twin_n)) {
    inf.status = ORC_ERR_INVALID_ARG;
    if (info) *info = inf;
    return inf.status;
  }
  orc_state* s = state_new(m, n, A, lda, b, k_max);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* u = (double*)malloc(sizeof(double) * (size_t)n);
  double* anorm = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)m);
  int* J = (int*)malloc(sizeof(int) * (size_t)k_max);
  int* elig = (int*)malloc(sizeof(int) * (size_t)n);
  int* qpos = (int*)malloc(sizeof(int) * (size_t)n);
  if (!s || !w || !u || !anorm || !y || !r || !J || !elig || !qpos) {
    state_free(s); free(w); free(u); free(anorm); free(y); free(r); free(J); free(elig); free(qpos);
    inf.status = ORC_ERR_ALLOC;
    if (info) *info = inf;
    return inf.status;
  }

  /* Setup (Algorithm 3, first lines): x = 0, w = A^T b, u = column norms. */
  double amax = 0.0, bnorm = sqrt(col_dot(b, b, m));
  for (int j = 0; j < n; ++j) {
    const double* a = A + (size_t)j * lda;
    anorm[j] = sqrt(col_dot(a, a, m));
    u[j] = anorm[j];
    w[j] = col_dot(a, b, m);
    if (anorm[j] > amax) amax = anorm[j];
  }
  const double tol_w = (prm->tol_w >= 0.0)
                           ? prm->tol_w
                           : 10.0 * ORC_EPS * (double)(m > n ? m : n) * amax * bnorm;
  const int max_outer = prm->max_outer > 0 ? prm->max_outer : 3 * n;
  inf.tol_w = tol_w;
  for (int i = 0; i < m; ++i) r[i] = b[i];

  for (;;) {
    /* outer-loop test over the eligible part of Z */
    int ne = 0;
    double wz_any = -INFINITY;
    for (int j = 0; j < n; ++j) {
      if (s->pos[j] >= 0 || twin_passive(s, j, twin_n)) continue;
      if (w[j] > wz_any) wz_any = w[j];
      if (u[j] > 100.0 * ORC_EPS * anorm[j]) elig[ne++] = j;
    }
    double wz_elig = -INFINITY;
    for (int t = 0; t < ne; ++t) if (w[elig[t]] > wz_elig) wz_elig = w[elig[t]];
    if (ne == 0 || !(wz_elig > tol_w)) {
      if (wz_any > tol_w) inf.rank_limited = 1;
      break;
    }
    if (inf.n_outer >= max_outer) { inf.status = ORC_ERR_MAX_ITER; break; }

    /* decision margin of this step (relative distance of the closest
       comparison to flipping): argmax gap and every y / x sign test */
    double margin = INFINITY;
    {
      double w1 = -INFINITY, w2 = -INFINITY;
      for (int t = 0; t < ne; ++t) {
        const double wv = w[elig[t]];
        if (wv > w1) { w2 = w1; w1 = wv; } else if (wv > w2) w2 = wv;
      }
      if (ne > 1 && w1 > 0.0) margin = (w1 - w2) / w1;
    }
    /* DM on C^(s) = trailing rows of the Z columns */
    const int L = m - s->nP;
    const int kdm = dm_select_core(L, s->nP, ne, elig, s->W, m, w, u, prm->tau1,
                                   prm->tau2, prm->delta, k_max, J);
    /* rank-k update (Algorithm 4), column by column in J order */
    s->nh = 0;
    int kk = 0;
    for (int t = 0; t < kdm; ++t) {
      if (state_append_one(s, J[t], 100.0 * ORC_EPS * anorm[J[t]])) break;
      ++kk;
    }
    if (kk == 0) { inf.rank_limited = 1; break; }
    state_solve(s, y);
    /* feasibility loop: while min y_J <= 0, delete the last element of J */
    int drops = 0;
    for (;;) {
      double ymin = INFINITY, ymax = 0.0;
      for (int t = 0; t < kk; ++t) if (y[J[t]] < ymin) ymin = y[J[t]];
      for (int p = 0; p < s->nP; ++p) ymax = fmax(ymax, fabs(y[s->order[p]]));
      for (int t = 0; t < kk; ++t)
        if (ymax > 0.0) margin = fmin(margin, fabs(y[J[t]]) / ymax);
      if (!(ymin <= 0.0) || kk <= 1) break;
      state_drop_last(s);
      --kk;
      ++drops;
      state_solve(s, y);
    }
    inf.n_drop += drops;
    /* sign flip (positivity trick, section 4.2): a passive column with
       y < 0 gives way to its twin; y keeps its values up to that sign */
    if (twin_n > 0 && prm->sign_flip) {
      int flips = 0;
      for (int p = 0; p < s->nP; ++p) {
        const int k = s->order[p];
        if (y[k] < 0.0) {
          const int kb = k < twin_n ? k + twin_n : k - twin_n;
          state_flip(s, p, twin_n);
          x[kb] = 0.0;  /* the twin was in Z: its previous iterate is 0 */
          x[k] = 0.0;
          ++flips;
        }
      }
      if (flips) state_solve(s, y);
      inf.n_flip += flips;
    }
    /* inner loop */
    int inner = 0, removed = 0;
    for (;;) {
      int neg = 0;
      double ymax = 0.0;
      for (int p = 0; p < s->nP; ++p) ymax = fmax(ymax, fabs(y[s->order[p]]));
      for (int p = 0; p < s->nP; ++p) {
        if (ymax > 0.0) margin = fmin(margin, fabs(y[s->order[p]]) / ymax);
        if (y[s->order[p]] <= 0.0) neg = 1;
      }
      if (!neg) break;
      if (inner > n) { inf.status = ORC_ERR_MAX_ITER; break; }
      ++inner;
      double alpha = INFINITY;
      int istar = -1;
      for (int p = 0; p < s->nP; ++p) {
        const int i = s->order[p];
        if (y[i] <= 0.0) {
          const double t = x[i] / (x[i] - y[i]);
          if (t < alpha || (t == alpha && i < istar)) { alpha = t; istar = i; }
        }
      }
      for (int p = 0; p < s->nP; ++p) {
        const int i = s->order[p];
        x[i] = x[i] + alpha * (y[i] - x[i]);
      }
      x[istar] = 0.0;
      {
        double xmax = 0.0;
        for (int p = 0; p < s->nP; ++p) xmax = fmax(xmax, fabs(x[s->order[p]]));
        for (int p = 0; p < s->nP; ++p)
          if (s->order[p] != istar && xmax > 0.0) margin = fmin(margin, fabs(x[s->order[p]]) / xmax);
      }
      int nq = 0;
      for (int p = 0; p < s->nP; ++p)
        if (x[s->order[p]] <= 0.0) { qpos[nq++] = p; x[s->order[p]] = 0.0; }
      removed += nq;
      if (state_delete(s, nq, qpos) != ORC_OK) { inf.status = ORC_ERR_INVALID_ARG; break; }
      state_solve(s, y);
    }
    inf.n_inner += inner;
    if (inf.status) break;
    /* x = y;  w = A^T (b - A x);  u = column norms of C */
    for (int j = 0; j < n; ++j) x[j] = (s->pos[j] >= 0) ? y[j] : 0.0;
    for (int i = 0; i < m; ++i) r[i] = b[i];
    for (int p = 0; p < s->nP; ++p) {
      const int c = s->order[p];
      const double* a = A + (size_t)c * lda;
      for (int i = 0; i < m; ++i) r[i] -= a[i] * x[c];
    }
    for (int j = 0; j < n; ++j) {
      if (s->pos[j] >= 0) { w[j] = 0.0; u[j] = 0.0; continue; }
      w[j] = col_dot(A + (size_t)j * lda, r, m);
      const double* cj = s->W + (size_t)j * m + s->nP;
      u[j] = sqrt(col_dot(cj, cj, m - s->nP));
    }
    if (trace_i && inf.n_outer < trace_cap) {
      trace_i[6 * inf.n_outer + 0] = kdm;
      trace_i[6 * inf.n_outer + 1] = kk;
      trace_i[6 * inf.n_outer + 2] = inner;
      trace_i[6 * inf.n_outer + 3] = s->nP;
      trace_i[6 * inf.n_outer + 4] = removed;
      trace_i[6 * inf.n_outer + 5] = J[0];
      if (trace_d) {
        trace_d[2 * inf.n_outer] = sqrt(col_dot(r, r, m));
        trace_d[2 * inf.n_outer + 1] = margin;
      }
    }
    inf.n_outer++;
  }

  /* outputs */
  for (int j = 0; j < n; ++j) if (s->pos[j] < 0) x[j] = 0.0;
  for (int p = 0; p < s->nP; ++p) p_order[p] = s->order[p];
  for (int i = 0; i < m; ++i) r[i] = b[i];
  for (int j = 0; j < n; ++j) {
    if (x[j] == 0.0) continue;
    const double* a = A + (size_t)j * lda;
    for (int i = 0; i < m; ++i) r[i] -= a[i] * x[j];
  }
  inf.resid_norm = sqrt(col_dot(r, r, m));
  inf.max_wZ = -INFINITY;
  for (int j = 0; j < n; ++j)
    if (s->pos[j] < 0 && !twin_passive(s, j, twin_n)) {
      const double wj = col_dot(A + (size_t)j * lda, r, m);
      if (wj > inf.max_wZ) inf.max_wZ = wj;
    }
  inf.n_passive = s->nP;
  if (R_out)
    for (int k = 0; k < s->nP; ++k)
      for (int i = 0; i < s->nP; ++i)
        R_out[i + (size_t)k * s->nP] = (i <= k) ? s->W[i + (size_t)s->order[k] * m] : 0.0;

  state_free(s); free(w); free(u); free(anorm); free(y); free(r); free(J); free(elig); free(qpos);
  if (info) *info = inf;
  return inf.status;
}
