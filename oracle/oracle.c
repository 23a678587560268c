/*
 * CPU FP64 ORACLE for AMGF-PCG (algebraic multigrid with filtering).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code
 * with the GPU library (paper_2505_18576_gb300/csrc) and includes none of its
 * headers; both only read the same seeded inputs from contactgen.
 *
 * What it computes, step by step, in plain loops (double precision):
 *   - the condensed IP-Newton matrix  A = K + J^T D J            (Section 3, eq. linsystem1)
 *   - the contact index set I_c = nonzero columns of J           (Section 4; Section 5.1 def. of I_c)
 *   - B := AMG(A): classical Ruge-Stueben AMG, unknown approach  (Remark "upper_bound_estimate";
 *     BoomerAMG in Section 6), with l1-Jacobi smoothing            (the l1 smoothers cited there)
 *   - the filter matrix A_w = P^T A P = A[I_c, I_c]               (Section 5.1, discrete operators)
 *   - AMGF:  I - M A = (I - B A)(I - P A_w^{-1} P^T A)(I - B A)   (Definition "AMGF", Section 5.1)
 *   - PCG with stop test on the relative preconditioned residual  (Section 4: sqrt(r^T z / r0^T z0))
 *
 * The paper fixes none of the AMG parameters (it uses hypre BoomerAMG); the
 * readings taken here (strength, coarsening, interpolation, tie-breaks and the
 * evaluation order of every sum) are the library's specification as well, so
 * that both sides build the same hierarchy:
 *   strength  : j != i is strong for i iff func(j) == func(i) and
 *               |a_ij| >= theta * max_{k != i, func(k) == func(i)} |a_ik| (> 0)
 *   coarsening: Ruge-Stueben first pass; measure = #undecided dependents + 2 #F dependents;
 *               pick max measure, ties -> smallest index; its undecided dependents become F
 *               (each new F point raises the measure of its undecided influencers by 1); the new
 *               C point lowers the measure of its undecided influencers by 1; when the maximal
 *               measure is 0, leftover points become C if they have a strong influencer, else F
 *   interp    : classical interpolation (Ruge-Stueben): strong C neighbours interpolate
 *               directly, each strong F neighbour k is distributed over the strong C points
 *               of i in proportion to the entries of row k whose sign is opposite to a_kk's,
 *               weak neighbours (and strong F points with an empty distribution) are lumped
 *               into the diagonal; a row whose lumped diagonal falls below 5% of a_ii in
 *               magnitude takes direct interpolation with the sign split instead (positive
 *               entries lumped into the diagonal when no positive strong C neighbour).  Only
 *               same-function couplings enter.  interp = 1 selects direct interpolation
 *               everywhere.  p_max > 0 truncates every F row with more weights to its p_max
 *               weights of largest magnitude (ties: smaller coarse index) and scales them by
 *               (sum of all weights) / (sum of the kept ones), so the row sum (interpolation
 *               of constants) is unchanged; a row whose kept weights sum to zero is left whole.
 *   Galerkin  : R = P^T, A_c = R (A P); every sum taken in ascending index order
 *   smoother  : nu sweeps of x <- x + (r - A x) / l1, l1_i = sum_j |a_ij|, zero start on the way
 *               down and the same sweeps on the way up (B symmetric); smoother = 1: the
 *               Chebyshev polynomial of degree nu in W A = diag(1/l1) A for [cheby_lower, 1]
 *               instead, the same polynomial down and up
 *   coarsest  : dense Cholesky when n_l <= max_coarse (or coarsening stalls)
 *   filter    : A_w factored by banded Cholesky after a reverse Cuthill-McKee ordering (exact solve)
 *
 * Parity pins for each step live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* status codes (same numeric meaning as the library's)                */
#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NONFINITE 2
#define ORC_NOT_SPD 3
#define ORC_BREAKDOWN 4
#define ORC_NOT_CONVERGED 5
#define ORC_OOM 7

typedef struct {
  int64_t nrows, ncols;
  int64_t* rp; /* nrows + 1 */
  int32_t* ci;
  double* v;
} ocsr;

typedef struct {
  double strength_theta; /* 0.52 */
  int max_coarse;        /* 1200 */
  int max_levels;        /* 25 */
  int num_functions;     /* 3: DOF i has function i % 3 on the finest level */
  int nu;                /* smoothing sweeps down and up (1) */
  int filter;            /* 0: M = B (AMG-PCG); 1: AMGF */
  int contact_components;/* 0: I_c = nonzero columns of J; 1: all 3 DOFs of those nodes; 2: all DOFs */
  int build_amg;         /* 1: full setup; 0: assemble A only (for A x on large problems) */
  int interp;            /* 0: classical interpolation (default); 1: direct interpolation */
  int p_max;             /* interpolation truncation: at most p_max weights per F row (4; 0: none) */
  int smoother;          /* 0: l1-Jacobi (nu sweeps); 1: Chebyshev of degree nu in W A */
  double cheby_lower;    /* Chebyshev: the polynomial damps eigenvalues of W A in [cheby_lower, 1] */
  int hier_from_K;       /* 1: strength, coarsening and interpolation from the stiffness hierarchy
                            K_{l+1} = R_l K_l P_l, operators A_l = K_l + J_l^T D J_l with
                            J_{l+1} = J_l P_l (a variant; the paper builds B := AMG(A)) */
} orc_opts;

typedef struct {
  int nlev;
  ocsr A[32];
  ocsr P[32];   /* P[l]: n_l x n_{l+1} */
  ocsr R[32];   /* R[l] = P[l]^T */
  double* l1[32];
  int32_t* func[32];
  int8_t* cf[32]; /* 1 = C, 0 = F */
  double* Lc;   /* dense Cholesky factor of coarsest A (row-major, lower) */
  int64_t nc_dense;
  double* theta[32]; /* per-row smoother weights (NULL: theta = 1) */
} orc_amg;

typedef struct {
  orc_opts o;
  int64_t n, m;
  ocsr S;
  orc_amg amg;
  /* filter */
  int64_t nc;
  int64_t* Ic;      /* sorted DOF indices */
  int64_t* perm;    /* position -> index into Ic (RCM order) */
  int64_t bw;       /* half bandwidth in the permuted order */
  double* Lb;       /* band factor: Lb[i*(bw+1) + (i-j)] = L_ij, 0 <= i-j <= bw */
  /* work */
  double* w[8];
  char err[256];
  double* dcontact;  /* diagonal of J^T D J (length n) */
  int8_t* ccontact;  /* 1 if the DOF is a nonzero column of J */
} orc_t;

static void* xmalloc(size_t n) {
  void* p = malloc(n ? n : 1);
  if (!p) { fprintf(stderr, "oracle: out of memory (%zu bytes)\n", n); abort(); }
  return p;
}
static void* xcalloc(size_t n, size_t s) {
  void* p = calloc(n ? n : 1, s ? s : 1);
  if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
  return p;
}

static void csr_free(ocsr* a) {
  free(a->rp); free(a->ci); free(a->v);
  memset(a, 0, sizeof(*a));
}

/* y = A x */
static void csr_mv(const ocsr* a, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < a->nrows; ++i) {
    double s = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) s += a->v[k] * x[a->ci[k]];
    y[i] = s;
  }
}

/* y = b - A x */
static void csr_resid(const ocsr* a, const double* b, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < a->nrows; ++i) {
    double s = 0.0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) s += a->v[k] * x[a->ci[k]];
    y[i] = b[i] - s;
  }
}

/* transpose (rows of the result in ascending column order) */
static void csr_transpose(const ocsr* a, ocsr* t) {
  t->nrows = a->ncols; t->ncols = a->nrows;
  t->rp = xcalloc(t->nrows + 1, sizeof(int64_t));
  int64_t nnz = a->rp[a->nrows];
  t->ci = xmalloc(nnz * sizeof(int32_t));
  t->v = xmalloc(nnz * sizeof(double));
  for (int64_t k = 0; k < nnz; ++k) t->rp[a->ci[k] + 1]++;
  for (int64_t i = 0; i < t->nrows; ++i) t->rp[i + 1] += t->rp[i];
  int64_t* pos = xmalloc((t->nrows + 1) * sizeof(int64_t));
  memcpy(pos, t->rp, (t->nrows + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < a->nrows; ++i)
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      int64_t j = a->ci[k];
      t->ci[pos[j]] = (int32_t)i;
      t->v[pos[j]] = a->v[k];
      pos[j]++;
    }
  free(pos);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* C = A * B.  Entry (i, J) accumulates a_ij * b_jJ over the entries of row i
 * of A in ascending j; result rows sorted by column. */
static void csr_matmul(const ocsr* a, const ocsr* b, ocsr* c) {
  c->nrows = a->nrows; c->ncols = b->ncols;
  c->rp = xcalloc(c->nrows + 1, sizeof(int64_t));
  int64_t cap = a->rp[a->nrows] + 16, nnz = 0;
  c->ci = xmalloc(cap * sizeof(int32_t));
  c->v = xmalloc(cap * sizeof(double));
  double* acc = xcalloc(b->ncols, sizeof(double));
  int64_t* mark = xmalloc(b->ncols * sizeof(int64_t));
  for (int64_t J = 0; J < b->ncols; ++J) mark[J] = -1;
  int32_t* cols = xmalloc((b->ncols + 1) * sizeof(int32_t));
  for (int64_t i = 0; i < a->nrows; ++i) {
    int64_t ncol = 0;
    for (int64_t k = a->rp[i]; k < a->rp[i + 1]; ++k) {
      int64_t j = a->ci[k];
      double aij = a->v[k];
      for (int64_t kk = b->rp[j]; kk < b->rp[j + 1]; ++kk) {
        int32_t J = b->ci[kk];
        if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; cols[ncol++] = J; }
        acc[J] += aij * b->v[kk];
      }
    }
    qsort(cols, ncol, sizeof(int32_t), cmp_i32);
    if (nnz + ncol > cap) {
      while (nnz + ncol > cap) cap *= 2;
      c->ci = realloc(c->ci, cap * sizeof(int32_t));
      c->v = realloc(c->v, cap * sizeof(double));
      if (!c->ci || !c->v) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    }
    for (int64_t t = 0; t < ncol; ++t) { c->ci[nnz] = cols[t]; c->v[nnz] = acc[cols[t]]; nnz++; }
    c->rp[i + 1] = nnz;
  }
  free(acc); free(mark); free(cols);
}

/* ------------------------------------------------------------------ */
/* A = K + J^T D J   (Section 3, eq. linsystem1)                       */
/* (J^T D J)_ab = sum_r J_ra D_r J_rb.  Built as the sum K + J^T (D J) with
 * entries of each row of J^T D J accumulated in ascending constraint r, then
 * merged with K (K entry first, then the contact sum added).               */
static void assemble_S(const ocsr* K, const ocsr* J, const double* D, ocsr* S) {
  ocsr Jt, DJ, C;
  memset(&Jt, 0, sizeof Jt);
  DJ.nrows = J->nrows; DJ.ncols = J->ncols;
  DJ.rp = xmalloc((J->nrows + 1) * sizeof(int64_t));
  memcpy(DJ.rp, J->rp, (J->nrows + 1) * sizeof(int64_t));
  int64_t jn = J->rp[J->nrows];
  DJ.ci = xmalloc(jn * sizeof(int32_t));
  DJ.v = xmalloc(jn * sizeof(double));
  for (int64_t r = 0; r < J->nrows; ++r)
    for (int64_t k = J->rp[r]; k < J->rp[r + 1]; ++k) { DJ.ci[k] = J->ci[k]; DJ.v[k] = D[r] * J->v[k]; }
  csr_transpose(J, &Jt);
  csr_matmul(&Jt, &DJ, &C); /* row a: sum over r ascending of J_ra * (D_r J_rb) */
  /* merge K and C row by row (union of columns, sorted) */
  S->nrows = K->nrows; S->ncols = K->ncols;
  S->rp = xcalloc(S->nrows + 1, sizeof(int64_t));
  int64_t cap = K->rp[K->nrows] + C.rp[C.nrows];
  S->ci = xmalloc(cap * sizeof(int32_t));
  S->v = xmalloc(cap * sizeof(double));
  int64_t nnz = 0;
  for (int64_t i = 0; i < K->nrows; ++i) {
    int64_t a = K->rp[i], ae = K->rp[i + 1], b = C.rp[i], be = C.rp[i + 1];
    while (a < ae || b < be) {
      if (b >= be || (a < ae && K->ci[a] < C.ci[b])) { S->ci[nnz] = K->ci[a]; S->v[nnz] = K->v[a]; a++; }
      else if (a >= ae || C.ci[b] < K->ci[a]) { S->ci[nnz] = C.ci[b]; S->v[nnz] = C.v[b]; b++; }
      else { S->ci[nnz] = K->ci[a]; S->v[nnz] = K->v[a] + C.v[b]; a++; b++; }
      nnz++;
    }
    S->rp[i + 1] = nnz;
  }
  csr_free(&Jt); csr_free(&DJ); csr_free(&C);
}

/* ------------------------------------------------------------------ */
/* AMG setup                                                           */

/* strong influences S_i (CSR pattern over rows of A) */
static void strength(const ocsr* A, const int32_t* func, double theta, ocsr* Sg) {
  int64_t n = A->nrows;
  Sg->nrows = n; Sg->ncols = n; Sg->v = NULL;
  Sg->rp = xcalloc(n + 1, sizeof(int64_t));
  Sg->ci = xmalloc((A->rp[n] + 1) * sizeof(int32_t));
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
      int64_t j = A->ci[k];
      if (j == i || func[j] != func[i]) continue;
      double a = fabs(A->v[k]);
      if (a > mx) mx = a;
    }
    if (mx > 0.0) {
      double thr = theta * mx;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int64_t j = A->ci[k];
        if (j == i || func[j] != func[i]) continue;
        if (fabs(A->v[k]) >= thr) Sg->ci[nnz++] = (int32_t)j;
      }
    }
    Sg->rp[i + 1] = nnz;
  }
}

/* segment tree: leftmost maximum over leaf values */
typedef struct { int64_t size; int64_t* t; } segtree;
static void seg_init(segtree* s, int64_t n, const int64_t* vals) {
  s->size = 1;
  while (s->size < n) s->size <<= 1;
  s->t = xmalloc(2 * s->size * sizeof(int64_t));
  for (int64_t i = 0; i < s->size; ++i) s->t[s->size + i] = (i < n) ? vals[i] : -1;
  for (int64_t i = s->size - 1; i >= 1; --i) {
    int64_t a = s->t[2 * i], b = s->t[2 * i + 1];
    s->t[i] = a > b ? a : b;
  }
}
static void seg_set(segtree* s, int64_t i, int64_t v) {
  int64_t p = s->size + i;
  s->t[p] = v;
  for (p >>= 1; p >= 1; p >>= 1) {
    int64_t a = s->t[2 * p], b = s->t[2 * p + 1];
    s->t[p] = a > b ? a : b;
  }
}
static int64_t seg_argmax(const segtree* s) {
  int64_t p = 1;
  while (p < s->size) p = (s->t[2 * p] == s->t[p]) ? 2 * p : 2 * p + 1;
  return p - s->size;
}

/* Ruge-Stueben first pass; cf[i] = 1 (C) or 0 (F) */
static void rs_coarsen(const ocsr* Sg, int8_t* cf) {
  int64_t n = Sg->nrows;
  ocsr St; /* St row j = points i that depend on j */
  ocsr tmp = *Sg;
  tmp.v = xcalloc(Sg->rp[n] + 1, sizeof(double));
  csr_transpose(&tmp, &St);
  free(tmp.v);
  enum { U = 0, F = 1, C = 2 };
  int8_t* st = xcalloc(n, 1);
  int64_t* lam = xmalloc((n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) lam[i] = St.rp[i + 1] - St.rp[i];
  segtree sg;
  seg_init(&sg, n, lam);
  for (;;) {
    if (sg.t[1] <= 0) break; /* no undecided point with positive measure */
    int64_t i = seg_argmax(&sg);
    st[i] = C;
    seg_set(&sg, i, -1);
    for (int64_t k = St.rp[i]; k < St.rp[i + 1]; ++k) {
      int64_t j = St.ci[k];
      if (st[j] != U) continue;
      st[j] = F;
      seg_set(&sg, j, -1);
      for (int64_t kk = Sg->rp[j]; kk < Sg->rp[j + 1]; ++kk) {
        int64_t q = Sg->ci[kk];
        if (st[q] == U) { lam[q] += 1; seg_set(&sg, q, lam[q]); }
      }
    }
    for (int64_t k = Sg->rp[i]; k < Sg->rp[i + 1]; ++k) {
      int64_t q = Sg->ci[k];
      if (st[q] == U) { lam[q] -= 1; seg_set(&sg, q, lam[q]); }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (st[i] == U) st[i] = (Sg->rp[i + 1] > Sg->rp[i]) ? C : F;
    cf[i] = (st[i] == C) ? 1 : 0;
  }
  free(st); free(lam); free(sg.t);
  csr_free(&St);
}

/* Direct interpolation weights of F point i (Stueben's sign split, same-function sums):
 * appended at P->ci/P->v[*nnz...]; strong[] marks the strong neighbours of i. */
static void direct_row(const ocsr* A, int64_t i, const int32_t* func, const int8_t* strong,
                       const int64_t* cidx, ocsr* P, int64_t* nnz) {
  double diag = 0.0, sn = 0.0, sp = 0.0, cn = 0.0, cp = 0.0;
  for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
    int64_t j = A->ci[k];
    double a = A->v[k];
    if (j == i) { diag = a; continue; }
    if (func[j] != func[i]) continue;
    if (a < 0.0) sn += a; else sp += a;
    if (strong[j] && cidx[j] >= 0) { if (a < 0.0) cn += a; else cp += a; }
  }
  if (cp == 0.0) diag += sp;
  double alpha = (cn != 0.0) ? sn / cn : 0.0;
  double beta = (cp != 0.0) ? sp / cp : 0.0;
  for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
    int64_t j = A->ci[k];
    if (j == i || !strong[j] || cidx[j] < 0) continue;
    double a = A->v[k];
    double w = (a < 0.0) ? -(alpha * a) / diag : -(beta * a) / diag;
    P->ci[*nnz] = (int32_t)cidx[j]; P->v[*nnz] = w; (*nnz)++;
  }
}

/* Truncate the F row P->ci/P->v[row0 .. *nnz) (ascending coarse index) to its p_max weights of
 * largest magnitude, ties to the smaller coarse index, rescaled to the old row sum; both
 * sums run in ascending index order.  Selection by repeated maximum over the row. */
static void truncate_row(ocsr* P, int64_t row0, int64_t* nnz, int p_max) {
  const int64_t len = *nnz - row0;
  if (p_max <= 0 || len <= p_max) return;
  int8_t* keep = xcalloc(len, 1);
  for (int t = 0; t < p_max; ++t) {
    int64_t best = -1;
    for (int64_t q = 0; q < len; ++q)
      if (!keep[q] && (best < 0 || fabs(P->v[row0 + q]) > fabs(P->v[row0 + best]))) best = q;
    keep[best] = 1;
  }
  double total = 0.0, kept = 0.0;
  for (int64_t q = 0; q < len; ++q) total += P->v[row0 + q];
  for (int64_t q = 0; q < len; ++q) if (keep[q]) kept += P->v[row0 + q];
  if (kept != 0.0) {
    const double scale = total / kept;
    int64_t m = row0;
    for (int64_t q = 0; q < len; ++q) {
      if (!keep[q]) continue;
      P->ci[m] = P->ci[row0 + q];
      P->v[m] = P->v[row0 + q] * scale;
      m++;
    }
    *nnz = m;
  }
  free(keep);
}

/* Interpolation P (n x n_c) from the C/F split.
 * interp = 0, classical interpolation (Ruge & Stueben), same-function couplings only:
 *   w_ij = -( a_ij + sum_{k in F_i^s} a_ik abar_kj / sum_{m in C_i^s} abar_km ) / d_i,
 *   d_i = a_ii + sum_{n weak} a_in  (+ a_ik of strong F points k with an empty sum),
 *   abar_km = a_km where its sign is opposite to a_kk's, else 0;
 *   rows with |d_i| < CLASSICAL_GUARD a_ii (lumping cancelled the diagonal) take the
 *   direct weights instead.
 * interp = 1, direct interpolation for every row.
 * C points interpolate by identity; F points without a strong C neighbour get an empty row. */
#define CLASSICAL_GUARD 0.05
static void build_interp(const ocsr* A, const ocsr* Sg, const int32_t* func, const int8_t* cf, int interp,
                         int p_max, ocsr* P, int64_t* ncoarse) {
  int64_t n = A->nrows;
  int64_t* cidx = xmalloc(n * sizeof(int64_t));
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) cidx[i] = cf[i] ? nc++ : -1;
  *ncoarse = nc;
  P->nrows = n; P->ncols = nc;
  P->rp = xcalloc(n + 1, sizeof(int64_t));
  int64_t cap = Sg->rp[n] + n + 1;
  P->ci = xmalloc(cap * sizeof(int32_t));
  P->v = xmalloc(cap * sizeof(double));
  int8_t* strong = xcalloc(n, 1);
  int64_t* pos = xmalloc(n * sizeof(int64_t)); /* position of strong C point m in row i's P entries */
  for (int64_t i = 0; i < n; ++i) pos[i] = -1;
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (cf[i]) {
      P->ci[nnz] = (int32_t)cidx[i]; P->v[nnz] = 1.0; nnz++;
      P->rp[i + 1] = nnz;
      continue;
    }
    int anyC = 0;
    for (int64_t k = Sg->rp[i]; k < Sg->rp[i + 1]; ++k) {
      strong[Sg->ci[k]] = 1;
      if (cf[Sg->ci[k]]) anyC = 1;
    }
    if (anyC && interp == 1) {
      direct_row(A, i, func, strong, cidx, P, &nnz);
    } else if (anyC) {
      const int64_t row0 = nnz;
      double diag = 0.0, aii = 0.0;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) { /* the strong C points, numerators a_ij */
        int64_t j = A->ci[k];
        if (j == i) { aii = A->v[k]; diag += A->v[k]; continue; }
        if (func[j] != func[i]) continue;
        if (strong[j] && cf[j]) { P->ci[nnz] = (int32_t)cidx[j]; P->v[nnz] = A->v[k]; pos[j] = nnz; nnz++; }
      }
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) {
        int64_t j = A->ci[k];
        if (j == i || func[j] != func[i] || (strong[j] && cf[j])) continue;
        double a = A->v[k];
        if (!strong[j]) { diag += a; continue; } /* weak neighbour: lumped */
        double akk = 0.0, den = 0.0;             /* strong F neighbour j: distributed over C_i^s */
        for (int64_t q = A->rp[j]; q < A->rp[j + 1]; ++q) if (A->ci[q] == j) akk = A->v[q];
        for (int64_t q = A->rp[j]; q < A->rp[j + 1]; ++q) {
          int64_t m2 = A->ci[q];
          if (m2 == j || pos[m2] < 0) continue;
          double am = A->v[q];
          if ((am < 0.0) != (akk < 0.0)) den += am;
        }
        if (den == 0.0) { diag += a; continue; }
        for (int64_t q = A->rp[j]; q < A->rp[j + 1]; ++q) {
          int64_t m2 = A->ci[q];
          if (m2 == j || pos[m2] < 0) continue;
          double am = A->v[q];
          if ((am < 0.0) != (akk < 0.0)) P->v[pos[m2]] += a * am / den;
        }
      }
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) pos[A->ci[k]] = -1;
      if (fabs(diag) < CLASSICAL_GUARD * aii) {
        nnz = row0;
        direct_row(A, i, func, strong, cidx, P, &nnz);
      } else {
        for (int64_t q = row0; q < nnz; ++q) P->v[q] = -P->v[q] / diag;
      }
    }
    for (int64_t k = Sg->rp[i]; k < Sg->rp[i + 1]; ++k) strong[Sg->ci[k]] = 0;
    truncate_row(P, P->rp[i], &nnz, p_max);
    P->rp[i + 1] = nnz;
  }
  free(strong); free(pos); free(cidx);
}

/* dense Cholesky (row-major lower); returns ORC_NOT_SPD on a non-positive pivot */
static int dense_chol(double* a, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    double s = a[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= a[j * n + k] * a[j * n + k];
    if (!(s > 0.0)) return ORC_NOT_SPD;
    double d = sqrt(s);
    a[j * n + j] = d;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = a[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = t / d;
    }
    for (int64_t i = 0; i < j; ++i) a[i * n + j] = 0.0;
  }
  return ORC_OK;
}
static void dense_chol_solve(const double* L, int64_t n, const double* b, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * x[k];
    x[i] = s / L[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = x[i];
    for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

static void csr_copy(const ocsr* a, ocsr* b) {
  const int64_t nnz = a->rp[a->nrows];
  b->nrows = a->nrows; b->ncols = a->ncols;
  b->rp = xmalloc((a->nrows + 1) * sizeof(int64_t));
  b->ci = xmalloc((nnz ? nnz : 1) * sizeof(int32_t));
  b->v = xmalloc((nnz ? nnz : 1) * sizeof(double));
  memcpy(b->rp, a->rp, (a->nrows + 1) * sizeof(int64_t));
  memcpy(b->ci, a->ci, nnz * sizeof(int32_t));
  memcpy(b->v, a->v, nnz * sizeof(double));
}

/* K, J, D: the inputs, used by the K-based variant (o->hier_from_K) only:
 *   strength, coarsening and interpolation of level l from K_l (K_0 = K, K_{l+1} = R_l K_l P_l),
 *   J_{l+1} = J_l P_l, and the level operator A_{l+1} = K_{l+1} + J_{l+1}^T D J_{l+1}
 *   (the same matrix as R_l A_l P_l in exact arithmetic). */
static int amg_setup(orc_t* h, const ocsr* K, const ocsr* J, const double* D) {
  orc_amg* g = &h->amg;
  const orc_opts* o = &h->o;
  const int fromK = o->hier_from_K && K;
  ocsr Kl, Jl;
  memset(&Kl, 0, sizeof Kl);
  memset(&Jl, 0, sizeof Jl);
  if (fromK) {
    csr_copy(K, &Kl);
    if (J && J->nrows > 0) csr_copy(J, &Jl);
  }
  /* level 0 operator is a copy of S */
  ocsr* A0 = &g->A[0];
  A0->nrows = h->S.nrows; A0->ncols = h->S.ncols;
  int64_t nnz = h->S.rp[h->S.nrows];
  A0->rp = xmalloc((A0->nrows + 1) * sizeof(int64_t));
  A0->ci = xmalloc(nnz * sizeof(int32_t));
  A0->v = xmalloc(nnz * sizeof(double));
  memcpy(A0->rp, h->S.rp, (A0->nrows + 1) * sizeof(int64_t));
  memcpy(A0->ci, h->S.ci, nnz * sizeof(int32_t));
  memcpy(A0->v, h->S.v, nnz * sizeof(double));
  g->func[0] = xmalloc(A0->nrows * sizeof(int32_t));
  for (int64_t i = 0; i < A0->nrows; ++i) g->func[0][i] = (int32_t)(o->num_functions > 1 ? i % o->num_functions : 0);
  int l = 0;
  for (;;) {
    ocsr* A = &g->A[l];
    int64_t n = A->nrows;
    g->l1[l] = xmalloc(n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k) s += fabs(A->v[k]);
      g->l1[l][i] = s;
    }
    if (n <= o->max_coarse || l + 1 >= o->max_levels || l + 1 >= 32) break;
    const ocsr* H = fromK ? &Kl : A; /* the matrix the hierarchy is built from */
    ocsr Sg;
    strength(H, g->func[l], o->strength_theta, &Sg);
    g->cf[l] = xmalloc(n);
    rs_coarsen(&Sg, g->cf[l]);
    int64_t nc = 0;
    build_interp(H, &Sg, g->func[l], g->cf[l], o->interp, o->p_max, &g->P[l], &nc);
    csr_free(&Sg);
    if (nc == 0 || nc == n) { /* coarsening stalled: this level is the coarsest */
      csr_free(&g->P[l]); free(g->cf[l]); g->cf[l] = NULL;
      break;
    }
    csr_transpose(&g->P[l], &g->R[l]);
    ocsr AP;
    if (fromK) {
      /* K_{l+1} = R K_l P, J_{l+1} = J_l P, A_{l+1} = K_{l+1} + J_{l+1}^T D J_{l+1} */
      ocsr Kc, JP;
      csr_matmul(&Kl, &g->P[l], &AP);
      csr_matmul(&g->R[l], &AP, &Kc);
      csr_free(&AP);
      csr_free(&Kl);
      Kl = Kc;
      if (Jl.nrows > 0) {
        csr_matmul(&Jl, &g->P[l], &JP);
        csr_free(&Jl);
        Jl = JP;
        assemble_S(&Kl, &Jl, D, &g->A[l + 1]);
      } else {
        csr_copy(&Kl, &g->A[l + 1]);
      }
    } else {
      csr_matmul(A, &g->P[l], &AP);
      csr_matmul(&g->R[l], &AP, &g->A[l + 1]);
      csr_free(&AP);
    }
    g->func[l + 1] = xmalloc(nc * sizeof(int32_t));
    for (int64_t i = 0, c = 0; i < n; ++i)
      if (g->cf[l][i]) g->func[l + 1][c++] = g->func[l][i];
    l++;
  }
  g->nlev = l + 1;
  if (fromK) { csr_free(&Kl); csr_free(&Jl); }
  /* coarsest: dense Cholesky */
  ocsr* AL = &g->A[l];
  int64_t nL = AL->nrows;
  if (nL > 8192) { snprintf(h->err, sizeof h->err, "coarsest level too large (%lld)", (long long)nL); return ORC_INVALID; }
  g->nc_dense = nL;
  g->Lc = xcalloc(nL * nL, sizeof(double));
  for (int64_t i = 0; i < nL; ++i)
    for (int64_t k = AL->rp[i]; k < AL->rp[i + 1]; ++k) g->Lc[i * nL + AL->ci[k]] = AL->v[k];
  if (dense_chol(g->Lc, nL) != ORC_OK) { snprintf(h->err, sizeof h->err, "coarsest matrix not SPD"); return ORC_NOT_SPD; }
  return ORC_OK;
}

/* x = B_l r  (V-cycle, recursive) */
/* Chebyshev smoothing of A x = b with the l1-scaled operator W A, W = diag(1 / l1): its
 * eigenvalues lie in (0, 1] (l1 row sums bound the spectrum), and the polynomial is the
 * shifted Chebyshev polynomial of the interval [lo, 1], applied by the three-term recurrence
 * of Chebyshev acceleration (Saad, Iterative Methods for Sparse Linear Systems, Algorithm
 * 12.1) with centre c = (1 + lo) / 2, half-width h = (1 - lo) / 2, s = c / h:
 *   rho_0 = 1 / s,  d_0 = W r_0 / c,  x_1 = x_0 + d_0,
 *   rho_j = 1 / (2 s - rho_{j-1}),  d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / h) W r_j,
 *   x_{j+1} = x_j + d_j,  r_j = b - A x_j.
 * k steps leave the error q_k(W A) e_0, q_k(l) = T_k((c - l) / h) / T_k(s).  from_zero: x_0 = 0
 * (r_0 = b, no product). */
static void cheby_smooth(const ocsr* A, const double* l1, const double* b, double* x, int k, double lo,
                         int from_zero, double* res, double* d) {
  const int64_t n = A->nrows;
  const double c = 0.5 * (1.0 + lo), hw = 0.5 * (1.0 - lo), sg = c / hw;
  double rho = 1.0 / sg;
  if (from_zero) {
    for (int64_t i = 0; i < n; ++i) { d[i] = (b[i] / l1[i]) / c; x[i] = d[i]; }
  } else {
    csr_resid(A, b, x, res);
    for (int64_t i = 0; i < n; ++i) { d[i] = (res[i] / l1[i]) / c; x[i] += d[i]; }
  }
  for (int j = 1; j < k; ++j) {
    const double rho_new = 1.0 / (2.0 * sg - rho);
    const double a = rho_new * rho, bc = 2.0 * rho_new / hw;
    csr_resid(A, b, x, res);
    for (int64_t i = 0; i < n; ++i) { d[i] = a * d[i] + bc * (res[i] / l1[i]); x[i] += d[i]; }
    rho = rho_new;
  }
}

static void vcycle(orc_t* h, int l, const double* r, double* x) {
  orc_amg* g = &h->amg;
  const ocsr* A = &g->A[l];
  int64_t n = A->nrows;
  if (l == g->nlev - 1) { dense_chol_solve(g->Lc, n, r, x); return; }
  const double* l1 = g->l1[l];
  const double* th = g->theta[l];
  double* res = xmalloc(n * sizeof(double));
  const int cheb = h->o.smoother == 1;
  double* d = cheb ? xmalloc(n * sizeof(double)) : NULL;
  if (cheb) {
    cheby_smooth(A, l1, r, x, h->o.nu, h->o.cheby_lower, 1, res, d);
  } else {
    /* pre-smoothing from x = 0: x = W r, W = diag(theta / l1) (theta = 1 without weights) */
    for (int64_t i = 0; i < n; ++i) x[i] = th ? (th[i] / l1[i]) * r[i] : r[i] / l1[i];
    for (int s = 1; s < h->o.nu; ++s) {
      csr_resid(A, r, x, res);
      for (int64_t i = 0; i < n; ++i) x[i] += th ? (th[i] / l1[i]) * res[i] : res[i] / l1[i];
    }
  }
  /* coarse-grid correction */
  csr_resid(A, r, x, res);
  int64_t nc = g->A[l + 1].nrows;
  double* rc = xmalloc(nc * sizeof(double));
  double* ec = xmalloc(nc * sizeof(double));
  csr_mv(&g->R[l], res, rc);
  vcycle(h, l + 1, rc, ec);
  double* pe = xmalloc(n * sizeof(double));
  csr_mv(&g->P[l], ec, pe);
  for (int64_t i = 0; i < n; ++i) x[i] += pe[i];
  /* post-smoothing (the same smoother as before the coarse correction, so B stays symmetric) */
  if (cheb) {
    cheby_smooth(A, l1, r, x, h->o.nu, h->o.cheby_lower, 0, res, d);
  } else {
    for (int s = 0; s < h->o.nu; ++s) {
      csr_resid(A, r, x, res);
      for (int64_t i = 0; i < n; ++i) x[i] += th ? (th[i] / l1[i]) * res[i] : res[i] / l1[i];
    }
  }
  free(res); free(rc); free(ec); free(pe); free(d);
}

/* ------------------------------------------------------------------ */
/* filter: I_c, A_w = A[I_c, I_c], RCM ordering, banded Cholesky        */

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

static void contact_set(orc_t* h, const ocsr* J) {
  int64_t n = h->n;
  int8_t* in = xcalloc(n, 1);
  if (h->o.contact_components == 2) {
    for (int64_t i = 0; i < n; ++i) in[i] = 1;
  } else {
    for (int64_t k = 0; k < J->rp[J->nrows]; ++k)
      if (J->v[k] != 0.0) {
        int64_t c = J->ci[k];
        if (h->o.contact_components == 1) { int64_t nd = c / 3; for (int d = 0; d < 3; ++d) if (3 * nd + d < n) in[3 * nd + d] = 1; }
        else in[c] = 1;
      }
  }
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) nc += in[i];
  h->nc = nc;
  h->Ic = xmalloc((nc + 1) * sizeof(int64_t));
  for (int64_t i = 0, t = 0; i < n; ++i) if (in[i]) h->Ic[t++] = i;
  free(in);
}

typedef struct { int64_t deg, idx; } degidx;
static int cmp_degidx(const void* a, const void* b) {
  const degidx* x = a; const degidx* y = b;
  if (x->deg != y->deg) return (x->deg > y->deg) - (x->deg < y->deg);
  return (x->idx > y->idx) - (x->idx < y->idx);
}

static int filter_setup(orc_t* h) {
  int64_t nc = h->nc;
  if (nc == 0) return ORC_OK;
  /* position of each DOF in I_c */
  int64_t* pos = xmalloc(h->n * sizeof(int64_t));
  for (int64_t i = 0; i < h->n; ++i) pos[i] = -1;
  for (int64_t t = 0; t < nc; ++t) pos[h->Ic[t]] = t;
  /* A_w = P^T A P: rows/cols of A restricted to I_c (CSR in I_c numbering) */
  ocsr Aw;
  Aw.nrows = nc; Aw.ncols = nc;
  Aw.rp = xcalloc(nc + 1, sizeof(int64_t));
  int64_t cap = 0;
  for (int64_t t = 0; t < nc; ++t) cap += h->S.rp[h->Ic[t] + 1] - h->S.rp[h->Ic[t]];
  Aw.ci = xmalloc((cap + 1) * sizeof(int32_t));
  Aw.v = xmalloc((cap + 1) * sizeof(double));
  int64_t nnz = 0;
  for (int64_t t = 0; t < nc; ++t) {
    int64_t i = h->Ic[t];
    for (int64_t k = h->S.rp[i]; k < h->S.rp[i + 1]; ++k) {
      int64_t p = pos[h->S.ci[k]];
      if (p >= 0) { Aw.ci[nnz] = (int32_t)p; Aw.v[nnz] = h->S.v[k]; nnz++; }
    }
    Aw.rp[t + 1] = nnz;
  }
  free(pos);
  /* reverse Cuthill-McKee: BFS from a minimum-degree unvisited vertex (ties: smallest
   * index), neighbours enqueued by increasing degree (ties: smallest index), then reversed */
  int64_t* deg = xmalloc(nc * sizeof(int64_t));
  for (int64_t t = 0; t < nc; ++t) deg[t] = Aw.rp[t + 1] - Aw.rp[t];
  int8_t* vis = xcalloc(nc, 1);
  int64_t* order = xmalloc(nc * sizeof(int64_t));
  degidx* nb = xmalloc((nc + 1) * sizeof(degidx));
  int64_t head = 0, tail = 0;
  while (tail < nc) {
    int64_t s = -1;
    for (int64_t t = 0; t < nc; ++t)
      if (!vis[t] && (s < 0 || deg[t] < deg[s])) s = t;
    vis[s] = 1; order[tail++] = s;
    while (head < tail) {
      int64_t u = order[head++], cnt = 0;
      for (int64_t k = Aw.rp[u]; k < Aw.rp[u + 1]; ++k) {
        int64_t v = Aw.ci[k];
        if (!vis[v]) { vis[v] = 1; nb[cnt].deg = deg[v]; nb[cnt].idx = v; cnt++; }
      }
      qsort(nb, cnt, sizeof(degidx), cmp_degidx);
      for (int64_t c = 0; c < cnt; ++c) order[tail++] = nb[c].idx;
    }
  }
  h->perm = xmalloc(nc * sizeof(int64_t));
  for (int64_t t = 0; t < nc; ++t) h->perm[t] = order[nc - 1 - t];
  int64_t* ipos = xmalloc(nc * sizeof(int64_t));
  for (int64_t t = 0; t < nc; ++t) ipos[h->perm[t]] = t;
  int64_t bw = 0;
  for (int64_t t = 0; t < nc; ++t)
    for (int64_t k = Aw.rp[t]; k < Aw.rp[t + 1]; ++k) {
      int64_t d = ipos[t] - ipos[Aw.ci[k]];
      if (d < 0) d = -d;
      if (d > bw) bw = d;
    }
  h->bw = bw;
  /* band storage of the permuted matrix, lower part: Lb[i*(bw+1) + (i-j)] */
  int64_t W = bw + 1;
  h->Lb = xcalloc((size_t)(nc > 0 ? nc : 1) * (size_t)(W > 0 ? W : 1), sizeof(double));
  for (int64_t t = 0; t < nc; ++t)
    for (int64_t k = Aw.rp[t]; k < Aw.rp[t + 1]; ++k) {
      int64_t i = ipos[t], j = ipos[Aw.ci[k]];
      if (j <= i) h->Lb[i * W + (i - j)] = Aw.v[k];
    }
  free(deg); free(vis); free(order); free(nb); free(ipos);
  csr_free(&Aw);
  /* banded Cholesky */
  double* L = h->Lb;
  for (int64_t j = 0; j < nc; ++j) {
    double s = L[j * W];
    int64_t k0 = j - bw > 0 ? j - bw : 0;
    for (int64_t k = k0; k < j; ++k) s -= L[j * W + (j - k)] * L[j * W + (j - k)];
    if (!(s > 0.0)) { snprintf(h->err, sizeof h->err, "filter matrix not SPD (pivot %lld)", (long long)j); return ORC_NOT_SPD; }
    double d = sqrt(s);
    L[j * W] = d;
    int64_t i1 = j + bw < nc - 1 ? j + bw : nc - 1;
    for (int64_t i = j + 1; i <= i1; ++i) {
      double t = L[i * W + (i - j)];
      int64_t kk0 = i - bw > 0 ? i - bw : 0;
      for (int64_t k = kk0; k < j; ++k) t -= L[i * W + (i - k)] * L[j * W + (j - k)];
      L[i * W + (i - j)] = t / d;
    }
  }
  return ORC_OK;
}

/* w = A_w^{-1} v  (v, w in I_c numbering) */
static void filter_solve(orc_t* h, const double* v, double* w) {
  int64_t nc = h->nc, bw = h->bw, W = bw + 1;
  const double* L = h->Lb;
  double* y = xmalloc(nc * sizeof(double));
  for (int64_t i = 0; i < nc; ++i) {
    double s = v[h->perm[i]];
    int64_t k0 = i - bw > 0 ? i - bw : 0;
    for (int64_t k = k0; k < i; ++k) s -= L[i * W + (i - k)] * y[k];
    y[i] = s / L[i * W];
  }
  for (int64_t i = nc - 1; i >= 0; --i) {
    double s = y[i];
    int64_t k1 = i + bw < nc - 1 ? i + bw : nc - 1;
    for (int64_t k = i + 1; k <= k1; ++k) s -= L[k * W + (k - i)] * y[k];
    y[i] = s / L[i * W];
  }
  for (int64_t i = 0; i < nc; ++i) w[h->perm[i]] = y[i];
  free(y);
}

/* ------------------------------------------------------------------ */
/* public API                                                          */

void orc_opts_default(orc_opts* o) {
  o->strength_theta = 0.52;
  o->max_coarse = 1200;
  o->max_levels = 25;
  o->num_functions = 3;
  o->nu = 1;
  o->filter = 1;
  o->contact_components = 0;
  o->build_amg = 1;
  o->interp = 0;
  o->p_max = 4;
  o->smoother = 0;
  o->cheby_lower = 0.3;
  o->hier_from_K = 0;
}

const char* orc_error(orc_t* h) { return h ? h->err : "null handle"; }

/* Bound-constrained variant (Remark on bound constraints, Section 3): with
 * J~ = [J; I; -I] and D~ = diag(D, D_lo, D_hi) the matrix is K + J~^T D~ J~ =
 * K + J^T D J + diag(D_lo + D_hi).  E = D_lo + D_hi (length n, entries >= 0, NULL = 0) is
 * added to the diagonal after the J^T D J term.  The filter space stays the nonzero
 * columns of J: the bound rows would make every DOF a "contact" DOF. */
int orc_create_bounds(int64_t n,
                      const int64_t* Krp, const int32_t* Kci, const double* Kv,
                      int64_t m,
                      const int64_t* Jrp, const int32_t* Jci, const double* Jv,
                      const double* D, const double* E, const orc_opts* opts, orc_t** out);
void orc_free(orc_t* h);

int orc_create(int64_t n,
               const int64_t* Krp, const int32_t* Kci, const double* Kv,
               int64_t m,
               const int64_t* Jrp, const int32_t* Jci, const double* Jv,
               const double* D, const orc_opts* opts, orc_t** out) {
  return orc_create_bounds(n, Krp, Kci, Kv, m, Jrp, Jci, Jv, D, NULL, opts, out);
}

int orc_create_bounds(int64_t n,
                      const int64_t* Krp, const int32_t* Kci, const double* Kv,
                      int64_t m,
                      const int64_t* Jrp, const int32_t* Jci, const double* Jv,
                      const double* D, const double* E, const orc_opts* opts, orc_t** out) {
  *out = NULL;
  if (n <= 0 || m < 0) return ORC_INVALID;
  if (opts->smoother < 0 || opts->smoother > 1 || !(opts->cheby_lower > 0.0 && opts->cheby_lower < 1.0))
    return ORC_INVALID;
  orc_t* h = xcalloc(1, sizeof(orc_t));
  h->o = *opts;
  h->n = n; h->m = m;
  for (int64_t r = 0; r < m; ++r)
    if (!isfinite(D[r])) { free(h); return ORC_NONFINITE; }
    else if (!(D[r] > 0.0)) { free(h); return ORC_NOT_SPD; }
  if (E)
    for (int64_t i = 0; i < n; ++i)
      if (!isfinite(E[i])) { free(h); return ORC_NONFINITE; }
      else if (E[i] < 0.0) { free(h); return ORC_NOT_SPD; }
  ocsr K = {n, n, (int64_t*)Krp, (int32_t*)Kci, (double*)Kv};
  ocsr J = {m, n, (int64_t*)Jrp, (int32_t*)Jci, (double*)Jv};
  /* per-DOF contact data for the learned smoother's features: (J^T D J)_aa and the flag */
  h->dcontact = xcalloc(n, sizeof(double));
  h->ccontact = xcalloc(n, 1);
  for (int64_t r = 0; r < m; ++r)
    for (int64_t k = Jrp[r]; k < Jrp[r + 1]; ++k) {
      h->dcontact[Jci[k]] += Jv[k] * (D[r] * Jv[k]);
      if (Jv[k] != 0.0) h->ccontact[Jci[k]] = 1;
    }
  if (m > 0) assemble_S(&K, &J, D, &h->S);
  else {
    int64_t nnz = Krp[n];
    h->S.nrows = n; h->S.ncols = n;
    h->S.rp = xmalloc((n + 1) * sizeof(int64_t)); memcpy(h->S.rp, Krp, (n + 1) * sizeof(int64_t));
    h->S.ci = xmalloc(nnz * sizeof(int32_t)); memcpy(h->S.ci, Kci, nnz * sizeof(int32_t));
    h->S.v = xmalloc(nnz * sizeof(double)); memcpy(h->S.v, Kv, nnz * sizeof(double));
  }
  if (E) {
    for (int64_t i = 0; i < n; ++i) {
      int found = 0;
      for (int64_t k = h->S.rp[i]; k < h->S.rp[i + 1]; ++k)
        if (h->S.ci[k] == i) { h->S.v[k] += E[i]; found = 1; }
      if (!found && E[i] != 0.0) { orc_free(h); return ORC_INVALID; } /* K stores its diagonal */
      h->dcontact[i] += E[i];
    }
  }
  if (!h->o.build_amg) {
    for (int i = 0; i < 8; ++i) h->w[i] = xmalloc(n * sizeof(double));
    *out = h;
    return ORC_OK;
  }
  if (h->o.hier_from_K && E) { orc_free(h); return ORC_INVALID; } /* variant without bound terms */
  int st = amg_setup(h, &K, &J, D);
  if (st != ORC_OK) { *out = h; return st; }
  if (h->o.filter) {
    if (m > 0 || h->o.contact_components == 2) contact_set(h, &J);
    st = filter_setup(h);
    if (st != ORC_OK) { *out = h; return st; }
  }
  for (int i = 0; i < 8; ++i) h->w[i] = xmalloc(n * sizeof(double));
  *out = h;
  return ORC_OK;
}

void orc_free(orc_t* h) {
  if (!h) return;
  csr_free(&h->S);
  for (int l = 0; l < 32; ++l) {
    csr_free(&h->amg.A[l]); csr_free(&h->amg.P[l]); csr_free(&h->amg.R[l]);
    free(h->amg.l1[l]); free(h->amg.func[l]); free(h->amg.cf[l]); free(h->amg.theta[l]);
  }
  free(h->dcontact); free(h->ccontact);
  free(h->amg.Lc); free(h->Ic); free(h->perm); free(h->Lb);
  for (int i = 0; i < 8; ++i) free(h->w[i]);
  free(h);
}

/* y = A x */
void orc_S_apply(orc_t* h, const double* x, double* y) { csr_mv(&h->S, x, y); }

/* x = B r  (one V-cycle, zero initial guess) */
void orc_vcycle(orc_t* h, const double* r, double* x) { vcycle(h, 0, r, x); }

/* w = A_w^{-1} v, v and w of length n_c in I_c order */
void orc_filter_solve(orc_t* h, const double* v, double* w) { filter_solve(h, v, w); }

/* z = M r.  filter == 0: M = B.  filter == 1: AMGF (Definition "AMGF"):
 *   y1 = B r; r1 = r - A y1; w = A_w^{-1} P^T r1; y2 = y1 + P w; r2 = r - A y2; z = y2 + B r2 */
void orc_apply(orc_t* h, const double* r, double* z) {
  int64_t n = h->n;
  if (!h->o.filter) { vcycle(h, 0, r, z); return; }
  double* y = h->w[0];
  double* r1 = h->w[1];
  double* t = h->w[2];
  vcycle(h, 0, r, y);                      /* y1 */
  csr_resid(&h->S, r, y, r1);              /* r1 = r - A y1 */
  if (h->nc > 0) {
    double* v = xmalloc(h->nc * sizeof(double));
    double* w = xmalloc(h->nc * sizeof(double));
    for (int64_t k = 0; k < h->nc; ++k) v[k] = r1[h->Ic[k]];   /* P^T r1 */
    filter_solve(h, v, w);
    for (int64_t k = 0; k < h->nc; ++k) y[h->Ic[k]] += w[k];  /* y2 = y1 + P w */
    free(v); free(w);
  }
  csr_resid(&h->S, r, y, r1);              /* r2 = r - A y2 */
  vcycle(h, 0, r1, t);                     /* B r2 */
  for (int64_t i = 0; i < n; ++i) z[i] = y[i] + t[i];
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Preconditioned CG (x holds x0 on entry).  Stops when sqrt(r_k^T z_k / r_0^T z_0) < tol,
 * evaluated after each update; *iters = number of A p products.  alphas/betas (length
 * maxit, may be NULL) receive the CG coefficients; relres (length maxit+1) the
 * relative preconditioned residual after each iteration (entry 0 = 1). */
int orc_pcg(orc_t* h, const double* b, double* x, double tol, int maxit,
            int* iters, double* alphas, double* betas, double* relres) {
  int64_t n = h->n;
  double* r = xmalloc(n * sizeof(double));
  double* z = xmalloc(n * sizeof(double));
  double* p = xmalloc(n * sizeof(double));
  double* q = xmalloc(n * sizeof(double));
  *iters = 0;
  int status = ORC_NOT_CONVERGED;
  csr_resid(&h->S, b, x, r);
  orc_apply(h, r, z);
  double rz = dot(r, z, n);
  if (!isfinite(rz)) { status = ORC_NONFINITE; goto done; }
  double rz0 = rz;
  if (relres) relres[0] = 1.0;
  if (rz0 == 0.0) { status = ORC_OK; goto done; }
  if (rz0 < 0.0) { status = ORC_BREAKDOWN; goto done; }
  memcpy(p, z, n * sizeof(double));
  for (int k = 1; k <= maxit; ++k) {
    csr_mv(&h->S, p, q);
    double pq = dot(p, q, n);
    if (!(pq > 0.0)) { status = isfinite(pq) ? ORC_BREAKDOWN : ORC_NONFINITE; break; }
    double alpha = rz / pq;
    for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
    orc_apply(h, r, z);
    double rzn = dot(r, z, n);
    *iters = k;
    if (alphas) alphas[k - 1] = alpha;
    if (!isfinite(rzn)) { status = ORC_NONFINITE; break; }
    if (rzn < 0.0) { status = ORC_BREAKDOWN; break; }
    double rel = sqrt(rzn / rz0);
    if (relres) relres[k] = rel;
    double beta = rzn / rz;
    if (betas) betas[k - 1] = beta;
    if (rel < tol) { status = ORC_OK; break; }
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rzn;
  }
done:
  free(r); free(z); free(p); free(q);
  return status;
}

/* ---------------- learned smoother weights (test infrastructure) ----------------
 * Per-row damping theta_i of the l1-Jacobi smoother, W = diag(theta / l1), predicted by a
 * small MLP from local features; theta = 0.3 + 0.9 sigmoid(o) keeps theta in [0.3, 1.2]
 * (< 2, so the l1 smoother stays convergent and B stays SPD).  Features of row i on level l:
 *   f0 = log10(a_ii) / 10, f1 = log10(l1_i) / 10, f2 = a_ii / l1_i, f3 = contact flag,
 *   f4 = log10(1 + d_i) / 10 with d = diag(J^T D J) on level 0, f5 = l / (nlev - 1);
 * the flag and d of a coarse row are those of the fine C point it comes from.
 * Weights (1313): W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3. */
#define MLP_NW 1313

static void mlp_features(orc_t* h, int l, const double* dl, const int8_t* cl, double* f /* n_l x 6 */) {
  const ocsr* A = &h->amg.A[l];
  int nlev = h->amg.nlev;
  for (int64_t i = 0; i < A->nrows; ++i) {
    double aii = 0.0;
    for (int64_t k = A->rp[i]; k < A->rp[i + 1]; ++k)
      if (A->ci[k] == i) aii = A->v[k];
    double l1 = h->amg.l1[l][i];
    f[6 * i + 0] = log10(aii) / 10.0;
    f[6 * i + 1] = log10(l1) / 10.0;
    f[6 * i + 2] = aii / l1;
    f[6 * i + 3] = cl[i] ? 1.0 : 0.0;
    f[6 * i + 4] = log10(1.0 + dl[i]) / 10.0;
    f[6 * i + 5] = nlev > 1 ? (double)l / (double)(nlev - 1) : 0.0;
  }
}

static double mlp_theta(const double* w, const double* f) {
  const double* W1 = w;          /* [32][6] */
  const double* b1 = w + 192;
  const double* W2 = w + 224;    /* [32][32] */
  const double* b2 = w + 1248;
  const double* w3 = w + 1280;
  const double b3 = w[1312];
  double h1[32], h2[32];
  for (int j = 0; j < 32; ++j) {
    double s = b1[j];
    for (int k = 0; k < 6; ++k) s += W1[6 * j + k] * f[k];
    h1[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < 32; ++j) {
    double s = b2[j];
    for (int k = 0; k < 32; ++k) s += W2[32 * j + k] * h1[k];
    h2[j] = s > 0.0 ? s : 0.0;
  }
  double o = b3;
  for (int k = 0; k < 32; ++k) o += w3[k] * h2[k];
  return 0.3 + 0.9 / (1.0 + exp(-o));
}

/* Set (w != NULL) or clear (w == NULL) the learned weights of every smoothed level. */
int orc_set_mlp(orc_t* h, const double* w, int64_t nw) {
  orc_amg* g = &h->amg;
  for (int l = 0; l < 32; ++l) { free(g->theta[l]); g->theta[l] = NULL; }
  if (!w) return ORC_OK;
  if (nw != MLP_NW) return ORC_INVALID;
  int64_t n0 = g->A[0].nrows;
  double* dl = xmalloc(n0 * sizeof(double));
  int8_t* cl = xmalloc(n0);
  memcpy(dl, h->dcontact, n0 * sizeof(double));
  memcpy(cl, h->ccontact, n0);
  for (int l = 0; l + 1 < g->nlev; ++l) {
    int64_t n = g->A[l].nrows;
    double* f = xmalloc(6 * n * sizeof(double));
    mlp_features(h, l, dl, cl, f);
    g->theta[l] = xmalloc(n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) g->theta[l][i] = mlp_theta(w, f + 6 * i);
    free(f);
    /* inherit d and the flag to the coarse level through the C points */
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
      if (g->cf[l][i]) { dl[c] = dl[i]; cl[c] = cl[i]; c++; }
  }
  free(dl); free(cl);
  return ORC_OK;
}

/* Training objective of the learned smoother (not in the paper): the error reduction of one
 * damped l1-Jacobi step on given vectors, averaged over the smoothed levels,
 *   L = (1 / (nlev - 1)) sum_l ||(I - A_l W_l) r_l||^2 / ||r_l||^2,   W_l = diag(theta_l / l1_l),
 * theta from the active weights (orc_set_mlp), theta = 1 without them.  r_all holds r_0, r_1,
 * ..., r_{nlev-2} back to back (n_l values each). */
int orc_mlp_loss(orc_t* h, const double* r_all, double* loss) {
  orc_amg* g = &h->amg;
  if (g->nlev < 2) return ORC_INVALID;
  double sum = 0.0;
  const double* r = r_all;
  for (int l = 0; l + 1 < g->nlev; ++l) {
    const ocsr* A = &g->A[l];
    const int64_t n = A->nrows;
    double* x = xmalloc(n * sizeof(double));
    double* e = xmalloc(n * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
      const double th = g->theta[l] ? g->theta[l][i] : 1.0;
      x[i] = (th / g->l1[l][i]) * r[i];
    }
    csr_resid(A, r, x, e); /* e = r - A W r */
    double ee = 0.0, rr = 0.0;
    for (int64_t i = 0; i < n; ++i) { ee += e[i] * e[i]; rr += r[i] * r[i]; }
    sum += ee / rr;
    free(x); free(e);
    r += n;
  }
  *loss = sum / (double)(g->nlev - 1);
  return ORC_OK;
}

/* Threads of the parallel loops (A x and residuals); returns the previous setting.  Used by the
 * benchmark to time the oracle single-threaded and on all cores. */
int orc_set_threads(int k) {
#ifdef _OPENMP
  const int prev = omp_get_max_threads();
  if (k > 0) omp_set_num_threads(k);
  return prev;
#else
  (void)k;
  return 1;
#endif
}

int orc_get_theta(orc_t* h, int l, double* out) {
  if (l < 0 || l >= h->amg.nlev - 1 || !h->amg.theta[l]) return ORC_INVALID;
  memcpy(out, h->amg.theta[l], h->amg.A[l].nrows * sizeof(double));
  return ORC_OK;
}

/* ---------------- introspection (tests) ---------------- */
int orc_num_levels(orc_t* h) { return h->amg.nlev; }
int64_t orc_n(orc_t* h) { return h->n; }
int64_t orc_nc(orc_t* h) { return h->nc; }
int64_t orc_bandwidth(orc_t* h) { return h->bw; }
void orc_get_Ic(orc_t* h, int64_t* Ic) { memcpy(Ic, h->Ic, h->nc * sizeof(int64_t)); }

/* which: 0 = A_l, 1 = P_l, 2 = R_l, 3 = S (level ignored) */
static const ocsr* pick(orc_t* h, int which, int l) {
  if (which == 3) return &h->S;
  if (l < 0 || l >= h->amg.nlev) return NULL;
  if (which == 0) return &h->amg.A[l];
  if (l >= h->amg.nlev - 1) return NULL;
  return which == 1 ? &h->amg.P[l] : &h->amg.R[l];
}
int orc_mat_shape(orc_t* h, int which, int l, int64_t* nrows, int64_t* ncols, int64_t* nnz) {
  const ocsr* a = pick(h, which, l);
  if (!a) return ORC_INVALID;
  *nrows = a->nrows; *ncols = a->ncols; *nnz = a->rp[a->nrows];
  return ORC_OK;
}
int orc_mat_get(orc_t* h, int which, int l, int64_t* rp, int32_t* ci, double* v) {
  const ocsr* a = pick(h, which, l);
  if (!a) return ORC_INVALID;
  memcpy(rp, a->rp, (a->nrows + 1) * sizeof(int64_t));
  memcpy(ci, a->ci, a->rp[a->nrows] * sizeof(int32_t));
  memcpy(v, a->v, a->rp[a->nrows] * sizeof(double));
  return ORC_OK;
}
int orc_get_cf(orc_t* h, int l, int8_t* cf) {
  if (l < 0 || l >= h->amg.nlev - 1 || !h->amg.cf[l]) return ORC_INVALID;
  memcpy(cf, h->amg.cf[l], h->amg.A[l].nrows);
  return ORC_OK;
}
int orc_get_l1(orc_t* h, int l, double* out) {
  if (l < 0 || l >= h->amg.nlev) return ORC_INVALID;
  memcpy(out, h->amg.l1[l], h->amg.A[l].nrows * sizeof(double));
  return ORC_OK;
}
int orc_get_func(orc_t* h, int l, int32_t* out) {
  if (l < 0 || l >= h->amg.nlev) return ORC_INVALID;
  memcpy(out, h->amg.func[l], h->amg.A[l].nrows * sizeof(int32_t));
  return ORC_OK;
}
