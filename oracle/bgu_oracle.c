/*
 * bgu_oracle.c -- plain FP64 CPU oracle for the Givens bidiagonal update (BGU).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path and is written for a reader who checks it against the
 * paper (Brust & Saunders, "Fast and Accurate SVD-Type Updating in Streaming
 * Data"), not for speed: one rotation at a time, in the order the algorithm
 * generates them.
 *
 * What it computes (Sec. 3.2, Eqs. rk1, bidiagsubproblem, bidiagplus):
 *   given A = Q * Bd * P^T (Q m x m, P n x n orthogonal, Bd n x n upper
 *   bidiagonal with diagonal d and superdiagonal e, m >= n) and an update
 *   B (m x r), C (n x r), produce Q+, Bd+, P+ with Q+ Bd+ P+^T = A + B C^T.
 *   Rank r is processed as r rank-1 steps (Sec. 3.2: "repeating the
 *   process"); U = Q^T B and V = P^T C are formed once with the old factors
 *   and the later columns are rotated along with every rotation of the
 *   earlier ones, which is exact because Q+^T b = G (Q^T b).
 *
 * The reduction of B + b+ c+^T (Sec. 3.4, Algorithm 2, Eqs. giv, giv1, gfill)
 * follows one fixed schedule, because the paper's phase-1 figure is not
 * available and bidiagonal factorizations are only unique up to the choice
 * of the first right vector.  The schedule used here never rotates column 1
 * of P (so P+(:,1) = P(:,1)), which makes Bd+ unique up to signs and lets
 * textbook bidiagonalizations of A+ P pin it:
 *
 *   rot(f,g): [c s; -s c][f; g] = [r; 0].  g == 0: no rotation (not counted).
 *             f == 0: c = 0, s = 1, r = g (the paper's permutation case).
 *             otherwise r = sign(f) * hypot(f, g), c = f / r, s = g / r.
 *             The eliminated entry is set to exactly 0 and the pivot to r.
 *   pair update of two vectors: x_a <- c x_a + s x_b, x_b <- -s x_a + c x_b.
 *   A left rotation on rows (a, a+1) updates those rows of the core, of u and
 *   of the later columns of U, and columns a, a+1 of Q (Q <- Q G^T).
 *   A right rotation on columns (a, a+1) updates those columns of the core,
 *   of v and of the later columns of V, and columns a, a+1 of P (P <- P H).
 *
 *   spike (m > n): for j = m, ..., n+2, left rotation (j-1, j) zeroing u(j)
 *             (the paper's order G_{m,m-1} first; rows > n of the core are
 *             zero, so Bd is untouched).  The core then has N = n+1 rows,
 *             otherwise N = n.
 *   phase 1:  for j = N, ..., 2: left rotation (j-1, j) zeroing u(j), then
 *             chase with i = j-1: while i+2 <= n and M(i,i+2) != 0:
 *             right rotation (i+1, i+2) zeroing M(i,i+2); if i+3 <= N and
 *             M(i+3,i+1) != 0: left rotation (i+2, i+3) zeroing M(i+3,i+1);
 *             i += 2.
 *   fold:     row 1 of the core += u(1) v^T; u, v := 0.
 *   phase 2:  for j = n, ..., 3: right rotation (j-1, j) zeroing M(1,j),
 *             then chase_lower(j-1).
 *   phase 3:  for i = 1, ..., n-1 (and i = n when N = n+1):
 *             (a) left rotation (i, i+1) zeroing M(i+1,i);
 *             (b) if i+3 <= n: right rotation (i+2, i+3) zeroing M(i,i+3),
 *                 then chase_lower(i+2);
 *             (c) if i+2 <= n: right rotation (i+1, i+2) zeroing M(i,i+2),
 *                 then chase_lower(i+1).
 *   chase_lower(k): while k+2 <= N and M(k+2,k) != 0: left rotation
 *             (k+1, k+2) zeroing M(k+2,k); if k+4 <= n and M(k+1,k+4) != 0:
 *             right rotation (k+3, k+4) zeroing M(k+1,k+4); k += 3.
 *
 * Storage of the core: a band with offsets -2..+3 around the diagonal (the
 * widest pattern any phase creates: the p = 1, q = 2 band of Sec. 3.4 plus
 * one bulge slot on each side) and, between the fold and the end of phase 2,
 * a dense copy of row 1.  A rotation visits every stored entry of its two
 * rows (columns) -- entries outside the band are structurally zero.  Writing
 * a nonzero outside the band is reported as ORC_EBAND, so the band
 * invariants of the schedule are checked on every rotation.
 *
 * Indices in this file are 1-based, as in the paper.  Matrices passed in are
 * column-major with the stated leading dimensions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EBAND = 3, ORC_EZERO = 4 };
enum { PH_SPIKE = 0, PH_1 = 1, PH_2 = 2, PH_3 = 3 };

/* A list of rotations in generation order; pair (a, a+1) is 1-based. */
typedef struct {
  int64_t count, cap;
  double *c, *s;
  int32_t *a;
  int8_t *phase;
} orc_rotlist;

typedef struct {
  int64_t left[4], right[4]; /* rotations by phase: spike, 1, 2, 3 */
  int64_t band_violations;
  int64_t zero_violations;   /* an entry that the schedule must leave exactly 0 was not */
} orc_counts;

/* ------------------------------------------------------------------------ */
/* Rotation generator (Eqs. giv, giv1; zero handling of Sec. 3.4)           */
/*                                                                          */
/* r = sign(f) * hypot(f, g) with safe scaling.  The scaling is by an exact  */
/* power of two chosen from the larger magnitude (the idea of Anderson's     */
/* "safe scaling", ACM TOMS Algorithm 978), so that f^2 + g^2 neither        */
/* overflows nor loses the larger term to underflow:                         */
/*   a = max(|f|, |g|);  sigma = 2^-600 if a > 2^500, 2^600 if a < 2^-500,   */
/*   else 1;  fs = sigma f, gs = sigma g  (exact);                           */
/*   h = sqrt(fs*fs + gs*gs);  rs = sign(f) h;  c = fs / rs;  s = gs / rs;   */
/*   r = rs / sigma  (exact).                                                */
/* Every step is one correctly rounded IEEE operation (the library is built  */
/* with -ffp-contract=off), so the result is fully determined by (f, g).     */
/* ------------------------------------------------------------------------ */
int orc_rot(double f, double g, double *c, double *s, double *r) {
  if (g == 0.0) return 0;
  if (f == 0.0) { *c = 0.0; *s = 1.0; *r = g; return 1; }
  const double big = 0x1p500, small = 0x1p-500;
  double a = fabs(f) > fabs(g) ? fabs(f) : fabs(g);
  double sigma = 1.0;
  if (a > big) sigma = 0x1p-600;
  else if (a < small) sigma = 0x1p600;
  double fs = f * sigma, gs = g * sigma;
  double h = sqrt(fs * fs + gs * gs);
  double rs = copysign(h, f);
  *c = fs / rs;
  *s = gs / rs;
  *r = rs / sigma;
  return 1;
}

static int list_push(orc_rotlist *L, double c, double s, int32_t a, int8_t ph) {
  if (L->count == L->cap) {
    int64_t nc = L->cap ? 2 * L->cap : 1024;
    double *c2 = realloc(L->c, nc * sizeof(double));
    if (c2) L->c = c2;
    double *s2 = realloc(L->s, nc * sizeof(double));
    if (s2) L->s = s2;
    int32_t *a2 = realloc(L->a, nc * sizeof(int32_t));
    if (a2) L->a = a2;
    int8_t *p2 = realloc(L->phase, nc * sizeof(int8_t));
    if (p2) L->phase = p2;
    if (!c2 || !s2 || !a2 || !p2) return ORC_ENOMEM;
    L->cap = nc;
  }
  L->c[L->count] = c;
  L->s[L->count] = s;
  L->a[L->count] = a;
  L->phase[L->count] = ph;
  L->count++;
  return ORC_OK;
}

void orc_free_list(orc_rotlist *L) {
  free(L->c); free(L->s); free(L->a); free(L->phase);
  memset(L, 0, sizeof(*L));
}

/* ------------------------------------------------------------------------ */
/* The core M = band + u v^T (Eq. sparsity) and the vectors rotated along   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int m, n, N;
  double *bd[6];  /* bd[o+2][i] = M(i, i+o), o = -2..3, i = 1..N */
  double *row1;   /* dense row 1, row1[j] = M(1, j), j = 1..n, while row1_dense */
  int row1_dense;
  double *u;      /* u(1..m) */
  double *v;      /* v(1..n) */
  int rx;         /* later columns rotated along (rank r > 1) */
  double *Ux;     /* Ux[(t)*m + (i-1)], t = 0..rx-1: later columns of U */
  double *Vx;     /* Vx[(t)*n + (j-1)] */
  orc_rotlist *L, *R;
  orc_counts *cnt;
  int phase;
  int err;
} core_t;

static double Mget(const core_t *k, int i, int j) {
  if (i < 1 || i > k->N || j < 1 || j > k->n) return 0.0;
  if (i == 1 && k->row1_dense) return k->row1[j];
  int o = j - i;
  if (o < -2 || o > 3) return 0.0;
  return k->bd[o + 2][i];
}

static void Mset(core_t *k, int i, int j, double x) {
  if (i < 1 || i > k->N || j < 1 || j > k->n) {
    if (x != 0.0) k->cnt->band_violations++;
    return;
  }
  if (i == 1 && k->row1_dense) { k->row1[j] = x; return; }
  int o = j - i;
  if (o < -2 || o > 3) {
    if (x != 0.0) k->cnt->band_violations++;
    return;
  }
  k->bd[o + 2][i] = x;
}

/* Left rotation on rows (a, a+1); (ie, je) is the eliminated entry, set to 0,
 * and (ip, jp) the pivot, set to r.  ie == 0 means the eliminated entry is
 * u(a+1) (phase-1 start and spike), whose pivot is u(a). */
static void rot_rows(core_t *k, int a, double c, double s, double r, int je) {
  int jlo = a - 2 < 1 ? 1 : a - 2;
  int jhi = a + 4 > k->n ? k->n : a + 4;
  if (a <= k->N) { /* the spike's rows lie below the core: no core entries */
    for (int j = jlo; j <= jhi; j++) {
      double x = Mget(k, a, j), y = Mget(k, a + 1, j);
      Mset(k, a, j, c * x + s * y);
      Mset(k, a + 1, j, -s * x + c * y);
    }
  }
  if (je > 0) { Mset(k, a, je, r); Mset(k, a + 1, je, 0.0); }
  double x = k->u[a], y = k->u[a + 1];
  k->u[a] = c * x + s * y;
  k->u[a + 1] = -s * x + c * y;
  if (je == 0) { k->u[a] = r; k->u[a + 1] = 0.0; }
  for (int t = 0; t < k->rx; t++) {
    double *U = k->Ux + (size_t)t * k->m - 1; /* 1-based */
    double xu = U[a], yu = U[a + 1];
    U[a] = c * xu + s * yu;
    U[a + 1] = -s * xu + c * yu;
  }
  if (list_push(k->L, c, s, a, (int8_t)k->phase)) k->err = ORC_ENOMEM;
  k->cnt->left[k->phase]++;
}

/* Right rotation on columns (a, a+1); (ie, a+1) is the eliminated entry and
 * (ie, a) the pivot. */
static void rot_cols(core_t *k, int a, double c, double s, double r, int ie) {
  int ilo = a - 3 < 1 ? 1 : a - 3;
  int ihi = a + 3 > k->N ? k->N : a + 3;
  if (k->row1_dense && ilo > 1) {
    double x = Mget(k, 1, a), y = Mget(k, 1, a + 1);
    Mset(k, 1, a, c * x + s * y);
    Mset(k, 1, a + 1, -s * x + c * y);
  }
  for (int i = ilo; i <= ihi; i++) {
    double x = Mget(k, i, a), y = Mget(k, i, a + 1);
    Mset(k, i, a, c * x + s * y);
    Mset(k, i, a + 1, -s * x + c * y);
  }
  Mset(k, ie, a, r);
  Mset(k, ie, a + 1, 0.0);
  double x = k->v[a], y = k->v[a + 1];
  k->v[a] = c * x + s * y;
  k->v[a + 1] = -s * x + c * y;
  for (int t = 0; t < k->rx; t++) {
    double *V = k->Vx + (size_t)t * k->n - 1;
    double xv = V[a], yv = V[a + 1];
    V[a] = c * xv + s * yv;
    V[a + 1] = -s * xv + c * yv;
  }
  if (list_push(k->R, c, s, a, (int8_t)k->phase)) k->err = ORC_ENOMEM;
  k->cnt->right[k->phase]++;
}

/* Eliminate M(ie, je) against M(ie, je-1) with a right rotation on columns
 * (je-1, je).  Returns 1 if a rotation was applied. */
static int zero_by_cols(core_t *k, int ie, int je) {
  double c, s, r;
  if (!orc_rot(Mget(k, ie, je - 1), Mget(k, ie, je), &c, &s, &r)) return 0;
  rot_cols(k, je - 1, c, s, r, ie);
  return 1;
}

/* Eliminate M(ie, je) against M(ie-1, je) with a left rotation on rows
 * (ie-1, ie). */
static int zero_by_rows(core_t *k, int ie, int je) {
  double c, s, r;
  if (!orc_rot(Mget(k, ie - 1, je), Mget(k, ie, je), &c, &s, &r)) return 0;
  rot_rows(k, ie - 1, c, s, r, je);
  return 1;
}

/* Eliminate u(j) against u(j-1) with a left rotation on rows (j-1, j). */
static int zero_u(core_t *k, int j) {
  double c, s, r;
  if (!orc_rot(k->u[j - 1], k->u[j], &c, &s, &r)) return 0;
  rot_rows(k, j - 1, c, s, r, 0);
  return 1;
}

static void chase_lower(core_t *k, int kk) {
  while (kk + 2 <= k->N && Mget(k, kk + 2, kk) != 0.0) {
    zero_by_rows(k, kk + 2, kk);
    if (kk + 4 <= k->n && Mget(k, kk + 1, kk + 4) != 0.0) zero_by_cols(k, kk + 1, kk + 4);
    kk += 3;
  }
}

/* One rank-1 step on the core (d, e) with u (length m) and v (length n). */
static int bgu_rank1(core_t *k) {
  const int m = k->m, n = k->n;
  /* spike (m > n) */
  k->phase = PH_SPIKE;
  for (int j = m; j >= n + 2; j--) zero_u(k, j);
  for (int j = n + 2; j <= m; j++)
    if (k->u[j] != 0.0) k->cnt->zero_violations++;
  /* phase 1: absorb u bottom-up */
  k->phase = PH_1;
  const int N = k->N;
  for (int j = N; j >= 2; j--) {
    zero_u(k, j);
    int i = j - 1;
    while (i + 2 <= n && Mget(k, i, i + 2) != 0.0) {
      zero_by_cols(k, i, i + 2);
      if (i + 3 <= N && Mget(k, i + 3, i + 1) != 0.0) zero_by_rows(k, i + 3, i + 1);
      i += 2;
    }
  }
  for (int j = 2; j <= N; j++)
    if (k->u[j] != 0.0) k->cnt->zero_violations++;
  /* fold: row 1 += u(1) v^T */
  for (int j = 1; j <= n; j++) k->row1[j] = Mget(k, 1, j) + k->u[1] * k->v[j];
  for (int o = -2; o <= 3; o++) k->bd[o + 2][1] = 0.0;
  k->row1_dense = 1;
  for (int j = 1; j <= m; j++) k->u[j] = 0.0;
  for (int j = 1; j <= n; j++) k->v[j] = 0.0;
  /* phase 2: clear row 1 right to left */
  k->phase = PH_2;
  for (int j = n; j >= 3; j--) {
    zero_by_cols(k, 1, j);
    chase_lower(k, j - 1);
  }
  /* row 1 is back inside the band */
  for (int j = 3; j <= n; j++)
    if (k->row1[j] != 0.0) k->cnt->zero_violations++;
  k->row1_dense = 0;
  for (int j = 1; j <= n && j <= 4; j++) Mset(k, 1, j, k->row1[j]);
  /* phase 3: band -> bidiagonal */
  k->phase = PH_3;
  int ilast = (N == n + 1) ? n : n - 1;
  for (int i = 1; i <= ilast; i++) {
    if (i + 1 <= N) zero_by_rows(k, i + 1, i);
    if (i + 3 <= n && zero_by_cols(k, i, i + 3)) chase_lower(k, i + 2);
    if (i + 2 <= n && zero_by_cols(k, i, i + 2)) chase_lower(k, i + 1);
  }
  /* every entry off the diagonal and first superdiagonal is exactly 0 */
  for (int i = 1; i <= N; i++)
    for (int o = -2; o <= 3; o++) {
      if (o == 0 || o == 1) continue;
      int j = i + o;
      if (j >= 1 && j <= n && k->bd[o + 2][i] != 0.0) k->cnt->zero_violations++;
    }
  return k->err;
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

/* U = Q^T B (m x r), V = P^T C (n x r); Eq. bidiagsubproblem. */
void orc_project(int m, int n, int r, const double *Q, int ldq, const double *P, int ldp,
                 const double *B, int ldb, const double *C, int ldc, double *U, double *V) {
  for (int t = 0; t < r; t++) {
    for (int i = 0; i < m; i++) {
      double acc = 0.0;
      for (int l = 0; l < m; l++) acc += Q[(size_t)i * ldq + l] * B[(size_t)t * ldb + l];
      U[(size_t)t * m + i] = acc;
    }
    for (int i = 0; i < n; i++) {
      double acc = 0.0;
      for (int l = 0; l < n; l++) acc += P[(size_t)i * ldp + l] * C[(size_t)t * ldc + l];
      V[(size_t)t * n + i] = acc;
    }
  }
}

/* Runs the reduction for r rank-1 columns on the bidiagonal (d, e), given the
 * projected update U (m x r) and V (n x r), which are consumed (rotated in
 * place).  d (n) and e (n-1) are updated in place.  The left rotations (for Q)
 * and right rotations (for P) are appended to *L and *R in generation order. */
int orc_generate(int m, int n, int r, double *d, double *e, double *U, double *V,
                 orc_rotlist *L, orc_rotlist *R, orc_counts *cnt) {
  if (m < n || n < 1 || r < 0) return ORC_EINVAL;
  core_t k;
  memset(&k, 0, sizeof(k));
  k.m = m; k.n = n; k.N = (m > n) ? n + 1 : n;
  k.L = L; k.R = R; k.cnt = cnt;
  for (int o = 0; o < 6; o++) {
    k.bd[o] = calloc((size_t)k.N + 2, sizeof(double));
    if (!k.bd[o]) return ORC_ENOMEM;
  }
  k.row1 = calloc((size_t)n + 2, sizeof(double));
  k.u = calloc((size_t)m + 2, sizeof(double));
  k.v = calloc((size_t)n + 2, sizeof(double));
  if (!k.row1 || !k.u || !k.v) return ORC_ENOMEM;
  int rc = ORC_OK;
  for (int col = 0; col < r && rc == ORC_OK; col++) {
    for (int o = 0; o < 6; o++) memset(k.bd[o], 0, ((size_t)k.N + 2) * sizeof(double));
    for (int i = 1; i <= n; i++) k.bd[2][i] = d[i - 1];
    for (int i = 1; i <= n - 1; i++) k.bd[3][i] = e[i - 1];
    for (int i = 1; i <= m; i++) k.u[i] = U[(size_t)col * m + i - 1];
    for (int i = 1; i <= n; i++) k.v[i] = V[(size_t)col * n + i - 1];
    k.rx = r - col - 1;
    k.Ux = U + (size_t)(col + 1) * m;
    k.Vx = V + (size_t)(col + 1) * n;
    k.row1_dense = 0;
    rc = bgu_rank1(&k);
    for (int i = 1; i <= n; i++) d[i - 1] = k.bd[2][i];
    for (int i = 1; i <= n - 1; i++) e[i - 1] = k.bd[3][i];
  }
  for (int o = 0; o < 6; o++) free(k.bd[o]);
  free(k.row1); free(k.u); free(k.v);
  if (rc == ORC_OK && cnt->band_violations) rc = ORC_EBAND;
  if (rc == ORC_OK && cnt->zero_violations) rc = ORC_EZERO;
  return rc;
}

/* Applies the rotations of *L (in order) to the listed rows of X, an
 * nrow_total x ncol column-major matrix with leading dimension ldx:
 * X(i, a), X(i, a+1) <- pair update.  This forms Q+ = Q * prod G^T from the
 * left list and P+ = P * prod H from the right list (Eq. bidiagplus).  Rows
 * are independent, so they are processed in parallel when OpenMP is on. */
void orc_apply_rows(double *X, int ldx, int ncol, const int32_t *rows, int nrows,
                    const orc_rotlist *L) {
#pragma omp parallel
  {
    double *x = malloc(((size_t)ncol + 2) * sizeof(double));
#pragma omp for schedule(static)
    for (int t = 0; t < nrows; t++) {
      int i = rows[t];
      for (int j = 1; j <= ncol; j++) x[j] = X[(size_t)(j - 1) * ldx + i];
      for (int64_t q = 0; q < L->count; q++) {
        int a = L->a[q];
        double c = L->c[q], s = L->s[q];
        double xa = x[a], xb = x[a + 1];
        x[a] = c * xa + s * xb;
        x[a + 1] = -s * xa + c * xb;
      }
      for (int j = 1; j <= ncol; j++) X[(size_t)(j - 1) * ldx + i] = x[j];
    }
    free(x);
  }
}

/* Full update: Q (m x m, ldq), d, e, P (n x n, ldp) are replaced by Q+, d+,
 * e+, P+ for A + B C^T.  Rank-1 columns are reduced in order and all
 * rotations are then applied to Q and P. */
int orc_update(int m, int n, int r, double *Q, int ldq, double *d, double *e, double *P,
               int ldp, const double *B, int ldb, const double *C, int ldc, orc_counts *cnt) {
  if (m < n || n < 1 || r < 0 || ldq < m || ldp < n) return ORC_EINVAL;
  double *U = malloc((size_t)m * (r > 0 ? r : 1) * sizeof(double));
  double *V = malloc((size_t)n * (r > 0 ? r : 1) * sizeof(double));
  int32_t *rows = malloc((size_t)m * sizeof(int32_t));
  if (!U || !V || !rows) return ORC_ENOMEM;
  orc_project(m, n, r, Q, ldq, P, ldp, B, ldb, C, ldc, U, V);
  orc_rotlist L = {0}, R = {0};
  int rc = orc_generate(m, n, r, d, e, U, V, &L, &R, cnt);
  if (rc == ORC_OK || rc == ORC_EBAND || rc == ORC_EZERO) {
    for (int i = 0; i < m; i++) rows[i] = i;
    orc_apply_rows(Q, ldq, m, rows, m, &L);
    orc_apply_rows(P, ldp, n, rows, n, &R);
  }
  orc_free_list(&L);
  orc_free_list(&R);
  free(U); free(V); free(rows);
  return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes) for tiny matrices: an independent way to  */
/* get singular values.  X (rows x cols, column-major) is overwritten; sv    */
/* receives the column norms after convergence (unsorted).                   */
/* ------------------------------------------------------------------------ */
int orc_jacobi_sv(double *X, int rows, int cols, double *sv, int max_sweeps) {
  /* A column whose squared norm falls below (rows eps)^2 ||X||_F^2 is
   * numerically zero (X is rank deficient): it cannot be made orthogonal to
   * the others beyond rounding, so its pairs count as converged.  The
   * rotations preserve ||X||_F, so it is taken once. */
  double fro2 = 0.0;
  for (size_t i = 0; i < (size_t)rows * cols; i++) fro2 += X[i] * X[i];
  const double null2 = (rows * 0x1p-52) * (rows * 0x1p-52) * fro2;
  for (int sweep = 0; sweep < max_sweeps; sweep++) {
    double off = 0.0;
    for (int p = 0; p < cols - 1; p++)
      for (int q = p + 1; q < cols; q++) {
        double *xp = X + (size_t)p * rows, *xq = X + (size_t)q * rows;
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < rows; i++) {
          alpha += xp[i] * xp[i];
          beta += xq[i] * xq[i];
          gamma += xp[i] * xq[i];
        }
        if (gamma == 0.0 || alpha <= null2 || beta <= null2) continue;
        double rel = fabs(gamma) / sqrt(alpha * beta);
        if (rel > off) off = rel;
        if (rel < 1e-15) continue;
        /* rotation angle that makes columns p and q orthogonal */
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < rows; i++) {
          double a = xp[i], b = xq[i];
          xp[i] = cs * a - sn * b;
          xq[i] = sn * a + cs * b;
        }
      }
    if (off < 1e-15) {
      for (int p = 0; p < cols; p++) {
        double acc = 0.0;
        for (int i = 0; i < rows; i++) acc += X[(size_t)p * rows + i] * X[(size_t)p * rows + i];
        sv[p] = sqrt(acc);
      }
      return sweep + 1;
    }
  }
  return -1;
}
