/* Drives the oracle's C library (oracle/bgu_oracle.c) through randomized
 * small problems with structured exact zeros, extreme magnitudes and every
 * entry point, for a build with AddressSanitizer and UndefinedBehavior-
 * Sanitizer: any out-of-bounds access, leak or undefined operation aborts
 * the run.  The declarations below restate the library's interface. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t count, cap;
  double *c, *s;
  int32_t *a;
  int8_t *phase;
} orc_rotlist;

typedef struct {
  int64_t left[4], right[4];
  int64_t band_violations;
  int64_t zero_violations;
} orc_counts;

int orc_rot(double f, double g, double *c, double *s, double *r);
void orc_free_list(orc_rotlist *L);
void orc_project(int m, int n, int r, const double *Q, int ldq, const double *P, int ldp, const double *B, int ldb,
                 const double *C, int ldc, double *U, double *V);
int orc_generate(int m, int n, int r, double *d, double *e, double *U, double *V, orc_rotlist *L, orc_rotlist *R,
                 orc_counts *cnt);
void orc_apply_rows(double *X, int ldx, int ncol, const int32_t *rows, int nrows, const orc_rotlist *L);
int orc_update(int m, int n, int r, double *Q, int ldq, double *d, double *e, double *P, int ldp, const double *B,
               int ldb, const double *C, int ldc, orc_counts *cnt);
int orc_jacobi_sv(double *X, int rows, int cols, double *sv, int max_sweeps);

static uint64_t rs = 0x9E3779B97F4A7C15ull;
static double unif(void) { /* xorshift64*, uniform in [0, 1) */
  rs ^= rs >> 12; rs ^= rs << 25; rs ^= rs >> 27;
  return (double)((rs * 0x2545F4914F6CDD1Dull) >> 11) * 0x1p-53;
}
static double gauss(void) { return sqrt(-2.0 * log(1.0 - unif())) * cos(6.283185307179586 * unif()); }

/* a product of k Householder reflectors, n x n column-major */
static void orthogonal(double *X, int n, int k) {
  double *v = malloc(sizeof(double) * n);
  memset(X, 0, sizeof(double) * n * n);
  for (int i = 0; i < n; i++) X[i * n + i] = 1.0;
  for (int t = 0; t < k; t++) {
    double nv = 0.0;
    for (int i = 0; i < n; i++) { v[i] = gauss(); nv += v[i] * v[i]; }
    for (int j = 0; j < n; j++) {
      double dot = 0.0;
      for (int i = 0; i < n; i++) dot += v[i] * X[j * n + i];
      for (int i = 0; i < n; i++) X[j * n + i] -= 2.0 * dot / nv * v[i];
    }
  }
  free(v);
}

int main(void) {
  int fails = 0;
  /* rotation generator at the extremes */
  const double vals[] = {0.0, -0.0, 1.0, -3.0, 0x1p-1074, 0x1p-1022, 0x1p1000, -0x1p1020, 1e-300, 1e300};
  const int nv = (int)(sizeof(vals) / sizeof(vals[0]));
  for (int i = 0; i < nv; i++)
    for (int j = 0; j < nv; j++) {
      double c = 0, s = 0, r = 0;
      if (orc_rot(vals[i], vals[j], &c, &s, &r) && !(isfinite(c) && isfinite(s) && isfinite(r))) fails++;
    }
  for (int trial = 0; trial < 400; trial++) {
    const int n = 1 + (int)(unif() * 12), m = n + (int)(unif() * 6), r = 1 + (int)(unif() * 3);
    double *Q = malloc(sizeof(double) * m * m), *P = malloc(sizeof(double) * n * n);
    double *d = malloc(sizeof(double) * n), *e = malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
    double *B = malloc(sizeof(double) * m * r), *C = malloc(sizeof(double) * n * r);
    orthogonal(Q, m, 3);
    orthogonal(P, n, 3);
    const double scale = (trial % 7 == 0) ? 0x1p600 : (trial % 11 == 0 ? 0x1p-600 : 1.0);
    for (int i = 0; i < n; i++) d[i] = unif() < 0.3 ? 0.0 : gauss() * scale;
    for (int i = 0; i + 1 < n; i++) e[i] = unif() < 0.3 ? 0.0 : gauss() * scale;
    for (int i = 0; i < m * r; i++) B[i] = unif() < 0.5 ? 0.0 : gauss() * scale;
    for (int i = 0; i < n * r; i++) C[i] = unif() < 0.5 ? 0.0 : gauss();
    orc_counts cnt;
    memset(&cnt, 0, sizeof(cnt));
    if (orc_update(m, n, r, Q, m, d, e, P, n, B, m, C, n, &cnt) != 0) fails++;
    /* the reduction alone, and its application to every row */
    double *U = malloc(sizeof(double) * m * r), *V = malloc(sizeof(double) * n * r);
    orc_project(m, n, r, Q, m, P, n, B, m, C, n, U, V);
    orc_rotlist L, R;
    memset(&L, 0, sizeof(L));
    memset(&R, 0, sizeof(R));
    memset(&cnt, 0, sizeof(cnt));
    if (orc_generate(m, n, r, d, e, U, V, &L, &R, &cnt) != 0) fails++;
    int32_t *rows = malloc(sizeof(int32_t) * m);
    for (int i = 0; i < m; i++) rows[i] = i;
    orc_apply_rows(Q, m, m, rows, m, &L);
    orc_apply_rows(P, n, n, rows, n, &R);
    orc_free_list(&L);
    orc_free_list(&R);
    /* singular values of the dense bidiagonal */
    double *X = calloc((size_t)m * n, sizeof(double)), *sv = malloc(sizeof(double) * n);
    for (int i = 0; i < n; i++) {
      X[i * m + i] = d[i];
      if (i + 1 < n) X[(i + 1) * m + i] = e[i];
    }
    if (orc_jacobi_sv(X, m, n, sv, 60) < 0) fails++;
    free(Q); free(P); free(d); free(e); free(B); free(C); free(U); free(V); free(rows); free(X); free(sv);
  }
  printf("oracle_sanitize %s (%d failures)\n", fails ? "FAILED" : "ok", fails);
  return fails != 0;
}
