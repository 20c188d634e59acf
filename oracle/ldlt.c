/* Oracle: plain up-looking sparse LDL^T of a complex symmetric matrix.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/sparse_ldlt.py for the tests,
 * smoke() and the CPU baseline of bench.py.  Shares nothing with the GPU
 * library.
 *
 * A = L D L^T with L unit lower triangular and D diagonal, transposes taken
 * without conjugation (A^T = A for the shifted matrices K - xi M of Section 3.1).
 * No pivoting: for Re(xi) < 0 the real part K - Re(xi) M is positive definite,
 * so every leading principal submatrix is nonsingular.
 *
 * Method: the up-looking sparse LDL^T of T. A. Davis, "Algorithm 849: A concise
 * sparse Cholesky factorization package", ACM Trans. Math. Softw. 31(4), 2005
 * (elimination tree, column counts, then a row-by-row numeric phase), restated
 * here for complex symmetric matrices with transposes taken without conjugation.
 *
 * The factorisation goes row by row.  Row k of L is found by a sparse
 * triangular solve L(0:k,0:k) D y = A(0:k,k), whose pattern is the set of
 * elimination-tree ancestors reachable from the nonzeros of A(0:k,k).
 * Input: the upper triangle of the (already permuted) matrix in compressed
 * columns (column k holds rows i <= k).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>

typedef double complex cplx;

/* Elimination tree and column counts of L. */
int64_t ldl_symbolic(int64_t n, const int64_t *Ap, const int64_t *Ai,
                     int64_t *Lp, int64_t *parent, int64_t *lnz, int64_t *flag) {
  for (int64_t k = 0; k < n; k++) {
    parent[k] = -1;
    flag[k] = k;
    lnz[k] = 0;
    for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
      int64_t i = Ai[p];
      if (i >= k) continue;
      for (; flag[i] != k; i = parent[i]) {
        if (parent[i] == -1) parent[i] = k;
        lnz[i]++;
        flag[i] = k;
      }
    }
  }
  Lp[0] = 0;
  for (int64_t k = 0; k < n; k++) Lp[k + 1] = Lp[k] + lnz[k];
  return Lp[n];
}

/* Numeric factorisation.  Returns n on success, or the index of the first
 * zero pivot. */
int64_t ldl_numeric(int64_t n, const int64_t *Ap, const int64_t *Ai, const cplx *Ax,
                    const int64_t *Lp, const int64_t *parent, int64_t *lnz,
                    int64_t *Li, cplx *Lx, cplx *D) {
  cplx *Y = (cplx *)calloc((size_t)n, sizeof(cplx));
  int64_t *pattern = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *flag = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t status = n;
  for (int64_t k = 0; k < n; k++) {
    Y[k] = 0.0;
    int64_t top = n;
    flag[k] = k;
    lnz[k] = 0;
    for (int64_t p = Ap[k]; p < Ap[k + 1]; p++) {
      int64_t i = Ai[p];
      if (i > k) continue;
      Y[i] += Ax[p];
      int64_t len = 0;
      for (; flag[i] != k; i = parent[i]) {
        pattern[len++] = i;
        flag[i] = k;
      }
      while (len > 0) pattern[--top] = pattern[--len];
    }
    D[k] = Y[k];
    Y[k] = 0.0;
    for (; top < n; top++) {
      int64_t i = pattern[top];
      cplx yi = Y[i];
      Y[i] = 0.0;
      int64_t p2 = Lp[i] + lnz[i];
      for (int64_t p = Lp[i]; p < p2; p++) Y[Li[p]] -= Lx[p] * yi;
      cplx lki = yi / D[i];
      D[k] -= lki * yi;
      Li[p2] = k;
      Lx[p2] = lki;
      lnz[i]++;
    }
    if (D[k] == 0.0) {
      status = k;
      break;
    }
  }
  free(Y);
  free(pattern);
  free(flag);
  return status;
}

/* Solve L D L^T X = B in place for nrhs columns (column-major, leading dim n). */
void ldl_solve(int64_t n, int64_t nrhs, const int64_t *Lp, const int64_t *Li,
               const cplx *Lx, const cplx *D, cplx *X) {
  for (int64_t c = 0; c < nrhs; c++) {
    cplx *x = X + c * n;
    for (int64_t j = 0; j < n; j++) {
      cplx xj = x[j];
      for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) x[Li[p]] -= Lx[p] * xj;
    }
    for (int64_t j = 0; j < n; j++) x[j] /= D[j];
    for (int64_t j = n - 1; j >= 0; j--) {
      cplx s = x[j];
      for (int64_t p = Lp[j]; p < Lp[j + 1]; p++) s -= Lx[p] * x[Li[p]];
      x[j] = s;
    }
  }
}
