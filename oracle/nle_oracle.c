/*
 * Oracle (test infrastructure only): plain, slow FP64 reference of the sparse
 * building blocks of the DACG-Newton eigensolver of Bergamaschi & Martinez,
 * "Efficiently preconditioned Inexact Newton methods for large symmetric
 * eigenvalue problems".  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file; the CUDA library shares no code with it.
 *
 * Contents
 *   orc_ict      IC(lfil, tau_IC) incomplete Cholesky factor of A
 *                (Section 2, the initial preconditioner P0 = (L L^T)^{-1}).
 *   orc_levels   level of every row of a triangular factor (longest chain of
 *                dependencies), used to schedule the triangular solves.
 *   orc_spmv     y = A x for CSR A (the "MV product", Section 5).
 *   orc_lsolve   solve L y = b (L lower triangular, CSR, diagonal last).
 *   orc_usolve   solve U y = b (U upper triangular, CSR, diagonal first).
 *
 * The paper fixes neither the IC variant nor the meaning of lfil precisely
 * (it cites Saad's dual-threshold idea).  The reading implemented here:
 *   - left-looking, column by column, j = 0..n-1;
 *   - w = lower part of column j of A (A is symmetric, so this is row j of
 *     the CSR restricted to columns >= j);
 *   - for every k < j with L(j,k) != 0, in ascending k, and for every row
 *     i >= j of column k: w[i] -= L(i,k) * L(j,k);
 *   - pivot d = w[j]; d <= 0 is a breakdown (return -2);
 *   - L(j,j) = sqrt(d), L(i,j) = w[i] / L(j,j) for the touched rows i > j;
 *   - an off-diagonal is dropped when |L(i,j)| < tau * ||A(:,j)||_2, the norm
 *     summed in ascending column order of row j of A;
 *   - of the survivors the lfil largest |L(i,j)| are kept, ties going to the
 *     smaller row index; kept entries are stored by ascending row.
 * Compile with -ffp-contract=off: the drop decisions depend on every
 * rounding, and no multiply-add may be fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t i;
  double v;
  double a;
} cand_t;

/* Order by |value| descending, then row ascending. */
static int cand_cmp(const void *x, const void *y) {
  const cand_t *p = (const cand_t *)x, *q = (const cand_t *)y;
  if (p->a > q->a) return -1;
  if (p->a < q->a) return 1;
  return (p->i < q->i) ? -1 : (p->i > q->i);
}

static int row_cmp(const void *x, const void *y) {
  const cand_t *p = (const cand_t *)x, *q = (const cand_t *)y;
  return (p->i < q->i) ? -1 : (p->i > q->i);
}

/*
 * IC(lfil, tau) of the symmetric CSR matrix (rowptr, col, val).
 * Output U = L^T in CSR: row j holds column j of L, diagonal first, then the
 * kept rows i > j ascending.  cap is the capacity of Ucol/Uval; on success
 * *nnzU receives the number of stored entries.
 * Returns 0 on success, -1 if cap is too small, -2 on a non-positive pivot
 * (its column in *bad_col), -3 on allocation failure.
 */
int orc_ict(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, int lfil,
            double tau, int64_t cap, int64_t *Urowptr, int32_t *Ucol, double *Uval, int64_t *nnzU,
            int64_t *bad_col) {
  double *w = (double *)calloc((size_t)n, sizeof(double));
  char *touched = (char *)calloc((size_t)n, 1);
  int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  cand_t *cand = (cand_t *)malloc(sizeof(cand_t) * (size_t)n);
  /* rows of L built so far: for row i, the columns k with L(i,k) != 0 and
     their values, as a singly linked list in ascending k */
  int64_t *rhead = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *rtail = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *rnext = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
  int64_t *rcol = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap > 0 ? cap : 1));
  double *rval = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
  int rc = 0;
  if (!w || !touched || !list || !cand || !rhead || !rtail || !rnext || !rcol || !rval) {
    rc = -3;
    goto done;
  }
  for (int64_t i = 0; i < n; i++) rhead[i] = rtail[i] = -1;
  int64_t nr = 0, pos = 0;
  Urowptr[0] = 0;
  for (int64_t j = 0; j < n; j++) {
    int64_t nt = 0;
    double nrm2 = 0.0;
    /* lower part of column j of A, and the column norm */
    for (int64_t e = rowptr[j]; e < rowptr[j + 1]; e++) {
      int64_t i = col[e];
      nrm2 += val[e] * val[e];
      if (i >= j) {
        if (!touched[i]) {
          touched[i] = 1;
          list[nt++] = i;
        }
        w[i] += val[e];
      }
    }
    double anorm = sqrt(nrm2);
    /* left-looking updates with every earlier column k having L(j,k) != 0 */
    for (int64_t t = rhead[j]; t >= 0; t = rnext[t]) {
      int64_t k = rcol[t];
      double ljk = rval[t];
      for (int64_t e = Urowptr[k]; e < Urowptr[k + 1]; e++) {
        int64_t i = Ucol[e];
        if (i < j) continue;
        if (!touched[i]) {
          touched[i] = 1;
          list[nt++] = i;
        }
        w[i] -= Uval[e] * ljk;
      }
    }
    double d = w[j];
    if (!(d > 0.0)) {
      if (bad_col) *bad_col = j;
      rc = -2;
      for (int64_t t = 0; t < nt; t++) {
        w[list[t]] = 0.0;
        touched[list[t]] = 0;
      }
      goto done;
    }
    double ljj = sqrt(d);
    int64_t nc = 0;
    for (int64_t t = 0; t < nt; t++) {
      int64_t i = list[t];
      if (i != j) {
        double lij = w[i] / ljj;
        if (!(fabs(lij) < tau * anorm)) {
          cand[nc].i = i;
          cand[nc].v = lij;
          cand[nc].a = fabs(lij);
          nc++;
        }
      }
      w[i] = 0.0;
      touched[i] = 0;
    }
    if (nc > lfil) {
      qsort(cand, (size_t)nc, sizeof(cand_t), cand_cmp);
      nc = lfil;
    }
    qsort(cand, (size_t)nc, sizeof(cand_t), row_cmp);
    if (pos + 1 + nc > cap) {
      rc = -1;
      goto done;
    }
    Ucol[pos] = (int32_t)j;
    Uval[pos] = ljj;
    pos++;
    for (int64_t t = 0; t < nc; t++) {
      Ucol[pos] = (int32_t)cand[t].i;
      Uval[pos] = cand[t].v;
      pos++;
      /* append (j, L(i,j)) to row i */
      int64_t i = cand[t].i;
      rcol[nr] = j;
      rval[nr] = cand[t].v;
      rnext[nr] = -1;
      if (rtail[i] < 0)
        rhead[i] = nr;
      else
        rnext[rtail[i]] = nr;
      rtail[i] = nr;
      nr++;
    }
    Urowptr[j + 1] = pos;
  }
  *nnzU = pos;
done:
  free(w);
  free(touched);
  free(list);
  free(cand);
  free(rhead);
  free(rtail);
  free(rnext);
  free(rcol);
  free(rval);
  return rc;
}

/* Transpose of an n x n CSR matrix; columns of the result come out sorted. */
void orc_transpose(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   int64_t *trowptr, int32_t *tcol, double *tval) {
  for (int64_t i = 0; i <= n; i++) trowptr[i] = 0;
  for (int64_t e = 0; e < rowptr[n]; e++) trowptr[col[e] + 1]++;
  for (int64_t i = 0; i < n; i++) trowptr[i + 1] += trowptr[i];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; i++) fill[i] = trowptr[i];
  for (int64_t i = 0; i < n; i++)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
      int64_t c = col[e];
      tcol[fill[c]] = (int32_t)i;
      tval[fill[c]] = val[e];
      fill[c]++;
    }
  free(fill);
}

/*
 * Level of every row of a triangular CSR factor.  lower != 0: row i depends
 * on the columns j < i of its row and lev(i) = 1 + max lev(j) (0 when it has
 * none); lower == 0: dependencies are the columns j > i, computed from the
 * last row upwards.  Returns the number of levels.
 */
int64_t orc_levels(int64_t n, const int64_t *rowptr, const int32_t *col, int lower, int32_t *lev) {
  int64_t nlev = 0;
  for (int64_t s = 0; s < n; s++) {
    int64_t i = lower ? s : n - 1 - s;
    int32_t l = 0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
      int64_t j = col[e];
      if ((lower && j < i) || (!lower && j > i))
        if (lev[j] + 1 > l) l = lev[j] + 1;
    }
    lev[i] = l;
    if (l + 1 > nlev) nlev = l + 1;
  }
  return nlev;
}

/* Rows listed level by level, ascending row within a level. */
void orc_level_sets(int64_t n, const int32_t *lev, int64_t nlev, int64_t *lptr, int32_t *rows) {
  for (int64_t l = 0; l <= nlev; l++) lptr[l] = 0;
  for (int64_t i = 0; i < n; i++) lptr[lev[i] + 1]++;
  for (int64_t l = 0; l < nlev; l++) lptr[l + 1] += lptr[l];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nlev > 0 ? nlev : 1));
  for (int64_t l = 0; l < nlev; l++) fill[l] = lptr[l];
  for (int64_t i = 0; i < n; i++) rows[fill[lev[i]]++] = (int32_t)i;
  free(fill);
}

/* y = A x */
void orc_spmv(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, const double *x,
              double *y) {
  for (int64_t i = 0; i < n; i++) {
    double acc = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) acc += val[e] * x[col[e]];
    y[i] = acc;
  }
}

/* Forward substitution L y = b; L lower triangular CSR with the diagonal as
   the last entry of each row. */
void orc_lsolve(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, const double *b,
                double *y) {
  for (int64_t i = 0; i < n; i++) {
    double acc = b[i];
    int64_t e1 = rowptr[i + 1] - 1;
    for (int64_t e = rowptr[i]; e < e1; e++) acc -= val[e] * y[col[e]];
    y[i] = acc / val[e1];
  }
}

/* Back substitution U y = b; U upper triangular CSR with the diagonal as the
   first entry of each row. */
void orc_usolve(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, const double *b,
                double *y) {
  for (int64_t i = n - 1; i >= 0; i--) {
    double acc = b[i];
    int64_t e0 = rowptr[i];
    for (int64_t e = e0 + 1; e < rowptr[i + 1]; e++) acc -= val[e] * y[col[e]];
    y[i] = acc / val[e0];
  }
}
