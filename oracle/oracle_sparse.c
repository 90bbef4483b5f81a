/*
 * Oracle, part 2: sparse helpers, block splitting, decoupling and the SIMPLE
 * approximate Schur complement. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Arithmetic order (stated so another implementation can reproduce the
 * results bit for bit): every sum runs in ascending column (or inner-index)
 * order and the first term of a sum is taken as the rounded product itself
 * (no 0 + x). In the sparse products (or_spgemm and the product inside
 * or_simple_schur) every later term is accumulated by a fused multiply-add,
 * acc = fma(a, b, acc), one rounding per term; elsewhere each product is
 * rounded before it is added.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static void *xmalloc(size_t n) {
  void *p = malloc(n ? n : 1);
  if (!p) abort();
  return p;
}

or_csr *or_csr_alloc(int32_t n, int32_t m, int32_t nnz) {
  or_csr *A = xmalloc(sizeof(or_csr));
  A->n = n;
  A->m = m;
  A->nnz = nnz;
  A->rowptr = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  A->col = xmalloc(sizeof(int32_t) * (size_t)nnz);
  A->val = xmalloc(sizeof(double) * (size_t)nnz);
  return A;
}

or_csr *or_csr_new(int32_t n, int32_t m, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                   const double *val) {
  or_csr *A = or_csr_alloc(n, m, nnz);
  memcpy(A->rowptr, rowptr, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(A->col, col, sizeof(int32_t) * (size_t)nnz);
  memcpy(A->val, val, sizeof(double) * (size_t)nnz);
  return A;
}

void or_csr_free(or_csr *A) {
  if (!A) return;
  free(A->rowptr);
  free(A->col);
  free(A->val);
  free(A);
}

void or_csr_info(const or_csr *A, int32_t *o) {
  o[0] = A->n;
  o[1] = A->m;
  o[2] = A->nnz;
}

void or_csr_copy(const or_csr *A, int32_t *rowptr, int32_t *col, double *val) {
  memcpy(rowptr, A->rowptr, sizeof(int32_t) * ((size_t)A->n + 1));
  memcpy(col, A->col, sizeof(int32_t) * (size_t)A->nnz);
  memcpy(val, A->val, sizeof(double) * (size_t)A->nnz);
}

void or_csr_spmv(const or_csr *A, const double *x, double *y) {
  for (int32_t i = 0; i < A->n; i++) {
    double s = 0.0;
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) s += A->val[k] * x[A->col[k]];
    y[i] = s;
  }
}

/* Point-ordered scalar view of a 2x2 block matrix (Sec. 3.2, the "point"
 * ordering): unknown 2i is P_w of cell i, 2i+1 is S_n. */
or_csr *or_scalar_from_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val) {
  int32_t nnzb = rowptr[nb];
  or_csr *A = or_csr_alloc(2 * nb, 2 * nb, 4 * nnzb);
  int32_t pos = 0;
  A->rowptr[0] = 0;
  for (int32_t i = 0; i < nb; i++) {
    for (int r = 0; r < 2; r++) {
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
        for (int c = 0; c < 2; c++) {
          A->col[pos] = 2 * col[k] + c;
          A->val[pos] = val[4 * (size_t)k + 2 * r + c];
          pos++;
        }
      }
      A->rowptr[2 * i + r + 1] = pos;
    }
  }
  return A;
}

/* One scalar block of J (eq. jacobian): (r,c) = (0,0) A_pp, (0,1) A_ps,
 * (1,0) A_sp, (1,1) A_ss. Keeps J's block pattern, structural zeros included. */
or_csr *or_bsr2_part(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, int32_t r,
                     int32_t c) {
  int32_t nnzb = rowptr[nb];
  or_csr *A = or_csr_alloc(nb, nb, nnzb);
  memcpy(A->rowptr, rowptr, sizeof(int32_t) * ((size_t)nb + 1));
  memcpy(A->col, col, sizeof(int32_t) * (size_t)nnzb);
  for (int32_t k = 0; k < nnzb; k++) A->val[k] = val[4 * (size_t)k + 2 * r + c];
  return A;
}

/* Inverse of a 2x2 block [a b; c d]: [d -b; -c a] / (a d - b c). */
static void inv2(const double *m, double *o) {
  double ad = m[0] * m[3], bc = m[1] * m[2];
  double det = ad - bc;
  o[0] = m[3] / det;
  o[1] = -(m[1] / det);
  o[2] = -(m[2] / det);
  o[3] = m[0] / det;
}

/* 2x2 product o = x y, each entry x_r0 y_0c + x_r1 y_1c. */
static void mul2(const double *x, const double *y, double *o) {
  for (int r = 0; r < 2; r++)
    for (int c = 0; c < 2; c++) {
      double t0 = x[2 * r] * y[c];
      double t1 = x[2 * r + 1] * y[2 + c];
      o[2 * r + c] = t0 + t1;
    }
}

/* D^{-1} J with D the per-cell 2x2 diagonal block: the IMPES-type operator
 * D = [diag A_pp, diag A_ps; diag A_sp, diag A_ss] of Sec. 3.1 applied as a
 * left scaling (alternate block factorisation). A zero-determinant diagonal
 * block leaves its block row unscaled. */
void or_decouple_abf(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *out) {
  for (int32_t i = 0; i < nb; i++) {
    const double *dblk = NULL;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
      if (col[k] == i) dblk = val + 4 * (size_t)k;
    double di[4];
    int ok = 0;
    if (dblk) {
      double ad = dblk[0] * dblk[3], bc = dblk[1] * dblk[2];
      ok = (ad - bc) != 0.0;
      if (ok) inv2(dblk, di);
    }
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      if (ok) mul2(di, val + 4 * (size_t)k, out + 4 * (size_t)k);
      else memcpy(out + 4 * (size_t)k, val + 4 * (size_t)k, 4 * sizeof(double));
    }
  }
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* C = A B, Gustavson row by row. For each (i, j) the terms a_ik b_kj are
 * added in ascending k; the first term (rounded) initialises the sum, every
 * later one is fused into it (fma). The pattern is every (i, j) reached by
 * some product, zeros included. */
or_csr *or_spgemm(const or_csr *A, const or_csr *B) {
  int32_t n = A->n, m = B->m;
  int32_t *mark = xmalloc(sizeof(int32_t) * (size_t)m);
  double *acc = xmalloc(sizeof(double) * (size_t)m);
  for (int32_t j = 0; j < m; j++) mark[j] = -1;
  /* symbolic */
  int64_t tot = 0;
  for (int32_t i = 0; i < n; i++) {
    for (int32_t ka = A->rowptr[i]; ka < A->rowptr[i + 1]; ka++) {
      int32_t k = A->col[ka];
      for (int32_t kb = B->rowptr[k]; kb < B->rowptr[k + 1]; kb++) {
        int32_t j = B->col[kb];
        if (mark[j] != i) { mark[j] = i; tot++; }
      }
    }
  }
  or_csr *C = or_csr_alloc(n, m, (int32_t)tot);
  for (int32_t j = 0; j < m; j++) mark[j] = -1;
  int32_t pos = 0;
  C->rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t start = pos;
    for (int32_t ka = A->rowptr[i]; ka < A->rowptr[i + 1]; ka++) {
      int32_t k = A->col[ka];
      double a = A->val[ka];
      for (int32_t kb = B->rowptr[k]; kb < B->rowptr[k + 1]; kb++) {
        int32_t j = B->col[kb];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = a * B->val[kb];
          C->col[pos++] = j;
        } else {
          acc[j] = fma(a, B->val[kb], acc[j]);
        }
      }
    }
    qsort(C->col + start, (size_t)(pos - start), sizeof(int32_t), cmp_i32);
    for (int32_t q = start; q < pos; q++) C->val[q] = acc[C->col[q]];
    C->rowptr[i + 1] = pos;
  }
  free(mark);
  free(acc);
  return C;
}

/* Transpose; row J of the result lists the rows i of A in ascending order. */
or_csr *or_transpose(const or_csr *A) {
  or_csr *T = or_csr_alloc(A->m, A->n, A->nnz);
  memset(T->rowptr, 0, sizeof(int32_t) * ((size_t)A->m + 1));
  for (int32_t k = 0; k < A->nnz; k++) T->rowptr[A->col[k] + 1]++;
  for (int32_t j = 0; j < A->m; j++) T->rowptr[j + 1] += T->rowptr[j];
  int32_t *fill = xmalloc(sizeof(int32_t) * (size_t)A->m);
  memcpy(fill, T->rowptr, sizeof(int32_t) * (size_t)A->m);
  for (int32_t i = 0; i < A->n; i++)
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      int32_t q = fill[A->col[k]]++;
      T->col[q] = i;
      T->val[q] = A->val[k];
    }
  free(fill);
  return T;
}

/* SIMPLE-type Schur complement (Sec. 3.4, eq. SIMPLE-Schur), read with A_sp
 * in the last factor:  S~ = A_pp - A_ps diag(A_ss)^{-1} A_sp.
 * Row i: for each k of A_ps(i,:) ascending, t = a_ps(i,k) / d_ss(k); for each
 * j of A_sp(k,:) ascending, acc_j gets t * a_sp(k,j) (the rounded product
 * initialises, later terms are fused in: acc_j = fma(t, a_sp(k,j), acc_j)).
 * The pattern is the union of A_pp's and the product's; entry = a_pp - acc
 * with a missing operand read as 0. A zero d_ss(k) skips column k. */
or_csr *or_simple_schur(const or_csr *App, const or_csr *Aps, const or_csr *Asp, const or_csr *Ass) {
  int32_t n = App->n;
  double *dss = xmalloc(sizeof(double) * (size_t)n);
  for (int32_t i = 0; i < n; i++) {
    dss[i] = 0.0;
    for (int32_t k = Ass->rowptr[i]; k < Ass->rowptr[i + 1]; k++)
      if (Ass->col[k] == i) dss[i] = Ass->val[k];
  }
  int32_t *mark = xmalloc(sizeof(int32_t) * (size_t)n);
  int8_t *has = xmalloc((size_t)n);
  double *acc = xmalloc(sizeof(double) * (size_t)n);
  double *app = xmalloc(sizeof(double) * (size_t)n);
  int32_t *cols = xmalloc(sizeof(int32_t) * (size_t)n);
  for (int32_t j = 0; j < n; j++) mark[j] = -1;
  /* first pass: count */
  int64_t tot = 0;
  for (int32_t i = 0; i < n; i++) {
    for (int32_t k = App->rowptr[i]; k < App->rowptr[i + 1]; k++)
      if (mark[App->col[k]] != i) { mark[App->col[k]] = i; tot++; }
    for (int32_t ka = Aps->rowptr[i]; ka < Aps->rowptr[i + 1]; ka++) {
      int32_t k = Aps->col[ka];
      if (dss[k] == 0.0) continue;
      for (int32_t kb = Asp->rowptr[k]; kb < Asp->rowptr[k + 1]; kb++)
        if (mark[Asp->col[kb]] != i) { mark[Asp->col[kb]] = i; tot++; }
    }
  }
  or_csr *S = or_csr_alloc(n, n, (int32_t)tot);
  for (int32_t j = 0; j < n; j++) mark[j] = -1;
  int32_t pos = 0;
  S->rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t cnt = 0;
    for (int32_t k = App->rowptr[i]; k < App->rowptr[i + 1]; k++) {
      int32_t j = App->col[k];
      if (mark[j] != i) { mark[j] = i; has[j] = 0; app[j] = 0.0; cols[cnt++] = j; }
      app[j] = App->val[k];
    }
    for (int32_t ka = Aps->rowptr[i]; ka < Aps->rowptr[i + 1]; ka++) {
      int32_t k = Aps->col[ka];
      if (dss[k] == 0.0) continue;
      double t = Aps->val[ka] / dss[k];
      for (int32_t kb = Asp->rowptr[k]; kb < Asp->rowptr[k + 1]; kb++) {
        int32_t j = Asp->col[kb];
        if (mark[j] != i) { mark[j] = i; has[j] = 0; app[j] = 0.0; cols[cnt++] = j; }
        if (!has[j]) { acc[j] = t * Asp->val[kb]; has[j] = 1; }
        else acc[j] = fma(t, Asp->val[kb], acc[j]);
      }
    }
    qsort(cols, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int32_t q = 0; q < cnt; q++) {
      int32_t j = cols[q];
      S->col[pos] = j;
      S->val[pos] = has[j] ? app[j] - acc[j] : app[j];
      pos++;
    }
    S->rowptr[i + 1] = pos;
  }
  free(dss); free(mark); free(has); free(acc); free(app); free(cols);
  return S;
}

/* Quasi-IMPES decoupling (Lacroix et al. 2003, named in Sec. 3.1 next to the
 * IMPES-type operator): in every block row the water equation gets
 * w_i = -(a_ps,ii / a_ss,ii) times the oil equation added to it,
 * row0 <- row0 + w_i row1, so the pressure equation loses the saturation
 * derivative of its own cell. Entry order: w = -(a_ps / a_ss); new = r0 + w r1.
 * A zero a_ss,ii leaves the row unchanged. Writes the weights to w_out. */
void or_decouple_qimpes(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                        double *out, double *w_out) {
  for (int32_t i = 0; i < nb; i++) {
    double w = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
      if (col[k] == i && val[4 * (size_t)k + 3] != 0.0) w = -(val[4 * (size_t)k + 1] / val[4 * (size_t)k + 3]);
    w_out[i] = w;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      const double *b = val + 4 * (size_t)k;
      double *o = out + 4 * (size_t)k;
      o[0] = b[0] + w * b[2];
      o[1] = b[1] + w * b[3];
      o[2] = b[2];
      o[3] = b[3];
    }
  }
}
