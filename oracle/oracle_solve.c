/*
 * Oracle, part 4: the four preconditioners (Sec. 3.2-3.4), right-preconditioned
 * flexible GMRES (Sec. 3, eq. precon-system) and Newton's method (Sec. 3).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 *  AMG_J : one V-cycle of scalar AMG on the point-ordered J (Sec. 3.2).
 *  CPR1  : Algorithm 1. u = P1^{-1} r; r' = r - J u; A_pp dp = R_p r' by one
 *          V-cycle; u += R_p^T dp.
 *  CPR2  : Algorithm 2: as CPR1 plus A_ss ds = R_s r' by one V-cycle,
 *          u += R_s^T ds, both corrections from the same r'.
 *  BF    : Algorithm 3. A_ss s = R_s r by one V-cycle; r_p = R_p r - A_ps s;
 *          S~ p = r_p by one V-cycle with S~ the SIMPLE Schur complement.
 *  For CPR, `decouple` = 1 applies everything to D^{-1} J and D^{-1} r with D
 *  the per-cell 2x2 diagonal block (the IMPES-type operator of Sec. 3.1).
 *  P1 is the point-block Jacobi inverse (p1 = 0) or ILU(0) of the
 *  point-ordered matrix (p1 = 1, the paper's choice in Sec. 3.3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

or_csr *or_csr_alloc(int32_t n, int32_t m, int32_t nnz);

static void *xmalloc(size_t n) {
  void *p = malloc(n ? n : 1);
  if (!p) abort();
  return p;
}

struct or_precond {
  or_precond_params prm;
  int32_t nb;
  int32_t *rowptr, *col;
  double *Jt;          /* matrix the preconditioner works on (J or D^{-1} J) */
  double *Dinv;        /* per-cell inverse diagonal block used for decoupling */
  double *qw;          /* quasi-IMPES weights */
  double *P1inv;       /* per-cell inverse of Jt's diagonal block (point-block Jacobi) */
  or_csr *ilu;         /* ILU(0) factors on the point-ordered Jt */
  int32_t *ilu_diag;
  or_amg *Hp, *Hs, *Hj;
  or_csr *Aps;
};

static void inv2(const double *m, double *o) {
  double ad = m[0] * m[3], bc = m[1] * m[2];
  double det = ad - bc;
  if (det == 0.0) { o[0] = 1; o[1] = 0; o[2] = 0; o[3] = 1; return; }
  o[0] = m[3] / det;
  o[1] = -(m[1] / det);
  o[2] = -(m[2] / det);
  o[3] = m[0] / det;
}

static void diag_inverses(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *out) {
  for (int32_t i = 0; i < nb; i++) {
    double z[4] = {0, 0, 0, 0};
    const double *d = z;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
      if (col[k] == i) d = val + 4 * (size_t)k;
    inv2(d, out + 4 * (size_t)i);
  }
}

/* ILU(0) of a scalar CSR in place (IKJ form, pattern of A only). */
static void ilu0(or_csr *A, int32_t *dpos) {
  int32_t n = A->n;
  int32_t *where = xmalloc(sizeof(int32_t) * (size_t)n);
  for (int32_t j = 0; j < n; j++) where[j] = -1;
  for (int32_t i = 0; i < n; i++) {
    dpos[i] = -1;
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      where[A->col[q]] = q;
      if (A->col[q] == i) dpos[i] = q;
    }
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t k = A->col[q];
      if (k >= i) break;
      double dk = A->val[dpos[k]];
      if (dk == 0.0) continue;
      A->val[q] = A->val[q] / dk;
      double l = A->val[q];
      for (int32_t t = dpos[k] + 1; t < A->rowptr[k + 1]; t++) {
        int32_t j = A->col[t];
        if (where[j] >= 0) A->val[where[j]] -= l * A->val[t];
      }
    }
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) where[A->col[q]] = -1;
  }
  free(where);
}

static void ilu0_solve(const or_csr *A, const int32_t *dpos, const double *b, double *x) {
  int32_t n = A->n;
  for (int32_t i = 0; i < n; i++) {
    double s = b[i];
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1] && A->col[q] < i; q++) s -= A->val[q] * x[A->col[q]];
    x[i] = s;
  }
  for (int32_t i = n - 1; i >= 0; i--) {
    double s = x[i];
    for (int32_t q = dpos[i] + 1; q < A->rowptr[i + 1]; q++) s -= A->val[q] * x[A->col[q]];
    double d = A->val[dpos[i]];
    x[i] = d != 0.0 ? s / d : s;
  }
}

/* ILU(0) of the point-ordered scalar matrix of a 2x2-block matrix (the
 * paper's P1, Sec. 3.3), its factors returned in the block layout:
 * lu[4k + 2r + cc] is the factor entry of scalar row 2i+r, column
 * 2 col[k] + cc (L strictly lower with unit diagonal, U upper). */
void or_ilu0_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *lu) {
  or_csr *A = or_scalar_from_bsr2(nb, rowptr, col, val);
  int32_t *dpos = xmalloc(sizeof(int32_t) * (size_t)(2 * nb + 1));
  ilu0(A, dpos);
  for (int32_t i = 0; i < nb; i++)
    for (int r = 0; r < 2; r++) {
      int32_t q = A->rowptr[2 * i + r];
      for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
        for (int c = 0; c < 2; c++) lu[4 * (size_t)k + 2 * r + c] = A->val[q++];
    }
  free(dpos);
  or_csr_free(A);
}

/* x = (L U)^{-1} b with the factors of or_ilu0_bsr2. */
void or_ilu0_solve_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *lu, const double *b,
                        double *x) {
  or_csr *A = or_scalar_from_bsr2(nb, rowptr, col, lu);
  int32_t *dpos = xmalloc(sizeof(int32_t) * (size_t)(2 * nb + 1));
  for (int32_t i = 0; i < 2 * nb; i++) {
    dpos[i] = -1;
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++)
      if (A->col[q] == i) dpos[i] = q;
  }
  ilu0_solve(A, dpos, b, x);
  free(dpos);
  or_csr_free(A);
}

or_precond *or_precond_create(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                              const or_precond_params *prm) {
  or_precond *M = xmalloc(sizeof(or_precond));
  memset(M, 0, sizeof(or_precond));
  M->prm = *prm;
  M->nb = nb;
  int32_t nnzb = rowptr[nb];
  M->rowptr = xmalloc(sizeof(int32_t) * ((size_t)nb + 1));
  M->col = xmalloc(sizeof(int32_t) * ((size_t)nnzb + 1));
  M->Jt = xmalloc(sizeof(double) * 4 * ((size_t)nnzb + 1));
  memcpy(M->rowptr, rowptr, sizeof(int32_t) * ((size_t)nb + 1));
  memcpy(M->col, col, sizeof(int32_t) * (size_t)nnzb);
  int cpr = prm->kind == OR_CPR1 || prm->kind == OR_CPR2;
  if (cpr && prm->decouple == 1) {
    M->Dinv = xmalloc(sizeof(double) * 4 * ((size_t)nb + 1));
    diag_inverses(nb, rowptr, col, val, M->Dinv);
    or_decouple_abf(nb, rowptr, col, val, M->Jt);
  } else if (cpr && prm->decouple == 2) {
    M->qw = xmalloc(sizeof(double) * ((size_t)nb + 1));
    or_decouple_qimpes(nb, rowptr, col, val, M->Jt, M->qw);
  } else {
    memcpy(M->Jt, val, sizeof(double) * 4 * (size_t)nnzb);
  }
  if (prm->kind == OR_AMG_J || prm->kind == OR_AMG_J_SCALAR) {
    /* black-box AMG on the point-ordered J (Sec. 3.2): the point method with
     * (p_w, S_n) per cell, or unknown-agnostic scalar AMG */
    or_csr *A = or_scalar_from_bsr2(nb, rowptr, col, val);
    or_amg_params ap = prm->amg;
    ap.num_functions = prm->kind == OR_AMG_J ? 2 : 1;
    M->Hj = or_amg_setup(A, &ap);
    or_csr_free(A);
  } else if (cpr) {
    if (prm->p1 == 1) {
      M->ilu = or_scalar_from_bsr2(nb, rowptr, col, M->Jt);
      M->ilu_diag = xmalloc(sizeof(int32_t) * (size_t)(2 * nb + 1));
      ilu0(M->ilu, M->ilu_diag);
    } else {
      M->P1inv = xmalloc(sizeof(double) * 4 * ((size_t)nb + 1));
      diag_inverses(nb, rowptr, col, M->Jt, M->P1inv);
    }
    or_csr *App = or_bsr2_part(nb, rowptr, col, M->Jt, 0, 0);
    M->Hp = or_amg_setup(App, &prm->amg);
    or_csr_free(App);
    if (prm->kind == OR_CPR2) {
      or_csr *Ass = or_bsr2_part(nb, rowptr, col, M->Jt, 1, 1);
      M->Hs = or_amg_setup(Ass, &prm->amg);
      or_csr_free(Ass);
    }
  } else {
    or_csr *App = or_bsr2_part(nb, rowptr, col, val, 0, 0);
    or_csr *Aps = or_bsr2_part(nb, rowptr, col, val, 0, 1);
    or_csr *Asp = or_bsr2_part(nb, rowptr, col, val, 1, 0);
    or_csr *Ass = or_bsr2_part(nb, rowptr, col, val, 1, 1);
    or_csr *S = or_simple_schur(App, Aps, Asp, Ass);
    M->Hs = or_amg_setup(Ass, &prm->amg);
    M->Hp = or_amg_setup(S, &prm->amg);
    M->Aps = Aps;
    or_csr_free(App); or_csr_free(Asp); or_csr_free(Ass); or_csr_free(S);
  }
  return M;
}

void or_precond_free(or_precond *M) {
  if (!M) return;
  free(M->rowptr); free(M->col); free(M->Jt); free(M->Dinv); free(M->qw); free(M->P1inv);
  or_csr_free(M->ilu); free(M->ilu_diag);
  or_amg_free(M->Hp); or_amg_free(M->Hs); or_amg_free(M->Hj);
  or_csr_free(M->Aps);
  free(M);
}

const or_amg *or_precond_amg(const or_precond *M, int32_t which) {
  if (which == 0) return M->Hj ? M->Hj : M->Hp;
  return M->Hs;
}

static void apply2(const double *m, const double *x, double *y) {
  double a = m[0] * x[0] + m[1] * x[1];
  double b = m[2] * x[0] + m[3] * x[1];
  y[0] = a;
  y[1] = b;
}

void or_precond_apply(const or_precond *M, const double *r, double *z) {
  int32_t nb = M->nb, n = 2 * nb;
  if (M->prm.kind == OR_AMG_J || M->prm.kind == OR_AMG_J_SCALAR) {
    or_amg_vcycle(M->Hj, r, z);
    return;
  }
  double *tmp = xmalloc(sizeof(double) * (size_t)n);
  double *sb = xmalloc(sizeof(double) * (size_t)nb);
  double *sx = xmalloc(sizeof(double) * (size_t)nb);
  if (M->prm.kind == OR_BF) {
    for (int32_t i = 0; i < nb; i++) sb[i] = r[2 * i + 1];
    or_amg_vcycle(M->Hs, sb, sx);                        /* A_ss s = R_s r */
    double *ps = xmalloc(sizeof(double) * (size_t)nb);
    or_csr_spmv(M->Aps, sx, ps);
    for (int32_t i = 0; i < nb; i++) sb[i] = r[2 * i] - ps[i];   /* r_p = R_p r - A_ps s */
    double *px = xmalloc(sizeof(double) * (size_t)nb);
    or_amg_vcycle(M->Hp, sb, px);                        /* S~ p = r_p */
    for (int32_t i = 0; i < nb; i++) { z[2 * i] = px[i]; z[2 * i + 1] = sx[i]; }
    free(ps); free(px);
  } else {
    const double *rt = r;
    double *rd = NULL;
    if (M->Dinv) {
      rd = xmalloc(sizeof(double) * (size_t)n);
      for (int32_t i = 0; i < nb; i++) apply2(M->Dinv + 4 * (size_t)i, r + 2 * i, rd + 2 * i);
      rt = rd;
    } else if (M->qw) {
      rd = xmalloc(sizeof(double) * (size_t)n);
      for (int32_t i = 0; i < nb; i++) {
        rd[2 * i] = r[2 * i] + M->qw[i] * r[2 * i + 1];
        rd[2 * i + 1] = r[2 * i + 1];
      }
      rt = rd;
    }
    /* step 2: u = P1^{-1} r */
    if (M->ilu) ilu0_solve(M->ilu, M->ilu_diag, rt, z);
    else
      for (int32_t i = 0; i < nb; i++) apply2(M->P1inv + 4 * (size_t)i, rt + 2 * i, z + 2 * i);
    /* step 3: r' = r - Jt u */
    or_bsr2_spmv(nb, M->rowptr, M->col, M->Jt, z, tmp);
    for (int32_t i = 0; i < n; i++) tmp[i] = rt[i] - tmp[i];
    /* step 4: pressure correction */
    for (int32_t i = 0; i < nb; i++) sb[i] = tmp[2 * i];
    or_amg_vcycle(M->Hp, sb, sx);
    double *ds = NULL;
    if (M->prm.kind == OR_CPR2) {
      ds = xmalloc(sizeof(double) * (size_t)nb);
      for (int32_t i = 0; i < nb; i++) sb[i] = tmp[2 * i + 1];
      or_amg_vcycle(M->Hs, sb, ds);
    }
    for (int32_t i = 0; i < nb; i++) z[2 * i] += sx[i];
    if (ds)
      for (int32_t i = 0; i < nb; i++) z[2 * i + 1] += ds[i];
    free(ds);
    free(rd);
  }
  free(tmp); free(sb); free(sx);
}

static double dot(int32_t n, const double *a, const double *b) {
  double s = 0.0;
  for (int32_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}

/* Right-preconditioned flexible GMRES(m) with modified Gram-Schmidt and Givens
 * rotations; x holds x0 on entry. Stops when ||b - J x|| <= rtol ||b||,
 * checked on the true residual at each restart and at exit.
 * Returns 0 converged, 1 not converged. */
int32_t or_fgmres(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                  const or_precond *M, const double *b, double *x, int32_t m, double rtol,
                  int32_t maxit, int32_t *its_out, double *relres) {
  int32_t n = 2 * nb;
  double *V = xmalloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
  double *Z = xmalloc(sizeof(double) * (size_t)n * (size_t)m);
  double *H = xmalloc(sizeof(double) * (size_t)(m + 1) * (size_t)m);
  double *cs = xmalloc(sizeof(double) * (size_t)m), *sn = xmalloc(sizeof(double) * (size_t)m);
  double *g = xmalloc(sizeof(double) * (size_t)(m + 1)), *y = xmalloc(sizeof(double) * (size_t)m);
  double *r = xmalloc(sizeof(double) * (size_t)n);
  double bn = sqrt(dot(n, b, b));
  if (bn == 0.0) bn = 1.0;
  int32_t its = 0, status = 1;
  double beta = 0.0;
  for (;;) {
    or_bsr2_spmv(nb, rowptr, col, val, x, r);
    for (int32_t i = 0; i < n; i++) r[i] = b[i] - r[i];
    beta = sqrt(dot(n, r, r));
    if (beta <= rtol * bn) { status = 0; break; }
    if (its >= maxit) break;
    for (int32_t i = 0; i < n; i++) V[i] = r[i] / beta;
    for (int32_t i = 0; i <= m; i++) g[i] = 0.0;
    g[0] = beta;
    int32_t k = 0;
    for (int32_t j = 0; j < m; j++) {
      double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
      if (M) or_precond_apply(M, vj, zj);
      else memcpy(zj, vj, sizeof(double) * (size_t)n);
      or_bsr2_spmv(nb, rowptr, col, val, zj, w);
      for (int32_t i = 0; i <= j; i++) {
        double h = dot(n, w, V + (size_t)i * n);
        H[(size_t)i * m + j] = h;
        for (int32_t t = 0; t < n; t++) w[t] -= h * V[(size_t)i * n + t];
      }
      double hn = sqrt(dot(n, w, w));
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (int32_t t = 0; t < n; t++) w[t] /= hn;
      for (int32_t i = 0; i < j; i++) {
        double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[(size_t)j * m + j], c = H[(size_t)(j + 1) * m + j];
      double d = sqrt(a * a + c * c);
      cs[j] = d != 0.0 ? a / d : 1.0;
      sn[j] = d != 0.0 ? c / d : 0.0;
      H[(size_t)j * m + j] = d;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      its++;
      k = j + 1;
      if (fabs(g[j + 1]) <= rtol * bn || its >= maxit || hn == 0.0) break;
    }
    for (int32_t i = k - 1; i >= 0; i--) {
      double s = g[i];
      for (int32_t t = i + 1; t < k; t++) s -= H[(size_t)i * m + t] * y[t];
      y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
    }
    for (int32_t i = 0; i < k; i++)
      for (int32_t t = 0; t < n; t++) x[t] += y[i] * Z[(size_t)i * n + t];
  }
  *its_out = its;
  *relres = beta / bn;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(r);
  return status;
}

/* Newton's method for one backward-Euler step: J(u_k) du = -F(u_k),
 * u_{k+1} = u_k + du, each cell's S_n change first cut to [-max_ds, max_ds]
 * when max_ds > 0 (Appleyard chop; the paper does not state its damping),
 * then S_n clamped to [0, 1 - S_wr - 1e-12]. Converged when the scaled
 * residual (or_scaled_fnorm) is <= ftol. Returns 0 on convergence, 1 if
 * max_newton is reached, 2 if a linear solve failed, 3 if the residual is not
 * finite. */
int32_t or_newton(const or_problem *p, double *u, const double *u_old, double dt,
                  const or_newton_params *prm, int32_t *newton_its, int32_t *linear_its,
                  double *fnorm_hist) {
  int32_t nb = p->nx * p->ny * p->nz, n = 2 * nb;
  int32_t nnzb = or_bsr2_nnzb(p);
  int32_t *rowptr = xmalloc(sizeof(int32_t) * ((size_t)nb + 1));
  int32_t *col = xmalloc(sizeof(int32_t) * (size_t)nnzb);
  double *J = xmalloc(sizeof(double) * 4 * (size_t)nnzb);
  double *F = xmalloc(sizeof(double) * (size_t)n);
  double *du = xmalloc(sizeof(double) * (size_t)n);
  or_bsr2_pattern(p, rowptr, col);
  int32_t status = 1, lin = 0, k;
  for (k = 0; k <= prm->max_newton; k++) {
    or_assemble(p, u, u_old, dt, rowptr, col, J, F);
    double fn = or_scaled_fnorm(p, F, dt);
    if (fnorm_hist) fnorm_hist[k] = fn;
    if (fn <= prm->ftol) { status = 0; break; }
    if (k == prm->max_newton) break;
    if (!isfinite(fn)) { status = 3; break; }
    for (int32_t i = 0; i < n; i++) { F[i] = -F[i]; du[i] = 0.0; }
    or_precond *M = or_precond_create(nb, rowptr, col, J, &prm->prec);
    int32_t its = 0;
    double rr = 0.0;
    int32_t st = or_fgmres(nb, rowptr, col, J, M, F, du, prm->gmres_m, prm->gmres_rtol, prm->gmres_maxit, &its, &rr);
    or_precond_free(M);
    lin += its;
    if (st != 0) { status = 2; break; }
    double smax = 1.0 - p->s_wr - 1e-12;
    for (int32_t i = 0; i < nb; i++) {
      u[2 * i] += du[2 * i];
      double ds = du[2 * i + 1];
      if (prm->max_ds > 0.0 && fabs(ds) > prm->max_ds) ds = ds > 0.0 ? prm->max_ds : -prm->max_ds;
      double s = u[2 * i + 1] + ds;
      u[2 * i + 1] = s < 0.0 ? 0.0 : (s > smax ? smax : s);
    }
  }
  *newton_its = k;
  *linear_its = lin;
  free(rowptr); free(col); free(J); free(F); free(du);
  return status;
}
