/*
 * Oracle, part 1: the discrete two-phase model and its exact Jacobian.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Model (Sec. 2): unknowns u = (P_w, S_n) per cell (eqs. balance1, balance2);
 * cell-centred finite volumes with two-point fluxes, phase upwinding and
 * harmonic face permeability; backward Euler in time
 * (eq. fully_discrete_system). The residual is kept in mass-rate form,
 *
 *   F_a,i = V (xi_a(u_i) - xi_a(u_old,i)) / dt
 *         + sum_j T_ij rho_a lambda_a,up (Phi_a,i - Phi_a,j) - q_a,i ,
 *
 * with xi_w = phi rho_w (1 - S_n), xi_n = phi rho_n S_n, Phi_w = P_w - rho_w g D,
 * Phi_n = P_w + P_c(S_n) - rho_n g D, lambda_a = k_ra / mu_a and
 * T_ij = (face area) K_ij / (centre distance). The paper's form of the
 * equation is this F times dt / V.
 *
 * Readings of points the paper leaves open:
 *  - Relative permeability (never stated): Brooks-Corey-Burdine with the same
 *    lambda as P_c: k_rw = Sb^((2+3L)/L), k_rn = (1-Sb)^2 (1 - Sb^((2+L)/L)),
 *    Sb = (S_w - S_wr)/(1 - S_wr - S_nr), clamped to [0, 1].
 *  - Brooks-Corey P_c = P_d Sb^(-1/L) (Sec. 4.1) is continued linearly below
 *    Sb = 1e-4 with the slope there, so the Jacobian stays exact.
 *  - Upwinding (Sec. 2): phase mobility from cell i iff Phi_i - Phi_j > 0,
 *    else from j; the exact Jacobian keeps that choice fixed.
 *  - Boundaries: water enters through the x = 0 face at Darcy flux u_in
 *    (mass source rho_w u_in A on those cells); the x = L face is a Dirichlet
 *    face at P_w = p_out with inflowing oil saturation sn_out, using the half
 *    transmissibility A K_i / (h/2); all other faces are closed. Point wells
 *    (the corner wells of the examples of Sec. 4): with well_in >= 0 the
 *    water enters only as a mass source rho_w q_in in that cell; with
 *    well_out >= 0 only that cell's x = L face is the outlet.
 *  - Depth D is the last coordinate (y in 2D, z in 3D), cell centres.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static double sbar_w(const or_problem *p, double sn) {
  return (1.0 - sn - p->s_wr) / (1.0 - p->s_wr - p->s_nr);
}

static double dsbar_dsn(const or_problem *p) { return -1.0 / (1.0 - p->s_wr - p->s_nr); }

/* Mobilities lambda_w, lambda_n and their derivatives with respect to S_n. */
static void mobility(const or_problem *p, double sn, double *lw, double *ln, double *dlw, double *dln) {
  double s = sbar_w(p, sn), L = p->bc_lambda;
  double ew = (2.0 + 3.0 * L) / L, en = (2.0 + L) / L;
  double krw, krn, dkrw, dkrn;
  if (s <= 0.0) {
    krw = 0.0; krn = 1.0; dkrw = 0.0; dkrn = 0.0;
  } else if (s >= 1.0) {
    krw = 1.0; krn = 0.0; dkrw = 0.0; dkrn = 0.0;
  } else {
    double t = pow(s, en);
    krw = pow(s, ew);
    dkrw = ew * pow(s, ew - 1.0);
    krn = (1.0 - s) * (1.0 - s) * (1.0 - t);
    dkrn = -2.0 * (1.0 - s) * (1.0 - t) - (1.0 - s) * (1.0 - s) * en * pow(s, en - 1.0);
  }
  double ds = dsbar_dsn(p);
  *lw = krw / p->mu_w;
  *ln = krn / p->mu_n;
  *dlw = dkrw * ds / p->mu_w;
  *dln = dkrn * ds / p->mu_n;
}

/* Capillary pressure P_c(S_n) and dP_c/dS_n (Sec. 4.1 models). */
static void capillary(const or_problem *p, double sn, double *pc, double *dpc) {
  double s = sbar_w(p, sn), ds = dsbar_dsn(p);
  if (p->pc_model == 1) {
    *pc = p->pc_p0 * (1.0 - s);
    *dpc = -p->pc_p0 * ds;
  } else if (p->pc_model == 2) {
    const double eps = 1e-4;
    double L = p->bc_lambda, d;
    if (s >= eps) {
      *pc = p->pc_pd * pow(s, -1.0 / L);
      d = -(p->pc_pd / L) * pow(s, -1.0 / L - 1.0);
    } else {
      double pce = p->pc_pd * pow(eps, -1.0 / L);
      d = -(p->pc_pd / L) * pow(eps, -1.0 / L - 1.0);
      *pc = pce + d * (s - eps);
    }
    *dpc = d * ds;
  } else {
    *pc = 0.0;
    *dpc = 0.0;
  }
}

void or_constitutive(const or_problem *p, double sn, double *o) {
  mobility(p, sn, &o[0], &o[1], &o[2], &o[3]);
  capillary(p, sn, &o[4], &o[5]);
}

/* Neighbours of cell i in ascending index order; returns count.
 * dir[k] = 0 x, 1 y, 2 z. */
static int neighbours(const or_problem *p, int32_t i, int32_t *nb, int *dir) {
  int32_t nx = p->nx, ny = p->ny, nz = p->nz;
  int32_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  int c = 0;
  if (p->dim == 3 && iz > 0) { nb[c] = i - nx * ny; dir[c++] = 2; }
  if (iy > 0) { nb[c] = i - nx; dir[c++] = 1; }
  if (ix > 0) { nb[c] = i - 1; dir[c++] = 0; }
  if (ix < nx - 1) { nb[c] = i + 1; dir[c++] = 0; }
  if (iy < ny - 1) { nb[c] = i + nx; dir[c++] = 1; }
  if (p->dim == 3 && iz < nz - 1) { nb[c] = i + nx * ny; dir[c++] = 2; }
  (void)nz;
  return c;
}

int32_t or_bsr2_nnzb(const or_problem *p) {
  int32_t n = p->nx * p->ny * p->nz, tot = 0, nb[6];
  int dir[6];
  for (int32_t i = 0; i < n; i++) tot += 1 + neighbours(p, i, nb, dir);
  return tot;
}

void or_bsr2_pattern(const or_problem *p, int32_t *rowptr, int32_t *col) {
  int32_t n = p->nx * p->ny * p->nz, nb[6], pos = 0;
  int dir[6];
  rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int c = neighbours(p, i, nb, dir);
    int placed = 0;
    for (int k = 0; k < c; k++) {
      if (!placed && nb[k] > i) { col[pos++] = i; placed = 1; }
      col[pos++] = nb[k];
    }
    if (!placed) col[pos++] = i;
    rowptr[i + 1] = pos;
  }
}

static double face_area(const or_problem *p, int d) {
  double hz = p->dim == 3 ? p->hz : 1.0;
  if (d == 0) return p->hy * hz;
  if (d == 1) return p->hx * hz;
  return p->hx * p->hy;
}

static double spacing(const or_problem *p, int d) { return d == 0 ? p->hx : (d == 1 ? p->hy : p->hz); }

static double perm(const or_problem *p, int d, int32_t i) {
  return d == 0 ? p->kx[i] : (d == 1 ? p->ky[i] : p->kz[i]);
}

static double depth(const or_problem *p, int32_t i) {
  if (p->dim == 3) return ((double)(i / (p->nx * p->ny)) + 0.5) * p->hz;
  return ((double)((i / p->nx) % p->ny) + 0.5) * p->hy;
}

/* Position of block column j in block row i. */
static int32_t find_block(const int32_t *rowptr, const int32_t *col, int32_t i, int32_t j) {
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
    if (col[k] == j) return k;
  return -1;
}

/* Residual F (length 2N) and, if Jval != NULL, the exact Jacobian blocks.
 * Block (i,j) is stored row-major: [dFw/dp, dFw/dS; dFn/dp, dFn/dS]. */
void or_assemble(const or_problem *p, const double *u, const double *u_old, double dt,
                 const int32_t *rowptr, const int32_t *col, double *Jval, double *F) {
  int32_t n = p->nx * p->ny * p->nz;
  double hz = p->dim == 3 ? p->hz : 1.0;
  double V = p->hx * p->hy * hz;
  double rho[2] = {p->rho_w, p->rho_n};
  if (Jval) memset(Jval, 0, sizeof(double) * 4 * (size_t)rowptr[n]);
  for (int32_t i = 0; i < n; i++) {
    double pi = u[2 * i], si = u[2 * i + 1], so = u_old[2 * i + 1];
    double mob_i[6];
    or_constitutive(p, si, mob_i);
    double Di = depth(p, i);
    /* storage */
    double xiw = p->phi * p->rho_w * (1.0 - si), xiw0 = p->phi * p->rho_w * (1.0 - so);
    double xin = p->phi * p->rho_n * si, xin0 = p->phi * p->rho_n * so;
    double Fw = V * (xiw - xiw0) / dt;
    double Fn = V * (xin - xin0) / dt;
    int32_t kd = Jval ? find_block(rowptr, col, i, i) : -1;
    if (Jval) {
      Jval[4 * kd + 1] += -V * p->phi * p->rho_w / dt;
      Jval[4 * kd + 3] += V * p->phi * p->rho_n / dt;
    }
    /* interior faces */
    int32_t nb[6];
    int dir[6];
    int c = neighbours(p, i, nb, dir);
    for (int k = 0; k < c; k++) {
      int32_t j = nb[k];
      int d = dir[k];
      double ki = perm(p, d, i), kj = perm(p, d, j);
      double kh = (ki + kj) > 0.0 ? 2.0 * ki * kj / (ki + kj) : 0.0;
      double T = face_area(p, d) * kh / spacing(p, d);
      double pj = u[2 * j], sj = u[2 * j + 1];
      double mob_j[6];
      or_constitutive(p, sj, mob_j);
      double Dj = depth(p, j);
      int32_t kj_blk = Jval ? find_block(rowptr, col, i, j) : -1;
      for (int a = 0; a < 2; a++) {
        double phi_i = pi - rho[a] * p->g * Di + (a == 1 ? mob_i[4] : 0.0);
        double phi_j = pj - rho[a] * p->g * Dj + (a == 1 ? mob_j[4] : 0.0);
        double dphi = phi_i - phi_j;
        int up_i = dphi > 0.0;
        double lam = up_i ? mob_i[a] : mob_j[a];
        double dlam = up_i ? mob_i[2 + a] : mob_j[2 + a];
        double cc = T * rho[a];
        double flux = cc * lam * dphi;
        if (a == 0) Fw += flux; else Fn += flux;
        if (Jval) {
          Jval[4 * kd + 2 * a + 0] += cc * lam;
          Jval[4 * kj_blk + 2 * a + 0] += -cc * lam;
          if (a == 1) {
            Jval[4 * kd + 2 * a + 1] += cc * lam * mob_i[5];
            Jval[4 * kj_blk + 2 * a + 1] += -cc * lam * mob_j[5];
          }
          if (up_i) Jval[4 * kd + 2 * a + 1] += cc * dlam * dphi;
          else Jval[4 * kj_blk + 2 * a + 1] += cc * dlam * dphi;
        }
      }
    }
    int32_t ix = i % p->nx;
    /* Dirichlet outlet face at x = L (the whole face, or one cell's) */
    if (ix == p->nx - 1 && (p->well_out < 0 || i == p->well_out)) {
      double T = face_area(p, 0) * p->kx[i] / (0.5 * p->hx);
      double mob_b[6];
      or_constitutive(p, p->sn_out, mob_b);
      for (int a = 0; a < 2; a++) {
        double phi_i = pi - rho[a] * p->g * Di + (a == 1 ? mob_i[4] : 0.0);
        double phi_b = p->p_out - rho[a] * p->g * Di + (a == 1 ? mob_b[4] : 0.0);
        double dphi = phi_i - phi_b;
        int up_i = dphi > 0.0;
        double lam = up_i ? mob_i[a] : mob_b[a];
        double cc = T * rho[a];
        double flux = cc * lam * dphi;
        if (a == 0) Fw += flux; else Fn += flux;
        if (Jval) {
          Jval[4 * kd + 2 * a + 0] += cc * lam;
          if (a == 1) Jval[4 * kd + 2 * a + 1] += cc * lam * mob_i[5];
          if (up_i) Jval[4 * kd + 2 * a + 1] += cc * mob_i[2 + a] * dphi;
        }
      }
    }
    /* injection through x = 0, or at the injection well */
    if (p->well_in < 0) {
      if (ix == 0) Fw -= p->rho_w * p->u_in * face_area(p, 0);
    } else if (i == p->well_in) {
      Fw -= p->rho_w * p->q_in;
    }
    F[2 * i] = Fw;
    F[2 * i + 1] = Fn;
  }
}

void or_bsr2_spmv(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                  const double *x, double *y) {
  for (int32_t i = 0; i < nb; i++) {
    double y0 = 0.0, y1 = 0.0;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
      const double *b = val + 4 * (size_t)k;
      double x0 = x[2 * col[k]], x1 = x[2 * col[k] + 1];
      y0 += b[0] * x0 + b[1] * x1;
      y1 += b[2] * x0 + b[3] * x1;
    }
    y[2 * i] = y0;
    y[2 * i + 1] = y1;
  }
}

/* Newton convergence measure: max over cells and phases of |F| dt / (V phi rho_a),
 * i.e. the residual of the paper's fully discrete equation in saturation units. */
double or_scaled_fnorm(const or_problem *p, const double *F, double dt) {
  int32_t n = p->nx * p->ny * p->nz;
  double hz = p->dim == 3 ? p->hz : 1.0;
  double V = p->hx * p->hy * hz, m = 0.0;
  for (int32_t i = 0; i < n; i++) {
    double a = fabs(F[2 * i]) * dt / (V * p->phi * p->rho_w);
    double b = fabs(F[2 * i + 1]) * dt / (V * p->phi * p->rho_n);
    if (a > m) m = a;
    if (b > m) m = b;
  }
  return m;
}
