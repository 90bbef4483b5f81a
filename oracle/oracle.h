/*
 * Plain FP64 CPU oracle of Bui, Elman and Moulton, "Algebraic Multigrid
 * Preconditioners for Multiphase Flow in Porous Media" (arXiv:1611.00127).
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA library: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it. It shares no code, header or table with the CUDA path.
 *
 * Everything is single-threaded, FP64, with loops written in the order of the
 * paper's definitions. Where floating point decides an integer (strength of
 * connection, C/F splitting, colouring) the sums are taken in ascending
 * column order with separate multiply and add (no fused multiply-add), so the
 * same decision can be reproduced exactly by another implementation that
 * follows the same stated order.
 */
#ifndef RS_ORACLE_H
#define RS_ORACLE_H
#include <stdint.h>

typedef struct {
  int32_t dim, nx, ny, nz;
  double hx, hy, hz;
  const double *kx, *ky, *kz;          /* per-cell permeability [m^2] */
  double phi, mu_w, mu_n, rho_w, rho_n, g;
  int32_t pc_model;                    /* 0 none, 1 linear, 2 Brooks-Corey */
  double pc_p0, pc_pd, bc_lambda;
  double s_wr, s_nr;
  double u_in, p_out, sn_out;
  double q_in;                         /* point wells, see or_assemble */
  int32_t well_in, well_out;
} or_problem;

/* Scalar CSR, n rows by m columns, columns ascending in each row. */
typedef struct {
  int32_t n, m, nnz;
  int32_t *rowptr, *col;
  double *val;
} or_csr;

typedef struct {
  double theta;        /* strength threshold */
  uint64_t seed;       /* PMIS and colouring random stream */
  int32_t max_levels;
  int32_t coarse_n;    /* stop coarsening at or below this many rows */
  int32_t max_dense;   /* largest coarsest level solved by dense LU */
  int32_t smoother;    /* 0 multicolour Gauss-Seidel, 1 l1-Jacobi, 2 hybrid multicolour GS */
  int32_t nu1, nu2;
  int32_t interp;      /* 0 classical, 1 extended+i */
  int32_t num_functions; /* 2: systems (point) AMG, 2 interleaved unknowns per point; else scalar */
  int32_t chunk;       /* rows per block of the hybrid smoother */
  int32_t agg_levels;  /* aggressive coarsening: the first agg_levels coarse grids are
                          two coarsening stages each (P = P_l P_{l+1}, level l+1 dropped) */
  int32_t chunk_coarse; /* hybrid-smoother chunk on levels >= 1 (0: `chunk` everywhere) */
  int32_t restriction;  /* scalar AMG: 0 R = P^T (Galerkin); 1, 2 approximate ideal restriction
                           over distance-1 / distance-2 F neighbourhoods, 3 over the distance-1
                           strongly coupled F points (lAIR); Petrov-Galerkin R A P */
} or_amg_params;

typedef struct or_amg or_amg;
typedef struct or_precond or_precond;

/* ---- physics (Sec. 2) ---- */
int32_t or_bsr2_nnzb(const or_problem *p);
void or_bsr2_pattern(const or_problem *p, int32_t *rowptr, int32_t *col);
void or_assemble(const or_problem *p, const double *u, const double *u_old, double dt,
                 const int32_t *rowptr, const int32_t *col, double *Jval, double *F);
void or_constitutive(const or_problem *p, double sn, double *out6);

/* ---- sparse helpers ---- */
void or_bsr2_spmv(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                  const double *x, double *y);
or_csr *or_csr_new(int32_t n, int32_t m, int32_t nnz, const int32_t *rowptr, const int32_t *col,
                   const double *val);
void or_csr_free(or_csr *A);
void or_csr_info(const or_csr *A, int32_t *nmnnz);
void or_csr_copy(const or_csr *A, int32_t *rowptr, int32_t *col, double *val);
or_csr *or_scalar_from_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val);
or_csr *or_bsr2_part(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, int32_t r, int32_t c);
void or_decouple_abf(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *out);
void or_decouple_qimpes(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *out,
                        double *w_out);
or_csr *or_simple_schur(const or_csr *App, const or_csr *Aps, const or_csr *Asp, const or_csr *Ass);
or_csr *or_transpose(const or_csr *A);
or_csr *or_spgemm(const or_csr *A, const or_csr *B);
void or_csr_spmv(const or_csr *A, const double *x, double *y);

/* ---- AMG pieces (Sec. 3.2, Sec. 4 solver settings) ---- */
uint64_t or_splitmix64(uint64_t seed, uint64_t counter);
void or_strength(const or_csr *A, double theta, uint8_t *strong);
void or_strength_nf(const or_csr *A, double theta, int32_t nfun, uint8_t *strong);
void or_pmis(const or_csr *A, const uint8_t *strong, uint64_t seed, int32_t level, int8_t *cf);
or_csr *or_interp(const or_csr *A, const uint8_t *strong, const int8_t *cf);
or_csr *or_interp_ext(const or_csr *A, const uint8_t *strong, const int8_t *cf);
or_csr *or_galerkin(const or_csr *A, const or_csr *P);
or_csr *or_air_restriction(const or_csr *A, const int8_t *cf, int32_t dist, const uint8_t *strong);
int32_t or_jp_colour(const or_csr *A, uint64_t seed, int32_t level, int32_t *colour);
int32_t or_chunk_rows(const or_csr *A, int32_t chunk);
int32_t or_chunk_colour(const or_csr *A, int32_t chunk, int32_t *colour);
int32_t or_chunk_colour_pt(const or_csr *A, int32_t chunk, int32_t b, int32_t *colour);
or_csr *or_func_part(const or_csr *A, int32_t b, int32_t f);

or_amg *or_amg_setup(const or_csr *A, const or_amg_params *prm);
void or_amg_free(or_amg *H);
int32_t or_amg_nlevels(const or_amg *H);
const or_csr *or_amg_A(const or_amg *H, int32_t l);
const or_csr *or_amg_P(const or_amg *H, int32_t l);
void or_amg_cf(const or_amg *H, int32_t l, int8_t *cf);
int32_t or_amg_colours(const or_amg *H, int32_t l, int32_t *colour);
void or_amg_vcycle(const or_amg *H, const double *b, double *x);
void or_amg_smooth(const or_amg *H, int32_t l, const double *b, double *x);

/* ---- dense LU (coarsest level and tests) ---- */
int32_t or_dense_lu(int32_t n, double *a, int32_t *piv);
void or_dense_lu_solve(int32_t n, const double *a, const int32_t *piv, const double *b, double *x);

/* ---- preconditioners (Sec. 3.2-3.4) ---- */
enum { OR_AMG_J = 0, OR_CPR1 = 1, OR_CPR2 = 2, OR_BF = 3, OR_AMG_J_SCALAR = 4 };
typedef struct {
  int32_t kind;
  int32_t decouple;   /* CPR only: 0 none, 1 per-cell inverse of the 2x2 diagonal block,
                         2 quasi-IMPES row combination */
  int32_t p1;         /* CPR only: 0 point-block Jacobi, 1 ILU(0) on the point-ordered matrix */
  or_amg_params amg;
} or_precond_params;
or_precond *or_precond_create(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                              const or_precond_params *prm);
void or_precond_free(or_precond *M);
void or_precond_apply(const or_precond *M, const double *r, double *z);
const or_amg *or_precond_amg(const or_precond *M, int32_t which);

/* ---- Krylov (Sec. 3, eq. precon-system) ---- */
int32_t or_fgmres(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                  const or_precond *M, const double *b, double *x, int32_t m, double rtol,
                  int32_t maxit, int32_t *its, double *relres);

/* ILU(0) of the point-ordered scalar matrix (P1 of CPR, Sec. 3.3): factors in
 * the block layout (lu[4k + 2r + c]: scalar row 2i+r, column 2 col[k] + c),
 * and the forward/backward solve with them. */
void or_ilu0_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *lu);
void or_ilu0_solve_bsr2(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *lu, const double *b,
                        double *x);

/* ---- Newton (Sec. 3) ---- */
typedef struct {
  int32_t max_newton;
  double ftol;          /* on max |F| * dt / (V phi rho_alpha): saturation units */
  int32_t gmres_m, gmres_maxit;
  double gmres_rtol;
  or_precond_params prec;
  double max_ds;        /* > 0: cut each cell's S_n change to [-max_ds, max_ds] */
} or_newton_params;
int32_t or_newton(const or_problem *p, double *u, const double *u_old, double dt,
                  const or_newton_params *prm, int32_t *newton_its, int32_t *linear_its,
                  double *fnorm_hist);
double or_scaled_fnorm(const or_problem *p, const double *F, double dt);

#endif
