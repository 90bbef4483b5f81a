/*
 * rsflow: GB300 (sm_103a) solver for the Newton Jacobians of a fully implicit
 * two-phase (water/oil) cell-centred finite-volume model, after Bui, Elman and
 * Moulton, "Algebraic Multigrid Preconditioners for Multiphase Flow in Porous
 * Media" (arXiv:1611.00127).
 *
 * Conventions for every call:
 *  - Return value: 0 (RS_OK) on success; > 0 a non-fatal outcome
 *    (RS_NOT_CONVERGED); < 0 an error (the call did nothing further). The
 *    text of the last error of the calling thread is available from
 *    rs_last_error().
 *  - Array arguments are DEVICE pointers owned by the caller unless a field
 *    says "host". They must stay valid and unmodified while a call that uses
 *    them is in flight on the stream, and, for a preconditioner, for as long
 *    as the preconditioner is applied (it keeps a reference to J).
 *  - Every call takes a cudaStream_t and enqueues its GPU work there. Calls
 *    marked (sync) wait for their own work before returning, to fill host
 *    statistics; all others are asynchronous.
 *  - Handles (rs_amg, rs_precond) own device memory allocated by the library;
 *    free them with the matching *_destroy. A handle is not thread-safe.
 *  - Unknowns are interleaved per cell: entry 2i is the water pressure P_w of
 *    cell i [Pa], entry 2i+1 its oil saturation S_n (Sec. 2, u = (P_w, S_n)).
 *  - Batches: a matrix may hold several independent systems stacked as a
 *    block-diagonal matrix. seg_off (host array of nseg+1 block-row offsets)
 *    marks them; all solver work (AMG hierarchies, orthogonalisation,
 *    convergence tests) is then done per system, in one set of launches.
 */
#ifndef RSFLOW_H
#define RSFLOW_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RS_OK 0
#define RS_NOT_CONVERGED 1
#define RS_EINVAL (-1)
#define RS_ECUDA (-2)
#define RS_ETIMEOUT (-3)
#define RS_ENOMEM (-4)
#define RS_ESETUP (-5)
#define RS_EBREAKDOWN (-6)

/* Empty systems (nb = 0, n = 0) are valid everywhere: vector arguments may
 * then be NULL, set-up builds nothing, applies and solves return RS_OK at once
 * (a solve reports 0 iterations, converged). */

/* 2x2-block CSR matrix, FP64. Block k (columns col[k]) is stored row-major at
 * val[4k..4k+3] = [dF_w/dP_w, dF_w/dS_n, dF_n/dP_w, dF_n/dS_n]; this is the
 * grid-point ordering of Sec. 3.2, with the blocks A_pp, A_ps, A_sp, A_ss of
 * eq. (jacobian) interleaved. Columns ascending in every block row, diagonal
 * block present. nseg = 0 or seg_off = NULL means one system. */
typedef struct rs_bsr2 {
  int32_t nb;              /* block rows (cells) */
  int32_t nnzb;            /* stored blocks */
  const int32_t *row_ptr;  /* [nb+1] */
  const int32_t *col;      /* [nnzb] */
  double *val;             /* [4*nnzb] */
  int32_t nseg;            /* number of stacked systems (0 or 1: one) */
  const int32_t *seg_off;  /* host [nseg+1] block-row offsets, seg_off[0]=0, seg_off[nseg]=nb */
} rs_bsr2;

/* Scalar CSR matrix, FP64, square, columns ascending. */
typedef struct rs_csr {
  int32_t n, nnz;
  const int32_t *row_ptr;  /* [n+1] */
  const int32_t *col;      /* [nnz] */
  const double *val;       /* [nnz] */
  int32_t nseg;
  const int32_t *seg_off;  /* host [nseg+1] row offsets, or NULL */
} rs_csr;

/* One Cartesian grid (Sec. 2): cells numbered x fastest,
 * i = ix + nx (iy + ny iz); 2D grids have nz = 1 and unit thickness. */
typedef struct rs_problem {
  int32_t dim, nx, ny, nz;
  double hx, hy, hz;                  /* cell sizes [m] */
  const double *kx, *ky, *kz;         /* device [ncell] permeability [m^2] */
  double phi, mu_w, mu_n, rho_w, rho_n, g;
  int32_t pc_model;                   /* 0 none, 1 linear P_0 (1-Sb), 2 Brooks-Corey P_d Sb^(-1/lambda) */
  double pc_p0, pc_pd, bc_lambda;     /* lambda also sets the Brooks-Corey relative permeabilities */
  double s_wr, s_nr;                  /* residual saturations */
  double u_in;                        /* water Darcy flux injected through the x = 0 face [m/s] */
  double p_out, sn_out;               /* Dirichlet outlet on the x = L face */
  /* point wells (the corner wells of the paper's examples, Sec. 4):
   * well_in >= 0: water enters only as a source of q_in [m^3/s] in that cell
   * (u_in unused); well_out >= 0: only that cell's x = L face (ix = nx-1) is
   * the outlet. -1: the face conditions above. */
  double q_in;
  int32_t well_in, well_out;
} rs_problem;

#define RS_SMOOTH_MCGS 0      /* multicolour Gauss-Seidel over the whole level */
#define RS_SMOOTH_L1JACOBI 1  /* l1-Jacobi */
#define RS_SMOOTH_HYBRID 2    /* Gauss-Seidel by colour inside chunks of `chunk` rows, Jacobi between chunks */
#define RS_INTERP_CLASSICAL 0
#define RS_INTERP_EXTI 1
#define RS_PREC_FP32 0   /* V-cycle values, vectors and sums in FP32 */
#define RS_PREC_FP64 1

typedef struct rs_amg_params {
  double theta;            /* strength threshold (e.g. 0.25 in 2D, 0.5 in 3D) */
  uint64_t seed;           /* PMIS and colouring random stream (SplitMix64) */
  int32_t max_levels;      /* <= 25 */
  int32_t coarse_n;        /* a system stops coarsening at or below this many rows */
  int32_t max_dense;       /* largest coarsest level handled by the dense solve */
  int32_t smoother;        /* RS_SMOOTH_* */
  int32_t nu1, nu2;        /* pre- and post-smoothing sweeps */
  int32_t interp;          /* RS_INTERP_* */
  int32_t num_functions;   /* 2: systems (point) AMG with 2 interleaved unknowns per point
                              (row 2i + f is unknown f of point i): points coarsened on the
                              unknown-0 part, each unknown interpolated from the same unknown,
                              point-block hybrid Gauss-Seidel smoother; 1: scalar AMG */
  int32_t precision;       /* RS_PREC_* of the V-cycle */
  int32_t chunk;           /* rows per chunk of the hybrid smoother (32..512) */
  int32_t agg_levels;      /* aggressive coarsening (0..8): the first agg_levels coarse grids are
                              each two coarsening stages, interpolated by the product of the
                              two stages' P (the intermediate level is dropped); 0: off */
  int32_t chunk_coarse;    /* rows per chunk of the hybrid smoother on levels >= 1 (32..512);
                              0: `chunk` on every level */
  int32_t restriction;     /* scalar AMG (num_functions 1): 0 Galerkin, R = P^T; 1 approximate
                              ideal restriction (AIR, Manteuffel, Southworth et al. 2018),
                              distance 1: R's row for C point i is 1 at i and -z on the F
                              points N_i coupled to i, A(N_i, N_i)^T z = A(i, N_i)^T, so
                              (R A)(i, N_i) = 0; A_{l+1} = R A P. 3: the same over the F
                              points that strongly influence i only (lAIR, Manteuffel,
                              Muenzenmaier, Ruge, Southworth 2019), which keeps R A P as
                              sparse as Galerkin's on transport-dominated levels. For
                              non-symmetric levels such as the block factorisation's S~ and
                              A_ss. Ignored by systems AMG */
} rs_amg_params;

typedef struct rs_amg rs_amg;
typedef struct rs_precond rs_precond;
typedef struct rs_ilu0 rs_ilu0;

#define RS_P1_BLOCK_JACOBI 0  /* inverse of each cell's 2x2 diagonal block */
#define RS_P1_ILU0 1          /* ILU(0) of the point-ordered matrix (Sec. 3.3) */

#define RS_PC_AMG_J 0   /* black-box AMG on the point-ordered J (Sec. 3.2), the point method */
#define RS_PC_CPR1 1    /* Algorithm 1, combinative two-stage CPR-AMG(1) */
#define RS_PC_CPR2 2    /* Algorithm 2, additive two-stage CPR-AMG(2) */
#define RS_PC_BF 3      /* Algorithm 3, block factorisation with SIMPLE Schur */
#define RS_PC_AMG_J_SCALAR 4  /* scalar AMG on the interleaved J (no point structure) */

#define RS_DECOUPLE_NONE 0
#define RS_DECOUPLE_ABF 1     /* D^{-1} J, D = per-cell 2x2 diagonal block */
#define RS_DECOUPLE_QIMPES 2  /* pressure row += -(a_ps,ii / a_ss,ii) oil row */

typedef struct rs_precond_params {
  int32_t kind;            /* RS_PC_* */
  int32_t decouple;        /* CPR only: RS_DECOUPLE_* */
  int32_t p1;              /* CPR only: RS_P1_* first-stage preconditioner */
  rs_amg_params amg;
} rs_precond_params;

typedef struct rs_gmres_params {
  int32_t m;               /* restart length */
  int32_t maxit;           /* total Arnoldi steps per system */
  double rtol;             /* stop when ||b - J x||_2 <= rtol ||b||_2 */
} rs_gmres_params;

typedef struct rs_gmres_stats {
  int32_t iterations;      /* max over systems */
  int32_t converged;       /* number of systems that reached rtol */
  double relres;           /* max over systems of the true relative residual */
  int32_t *its;            /* host [nseg] per-system iterations, or NULL */
  double *relres_seg;      /* host [nseg] per-system true relative residual, or NULL */
} rs_gmres_stats;

typedef struct rs_newton_params {
  int32_t max_newton;
  double ftol;             /* on max_i |F_a,i| dt / (V phi rho_a) */
  rs_gmres_params gmres;
  rs_precond_params prec;
  double max_ds;           /* > 0: each cell's S_n change per iteration is cut to
                              [-max_ds, max_ds] (Appleyard chop); <= 0: full steps */
} rs_newton_params;

typedef struct rs_newton_stats {
  int32_t newton_its;
  int32_t linear_its;      /* summed over Newton iterations */
  double fnorm;            /* final scaled residual */
  double setup_ms, solve_ms, assemble_ms;
} rs_newton_stats;

/* Text of the last error on this thread (never NULL). */
const char *rs_last_error(void);

/* Library version and the CUDA architecture it was built for. */
int rs_version(int *major, int *minor, int *arch);

/* Number of CUDA kernels the library has launched in this process so far
 * (all threads, all devices). */
long long rs_launch_count(void);

/* Kernel profiling for measurement: between rs_profile_begin and
 * rs_profile_end the library brackets launches of its main kernel classes
 * with CUDA events on their own stream (and runs preconditioner applies
 * without graph replay). rs_profile_end fills, per class, the summed device
 * time [ms], the summed algorithmic bytes and the launch count, and returns
 * the number of classes: 0 hybrid GS sweep, 1 CSR residual/restriction/
 * prolongation, 2 block SpMV (and CPR residual), 3 GMRES dot/update,
 * 4 setup sparse products, 5 interpolation, 6 other. Not for use inside stream
 * capture. */
int rs_profile_begin(void);
int rs_profile_end(double *ms, double *bytes, long long *launches, int nclasses);

/* Lanes per block row of the block SpMV (1, 2, 4 or 8; default 4), a tuning
 * knob chosen by measurement; rs_autotune_bsr2 times every choice on J
 * (CUDA events on `stream`, x and y as work vectors) and keeps the fastest,
 * returning it in *best. */
int rs_tune_set_bsr2_lpr(int lanes);
int rs_autotune_bsr2(const rs_bsr2 *J, const double *x, double *y, int *best, cudaStream_t stream);

/* ---------------------------------------------------------------- grid --- */
/* Number of stored blocks of the two-point-flux pattern of `nprob` grids
 * stacked in order (host call, no GPU work). */
int64_t rs_bsr2_nnzb(const rs_problem *probs, int32_t nprob);

/* Block pattern (Sec. 2, TPFA neighbours plus the diagonal) of the stacked
 * grids: row_ptr [ncell_total+1], col [nnzb] (device outputs). */
int rs_bsr2_pattern(const rs_problem *probs, int32_t nprob, int32_t *row_ptr, int32_t *col,
                    cudaStream_t stream);

/* ------------------------------------------------------------ the calls --- */
/* Residual F(u) and exact Jacobian J(u) of the backward-Euler TPFA system
 * (eq. fully_discrete_system; Jacobian eq. linearize_fc / eq. jacobian), for
 * `nprob` grids stacked in order. u, u_old: [2 N] interleaved (P_w, S_n).
 * F: [2 N] output (mass-rate form, kg/s). J->val is overwritten on the
 * pattern from rs_bsr2_pattern; J may be NULL to form F only. */
int jacobian_assemble(const rs_problem *probs, int32_t nprob, const double *u, const double *u_old,
                      double dt, rs_bsr2 *J, double *F, cudaStream_t stream);

/* Same as jacobian_assemble, but the call allocates no device memory: for
 * callers that cannot call cudaMalloc at that point (the device allocator is
 * owned by another component or fully reserved, or the call sits in a loop
 * that must not allocate). The paper has no counterpart; this is a service of
 * the library. Scratch lives in fixed arrays of the library's device image
 * (about 3.2 MB held on every GPU that loads the library, until exit).
 * Limits: at most 65536 cells and 64 grids per call, else RS_EINVAL with a
 * message naming the limit. The grid descriptions reach the device as a
 * kernel parameter; the call copies nothing from host memory. The first call
 * on a device looks up the arrays' device addresses (cudaGetSymbolAddress);
 * make that first call before any stream capture. All calls share the
 * arrays, which keep the last call's contents (every call overwrites what it
 * reads): calls that overlap on the GPU race. Arguments and outputs as for
 * jacobian_assemble. */
int jacobian_assemble_noalloc(const rs_problem *probs, int32_t nprob, const double *u, const double *u_old,
                              double dt, rs_bsr2 *J, double *F, cudaStream_t stream);

/* Classical AMG hierarchy for a scalar matrix (Sec. 3.2; solver settings of
 * Sec. 4 with PMIS coarsening and the stated interpolation): strength graph,
 * PMIS C/F splitting, interpolation, Galerkin A_c = P^T A P, colouring,
 * coarsest dense inverse. A is read during the call only. (sync) */
int amg_setup(const rs_csr *A, const rs_amg_params *params, rs_amg **H, cudaStream_t stream);
int amg_destroy(rs_amg *H);

/* x = one V(nu1,nu2)-cycle applied to b with zero initial guess (FP64 in and
 * out; the cycle itself runs in params.precision). */
int amg_apply(const rs_amg *H, const double *b, double *x, cudaStream_t stream);

/* Preconditioner M for J (Sec. 3.2-3.4): builds the needed blocks, decoupling
 * and AMG hierarchies. (sync) */
int precond_create(const rs_bsr2 *J, const rs_precond_params *params, rs_precond **M,
                   cudaStream_t stream);
int precond_destroy(rs_precond *M);

/* z = M^{-1} r (Algorithms 1-3 or the black-box V-cycle), FP64 [2N]. */
int precond_apply(const rs_precond *M, const double *r, double *z, cudaStream_t stream);

/* Capped device waits. A smoother CTA whose staging copies have not landed
 * within its wait limit leaves its rows unswept and raises a device flag
 * (no counterpart in the paper: a guard of this implementation).
 * gmres_solve and newton_step check the flag before they return and report
 * RS_ETIMEOUT. After the asynchronous calls (precond_apply, amg_apply,
 * amg_level_smooth) call rs_wait_status: it synchronises `stream`, returns
 * RS_ETIMEOUT and clears the flag if it was raised, else RS_OK.
 * rs_raise_wait_flag sets the flag as a capped wait would, without running a
 * kernel, so that callers can test their handling of the error. */
int rs_wait_status(cudaStream_t stream);
int rs_raise_wait_flag(cudaStream_t stream);

/* Right-preconditioned flexible GMRES(m) (Sec. 3, eq. precon-system) for/* Right-preconditioned flexible GMRES(m) (Sec. 3, eq. precon-system) for
 * J x = b, per system of the batch, with classical Gram-Schmidt applied twice
 * and Givens rotations in FP64. x holds the initial guess on entry. M may be
 * NULL (no preconditioner). Returns RS_OK when every system converged, else
 * RS_NOT_CONVERGED. (sync) */
int gmres_solve(const rs_bsr2 *J, const rs_precond *M, const double *b, double *x,
                const rs_gmres_params *params, rs_gmres_stats *stats, cudaStream_t stream);

/* One backward-Euler step by Newton's method (Sec. 3): repeats
 * assemble -> precond_create -> gmres_solve(J du = -F) -> u += du (S_n
 * change cut to +-max_ds when max_ds > 0, S_n clamped to
 * [0, 1 - S_wr - 1e-12]) until the scaled residual is <= ftol. Returns
 * RS_NOT_CONVERGED after max_newton iterations, when FGMRES does not converge,
 * or when the residual is not finite; u then holds the last iterate.
 * u: [2N] in/out. (sync) */
int newton_step(const rs_problem *probs, int32_t nprob, double *u, const double *u_old, double dt,
                const rs_newton_params *params, rs_newton_stats *stats, cudaStream_t stream);

/* ------------------------------------------------------- building blocks --- */
/* y = J x (FP64). */
int bsr2_spmv(const rs_bsr2 *J, const double *x, double *y, cudaStream_t stream);
/* r = b - J x (FP64). */
int bsr2_residual(const rs_bsr2 *J, const double *x, const double *b, double *r,
                  cudaStream_t stream);

/* ILU(0) (Sec. 3.3: the first stage P1 of CPR, Algorithms 1 and 2) of the
 * point-ordered scalar matrix of J: rows 2i, 2i+1 per cell, the pattern of
 * J's blocks with their structural zeros, no fill. Factored in IKJ order
 * (a zero pivot skips the elimination; the solve then divides by one) and
 * applied as the forward and backward triangular solves, both level-scheduled
 * over the cells: each phase is one launch of a single thread-block cluster
 * (1..8 CTAs) walking the levels with a cluster barrier. J's block pattern
 * must be structurally symmetric with every diagonal block present
 * (RS_EINVAL otherwise). The factors are computed in FP64; precision
 * (RS_PREC_*) is the arithmetic of the solves (FP32: the factors rounded
 * once, RS_ESETUP if one leaves the FP32 range; vectors stay FP64). Inside
 * CPR the solves take the V-cycle precision. The handle keeps a reference to
 * J's row_ptr and col and its own copy of the factors; J.val may change
 * afterwards. (sync) */
int ilu0_create(const rs_bsr2 *J, int32_t precision, rs_ilu0 **out, cudaStream_t stream);
/* x = (L U)^{-1} b; b, x [2 nb], not aliased. */
int ilu0_apply(const rs_ilu0 *F, const double *b, double *x, cudaStream_t stream);
/* Level count, widest level and CTAs per cluster of the schedule. */
int ilu0_info(const rs_ilu0 *F, int32_t *nlevels, int32_t *max_width, int32_t *cluster_ctas);
/* Copy of the factors into lu (device [4 nnzb], J's block layout:
 * lu[4k + 2r + c] is the entry of scalar row 2i+r, column 2 col[k] + c;
 * L strictly lower with unit diagonal, U upper). */
int ilu0_factors(const rs_ilu0 *F, double *lu, cudaStream_t stream);
int ilu0_destroy(rs_ilu0 *F);

/* ------------------------------------------------------ introspection --- */
/* Number of levels of a hierarchy, and level l's size and stored entries
 * (host outputs; sync). */
int amg_levels(const rs_amg *H, int32_t *nlevels);
int amg_level_info(const rs_amg *H, int32_t l, int32_t *n, int32_t *nnz, int32_t *nnz_p,
                   int32_t *ncolours);
/* Copies of level l (device outputs, any may be NULL): A_l in CSR, the C/F
 * marks of level l (1 C, -1 F, int8 [n]), P_l in CSR (n x n_{l+1}),
 * colours int32 [n]. */
int amg_level_copy(const rs_amg *H, int32_t l, int32_t *a_row_ptr, int32_t *a_col, double *a_val,
                   int8_t *cf, int32_t *p_row_ptr, int32_t *p_col, double *p_val, int32_t *colour,
                   cudaStream_t stream);
/* `sweeps` sweeps of level l's smoother on the hierarchy's own work vectors
 * (right-hand side as left by the last cycle), for measuring the smoother in
 * isolation; *bytes_per_sweep receives the algorithmic bytes one sweep moves
 * (matrix entries, row pointers, and the vectors read and written once). */
int amg_level_smooth(const rs_amg *H, int32_t l, int32_t sweeps, double *bytes_per_sweep, cudaStream_t stream);
/* `reps` back-to-back launches of one transfer kernel of the V-cycle on
 * level l (l below the coarsest), on the hierarchy's own work vectors, for
 * measuring it in isolation: which = 0 residual r_l = b_l - A_l x_l,
 * 1 restriction b_{l+1} = R_l r_l, 2 prolongation with correction
 * x_l += P_l x_{l+1}. *bytes_per_launch receives the algorithmic bytes of one
 * launch (matrix entries and row pointers, vectors read and written once).
 * RS_EINVAL for a level without a coarser one or an unknown `which`. */
int amg_level_transfer(const rs_amg *H, int32_t l, int32_t which, int32_t reps, double *bytes_per_launch,
                       cudaStream_t stream);

/* Hierarchy inside a preconditioner: which = 0 pressure / Schur / black-box,
 * 1 saturation. NULL if absent. */
const rs_amg *precond_amg(const rs_precond *M, int32_t which);

#ifdef __cplusplus
}
#endif
#endif
