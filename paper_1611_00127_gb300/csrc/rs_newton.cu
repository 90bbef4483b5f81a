// One backward-Euler step by Newton's method (Sec. 3): J(u_k) du = -F(u_k),
// u_{k+1} = u_k + du with S_n clamped to [0, 1 - S_wr - 1e-12] (and, when
// asked, each cell's S_n change cut to +-max_ds: an Appleyard chop), until the
// scaled residual max |F_a,i| dt / (V phi rho_a) is at most ftol. Each
// iteration re-assembles F and the exact J, rebuilds the preconditioner and
// solves with FGMRES; several grids may be stepped together as one batch.
#include <chrono>
#include <cmath>

#include "rs_internal.cuh"

namespace rs {
int scaled_fnorm(const rs_problem *probs, int32_t nprob, const double *F, double dt, double *out, cudaStream_t s);
int newton_update(const rs_problem *probs, int32_t nprob, const double *du, double sign, double max_ds, double *u,
                  cudaStream_t s);
}  // namespace rs
using namespace rs;

static double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

extern "C" int newton_step(const rs_problem *probs, int32_t nprob, double *u, const double *u_old, double dt,
                           const rs_newton_params *params, rs_newton_stats *stats, cudaStream_t s) {
  if (!probs || nprob < 1 || !u || !u_old || !params) return fail(RS_EINVAL, "null argument");
  if (params->max_newton < 0) return fail(RS_EINVAL, "bad Newton limit");
  const int64_t nnzb = rs_bsr2_nnzb(probs, nprob);
  std::vector<int32_t> off(nprob + 1, 0);
  int64_t tot = 0;
  for (int32_t k = 0; k < nprob; k++) {
    if (probs[k].nx < 1 || probs[k].ny < 1 || probs[k].nz < 1) return fail(RS_EINVAL, "bad grid dimensions");
    tot += (int64_t)probs[k].nx * probs[k].ny * (probs[k].dim == 3 ? probs[k].nz : 1);
    if (tot > 0x3fffffff) return fail(RS_EINVAL, "too many cells");
    off[k + 1] = (int32_t)tot;
  }
  const int32_t nb = off[nprob];
  if (nnzb < 0 || nnzb > 0x7fffffff) return fail(RS_EINVAL, "pattern too large");
  Scratch sc(s);
  int32_t *rowptr = nullptr, *col = nullptr;
  double *val = nullptr, *F = nullptr, *du = nullptr;
  RS_TRY(sc.get(&rowptr, (size_t)nb + 1));
  RS_TRY(sc.get(&col, (size_t)nnzb));
  RS_TRY(sc.get(&val, 4 * (size_t)nnzb));
  RS_TRY(sc.get(&F, 2 * (size_t)nb));
  RS_TRY(sc.get(&du, 2 * (size_t)nb));
  RS_TRY(rs_bsr2_pattern(probs, nprob, rowptr, col, s));
  rs_bsr2 J{nb, (int32_t)nnzb, rowptr, col, val, nprob, off.data()};
  rs_newton_stats st{};
  if (stats) *stats = st;
  // every return from here on reports the work done so far in `stats`
#define NEWTON_TRY(expr)            \
  do {                              \
    const int r__ = (expr);         \
    if (r__ < 0) {                  \
      st.newton_its = k;            \
      if (stats) *stats = st;       \
      return r__;                   \
    }                               \
  } while (0)
  int status = RS_NOT_CONVERGED;
  bool nonfinite = false;   // the residual became NaN or infinite: the step failed
  int k = 0;
  for (;; k++) {
    auto t0 = std::chrono::steady_clock::now();
    NEWTON_TRY(jacobian_assemble(probs, nprob, u, u_old, dt, &J, F, s));
    double fn = 0.0;
    NEWTON_TRY(scaled_fnorm(probs, nprob, F, dt, &fn, s));
    st.assemble_ms += ms_since(t0);
    st.fnorm = fn;
    if (fn <= params->ftol) { status = RS_OK; break; }
    if (k >= params->max_newton) break;
    if (!std::isfinite(fn)) { nonfinite = true; break; }
    NEWTON_TRY(cudaMemsetAsync(du, 0, sizeof(double) * 2 * (size_t)nb, s) == cudaSuccess ? 0 : fail(RS_ECUDA, "cudaMemsetAsync"));
    t0 = std::chrono::steady_clock::now();
    rs_precond *M = nullptr;
    NEWTON_TRY(precond_create(&J, &params->prec, &M, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      precond_destroy(M);
      NEWTON_TRY(fail(RS_ECUDA, "cudaStreamSynchronize after the preconditioner set-up"));
    }
    st.setup_ms += ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    // solve J du = -F as J (-du) = F and negate afterwards
    rs_gmres_stats gs{};
    int r = gmres_solve(&J, M, F, du, &params->gmres, &gs, s);
    precond_destroy(M);
    st.solve_ms += ms_since(t0);
    st.linear_its += gs.iterations;
    if (r < 0) {
      st.newton_its = k + 1;
      if (stats) *stats = st;
      return r;
    }
    if (r == RS_NOT_CONVERGED) { status = RS_NOT_CONVERGED; st.newton_its = k + 1; break; }
    // u -= du (du solves J du = F)
    NEWTON_TRY(newton_update(probs, nprob, du, -1.0, params->max_ds, u, s));
  }
  if (nonfinite || status == RS_OK || k >= params->max_newton) st.newton_its = k;
  if (stats) *stats = st;
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  return status;
#undef NEWTON_TRY
}
