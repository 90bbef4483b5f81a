// C-ABI for stand-alone AMG hierarchies and level introspection.
#include "rs_internal.cuh"

using namespace rs;

namespace rs {
// Host-side check of AMG parameters (RS_EINVAL with a message naming the
// parameter); shared by amg_setup and precond_create.
int check_amg_params(const rs_amg_params &a) {
  if (!(a.theta >= 0.0 && a.theta <= 1.0)) return fail(RS_EINVAL, "theta outside [0,1]");
  if (a.max_levels < 1 || a.coarse_n < 1 || a.max_dense < 1 || a.max_dense > 8192)
    return fail(RS_EINVAL, "bad level limits");
  if (a.smoother != RS_SMOOTH_MCGS && a.smoother != RS_SMOOTH_L1JACOBI && a.smoother != RS_SMOOTH_HYBRID)
    return fail(RS_EINVAL, "bad smoother");
  if (a.smoother == RS_SMOOTH_HYBRID && (a.chunk < 32 || a.chunk > 512)) return fail(RS_EINVAL, "chunk outside [32, 512]");
  if (a.num_functions < 0 || a.num_functions > 2) return fail(RS_EINVAL, "num_functions must be 1 or 2");
  if (a.nu1 < 0 || a.nu2 < 0 || a.nu1 > 16 || a.nu2 > 16) return fail(RS_EINVAL, "bad sweep counts");
  if (a.interp != RS_INTERP_CLASSICAL && a.interp != RS_INTERP_EXTI) return fail(RS_EINVAL, "bad interpolation");
  if (a.precision != RS_PREC_FP32 && a.precision != RS_PREC_FP64) return fail(RS_EINVAL, "bad precision");
  if (a.agg_levels < 0 || a.agg_levels > 8) return fail(RS_EINVAL, "agg_levels outside [0, 8]");
  if (a.chunk_coarse != 0 && (a.chunk_coarse < 32 || a.chunk_coarse > 512))
    return fail(RS_EINVAL, "chunk_coarse outside [32, 512]");
  if (a.restriction != 0 && a.restriction != 1 && a.restriction != 3)
    return fail(RS_EINVAL, "restriction must be 0 (Galerkin), 1 (AIR, distance 1) or 3 (lAIR)");
  return 0;
}
}  // namespace rs

extern "C" int amg_setup(const rs_csr *A, const rs_amg_params *params, rs_amg **H, cudaStream_t stream) {
  if (!H) return fail(RS_EINVAL, "null output handle");
  *H = nullptr;
  if (!A || !params || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->row_ptr || !A->col || !A->val)))
    return fail(RS_EINVAL, "invalid matrix");
  RS_TRY(check_amg_params(*params));
  std::vector<int32_t> off = seg_offsets(A->n, A->nseg, A->seg_off);
  if (off.front() != 0 || off.back() != A->n) return fail(RS_EINVAL, "segment offsets must run from 0 to n");
  DCsr view;
  view.n = view.m = A->n;
  view.nnz = A->nnz;
  view.rowptr = const_cast<int32_t *>(A->row_ptr);
  view.col = const_cast<int32_t *>(A->col);
  view.val = const_cast<double *>(A->val);
  rs_amg *h = new rs_amg();
  h->stream = stream;
  int r = amg_build(view, off, *params, h->H, stream);
  if (r) {
    cudaStreamSynchronize(stream);
    amg_free(h->H, stream);
    cudaStreamSynchronize(stream);
    delete h;
    return r;
  }
  *H = h;
  return RS_OK;
}

extern "C" int amg_destroy(rs_amg *H) {
  if (!H) return RS_OK;
  cudaStreamSynchronize(H->stream);
  amg_free(H->H, H->stream);
  cudaStreamSynchronize(H->stream);
  delete H;
  return RS_OK;
}

extern "C" int amg_apply(const rs_amg *H, const double *b, double *x, cudaStream_t stream) {
  if (!H) return fail(RS_EINVAL, "null argument");
  if ((!b || !x) && H->H.nlev > 0 && H->H.L[0].A.n > 0) return fail(RS_EINVAL, "null argument");
  return amg_vcycle(H->H, b, x, stream);
}

extern "C" int amg_levels(const rs_amg *H, int32_t *nlevels) {
  if (!H || !nlevels) return fail(RS_EINVAL, "null argument");
  *nlevels = H->H.nlev;
  return RS_OK;
}

extern "C" int amg_level_info(const rs_amg *H, int32_t l, int32_t *n, int32_t *nnz, int32_t *nnz_p,
                              int32_t *ncolours) {
  if (!H || l < 0 || l >= H->H.nlev) return fail(RS_EINVAL, "level out of range");
  const Level &L = H->H.L[l];
  if (n) *n = L.A.n;
  if (nnz) *nnz = L.A.nnz;
  if (nnz_p) *nnz_p = L.P.rowptr ? L.P.nnz : 0;
  if (ncolours) *ncolours = L.ncolour;
  return RS_OK;
}

__global__ void k_fill_i8(int32_t n, int8_t v, int8_t *a) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}
__global__ void k_fill_i32(int32_t n, int32_t v, int32_t *a) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

extern "C" int amg_level_copy(const rs_amg *H, int32_t l, int32_t *a_row_ptr, int32_t *a_col, double *a_val,
                              int8_t *cf, int32_t *p_row_ptr, int32_t *p_col, double *p_val, int32_t *colour,
                              cudaStream_t s) {
  if (!H || l < 0 || l >= H->H.nlev) return fail(RS_EINVAL, "level out of range");
  const Level &L = H->H.L[l];
  const size_t n = (size_t)L.A.n;
  if (a_row_ptr) RS_CHECK_CUDA(cudaMemcpyAsync(a_row_ptr, L.A.rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
  if (a_col) RS_CHECK_CUDA(cudaMemcpyAsync(a_col, L.A.col, sizeof(int32_t) * L.A.nnz, cudaMemcpyDeviceToDevice, s));
  if (a_val) RS_CHECK_CUDA(cudaMemcpyAsync(a_val, L.A.val, sizeof(double) * L.A.nnz, cudaMemcpyDeviceToDevice, s));
  if (cf) {
    if (L.cf) RS_CHECK_CUDA(cudaMemcpyAsync(cf, L.cf, n, cudaMemcpyDeviceToDevice, s));
    else if (n) RS_COUNTED k_fill_i8<<<grid_for(n), kBlock, 0, s>>>((int32_t)n, 0, cf);
  }
  if (L.P.rowptr) {
    if (p_row_ptr) RS_CHECK_CUDA(cudaMemcpyAsync(p_row_ptr, L.P.rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    if (p_col) RS_CHECK_CUDA(cudaMemcpyAsync(p_col, L.P.col, sizeof(int32_t) * L.P.nnz, cudaMemcpyDeviceToDevice, s));
    if (p_val) RS_CHECK_CUDA(cudaMemcpyAsync(p_val, L.P.val, sizeof(double) * L.P.nnz, cudaMemcpyDeviceToDevice, s));
  }
  if (colour) {
    if (L.colour) RS_CHECK_CUDA(cudaMemcpyAsync(colour, L.colour, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    else if (n) RS_COUNTED k_fill_i32<<<grid_for(n), kBlock, 0, s>>>((int32_t)n, -2, colour);
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return RS_OK;
}

extern "C" int amg_level_smooth(const rs_amg *H, int32_t l, int32_t sweeps, double *bytes_per_sweep,
                                cudaStream_t stream) {
  if (!H || sweeps < 0) return fail(RS_EINVAL, "invalid arguments");
  return amg_level_sweeps(H->H, l, sweeps, bytes_per_sweep, stream);
}

extern "C" int amg_level_transfer(const rs_amg *H, int32_t l, int32_t which, int32_t reps, double *bytes_per_launch,
                                  cudaStream_t stream) {
  if (!H || reps < 0) return fail(RS_EINVAL, "invalid arguments");
  return rs::amg_level_xfer(H->H, l, which, reps, bytes_per_launch, stream);
}
