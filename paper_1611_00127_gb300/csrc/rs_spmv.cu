// 2x2-block CSR SpMV, FP64: y = J x and r = b - J x (Sec. 3, eq. precon-system:
// the operator of every Krylov step). HBM-bound: each stored block moves 32 B
// of values and 4 B of column index and costs 4 FP64 FMAs.
//
// Layout: a group of LPR consecutive lanes owns one block row; lane l reads
// blocks start+l, start+l+LPR, ... so a warp's value loads are contiguous
// 32-byte blocks (fully coalesced) and x is gathered as one 16-byte (P_w, S_n)
// pair per block. Partial sums are combined with shuffles inside the group.
#include "rs_internal.cuh"

namespace rs {

template <int LPR, bool RESID>
__global__ void __launch_bounds__(256) k_bsr2_spmv(int32_t nb, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ col,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ x,
                                                   const double *__restrict__ b, double *__restrict__ y,
                                                   const uint8_t *__restrict__ act,
                                                   const int32_t *__restrict__ rseg) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / LPR;
  const int lane = threadIdx.x % LPR;
  double y0 = 0.0, y1 = 0.0;
  // a row of a retired system of a batch (act[system] = 0) gets y = 0
  // without reading its blocks
  const bool live = row < nb && (act == nullptr || act[rseg[row]]);
  if (live) {
    const int32_t s = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
    for (int32_t k = s + lane; k < e; k += LPR) {
      const double2 v01 = __ldg(reinterpret_cast<const double2 *>(val) + 2 * (int64_t)k);
      const double2 v23 = __ldg(reinterpret_cast<const double2 *>(val) + 2 * (int64_t)k + 1);
      const double2 xv = __ldg(reinterpret_cast<const double2 *>(x) + __ldg(col + k));
      y0 = fma(v01.x, xv.x, y0);
      y0 = fma(v01.y, xv.y, y0);
      y1 = fma(v23.x, xv.x, y1);
      y1 = fma(v23.y, xv.y, y1);
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) {
    y0 += __shfl_down_sync(0xffffffffu, y0, o, LPR);
    y1 += __shfl_down_sync(0xffffffffu, y1, o, LPR);
  }
  if (row < nb && lane == 0) {
    double2 out;
    if (!live) {
      out = make_double2(0.0, 0.0);
    } else if (RESID) {
      const double2 bv = reinterpret_cast<const double2 *>(b)[row];
      out = make_double2(bv.x - y0, bv.y - y1);
    } else {
      out = make_double2(y0, y1);
    }
    reinterpret_cast<double2 *>(y)[row] = out;
  }
}

static int g_bsr2_lpr = 4;   // lanes per block row; set by the tuner

extern "C" int rs_tune_set_bsr2_lpr(int lpr) {
  if (lpr != 1 && lpr != 2 && lpr != 4 && lpr != 8) return RS_EINVAL;
  g_bsr2_lpr = lpr;
  return RS_OK;
}

template <bool RESID>
static int launch(const rs_bsr2 &J, const double *x, const double *b, double *y, cudaStream_t s,
                  const uint8_t *act = nullptr, const int32_t *rseg = nullptr) {
  if (J.nb <= 0) return 0;
  const int64_t threads = (int64_t)J.nb * g_bsr2_lpr;
  const unsigned grid = grid_for(threads);
  ProfScope ps(kProfBsr2, J.nnzb * 36.0 + (J.nb + 1) * 4.0 + J.nb * (RESID ? 48.0 : 32.0), s);
  switch (g_bsr2_lpr) {
    case 1: RS_COUNTED k_bsr2_spmv<1, RESID><<<grid, kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, x, b, y, act, rseg); break;
    case 2: RS_COUNTED k_bsr2_spmv<2, RESID><<<grid, kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, x, b, y, act, rseg); break;
    case 8: RS_COUNTED k_bsr2_spmv<8, RESID><<<grid, kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, x, b, y, act, rseg); break;
    default: RS_COUNTED k_bsr2_spmv<4, RESID><<<grid, kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, x, b, y, act, rseg); break;
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int launch_bsr2_spmv(const rs_bsr2 &J, const double *x, double *y, cudaStream_t s, const uint8_t *act,
                     const int32_t *rseg) {
  return launch<false>(J, x, nullptr, y, s, act, rseg);
}

int launch_bsr2_residual(const rs_bsr2 &J, const double *x, const double *b, double *r, cudaStream_t s) {
  return launch<true>(J, x, b, r, s);
}

}  // namespace rs

using namespace rs;

static int check_bsr2(const rs_bsr2 *J) {
  if (!J || J->nb < 0 || J->nnzb < 0 || (J->nb > 0 && (!J->row_ptr || !J->col || !J->val)))
    return fail(RS_EINVAL, "invalid block matrix");
  return 0;
}

extern "C" int bsr2_spmv(const rs_bsr2 *J, const double *x, double *y, cudaStream_t stream) {
  RS_TRY(check_bsr2(J));
  if ((!x || !y) && J->nb > 0) return fail(RS_EINVAL, "null vector");
  return launch_bsr2_spmv(*J, x, y, stream);
}

extern "C" int bsr2_residual(const rs_bsr2 *J, const double *x, const double *b, double *r,
                             cudaStream_t stream) {
  RS_TRY(check_bsr2(J));
  if ((!x || !b || !r) && J->nb > 0) return fail(RS_EINVAL, "null vector");
  return launch_bsr2_residual(*J, x, b, r, stream);
}

// Autotuner: times y = J x for each lanes-per-row choice (CUDA events on the
// caller's stream, after a warm-up) and keeps the fastest.
extern "C" int rs_autotune_bsr2(const rs_bsr2 *J, const double *x, double *y, int *best, cudaStream_t stream) {
  RS_TRY(check_bsr2(J));
  if ((!x || !y) && J->nb > 0) return fail(RS_EINVAL, "null vector");
  const int cand[4] = {1, 2, 4, 8};
  float bt = 1e30f;
  int bl = g_bsr2_lpr;
  cudaEvent_t e0, e1;
  RS_CHECK_CUDA(cudaEventCreate(&e0));
  RS_CHECK_CUDA(cudaEventCreate(&e1));
  for (int c : cand) {
    g_bsr2_lpr = c;
    for (int w = 0; w < 3; w++) RS_TRY(launch_bsr2_spmv(*J, x, y, stream));
    RS_CHECK_CUDA(cudaEventRecord(e0, stream));
    for (int r = 0; r < 10; r++) RS_TRY(launch_bsr2_spmv(*J, x, y, stream));
    RS_CHECK_CUDA(cudaEventRecord(e1, stream));
    RS_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < bt) { bt = ms; bl = c; }
  }
  g_bsr2_lpr = bl;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best) *best = bl;
  return RS_OK;
}
