// AMG V(nu1, nu2)-cycle (Sec. 3.2: one V-cycle per preconditioner application,
// Sec. 4), in FP32 (values, vectors and sums) or FP64, with the coarsest
// levels solved by a dense FP64 inverse.
//
// Every kernel here streams CSR rows from HBM: a group of LPR lanes owns a row
// and strides over its entries (coalesced column/value loads, one gathered x
// per entry), then reduces with shuffles. LPR is picked per level from the
// mean row length. Per level: multicolour Gauss-Seidel sweeps (one launch per
// colour, rows of a colour taken from a per-colour row list, no two rows of a
// colour coupled, so each sweep is an exact Gauss-Seidel update in colour
// order), residual, restriction by R = P^T, recursion, prolongation with
// correction, post-sweeps.
#include "rs_internal.cuh"

namespace rs {

template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_gs_colour(int32_t nrows, const int32_t *__restrict__ rows,
                                                   const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                   const T *__restrict__ val, const T *__restrict__ dinv,
                                                   const T *__restrict__ b, T *x) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = tid / LPR;
  const int lane = threadIdx.x % LPR;
  int32_t i = -1;
  T s = T(0);
  if (r < nrows) {
    i = __ldg(rows + r);
    const int32_t e = __ldg(rp + i + 1);
    for (int32_t k = __ldg(rp + i) + lane; k < e; k += LPR) {
      const int32_t j = __ldg(col + k);
      if (j != i) s += __ldg(val + k) * x[j];
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LPR);
  if (i >= 0 && lane == 0) {
    const T di = __ldg(dinv + i);
    if (di != T(0)) x[i] = (__ldg(b + i) - s) * di;
  }
}

// t_i = b_i - (A x)_i for listed rows (first half of an l1-Jacobi sweep)
template <typename T, int LPR>
__global__ void __launch_bounds__(256) k_resid_rows(int32_t nrows, const int32_t *__restrict__ rows,
                                                    const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                    const T *__restrict__ val, const T *__restrict__ b,
                                                    const T *__restrict__ x, T *__restrict__ t) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = tid / LPR;
  const int lane = threadIdx.x % LPR;
  int32_t i = -1;
  T s = T(0);
  if (r < nrows) {
    i = __ldg(rows + r);
    const int32_t e = __ldg(rp + i + 1);
    for (int32_t k = __ldg(rp + i) + lane; k < e; k += LPR) s += __ldg(val + k) * __ldg(x + __ldg(col + k));
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LPR);
  if (i >= 0 && lane == 0) t[i] = __ldg(b + i) - s;
}

template <typename T>
__global__ void k_jacobi_update(int32_t nrows, const int32_t *__restrict__ rows, const T *__restrict__ inv,
                                const T *__restrict__ t, T *__restrict__ x) {
  int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int32_t i = rows[r];
  x[i] += t[i] * inv[i];
}

// y = b - A x over all rows (b == nullptr: y = A x); `accum`: y += A x
template <typename T, int LPR, int MODE>
__global__ void __launch_bounds__(256) k_csr(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                             const T *__restrict__ val, const T *__restrict__ x,
                                             const T *__restrict__ b, T *__restrict__ y) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = tid / LPR;
  const int lane = threadIdx.x % LPR;
  T s = T(0);
  if (i < n) {
    const int32_t e = __ldg(rp + i + 1);
    for (int32_t k = __ldg(rp + i) + lane; k < e; k += LPR) s += __ldg(val + k) * __ldg(x + __ldg(col + k));
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LPR);
  if (i < n && lane == 0) {
    if (MODE == 0) y[i] = s;                 // y = A x
    else if (MODE == 1) y[i] = b[i] - s;     // y = b - A x
    else y[i] += s;                          // y += A x
  }
}

// x[row] = A_c^{-1} b over the systems solved directly at this level, FP64
template <typename T>
__global__ void k_coarse_solve(int32_t nrows, const int32_t *__restrict__ crows, const int32_t *__restrict__ crow_seg,
                               const int4 *__restrict__ info, const int64_t *__restrict__ inv_off,
                               const double *__restrict__ inv, const T *__restrict__ b, T *__restrict__ x) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int32_t row = crows[w];
  const int32_t q = crow_seg[w];
  const int4 in = info[q];
  const int32_t r0 = in.x, n = in.y;
  const double *a = inv + inv_off[q] + (int64_t)(row - r0) * n;
  double s = 0.0;
  for (int32_t c = lane; c < n; c += 32) s = fma(a[c], (double)b[r0 + c], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = (T)s;
}

template <typename A, typename B>
__global__ void k_cast(int64_t n, const A *__restrict__ a, B *__restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

static int pick_lpr(int32_t n, int32_t nnz) {
  const double avg = n > 0 ? (double)nnz / n : 1.0;
  if (avg <= 6.0) return 4;
  if (avg <= 14.0) return 8;
  if (avg <= 40.0) return 16;
  return 32;
}

#define RS_LPR_SWITCH(lpr, ...)                  \
  switch (lpr) {                                 \
    case 4: { constexpr int L_ = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int L_ = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int L_ = 16; __VA_ARGS__; } break; \
    default: { constexpr int L_ = 32; __VA_ARGS__; } break; \
  }

template <typename T>
static const T *vals(const DCsr &A);
template <>
const float *vals<float>(const DCsr &A) { return A.valf; }
template <>
const double *vals<double>(const DCsr &A) { return A.val; }

template <typename T>
static const T *dinv_of(const Level &L);
template <>
const float *dinv_of<float>(const Level &L) { return L.dinvf; }
template <>
const double *dinv_of<double>(const Level &L) { return L.dinv; }

template <typename T>
static void smooth(const Hier &H, const Level &L, int sweeps, cudaStream_t s) {
  if (L.nsmooth == 0 || sweeps <= 0) return;
  const int lpr = pick_lpr(L.A.n, L.A.nnz);
  const T *val = vals<T>(L.A);
  const T *dinv = dinv_of<T>(L);
  T *x = static_cast<T *>(L.x);
  const T *b = static_cast<const T *>(L.b);
  for (int sw = 0; sw < sweeps; sw++) {
    if (H.prm.smoother == RS_SMOOTH_L1JACOBI) {
      T *t = static_cast<T *>(L.t);
      const int32_t nr = L.nsmooth;
      RS_LPR_SWITCH(lpr, k_resid_rows<T, L_><<<grid_for((int64_t)nr * L_), kBlock, 0, s>>>(
                             nr, L.colour_rows, L.A.rowptr, L.A.col, val, b, x, t));
      k_jacobi_update<T><<<grid_for(nr), kBlock, 0, s>>>(nr, L.colour_rows, dinv, t, x);
    } else {
      for (int c = 0; c < L.ncolour; c++) {
        const int32_t r0 = L.colour_off[c], nr = L.colour_off[c + 1] - r0;
        if (nr == 0) continue;
        RS_LPR_SWITCH(lpr, k_gs_colour<T, L_><<<grid_for((int64_t)nr * L_), kBlock, 0, s>>>(
                               nr, L.colour_rows + r0, L.A.rowptr, L.A.col, val, dinv, b, x));
      }
    }
  }
}

template <typename T>
static void cycle(const Hier &H, int32_t l, cudaStream_t s) {
  const Level &L = H.L[l];
  T *x = static_cast<T *>(L.x);
  if (L.A.n > 0) cudaMemsetAsync(x, 0, sizeof(T) * (size_t)L.A.n, s);
  smooth<T>(H, L, H.prm.nu1, s);
  if (l + 1 < H.nlev && L.P.rowptr) {
    const Level &N = H.L[l + 1];
    T *r = static_cast<T *>(L.r);
    const int lpr = pick_lpr(L.A.n, L.A.nnz);
    RS_LPR_SWITCH(lpr, k_csr<T, L_, 1><<<grid_for((int64_t)L.A.n * L_), kBlock, 0, s>>>(
                           L.A.n, L.A.rowptr, L.A.col, vals<T>(L.A), x, static_cast<const T *>(L.b), r));
    const int lr = pick_lpr(L.R.n, L.R.nnz);
    RS_LPR_SWITCH(lr, k_csr<T, L_, 0><<<grid_for((int64_t)L.R.n * L_), kBlock, 0, s>>>(
                          L.R.n, L.R.rowptr, L.R.col, vals<T>(L.R), r, nullptr, static_cast<T *>(N.b)));
    cycle<T>(H, l + 1, s);
    const int lp = pick_lpr(L.P.n, L.P.nnz);
    RS_LPR_SWITCH(lp, k_csr<T, L_, 2><<<grid_for((int64_t)L.P.n * L_), kBlock, 0, s>>>(
                          L.P.n, L.P.rowptr, L.P.col, vals<T>(L.P), static_cast<const T *>(N.x), nullptr, x));
  }
  smooth<T>(H, L, H.prm.nu2, s);
  if (L.ncoarse_rows > 0) {
    k_coarse_solve<T><<<grid_for((int64_t)L.ncoarse_rows * 32), kBlock, 0, s>>>(
        L.ncoarse_rows, L.crows, L.crow_seg, L.cinfo, L.cinv_off, L.cinv, static_cast<const T *>(L.b), x);
  }
}

int amg_vcycle(const Hier &H, const double *b, double *x, cudaStream_t s) {
  if (H.nlev == 0) return fail(RS_EINVAL, "empty hierarchy");
  const Level &L0 = H.L[0];
  const int64_t n = L0.A.n;
  if (n == 0) return 0;
  if (H.precision == RS_PREC_FP32) {
    k_cast<double, float><<<grid_for(n), kBlock, 0, s>>>(n, b, static_cast<float *>(L0.b));
    cycle<float>(H, 0, s);
    k_cast<float, double><<<grid_for(n), kBlock, 0, s>>>(n, static_cast<const float *>(L0.x), x);
  } else {
    RS_CHECK_CUDA(cudaMemcpyAsync(L0.b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    cycle<double>(H, 0, s);
    RS_CHECK_CUDA(cudaMemcpyAsync(x, L0.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace rs
