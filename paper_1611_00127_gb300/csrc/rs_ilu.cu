// ILU(0) of the point-ordered scalar matrix of a 2x2-block BSR matrix: the
// first stage P1 of CPR (Sec. 3.3, Algorithms 1 and 2), factored and applied
// on the GPU in level-scheduled form.
//
// The scalar matrix has rows 2c and 2c+1 for cell c; row 2c+r holds the
// entries (2 col[k] + cc), cc = 0, 1, of every block k of block row c -- the
// block pattern with its structural zeros. ILU(0) keeps exactly that pattern.
// In IKJ order row i eliminates its lower entries in ascending column order:
// for lower entry j, l = a_ij / u_jj (skipped when u_jj = 0), then every
// entry of row j right of its diagonal updates the entry of row i in the same
// column, when row i has one. The factors overwrite a copy of the values in
// the BSR layout: L strictly lower with a unit diagonal, U upper. The solve
// is L y = b forward, then U x = y backward (a zero pivot divides by one).
//
// Dependencies: row 2c+1 needs row 2c, and both need the rows of the
// lower-numbered neighbour cells. Cells are grouped into levels (Kahn's
// layering of that dependency DAG: level 0 has no lower neighbour, a cell
// sits one level above its highest lower neighbour); cells of one level are
// independent. Each phase -- layering, factorisation, forward + backward
// solve -- is one launch of a single thread-block cluster (1..8 CTAs of up to
// 1024 threads for the set-up and 512 for the solve, sized to the widest
// level) that walks the levels with a cluster barrier between them (hardware
// barrier; no spin loop). One thread
// handles both rows of a cell in the sequential algorithm's operation order,
// and this file is compiled without FMA contraction, so factors and solves
// round exactly as the sequential algorithm does. With FP32 solves (the
// mixed-precision preconditioner) the FP64 factors are rounded to FP32 once
// and both sweeps compute in FP32 -- GB300 issues FP32 at 64 times its FP64
// rate, and a level's arithmetic sits on the critical path; vectors stay FP64
// in memory. Values that other threads
// wrote earlier in the same launch are read with ld.global.cg (L2) when the
// cluster has several CTAs, so no stale L1 line is ever used; a single-CTA
// solve separates its levels by __syncthreads, which makes them visible to
// plain loads.
//
// The block pattern must be structurally symmetric (TPFA Jacobians are): the
// layering releases a cell's upper neighbours from its own row and the
// backward solve walks the levels in reverse. Set-up checks the symmetry and
// that the layering placed every cell once.
#include <cooperative_groups.h>

#include "rs_internal.cuh"

namespace cg = cooperative_groups;
using namespace rs;

struct rs_ilu0 {
  int32_t nb = 0, nnzb = 0;
  const int32_t *row_ptr = nullptr, *col = nullptr;   // caller's pattern (kept by reference)
  double *lu = nullptr;            // factors, BSR layout [4 nnzb]
  float *luf = nullptr;            // FP32 copy of the factors (FP32 solves) [4 nnzb]
  int precision = RS_PREC_FP64;    // arithmetic of the solves
  int32_t *dblk = nullptr;         // diagonal block of each block row [nb]
  int32_t *lvl_cells = nullptr;    // cells ordered by level [nb]
  int32_t *lvl_ptr = nullptr;      // level offsets [nb + 1]
  int32_t *nlev_d = nullptr;       // level count on the device [1]
  int4 *rec = nullptr;             // level-ordered solve records [3 nb]
  int32_t nlev = 0, maxw = 0;
  int cluster = 1, threads = 32;   // factorisation launch
  int cluster_s = 1, threads_s = 32;   // solve launch
  cudaStream_t stream = nullptr;
};

namespace {

constexpr int kIluThreads = 1024;       // layering and factorisation
constexpr int kIluSolveThreads = 512;   // triangular solves (room for the prefetched records)
constexpr int kIluMaxCluster = 8;

struct ClusterIdx {
  int64_t tid, nthreads;
};

__device__ __forceinline__ ClusterIdx cluster_idx() {
  cg::cluster_group cl = cg::this_cluster();
  return {(int64_t)cl.block_rank() * blockDim.x + threadIdx.x, (int64_t)cl.num_blocks() * blockDim.x};
}

// diagonal block of every block row, and the structural symmetry of the
// pattern: err |= 1 (no diagonal block), 2 (block (c,d) without (d,c)).
__global__ void k_ilu_check(int32_t nb, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                            int32_t *__restrict__ dblk, int32_t *__restrict__ err) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb) return;
  int32_t kd = -1;
  for (int32_t k = rowptr[c]; k < rowptr[c + 1]; k++) {
    const int32_t d = col[k];
    if (d == c) kd = k;
    if (d < 0 || d >= nb) { atomicOr(err, 2); continue; }
    int32_t lo = rowptr[d], hi = rowptr[d + 1];
    while (lo < hi) {
      const int32_t m = (lo + hi) >> 1;
      if (col[m] < c) lo = m + 1; else hi = m;
    }
    if (lo == rowptr[d + 1] || col[lo] != c) atomicOr(err, 2);
  }
  dblk[c] = kd;
  if (kd < 0) atomicOr(err, 1);
}

// Kahn's layering. cnt[t] counts the cells of level t (zeroed before the
// launch): level t's cells are lvl_cells[b, e); a cell released while level
// t is processed lands at e + atomicAdd(&cnt[t + 1], 1). Every thread keeps
// b, e and t itself; all read cnt[t + 1] only after the barrier that ends
// level t, and nothing writes it afterwards, so the loop is uniform over the
// cluster. lvl_ptr[0..nlev] receives the level offsets. ctrl: [0] level
// count, [1] widest level, [2] cells placed, [3] error (a cell released more
// often than it has lower neighbours).
__global__ void __launch_bounds__(kIluThreads, 1)
    k_ilu_levels(int32_t nb, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                 int32_t *__restrict__ indeg, int32_t *__restrict__ cnt, int32_t *__restrict__ lvl_cells,
                 int32_t *__restrict__ lvl_ptr, int32_t *__restrict__ nlev_d, int32_t *__restrict__ ctrl) {
  cg::cluster_group cl = cg::this_cluster();
  const ClusterIdx ix = cluster_idx();
  for (int64_t c = ix.tid; c < nb; c += ix.nthreads) {
    int32_t d = 0;
    for (int32_t k = rowptr[c]; k < rowptr[c + 1]; k++) d += col[k] < c;
    indeg[c] = d;
    if (d == 0) lvl_cells[atomicAdd(&cnt[0], 1)] = (int32_t)c;
  }
  cl.sync();
  int32_t b = 0, e = __ldcg(&cnt[0]), t = 0, maxw = e;
  if (ix.tid == 0) lvl_ptr[0] = 0;
  while (e > b && t < nb) {
    for (int64_t q = b + ix.tid; q < e; q += ix.nthreads) {
      const int32_t c = __ldcg(&lvl_cells[q]);
      for (int32_t k = rowptr[c]; k < rowptr[c + 1]; k++) {
        const int32_t d = col[k];
        if (d <= c) continue;
        const int32_t old = atomicSub(&indeg[d], 1);
        if (old == 1) lvl_cells[e + atomicAdd(&cnt[t + 1], 1)] = d;
        else if (old <= 0) atomicOr(&ctrl[3], 1);
      }
    }
    cl.sync();
    t++;
    b = e;
    e += __ldcg(&cnt[t]);
    maxw = max(maxw, e - b);
    if (ix.tid == 0) lvl_ptr[t] = b;
  }
  // here lvl_ptr[t] = b = e: the level offsets end with the cell count
  if (ix.tid == 0) {
    *nlev_d = t;
    ctrl[0] = t;
    ctrl[1] = maxw;
    ctrl[2] = e;
  }
}

// row 2c+r of cell c: position of column (2 cb + cc) in it, or -1
__device__ __forceinline__ int32_t find_block(const int32_t *__restrict__ col, int32_t kb, int32_t ke, int32_t cb) {
  for (int32_t k = kb; k < ke; k++) {
    const int32_t v = col[k];
    if (v == cb) return k;
    if (v > cb) break;
  }
  return -1;
}

// Eliminate lower entry (block k, column part cc) of row 2c+r: pivot row
// j = 2 col[k] + cc.
__device__ __forceinline__ void ilu_eliminate(int32_t c, int r, int32_t k, int cc, const int32_t *__restrict__ rowptr,
                                              const int32_t *__restrict__ col, const int32_t *__restrict__ dblk,
                                              double *lu) {
  const int32_t cp = col[k];
  const int32_t kdp = dblk[cp];
  const double dk = __ldcg(&lu[4 * (int64_t)kdp + 3 * cc]);
  if (dk == 0.0) return;
  double *q = &lu[4 * (int64_t)k + 2 * r + cc];
  const double l = *q / dk;
  *q = l;
  const int32_t kb = rowptr[c], ke = rowptr[c + 1];
  // row j right of its diagonal: the rest of its diagonal block, then the
  // blocks after it
  if (cc == 0) {
    const int32_t kt = find_block(col, kb, ke, cp);
    if (kt >= 0) lu[4 * (int64_t)kt + 2 * r + 1] -= l * __ldcg(&lu[4 * (int64_t)kdp + 1]);
  }
  const int32_t pe = rowptr[cp + 1];
  int32_t kt = kb;
  for (int32_t k2 = kdp + 1; k2 < pe; k2++) {
    const int32_t cj = col[k2];
    while (kt < ke && col[kt] < cj) kt++;
    if (kt == ke) break;
    if (col[kt] != cj) continue;
    lu[4 * (int64_t)kt + 2 * r] -= l * __ldcg(&lu[4 * (int64_t)k2 + 2 * cc]);
    lu[4 * (int64_t)kt + 2 * r + 1] -= l * __ldcg(&lu[4 * (int64_t)k2 + 2 * cc + 1]);
  }
}

__global__ void __launch_bounds__(kIluThreads, 1)
    k_ilu_factor(const int32_t *__restrict__ nlev_d, const int32_t *__restrict__ lvl_ptr,
                 const int32_t *__restrict__ lvl_cells, const int32_t *__restrict__ rowptr,
                 const int32_t *__restrict__ col, const int32_t *__restrict__ dblk, double *lu) {
  cg::cluster_group cl = cg::this_cluster();
  const ClusterIdx ix = cluster_idx();
  const int32_t nlev = *nlev_d;
  for (int32_t t = 0; t < nlev; t++) {
    const int32_t b = lvl_ptr[t], e = lvl_ptr[t + 1];
    for (int64_t q = b + ix.tid; q < e; q += ix.nthreads) {
      const int32_t c = lvl_cells[q];
      const int32_t kb = rowptr[c], kd = dblk[c];
      for (int r = 0; r < 2; r++) {
        for (int32_t k = kb; k < kd; k++) {
          ilu_eliminate(c, r, k, 0, rowptr, col, dblk, lu);
          ilu_eliminate(c, r, k, 1, rowptr, col, dblk, lu);
        }
        if (r == 1) ilu_eliminate(c, 1, kd, 0, rowptr, col, dblk, lu);
      }
    }
    cl.sync();
  }
}

// Level-ordered record of the cell at position q: {c, first block, diagonal
// block, end of row} and the columns of its first four lower and first four
// upper neighbour blocks (-1 past them). A solve thread reads one record
// (three int4) per cell, prefetched before the barrier that precedes the
// cell's level, so that after the barrier only the neighbours' x values
// (and the factor entries) are on the critical path.
__global__ void k_ilu_records(int32_t nb, const int32_t *__restrict__ lvl_cells, const int32_t *__restrict__ rowptr,
                              const int32_t *__restrict__ col, const int32_t *__restrict__ dblk,
                              int4 *__restrict__ rec) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nb) return;
  const int32_t c = lvl_cells[q], kb = rowptr[c], kd = dblk[c], ke = rowptr[c + 1];
  int32_t lo[4], up[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    lo[i] = kb + i < kd ? col[kb + i] : -1;
    up[i] = kd + 1 + i < ke ? col[kd + 1 + i] : -1;
  }
  rec[3 * q] = make_int4(c, kb, kd, ke);
  rec[3 * q + 1] = make_int4(lo[0], lo[1], lo[2], lo[3]);
  rec[3 * q + 2] = make_int4(up[0], up[1], up[2], up[3]);
}

__device__ __forceinline__ int32_t pick(const int4 v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// a value another thread of the launch wrote before the last barrier: within
// one CTA the barrier makes it visible to a plain (L1) load; across the CTAs
// of a cluster it is read from L2
template <bool ONE>
__device__ __forceinline__ double ld_shared_state(const double *p) {
  if constexpr (ONE) return *p;
  else return __ldcg(p);
}

template <bool ONE>
__device__ __forceinline__ void level_barrier() {
  if constexpr (ONE) __syncthreads();
  else cg::this_cluster().sync();
}

// forward rows 2c, 2c+1 of one cell (L y = b, unit diagonal); b0, b1 = b
template <bool ONE, typename T>
__device__ __forceinline__ void ilu_forward_cell(const int4 a, const int4 lo, T b0, T b1,
                                                 const int32_t *__restrict__ col, const T *__restrict__ lu,
                                                 double *x) {
  const int32_t c = a.x, kb = a.y, kd = a.z;
  const int32_t nl = kd - kb;
  T xa[4], xb[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nl) {
      const int64_t j = 2 * (int64_t)pick(lo, i);
      xa[i] = (T)ld_shared_state<ONE>(&x[j]);
      xb[i] = (T)ld_shared_state<ONE>(&x[j + 1]);
    }
  }
  T s0 = b0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nl) {
      const int64_t k = kb + i;
      s0 -= lu[4 * k] * xa[i];
      s0 -= lu[4 * k + 1] * xb[i];
    }
  }
  for (int32_t k = kb + 4; k < kd; k++) {
    const int64_t j = 2 * (int64_t)col[k];
    s0 -= lu[4 * (int64_t)k] * (T)ld_shared_state<ONE>(&x[j]);
    s0 -= lu[4 * (int64_t)k + 1] * (T)ld_shared_state<ONE>(&x[j + 1]);
  }
  x[2 * (int64_t)c] = (double)s0;
  T s1 = b1;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nl) {
      const int64_t k = kb + i;
      s1 -= lu[4 * k + 2] * xa[i];
      s1 -= lu[4 * k + 3] * xb[i];
    }
  }
  for (int32_t k = kb + 4; k < kd; k++) {
    const int64_t j = 2 * (int64_t)col[k];
    s1 -= lu[4 * (int64_t)k + 2] * (T)ld_shared_state<ONE>(&x[j]);
    s1 -= lu[4 * (int64_t)k + 3] * (T)ld_shared_state<ONE>(&x[j + 1]);
  }
  s1 -= lu[4 * (int64_t)kd + 2] * s0;
  x[2 * (int64_t)c + 1] = (double)s1;
}

// backward rows 2c+1, then 2c of one cell (U x = y); y0, y1 = the cell's y
template <bool ONE, typename T>
__device__ __forceinline__ void ilu_backward_cell(const int4 a, const int4 up, T y0, T y1,
                                                  const int32_t *__restrict__ col, const T *__restrict__ lu,
                                                  double *x) {
  const int32_t c = a.x, kd = a.z, ke = a.w;
  const int32_t nu = ke - kd - 1;
  T xa[4], xb[4];
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nu) {
      const int64_t j = 2 * (int64_t)pick(up, i);
      xa[i] = (T)ld_shared_state<ONE>(&x[j]);
      xb[i] = (T)ld_shared_state<ONE>(&x[j + 1]);
    }
  }
  T s1 = y1;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nu) {
      const int64_t k = kd + 1 + i;
      s1 -= lu[4 * k + 2] * xa[i];
      s1 -= lu[4 * k + 3] * xb[i];
    }
  }
  for (int32_t k = kd + 5; k < ke; k++) {
    const int64_t j = 2 * (int64_t)col[k];
    s1 -= lu[4 * (int64_t)k + 2] * (T)ld_shared_state<ONE>(&x[j]);
    s1 -= lu[4 * (int64_t)k + 3] * (T)ld_shared_state<ONE>(&x[j + 1]);
  }
  const T d1 = lu[4 * (int64_t)kd + 3];
  s1 = d1 != T(0) ? s1 / d1 : s1;
  x[2 * (int64_t)c + 1] = (double)s1;
  T s0 = y0;
  s0 -= lu[4 * (int64_t)kd + 1] * s1;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (i < nu) {
      const int64_t k = kd + 1 + i;
      s0 -= lu[4 * k] * xa[i];
      s0 -= lu[4 * k + 1] * xb[i];
    }
  }
  for (int32_t k = kd + 5; k < ke; k++) {
    const int64_t j = 2 * (int64_t)col[k];
    s0 -= lu[4 * (int64_t)k] * (T)ld_shared_state<ONE>(&x[j]);
    s0 -= lu[4 * (int64_t)k + 1] * (T)ld_shared_state<ONE>(&x[j + 1]);
  }
  const T d0 = lu[4 * (int64_t)kd];
  x[2 * (int64_t)c] = (double)(d0 != T(0) ? s0 / d0 : s0);
}

// x = U^{-1} L^{-1} b: the forward sweep over the levels, then the backward
// sweep over them in reverse. Position q of level t goes to thread
// q - lvl_ptr[t] (then + nthreads, ...), in both sweeps.
template <bool ONE, typename T>
__global__ void __launch_bounds__(kIluSolveThreads, 1)
    k_ilu_solve(const int32_t *__restrict__ nlev_d, const int32_t *__restrict__ lvl_ptr,
                const int4 *__restrict__ rec, const int32_t *__restrict__ col, const T *__restrict__ lu,
                const double *__restrict__ b, double *x) {
  const ClusterIdx ix = cluster_idx();
  const int32_t nlev = *nlev_d;
  int4 ra = make_int4(0, 0, 0, 0), rl = ra, ru = ra;
  T p0 = T(0), p1 = T(0);
  auto fetch = [&](int64_t q) {
    ra = rec[3 * q];
    rl = rec[3 * q + 1];
    ru = rec[3 * q + 2];
  };
  if (nlev > 0 && lvl_ptr[0] + ix.tid < lvl_ptr[1]) {
    fetch(lvl_ptr[0] + ix.tid);
    p0 = (T)b[2 * (int64_t)ra.x];
    p1 = (T)b[2 * (int64_t)ra.x + 1];
  }
  for (int32_t t = 0; t < nlev; t++) {
    const int32_t lb = lvl_ptr[t], le = lvl_ptr[t + 1];
    for (int64_t q = lb + ix.tid; q < le; q += ix.nthreads) {
      if (q != lb + ix.tid) {
        fetch(q);
        p0 = (T)b[2 * (int64_t)ra.x];
        p1 = (T)b[2 * (int64_t)ra.x + 1];
      }
      ilu_forward_cell<ONE, T>(ra, rl, p0, p1, col, lu, x);
    }
    if (t + 1 < nlev && le + ix.tid < lvl_ptr[t + 2]) {    // next level's first cell
      fetch(le + ix.tid);
      p0 = (T)b[2 * (int64_t)ra.x];
      p1 = (T)b[2 * (int64_t)ra.x + 1];
    }
    level_barrier<ONE>();
  }
  if (nlev > 0 && lvl_ptr[nlev - 1] + ix.tid < lvl_ptr[nlev]) {
    fetch(lvl_ptr[nlev - 1] + ix.tid);
    p0 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x]);
    p1 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x + 1]);
  }
  for (int32_t t = nlev - 1; t >= 0; t--) {
    const int32_t lb = lvl_ptr[t], le = lvl_ptr[t + 1];
    for (int64_t q = lb + ix.tid; q < le; q += ix.nthreads) {
      if (q != lb + ix.tid) {
        fetch(q);
        p0 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x]);
        p1 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x + 1]);
      }
      ilu_backward_cell<ONE, T>(ra, ru, p0, p1, col, lu, x);
    }
    // the previous level's first cell: its y values are final since the
    // forward sweep, and no thread writes them before its own turn
    if (t > 0 && lvl_ptr[t - 1] + ix.tid < lb) {
      fetch(lvl_ptr[t - 1] + ix.tid);
      p0 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x]);
      p1 = (T)ld_shared_state<ONE>(&x[2 * (int64_t)ra.x + 1]);
    }
    level_barrier<ONE>();
  }
}

// FP32 copy of the factors; err |= 1 where a value is not finite in FP32
__global__ void k_ilu_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ f, int32_t *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = (float)a[i];
  if (!isfinite(v)) atomicOr(err, 1);
  f[i] = v;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(void (*kern)(KArgs...), int cluster, int threads, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

void ilu_free(rs_ilu0 *F) {
  cudaStream_t s = F->stream;
  dfree(F->lu, s);
  dfree(F->dblk, s);
  dfree(F->lvl_cells, s);
  dfree(F->lvl_ptr, s);
  dfree(F->nlev_d, s);
  dfree(F->rec, s);
  dfree(F->luf, s);
  delete F;
}

}  // namespace

namespace rs {

int ilu0_build(const rs_bsr2 &J, int precision, rs_ilu0 **out, cudaStream_t s) {
  *out = nullptr;
  rs_ilu0 *F = new rs_ilu0();
  F->nb = J.nb;
  F->nnzb = J.nnzb;
  F->row_ptr = J.row_ptr;
  F->col = J.col;
  F->stream = s;
  F->precision = precision;
  const int32_t nb = J.nb;
  if (nb == 0) { *out = F; return 0; }
  int rc = 0;
  Scratch sc(s);
  int32_t *indeg = nullptr, *cnt = nullptr, *ctrl = nullptr;
  auto attempt = [&]() -> int {
    RS_TRY(dalloc_n(&F->lu, 4 * (size_t)J.nnzb, s));
    RS_TRY(dalloc_n(&F->dblk, (size_t)nb, s));
    RS_TRY(dalloc_n(&F->lvl_cells, (size_t)nb, s));
    RS_TRY(dalloc_n(&F->lvl_ptr, (size_t)nb + 1, s));
    RS_TRY(dalloc_n(&F->nlev_d, 1, s));
    RS_TRY(dalloc_n(&F->rec, 3 * (size_t)nb, s));
    RS_TRY(sc.get(&indeg, (size_t)nb));
    RS_TRY(sc.get(&cnt, (size_t)nb + 1));
    RS_TRY(sc.get(&ctrl, 5));
    RS_CHECK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)nb + 1), s));
    RS_CHECK_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(int32_t) * 5, s));
    RS_COUNTED k_ilu_check<<<grid_for(nb), kBlock, 0, s>>>(nb, J.row_ptr, J.col, F->dblk, ctrl + 4);
    RS_CHECK_CUDA(cudaGetLastError());
    // the layering runs with the largest cluster: its widest level is not
    // known yet
    RS_CHECK_CUDA(launch_cluster(k_ilu_levels, kIluMaxCluster, kIluThreads, s, nb, J.row_ptr, J.col, indeg, cnt,
                                 F->lvl_cells, F->lvl_ptr, F->nlev_d, ctrl));
    int32_t h[5];
    RS_CHECK_CUDA(cudaMemcpyAsync(h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    if (h[4] & 1) return fail(RS_EINVAL, "ILU(0): a block row has no diagonal block");
    if (h[4] & 2) return fail(RS_EINVAL, "ILU(0): the block pattern is not structurally symmetric");
    if (h[3] || h[2] != nb) return fail(RS_ESETUP, "ILU(0): level scheduling did not place every cell once");
    F->nlev = h[0];
    F->maxw = h[1];
    const int64_t per = (F->maxw + 31) / 32 * 32;
    F->cluster = 1;
    while (F->cluster < kIluMaxCluster && per > (int64_t)F->cluster * kIluThreads) F->cluster *= 2;
    F->threads = (int)std::min<int64_t>(kIluThreads, std::max<int64_t>(32, per));
    F->cluster_s = 1;
    while (F->cluster_s < kIluMaxCluster && per > (int64_t)F->cluster_s * kIluSolveThreads) F->cluster_s *= 2;
    F->threads_s = (int)std::min<int64_t>(kIluSolveThreads, std::max<int64_t>(32, per));
    RS_COUNTED k_ilu_records<<<grid_for(nb), kBlock, 0, s>>>(nb, F->lvl_cells, J.row_ptr, J.col, F->dblk, F->rec);
    RS_CHECK_CUDA(cudaGetLastError());
    RS_CHECK_CUDA(cudaMemcpyAsync(F->lu, J.val, sizeof(double) * 4 * (size_t)J.nnzb, cudaMemcpyDeviceToDevice, s));
    RS_CHECK_CUDA(launch_cluster(k_ilu_factor, F->cluster, F->threads, s, F->nlev_d, F->lvl_ptr, F->lvl_cells,
                                 J.row_ptr, J.col, F->dblk, F->lu));
    if (precision == RS_PREC_FP32) {
      RS_TRY(dalloc_n(&F->luf, 4 * (size_t)J.nnzb, s));
      RS_CHECK_CUDA(cudaMemsetAsync(ctrl, 0, sizeof(int32_t), s));
      RS_COUNTED k_ilu_to_f32<<<grid_for(4 * (int64_t)J.nnzb), kBlock, 0, s>>>(4 * (int64_t)J.nnzb, F->lu, F->luf, ctrl);
      RS_CHECK_CUDA(cudaGetLastError());
      int32_t e = 0;
      RS_CHECK_CUDA(cudaMemcpyAsync(&e, ctrl, sizeof(e), cudaMemcpyDeviceToHost, s));
      RS_CHECK_CUDA(cudaStreamSynchronize(s));
      if (e) return fail(RS_ESETUP, "ILU(0): factors beyond the FP32 range");
    }
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    return 0;
  };
  rc = attempt();
  if (rc) {
    ilu_free(F);
    return rc;
  }
  *out = F;
  return 0;
}

int ilu0_solve(const rs_ilu0 *F, const double *b, double *x, cudaStream_t s) {
  if (F->nb == 0) return 0;
  const bool one = F->cluster_s == 1;
  if (F->precision == RS_PREC_FP32) {
    if (one)
      RS_CHECK_CUDA(launch_cluster(k_ilu_solve<true, float>, 1, F->threads_s, s, F->nlev_d, F->lvl_ptr, F->rec, F->col,
                                   F->luf, b, x));
    else
      RS_CHECK_CUDA(launch_cluster(k_ilu_solve<false, float>, F->cluster_s, F->threads_s, s, F->nlev_d, F->lvl_ptr,
                                   F->rec, F->col, F->luf, b, x));
  } else {
    if (one)
      RS_CHECK_CUDA(launch_cluster(k_ilu_solve<true, double>, 1, F->threads_s, s, F->nlev_d, F->lvl_ptr, F->rec,
                                   F->col, F->lu, b, x));
    else
      RS_CHECK_CUDA(launch_cluster(k_ilu_solve<false, double>, F->cluster_s, F->threads_s, s, F->nlev_d, F->lvl_ptr,
                                   F->rec, F->col, F->lu, b, x));
  }
  return 0;
}

void ilu0_free(rs_ilu0 *F) {
  if (F) ilu_free(F);
}

}  // namespace rs

extern "C" int ilu0_create(const rs_bsr2 *J, int32_t precision, rs_ilu0 **out, cudaStream_t stream) {
  if (!out) return fail(RS_EINVAL, "null output handle");
  *out = nullptr;
  if (!J || J->nb < 0 || J->nnzb < 0 || (J->nb > 0 && (!J->row_ptr || !J->col || !J->val)))
    return fail(RS_EINVAL, "invalid arguments");
  if (precision != RS_PREC_FP32 && precision != RS_PREC_FP64) return fail(RS_EINVAL, "bad precision");
  return ilu0_build(*J, precision, out, stream);
}

extern "C" int ilu0_apply(const rs_ilu0 *F, const double *b, double *x, cudaStream_t stream) {
  if (!F || ((!b || !x) && F->nb > 0)) return fail(RS_EINVAL, "null argument");
  if (b == x && F->nb > 0) return fail(RS_EINVAL, "b and x must not alias");
  return ilu0_solve(F, b, x, stream);
}

extern "C" int ilu0_info(const rs_ilu0 *F, int32_t *nlevels, int32_t *max_width, int32_t *cluster_ctas) {
  if (!F) return fail(RS_EINVAL, "null handle");
  if (nlevels) *nlevels = F->nlev;
  if (max_width) *max_width = F->maxw;
  if (cluster_ctas) *cluster_ctas = F->nb ? F->cluster : 0;
  return RS_OK;
}

extern "C" int ilu0_factors(const rs_ilu0 *F, double *lu, cudaStream_t stream) {
  if (!F || (!lu && F->nnzb > 0)) return fail(RS_EINVAL, "null argument");
  if (F->nnzb > 0)
    RS_CHECK_CUDA(cudaMemcpyAsync(lu, F->lu, sizeof(double) * 4 * (size_t)F->nnzb, cudaMemcpyDeviceToDevice, stream));
  return RS_OK;
}

extern "C" int ilu0_destroy(rs_ilu0 *F) {
  if (F) {
    cudaStreamSynchronize(F->stream);
    ilu_free(F);
  }
  return RS_OK;
}
