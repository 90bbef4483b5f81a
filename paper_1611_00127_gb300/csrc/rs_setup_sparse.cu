// Setup-time sparse operations, FP64 (compiled without fused multiply-add):
// block extraction, decoupling, SIMPLE Schur complement (Sec. 3.4), sparse
// products and transposes for the Galerkin operator.
//
// Arithmetic order, shared with the CPU check so that the integer decisions
// taken on the results (strength, C/F splitting) are reproduced exactly:
// sums run in ascending inner index and the first term of a sum is the
// rounded product itself; in the sparse products every later term is fused
// into the sum (fma, one rounding), elsewhere each product is rounded before
// it is added.
#include <type_traits>

#include "rs_internal.cuh"

namespace rs {

// ------------------------------------------------------------------ blocks
__global__ void k_part(int32_t nnzb, const double *val, int off, double *out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnzb) out[k] = val[4 * k + off];
}

int bsr2_part(const rs_bsr2 &J, int r, int c, DCsr &out, cudaStream_t s) {
  out.n = out.m = J.nb;
  out.nnz = J.nnzb;
  RS_TRY(dalloc_n(&out.rowptr, (size_t)J.nb + 1, s));
  RS_TRY(dalloc_n(&out.col, (size_t)J.nnzb, s));
  RS_TRY(dalloc_n(&out.val, (size_t)J.nnzb, s));
  RS_CHECK_CUDA(cudaMemcpyAsync(out.rowptr, J.row_ptr, sizeof(int32_t) * ((size_t)J.nb + 1), cudaMemcpyDeviceToDevice, s));
  RS_CHECK_CUDA(cudaMemcpyAsync(out.col, J.col, sizeof(int32_t) * (size_t)J.nnzb, cudaMemcpyDeviceToDevice, s));
  if (J.nnzb > 0) RS_COUNTED k_part<<<grid_for(J.nnzb), kBlock, 0, s>>>(J.nnzb, J.val, 2 * r + c, out.val);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// Point-ordered scalar matrix: unknown 2i = P_w, 2i+1 = S_n of cell i.
__global__ void k_scalar(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                         int32_t *orp, int32_t *ocol, double *oval) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const int32_t s = rowptr[i], e = rowptr[i + 1], len = e - s;
  for (int r = 0; r < 2; r++) {
    int32_t pos = 4 * s + r * 2 * len;
    orp[2 * i + r] = pos;
    for (int32_t k = s; k < e; k++)
      for (int c = 0; c < 2; c++) {
        ocol[pos] = 2 * col[k] + c;
        oval[pos] = val[4 * (int64_t)k + 2 * r + c];
        pos++;
      }
  }
  if (i == nb - 1) orp[2 * nb] = 4 * e;
}

int bsr2_scalar(const rs_bsr2 &J, DCsr &out, cudaStream_t s) {
  out.n = out.m = 2 * J.nb;
  out.nnz = 4 * J.nnzb;
  RS_TRY(dalloc_n(&out.rowptr, (size_t)out.n + 1, s));
  RS_TRY(dalloc_n(&out.col, (size_t)out.nnz, s));
  RS_TRY(dalloc_n(&out.val, (size_t)out.nnz, s));
  if (J.nb > 0) RS_COUNTED k_scalar<<<grid_for(J.nb), kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, out.rowptr, out.col, out.val);
  else RS_CHECK_CUDA(cudaMemsetAsync(out.rowptr, 0, sizeof(int32_t), s));
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// Quasi-IMPES: w_i = -(a_ps,ii / a_ss,ii); pressure row += w_i * oil row.
__global__ void k_qimpes(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val,
                         double *out, double *w_out) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double w = 0.0;
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
    if (col[k] == i && val[4 * (int64_t)k + 3] != 0.0) w = -(val[4 * (int64_t)k + 1] / val[4 * (int64_t)k + 3]);
  w_out[i] = w;
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
    const double *b = val + 4 * (int64_t)k;
    double *o = out + 4 * (int64_t)k;
    const double t0 = w * b[2], t1 = w * b[3];
    o[0] = b[0] + t0;
    o[1] = b[1] + t1;
    o[2] = b[2];
    o[3] = b[3];
  }
}

__device__ __forceinline__ bool inv2x2(const double *m, double *o) {
  const double ad = m[0] * m[3], bc = m[1] * m[2];
  const double det = ad - bc;
  if (det == 0.0) return false;
  o[0] = m[3] / det;
  o[1] = -(m[1] / det);
  o[2] = -(m[2] / det);
  o[3] = m[0] / det;
  return true;
}

// D^{-1} J with D the diagonal 2x2 block (rows with singular D unchanged);
// also the inverse blocks (identity where singular).
__global__ void k_abf(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *out,
                      double *dinv) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double di[4] = {1.0, 0.0, 0.0, 1.0};
  bool ok = false;
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
    if (col[k] == i) ok = inv2x2(val + 4 * (int64_t)k, di);
  if (!ok) { di[0] = 1.0; di[1] = 0.0; di[2] = 0.0; di[3] = 1.0; }
  for (int q = 0; q < 4; q++) dinv[4 * (int64_t)i + q] = di[q];
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
    const double *y = val + 4 * (int64_t)k;
    double *o = out + 4 * (int64_t)k;
    if (!ok) {
      for (int q = 0; q < 4; q++) o[q] = y[q];
      continue;
    }
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 2; c++) {
        const double t0 = di[2 * r] * y[c];
        const double t1 = di[2 * r + 1] * y[2 + c];
        o[2 * r + c] = t0 + t1;
      }
  }
}

// Inverse of each diagonal block (identity where singular): point-block Jacobi.
__global__ void k_diag_inv(int32_t nb, const int32_t *rowptr, const int32_t *col, const double *val, double *dinv) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double z[4] = {0.0, 0.0, 0.0, 0.0}, di[4];
  const double *d = z;
  for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
    if (col[k] == i) d = val + 4 * (int64_t)k;
  if (!inv2x2(d, di)) { di[0] = 1.0; di[1] = 0.0; di[2] = 0.0; di[3] = 1.0; }
  for (int q = 0; q < 4; q++) dinv[4 * (int64_t)i + q] = di[q];
}

int decouple_qimpes(const rs_bsr2 &J, double *out, double *w, cudaStream_t s) {
  if (J.nb > 0) RS_COUNTED k_qimpes<<<grid_for(J.nb), kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, out, w);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int decouple_abf(const rs_bsr2 &J, double *out, double *dinv, cudaStream_t s) {
  if (J.nb > 0) RS_COUNTED k_abf<<<grid_for(J.nb), kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, out, dinv);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int block_diag_inverse(const rs_bsr2 &J, double *dinv, cudaStream_t s) {
  if (J.nb > 0) RS_COUNTED k_diag_inv<<<grid_for(J.nb), kBlock, 0, s>>>(J.nb, J.row_ptr, J.col, J.val, dinv);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ SpGEMM
// C = A B. One warp per row of C with an open-addressing hash table in shared
// memory. The warp walks A's row in ascending column k; for each k the lanes
// take the (distinct) entries of B's row k, so every C(i,j) receives its
// terms in ascending k. Pass 1 counts distinct columns, pass 2 accumulates,
// sorts the row by column and writes it.
//
// Rows are binned by the table they need, so that the many short rows run
// with small tables (many warps per SM) and only the long ones with large
// tables: pass 1 sizes a row's table from its product count (an upper bound
// of its distinct columns), pass 2 from twice the exact distinct count that
// pass 1 found (short probe sequences).
constexpr int kHashBits = 11;
constexpr int kHash = 1 << kHashBits;     // largest per-row table (slots)
constexpr int kGemmThreads = 256;
constexpr int kGemmBins = kHashBits - 4;  // tables of 32 .. kHash slots
constexpr int kGemmSmem = 96 * 1024;      // shared memory budget of one CTA
constexpr int kRankE = 4;                 // entries per lane of the rank placement

// table slot of a column key (Fibonacci hashing into 2^tbits slots)
__device__ __forceinline__ int hslot(int32_t key, int tbits) {
  return (int)(((uint32_t)key * 2654435761u) >> (32 - tbits));
}

// bin of a row that needs `need` slots: the smallest table of 32 << b slots
// that holds them (the largest bin when none does; the product kernel then
// reports the overflow)
__device__ __forceinline__ int gemm_bin(int64_t need) {
  int b = 0;
  while (b < kGemmBins - 1 && (int64_t(32) << b) < need) b++;
  return b;
}

// Adds one to bin b's counter for every lane of the warp, one atomic per
// distinct bin of the warp (all 32 lanes call it; `ok` lanes count).
__device__ __forceinline__ void warp_bin_add(bool ok, int b, int32_t *cnt) {
  const unsigned act = __ballot_sync(0xffffffffu, ok);
  if (!ok) return;
  const unsigned same = __match_any_sync(act, b);
  if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[b], __popc(same));
}

// pass-1 bins: the number of products of each row of A with B
__global__ void k_spgemm_bin1(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                              const int32_t *__restrict__ brp, uint8_t *bin, int32_t *bincnt, int32_t *npcap,
                              unsigned long long *captot) {
  const int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0;
  int32_t cap = 0;
  if (row < n) {
    int64_t np = 0;
    for (int32_t ka = arp[row]; ka < arp[row + 1]; ka++) {
      const int32_t k = acol[ka];
      np += brp[k + 1] - brp[k];
    }
    b = gemm_bin(np);
    bin[row] = (uint8_t)b;
    // the most entries the row can have (its products, at most a full table)
    cap = (int32_t)(np < kHash ? np : kHash);
    npcap[row] = cap;
  }
  // the reservation's total in 64 bits (one atomic per warp; a warp's sum
  // is at most 32 * kHash)
  const unsigned ws = __reduce_add_sync(0xffffffffu, (unsigned)cap);
  if ((threadIdx.x & 31) == 0 && ws) atomicAdd(captot, (unsigned long long)ws);
  warp_bin_add(row < n, b, bincnt);
}

// pass-2 bins: twice the distinct count found by pass 1 (crp scanned)
__global__ void k_spgemm_bin2(int32_t n, const int32_t *__restrict__ crp, uint8_t *bin, int32_t *bincnt) {
  const int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
  int b = 0;
  if (row < n) {
    b = gemm_bin(2 * (int64_t)(crp[row + 1] - crp[row]));
    bin[row] = (uint8_t)b;
  }
  warp_bin_add(row < n, b, bincnt);
}

// rows listed bin after bin (any order inside a bin); one atomic per
// distinct bin of a warp
__global__ void k_spgemm_binfill(int32_t n, const uint8_t *__restrict__ bin, int32_t *cursor, int32_t *rows) {
  const int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = row < n;
  const unsigned act = __ballot_sync(0xffffffffu, ok);
  if (!ok) return;
  const int b = bin[row];
  const unsigned same = __match_any_sync(act, b);
  const int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(&cursor[b], __popc(same));
  base = __shfl_sync(same, base, leader);
  rows[base + __popc(same & ((1u << lane) - 1u))] = row;
}

// Sorts the pairs (key[t], val[t]), t < cnt, by key (keys distinct) with
// the G lanes of a group (lane gl of the group, mask gmask); the arrays have
// room for the next power of two of cnt (<= tsize). Up to G pairs: bitonic
// network in registers; more: bitonic network in place.
template <int G>
__device__ void group_sort_pairs(int32_t *key, double *val, int32_t cnt, int tsize, int gl, unsigned gmask) {
  if (cnt <= G) {
    int32_t k = gl < cnt ? key[gl] : INT32_MAX;
    double v = gl < cnt ? val[gl] : 0.0;
    for (int kk = 2; kk <= G; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        const int32_t ok = __shfl_xor_sync(gmask, k, j, G);
        const double ov = __shfl_xor_sync(gmask, v, j, G);
        const bool up = (gl & kk) == 0, lower = (gl & j) == 0;
        const bool take = (lower == up) ? (ok < k) : (ok > k);
        if (take) { k = ok; v = ov; }
      }
    __syncwarp(gmask);
    if (gl < cnt) { key[gl] = k; val[gl] = v; }
    __syncwarp(gmask);
    return;
  }
  int32_t P = 2 * G;
  while (P < cnt) P <<= 1;
  if (P > tsize) P = tsize;
  for (int32_t t = cnt + gl; t < P; t += G) key[t] = INT32_MAX;
  __syncwarp(gmask);
  for (int32_t kk = 2; kk <= P; kk <<= 1)
    for (int32_t j = kk >> 1; j > 0; j >>= 1) {
      for (int32_t t = gl; t < P / 2; t += G) {
        const int32_t a = (t / j) * 2 * j + (t % j), b = a + j;
        const bool up = (a & kk) == 0;
        const int32_t x = key[a], y = key[b];
        if ((x > y) == up) {
          key[a] = y;
          key[b] = x;
          const double w = val[a];
          val[a] = val[b];
          val[b] = w;
        }
      }
      __syncwarp(gmask);
    }
}

// Groups of G lanes take one listed row each (32 / G rows per warp), each
// group with its own table of 2^tbits slots in shared memory. The loops over
// A's row and B's rows run to the warp's longest, so the groups stay in step
// and every FP64 multiply or add is one instruction for all of the warp's
// rows (GB300 issues FP64 at a low rate per instruction, whatever the number
// of active lanes). Products are accumulated in ascending inner index (the
// A-row loop is sequential, a B row holds each column once), so sums are
// reproducible.
template <int G, bool NUMERIC>
__global__ void __launch_bounds__(kGemmThreads) k_spgemm(int32_t nrows, const int32_t *__restrict__ rows, int tbits,
                                                         const int32_t *__restrict__ arp,
                                                         const int32_t *__restrict__ acol,
                                                         const double *__restrict__ aval,
                                                         const int32_t *__restrict__ brp,
                                                         const int32_t *__restrict__ bcol,
                                                         const double *__restrict__ bval,
                                                         int32_t *__restrict__ crp, int32_t *__restrict__ ccol,
                                                         double *__restrict__ cval, int32_t *err,
                                                         int32_t *__restrict__ defer, int32_t *__restrict__ ccnt) {
  constexpr int R = 32 / G;
  extern __shared__ unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  const unsigned glow = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const int tsize = 1 << tbits;
  const int tab = warp * R + grp;
  // tables tsize + G elements apart, so that the groups of a warp reading
  // the same slot index of their own tables hit different banks
  const int tstride = tsize + G;
  double *vals = reinterpret_cast<double *>(smem) + (int64_t)tab * tstride;
  int32_t *keys =
      reinterpret_cast<int32_t *>(smem + sizeof(double) * (size_t)tstride * nwarps * R) + (int64_t)tab * tstride;
  __shared__ int32_t cnt_s[kGemmThreads / 32 * 4];
  __shared__ int32_t ovf_s[kGemmThreads / 32 * 4];
  for (int64_t base = ((int64_t)blockIdx.x * nwarps + warp) * R; base < nrows;
       base += (int64_t)gridDim.x * nwarps * R) {
    const bool has = base + grp < nrows;
    const int32_t row = has ? rows[base + grp] : 0;
    const int32_t as = has ? arp[row] : 0, alen = has ? arp[row + 1] - as : 0;
    for (int h = gl; h < tsize; h += G) keys[h] = -1;
    if (gl == 0) { cnt_s[tab] = 0; ovf_s[tab] = 0; }
    __syncwarp();
    const int32_t amax = __reduce_max_sync(0xffffffffu, alen);
    for (int32_t t = 0; t < amax; t++) {
      const bool on = t < alen;
      const int32_t k = on ? acol[as + t] : 0;
      const double a = on ? aval[as + t] : 0.0;
      const int32_t bs = on ? brp[k] : 0, blen = on ? brp[k + 1] - bs : 0;
      const int32_t bmax = __reduce_max_sync(0xffffffffu, blen);
      for (int32_t u0 = 0; u0 < bmax; u0 += G) {
        const int32_t u = u0 + gl;
        const bool live = u < blen;
        const int32_t j = live ? bcol[bs + u] : -1;
        const double b = (NUMERIC && live) ? bval[bs + u] : 0.0;
        int h = -1;
        bool fresh = false;
        if (live) {
          h = hslot(j, tbits);
          for (int probes = 0;; probes++) {
            const int32_t prev = atomicCAS(&keys[h], -1, j);
            if (prev == -1) { fresh = true; atomicAdd(&cnt_s[tab], 1); break; }
            if (prev == j) break;
            h = (h + 1) & (tsize - 1);
            if (probes + 1 >= tsize) { ovf_s[tab] = 1; h = -1; break; }
          }
        }
        __syncwarp();
        // a fresh entry takes the rounded product (a b + -0 = a b exactly),
        // a present one fuses the term into its sum: one FP64 instruction
        if (NUMERIC && h >= 0) vals[h] = fma(a, b, fresh ? -0.0 : vals[h]);
        __syncwarp();
      }
    }
    const int32_t cnt = cnt_s[tab];
    const bool over = ovf_s[tab] != 0 || cnt > tsize;
    if (!NUMERIC) {
      // a row whose distinct columns overflow this table is listed in
      // `defer` for a pass with the largest table (without a list: error)
      if (has && gl == 0) {
        if (over && defer) {
          defer[1 + atomicAdd(&defer[0], 1)] = row;
          crp[row] = 0;
        } else {
          if (over) atomicExch(err, 1);
          crp[row] = cnt;
        }
      }
    } else {
      // one pass into reserved rows (ccnt given: crp holds each row's
      // reserved capacity, the count goes to ccnt): a row whose distinct
      // columns overflow this table is listed in `defer` for a pass with the
      // largest table (without a list: error)
      if (has && over && gl == 0) {
        if (defer) defer[1 + atomicAdd(&defer[0], 1)] = row;
        else atomicExch(err, 1);
      }
      // compact the occupied slots to the front of the table (in place: a
      // slot moves only to a lower index, after the whole group has read its
      // chunk), sort them by column and write the output row
      int32_t base_c = 0;
      for (int h0 = 0; h0 < tsize; h0 += G) {
        const int32_t j = keys[h0 + gl];
        const double v = vals[h0 + gl];
        const unsigned occ = (__ballot_sync(0xffffffffu, j >= 0) >> (grp * G)) & glow;
        __syncwarp();
        if (j >= 0) {
          const int32_t pos = base_c + __popc(occ & ((1u << gl) - 1u));
          keys[pos] = j;
          vals[pos] = v;
        }
        base_c += __popc(occ);
        __syncwarp();
      }
      const int32_t scnt = has && !over ? cnt : 0;
      const int32_t cb = has ? crp[row] : 0, room = has ? crp[row + 1] - cb : 0;
      if (has && !over) {
        if ((ccnt ? cnt > room : room != cnt) && gl == 0) atomicExch(err, 1);
        if (ccnt && gl == 0) ccnt[row] = cnt;
      }
      if (scnt <= G * kRankE) {
        // each entry goes to its rank among the row's columns (distinct):
        // lane gl holds entries gl + G u and counts the smaller columns
        // against every entry of the compacted table
        int32_t kk[kRankE], rk[kRankE];
#pragma unroll
        for (int u = 0; u < kRankE; u++) {
          const int32_t e = gl + G * u;
          kk[u] = e < scnt ? keys[e] : INT32_MAX;
          rk[u] = 0;
        }
        for (int32_t x = 0; x < scnt; x++) {
          const int32_t kx = keys[x];
#pragma unroll
          for (int u = 0; u < kRankE; u++) rk[u] += kx < kk[u];
        }
#pragma unroll
        for (int u = 0; u < kRankE; u++) {
          const int32_t e = gl + G * u;
          if (e < scnt && rk[u] < room) {
            ccol[cb + rk[u]] = kk[u];
            cval[cb + rk[u]] = vals[e];
          }
        }
      } else {
        group_sort_pairs<G>(keys, vals, scnt, tsize, gl, gmask);
        for (int32_t a = gl; a < scnt && a < room; a += G) {
          ccol[cb + a] = keys[a];
          cval[cb + a] = vals[a];
        }
      }
    }
    __syncwarp();
  }
}

// Lists the rows bin by bin (bin counts bincnt_d on the device) and launches
// the product kernel once per non-empty bin with that bin's table size.
// Lists the rows bin by bin (bin counts bincnt_d on the device) and launches
// the product kernel once per non-empty bin with that bin's table size. In
// the first pass (tables sized by the product count, often several times the
// distinct count) a bin's rows first try a table of at most kGemmTry slots;
// the rows it cannot hold run again with the largest table.
constexpr int kGemmTryBits = 8;
template <bool NUMERIC>
static int spgemm_pass(const DCsr &A, const DCsr &B, DCsr &C, const uint8_t *bin, const int32_t *bincnt_d,
                       int32_t *cursor, int32_t *rows, int32_t *err, int32_t *defer, cudaStream_t s,
                       int32_t *ccnt = nullptr, int32_t *ccol = nullptr, double *cval = nullptr) {
  // output rows: C's, or (ccnt given) rows reserved at C.rowptr's offsets
  int32_t *ocol = ccol ? ccol : C.col;
  double *oval = cval ? cval : C.val;
  int32_t hcnt[kGemmBins];
  RS_CHECK_CUDA(cudaMemcpyAsync(hcnt, bincnt_d, sizeof(hcnt), cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  int32_t hoff[kGemmBins + 1];
  hoff[0] = 0;
  for (int b = 0; b < kGemmBins; b++) hoff[b + 1] = hoff[b] + hcnt[b];
  // (cudaMemcpyAsync from the pageable stack array hoff stages the data
  // before it returns)
  RS_CHECK_CUDA(cudaMemcpyAsync(cursor, hoff, sizeof(int32_t) * kGemmBins, cudaMemcpyHostToDevice, s));
  RS_COUNTED k_spgemm_binfill<<<grid_for(A.n), kBlock, 0, s>>>(A.n, bin, cursor, rows);
  if (defer) RS_CHECK_CUDA(cudaMemsetAsync(defer, 0, sizeof(int32_t), s));
  auto run = [&](int tbits, int32_t nrows, const int32_t *list, int32_t *dfr) {
    const int tsize = 1 << tbits;
    // lanes per row: 8 for tables of up to 64 slots, 16 for 128, else 32
    const int G = tsize <= 64 ? 8 : (tsize <= 128 ? 16 : 32), R = 32 / G;
    const int warps = (int)std::max<int64_t>(
        1, std::min<int64_t>(kGemmThreads / 32, kGemmSmem / (12 * (int64_t)(tsize + G) * R)));
    const size_t shm = (sizeof(double) + sizeof(int32_t)) * (size_t)(tsize + G) * warps * R;
    const int64_t per_cta = (int64_t)warps * R;
    const unsigned grid = (unsigned)std::min<int64_t>((nrows + per_cta - 1) / per_cta, (int64_t)num_sms() * 32);
    auto kern = G == 8 ? k_spgemm<8, NUMERIC> : (G == 16 ? k_spgemm<16, NUMERIC> : k_spgemm<32, NUMERIC>);
    RS_COUNTED kern<<<grid, 32 * warps, shm, s>>>(nrows, list, tbits, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val,
                                                  C.rowptr, ocol, oval, err, dfr, ccnt);
  };
  bool tried = false;
  for (int b = 0; b < kGemmBins; b++) {
    if (hcnt[b] == 0) continue;
    const int tbits = 5 + b;
    if (defer && tbits > kGemmTryBits) {
      run(kGemmTryBits, hcnt[b], rows + hoff[b], defer);
      tried = true;
    } else {
      run(tbits, hcnt[b], rows + hoff[b], nullptr);
    }
  }
  if (tried) {
    int32_t nd = 0;
    RS_CHECK_CUDA(cudaMemcpyAsync(&nd, defer, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    if (nd > 0) run(kHashBits, nd, defer + 1, nullptr);
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// Moves row i's crp[i+1] - crp[i] entries from toff[i] to crp[i], G lanes
// per row: consecutive lanes take consecutive entries, so each group's loads
// and stores are contiguous.
template <int G>
__global__ void k_copy_rows(int32_t n, const int32_t *__restrict__ toff, const int32_t *__restrict__ crp,
                            const int32_t *__restrict__ tcol, const double *__restrict__ tval,
                            int32_t *__restrict__ ccol, double *__restrict__ cval) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid / G;
  if (i >= n) return;
  const int gl = (int)(gid % G);
  const int32_t a = __ldg(toff + i), b = __ldg(crp + i), c = __ldg(crp + i + 1) - b;
  for (int32_t t = gl; t < c; t += G) {
    ccol[b + t] = __ldg(tcol + a + t);
    cval[b + t] = __ldg(tval + a + t);
  }
}

int copy_rows(int32_t n, int64_t nnz, const int32_t *toff, const int32_t *crp, const int32_t *tcol,
              const double *tval, int32_t *ccol, double *cval, cudaStream_t s) {
  if (n <= 0) return 0;
  const double avg = (double)nnz / n;
  const int G = avg <= 6.0 ? 4 : (avg <= 16.0 ? 8 : (avg <= 40.0 ? 16 : 32));
  const unsigned grid = (unsigned)(((int64_t)n * G + kBlock - 1) / kBlock);
  switch (G) {
    case 4: RS_COUNTED k_copy_rows<4><<<grid, kBlock, 0, s>>>(n, toff, crp, tcol, tval, ccol, cval); break;
    case 8: RS_COUNTED k_copy_rows<8><<<grid, kBlock, 0, s>>>(n, toff, crp, tcol, tval, ccol, cval); break;
    case 16: RS_COUNTED k_copy_rows<16><<<grid, kBlock, 0, s>>>(n, toff, crp, tcol, tval, ccol, cval); break;
    default: RS_COUNTED k_copy_rows<32><<<grid, kBlock, 0, s>>>(n, toff, crp, tcol, tval, ccol, cval); break;
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// C = A B. When the rows' worst cases (each row's product count, at most a
// full table) fit in a quarter of the free device memory, one numeric pass
// writes every row into a reserved row of that size and a compaction moves
// them into C; otherwise a counting pass sizes C's rows first.
int spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
  C.n = A.n;
  C.m = B.m;
  RS_TRY(dalloc_n(&C.rowptr, (size_t)A.n + 1, s));
  Scratch sc(s);
  int32_t *err = nullptr, *bincnt = nullptr, *cursor = nullptr, *rows = nullptr, *defer = nullptr, *npcap = nullptr;
  uint8_t *bin = nullptr;
  unsigned long long *captot = nullptr;
  RS_TRY(sc.get(&err, 2));
  RS_TRY(sc.get(&bincnt, 2 * kGemmBins));
  RS_TRY(sc.get(&cursor, kGemmBins));
  RS_TRY(sc.get(&rows, (size_t)A.n + 1));
  RS_TRY(sc.get(&bin, (size_t)A.n + 1));
  RS_TRY(sc.get(&defer, (size_t)A.n + 1));
  RS_TRY(sc.get(&npcap, (size_t)A.n + 1));
  RS_TRY(sc.get(&captot, 1));
  RS_CHECK_CUDA(cudaMemsetAsync(captot, 0, sizeof(unsigned long long), s));
  RS_CHECK_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), s));
  RS_CHECK_CUDA(cudaMemsetAsync(bincnt, 0, 2 * kGemmBins * sizeof(int32_t), s));
  static bool attr = false;
  if (!attr) {
    const void *ks[6] = {(const void *)k_spgemm<8, false>, (const void *)k_spgemm<16, false>,
                         (const void *)k_spgemm<32, false>, (const void *)k_spgemm<8, true>,
                         (const void *)k_spgemm<16, true>, (const void *)k_spgemm<32, true>};
    for (const void *k : ks)
      RS_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
    attr = true;
  }
  ProfScope ps(kProfSpgemm, A.nnz * 12.0 + B.nnz * 12.0, s);
  int32_t herr = 0;
  if (A.n > 0) {
    RS_COUNTED k_spgemm_bin1<<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, B.rowptr, bin, bincnt, npcap,
                                                              captot);
    unsigned long long hcap = 0;
    RS_CHECK_CUDA(cudaMemcpyAsync(&hcap, captot, sizeof(hcap), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    size_t fr = 0, tot_mem = 0;
    RS_CHECK_CUDA(cudaMemGetInfo(&fr, &tot_mem));
    if (hcap < 0x7fffffffULL && hcap * 12 <= fr / 4) {
      // reserved rows: offsets of the capped product counts
      int32_t *toff = nullptr;
      RS_TRY(sc.get(&toff, (size_t)A.n + 1));
      int32_t reserve = 0;
      RS_TRY(exclusive_scan(npcap, toff, A.n, s, nullptr));
      reserve = (int32_t)hcap;
      Scratch st(s);
      int32_t *tcol = nullptr, *ccnt = nullptr;
      double *tval = nullptr;
      RS_TRY(st.get(&tcol, (size_t)reserve + 1));
      RS_TRY(st.get(&tval, (size_t)reserve + 1));
      RS_TRY(st.get(&ccnt, (size_t)A.n + 1));
      DCsr T;
      T.n = A.n;
      T.rowptr = toff;
      RS_TRY(spgemm_pass<true>(A, B, T, bin, bincnt, cursor, rows, err, defer, s, ccnt, tcol, tval));
      int32_t tot = 0;
      RS_TRY(exclusive_scan(ccnt, C.rowptr, A.n, s, &tot));
      RS_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RS_CHECK_CUDA(cudaStreamSynchronize(s));
      if (herr) return fail(RS_ESETUP, "sparse product row exceeds the per-row table");
      C.nnz = tot;
      RS_TRY(dalloc_n(&C.col, (size_t)tot, s));
      RS_TRY(dalloc_n(&C.val, (size_t)tot, s));
      return copy_rows(A.n, tot, toff, C.rowptr, tcol, tval, C.col, C.val, s);
    }
    RS_TRY(spgemm_pass<false>(A, B, C, bin, bincnt, cursor, rows, err, defer, s));
  }
  int32_t tot = 0;
  RS_TRY(exclusive_scan(C.rowptr, C.rowptr, A.n, s, &tot));
  RS_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(RS_ESETUP, "sparse product row exceeds the per-row table");
  C.nnz = tot;
  RS_TRY(dalloc_n(&C.col, (size_t)tot, s));
  RS_TRY(dalloc_n(&C.val, (size_t)tot, s));
  if (A.n > 0) {
    RS_COUNTED k_spgemm_bin2<<<grid_for(A.n), kBlock, 0, s>>>(A.n, C.rowptr, bin, bincnt + kGemmBins);
    RS_TRY(spgemm_pass<true>(A, B, C, bin, bincnt + kGemmBins, cursor, rows, err, nullptr, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    if (herr) return fail(RS_ESETUP, "sparse product row exceeds the per-row table");
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ transpose
__global__ void k_col_count(int32_t nnz, const int32_t *col, int32_t *cnt) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) atomicAdd(&cnt[col[k]], 1);
}

__global__ void k_transpose_fill(int32_t n, const int32_t *rp, const int32_t *col, const double *val,
                                 int32_t *fill, int32_t *tcol, double *tval) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
    const int32_t q = atomicAdd(&fill[col[k]], 1);
    tcol[q] = i;
    tval[q] = val[k];
  }
}

// Sorts each row by column (the columns of a row are distinct), a warp per
// row. A row of up to 32 * kSortE entries is held in registers (kSortE per
// lane); each entry's rank, the number of smaller columns in the row, is
// counted against every entry by shuffles, and the entry is stored at its
// rank. A longer row is insertion-sorted by lane 0.
constexpr int kSortE = 8;
__global__ void k_row_sort(int32_t n, const int32_t *__restrict__ rp, int32_t *col, double *val) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;   // whole warps
  const int32_t s = rp[w], e = rp[w + 1], len = e - s;
  if (len <= 1) return;
  if (len > 32 * kSortE) {
    if (lane != 0) return;
    for (int32_t a = s + 1; a < e; a++) {
      const int32_t c = col[a];
      const double v = val[a];
      int32_t b = a - 1;
      while (b >= s && col[b] > c) {
        col[b + 1] = col[b];
        val[b + 1] = val[b];
        b--;
      }
      col[b + 1] = c;
      val[b + 1] = v;
    }
    return;
  }
  int32_t key[kSortE], rank[kSortE];
  double v[kSortE];
#pragma unroll
  for (int u = 0; u < kSortE; u++) {
    const int32_t t = u * 32 + lane;
    key[u] = t < len ? col[s + t] : INT32_MAX;
    v[u] = t < len ? val[s + t] : 0.0;
    rank[u] = 0;
  }
#pragma unroll
  for (int u2 = 0; u2 < kSortE; u2++) {
    if (u2 * 32 >= len) break;   // warp-uniform
    for (int src = 0; src < 32; src++) {
      const int32_t k = __shfl_sync(0xffffffffu, key[u2], src);
#pragma unroll
      for (int u = 0; u < kSortE; u++) rank[u] += k < key[u];
    }
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < kSortE; u++) {
    const int32_t t = u * 32 + lane;
    if (t < len) {
      col[s + rank[u]] = key[u];
      val[s + rank[u]] = v[u];
    }
  }
}

int transpose(const DCsr &A, DCsr &T, cudaStream_t s) {
  T.n = A.m;
  T.m = A.n;
  T.nnz = A.nnz;
  RS_TRY(dalloc_n(&T.rowptr, (size_t)A.m + 1, s));
  RS_TRY(dalloc_n(&T.col, (size_t)A.nnz, s));
  RS_TRY(dalloc_n(&T.val, (size_t)A.nnz, s));
  Scratch sc(s);
  int32_t *fill = nullptr;
  RS_TRY(sc.get(&fill, (size_t)A.m + 1));
  RS_CHECK_CUDA(cudaMemsetAsync(T.rowptr, 0, sizeof(int32_t) * ((size_t)A.m + 1), s));
  if (A.nnz > 0) RS_COUNTED k_col_count<<<grid_for(A.nnz), kBlock, 0, s>>>(A.nnz, A.col, T.rowptr);
  RS_TRY(exclusive_scan(T.rowptr, T.rowptr, A.m, s, nullptr));
  RS_CHECK_CUDA(cudaMemcpyAsync(fill, T.rowptr, sizeof(int32_t) * ((size_t)A.m + 1), cudaMemcpyDeviceToDevice, s));
  if (A.n > 0) RS_COUNTED k_transpose_fill<<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, fill, T.col, T.val);
  if (A.m > 0) RS_COUNTED k_row_sort<<<grid_for((int64_t)A.m * 32), kBlock, 0, s>>>(A.m, T.rowptr, T.col, T.val);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ SIMPLE Schur
__global__ void k_diag_vals(int32_t n, const int32_t *rp, const int32_t *col, const double *val, double *d) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = 0.0;
  for (int32_t k = rp[i]; k < rp[i + 1]; k++)
    if (col[k] == i) v = val[k];
  d[i] = v;
}

// X = A_ps diag(d)^{-1}: x_ik = a_ps,ik / d_k (0 kept as a structural entry when d_k = 0).
__global__ void k_scale_cols(int32_t nnz, const int32_t *col, const double *val, const double *d, double *out) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const double dk = d[col[k]];
  out[k] = dk != 0.0 ? val[k] / dk : 0.0;
}

// position of column v in the sorted columns a[0..m), or -1
__device__ __forceinline__ int32_t find_col(const int32_t *a, int32_t m, int32_t v) {
  int32_t lo = 0, hi = m - 1;
  while (lo <= hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t x = a[mid];
    if (x == v) return mid;
    if (x < v) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// C = A - B on the union pattern; an entry missing from A counts as 0.0
// (so the result is 0.0 - b), one missing from B leaves a. G lanes per row:
// the count pass looks A's columns up in B's row; the fill writes B's row
// lane-parallel when A's pattern lies inside it (the union is then B's
// pattern), else the group's first lane merges the two rows.
template <bool FILL, int G>
__global__ void k_sub(int32_t n, const int32_t *arp, const int32_t *acol, const double *aval, const int32_t *brp,
                      const int32_t *bcol, const double *bval, int32_t *crp, int32_t *ccol, double *cval) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid / G;
  const int gl = (int)(gid % G);
  const bool ok = i < n;
  const int32_t p = ok ? arp[i] : 0, na = ok ? arp[i + 1] - p : 0;
  const int32_t q = ok ? brp[i] : 0, nb = ok ? brp[i + 1] - q : 0;
  if (!FILL) {
    // the union's size: B's entries and A's entries missing from B
    int32_t extra = 0;
    for (int32_t t = gl; t < na; t += G) extra += find_col(bcol + q, nb, acol[p + t]) < 0;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) extra += __shfl_xor_sync(0xffffffffu, extra, o, G);
    if (ok && gl == 0) crp[i] = nb + extra;
    return;
  }
  if (!ok) return;
  const int32_t o = crp[i], c = crp[i + 1] - o;
  if (c == nb) {
    // A's pattern inside B's (the usual case): the union is B's row
    for (int32_t t = gl; t < nb; t += G) {
      const int32_t j = bcol[q + t];
      const int32_t pa = find_col(acol + p, na, j);
      ccol[o + t] = j;
      cval[o + t] = (pa >= 0 ? aval[p + pa] : 0.0) - bval[q + t];
    }
    return;
  }
  if (gl != 0) return;
  int32_t pp = p, pe = p + na, qq = q, qe = q + nb, k = 0;
  while (pp < pe || qq < qe) {
    const int32_t ja = pp < pe ? acol[pp] : 0x7fffffff, jb = qq < qe ? bcol[qq] : 0x7fffffff;
    if (ja == jb) {
      ccol[o + k] = ja;
      cval[o + k] = aval[pp] - bval[qq];
      pp++;
      qq++;
    } else if (ja < jb) {
      ccol[o + k] = ja;
      cval[o + k] = aval[pp];
      pp++;
    } else {
      ccol[o + k] = jb;
      cval[o + k] = 0.0 - bval[qq];
      qq++;
    }
    k++;
  }
}

int csr_sub(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
  C.n = A.n;
  C.m = A.m;
  RS_TRY(dalloc_n(&C.rowptr, (size_t)A.n + 1, s));
  const double avg = A.n > 0 ? (double)B.nnz / A.n : 1.0;
  const int G = avg <= 12.0 ? 8 : (avg <= 32.0 ? 16 : 32);
  const unsigned grid = grid_for((int64_t)A.n * G);
  auto launch = [&](auto fill) {
    constexpr bool F = decltype(fill)::value;
    if (G == 8)
      RS_COUNTED k_sub<F, 8><<<grid, kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, C.rowptr,
                                                    C.col, C.val);
    else if (G == 16)
      RS_COUNTED k_sub<F, 16><<<grid, kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, C.rowptr,
                                                     C.col, C.val);
    else
      RS_COUNTED k_sub<F, 32><<<grid, kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, C.rowptr,
                                                     C.col, C.val);
  };
  if (A.n > 0) launch(std::false_type{});
  int32_t tot = 0;
  RS_TRY(exclusive_scan(C.rowptr, C.rowptr, A.n, s, &tot));
  C.nnz = tot;
  RS_TRY(dalloc_n(&C.col, (size_t)tot, s));
  RS_TRY(dalloc_n(&C.val, (size_t)tot, s));
  if (A.n > 0) launch(std::true_type{});
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int simple_schur(const DCsr &App, const DCsr &Aps, const DCsr &Asp, const DCsr &Ass, DCsr &out, cudaStream_t s) {
  Scratch sc(s);
  double *dss = nullptr;
  RS_TRY(sc.get(&dss, (size_t)Ass.n + 1));
  if (Ass.n > 0) RS_COUNTED k_diag_vals<<<grid_for(Ass.n), kBlock, 0, s>>>(Ass.n, Ass.rowptr, Ass.col, Ass.val, dss);
  DCsr X = Aps;                      // shares pattern arrays with A_ps
  X.val = nullptr;
  X.valf = nullptr;
  RS_TRY(sc.get(&X.val, (size_t)Aps.nnz + 1));
  if (Aps.nnz > 0) RS_COUNTED k_scale_cols<<<grid_for(Aps.nnz), kBlock, 0, s>>>(Aps.nnz, Aps.col, Aps.val, dss, X.val);
  DCsr Pm;
  int r = spgemm(X, Asp, Pm, s);
  if (r) { dcsr_free(Pm, s); return r; }
  r = csr_sub(App, Pm, out, s);
  dcsr_free(Pm, s);
  return r;
}

}  // namespace rs
