// Setup-time sparse operations, FP64 (compiled without fused multiply-add):
// block extraction, decoupling, SIMPLE Schur complement (Sec. 3.4), sparse
// products and transposes for the Galerkin operator.
//
// Arithmetic order, shared with the CPU check so that the integer decisions
// taken on the results (strength, C/F splitting) are reproduced exactly:
// sums run in ascending inner index, each product is rounded before it is
// added, and the first term of a sum is the rounded product itself.
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
constexpr int kHash = 2048;       // largest per-row table (slots)
constexpr int kGemmThreads = 256;

// table slot of a column key (Fibonacci hashing into 2^tbits slots)
__device__ __forceinline__ int hslot(int32_t key, int tbits) {
  return (int)(((uint32_t)key * 2654435761u) >> (32 - tbits));
}

// largest number of products of one row of A with B (an upper bound of the
// row's distinct output columns)
__global__ void k_spgemm_maxprod(int32_t n, const int32_t *__restrict__ arp, const int32_t *__restrict__ acol,
                                 const int32_t *__restrict__ brp, int32_t *mx) {
  const int32_t row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  int32_t np = 0;
  for (int32_t ka = arp[row]; ka < arp[row + 1]; ka++) {
    const int32_t k = acol[ka];
    np += brp[k + 1] - brp[k];
  }
  atomicMax(mx, np);
}

// One warp per row, with a hash table of `tcap` slots per warp in shared
// memory (tcap sized from the level's largest row, so small rows leave room
// for many warps per SM); each row uses the smallest power of two >= 2x its
// product count. Products are accumulated in ascending inner index (the ka
// loop is sequential, a B row holds each column once), so sums are
// reproducible.
template <bool NUMERIC>
__global__ void __launch_bounds__(kGemmThreads) k_spgemm(int32_t n, int32_t tcap, const int32_t *__restrict__ arp,
                                                         const int32_t *__restrict__ acol,
                                                         const double *__restrict__ aval,
                                                         const int32_t *__restrict__ brp,
                                                         const int32_t *__restrict__ bcol,
                                                         const double *__restrict__ bval,
                                                         int32_t *__restrict__ crp, int32_t *__restrict__ ccol,
                                                         double *__restrict__ cval, int32_t *err) {
  extern __shared__ unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  double *vals = reinterpret_cast<double *>(smem) + (int64_t)warp * tcap;
  int32_t *keys = reinterpret_cast<int32_t *>(smem + sizeof(double) * (size_t)tcap * nwarps) + (int64_t)warp * tcap;
  __shared__ int32_t cnt_s[kGemmThreads / 32];
  for (int32_t row = blockIdx.x * nwarps + warp; row < n; row += gridDim.x * nwarps) {
    const int32_t as = arp[row], ae = arp[row + 1];
    // upper bound of distinct columns: the number of products
    int32_t np = 0;
    for (int32_t ka = as + lane; ka < ae; ka += 32) {
      const int32_t k = acol[ka];
      np += brp[k + 1] - brp[k];
    }
    np = __reduce_add_sync(0xffffffffu, np);
    int tbits = 5;
    while ((1 << tbits) < tcap && (1 << tbits) < 2 * np) tbits++;
    const int tsize = 1 << tbits;
    for (int h = lane; h < tsize; h += 32) keys[h] = -1;
    if (lane == 0) cnt_s[warp] = 0;
    __syncwarp();
    for (int32_t ka = as; ka < ae; ka++) {
      const int32_t k = acol[ka];
      const double a = aval[ka];
      const int32_t bs = brp[k], be = brp[k + 1];
      for (int32_t kb = bs + lane; kb < be; kb += 32) {
        const int32_t j = bcol[kb];
        int h = hslot(j, tbits);
        int probes = 0;
        for (;;) {
          int32_t prev = atomicCAS(&keys[h], -1, j);
          if (prev == -1) {
            atomicAdd(&cnt_s[warp], 1);
            if (NUMERIC) vals[h] = a * bval[kb];
            break;
          }
          if (prev == j) {
            if (NUMERIC) vals[h] = vals[h] + a * bval[kb];
            break;
          }
          h = (h + 1) & (tsize - 1);
          if (++probes >= tsize) { atomicExch(err, 1); break; }
        }
      }
      __syncwarp();
    }
    __syncwarp();
    const int32_t cnt = cnt_s[warp];
    if (cnt > tsize && lane == 0) atomicExch(err, 1);
    if (!NUMERIC) {
      if (lane == 0) crp[row] = cnt;
    } else {
      // compact the occupied slots to the front of the table (in place: a
      // slot moves only to a lower index, after the whole warp has read its
      // chunk), then rank each entry by column and scatter to the output row
      int32_t base_c = 0;
      for (int h0 = 0; h0 < tsize; h0 += 32) {
        const int32_t j = keys[h0 + lane];
        const double v = vals[h0 + lane];
        const unsigned occ = __ballot_sync(0xffffffffu, j >= 0);
        __syncwarp();
        if (j >= 0) {
          const int32_t pos = base_c + __popc(occ & ((1u << lane) - 1u));
          keys[pos] = j;
          vals[pos] = v;
        }
        base_c += __popc(occ);
        __syncwarp();
      }
      const int32_t base = crp[row];
      for (int32_t a = lane; a < cnt; a += 32) {
        const int32_t j = keys[a];
        int32_t rank = 0;
        for (int32_t g = 0; g < cnt; g++) rank += keys[g] < j;
        ccol[base + rank] = j;
        cval[base + rank] = vals[a];
      }
    }
    __syncwarp();
  }
}

int spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
  C.n = A.n;
  C.m = B.m;
  RS_TRY(dalloc_n(&C.rowptr, (size_t)A.n + 1, s));
  Scratch sc(s);
  int32_t *err = nullptr;
  RS_TRY(sc.get(&err, 2));
  RS_CHECK_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int32_t), s));
  static bool attr = false;
  if (!attr) {
    const int mx = (int)(sizeof(double) + sizeof(int32_t)) * kHash * (kGemmThreads / 32);
    RS_CHECK_CUDA(cudaFuncSetAttribute(k_spgemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    RS_CHECK_CUDA(cudaFuncSetAttribute(k_spgemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    attr = true;
  }
  // per-warp table: twice the largest row's product count, as a power of two
  // (32..kHash); rows with more products than kHash / 2 are an error
  int32_t maxprod = 0;
  if (A.n > 0) {
    RS_COUNTED k_spgemm_maxprod<<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, B.rowptr, err + 1);
    RS_CHECK_CUDA(cudaMemcpyAsync(&maxprod, err + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  int32_t tcap = 32;
  while (tcap < kHash && tcap < 2 * maxprod) tcap *= 2;
  // as many warps per CTA as keep a CTA's tables within 48 KB (1..8)
  int warps = (int)std::min<int64_t>(kGemmThreads / 32, std::max<int64_t>(1, (48 * 1024) / (12 * (int64_t)tcap)));
  const size_t shm = (sizeof(double) + sizeof(int32_t)) * (size_t)tcap * warps;
  const unsigned grid = (unsigned)std::min<int64_t>((A.n + warps - 1) / warps, (int64_t)num_sms() * 32);
  ProfScope ps(kProfSpgemm, A.nnz * 12.0 + B.nnz * 12.0, s);
  if (A.n > 0)
    RS_COUNTED k_spgemm<false><<<grid, 32 * warps, shm, s>>>(A.n, tcap, A.rowptr, A.col, A.val, B.rowptr, B.col,
                                                             B.val, C.rowptr, nullptr, nullptr, err);
  int32_t tot = 0;
  RS_TRY(exclusive_scan(C.rowptr, C.rowptr, A.n, s, &tot));
  int32_t herr = 0;
  RS_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (herr) return fail(RS_ESETUP, "sparse product row exceeds the per-row table");
  C.nnz = tot;
  RS_TRY(dalloc_n(&C.col, (size_t)tot, s));
  RS_TRY(dalloc_n(&C.val, (size_t)tot, s));
  if (A.n > 0)
    RS_COUNTED k_spgemm<true><<<grid, 32 * warps, shm, s>>>(A.n, tcap, A.rowptr, A.col, A.val, B.rowptr, B.col,
                                                            B.val, C.rowptr, C.col, C.val, err);
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

// Sort each row by column (rows of a transpose are short).
__global__ void k_row_sort(int32_t n, const int32_t *rp, int32_t *col, double *val) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t s = rp[i], e = rp[i + 1];
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
  if (A.m > 0) RS_COUNTED k_row_sort<<<grid_for(A.m), kBlock, 0, s>>>(A.m, T.rowptr, T.col, T.val);
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

// C = A - B on the union pattern; an entry missing from A counts as 0.0
// (so the result is 0.0 - b), one missing from B leaves a.
template <bool FILL>
__global__ void k_sub(int32_t n, const int32_t *arp, const int32_t *acol, const double *aval, const int32_t *brp,
                      const int32_t *bcol, const double *bval, int32_t *crp, int32_t *ccol, double *cval) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t p = arp[i], pe = arp[i + 1], q = brp[i], qe = brp[i + 1], o = FILL ? crp[i] : 0, c = 0;
  while (p < pe || q < qe) {
    const int32_t ja = p < pe ? acol[p] : 0x7fffffff, jb = q < qe ? bcol[q] : 0x7fffffff;
    if (ja == jb) {
      if (FILL) { ccol[o + c] = ja; cval[o + c] = aval[p] - bval[q]; }
      p++; q++;
    } else if (ja < jb) {
      if (FILL) { ccol[o + c] = ja; cval[o + c] = aval[p]; }
      p++;
    } else {
      if (FILL) { ccol[o + c] = jb; cval[o + c] = 0.0 - bval[q]; }
      q++;
    }
    c++;
  }
  if (!FILL) crp[i] = c;
}

int csr_sub(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
  C.n = A.n;
  C.m = A.m;
  RS_TRY(dalloc_n(&C.rowptr, (size_t)A.n + 1, s));
  if (A.n > 0)
    RS_COUNTED k_sub<false><<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, C.rowptr,
                                                  nullptr, nullptr);
  int32_t tot = 0;
  RS_TRY(exclusive_scan(C.rowptr, C.rowptr, A.n, s, &tot));
  C.nnz = tot;
  RS_TRY(dalloc_n(&C.col, (size_t)tot, s));
  RS_TRY(dalloc_n(&C.val, (size_t)tot, s));
  if (A.n > 0)
    RS_COUNTED k_sub<true><<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, C.rowptr,
                                                 C.col, C.val);
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
