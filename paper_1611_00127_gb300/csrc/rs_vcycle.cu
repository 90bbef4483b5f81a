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
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "rs_internal.cuh"

namespace cg = cooperative_groups;

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

// Hybrid multicolour Gauss-Seidel sweep, one CTA per chunk of consecutive
// rows, on the level's packed smoother operator (per row: the off-diagonal
// entries inside the chunk with chunk-local columns, then the entries
// coupling to other chunks with global columns; the diagonal enters through
// its inverse). Couplings to other chunks read `xold` (the iterate at the
// start of the sweep; nullptr means the zero vector), so their contribution to
// each row is a constant of the sweep.
//
// Staging. Everything the CTA reads from HBM, apart from the xold values of
// other chunks, is a contiguous range: the chunk's packed row starts and
// split points, right-hand side, inverse diagonal, start iterate, rows by
// colour, and its packed columns and values. One thread issues a bulk
// asynchronous copy (cp.async.bulk, the TMA engine's 1D form) for the
// 16-byte-aligned interior of each range, all tracked by one mbarrier, so the
// whole chunk is in flight at once; the few elements before the first and
// after the last 16-byte boundary are loaded by plain loads. Each range lands
// in its shared-memory segment shifted by its global address mod 16, which
// keeps both sides of every bulk copy 16-byte aligned. Then each row's sum
// over other chunks is formed (gathers of xold, mostly from L2) and the
// colours are swept in order, a __syncthreads apart, on shared memory only.
// Chunks with more entries than the staging area read their entries from
// global memory instead. Result in `xnew`; the order of CTAs does not affect
// it.
// 16384 packed entries cover a 512-row chunk of a 25-point (3D Schur
// complement) level: 210 KB of shared memory in FP64 at the largest.
constexpr int kHgsStageEntries = 16384;
constexpr int kHgsMaxColours = 128;
constexpr int kHgsSpin = 1 << 20;     // bound on the mbarrier wait (iterations)
constexpr int kHgsThreads = 256;      // threads per chunk CTA

// Set when a smoother CTA gave up waiting for its staging copies; read and
// cleared by vcycle_wait_status().
__device__ int g_hgs_wait_timeout;

__host__ __device__ constexpr size_t hgs_seg(size_t bytes) { return ((bytes + 15) & ~size_t(15)) + 16; }

// Bounded wait of every thread of the CTA on the staging mbarrier (phase 0).
// Returns true, after a barrier, when the copies have landed. When a wait
// runs out it raises the timeout flag and waits once more, with the same
// bound, for the copies still in flight; the CTA then agrees (a barrier
// with a vote) to leave its rows unswept, so no thread reads shared memory
// the copies may not have filled and no thread exits while a copy of its
// CTA can still be writing, unless that second wait ran out as well.
__device__ __forceinline__ bool hgs_wait_staged(uint32_t ubar) {
  uint32_t done = 0;
  for (int it = 0; it < kHgsSpin && !done; it++)
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(ubar) : "memory");
  const bool first = done != 0;
  if (!first) {
    atomicOr(&g_hgs_wait_timeout, 1);
    for (int it = 0; it < kHgsSpin && !done; it++)
      asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                   : "=r"(done) : "r"(ubar) : "memory");
  }
  return __syncthreads_and(first ? 1 : 0) != 0;
}

// Dynamic shared memory of a sweep CTA: chunks of up to cmax rows, up to
// `stage` packed entries staged, ncol colours (the colour offsets come last,
// so a smaller ncol only trims the end).
template <typename T>
constexpr size_t hgs_smem(int cmax, int stage, int ncol = kHgsMaxColours) {
  return 3 * hgs_seg(sizeof(T) * (size_t)cmax) + hgs_seg(sizeof(T) * (size_t)stage) +
         hgs_seg(sizeof(int32_t) * (size_t)stage) + hgs_seg(sizeof(int32_t) * ((size_t)cmax + 1)) +
         2 * hgs_seg(sizeof(int32_t) * (size_t)cmax) + sizeof(int32_t) * ((size_t)ncol + 1);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Where the elements [off, off + cnt) of global array g go in a segment: the
// shifted base (same address mod 16 as g + off), the number of leading
// elements before the first 16-byte boundary, and the aligned interior bytes.
template <typename E>
struct BulkRange {
  E *dst;
  const E *src;
  int32_t cnt, head;
  uint32_t bytes;
  __device__ BulkRange(unsigned char *seg, const E *g, int64_t off, int32_t n) {
    src = g + off;
    const uint32_t shift = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15u);
    dst = reinterpret_cast<E *>(seg + shift);
    cnt = n;
    head = min(n, static_cast<int32_t>(((16u - shift) & 15u) / sizeof(E)));
    bytes = static_cast<uint32_t>(((int64_t)(n - head) * (int64_t)sizeof(E)) & ~int64_t(15));
  }
  __device__ int32_t tail_begin() const { return head + static_cast<int32_t>(bytes / sizeof(E)); }
  // thread 0: bulk copy of the interior
  __device__ void issue(uint32_t bar) const {
    if (bytes == 0) return;
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_addr(dst + head)), "l"(src + head), "r"(bytes), "r"(bar) : "memory");
  }
  // every thread: its share of the head and tail elements
  __device__ void edges(int t, int nt) const {
    for (int32_t e = t; e < head; e += nt) dst[e] = __ldg(src + e);
    for (int32_t e = tail_begin() + t; e < cnt; e += nt) dst[e] = __ldg(src + e);
  }
};

template <typename T, int LPR>
__global__ void __launch_bounds__(kHgsThreads) k_hgs(const int32_t *__restrict__ cr, const int32_t *__restrict__ coff,
                                             const int32_t *__restrict__ crows, int32_t ncol, int32_t cmax,
                                             int32_t stage_cap, const int32_t *__restrict__ hrp,
                                             const int32_t *__restrict__ hmid, const int32_t *__restrict__ hcol,
                                             const T *__restrict__ hval, const T *__restrict__ dinv,
                                             const T *__restrict__ b, const T *__restrict__ xold,
                                             T *__restrict__ xnew, const uint8_t *__restrict__ act,
                                             const int32_t *__restrict__ csys) {
  RS_PDL_ENTRY();
  if (act && !act[csys[blockIdx.x]]) {   // a retired system of a batch: zeros
    const int32_t q0 = __ldg(cr + 2 * blockIdx.x), q1 = __ldg(cr + 2 * blockIdx.x + 1);
    for (int32_t t = q0 + threadIdx.x; t < q1; t += blockDim.x) xnew[t] = T(0);
    return;
  }
  // entries of the out-of-chunk pass in flight per lane: four for FP32; two
  // for FP64, where every issued FMA costs FP64-pipe time even for lanes
  // past their row's end (rows of 7-point levels have two or three such
  // entries)
  constexpr int kOffU = sizeof(T) == 8 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  unsigned char *seg = smem;
  unsigned char *seg_x = seg;    seg += hgs_seg(sizeof(T) * cmax);
  unsigned char *seg_b = seg;    seg += hgs_seg(sizeof(T) * cmax);
  unsigned char *seg_d = seg;    seg += hgs_seg(sizeof(T) * cmax);
  unsigned char *seg_v = seg;    seg += hgs_seg(sizeof(T) * stage_cap);
  unsigned char *seg_c = seg;    seg += hgs_seg(sizeof(int32_t) * stage_cap);
  unsigned char *seg_rp = seg;   seg += hgs_seg(sizeof(int32_t) * (cmax + 1));
  unsigned char *seg_md = seg;   seg += hgs_seg(sizeof(int32_t) * cmax);
  unsigned char *seg_rw = seg;   seg += hgs_seg(sizeof(int32_t) * cmax);
  int32_t *scof = reinterpret_cast<int32_t *>(seg);            // colour offsets [ncol+1]

  const int32_t k = blockIdx.x;
  const int32_t r0 = __ldg(cr + 2 * k), r1 = __ldg(cr + 2 * k + 1), len = r1 - r0;
  const int32_t p0 = __ldg(hrp + r0), np = __ldg(hrp + r1) - p0;
  const bool staged = np <= stage_cap;
  const int32_t *cof = coff + (int64_t)k * (ncol + 1);

  const BulkRange<int32_t> g_rp(seg_rp, hrp, r0, len + 1);
  const BulkRange<int32_t> g_md(seg_md, hmid, r0, len);
  const BulkRange<T> g_b(seg_b, b, r0, len);
  const BulkRange<T> g_d(seg_d, dinv, r0, len);
  const BulkRange<int32_t> g_rw(seg_rw, crows, r0, len);
  const BulkRange<T> g_x(seg_x, xold ? xold : b, r0, xold ? len : 0);
  const BulkRange<int32_t> g_c(seg_c, hcol, p0, staged ? np : 0);
  const BulkRange<T> g_v(seg_v, hval, p0, staged ? np : 0);
  const uint32_t ubar = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ubar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t tx = g_rp.bytes + g_md.bytes + g_b.bytes + g_d.bytes + g_rw.bytes + g_x.bytes + g_c.bytes +
                        g_v.bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(ubar), "r"(tx) : "memory");
    g_c.issue(ubar);
    g_v.issue(ubar);
    g_rp.issue(ubar);
    g_md.issue(ubar);
    g_rw.issue(ubar);
    g_b.issue(ubar);
    g_d.issue(ubar);
    g_x.issue(ubar);
  } else {
    const int t = threadIdx.x - 1, nt = blockDim.x - 1;
    g_rp.edges(t, nt);
    g_md.edges(t, nt);
    g_b.edges(t, nt);
    g_d.edges(t, nt);
    g_rw.edges(t, nt);
    g_x.edges(t, nt);
    g_c.edges(t, nt);
    g_v.edges(t, nt);
  }
  for (int32_t c = threadIdx.x; c <= ncol; c += blockDim.x) scof[c] = __ldg(cof + c);
  T *xs = g_x.dst;
  if (!xold)
    for (int32_t t = threadIdx.x; t < len; t += blockDim.x) xs[t] = T(0);
  // bounded wait for the bulk copies (phase 0 of the barrier)
  if (!hgs_wait_staged(ubar)) return;
  const int32_t *lrp = g_rp.dst;       // packed row starts of rows r0..r1
  const int32_t *lmd = g_md.dst;       // packed split points
  T *rhs = g_b.dst;
  const T *dv = g_d.dst;
  const int32_t *srows = g_rw.dst;
  const int32_t *pcol = staged ? g_c.dst : hcol + p0;
  const T *pval = staged ? g_v.dst : hval + p0;
  const int group = threadIdx.x / LPR, lane = threadIdx.x % LPR, ngroups = blockDim.x / LPR;
  // rhs_i = b_i - sum_j a_ij xold_j over other chunks (uniform trip count:
  // the group shuffles see whole warps); kOffU gathers in flight per lane
  if (xold) {
    for (int32_t base = 0; base < len; base += ngroups) {
      const int32_t li = base + group;
      const bool act = li < len;
      T off = T(0);
      if (act) {
        if (lane == 0) off = rhs[li];
        const int32_t m = lmd[li] - p0, e = lrp[li + 1] - p0;
        for (int32_t q = m + lane; q < e; q += kOffU * LPR) {
          int32_t jj[kOffU];
          T aa[kOffU], xx[kOffU];
#pragma unroll
          for (int u = 0; u < kOffU; u++) {
            const int32_t qq = q + u * LPR;
            jj[u] = qq < e ? pcol[qq] : -1;
            aa[u] = qq < e ? pval[qq] : T(0);
          }
#pragma unroll
          for (int u = 0; u < kOffU; u++) xx[u] = jj[u] >= 0 ? __ldg(xold + jj[u]) : T(0);
#pragma unroll
          for (int u = 0; u < kOffU; u++)
            if (jj[u] >= 0) off -= aa[u] * xx[u];
        }
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) off += __shfl_down_sync(0xffffffffu, off, o, LPR);
      if (act && lane == 0) rhs[li] = off;
    }
  }
  __syncthreads();
  // colour passes over the entries inside the chunk
  for (int32_t c = 0; c < ncol; c++) {
    const int32_t beg = scof[c], end = scof[c + 1];
    for (int32_t base = beg; base < end; base += ngroups) {
      const int32_t pos = base + group;
      int32_t li = -1;
      T acc = T(0);
      if (pos < end) {
        li = srows[pos];
        if (lane == 0) acc = rhs[li];
        const int32_t s0 = lrp[li] - p0, m = lmd[li] - p0;
        for (int32_t q = s0 + lane; q < m; q += LPR) acc -= pval[q] * xs[pcol[q]];
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LPR);
      if (li >= 0 && lane == 0) {
        const T di = dv[li];
        if (di != T(0)) xs[li] = acc * di;
      }
    }
    __syncthreads();
  }
  for (int32_t t = threadIdx.x; t < len; t += blockDim.x) xnew[r0 + t] = xs[t];
}

// Point-block hybrid Gauss-Seidel sweep of systems AMG (two interleaved
// unknowns per point, rows 2i and 2i+1 of point i): the same chunking,
// staging and packed operator as k_hgs (the packed rows leave out the whole
// 2 x 2 diagonal block of their point), points coloured inside the chunk,
// and each point of the current colour set to the inverse of its diagonal
// block times its two right-hand sides less their couplings (a point whose
// block is singular keeps its values). One thread per point.
template <typename T>
constexpr size_t hgs2_smem(int cmax, int stage, int ncol = kHgsMaxColours) {
  return 2 * hgs_seg(sizeof(T) * (size_t)cmax) + hgs_seg(sizeof(T) * 2 * (size_t)cmax) +
         hgs_seg(sizeof(T) * (size_t)stage) + hgs_seg(sizeof(int32_t) * (size_t)stage) +
         hgs_seg(sizeof(int32_t) * ((size_t)cmax + 1)) + 2 * hgs_seg(sizeof(int32_t) * (size_t)cmax) +
         sizeof(int32_t) * ((size_t)ncol + 1);
}

template <typename T, int LPR>
__global__ void __launch_bounds__(kHgsThreads) k_hgs2(const int32_t *__restrict__ cr, const int32_t *__restrict__ coff,
                                              const int32_t *__restrict__ crows, int32_t ncol, int32_t cmax,
                                              int32_t stage_cap, const int32_t *__restrict__ hrp,
                                              const int32_t *__restrict__ hmid, const int32_t *__restrict__ hcol,
                                              const T *__restrict__ hval, const T *__restrict__ binv,
                                              const T *__restrict__ b, const T *__restrict__ xold,
                                              T *__restrict__ xnew, const uint8_t *__restrict__ act,
                                              const int32_t *__restrict__ csys) {
  RS_PDL_ENTRY();
  if (act && !act[csys[blockIdx.x]]) {   // a retired system of a batch: zeros
    const int32_t q0 = __ldg(cr + 2 * blockIdx.x), q1 = __ldg(cr + 2 * blockIdx.x + 1);
    for (int32_t t = q0 + threadIdx.x; t < q1; t += blockDim.x) xnew[t] = T(0);
    return;
  }
  // entries of the out-of-chunk pass in flight per lane: four for FP32; two
  // for FP64, where every issued FMA costs FP64-pipe time even for lanes
  // past their row's end (rows of 7-point levels have two or three such
  // entries)
  constexpr int kOffU = sizeof(T) == 8 ? 2 : 4;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;
  unsigned char *seg = smem;
  unsigned char *seg_x = seg;    seg += hgs_seg(sizeof(T) * cmax);
  unsigned char *seg_b = seg;    seg += hgs_seg(sizeof(T) * cmax);
  unsigned char *seg_d = seg;    seg += hgs_seg(sizeof(T) * 2 * cmax);
  unsigned char *seg_v = seg;    seg += hgs_seg(sizeof(T) * stage_cap);
  unsigned char *seg_c = seg;    seg += hgs_seg(sizeof(int32_t) * stage_cap);
  unsigned char *seg_rp = seg;   seg += hgs_seg(sizeof(int32_t) * (cmax + 1));
  unsigned char *seg_md = seg;   seg += hgs_seg(sizeof(int32_t) * cmax);
  unsigned char *seg_rw = seg;   seg += hgs_seg(sizeof(int32_t) * cmax);
  int32_t *scof = reinterpret_cast<int32_t *>(seg);            // colour offsets [ncol+1], in points

  const int32_t k = blockIdx.x;
  const int32_t r0 = __ldg(cr + 2 * k), r1 = __ldg(cr + 2 * k + 1), len = r1 - r0, npt = len / 2;
  const int32_t p0 = __ldg(hrp + r0), np = __ldg(hrp + r1) - p0;
  const bool staged = np <= stage_cap;
  const int32_t *cof = coff + (int64_t)k * (ncol + 1);

  const BulkRange<int32_t> g_rp(seg_rp, hrp, r0, len + 1);
  const BulkRange<int32_t> g_md(seg_md, hmid, r0, len);
  const BulkRange<T> g_b(seg_b, b, r0, len);
  const BulkRange<T> g_d(seg_d, binv, 2 * (int64_t)r0, 2 * len);
  const BulkRange<int32_t> g_rw(seg_rw, crows, r0 / 2, npt);
  const BulkRange<T> g_x(seg_x, xold ? xold : b, r0, xold ? len : 0);
  const BulkRange<int32_t> g_c(seg_c, hcol, p0, staged ? np : 0);
  const BulkRange<T> g_v(seg_v, hval, p0, staged ? np : 0);
  const uint32_t ubar = smem_addr(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(ubar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t tx = g_rp.bytes + g_md.bytes + g_b.bytes + g_d.bytes + g_rw.bytes + g_x.bytes + g_c.bytes +
                        g_v.bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(ubar), "r"(tx) : "memory");
    g_c.issue(ubar);
    g_v.issue(ubar);
    g_rp.issue(ubar);
    g_md.issue(ubar);
    g_rw.issue(ubar);
    g_b.issue(ubar);
    g_d.issue(ubar);
    g_x.issue(ubar);
  } else {
    const int t = threadIdx.x - 1, nt = blockDim.x - 1;
    g_rp.edges(t, nt);
    g_md.edges(t, nt);
    g_b.edges(t, nt);
    g_d.edges(t, nt);
    g_rw.edges(t, nt);
    g_x.edges(t, nt);
    g_c.edges(t, nt);
    g_v.edges(t, nt);
  }
  for (int32_t c = threadIdx.x; c <= ncol; c += blockDim.x) scof[c] = __ldg(cof + c);
  T *xs = g_x.dst;
  if (!xold)
    for (int32_t t = threadIdx.x; t < len; t += blockDim.x) xs[t] = T(0);
  if (!hgs_wait_staged(ubar)) return;
  const int32_t *lrp = g_rp.dst;
  const int32_t *lmd = g_md.dst;
  T *rhs = g_b.dst;
  const T *dv = g_d.dst;
  const int32_t *srows = g_rw.dst;
  const int32_t *pcol = staged ? g_c.dst : hcol + p0;
  const T *pval = staged ? g_v.dst : hval + p0;
  const int group = threadIdx.x / LPR, lane = threadIdx.x % LPR, ngroups = blockDim.x / LPR;
  // right-hand sides less the couplings to other chunks, a group of LPR
  // lanes per row (uniform trip count: the group shuffles see whole warps)
  if (xold) {
    for (int32_t base = 0; base < len; base += ngroups) {
      const int32_t lr = base + group;
      const bool act = lr < len;
      T acc = T(0);
      if (act) {
        if (lane == 0) acc = rhs[lr];
        const int32_t m = lmd[lr] - p0, e = lrp[lr + 1] - p0;
        for (int32_t q = m + lane; q < e; q += kOffU * LPR) {
          int32_t jj[kOffU];
          T aa[kOffU], xx[kOffU];
#pragma unroll
          for (int u = 0; u < kOffU; u++) {
            const int32_t qq = q + u * LPR;
            jj[u] = qq < e ? pcol[qq] : -1;
            aa[u] = qq < e ? pval[qq] : T(0);
          }
#pragma unroll
          for (int u = 0; u < kOffU; u++) xx[u] = jj[u] >= 0 ? __ldg(xold + jj[u]) : T(0);
#pragma unroll
          for (int u = 0; u < kOffU; u++)
            if (jj[u] >= 0) acc -= aa[u] * xx[u];
        }
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LPR);
      if (act && lane == 0) rhs[lr] = acc;
    }
  }
  __syncthreads();
  // colour passes: a group per point, its two rows' in-chunk sums, then the
  // 2 x 2 block solve
  for (int32_t c = 0; c < ncol; c++) {
    const int32_t beg = scof[c], end = scof[c + 1];
    for (int32_t base = beg; base < end; base += ngroups) {
      const int32_t pos = base + group;
      int32_t li = -1;
      T acc[2] = {T(0), T(0)};
      if (pos < end) {
        li = srows[pos];
#pragma unroll
        for (int f = 0; f < 2; f++) {
          const int32_t lr = 2 * li + f;
          T a = lane == 0 ? rhs[lr] : T(0);
          const int32_t s0 = lrp[lr] - p0, m = lmd[lr] - p0;
          for (int32_t q = s0 + lane; q < m; q += LPR) a -= pval[q] * xs[pcol[q]];
          acc[f] = a;
        }
      }
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) {
        acc[0] += __shfl_down_sync(0xffffffffu, acc[0], o, LPR);
        acc[1] += __shfl_down_sync(0xffffffffu, acc[1], o, LPR);
      }
      if (li >= 0 && lane == 0) {
        const T *mi = dv + 4 * li;
        if (mi[0] != T(0) || mi[1] != T(0) || mi[2] != T(0) || mi[3] != T(0)) {
          xs[2 * li] = mi[0] * acc[0] + mi[1] * acc[1];
          xs[2 * li + 1] = mi[2] * acc[0] + mi[3] * acc[1];
        }
      }
    }
    __syncthreads();
  }
  for (int32_t t = threadIdx.x; t < len; t += blockDim.x) xnew[r0 + t] = xs[t];
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

// y = b - A x over all rows (b == nullptr: y = A x); `accum`: y += A x.
// Groups of LPR lanes take rows in a grid-stride loop (the grid is capped at
// a few CTAs per SM, so large levels do not pay for tens of thousands of
// short-lived CTAs); the trip count is uniform across each warp.
// Batches: with `act`, the rows of a system whose flag is 0 get y = 0 (modes
// 0 and 1) or keep y (mode 2) without their sums being formed.
template <typename T, int LPR, int MODE>
__global__ void __launch_bounds__(256) k_csr(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                             const T *__restrict__ val, const T *__restrict__ x,
                                             const T *__restrict__ b, T *__restrict__ y,
                                             const uint8_t *__restrict__ act, const int32_t *__restrict__ rseg) {
  RS_PDL_ENTRY();
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / LPR;
  const int lane = threadIdx.x % LPR;
  for (int64_t base = 0; base < n; base += groups) {
    const int64_t i = base + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPR;
    const bool live = i < n && (act == nullptr || act[rseg[i]]);
    T s = T(0);
    if (live) {
      const int32_t e = __ldg(rp + i + 1);
      for (int32_t k = __ldg(rp + i) + lane; k < e; k += LPR) s += __ldg(val + k) * __ldg(x + __ldg(col + k));
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LPR);
    if (i < n && lane == 0) {
      if (MODE == 0) y[i] = live ? s : T(0);                 // y = A x
      else if (MODE == 1) y[i] = live ? b[i] - s : T(0);     // y = b - A x
      else if (live) y[i] += s;                              // y += A x
    }
  }
}

// grid of a k_csr launch over n rows with LPR lanes each
static unsigned csr_grid(int64_t n, int lpr) {
  const int64_t need = (n * lpr + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)num_sms() * 16;
  return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

// x[row] = A_c^{-1} b over the systems solved directly at this level, FP64
template <typename T>
__global__ void k_coarse_solve(int32_t nrows, const int32_t *__restrict__ crows, const int32_t *__restrict__ crow_seg,
                               const int4 *__restrict__ info, const int64_t *__restrict__ inv_off,
                               const double *__restrict__ inv, const T *__restrict__ b, T *__restrict__ x,
                               const uint8_t *__restrict__ act, const int32_t *__restrict__ crow_sys) {
  RS_PDL_ENTRY();
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;
  const int32_t row = crows[w];
  if (act && !act[crow_sys[w]]) {   // a retired system of a batch
    if (lane == 0) x[row] = T(0);
    return;
  }
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
  RS_PDL_ENTRY();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// Lanes per row. FP32: one lane for short rows (the row's entries share
// cache lines, and no reduction is needed), more for long coarse-level rows.
// FP64: GB300's FP64 pipe issues about 2 lanes per clock per SM, so every
// warp-wide FP64 instruction is costly even with idle lanes; FP64 kernels use
// one lane per row (two or four for long rows), which needs no FP64
// shuffle-reduction additions.
template <typename T>
static int pick_lpr(int32_t n, int32_t nnz) {
  const double avg = n > 0 ? (double)nnz / n : 1.0;
  if (sizeof(T) == 8) {
    if (avg <= 32.0) return 1;
    if (avg <= 128.0) return 2;
    return 4;
  }
  if (avg <= 16.0) return 1;
  if (avg <= 40.0) return 4;
  if (avg <= 96.0) return 8;
  return 16;
}

#define RS_LPR_SWITCH(lpr, ...)                  \
  switch (lpr) {                                 \
    case 1: { constexpr int L_ = 1; __VA_ARGS__; } break;   \
    case 2: { constexpr int L_ = 2; __VA_ARGS__; } break;   \
    case 4: { constexpr int L_ = 4; __VA_ARGS__; } break;   \
    case 8: { constexpr int L_ = 8; __VA_ARGS__; } break;   \
    case 16: { constexpr int L_ = 16; __VA_ARGS__; } break; \
    default: { constexpr int L_ = 32; __VA_ARGS__; } break; \
  }

// lanes per row of level L's transfer `which` (0 residual with A, 1
// restriction with R, 2 prolongation with P): the autotuned choice, else the
// rule above
template <typename T>
static int xfer_lpr(const Level &L, int which) {
  if (L.xfer_lpr[which] > 0) return L.xfer_lpr[which];
  const DCsr &M = which == 0 ? L.A : (which == 1 ? L.R : L.P);
  return pick_lpr<T>(M.n, M.nnz);
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
static const T *hs_vals(const Level &L);
template <>
const float *hs_vals<float>(const Level &L) { return L.hs_valf; }
template <>
const double *hs_vals<double>(const Level &L) { return L.hs_val; }

// Lanes per row of the hybrid sweep. Its inner loops run over a row's packed
// entries in shared memory. With at least half as many chunks as SMs the
// sweep is bandwidth-bound: one lane per row unless rows are long, which also
// keeps FP64 free of shuffle additions. With fewer chunks, a few CTAs walk
// the rows colour by colour, and the chains of dependent shared-memory loads
// and FMAs per row set the time, so more lanes shorten each chain; with very
// few chunks (under 16) even short rows are split.
static int hgs_lpr(int32_t n, int32_t nnz, int32_t nchunk) {
  const double avg = n > 0 ? (double)nnz / n : 1.0;
  if (2 * nchunk >= num_sms()) {
    if (avg <= 16.0) return 1;
    if (avg <= 64.0) return 4;
    return 8;
  }
  if (nchunk >= 16) {
    if (avg <= 6.0) return 1;
    if (avg <= 16.0) return 2;
    if (avg <= 32.0) return 4;
    if (avg <= 64.0) return 8;
    return 16;
  }
  if (avg <= 6.0) return 1;
  if (avg <= 12.0) return 2;
  if (avg <= 24.0) return 4;
  if (avg <= 48.0) return 8;
  return 16;
}

// Algorithmic bytes of one hybrid sweep over ns rows holding nz entries: the
// matrix entries and row pointers once, b once, the iterate written once and
// (unless it starts at zero) read once.
static double hgs_bytes(double ns, double nz, size_t es, bool xin) {
  return nz * (4.0 + es) + (ns + 1) * 4.0 + ns * es * (xin ? 3.0 : 2.0);
}

template <typename T>
static const T *binv_of(const Level &L);
template <>
const float *binv_of<float>(const Level &L) { return L.binvf; }
template <>
const double *binv_of<double>(const Level &L) { return L.binv; }

static_assert(hgs_smem<double>(512, kHgsStageEntries) + 16 <= 232448, "sweep staging exceeds shared memory");
static_assert(hgs2_smem<double>(512, kHgsStageEntries) + 16 <= 232448, "sweep staging exceeds shared memory");

template <typename T, int LPR>
static void hgs2_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_hgs2<T, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)hgs2_smem<T>(512, kHgsStageEntries));
    done = true;
  }
}

template <typename T, int LPR>
static void hgs_attr() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_hgs<T, LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)hgs_smem<T>(512, kHgsStageEntries));
    done = true;
  }
}

// Smoothing sweeps on level l. `cur` holds the current iterate on entry (or
// is nullptr when it is zero) and the buffer holding the result on exit.
template <typename T>
static void smooth(const Hier &H, const Level &L, int sweeps, T *&cur, cudaStream_t s) {
  if (sweeps <= 0) return;
  const int lpr = pick_lpr<T>(L.A.n, L.A.nnz);
  const T *val = vals<T>(L.A);
  const T *dinv = dinv_of<T>(L);
  const T *b = static_cast<const T *>(L.b);
  T *xa = static_cast<T *>(L.x), *xb = static_cast<T *>(L.x2);
  if (L.nsmooth == 0) {
    if (!cur) {
      cudaMemsetAsync(xa, 0, sizeof(T) * (size_t)L.A.n, s);
      cur = xa;
    }
    return;
  }
  if (H.prm.smoother == RS_SMOOTH_HYBRID) {
    // staging area: the level's largest chunk of packed entries (the diagonal
    // is not among them)
    const int32_t stage = std::min(L.hs_chunk_max, kHgsStageEntries);
    const int32_t cmax = L.chunk_c > 0 ? L.chunk_c : H.prm.chunk;   // the level's largest chunk
    const size_t shm = hgs_smem<T>(cmax, stage, L.ncolour);
    const double ns = L.nsmooth, nz = L.A.n ? (double)L.A.nnz * ns / L.A.n : 0.0;
    const int hl = L.hgs_lpr > 0 ? L.hgs_lpr : hgs_lpr(L.A.n, L.A.nnz, L.nchunk);
    if (L.nfun == 2) {
      const size_t shm2 = hgs2_smem<T>(cmax, stage, L.ncolour);
      for (int sw = 0; sw < sweeps; sw++) {
        T *out = (cur == xa) ? xb : xa;
        ProfScope ps(kProfHgs, hgs_bytes(ns, nz, sizeof(T), cur != nullptr), s);
        RS_LPR_SWITCH(hl, hgs2_attr<T, L_>(); RS_COUNTED launch_pdl(k_hgs2<T, L_>, dim3(L.nchunk), dim3(kHgsThreads),
                              shm2, s, L.chunk_row0, L.chunk_coff, L.chunk_rows, L.ncolour, cmax, stage,
                              L.hs_rp, L.hs_mid, L.hs_col, hs_vals<T>(L), binv_of<T>(L), b, (const T *)cur, out,
                              H.active, (const int32_t *)L.chunk_sys));
        cur = out;
      }
      return;
    }
    for (int sw = 0; sw < sweeps; sw++) {
      T *out = (cur == xa) ? xb : xa;
      ProfScope ps(kProfHgs, hgs_bytes(ns, nz, sizeof(T), cur != nullptr), s);
      RS_LPR_SWITCH(hl, hgs_attr<T, L_>(); RS_COUNTED launch_pdl(k_hgs<T, L_>, dim3(L.nchunk), dim3(kHgsThreads), shm, s,
                            L.chunk_row0, L.chunk_coff, L.chunk_rows, L.ncolour, cmax, stage, L.hs_rp,
                            L.hs_mid, L.hs_col, hs_vals<T>(L), dinv, b, (const T *)cur, out, H.active,
                            (const int32_t *)L.chunk_sys));
      cur = out;
    }
    return;
  }
  if (!cur) {
    cudaMemsetAsync(xa, 0, sizeof(T) * (size_t)L.A.n, s);
    cur = xa;
  }
  T *x = cur;
  for (int sw = 0; sw < sweeps; sw++) {
    if (H.prm.smoother == RS_SMOOTH_L1JACOBI) {
      T *t = static_cast<T *>(L.t);
      const int32_t nr = L.nsmooth;
      RS_LPR_SWITCH(lpr, RS_COUNTED k_resid_rows<T, L_><<<grid_for((int64_t)nr * L_), kBlock, 0, s>>>(
                             nr, L.colour_rows, L.A.rowptr, L.A.col, val, b, x, t));
      RS_COUNTED k_jacobi_update<T><<<grid_for(nr), kBlock, 0, s>>>(nr, L.colour_rows, dinv, t, x);
    } else {
      for (int c = 0; c < L.ncolour; c++) {
        const int32_t r0 = L.colour_off[c], nr = L.colour_off[c + 1] - r0;
        if (nr == 0) continue;
        RS_LPR_SWITCH(lpr, RS_COUNTED k_gs_colour<T, L_><<<grid_for((int64_t)nr * L_), kBlock, 0, s>>>(
                               nr, L.colour_rows + r0, L.A.rowptr, L.A.col, val, dinv, b, x));
      }
    }
  }
}

// One V-cycle on level l with zero initial guess; returns the buffer that
// holds x_l.
template <typename T>
static T *cycle(const Hier &H, int32_t l, cudaStream_t s) {
  const Level &L = H.L[l];
  T *cur = nullptr;
  smooth<T>(H, L, H.prm.nu1, cur, s);
  if (!cur) {
    cur = static_cast<T *>(L.x);
    cudaMemsetAsync(cur, 0, sizeof(T) * (size_t)L.A.n, s);
  }
  if (l + 1 < H.nlev && L.P.rowptr) {
    const Level &N = H.L[l + 1];
    T *r = static_cast<T *>(L.r);
    const double sz = sizeof(T);
    const int lpr = xfer_lpr<T>(L, 0);
    {
      ProfScope ps(kProfCsr, L.A.nnz * (4.0 + sz) + (L.A.n + 1) * 4.0 + 3.0 * L.A.n * sz, s);
      RS_LPR_SWITCH(lpr, RS_COUNTED launch_pdl(k_csr<T, L_, 1>, dim3(csr_grid(L.A.n, L_)), dim3(kBlock), 0, s,
                             L.A.n, L.A.rowptr, L.A.col, vals<T>(L.A), (const T *)cur, static_cast<const T *>(L.b), r,
                             H.active, (const int32_t *)L.row_seg));
    }
    const int lr = xfer_lpr<T>(L, 1);
    {
      ProfScope ps(kProfCsr, L.R.nnz * (4.0 + sz) + (L.R.n + 1) * 4.0 + (L.R.n + L.A.n) * sz, s);
      RS_LPR_SWITCH(lr, RS_COUNTED launch_pdl(k_csr<T, L_, 0>, dim3(csr_grid(L.R.n, L_)), dim3(kBlock), 0, s,
                            L.R.n, L.R.rowptr, L.R.col, vals<T>(L.R), (const T *)r, (const T *)nullptr, static_cast<T *>(N.b),
                            H.active, (const int32_t *)N.row_seg));
    }
    const T *xc = cycle<T>(H, l + 1, s);
    const int lp = xfer_lpr<T>(L, 2);
    {
      ProfScope ps(kProfCsr, L.P.nnz * (4.0 + sz) + (L.P.n + 1) * 4.0 + (2.0 * L.P.n + L.R.n) * sz, s);
      RS_LPR_SWITCH(lp, RS_COUNTED launch_pdl(k_csr<T, L_, 2>, dim3(csr_grid(L.P.n, L_)), dim3(kBlock), 0, s,
                            L.P.n, L.P.rowptr, L.P.col, vals<T>(L.P), xc, (const T *)nullptr, cur, H.active,
                            (const int32_t *)L.row_seg));
    }
  }
  smooth<T>(H, L, H.prm.nu2, cur, s);
  if (L.ncoarse_rows > 0) {
    RS_COUNTED launch_pdl(k_coarse_solve<T>, dim3(grid_for((int64_t)L.ncoarse_rows * 32)), dim3(kBlock), 0, s,
        L.ncoarse_rows, (const int32_t *)L.crows, (const int32_t *)L.crow_seg, (const int4 *)L.cinfo,
        (const int64_t *)L.cinv_off, (const double *)L.cinv, static_cast<const T *>(L.b), cur, H.active,
        (const int32_t *)L.crow_sys);
  }
  return cur;
}

// Sweeps of level l's smoother on the hierarchy's own vectors (right-hand
// side b_l as left by the last cycle, iterate x_l), for measurement.
template <typename T>
static double level_sweeps(const Hier &H, int32_t l, int sweeps, cudaStream_t s) {
  const Level &L = H.L[l];
  T *cur = static_cast<T *>(L.x);
  smooth<T>(H, L, sweeps, cur, s);
  const double ns = L.nsmooth, nz = L.A.n ? (double)L.A.nnz * ns / L.A.n : 0.0;
  return hgs_bytes(ns, nz, sizeof(T), true);
}

// Transfer kernels of level l, as the V-cycle launches them (same lanes per
// row), on the level's own vectors.
template <typename T>
static double level_xfer(const Hier &H, int32_t l, int which, int reps, cudaStream_t s) {
  const Level &L = H.L[l];
  const Level &N = H.L[l + 1];
  const double sz = sizeof(T);
  T *x = static_cast<T *>(L.x), *r = static_cast<T *>(L.r);
  for (int k = 0; k < reps; k++) {
    if (which == 0) {
      const int lpr = xfer_lpr<T>(L, 0);
      RS_LPR_SWITCH(lpr, RS_COUNTED launch_pdl(k_csr<T, L_, 1>, dim3(csr_grid(L.A.n, L_)), dim3(kBlock), 0,
                                               s, L.A.n, L.A.rowptr, L.A.col, vals<T>(L.A), (const T *)x,
                                               static_cast<const T *>(L.b), r, H.active, (const int32_t *)L.row_seg));
    } else if (which == 1) {
      const int lr = xfer_lpr<T>(L, 1);
      RS_LPR_SWITCH(lr, RS_COUNTED launch_pdl(k_csr<T, L_, 0>, dim3(csr_grid(L.R.n, L_)), dim3(kBlock), 0,
                                              s, L.R.n, L.R.rowptr, L.R.col, vals<T>(L.R), (const T *)r,
                                              (const T *)nullptr, static_cast<T *>(N.b), H.active,
                                              (const int32_t *)N.row_seg));
    } else {
      const int lp = xfer_lpr<T>(L, 2);
      RS_LPR_SWITCH(lp, RS_COUNTED launch_pdl(k_csr<T, L_, 2>, dim3(csr_grid(L.P.n, L_)), dim3(kBlock), 0,
                                              s, L.P.n, L.P.rowptr, L.P.col, vals<T>(L.P),
                                              (const T *)static_cast<T *>(N.x), (const T *)nullptr, x, H.active,
                                              (const int32_t *)L.row_seg));
    }
  }
  if (which == 0) return L.A.nnz * (4.0 + sz) + (L.A.n + 1) * 4.0 + 3.0 * L.A.n * sz;
  if (which == 1) return L.R.nnz * (4.0 + sz) + (L.R.n + 1) * 4.0 + (L.R.n + L.A.n) * sz;
  return L.P.nnz * (4.0 + sz) + (L.P.n + 1) * 4.0 + (2.0 * L.P.n + L.R.n) * sz;
}

int amg_level_xfer(const Hier &H, int32_t l, int which, int reps, double *bytes_per_launch, cudaStream_t s) {
  if (l < 0 || l + 1 >= H.nlev || !H.L[l].P.rowptr) return fail(RS_EINVAL, "level has no coarser level");
  if (which < 0 || which > 2) return fail(RS_EINVAL, "unknown transfer kernel");
  const double by = H.precision == RS_PREC_FP32 ? level_xfer<float>(H, l, which, reps, s)
                                                : level_xfer<double>(H, l, which, reps, s);
  if (bytes_per_launch) *bytes_per_launch = by;
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ smoother autotuner
// Key of a level shape: precision, unknowns per point, and log2 buckets of
// the chunk count and of the mean row length (x4); levels of one key get the
// same lanes per row.
static std::mutex g_hgs_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_hgs_tune;

static int ilog2(double v) {
  int k = 0;
  while (v >= 2.0 && k < 40) { v *= 0.5; k++; }
  return k;
}

template <typename T>
static int tune_level(const Hier &H, Level &L, cudaStream_t s) {
  static const int cand[] = {1, 2, 4, 8, 16};
  cudaEvent_t e0, e1;
  RS_CHECK_CUDA(cudaEventCreate(&e0));
  RS_CHECK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int bestl = 0;
  for (int c : cand) {
    L.hgs_lpr = c;
    T *cur = static_cast<T *>(L.x);
    smooth<T>(H, L, 1, cur, s);          // warm-up (kernel attributes, caches)
    RS_CHECK_CUDA(cudaEventRecord(e0, s));
    smooth<T>(H, L, 4, cur, s);
    RS_CHECK_CUDA(cudaEventRecord(e1, s));
    RS_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (bestl == 0 || ms < best) { best = ms; bestl = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.hgs_lpr = bestl;
  return 0;
}

// Transfers, the same way: each level's residual, restriction and
// prolongation time every lanes-per-row choice on the level's own vectors;
// decisions are cached per (precision, transfer, log2 rows, log2 of 4x the
// mean row length).
static std::mutex g_xfer_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_xfer_tune;

template <typename T>
static int tune_xfer(Hier &H, int32_t l, int which, cudaStream_t s) {
  static const int cand64[] = {1, 2, 4, 8}, cand32[] = {1, 2, 4, 8, 16};
  const int *cand = sizeof(T) == 8 ? cand64 : cand32;
  const int ncand = sizeof(T) == 8 ? 4 : 5;
  Level &L = H.L[l];
  cudaEvent_t e0, e1;
  RS_CHECK_CUDA(cudaEventCreate(&e0));
  RS_CHECK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int bestl = 0;
  for (int k = 0; k < ncand; k++) {
    L.xfer_lpr[which] = (int8_t)cand[k];
    level_xfer<T>(H, l, which, 1, s);     // warm-up
    RS_CHECK_CUDA(cudaEventRecord(e0, s));
    level_xfer<T>(H, l, which, 4, s);
    RS_CHECK_CUDA(cudaEventRecord(e1, s));
    RS_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RS_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (bestl == 0 || ms < best) { best = ms; bestl = cand[k]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.xfer_lpr[which] = (int8_t)bestl;
  return 0;
}

static int tune_transfers(Hier &H, cudaStream_t s) {
  for (int32_t l = 0; l + 1 < H.nlev; l++) {
    Level &L = H.L[l];
    if (!L.P.rowptr || L.A.n == 0) continue;
    for (int which = 0; which < 3; which++) {
      const DCsr &M = which == 0 ? L.A : (which == 1 ? L.R : L.P);
      if (M.n == 0) continue;
      const auto key = std::make_tuple(H.precision, which, ilog2((double)M.n),
                                       ilog2(4.0 * (double)M.nnz / (double)M.n));
      {
        std::lock_guard<std::mutex> lock(g_xfer_tune_mu);
        auto it = g_xfer_tune.find(key);
        if (it != g_xfer_tune.end()) {
          L.xfer_lpr[which] = (int8_t)it->second;
          continue;
        }
      }
      RS_TRY(H.precision == RS_PREC_FP32 ? tune_xfer<float>(H, l, which, s) : tune_xfer<double>(H, l, which, s));
      std::lock_guard<std::mutex> lock(g_xfer_tune_mu);
      g_xfer_tune[key] = L.xfer_lpr[which];
    }
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int amg_tune_smoother(Hier &H, cudaStream_t s) {
  RS_TRY(tune_transfers(H, s));
  if (H.prm.smoother != RS_SMOOTH_HYBRID) return 0;
  for (int32_t l = 0; l < H.nlev; l++) {
    Level &L = H.L[l];
    if (L.nsmooth == 0 || L.nchunk == 0 || L.A.n == 0) continue;
    const auto key = std::make_tuple(H.precision, (int)L.nfun, ilog2((double)L.nchunk),
                                     ilog2(4.0 * (double)L.A.nnz / (double)L.A.n));
    {
      std::lock_guard<std::mutex> lock(g_hgs_tune_mu);
      auto it = g_hgs_tune.find(key);
      if (it != g_hgs_tune.end()) {
        L.hgs_lpr = it->second;
        continue;
      }
    }
    RS_TRY(H.precision == RS_PREC_FP32 ? tune_level<float>(H, L, s) : tune_level<double>(H, L, s));
    std::lock_guard<std::mutex> lock(g_hgs_tune_mu);
    g_hgs_tune[key] = L.hgs_lpr;
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int vcycle_wait_status(cudaStream_t s) {
  int h = 0;
  RS_CHECK_CUDA(cudaMemcpyFromSymbolAsync(&h, g_hgs_wait_timeout, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  if (h == 0) return 0;
  const int z = 0;
  RS_CHECK_CUDA(cudaMemcpyToSymbolAsync(g_hgs_wait_timeout, &z, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  return fail(RS_ETIMEOUT, "smoother: a staging copy did not complete within the wait limit");
}

int vcycle_raise_wait_flag(cudaStream_t s) {
  const int one = 1;
  RS_CHECK_CUDA(cudaMemcpyToSymbolAsync(g_hgs_wait_timeout, &one, sizeof(int), 0, cudaMemcpyHostToDevice, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  return 0;
}

int amg_level_sweeps(const Hier &H, int32_t l, int sweeps, double *bytes_per_sweep, cudaStream_t s) {
  if (l < 0 || l >= H.nlev) return fail(RS_EINVAL, "level out of range");
  const double by = H.precision == RS_PREC_FP32 ? level_sweeps<float>(H, l, sweeps, s)
                                                : level_sweeps<double>(H, l, sweeps, s);
  if (bytes_per_sweep) *bytes_per_sweep = by;
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

int amg_vcycle(const Hier &H, const double *b, double *x, cudaStream_t s) {
  if (H.nlev == 0) return fail(RS_EINVAL, "empty hierarchy");
  const Level &L0 = H.L[0];
  const int64_t n = L0.A.n;
  if (n == 0) return 0;
  if (H.precision == RS_PREC_FP32) {
    RS_COUNTED launch_pdl(k_cast<double, float>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, b, static_cast<float *>(L0.b));
    const float *x0 = cycle<float>(H, 0, s);
    RS_COUNTED launch_pdl(k_cast<float, double>, dim3(grid_for(n)), dim3(kBlock), 0, s, n, x0, x);
  } else {
    RS_CHECK_CUDA(cudaMemcpyAsync(L0.b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    const double *x0 = cycle<double>(H, 0, s);
    RS_CHECK_CUDA(cudaMemcpyAsync(x, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace rs

extern "C" int rs_wait_status(cudaStream_t stream) { return rs::vcycle_wait_status(stream); }

extern "C" int rs_raise_wait_flag(cudaStream_t stream) { return rs::vcycle_raise_wait_flag(stream); }
