// Right-preconditioned flexible GMRES(m) (Sec. 3, eq. precon-system: solve
// J M^{-1} c^ = q, c = M^{-1} c^; flexible because the AMG preconditioner
// changes from one application to the next in FP32), FP64, per system of a
// batch. Orthogonalisation is classical Gram-Schmidt applied twice (CGS2):
// each pass is one multi-dot kernel (all j+1 inner products against the new
// vector, which a block keeps in shared memory) plus one update kernel, in
// place of the paper solver's modified Gram-Schmidt, whose j+1 dependent dot
// products would each need a grid-wide reduction.
//
// Reductions are deterministic: each block reduces a fixed chunk of one
// system's rows, then one thread per (system, vector) sums the chunk partials
// in order. Givens rotations, the residual estimate and the convergence test
// run on the device, one thread per system.
#include <algorithm>
#include <cmath>

#include "rs_internal.cuh"

namespace rs {
int precond_apply_impl(const rs_precond *M, const double *r, double *z, cudaStream_t s);
int precond_set_active(const rs_precond *M, const uint8_t *active, cudaStream_t s);
}
using namespace rs;

namespace {

// Rows per reduction block: the CGS2 passes are FP64-FMA work, so a solve
// uses about four blocks per SM (at least 512 rows each, at most kChunk).
constexpr int kChunk = 4096;   // largest block (shared-memory copy of w)
static int64_t chunk_rows(int64_t n) {
  const int64_t want = (n + 4 * (int64_t)num_sms() - 1) / (4 * (int64_t)num_sms());
  int64_t c = 512;
  while (c < want && c < kChunk) c *= 2;
  return c;
}
constexpr int kRedThreads = 256;

struct Chunk {
  int32_t seg, beg, end;
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kRedThreads / 32; k++) t += sh[k];
  return t;
}

// part[c][i] = sum over chunk c of V_i . w, i < nvec  (V_i = V + i*ldv)
__global__ void __launch_bounds__(kRedThreads) k_multidot(const Chunk *__restrict__ chunks, const double *__restrict__ V,
                                                          int64_t ldv, int nvec, const double *__restrict__ w,
                                                          int stride, double *__restrict__ part) {
  __shared__ double ws[kChunk];
  __shared__ double sh[kRedThreads / 32];
  const Chunk ch = chunks[blockIdx.x];
  const int len = ch.end - ch.beg;
  for (int t = threadIdx.x; t < len; t += kRedThreads) ws[t] = w[ch.beg + t];
  __syncthreads();
  for (int i = 0; i < nvec; i++) {
    const double *vi = V + i * ldv + ch.beg;
    double acc = 0.0;
    for (int t = threadIdx.x; t < len; t += kRedThreads) acc = fma(vi[t], ws[t], acc);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * stride + i] = tot;
  }
}

// h[s][i] = sum of the partials of system s (in chunk order). mode 1: out = h
// and H(i, col) = h; mode 2: out = h and H(i, col) += h; mode 3 (norm):
// out[s] = sqrt(h). Inactive systems get h = 0.
__global__ void k_reduce(int32_t nseg, const int32_t *__restrict__ seg_chunk, int nvec, int stride,
                         const double *__restrict__ part, double *__restrict__ out, double *__restrict__ H,
                         int ldh_seg, int col, int mode, const uint8_t *__restrict__ active) {
  RS_PDL_ENTRY();
  // one warp per (system, vector): lane l sums chunks l, l+32, ... in order,
  // then a fixed shuffle tree adds the lanes (deterministic)
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)nseg * nvec) return;
  const int32_t s = (int32_t)(t / nvec);
  const int i = (int)(t % nvec);
  double acc = 0.0;
  for (int32_t c = seg_chunk[s] + lane; c < seg_chunk[s + 1]; c += 32) acc += part[(int64_t)c * stride + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane != 0) return;
  if (active && !active[s]) acc = 0.0;
  if (mode == 3) {
    out[s] = sqrt(acc);
    return;
  }
  out[(int64_t)s * stride + i] = acc;
  if (mode == 1) H[(int64_t)s * ldh_seg + (int64_t)i * 64 + col] = acc;
  else if (mode == 2) H[(int64_t)s * ldh_seg + (int64_t)i * 64 + col] += acc;
}

// w -= sum_i V_i h[seg][i]
__global__ void __launch_bounds__(kRedThreads) k_update(const Chunk *__restrict__ chunks, const double *__restrict__ V,
                                                        int64_t ldv, int nvec, const double *__restrict__ h,
                                                        int stride, double *__restrict__ w) {
  const Chunk ch = chunks[blockIdx.x];
  const double *hs = h + (int64_t)ch.seg * stride;
  for (int t = ch.beg + threadIdx.x; t < ch.end; t += kRedThreads) {
    double acc = w[t];
    for (int i = 0; i < nvec; i++) acc = fma(-V[i * ldv + t], hs[i], acc);
    w[t] = acc;
  }
}

// y = x * f[seg] (0 where f is 0 or not finite)
// y = x / nrm per system; also clears *zero (the next Givens step's counter
// of still-active systems) when given
__global__ void __launch_bounds__(kRedThreads) k_scale(const Chunk *__restrict__ chunks, const double *__restrict__ nrm,
                                                       const double *__restrict__ x, double *__restrict__ y,
                                                       int32_t *zero) {
  RS_PDL_ENTRY();
  if (zero && blockIdx.x == 0 && threadIdx.x == 0) *zero = 0;
  const Chunk ch = chunks[blockIdx.x];
  const double d = nrm[ch.seg];
  const double f = (d > 0.0 && isfinite(d)) ? 1.0 / d : 0.0;
  for (int t = ch.beg + threadIdx.x; t < ch.end; t += kRedThreads) y[t] = x[t] * f;
}

// x += sum_{i < k[seg]} y[seg][i] Z_i
__global__ void __launch_bounds__(kRedThreads) k_xupdate(const Chunk *__restrict__ chunks, const double *__restrict__ Z,
                                                         int64_t ldz, const double *__restrict__ y, int m,
                                                         const int32_t *__restrict__ kseg, double *__restrict__ x) {
  const Chunk ch = chunks[blockIdx.x];
  const int k = kseg[ch.seg];
  const double *ys = y + (int64_t)ch.seg * m;
  for (int t = ch.beg + threadIdx.x; t < ch.end; t += kRedThreads) {
    double acc = x[t];
    for (int i = 0; i < k; i++) acc = fma(ys[i], Z[i * ldz + t], acc);
    x[t] = acc;
  }
}

// Tiled multi-dot: part[c][i] = V_i . w over chunk c for i < nvec. Each thread
// keeps TILE running sums in registers, so a block does one reduction per
// tile of TILE vectors instead of one per vector; w is read from shared memory.
constexpr int kTile = 8;

__device__ __forceinline__ void block_sum_tile(double (&v)[kTile], double *sh, double *out, int nv) {
  // sh: [kRedThreads/32][kTile]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kTile; t++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[t] += __shfl_down_sync(0xffffffffu, v[t], o);
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < kTile; t++) sh[wid * kTile + t] = v[t];
  __syncthreads();
  if (threadIdx.x < nv) {
    double acc = 0.0;
    for (int w = 0; w < kRedThreads / 32; w++) acc += sh[w * kTile + threadIdx.x];
    out[threadIdx.x] = acc;
  }
}

// MODE 0: part = V_{0..nvec-1} . w
// MODE 1: w -= sum_i V_i h[seg][i], then part = V_{0..nvec-1} . w (next CGS pass)
// MODE 2: w -= sum_i V_i h[seg][i], then part[0] = w . w
// Chunks of a retired system (active[seg] = 0) do nothing: their partial
// sums are not read (the reductions mask retired systems).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_arnoldi(const Chunk *__restrict__ chunks, const double *__restrict__ V,
                                                         int64_t ldv, int nvec, const double *__restrict__ h, int stride,
                                                         double *__restrict__ w, double *__restrict__ part,
                                                         const uint8_t *__restrict__ active) {
  RS_PDL_ENTRY();
  if (active && !active[chunks[blockIdx.x].seg]) return;
  __shared__ double ws[kChunk];
  __shared__ double sh[(kRedThreads / 32) * kTile];
  const Chunk ch = chunks[blockIdx.x];
  const int len = ch.end - ch.beg;
  const double *hs = h ? h + (int64_t)ch.seg * stride : nullptr;
  for (int t = threadIdx.x; t < len; t += kRedThreads) {
    double x = w[ch.beg + t];
    if (MODE != 0) {
      for (int i = 0; i < nvec; i++) x = fma(-V[i * ldv + ch.beg + t], hs[i], x);
      w[ch.beg + t] = x;
    }
    ws[t] = x;
  }
  __syncthreads();
  if (MODE == 2) {
    double v[kTile] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < len; t += kRedThreads) v[0] = fma(ws[t], ws[t], v[0]);
    block_sum_tile(v, sh, part + (int64_t)blockIdx.x * stride, 1);
    return;
  }
  for (int i0 = 0; i0 < nvec; i0 += kTile) {
    const int nv = min(kTile, nvec - i0);
    double v[kTile] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < len; t += kRedThreads) {
      const double x = ws[t];
#pragma unroll
      for (int q = 0; q < kTile; q++)
        if (q < nv) v[q] = fma(V[(i0 + q) * ldv + ch.beg + t], x, v[q]);
    }
    block_sum_tile(v, sh, part + (int64_t)blockIdx.x * stride + i0, nv);
  }
}

struct SegState {
  double g[65];
  double cs[64], sn[64];
};

// Givens update of column j for every active system; convergence test on the
// residual estimate |g_{j+1}|.
__global__ void k_givens(int32_t nseg, int j, int m, double *__restrict__ H, int ldh_seg, const double *__restrict__ hnext,
                         SegState *__restrict__ st, uint8_t *__restrict__ active, int32_t *__restrict__ kseg,
                         const double *__restrict__ tol, int32_t *__restrict__ its, int32_t maxit,
                         int32_t *__restrict__ nactive, uint8_t *__restrict__ bad) {
  RS_PDL_ENTRY();
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg || !active[s]) return;
  double *Hs = H + (int64_t)s * ldh_seg;
  SegState &S = st[s];
  Hs[(int64_t)(j + 1) * 64 + j] = hnext[s];
  for (int i = 0; i < j; i++) {
    const double a = Hs[(int64_t)i * 64 + j], c = Hs[(int64_t)(i + 1) * 64 + j];
    Hs[(int64_t)i * 64 + j] = S.cs[i] * a + S.sn[i] * c;
    Hs[(int64_t)(i + 1) * 64 + j] = -S.sn[i] * a + S.cs[i] * c;
  }
  const double a = Hs[(int64_t)j * 64 + j], c = Hs[(int64_t)(j + 1) * 64 + j];
  const double d = sqrt(a * a + c * c);
  S.cs[j] = d != 0.0 ? a / d : 1.0;
  S.sn[j] = d != 0.0 ? c / d : 0.0;
  Hs[(int64_t)j * 64 + j] = d;
  Hs[(int64_t)(j + 1) * 64 + j] = 0.0;
  S.g[j + 1] = -S.sn[j] * S.g[j];
  S.g[j] = S.cs[j] * S.g[j];
  kseg[s] = j + 1;
  its[s] += 1;
  const double est = fabs(S.g[j + 1]);
  if (!isfinite(est) || !isfinite(d)) {
    bad[s] = 1;
    active[s] = 0;
    kseg[s] = j;   // drop the failed column
    its[s] -= 1;
    return;
  }
  if (est <= tol[s] || its[s] >= maxit || j + 1 >= m || hnext[s] == 0.0) active[s] = 0;
  else atomicAdd(nactive, 1);
}

// back substitution y = R^{-1} g per system
__global__ void k_backsolve(int32_t nseg, int m, const double *__restrict__ H, int ldh_seg,
                            const SegState *__restrict__ st, const int32_t *__restrict__ kseg, double *__restrict__ y) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const int k = kseg[s];
  const double *Hs = H + (int64_t)s * ldh_seg;
  double *ys = y + (int64_t)s * m;
  for (int i = k - 1; i >= 0; i--) {
    double acc = st[s].g[i];
    for (int t = i + 1; t < k; t++) acc -= Hs[(int64_t)i * 64 + t] * ys[t];
    const double d = Hs[(int64_t)i * 64 + i];
    ys[i] = d != 0.0 ? acc / d : 0.0;
  }
}

__global__ void k_cycle_start(int32_t nseg, const double *__restrict__ beta, const double *__restrict__ tol,
                              const int32_t *__restrict__ its, int32_t maxit, const uint8_t *__restrict__ bad,
                              uint8_t *__restrict__ active, int32_t *__restrict__ kseg, SegState *__restrict__ st) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  const bool go = !bad[s] && beta[s] > tol[s] && its[s] < maxit && isfinite(beta[s]);
  active[s] = go ? 1 : 0;
  kseg[s] = 0;
  st[s].g[0] = go ? beta[s] : 0.0;
}

}  // namespace

extern "C" int gmres_solve(const rs_bsr2 *J, const rs_precond *M, const double *b, double *x,
                           const rs_gmres_params *params, rs_gmres_stats *stats, cudaStream_t s) {
  if (!J || !params || ((!b || !x) && J->nb > 0)) return fail(RS_EINVAL, "null argument");
  if (J->nb < 0 || (J->nb > 0 && (!J->row_ptr || !J->col || !J->val))) return fail(RS_EINVAL, "invalid matrix");
  const int m = params->m;
  if (m < 1 || m > 63) return fail(RS_EINVAL, "restart length must be in [1, 63]");
  if (params->maxit < 0 || !(params->rtol >= 0.0)) return fail(RS_EINVAL, "bad tolerance or iteration limit");
  const std::vector<int32_t> boff = seg_offsets(J->nb, J->nseg, J->seg_off);
  if (boff.front() != 0 || boff.back() != J->nb) return fail(RS_EINVAL, "segment offsets must run from 0 to nb");
  const int32_t nseg = (int32_t)boff.size() - 1;
  const int64_t n = 2 * (int64_t)J->nb;
  if (n == 0) {   // empty system(s): converged with no iterations
    if (stats) {
      stats->iterations = 0;
      stats->converged = nseg;
      stats->relres = 0.0;
      for (int32_t q = 0; q < nseg; q++) {
        if (stats->its) stats->its[q] = 0;
        if (stats->relres_seg) stats->relres_seg[q] = 0.0;
      }
    }
    return RS_OK;
  }
  // chunk table
  const int64_t crows = chunk_rows(n);
  std::vector<Chunk> chunks;
  std::vector<int32_t> seg_chunk(nseg + 1, 0);
  for (int32_t q = 0; q < nseg; q++) {
    seg_chunk[q] = (int32_t)chunks.size();
    for (int64_t r0 = 2 * (int64_t)boff[q]; r0 < 2 * (int64_t)boff[q + 1]; r0 += crows)
      chunks.push_back({q, (int32_t)r0, (int32_t)std::min<int64_t>(r0 + crows, 2 * (int64_t)boff[q + 1])});
  }
  seg_chunk[nseg] = (int32_t)chunks.size();
  const int32_t nch = (int32_t)chunks.size();
  const int stride = 64;
  const int ldh = 65 * 64;
  Scratch sc(s);
  double *V = nullptr, *Z = nullptr, *H = nullptr, *part = nullptr, *hbuf = nullptr, *nrm = nullptr, *y = nullptr,
         *tol = nullptr;
  Chunk *dch = nullptr;
  int32_t *dsegc = nullptr, *kseg = nullptr, *its = nullptr, *nact = nullptr;
  uint8_t *active = nullptr, *bad = nullptr;
  SegState *st = nullptr;
  RS_TRY(sc.get(&V, (size_t)n * (m + 1) + 1));
  RS_TRY(sc.get(&Z, (size_t)n * m + 1));
  RS_TRY(sc.get(&H, (size_t)nseg * ldh));
  RS_TRY(sc.get(&part, (size_t)std::max(nch, 1) * stride));
  RS_TRY(sc.get(&hbuf, (size_t)nseg * stride));
  RS_TRY(sc.get(&nrm, (size_t)nseg));
  RS_TRY(sc.get(&y, (size_t)nseg * m));
  RS_TRY(sc.get(&tol, (size_t)nseg));
  RS_TRY(sc.get(&dch, (size_t)std::max(nch, 1)));
  RS_TRY(sc.get(&dsegc, (size_t)nseg + 1));
  RS_TRY(sc.get(&kseg, (size_t)nseg));
  RS_TRY(sc.get(&its, (size_t)nseg));
  RS_TRY(sc.get(&nact, 2));
  RS_TRY(sc.get(&active, (size_t)nseg));
  RS_TRY(sc.get(&bad, (size_t)nseg));
  RS_TRY(sc.get(&st, (size_t)nseg));
  // batches: the system of every block row, read by the block SpMV to skip
  // the rows of retired systems
  int32_t *brseg = nullptr;
  if (nseg > 1) {
    RS_TRY(seg_ids(boff, J->nb, &brseg, s));
    sc.ptrs.push_back(brseg);
  }
  if (nch > 0) RS_CHECK_CUDA(cudaMemcpyAsync(dch, chunks.data(), sizeof(Chunk) * nch, cudaMemcpyHostToDevice, s));
  RS_CHECK_CUDA(cudaMemcpyAsync(dsegc, seg_chunk.data(), sizeof(int32_t) * (nseg + 1), cudaMemcpyHostToDevice, s));
  RS_CHECK_CUDA(cudaMemsetAsync(its, 0, sizeof(int32_t) * nseg, s));
  RS_CHECK_CUDA(cudaMemsetAsync(bad, 0, (size_t)nseg, s));
  RS_CHECK_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * nseg * ldh, s));
  const unsigned gseg = grid_for(nseg);
  auto norms = [&](const double *vec, double *out) -> int {
    if (nch > 0) RS_COUNTED k_multidot<<<nch, kRedThreads, 0, s>>>(dch, vec, 0, 1, vec, stride, part);
    RS_COUNTED k_reduce<<<grid_for((int64_t)nseg * 32), kBlock, 0, s>>>(nseg, dsegc, 1, stride, part, out, nullptr, 0,
                                                                        0, 3, nullptr);
    RS_CHECK_CUDA(cudaGetLastError());
    return 0;
  };
  // tolerances from ||b||
  RS_TRY(norms(b, nrm));
  std::vector<double> hb(nseg), hbeta(nseg);
  RS_CHECK_CUDA(cudaMemcpyAsync(hb.data(), nrm, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  std::vector<double> htol(nseg);
  for (int32_t q = 0; q < nseg; q++) htol[q] = params->rtol * (hb[q] > 0.0 ? hb[q] : 1.0);
  RS_CHECK_CUDA(cudaMemcpyAsync(tol, htol.data(), sizeof(double) * nseg, cudaMemcpyHostToDevice, s));
  // convergence flags come back through pinned memory one iteration late: the
  // host waits for step j-1's count while step j is already queued, so the GPU
  // does not idle between steps (a step queued after every system stopped
  // changes nothing: stopped systems are frozen)
  static thread_local int32_t *hnact = nullptr;   // pinned, kept for the thread's lifetime
  if (!hnact) RS_CHECK_CUDA(cudaMallocHost(&hnact, 2 * sizeof(int32_t)));
  cudaEvent_t evn[2];
  RS_CHECK_CUDA(cudaEventCreateWithFlags(&evn[0], cudaEventDisableTiming));
  RS_CHECK_CUDA(cudaEventCreateWithFlags(&evn[1], cudaEventDisableTiming));
  std::vector<int32_t> hits(nseg, 0);
  std::vector<uint8_t> hbad(nseg, 0);
  std::vector<double> hprev(nseg, -1.0);
  std::vector<uint8_t> stalled(nseg, 0);
  int rc = RS_OK;
  for (int cycle = 0;; cycle++) {
    // true residual
    rc = launch_bsr2_residual(*J, x, b, V, s);
    if (rc) break;
    rc = norms(V, nrm);
    if (rc) break;
    RS_CHECK_CUDA(cudaMemcpyAsync(hbeta.data(), nrm, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(hits.data(), its, sizeof(int32_t) * nseg, cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(hbad.data(), bad, (size_t)nseg, cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    // a system whose true residual fell by less than 0.1 % over a whole
    // restart cycle (or grew past 1e3 ||b||) has stalled and stops
    bool more = false, newly = false;
    for (int32_t q = 0; q < nseg; q++) {
      if (!stalled[q] && hprev[q] >= 0.0 && hbeta[q] > htol[q] &&
          (hbeta[q] > 0.999 * hprev[q] || hbeta[q] > 1e3 * (hb[q] > 0.0 ? hb[q] : 1.0))) {
        stalled[q] = 1;
        newly = true;
      }
      hprev[q] = hbeta[q];
      if (!stalled[q] && !hbad[q] && std::isfinite(hbeta[q]) && hbeta[q] > htol[q] && hits[q] < params->maxit)
        more = true;
    }
    if (newly)
      for (int32_t q = 0; q < nseg; q++)
        if (stalled[q]) hbad[q] = 2;
    if (newly) RS_CHECK_CUDA(cudaMemcpyAsync(bad, hbad.data(), (size_t)nseg, cudaMemcpyHostToDevice, s));
    if (!more) break;
    RS_COUNTED k_cycle_start<<<gseg, kBlock, 0, s>>>(nseg, nrm, tol, its, params->maxit, bad, active, kseg, st);
    if (nch > 0) RS_COUNTED k_scale<<<nch, kRedThreads, 0, s>>>(dch, nrm, V, V, nullptr);
    for (int j = 0; j < m; j++) {
      double *vj = V + (int64_t)j * n, *zj = Z + (int64_t)j * n, *w = V + (int64_t)(j + 1) * n;
      // retired systems (converged or out of iterations in this cycle) are
      // skipped by the preconditioner's V-cycles
      if (M && nseg > 1) rc = precond_set_active(M, active, s);
      if (M && !rc) rc = precond_apply_impl(M, vj, zj, s);
      else RS_CHECK_CUDA(cudaMemcpyAsync(zj, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      if (rc) break;
      rc = launch_bsr2_spmv(*J, zj, w, s, brseg ? active : nullptr, brseg);
      if (rc) break;
      // CGS2: dots, reduce, (update + second dots), reduce, (update + norm)
      const double nv = j + 1;
      if (nch > 0) {
        ProfScope ps(kProfArnoldi, (nv + 1) * 8.0 * n, s);
        RS_COUNTED launch_pdl(k_arnoldi<0>, dim3(nch), dim3(kRedThreads), 0, s, (const Chunk *)dch, (const double *)V,
                              (int64_t)n, j + 1, (const double *)nullptr, stride, w, part, (const uint8_t *)active);
      }
      RS_COUNTED launch_pdl(k_reduce, dim3(grid_for((int64_t)nseg * (j + 1) * 32)), dim3(kBlock), 0, s, nseg,
                            (const int32_t *)dsegc, j + 1, stride, (const double *)part, hbuf, H, ldh, j, 1,
                            (const uint8_t *)active);
      if (nch > 0) {
        ProfScope ps(kProfArnoldi, (2.0 * nv + 2) * 8.0 * n, s);
        RS_COUNTED launch_pdl(k_arnoldi<1>, dim3(nch), dim3(kRedThreads), 0, s, (const Chunk *)dch, (const double *)V,
                              (int64_t)n, j + 1, (const double *)hbuf, stride, w, part, (const uint8_t *)active);
      }
      RS_COUNTED launch_pdl(k_reduce, dim3(grid_for((int64_t)nseg * (j + 1) * 32)), dim3(kBlock), 0, s, nseg,
                            (const int32_t *)dsegc, j + 1, stride, (const double *)part, hbuf, H, ldh, j, 2,
                            (const uint8_t *)active);
      if (nch > 0) {
        ProfScope ps(kProfArnoldi, (nv + 2) * 8.0 * n, s);
        RS_COUNTED launch_pdl(k_arnoldi<2>, dim3(nch), dim3(kRedThreads), 0, s, (const Chunk *)dch, (const double *)V,
                              (int64_t)n, j + 1, (const double *)hbuf, stride, w, part, (const uint8_t *)active);
      }
      RS_COUNTED launch_pdl(k_reduce, dim3(grid_for((int64_t)nseg * 32)), dim3(kBlock), 0, s, nseg,
                            (const int32_t *)dsegc, 1, stride, (const double *)part, nrm, (double *)nullptr, 0, 0, 3,
                            (const uint8_t *)active);   // retired systems: norm 0, so their next basis vector is 0
      const int slot = j & 1;
      RS_COUNTED launch_pdl(k_scale, dim3(nch), dim3(kRedThreads), 0, s, (const Chunk *)dch, (const double *)nrm,
                            (const double *)w, w, nact + slot);
      RS_COUNTED launch_pdl(k_givens, dim3(gseg), dim3(kBlock), 0, s, nseg, j, m, H, ldh, (const double *)nrm, st,
                            active, kseg, (const double *)tol, its, params->maxit, nact + slot, bad);
      RS_CHECK_CUDA(cudaMemcpyAsync(hnact + slot, nact + slot, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      RS_CHECK_CUDA(cudaEventRecord(evn[slot], s));
      if (j >= 1) {
        RS_CHECK_CUDA(cudaEventSynchronize(evn[slot ^ 1]));
        if (hnact[slot ^ 1] == 0) break;
      }
    }
    if (rc) break;
    RS_COUNTED k_backsolve<<<gseg, kBlock, 0, s>>>(nseg, m, H, ldh, st, kseg, y);
    if (nch > 0) RS_COUNTED k_xupdate<<<nch, kRedThreads, 0, s>>>(dch, Z, n, y, m, kseg, x);
    RS_CHECK_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * nseg * ldh, s));
    RS_CHECK_CUDA(cudaGetLastError());
  }
  cudaEventDestroy(evn[0]);
  cudaEventDestroy(evn[1]);
  if (rc) return rc;
  int32_t conv = 0, itmax = 0;
  double rmax = 0.0;
  for (int32_t q = 0; q < nseg; q++) {
    const double bn = hb[q] > 0.0 ? hb[q] : 1.0;
    const double rr = hbeta[q] / bn;
    if (hbad[q] != 1 && rr <= params->rtol) conv++;
    if (!(rr <= rmax)) rmax = rr;
    itmax = std::max(itmax, hits[q]);
    if (stats && stats->its) stats->its[q] = hits[q];
    if (stats && stats->relres_seg) stats->relres_seg[q] = rr;
  }
  if (stats) {
    stats->iterations = itmax;
    stats->converged = conv;
    stats->relres = rmax;
  }
  // a smoother CTA that gave up waiting for its staging copies left rows
  // unswept: the statistics above describe the work done, the call fails
  rc = vcycle_wait_status(s);
  if (rc) return rc;
  return conv == nseg ? RS_OK : RS_NOT_CONVERGED;
}
