// On-device classical AMG setup (Sec. 3.2; solver settings of Sec. 4), FP64,
// compiled without fused multiply-add so that every floating-point decision
// (strength threshold, interpolation weights feeding the next level's
// strength) matches the CPU check bit for bit.
//
//  strength   : with s_i = sign of a_ii (+1 for 0), j != i is strong for i iff
//               -s_i a_ij >= theta * max_{k != i}(-s_i a_ik) and that max > 0;
//               with num_functions > 1 on the finest level only couplings
//               between unknowns of the same kind (i mod nf == j mod nf) count.
//  coarsening : PMIS (De Sterck, Yang, Heys 2006) in place of the paper's
//               CLJP. key_i = (|S^T_i| << 24) | (SplitMix64 bits >> 40); i
//               beats j iff key_i > key_j or (equal and i < j). Points nobody
//               depends on start as F. Each round an undecided point beating
//               all undecided neighbours in S u S^T becomes C, then undecided
//               points strongly depending on a C point become F.
//  random bits: SplitMix64 (Steele, Lea, Flood 2014), c-th output for seed s =
//               mix(s + (c+1) 0x9E3779B97F4A7C15); counter ((2l) << 32) + i
//               for PMIS and ((2l+1) << 32) + i for colouring, i the row's
//               index within its own system, so a batch member coarsens
//               exactly as it would alone.
//  interp.    : extended+i (De Sterck, Falgout, Nolting, Yang 2008) or classical
//               Ruge-Stueben; see k_interp_ext / k_interp_classical.
//  Galerkin   : A_c = P^T (A P) by the ordered sparse products.
//  colouring  : Jones-Plassmann on the symmetrised pattern, lowest free colour.
//  stopping   : per system: at or below coarse_n rows, at max_levels, or when
//               a coarsening keeps more than 0.9 n (or no) points; that system
//               is then solved there by a dense FP64 inverse.
#include <algorithm>

#include "rs_internal.cuh"

namespace rs {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool beats(uint64_t ki, int32_t i, uint64_t kj, int32_t j) {
  return ki > kj || (ki == kj && i < j);
}

// Row-wise kernels below take G lanes per row (G = 8, 16 or 32 from the mean
// row length, row_lanes): consecutive lanes read consecutive entries of the
// row, so a group's loads are contiguous; the grid covers n * G threads in
// whole warps.
static int row_lanes(int64_t n, int64_t nnz) {
  const double avg = n > 0 ? (double)nnz / (double)n : 1.0;
  return avg <= 10.0 ? 8 : (avg <= 24.0 ? 16 : 32);
}
#define RS_ROWG_SWITCH(g, ...)                                   \
  switch (g) {                                                   \
    case 8: { constexpr int G_ = 8; __VA_ARGS__; } break;        \
    case 16: { constexpr int G_ = 16; __VA_ARGS__; } break;      \
    default: { constexpr int G_ = 32; __VA_ARGS__; } break;      \
  }

// this thread's group's bits of a warp ballot
template <int G>
__device__ __forceinline__ unsigned group_bits(unsigned ballot) {
  if constexpr (G == 32) return ballot;
  else return (ballot >> ((threadIdx.x & 31) & ~(G - 1))) & ((1u << G) - 1u);
}

template <int G>
__global__ void k_diag(int32_t n, const int32_t *rp, const int32_t *col, const double *val, double *d) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid / G;
  const int gl = (int)(gid % G);
  double v = 0.0;
  bool f = false;
  if (i < n)
    for (int32_t k = rp[i] + gl; k < rp[i + 1]; k += G)
      if (col[k] == i) { v = val[k]; f = true; }
  // the lane holding the diagonal (columns of a row are distinct)
  const unsigned m = group_bits<G>(__ballot_sync(0xffffffffu, f));
  const int base = (threadIdx.x & 31) & ~(G - 1);
  const double dv = __shfl_sync(0xffffffffu, v, m ? base + __ffs(m) - 1 : base);
  if (i < n && gl == 0) d[i] = m ? dv : 0.0;
}

// rows of systems that do not coarsen at this level get no strong entries
template <int G>
__global__ void k_strength(int32_t n, const int32_t *rp, const int32_t *col, const double *val, const double *diag,
                           const int32_t *seg, const uint8_t *seg_act, double theta, int32_t nfun,
                           uint8_t *strong) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i64 = gid / G;
  const int gl = (int)(gid % G);
  const bool ok = i64 < n;
  const int32_t i = ok ? (int32_t)i64 : 0;
  int32_t s = 0, e = 0;
  bool act = false;
  double sg = 1.0;
  if (ok) {
    s = rp[i];
    e = rp[i + 1];
    act = seg_act[seg[i]] != 0;
    sg = diag[i] < 0.0 ? -1.0 : 1.0;
  }
  double mx = 0.0;
  if (act)
    for (int32_t k = s + gl; k < e; k += G) {
      const int32_t j = col[k];
      if (j == i || (j % nfun) != (i % nfun)) continue;
      const double v = -(sg * val[k]);
      if (v > mx) mx = v;
    }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, mx, o, G);
    if (w > mx) mx = w;
  }
  if (!ok) return;
  const double thr = theta * mx;
  for (int32_t k = s + gl; k < e; k += G) {
    uint8_t st = 0;
    if (act) {
      const int32_t j = col[k];
      if (j != i && (j % nfun) == (i % nfun) && mx > 0.0) st = (-(sg * val[k]) >= thr) ? 1 : 0;
    }
    strong[k] = st;
  }
}

template <int G>
__global__ void k_lambda(int32_t n, const int32_t *rp, const int32_t *col, const uint8_t *strong, int32_t *lam) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid / G;
  if (i >= n) return;
  for (int32_t k = rp[i] + (int)(gid % G); k < rp[i + 1]; k += G)
    if (strong[k]) atomicAdd(&lam[col[k]], 1);
}

// cf: 0 undecided, 1 C, -1 F
__global__ void k_pmis_init(int32_t n, const int32_t *lam, const int32_t *seg, const int32_t *seg_off,
                            const uint8_t *seg_act, uint64_t seed, int32_t level, uint64_t *key, int8_t *cf) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t sg = seg[i];
  const uint64_t local = (uint64_t)(i - seg_off[sg]);
  const uint64_t r = splitmix64(seed, ((uint64_t)(2 * level) << 32) + local);
  key[i] = ((uint64_t)lam[i] << 24) | (r >> 40);
  cf[i] = (seg_act[sg] && lam[i] > 0) ? 0 : -1;
}

// every strong edge between two undecided points marks its loser
template <int G>
__global__ void k_pmis_losers(int32_t n, const int32_t *rp, const int32_t *col, const uint8_t *strong,
                              const uint64_t *key, const int8_t *cf, uint8_t *notmax) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j64 = gid / G;
  if (j64 >= n) return;
  const int32_t j = (int32_t)j64;
  if (cf[j] != 0) return;
  const uint64_t kj = key[j];
  for (int32_t q = rp[j] + (int)(gid % G); q < rp[j + 1]; q += G) {
    if (!strong[q]) continue;
    const int32_t k = col[q];
    if (cf[k] != 0) continue;
    if (beats(kj, j, key[k], k)) notmax[k] = 1;
    else notmax[j] = 1;
  }
}

// (also clears the marks it read, so the next round starts clean)
__global__ void k_pmis_select(int32_t n, uint8_t *notmax, int8_t *cf) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] != 0) return;
  if (!notmax[i]) cf[i] = 1;
  notmax[i] = 0;
}

// undecided points strongly depending on a C point become F; count the rest
// (one atomic per warp)
template <int G>
__global__ void k_pmis_fmark(int32_t n, const int32_t *rp, const int32_t *col, const uint8_t *strong, int8_t *cf,
                             int32_t *left) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j64 = gid / G;
  const int gl = (int)(gid % G);
  const int32_t j = j64 < n ? (int32_t)j64 : 0;
  const bool und = j64 < n && cf[j] == 0;
  bool hit = false;
  if (und)
    for (int32_t q = rp[j] + gl; q < rp[j + 1]; q += G)
      if (strong[q] && cf[col[q]] == 1) { hit = true; break; }
  const bool anyhit = group_bits<G>(__ballot_sync(0xffffffffu, hit)) != 0;
  if (und && gl == 0 && anyhit) cf[j] = -1;
  const unsigned rest = __ballot_sync(0xffffffffu, und && gl == 0 && !anyhit);
  if ((threadIdx.x & 31) == 0 && rest) atomicAdd(left, __popc(rest));
}

// (one atomic per distinct system of a warp)
__global__ void k_seg_count_c(int32_t n, const int8_t *cf, const int32_t *seg, int32_t *cnt) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool c = i < n && cf[i] == 1;
  const unsigned act = __ballot_sync(0xffffffffu, c);
  if (!c) return;
  const unsigned same = __match_any_sync(act, seg[i]);
  if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&cnt[seg[i]], __popc(same));
}

// systems that stop here lose their C points; C flags for the numbering
__global__ void k_seg_revert(int32_t n, int8_t *cf, const int32_t *seg, const uint8_t *seg_act, int32_t *isc) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!seg_act[seg[i]]) cf[i] = -1;
  isc[i] = cf[i] == 1 ? 1 : 0;
}

__global__ void k_gather_offsets(int32_t m, const int32_t *at, const int32_t *v, int32_t *out) {
  int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < m) out[q] = v[at[q]];
}

// ------------------------------------------------------------------ interpolation
constexpr int kMaxChat = 96;

__device__ __forceinline__ int find_sorted(const int32_t *a, int m, int32_t v) {
  int lo = 0, hi = m - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int32_t x = a[mid];
    if (x == v) return mid;
    if (x < v) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ bool insert_sorted(int32_t *a, int &m, int32_t v) {
  int p = m;
  while (p > 0 && a[p - 1] > v) p--;
  if (p > 0 && a[p - 1] == v) return true;
  if (m >= kMaxChat) return false;
  for (int q = m; q > p; q--) a[q] = a[q - 1];
  a[p] = v;
  m++;
  return true;
}

struct Acc {
  double v;
  bool set;
  __device__ __forceinline__ void add(double x) {
    if (!set) { v = x; set = true; } else v = v + x;
  }
};

// Extended+i weights for F row i (see the CPU check for the same wording):
//   Chat_i = strong C neighbours of i and of its strong F neighbours;
//   pass A over row i (ascending): a_ii, weak a_ij outside Chat_i, and strong F
//   a_ik with d_k = 0 go to dtil; a_ij with j in Chat_i start num_j;
//   pass B over the strong F neighbours k (ascending) with d_k != 0:
//   t = a_ik / d_k, then over row k (ascending, opposite sign to a_kk only)
//   t * a_kl goes to num_l (l in Chat_i) or dtil (l = i);
//   w_ij = -(num_j / dtil) for the num_j that were set; dtil = 0: empty row.
// WRITE = false returns the row length only.
template <bool WRITE>
__global__ void k_interp_ext(int32_t n, const int32_t *rp, const int32_t *col, const double *val, const double *diag,
                             const uint8_t *strong, const int8_t *cf, const int32_t *cidx, int32_t *prp,
                             int32_t *pcol, double *pval, int32_t *err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] == 1) {
    if (WRITE) { pcol[prp[i]] = cidx[i]; pval[prp[i]] = 1.0; }
    else prp[i] = 1;
    return;
  }
  int32_t chat[kMaxChat];
  double num[kMaxChat];
  bool nset[kMaxChat];
  int m = 0;
  bool ok = true;
  const int32_t s = rp[i], e = rp[i + 1];
  for (int32_t q = s; q < e && ok; q++) {
    const int32_t j = col[q];
    if (j == i || !strong[q]) continue;
    if (cf[j] == 1) ok = insert_sorted(chat, m, j);
    else
      for (int32_t t = rp[j]; t < rp[j + 1] && ok; t++) {
        const int32_t l = col[t];
        if (l != j && strong[t] && cf[l] == 1) ok = insert_sorted(chat, m, l);
      }
  }
  if (!ok) { atomicExch(err, 1); if (!WRITE) prp[i] = 0; return; }
  if (m == 0) { if (!WRITE) prp[i] = 0; return; }
  for (int q = 0; q < m; q++) { nset[q] = false; num[q] = 0.0; }
  Acc dt{0.0, false};
  // pass A
  for (int32_t q = s; q < e; q++) {
    const int32_t j = col[q];
    const double a = val[q];
    if (j == i) { dt.add(a); continue; }
    const int mj = find_sorted(chat, m, j);
    if (mj >= 0) { num[mj] = a; nset[mj] = true; continue; }
    if (strong[q] && cf[j] != 1) {
      const double sk = diag[j] < 0.0 ? -1.0 : 1.0;
      Acc d{0.0, false};
      for (int32_t t = rp[j]; t < rp[j + 1]; t++) {
        const int32_t l = col[t];
        if (l == j || !(l == i || find_sorted(chat, m, l) >= 0)) continue;
        const double av = val[t];
        if (!(sk * av < 0.0)) continue;
        d.add(av);
      }
      if (d.v == 0.0) dt.add(a);
      continue;
    }
    dt.add(a);
  }
  // pass B
  for (int32_t q = s; q < e; q++) {
    const int32_t k = col[q];
    if (k == i || !strong[q] || cf[k] == 1) continue;
    const double sk = diag[k] < 0.0 ? -1.0 : 1.0;
    Acc d{0.0, false};
    for (int32_t t = rp[k]; t < rp[k + 1]; t++) {
      const int32_t l = col[t];
      if (l == k || !(l == i || find_sorted(chat, m, l) >= 0)) continue;
      const double av = val[t];
      if (!(sk * av < 0.0)) continue;
      d.add(av);
    }
    if (d.v == 0.0) continue;
    const double tq = val[q] / d.v;
    for (int32_t t = rp[k]; t < rp[k + 1]; t++) {
      const int32_t l = col[t];
      if (l == k) continue;
      const int ml = l == i ? -2 : find_sorted(chat, m, l);
      if (ml == -1) continue;
      const double av = val[t];
      if (!(sk * av < 0.0)) continue;
      const double pr = tq * av;
      if (ml == -2) dt.add(pr);
      else if (!nset[ml]) { num[ml] = pr; nset[ml] = true; }
      else num[ml] = num[ml] + pr;
    }
  }
  int32_t cnt = 0;
  const int32_t base = WRITE ? prp[i] : 0;
  if (dt.v != 0.0) {
    for (int q = 0; q < m; q++) {
      if (!nset[q]) continue;
      if (WRITE) { pcol[base + cnt] = cidx[chat[q]]; pval[base + cnt] = -(num[q] / dt.v); }
      cnt++;
    }
  }
  if (!WRITE) prp[i] = cnt;
}

// Warp-per-row form of the extended+i weights above (same sets, same sums in
// the same order, so the same bits): the lanes share the work that has no
// ordering constraint (gathering Chat_i, the denominators d_k, one lane per
// k, and the numerators, one lane per target column j, each summing over k
// ascending), while the single ordered accumulation of dtil is done by lane 0.
constexpr int kICand = 2048;
constexpr int kICap = 256;
constexpr int kIF = 256;

// Per-warp work arrays of the interpolation kernels, carved from dynamic
// shared memory with capacities sized for the level (ccap candidates, hcap
// interpolation points, fcap strong F neighbours; at most kICand, kICap,
// kIF): small capacities on the fine levels let many warps share an SM.
struct IWarp {
  double *num, *fa, *fd;
  int32_t *hkey, *chat, *nset, *fk, *fb, *fe, *fneg, *cnt;   // hkey: candidate hash set; cnt: -, m, nf
  int16_t *hidx;   // per hash slot: the key's position in the sorted Chat_i
};

__host__ __device__ inline size_t iwarp_bytes(int ccap, int hcap, int fcap) {
  return 8 * (size_t)(hcap + 2 * fcap) + 4 * (size_t)(ccap + 2 * hcap + 4 * fcap + 4) + 2 * (size_t)ccap;
}

__device__ inline IWarp iwarp_at(unsigned char *base, int ccap, int hcap, int fcap) {
  IWarp W;
  W.num = reinterpret_cast<double *>(base);
  W.fa = W.num + hcap;
  W.fd = W.fa + fcap;
  W.hkey = reinterpret_cast<int32_t *>(W.fd + fcap);
  W.chat = W.hkey + ccap;
  W.nset = W.chat + hcap;
  W.fk = W.nset + hcap;
  W.fb = W.fk + fcap;
  W.fe = W.fb + fcap;
  W.fneg = W.fe + fcap;
  W.cnt = W.fneg + fcap;
  W.hidx = reinterpret_cast<int16_t *>(W.cnt + 4);
  return W;
}

// Position of `key` in the sorted Chat_i through the row's hash set (-1: not
// a member).
__device__ __forceinline__ int32_t hfind(const IWarp &W, int tbits, int32_t key) {
  const int size = 1 << tbits;
  int h = (int)(((uint32_t)key * 2654435761u) >> (32 - tbits));
  for (int p = 0; p < size; p++) {
    const int32_t k = W.hkey[h];
    if (k == key) return W.hidx[h];
    if (k < 0) return -1;
    h = (h + 1) & (size - 1);
  }
  return -1;
}

// Sign tests on the bit pattern (integer instructions; GB300 issues FP64
// comparisons on its slow FP64 pipe): v < 0, v > 0 (false for +-0 and NaN),
// and v == +-0.
__device__ __forceinline__ bool dneg(double v) {
  const long long b = __double_as_longlong(v), a = b & 0x7fffffffffffffffLL;
  return b < 0 && a != 0 && a <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dpos(double v) {
  const long long b = __double_as_longlong(v);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dzero(double v) { return (__double_as_longlong(v) & 0x7fffffffffffffffLL) == 0; }
// a_kl has the sign opposite to a_kk (a_kk < 0: a_kl > 0; else a_kl < 0)
__device__ __forceinline__ bool dopposite(int neg_kk, double akl) { return neg_kk ? dpos(akl) : dneg(akl); }

// Inserts key into the warp's open-addressing set of 2^tbits slots (-1 =
// empty), counting new keys in *distinct; false when the set is full.
__device__ __forceinline__ bool hset_insert(int32_t *keys, int tbits, int32_t key, int32_t *distinct) {
  const int size = 1 << tbits;
  int h = (int)(((uint32_t)key * 2654435761u) >> (32 - tbits));
  for (int probes = 0; probes < size; probes++) {
    const int32_t prev = atomicCAS(&keys[h], -1, key);
    if (prev == -1) {
      atomicAdd(distinct, 1);
      return true;
    }
    if (prev == key) return true;
    h = (h + 1) & (size - 1);
  }
  return false;
}

// Sorts a[0..m) ascending, one warp; a has room for the next power of two
// of m (cap, a power of two). Up to 32 values: bitonic network in registers;
// more: bitonic network in place over the padded array.
__device__ void warp_sort_asc(int32_t *a, int32_t m, int32_t cap) {
  const int lane = threadIdx.x & 31;
  if (m <= 1) return;
  if (m <= 32) {
    int32_t v = lane < m ? a[lane] : INT32_MAX;
    for (int k = 2; k <= 32; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        v = (lower == up) ? min(v, o) : max(v, o);
      }
    __syncwarp();
    if (lane < m) a[lane] = v;
    __syncwarp();
    return;
  }
  int32_t P = 64;
  while (P < m) P <<= 1;
  if (P > cap) P = cap;   // (m <= cap, and cap is a power of two)
  for (int32_t t = m + lane; t < P; t += 32) a[t] = INT32_MAX;
  __syncwarp();
  for (int32_t k = 2; k <= P; k <<= 1)
    for (int32_t j = k >> 1; j > 0; j >>= 1) {
      for (int32_t t = lane; t < P / 2; t += 32) {
        const int32_t i = (t / j) * 2 * j + (t % j), q = i + j;
        const bool up = (i & k) == 0;
        const int32_t x = a[i], y = a[q];
        if ((x > y) == up) { a[i] = y; a[q] = x; }
      }
      __syncwarp();
    }
}

// bounds of a level for the interpolation capacities: the largest number of
// entries of a row plus its neighbours' rows (bounds the candidate count),
// and the largest row
// (the maxima reduced over the warp first: one atomic per warp)
__global__ void k_interp_bounds(int32_t n, const int32_t *rp, const int32_t *col, int32_t *mx) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t c = 0, len = 0;
  if (i < n) {
    len = rp[i + 1] - rp[i];
    c = len;
    for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
      const int32_t j = col[q];
      c += rp[j + 1] - rp[j];
    }
  }
  c = __reduce_max_sync(0xffffffffu, c);
  len = __reduce_max_sync(0xffffffffu, len);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx, c);
    atomicMax(mx + 1, len);
  }
}

__device__ __forceinline__ int find_row(const int32_t *col, int32_t s, int32_t e, int32_t v) {
  int32_t lo = s, hi = e - 1;
  while (lo <= hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t x = col[mid];
    if (x == v) return mid;
    if (x < v) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Room for row i of P: 1 for a C row; for an F row its candidate count with
// repeats (1 per strong C neighbour, the length of each strong F neighbour's
// row), which bounds |Chat_i|, capped at Chat's capacity hcap. The total is
// summed in 64 bits (one atomic per warp).
__global__ void k_interp_cap(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const uint8_t *__restrict__ strong, const int8_t *__restrict__ cf, int32_t hcap,
                             int32_t *__restrict__ cap, unsigned long long *captot) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t c = 0;
  if (i < n) {
    if (cf[i] == 1) {
      c = 1;
    } else {
      int64_t b = 0;
      for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
        const int32_t j = col[q];
        if (j != i && strong[q]) b += cf[j] == 1 ? 1 : rp[j + 1] - rp[j];
      }
      c = (int32_t)(b < hcap ? b : hcap);
    }
    cap[i] = c;
  }
  const unsigned ws = __reduce_add_sync(0xffffffffu, (unsigned)c);
  if ((threadIdx.x & 31) == 0 && ws) atomicAdd(captot, (unsigned long long)ws);
}

// SIZE = true: prp[i] = the size of Chat_i (1 for a C row), an upper bound
// of row i's entries. SIZE = false: row i's entries at pcol/pval + prp[i]
// (offsets of the sizes) and their number in cnt[i].
template <bool SIZE>
__global__ void __launch_bounds__(256) k_interp_ext_w(int32_t n, int ccap, int hcap, int fcap,
                                                     const int32_t *__restrict__ rp,
                                                     const int32_t *__restrict__ col,
                                                     const double *__restrict__ val,
                                                     const double *__restrict__ diag,
                                                     const uint8_t *__restrict__ strong,
                                                     const int8_t *__restrict__ cf,
                                                     const int32_t *__restrict__ cidx, int32_t *prp,
                                                     int32_t *__restrict__ pcol, double *__restrict__ pval,
                                                     int32_t *__restrict__ cnt, int32_t *err,
                                                     const int32_t *__restrict__ rlist, int32_t nlist,
                                                     uint8_t *__restrict__ big, int32_t *__restrict__ defer) {
  extern __shared__ __align__(16) unsigned char iwsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const IWarp W = iwarp_at(iwsm + (size_t)warp * iwarp_bytes(ccap, hcap, fcap), ccap, hcap, fcap);
  const unsigned lt = (1u << lane) - 1u;
  // rows: all n, or the listed ones; the rows a small-workspace size pass
  // deferred (big[i] = 1) are left to the pass over their list
  const int32_t nrow = rlist ? nlist : n;
  const bool skip_big = !SIZE && big != nullptr && rlist == nullptr;
  for (int32_t idx = blockIdx.x * nwarps + warp; idx < nrow; idx += gridDim.x * nwarps) {
    const int32_t i = rlist ? rlist[idx] : idx;
    if (skip_big && big[i]) continue;
    if (cf[i] == 1) {
      if (lane == 0) {
        if (SIZE) prp[i] = 1;
        else { pcol[prp[i]] = cidx[i]; pval[prp[i]] = 1.0; cnt[i] = 1; }
      }
      continue;
    }
    const int32_t s = rp[i], e = rp[i + 1];
    // this row's hash set: a power of two at least twice its number of
    // candidate entries (with repeats), within the level's capacity
    int32_t bnd = 0;
    for (int32_t q = s + lane; q < e; q += 32) {
      const int32_t j = col[q];
      if (j != i && strong[q]) bnd += cf[j] == 1 ? 1 : rp[j + 1] - rp[j];
    }
    bnd = __reduce_add_sync(0xffffffffu, bnd);
    int tbits = 5;
    while ((1 << tbits) < ccap && (1 << tbits) < 2 * bnd) tbits++;
    for (int h = lane; h < (1 << tbits); h += 32) W.hkey[h] = -1;
    if (lane == 0) { W.cnt[1] = 0; W.cnt[2] = 0; }
    __syncwarp();
    // candidates for Chat_i (strong C neighbours of i and of its strong F
    // neighbours) into the set, and the strong F neighbours in row order
    bool ovf = false;
    for (int32_t b0 = s; b0 < e; b0 += 32) {
      const int32_t q = b0 + lane;
      int32_t j = -1;
      bool st = false;
      if (q < e) { j = col[q]; st = j != i && strong[q]; }
      const bool isC = st && cf[j] == 1;
      const bool isF = st && cf[j] != 1;
      if (isC && !hset_insert(W.hkey, tbits, j, &W.cnt[1])) ovf = true;
      if (isF) {
        for (int32_t t = rp[j]; t < rp[j + 1]; t++) {
          const int32_t l = col[t];
          if (l != j && strong[t] && cf[l] == 1 && !hset_insert(W.hkey, tbits, l, &W.cnt[1])) ovf = true;
        }
      }
      const unsigned fm = __ballot_sync(0xffffffffu, isF);
      const int32_t nf0 = W.cnt[2];
      __syncwarp();
      if (isF) {
        const int32_t p = nf0 + __popc(fm & lt);
        if (p < fcap) { W.fk[p] = j; W.fa[p] = val[q]; } else ovf = true;
      }
      __syncwarp();
      if (lane == 0) W.cnt[2] = nf0 + __popc(fm);
      __syncwarp();
    }
    const int32_t m = W.cnt[1], nf = W.cnt[2];
    ovf = __any_sync(0xffffffffu, ovf) || m > hcap || nf > fcap;
    if (SIZE) {
      if (lane == 0) {
        if (ovf && defer) {        // too large for this workspace: defer the row
          big[i] = 1;
          defer[1 + atomicAdd(&defer[0], 1)] = i;
          prp[i] = 0;
        } else {
          if (ovf) atomicExch(err, 1);
          prp[i] = ovf ? 0 : m;
        }
      }
      __syncwarp();
      continue;
    }
    // Chat_i: the distinct candidates in ascending order
    if (!ovf) {
      int32_t base = 0;
      for (int32_t h0 = 0; h0 < (1 << tbits); h0 += 32) {
        const int32_t v = W.hkey[h0 + lane];
        const unsigned occ = __ballot_sync(0xffffffffu, v >= 0);
        if (v >= 0) W.chat[base + __popc(occ & lt)] = v;
        base += __popc(occ);
      }
      __syncwarp();
      warp_sort_asc(W.chat, m, hcap);
      // map each hash slot to its key's position in Chat_i
      for (int32_t idx = lane; idx < m; idx += 32) {
        const int32_t key = W.chat[idx];
        int h = (int)(((uint32_t)key * 2654435761u) >> (32 - tbits));
        while (W.hkey[h] != key) h = (h + 1) & ((1 << tbits) - 1);
        W.hidx[h] = (int16_t)idx;
      }
    }
    __syncwarp();
    if (ovf) {
      if (lane == 0) {
        if (defer) defer[1 + atomicAdd(&defer[0], 1)] = i;   // for the full workspace
        else atomicExch(err, 1);
        cnt[i] = 0;
      }
      continue;
    }
    if (m == 0) {
      if (lane == 0) cnt[i] = 0;
      continue;
    }
    // denominators d_k = sum over row k (ascending) of entries in Chat_i + {i}
    // whose sign is opposite to a_kk; one lane per k
    // (each k's row bounds and diagonal sign are kept for the passes below,
    // and fa becomes t_k = a_ik / d_k, divided once per k)
    for (int32_t f = lane; f < nf; f += 32) {
      const int32_t k = W.fk[f];
      const int neg = dneg(diag[k]) ? 1 : 0;
      const int32_t kb = rp[k], ke = rp[k + 1];
      Acc d{0.0, false};
      for (int32_t t = kb; t < ke; t++) {
        const int32_t l = col[t];
        if (l == k || !(l == i || hfind(W, tbits, l) >= 0)) continue;
        const double av = val[t];
        if (!dopposite(neg, av)) continue;
        d.add(av);
      }
      W.fd[f] = d.v;
      W.fa[f] = dzero(d.v) ? 0.0 : W.fa[f] / d.v;
      W.fb[f] = kb;
      W.fe[f] = ke;
      W.fneg[f] = neg;
    }
    __syncwarp();
    // numerators, scattered: a_ij first (from row i), then t_k * abar_kj for
    // the k in ascending order, each k's row spread over the lanes (a row
    // holds each target at most once, so no two lanes add to one target in a
    // pass, and every target's terms arrive in the order of a sequential sum)
    for (int32_t idx = lane; idx < m; idx += 32) {
      W.num[idx] = 0.0;
      W.nset[idx] = 0;
    }
    __syncwarp();
    for (int32_t q = s + lane; q < e; q += 32) {
      const int32_t x = hfind(W, tbits, col[q]);
      if (x >= 0) {
        W.num[x] = val[q];
        W.nset[x] = 1;
      }
    }
    __syncwarp();
    for (int32_t f = 0; f < nf; f++) {
      if (dzero(W.fd[f])) continue;
      const double tq = W.fa[f];
      const int neg = W.fneg[f];
      const int32_t ke = W.fe[f];
      for (int32_t q = W.fb[f] + lane; q < ke; q += 32) {
        const int32_t x = hfind(W, tbits, col[q]);
        if (x < 0) continue;
        const double av = val[q];
        if (!dopposite(neg, av)) continue;
        const double t = tq * av;
        W.num[x] = W.nset[x] ? W.num[x] + t : t;
        W.nset[x] = 1;
      }
      __syncwarp();
    }
    // dtil: pass A over row i, then the "+i" terms of the k (ascending). The
    // lanes look up the terms of 32 entries at a time; lane 0 adds them in
    // row order (the order, and so the rounding, of a sequential sum).
    Acc a{0.0, false};
    {
      int32_t fbase = 0;   // strong F entries of row i before this chunk
      for (int32_t b0 = s; b0 < e; b0 += 32) {
        const int32_t q = b0 + lane;
        bool has = false, isF = false;
        double v = 0.0;
        if (q < e) {
          const int32_t j = col[q];
          v = val[q];
          if (j == i) has = true;
          else if (hfind(W, tbits, j) < 0) {
            isF = strong[q] && cf[j] != 1;
            has = !isF;
          }
        }
        const unsigned fm = __ballot_sync(0xffffffffu, isF);
        if (isF) has = dzero(W.fd[fbase + __popc(fm & lt)]);
        fbase += __popc(fm);
        // (only the lanes holding a term: one FP64 add per term)
        for (unsigned hm = __ballot_sync(0xffffffffu, has); hm; hm &= hm - 1u) {
          const double vt = __shfl_sync(0xffffffffu, v, __ffs(hm) - 1);
          if (lane == 0) a.add(vt);
        }
      }
      for (int32_t g0 = 0; g0 < nf; g0 += 32) {
        const int32_t g = g0 + lane;
        bool has = false;
        double term = 0.0;
        if (g < nf && !dzero(W.fd[g])) {
          const int32_t qk = find_row(col, W.fb[g], W.fe[g], i);
          if (qk >= 0) {
            const double av = val[qk];
            if (dopposite(W.fneg[g], av)) {
              term = W.fa[g] * av;
              has = true;
            }
          }
        }
        for (unsigned hm = __ballot_sync(0xffffffffu, has); hm; hm &= hm - 1u) {
          const double vt = __shfl_sync(0xffffffffu, term, __ffs(hm) - 1);
          if (lane == 0) a.add(vt);
        }
      }
    }
    double dt = a.v;
    dt = __shfl_sync(0xffffffffu, dt, 0);
    __syncwarp();
    // output the set entries in Chat order
    int32_t base = 0;
    for (int32_t b0 = 0; b0 < m; b0 += 32) {
      const int32_t idx = b0 + lane;
      const bool on = idx < m && W.nset[idx] && dt != 0.0;
      const unsigned om = __ballot_sync(0xffffffffu, on);
      if (on) {
        const int32_t p = prp[i] + base + __popc(om & lt);
        pcol[p] = cidx[W.chat[idx]];
        pval[p] = -(W.num[idx] / dt);
      }
      base += __popc(om);
    }
    if (lane == 0) cnt[i] = base;
    __syncwarp();
  }
}

// Classical Ruge-Stueben weights (C_i = strong C neighbours, distribution of
// strong F neighbours m through C_i with entries of sign opposite to a_mm; a
// strong F neighbour sharing no such entry, and weak neighbours, go to the
// diagonal). Same accumulation order rules as above.
template <bool WRITE>
__global__ void k_interp_classical(int32_t n, const int32_t *rp, const int32_t *col, const double *val,
                                   const double *diag, const uint8_t *strong, const int8_t *cf,
                                   const int32_t *cidx, int32_t *prp, int32_t *pcol, double *pval, int32_t *err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] == 1) {
    if (WRITE) { pcol[prp[i]] = cidx[i]; pval[prp[i]] = 1.0; }
    else prp[i] = 1;
    return;
  }
  int32_t ci[kMaxChat];
  double num[kMaxChat];
  int m = 0;
  const int32_t s = rp[i], e = rp[i + 1];
  for (int32_t q = s; q < e; q++)
    if (strong[q] && col[q] != i && cf[col[q]] == 1) {
      if (m >= kMaxChat) { atomicExch(err, 1); if (!WRITE) prp[i] = 0; return; }
      ci[m++] = col[q];
    }
  if (m == 0) { if (!WRITE) prp[i] = 0; return; }
  Acc dt{0.0, false};
  for (int32_t q = s; q < e; q++) {
    const int32_t j = col[q];
    const double a = val[q];
    if (j == i || !strong[q]) { dt.add(a); continue; }
    if (cf[j] == 1) { num[find_sorted(ci, m, j)] = a; continue; }
    const double sm = diag[j] < 0.0 ? -1.0 : 1.0;
    Acc d{0.0, false};
    for (int32_t t = rp[j]; t < rp[j + 1]; t++) {
      const int32_t kk = col[t];
      if (kk == j || find_sorted(ci, m, kk) < 0) continue;
      const double av = val[t];
      if (!(sm * av < 0.0)) continue;
      d.add(av);
    }
    if (d.v == 0.0) dt.add(a);
  }
  for (int32_t q = s; q < e; q++) {
    const int32_t mm = col[q];
    if (mm == i || !strong[q] || cf[mm] == 1) continue;
    const double sm = diag[mm] < 0.0 ? -1.0 : 1.0;
    Acc d{0.0, false};
    for (int32_t t = rp[mm]; t < rp[mm + 1]; t++) {
      const int32_t kk = col[t];
      if (kk == mm || find_sorted(ci, m, kk) < 0) continue;
      const double av = val[t];
      if (!(sm * av < 0.0)) continue;
      d.add(av);
    }
    if (d.v == 0.0) continue;
    const double tq = val[q] / d.v;
    for (int32_t t = rp[mm]; t < rp[mm + 1]; t++) {
      const int32_t kk = col[t];
      if (kk == mm) continue;
      const int mk = find_sorted(ci, m, kk);
      if (mk < 0) continue;
      const double av = val[t];
      if (!(sm * av < 0.0)) continue;
      num[mk] = num[mk] + tq * av;
    }
  }
  if (dt.v == 0.0) { if (!WRITE) prp[i] = 0; return; }
  if (WRITE)
    for (int q = 0; q < m; q++) { pcol[prp[i] + q] = cidx[ci[q]]; pval[prp[i] + q] = -(num[q] / dt.v); }
  else prp[i] = m;
}

// ------------------------------------------------------------------ colouring
constexpr int kColourWords = 4;   // up to 256 colours

__global__ void k_jp_init(int32_t n, const int32_t *seg, const int32_t *seg_off, const uint8_t *seg_smooth,
                          uint64_t seed, int32_t level, uint64_t *key, int32_t *colour) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t sg = seg[i];
  key[i] = splitmix64(seed, ((uint64_t)(2 * level + 1) << 32) + (uint64_t)(i - seg_off[sg]));
  colour[i] = seg_smooth[sg] ? -1 : -2;     // -2: not coloured at this level
}

__global__ void k_jp_losers(int32_t n, const int32_t *rp, const int32_t *col, const uint64_t *key,
                            const int32_t *colour, uint8_t *notmax) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || colour[j] != -1) return;
  const uint64_t kj = key[j];
  for (int32_t q = rp[j]; q < rp[j + 1]; q++) {
    const int32_t k = col[q];
    if (k == j || colour[k] != -1) continue;
    if (beats(kj, j, key[k], k)) notmax[k] = 1;
    else notmax[j] = 1;
  }
}

// forbidden colours of the selected points, from coloured neighbours in both directions
__global__ void k_jp_forbid(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *colour,
                            const uint8_t *notmax, unsigned long long *mask) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int32_t cj = colour[j];
  const bool sel_j = cj == -1 && !notmax[j];
  for (int32_t q = rp[j]; q < rp[j + 1]; q++) {
    const int32_t k = col[q];
    if (k == j) continue;
    const int32_t ck = colour[k];
    if (sel_j && ck >= 0) atomicOr(&mask[(int64_t)j * kColourWords + (ck >> 6)], 1ull << (ck & 63));
    if (cj >= 0 && ck == -1 && !notmax[k]) atomicOr(&mask[(int64_t)k * kColourWords + (cj >> 6)], 1ull << (cj & 63));
  }
}

// (also clears the marks and masks it read, so the next round starts clean)
__global__ void k_jp_assign(int32_t n, uint8_t *notmax, unsigned long long *mask, int32_t *colour,
                            int32_t *left, int32_t *maxc, int32_t *err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || colour[i] != -1) return;
  if (notmax[i]) { notmax[i] = 0; atomicAdd(left, 1); return; }
  int c = -1;
  for (int w = 0; w < kColourWords; w++) {
    const unsigned long long fm = ~mask[(int64_t)i * kColourWords + w];
    if (fm && c < 0) c = 64 * w + __ffsll((long long)fm) - 1;
    mask[(int64_t)i * kColourWords + w] = 0ull;
  }
  if (c < 0) { atomicExch(err, 1); c = 0; }
  colour[i] = c;
  atomicMax(maxc, c + 1);
}

__global__ void k_colour_count(int32_t n, const int32_t *colour, int32_t *cnt) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && colour[i] >= 0) atomicAdd(&cnt[colour[i]], 1);
}

__global__ void k_colour_fill(int32_t n, const int32_t *colour, int32_t *fill, int32_t *rows) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && colour[i] >= 0) rows[atomicAdd(&fill[colour[i]], 1)] = i;
}

// Colouring for the hybrid smoother, one CTA per chunk (rows [cr[2k],
// cr[2k+1]), at most 512): rows are coloured first-fit in ascending order,
// each taking the lowest colour (< 128) not used by an already coloured row
// of the chunk coupled to it in either direction. The chunk's coupling graph
// is built as a bit matrix in shared memory; warp 0 then walks the rows, the
// lanes OR-ing the colours of the coloured neighbours found in their words.
constexpr int kCCMax = 512;
constexpr int kCCWords = kCCMax / 32;

// B unknowns per point (B = 1: rows are the points): the graph and the
// colours are those of the chunk's points, and every unknown of a point gets
// the point's colour.
template <int B>
__global__ void __launch_bounds__(256) k_chunk_colour(const int32_t *cr, const int32_t *rp, const int32_t *col,
                                                      int32_t *colour, int32_t *maxc, int32_t *err) {
  __shared__ uint32_t adj[kCCMax * kCCWords];
  __shared__ int32_t cs[kCCMax];
  const int32_t k = blockIdx.x;
  const int32_t r0 = cr[2 * k], nrow = cr[2 * k + 1] - r0, len = nrow / B;
  if (len > kCCMax) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  for (int32_t t = threadIdx.x; t < len * kCCWords; t += blockDim.x) adj[t] = 0u;
  __syncthreads();
  for (int32_t lr = threadIdx.x; lr < nrow; lr += blockDim.x) {
    const int32_t i = r0 + lr, li = lr / B;
    for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
      const int32_t lc = col[q] - r0;
      if (lc < 0 || lc >= nrow) continue;
      const int32_t lj = lc / B;
      if (lj == li) continue;
      atomicOr(&adj[li * kCCWords + (lj >> 5)], 1u << (lj & 31));
      atomicOr(&adj[lj * kCCWords + (li >> 5)], 1u << (li & 31));
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // greedy in point order, one warp: lane w gathers the colours of the
    // earlier neighbours in adjacency word w, the warp ORs them together,
    // and every lane takes the lowest free colour
    const int lane = threadIdx.x;
    int32_t localmax = 0;
    for (int32_t li = 0; li < len; li++) {
      unsigned long long u0 = 0ull, u1 = 0ull;
      const int32_t wl = li >> 5;
      if (lane < kCCWords && lane <= wl) {
        uint32_t w = adj[li * kCCWords + lane];
        if (lane == wl) w &= (li & 31) ? ((1u << (li & 31)) - 1u) : 0u;
        while (w) {
          const int b = __ffs(w) - 1;
          w &= w - 1u;
          const int32_t c = cs[lane * 32 + b];
          if (c < 64) u0 |= 1ull << c; else u1 |= 1ull << (c - 64);
        }
      }
      const unsigned m0 = __reduce_or_sync(0xffffffffu, (unsigned)u0);
      const unsigned m1 = __reduce_or_sync(0xffffffffu, (unsigned)(u0 >> 32));
      const unsigned m2 = __reduce_or_sync(0xffffffffu, (unsigned)u1);
      const unsigned m3 = __reduce_or_sync(0xffffffffu, (unsigned)(u1 >> 32));
      int32_t c;
      if (~m0) c = __ffs(~m0) - 1;
      else if (~m1) c = 32 + __ffs(~m1) - 1;
      else if (~m2) c = 64 + __ffs(~m2) - 1;
      else if (~m3) c = 96 + __ffs(~m3) - 1;
      else { c = 0; if (lane == 0) atomicExch(err, 2); }
      if (lane == 0) cs[li] = c;
      if (c + 1 > localmax) localmax = c + 1;
      __syncwarp();
    }
    if (lane == 0) atomicMax(maxc, localmax);
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < nrow; t += blockDim.x) colour[r0 + t] = cs[t / B];
}

__global__ void k_chunk_nnz_max(int32_t nchunk, const int32_t *cr, const int32_t *rp, int32_t *mx) {
  int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nchunk) atomicMax(mx, rp[cr[2 * k + 1]] - rp[cr[2 * k]]);
}

__global__ void k_fill_colour(int32_t n, int32_t *c) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = -2;
}

// Hybrid smoother tables: for chunk k (rows [cr[2k], cr[2k+1])), the local rows
// sorted by (colour, row) and the offset of each colour inside the chunk.
// With B unknowns per point the entries are the chunk's local points, stored
// from position r0 / B.
template <int B>
__global__ void k_chunk_sort(const int32_t *cr, const int32_t *colour, int32_t ncol, int32_t *coff,
                             int32_t *rows) {
  __shared__ int32_t cs[1024];
  const int32_t k = blockIdx.x;
  const int32_t r0 = cr[2 * k], len = (cr[2 * k + 1] - r0) / B;
  for (int32_t t = threadIdx.x; t < len; t += blockDim.x) cs[t] = colour[r0 + B * t];
  __syncthreads();
  for (int32_t c = threadIdx.x; c <= ncol; c += blockDim.x) {
    int32_t cnt = 0;
    for (int32_t t = 0; t < len; t++) cnt += cs[t] < c;
    coff[(int64_t)k * (ncol + 1) + c] = cnt;
  }
  for (int32_t t = threadIdx.x; t < len; t += blockDim.x) {
    const int32_t c = cs[t];
    int32_t rank = 0;
    for (int32_t q = 0; q < len; q++) rank += (cs[q] < c) || (cs[q] == c && q < t);
    rows[r0 / B + rank] = t;
  }
}

// inverse diagonal (GS) or inverse l1 row weight (Jacobi), FP64 and FP32
__global__ void k_smoother_diag(int32_t n, const int32_t *rp, const int32_t *col, const double *val, int32_t l1,
                                double *dinv, float *dinvf, int32_t *range_err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0, off = 0.0;
  for (int32_t k = rp[i]; k < rp[i + 1]; k++) {
    if (col[k] == i) d = val[k];
    else off += fabs(val[k]);
  }
  if (l1) d = d < 0.0 ? d - off : d + off;
  const double inv = d != 0.0 ? 1.0 / d : 0.0;
  dinv[i] = inv;
  dinvf[i] = (float)inv;
  if (range_err && isinf(dinvf[i]) && isfinite(inv)) atomicOr(range_err, 1);
}

// ---- systems (point) AMG: B interleaved unknowns per point, row B*i + f
// function f of point i (Sec. 3.2, the point method)
// rows B*i + f and columns B*j + f of A as an N x N matrix
__global__ void k_func_count(int32_t N, int32_t B, int32_t f, const int32_t *rp, const int32_t *col,
                             int32_t *cnt) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int32_t c = 0;
  for (int32_t q = rp[B * i + f]; q < rp[B * i + f + 1]; q++) c += col[q] % B == f;
  cnt[i] = c;
}

__global__ void k_func_fill(int32_t N, int32_t B, int32_t f, const int32_t *rp, const int32_t *col,
                            const double *val, const int32_t *orp, int32_t *ocol, double *oval) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int32_t pos = orp[i];
  for (int32_t q = rp[B * i + f]; q < rp[B * i + f + 1]; q++)
    if (col[q] % B == f) {
      ocol[pos] = col[q] / B;
      oval[pos++] = val[q];
    }
}

// interleaved interpolation: row B*i + f is row i of Pf with column c -> B*c + f
__global__ void k_ileave_count(int32_t N, int32_t B, int32_t f, const int32_t *prp, int32_t *cnt) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) cnt[B * i + f] = prp[i + 1] - prp[i];
}

__global__ void k_ileave_fill(int32_t N, int32_t B, int32_t f, const int32_t *prp, const int32_t *pcol,
                              const double *pval, const int32_t *orp, int32_t *ocol, double *oval) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int32_t pos = orp[B * i + f];
  for (int32_t q = prp[i]; q < prp[i + 1]; q++) {
    ocol[pos] = B * pcol[q] + f;
    oval[pos++] = pval[q];
  }
}

__global__ void k_cf_expand(int32_t N, int32_t B, const int8_t *cfp, int8_t *cf) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N)
    for (int32_t f = 0; f < B; f++) cf[B * i + f] = cfp[i];
}

// inverses of the 2 x 2 diagonal blocks of the points (row-major, FP64 and an
// FP32 copy); a singular block gets zeros (that point is left unchanged)
__global__ void k_block_inv2(int32_t N, const int32_t *rp, const int32_t *col, const double *val, double *inv,
                             float *invf, int32_t *range_err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double d[4] = {0.0, 0.0, 0.0, 0.0};
  for (int32_t f = 0; f < 2; f++)
    for (int32_t q = rp[2 * i + f]; q < rp[2 * i + f + 1]; q++)
      if (col[q] / 2 == i) d[2 * f + col[q] % 2] = val[q];
  const double det = d[0] * d[3] - d[1] * d[2];
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  if (det != 0.0) {
    m[0] = d[3] / det;
    m[1] = -d[1] / det;
    m[2] = -d[2] / det;
    m[3] = d[0] / det;
  }
  for (int q = 0; q < 4; q++) {
    inv[4 * (int64_t)i + q] = m[q];
    invf[4 * (int64_t)i + q] = (float)m[q];
    if (range_err && isinf((float)m[q]) && isfinite(m[q])) atomicOr(range_err, 1);
  }
}

static int func_part(const DCsr &A, int32_t B, int32_t f, DCsr &out, cudaStream_t s) {
  const int32_t N = A.n / B;
  out.n = N;
  out.m = A.m / B;
  RS_TRY(dalloc_n(&out.rowptr, (size_t)N + 1, s));
  if (N > 0) RS_COUNTED k_func_count<<<grid_for(N), kBlock, 0, s>>>(N, B, f, A.rowptr, A.col, out.rowptr);
  int32_t nnz = 0;
  RS_TRY(exclusive_scan(out.rowptr, out.rowptr, N, s, &nnz));
  out.nnz = nnz;
  RS_TRY(dalloc_n(&out.col, (size_t)nnz + 1, s));
  RS_TRY(dalloc_n(&out.val, (size_t)nnz + 1, s));
  if (N > 0)
    RS_COUNTED k_func_fill<<<grid_for(N), kBlock, 0, s>>>(N, B, f, A.rowptr, A.col, A.val, out.rowptr, out.col,
                                                          out.val);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// FP32 copy; a finite value beyond the FP32 range sets *range_err
__global__ void k_to_f32(int64_t n, const double *a, float *b, int32_t *range_err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = (float)a[i];
  b[i] = f;
  if (isinf(f) && isfinite(a[i])) atomicOr(range_err, 1);
}

// Hybrid smoother operator. For every row of a chunk: its off-diagonal
// entries coupling to rows of the same chunk (column stored as the position
// inside the chunk), then those coupling to other rows (global column), each
// part in ascending column order; the diagonal is left out (the smoother
// uses its inverse). hs_mid[i] is where row i's second part begins.
// With B unknowns per point the whole diagonal block of the row's point is
// left out (the point-block smoother uses its inverse).
// G lanes per row (rows of a chunk in a loop of the CTA; the lanes of a
// group stay together, groups of one warp may part at a chunk's end).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) return 0xffffffffu;
  else return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

template <int B, int G>
__global__ void k_hs_count(const int32_t *cr, const int32_t *rp, const int32_t *col, int32_t *cnt) {
  const int32_t k = blockIdx.x;
  const int32_t r0 = cr[2 * k], r1 = cr[2 * k + 1];
  const int gl = threadIdx.x % G;
  const unsigned gm = group_mask<G>();
  for (int32_t i = r0 + (int32_t)(threadIdx.x / G); i < r1; i += blockDim.x / G) {
    int32_t c = 0;
    for (int32_t q = rp[i] + gl; q < rp[i + 1]; q += G) c += col[q] / B != i / B;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) c += __shfl_xor_sync(gm, c, o, G);
    if (gl == 0) cnt[i] = c;
  }
}

// Each row's in-chunk entries (less its point's own block), then its
// out-of-chunk entries, each part in the row's order: a group's lanes take G
// entries at a time and place the kept ones by their rank among the kept.
template <typename T, int B, int G>
__global__ void k_hs_fill(const int32_t *cr, const int32_t *rp, const int32_t *col, const double *val,
                          const int32_t *hrp, int32_t *hmid, int32_t *hcol, T *hval) {
  const int32_t k = blockIdx.x;
  const int32_t r0 = cr[2 * k], r1 = cr[2 * k + 1];
  const int gl = threadIdx.x % G;
  const unsigned gm = group_mask<G>();
  const unsigned below = (1u << gl) - 1u;
  for (int32_t i = r0 + (int32_t)(threadIdx.x / G); i < r1; i += blockDim.x / G) {
    int32_t pos = hrp[i];
    const int32_t qs = rp[i], qe = rp[i + 1];
    for (int pass = 0; pass < 2; pass++) {
      for (int32_t q0 = qs; q0 < qe; q0 += G) {
        const int32_t q = q0 + gl;
        int32_t j = 0;
        bool keep = false;
        if (q < qe) {
          j = col[q];
          const bool inside = j >= r0 && j < r1;
          keep = pass == 0 ? (inside && j / B != i / B) : !inside;
        }
        const unsigned m = group_bits<G>(__ballot_sync(gm, keep));
        if (keep) {
          const int32_t p = pos + __popc(m & below);
          hcol[p] = pass == 0 ? j - r0 : j;
          hval[p] = (T)val[q];
        }
        pos += __popc(m);
      }
      if (pass == 0 && gl == 0) hmid[i] = pos;
    }
  }
}

// ------------------------------------------------------------------ coarse inverse
// Gauss-Jordan with partial pivoting (largest |a|, first on ties), one CTA per
// system, dense FP64 in global scratch: [A | I] -> [I | A^{-1}].
template <bool SMEM>
__global__ void k_coarse_dense(const int32_t *rp, const int32_t *col, const double *val, const int4 *info,
                               const int64_t *inv_off, double *work, double *inv) {
  extern __shared__ __align__(16) unsigned char cdsm[];
  const int4 in = info[blockIdx.x];
  const int32_t r0 = in.x, n = in.y;
  const int64_t off = inv_off[blockIdx.x];
  // n x n matrix followed by the n x n identity, row-major each, in shared
  // memory when they fit, else in the global work area
  double *a = SMEM ? reinterpret_cast<double *>(cdsm) : work + 2 * off;
  double *b = a + (int64_t)n * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int64_t t = threadIdx.x; t < 2 * (int64_t)n * n; t += blockDim.x) a[t] = 0.0;
  __syncthreads();
  for (int32_t r = threadIdx.x; r < n; r += blockDim.x) {
    for (int32_t k = rp[r0 + r]; k < rp[r0 + r + 1]; k++) {
      const int32_t c = col[k] - r0;
      if (c >= 0 && c < n) a[(int64_t)r * n + c] = val[k];
    }
    b[(int64_t)r * n + r] = 1.0;
  }
  __syncthreads();
  __shared__ int32_t piv;
  __shared__ double red_v[32];
  __shared__ int32_t red_i[32];
  for (int32_t k = 0; k < n; k++) {
    // pivot search: largest |a_rk| for r >= k, lowest row on ties (block-wide argmax)
    double best = -1.0;
    int32_t bi = n;
    for (int32_t r = k + threadIdx.x; r < n; r += blockDim.x) {
      const double v = fabs(a[(int64_t)r * n + k]);
      if (v > best || (v == best && r < bi)) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int32_t oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bv = -1.0;
      int32_t bix = n;
      for (int t = 0; t < nwarps; t++)
        if (red_v[t] > bv || (red_v[t] == bv && red_i[t] < bix)) { bv = red_v[t]; bix = red_i[t]; }
      piv = bix < n ? bix : k;
    }
    __syncthreads();
    const int32_t p = piv;
    if (p != k)
      for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
        double t = a[(int64_t)k * n + c]; a[(int64_t)k * n + c] = a[(int64_t)p * n + c]; a[(int64_t)p * n + c] = t;
        t = b[(int64_t)k * n + c]; b[(int64_t)k * n + c] = b[(int64_t)p * n + c]; b[(int64_t)p * n + c] = t;
      }
    __syncthreads();
    const double d = a[(int64_t)k * n + k];
    const double dinv = d != 0.0 ? 1.0 / d : 0.0;
    __syncthreads();
    for (int32_t c = threadIdx.x; c < n; c += blockDim.x) {
      a[(int64_t)k * n + c] *= dinv;
      b[(int64_t)k * n + c] *= dinv;
    }
    __syncthreads();
    // eliminate column k from every other row: a warp per row, lanes over columns
    for (int32_t r = warp; r < n; r += nwarps) {
      if (r == k) continue;
      const double f = a[(int64_t)r * n + k];
      if (f == 0.0) continue;
      for (int32_t c = lane; c < n; c += 32) {
        if (c != k) a[(int64_t)r * n + c] -= f * a[(int64_t)k * n + c];
        b[(int64_t)r * n + c] -= f * b[(int64_t)k * n + c];
      }
    }
    __syncthreads();
    for (int32_t r = threadIdx.x; r < n; r += blockDim.x)
      if (r != k) a[(int64_t)r * n + k] = 0.0;
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) inv[off + t] = b[t];
}

// largest coarse system staged in shared memory (2 n^2 doubles <= 96 KB)
constexpr int kCoarseSmemN = 78;

// ------------------------------------------------------------------ driver
static int sync_copy(void *h, const void *d, size_t bytes, cudaStream_t s) {
  RS_CHECK_CUDA(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  return 0;
}

template <typename T>
static int upload(T **d, const std::vector<T> &h, cudaStream_t s) {
  RS_TRY(dalloc_n(d, h.size() + 1, s));
  if (!h.empty()) RS_CHECK_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return 0;
}

static int colour_level(Level &L, const int32_t *seg, const int32_t *dseg_off, const std::vector<uint8_t> &smooth_seg,
                        uint64_t seed, int32_t level, cudaStream_t s) {
  const int32_t n = L.A.n;
  const int32_t nseg = (int32_t)smooth_seg.size();
  Scratch sc(s);
  uint64_t *key = nullptr;
  uint8_t *notmax = nullptr, *dsm = nullptr;
  unsigned long long *mask = nullptr;
  int32_t *cnt3 = nullptr;   // left, maxc, err
  RS_TRY(sc.get(&key, (size_t)n));
  RS_TRY(sc.get(&notmax, (size_t)n));
  RS_TRY(sc.get(&mask, (size_t)n * kColourWords));
  RS_TRY(sc.get(&cnt3, 3));
  RS_TRY(dalloc_n(&L.colour, (size_t)n, s));
  std::vector<uint8_t> sm(smooth_seg);
  RS_TRY(sc.get(&dsm, (size_t)nseg));
  RS_CHECK_CUDA(cudaMemcpyAsync(dsm, sm.data(), nseg, cudaMemcpyHostToDevice, s));
  RS_CHECK_CUDA(cudaMemsetAsync(cnt3, 0, 3 * sizeof(int32_t), s));
  RS_CHECK_CUDA(cudaMemsetAsync(notmax, 0, (size_t)n, s));
  RS_CHECK_CUDA(cudaMemsetAsync(mask, 0, sizeof(unsigned long long) * (size_t)n * kColourWords, s));
  RS_COUNTED k_jp_init<<<grid_for(n), kBlock, 0, s>>>(n, seg, dseg_off, dsm, seed, level, key, L.colour);
  int32_t h3[3] = {1, 0, 0};
  // rounds run in batches between host checks; a round with nothing left to
  // colour changes nothing
  for (int round = 0; round < 100000 && h3[0] > 0; round += 6) {
    for (int r = 0; r < 6; r++) {
      RS_CHECK_CUDA(cudaMemsetAsync(cnt3, 0, sizeof(int32_t), s));
      RS_COUNTED k_jp_losers<<<grid_for(n), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, key, L.colour, notmax);
      RS_COUNTED k_jp_forbid<<<grid_for(n), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, L.colour, notmax, mask);
      RS_COUNTED k_jp_assign<<<grid_for(n), kBlock, 0, s>>>(n, notmax, mask, L.colour, cnt3, cnt3 + 1, cnt3 + 2);
    }
    RS_TRY(sync_copy(h3, cnt3, sizeof(h3), s));
    if (h3[2]) return fail(RS_ESETUP, "more than 256 colours needed on level " + std::to_string(level));
  }
  const int32_t nc = h3[1];
  L.ncolour = nc;
  int32_t *ccnt = nullptr;
  RS_TRY(sc.get(&ccnt, (size_t)nc + 1));
  RS_CHECK_CUDA(cudaMemsetAsync(ccnt, 0, sizeof(int32_t) * ((size_t)nc + 1), s));
  if (n > 0) RS_COUNTED k_colour_count<<<grid_for(n), kBlock, 0, s>>>(n, L.colour, ccnt);
  RS_TRY(exclusive_scan(ccnt, ccnt, nc, s, &L.nsmooth));
  L.colour_off.resize(nc + 1);
  RS_TRY(sync_copy(L.colour_off.data(), ccnt, sizeof(int32_t) * (nc + 1), s));
  RS_TRY(dalloc_n(&L.colour_rows, (size_t)L.nsmooth, s));
  int32_t *fill = nullptr;
  RS_TRY(sc.get(&fill, (size_t)nc + 1));
  RS_CHECK_CUDA(cudaMemcpyAsync(fill, ccnt, sizeof(int32_t) * (nc + 1), cudaMemcpyDeviceToDevice, s));
  if (n > 0) RS_COUNTED k_colour_fill<<<grid_for(n), kBlock, 0, s>>>(n, L.colour, fill, L.colour_rows);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

static void level_free(Level &L, cudaStream_t s);

// fine C/F marks after two coarsening stages: C iff C in both (the first
// stage's C points, in order, are the second stage's rows)
__global__ void k_cf_merge(int32_t n, const int8_t *__restrict__ cf0, const int32_t *__restrict__ cidx,
                           const int8_t *__restrict__ cf1, int8_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cf0[i] == 1 ? cf1[cidx[i]] : (int8_t)-1;
}

__global__ void k_is_c(int32_t n, const int8_t *__restrict__ cf, int32_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cf[i] == 1;
}

// ------------------------------------------------------------------ approximate ideal restriction
// AIR (Manteuffel, Southworth et al., "Nonsymmetric algebraic multigrid based
// on local approximate ideal restriction", 2018), distance 1: row r of R, for
// the r-th C point i, is 1 at i and -z on N_i, the F points coupled to i in
// row i (ascending, each once), with A(N_i, N_i)^T z = A(i, N_i)^T, so that
// (R A)(i, N_i) = 0. With a strength array (one flag per entry of A) N_i
// keeps only the strong couplings: the localised form lAIR (Manteuffel,
// Muenzenmaier, Ruge, Southworth 2019), whose coarse operators stay as
// sparse as Galerkin's on transport-dominated levels. The local system is solved by LU with partial pivoting
// (largest magnitude, the first one on ties; a zero pivot leaves its column
// uneliminated and its solution component zero) in the operation order of a
// plain sequential elimination, which this unit, compiled without FMA
// contraction, reproduces bit for bit.

// Per C point: its row length |N_i| + 1 in R, its fine index, and the
// largest |N_i|.
__global__ void k_air_count(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int8_t *__restrict__ cf, const uint8_t *__restrict__ strong,
                            const int32_t *__restrict__ cidx, int32_t *__restrict__ rlen,
                            int32_t *__restrict__ cpt, int32_t *__restrict__ mmax) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] != 1) return;
  int32_t m = 0;
  for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
    const int32_t j = col[q];
    if (j == i || cf[j] == 1 || (strong && !strong[q])) continue;
    bool dup = false;
    for (int32_t q2 = rp[i]; q2 < q && !dup; q2++) dup = col[q2] == j && (!strong || strong[q2]);
    if (!dup) m++;
  }
  const int32_t r = cidx[i];
  rlen[r] = m + 1;
  cpt[r] = i;
  atomicMax(mmax, m);
}

// Position of j in the ascending list nb (element a at nb[a * T]), or -1.
__device__ __forceinline__ int32_t air_find(const int32_t *nb, size_t T, int32_t m, int32_t j) {
  int32_t lo = 0, hi = m - 1;
  while (lo <= hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t v = nb[(size_t)mid * T];
    if (v == j) return mid;
    if (v < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// T threads, each working through rows t, t + T, ... with its own slice of
// the work arrays, interleaved across threads (element e of thread t at
// e * T + t): the local matrix (mx^2), the right-hand side / solution (mx),
// N_i and the pivots (mx each).
__global__ void __launch_bounds__(128) k_air_fill(int32_t nc, int32_t T, int32_t mx, const int32_t *__restrict__ rp,
                                                  const int32_t *__restrict__ col, const double *__restrict__ val,
                                                  const int8_t *__restrict__ cf, const uint8_t *__restrict__ strong,
                                                  const int32_t *__restrict__ cpt,
                                                  const int32_t *__restrict__ rrp, double *__restrict__ ws,
                                                  int32_t *__restrict__ wi, int32_t *__restrict__ rcol,
                                                  double *__restrict__ rval) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const size_t S = (size_t)T;
  double *M = ws + t;
  double *x = ws + (size_t)mx * mx * S + t;
  int32_t *nb = wi + t;
  int32_t *piv = wi + (size_t)mx * S + t;
  for (int32_t r = t; r < nc; r += T) {
    const int32_t i = cpt[r];
    // N_i by insertion into an ascending list
    int32_t m = 0;
    for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
      const int32_t j = col[q];
      if (j == i || cf[j] == 1 || (strong && !strong[q])) continue;
      int32_t a = m;
      while (a > 0 && nb[(size_t)(a - 1) * S] > j) a--;
      if (a > 0 && nb[(size_t)(a - 1) * S] == j) continue;
      if (m >= mx) break;   // cannot happen: mx is the largest count
      for (int32_t b = m; b > a; b--) nb[(size_t)b * S] = nb[(size_t)(b - 1) * S];
      nb[(size_t)a * S] = j;
      m++;
    }
    // M = A(N_i, N_i)^T (row b of A(N_i, .) fills column b), x = A(i, N_i)^T
    for (int32_t e = 0; e < m * m; e++) M[(size_t)e * S] = 0.0;
    for (int32_t a = 0; a < m; a++) x[(size_t)a * S] = 0.0;
    for (int32_t b = 0; b < m; b++) {
      const int32_t k = nb[(size_t)b * S];
      for (int32_t q = rp[k]; q < rp[k + 1]; q++) {
        const int32_t a = air_find(nb, S, m, col[q]);
        if (a >= 0) M[(size_t)(a * m + b) * S] = val[q];
      }
    }
    for (int32_t q = rp[i]; q < rp[i + 1]; q++) {
      const int32_t a = air_find(nb, S, m, col[q]);
      if (a >= 0) x[(size_t)a * S] = val[q];
    }
    // LU with partial pivoting, in place
    for (int32_t k = 0; k < m; k++) {
      int32_t p = k;
      double big = fabs(M[(size_t)(k * m + k) * S]);
      for (int32_t a = k + 1; a < m; a++) {
        const double v = fabs(M[(size_t)(a * m + k) * S]);
        if (v > big) { big = v; p = a; }
      }
      piv[(size_t)k * S] = p;
      if (p != k)
        for (int32_t b = 0; b < m; b++) {
          const double tmp = M[(size_t)(k * m + b) * S];
          M[(size_t)(k * m + b) * S] = M[(size_t)(p * m + b) * S];
          M[(size_t)(p * m + b) * S] = tmp;
        }
      const double d = M[(size_t)(k * m + k) * S];
      if (d == 0.0) continue;
      for (int32_t a = k + 1; a < m; a++) {
        const double l = M[(size_t)(a * m + k) * S] / d;
        M[(size_t)(a * m + k) * S] = l;
        for (int32_t b = k + 1; b < m; b++) M[(size_t)(a * m + b) * S] -= l * M[(size_t)(k * m + b) * S];
      }
    }
    // solve: row interchanges, forward (unit L), backward (U)
    for (int32_t k = 0; k < m; k++) {
      const int32_t p = piv[(size_t)k * S];
      if (p != k) {
        const double tmp = x[(size_t)k * S];
        x[(size_t)k * S] = x[(size_t)p * S];
        x[(size_t)p * S] = tmp;
      }
    }
    for (int32_t a = 0; a < m; a++) {
      double v = x[(size_t)a * S];
      for (int32_t b = 0; b < a; b++) v -= M[(size_t)(a * m + b) * S] * x[(size_t)b * S];
      x[(size_t)a * S] = v;
    }
    for (int32_t a = m - 1; a >= 0; a--) {
      double v = x[(size_t)a * S];
      for (int32_t b = a + 1; b < m; b++) v -= M[(size_t)(a * m + b) * S] * x[(size_t)b * S];
      const double d = M[(size_t)(a * m + a) * S];
      x[(size_t)a * S] = d != 0.0 ? v / d : 0.0;
    }
    // the row: 1 at i, -z on N_i, ascending columns
    int32_t o = rrp[r];
    bool placed = false;
    for (int32_t a = 0; a < m; a++) {
      const int32_t j = nb[(size_t)a * S];
      if (!placed && i < j) { rcol[o] = i; rval[o] = 1.0; o++; placed = true; }
      rcol[o] = j;
      rval[o] = -x[(size_t)a * S];
      o++;
    }
    if (!placed) { rcol[o] = i; rval[o] = 1.0; }
  }
}

// R (nc x n) of level matrix A by approximate ideal restriction, for the marks
// cf (1 C) and the C index cidx of every C point; nc C points in all; strong
// (nullptr: every coupling) limits the neighbourhoods to strong couplings.
static int air_restriction(const DCsr &A, const int8_t *cf, const int32_t *cidx, int32_t nc, const uint8_t *strong,
                           DCsr &R, cudaStream_t s) {
  const int32_t n = A.n;
  R.n = nc;
  R.m = n;
  RS_TRY(dalloc_n(&R.rowptr, (size_t)nc + 1, s));
  Scratch sc(s);
  int32_t *cpt = nullptr, *mmax = nullptr;
  RS_TRY(sc.get(&cpt, (size_t)nc + 1));
  RS_TRY(sc.get(&mmax, 1));
  RS_CHECK_CUDA(cudaMemsetAsync(mmax, 0, sizeof(int32_t), s));
  RS_CHECK_CUDA(cudaMemsetAsync(R.rowptr, 0, sizeof(int32_t) * ((size_t)nc + 1), s));
  if (n > 0) RS_COUNTED k_air_count<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cf, strong, cidx, R.rowptr, cpt,
                                                                mmax);
  int32_t nnz = 0, mx = 0;
  RS_TRY(exclusive_scan(R.rowptr, R.rowptr, nc, s, &nnz));
  RS_TRY(sync_copy(&mx, mmax, sizeof(int32_t), s));
  if (mx > 4096) return fail(RS_ESETUP, "AIR neighbourhood of more than 4096 points");
  R.nnz = nnz;
  RS_TRY(dalloc_n(&R.col, (size_t)nnz + 1, s));
  RS_TRY(dalloc_n(&R.val, (size_t)nnz + 1, s));
  if (nc == 0) return 0;
  // threads bounded by a 256 MB work area
  const size_t per = ((size_t)mx * mx + mx) * sizeof(double) + 2 * (size_t)mx * sizeof(int32_t);
  size_t T = (size_t)num_sms() * 256;
  if (per > 0) T = std::min(T, std::max<size_t>(1, ((size_t)256 << 20) / per));
  T = std::min(T, (size_t)nc);
  double *ws = nullptr;
  int32_t *wi = nullptr;
  RS_TRY(sc.get(&ws, ((size_t)mx * mx + mx) * T + 1));
  RS_TRY(sc.get(&wi, 2 * (size_t)mx * T + 1));
  RS_COUNTED k_air_fill<<<(unsigned)((T + 127) / 128), 128, 0, s>>>(nc, (int32_t)T, mx, A.rowptr, A.col, A.val, cf,
                                                                     strong, cpt, R.rowptr, ws, wi, R.col, R.val);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// Aggressive coarsening, two-stage form: level l's coarse grid becomes the
// second of two PMIS stages and its interpolation the product of the two
// stages' interpolations, P = P_l P_{l+1}, R = P^T (with AIR the product of
// the stages' restrictions, R_{l+1} R_l); level l+1 is dropped and
// A_{l+2} = R_{l+1} (R_l A_l P_l) P_{l+1} stays the next operator. Applied
// to the first prm.agg_levels coarse grids while every system coarsens past
// the dropped level.
static int merge_levels(Hier &H, const rs_amg_params &prm, int32_t *f32err, cudaStream_t s) {
  for (int32_t l = 0; l < prm.agg_levels && l + 2 < (int32_t)H.L.size(); l++) {
    bool all = true;
    for (int32_t q = 0; q < H.nseg; q++) all = all && H.last_level[q] >= l + 2;
    if (!all) break;
    Level &L = H.L[l];
    Level &M = H.L[l + 1];
    DCsr P, R;
    RS_TRY(spgemm(L.P, M.P, P, s));
    if (L.nfun == 1 && prm.restriction > 0) RS_TRY(spgemm(M.R, L.R, R, s));
    else RS_TRY(transpose(P, R, s));
    const int32_t n = L.A.n;
    Scratch sc(s);
    int32_t *cidx = nullptr;
    int8_t *cf = nullptr;
    RS_TRY(sc.get(&cidx, (size_t)n + 1));
    RS_TRY(dalloc_n(&cf, (size_t)n + 1, s));
    if (n > 0) {
      RS_COUNTED k_is_c<<<grid_for(n), kBlock, 0, s>>>(n, L.cf, cidx);
      int32_t nc = 0;
      RS_TRY(exclusive_scan(cidx, cidx, n, s, &nc));
      RS_COUNTED k_cf_merge<<<grid_for(n), kBlock, 0, s>>>(n, L.cf, cidx, M.cf, cf);
    }
    if (H.precision == RS_PREC_FP32) {
      RS_TRY(dalloc_n(&P.valf, (size_t)P.nnz + 1, s));
      RS_TRY(dalloc_n(&R.valf, (size_t)R.nnz + 1, s));
      if (P.nnz) RS_COUNTED k_to_f32<<<grid_for(P.nnz), kBlock, 0, s>>>(P.nnz, P.val, P.valf, f32err);
      if (R.nnz) RS_COUNTED k_to_f32<<<grid_for(R.nnz), kBlock, 0, s>>>(R.nnz, R.val, R.valf, f32err);
    }
    RS_CHECK_CUDA(cudaGetLastError());
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    dcsr_free(L.P, s);
    dcsr_free(L.R, s);
    dfree(L.cf, s);
    L.P = P;
    L.R = R;
    L.cf = cf;
    level_free(M, s);
    H.L.erase(H.L.begin() + l + 1);
    for (int32_t q = 0; q < H.nseg; q++) H.last_level[q]--;
    H.nlev = (int32_t)H.L.size();
  }
  return 0;
}

int amg_build(const DCsr &A0, const std::vector<int32_t> &seg_off0, const rs_amg_params &prm, Hier &H,
              cudaStream_t s) {
  H.prm = prm;
  if (prm.num_functions == 2) {
    H.prm.smoother = RS_SMOOTH_HYBRID;   // point-block hybrid smoother
    if (prm.chunk < 32 || prm.chunk > 512) return fail(RS_EINVAL, "chunk outside [32, 512]");
    for (size_t q = 0; q < seg_off0.size(); q++)
      if (seg_off0[q] % 2) return fail(RS_EINVAL, "systems AMG needs whole points (even row counts per system)");
  }
  H.precision = prm.precision;
  H.nseg = (int32_t)seg_off0.size() - 1;
  H.L.clear();
  H.L.reserve(33);
  H.last_level.assign(H.nseg, -1);
  const int32_t maxl = std::max(1, std::min(prm.max_levels, 32));
  if (A0.n == 0) {   // empty system: one empty level, nothing to coarsen or solve
    H.L.emplace_back();
    H.L[0].seg_off = seg_off0;
    H.nlev = 1;
    H.last_level.assign(H.nseg, 0);
    return 0;
  }
  // set by the FP32 copies when a finite FP64 value lies beyond the FP32 range
  Scratch scb(s);
  int32_t *f32err = nullptr;
  RS_TRY(scb.get(&f32err, 1));
  RS_CHECK_CUDA(cudaMemsetAsync(f32err, 0, sizeof(int32_t), s));
  const int32_t nfun0 = std::max(1, prm.num_functions);
  // level 0 owns a copy of A
  H.L.emplace_back();
  {
    Level &L0 = H.L[0];
    L0.A.n = L0.A.m = A0.n;
    L0.A.nnz = A0.nnz;
    RS_TRY(dalloc_n(&L0.A.rowptr, (size_t)A0.n + 1, s));
    RS_TRY(dalloc_n(&L0.A.col, (size_t)A0.nnz, s));
    RS_TRY(dalloc_n(&L0.A.val, (size_t)A0.nnz, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(L0.A.rowptr, A0.rowptr, sizeof(int32_t) * ((size_t)A0.n + 1), cudaMemcpyDeviceToDevice, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(L0.A.col, A0.col, sizeof(int32_t) * (size_t)A0.nnz, cudaMemcpyDeviceToDevice, s));
    RS_CHECK_CUDA(cudaMemcpyAsync(L0.A.val, A0.val, sizeof(double) * (size_t)A0.nnz, cudaMemcpyDeviceToDevice, s));
    L0.seg_off = seg_off0;
  }
  // systems (point) AMG: B unknowns per point; points are coarsened on the
  // function-0 part and each function is interpolated on its own part
  const int32_t B = prm.num_functions == 2 ? 2 : 1;
  for (int32_t l = 0;; l++) {
    Level &L = H.L[l];
    const int32_t n = L.A.n, nseg = H.nseg;
    L.nfun = B;
    Scratch sc(s);
    int32_t *seg = nullptr, *dseg_off = nullptr;
    RS_TRY(seg_ids(L.seg_off, n, &seg, s));
    if (nseg > 1) L.row_seg = seg;     // kept for the V-cycle's retired-system test
    else sc.ptrs.push_back(seg);
    RS_TRY(upload(&dseg_off, L.seg_off, s));
    sc.ptrs.push_back(dseg_off);
    // which systems still coarsen
    std::vector<uint8_t> act(nseg, 0);
    int32_t nact = 0;
    for (int32_t g = 0; g < nseg; g++) {
      const int32_t ng = L.seg_off[g + 1] - L.seg_off[g];
      if (H.last_level[g] >= 0) continue;
      if (ng > prm.coarse_n && l < maxl - 1) { act[g] = 1; nact++; }
      else H.last_level[g] = l;
    }
    std::vector<uint8_t> smooth_seg(act);   // systems smoothed (not solved) at this level
    if (nact > 0) {
      // the matrix whose points are coarsened: A itself, or its function-0 part
      DCsr Ap;
      const DCsr &M = B > 1 ? Ap : L.A;
      const int32_t np = n / B;
      std::vector<int32_t> pseg_off(nseg + 1);
      for (int32_t q = 0; q <= nseg; q++) pseg_off[q] = L.seg_off[q] / B;
      int32_t *pseg = seg, *dpseg_off = dseg_off;
      if (B > 1) {
        RS_TRY(func_part(L.A, B, 0, Ap, s));
        RS_TRY(seg_ids(pseg_off, np, &pseg, s));
        sc.ptrs.push_back(pseg);
        RS_TRY(upload(&dpseg_off, pseg_off, s));
        sc.ptrs.push_back(dpseg_off);
      }
      uint8_t *dact = nullptr, *strong = nullptr, *notmax = nullptr;
      int32_t *lam = nullptr, *left = nullptr, *segc = nullptr, *isc = nullptr, *err = nullptr;
      uint64_t *key = nullptr;
      double *diag = nullptr;
      int8_t *cfp = nullptr;
      RS_TRY(sc.get(&dact, (size_t)nseg));
      RS_TRY(sc.get(&strong, (size_t)std::max(M.nnz, L.A.nnz) + 1));
      RS_TRY(sc.get(&notmax, (size_t)np + 1));
      RS_TRY(sc.get(&lam, (size_t)np + 1));
      RS_TRY(sc.get(&left, 2));
      RS_TRY(sc.get(&segc, (size_t)nseg));
      RS_TRY(sc.get(&isc, (size_t)np + 1));
      RS_TRY(sc.get(&key, (size_t)np + 1));
      RS_TRY(sc.get(&diag, (size_t)np + 1));
      RS_TRY(sc.get(&err, 1));
      RS_CHECK_CUDA(cudaMemcpyAsync(dact, act.data(), nseg, cudaMemcpyHostToDevice, s));
      RS_TRY(dalloc_n(&L.cf, (size_t)n, s));
      if (B > 1) RS_TRY(sc.get(&cfp, (size_t)np + 1));
      else cfp = L.cf;
      const unsigned g = grid_for(np);
      const int rg = row_lanes(np, M.nnz);
      const unsigned gg = grid_for((int64_t)np * rg);
      RS_ROWG_SWITCH(rg, RS_COUNTED k_diag<G_><<<gg, kBlock, 0, s>>>(np, M.rowptr, M.col, M.val, diag);
                     RS_COUNTED k_strength<G_><<<gg, kBlock, 0, s>>>(np, M.rowptr, M.col, M.val, diag, pseg, dact,
                                                                     prm.theta, 1, strong));
      RS_CHECK_CUDA(cudaMemsetAsync(lam, 0, sizeof(int32_t) * np, s));
      RS_ROWG_SWITCH(rg, RS_COUNTED k_lambda<G_><<<gg, kBlock, 0, s>>>(np, M.rowptr, M.col, strong, lam));
      RS_COUNTED k_pmis_init<<<g, kBlock, 0, s>>>(np, lam, pseg, dpseg_off, dact, prm.seed, l, key, cfp);
      RS_CHECK_CUDA(cudaMemsetAsync(notmax, 0, (size_t)np, s));
      int32_t hleft = 1, rounds = 0;
      while (hleft > 0) {
        if (++rounds > 100000) return fail(RS_ESETUP, "PMIS did not finish");
        // a few rounds between host checks; a round with nothing undecided does nothing
        for (int r = 0; r < 3; r++) {
          RS_CHECK_CUDA(cudaMemsetAsync(left, 0, sizeof(int32_t), s));
          // (a thread per point: after the first rounds most points are
          // decided and leave at once)
          RS_COUNTED k_pmis_losers<1><<<g, kBlock, 0, s>>>(np, M.rowptr, M.col, strong, key, cfp, notmax);
          RS_COUNTED k_pmis_select<<<g, kBlock, 0, s>>>(np, notmax, cfp);
          RS_COUNTED k_pmis_fmark<1><<<g, kBlock, 0, s>>>(np, M.rowptr, M.col, strong, cfp, left);
        }
        RS_TRY(sync_copy(&hleft, left, sizeof(int32_t), s));
      }
      // per-system C counts; systems that coarsen too little stop here
      RS_CHECK_CUDA(cudaMemsetAsync(segc, 0, sizeof(int32_t) * nseg, s));
      RS_COUNTED k_seg_count_c<<<g, kBlock, 0, s>>>(np, cfp, pseg, segc);
      std::vector<int32_t> hc(nseg);
      RS_TRY(sync_copy(hc.data(), segc, sizeof(int32_t) * nseg, s));
      nact = 0;
      bool dropped = false;   // a system stopped coarsening after PMIS
      for (int32_t q = 0; q < nseg; q++) {
        if (!act[q]) continue;
        const int32_t ng = pseg_off[q + 1] - pseg_off[q];
        if (hc[q] == 0 || (double)hc[q] > 0.9 * (double)ng) {
          act[q] = 0; smooth_seg[q] = 0; H.last_level[q] = l; dropped = true;
        } else {
          nact++;
        }
      }
      RS_CHECK_CUDA(cudaMemcpyAsync(dact, act.data(), nseg, cudaMemcpyHostToDevice, s));
      RS_COUNTED k_seg_revert<<<g, kBlock, 0, s>>>(np, cfp, pseg, dact, isc);
      if (B > 1 && np > 0) RS_COUNTED k_cf_expand<<<g, kBlock, 0, s>>>(np, B, cfp, L.cf);
      if (B > 1) dcsr_free(Ap, s);
      if (nact > 0) {
        int32_t nc = 0;
        RS_TRY(exclusive_scan(isc, isc, np, s, &nc));
        std::vector<int32_t> off_next(nseg + 1);
        int32_t *offd = nullptr;
        RS_TRY(sc.get(&offd, (size_t)nseg + 1));
        RS_COUNTED k_gather_offsets<<<grid_for(nseg + 1), kBlock, 0, s>>>(nseg + 1, dpseg_off, isc, offd);
        RS_TRY(sync_copy(off_next.data(), offd, sizeof(int32_t) * (nseg + 1), s));
        for (int32_t q = 0; q <= nseg; q++) off_next[q] *= B;
        // interpolation of one function part F (np rows) under the point splitting
        auto interpolate = [&](const DCsr &F, const int8_t *cfu, DCsr &Pf) -> int {
          const unsigned gf = grid_for(F.n);
          // the diagonal and strength of F: those PMIS used when F is the
          // coarsened matrix itself and no system stopped since, else formed
          if (B > 1 || dropped) {
            const int fg = row_lanes(F.n, F.nnz);
            const unsigned gfg = grid_for((int64_t)F.n * fg);
            RS_ROWG_SWITCH(fg, RS_COUNTED k_diag<G_><<<gfg, kBlock, 0, s>>>(F.n, F.rowptr, F.col, F.val, diag);
                           RS_COUNTED k_strength<G_><<<gfg, kBlock, 0, s>>>(F.n, F.rowptr, F.col, F.val, diag, pseg,
                                                                            dact, prm.theta, 1, strong));
          }
          Pf.n = F.n;
          Pf.m = nc;
          RS_TRY(dalloc_n(&Pf.rowptr, (size_t)F.n + 1, s));
          RS_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
          // ext+i work arrays sized for this level (see IWarp)
          int ccap = kICand, hcap = kICap, fcap = kIF;
          if (prm.interp != RS_INTERP_CLASSICAL && F.n > 0) {
            int32_t *bd = nullptr;
            RS_TRY(sc.get(&bd, 2));
            RS_CHECK_CUDA(cudaMemsetAsync(bd, 0, 2 * sizeof(int32_t), s));
            RS_COUNTED k_interp_bounds<<<gf, kBlock, 0, s>>>(F.n, F.rowptr, F.col, bd);
            int32_t hb[2] = {0, 0};
            RS_TRY(sync_copy(hb, bd, sizeof(hb), s));
            ccap = 32;
            while (ccap < kICand && ccap < hb[0]) ccap *= 2;
            hcap = std::min(ccap, kICap);
            // the candidate set never needs more than twice Chat's capacity
            // (more distinct candidates than hcap is an error either way)
            ccap = std::min(ccap, 2 * hcap);
            fcap = 8;
            while (fcap < kIF && fcap < hb[1]) fcap *= 2;
          }
          // algorithmic bytes of one pass: the level's rows once (column,
          // value, strength flag per entry; row start, diagonal, C/F mark
          // and coarse index per row)
          const double ibytes = (double)F.nnz * 13.0 + (double)F.n * 17.0;
          if (prm.interp == RS_INTERP_CLASSICAL) {
            {
              ProfScope ps(kProfInterp, ibytes, s);
              RS_COUNTED k_interp_classical<false><<<gf, kBlock, 0, s>>>(F.n, F.rowptr, F.col, F.val, diag, strong,
                                                                         cfu, isc, Pf.rowptr, nullptr, nullptr, err);
            }
            int32_t pnnz = 0;
            RS_TRY(exclusive_scan(Pf.rowptr, Pf.rowptr, F.n, s, &pnnz));
            int32_t herr = 0;
            RS_TRY(sync_copy(&herr, err, sizeof(int32_t), s));
            if (herr) return fail(RS_ESETUP, "interpolation set too large on level " + std::to_string(l));
            Pf.nnz = pnnz;
            RS_TRY(dalloc_n(&Pf.col, (size_t)pnnz + 1, s));
            RS_TRY(dalloc_n(&Pf.val, (size_t)pnnz + 1, s));
            ProfScope ps(kProfInterp, ibytes + (double)pnnz * 12.0, s);
            RS_COUNTED k_interp_classical<true><<<gf, kBlock, 0, s>>>(F.n, F.rowptr, F.col, F.val, diag, strong, cfu,
                                                                      isc, Pf.rowptr, Pf.col, Pf.val, err);
          } else {
            // ext+i: the size of every Chat_i (a cheap pass: candidates
            // only), the weights once into rows of that size, then the rows
            // moved together. Every row is first taken with a small
            // workspace (many warps per SM); the rows it cannot hold are
            // listed and taken again with the level's full workspace.
            Scratch si(s);
            int32_t *toff = nullptr, *tcnt = nullptr, *tcol = nullptr, *defer = nullptr;
            double *tval = nullptr;
            uint8_t *bigf = nullptr;
            RS_TRY(si.get(&toff, (size_t)F.n + 1));
            RS_TRY(si.get(&tcnt, (size_t)F.n + 1));
            struct Cfg { int c, h, f, iw; size_t shm; };
            auto cfg_of = [](int c, int h, int f) {
              const size_t wb = iwarp_bytes(c, h, f);
              const int w = (int)std::min<size_t>(8, std::max<size_t>(1, (48 * 1024) / wb));
              return Cfg{c, h, f, w, wb * w};
            };
            const Cfg cbig = cfg_of(ccap, hcap, fcap);
            const Cfg csmall = cfg_of(std::min(ccap, 256), std::min(hcap, 128), std::min(fcap, 64));
            const bool split = csmall.iw > cbig.iw;
            auto grid_w = [&](const Cfg &c, int64_t rows) {
              return (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + c.iw - 1) / c.iw, (int64_t)num_sms() * 64));
            };
            // one pass when the rows' bounds fit a quarter of the free memory:
            // rows reserved at their bound, the weights formed once (rows the
            // small workspace cannot hold again with the full one), then
            // compacted
            if (F.n > 0) {
              unsigned long long *captot = nullptr;
              RS_TRY(si.get(&captot, 1));
              RS_CHECK_CUDA(cudaMemsetAsync(captot, 0, sizeof(unsigned long long), s));
              RS_COUNTED k_interp_cap<<<gf, kBlock, 0, s>>>(F.n, F.rowptr, F.col, strong, cfu, cbig.h, toff, captot);
              unsigned long long hcapt = 0;
              RS_TRY(sync_copy(&hcapt, captot, sizeof(hcapt), s));
              size_t fr = 0, tm = 0;
              RS_CHECK_CUDA(cudaMemGetInfo(&fr, &tm));
              if (hcapt < 0x7fffffffULL && hcapt * 12 <= fr / 4) {
                RS_TRY(exclusive_scan(toff, toff, F.n, s, nullptr));
                RS_TRY(si.get(&tcol, (size_t)hcapt + 1));
                RS_TRY(si.get(&tval, (size_t)hcapt + 1));
                RS_TRY(si.get(&defer, (size_t)F.n + 1));
                RS_CHECK_CUDA(cudaMemsetAsync(defer, 0, sizeof(int32_t), s));
                int32_t nd = 0;
                {
                  ProfScope ps(kProfInterp, ibytes + (double)hcapt * 12.0, s);
                  const Cfg &c = split ? csmall : cbig;
                  RS_COUNTED k_interp_ext_w<false><<<grid_w(c, F.n), 32 * c.iw, c.shm, s>>>(
                      F.n, c.c, c.h, c.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, tcol, tval, tcnt, err,
                      nullptr, 0, nullptr, split ? defer : nullptr);
                  if (split) {
                    RS_TRY(sync_copy(&nd, defer, sizeof(int32_t), s));
                    if (nd > 0)
                      RS_COUNTED k_interp_ext_w<false><<<grid_w(cbig, nd), 32 * cbig.iw, cbig.shm, s>>>(
                          F.n, cbig.c, cbig.h, cbig.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, tcol,
                          tval, tcnt, err, defer + 1, nd, nullptr, nullptr);
                  }
                }
                int32_t pnnz = 0;
                RS_TRY(exclusive_scan(tcnt, Pf.rowptr, F.n, s, &pnnz));
                int32_t herr = 0;
                RS_TRY(sync_copy(&herr, err, sizeof(int32_t), s));
                if (herr) return fail(RS_ESETUP, "interpolation set too large on level " + std::to_string(l));
                Pf.nnz = pnnz;
                RS_TRY(dalloc_n(&Pf.col, (size_t)pnnz + 1, s));
                RS_TRY(dalloc_n(&Pf.val, (size_t)pnnz + 1, s));
                return copy_rows(F.n, pnnz, toff, Pf.rowptr, tcol, tval, Pf.col, Pf.val, s);
              }
            }
            int32_t nbig = 0;
            if (split) {
              RS_TRY(si.get(&bigf, (size_t)F.n + 1));
              RS_TRY(si.get(&defer, (size_t)F.n + 1));
              RS_CHECK_CUDA(cudaMemsetAsync(bigf, 0, (size_t)F.n + 1, s));
              RS_CHECK_CUDA(cudaMemsetAsync(defer, 0, sizeof(int32_t), s));
            }
            {
              ProfScope ps(kProfInterp, ibytes, s);
              const Cfg &c = split ? csmall : cbig;
              if (F.n > 0)
                RS_COUNTED k_interp_ext_w<true><<<grid_w(c, F.n), 32 * c.iw, c.shm, s>>>(
                    F.n, c.c, c.h, c.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, nullptr, nullptr,
                    nullptr, err, nullptr, 0, split ? bigf : nullptr, split ? defer : nullptr);
              if (split) {
                RS_TRY(sync_copy(&nbig, defer, sizeof(int32_t), s));
                if (nbig > 0)
                  RS_COUNTED k_interp_ext_w<true><<<grid_w(cbig, nbig), 32 * cbig.iw, cbig.shm, s>>>(
                      F.n, cbig.c, cbig.h, cbig.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, nullptr,
                      nullptr, nullptr, err, defer + 1, nbig, nullptr, nullptr);
              }
            }
            int32_t tnnz = 0;
            RS_TRY(exclusive_scan(toff, toff, F.n, s, &tnnz));
            int32_t herr = 0;
            RS_TRY(sync_copy(&herr, err, sizeof(int32_t), s));
            if (herr) return fail(RS_ESETUP, "interpolation set too large on level " + std::to_string(l));
            RS_TRY(si.get(&tcol, (size_t)tnnz + 1));
            RS_TRY(si.get(&tval, (size_t)tnnz + 1));
            {
              ProfScope ps(kProfInterp, ibytes + (double)tnnz * 12.0, s);
              const Cfg &c = split ? csmall : cbig;
              if (F.n > 0)
                RS_COUNTED k_interp_ext_w<false><<<grid_w(c, F.n), 32 * c.iw, c.shm, s>>>(
                    F.n, c.c, c.h, c.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, tcol, tval, tcnt, err,
                    nullptr, 0, split ? bigf : nullptr, nullptr);
              if (nbig > 0)
                RS_COUNTED k_interp_ext_w<false><<<grid_w(cbig, nbig), 32 * cbig.iw, cbig.shm, s>>>(
                    F.n, cbig.c, cbig.h, cbig.f, F.rowptr, F.col, F.val, diag, strong, cfu, isc, toff, tcol, tval,
                    tcnt, err, defer + 1, nbig, nullptr, nullptr);
            }
            int32_t pnnz = 0;
            RS_TRY(exclusive_scan(tcnt, Pf.rowptr, F.n, s, &pnnz));
            RS_TRY(sync_copy(&herr, err, sizeof(int32_t), s));
            if (herr) return fail(RS_ESETUP, "interpolation set too large on level " + std::to_string(l));
            Pf.nnz = pnnz;
            RS_TRY(dalloc_n(&Pf.col, (size_t)pnnz + 1, s));
            RS_TRY(dalloc_n(&Pf.val, (size_t)pnnz + 1, s));
            RS_TRY(copy_rows(F.n, pnnz, toff, Pf.rowptr, tcol, tval, Pf.col, Pf.val, s));
          }
          RS_CHECK_CUDA(cudaGetLastError());
          return 0;
        };
        DCsr &P = L.P;
        if (B == 1) {
          RS_TRY(interpolate(L.A, L.cf, P));
        } else {
          P.n = n;
          P.m = B * nc;
          RS_TRY(dalloc_n(&P.rowptr, (size_t)n + 1, s));
          DCsr Pf[2];
          for (int32_t f = 0; f < B; f++) {
            DCsr Af;
            RS_TRY(func_part(L.A, B, f, Af, s));
            const int r = interpolate(Af, cfp, Pf[f]);
            dcsr_free(Af, s);
            if (r) {
              for (int32_t q = 0; q <= f; q++) dcsr_free(Pf[q], s);
              return r;
            }
            if (np > 0) RS_COUNTED k_ileave_count<<<g, kBlock, 0, s>>>(np, B, f, Pf[f].rowptr, P.rowptr);
          }
          int32_t pnnz = 0;
          RS_TRY(exclusive_scan(P.rowptr, P.rowptr, n, s, &pnnz));
          P.nnz = pnnz;
          RS_TRY(dalloc_n(&P.col, (size_t)pnnz + 1, s));
          RS_TRY(dalloc_n(&P.val, (size_t)pnnz + 1, s));
          for (int32_t f = 0; f < B; f++) {
            if (np > 0)
              RS_COUNTED k_ileave_fill<<<g, kBlock, 0, s>>>(np, B, f, Pf[f].rowptr, Pf[f].col, Pf[f].val, P.rowptr,
                                                            P.col, P.val);
            dcsr_free(Pf[f], s);
          }
          RS_CHECK_CUDA(cudaGetLastError());
        }
        // (strong: the strength of L.A, as left by the interpolation)
        if (B == 1 && prm.restriction > 0)
          RS_TRY(air_restriction(L.A, L.cf, isc, nc, prm.restriction == 3 ? strong : nullptr, L.R, s));
        else RS_TRY(transpose(P, L.R, s));
        DCsr AP;
        RS_TRY(spgemm(L.A, P, AP, s));
        Level next;
        int r = spgemm(L.R, AP, next.A, s);
        dcsr_free(AP, s);
        if (r) return r;
        next.seg_off = off_next;
        H.L.push_back(next);
      } else {
        dfree(L.cf, s);
        L.cf = nullptr;
      }
    }
    Level &Lc = H.L[l];   // (reference may have moved after push_back)
    // smoother data for the systems smoothed here
    const bool any_smooth = std::any_of(smooth_seg.begin(), smooth_seg.end(), [](uint8_t v) { return v != 0; });
    if (any_smooth && H.prm.smoother == RS_SMOOTH_HYBRID) {
      // chunk k = rows [packed[2k], packed[2k+1]), never spanning two systems;
      // per system the chunk size is `chunk` (`chunk_coarse`, when set, on
      // levels >= 1)
      std::vector<int32_t> packed, csys;
      int32_t nsm = 0;
      const int32_t C0 = (l == 0 || prm.chunk_coarse <= 0) ? prm.chunk : prm.chunk_coarse;
      Lc.chunk_c = 0;
      for (int32_t q = 0; q < nseg; q++) {
        if (!smooth_seg[q]) continue;
        const int64_t nq = Lc.seg_off[q + 1] - Lc.seg_off[q];
        const int32_t C = C0;
        Lc.chunk_c = std::max(Lc.chunk_c, C);
        for (int32_t r = Lc.seg_off[q]; r < Lc.seg_off[q + 1]; r += C) {
          packed.push_back(r);
          csys.push_back(q);
          packed.push_back(std::min(r + C, Lc.seg_off[q + 1]));
        }
        nsm += (int32_t)nq;
      }
      Lc.nchunk = (int32_t)(packed.size() / 2);
      Lc.nsmooth = nsm;
      RS_TRY(upload(&Lc.chunk_row0, packed, s));
      if (nseg > 1 && !csys.empty()) RS_TRY(upload(&Lc.chunk_sys, csys, s));
      RS_TRY(dalloc_n(&Lc.colour, (size_t)n, s));
      int32_t *cc = nullptr;   // max colour, error flag, largest chunk
      RS_TRY(sc.get(&cc, 3));
      RS_CHECK_CUDA(cudaMemsetAsync(cc, 0, 3 * sizeof(int32_t), s));
      if (Lc.nchunk > 0)
        RS_COUNTED k_chunk_nnz_max<<<grid_for(Lc.nchunk), kBlock, 0, s>>>(Lc.nchunk, Lc.chunk_row0, Lc.A.rowptr, cc + 2);
      if (n > 0) RS_COUNTED k_fill_colour<<<grid_for(n), kBlock, 0, s>>>(n, Lc.colour);
      if (Lc.nchunk > 0)
        RS_COUNTED (B == 1 ? k_chunk_colour<1> : k_chunk_colour<2>)<<<Lc.nchunk, 256, 0, s>>>(
            Lc.chunk_row0, Lc.A.rowptr, Lc.A.col, Lc.colour, cc, cc + 1);
      int32_t hcc[3] = {0, 0, 0};
      RS_TRY(sync_copy(hcc, cc, sizeof(hcc), s));
      if (hcc[1]) return fail(RS_ESETUP, "chunk colouring failed on level " + std::to_string(l));
      Lc.ncolour = hcc[0];
      Lc.chunk_max_nnz = hcc[2];
      RS_TRY(dalloc_n(&Lc.chunk_coff, (size_t)Lc.nchunk * (Lc.ncolour + 1), s));
      RS_TRY(dalloc_n(&Lc.chunk_rows, (size_t)n, s));
      if (Lc.nchunk > 0)
        RS_COUNTED (B == 1 ? k_chunk_sort<1> : k_chunk_sort<2>)<<<Lc.nchunk, 512, 0, s>>>(Lc.chunk_row0, Lc.colour, Lc.ncolour, Lc.chunk_coff,
                                                          Lc.chunk_rows);
      RS_CHECK_CUDA(cudaGetLastError());
    } else if (any_smooth) {
      RS_TRY(colour_level(Lc, seg, dseg_off, smooth_seg, prm.seed, l, s));
    }
    RS_TRY(dalloc_n(&Lc.dinv, (size_t)n, s));
    RS_TRY(dalloc_n(&Lc.dinvf, (size_t)n, s));
    if (n > 0)
      RS_COUNTED k_smoother_diag<<<grid_for(n), kBlock, 0, s>>>(n, Lc.A.rowptr, Lc.A.col, Lc.A.val,
                                                     H.prm.smoother == RS_SMOOTH_L1JACOBI, Lc.dinv, Lc.dinvf,
                                                     H.precision == RS_PREC_FP32 ? f32err : nullptr);
    if (B == 2) {
      const int32_t np = n / 2;
      RS_TRY(dalloc_n(&Lc.binv, 4 * (size_t)np + 4, s));
      RS_TRY(dalloc_n(&Lc.binvf, 4 * (size_t)np + 4, s));
      if (np > 0)
        RS_COUNTED k_block_inv2<<<grid_for(np), kBlock, 0, s>>>(np, Lc.A.rowptr, Lc.A.col, Lc.A.val, Lc.binv,
                                                                Lc.binvf,
                                                                H.precision == RS_PREC_FP32 ? f32err : nullptr);
    }
    // systems solved directly here
    int64_t inv_tot = 0;
    std::vector<int4> info;
    std::vector<int64_t> ioff;
    std::vector<int32_t> rows;
    std::vector<int32_t> rowseg;
    for (int32_t q = 0; q < nseg; q++) {
      if (H.last_level[q] != l) continue;
      const int32_t r0 = Lc.seg_off[q], ng = Lc.seg_off[q + 1] - Lc.seg_off[q];
      if (ng == 0) continue;
      if (ng > prm.max_dense)
        return fail(RS_ESETUP, "coarsest level of system " + std::to_string(q) + " has " + std::to_string(ng) +
                                   " rows (> max_dense)");
      Lc.cseg.push_back(q);
      info.push_back(make_int4(r0, ng, 0, 0));
      ioff.push_back(inv_tot);
      for (int32_t t = 0; t < ng; t++) { rows.push_back(r0 + t); rowseg.push_back((int32_t)info.size() - 1); }
      inv_tot += (int64_t)ng * ng;
    }
    if (!info.empty()) {
      Lc.ncoarse_rows = (int32_t)rows.size();
      RS_TRY(upload(&Lc.cinfo, info, s));
      RS_TRY(upload(&Lc.cinv_off, ioff, s));
      RS_TRY(upload(&Lc.crows, rows, s));
      RS_TRY(upload(&Lc.crow_seg, rowseg, s));
      if (nseg > 1) {
        std::vector<int32_t> rsys(rowseg.size());
        for (size_t t = 0; t < rowseg.size(); t++) rsys[t] = Lc.cseg[rowseg[t]];
        RS_TRY(upload(&Lc.crow_sys, rsys, s));
      }
      RS_TRY(dalloc_n(&Lc.cinv, (size_t)inv_tot, s));
      int32_t maxng = 0;
      for (const int4 &in : info) maxng = std::max(maxng, in.y);
      if (maxng <= kCoarseSmemN) {
        const size_t shm = 2 * sizeof(double) * (size_t)maxng * maxng;
        static bool attr = false;
        if (!attr) {
          RS_CHECK_CUDA(cudaFuncSetAttribute(k_coarse_dense<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(2 * sizeof(double) * kCoarseSmemN * kCoarseSmemN)));
          attr = true;
        }
        RS_COUNTED k_coarse_dense<true><<<(unsigned)info.size(), 256, shm, s>>>(
            Lc.A.rowptr, Lc.A.col, Lc.A.val, Lc.cinfo, Lc.cinv_off, nullptr, Lc.cinv);
      } else {
        double *work = nullptr;
        RS_TRY(sc.get(&work, 2 * (size_t)inv_tot));
        RS_COUNTED k_coarse_dense<false><<<(unsigned)info.size(), 256, 0, s>>>(
            Lc.A.rowptr, Lc.A.col, Lc.A.val, Lc.cinfo, Lc.cinv_off, work, Lc.cinv);
      }
      RS_CHECK_CUDA(cudaGetLastError());
    }
    // FP32 copies for the FP32 cycle
    if (H.precision == RS_PREC_FP32) {
      RS_TRY(dalloc_n(&Lc.A.valf, (size_t)Lc.A.nnz, s));
      if (Lc.A.nnz) RS_COUNTED k_to_f32<<<grid_for(Lc.A.nnz), kBlock, 0, s>>>(Lc.A.nnz, Lc.A.val, Lc.A.valf, f32err);
      if (Lc.P.rowptr) {
        RS_TRY(dalloc_n(&Lc.P.valf, (size_t)Lc.P.nnz, s));
        RS_TRY(dalloc_n(&Lc.R.valf, (size_t)Lc.R.nnz, s));
        if (Lc.P.nnz) RS_COUNTED k_to_f32<<<grid_for(Lc.P.nnz), kBlock, 0, s>>>(Lc.P.nnz, Lc.P.val, Lc.P.valf, f32err);
        if (Lc.R.nnz) RS_COUNTED k_to_f32<<<grid_for(Lc.R.nnz), kBlock, 0, s>>>(Lc.R.nnz, Lc.R.val, Lc.R.valf, f32err);
      }
    }
    // packed operator of the hybrid smoother, in the cycle's precision
    if (H.prm.smoother == RS_SMOOTH_HYBRID && Lc.nchunk > 0) {
      RS_TRY(dalloc_n(&Lc.hs_rp, (size_t)n + 1, s));
      RS_TRY(dalloc_n(&Lc.hs_mid, (size_t)n, s));
      RS_CHECK_CUDA(cudaMemsetAsync(Lc.hs_rp, 0, sizeof(int32_t) * ((size_t)n + 1), s));
      const int hg = row_lanes(n, Lc.A.nnz);
      RS_ROWG_SWITCH(hg, RS_COUNTED (B == 1 ? k_hs_count<1, G_> : k_hs_count<2, G_>)<<<Lc.nchunk, 256, 0, s>>>(
                             Lc.chunk_row0, Lc.A.rowptr, Lc.A.col, Lc.hs_rp));
      int32_t tot = 0;
      RS_TRY(exclusive_scan(Lc.hs_rp, Lc.hs_rp, n, s, &tot));
      Lc.hs_nnz = tot;
      {
        int32_t *mx = nullptr;
        RS_TRY(sc.get(&mx, 1));
        RS_CHECK_CUDA(cudaMemsetAsync(mx, 0, sizeof(int32_t), s));
        RS_COUNTED k_chunk_nnz_max<<<grid_for(Lc.nchunk), kBlock, 0, s>>>(Lc.nchunk, Lc.chunk_row0, Lc.hs_rp, mx);
        RS_TRY(sync_copy(&Lc.hs_chunk_max, mx, sizeof(int32_t), s));
      }
      RS_TRY(dalloc_n(&Lc.hs_col, (size_t)tot + 1, s));
      if (H.precision == RS_PREC_FP32) {
        RS_TRY(dalloc_n(&Lc.hs_valf, (size_t)tot + 1, s));
        RS_ROWG_SWITCH(hg, RS_COUNTED (B == 1 ? k_hs_fill<float, 1, G_> : k_hs_fill<float, 2, G_>)<<<Lc.nchunk, 256,
                                                                                               0, s>>>(
                               Lc.chunk_row0, Lc.A.rowptr, Lc.A.col, Lc.A.val, Lc.hs_rp, Lc.hs_mid, Lc.hs_col,
                               Lc.hs_valf));
      } else {
        RS_TRY(dalloc_n(&Lc.hs_val, (size_t)tot + 1, s));
        RS_ROWG_SWITCH(hg, RS_COUNTED (B == 1 ? k_hs_fill<double, 1, G_> : k_hs_fill<double, 2, G_>)<<<Lc.nchunk,
                                                                                                 256, 0, s>>>(
                               Lc.chunk_row0, Lc.A.rowptr, Lc.A.col, Lc.A.val, Lc.hs_rp, Lc.hs_mid, Lc.hs_col,
                               Lc.hs_val));
      }
      RS_CHECK_CUDA(cudaGetLastError());
    }
    // work vectors
    const size_t es = H.precision == RS_PREC_FP32 ? sizeof(float) : sizeof(double);
    RS_TRY(dalloc(&Lc.x, es * ((size_t)n + 1), s));
    RS_TRY(dalloc(&Lc.x2, es * ((size_t)n + 1), s));
    RS_CHECK_CUDA(cudaMemsetAsync(Lc.x, 0, es * ((size_t)n + 1), s));
    RS_CHECK_CUDA(cudaMemsetAsync(Lc.x2, 0, es * ((size_t)n + 1), s));
    RS_TRY(dalloc(&Lc.b, es * ((size_t)n + 1), s));
    RS_TRY(dalloc(&Lc.r, es * ((size_t)n + 1), s));
    RS_TRY(dalloc(&Lc.t, es * ((size_t)n + 1), s));
    RS_CHECK_CUDA(cudaGetLastError());
    if ((int32_t)H.L.size() == l + 1) break;   // no next level
  }
  H.nlev = (int32_t)H.L.size();
  for (int32_t q = 0; q < H.nseg; q++)
    if (H.last_level[q] < 0) H.last_level[q] = H.nlev - 1;
  RS_TRY(merge_levels(H, prm, f32err, s));
  int32_t hrange = 0;
  RS_TRY(sync_copy(&hrange, f32err, sizeof(int32_t), s));
  if (hrange)
    return fail(RS_ESETUP, "hierarchy values lie beyond the FP32 range; use an FP64 hierarchy (RS_PREC_FP64)");
  return amg_tune_smoother(H, s);
}

static void level_free(Level &L, cudaStream_t s) {
  {
    dcsr_free(L.A, s);
    dcsr_free(L.P, s);
    dcsr_free(L.R, s);
    dfree(L.cf, s);
    dfree(L.colour, s);
    dfree(L.colour_rows, s);
    dfree(L.dinv, s);
    dfree(L.dinvf, s);
    dfree(L.cinfo, s);
    dfree(L.cinv_off, s);
    dfree(L.crows, s);
    dfree(L.crow_seg, s);
    dfree(L.cinv, s);
    dfree(L.x, s);
    dfree(L.x2, s);
    dfree(L.chunk_row0, s);
    dfree(L.chunk_coff, s);
    dfree(L.chunk_rows, s);
    dfree(L.hs_rp, s);
    dfree(L.hs_mid, s);
    dfree(L.hs_col, s);
    dfree(L.hs_val, s);
    dfree(L.hs_valf, s);
    dfree(L.binv, s);
    dfree(L.binvf, s);
    dfree(L.b, s);
    dfree(L.r, s);
    dfree(L.t, s);
    dfree(L.row_seg, s);
    dfree(L.chunk_sys, s);
    dfree(L.crow_sys, s);
  }
}

void amg_free(Hier &H, cudaStream_t s) {
  for (Level &L : H.L) level_free(L, s);
  H.L.clear();
  H.nlev = 0;
}

}  // namespace rs
