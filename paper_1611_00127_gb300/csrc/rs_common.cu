// Error state, memory pool, device scan and batch helpers.
#include <cstdio>
#include <atomic>
#include <mutex>

#include "rs_internal.cuh"

namespace rs {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::once_flag g_pool_once;

int dalloc(void **p, size_t bytes, cudaStream_t s) {
  std::call_once(g_pool_once, []() {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
    }
  });
  *p = nullptr;
  cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RS_ENOMEM, std::string("cudaMallocAsync(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return 0;
}

void dfree(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

void dcsr_free(DCsr &A, cudaStream_t s) {
  dfree(A.rowptr, s);
  dfree(A.col, s);
  dfree(A.val, s);
  dfree(A.valf, s);
  A = DCsr();
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 4;
constexpr int kScanTile = kBlock * kScanItems;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
  const unsigned lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the block total to *total.
__device__ int32_t block_excl_scan(int32_t v, int32_t *total) {
  __shared__ int32_t wsum[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < kBlock / 32 ? wsum[lane] : 0;
    int32_t wi = warp_incl_scan(w);
    if (lane < kBlock / 32) wsum[lane] = wi - w;
    if (lane == kBlock / 32 - 1) *total = wi;
  }
  __syncthreads();
  int32_t r = inc - v + wsum[wid];
  __syncthreads();
  return r;
}

__global__ void scan_tiles(const int32_t *in, int32_t *out, int32_t n, int32_t *tile_sums) {
  __shared__ int32_t tot;
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int32_t pre = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = pre;
    pre += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place; total to *total.
__global__ void scan_sums(int32_t *sums, int32_t nt, int32_t *total_out) {
  __shared__ int32_t tot;
  int32_t carry = 0;
  for (int32_t base = 0; base < nt; base += kBlock) {
    int32_t i = base + threadIdx.x;
    int32_t v = i < nt ? sums[i] : 0;
    int32_t pre = block_excl_scan(v, &tot);
    if (i < nt) sums[i] = pre + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void scan_add(int32_t *out, int32_t n, const int32_t *tile_off, const int32_t *total) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  int32_t add = tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t j = i + (int64_t)k * kBlock;
    if (j < n) out[j] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *total;
}

int exclusive_scan(const int32_t *in, int32_t *out, int32_t n, cudaStream_t s, int32_t *total) {
  int32_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt < 1) nt = 1;
  Scratch sc(s);
  int32_t *sums = nullptr;
  RS_TRY(sc.get(&sums, (size_t)nt + 1));
  RS_COUNTED scan_tiles<<<nt, kBlock, 0, s>>>(in, out, n, sums);
  RS_COUNTED scan_sums<<<1, kBlock, 0, s>>>(sums, nt, sums + nt);
  RS_COUNTED scan_add<<<nt, kBlock, 0, s>>>(out, n, sums, sums + nt);
  RS_CHECK_CUDA(cudaGetLastError());
  if (total) {
    RS_CHECK_CUDA(cudaMemcpyAsync(total, out + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  return 0;
}

// ------------------------------------------------------------------ batches
std::vector<int32_t> seg_offsets(int32_t n, int32_t nseg, const int32_t *seg_off) {
  std::vector<int32_t> o;
  if (nseg <= 1 || !seg_off) {
    o = {0, n};
  } else {
    o.assign(seg_off, seg_off + nseg + 1);
  }
  return o;
}

__global__ void k_seg_ids(const int32_t *off, int32_t nseg, int32_t n, int32_t *seg) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  seg[i] = lo;
}

int seg_ids(const std::vector<int32_t> &seg_off, int32_t n, int32_t **dseg, cudaStream_t s) {
  int32_t nseg = (int32_t)seg_off.size() - 1;
  RS_TRY(dalloc_n(dseg, (size_t)n + 1, s));
  int32_t *doff = nullptr;
  RS_TRY(dalloc_n(&doff, seg_off.size(), s));
  RS_CHECK_CUDA(cudaMemcpyAsync(doff, seg_off.data(), seg_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (n > 0) RS_COUNTED k_seg_ids<<<grid_for(n), kBlock, 0, s>>>(doff, nseg, n, *dseg);
  dfree(doff, s);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

// ------------------------------------------------------------------ profiling
struct ProfPending {
  int cls;
  double bytes;
  cudaEvent_t e0, e1;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfPending> g_prof_pending;
static double g_prof_ms[kProfCount], g_prof_bytes[kProfCount];
static long long g_prof_n[kProfCount];

bool profiling() { return g_prof_on; }

ProfScope::ProfScope(int c, double b, cudaStream_t st) : cls(c), bytes(b), s(st) {
  if (!g_prof_on) return;
  cudaEventCreate(&e0);
  cudaEventRecord(e0, s);
}

ProfScope::~ProfScope() {
  if (!e0) return;
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, s);
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_prof_pending.push_back({cls, bytes, e0, e1});
}

static void prof_resolve() {
  for (auto &p : g_prof_pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.e1);
    if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      g_prof_ms[p.cls] += ms;
      g_prof_bytes[p.cls] += p.bytes;
      g_prof_n[p.cls] += 1;
    }
    cudaEventDestroy(p.e0);
    cudaEventDestroy(p.e1);
  }
  g_prof_pending.clear();
}

}  // namespace rs

extern "C" int rs_profile_begin(void) {
  std::lock_guard<std::mutex> lock(rs::g_prof_mu);
  rs::prof_resolve();
  for (int c = 0; c < rs::kProfCount; c++) { rs::g_prof_ms[c] = 0; rs::g_prof_bytes[c] = 0; rs::g_prof_n[c] = 0; }
  rs::g_prof_on = true;
  return RS_OK;
}

extern "C" int rs_profile_end(double *ms, double *bytes, long long *launches, int ncls) {
  std::lock_guard<std::mutex> lock(rs::g_prof_mu);
  rs::g_prof_on = false;
  rs::prof_resolve();
  for (int c = 0; c < ncls && c < rs::kProfCount; c++) {
    if (ms) ms[c] = rs::g_prof_ms[c];
    if (bytes) bytes[c] = rs::g_prof_bytes[c];
    if (launches) launches[c] = rs::g_prof_n[c];
  }
  return rs::kProfCount;
}

extern "C" const char *rs_last_error(void) { return rs::g_last_error.c_str(); }

extern "C" long long rs_launch_count(void) { return rs::g_launches.load(); }

extern "C" int rs_version(int *major, int *minor, int *arch) {
  if (major) *major = 0;
  if (minor) *minor = 1;
  if (arch) *arch = 103;
  return RS_OK;
}
