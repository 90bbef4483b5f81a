// Internal declarations shared by the rsflow CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsflow.h"

namespace rs {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

#define RS_CHECK_CUDA(expr)                                                         \
  do {                                                                              \
    cudaError_t e__ = (expr);                                                       \
    if (e__ != cudaSuccess)                                                         \
      return ::rs::fail(RS_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)); \
  } while (0)

#define RS_TRY(expr)              \
  do {                            \
    int r__ = (expr);             \
    if (r__ < 0) return r__;      \
  } while (0)

// ------------------------------------------------------------------ memory
// Stream-ordered allocations from the device's default memory pool (kept
// resident between calls), freed with dfree (stream-ordered) or dfree_sync.
int dalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);
template <typename T>
inline int dalloc_n(T **p, size_t n, cudaStream_t s) {
  return dalloc(reinterpret_cast<void **>(p), n * sizeof(T) + 16, s);
}

// Scratch list freed together at scope end (stream-ordered).
struct Scratch {
  cudaStream_t s;
  std::vector<void *> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <typename T>
  int get(T **p, size_t n) {
    int r = dalloc_n(p, n, s);
    if (r == 0) ptrs.push_back(*p);
    return r;
  }
  ~Scratch() {
    for (void *p : ptrs) dfree(p, s);
  }
};

// ------------------------------------------------------------------ launch
// Every kernel launch of the library is written `RS_COUNTED kernel<<<...>>>(...)`
// so that rs_launch_count() can report how many kernels a call issued.
void count_launch();
void count_launches(long long n);
#define RS_COUNTED ::rs::count_launch(),
constexpr int kBlock = 256;

// Programmatic dependent launch: kernels launched with launch_pdl may be
// scheduled while their predecessor in the stream is still running; every such
// kernel starts with RS_PDL_ENTRY, which waits until the predecessor has
// finished and its writes are visible (so data dependences are unchanged) and
// then lets its own successor be scheduled, so each launch's latency overlaps
// the previous kernel's execution with at most one kernel waiting ahead.
#define RS_PDL_ENTRY()                                            \
  do {                                                            \
    asm volatile("griddepcontrol.wait;" ::: "memory");           \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
  } while (0)

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------------ profiling
// When profiling is on (rs_profile_begin), launches of the main kernel classes
// are bracketed by CUDA events on their stream and their algorithmic bytes are
// accumulated; preconditioner applies then run eagerly (no graph replay) so
// that every launch is seen.
enum ProfClass {
  kProfHgs = 0,       // hybrid Gauss-Seidel sweep
  kProfCsr,           // residual / restriction / prolongation
  kProfBsr2,          // block SpMV (and the CPR residual)
  kProfArnoldi,       // CGS2 dot / update kernels
  kProfSpgemm,        // sparse products of the setup
  kProfInterp,        // interpolation
  kProfOther,
  kProfCount
};
bool profiling();
struct ProfScope {
  int cls;
  double bytes;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(int c, double b, cudaStream_t st);
  ~ProfScope();
};
inline unsigned grid_for(int64_t n, int per_block = kBlock) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 0x7fffffff) g = 0x7fffffff;
  return (unsigned)g;
}
int num_sms();

// exclusive scan: out[i] = sum_{k<i} in[i], out[n] = total; in == out allowed.
// `total` (host, optional) receives the total after a stream sync.
int exclusive_scan(const int32_t *in, int32_t *out, int32_t n, cudaStream_t s, int32_t *total);

// ------------------------------------------------------------------ matrices
struct DCsr {
  int32_t n = 0, m = 0, nnz = 0;
  int32_t *rowptr = nullptr, *col = nullptr;
  double *val = nullptr;  // FP64 values (setup and FP64 cycles)
  float *valf = nullptr;  // FP32 copy (FP32 cycles)
};
void dcsr_free(DCsr &A, cudaStream_t s);

// ------------------------------------------------------------------ kernels shared across files
// y = J x, r = b - J x (bsr2, FP64)
// y = J x; with act (per-system flags) and rseg (system of each block row),
// rows of systems whose flag is 0 get y = 0 without being read
int launch_bsr2_spmv(const rs_bsr2 &J, const double *x, double *y, cudaStream_t s, const uint8_t *act = nullptr,
                     const int32_t *rseg = nullptr);
int launch_bsr2_residual(const rs_bsr2 &J, const double *x, const double *b, double *r,
                         cudaStream_t s);

// Block extraction and derived matrices (setup; exact operation order).
int bsr2_part(const rs_bsr2 &J, int r, int c, DCsr &out, cudaStream_t s);
int bsr2_scalar(const rs_bsr2 &J, DCsr &out, cudaStream_t s);
int simple_schur(const DCsr &App, const DCsr &Aps, const DCsr &Asp, const DCsr &Ass, DCsr &out,
                 cudaStream_t s);
int spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s);
int transpose(const DCsr &A, DCsr &T, cudaStream_t s);
// Moves row i's crp[i+1] - crp[i] entries from offset toff[i] of (tcol, tval)
// to offset crp[i] of (ccol, cval); nnz = crp[n] picks the lanes per row.
int copy_rows(int32_t n, int64_t nnz, const int32_t *toff, const int32_t *crp, const int32_t *tcol,
              const double *tval, int32_t *ccol, double *cval, cudaStream_t s);

// ------------------------------------------------------------------ AMG
struct Level {
  DCsr A, P, R;
  int8_t *cf = nullptr;          // C/F marks (1 C, -1 F) of this level (nullptr on the last)
  int32_t *colour = nullptr;     // colour per row (-1: not smoothed here)
  int32_t ncolour = 0;
  std::vector<int32_t> colour_off;   // host [ncolour+1] into colour_rows
  int32_t *colour_rows = nullptr;    // rows grouped by colour
  int32_t nsmooth = 0;               // rows smoothed at this level
  double *dinv = nullptr;            // 1 / a_ii (GS) or 1 / l1 row norm (Jacobi)
  float *dinvf = nullptr;
  std::vector<int32_t> seg_off;      // host [nseg+1]
  // coarse solve of the systems whose last level is this one
  std::vector<int32_t> cseg;         // systems solved here
  int32_t ncoarse_rows = 0;
  int32_t *crow_seg = nullptr;       // per coarse row: index into cinfo
  int4 *cinfo = nullptr;             // per solved system: (row0, n, inverse offset (in doubles, low), hi)
  int64_t *cinv_off = nullptr;
  int32_t *crows = nullptr;          // the rows solved directly
  double *cinv = nullptr;            // stacked dense inverses, row-major
  // hybrid smoother: chunks of consecutive rows (never spanning two systems)
  int32_t nchunk = 0;
  int32_t chunk_c = 0;               // largest chunk (rows) of this level
  int32_t chunk_max_nnz = 0;         // largest number of matrix entries in one chunk
  int32_t hs_chunk_max = 0;          // largest number of packed smoother entries in one chunk
  int32_t *chunk_row0 = nullptr;     // [2 nchunk] (first row, end row) of each chunk
  int32_t *chunk_coff = nullptr;     // [nchunk * (ncolour+1)] colour offsets inside each chunk
  int32_t *chunk_rows = nullptr;     // [n] local row of each position, sorted by (chunk, colour, row)
  // packed operator of the hybrid smoother: per chunk row, off-diagonal
  // entries inside the chunk (chunk-local column) in [hs_rp[i], hs_mid[i]),
  // then those coupling to other rows (global column) up to hs_rp[i+1];
  // values in the cycle's precision (hs_val FP64 or hs_valf FP32)
  // systems (point) AMG: unknowns per point, and the inverses of the 2 x 2
  // diagonal blocks of the points (row-major, FP64 and FP32)
  int32_t nfun = 1;
  int32_t hgs_lpr = 0;               // lanes per row of the hybrid sweep (0: by rule)
  int8_t xfer_lpr[3] = {0, 0, 0};    // lanes per row of residual, restriction, prolongation (0: by rule)
  // batches only (nullptr for one system): the system of every row, of every
  // smoother chunk and of every row solved directly here
  int32_t *row_seg = nullptr, *chunk_sys = nullptr, *crow_sys = nullptr;
  double *binv = nullptr;
  float *binvf = nullptr;
  int32_t hs_nnz = 0;
  int32_t *hs_rp = nullptr, *hs_mid = nullptr, *hs_col = nullptr;
  double *hs_val = nullptr;
  float *hs_valf = nullptr;
  // work vectors (FP32 or FP64 by the hierarchy's precision); x2 is the
  // second buffer of the hybrid smoother's old/new pair
  void *x = nullptr, *x2 = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
};

struct Hier {
  rs_amg_params prm;
  int32_t nlev = 0;
  int32_t nseg = 1;
  std::vector<Level> L;
  std::vector<int32_t> last_level;   // per system
  int precision = RS_PREC_FP32;
  // batches: per-system flags (nseg bytes, device; nullptr: every system
  // live). A V-cycle writes zeros for the rows of a system whose flag is 0
  // instead of computing them -- FGMRES retires converged systems this way.
  const uint8_t *active = nullptr;
};

int check_amg_params(const rs_amg_params &a);
int amg_build(const DCsr &A0, const std::vector<int32_t> &seg_off, const rs_amg_params &prm,
              Hier &H, cudaStream_t s);
void amg_free(Hier &H, cudaStream_t s);
// x = V-cycle(b); FP64 in/out. `xin_zero` is always true here (zero guess).
int amg_vcycle(const Hier &H, const double *b, double *x, cudaStream_t s);
int amg_level_sweeps(const Hier &H, int32_t l, int sweeps, double *bytes_per_sweep, cudaStream_t s);
int amg_level_xfer(const Hier &H, int32_t l, int which, int reps, double *bytes_per_launch, cudaStream_t s);
// Autotuner of the hybrid sweep's lanes per row: times the candidates on each
// smoothed level's own vectors and stores the fastest in Level::hgs_lpr
// (decisions cached per level shape). Not inside stream capture.
int amg_tune_smoother(Hier &H, cudaStream_t s);
// RS_ETIMEOUT (and clears the flag) if a smoother CTA gave up waiting for its
// staging copies since the last call; synchronises the stream.
int vcycle_wait_status(cudaStream_t s);
// Sets that flag as a capped wait would (no kernel runs).
int vcycle_raise_wait_flag(cudaStream_t s);
// ILU(0) of the point-ordered scalar matrix of J (rs_ilu.cu); the factors
// keep a reference to J's pattern
int ilu0_build(const rs_bsr2 &J, int precision, rs_ilu0 **out, cudaStream_t s);
int ilu0_solve(const rs_ilu0 *F, const double *b, double *x, cudaStream_t s);
void ilu0_free(rs_ilu0 *F);

// ------------------------------------------------------------------ helpers
std::vector<int32_t> seg_offsets(int32_t n, int32_t nseg, const int32_t *seg_off);
int seg_ids(const std::vector<int32_t> &seg_off, int32_t n, int32_t **dseg, cudaStream_t s);

}  // namespace rs

struct rs_amg {
  rs::Hier H;
  cudaStream_t stream;
};
