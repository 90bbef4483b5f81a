// Residual and exact Jacobian of the two-phase TPFA model (Sec. 2; Jacobian
// eq. linearize_fc / eq. jacobian), FP64, for one or several stacked grids.
//
// Two passes: (1) one thread per cell evaluates the constitutive laws
// (mobilities, capillary pressure and their S_n derivatives) once and stores
// them; (2) one thread per cell forms its two residual entries and its block
// row of J from its own and its neighbours' stored values. This keeps the
// FP64 transcendental work (pow) at one evaluation per cell, which matters on
// a part whose FP64 rate is a small fraction of its FP32 rate.
//
// Readings of the model (kept identical to the CPU check):
//  - Residual in mass-rate form: F_a,i = V (xi_a - xi_a,old)/dt
//    + sum_j T_ij rho_a lambda_a,up (Phi_a,i - Phi_a,j) - q_a,i, with
//    xi_w = phi rho_w (1 - S_n), xi_n = phi rho_n S_n, Phi_w = P_w - rho_w g D,
//    Phi_n = P_w + P_c - rho_n g D, T_ij = area * harmonic(K) / spacing.
//  - Upwind: mobility from cell i iff Phi_i - Phi_j > 0, else from j.
//  - k_r: Brooks-Corey-Burdine with the P_c lambda; Brooks-Corey P_c continued
//    linearly below Sb = 1e-4.
//  - Water injected through x = 0 at Darcy flux u_in; Dirichlet outlet on
//    x = L with half-cell transmissibility; other faces closed; depth is the
//    last coordinate. Point wells (the corner wells of the examples of
//    Sec. 4): a water source rho_w q_in in cell well_in instead of the x = 0
//    flux, and the outlet restricted to the x = L face of cell well_out.
#include <cstring>
#include <mutex>

#include "rs_internal.cuh"

namespace rs {

// Largest total cell count of one call (the block layout indexes rows and
// neighbours in 32-bit integers).
constexpr int64_t kMaxCells = 0x3fffffff;

struct DProb {
  int32_t dim, nx, ny, nz;
  double hx, hy, hz;
  const double *kx, *ky, *kz;
  double phi, mu_w, mu_n, rho_w, rho_n, g;
  int32_t pc_model;
  double pc_p0, pc_pd, bc_lambda, s_wr, s_nr, u_in, p_out, sn_out;
  double q_in;
  int32_t well_in, well_out;   // point wells (-1: face conditions)
  int32_t cell0;   // first global cell of this grid
  int32_t ncell;
};

__device__ __forceinline__ void constitutive(const DProb &p, double sn, double *o) {
  const double denom = 1.0 - p.s_wr - p.s_nr;
  const double s = (1.0 - sn - p.s_wr) / denom;
  const double ds = -1.0 / denom;
  const double L = p.bc_lambda;
  const double ew = (2.0 + 3.0 * L) / L, en = (2.0 + L) / L;
  double krw, krn, dkrw, dkrn;
  if (s <= 0.0) {
    krw = 0.0; krn = 1.0; dkrw = 0.0; dkrn = 0.0;
  } else if (s >= 1.0) {
    krw = 1.0; krn = 0.0; dkrw = 0.0; dkrn = 0.0;
  } else {
    const double t = pow(s, en);
    krw = pow(s, ew);
    dkrw = ew * pow(s, ew - 1.0);
    krn = (1.0 - s) * (1.0 - s) * (1.0 - t);
    dkrn = -2.0 * (1.0 - s) * (1.0 - t) - (1.0 - s) * (1.0 - s) * en * pow(s, en - 1.0);
  }
  o[0] = krw / p.mu_w;
  o[1] = krn / p.mu_n;
  o[2] = dkrw * ds / p.mu_w;
  o[3] = dkrn * ds / p.mu_n;
  double pc = 0.0, dpc = 0.0;
  if (p.pc_model == 1) {
    pc = p.pc_p0 * (1.0 - s);
    dpc = -p.pc_p0 * ds;
  } else if (p.pc_model == 2) {
    const double eps = 1e-4;
    double d;
    if (s >= eps) {
      pc = p.pc_pd * pow(s, -1.0 / L);
      d = -(p.pc_pd / L) * pow(s, -1.0 / L - 1.0);
    } else {
      const double pce = p.pc_pd * pow(eps, -1.0 / L);
      d = -(p.pc_pd / L) * pow(eps, -1.0 / L - 1.0);
      pc = pce + d * (s - eps);
    }
    dpc = d * ds;
  }
  o[4] = pc;
  o[5] = dpc;
}

__device__ __forceinline__ int find_prob(const DProb *probs, int32_t nprob, int32_t cell) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (probs[mid].cell0 <= cell) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Local neighbours in ascending order; returns count (<= 6).
__device__ __forceinline__ int neighbours(const DProb &p, int32_t i, int32_t *nb, int *dir) {
  const int32_t nx = p.nx, ny = p.ny, nz = p.nz;
  const int32_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
  int c = 0;
  if (p.dim == 3 && iz > 0) { nb[c] = i - nx * ny; dir[c++] = 2; }
  if (iy > 0) { nb[c] = i - nx; dir[c++] = 1; }
  if (ix > 0) { nb[c] = i - 1; dir[c++] = 0; }
  if (ix < nx - 1) { nb[c] = i + 1; dir[c++] = 0; }
  if (iy < ny - 1) { nb[c] = i + nx; dir[c++] = 1; }
  if (p.dim == 3 && iz < nz - 1) { nb[c] = i + nx * ny; dir[c++] = 2; }
  return c;
}

__global__ void k_pattern_counts(const DProb *probs, int32_t nprob, int32_t ncell, int32_t *cnt) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DProb &p = probs[find_prob(probs, nprob, g)];
  int32_t nb[6];
  int dir[6];
  cnt[g] = 1 + neighbours(p, g - p.cell0, nb, dir);
}

__global__ void k_pattern_fill(const DProb *probs, int32_t nprob, int32_t ncell, const int32_t *rowptr,
                               int32_t *col) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DProb &p = probs[find_prob(probs, nprob, g)];
  const int32_t i = g - p.cell0;
  int32_t nb[6];
  int dir[6];
  int c = neighbours(p, i, nb, dir);
  int32_t pos = rowptr[g];
  bool placed = false;
  for (int k = 0; k < c; k++) {
    if (!placed && nb[k] > i) { col[pos++] = g; placed = true; }
    col[pos++] = p.cell0 + nb[k];
  }
  if (!placed) col[pos++] = g;
}

__global__ void k_props(const DProb *probs, int32_t nprob, int32_t ncell, const double *u, double *props) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DProb &p = probs[find_prob(probs, nprob, g)];
  double o[6];
  constitutive(p, u[2 * (int64_t)g + 1], o);
#pragma unroll
  for (int k = 0; k < 6; k++) props[6 * (int64_t)g + k] = o[k];
}

__device__ __forceinline__ double face_area(const DProb &p, int d) {
  const double hz = p.dim == 3 ? p.hz : 1.0;
  return d == 0 ? p.hy * hz : (d == 1 ? p.hx * hz : p.hx * p.hy);
}
__device__ __forceinline__ double spacing(const DProb &p, int d) { return d == 0 ? p.hx : (d == 1 ? p.hy : p.hz); }
__device__ __forceinline__ double perm(const DProb &p, int d, int32_t i) {
  return d == 0 ? p.kx[i] : (d == 1 ? p.ky[i] : p.kz[i]);
}
__device__ __forceinline__ double depth(const DProb &p, int32_t i) {
  if (p.dim == 3) return ((double)(i / (p.nx * p.ny)) + 0.5) * p.hz;
  return ((double)((i / p.nx) % p.ny) + 0.5) * p.hy;
}

// One thread per cell: residual pair and block row of J.
__global__ void k_assemble(const DProb *probs, int32_t nprob, int32_t ncell, const double *u,
                           const double *u_old, double dt, const double *props, const int32_t *rowptr,
                           double *Jval, double *F) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DProb &p = probs[find_prob(probs, nprob, g)];
  const int32_t i = g - p.cell0;
  const double hz = p.dim == 3 ? p.hz : 1.0;
  const double V = p.hx * p.hy * hz;
  const double rho[2] = {p.rho_w, p.rho_n};
  const double pi = u[2 * (int64_t)g], si = u[2 * (int64_t)g + 1], so = u_old[2 * (int64_t)g + 1];
  double mi[6];
#pragma unroll
  for (int k = 0; k < 6; k++) mi[k] = props[6 * (int64_t)g + k];
  const double Di = depth(p, i);
  double Fw = V * (p.phi * p.rho_w * (1.0 - si) - p.phi * p.rho_w * (1.0 - so)) / dt;
  double Fn = V * (p.phi * p.rho_n * si - p.phi * p.rho_n * so) / dt;
  // block row accumulators: up to 7 blocks, diagonal at slot `kd`
  double blk[7][4];
#pragma unroll
  for (int k = 0; k < 7; k++) blk[k][0] = blk[k][1] = blk[k][2] = blk[k][3] = 0.0;
  int32_t nb[6];
  int dir[6];
  const int c = neighbours(p, i, nb, dir);
  int kd = 0;
  while (kd < c && nb[kd] < i) kd++;
  blk[kd][1] += -V * p.phi * p.rho_w / dt;
  blk[kd][3] += V * p.phi * p.rho_n / dt;
  for (int k = 0; k < c; k++) {
    const int32_t j = nb[k];
    const int32_t gj = p.cell0 + j;
    const int slot = k < kd ? k : k + 1;
    const int d = dir[k];
    const double ki = perm(p, d, i), kj = perm(p, d, j);
    const double kh = (ki + kj) > 0.0 ? 2.0 * ki * kj / (ki + kj) : 0.0;
    const double T = face_area(p, d) * kh / spacing(p, d);
    const double pj = u[2 * (int64_t)gj];
    double mj[6];
#pragma unroll
    for (int q = 0; q < 6; q++) mj[q] = props[6 * (int64_t)gj + q];
    const double Dj = depth(p, j);
#pragma unroll
    for (int a = 0; a < 2; a++) {
      const double phi_i = pi - rho[a] * p.g * Di + (a == 1 ? mi[4] : 0.0);
      const double phi_j = pj - rho[a] * p.g * Dj + (a == 1 ? mj[4] : 0.0);
      const double dphi = phi_i - phi_j;
      const bool up_i = dphi > 0.0;
      const double lam = up_i ? mi[a] : mj[a];
      const double dlam = up_i ? mi[2 + a] : mj[2 + a];
      const double cc = T * rho[a];
      const double flux = cc * lam * dphi;
      if (a == 0) Fw += flux; else Fn += flux;
      blk[kd][2 * a] += cc * lam;
      blk[slot][2 * a] += -cc * lam;
      if (a == 1) {
        blk[kd][3] += cc * lam * mi[5];
        blk[slot][3] += -cc * lam * mj[5];
      }
      if (up_i) blk[kd][2 * a + 1] += cc * dlam * dphi;
      else blk[slot][2 * a + 1] += cc * dlam * dphi;
    }
  }
  const int32_t ix = i % p.nx;
  if (ix == p.nx - 1 && (p.well_out < 0 || i == p.well_out)) {
    const double T = face_area(p, 0) * p.kx[i] / (0.5 * p.hx);
    double mb[6];
    constitutive(p, p.sn_out, mb);
#pragma unroll
    for (int a = 0; a < 2; a++) {
      const double phi_i = pi - rho[a] * p.g * Di + (a == 1 ? mi[4] : 0.0);
      const double phi_b = p.p_out - rho[a] * p.g * Di + (a == 1 ? mb[4] : 0.0);
      const double dphi = phi_i - phi_b;
      const bool up_i = dphi > 0.0;
      const double lam = up_i ? mi[a] : mb[a];
      const double cc = T * rho[a];
      const double flux = cc * lam * dphi;
      if (a == 0) Fw += flux; else Fn += flux;
      blk[kd][2 * a] += cc * lam;
      if (a == 1) blk[kd][3] += cc * lam * mi[5];
      if (up_i) blk[kd][2 * a + 1] += cc * mi[2 + a] * dphi;
    }
  }
  if (p.well_in < 0) {
    if (ix == 0) Fw -= p.rho_w * p.u_in * face_area(p, 0);
  } else if (i == p.well_in) {
    Fw -= p.rho_w * p.q_in;
  }
  F[2 * (int64_t)g] = Fw;
  F[2 * (int64_t)g + 1] = Fn;
  if (Jval) {
    double2 *out = reinterpret_cast<double2 *>(Jval + 4 * (int64_t)rowptr[g]);
    for (int k = 0; k <= c; k++) {
      out[2 * k] = make_double2(blk[k][0], blk[k][1]);
      out[2 * k + 1] = make_double2(blk[k][2], blk[k][3]);
    }
  }
}

// Checks one grid description and fills its device descriptor. Cell counts
// are formed in 64-bit integers: a product of dimensions that wraps in 32 bits
// would otherwise pass the limits and let the kernels index past the arrays.
static int check_grid(const rs_problem &q, int32_t k, int64_t cell0, DProb *out) {
  if (q.nx < 1 || q.ny < 1 || q.nz < 1 || (q.dim != 2 && q.dim != 3) || (q.dim == 2 && q.nz != 1))
    return fail(RS_EINVAL, "bad grid dimensions in problem " + std::to_string(k));
  const int64_t n = (int64_t)q.nx * (int64_t)q.ny * (int64_t)q.nz;
  if (n > kMaxCells || cell0 + n > kMaxCells)
    return fail(RS_EINVAL, "too many cells: problem " + std::to_string(k) + " brings the total to " +
                               std::to_string(cell0 + n) + ", above " + std::to_string(kMaxCells));
  if (!q.kx || !q.ky || (q.dim == 3 && !q.kz)) return fail(RS_EINVAL, "missing permeability");
  if (q.pc_model < 0 || q.pc_model > 2 || !(q.bc_lambda > 0) || !(q.mu_w > 0) || !(q.mu_n > 0))
    return fail(RS_EINVAL, "bad constitutive parameters");
  if (q.well_in < -1 || q.well_in >= n || q.well_out < -1 || q.well_out >= n ||
      (q.well_out >= 0 && q.well_out % q.nx != q.nx - 1))
    return fail(RS_EINVAL, "bad well cells in problem " + std::to_string(k));
  DProb &p = *out;
  p.dim = q.dim; p.nx = q.nx; p.ny = q.ny; p.nz = q.nz;
  p.hx = q.hx; p.hy = q.hy; p.hz = q.hz;
  p.kx = q.kx; p.ky = q.ky; p.kz = q.kz ? q.kz : q.kx;
  p.phi = q.phi; p.mu_w = q.mu_w; p.mu_n = q.mu_n; p.rho_w = q.rho_w; p.rho_n = q.rho_n; p.g = q.g;
  p.pc_model = q.pc_model; p.pc_p0 = q.pc_p0; p.pc_pd = q.pc_pd; p.bc_lambda = q.bc_lambda;
  p.s_wr = q.s_wr; p.s_nr = q.s_nr; p.u_in = q.u_in; p.p_out = q.p_out; p.sn_out = q.sn_out;
  p.q_in = q.q_in; p.well_in = q.well_in; p.well_out = q.well_out;
  p.cell0 = (int32_t)cell0;
  p.ncell = (int32_t)n;
  return 0;
}

static int upload_probs(const rs_problem *probs, int32_t nprob, DProb **d, int32_t *ncell, cudaStream_t s) {
  if (!probs || nprob < 1) return fail(RS_EINVAL, "no problem descriptions");
  std::vector<DProb> h(nprob);
  int64_t tot = 0;
  for (int32_t k = 0; k < nprob; k++) {
    RS_TRY(check_grid(probs[k], k, tot, &h[k]));
    tot += (int64_t)h[k].ncell;
  }
  *ncell = (int32_t)tot;
  RS_TRY(dalloc_n(d, (size_t)nprob, s));
  RS_CHECK_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(DProb) * nprob, cudaMemcpyHostToDevice, s));
  return 0;
}

}  // namespace rs

using namespace rs;

extern "C" int64_t rs_bsr2_nnzb(const rs_problem *probs, int32_t nprob) {
  if (!probs || nprob < 1) return -1;
  int64_t tot = 0;
  for (int32_t k = 0; k < nprob; k++) {
    const rs_problem &q = probs[k];
    int64_t nx = q.nx, ny = q.ny, nz = q.dim == 3 ? q.nz : 1;
    int64_t n = nx * ny * nz;
    int64_t faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + (q.dim == 3 ? nx * ny * (nz - 1) : 0);
    tot += n + 2 * faces;
  }
  return tot;
}

extern "C" int rs_bsr2_pattern(const rs_problem *probs, int32_t nprob, int32_t *row_ptr, int32_t *col,
                               cudaStream_t stream) {
  if (!row_ptr || !col) return fail(RS_EINVAL, "null output");
  DProb *d = nullptr;
  int32_t ncell = 0;
  RS_TRY(upload_probs(probs, nprob, &d, &ncell, stream));
  RS_COUNTED k_pattern_counts<<<grid_for(ncell), kBlock, 0, stream>>>(d, nprob, ncell, row_ptr);
  RS_TRY(exclusive_scan(row_ptr, row_ptr, ncell, stream, nullptr));
  RS_COUNTED k_pattern_fill<<<grid_for(ncell), kBlock, 0, stream>>>(d, nprob, ncell, row_ptr, col);
  dfree(d, stream);
  RS_CHECK_CUDA(cudaGetLastError());
  return RS_OK;
}

extern "C" int jacobian_assemble(const rs_problem *probs, int32_t nprob, const double *u, const double *u_old,
                                 double dt, rs_bsr2 *J, double *F, cudaStream_t stream) {
  if (!u || !u_old || !F) return fail(RS_EINVAL, "null vector");
  if (!(dt > 0)) return fail(RS_EINVAL, "dt must be positive");
  DProb *d = nullptr;
  int32_t ncell = 0;
  RS_TRY(upload_probs(probs, nprob, &d, &ncell, stream));
  if (J && (J->nb != ncell || !J->row_ptr || !J->val)) {
    dfree(d, stream);
    return fail(RS_EINVAL, "Jacobian does not match the grids");
  }
  double *props = nullptr;
  int r = dalloc_n(&props, 6 * (size_t)ncell, stream);
  if (r) { dfree(d, stream); return r; }
  RS_COUNTED k_props<<<grid_for(ncell), kBlock, 0, stream>>>(d, nprob, ncell, u, props);
  RS_COUNTED k_assemble<<<grid_for(ncell, 128), 128, 0, stream>>>(d, nprob, ncell, u, u_old, dt, props,
                                                      J ? J->row_ptr : nullptr, J ? J->val : nullptr, F);
  dfree(props, stream);
  dfree(d, stream);
  RS_CHECK_CUDA(cudaGetLastError());
  return RS_OK;
}

namespace rs {

// max over cells and phases of |F_a,i| dt / (V phi rho_a)
__global__ void k_scaled_fnorm(const DProb *probs, int32_t nprob, int32_t ncell, const double *F, double dt,
                               unsigned long long *out) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (g < ncell) {
    const DProb &p = probs[find_prob(probs, nprob, g)];
    const double V = p.hx * p.hy * (p.dim == 3 ? p.hz : 1.0);
    const double a = fabs(F[2 * (int64_t)g]) * dt / (V * p.phi * p.rho_w);
    const double b = fabs(F[2 * (int64_t)g + 1]) * dt / (V * p.phi * p.rho_n);
    v = a > b ? a : b;
    if (!(v == v)) v = __longlong_as_double(0x7ff0000000000000ll);   // NaN counts as infinite
  }
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
}

// u += sign * du, the S_n change cut to [-max_ds, max_ds] when max_ds > 0;
// S_n clamped to [0, 1 - S_wr - 1e-12]
__global__ void k_newton_update(const DProb *probs, int32_t nprob, int32_t ncell, const double *du, double sign,
                                double max_ds, double *u) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DProb &p = probs[find_prob(probs, nprob, g)];
  const double smax = 1.0 - p.s_wr - 1e-12;
  u[2 * (int64_t)g] += sign * du[2 * (int64_t)g];
  double ds = sign * du[2 * (int64_t)g + 1];
  if (max_ds > 0.0) ds = ds < -max_ds ? -max_ds : (ds > max_ds ? max_ds : ds);
  double sn = u[2 * (int64_t)g + 1] + ds;
  sn = sn < 0.0 ? 0.0 : (sn > smax ? smax : sn);
  u[2 * (int64_t)g + 1] = sn;
}

int scaled_fnorm(const rs_problem *probs, int32_t nprob, const double *F, double dt, double *out,
                 cudaStream_t s) {
  DProb *d = nullptr;
  int32_t ncell = 0;
  RS_TRY(upload_probs(probs, nprob, &d, &ncell, s));
  unsigned long long *acc = nullptr;
  RS_TRY(dalloc_n(&acc, 1, s));
  RS_CHECK_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
  if (ncell > 0) RS_COUNTED k_scaled_fnorm<<<grid_for(ncell), kBlock, 0, s>>>(d, nprob, ncell, F, dt, acc);
  unsigned long long h = 0;
  RS_CHECK_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  RS_CHECK_CUDA(cudaStreamSynchronize(s));
  dfree(acc, s);
  dfree(d, s);
  double v;
  memcpy(&v, &h, sizeof(v));
  *out = v;
  return 0;
}

int newton_update(const rs_problem *probs, int32_t nprob, const double *du, double sign, double max_ds, double *u,
                  cudaStream_t s) {
  DProb *d = nullptr;
  int32_t ncell = 0;
  RS_TRY(upload_probs(probs, nprob, &d, &ncell, s));
  if (ncell > 0) RS_COUNTED k_newton_update<<<grid_for(ncell), kBlock, 0, s>>>(d, nprob, ncell, du, sign, max_ds, u);
  dfree(d, s);
  RS_CHECK_CUDA(cudaGetLastError());
  return 0;
}

}  // namespace rs

// ------------------------------------------------------------------------
// Assembly without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual and Jacobian: code running while another component owns the
// device allocator (a framework that forbids outside cudaMalloc, or one whose
// memory is fully reserved), latency-critical loops where an allocation (and
// the synchronisation it can imply) is not acceptable, or memory-capped
// processes. For them, jacobian_assemble_noalloc does the same work as
// jacobian_assemble with its scratch (the per-cell constitutive table and the
// grid descriptors) held in fixed-size arrays that live in the library's
// device image, so the call itself allocates nothing on the device. The
// descriptors reach the device as a kernel parameter, not through a copy
// from host memory.
//
// Limits: at most kNoAllocMaxCells cells and kNoAllocMaxGrids grids per call.
// The arrays exist once per device for as long as the library is loaded
// (about 3.2 MB of device memory on every GPU that loads it). Each call
// overwrites them entirely (nothing has to start at zero); calls that overlap
// on the GPU (concurrent streams, threads) share the arrays and race.
namespace rs {
namespace {

constexpr int32_t kNoAllocMaxCells = 65536;
constexpr int32_t kNoAllocMaxGrids = 64;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_props[6 * kNoAllocMaxCells];
static __device__ __align__(256) DProb g_noalloc_grids[kNoAllocMaxGrids];

// The grid descriptors of one call, passed by value as a kernel parameter
// (64 descriptors of 208 bytes: within the 32 KB parameter limit).
struct NoAllocGridPack {
  DProb g[kNoAllocMaxGrids];
};
static_assert(sizeof(NoAllocGridPack) <= 32000, "grid pack exceeds the kernel parameter limit");

// Copies the first n descriptors of the parameter into the fixed array.
__global__ void k_noalloc_grids(const __grid_constant__ NoAllocGridPack pack, int32_t n) {
  const int i = threadIdx.x;
  if (i < n) g_noalloc_grids[i] = pack.g[i];
}

struct NoAllocPtrs {
  double *props = nullptr;
  DProb *grids = nullptr;
  bool ready = false;
};
static NoAllocPtrs g_noalloc_ptrs[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Device addresses of the two arrays for the current device, looked up once
// per device (the array names are host-side stand-ins, not device addresses).
int noalloc_ptrs(NoAllocPtrs *out) {
  int dev = 0;
  RS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(RS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocPtrs &p = g_noalloc_ptrs[dev];
  if (!p.ready) {
    void *a = nullptr, *b = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_props);
    if (e != cudaSuccess) return fail(RS_ECUDA, std::string("cudaGetSymbolAddress(props): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&b, g_noalloc_grids);
    if (e != cudaSuccess) return fail(RS_ECUDA, std::string("cudaGetSymbolAddress(grids): ") + cudaGetErrorString(e));
    p.props = static_cast<double *>(a);
    p.grids = static_cast<DProb *>(b);
    p.ready = true;
  }
  *out = p;
  return 0;
}

}  // namespace
}  // namespace rs

extern "C" int jacobian_assemble_noalloc(const rs_problem *probs, int32_t nprob, const double *u,
                                         const double *u_old, double dt, rs_bsr2 *J, double *F,
                                         cudaStream_t stream) {
  if (!u || !u_old || !F) return fail(RS_EINVAL, "null vector");
  if (!(dt > 0)) return fail(RS_EINVAL, "dt must be positive");
  if (!probs || nprob < 1) return fail(RS_EINVAL, "no problem descriptions");
  if (nprob > kNoAllocMaxGrids)
    return fail(RS_EINVAL, "jacobian_assemble_noalloc: " + std::to_string(nprob) + " grids exceed the limit of " +
                               std::to_string(kNoAllocMaxGrids));
  NoAllocGridPack pack;
  int64_t tot = 0;
  for (int32_t k = 0; k < nprob; k++) {
    RS_TRY(check_grid(probs[k], k, tot, &pack.g[k]));
    tot += (int64_t)pack.g[k].ncell;
    if (tot > kNoAllocMaxCells)
      return fail(RS_EINVAL, "jacobian_assemble_noalloc: " + std::to_string(tot) +
                                 " cells exceed the limit of " + std::to_string(kNoAllocMaxCells));
  }
  const int32_t ncell = (int32_t)tot;
  if (J && (J->nb != ncell || !J->row_ptr || !J->val)) return fail(RS_EINVAL, "Jacobian does not match the grids");
  NoAllocPtrs d;
  RS_TRY(noalloc_ptrs(&d));
  // The descriptors travel as a kernel parameter (copied at launch), so no
  // host buffer has to outlive this call.
  RS_COUNTED k_noalloc_grids<<<1, kNoAllocMaxGrids, 0, stream>>>(pack, nprob);
  RS_COUNTED k_props<<<grid_for(ncell), kBlock, 0, stream>>>(d.grids, nprob, ncell, u, d.props);
  RS_COUNTED k_assemble<<<grid_for(ncell, 128), 128, 0, stream>>>(d.grids, nprob, ncell, u, u_old, dt, d.props,
                                                                 J ? J->row_ptr : nullptr, J ? J->val : nullptr, F);
  RS_CHECK_CUDA(cudaGetLastError());
  return RS_OK;
}
