// Preconditioners M ~ J for the right-preconditioned Krylov solve (Sec. 3):
//   AMG_J : one scalar V-cycle on the point-ordered J (Sec. 3.2).
//   CPR1  : Algorithm 1. u = P1^{-1} r; r' = r - J u; A_pp dp = R_p r' (one
//           V-cycle); u += R_p^T dp.
//   CPR2  : Algorithm 2. CPR1 plus A_ss ds = R_s r' (one V-cycle), u += R_s^T ds.
//   BF    : Algorithm 3. A_ss s = R_s r (one V-cycle); r_p = R_p r - A_ps s;
//           S~ p = r_p (one V-cycle), S~ = A_pp - A_ps diag(A_ss)^{-1} A_sp
//           (eq. SIMPLE-Schur read with A_sp).
// CPR with decoupling W (per-cell 2x2: ABF D^{-1}, or quasi-IMPES
// [1, -a_ps,ii/a_ss,ii; 0, 1]) runs Algorithm 1/2 on W J and W r. P1 is the
// point-block Jacobi inverse of W J's diagonal blocks (p1 = 0, the parallel
// stand-in) or the paper's ILU(0) of the point-ordered W J (p1 = 1,
// level-scheduled factorisation and triangular solves).
//
// Glue kernels work in FP64 on interleaved (P_w, S_n) vectors; the V-cycles
// take FP64 in and out and run in the hierarchy's precision.
#include "rs_internal.cuh"

namespace rs {
int decouple_qimpes(const rs_bsr2 &J, double *out, double *w, cudaStream_t s);
int decouple_abf(const rs_bsr2 &J, double *out, double *dinv, cudaStream_t s);
int block_diag_inverse(const rs_bsr2 &J, double *dinv, cudaStream_t s);
}  // namespace rs

using namespace rs;

struct rs_precond {
  rs_precond_params prm;
  rs_bsr2 J;                       // caller's matrix (kept by reference)
  std::vector<int32_t> seg_off;    // block-row offsets
  int32_t nb = 0;
  double *qw = nullptr;            // quasi-IMPES weights [nb]
  double *dinv = nullptr;          // ABF D^{-1} blocks [4 nb]
  double *p1inv = nullptr;         // P1^{-1} blocks [4 nb] (point-block Jacobi)
  rs_ilu0 *ilu = nullptr;          // P1 = ILU(0) of W J
  uint8_t *act = nullptr;          // batches: per-system live flags read by the V-cycles (1 = live)
  int32_t *rseg = nullptr;         // batches: the system of every block row (glue kernels)
  Hier Hp, Hs, Hj;
  bool has_p = false, has_s = false, has_j = false;
  DCsr Aps;                        // BF coupling block
  double *rt = nullptr, *sb = nullptr, *ss = nullptr, *sx = nullptr, *sy = nullptr;
  cudaStream_t stream;
  // the apply sequence recorded once as a CUDA graph (on a private stream,
  // between fixed input/output buffers) and replayed on the caller's stream
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  double *gin = nullptr, *gout = nullptr;
  long long napply = 0;
  long long graph_launches = 0;
  bool use_graph = true;
};

namespace {

// Batches: block row i belongs to a retired system (its flag is 0); the glue
// kernels then write zeros for it without reading its data, as the V-cycles
// do (act == nullptr: a single system, never retired).
__device__ __forceinline__ bool retired(const uint8_t *act, const int32_t *rseg, int64_t i) {
  return act != nullptr && !act[rseg[i]];
}

// rt = W r; z = P1^{-1} rt when P1 is point-block Jacobi (p1inv != NULL)
__global__ void k_cpr_stage1(int32_t nb, int mode, const double *qw, const double *dinv, const double *p1inv,
                             const double *r, double *rt, double *z, const uint8_t *act, const int32_t *rseg) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  if (retired(act, rseg, i)) {
    reinterpret_cast<double2 *>(rt)[i] = make_double2(0.0, 0.0);
    if (p1inv) reinterpret_cast<double2 *>(z)[i] = make_double2(0.0, 0.0);
    return;
  }
  const double2 rv = reinterpret_cast<const double2 *>(r)[i];
  double2 t = rv;
  if (mode == RS_DECOUPLE_QIMPES) {
    t.x = rv.x + qw[i] * rv.y;
  } else if (mode == RS_DECOUPLE_ABF) {
    const double *d = dinv + 4 * (int64_t)i;
    t.x = d[0] * rv.x + d[1] * rv.y;
    t.y = d[2] * rv.x + d[3] * rv.y;
  }
  reinterpret_cast<double2 *>(rt)[i] = t;
  if (!p1inv) return;
  const double *p = p1inv + 4 * (int64_t)i;
  reinterpret_cast<double2 *>(z)[i] = make_double2(p[0] * t.x + p[1] * t.y, p[2] * t.x + p[3] * t.y);
}

// r' = rt - W (J z), split into its pressure (sb) and saturation (ss) parts
template <int LPR>
__global__ void __launch_bounds__(256) k_cpr_resid(int32_t nb, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ col, const double *__restrict__ val,
                                                   const double *__restrict__ z, const double *__restrict__ rt,
                                                   int mode, const double *__restrict__ qw,
                                                   const double *__restrict__ dinv, double *__restrict__ sb,
                                                   double *__restrict__ ss, const uint8_t *__restrict__ act,
                                                   const int32_t *__restrict__ rseg) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / LPR;
  const int lane = threadIdx.x % LPR;
  double y0 = 0.0, y1 = 0.0;
  const bool live = row < nb && !retired(act, rseg, row);
  if (live) {
    const int32_t e = rowptr[row + 1];
    for (int32_t k = rowptr[row] + lane; k < e; k += LPR) {
      const double2 v01 = reinterpret_cast<const double2 *>(val)[2 * (int64_t)k];
      const double2 v23 = reinterpret_cast<const double2 *>(val)[2 * (int64_t)k + 1];
      const double2 xv = reinterpret_cast<const double2 *>(z)[col[k]];
      y0 = fma(v01.x, xv.x, fma(v01.y, xv.y, y0));
      y1 = fma(v23.x, xv.x, fma(v23.y, xv.y, y1));
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) {
    y0 += __shfl_down_sync(0xffffffffu, y0, o, LPR);
    y1 += __shfl_down_sync(0xffffffffu, y1, o, LPR);
  }
  if (row < nb && lane == 0 && !live) {
    sb[row] = 0.0;
    if (ss) ss[row] = 0.0;
  } else if (row < nb && lane == 0) {
    double w0 = y0, w1 = y1;
    if (mode == RS_DECOUPLE_QIMPES) {
      w0 = y0 + qw[row] * y1;
    } else if (mode == RS_DECOUPLE_ABF) {
      const double *d = dinv + 4 * row;
      w0 = d[0] * y0 + d[1] * y1;
      w1 = d[2] * y0 + d[3] * y1;
    }
    const double2 t = reinterpret_cast<const double2 *>(rt)[row];
    sb[row] = t.x - w0;
    if (ss) ss[row] = t.y - w1;
  }
}

__global__ void k_cpr_update(int32_t nb, const double *dp, const double *ds, double *z, const uint8_t *act,
                             const int32_t *rseg) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb || retired(act, rseg, i)) return;
  z[2 * (int64_t)i] += dp[i];
  if (ds) z[2 * (int64_t)i + 1] += ds[i];
}

__global__ void k_take(int32_t nb, const double *r, int comp, double *out, const uint8_t *act,
                       const int32_t *rseg) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) out[i] = retired(act, rseg, i) ? 0.0 : r[2 * (int64_t)i + comp];
}

// rp_i = r_{2i} - (A_ps s)_i
// one thread per row (rows of A_ps hold a handful of entries; no FP64
// shuffle additions)
__global__ void k_bf_rp(int32_t nb, const int32_t *rp, const int32_t *col, const double *val, const double *s,
                        const double *r, double *out, const uint8_t *act, const int32_t *rseg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  if (retired(act, rseg, i)) {
    out[i] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int32_t k = rp[i]; k < rp[i + 1]; k++) acc = fma(val[k], s[col[k]], acc);
  out[i] = r[2 * i] - acc;
}

__global__ void k_interleave(int32_t nb, const double *p, const double *s, double *z, const uint8_t *act,
                             const int32_t *rseg) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb)
    reinterpret_cast<double2 *>(z)[i] = retired(act, rseg, i) ? make_double2(0.0, 0.0) : make_double2(p[i], s[i]);
}

std::vector<int32_t> dof_offsets(const std::vector<int32_t> &blk) {
  std::vector<int32_t> o(blk.size());
  for (size_t k = 0; k < blk.size(); k++) o[k] = 2 * blk[k];
  return o;
}

int build(rs_precond *M, cudaStream_t s) {
  const rs_bsr2 &J = M->J;
  const int32_t nb = J.nb;
  const rs_precond_params &p = M->prm;
  const int kind = p.kind;
  if (nb == 0) return 0;   // empty system: applying M is a no-op
  const int32_t nseg = (int32_t)M->seg_off.size() - 1;
  if (nseg > 1) {
    RS_TRY(dalloc_n(&M->act, (size_t)nseg, s));
    RS_CHECK_CUDA(cudaMemsetAsync(M->act, 1, (size_t)nseg, s));
    RS_TRY(seg_ids(M->seg_off, nb, &M->rseg, s));
  }
  RS_TRY(dalloc_n(&M->rt, 2 * (size_t)nb, s));
  RS_TRY(dalloc_n(&M->sb, (size_t)nb, s));
  RS_TRY(dalloc_n(&M->ss, (size_t)nb, s));
  RS_TRY(dalloc_n(&M->sx, (size_t)nb, s));
  RS_TRY(dalloc_n(&M->sy, (size_t)nb, s));
  if (kind == RS_PC_AMG_J || kind == RS_PC_AMG_J_SCALAR) {
    // black-box AMG on the point-ordered J (Sec. 3.2): the point method with
    // (p_w, S_n) per cell, or unknown-agnostic scalar AMG
    DCsr A;
    RS_TRY(bsr2_scalar(J, A, s));
    rs_amg_params ap = p.amg;
    ap.num_functions = kind == RS_PC_AMG_J ? 2 : 1;
    int r = amg_build(A, dof_offsets(M->seg_off), ap, M->Hj, s);
    dcsr_free(A, s);
    if (r) return r;
    M->has_j = true;
    M->Hj.active = M->act;
    return 0;
  }
  if (kind == RS_PC_CPR1 || kind == RS_PC_CPR2) {
    Scratch sc(s);
    rs_bsr2 Jt = J;
    double *jt = nullptr;
    if (p.decouple == RS_DECOUPLE_QIMPES) {
      RS_TRY(sc.get(&jt, 4 * (size_t)J.nnzb));
      RS_TRY(dalloc_n(&M->qw, (size_t)nb, s));
      RS_TRY(decouple_qimpes(J, jt, M->qw, s));
      Jt.val = jt;
    } else if (p.decouple == RS_DECOUPLE_ABF) {
      RS_TRY(sc.get(&jt, 4 * (size_t)J.nnzb));
      RS_TRY(dalloc_n(&M->dinv, 4 * (size_t)nb, s));
      RS_TRY(decouple_abf(J, jt, M->dinv, s));
      Jt.val = jt;
    }
    if (p.p1 == RS_P1_ILU0) {
      RS_TRY(ilu0_build(Jt, p.amg.precision, &M->ilu, s));   // solves in the V-cycle precision
    } else {
      RS_TRY(dalloc_n(&M->p1inv, 4 * (size_t)nb, s));
      RS_TRY(block_diag_inverse(Jt, M->p1inv, s));
    }
    DCsr App;
    RS_TRY(bsr2_part(Jt, 0, 0, App, s));
    int r = amg_build(App, M->seg_off, p.amg, M->Hp, s);
    dcsr_free(App, s);
    if (r) return r;
    M->has_p = true;
    M->Hp.active = M->act;
    if (kind == RS_PC_CPR2) {
      DCsr Ass;
      RS_TRY(bsr2_part(Jt, 1, 1, Ass, s));
      r = amg_build(Ass, M->seg_off, p.amg, M->Hs, s);
      dcsr_free(Ass, s);
      if (r) return r;
      M->has_s = true;
      M->Hs.active = M->act;
    }
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    return 0;
  }
  // block factorisation
  DCsr App, Asp, Ass, S;
  RS_TRY(bsr2_part(J, 0, 0, App, s));
  RS_TRY(bsr2_part(J, 0, 1, M->Aps, s));
  RS_TRY(bsr2_part(J, 1, 0, Asp, s));
  RS_TRY(bsr2_part(J, 1, 1, Ass, s));
  int r = simple_schur(App, M->Aps, Asp, Ass, S, s);
  if (!r) r = amg_build(Ass, M->seg_off, p.amg, M->Hs, s);
  if (!r) { M->has_s = true; M->Hs.active = M->act; r = amg_build(S, M->seg_off, p.amg, M->Hp, s); }
  if (!r) { M->has_p = true; M->Hp.active = M->act; }
  dcsr_free(App, s);
  dcsr_free(Asp, s);
  dcsr_free(Ass, s);
  dcsr_free(S, s);
  return r;
}

void destroy(rs_precond *M) {
  cudaStream_t s = M->stream;
  cudaStreamSynchronize(s);
  if (M->exec) cudaGraphExecDestroy(M->exec);
  if (M->cap_stream) cudaStreamDestroy(M->cap_stream);
  dfree(M->gin, s);
  dfree(M->gout, s);
  if (M->has_p) amg_free(M->Hp, s);
  if (M->has_s) amg_free(M->Hs, s);
  if (M->has_j) amg_free(M->Hj, s);
  dcsr_free(M->Aps, s);
  dfree(M->qw, s);
  dfree(M->dinv, s);
  dfree(M->p1inv, s);
  dfree(M->act, s);
  dfree(M->rseg, s);
  ilu0_free(M->ilu);
  dfree(M->rt, s);
  dfree(M->sb, s);
  dfree(M->ss, s);
  dfree(M->sx, s);
  dfree(M->sy, s);
  cudaStreamSynchronize(s);
  delete M;
}

}  // namespace

namespace rs {
static int apply_body(const rs_precond *M, const double *r, double *z, cudaStream_t s) {
  const int32_t nb = M->nb;
  if (nb == 0) return 0;
  const unsigned g = grid_for(nb);
  switch (M->prm.kind) {
    case RS_PC_AMG_J:
    case RS_PC_AMG_J_SCALAR:
      return amg_vcycle(M->Hj, r, z, s);
    case RS_PC_BF: {
      RS_COUNTED k_take<<<g, kBlock, 0, s>>>(nb, r, 1, M->sb, M->act, M->rseg);
      RS_TRY(amg_vcycle(M->Hs, M->sb, M->sx, s));                 // A_ss s = R_s r
      RS_COUNTED k_bf_rp<<<grid_for((int64_t)nb), kBlock, 0, s>>>(nb, M->Aps.rowptr, M->Aps.col, M->Aps.val, M->sx, r,
                                                           M->ss, M->act, M->rseg);    // r_p = R_p r - A_ps s
      RS_TRY(amg_vcycle(M->Hp, M->ss, M->sy, s));                 // S~ p = r_p
      RS_COUNTED k_interleave<<<g, kBlock, 0, s>>>(nb, M->sy, M->sx, z, M->act, M->rseg);
      RS_CHECK_CUDA(cudaGetLastError());
      return 0;
    }
    default: {
      const int mode = M->prm.decouple;
      const bool two = M->prm.kind == RS_PC_CPR2;
      RS_COUNTED k_cpr_stage1<<<g, kBlock, 0, s>>>(nb, mode, M->qw, M->dinv, M->p1inv, r, M->rt, z, M->act, M->rseg);
      if (M->ilu) RS_TRY(ilu0_solve(M->ilu, M->rt, z, s));
      {
        ProfScope ps(kProfBsr2, M->J.nnzb * 36.0 + (nb + 1) * 4.0 + nb * (16.0 + 16.0 + 16.0), s);
        // one lane per block row: on GB300 every FP64 shuffle addition costs
        // FP64-pipe time, and a row's blocks share cache lines
        RS_COUNTED k_cpr_resid<1><<<grid_for((int64_t)nb), kBlock, 0, s>>>(
            nb, M->J.row_ptr, M->J.col, M->J.val, z, M->rt, mode, M->qw, M->dinv, M->sb, two ? M->ss : nullptr, M->act,
            M->rseg);
      }
      RS_TRY(amg_vcycle(M->Hp, M->sb, M->sx, s));
      if (two) RS_TRY(amg_vcycle(M->Hs, M->ss, M->sy, s));
      RS_COUNTED k_cpr_update<<<g, kBlock, 0, s>>>(nb, M->sx, two ? M->sy : nullptr, z, M->act, M->rseg);
      RS_CHECK_CUDA(cudaGetLastError());
      return 0;
    }
  }
}

// Batches: the V-cycles of the next applies skip (write zeros for) the
// systems whose flag in `active` (nseg bytes, device) is 0.
int precond_set_active(const rs_precond *M, const uint8_t *active, cudaStream_t s) {
  if (!M->act || !active) return 0;
  RS_CHECK_CUDA(cudaMemcpyAsync(M->act, active, M->seg_off.size() - 1, cudaMemcpyDeviceToDevice, s));
  return 0;
}

int precond_apply_impl(const rs_precond *Mc, const double *r, double *z, cudaStream_t s) {
  rs_precond *M = const_cast<rs_precond *>(Mc);
  const size_t bytes = sizeof(double) * 2 * (size_t)M->nb;
  if (M->nb == 0) return 0;
  if (profiling()) {
    M->napply++;
    return apply_body(M, r, z, s);
  }
  if (M->use_graph && !M->exec && M->napply >= 1) {
    // record the apply once; the first apply ran eagerly (kernel attributes set)
    if (!M->cap_stream) RS_CHECK_CUDA(cudaStreamCreateWithFlags(&M->cap_stream, cudaStreamNonBlocking));
    if (!M->gin) RS_TRY(dalloc_n(&M->gin, 2 * (size_t)M->nb, s));
    if (!M->gout) RS_TRY(dalloc_n(&M->gout, 2 * (size_t)M->nb, s));
    RS_CHECK_CUDA(cudaStreamSynchronize(s));
    cudaGraph_t g = nullptr;
    RS_CHECK_CUDA(cudaStreamBeginCapture(M->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long l0 = rs_launch_count();
    int rc = apply_body(M, M->gin, M->gout, M->cap_stream);
    cudaError_t e = cudaStreamEndCapture(M->cap_stream, &g);
    M->graph_launches = rs_launch_count() - l0;
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      M->use_graph = false;
    } else {
      e = cudaGraphInstantiate(&M->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { cudaGetLastError(); M->exec = nullptr; M->use_graph = false; }
    }
  }
  M->napply++;
  if (M->exec) {
    RS_CHECK_CUDA(cudaMemcpyAsync(M->gin, r, bytes, cudaMemcpyDeviceToDevice, s));
    RS_CHECK_CUDA(cudaGraphLaunch(M->exec, s));
    count_launches(M->graph_launches);
    RS_CHECK_CUDA(cudaMemcpyAsync(z, M->gout, bytes, cudaMemcpyDeviceToDevice, s));
    return 0;
  }
  return apply_body(M, r, z, s);
}
}  // namespace rs

extern "C" int precond_create(const rs_bsr2 *J, const rs_precond_params *params, rs_precond **out,
                              cudaStream_t stream) {
  if (!out) return fail(RS_EINVAL, "null output handle");
  *out = nullptr;
  if (!J || !params || J->nb < 0 || J->nnzb < 0 || (J->nb > 0 && (!J->row_ptr || !J->col || !J->val)))
    return fail(RS_EINVAL, "invalid arguments");
  if (params->kind < RS_PC_AMG_J || params->kind > RS_PC_AMG_J_SCALAR)
    return fail(RS_EINVAL, "unknown preconditioner kind");
  if (params->decouple < RS_DECOUPLE_NONE || params->decouple > RS_DECOUPLE_QIMPES)
    return fail(RS_EINVAL, "unknown decoupling");
  if (params->p1 != RS_P1_BLOCK_JACOBI && params->p1 != RS_P1_ILU0) return fail(RS_EINVAL, "unknown P1");
  RS_TRY(check_amg_params(params->amg));
  rs_precond *M = new rs_precond();
  M->prm = *params;
  M->J = *J;
  M->nb = J->nb;
  M->seg_off = seg_offsets(J->nb, J->nseg, J->seg_off);
  M->J.seg_off = nullptr;
  M->stream = stream;
  if (M->seg_off.front() != 0 || M->seg_off.back() != J->nb) {
    delete M;
    return fail(RS_EINVAL, "segment offsets must run from 0 to nb");
  }
  int r = build(M, stream);
  if (r) {
    destroy(M);
    return r;
  }
  *out = M;
  return RS_OK;
}

extern "C" int precond_destroy(rs_precond *M) {
  if (M) destroy(M);
  return RS_OK;
}

extern "C" int precond_apply(const rs_precond *M, const double *r, double *z, cudaStream_t stream) {
  if (!M || ((!r || !z) && M->nb > 0)) return fail(RS_EINVAL, "null argument");
  return precond_apply_impl(M, r, z, stream);
}

extern "C" const rs_amg *precond_amg(const rs_precond *M, int32_t which) {
  if (!M) return nullptr;
  // views into the preconditioner's hierarchies (owned by M)
  static thread_local rs_amg view[3];
  const Hier *h = nullptr;
  if (which == 0) h = M->has_j ? &M->Hj : (M->has_p ? &M->Hp : nullptr);
  else if (which == 1) h = M->has_s ? &M->Hs : nullptr;
  if (!h) return nullptr;
  rs_amg *v = &view[which];
  v->H = *h;
  v->stream = M->stream;
  return v;
}
