/*
 * Oracle, part 3: classical algebraic multigrid (Sec. 3.2; solver settings of
 * Sec. 4: one V-cycle, classical Ruge-Stueben interpolation, Gauss-Seidel
 * smoothing). TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings and stated deviations (the same in the CUDA library):
 *  - Strength: with s_i = -1 if a_ii < 0 else +1, j != i is strong for i iff
 *    -s_i a_ij >= theta * max_{k != i} (-s_i a_ik) and that maximum is > 0.
 *  - Coarsening: PMIS (De Sterck, Yang, Heys 2006) in place of the paper's
 *    CLJP. Measure key_i = (|S^T_i| << 24) | (24 random bits); i beats j iff
 *    key_i > key_j, or equal keys and i < j. Points no one depends on become
 *    F. Each round, an undecided point that beats every undecided neighbour
 *    in S u S^T becomes C; then every undecided point that strongly depends
 *    on a new C point becomes F.
 *  - Random bits: SplitMix64 (Steele, Lea, Flood 2014): the c-th output for
 *    seed s is mix(s + (c + 1) * 0x9E3779B97F4A7C15). PMIS uses counter
 *    c = ((2 l) << 32) + i, colouring c = ((2 l + 1) << 32) + i at level l.
 *  - Interpolation: classical (direct plus distribution of strong F
 *    neighbours through the common C points), with only the entries of row m
 *    whose sign is opposite to a_mm distributed. Weak neighbours and strong F
 *    neighbours that share no C point are added to the diagonal. An F point
 *    with no strong C neighbour gets an empty row.
 *  - Galerkin coarse operator A_c = P^T (A P), both products by ascending
 *    inner index.
 *  - Smoother: hybrid multicolour Gauss-Seidel (the default, smoother = 2):
 *    the rows are cut into consecutive chunks of `chunk` rows; inside a chunk
 *    Gauss-Seidel runs colour by colour (Jones-Plassmann colouring of the
 *    symmetrised pattern, each point taking the lowest colour unused by its
 *    already coloured neighbours, colours ascending) on the newest values,
 *    while couplings to other chunks use the values from the start of the
 *    sweep. This is the paper's hybrid Gauss-Seidel with a chunk of rows in
 *    place of an MPI process. Alternatives: plain multicolour Gauss-Seidel
 *    over the whole level (smoother = 0) and l1-Jacobi (smoother = 1). Pre-
 *    and post-smoothing sweep the colours in the same ascending order.
 *  - Coarsest level: dense LU with partial pivoting.
 *  - Systems ("point") AMG, num_functions = b = 2 (Sec. 3.2: BoomerAMG on the
 *    Jacobian ordered by grid points, the point method of Stueben et al.):
 *    the unknowns are interleaved, b per point (row b*i + f is function f of
 *    point i). Each level coarsens the points by strength and PMIS on the
 *    function-0 (pressure) part A_00, the primary unknown; every unknown of a
 *    C point is a C unknown. Each function f is interpolated only from the
 *    same function at C points, with the weights of the interpolation of
 *    A_ff under the point splitting; couplings between functions enter only
 *    through the Galerkin product with the whole matrix. The smoother is the
 *    point-block hybrid Gauss-Seidel: chunks of consecutive points, points
 *    coloured first-fit inside the chunk, each point's b x b diagonal block
 *    solved with its inverse (no update where that block is singular).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

or_csr *or_csr_alloc(int32_t n, int32_t m, int32_t nnz);

static void *xmalloc(size_t n) {
  void *p = malloc(n ? n : 1);
  if (!p) abort();
  return p;
}

uint64_t or_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double diag_of(const or_csr *A, int32_t i) {
  for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
    if (A->col[k] == i) return A->val[k];
  return 0.0;
}

/* nfun > 1: unknown-based strength (hypre's "num_functions"): only entries
 * coupling unknowns of the same kind (i mod nfun == j mod nfun) compete. */
void or_strength_nf(const or_csr *A, double theta, int32_t nfun, uint8_t *strong) {
  if (nfun < 1) nfun = 1;
  for (int32_t i = 0; i < A->n; i++) {
    double s = diag_of(A, i) < 0.0 ? -1.0 : 1.0;
    double mx = 0.0;
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      if (A->col[k] == i || A->col[k] % nfun != i % nfun) continue;
      double v = -(s * A->val[k]);
      if (v > mx) mx = v;
    }
    double thr = theta * mx;
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      strong[k] = 0;
      if (A->col[k] == i || A->col[k] % nfun != i % nfun || !(mx > 0.0)) continue;
      double v = -(s * A->val[k]);
      if (v >= thr) strong[k] = 1;
    }
  }
}

void or_strength(const or_csr *A, double theta, uint8_t *strong) { or_strength_nf(A, theta, 1, strong); }

static int beats(uint64_t ki, int32_t i, uint64_t kj, int32_t j) {
  return ki > kj || (ki == kj && i < j);
}

/* cf: 1 = C, -1 = F. */
void or_pmis(const or_csr *A, const uint8_t *strong, uint64_t seed, int32_t level, int8_t *cf) {
  int32_t n = A->n;
  int32_t *lam = xmalloc(sizeof(int32_t) * (size_t)n);
  uint64_t *key = xmalloc(sizeof(uint64_t) * (size_t)n);
  int8_t *newc = xmalloc((size_t)n);
  memset(lam, 0, sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < n; i++)
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
      if (strong[k]) lam[A->col[k]]++;
  /* S^T adjacency, so each point can see who depends on it */
  int32_t *tp = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  memset(tp, 0, sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t i = 0; i < n; i++)
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
      if (strong[k]) tp[A->col[k] + 1]++;
  for (int32_t i = 0; i < n; i++) tp[i + 1] += tp[i];
  int32_t *tc = xmalloc(sizeof(int32_t) * ((size_t)tp[n] + 1));
  int32_t *fill = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  memcpy(fill, tp, sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < n; i++)
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
      if (strong[k]) tc[fill[A->col[k]]++] = i;
  int32_t undecided = 0;
  for (int32_t i = 0; i < n; i++) {
    uint64_t r = or_splitmix64(seed, ((uint64_t)(2 * level) << 32) + (uint64_t)i);
    key[i] = ((uint64_t)lam[i] << 24) | (r >> 40);
    if (lam[i] == 0) cf[i] = -1;
    else { cf[i] = 0; undecided++; }
  }
  while (undecided > 0) {
    for (int32_t i = 0; i < n; i++) {
      newc[i] = 0;
      if (cf[i] != 0) continue;
      int ok = 1;
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1] && ok; k++) {
        int32_t j = A->col[k];
        if (strong[k] && cf[j] == 0 && !beats(key[i], i, key[j], j)) ok = 0;
      }
      for (int32_t q = tp[i]; q < tp[i + 1] && ok; q++) {
        int32_t j = tc[q];
        if (cf[j] == 0 && !beats(key[i], i, key[j], j)) ok = 0;
      }
      newc[i] = (int8_t)ok;
    }
    for (int32_t i = 0; i < n; i++)
      if (newc[i]) { cf[i] = 1; undecided--; }
    for (int32_t i = 0; i < n; i++) {
      if (cf[i] != 0) continue;
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
        if (strong[k] && newc[A->col[k]]) { cf[i] = -1; undecided--; break; }
    }
  }
  free(lam); free(key); free(newc); free(tp); free(tc); free(fill);
}

/* Classical interpolation; see the header comment for the reading. Row i of
 * P for an F point, with C_i its strong C neighbours:
 *   pass A over row i in ascending column order accumulates the diagonal
 *     dacc from a_ii, weak a_ij, and strong F a_im whose row has no
 *     distributable entry in C_i (denominator exactly 0); num_j = a_ij for
 *     j in C_i;
 *   pass B over the strong F neighbours m (ascending) with nonzero
 *     denominator d_m = sum_{k in C_i} ahat_mk adds (a_im / d_m) * ahat_mj to
 *     num_j for each j in C_i found in row m (ascending k);
 *   w_ij = -(num_j / dacc); a zero dacc leaves the row empty. */
or_csr *or_interp(const or_csr *A, const uint8_t *strong, const int8_t *cf) {
  int32_t n = A->n;
  int32_t *cidx = xmalloc(sizeof(int32_t) * (size_t)n);
  int32_t nc = 0;
  for (int32_t i = 0; i < n; i++) cidx[i] = cf[i] == 1 ? nc++ : -1;
  /* row sizes */
  int32_t *cnt = xmalloc(sizeof(int32_t) * (size_t)n);
  int64_t tot = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t c = 0;
    if (cf[i] == 1) c = 1;
    else
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
        if (strong[k] && cf[A->col[k]] == 1) c++;
    cnt[i] = c;
    tot += c;
  }
  int32_t *mark = xmalloc(sizeof(int32_t) * (size_t)n);  /* position of j in C_i, or -1 */
  double *num = xmalloc(sizeof(double) * (size_t)n);
  for (int32_t j = 0; j < n; j++) mark[j] = -1;
  or_csr *P = or_csr_alloc(n, nc, (int32_t)tot);
  int32_t pos = 0;
  P->rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    if (cf[i] == 1) {
      P->col[pos] = cidx[i];
      P->val[pos] = 1.0;
      pos++;
      P->rowptr[i + 1] = pos;
      continue;
    }
    if (cnt[i] == 0) { P->rowptr[i + 1] = pos; continue; }
    int32_t base = pos;
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      int32_t j = A->col[k];
      if (strong[k] && cf[j] == 1) { mark[j] = pos - base; P->col[pos] = cidx[j]; pos++; }
    }
    /* pass A */
    double dacc = 0.0;
    int dinit = 0;
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      int32_t j = A->col[k];
      double a = A->val[k];
      int add = 0;
      if (j == i || !strong[k]) add = 1;
      else if (cf[j] == 1) num[mark[j]] = a;
      else {
        double sm = diag_of(A, j) < 0.0 ? -1.0 : 1.0;
        double d = 0.0;
        int dset = 0;
        for (int32_t q = A->rowptr[j]; q < A->rowptr[j + 1]; q++) {
          int32_t kk = A->col[q];
          if (kk == j || mark[kk] < 0) continue;
          double av = A->val[q];
          if (!(sm * av < 0.0)) continue;
          if (!dset) { d = av; dset = 1; } else d = d + av;
        }
        if (d == 0.0) add = 1;
      }
      if (add) {
        if (!dinit) { dacc = a; dinit = 1; } else dacc = dacc + a;
      }
    }
    /* pass B */
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
      int32_t m = A->col[k];
      if (m == i || !strong[k] || cf[m] == 1) continue;
      double sm = diag_of(A, m) < 0.0 ? -1.0 : 1.0;
      double d = 0.0;
      int dset = 0;
      for (int32_t q = A->rowptr[m]; q < A->rowptr[m + 1]; q++) {
        int32_t kk = A->col[q];
        if (kk == m || mark[kk] < 0) continue;
        double av = A->val[q];
        if (!(sm * av < 0.0)) continue;
        if (!dset) { d = av; dset = 1; } else d = d + av;
      }
      if (d == 0.0) continue;
      double t = A->val[k] / d;
      for (int32_t q = A->rowptr[m]; q < A->rowptr[m + 1]; q++) {
        int32_t kk = A->col[q];
        if (kk == m || mark[kk] < 0) continue;
        double av = A->val[q];
        if (!(sm * av < 0.0)) continue;
        num[mark[kk]] = num[mark[kk]] + t * av;
      }
    }
    if (dacc == 0.0) {
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) mark[A->col[k]] = -1;
      pos = base;
      P->rowptr[i + 1] = pos;
      continue;
    }
    for (int32_t q = base; q < pos; q++) P->val[q] = -(num[q - base] / dacc);
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) mark[A->col[k]] = -1;
    P->rowptr[i + 1] = pos;
  }
  P->nnz = pos;
  free(cidx); free(cnt); free(mark); free(num);
  return P;
}


static int cmp_i32_amg(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Distance-two "extended+i" interpolation (De Sterck, Falgout, Nolting, Yang
 * 2008), the usual companion of PMIS. For an F point i with strong F
 * neighbours F_i and strong C neighbours C_i, the interpolatory set is
 * Chat_i = C_i united with the strong C neighbours of every k in F_i, and
 *   w_ij = -(1/dtil) (a_ij + sum_{k in F_i} a_ik abar_kj / d_k),  j in Chat_i,
 *   dtil = a_ii + sum_{weak n not in Chat_i} a_in + sum_{k in F_i} a_ik abar_ki / d_k,
 *   d_k  = sum_{l in Chat_i + {i}} abar_kl,
 * with abar_kl = a_kl when its sign is opposite to a_kk, else 0 (a_ij = 0
 * when j is not a neighbour of i). A strong F neighbour with d_k = 0 is added
 * to the diagonal. Arithmetic order: pass A runs over row i ascending
 * (diagonal, weak lumps and d_k = 0 lumps into dtil; a_ij into num_j); pass B
 * over the k of F_i ascending, t = a_ik / d_k, then over row k ascending adds
 * t * abar_kl to num_l (l in Chat_i) or to dtil (l = i). Every sum starts from
 * its first term. Entries whose num_j was never set are left out; a zero
 * dtil or an empty Chat_i gives an empty row. */
or_csr *or_interp_ext(const or_csr *A, const uint8_t *strong, const int8_t *cf) {
  int32_t n = A->n;
  int32_t *cidx = xmalloc(sizeof(int32_t) * (size_t)n);
  int32_t nc = 0;
  for (int32_t i = 0; i < n; i++) cidx[i] = cf[i] == 1 ? nc++ : -1;
  int32_t *mark = xmalloc(sizeof(int32_t) * (size_t)n);
  for (int32_t j = 0; j < n; j++) mark[j] = -1;
  int32_t cap = 1024, rowcap = 4096;
  int32_t *chat = xmalloc(sizeof(int32_t) * (size_t)rowcap);
  double *num = xmalloc(sizeof(double) * (size_t)rowcap);
  int8_t *nset = xmalloc((size_t)rowcap);
  int32_t *pc = xmalloc(sizeof(int32_t) * (size_t)cap);
  double *pv = xmalloc(sizeof(double) * (size_t)cap);
  int32_t *rp = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t pos = 0;
  rp[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    int32_t m = 0;
    if (cf[i] == 1) {
      if (pos + 1 > cap) { cap *= 2; pc = realloc(pc, sizeof(int32_t) * (size_t)cap); pv = realloc(pv, sizeof(double) * (size_t)cap); }
      pc[pos] = cidx[i]; pv[pos] = 1.0; pos++;
      rp[i + 1] = pos;
      continue;
    }
    /* Chat_i */
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t j = A->col[q];
      if (j == i || !strong[q]) continue;
      if (cf[j] == 1) {
        if (mark[j] < 0) { mark[j] = 0; chat[m++] = j; }
      } else {
        for (int32_t t = A->rowptr[j]; t < A->rowptr[j + 1]; t++) {
          int32_t l = A->col[t];
          if (l != j && strong[t] && cf[l] == 1 && mark[l] < 0) { mark[l] = 0; chat[m++] = l; }
        }
      }
    }
    if (m == 0) { rp[i + 1] = pos; continue; }
    qsort(chat, (size_t)m, sizeof(int32_t), cmp_i32_amg);
    for (int32_t q = 0; q < m; q++) { mark[chat[q]] = q; nset[q] = 0; num[q] = 0.0; }
    double dacc = 0.0;
    int dinit = 0;
#define DADD(v) do { if (!dinit) { dacc = (v); dinit = 1; } else dacc = dacc + (v); } while (0)
    /* pass A */
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t j = A->col[q];
      double a = A->val[q];
      if (j == i) { DADD(a); continue; }
      if (mark[j] >= 0) { num[mark[j]] = a; nset[mark[j]] = 1; continue; }
      if (strong[q] && cf[j] != 1) {
        double sk = diag_of(A, j) < 0.0 ? -1.0 : 1.0, d = 0.0;
        int ds = 0;
        for (int32_t t = A->rowptr[j]; t < A->rowptr[j + 1]; t++) {
          int32_t l = A->col[t];
          if (l == j || !(l == i || mark[l] >= 0)) continue;
          double av = A->val[t];
          if (!(sk * av < 0.0)) continue;
          if (!ds) { d = av; ds = 1; } else d = d + av;
        }
        if (d == 0.0) DADD(a);
        continue;
      }
      DADD(a);
    }
    /* pass B */
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t k = A->col[q];
      if (k == i || !strong[q] || cf[k] == 1 || mark[k] >= 0) continue;
      double sk = diag_of(A, k) < 0.0 ? -1.0 : 1.0, d = 0.0;
      int ds = 0;
      for (int32_t t = A->rowptr[k]; t < A->rowptr[k + 1]; t++) {
        int32_t l = A->col[t];
        if (l == k || !(l == i || mark[l] >= 0)) continue;
        double av = A->val[t];
        if (!(sk * av < 0.0)) continue;
        if (!ds) { d = av; ds = 1; } else d = d + av;
      }
      if (d == 0.0) continue;
      double tq = A->val[q] / d;
      for (int32_t t = A->rowptr[k]; t < A->rowptr[k + 1]; t++) {
        int32_t l = A->col[t];
        if (l == k || !(l == i || mark[l] >= 0)) continue;
        double av = A->val[t];
        if (!(sk * av < 0.0)) continue;
        double pr = tq * av;
        if (l == i) DADD(pr);
        else if (!nset[mark[l]]) { num[mark[l]] = pr; nset[mark[l]] = 1; }
        else num[mark[l]] = num[mark[l]] + pr;
      }
    }
#undef DADD
    if (dacc != 0.0) {
      if (pos + m > cap) { while (pos + m > cap) cap *= 2; pc = realloc(pc, sizeof(int32_t) * (size_t)cap); pv = realloc(pv, sizeof(double) * (size_t)cap); }
      for (int32_t q = 0; q < m; q++) {
        if (!nset[q]) continue;
        pc[pos] = cidx[chat[q]];
        pv[pos] = -(num[q] / dacc);
        pos++;
      }
    }
    for (int32_t q = 0; q < m; q++) mark[chat[q]] = -1;
    rp[i + 1] = pos;
  }
  or_csr *P = or_csr_alloc(n, nc, pos);
  memcpy(P->rowptr, rp, sizeof(int32_t) * ((size_t)n + 1));
  memcpy(P->col, pc, sizeof(int32_t) * (size_t)pos);
  memcpy(P->val, pv, sizeof(double) * (size_t)pos);
  free(cidx); free(mark); free(chat); free(num); free(nset); free(pc); free(pv); free(rp);
  return P;
}

or_csr *or_spgemm(const or_csr *A, const or_csr *B);
or_csr *or_transpose(const or_csr *A);
void or_csr_free(or_csr *A);

or_csr *or_galerkin(const or_csr *A, const or_csr *P) {
  or_csr *AP = or_spgemm(A, P);
  or_csr *R = or_transpose(P);
  or_csr *Ac = or_spgemm(R, AP);
  or_csr_free(AP);
  or_csr_free(R);
  return Ac;
}

/* Jones-Plassmann colouring of the symmetrised pattern of A (diagonal
 * ignored). Returns the number of colours. */
int32_t or_jp_colour(const or_csr *A, uint64_t seed, int32_t level, int32_t *colour) {
  int32_t n = A->n;
  uint64_t *key = xmalloc(sizeof(uint64_t) * (size_t)n);
  int8_t *sel = xmalloc((size_t)n);
  /* transpose adjacency */
  int32_t *tp = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  memset(tp, 0, sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t k = 0; k < A->nnz; k++) tp[A->col[k] + 1]++;
  for (int32_t i = 0; i < n; i++) tp[i + 1] += tp[i];
  int32_t *tc = xmalloc(sizeof(int32_t) * ((size_t)A->nnz + 1));
  int32_t *fill = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  memcpy(fill, tp, sizeof(int32_t) * (size_t)n);
  for (int32_t i = 0; i < n; i++)
    for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) tc[fill[A->col[k]]++] = i;
  for (int32_t i = 0; i < n; i++) {
    key[i] = or_splitmix64(seed, ((uint64_t)(2 * level + 1) << 32) + (uint64_t)i);
    colour[i] = -1;
  }
  int32_t left = n, ncol = 0;
  uint8_t *used = xmalloc(1024);
  while (left > 0) {
    for (int32_t i = 0; i < n; i++) {
      sel[i] = 0;
      if (colour[i] >= 0) continue;
      int ok = 1;
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1] && ok; k++) {
        int32_t j = A->col[k];
        if (j != i && colour[j] < 0 && !beats(key[i], i, key[j], j)) ok = 0;
      }
      for (int32_t q = tp[i]; q < tp[i + 1] && ok; q++) {
        int32_t j = tc[q];
        if (j != i && colour[j] < 0 && !beats(key[i], i, key[j], j)) ok = 0;
      }
      sel[i] = (int8_t)ok;
    }
    for (int32_t i = 0; i < n; i++) {
      if (!sel[i]) continue;
      memset(used, 0, 1024);
      for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) {
        int32_t j = A->col[k];
        if (j != i && colour[j] >= 0 && colour[j] < 1024) used[colour[j]] = 1;
      }
      for (int32_t q = tp[i]; q < tp[i + 1]; q++) {
        int32_t j = tc[q];
        if (j != i && colour[j] >= 0 && colour[j] < 1024) used[colour[j]] = 1;
      }
      int32_t c = 0;
      while (c < 1024 && used[c]) c++;
      colour[i] = c;
    }
    for (int32_t i = 0; i < n; i++)
      if (sel[i]) { left--; if (colour[i] + 1 > ncol) ncol = colour[i] + 1; }
  }
  free(key); free(sel); free(tp); free(tc); free(fill); free(used);
  return ncol;
}

/* Rows per chunk of the hybrid smoother: the `chunk` parameter (512 when
 * unset), a plain method parameter like the number of processes of the
 * parallel hybrid Gauss-Seidel it stands in for (Sec. 4.1). The matrix does
 * not enter. */
int32_t or_chunk_rows(const or_csr *A, int32_t chunk) {
  (void)A;
  return chunk > 0 ? chunk : 512;
}

/* The hybrid smoother's chunk parameter on level l: `chunk` on level 0,
 * `chunk_coarse` (when set) on the coarser levels. */
static int32_t level_chunk(const or_amg_params *p, int32_t l) {
  return (l == 0 || p->chunk_coarse <= 0) ? p->chunk : p->chunk_coarse;
}

/* Colouring used by the hybrid smoother: rows are cut into chunks of
 * or_chunk_rows(A) consecutive rows; inside each chunk, rows are coloured
 * first-fit in ascending order, each taking the lowest colour not used by an
 * already coloured row of the same chunk that it is coupled to in either
 * direction (a_ij or a_ji stored, i != j). Couplings across chunks are
 * ignored: the smoother treats them with old values. Returns the number of
 * colours (maximum over chunks). */
int32_t or_chunk_colour(const or_csr *A, int32_t chunk, int32_t *colour) {
  int32_t n = A->n, C = or_chunk_rows(A, chunk), ncol = 0;
  int32_t *tp = xmalloc(sizeof(int32_t) * ((size_t)C + 1));
  int32_t *tc = xmalloc(sizeof(int32_t) * ((size_t)A->nnz + 1));
  int32_t *stamp = xmalloc(sizeof(int32_t) * ((size_t)n + 2));
  for (int32_t c = 0; c <= n; c++) stamp[c] = -1;
  for (int32_t c0 = 0; c0 < n; c0 += C) {
    int32_t c1 = c0 + C < n ? c0 + C : n, len = c1 - c0;
    /* in-chunk transpose adjacency: tc[tp[i]..tp[i+1]) = rows k of the chunk with a_ki stored */
    for (int32_t t = 0; t <= len; t++) tp[t] = 0;
    for (int32_t k = c0; k < c1; k++)
      for (int32_t q = A->rowptr[k]; q < A->rowptr[k + 1]; q++) {
        int32_t j = A->col[q];
        if (j != k && j >= c0 && j < c1) tp[j - c0 + 1]++;
      }
    for (int32_t t = 0; t < len; t++) tp[t + 1] += tp[t];
    int32_t *cnt = xmalloc(sizeof(int32_t) * ((size_t)len + 1));
    for (int32_t t = 0; t < len; t++) cnt[t] = tp[t];
    for (int32_t k = c0; k < c1; k++)
      for (int32_t q = A->rowptr[k]; q < A->rowptr[k + 1]; q++) {
        int32_t j = A->col[q];
        if (j != k && j >= c0 && j < c1) tc[cnt[j - c0]++] = k;
      }
    free(cnt);
    for (int32_t i = c0; i < c1; i++) {
      /* mark colours of coloured in-chunk neighbours (rows < i) */
      for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
        int32_t j = A->col[q];
        if (j != i && j >= c0 && j < i) stamp[colour[j]] = i;
      }
      for (int32_t t = tp[i - c0]; t < tp[i - c0 + 1]; t++) {
        int32_t k = tc[t];
        if (k < i) stamp[colour[k]] = i;
      }
      int32_t c = 0;
      while (stamp[c] == i) c++;
      colour[i] = c;
      if (c + 1 > ncol) ncol = c + 1;
    }
  }
  free(tp); free(tc); free(stamp);
  return ncol;
}

/* Function f of b interleaved unknowns per point: rows b*i + f, columns
 * b*j + f of A, as an N x N matrix (N = n / b). */
or_csr *or_func_part(const or_csr *A, int32_t b, int32_t f) {
  int32_t N = A->n / b, nnz = 0;
  for (int32_t i = 0; i < N; i++)
    for (int32_t q = A->rowptr[b * i + f]; q < A->rowptr[b * i + f + 1]; q++) nnz += A->col[q] % b == f;
  or_csr *B = or_csr_alloc(N, A->m / b, nnz);
  int32_t pos = 0;
  B->rowptr[0] = 0;
  for (int32_t i = 0; i < N; i++) {
    for (int32_t q = A->rowptr[b * i + f]; q < A->rowptr[b * i + f + 1]; q++)
      if (A->col[q] % b == f) {
        B->col[pos] = A->col[q] / b;
        B->val[pos++] = A->val[q];
      }
    B->rowptr[i + 1] = pos;
  }
  return B;
}

/* Interleaved interpolation: row b*i + f of P is row i of Pf[f] with column
 * c mapped to b*c + f. */
static or_csr *interleave_P(or_csr **Pf, int32_t b) {
  int32_t N = Pf[0]->n, nc = Pf[0]->m, nnz = 0;
  for (int32_t f = 0; f < b; f++) nnz += Pf[f]->nnz;
  or_csr *P = or_csr_alloc(b * N, b * nc, nnz);
  int32_t pos = 0;
  P->rowptr[0] = 0;
  for (int32_t i = 0; i < N; i++)
    for (int32_t f = 0; f < b; f++) {
      const or_csr *Q = Pf[f];
      for (int32_t q = Q->rowptr[i]; q < Q->rowptr[i + 1]; q++) {
        P->col[pos] = b * Q->col[q] + f;
        P->val[pos++] = Q->val[q];
      }
      P->rowptr[b * i + f + 1] = pos;
    }
  return P;
}

/* Point colouring of the point-block hybrid smoother: chunks of
 * or_chunk_rows(A) consecutive rows (a whole number of points); inside a
 * chunk the points are coloured first-fit in ascending order, each taking the
 * lowest colour not used by an already coloured point of the chunk that it
 * is coupled to in either direction (some a_rc or a_cr stored with r in
 * point i and c in point k != i). Every unknown of a point gets the point's
 * colour. Returns the number of colours. */
int32_t or_chunk_colour_pt(const or_csr *A, int32_t chunk, int32_t b, int32_t *colour) {
  int32_t n = A->n, C = or_chunk_rows(A, chunk), ncol = 0;
  int32_t N = n / b;
  int32_t *pc = xmalloc(sizeof(int32_t) * ((size_t)N + 1));
  int32_t *stamp = xmalloc(sizeof(int32_t) * ((size_t)n + 2));
  for (int32_t c = 0; c <= n; c++) stamp[c] = -1;
  for (int32_t c0 = 0; c0 < n; c0 += C) {
    int32_t c1 = c0 + C < n ? c0 + C : n;
    int32_t p0 = c0 / b, p1 = c1 / b;
    for (int32_t i = p0; i < p1; i++) {
      /* in-chunk neighbours through the rows of point i */
      for (int32_t f = 0; f < b; f++)
        for (int32_t q = A->rowptr[b * i + f]; q < A->rowptr[b * i + f + 1]; q++) {
          int32_t k = A->col[q] / b;
          if (k != i && k >= p0 && k < i) stamp[pc[k]] = i;
        }
      /* and through the rows of earlier points of the chunk */
      for (int32_t k = p0; k < i; k++)
        for (int32_t f = 0; f < b; f++)
          for (int32_t q = A->rowptr[b * k + f]; q < A->rowptr[b * k + f + 1]; q++)
            if (A->col[q] / b == i) stamp[pc[k]] = i;
      int32_t c = 0;
      while (stamp[c] == i) c++;
      pc[i] = c;
      if (c + 1 > ncol) ncol = c + 1;
    }
  }
  for (int32_t i = 0; i < N; i++)
    for (int32_t f = 0; f < b; f++) colour[b * i + f] = pc[i];
  free(pc); free(stamp);
  return ncol;
}

/* Inverses of the 2 x 2 diagonal blocks of the points, row-major; a singular
 * block gets four zeros (the smoother then leaves that point unchanged). */
static double *block_inverses2(const or_csr *A) {
  int32_t N = A->n / 2;
  double *inv = xmalloc(sizeof(double) * 4 * ((size_t)N + 1));
  for (int32_t i = 0; i < N; i++) {
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    for (int32_t f = 0; f < 2; f++)
      for (int32_t q = A->rowptr[2 * i + f]; q < A->rowptr[2 * i + f + 1]; q++)
        if (A->col[q] / 2 == i) d[2 * f + A->col[q] % 2] = A->val[q];
    double det = d[0] * d[3] - d[1] * d[2];
    if (det != 0.0) {
      inv[4 * i + 0] = d[3] / det;
      inv[4 * i + 1] = -d[1] / det;
      inv[4 * i + 2] = -d[2] / det;
      inv[4 * i + 3] = d[0] / det;
    } else {
      inv[4 * i + 0] = inv[4 * i + 1] = inv[4 * i + 2] = inv[4 * i + 3] = 0.0;
    }
  }
  return inv;
}

/* ---------------- dense LU ---------------- */
int32_t or_dense_lu(int32_t n, double *a, int32_t *piv) {
  int32_t sing = 0;
  for (int32_t k = 0; k < n; k++) {
    int32_t p = k;
    double mx = fabs(a[(size_t)k * n + k]);
    for (int32_t i = k + 1; i < n; i++)
      if (fabs(a[(size_t)i * n + k]) > mx) { mx = fabs(a[(size_t)i * n + k]); p = i; }
    piv[k] = p;
    if (p != k)
      for (int32_t j = 0; j < n; j++) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    double d = a[(size_t)k * n + k];
    if (d == 0.0) { sing = 1; continue; }
    for (int32_t i = k + 1; i < n; i++) {
      double l = a[(size_t)i * n + k] / d;
      a[(size_t)i * n + k] = l;
      for (int32_t j = k + 1; j < n; j++) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return sing;
}

void or_dense_lu_solve(int32_t n, const double *a, const int32_t *piv, const double *b, double *x) {
  for (int32_t i = 0; i < n; i++) x[i] = b[i];
  for (int32_t k = 0; k < n; k++)
    if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int32_t i = 0; i < n; i++)
    for (int32_t j = 0; j < i; j++) x[i] -= a[(size_t)i * n + j] * x[j];
  for (int32_t i = n - 1; i >= 0; i--) {
    for (int32_t j = i + 1; j < n; j++) x[i] -= a[(size_t)i * n + j] * x[j];
    double d = a[(size_t)i * n + i];
    x[i] = d != 0.0 ? x[i] / d : 0.0;
  }
}

/* Approximate ideal restriction (AIR; Manteuffel, Southworth et al.,
 * "Nonsymmetric algebraic multigrid based on local approximate ideal
 * restriction", 2018) for the C/F splitting cf. The ideal restriction makes
 * (R A)(i, F) = 0 for every coarse point i; AIR imposes it on a small
 * neighbourhood: row r of R (the r-th C point i, in order) is e_i - z with z
 * supported on N_i and A(N_i, N_i)^T z = A(i, N_i)^T, so (R A)(i, N_i) = 0.
 * N_i: the F points coupled to i in row i (dist = 1), and for dist = 2 also
 * the F points coupled to those in their rows; ascending. With `strong`
 * (one flag per entry of A, NULL: every entry) only strong couplings count,
 * the neighbourhoods of the localised form lAIR (Manteuffel, Muenzenmaier,
 * Ruge, Southworth 2019). The local systems are solved by dense LU with
 * partial pivoting. */
or_csr *or_air_restriction(const or_csr *A, const int8_t *cf, int32_t dist, const uint8_t *strong) {
  int32_t n = A->n, nc = 0;
  for (int32_t i = 0; i < n; i++) nc += cf[i] == 1;
  int32_t *mark = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  int32_t *pos = xmalloc(sizeof(int32_t) * ((size_t)n + 1));
  for (int32_t j = 0; j < n; j++) { mark[j] = -1; pos[j] = -1; }
  size_t cap = (size_t)A->nnz + (size_t)nc + 16, used = 0;
  int32_t *rcol = xmalloc(sizeof(int32_t) * cap);
  double *rval = xmalloc(sizeof(double) * cap);
  or_csr *R = or_csr_alloc(nc, n, 0);
  int32_t ncap = 64, *nb = xmalloc(sizeof(int32_t) * (size_t)ncap);
  int32_t r = 0;
  R->rowptr[0] = 0;
  for (int32_t i = 0; i < n; i++) {
    if (cf[i] != 1) continue;
    int32_t m = 0;
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t j = A->col[q];
      if (j == i || cf[j] == 1 || mark[j] == i || (strong && !strong[q])) continue;
      if (m == ncap) { ncap *= 2; nb = realloc(nb, sizeof(int32_t) * (size_t)ncap); if (!nb) abort(); }
      mark[j] = i;
      nb[m++] = j;
    }
    if (dist >= 2) {
      int32_t m1 = m;
      for (int32_t a = 0; a < m1; a++)
        for (int32_t q = A->rowptr[nb[a]]; q < A->rowptr[nb[a] + 1]; q++) {
          int32_t j = A->col[q];
          if (j == i || cf[j] == 1 || mark[j] == i || (strong && !strong[q])) continue;
          if (m == ncap) { ncap *= 2; nb = realloc(nb, sizeof(int32_t) * (size_t)ncap); if (!nb) abort(); }
          mark[j] = i;
          nb[m++] = j;
        }
    }
    qsort(nb, (size_t)m, sizeof(int32_t), cmp_i32_amg);
    for (int32_t a = 0; a < m; a++) pos[nb[a]] = a;
    double *M = xmalloc(sizeof(double) * ((size_t)m * m + 1));
    double *rhs = xmalloc(sizeof(double) * ((size_t)m + 1));
    double *z = xmalloc(sizeof(double) * ((size_t)m + 1));
    int32_t *piv = xmalloc(sizeof(int32_t) * ((size_t)m + 1));
    for (size_t t = 0; t < (size_t)m * m; t++) M[t] = 0.0;
    for (int32_t a = 0; a < m; a++) rhs[a] = 0.0;
    /* M = A(N_i, N_i)^T: row b of A(N_i, .) fills column b of M */
    for (int32_t b = 0; b < m; b++)
      for (int32_t q = A->rowptr[nb[b]]; q < A->rowptr[nb[b] + 1]; q++) {
        int32_t a = A->col[q] < n ? pos[A->col[q]] : -1;
        if (a >= 0) M[(size_t)a * m + b] = A->val[q];
      }
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
      int32_t a = pos[A->col[q]];
      if (a >= 0) rhs[a] = A->val[q];
    }
    if (m > 0) {
      or_dense_lu(m, M, piv);
      or_dense_lu_solve(m, M, piv, rhs, z);
    }
    if (used + (size_t)m + 1 > cap) {
      cap = 2 * (used + (size_t)m + 1);
      rcol = realloc(rcol, sizeof(int32_t) * cap);
      rval = realloc(rval, sizeof(double) * cap);
      if (!rcol || !rval) abort();
    }
    /* the row: -z on N_i and 1 at i, ascending columns */
    int placed = 0;
    for (int32_t a = 0; a < m; a++) {
      if (!placed && i < nb[a]) { rcol[used] = i; rval[used] = 1.0; used++; placed = 1; }
      rcol[used] = nb[a];
      rval[used] = -z[a];
      used++;
    }
    if (!placed) { rcol[used] = i; rval[used] = 1.0; used++; }
    for (int32_t a = 0; a < m; a++) pos[nb[a]] = -1;
    free(M); free(rhs); free(z); free(piv);
    R->rowptr[++r] = (int32_t)used;
  }
  free(R->col); free(R->val);
  R->col = rcol;
  R->val = rval;
  R->nnz = (int32_t)used;
  free(mark); free(pos); free(nb);
  return R;
}

/* ---------------- hierarchy ---------------- */
#define OR_MAXLEV 32
struct or_amg {
  or_amg_params prm;
  int32_t nlev;
  or_csr *A[OR_MAXLEV];
  or_csr *P[OR_MAXLEV];
  or_csr *R[OR_MAXLEV];
  int8_t *cf[OR_MAXLEV];
  int32_t *colour[OR_MAXLEV];
  int32_t ncol[OR_MAXLEV];
  double *l1[OR_MAXLEV];
  double *binv[OR_MAXLEV];  /* point mode: inverses of the 2 x 2 diagonal blocks */
  int32_t b;                /* unknowns per point (1: scalar AMG) */
  double *lu;        /* coarsest dense LU */
  int32_t *piv;
  int32_t dense;     /* 1 if the coarsest level is solved by LU */
};

or_amg *or_amg_setup(const or_csr *A0, const or_amg_params *prm) {
  or_amg *H = xmalloc(sizeof(or_amg));
  memset(H, 0, sizeof(or_amg));
  H->prm = *prm;
  H->b = prm->num_functions == 2 ? 2 : 1;
  if (H->b > 1) H->prm.smoother = 2;   /* point mode uses the point-block hybrid smoother */
  int32_t maxl = prm->max_levels < OR_MAXLEV ? prm->max_levels : OR_MAXLEV;
  H->A[0] = or_csr_alloc(A0->n, A0->m, A0->nnz);
  memcpy(H->A[0]->rowptr, A0->rowptr, sizeof(int32_t) * ((size_t)A0->n + 1));
  memcpy(H->A[0]->col, A0->col, sizeof(int32_t) * (size_t)A0->nnz);
  memcpy(H->A[0]->val, A0->val, sizeof(double) * (size_t)A0->nnz);
  int32_t l = 0;
  for (;;) {
    or_csr *A = H->A[l];
    int32_t n = A->n;
    H->cf[l] = NULL;
    if (n <= prm->coarse_n || l == maxl - 1) break;
    if (H->b > 1) {
      /* point mode: coarsen the points on the pressure part */
      int32_t b = H->b, N = n / b;
      or_csr *Ap = or_func_part(A, b, 0);
      uint8_t *st = xmalloc((size_t)Ap->nnz + 1);
      or_strength_nf(Ap, prm->theta, 1, st);
      int8_t *cfp = xmalloc((size_t)N + 1);
      or_pmis(Ap, st, prm->seed, l, cfp);
      free(st);
      or_csr_free(Ap);
      int32_t nc = 0;
      for (int32_t i = 0; i < N; i++) nc += cfp[i] == 1;
      if (nc == 0 || (double)nc > 0.9 * (double)N) { free(cfp); break; }
      or_csr *Pf[2];
      for (int32_t f = 0; f < b; f++) {
        or_csr *Af = or_func_part(A, b, f);
        uint8_t *sf = xmalloc((size_t)Af->nnz + 1);
        or_strength_nf(Af, prm->theta, 1, sf);
        Pf[f] = prm->interp == 1 ? or_interp_ext(Af, sf, cfp) : or_interp(Af, sf, cfp);
        free(sf);
        or_csr_free(Af);
      }
      H->P[l] = interleave_P(Pf, b);
      for (int32_t f = 0; f < b; f++) or_csr_free(Pf[f]);
      int8_t *cf = xmalloc((size_t)n);
      for (int32_t i = 0; i < N; i++)
        for (int32_t f = 0; f < b; f++) cf[b * i + f] = cfp[i];
      free(cfp);
      H->cf[l] = cf;
    } else {
      uint8_t *st = xmalloc((size_t)A->nnz);
      or_strength_nf(A, prm->theta, 1, st);
      int8_t *cf = xmalloc((size_t)n);
      or_pmis(A, st, prm->seed, l, cf);
      int32_t nc = 0;
      for (int32_t i = 0; i < n; i++) nc += cf[i] == 1;
      if (nc == 0 || (double)nc > 0.9 * (double)n) { free(st); free(cf); break; }
      H->cf[l] = cf;
      H->P[l] = prm->interp == 1 ? or_interp_ext(A, st, cf) : or_interp(A, st, cf);
      /* AIR restriction, Petrov-Galerkin coarse operator R A P; restriction 3
       * takes distance-1 neighbourhoods of strong couplings (lAIR) */
      if (prm->restriction > 0)
        H->R[l] = prm->restriction == 3 ? or_air_restriction(A, cf, 1, st)
                                        : or_air_restriction(A, cf, prm->restriction, NULL);
      free(st);
    }
    if (H->b == 1 && prm->restriction > 0) {
      or_csr *AP = or_spgemm(A, H->P[l]);
      H->A[l + 1] = or_spgemm(H->R[l], AP);
      or_csr_free(AP);
    } else {
      H->R[l] = or_transpose(H->P[l]);
      H->A[l + 1] = or_galerkin(A, H->P[l]);
    }
    l++;
  }
  H->nlev = l + 1;
  /* Aggressive coarsening, two-stage form: the coarse grid of level k is the
   * second of two PMIS stages, C2 within C1, and its interpolation the product
   * of the two stages' interpolations, P = P_k P_{k+1} (each stage extended+i
   * or classical on its own Galerkin operator); the intermediate level is
   * dropped, its operator A_{k+2} = P_{k+1}^T (P_k^T A_k P_k) P_{k+1} kept as
   * the next level's. A fine point is C when it is C in both stages. Applied
   * to the first agg_levels coarse grids while two more levels exist. */
  for (int32_t k = 0; k < prm->agg_levels && k + 2 < H->nlev; k++) {
    or_csr *P = or_spgemm(H->P[k], H->P[k + 1]);
    int8_t *cf = xmalloc((size_t)H->A[k]->n + 1);
    int32_t ic = 0;
    for (int32_t i = 0; i < H->A[k]->n; i++) cf[i] = H->cf[k][i] == 1 ? H->cf[k + 1][ic++] : (int8_t)-1;
    or_csr *Rk = (H->b == 1 && prm->restriction > 0) ? or_spgemm(H->R[k + 1], H->R[k]) : or_transpose(P);
    or_csr_free(H->P[k]); or_csr_free(H->R[k]); free(H->cf[k]);
    H->P[k] = P;
    H->R[k] = Rk;
    H->cf[k] = cf;
    or_csr_free(H->A[k + 1]); or_csr_free(H->P[k + 1]); or_csr_free(H->R[k + 1]); free(H->cf[k + 1]);
    for (int32_t j = k + 1; j + 1 < H->nlev; j++) {
      H->A[j] = H->A[j + 1]; H->P[j] = H->P[j + 1]; H->R[j] = H->R[j + 1]; H->cf[j] = H->cf[j + 1];
    }
    H->nlev--;
    H->A[H->nlev] = NULL; H->P[H->nlev] = NULL; H->R[H->nlev] = NULL; H->cf[H->nlev] = NULL;
  }
  for (int32_t k = 0; k < H->nlev - 1; k++) {
    or_csr *A = H->A[k];
    H->colour[k] = xmalloc(sizeof(int32_t) * ((size_t)A->n + 1));
    if (H->b > 1) {
      H->ncol[k] = or_chunk_colour_pt(A, level_chunk(prm, k), H->b, H->colour[k]);
      H->binv[k] = block_inverses2(A);
    } else if (prm->smoother == 2) H->ncol[k] = or_chunk_colour(A, level_chunk(prm, k), H->colour[k]);
    else H->ncol[k] = or_jp_colour(A, prm->seed, k, H->colour[k]);
    H->l1[k] = xmalloc(sizeof(double) * ((size_t)A->n + 1));
    for (int32_t i = 0; i < A->n; i++) {
      double d = 0.0, off = 0.0;
      for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
        if (A->col[q] == i) d = A->val[q];
        else off += fabs(A->val[q]);
      }
      H->l1[k][i] = d < 0.0 ? d - off : d + off;
    }
  }
  or_csr *Ac = H->A[H->nlev - 1];
  int32_t nc = Ac->n;
  if (nc <= prm->max_dense) {
    H->dense = 1;
    H->lu = xmalloc(sizeof(double) * (size_t)nc * (size_t)nc + 1);
    H->piv = xmalloc(sizeof(int32_t) * ((size_t)nc + 1));
    memset(H->lu, 0, sizeof(double) * (size_t)nc * (size_t)nc);
    for (int32_t i = 0; i < nc; i++)
      for (int32_t q = Ac->rowptr[i]; q < Ac->rowptr[i + 1]; q++)
        H->lu[(size_t)i * nc + Ac->col[q]] = Ac->val[q];
    or_dense_lu(nc, H->lu, H->piv);
  } else {
    /* coarsest level too large for a dense factorisation: smooth it instead */
    int32_t k = H->nlev - 1;
    H->colour[k] = xmalloc(sizeof(int32_t) * ((size_t)nc + 1));
    if (H->b > 1) {
      H->ncol[k] = or_chunk_colour_pt(Ac, level_chunk(prm, k), H->b, H->colour[k]);
      H->binv[k] = block_inverses2(Ac);
    } else if (prm->smoother == 2) H->ncol[k] = or_chunk_colour(Ac, level_chunk(prm, k), H->colour[k]);
    else H->ncol[k] = or_jp_colour(Ac, prm->seed, k, H->colour[k]);
    H->l1[k] = xmalloc(sizeof(double) * ((size_t)nc + 1));
    for (int32_t i = 0; i < nc; i++) {
      double d = 0.0, off = 0.0;
      for (int32_t q = Ac->rowptr[i]; q < Ac->rowptr[i + 1]; q++) {
        if (Ac->col[q] == i) d = Ac->val[q];
        else off += fabs(Ac->val[q]);
      }
      H->l1[k][i] = d < 0.0 ? d - off : d + off;
    }
  }
  return H;
}

void or_amg_free(or_amg *H) {
  if (!H) return;
  for (int32_t l = 0; l < H->nlev; l++) {
    or_csr_free(H->A[l]);
    or_csr_free(H->P[l]);
    or_csr_free(H->R[l]);
    free(H->cf[l]);
    free(H->colour[l]);
    free(H->l1[l]);
    free(H->binv[l]);
  }
  free(H->lu);
  free(H->piv);
  free(H);
}

int32_t or_amg_nlevels(const or_amg *H) { return H->nlev; }
const or_csr *or_amg_A(const or_amg *H, int32_t l) { return H->A[l]; }
const or_csr *or_amg_P(const or_amg *H, int32_t l) { return H->P[l]; }
void or_amg_cf(const or_amg *H, int32_t l, int8_t *cf) {
  if (H->cf[l]) memcpy(cf, H->cf[l], (size_t)H->A[l]->n);
}
int32_t or_amg_colours(const or_amg *H, int32_t l, int32_t *colour) {
  if (!H->colour[l]) return 0;
  memcpy(colour, H->colour[l], sizeof(int32_t) * (size_t)H->A[l]->n);
  return H->ncol[l];
}

/* One smoothing sweep on level l (x updated in place). */
void or_amg_smooth(const or_amg *H, int32_t l, const double *b, double *x) {
  const or_csr *A = H->A[l];
  if (H->prm.smoother == 1) {
    double *r = xmalloc(sizeof(double) * ((size_t)A->n + 1));
    for (int32_t i = 0; i < A->n; i++) {
      double s = 0.0;
      for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) s += A->val[q] * x[A->col[q]];
      r[i] = b[i] - s;
    }
    for (int32_t i = 0; i < A->n; i++)
      if (H->l1[l][i] != 0.0) x[i] += r[i] / H->l1[l][i];
    free(r);
    return;
  }
  if (H->b == 2) {
    /* point-block hybrid Gauss-Seidel: as below with points in place of rows;
     * for a point of the current colour, each of its rows takes b minus the
     * couplings outside the point (newest values inside the chunk, start
     * values outside it), then the point's two unknowns are set to the
     * inverse diagonal block times those two numbers */
    double *xo = xmalloc(sizeof(double) * ((size_t)A->n + 1));
    memcpy(xo, x, sizeof(double) * (size_t)A->n);
    int32_t C = or_chunk_rows(A, level_chunk(&H->prm, l));
    for (int32_t c0 = 0; c0 < A->n; c0 += C) {
      int32_t c1 = c0 + C < A->n ? c0 + C : A->n;
      for (int32_t c = 0; c < H->ncol[l]; c++) {
        for (int32_t i = c0 / 2; i < c1 / 2; i++) {
          if (H->colour[l][2 * i] != c) continue;
          double r[2];
          for (int32_t f = 0; f < 2; f++) {
            double t = b[2 * i + f];
            for (int32_t q = A->rowptr[2 * i + f]; q < A->rowptr[2 * i + f + 1]; q++) {
              int32_t j = A->col[q];
              if (j / 2 == i) continue;
              t -= A->val[q] * ((j >= c0 && j < c1) ? x[j] : xo[j]);
            }
            r[f] = t;
          }
          const double *m = H->binv[l] + 4 * (size_t)i;
          if (m[0] == 0.0 && m[1] == 0.0 && m[2] == 0.0 && m[3] == 0.0) continue;
          x[2 * i] = m[0] * r[0] + m[1] * r[1];
          x[2 * i + 1] = m[2] * r[0] + m[3] * r[1];
        }
      }
    }
    free(xo);
    return;
  }
  if (H->prm.smoother == 2) {
    /* hybrid multicolour Gauss-Seidel: rows are cut into consecutive chunks of
     * `chunk` rows; inside a chunk the colours are swept in order using the
     * chunk's newest values, couplings to other chunks use the values from the
     * start of the sweep (block Jacobi between chunks, as in the hybrid
     * Gauss-Seidel of parallel AMG codes, with a chunk in place of a process). */
    double *xo = xmalloc(sizeof(double) * ((size_t)A->n + 1));
    memcpy(xo, x, sizeof(double) * (size_t)A->n);
    /* chunk size: the level's `chunk` parameter */
    int32_t C = or_chunk_rows(A, level_chunk(&H->prm, l));
    for (int32_t c0 = 0; c0 < A->n; c0 += C) {
      int32_t c1 = c0 + C < A->n ? c0 + C : A->n;
      for (int32_t c = 0; c < H->ncol[l]; c++) {
        for (int32_t i = c0; i < c1; i++) {
          if (H->colour[l][i] != c) continue;
          double s = 0.0, d = 0.0;
          for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
            int32_t j = A->col[q];
            if (j == i) d = A->val[q];
            else s += A->val[q] * ((j >= c0 && j < c1) ? x[j] : xo[j]);
          }
          if (d != 0.0) x[i] = (b[i] - s) / d;
        }
      }
    }
    free(xo);
    return;
  }
  for (int32_t c = 0; c < H->ncol[l]; c++) {
    for (int32_t i = 0; i < A->n; i++) {
      if (H->colour[l][i] != c) continue;
      double s = 0.0, d = 0.0;
      for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) {
        if (A->col[q] == i) d = A->val[q];
        else s += A->val[q] * x[A->col[q]];
      }
      if (d != 0.0) x[i] = (b[i] - s) / d;
    }
  }
}

static void vcycle(const or_amg *H, int32_t l, const double *b, double *x) {
  const or_csr *A = H->A[l];
  int32_t n = A->n;
  if (l == H->nlev - 1) {
    if (H->dense) {
      or_dense_lu_solve(n, H->lu, H->piv, b, x);
    } else {
      for (int32_t i = 0; i < n; i++) x[i] = 0.0;
      for (int32_t s = 0; s < H->prm.nu1 + H->prm.nu2; s++) or_amg_smooth(H, l, b, x);
    }
    return;
  }
  for (int32_t i = 0; i < n; i++) x[i] = 0.0;
  for (int32_t s = 0; s < H->prm.nu1; s++) or_amg_smooth(H, l, b, x);
  double *r = xmalloc(sizeof(double) * ((size_t)n + 1));
  for (int32_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int32_t q = A->rowptr[i]; q < A->rowptr[i + 1]; q++) s += A->val[q] * x[A->col[q]];
    r[i] = b[i] - s;
  }
  int32_t nc = H->A[l + 1]->n;
  double *bc = xmalloc(sizeof(double) * ((size_t)nc + 1));
  double *xc = xmalloc(sizeof(double) * ((size_t)nc + 1));
  or_csr_spmv(H->R[l], r, bc);
  vcycle(H, l + 1, bc, xc);
  const or_csr *P = H->P[l];
  for (int32_t i = 0; i < n; i++)
    for (int32_t q = P->rowptr[i]; q < P->rowptr[i + 1]; q++) x[i] += P->val[q] * xc[P->col[q]];
  for (int32_t s = 0; s < H->prm.nu2; s++) or_amg_smooth(H, l, b, x);
  free(r); free(bc); free(xc);
}

void or_amg_vcycle(const or_amg *H, const double *b, double *x) { vcycle(H, 0, b, x); }
