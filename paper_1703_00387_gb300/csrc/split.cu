// Two-site split with truncation by the eigendecomposition route (Sec. 2,
// Eq. AAD_ULLUD and Eq. ThetaAL), entirely in float64:
//   left-to-right: G = M M^T (Gram matrix), G = U lambda^2 U^T (float64
//                  eigenpairs), A1 = U_kept, A2 = U_kept^T M / ||.||
//   right-to-left: G = M^T M, A2 = V_kept^T, A1 = M V_kept / ||.||
// with M = theta viewed as (chi_l d1) x (d2 chi_r). The number kept follows
// the local tolerance (Eq. elocal, Sec. 3.4): chi' = min(chi_max, smallest n
// with discarded weight <= eps_local), lambda^2 normalised to sum 1. The
// eigenvalues are copied to the host to fix chi' (the next shapes depend on it).
//
// Arithmetic: the eigenpairs are float64, from the tridiagonal route of
// eig.cu (this library's Householder tridiagonalisation, then multisection,
// inverse iteration, Cholesky QR and blocked back-transformation on
// emulated-float64 GEMMs; the default from Gram dimension 64 on) or from
// cuSOLVER (dsyevdx for the largest min(chi_max, rank) only, dsyevd when
// that is all of them; the default below 64), as osmps_ctx_set_eig_solver
// selects. The
// Gram matrix and the projection are float64 GEMMs: on the DMMA kernel for
// OSMPS_PREC_FP64, on the float64-accurate emulated tensor-core GEMM for
// every other precision.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace osmps {

namespace {

// dst[j * n + c] = Y[idx[j] * n + c]
__global__ void k_gather_idx_rows(const double* __restrict__ Y, const int* __restrict__ idx,
                                  int64_t n, int64_t keep, double* __restrict__ dst) {
  const int64_t total = n * keep;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, c = e - j * n;
    dst[e] = Y[(int64_t)idx[j] * n + c];
  }
}

// dst[r * keep + j] = Yk[j * n + r]
__global__ void k_transpose_keep(const double* __restrict__ Yk, int64_t n, int64_t keep,
                                 double* __restrict__ dst) {
  const int64_t total = n * keep;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / keep, j = e - r * keep;
    dst[e] = Yk[j * n + r];
  }
}

int blocks_for(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 16384) b = 16384;
  return (int)b;
}

}  // namespace

// Truncation from the computed (largest) eigenvalues of the Gram matrix, in
// any order: returns the indices of the kept values (descending) and fills
// chi', the discarded weight and the entropy. The Gram route squares the
// singular values, so eigenvalues below ~n eps ||theta||^2 are rounding
// noise; the discarded weight is therefore taken as 1 - (kept sum) / tr with
// tr = ||theta||^2 computed directly, the kept sum accumulated with
// compensated summation, instead of as a sum over the noisy tail.
osmps_status truncate_spectrum(const double* ev, int64_t n, double tr, int64_t rank,
                                      int64_t chi_max, double eps_local, Trunc* t) {
  t->order.resize(n);
  for (int64_t i = 0; i < n; ++i) t->order[i] = (int)i;
  std::stable_sort(t->order.begin(), t->order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
  if (!(tr > 0.0) || !std::isfinite(tr))
    return set_error(OSMPS_ENAN, "split: theta has zero or non-finite norm");
  t->lam2.resize(n);
  for (int64_t i = 0; i < n; ++i) t->lam2[i] = std::max(ev[t->order[i]], 0.0) / tr;
  const int64_t cap = std::min<int64_t>(chi_max, rank);
  double kept = 0.0, kc = 0.0;
  int64_t keep = 0;
  while (keep < n) {
    const double y = t->lam2[keep] - kc, u = kept + y;
    kc = (u - kept) - y;
    kept = u;
    ++keep;
    if (1.0 - kept <= eps_local || keep >= cap) break;
  }
  t->keep = keep;
  t->discarded = std::max(1.0 - kept, 0.0);
  double S = 0.0;
  for (int64_t i = 0; i < keep; ++i) {
    const double p = t->lam2[i] / kept;
    if (p > 0.0) S -= p * std::log(p);
  }
  t->entropy = S;
  return OSMPS_OK;
}

// Truncate from the eigenpairs (Y: eigenvectors as rows, ev: eigenvalues on
// the host, any order), then form the two site tensors:
//   move_right: A1 = U_kept (left-canonical), A2 = U_kept^T M, renormalised;
//   else:       A2 = V_kept^T (right-canonical), A1 = M V_kept, renormalised.
static osmps_status finish_split(osmps_ctx* ctx, const double* theta, const double* Y,
                                 const double* ev, int64_t nev, double tr, int64_t rows,
                                 int64_t cols, int move_right, int64_t chi_max, double eps_local,
                                 bool emu, double* A1, double* A2, int64_t* chi_new,
                                 double* discarded, double* entropy, double* lam2_out,
                                 cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t n = move_right ? rows : cols;
  Trunc t;
  OSMPS_TRY(truncate_spectrum(ev, nev, tr, std::min(rows, cols), chi_max, eps_local, &t));
  const int64_t keep = t.keep;
  if (lam2_out)
    for (int64_t i = 0; i < std::min(rows, cols); ++i) lam2_out[i] = i < nev ? t.lam2[i] : 0.0;
  *chi_new = keep;
  *discarded = t.discarded;
  *entropy = t.entropy;

  int* idx = (int*)ws_get(ctx, SLOT_QR_TAU, (size_t)keep * sizeof(int) + 256, s, &st);
  if (!idx) return st;
  OSMPS_CUDA(cudaMemcpyAsync(idx, t.order.data(), (size_t)keep * sizeof(int), cudaMemcpyHostToDevice, s));
  double* Yk = (double*)ws_get(ctx, SLOT_SPLIT_TMP, (size_t)keep * n * 8 + 256, s, &st);
  if (!Yk) return st;
  { k_gather_idx_rows<<<blocks_for(n * keep), 256, 0, s>>>(Y, idx, n, keep, Yk); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  double* nrm = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);
  if (!nrm) return st;
  if (move_right) {
    { k_transpose_keep<<<blocks_for(n * keep), 256, 0, s>>>(Yk, n, keep, A1); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    if (emu) {
      SplitView a; a.src = Yk; a.rows = keep; a.K = rows; a.s0 = rows; a.sk = 1;
      SplitView b; b.src = theta; b.rows = cols; b.K = rows; b.s0 = 1; b.sk = cols;
      OSMPS_TRY(gemm_emu(ctx, a, b, keep, cols, rows, A2, cols, s));
    } else {
      GemmF64 p;
      p.M = keep; p.N = cols; p.K = rows;
      p.A = Yk; p.sam = rows; p.sak = 1;
      p.B = theta; p.sbk = cols; p.sbn = 1;
      p.C = A2; p.scm = cols; p.scn = 1;
      OSMPS_TRY(gemm_f64(p, s));
    }
    OSMPS_TRY(vec_norm2(ctx, A2, keep * cols, nrm, s));
    OSMPS_TRY(vec_scale_by_inv_sqrt(A2, keep * cols, nrm, s));
  } else {
    OSMPS_CUDA(cudaMemcpyAsync(A2, Yk, (size_t)keep * cols * 8, cudaMemcpyDeviceToDevice, s));
    if (emu) {
      SplitView a; a.src = theta; a.rows = rows; a.K = cols; a.s0 = cols; a.sk = 1;
      SplitView b; b.src = Yk; b.rows = keep; b.K = cols; b.s0 = cols; b.sk = 1;
      OSMPS_TRY(gemm_emu(ctx, a, b, rows, keep, cols, A1, keep, s));
    } else {
      GemmF64 p;
      p.M = rows; p.N = keep; p.K = cols;
      p.A = theta; p.sam = cols; p.sak = 1;
      p.B = Yk; p.sbk = 1; p.sbn = cols;
      p.C = A1; p.scm = keep; p.scn = 1;
      OSMPS_TRY(gemm_f64(p, s));
    }
    OSMPS_TRY(vec_norm2(ctx, A1, rows * keep, nrm, s));
    OSMPS_TRY(vec_scale_by_inv_sqrt(A1, rows * keep, nrm, s));
  }
  return OSMPS_OK;
}

osmps_status split_impl(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                        int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int move_right,
                        int64_t chi_max, double eps_local, int64_t* chi_new, double* discarded,
                        double* entropy, double* lam2_out, int precision, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t rows = chi_l * d1, cols = d2 * chi_r;
  const int64_t n = move_right ? rows : cols;
  if (n > 46340) return set_error(OSMPS_ESHAPE, "split: Gram dimension %lld too large", (long long)n);
  const bool emu = precision != OSMPS_PREC_FP64;
  double* G = (double*)ws_get(ctx, SLOT_SPLIT_G, (size_t)n * n * 8, s, &st);
  if (!G) return st;
  double* ev = (double*)ws_get(ctx, SLOT_SPLIT_EV, (size_t)(n + 8) * 8, s, &st);
  if (!ev) return st;
  double* tr_dev = ev + n;  // ||theta||^2
  OSMPS_TRY(vec_norm2(ctx, theta, rows * cols, tr_dev, s));
  // Gram matrix: G = M M^T (move_right) or M^T M, M = theta as rows x cols
  if (emu) {
    SplitView mv;
    if (move_right) { mv.src = theta; mv.rows = rows; mv.K = cols; mv.s0 = cols; mv.sk = 1; }
    else { mv.src = theta; mv.rows = cols; mv.K = rows; mv.s0 = 1; mv.sk = cols; }
    OSMPS_TRY(gemm_emu(ctx, mv, mv, n, n, mv.K, G, n, s));
  } else {
    GemmF64 g;
    if (move_right) {
      g.M = rows; g.N = rows; g.K = cols;
      g.A = theta; g.sam = cols; g.sak = 1;
      g.B = theta; g.sbk = 1; g.sbn = cols;
    } else {
      g.M = cols; g.N = cols; g.K = rows;
      g.A = theta; g.sam = 1; g.sak = cols;
      g.B = theta; g.sbk = cols; g.sbn = 1;
    }
    g.C = G; g.scm = n; g.scn = 1;
    OSMPS_TRY(gemm_f64(g, s));
  }
  // Only the largest min(chi_max, rank) eigenpairs can be kept: compute just
  // those (the discarded weight comes from ||theta||^2, not from the rest).
  const int64_t nev = std::min<int64_t>(n, std::min<int64_t>(chi_max, std::min(rows, cols)));
  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lwork = 0, found = 0;
  double* Z = nullptr;  // eigenvectors, column-major n x nev (rows of a row-major nev x n)
  // AUTO: this library's route from Gram dimension 64 on, where it measured
  // faster than cuSOLVER on GB300 (n = 64 ... 2048), cuSOLVER below
  const bool tridiag = ctx->eig_solver == OSMPS_EIG_TRIDIAG ||
                       (ctx->eig_solver == OSMPS_EIG_AUTO && n >= 64);
  if (tridiag && n >= 2) {
    double* Y = (double*)ws_get(ctx, SLOT_SPLIT_TMP2, (size_t)nev * n * 8, s, &st);
    if (!Y) return st;
    OSMPS_TRY(eig_top(ctx, G, n, nev, ev, Y, s));
    found = (int)nev;
    Z = Y;
    OSMPS_CUDA(cudaMemsetAsync(ctx->dev_info, 0, sizeof(int), s));
  } else if (nev == n) {
    OSMPS_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n, ev, &lwork));
    double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 8, s, &st);
    if (!work) return st;
    OSMPS_SOLVER(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  (int)n, G, (int)n, ev, work, lwork, ctx->dev_info));
    found = (int)n;
    Z = G;
  } else {
    const int il = (int)(n - nev + 1), iu = (int)n;
    OSMPS_SOLVER(cusolverDnDsyevdx_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                              CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, (int)n,
                                              G, (int)n, 0.0, 0.0, il, iu, &found, ev, &lwork));
    double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 8, s, &st);
    if (!work) return st;
    OSMPS_SOLVER(cusolverDnDsyevdx(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                   CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n, 0.0, 0.0, il, iu,
                                   &found, ev, work, lwork, ctx->dev_info));
    Z = G;  // the selected eigenvectors occupy the first `found` columns of G
  }
  OSMPS_TRY(pinned_reserve(ctx, (size_t)n + 16));
  double* h = ctx->host_pinned;
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(h, ev, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) return set_error(OSMPS_ECUDA, "split: syevd info %d", info);
  if (found < 1 || found > n) return set_error(OSMPS_ECUDA, "split: syevdx found %d eigenpairs", found);
  const double trace = h[n];  // ||theta||^2, stored after the n eigenvalue slots
  std::vector<double> ev_host(h, h + found);
  return finish_split(ctx, theta, Z, ev_host.data(), found, trace, rows, cols, move_right,
                      chi_max, eps_local, emu, A1, A2, chi_new, discarded, entropy, lam2_out, s);
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_split(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                                    int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                    int move_right, int64_t chi_max, double eps_local,
                                    int64_t* chi_new_out, double* discarded_out,
                                    double* entropy_out, double* lam2_out, int precision,
                                    void* stream) {
  clear_error();
  if (!ctx || !theta || !A1 || !A2 || !chi_new_out || !discarded_out || !entropy_out)
    return set_error(OSMPS_EINVAL, "osmps_split: null argument");
  if (A1 == theta || A2 == theta || A1 == A2)
    return set_error(OSMPS_EINVAL, "osmps_split: outputs alias each other or theta");
  if (move_right != 0 && move_right != 1)
    return set_error(OSMPS_EINVAL, "osmps_split: move_right %d", move_right);
  if (chi_max < 1) return set_error(OSMPS_EINVAL, "osmps_split: chi_max %lld", (long long)chi_max);
  if (!valid_precision(precision)) return set_error(OSMPS_EINVAL, "osmps_split: precision %d", precision);
  if (!(eps_local >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_split: eps_local %g", eps_local);
  for (int64_t x : {chi_l, d1, d2, chi_r})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_split: non-positive or oversized dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return split_impl(ctx, theta, A1, A2, chi_l, d1, d2, chi_r, move_right, chi_max, eps_local,
                    chi_new_out, discarded_out, entropy_out, lam2_out, precision, (cudaStream_t)stream);
}
