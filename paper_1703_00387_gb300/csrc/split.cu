// Two-site split with truncation by the eigendecomposition route (Sec. 2,
// Eq. AAD_ULLUD and Eq. ThetaAL), entirely in float64:
//   left-to-right: G = M M^T (Gram on the DMMA GEMM), G = U lambda^2 U^T
//                  (cuSOLVER syevd), A1 = U_kept, A2 = U_kept^T M / ||.||
//   right-to-left: G = M^T M, A2 = V_kept^T, A1 = M V_kept / ||.||
// with M = theta viewed as (chi_l d1) x (d2 chi_r). The number kept follows
// the local tolerance (Eq. elocal, Sec. 3.4): chi' = min(chi_max, smallest n
// with discarded weight sum_{i>=n} lambda_i^2 <= eps_local), lambda^2
// normalised to sum 1. The eigenvalues are copied to the host to fix chi'
// (the next shapes depend on it).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace osmps {

namespace {

// dst[r * keep + j] = Gmem[(n - 1 - j) * n + r] (descending eigenvector j, row r)
__global__ void k_gather_cols(const double* __restrict__ G, int64_t n, int64_t keep,
                              double* __restrict__ dst) {
  const int64_t total = n * keep;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / keep, j = e - r * keep;
    dst[e] = G[(n - 1 - j) * n + r];
  }
}

// dst[j * n + c] = Gmem[(n - 1 - j) * n + c]  (descending eigenvectors as rows)
__global__ void k_gather_rows(const double* __restrict__ G, int64_t n, int64_t keep,
                              double* __restrict__ dst) {
  const int64_t total = n * keep;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, c = e - j * n;
    dst[e] = G[(n - 1 - j) * n + c];
  }
}

int blocks_for(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 16384) b = 16384;
  return (int)b;
}

}  // namespace

osmps_status split_impl(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                        int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int move_right,
                        int64_t chi_max, double eps_local, int64_t* chi_new, double* discarded,
                        double* entropy, double* lam2_out, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t rows = chi_l * d1, cols = d2 * chi_r;
  const int64_t n = move_right ? rows : cols;
  if (n > 46340) return set_error(OSMPS_ESHAPE, "split: Gram dimension %lld too large", (long long)n);
  double* G = (double*)ws_get(ctx, SLOT_SPLIT_G, (size_t)n * n * 8, s, &st);
  if (!G) return st;
  double* ev = (double*)ws_get(ctx, SLOT_SPLIT_EV, (size_t)n * 8, s, &st);
  if (!ev) return st;

  GemmF64 g;
  if (move_right) {  // G = M M^T
    g.M = rows; g.N = rows; g.K = cols;
    g.A = theta; g.sam = cols; g.sak = 1;
    g.B = theta; g.sbk = 1; g.sbn = cols;
  } else {  // G = M^T M
    g.M = cols; g.N = cols; g.K = rows;
    g.A = theta; g.sam = 1; g.sak = cols;
    g.B = theta; g.sbk = cols; g.sbn = 1;
  }
  g.C = G; g.scm = n; g.scn = 1;
  OSMPS_TRY(gemm_f64(g, s));

  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lwork = 0;
  OSMPS_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                           CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n, ev, &lwork));
  double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 8, s, &st);
  if (!work) return st;
  OSMPS_SOLVER(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                (int)n, G, (int)n, ev, work, lwork, ctx->dev_info));
  OSMPS_TRY(pinned_reserve(ctx, (size_t)n + 8));
  double* h = ctx->host_pinned;
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(h, ev, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) return set_error(OSMPS_ECUDA, "split: syevd info %d", info);

  // descending, clipped, normalised lambda^2
  std::vector<double> lam2(n);
  double tot = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    lam2[i] = std::max(h[n - 1 - i], 0.0);
    tot += lam2[i];
  }
  if (!(tot > 0.0) || !std::isfinite(tot)) return set_error(OSMPS_ENAN, "split: theta has zero or non-finite norm");
  for (auto& x : lam2) x /= tot;
  // tail[i] = sum_{k >= i} lam2[k], summed from the small end
  std::vector<double> tail(n + 1, 0.0);
  for (int64_t i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + lam2[i];
  int64_t keep = 1;
  while (keep < n && tail[keep] > eps_local) ++keep;
  keep = std::min<int64_t>(keep, std::min<int64_t>(chi_max, std::min(rows, cols)));
  double kept = 0.0;
  for (int64_t i = 0; i < keep; ++i) kept += lam2[i];
  double S = 0.0;
  for (int64_t i = 0; i < keep; ++i) {
    const double p = lam2[i] / kept;
    if (p > 0.0) S -= p * std::log(p);
  }
  if (lam2_out)
    for (int64_t i = 0; i < std::min(rows, cols); ++i) lam2_out[i] = lam2[i];
  *chi_new = keep;
  *discarded = tail[keep];
  *entropy = S;

  double* nrm = (double*)ws_get(ctx, SLOT_SPLIT_TMP, 64, s, &st);
  if (!nrm) return st;
  if (move_right) {
    // A1[(a,s1), j] = U[:, j];  A2[j, (s2,c)] = sum_r A1[r, j] M[r, (s2,c)]
    { k_gather_cols<<<blocks_for(n * keep), 256, 0, s>>>(G, n, keep, A1); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    GemmF64 p;
    p.M = keep; p.N = cols; p.K = rows;
    p.A = A1; p.sam = 1; p.sak = keep;
    p.B = theta; p.sbk = cols; p.sbn = 1;
    p.C = A2; p.scm = cols; p.scn = 1;
    OSMPS_TRY(gemm_f64(p, s));
    OSMPS_TRY(vec_norm2(ctx, A2, keep * cols, nrm, s));
    OSMPS_TRY(vec_scale_by_inv_sqrt(A2, keep * cols, nrm, s));
  } else {
    // A2[j, (s2,c)] = V[:, j]^T;  A1[(a,s1), j] = sum_c M[(a,s1), c] A2[j, c]
    { k_gather_rows<<<blocks_for(n * keep), 256, 0, s>>>(G, n, keep, A2); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    GemmF64 p;
    p.M = rows; p.N = keep; p.K = cols;
    p.A = theta; p.sam = cols; p.sak = 1;
    p.B = A2; p.sbk = 1; p.sbn = cols;
    p.C = A1; p.scm = keep; p.scn = 1;
    OSMPS_TRY(gemm_f64(p, s));
    OSMPS_TRY(vec_norm2(ctx, A1, rows * keep, nrm, s));
    OSMPS_TRY(vec_scale_by_inv_sqrt(A1, rows * keep, nrm, s));
  }
  return OSMPS_OK;
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_split(osmps_ctx* ctx, const double* theta, double* A1, double* A2,
                                    int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                    int move_right, int64_t chi_max, double eps_local,
                                    int64_t* chi_new_out, double* discarded_out,
                                    double* entropy_out, double* lam2_out, void* stream) {
  clear_error();
  if (!ctx || !theta || !A1 || !A2 || !chi_new_out || !discarded_out || !entropy_out)
    return set_error(OSMPS_EINVAL, "osmps_split: null argument");
  if (A1 == theta || A2 == theta || A1 == A2)
    return set_error(OSMPS_EINVAL, "osmps_split: outputs alias each other or theta");
  if (move_right != 0 && move_right != 1)
    return set_error(OSMPS_EINVAL, "osmps_split: move_right %d", move_right);
  if (chi_max < 1) return set_error(OSMPS_EINVAL, "osmps_split: chi_max %lld", (long long)chi_max);
  if (!(eps_local >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_split: eps_local %g", eps_local);
  for (int64_t x : {chi_l, d1, d2, chi_r})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_split: non-positive or oversized dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return split_impl(ctx, theta, A1, A2, chi_l, d1, d2, chi_r, move_right, chi_max, eps_local,
                    chi_new_out, discarded_out, entropy_out, lam2_out, (cudaStream_t)stream);
}
