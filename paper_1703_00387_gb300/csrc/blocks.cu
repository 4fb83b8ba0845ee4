// Block operations for block-sparse (U(1)-symmetric) tensors: the sweep over
// a particle-number-conserving MPS (Sec. 3.4 with symmetries) works on the
// dense blocks of its tensors, one per combination of charge sectors, so
// theta formation, the per-sector Gram matrices and projections of the split
// (Sec. 2, Eq. AAD_ULLUD), and the environment updates become lists of
// float64 products and copies of strided matrix views. The host builds the
// lists from the sector bookkeeping; this file runs them:
//   osmps_gemm_list      C = alpha A B + beta C per entry (float64 DMMA
//                        kernel, element strides of either sign);
//   osmps_copy_list      dst = alpha src per entry (strided 2-D views), all
//                        entries in one launch, one block per entry;
//   osmps_sym_eig_top    the largest eigenpairs of a symmetric matrix (this
//                        library's route from n = 64 on, cuSOLVER below);
//   osmps_vec_norm2      ||x||^2 to the host.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace osmps {
namespace {

struct CopyDesc {
  const double* src;
  double* dst;
  int64_t rows, cols;
  int64_t srs, scs;  // source element strides (row, column), either sign
  int64_t drs;       // destination row stride (columns contiguous)
  double alpha;
};

// blockIdx.x = entry, blockIdx.y = chunk of it: dst[r drs + c] =
// alpha src[r srs + c scs] (src null: dst = 0)
__global__ void k_copy_list(const CopyDesc* __restrict__ d, int n) {
  const CopyDesc c = d[blockIdx.x];
  const int64_t total = c.rows * c.cols;
  const int64_t step = (int64_t)gridDim.y * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t r = e / c.cols, k = e - r * c.cols;
    c.dst[r * c.drs + k] = c.src ? c.alpha * c.src[r * c.srs + k * c.scs] : 0.0;
  }
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_gemm_list(osmps_ctx* ctx, const osmps_gemm_desc* descs, int64_t n,
                                        void* stream) {
  clear_error();
  if (!ctx || (n > 0 && !descs)) return set_error(OSMPS_EINVAL, "osmps_gemm_list: null argument");
  if (n < 0) return set_error(OSMPS_EINVAL, "osmps_gemm_list: n=%lld", (long long)n);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t i = 0; i < n; ++i) {
    const osmps_gemm_desc& d = descs[i];
    if (!d.A || !d.B || !d.C)
      return set_error(OSMPS_EINVAL, "osmps_gemm_list: entry %lld has a null pointer", (long long)i);
    if (d.M < 0 || d.N < 0 || d.K < 0)
      return set_error(OSMPS_ESHAPE, "osmps_gemm_list: entry %lld has a negative size", (long long)i);
    if (d.M == 0 || d.N == 0) continue;
    GemmF64 g;
    g.M = d.M; g.N = d.N; g.K = d.K;
    g.A = d.A; g.sam = d.sam; g.sak = d.sak;
    g.B = d.B; g.sbk = d.sbk; g.sbn = d.sbn;
    g.C = d.C; g.scm = d.scm; g.scn = d.scn;
    g.alpha = d.alpha; g.beta = d.beta;
    if (d.K == 0) {  // an empty sum: C = beta C
      g.K = 1;
      g.alpha = 0.0;
    }
    OSMPS_TRY(gemm_f64(g, s));
  }
  return OSMPS_OK;
}

extern "C" osmps_status osmps_copy_list(osmps_ctx* ctx, const osmps_copy_desc* descs, int64_t n,
                                        void* stream) {
  clear_error();
  if (!ctx || (n > 0 && !descs)) return set_error(OSMPS_EINVAL, "osmps_copy_list: null argument");
  if (n < 0 || n > INT32_MAX) return set_error(OSMPS_EINVAL, "osmps_copy_list: n=%lld", (long long)n);
  if (n == 0) return OSMPS_OK;
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<CopyDesc> h((size_t)n);
  int64_t largest = 0;
  for (int64_t i = 0; i < n; ++i) {
    const osmps_copy_desc& d = descs[i];
    if (!d.dst || d.rows < 0 || d.cols < 0 || (d.cols > 0 && d.rows > INT64_MAX / d.cols))
      return set_error(OSMPS_EINVAL, "osmps_copy_list: entry %lld", (long long)i);
    h[(size_t)i] = CopyDesc{d.src, d.dst, d.rows, d.cols, d.srs, d.scs, d.drs, d.alpha};
    largest = std::max(largest, d.rows * d.cols);
  }
  if (largest == 0) return OSMPS_OK;
  // enough chunks that the largest entry gets ~8 elements per thread, at most
  // 4 resident blocks' worth per SM in total
  const int64_t want = (largest + 2047) / 2048;
  const int64_t cap = std::max<int64_t>(1, (int64_t)4 * ctx->sm_count / std::min<int64_t>(n, 65535));
  const unsigned chunks = (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, cap, 65535}));
  osmps_status st = OSMPS_OK;
  auto* dd = (CopyDesc*)ws_get(ctx, SLOT_RED, (size_t)n * sizeof(CopyDesc), s, &st);
  if (!dd) return st;
  OSMPS_CUDA(cudaMemcpyAsync(dd, h.data(), (size_t)n * sizeof(CopyDesc), cudaMemcpyHostToDevice, s));
  { k_copy_list<<<dim3((unsigned)n, chunks), 256, 0, s>>>(dd, (int)n); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  // the host descriptors must outlive the copy
  OSMPS_CUDA(cudaStreamSynchronize(s));
  return OSMPS_OK;
}

extern "C" osmps_status osmps_sym_eig_top(osmps_ctx* ctx, double* G, int64_t n, int64_t nev,
                                          double* ev_host, double* Y, void* stream) {
  clear_error();
  if (!ctx || !G || !ev_host || !Y) return set_error(OSMPS_EINVAL, "osmps_sym_eig_top: null argument");
  if (n < 1 || n > 46340 || nev < 1 || nev > n)
    return set_error(OSMPS_ESHAPE, "osmps_sym_eig_top: n=%lld nev=%lld", (long long)n, (long long)nev);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  double* ev = (double*)ws_get(ctx, SLOT_SPLIT_EV, (size_t)(n + 8) * 8, s, &st);
  if (!ev) return st;
  const bool own = ctx->eig_solver == OSMPS_EIG_TRIDIAG ||
                   (ctx->eig_solver == OSMPS_EIG_AUTO && n >= 64);
  if (own && n >= 2) {
    OSMPS_TRY(eig_top(ctx, G, n, nev, ev, Y, s));
    OSMPS_CUDA(cudaMemcpyAsync(ev_host, ev, (size_t)nev * 8, cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    return OSMPS_OK;
  }
  // cuSOLVER dsyevd: all pairs ascending, vectors as the columns of the
  // column-major G (= rows of the row-major view); the top nev are the last
  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lwork = 0;
  OSMPS_SOLVER(cusolverDnDsyevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                           CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n, ev, &lwork));
  double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 8, s, &st);
  if (!work) return st;
  OSMPS_SOLVER(cusolverDnDsyevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                (int)n, G, (int)n, ev, work, lwork, ctx->dev_info));
  OSMPS_CUDA(cudaMemcpyAsync(Y, G + (n - nev) * n, (size_t)nev * n * 8, cudaMemcpyDeviceToDevice, s));
  OSMPS_CUDA(cudaMemcpyAsync(ev_host, ev + (n - nev), (size_t)nev * 8, cudaMemcpyDeviceToHost, s));
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) return set_error(OSMPS_ECUDA, "osmps_sym_eig_top: syevd info %d", info);
  return OSMPS_OK;
}

extern "C" osmps_status osmps_vec_norm2(osmps_ctx* ctx, const double* x, int64_t n, double* out_host,
                                        void* stream) {
  clear_error();
  if (!ctx || !x || !out_host) return set_error(OSMPS_EINVAL, "osmps_vec_norm2: null argument");
  if (n < 1) return set_error(OSMPS_ESHAPE, "osmps_vec_norm2: n=%lld", (long long)n);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  double* d = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);
  if (!d) return st;
  OSMPS_TRY(vec_norm2(ctx, x, n, d, s));
  OSMPS_CUDA(cudaMemcpyAsync(out_host, d, 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  return OSMPS_OK;
}
