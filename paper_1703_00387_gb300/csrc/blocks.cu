// Block operations for block-sparse (U(1)-symmetric) tensors: the sweep over
// a particle-number-conserving MPS (Sec. 3.4 with symmetries) works on the
// dense blocks of its tensors, one per combination of charge sectors, so
// theta formation, the per-sector Gram matrices and projections of the split
// (Sec. 2, Eq. AAD_ULLUD), and the environment updates become lists of
// float64 products and copies of strided matrix views. The host builds the
// lists from the sector bookkeeping; this file runs them:
//   osmps_gemm_grouped   per output C = sum over its terms of alpha A B +
//                        beta C, every output in one launch of a float64
//                        DMMA kernel (element strides of either sign);
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

// ---------------------------------------------------------------------------
// Grouped segmented-K float64 GEMM. One CTA per 64 x 64 tile of one output;
// the CTA runs through the K ranges of the output's terms in order, 16 at a
// time, double-buffered through shared memory (the tiling of the strided
// float64 kernel: 8 warps as 2 x 4, each a 32 x 16 sub-tile of 8 x 8
// mma.sync f64 fragments). A term's alpha scales its A tile as it is staged.
// ---------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 64, GB_K = 16, GB_PAD = 4, GB_THREADS = 256;

struct GTerm {
  const double* A;
  int64_t sam, sak;
  const double* B;
  int64_t sbk, sbn;
  int64_t K;
  double alpha;
};
struct GOut {
  double* C;
  int64_t scm, scn, M, N;
  double beta;
  int64_t t0, tn;    // term range
  int64_t tile0;     // first tile of this output in the launch
};

__device__ __forceinline__ void dmma884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(GB_THREADS) k_gemm_grouped(const GOut* __restrict__ outs, int n_out,
                                                              const GTerm* __restrict__ terms) {
  __shared__ double As[2][GB_K][GB_M + GB_PAD];
  __shared__ double Bs[2][GB_K][GB_N + GB_PAD];
  __shared__ int s_out;
  const int tid = threadIdx.x;
  if (tid == 0) {  // the last output whose first tile is at or before this one
    int lo = 0, hi = n_out - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (outs[mid].tile0 <= (int64_t)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_out = lo;
  }
  __syncthreads();
  const GOut o = outs[s_out];
  const int64_t t = (int64_t)blockIdx.x - o.tile0;
  const int64_t tiles_n = cdiv(o.N, GB_N);
  const int64_t m0 = (t / tiles_n) * GB_M, n0 = (t % tiles_n) * GB_N;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;

  double ra[4], rb[4];
  auto load = [&](int64_t ti, int64_t k0) {
    const GTerm& tm = terms[ti];
    const bool akf = tm.sak == 1, bnf = tm.sbn == 1;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * GB_THREADS;
      int mm, kk;
      if (akf) { kk = e % GB_K; mm = e / GB_K; } else { mm = e % GB_M; kk = e / GB_M; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < o.M && gk < tm.K) ? tm.alpha * tm.A[gm * tm.sam + gk * tm.sak] : 0.0;
      int nn;
      if (bnf) { nn = e % GB_N; kk = e / GB_N; } else { kk = e % GB_K; nn = e / GB_K; }
      const int64_t gn = n0 + nn;
      gk = k0 + kk;
      rb[r] = (gn < o.N && gk < tm.K) ? tm.B[gk * tm.sbk + gn * tm.sbn] : 0.0;
    }
  };
  auto store = [&](int64_t ti, int buf) {
    const bool akf = terms[ti].sak == 1, bnf = terms[ti].sbn == 1;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + r * GB_THREADS;
      int mm, kk;
      if (akf) { kk = e % GB_K; mm = e / GB_K; } else { mm = e % GB_M; kk = e / GB_M; }
      As[buf][kk][mm] = ra[r];
      int nn;
      if (bnf) { nn = e % GB_N; kk = e / GB_N; } else { kk = e % GB_K; nn = e / GB_K; }
      Bs[buf][kk][nn] = rb[r];
    }
  };

  double acc[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int64_t te = o.t0 + o.tn;
  int64_t ti = o.t0, k0 = 0;
  bool have = ti < te;
  if (have) {
    load(ti, 0);
    store(ti, 0);
  }
  __syncthreads();
  int buf = 0;
  while (have) {
    int64_t nti = ti, nk0 = k0 + GB_K;
    if (nk0 >= terms[ti].K) {
      nti = ti + 1;
      nk0 = 0;
    }
    const bool nhave = nti < te;
    if (nhave) load(nti, nk0);
#pragma unroll
    for (int k4 = 0; k4 < GB_K; k4 += 4) {
      double a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][k4 + tq][wm + i * 8 + g];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Bs[buf][k4 + tq][wn + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dmma884(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
    if (nhave) store(nti, buf ^ 1);
    __syncthreads();
    buf ^= 1;
    ti = nti;
    k0 = nk0;
    have = nhave;
  }

#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int64_t gm = m0 + wm + i * 8 + g;
        const int64_t gn = n0 + wn + j * 8 + tq * 2 + r;
        if (gm < o.M && gn < o.N) {
          double* c = o.C + gm * o.scm + gn * o.scn;
          double v = acc[i][j][r];
          if (o.beta != 0.0) v = fma(o.beta, *c, v);
          *c = v;
        }
      }
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_gemm_grouped(osmps_ctx* ctx, const osmps_gemm_out* outs, int64_t n_out,
                                           const osmps_gemm_term* terms, int64_t n_terms, void* stream) {
  clear_error();
  if (!ctx || (n_out > 0 && !outs) || (n_terms > 0 && !terms))
    return set_error(OSMPS_EINVAL, "osmps_gemm_grouped: null argument");
  if (n_out < 0 || n_terms < 0 || n_out > INT32_MAX || n_terms > INT32_MAX)
    return set_error(OSMPS_EINVAL, "osmps_gemm_grouped: n_out=%lld n_terms=%lld", (long long)n_out,
                     (long long)n_terms);
  for (int64_t i = 0; i < n_terms; ++i) {
    const osmps_gemm_term& t = terms[i];
    if (!t.A || !t.B) return set_error(OSMPS_EINVAL, "osmps_gemm_grouped: term %lld has a null pointer", (long long)i);
    if (t.K < 1) return set_error(OSMPS_ESHAPE, "osmps_gemm_grouped: term %lld has K=%lld", (long long)i, (long long)t.K);
  }
  std::vector<GOut> h;
  h.reserve((size_t)n_out);
  int64_t tiles = 0;
  for (int64_t i = 0; i < n_out; ++i) {
    const osmps_gemm_out& o = outs[i];
    if (o.M < 0 || o.N < 0) return set_error(OSMPS_ESHAPE, "osmps_gemm_grouped: output %lld has a negative size", (long long)i);
    if (o.term_begin < 0 || o.term_count < 0 || o.term_begin > n_terms - o.term_count)
      return set_error(OSMPS_EINVAL, "osmps_gemm_grouped: output %lld has terms [%lld, +%lld) outside [0, %lld)",
                       (long long)i, (long long)o.term_begin, (long long)o.term_count, (long long)n_terms);
    if (o.M == 0 || o.N == 0) continue;
    if (!o.C) return set_error(OSMPS_EINVAL, "osmps_gemm_grouped: output %lld has a null pointer", (long long)i);
    h.push_back(GOut{o.C, o.scm, o.scn, o.M, o.N, o.beta, o.term_begin, o.term_count, tiles});
    tiles += cdiv(o.M, GB_M) * cdiv(o.N, GB_N);
    if (tiles > INT32_MAX) return set_error(OSMPS_ESHAPE, "osmps_gemm_grouped: more than 2^31 tiles");
  }
  if (h.empty()) return OSMPS_OK;
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = round_up((int64_t)(h.size() * sizeof(GOut)), 256), tb = (size_t)n_terms * sizeof(GTerm);
  osmps_status st = OSMPS_OK;
  auto* dd = (char*)ws_get(ctx, SLOT_RED, ob + tb + 8, s, &st);
  if (!dd) return st;
  std::vector<GTerm> ht((size_t)n_terms);
  for (int64_t i = 0; i < n_terms; ++i) {
    const osmps_gemm_term& t = terms[i];
    ht[(size_t)i] = GTerm{t.A, t.sam, t.sak, t.B, t.sbk, t.sbn, t.K, t.alpha};
  }
  OSMPS_CUDA(cudaMemcpyAsync(dd, h.data(), h.size() * sizeof(GOut), cudaMemcpyHostToDevice, s));
  if (tb) OSMPS_CUDA(cudaMemcpyAsync(dd + ob, ht.data(), tb, cudaMemcpyHostToDevice, s));
  double flops = 0.0;
  for (const GOut& o : h)
    for (int64_t k = o.t0; k < o.t0 + o.tn; ++k) flops += 2.0 * (double)o.M * (double)o.N * (double)ht[(size_t)k].K;
  const int ph = prof_begin(s);
  k_gemm_grouped<<<(unsigned)tiles, GB_THREADS, 0, s>>>((const GOut*)dd, (int)h.size(), (const GTerm*)(dd + ob));
  note_launch();
  OSMPS_LAUNCH_CHECK();
  prof_end(ph, s, OSMPS_KERNEL_GEMM_F64, flops, flops);
  // the host descriptor arrays must outlive the upload
  OSMPS_CUDA(cudaStreamSynchronize(s));
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
