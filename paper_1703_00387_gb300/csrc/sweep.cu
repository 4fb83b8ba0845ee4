// Whole-chain handles and the two-site sweeps of Sec. 3.4.
//
// A sweep optimises the pairs (0,1) ... (L-2,L-1) left to right and back,
// each step being: theta = A_k A_{k+1} (Sec. 2 "Contractions"), the lowest
// eigenpair of H_eff by Lanczos, the eigendecomposition split with
// truncation (Eq. AAD_ULLUD, Eq. elocal) and one environment update. The
// initial state is brought to mixed-canonical form by QR shifts of the
// orthogonality centre (Sec. 2 "Shifting", Eq. oc). All state lives on the
// device; only shapes and per-step scalars go to the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

namespace osmps {

namespace {

__global__ void k_transpose(const double* __restrict__ src, int64_t rows, int64_t cols,
                            double* __restrict__ dst) {
  // dst[j * rows + i] = src[i * cols + j]
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < rows && j < cols) t[r][threadIdx.x] = src[i * cols + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (i < rows && j < cols) dst[j * rows + i] = t[threadIdx.x][r];
  }
}

osmps_status transpose(const double* src, int64_t rows, int64_t cols, double* dst, cudaStream_t s) {
  dim3 grid((unsigned)cdiv(cols, 32), (unsigned)cdiv(rows, 32));
  if (grid.y > 65535) return set_error(OSMPS_ESHAPE, "transpose: %lld rows", (long long)rows);
  { k_transpose<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, dst); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

// Rout[i][j] = X[j * nr + i] for i <= j, 0 below the diagonal (i < r, j < nc)
__global__ void k_extract_r(const double* __restrict__ X, int64_t nr, int64_t nc, int64_t r,
                            double* __restrict__ Rout) {
  const int64_t total = r * nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / nc, j = e - i * nc;
    Rout[e] = (i <= j) ? X[j * nr + i] : 0.0;
  }
}

__global__ void k_fill(double* p, int64_t n, double v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

__global__ void k_identity_op(double* p, int64_t d) {
  for (int64_t e = threadIdx.x; e < d * d; e += blockDim.x) p[e] = (e / d == e % d) ? 1.0 : 0.0;
}

int nblk(int64_t n) {
  int64_t b = cdiv(n, 1024);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 16384));
}

// Thin QR of the column-major nr x nc matrix X (ld = nr), overwritten by Q
// (first r = min(nr, nc) columns); R (r x nc, row-major, upper) to Rout.
osmps_status qr_inplace(osmps_ctx* ctx, double* X, int64_t nr, int64_t nc, double* Rout,
                        int64_t* r_out, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t r = std::min(nr, nc);
  double* tau = (double*)ws_get(ctx, SLOT_QR_TAU, (size_t)r * 8, s, &st);
  if (!tau) return st;
  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lw1 = 0, lw2 = 0;
  OSMPS_SOLVER(cusolverDnDgeqrf_bufferSize(ctx->solver, (int)nr, (int)nc, X, (int)nr, &lw1));
  OSMPS_SOLVER(cusolverDnDorgqr_bufferSize(ctx->solver, (int)nr, (int)r, (int)r, X, (int)nr, tau, &lw2));
  const int lw = std::max(std::max(lw1, lw2), 1);
  double* work = (double*)ws_get(ctx, SLOT_QR_WORK, (size_t)lw * 8, s, &st);
  if (!work) return st;
  OSMPS_SOLVER(cusolverDnDgeqrf(ctx->solver, (int)nr, (int)nc, X, (int)nr, tau, work, lw, ctx->dev_info));
  { k_extract_r<<<nblk(r * nc), 256, 0, s>>>(X, nr, nc, r, Rout); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  OSMPS_SOLVER(cusolverDnDorgqr(ctx->solver, (int)nr, (int)r, (int)r, X, (int)nr, tau, work, lw, ctx->dev_info));
  *r_out = r;
  return OSMPS_OK;
}

// Make site k left-canonical and push R into site k+1.
osmps_status shift_right(osmps_ctx* ctx, osmps_mps* m, int64_t k, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t chl = m->chi[k], d = m->d[k], chr = m->chi[k + 1];
  const int64_t rows = chl * d, cols = chr;
  double* X = (double*)ws_get(ctx, SLOT_SPLIT_G, (size_t)rows * cols * 8, s, &st);
  if (!X) return st;
  double* R = (double*)ws_get(ctx, SLOT_QR_R, (size_t)std::min(rows, cols) * cols * 8, s, &st);
  if (!R) return st;
  OSMPS_TRY(transpose(m->A[k], rows, cols, X, s));  // column-major copy of A_k as (chl d) x chr
  int64_t r = 0;
  OSMPS_TRY(qr_inplace(ctx, X, rows, cols, R, &r, s));
  OSMPS_TRY(transpose(X, r, rows, m->A[k], s));  // Q^T (col-major r x rows) -> row-major rows x r
  const int64_t d2 = m->d[k + 1], chr2 = m->chi[k + 2];
  double* tmp = (double*)ws_get(ctx, SLOT_SPLIT_TMP, (size_t)r * d2 * chr2 * 8, s, &st);
  if (!tmp) return st;
  GemmF64 g;  // A_{k+1} <- R A_{k+1}
  g.M = r; g.N = d2 * chr2; g.K = cols;
  g.A = R; g.sam = cols; g.sak = 1;
  g.B = m->A[k + 1]; g.sbk = d2 * chr2; g.sbn = 1;
  g.C = tmp; g.scm = d2 * chr2; g.scn = 1;
  OSMPS_TRY(gemm_f64(g, s));
  OSMPS_CUDA(cudaMemcpyAsync(m->A[k + 1], tmp, (size_t)r * d2 * chr2 * 8, cudaMemcpyDeviceToDevice, s));
  m->chi[k + 1] = r;
  // The state is defined up to a scalar: keep the receiving tensor at unit
  // norm so that products of many unnormalised sites cannot overflow.
  double* nrm = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);
  if (!nrm) return st;
  OSMPS_TRY(vec_norm2(ctx, m->A[k + 1], r * d2 * chr2, nrm, s));
  return vec_scale_by_inv_sqrt(m->A[k + 1], r * d2 * chr2, nrm, s);
}

// Make site k right-canonical and push R^T into site k-1.
osmps_status shift_left(osmps_ctx* ctx, osmps_mps* m, int64_t k, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t chl = m->chi[k], d = m->d[k], chr = m->chi[k + 1];
  const int64_t nr = d * chr, nc = chl;  // A_k row-major (chl, d chr) == column-major (d chr) x chl
  double* R = (double*)ws_get(ctx, SLOT_QR_R, (size_t)std::min(nr, nc) * nc * 8, s, &st);
  if (!R) return st;
  int64_t r = 0;
  OSMPS_TRY(qr_inplace(ctx, m->A[k], nr, nc, R, &r, s));  // A_k now holds Q^T (r, d, chr)
  const int64_t chl0 = m->chi[k - 1], d0 = m->d[k - 1];
  double* tmp = (double*)ws_get(ctx, SLOT_SPLIT_TMP, (size_t)chl0 * d0 * r * 8, s, &st);
  if (!tmp) return st;
  GemmF64 g;  // A_{k-1} <- A_{k-1} R^T
  g.M = chl0 * d0; g.N = r; g.K = chl;
  g.A = m->A[k - 1]; g.sam = chl; g.sak = 1;
  g.B = R; g.sbk = 1; g.sbn = nc;
  g.C = tmp; g.scm = r; g.scn = 1;
  OSMPS_TRY(gemm_f64(g, s));
  OSMPS_CUDA(cudaMemcpyAsync(m->A[k - 1], tmp, (size_t)chl0 * d0 * r * 8, cudaMemcpyDeviceToDevice, s));
  m->chi[k] = r;
  double* nrm = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);  // unit norm, as in shift_right
  if (!nrm) return st;
  OSMPS_TRY(vec_norm2(ctx, m->A[k - 1], chl0 * d0 * r, nrm, s));
  return vec_scale_by_inv_sqrt(m->A[k - 1], chl0 * d0 * r, nrm, s);
}

osmps_status ensure_envs(osmps_ctx* ctx, osmps_mps* m, const osmps_mpo* h, cudaStream_t s) {
  const int64_t L = m->L;
  bool realloc = m->Lenv.empty() || m->env_w != h->w;
  if (!realloc) return OSMPS_OK;
  OSMPS_CUDA(cudaStreamSynchronize(s));
  for (auto p : m->Lenv) if (p) cudaFree(p);
  for (auto p : m->Renv) if (p) cudaFree(p);
  m->Lenv.assign(L + 1, nullptr);
  m->Renv.assign(L + 1, nullptr);
  m->lvalid.assign(L + 1, 0);
  m->rvalid.assign(L + 1, 0);
  for (int64_t k = 0; k <= L; ++k) {
    const size_t bytes = (size_t)m->cap[k] * h->w[k] * m->cap[k] * 8;
    if (cudaMalloc(&m->Lenv[k], bytes) != cudaSuccess || cudaMalloc(&m->Renv[k], bytes) != cudaSuccess) {
      cudaGetLastError();
      return set_error(OSMPS_ENOMEM, "environments: cudaMalloc failed at bond %lld", (long long)k);
    }
  }
  m->env_w = h->w;
  { k_fill<<<1, 32, 0, s>>>(m->Lenv[0], 1, 1.0); note_launch(); }
  { k_fill<<<1, 32, 0, s>>>(m->Renv[L], 1, 1.0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  m->lvalid[0] = 1;
  m->rvalid[L] = 1;
  return OSMPS_OK;
}

// Mixed-canonical form with the orthogonality centre at `center`, normalised,
// with L environments up to `center` and R environments from center + 2.
osmps_status canonicalize(osmps_ctx* ctx, osmps_mps* m, const osmps_mpo* h, int64_t center,
                          int precision, cudaStream_t s) {
  OSMPS_TRY(ensure_envs(ctx, m, h, s));
  const int64_t L = m->L;
  for (int64_t k = 0; k < center; ++k) OSMPS_TRY(shift_right(ctx, m, k, s));
  for (int64_t k = L - 1; k > center; --k) OSMPS_TRY(shift_left(ctx, m, k, s));
  osmps_status st = OSMPS_OK;
  const int64_t nc = m->chi[center] * m->d[center] * m->chi[center + 1];
  double* nrm = (double*)ws_get(ctx, SLOT_SWEEP_ENV2, 64, s, &st);
  if (!nrm) return st;
  OSMPS_TRY(vec_norm2(ctx, m->A[center], nc, nrm, s));
  OSMPS_TRY(vec_scale_by_inv_sqrt(m->A[center], nc, nrm, s));
  std::fill(m->lvalid.begin(), m->lvalid.end(), 0);
  std::fill(m->rvalid.begin(), m->rvalid.end(), 0);
  m->lvalid[0] = 1;
  m->rvalid[L] = 1;
  for (int64_t k = 0; k < center; ++k) {
    OSMPS_TRY(env_update_impl(ctx, 0, m->Lenv[k], m->A[k], h->W[k], m->Lenv[k + 1], m->chi[k],
                              m->d[k], m->chi[k + 1], h->w[k], h->w[k + 1], precision, s));
    m->lvalid[k + 1] = 1;
  }
  for (int64_t k = L - 1; k >= center + 2; --k) {
    OSMPS_TRY(env_update_impl(ctx, 1, m->Renv[k + 1], m->A[k], h->W[k], m->Renv[k], m->chi[k],
                              m->d[k], m->chi[k + 1], h->w[k + 1], h->w[k], precision, s));
    m->rvalid[k] = 1;
  }
  m->center = center;
  return OSMPS_OK;
}

struct StepOut {
  double energy = 0.0, discarded = 0.0, entropy = 0.0, resid = 0.0;
  int iters = 0;
  int64_t chi_new = 0;
  bool converged = true;
};

osmps_status two_site_step(osmps_ctx* ctx, osmps_mps* m, const osmps_mpo* h, int64_t k,
                           bool move_right, int64_t chi_max, double eps_local, double tol,
                           int max_iter, int precision, StepOut* out, cudaStream_t s) {
  if (!m->lvalid[k] || !m->rvalid[k + 2])
    return set_error(OSMPS_EINVAL, "step at (%lld,%lld): environments not built for this centre",
                     (long long)k, (long long)(k + 1));
  osmps_status st = OSMPS_OK;
  const int64_t chl = m->chi[k], chm = m->chi[k + 1], chr = m->chi[k + 2];
  const int64_t d1 = m->d[k], d2 = m->d[k + 1];
  double* theta = (double*)ws_get(ctx, SLOT_SWEEP_THETA, (size_t)chl * d1 * d2 * chr * 8, s, &st);
  if (!theta) return st;
  if (precision == OSMPS_PREC_FP64)
    OSMPS_TRY(theta_form_impl(m->A[k], m->A[k + 1], theta, chl, d1, chm, d2, chr, s));
  else
    OSMPS_TRY(theta_form_tc(ctx, m->A[k], m->A[k + 1], theta, chl, d1, chm, d2, chr, precision, s));
  double e = 0.0, res = 0.0;
  int it = 0;
  osmps_status ls = lanczos_impl(ctx, m->Lenv[k], h->W[k], h->W[k + 1], m->Renv[k + 2], theta, chl,
                                 d1, d2, chr, h->w[k], h->w[k + 1], h->w[k + 2], max_iter, tol,
                                 precision, &e, &it, &res, s);
  if (ls != OSMPS_OK && ls != OSMPS_ENOCONV) return ls;
  int64_t chn = 0;
  double disc = 0.0, ent = 0.0;
  OSMPS_TRY(split_impl(ctx, theta, m->A[k], m->A[k + 1], chl, d1, d2, chr, move_right ? 1 : 0,
                       chi_max, eps_local, &chn, &disc, &ent, nullptr, precision, s));
  m->chi[k + 1] = chn;
  if (move_right) {
    OSMPS_TRY(env_update_impl(ctx, 0, m->Lenv[k], m->A[k], h->W[k], m->Lenv[k + 1], chl, d1, chn,
                              h->w[k], h->w[k + 1], precision, s));
    m->lvalid[k + 1] = 1;
    m->rvalid[k + 1] = 0;
    m->center = k + 1;
  } else {
    OSMPS_TRY(env_update_impl(ctx, 1, m->Renv[k + 2], m->A[k + 1], h->W[k + 1], m->Renv[k + 1],
                              chn, d2, chr, h->w[k + 2], h->w[k + 1], precision, s));
    m->rvalid[k + 1] = 1;
    m->lvalid[k + 1] = 0;
    m->center = k;
  }
  out->energy = e;
  out->iters = it;
  out->resid = res;
  out->chi_new = chn;
  out->discarded = disc;
  out->entropy = ent;
  out->converged = (ls == OSMPS_OK);
  return OSMPS_OK;
}

osmps_status energy_impl(osmps_ctx* ctx, const osmps_mps* m, const osmps_mpo* h, double* E,
                         cudaStream_t s, double* norm_out = nullptr) {
  osmps_status st = OSMPS_OK;
  int64_t maxsz = 1;
  for (int64_t k = 0; k <= m->L; ++k) maxsz = std::max(maxsz, m->chi[k] * m->chi[k] * h->w[k]);
  double* e1 = (double*)ws_get(ctx, SLOT_SWEEP_ENV, (size_t)maxsz * 8, s, &st);
  if (!e1) return st;
  double* e2 = (double*)ws_get(ctx, SLOT_SWEEP_ENV2, (size_t)maxsz * 8, s, &st);
  if (!e2) return st;
  double vals[2];
  for (int pass = 0; pass < 2; ++pass) {  // pass 0: <psi|H|psi>, pass 1: <psi|psi>
    { k_fill<<<1, 32, 0, s>>>(e1, 1, 1.0); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    double* a = e1;
    double* b = e2;
    for (int64_t k = 0; k < m->L; ++k) {
      const double* W = pass == 0 ? h->W[k] : h->ident[k];
      const int64_t wi = pass == 0 ? h->w[k] : 1, wo = pass == 0 ? h->w[k + 1] : 1;
      OSMPS_TRY(env_update_impl(ctx, 0, a, m->A[k], W, b, m->chi[k], m->d[k], m->chi[k + 1], wi, wo,
                                OSMPS_PREC_FP64_EMU, s));
      std::swap(a, b);
    }
    OSMPS_CUDA(cudaMemcpyAsync(&vals[pass], a, 8, cudaMemcpyDeviceToHost, s));
  }
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (!(vals[1] > 0.0)) return set_error(OSMPS_ENAN, "energy: state norm %g", vals[1]);
  *E = vals[0] / vals[1];
  if (norm_out) *norm_out = vals[1];
  return OSMPS_OK;
}

// Site tensor of (H - c)^2 from W[a,t,u,x] (dims wl, d, d, wr):
//   out[(a wl + b), t, s, (x wr + y)] = sum_u W'[a,t,u,x] W'[b,u,s,y],
//   W' = W - (c / L) 1 on the local-term block [start = wl - 1, :, :, done = 0].
__global__ void k_mpo_shift_square(const double* __restrict__ W, int wl, int d, int wr, double cl,
                                   double* __restrict__ out) {
  const int64_t total = (int64_t)wl * wl * d * d * wr * wr;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e;
    const int y = (int)(r % wr); r /= wr;
    const int x = (int)(r % wr); r /= wr;
    const int sx = (int)(r % d); r /= d;
    const int t = (int)(r % d); r /= d;
    const int b = (int)(r % wl);
    const int a = (int)(r / wl);
    double acc = 0.0;
    for (int u = 0; u < d; ++u) {
      double w1 = W[(((int64_t)a * d + t) * d + u) * wr + x];
      double w2 = W[(((int64_t)b * d + u) * d + sx) * wr + y];
      if (a == wl - 1 && x == 0 && t == u) w1 -= cl;
      if (b == wl - 1 && y == 0 && u == sx) w2 -= cl;
      acc = fma(w1, w2, acc);
    }
    out[e] = acc;
  }
}

// V = <psi|(H - E)^2|psi> / <psi|psi> (Sec. 3.4 convergence parameters: the
// variance of the state), formed without the cancellation of <H^2> - E^2:
// E first, then the squared shifted MPO contracted with the state by
// float64-accurate left environment updates.
osmps_status variance_impl(osmps_ctx* ctx, const osmps_mps* m, const osmps_mpo* h, double* E,
                           double* V, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  double nrm = 0.0;
  OSMPS_TRY(energy_impl(ctx, m, h, E, s, &nrm));
  const int64_t L = m->L;
  std::vector<int64_t> off(L + 1, 0);
  int64_t maxsz = 1;
  for (int64_t k = 0; k < L; ++k) {
    const int64_t wl = h->w[k], wr = h->w[k + 1], d = h->d[k];
    if (wl * wl * d > 64 || d * wr * wr > 64)
      return set_error(OSMPS_EUNSUPPORTED, "variance: squared MPO block (w^2 d = %lld) above 64",
                       (long long)std::max(wl * wl * d, d * wr * wr));
    off[k + 1] = off[k] + wl * wl * d * d * wr * wr;
  }
  for (int64_t k = 0; k <= L; ++k) maxsz = std::max(maxsz, m->chi[k] * m->chi[k] * h->w[k] * h->w[k]);
  double* W2 = (double*)ws_get(ctx, SLOT_VAR, (size_t)off[L] * 8, s, &st);
  if (!W2) return st;
  for (int64_t k = 0; k < L; ++k) {
    const int64_t n = off[k + 1] - off[k];
    { k_mpo_shift_square<<<(int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 4096)), 256, 0, s>>>(
          h->W[k], (int)h->w[k], (int)h->d[k], (int)h->w[k + 1], *E / (double)L, W2 + off[k]); note_launch(); }
  }
  OSMPS_LAUNCH_CHECK();
  double* e1 = (double*)ws_get(ctx, SLOT_SWEEP_ENV, (size_t)maxsz * 8, s, &st);
  if (!e1) return st;
  double* e2 = (double*)ws_get(ctx, SLOT_SWEEP_ENV2, (size_t)maxsz * 8, s, &st);
  if (!e2) return st;
  { k_fill<<<1, 32, 0, s>>>(e1, 1, 1.0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  double* a = e1;
  double* b = e2;
  for (int64_t k = 0; k < L; ++k) {
    OSMPS_TRY(env_update_impl(ctx, 0, a, m->A[k], W2 + off[k], b, m->chi[k], m->d[k], m->chi[k + 1],
                              h->w[k] * h->w[k], h->w[k + 1] * h->w[k + 1], OSMPS_PREC_FP64_EMU, s));
    std::swap(a, b);
  }
  double v = 0.0;
  OSMPS_CUDA(cudaMemcpyAsync(&v, a, 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  *V = v / nrm;
  return OSMPS_OK;
}

// dE/dW_k for every site at a fixed state (Eq. mpo: H is linear in each W_k,
// so dE/dW_k = G_k / <psi|psi> with G_k the contraction of everything else).
// Right environments R_1..R_L come from one pass from the right; with
// `every` > 1 only R_L and the R_k with k a multiple of `every` are kept and
// the others are rebuilt block by block from the checkpoint above them, so
// about L/every + every environments are alive instead of L. The left
// environment is carried along (one alive at a time).
osmps_status energy_grad_impl(osmps_ctx* ctx, const osmps_mps* m, const osmps_mpo* h, double* gW,
                              int64_t every, int prec, double* E, double* norm_out,
                              cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t L = m->L;
  const int64_t stride = every > 1 ? std::min<int64_t>(every, L) : 1;
  auto envsz = [&](int64_t k) { return m->chi[k] * h->w[k] * m->chi[k]; };
  int64_t maxsz = 1;
  for (int64_t k = 0; k <= L; ++k) maxsz = std::max(maxsz, envsz(k));
  double* t0 = (double*)ws_get(ctx, SLOT_SWEEP_ENV, (size_t)maxsz * 8, s, &st);
  if (!t0) return st;
  double* t1 = (double*)ws_get(ctx, SLOT_SWEEP_ENV2, (size_t)maxsz * 8, s, &st);
  if (!t1) return st;
  // <psi|psi>: left pass with identity operators
  { k_fill<<<1, 32, 0, s>>>(t0, 1, 1.0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  {
    double* a = t0;
    double* b = t1;
    for (int64_t k = 0; k < L; ++k) {
      OSMPS_TRY(env_update_impl(ctx, 0, a, m->A[k], h->ident[k], b, m->chi[k], m->d[k],
                                m->chi[k + 1], 1, 1, prec, s));
      std::swap(a, b);
    }
    double nrm = 0.0;
    OSMPS_CUDA(cudaMemcpyAsync(&nrm, a, 8, cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return set_error(OSMPS_ENAN, "energy gradient: state norm %g", nrm);
    *norm_out = nrm;
  }
  const double inv_norm = 1.0 / *norm_out;
  // storage: checkpoints (k = L and multiples of stride in [1, L)), then a
  // segment of stride - 1 environments rebuilt per block
  auto is_ckpt = [&](int64_t k) { return k == L || (k >= 1 && k % stride == 0); };
  std::vector<int64_t> off(L + 1, -1);
  int64_t total = 0;
  for (int64_t k = 1; k <= L; ++k)
    if (is_ckpt(k)) { off[k] = total; total += envsz(k); }
  const int64_t seg_off = total;
  total += (stride - 1) * maxsz;
  double* store = (double*)ws_get(ctx, SLOT_GRAD_ENVS, (size_t)std::max<int64_t>(total, 1) * 8, s, &st);
  if (!store) return st;
  auto renv = [&](int64_t k, int64_t seg_base) -> double* {
    if (is_ckpt(k)) return store + off[k];
    return store + seg_off + (k - seg_base - 1) * maxsz;  // seg_base < k < seg_base + stride
  };
  // R_L = 1, then R_k = env(R_{k+1}, A_k, W_k) down to k = 1, keeping checkpoints
  { k_fill<<<1, 32, 0, s>>>(store + off[L], 1, 1.0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  {
    const double* cur = store + off[L];
    for (int64_t k = L - 1; k >= 1; --k) {
      double* out = is_ckpt(k) ? store + off[k] : (cur == t0 ? t1 : t0);
      OSMPS_TRY(env_update_impl(ctx, 1, cur, m->A[k], h->W[k], out, m->chi[k], m->d[k],
                                m->chi[k + 1], h->w[k + 1], h->w[k], prec, s));
      cur = out;
    }
  }
  // left to right: G_k from L_k and R_{k+1}, then L_{k+1}
  { k_fill<<<1, 32, 0, s>>>(t0, 1, 1.0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  double* a = t0;
  double* b = t1;
  int64_t goff = 0;
  for (int64_t base = 0; base < L; base += stride) {
    const int64_t top = std::min(base + stride, L);
    for (int64_t j = top - 1; j > base; --j)  // rebuild R_j for base < j < top
      OSMPS_TRY(env_update_impl(ctx, 1, renv(j + 1, base), m->A[j], h->W[j], renv(j, base),
                                m->chi[j], m->d[j], m->chi[j + 1], h->w[j + 1], h->w[j], prec, s));
    for (int64_t k = base; k < top; ++k) {
      OSMPS_TRY(site_energy_grad(ctx, a, m->A[k], renv(k + 1, base), gW + goff, m->chi[k], m->d[k],
                                 m->chi[k + 1], h->w[k], h->w[k + 1], inv_norm, prec, s));
      goff += h->w[k] * m->d[k] * m->d[k] * h->w[k + 1];
      OSMPS_TRY(env_update_impl(ctx, 0, a, m->A[k], h->W[k], b, m->chi[k], m->d[k], m->chi[k + 1],
                                h->w[k], h->w[k + 1], prec, s));
      std::swap(a, b);
    }
  }
  double num = 0.0;
  OSMPS_CUDA(cudaMemcpyAsync(&num, a, 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  *E = num * inv_norm;
  return OSMPS_OK;
}

}  // namespace

}  // namespace osmps

using namespace osmps;

extern "C" {

osmps_status osmps_mps_create(osmps_ctx* ctx, int64_t L, const int64_t* d, const int64_t* chi,
                              const double* const* host_tensors, int64_t chi_cap,
                              osmps_mps** out) {
  clear_error();
  if (!ctx || !d || !chi || !host_tensors || !out) return set_error(OSMPS_EINVAL, "osmps_mps_create: null argument");
  *out = nullptr;
  if (L < 2) return set_error(OSMPS_ESHAPE, "osmps_mps_create: L=%lld (need >= 2)", (long long)L);
  if (chi[0] != 1 || chi[L] != 1) return set_error(OSMPS_ESHAPE, "osmps_mps_create: boundary bonds must be 1");
  if (chi_cap < 1) return set_error(OSMPS_EINVAL, "osmps_mps_create: chi_cap %lld", (long long)chi_cap);
  for (int64_t k = 0; k < L; ++k) {
    if (d[k] < 1 || chi[k] < 1 || chi[k + 1] < 1 || !host_tensors[k])
      return set_error(OSMPS_ESHAPE, "osmps_mps_create: bad site %lld", (long long)k);
  }
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  osmps_mps* m = new osmps_mps();
  m->ctx = ctx;
  m->L = L;
  m->d.assign(d, d + L);
  m->chi.assign(chi, chi + L + 1);
  m->cap.assign(L + 1, 1);
  // cap[k] = max(chi[k], min(chi_cap, dims of either side))
  std::vector<double> left(L + 1, 1.0), right(L + 1, 1.0);
  for (int64_t k = 1; k <= L; ++k) left[k] = std::min(1e18, left[k - 1] * (double)d[k - 1]);
  for (int64_t k = L - 1; k >= 0; --k) right[k] = std::min(1e18, right[k + 1] * (double)d[k]);
  for (int64_t k = 0; k <= L; ++k) {
    const double b = std::min(left[k], right[k]);
    m->cap[k] = std::max<int64_t>(chi[k], (int64_t)std::min<double>((double)chi_cap, b));
  }
  m->A.assign(L, nullptr);
  for (int64_t k = 0; k < L; ++k) {
    const size_t bytes = (size_t)m->cap[k] * d[k] * m->cap[k + 1] * 8;
    if (cudaMalloc(&m->A[k], bytes) != cudaSuccess) {
      cudaGetLastError();
      osmps_mps_destroy(m);
      return set_error(OSMPS_ENOMEM, "osmps_mps_create: cudaMalloc failed at site %lld", (long long)k);
    }
    cudaError_t e = cudaMemcpy(m->A[k], host_tensors[k], (size_t)chi[k] * d[k] * chi[k + 1] * 8,
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      osmps_mps_destroy(m);
      return set_error(OSMPS_ECUDA, "osmps_mps_create: copy failed: %s", cudaGetErrorString(e));
    }
  }
  *out = m;
  return OSMPS_OK;
}

osmps_status osmps_mps_destroy(osmps_mps* m) {
  if (!m) return OSMPS_OK;
  cudaSetDevice(m->ctx->device);
  cudaDeviceSynchronize();
  for (auto p : m->A) if (p) cudaFree(p);
  for (auto p : m->Lenv) if (p) cudaFree(p);
  for (auto p : m->Renv) if (p) cudaFree(p);
  delete m;
  return OSMPS_OK;
}

osmps_status osmps_mps_bond_dims(const osmps_mps* m, int64_t* chi_out) {
  clear_error();
  if (!m || !chi_out) return set_error(OSMPS_EINVAL, "osmps_mps_bond_dims: null argument");
  for (int64_t k = 0; k <= m->L; ++k) chi_out[k] = m->chi[k];
  return OSMPS_OK;
}

osmps_status osmps_mps_get_tensor(const osmps_mps* m, int64_t k, double* host_out) {
  clear_error();
  if (!m || !host_out) return set_error(OSMPS_EINVAL, "osmps_mps_get_tensor: null argument");
  if (k < 0 || k >= m->L) return set_error(OSMPS_EINVAL, "osmps_mps_get_tensor: site %lld", (long long)k);
  OSMPS_CUDA(cudaSetDevice(m->ctx->device));
  OSMPS_CUDA(cudaDeviceSynchronize());
  OSMPS_CUDA(cudaMemcpy(host_out, m->A[k], (size_t)m->chi[k] * m->d[k] * m->chi[k + 1] * 8,
                        cudaMemcpyDeviceToHost));
  return OSMPS_OK;
}

const double* osmps_mps_device_tensor(const osmps_mps* m, int64_t k) {
  if (!m || k < 0 || k >= m->L) return nullptr;
  return m->A[k];
}

osmps_status osmps_mpo_create(osmps_ctx* ctx, int64_t L, const int64_t* d, const int64_t* w,
                              const double* const* host_W, osmps_mpo** out) {
  clear_error();
  if (!ctx || !d || !w || !host_W || !out) return set_error(OSMPS_EINVAL, "osmps_mpo_create: null argument");
  *out = nullptr;
  if (L < 2) return set_error(OSMPS_ESHAPE, "osmps_mpo_create: L=%lld", (long long)L);
  if (w[0] != 1 || w[L] != 1) return set_error(OSMPS_ESHAPE, "osmps_mpo_create: boundary MPO bonds must be 1");
  for (int64_t k = 0; k < L; ++k)
    if (d[k] < 1 || w[k] < 1 || w[k + 1] < 1 || !host_W[k])
      return set_error(OSMPS_ESHAPE, "osmps_mpo_create: bad site %lld", (long long)k);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  osmps_mpo* h = new osmps_mpo();
  h->ctx = ctx;
  h->L = L;
  h->d.assign(d, d + L);
  h->w.assign(w, w + L + 1);
  h->W.assign(L, nullptr);
  h->ident.assign(L, nullptr);
  for (int64_t k = 0; k < L; ++k) {
    const size_t bytes = (size_t)w[k] * d[k] * d[k] * w[k + 1] * 8;
    if (cudaMalloc(&h->W[k], bytes) != cudaSuccess || cudaMalloc(&h->ident[k], (size_t)d[k] * d[k] * 8) != cudaSuccess) {
      cudaGetLastError();
      osmps_mpo_destroy(h);
      return set_error(OSMPS_ENOMEM, "osmps_mpo_create: cudaMalloc failed");
    }
    OSMPS_CUDA(cudaMemcpy(h->W[k], host_W[k], bytes, cudaMemcpyHostToDevice));
    { k_identity_op<<<1, 64>>>(h->ident[k], d[k]); note_launch(); }
  }
  OSMPS_CUDA(cudaDeviceSynchronize());
  *out = h;
  return OSMPS_OK;
}

osmps_status osmps_mpo_destroy(osmps_mpo* h) {
  if (!h) return OSMPS_OK;
  cudaSetDevice(h->ctx->device);
  cudaDeviceSynchronize();
  for (auto p : h->W) if (p) cudaFree(p);
  for (auto p : h->ident) if (p) cudaFree(p);
  delete h;
  return OSMPS_OK;
}

static osmps_status check_pair(const osmps_mps* m, const osmps_mpo* h) {
  if (m->L != h->L) return set_error(OSMPS_ESHAPE, "MPS has %lld sites, MPO %lld", (long long)m->L, (long long)h->L);
  for (int64_t k = 0; k < m->L; ++k)
    if (m->d[k] != h->d[k]) return set_error(OSMPS_ESHAPE, "site %lld: MPS d=%lld, MPO d=%lld",
                                             (long long)k, (long long)m->d[k], (long long)h->d[k]);
  return OSMPS_OK;
}

osmps_status osmps_mps_canonicalize(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo,
                                    int64_t center, int precision, void* stream) {
  clear_error();
  if (!ctx || !mps || !mpo) return set_error(OSMPS_EINVAL, "osmps_mps_canonicalize: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  if (center < 0 || center >= mps->L - 1)
    return set_error(OSMPS_EINVAL, "osmps_mps_canonicalize: centre %lld", (long long)center);
  if (!valid_precision(precision)) return set_error(OSMPS_EINVAL, "osmps_mps_canonicalize: precision");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  OSMPS_TRY(canonicalize(ctx, mps, mpo, center, precision, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  return OSMPS_OK;
}

osmps_status osmps_sweep_step(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo, int64_t k,
                              int move_right, const osmps_sweep_params* p,
                              osmps_step_stats* out, void* stream) {
  clear_error();
  if (!ctx || !mps || !mpo || !p) return set_error(OSMPS_EINVAL, "osmps_sweep_step: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  if (k < 0 || k >= mps->L - 1) return set_error(OSMPS_EINVAL, "osmps_sweep_step: pair %lld", (long long)k);
  if (p->chi_max < 1 || p->lanczos_max_iter < 1 || p->lanczos_max_iter > 512 || !valid_precision(p->precision))
    return set_error(OSMPS_EINVAL, "osmps_sweep_step: bad parameters");
  if (mps->Lenv.empty()) return set_error(OSMPS_EINVAL, "osmps_sweep_step: call osmps_mps_canonicalize first");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  const double eps = p->eps_local < 0.0 ? 1e-12 / (4.0 * mps->L) : p->eps_local;
  StepOut so;
  OSMPS_TRY(two_site_step(ctx, mps, mpo, k, move_right != 0, std::min(p->chi_max, mps->cap[k + 1]),
                          eps, p->lanczos_tol, p->lanczos_max_iter, p->precision, &so,
                          (cudaStream_t)stream));
  if (out) {
    out->energy = so.energy;
    out->resid = so.resid;
    out->discarded = so.discarded;
    out->entropy = so.entropy;
    out->chi_new = so.chi_new;
    out->iters = so.iters;
    out->converged = so.converged ? 1 : 0;
  }
  return OSMPS_OK;
}

osmps_status osmps_sweep(osmps_ctx* ctx, osmps_mps* mps, const osmps_mpo* mpo,
                         const osmps_sweep_params* p, osmps_sweep_stats* stats, void* stream) {
  clear_error();
  auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !mps || !mpo || !p) return set_error(OSMPS_EINVAL, "osmps_sweep: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  if (p->chi_max < 1 || p->n_sweeps < 0 || p->refine_sweeps < 0 || p->lanczos_max_iter < 1 ||
      p->lanczos_max_iter > 512 || !valid_precision(p->precision) || !(p->lanczos_tol >= 0.0))
    return set_error(OSMPS_EINVAL, "osmps_sweep: bad parameters");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t L = mps->L;
  const double eps = p->eps_local < 0.0 ? 1e-12 / (4.0 * L) : p->eps_local;
  const int total_sweeps = p->n_sweeps + p->refine_sweeps;
  OSMPS_TRY(canonicalize(ctx, mps, mpo, 0, total_sweeps > 0 && p->n_sweeps > 0 ? p->precision : OSMPS_PREC_FP64, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  auto t_sweeps = std::chrono::steady_clock::now();
  osmps_sweep_stats st{};
  if (stats) {
    st.step_energies = stats->step_energies;
    st.step_iters = stats->step_iters;
  }
  int64_t idx = 0;
  // Refinement sweeps run float64-accurate contractions: emulated on the
  // tensor cores after tensor-core sweeps, plain float64 otherwise.
  const int refine_prec = p->precision == OSMPS_PREC_FP64 ? OSMPS_PREC_FP64 : OSMPS_PREC_FP64_EMU;
  for (int sw = 0; sw < total_sweeps; ++sw) {
    const int prec = sw < p->n_sweeps ? p->precision : refine_prec;
    if (sw == p->n_sweeps && sw > 0 && prec != p->precision) {
      // refinement: rebuild the right environments in the refinement precision
      OSMPS_TRY(canonicalize(ctx, mps, mpo, 0, refine_prec, s));
    }
    for (int dir = 0; dir < 2; ++dir) {
      for (int64_t i = 0; i < L - 1; ++i) {
        const int64_t k = dir == 0 ? i : L - 2 - i;
        StepOut so;
        OSMPS_TRY(two_site_step(ctx, mps, mpo, k, dir == 0, std::min(p->chi_max, mps->cap[k + 1]),
                                eps, p->lanczos_tol, p->lanczos_max_iter, prec, &so, s));
        st.last_step_energy = so.energy;
        st.max_discarded = std::max(st.max_discarded, so.discarded);
        st.max_chi = std::max(st.max_chi, so.chi_new);
        st.lanczos_iters += so.iters;
        st.nonconverged += so.converged ? 0 : 1;
        if (k == (L - 1) / 2) st.entropy_center = so.entropy;
        if (st.step_energies) st.step_energies[idx] = so.energy;
        if (st.step_iters) st.step_iters[idx] = so.iters;
        ++idx;
        st.steps++;
      }
    }
  }
  OSMPS_CUDA(cudaStreamSynchronize(s));
  auto t_energy = std::chrono::steady_clock::now();
  OSMPS_TRY(energy_impl(ctx, mps, mpo, &st.energy, s));
  auto t_end = std::chrono::steady_clock::now();
  st.seconds = std::chrono::duration<double>(t_end - t0).count();
  st.sweep_seconds = std::chrono::duration<double>(t_energy - t_sweeps).count();
  st.setup_seconds = std::chrono::duration<double>(t_sweeps - t0).count();
  st.energy_seconds = std::chrono::duration<double>(t_end - t_energy).count();
  if (stats) *stats = st;
  return OSMPS_OK;
}

osmps_status osmps_energy(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                          double* energy_out, void* stream) {
  clear_error();
  if (!ctx || !mps || !mpo || !energy_out) return set_error(OSMPS_EINVAL, "osmps_energy: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return energy_impl(ctx, mps, mpo, energy_out, (cudaStream_t)stream);
}

osmps_status osmps_energy_grad(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                               double* gW, int64_t gW_count, int64_t checkpoint_every,
                               int precision, double* energy_out, double* norm_out, void* stream) {
  clear_error();
  if (!ctx || !mps || !mpo || !gW) return set_error(OSMPS_EINVAL, "osmps_energy_grad: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  if (precision != OSMPS_PREC_FP64 && precision != OSMPS_PREC_FP64_EMU)
    return set_error(OSMPS_EINVAL, "osmps_energy_grad: precision %d (FP64 or FP64_EMU)", precision);
  if (checkpoint_every < 0) return set_error(OSMPS_EINVAL, "osmps_energy_grad: checkpoint_every < 0");
  int64_t need = 0;
  for (int64_t k = 0; k < mpo->L; ++k) {
    if (mpo->w[k] * mpo->d[k] > 64 || mpo->d[k] * mpo->w[k + 1] > 64)
      return set_error(OSMPS_EUNSUPPORTED, "osmps_energy_grad: site %lld MPO block too large", (long long)k);
    need += mpo->w[k] * mpo->d[k] * mpo->d[k] * mpo->w[k + 1];
  }
  if (gW_count != need)
    return set_error(OSMPS_ESHAPE, "osmps_energy_grad: gW holds %lld values, the MPO %lld",
                     (long long)gW_count, (long long)need);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  double E = 0.0, nrm = 0.0;
  OSMPS_TRY(energy_grad_impl(ctx, mps, mpo, gW, checkpoint_every, precision, &E, &nrm,
                             (cudaStream_t)stream));
  if (energy_out) *energy_out = E;
  if (norm_out) *norm_out = nrm;
  return OSMPS_OK;
}

osmps_status osmps_variance(osmps_ctx* ctx, const osmps_mps* mps, const osmps_mpo* mpo,
                            double* energy_out, double* variance_out, void* stream) {
  clear_error();
  if (!ctx || !mps || !mpo || !variance_out) return set_error(OSMPS_EINVAL, "osmps_variance: null argument");
  OSMPS_TRY(check_pair(mps, mpo));
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  double E = 0.0, V = 0.0;
  OSMPS_TRY(variance_impl(ctx, mps, mpo, &E, &V, (cudaStream_t)stream));
  if (energy_out) *energy_out = E;
  *variance_out = V;
  return OSMPS_OK;
}

osmps_status osmps_mpo_set(osmps_mpo* mpo, const double* const* host_W) {
  clear_error();
  if (!mpo || !host_W) return set_error(OSMPS_EINVAL, "osmps_mpo_set: null argument");
  for (int64_t k = 0; k < mpo->L; ++k)
    if (!host_W[k]) return set_error(OSMPS_EINVAL, "osmps_mpo_set: site %lld is NULL", (long long)k);
  OSMPS_CUDA(cudaSetDevice(mpo->ctx->device));
  OSMPS_CUDA(cudaDeviceSynchronize());
  for (int64_t k = 0; k < mpo->L; ++k) {
    const size_t bytes = (size_t)mpo->w[k] * mpo->d[k] * mpo->d[k] * mpo->w[k + 1] * 8;
    OSMPS_CUDA(cudaMemcpy(mpo->W[k], host_W[k], bytes, cudaMemcpyHostToDevice));
  }
  return OSMPS_OK;
}

}  // extern "C"
