// Lanczos ground state of H_eff (Sec. 3.4: the local eigenproblem is solved
// with matrix-vector products only).
//
// Krylov vectors, orthogonalisation and the tridiagonal eigensolve are all
// float64 on the device. Each step applies H_eff (any precision), projects
// the result against every stored Krylov vector twice (classical
// Gram-Schmidt, two passes: full reorthogonalisation), normalises, and
// solves the small tridiagonal problem for the lowest Ritz pair:
//   * the eigenvalue by Sturm-count multisection (32 points per round, one warp),
//   * its eigenvector by inverse iteration with a partially pivoted
//     tridiagonal LU (Gaussian elimination with row interchanges).
// The host reads three numbers per step (energy, residual estimate, beta)
// to decide whether to stop: residual estimate beta_j |s_j| <= tol.
#include <cmath>

#include "common.cuh"

namespace osmps {

namespace {

constexpr int MAXIT = 512;
constexpr int DOT_THREADS = 256;
constexpr int DOT_GROUP = 8;
constexpr int DOT_MAX_BLOCKS = 1024;

// scalar layout in SLOT_LZ_SCAL (doubles)
constexpr int OFF_ALPHA = 0;
constexpr int OFF_BETA = MAXIT;
constexpr int OFF_C1 = 2 * MAXIT;
constexpr int OFF_C2 = 3 * MAXIT;
constexpr int OFF_S = 4 * MAXIT;
constexpr int OFF_MISC = 5 * MAXIT;  // [0] e, [1] resid, [2] beta, [3] ||w||^2, [4] ||theta||^2
constexpr int OFF_PROJ = 5 * MAXIT + 16;  // coefficients against the projector rows
constexpr int MAX_PROJ = 64;
constexpr int SCAL_COUNT = 5 * MAXIT + 16 + 2 * MAX_PROJ;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-partial dot products of G consecutive Krylov vectors with w:
// part[(g0 + v) * nb + b] = sum over block b's elements of V[g0 + v][e] w[e].
// The float64 pipe is the narrowest unit on this GPU, so exactly one fused
// multiply-add is issued per (vector, element): the group size is a template
// parameter (no predicated-off FMAs), and each thread covers many elements so
// the warp reductions stay a small fraction of the float64 work.
template <int G>
__device__ __forceinline__ void multidot_group(const double* __restrict__ V, int64_t ld, int g0,
                                               const double* __restrict__ w, int64_t n,
                                               double* __restrict__ part,
                                               double (*sh)[DOT_GROUP]) {
  const int nb = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n2 = n >> 1;  // element pairs (16-byte loads); odd tail below
  const double2* V0 = reinterpret_cast<const double2*>(V + (int64_t)g0 * ld);
  const int64_t ld2 = ld >> 1;  // ld is even
  double acc[G];
#pragma unroll
  for (int v = 0; v < G; ++v) acc[v] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; e < n2;
       e += (int64_t)nb * DOT_THREADS) {
    const double2 wv = reinterpret_cast<const double2*>(w)[e];
    double2 x[G];
#pragma unroll
    for (int v = 0; v < G; ++v) x[v] = V0[v * ld2 + e];
#pragma unroll
    for (int v = 0; v < G; ++v) acc[v] = fma(x[v].x, wv.x, fma(x[v].y, wv.y, acc[v]));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < G; ++v) acc[v] = fma(V[(int64_t)(g0 + v) * ld + n - 1], w[n - 1], acc[v]);
  }
#pragma unroll
  for (int v = 0; v < G; ++v) {
    const double t = warp_sum(acc[v]);
    if (lane == 0) sh[warp][v] = t;
  }
  __syncthreads();
  if (threadIdx.x < G) {
    double t = 0.0;
    for (int k = 0; k < DOT_THREADS / 32; ++k) t += sh[k][threadIdx.x];
    part[(int64_t)(g0 + threadIdx.x) * nb + blockIdx.x] = t;
  }
  __syncthreads();
}

// part[i * nb + b] = sum over block b's elements of V[i][e] * w[e], i < nv:
// groups of DOT_GROUP vectors, then one group of the remainder.
__global__ void __launch_bounds__(DOT_THREADS, 3) k_multidot(const double* __restrict__ V, int64_t ld,
                                                          int nv, const double* __restrict__ w,
                                                          int64_t n, double* __restrict__ part) {
  __shared__ double sh[DOT_THREADS / 32][DOT_GROUP];
  int g0 = 0;
  for (; g0 + DOT_GROUP <= nv; g0 += DOT_GROUP) multidot_group<DOT_GROUP>(V, ld, g0, w, n, part, sh);
  switch (nv - g0) {
    case 1: multidot_group<1>(V, ld, g0, w, n, part, sh); break;
    case 2: multidot_group<2>(V, ld, g0, w, n, part, sh); break;
    case 3: multidot_group<3>(V, ld, g0, w, n, part, sh); break;
    case 4: multidot_group<4>(V, ld, g0, w, n, part, sh); break;
    case 5: multidot_group<5>(V, ld, g0, w, n, part, sh); break;
    case 6: multidot_group<6>(V, ld, g0, w, n, part, sh); break;
    case 7: multidot_group<7>(V, ld, g0, w, n, part, sh); break;
    default: break;
  }
}

// out[i] = sum_b part[i * nb + b] in a fixed order (one block per vector).
__global__ void k_multidot_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)blockIdx.x * nb + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
  }
}

// mode 0: w[e] -= sum_i c[i] V[i][e];  mode 1: w[e] = sum_i c[i] V[i][e]
// (two consecutive elements per thread, 16-byte loads; the vectors are
// 256-byte aligned with an even stride).
__global__ void k_combine(const double* __restrict__ V, int64_t ld, int nv,
                          const double* __restrict__ c, double* __restrict__ w, int64_t n,
                          int mode) {
  __shared__ double cs[MAXIT];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  const int64_t n2 = n >> 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double ax = 0.0, ay = 0.0;
    for (int i = 0; i < nv; ++i) {
      const double2 x = reinterpret_cast<const double2*>(V + (int64_t)i * ld)[e];
      ax = fma(cs[i], x.x, ax);
      ay = fma(cs[i], x.y, ay);
    }
    double2* wp = reinterpret_cast<double2*>(w) + e;
    if (mode == 0) {
      const double2 o = *wp;
      *wp = make_double2(o.x - ax, o.y - ay);
    } else {
      *wp = make_double2(ax, ay);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cs[i], V[(int64_t)i * ld + n - 1], a);
    w[n - 1] = (mode == 0) ? (w[n - 1] - a) : a;
  }
}

// x[e] = sum_i c[i] V[i][e] into an arbitrary (8-byte aligned) caller buffer.
__global__ void k_combine_scalar(const double* __restrict__ V, int64_t ld, int nv,
                                 const double* __restrict__ c, double* __restrict__ x, int64_t n) {
  __shared__ double cs[MAXIT];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cs[i], V[(int64_t)i * ld + e], a);
    x[e] = a;
  }
}

__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  // number of eigenvalues of the tridiagonal (a, b) below x
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < m; ++i) {
    if (q == 0.0) q = 1e-300;
    q = (a[i] - x) - b[i - 1] * b[i - 1] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Record alpha_j, beta_j, then the lowest eigenpair of T_{j+1}; one warp.
// Eigenvalue: Sturm-count multisection, 32 points per round (5 bits).
// Eigenvector: inverse iteration (3 solves) with a partially pivoted
// tridiagonal LU, run by lane 0.
__global__ void __launch_bounds__(32) k_tridiag(double* __restrict__ sc, int j) {
  __shared__ double a[MAXIT], b[MAXIT], x[MAXIT], dl[MAXIT], dd[MAXIT], du[MAXIT];
  const int m = j + 1;
  const int lane = threadIdx.x;
  if (lane == 0) {
    sc[OFF_ALPHA + j] = sc[OFF_C1 + j] + sc[OFF_C2 + j];
    sc[OFF_BETA + j] = sqrt(sc[OFF_MISC + 3]);
  }
  __syncwarp();
  for (int i = lane; i < m; i += 32) {
    a[i] = sc[OFF_ALPHA + i];
    b[i] = sc[OFF_BETA + i];  // b[i] couples i and i+1 (b[j] is the residual norm)
  }
  __syncwarp();
  double l = 1e300, h = -1e300;
  for (int i = lane; i < m; i += 32) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    l = fmin(l, a[i] - r);
    h = fmax(h, a[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
  }
  const double pad = 1e-12 * fmax(fabs(l), fabs(h)) + 1e-300;
  double lo = l - pad, hi = h + pad;
  for (int round = 0; round < 16; ++round) {
    if (!(hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double xt = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const unsigned hit = __ballot_sync(0xffffffffu, sturm_count(a, b, m, xt) >= 1);
    const int t = hit ? (__ffs(hit) - 1) : 32;
    const double nlo = lo + (hi - lo) * (double)t / 33.0;
    const double nhi = (t < 32) ? lo + (hi - lo) * (double)(t + 1) / 33.0 : hi;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) {
    const double e = 0.5 * (lo + hi);
    double tnorm = 0.0;
    for (int i = 0; i < m; ++i) tnorm = fmax(tnorm, fabs(a[i]) + 2.0 * fabs(b[i]));
    const double tiny = 1e-300 + 1e-18 * tnorm;
    for (int i = 0; i < m; ++i) x[i] = 1.0 / sqrt((double)m);
    for (int iter = 0; iter < 3; ++iter) {
      for (int i = 0; i < m; ++i) {
        dd[i] = a[i] - e;
        du[i] = (i < m - 1) ? b[i] : 0.0;
        dl[i] = (i < m - 1) ? b[i] : 0.0;
      }
      // Gaussian elimination with partial pivoting; dl[i] becomes the second
      // superdiagonal entry of row i after the sweep.
      for (int i = 0; i + 1 < m; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
          if (dd[i] == 0.0) dd[i] = tiny;
          const double f = dl[i] / dd[i];
          dd[i + 1] -= f * du[i];
          x[i + 1] -= f * x[i];
          dl[i] = 0.0;
        } else {
          const double f = dd[i] / dl[i];
          dd[i] = dl[i];
          const double t = dd[i + 1];
          dd[i + 1] = du[i] - f * t;
          if (i + 2 < m) {
            dl[i] = du[i + 1];
            du[i + 1] = -f * dl[i];
          } else {
            dl[i] = 0.0;
          }
          du[i] = t;
          const double bt = x[i];
          x[i] = x[i + 1];
          x[i + 1] = bt - f * x[i + 1];
        }
      }
      if (dd[m - 1] == 0.0) dd[m - 1] = tiny;
      x[m - 1] /= dd[m - 1];
      if (m > 1) x[m - 2] = (x[m - 2] - du[m - 2] * x[m - 1]) / dd[m - 2];
      for (int i = m - 3; i >= 0; --i)
        x[i] = (x[i] - du[i] * x[i + 1] - dl[i] * x[i + 2]) / dd[i];
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
      nrm = sqrt(nrm);
      if (!(nrm > 0.0) || !isfinite(nrm)) {
        for (int i = 0; i < m; ++i) x[i] = (i == 0) ? 1.0 : 0.0;
        break;
      }
      for (int i = 0; i < m; ++i) x[i] /= nrm;
    }
    for (int i = 0; i < m; ++i) sc[OFF_S + i] = x[i];
    sc[OFF_MISC + 0] = e;
    sc[OFF_MISC + 1] = b[j] * fabs(x[m - 1]);
    sc[OFF_MISC + 2] = b[j];
  }
}

// Blocks for k_multidot: at least 16 element pairs per thread, and no more
// blocks than fit on the GPU in one wave (3 per SM at its register use).
int dot_blocks(int64_t n, int sm_count) {
  int64_t b = cdiv(n, DOT_THREADS * 32);
  const int64_t wave = 3 * (int64_t)(sm_count > 0 ? sm_count : 1);
  if (b > wave) b = wave;
  if (b > DOT_MAX_BLOCKS) b = DOT_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

int ew_blocks(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

// w -= V^T-projection of w onto the nv stored Krylov vectors (rows of V with
// an even stride ld, 16-byte aligned like w), coefficients to coef.
osmps_status project(osmps_ctx* ctx, const double* V, int64_t ld, int64_t n, int nv, double* w,
                     double* part, double* coef, cudaStream_t s) {
  const int nb = dot_blocks(n, ctx->sm_count);
  { k_multidot<<<nb, DOT_THREADS, 0, s>>>(V, ld, nv, w, n, part); note_launch(); }
  { k_multidot_final<<<nv, 256, 0, s>>>(part, nb, coef); note_launch(); }
  { k_combine<<<ew_blocks(n), 256, 0, s>>>(V, ld, nv, coef, w, n, 0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

}  // namespace

osmps_status lanczos_core(osmps_ctx* ctx, int64_t n, double* theta, int max_iter, double tol,
                          const Matvec& matvec, double* energy, int* iters, double* resid,
                          cudaStream_t s, const double* P, int64_t ldp, int kp) {
  osmps_status st = OSMPS_OK;
  const int64_t ld = (n + 1) & ~(int64_t)1;  // even row stride: 16-byte aligned rows
  if (max_iter > n) max_iter = (int)n;
  double* V = (double*)ws_get(ctx, SLOT_LZ_BASIS, (size_t)max_iter * ld * 8, s, &st);
  if (!V) return st;
  double* w = (double*)ws_get(ctx, SLOT_LZ_W, (size_t)n * 8, s, &st);
  if (!w) return st;
  double* sc = (double*)ws_get(ctx, SLOT_LZ_SCAL, SCAL_COUNT * 8, s, &st);
  if (!sc) return st;
  double* part = (double*)ws_get(ctx, SLOT_LZ_PART, (size_t)MAXIT * DOT_MAX_BLOCKS * 8, s, &st);
  if (!part) return st;
  OSMPS_TRY(pinned_reserve(ctx, 16));

  // v_0 = theta / ||theta||
  OSMPS_TRY(vec_norm2(ctx, theta, n, sc + OFF_MISC + 4, s));
  OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC + 4, 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (!(ctx->host_pinned[0] > 0.0) || !std::isfinite(ctx->host_pinned[0]))
    return set_error(ctx->host_pinned[0] == 0.0 ? OSMPS_EINVAL : OSMPS_ENAN,
                     "lanczos: start vector has norm^2 %g", ctx->host_pinned[0]);
  OSMPS_CUDA(cudaMemcpyAsync(V, theta, n * 8, cudaMemcpyDeviceToDevice, s));
  if (kp > 0) {
    // start in the orthogonal complement of the projector rows (two passes)
    OSMPS_TRY(project(ctx, P, ldp, n, kp, V, part, sc + OFF_PROJ, s));
    OSMPS_TRY(project(ctx, P, ldp, n, kp, V, part, sc + OFF_PROJ + MAX_PROJ, s));
    OSMPS_TRY(vec_norm2(ctx, V, n, sc + OFF_MISC + 4, s));
    OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC + 4, 8, cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    if (!(ctx->host_pinned[0] > 0.0))
      return set_error(OSMPS_EINVAL, "lanczos: start vector lies in the span of the projector rows");
  }
  OSMPS_TRY(vec_scale_by_inv_sqrt(V, n, sc + OFF_MISC + 4, s));

  int m = 0;
  double e = 0.0, res = 0.0;
  bool converged = false;
  for (int j = 0; j < max_iter; ++j) {
    double* vj = V + (int64_t)j * ld;
    OSMPS_TRY(matvec(vj, w));
    if (kp > 0) {  // the operator restricted to the complement: w <- (1 - P^T P) H v_j
      OSMPS_TRY(project(ctx, P, ldp, n, kp, w, part, sc + OFF_PROJ, s));
      OSMPS_TRY(project(ctx, P, ldp, n, kp, w, part, sc + OFF_PROJ + MAX_PROJ, s));
    }
    OSMPS_TRY(project(ctx, V, ld, n, j + 1, w, part, sc + OFF_C1, s));
    OSMPS_TRY(project(ctx, V, ld, n, j + 1, w, part, sc + OFF_C2, s));
    OSMPS_TRY(vec_norm2(ctx, w, n, sc + OFF_MISC + 3, s));
    { k_tridiag<<<1, 32, 0, s>>>(sc, j); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC, 3 * 8, cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    e = ctx->host_pinned[0];
    res = ctx->host_pinned[1];
    const double beta = ctx->host_pinned[2];
    m = j + 1;
    if (!std::isfinite(e) || !std::isfinite(res))
      return set_error(OSMPS_ENAN, "lanczos: non-finite Ritz value at step %d", j);
    if (res <= tol || beta == 0.0 || m == n) {
      converged = true;
      break;
    }
    if (j + 1 == max_iter) break;
    OSMPS_TRY(vec_scale_by_inv(V + (int64_t)(j + 1) * ld, w, n, sc + OFF_BETA + j, s));
  }
  // Ritz vector theta = sum_i s_i v_i, normalised
  { k_combine_scalar<<<ew_blocks(n), 256, 0, s>>>(V, ld, m, sc + OFF_S, theta, n); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  OSMPS_TRY(vec_norm2(ctx, theta, n, sc + OFF_MISC + 4, s));
  OSMPS_TRY(vec_scale_by_inv_sqrt(theta, n, sc + OFF_MISC + 4, s));
  int flag = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&flag, ctx->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (flag & 1) {
    cudaMemsetAsync(ctx->dev_flags, 0, sizeof(int), s);
    return set_error(OSMPS_ETIMEOUT, "lanczos: a bounded device wait gave up");
  }
  *energy = e;
  *iters = m;
  if (resid) *resid = res;
  if (!converged)
    return set_error(OSMPS_ENOCONV, "lanczos: residual %.3e above tol %.3e after %d steps", res,
                     tol, m);
  return OSMPS_OK;
}

osmps_status lanczos_impl(osmps_ctx* ctx, const double* L, const double* W1, const double* W2,
                          const double* R, double* theta, int64_t chi_l, int64_t d1, int64_t d2,
                          int64_t chi_r, int64_t wl, int64_t wm, int64_t wr, int max_iter,
                          double tol, int precision, double* energy, int* iters, double* resid,
                          cudaStream_t s) {
  OSMPS_TRY(heff_prepare(ctx, L, W1, W2, R, chi_l, d1, d2, chi_r, wl, wm, wr, precision, s));
  const Matvec mv = [&](const double* x, double* y) {
    return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, x, y, chi_l, d1, d2, chi_r,
                           wl, wm, wr, precision, s, true);
  };
  return lanczos_core(ctx, chi_l * d1 * d2 * chi_r, theta, max_iter, tol, mv, energy, iters,
                      resid, s);
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_lanczos_ground(osmps_ctx* ctx, const double* L, const double* W1,
                                             const double* W2, const double* R,
                                             double* theta_inout, int64_t chi_l, int64_t d1,
                                             int64_t d2, int64_t chi_r, int64_t wl, int64_t wm,
                                             int64_t wr, int max_iter, double tol, int precision,
                                             double* energy_out, int* iters_out,
                                             double* resid_out, void* stream) {
  clear_error();
  if (!ctx || !L || !W1 || !W2 || !R || !theta_inout || !energy_out || !iters_out)
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground: null argument");
  if (max_iter < 1 || max_iter > MAXIT)
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground: max_iter %d outside [1, %d]", max_iter,
                     MAXIT);
  if (!(tol >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_lanczos_ground: tol %g", tol);
  if (!valid_precision(precision))
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground: precision %d", precision);
  for (int64_t x : {chi_l, d1, d2, chi_r, wl, wm, wr})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_lanczos_ground: non-positive or oversized dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return lanczos_impl(ctx, L, W1, W2, R, theta_inout, chi_l, d1, d2, chi_r, wl, wm, wr, max_iter,
                      tol, precision, energy_out, iters_out, resid_out, (cudaStream_t)stream);
}

// Lanczos on the operator restricted to the orthogonal complement of k given
// vectors (the local problem of the excited-state search, Sec. 4.1 eMPS,
// Eq. emps_lagrange: the Lagrange multipliers keep the state orthogonal to
// the lower eigenstates). The rows of P are copied, orthonormalised (two
// Gram-Schmidt passes each) and used as the projector.
extern "C" osmps_status osmps_lanczos_ground_projected(
    osmps_ctx* ctx, const double* L, const double* W1, const double* W2, const double* R,
    double* theta_inout, const double* P, int k, int64_t chi_l, int64_t d1, int64_t d2,
    int64_t chi_r, int64_t wl, int64_t wm, int64_t wr, int max_iter, double tol, int precision,
    double* energy_out, int* iters_out, double* resid_out, void* stream) {
  clear_error();
  if (!ctx || !L || !W1 || !W2 || !R || !theta_inout || !energy_out || !iters_out || (k > 0 && !P))
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: null argument");
  if (k < 0 || k > MAX_PROJ) return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: k=%d outside [0, %d]", k, MAX_PROJ);
  if (max_iter < 1 || max_iter > MAXIT)
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: max_iter %d", max_iter);
  if (!(tol >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: tol %g", tol);
  if (!valid_precision(precision))
    return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: precision %d", precision);
  for (int64_t x : {chi_l, d1, d2, chi_r, wl, wm, wr})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_lanczos_ground_projected: bad dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  const int64_t n = chi_l * d1 * d2 * chi_r;
  const int64_t ld = (n + 1) & ~(int64_t)1;
  double* Q = nullptr;
  if (k > 0) {
    Q = (double*)ws_get(ctx, SLOT_LZ_PROJ, (size_t)k * ld * 8, s, &st);
    if (!Q) return st;
    double* part = (double*)ws_get(ctx, SLOT_LZ_PART, (size_t)MAXIT * DOT_MAX_BLOCKS * 8, s, &st);
    if (!part) return st;
    double* sc = (double*)ws_get(ctx, SLOT_LZ_SCAL, SCAL_COUNT * 8, s, &st);
    if (!sc) return st;
    OSMPS_TRY(pinned_reserve(ctx, 16));
    for (int i = 0; i < k; ++i) {
      double* qi = Q + (int64_t)i * ld;
      OSMPS_CUDA(cudaMemcpyAsync(qi, P + (int64_t)i * n, n * 8, cudaMemcpyDeviceToDevice, s));
      if (i > 0) {
        OSMPS_TRY(project(ctx, Q, ld, n, i, qi, part, sc + OFF_PROJ, s));
        OSMPS_TRY(project(ctx, Q, ld, n, i, qi, part, sc + OFF_PROJ + MAX_PROJ, s));
      }
      OSMPS_TRY(vec_norm2(ctx, qi, n, sc + OFF_MISC + 5, s));
      OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC + 5, 8, cudaMemcpyDeviceToHost, s));
      OSMPS_CUDA(cudaStreamSynchronize(s));
      if (!(ctx->host_pinned[0] > 1e-300))
        return set_error(OSMPS_EINVAL, "osmps_lanczos_ground_projected: projector row %d is dependent", i);
      OSMPS_TRY(vec_scale_by_inv_sqrt(qi, n, sc + OFF_MISC + 5, s));
    }
  }
  OSMPS_TRY(heff_prepare(ctx, L, W1, W2, R, chi_l, d1, d2, chi_r, wl, wm, wr, precision, s));
  const Matvec mv = [&](const double* x, double* y) {
    return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, x, y, chi_l, d1, d2, chi_r,
                           wl, wm, wr, precision, s, true);
  };
  return lanczos_core(ctx, n, theta_inout, max_iter, tol, mv, energy_out, iters_out, resid_out, s,
                      Q, ld, k);
}

