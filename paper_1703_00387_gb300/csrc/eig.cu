// Largest eigenpairs of a symmetric matrix in float64 for the split (Sec. 2,
// Eq. AAD_ULLUD: the eigendecomposition route to the truncated SVD), with the
// work that is not the Householder reduction taken off the float64 pipe.
//
//   1. T = Q^T G Q, tridiagonal, by Householder reflections (sytrd.cu: panels
//      on a cooperative kernel, trailing updates on the emulated GEMM; cuSOLVER
//      dsytrd above n = 8192).
//   2. The wanted eigenvalues of T by bisection on Sturm counts (one thread
//      per eigenvalue; a count is the number of negative pivots of the LDL^T
//      factorisation of T - x I, with the usual tiny-pivot guard).
//   3. One eigenvector per eigenvalue by inverse iteration: two solves with
//      T - lambda I (Gaussian elimination with partial pivoting on the
//      tridiagonal) from a pseudo-random start, one thread per eigenvalue.
//   4. Orthonormalisation of the vectors by Cholesky QR applied twice: the
//      Gram matrix and the products on the float64-accurate emulated GEMM.
//      Vectors of nearly equal eigenvalues come out of step 3 as independent
//      combinations inside their cluster; step 4 turns them into an
//      orthonormal basis of it, so the kept space is right even where the
//      individual vectors of a cluster are not determined.
//   5. The back-transformation U = Q Z by blocks of reflectors in compact WY
//      form, Q_b = I - V T V^T (T from the Schreiber-Van Loan recurrence), each
//      block two emulated-float64 GEMMs.
// Output: eigenvalues ascending, eigenvectors as rows (the layout the split uses).
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "sturm.cuh"

namespace osmps {
namespace {

constexpr int WY = 512;  // reflectors per back-transformation block

// bounds = {gl, gu, pivmin, tnorm}; e2[i] = e[i]^2
__global__ void k_gersh(const double* __restrict__ d, const double* __restrict__ e, int n,
                        double* __restrict__ e2, double* __restrict__ bounds) {
  __shared__ double smin[256], smax[256], se2[256];
  double lo = DBL_MAX, hi = -DBL_MAX, m2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i < n - 1 ? fabs(e[i]) : 0.0;
    lo = fmin(lo, d[i] - el - er);
    hi = fmax(hi, d[i] + el + er);
    if (i < n - 1) {
      e2[i] = e[i] * e[i];
      m2 = fmax(m2, e2[i]);
    }
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  se2[threadIdx.x] = m2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
      se2[threadIdx.x] = fmax(se2[threadIdx.x], se2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double tnorm = fmax(fmax(fabs(smin[0]), fabs(smax[0])), DBL_MIN);
    const double pivmin = DBL_MIN * fmax(1.0, se2[0]);
    const double pad = 2.0 * DBL_EPSILON * tnorm + 2.0 * pivmin;
    bounds[0] = smin[0] - pad;
    bounds[1] = smax[0] + pad;
    bounds[2] = pivmin;
    bounds[3] = tnorm;
  }
}

// ds = d / tnorm, e2s = e^2 / tnorm^2 (the bisection works on T / ||T||)
__global__ void k_scale_t(const double* __restrict__ d, const double* __restrict__ e2, int n,
                          const double* __restrict__ bounds, double* __restrict__ ds,
                          double* __restrict__ e2s) {
  const double inv = 1.0 / bounds[3];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    ds[i] = d[i] * inv;
    if (i < n - 1) e2s[i] = e2[i] * inv * inv;
  }
}

// ev[j] = eigenvalue n - nev + j of T (ascending), by bisection on T / ||T||
// (one Sturm chain per thread: on this GPU's float64 pipe, several chains per
// thread with multisection measured slower than plain bisection).
__global__ void k_bisect(const double* __restrict__ ds, const double* __restrict__ e2s, int n,
                         int nev, const double* __restrict__ bounds, double* __restrict__ ev) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nev) return;
  const int idx = n - nev + j;
  const double tn = bounds[3];
  double lo = bounds[0] / tn, hi = bounds[1] / tn;
  // absolute tolerance eps ||T||: the eigenvalues of a Gram matrix carry that
  // much rounding anyway, and it bounds the count of halvings (~53)
  const double tol = DBL_EPSILON;
  for (int it = 0; it < 160; ++it) {
    if (hi - lo <= tol) break;
    const double mid[1] = {0.5 * (lo + hi)};
    if (!(mid[0] > lo && mid[0] < hi)) break;
    int c[1];
    sturm_counts<1>(ds, e2s, n, mid, c);
    if (c[0] > idx) hi = mid[0];
    else lo = mid[0];
  }
  ev[j] = 0.5 * (lo + hi) * tn;
}

__device__ __forceinline__ double hash_uniform(uint64_t seed, uint64_t a, uint64_t b) {
  uint64_t z = seed + a * 0x9E3779B97F4A7C15ull + b * 0xD1B54A32D192ED03ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;  // (-1, 1)
}

// Inverse iteration for eigenvalue j: x = (T - ev[j] I)^-1 x twice from a
// pseudo-random start, normalised, stored in column c = nev - 1 - j of Z
// (columns by decreasing eigenvalue): Z[i * nev + c] = x[i]. Eigenvalues at
// or below `noise` (the resolution of the Gram route, n eps ||T||) are not
// determined by the data; their columns get the normalised pseudo-random
// start instead, and the orthonormalisation that follows (columns in order)
// turns them into an orthonormal completion of the resolved ones. Work arrays
// are interleaved across eigenvalues (W[(k n + i) nev + j]) so that
// neighbouring threads touch neighbouring addresses.
__global__ void k_inviter(const double* __restrict__ d, const double* __restrict__ e, int n,
                          int nev, const double* __restrict__ ev,
                          const double* __restrict__ bounds, double* __restrict__ W,
                          double* __restrict__ Z, uint64_t seed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nev) return;
  const double lam = ev[j];
  const double tiny = DBL_EPSILON * fmax(bounds[3], DBL_MIN);
  const int64_t col = nev - 1 - j;
  if (lam <= (double)n * DBL_EPSILON * bounds[3]) {
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      const double v = hash_uniform(seed, (uint64_t)j, (uint64_t)i);
      nrm = fma(v, v, nrm);
    }
    const double sc = 1.0 / sqrt(nrm);
    for (int i = 0; i < n; ++i) Z[(int64_t)i * nev + col] = sc * hash_uniform(seed, (uint64_t)j, (uint64_t)i);
    return;
  }
  const int64_t ld = nev;
  double* md = W;                              // U diagonal
  double* mu = W + (int64_t)n * ld;            // U first superdiagonal
  double* mu2 = W + 2 * (int64_t)n * ld;       // U second superdiagonal
  double* ml = W + 3 * (int64_t)n * ld;        // multipliers
  double* mp = W + 4 * (int64_t)n * ld;        // 1 where rows i, i+1 were swapped
  double* x = W + 5 * (int64_t)n * ld;         // right-hand side / solution
#define AT(a, i) a[(int64_t)(i) * ld + j]
  for (int i = 0; i < n; ++i) {
    AT(md, i) = d[i] - lam;
    AT(mu, i) = i < n - 1 ? e[i] : 0.0;
    AT(mu2, i) = 0.0;
    AT(x, i) = hash_uniform(seed, (uint64_t)j, (uint64_t)i);
  }
  // LU with partial pivoting of the tridiagonal (subdiagonal e)
  for (int i = 0; i < n - 1; ++i) {
    const double di = AT(md, i), li = e[i];
    if (fabs(di) >= fabs(li)) {
      const double f = di != 0.0 ? li / di : 0.0;
      AT(ml, i) = f;
      AT(mp, i) = 0.0;
      AT(md, i + 1) -= f * AT(mu, i);
    } else {
      const double f = di / li;
      AT(md, i) = li;
      AT(ml, i) = f;
      AT(mp, i) = 1.0;
      const double t = AT(mu, i);
      AT(mu, i) = AT(md, i + 1);
      AT(md, i + 1) = t - f * AT(md, i + 1);
      if (i < n - 2) {
        AT(mu2, i) = AT(mu, i + 1);
        AT(mu, i + 1) = -f * AT(mu, i + 1);
      }
    }
  }
  for (int i = 0; i < n; ++i)  // a zero (or tiny) pivot is replaced by a tiny one
    if (fabs(AT(md, i)) < tiny) AT(md, i) = AT(md, i) < 0.0 ? -tiny : tiny;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n - 1; ++i) {  // forward: apply the row swaps and multipliers
      if (AT(mp, i) == 0.0) {
        AT(x, i + 1) -= AT(ml, i) * AT(x, i);
      } else {
        const double t = AT(x, i);
        AT(x, i) = AT(x, i + 1);
        AT(x, i + 1) = t - AT(ml, i) * AT(x, i + 1);
      }
    }
    double nrm = 0.0;
    for (int i = n - 1; i >= 0; --i) {  // back substitution with U
      double v = AT(x, i);
      if (i + 1 < n) v -= AT(mu, i) * AT(x, i + 1);
      if (i + 2 < n) v -= AT(mu2, i) * AT(x, i + 2);
      v /= AT(md, i);
      AT(x, i) = v;
      nrm = fma(v, v, nrm);
    }
    const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int i = 0; i < n; ++i) AT(x, i) *= sc;
  }
  for (int i = 0; i < n; ++i) Z[(int64_t)i * nev + col] = AT(x, i);
#undef AT
}

// Zero the strictly lower part of a column-major m x m matrix.
__global__ void k_zero_strict_lower(double* __restrict__ A, int64_t m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, r = e - c * m;
    if (r > c) A[e] = 0.0;
  }
}

// Reflectors i0 .. i0+mb-1 of dsytrd (lower) as a dense n x mb row-major V:
// column c holds v = (0,...,0, 1 at row i+1, A[i+2.., i]) with i = i0 + c,
// or zeros where tau_i = 0 (that reflector is the identity).
__global__ void k_build_v(const double* __restrict__ A, const double* __restrict__ tau, int64_t n,
                          int64_t i0, int64_t mb, double* __restrict__ V) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * mb;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / mb, c = e - r * mb, i = i0 + c;
    double v = 0.0;
    if (tau[i] != 0.0) {
      if (r == i + 1) v = 1.0;
      else if (r > i + 1) v = A[i * n + r];
    }
    V[e] = v;
  }
}

// T^-1 of the compact WY form, column-major upper triangular, in place over
// S = V^T V: T^-1 = strictly-upper(S) + diag(1 / tau) (Puglisi), with 1 on
// the diagonal where tau = 0 (V's column is zero there, so T's row and
// column do not enter V T V^T).
__global__ void k_tinv(double* __restrict__ S, const double* __restrict__ tau, int64_t mb) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < mb * mb;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / mb, r = e - c * mb;  // column-major (S is symmetric)
    if (r > c) S[e] = 0.0;
    else if (r == c) S[e] = tau[r] != 0.0 ? 1.0 / tau[r] : 1.0;
  }
}

__global__ void k_add_diag(double* __restrict__ S, int64_t k, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k;
       i += (int64_t)gridDim.x * blockDim.x)
    S[i * k + i] += v;
}

__global__ void k_sub_inplace(double* __restrict__ Z, const double* __restrict__ D, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    Z[e] -= D[e];
}

// Y[j * n + i] = U[i * nev + (nev - 1 - j)] (U's columns by decreasing eigenvalue)
__global__ void k_transpose_nk(const double* __restrict__ U, int64_t n, int64_t nev,
                               double* __restrict__ Y) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < nev) t[r][threadIdx.x] = U[i * nev + (nev - 1 - j)];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (i < n && j < nev) Y[j * n + i] = t[threadIdx.x][r];
  }
}

int grid1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 16384)); }

// One Cholesky QR pass: dst = src R^-1 with R^T R = src^T src + shift I
// (src, dst n x k row-major; S k x k scratch). Returns false in *ok when the
// Cholesky factorisation breaks down (the columns are numerically dependent).
osmps_status cholqr_pass(osmps_ctx* ctx, const double* src, double* dst, int64_t n, int64_t k,
                         double* S, double shift, cudaStream_t s, bool* ok) {
  osmps_status st = OSMPS_OK;
  SplitView zt; zt.src = src; zt.rows = k; zt.K = n; zt.s0 = 1; zt.sk = k;  // S = src^T src
  OSMPS_TRY(gemm_emu(ctx, zt, zt, k, k, n, S, k, s));
  if (shift > 0.0) { k_add_diag<<<grid1(k), 256, 0, s>>>(S, k, shift); note_launch(); }
  int lw = 0;
  OSMPS_SOLVER(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)k, S, (int)k, &lw));
  size_t dbytes = 0, hbytes = 0;
  OSMPS_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT,
                                           k, CUDA_R_64F, S, k, &dbytes, &hbytes));
  const size_t wbytes = std::max<size_t>((size_t)std::max(lw, 1) * 8, dbytes) + 256;
  double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, wbytes, s, &st);
  if (!work) return st;
  OSMPS_SOLVER(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)k, S, (int)k, work, lw,
                                ctx->dev_info));
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) {
    *ok = false;
    return OSMPS_OK;
  }
  std::vector<char> hbuf(std::max<size_t>(hbytes, 1));
  OSMPS_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, k,
                                CUDA_R_64F, S, k, work, dbytes, hbuf.data(), hbytes, ctx->dev_info));
  { k_zero_strict_lower<<<grid1(k * k), 256, 0, s>>>(S, k); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  // dst[i][c] = sum_j src[i][j] Rinv(j, c), Rinv column-major (upper)
  SplitView a; a.src = src; a.rows = n; a.K = k; a.s0 = k; a.sk = 1;
  SplitView b; b.src = S; b.rows = k; b.K = k; b.s0 = k; b.sk = 1;
  OSMPS_TRY(gemm_emu(ctx, a, b, n, k, k, dst, k, s));
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) return set_error(OSMPS_ECUDA, "eigensolver: triangular inverse failed (%d)", info);
  *ok = true;
  return OSMPS_OK;
}

// Orthonormal columns spanning Z's, result in Z: Cholesky QR twice; if that
// breaks down, shifted Cholesky QR (shift 11 (n k + k (k + 1)) u ||Z||^2 with
// ||Z||^2 <= k for unit columns) followed by Cholesky QR twice.
osmps_status orthonormalize(osmps_ctx* ctx, double* Z, double* Z2, int64_t n, int64_t k,
                            double* S, cudaStream_t s) {
  bool ok = true;
  OSMPS_TRY(cholqr_pass(ctx, Z, Z2, n, k, S, 0.0, s, &ok));
  if (ok) OSMPS_TRY(cholqr_pass(ctx, Z2, Z, n, k, S, 0.0, s, &ok));
  if (ok) return OSMPS_OK;
  // Z still holds the input (a failed pass writes nothing)
  const double shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * DBL_EPSILON * 0.5 * (double)k;
  OSMPS_TRY(cholqr_pass(ctx, Z, Z2, n, k, S, shift, s, &ok));
  if (!ok) return set_error(OSMPS_ECUDA, "eigensolver: shifted Cholesky QR failed");
  OSMPS_TRY(cholqr_pass(ctx, Z2, Z, n, k, S, 0.0, s, &ok));
  if (ok) OSMPS_TRY(cholqr_pass(ctx, Z, Z2, n, k, S, 0.0, s, &ok));
  if (!ok) return set_error(OSMPS_ECUDA, "eigensolver: Cholesky QR failed after the shifted pass");
  OSMPS_CUDA(cudaMemcpyAsync(Z, Z2, (size_t)n * k * 8, cudaMemcpyDeviceToDevice, s));
  return OSMPS_OK;
}

}  // namespace

osmps_status eig_top(osmps_ctx* ctx, double* G, int64_t n, int64_t nev, double* ev, double* Y,
                     cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  if (n < 2 || nev < 1 || nev > n) return set_error(OSMPS_ESHAPE, "eig_top: n=%lld nev=%lld", (long long)n, (long long)nev);
  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  double* dvec = (double*)ws_get(ctx, SLOT_EIG_E, (size_t)(6 * n + 16) * 8, s, &st);
  if (!dvec) return st;
  double* evec = dvec + n;
  double* tau = evec + n;
  double* e2 = tau + n;
  double* ds = e2 + n;
  double* e2s = ds + n;
  double* bounds = e2s + n;
  if (sytrd_supported(n)) {
    OSMPS_TRY(sytrd_tc(ctx, G, n, dvec, evec, tau, s));
  } else {
    int lw = 0;
    OSMPS_SOLVER(cusolverDnDsytrd_bufferSize(ctx->solver, CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n,
                                             dvec, evec, tau, &lw));
    double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lw, 1) * 8, s, &st);
    if (!work) return st;
    OSMPS_SOLVER(cusolverDnDsytrd(ctx->solver, CUBLAS_FILL_MODE_LOWER, (int)n, G, (int)n, dvec,
                                  evec, tau, work, lw, ctx->dev_info));
  }
  { k_gersh<<<1, 256, 0, s>>>(dvec, evec, (int)n, e2, bounds); note_launch(); }
  { k_scale_t<<<grid1(n), 256, 0, s>>>(dvec, e2, (int)n, bounds, ds, e2s); note_launch(); }
  // 8 eigenvalues per block: the multisections spread over the SMs
  { k_bisect<<<(int)cdiv(nev, 8), 8, 0, s>>>(ds, e2s, (int)n, (int)nev, bounds, ev); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  double* Wk = (double*)ws_get(ctx, SLOT_EIG_X, (size_t)6 * n * nev * 8, s, &st);
  if (!Wk) return st;
  double* Z = (double*)ws_get(ctx, SLOT_EIG_R, (size_t)2 * n * nev * 8, s, &st);
  if (!Z) return st;
  double* Z2 = Z + n * nev;
  { k_inviter<<<(int)cdiv(nev, 32), 32, 0, s>>>(dvec, evec, (int)n, (int)nev, ev, bounds, Wk, Z,
                                                0x5DEECE66Dull); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  const int64_t mbmax = std::min<int64_t>(WY, n - 1);
  double* S = (double*)ws_get(ctx, SLOT_EIG_S,
                              (size_t)(nev * nev + 2 * mbmax * nev + mbmax * mbmax + 64) * 8, s, &st);
  if (!S) return st;
  OSMPS_TRY(orthonormalize(ctx, Z, Z2, n, nev, S, s));  // result back in Z
  // U = Q Z, Q = H(0) ... H(n-2): blocks applied last to first,
  // Q_b = I - V T V^T, so Q_b Z = Z - V (T (V^T Z))
  double* W1 = S + nev * nev;
  double* W2 = W1 + mbmax * nev;
  double* Tb = W2 + mbmax * nev;
  double* V = (double*)ws_get(ctx, SLOT_EIG_P, (size_t)(n * mbmax + n * nev + 64) * 8, s, &st);
  if (!V) return st;
  double* D = V + n * mbmax;
  const int64_t nref = n - 1;
  for (int64_t i0 = ((nref - 1) / WY) * WY; i0 >= 0; i0 -= WY) {
    const int64_t mb = std::min<int64_t>(WY, nref - i0);
    { k_build_v<<<grid1(n * mb), 256, 0, s>>>(G, tau, n, i0, mb, V); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    SplitView vt; vt.src = V; vt.rows = mb; vt.K = n; vt.s0 = 1; vt.sk = mb;  // V^T rows
    OSMPS_TRY(gemm_emu(ctx, vt, vt, mb, mb, n, Tb, mb, s));                  // V^T V
    { k_tinv<<<grid1(mb * mb), 256, 0, s>>>(Tb, tau + i0, mb); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    size_t dbytes = 0, hbytes = 0;
    OSMPS_SOLVER(cusolverDnXtrtri_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT,
                                             mb, CUDA_R_64F, Tb, mb, &dbytes, &hbytes));
    double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, dbytes + 256, s, &st);
    if (!work) return st;
    std::vector<char> hbuf(std::max<size_t>(hbytes, 1));
    OSMPS_SOLVER(cusolverDnXtrtri(ctx->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, mb,
                                  CUDA_R_64F, Tb, mb, work, dbytes, hbuf.data(), hbytes,
                                  ctx->dev_info + 2));
    SplitView zt; zt.src = Z; zt.rows = nev; zt.K = n; zt.s0 = 1; zt.sk = nev;  // Z^T rows
    OSMPS_TRY(gemm_emu(ctx, vt, zt, mb, nev, n, W1, nev, s));                  // W1 = V^T Z
    SplitView ta; ta.src = Tb; ta.rows = mb; ta.K = mb; ta.s0 = 1; ta.sk = mb;  // T rows (col-major)
    SplitView w1t; w1t.src = W1; w1t.rows = nev; w1t.K = mb; w1t.s0 = 1; w1t.sk = nev;
    OSMPS_TRY(gemm_emu(ctx, ta, w1t, mb, nev, mb, W2, nev, s));                // W2 = T W1
    SplitView vr; vr.src = V; vr.rows = n; vr.K = mb; vr.s0 = mb; vr.sk = 1;
    SplitView w2t; w2t.src = W2; w2t.rows = nev; w2t.K = mb; w2t.s0 = 1; w2t.sk = nev;
    OSMPS_TRY(gemm_emu(ctx, vr, w2t, n, nev, mb, D, nev, s));                  // D = V W2
    { k_sub_inplace<<<grid1(n * nev), 256, 0, s>>>(Z, D, n * nev); note_launch(); }
    OSMPS_LAUNCH_CHECK();
  }
  {
    int info = 0;
    OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    if (info != 0) return set_error(OSMPS_ECUDA, "eigensolver: WY factor inverse failed (%d)", info);
  }
  dim3 grid((unsigned)cdiv(n, 32), (unsigned)cdiv(nev, 32));
  { k_transpose_nk<<<grid, dim3(32, 8), 0, s>>>(Z, n, nev, Y); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

}  // namespace osmps
