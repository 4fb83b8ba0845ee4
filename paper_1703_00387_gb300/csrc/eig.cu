// Largest eigenpairs of a symmetric matrix in float64 for the split (Sec. 2,
// Eq. AAD_ULLUD: the eigendecomposition route to the truncated SVD), with the
// work that is not the Householder reduction taken off the float64 pipe.
//
//   1. T = Q^T G Q, tridiagonal, by Householder reflections (sytrd.cu: panels
//      on a cooperative kernel, trailing updates on the emulated GEMM; cuSOLVER
//      dsytrd above n = 8192).
//   2. The wanted eigenvalues of T by multisection on Sturm counts (sign
//      changes of the leading principal minors of T - x I), eight points per
//      eigenvalue on eight lanes: float32 counts on T / ||T|| narrow the
//      bracket to ~1e-5 ||T||; the padded bracket is checked at both ends
//      with float64 counts (the Gershgorin interval again if the check
//      fails) and narrowed to eps ||T|| with float64 counts.
//   3. One eigenvector per eigenvalue by inverse iteration: two solves with
//      T - lambda I (Gaussian elimination with partial pivoting on the
//      tridiagonal) from a pseudo-random start, one thread per eigenvalue;
//      the elimination keeps its running row in registers and the back
//      substitution multiplies by pivot reciprocals formed off the chain.
//   4. Orthonormalisation of the vectors by Cholesky QR applied twice: the
//      Gram matrix and the products on the float64-accurate emulated GEMM.
//      Vectors of nearly equal eigenvalues come out of step 3 as independent
//      combinations inside their cluster; step 4 turns them into an
//      orthonormal basis of it, so the kept space is right even where the
//      individual vectors of a cluster are not determined.
//   5. The back-transformation U = Q Z by blocks of reflectors in compact WY
//      form, Q_b = I - V T V^T, T the inverse of triu(V^T V, 1) + diag(1/tau),
//      each block three emulated-float64 GEMMs.
// The triangular inverses (of the Cholesky factor in step 4 and of T^-1 in
// step 5) are this file's column-parallel back substitution.
// Output: eigenvalues ascending, eigenvectors as rows (the layout the split uses).
#include <cfloat>
#include <cmath>
#include <cstring>

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

// float32 copies of T / ||T|| for the first multisection rounds
__global__ void k_t_to_f32(const double* __restrict__ ds, const double* __restrict__ e2s, int n,
                           float* __restrict__ d32, float* __restrict__ e232) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d32[i] = (float)ds[i];
    if (i < n - 1) e232[i] = (float)e2s[i];
  }
}

constexpr int MS_PTS = 16;  // multisection points (lanes) per eigenvalue
// Sixteen points (two eigenvalues per warp, four warps per block): measured
// 4.70 ms for the top 1024 of n = 2048 against 5.0 ms with 8 points in
// one-warp blocks and 5.8 ms with 32 (the chains are float64-bound).
constexpr int MS_BLOCK = 128;

// ev[j] = eigenvalue n - nev + j of T (ascending). A group of MS_PTS lanes
// works on one eigenvalue: each round every lane counts the eigenvalues of
// T / ||T|| below its point, and the group keeps the subinterval that holds
// the wanted one (the points with count <= idx form a prefix).
__global__ void __launch_bounds__(MS_BLOCK) k_multisect(const double* __restrict__ ds,
                                                  const double* __restrict__ e2s,
                                                  const float* __restrict__ d32,
                                                  const float* __restrict__ e232, int n, int nev,
                                                  const double* __restrict__ bounds,
                                                  double* __restrict__ ev) {
  const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / MS_PTS;
  const int p = threadIdx.x % MS_PTS;
  const int lane = threadIdx.x & 31;
  const int g0 = lane - p;  // first lane of the group
  const unsigned gmask = ((1u << MS_PTS) - 1u) << g0;  // MS_PTS < 32
  if (gid >= nev) return;  // whole groups leave together
  const int idx = n - nev + gid;
  const double tn = bounds[3];
  const double glo = bounds[0] / tn, ghi = bounds[1] / tn;
  // float32 rounds to a bracket of ~1e-5
  float flo = (float)glo, fhi = (float)ghi;
  flo = nextafterf(flo, -INFINITY);
  fhi = nextafterf(fhi, INFINITY);
  for (int it = 0; it < 24 && fhi - flo > 1e-5f; ++it) {
    const float x = flo + (fhi - flo) * (float)(p + 1) / (float)(MS_PTS + 1);
    const int c = sturm_count_f32(d32, e232, n, x);
    const int k = __popc(__ballot_sync(gmask, c <= idx) & gmask);
    const float xl = __shfl_sync(gmask, x, g0 + (k > 0 ? k - 1 : 0));
    const float xh = __shfl_sync(gmask, x, g0 + (k < MS_PTS ? k : MS_PTS - 1));
    if (k > 0) flo = xl;
    if (k < MS_PTS) fhi = xh;
  }
  // float64: check the padded bracket at both ends on the first round
  double lo = (double)flo - 1e-6, hi = (double)fhi + 1e-6;
  lo = fmax(lo, glo);
  hi = fmin(hi, ghi);
  {
    const double x = p == 0 ? lo : (p == MS_PTS - 1 ? hi : lo + (hi - lo) * p / (MS_PTS - 1));
    const double xs[1] = {x};
    int c[1];
    sturm_counts<1>(ds, e2s, n, xs, c);
    const unsigned below = __ballot_sync(gmask, c[0] <= idx) & gmask;
    const int k = __popc(below);
    const bool valid = ((below >> g0) & 1u) && !((below >> (g0 + MS_PTS - 1)) & 1u);
    const double xl = __shfl_sync(gmask, x, g0 + (k > 0 ? k - 1 : 0));
    const double xh = __shfl_sync(gmask, x, g0 + (k < MS_PTS ? k : MS_PTS - 1));
    if (valid) {
      lo = xl;
      hi = xh;
    } else {
      lo = glo;
      hi = ghi;
    }
  }
  // absolute tolerance eps ||T||: the eigenvalues of a Gram matrix carry that
  // much rounding anyway
  const double tol = DBL_EPSILON;
  for (int it = 0; it < 80 && hi - lo > tol; ++it) {
    const double x = lo + (hi - lo) * (p + 1) / (MS_PTS + 1);
    const bool inside = x > lo && x < hi;
    if (!__all_sync(gmask, inside)) break;  // no representable point left between
    const double xs[1] = {x};
    int c[1];
    sturm_counts<1>(ds, e2s, n, xs, c);
    const int k = __popc(__ballot_sync(gmask, c[0] <= idx) & gmask);
    const double xl = __shfl_sync(gmask, x, g0 + (k > 0 ? k - 1 : 0));
    const double xh = __shfl_sync(gmask, x, g0 + (k < MS_PTS ? k : MS_PTS - 1));
    if (k > 0) lo = xl;
    if (k < MS_PTS) hi = xh;
  }
  if (p == 0) ev[gid] = 0.5 * (lo + hi) * tn;
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
// turns them into an orthonormal completion of the resolved ones.
// The elimination with partial pivoting runs down the rows with the current
// row in registers (only the pivot division is on the dependence chain) and
// stores, per row, the reciprocal of the final pivot, the first
// superdiagonal of U, the multiplier and whether rows i, i+1 were swapped (a
// swap puts e[i+1] on the second superdiagonal, so that needs no storage).
// Work arrays are interleaved across eigenvalues (W[i * nev + j]) so that
// neighbouring threads touch neighbouring addresses. The two sweeps of each
// solve carry a dependence chain of one or three float64 operations per row,
// and the row's stored factors come from L2: they are loaded IV_AHEAD rows at
// a time into registers before that chunk's chain runs, so the chain does not
// wait for one load round trip per row. (The arithmetic and its order are
// those of the plain row loop.)
constexpr int IV_AHEAD = 8;

__global__ void k_inviter(const double* __restrict__ d, const double* __restrict__ e, int n,
                          int nev, const double* __restrict__ ev,
                          const double* __restrict__ bounds, double* __restrict__ rcp,
                          double* __restrict__ mu, double* __restrict__ ml, double* __restrict__ x,
                          unsigned char* __restrict__ piv, double* __restrict__ Z, uint64_t seed) {
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
  // rcp: 1 / pivot of row i (tiny pivots replaced); mu: first superdiagonal
  // of U; ml: multipliers; x: right-hand side / solution
#define AT(a, i) a[(int64_t)(i) * ld + j]
  auto store_pivot = [&](int i, double p) {
    if (fabs(p) < tiny) p = p < 0.0 ? -tiny : tiny;  // a zero (or tiny) pivot becomes a tiny one
    AT(rcp, i) = 1.0 / p;
  };
  // LU with partial pivoting of the tridiagonal (subdiagonal e): the running
  // row i is (di at column i, ui at column i+1)
  double di = d[0] - lam, ui = n > 1 ? e[0] : 0.0;
  for (int i = 0; i + 1 < n; ++i) {
    const double li = e[i], dn = d[i + 1] - lam, un = i + 2 < n ? e[i + 1] : 0.0;
    if (fabs(di) >= fabs(li)) {
      const double f = di != 0.0 ? li / di : 0.0;
      store_pivot(i, di);
      AT(mu, i) = ui;
      AT(ml, i) = f;
      AT(piv, i) = 0;
      di = fma(-f, ui, dn);
      ui = un;
    } else {
      const double f = di / li;
      store_pivot(i, li);
      AT(mu, i) = dn;
      AT(ml, i) = f;
      AT(piv, i) = 1;
      di = fma(-f, dn, ui);
      ui = -f * un;
    }
  }
  store_pivot(n - 1, di);
  for (int pass = 0; pass < 2; ++pass) {
    // forward: the row swaps and multipliers applied to the right-hand side;
    // row i reads x[i+1] (the previous solve, or the start vector) before row
    // i+1 overwrites it, as in the plain loop
    double xi = pass == 0 ? hash_uniform(seed, (uint64_t)j, 0) : AT(x, 0);
    int i = 0;
    for (; i + IV_AHEAD < n; i += IV_AHEAD) {
      double fq[IV_AHEAD], xq[IV_AHEAD];
      unsigned char pq[IV_AHEAD];
#pragma unroll
      for (int u = 0; u < IV_AHEAD; ++u) {
        fq[u] = AT(ml, i + u);
        pq[u] = AT(piv, i + u);
        xq[u] = pass == 0 ? hash_uniform(seed, (uint64_t)j, (uint64_t)(i + u + 1)) : AT(x, i + u + 1);
      }
#pragma unroll
      for (int u = 0; u < IV_AHEAD; ++u) {
        if (pq[u] == 0) {
          AT(x, i + u) = xi;
          xi = fma(-fq[u], xi, xq[u]);
        } else {
          AT(x, i + u) = xq[u];
          xi = fma(-fq[u], xq[u], xi);
        }
      }
    }
    for (; i + 1 < n; ++i) {
      const double xn = pass == 0 ? hash_uniform(seed, (uint64_t)j, (uint64_t)(i + 1)) : AT(x, i + 1);
      const double f = AT(ml, i);
      if (AT(piv, i) == 0) {
        AT(x, i) = xi;
        xi = fma(-f, xi, xn);
      } else {
        AT(x, i) = xn;
        xi = fma(-f, xn, xi);
      }
    }
    AT(x, n - 1) = xi;
    // back substitution with U (second superdiagonal e[i+1] where rows swapped)
    double x1 = 0.0, x2 = 0.0, nrm = 0.0;
    int r = n - 1;
    for (; r + 1 >= IV_AHEAD; r -= IV_AHEAD) {  // rows r, r-1, .., r-IV_AHEAD+1 (all >= 0)
      double vq[IV_AHEAD], mq[IV_AHEAD], eq[IV_AHEAD], rq[IV_AHEAD];
      unsigned char pq[IV_AHEAD];
#pragma unroll
      for (int u = 0; u < IV_AHEAD; ++u) {
        const int ii = r - u;
        vq[u] = AT(x, ii);
        mq[u] = ii + 1 < n ? AT(mu, ii) : 0.0;
        pq[u] = ii + 2 < n ? AT(piv, ii) : 0;
        eq[u] = ii + 2 < n ? e[ii + 1] : 0.0;
        rq[u] = AT(rcp, ii);
      }
#pragma unroll
      for (int u = 0; u < IV_AHEAD; ++u) {
        const int ii = r - u;
        double v = vq[u];
        if (ii + 1 < n) v = fma(-mq[u], x1, v);
        if (pq[u]) v = fma(-eq[u], x2, v);
        v *= rq[u];
        AT(x, ii) = v;
        nrm = fma(v, v, nrm);
        x2 = x1;
        x1 = v;
      }
    }
    for (; r >= 0; --r) {
      double v = AT(x, r);
      if (r + 1 < n) v = fma(-AT(mu, r), x1, v);
      if (r + 2 < n && AT(piv, r)) v = fma(-e[r + 1], x2, v);
      v *= AT(rcp, r);
      AT(x, r) = v;
      nrm = fma(v, v, nrm);
      x2 = x1;
      x1 = v;
    }
    const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    if (pass == 0)
      for (int k = 0; k < n; ++k) AT(x, k) *= sc;
    else
      for (int k = 0; k < n; ++k) Z[(int64_t)k * nev + col] = AT(x, k) * sc;
  }
#undef AT
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

// *emax = max |S_ij - delta_ij| over the k x k matrix S, as the bits of a
// non-negative double (which order like the double values)
__global__ void k_identity_err(const double* __restrict__ S, int64_t k,
                               unsigned long long* __restrict__ emax) {
  unsigned long long m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, c = e - r * k;
    const double d = fabs(S[e] - (r == c ? 1.0 : 0.0));
    const unsigned long long b = isfinite(d) ? (unsigned long long)__double_as_longlong(d)
                                             : 0x7FF0000000000000ull;
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
    m = x > m ? x : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(emax, m);
}

// rd[i] = 1 / U[i][i] (U column-major with leading dimension m)
__global__ void k_diag_rcp(const double* __restrict__ U, int64_t m, double* __restrict__ rd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    rd[i] = 1.0 / U[i * m + i];
}

// X = U^-1 for an upper-triangular m x m U (column-major, leading dimension
// m; the strict lower part is not read), X column-major with zeros below the
// diagonal. One block per column c of X solves U x = e_c by back
// substitution in column (axpy) order: x_i = x_i / U_ii, then x_r -= U_ri x_i
// for r < i, down to i = 0. Thread t holds rows t, t + NT, ... in registers;
// the finished x_i goes through a two-slot shared broadcast (one barrier
// per step); the next column of U is loaded one step ahead and the diagonal
// reciprocals (rd) come precomputed, so a step's dependence chain is one FMA
// and one multiplication.
template <int NT, int RPT>
__global__ void __launch_bounds__(NT) k_trtri_upper(const double* __restrict__ U,
                                                    const double* __restrict__ rd,
                                                    double* __restrict__ X, int m) {
  const int c = blockIdx.x, t = threadIdx.x;
  __shared__ double sx[2];
  double xr[RPT], ucur[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = t + NT * k;
    xr[k] = r == c ? rd[c] : 0.0;
    ucur[k] = r < c ? U[(int64_t)c * m + r] : 0.0;
    if (r == c) sx[c & 1] = xr[k];
  }
  __syncthreads();
  for (int i = c; i >= 1; --i) {
    const double xi = sx[i & 1];
    double unext[RPT];
    // a warp whose rows in slot k are all >= i has nothing left to do there
    // (x_r is final once the step passes r): the test is the same for every
    // lane of the warp, so such warps skip the float64 instructions instead of
    // issuing them with every lane masked off
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = t + NT * k;
      unext[k] = (t & ~31) + NT * k < i - 1 && r < i - 1 ? U[(int64_t)(i - 1) * m + r] : 0.0;
    }
    const double rnext = rd[i - 1];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const int r = t + NT * k;
      if ((t & ~31) + NT * k < i) {
        if (r < i) xr[k] = fma(-ucur[k], xi, xr[k]);
        if (r == i - 1) {
          xr[k] *= rnext;
          sx[(i - 1) & 1] = xr[k];
        }
        ucur[k] = unext[k];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = t + NT * k;
    if (r < m) X[(int64_t)c * m + r] = r <= c ? xr[k] : 0.0;
  }
}

// X = U^-1 (upper triangular, column-major, m <= 8192); rd: m doubles of scratch.
osmps_status trtri_upper(const double* U, double* X, double* rd, int64_t m, cudaStream_t s) {
  if (m < 1 || m > 8192) return set_error(OSMPS_ESHAPE, "triangular inverse: m=%lld", (long long)m);
  { k_diag_rcp<<<grid1(m), 256, 0, s>>>(U, m, rd); note_launch(); }
  const int mi = (int)m;
  if (m <= 256) { k_trtri_upper<256, 1><<<mi, 256, 0, s>>>(U, rd, X, mi); }
  else if (m <= 512) { k_trtri_upper<256, 2><<<mi, 256, 0, s>>>(U, rd, X, mi); }
  else if (m <= 1024) { k_trtri_upper<256, 4><<<mi, 256, 0, s>>>(U, rd, X, mi); }
  else if (m <= 2048) { k_trtri_upper<256, 8><<<mi, 256, 0, s>>>(U, rd, X, mi); }
  else if (m <= 4096) { k_trtri_upper<512, 8><<<mi, 512, 0, s>>>(U, rd, X, mi); }
  else { k_trtri_upper<512, 16><<<mi, 512, 0, s>>>(U, rd, X, mi); }
  note_launch();
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

// One Cholesky QR pass: dst = src R^-1 with R^T R = src^T src + shift I
// (src, dst n x k row-major; S k x k scratch). Returns false in *ok when the
// Cholesky factorisation breaks down (the columns are numerically dependent).
osmps_status cholqr_pass(osmps_ctx* ctx, const double* src, double* dst, int64_t n, int64_t k,
                         double* S, double shift, cudaStream_t s, bool* ok,
                         bool have_gram = false) {
  osmps_status st = OSMPS_OK;
  SplitView zt; zt.src = src; zt.rows = k; zt.K = n; zt.s0 = 1; zt.sk = k;  // S = src^T src
  if (!have_gram) OSMPS_TRY(gemm_emu(ctx, zt, zt, k, k, n, S, k, s));
  if (shift > 0.0) { k_add_diag<<<grid1(k), 256, 0, s>>>(S, k, shift); note_launch(); }
  int lw = 0;
  OSMPS_SOLVER(cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)k, S, (int)k, &lw));
  double* work = (double*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lw, 1) * 8 + 256, s, &st);
  if (!work) return st;
  double* Rinv = (double*)ws_get(ctx, SLOT_EIG_SCAL, (size_t)(k * k + k + 64) * 8, s, &st);
  if (!Rinv) return st;
  OSMPS_SOLVER(cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, (int)k, S, (int)k, work, lw,
                                ctx->dev_info));
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) {
    *ok = false;
    return OSMPS_OK;
  }
  OSMPS_TRY(trtri_upper(S, Rinv, Rinv + k * k, k, s));
  // dst[i][c] = sum_j src[i][j] Rinv(j, c), Rinv column-major (upper)
  SplitView a; a.src = src; a.rows = n; a.K = k; a.s0 = k; a.sk = 1;
  SplitView b; b.src = Rinv; b.rows = k; b.K = k; b.s0 = k; b.sk = 1;
  OSMPS_TRY(gemm_emu(ctx, a, b, n, k, k, dst, k, s));
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
  if (ok) {
    // the second pass is skipped when the first already left the columns
    // orthonormal to 32 eps (max |Z2^T Z2 - I|)
    SplitView zt; zt.src = Z2; zt.rows = k; zt.K = n; zt.s0 = 1; zt.sk = k;
    OSMPS_TRY(gemm_emu(ctx, zt, zt, k, k, n, S, k, s));
    unsigned long long* dmax = reinterpret_cast<unsigned long long*>(ctx->dev_flags + 10);
    OSMPS_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
    { k_identity_err<<<grid1(k * k), 256, 0, s>>>(S, k, dmax); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    unsigned long long h = 0;
    OSMPS_CUDA(cudaMemcpyAsync(&h, dmax, sizeof(h), cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    double err = 0.0;
    memcpy(&err, &h, sizeof(err));
    if (err <= 32.0 * DBL_EPSILON) {
      OSMPS_CUDA(cudaMemcpyAsync(Z, Z2, (size_t)n * k * 8, cudaMemcpyDeviceToDevice, s));
      return OSMPS_OK;
    }
    OSMPS_TRY(cholqr_pass(ctx, Z2, Z, n, k, S, 0.0, s, &ok, true));
  }
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
  float* d32 = (float*)ws_get(ctx, SLOT_EIG_F32, (size_t)(2 * n + 64) * 4, s, &st);
  if (!d32) return st;
  float* e232 = d32 + n;
  { k_t_to_f32<<<grid1(n), 256, 0, s>>>(ds, e2s, (int)n, d32, e232); note_launch(); }
  // MS_PTS lanes per eigenvalue, MS_BLOCK / MS_PTS eigenvalues per block
  { k_multisect<<<(int)cdiv(nev * MS_PTS, MS_BLOCK), MS_BLOCK, 0, s>>>(ds, e2s, d32, e232, (int)n,
                                                                     (int)nev, bounds, ev); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  double* Wk = (double*)ws_get(ctx, SLOT_EIG_X, (size_t)4 * n * nev * 8 + (size_t)n * nev + 256,
                              s, &st);
  if (!Wk) return st;
  unsigned char* pivk = reinterpret_cast<unsigned char*>(Wk + 4 * n * nev);
  double* Z = (double*)ws_get(ctx, SLOT_EIG_R, (size_t)2 * n * nev * 8, s, &st);
  if (!Z) return st;
  double* Z2 = Z + n * nev;
  // 8 eigenvalues per block: the sequential chains spread over the SMs
  { k_inviter<<<(int)cdiv(nev, 8), 8, 0, s>>>(dvec, evec, (int)n, (int)nev, ev, bounds, Wk,
                                              Wk + n * nev, Wk + 2 * n * nev, Wk + 3 * n * nev, pivk,
                                              Z, 0x5DEECE66Dull); note_launch(); }
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
  double* V = (double*)ws_get(ctx, SLOT_EIG_P, (size_t)(n * mbmax + 64) * 8, s, &st);
  if (!V) return st;
  double* Tw = (double*)ws_get(ctx, SLOT_EIG_SCAL, (size_t)(mbmax * mbmax + mbmax + 64) * 8, s, &st);
  if (!Tw) return st;
  const int64_t nref = n - 1;
  for (int64_t i0 = ((nref - 1) / WY) * WY; i0 >= 0; i0 -= WY) {
    const int64_t mb = std::min<int64_t>(WY, nref - i0);
    { k_build_v<<<grid1(n * mb), 256, 0, s>>>(G, tau, n, i0, mb, V); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    SplitView vt; vt.src = V; vt.rows = mb; vt.K = n; vt.s0 = 1; vt.sk = mb;  // V^T rows
    OSMPS_TRY(gemm_emu(ctx, vt, vt, mb, mb, n, Tb, mb, s));                  // V^T V
    { k_tinv<<<grid1(mb * mb), 256, 0, s>>>(Tb, tau + i0, mb); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    OSMPS_TRY(trtri_upper(Tb, Tw, Tw + mb * mb, mb, s));                        // T = (T^-1)^-1
    SplitView zt; zt.src = Z; zt.rows = nev; zt.K = n; zt.s0 = 1; zt.sk = nev;  // Z^T rows
    OSMPS_TRY(gemm_emu(ctx, vt, zt, mb, nev, n, W1, nev, s));                  // W1 = V^T Z
    SplitView ta; ta.src = Tw; ta.rows = mb; ta.K = mb; ta.s0 = 1; ta.sk = mb;  // T rows (col-major)
    SplitView w1t; w1t.src = W1; w1t.rows = nev; w1t.K = mb; w1t.s0 = 1; w1t.sk = nev;
    OSMPS_TRY(gemm_emu(ctx, ta, w1t, mb, nev, mb, W2, nev, s));                // W2 = T W1
    SplitView vr; vr.src = V; vr.rows = n; vr.K = mb; vr.s0 = mb; vr.sk = 1;
    SplitView w2t; w2t.src = W2; w2t.rows = nev; w2t.K = mb; w2t.s0 = 1; w2t.sk = nev;
    OSMPS_TRY(gemm_emu(ctx, vr, w2t, n, nev, mb, Z, nev, s, true));            // Z -= V W2
  }
  {
    int flag = 0;
    OSMPS_CUDA(cudaMemcpyAsync(&flag, ctx->dev_flags + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    if (flag != 0) {
      cudaMemsetAsync(ctx->dev_flags + 3, 0, sizeof(int), s);
      return set_error(OSMPS_ETIMEOUT, "eigensolver: a grid barrier wait of the reduction gave up");
    }
  }
  dim3 grid((unsigned)cdiv(n, 32), (unsigned)cdiv(nev, 32));
  { k_transpose_nk<<<grid, dim3(32, 8), 0, s>>>(Z, n, nev, Y); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

}  // namespace osmps
