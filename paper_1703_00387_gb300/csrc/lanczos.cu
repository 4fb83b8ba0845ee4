// Lanczos ground state of H_eff (Sec. 3.4: the local eigenproblem is solved
// with matrix-vector products only).
//
// Krylov vectors, orthogonalisation and the tridiagonal eigensolve are all
// float64 on the device. Each step applies H_eff (any precision), projects
// the result against every stored Krylov vector twice (classical
// Gram-Schmidt, two passes: full reorthogonalisation), normalises, and
// solves the small tridiagonal problem for the lowest Ritz pair:
//   * the eigenvalue by Sturm-count multisection (128 points per round),
//   * its eigenvector from the twisted factorisation of T - e I.
// The stopping test (residual estimate beta_j |s_j| <= tol, the iteration
// cap, an exhausted Krylov space) is taken on the device, by the kernel that
// solves the tridiagonal problem, and kept with the index of the current
// Krylov vector in device memory. So one step is the same sequence of
// launches whatever the step number, and the steps can run either from a
// host loop that reads the decision after each step or as one CUDA graph
// whose conditional while-node repeats the recorded step on the device.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "sturm.cuh"

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
constexpr int OFF_STATE = OFF_MISC + 8;  // 4 ints in two double slots, below
constexpr int OFF_PROJ = 5 * MAXIT + 16;  // coefficients against the projector rows
constexpr int MAX_PROJ = 64;
constexpr int OFF_URE = 5 * MAXIT + 16 + 2 * MAX_PROJ;  // exp(-i tau T) e_1 (Krylov propagator)
constexpr int OFF_UIM = OFF_URE + MAXIT;
constexpr int SCAL_COUNT = OFF_UIM + MAXIT;
constexpr int MISC_READ = 10;  // doubles of OFF_MISC the host reads (the state included)

// Iteration state (ints at OFF_STATE): the index J of the Krylov vector the
// next step applies H_eff to, the stop code, and the number of Krylov vectors
// the Ritz vector combines.
constexpr int ST_J = 0, ST_STOP = 1, ST_M = 2;
constexpr int STOP_NONE = 0, STOP_CONVERGED = 1, STOP_CAP = 2, STOP_NONFINITE = 3;

__host__ __device__ inline int* lz_state(double* sc) { return reinterpret_cast<int*>(sc + OFF_STATE); }
__host__ __device__ inline const int* lz_state(const double* sc) {
  return reinterpret_cast<const int*>(sc + OFF_STATE);
}
// The state inside a host copy of the MISC_READ doubles from OFF_MISC on.
inline const int* lz_state_in_misc(const double* misc) {
  return reinterpret_cast<const int*>(misc + (OFF_STATE - OFF_MISC));
}

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
// block (b, y) takes element chunk b (nb = gridDim.x chunks) of the vector
// group starting at y * DOT_GROUP, so small vectors still spread over many
// SMs (the float64 FMA rate of one SM is the limit there).
// With jcur set, nv = jcur[0] + 1 (the Krylov vectors up to the current one).
__global__ void __launch_bounds__(DOT_THREADS, 3) k_multidot(const double* __restrict__ V, int64_t ld,
                                                          int nv, const double* __restrict__ w,
                                                          int64_t n, double* __restrict__ part,
                                                          const int* __restrict__ jcur,
                                                          const int* __restrict__ skip) {
  __shared__ double sh[DOT_THREADS / 32][DOT_GROUP];
  if (skip && *skip) return;
  if (jcur) nv = jcur[0] + 1;
  const int g0 = (int)blockIdx.y * DOT_GROUP;
  if (g0 >= nv) return;
  if (g0 + DOT_GROUP <= nv) {
    multidot_group<DOT_GROUP>(V, ld, g0, w, n, part, sh);
    return;
  }
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

// out[i] = sum_b part[i * nb + b] in a fixed order (one block per vector;
// with jcur set, blocks past vector jcur[0] return at once).
__global__ void k_multidot_final(const double* __restrict__ part, int nb, double* __restrict__ out,
                                 const int* __restrict__ jcur, const int* __restrict__ skip) {
  __shared__ double sh[32];
  if (jcur && (int)blockIdx.x > jcur[0]) return;
  if (skip && *skip) {  // a skipped pass contributes nothing
    if (threadIdx.x == 0) out[blockIdx.x] = 0.0;
    return;
  }
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
// 256-byte aligned with an even stride). With ACC = 4 the sum over i runs
// in four interleaved partial sums (i mod 4), added in a fixed order, which
// cuts the dependent float64 chain per element by four: the form for small
// vectors, where that chain is the cost. Large vectors are bandwidth-bound
// and stream one vector at a time faster (ACC = 1).
template <int ACC>
__global__ void k_combine(const double* __restrict__ V, int64_t ld, int nv,
                          const double* __restrict__ c, double* __restrict__ w, int64_t n,
                          int mode, const int* __restrict__ jcur,
                          const int* __restrict__ skip = nullptr) {
  __shared__ double cs[MAXIT];
  if (skip && *skip) return;
  if (jcur) nv = jcur[0] + 1;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  const int64_t n2 = n >> 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    double ax[ACC], ay[ACC];
#pragma unroll
    for (int q = 0; q < ACC; ++q) ax[q] = ay[q] = 0.0;
    int i = 0;
    for (; i + ACC <= nv; i += ACC) {
#pragma unroll
      for (int q = 0; q < ACC; ++q) {
        const double2 x = reinterpret_cast<const double2*>(V + (int64_t)(i + q) * ld)[e];
        ax[q] = fma(cs[i + q], x.x, ax[q]);
        ay[q] = fma(cs[i + q], x.y, ay[q]);
      }
    }
    for (int q = 0; i < nv; ++i, ++q) {
      const double2 x = reinterpret_cast<const double2*>(V + (int64_t)i * ld)[e];
      ax[q] = fma(cs[i], x.x, ax[q]);
      ay[q] = fma(cs[i], x.y, ay[q]);
    }
    double sx = ax[0], sy = ay[0];
    if (ACC == 4) {
      sx = (ax[0] + ax[1 % ACC]) + (ax[2 % ACC] + ax[3 % ACC]);
      sy = (ay[0] + ay[1 % ACC]) + (ay[2 % ACC] + ay[3 % ACC]);
    }
    double2* wp = reinterpret_cast<double2*>(w) + e;
    if (mode == 0) {
      const double2 o = *wp;
      *wp = make_double2(o.x - sx, o.y - sy);
    } else {
      *wp = make_double2(sx, sy);
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cs[i], V[(int64_t)i * ld + n - 1], a);
    w[n - 1] = (mode == 0) ? (w[n - 1] - a) : a;
  }
}

// The Ritz vector x[e] = sum_i s[i] V[i][e], i < m (the state's vector
// count), into an arbitrary (8-byte aligned) caller buffer; x is left as it
// is when the iteration stopped on a non-finite value.
__global__ void k_combine_scalar(const double* __restrict__ V, int64_t ld,
                                 const double* __restrict__ sc, double* __restrict__ x, int64_t n) {
  __shared__ double cs[MAXIT];
  const int* st = lz_state(sc);
  if (st[ST_STOP] == STOP_NONFINITE) return;
  const int nv = st[ST_M];
  const double* c = sc + OFF_S;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < nv; ++i) a = fma(cs[i], V[(int64_t)i * ld + e], a);
    x[e] = a;
  }
}

// Step j = state J: record alpha_j, beta_j, then the lowest eigenpair of
// T_{j+1}; one block of four warps (one per SM sub-partition: the float64
// pipe of a sub-partition is the limit for a single warp).
//   * Eigenvalue: multisection, 128 points per round (one per thread),
//     from the Gershgorin interval: first on float32 Sturm counts of T/||T||
//     down to 1e-5 ||T|| (the float32 pipe is far wider), then the bracket
//     is padded, checked with float64 counts at its ends (the full interval
//     again if the check fails), and narrowed to 4e-16 relative width on
//     division-free float64 counts (sturm.cuh).
//   * Eigenvector: the twisted factorisation of T - e I (top-down and
//     bottom-up pivot chains on two warps, twist index where |gamma| is
//     least, the vector by two product chains from it), normalised in
//     parallel.
// Then the stopping decision: a non-finite Ritz value or residual; converged
// (residual estimate <= tol, beta = 0, or the Krylov space is the whole
// space); the step cap. Without a stop, J advances. With set_cond, the
// decision is also the loop condition of the CUDA graph this kernel runs in
// (1 = run another step), so a graph loop ends after at most max_iter steps:
// J only advances below max_iter - 1.
constexpr int TRI_THREADS = 128;

// The first thread index whose flag is set (TRI_THREADS if none), for every
// thread of the block; flags grow with the index (Sturm counts grow with x).
__device__ __forceinline__ int first_set(bool flag, int* sh4) {
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh4[warp] = m ? warp * 32 + __ffs(m) - 1 : TRI_THREADS;
  __syncthreads();
  int t = TRI_THREADS;
  for (int w = 0; w < TRI_THREADS / 32; ++w) t = min(t, sh4[w]);
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(TRI_THREADS) k_tridiag(double* __restrict__ sc, int max_iter,
                                                         double tol, long long n,
                                                         cudaGraphConditionalHandle cond,
                                                         int set_cond) {
  __shared__ double a[MAXIT], b[MAXIT], b2[MAXIT], x[MAXIT], dd[MAXIT], du[MAXIT], ml[MAXIT],
      rd[MAXIT];
  __shared__ float af[MAXIT], b2f[MAXIT];
  __shared__ double red[2][TRI_THREADS / 32];
  __shared__ int sh4[TRI_THREADS / 32];
  int* st = lz_state(sc);
  const int j = st[ST_J];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (j < 0 || j >= max_iter || j >= MAXIT) {  // not reachable from the drivers below
    if (tid == 0) {
      st[ST_STOP] = STOP_NONFINITE;
      st[ST_M] = 1;
      if (set_cond) cudaGraphSetConditional(cond, 0u);
    }
    return;
  }
  const int m = j + 1;
  if (tid == 0) {
    sc[OFF_ALPHA + j] = sc[OFF_C1 + j] + sc[OFF_C2 + j];
    sc[OFF_BETA + j] = sqrt(sc[OFF_MISC + 3]);
  }
  __syncthreads();
  for (int i = tid; i < m; i += TRI_THREADS) {
    a[i] = sc[OFF_ALPHA + i];
    b[i] = sc[OFF_BETA + i];  // b[i] couples i and i+1 (b[j] is the residual norm)
    b2[i] = b[i] * b[i];
  }
  __syncthreads();
  double l = 1e300, h = -1e300;
  for (int i = tid; i < m; i += TRI_THREADS) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    l = fmin(l, a[i] - r);
    h = fmax(h, a[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
  }
  if (lane == 0) {
    red[0][warp] = l;
    red[1][warp] = h;
  }
  __syncthreads();
  l = red[0][0];
  h = red[1][0];
  for (int w = 1; w < TRI_THREADS / 32; ++w) {
    l = fmin(l, red[0][w]);
    h = fmax(h, red[1][w]);
  }
  const double tn = fmax(fabs(l), fabs(h)) + 1e-300;
  const double pad = 1e-12 * tn + 1e-300;
  const double gl = l - pad, gh = h + pad;  // the Gershgorin interval
  // float32 phase on T / tn
  const double inv = 1.0 / tn;
  for (int i = tid; i < m; i += TRI_THREADS) {
    af[i] = (float)(a[i] * inv);
    b2f[i] = (float)(b2[i] * inv * inv);
  }
  __syncthreads();
  double lo = gl, hi = gh;
  for (int round = 0; round < 8; ++round) {
    if (!(hi - lo > 1e-5 * tn)) break;
    const double step = (hi - lo) * (1.0 / (TRI_THREADS + 1));
    const double xt = lo + step * (double)(tid + 1);
    const bool hit = sturm_count_f32(af, b2f, m, (float)(xt * inv)) >= 1;
    const int t = first_set(hit, sh4);
    const double nlo = lo + step * (double)t;
    const double nhi = (t < TRI_THREADS) ? lo + step * (double)(t + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  // float64 phase: the padded bracket, its ends checked in the first round
  {
    const double fpad = 4e-5 * tn;
    lo = fmax(gl, lo - fpad);
    hi = fmin(gh, hi + fpad);
  }
  bool check = true;  // this round includes the bracket's ends
  for (int round = 0; round < 40; ++round) {
    if (!check && !(hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
    double xt, step;
    if (check) {  // points lo, ..., hi (ends included)
      step = (hi - lo) * (1.0 / (TRI_THREADS - 1));
      xt = (tid == TRI_THREADS - 1) ? hi : lo + step * (double)tid;
    } else {
      step = (hi - lo) * (1.0 / (TRI_THREADS + 1));
      xt = lo + step * (double)(tid + 1);
    }
    const double xs[1] = {xt};
    int c[1];
    sturm_counts<1>(a, b2, m, xs, c);
    const int t = first_set(c[0] >= 1, sh4);
    if (check) {
      check = false;
      if (t == 0 || t == TRI_THREADS) {  // the float32 bracket missed: the full interval
        lo = gl;
        hi = gh;
        continue;
      }
      const double nlo = lo + step * (double)(t - 1);
      const double nhi = (t == TRI_THREADS - 1) ? hi : lo + step * (double)t;
      lo = nlo;
      hi = nhi;
    } else {
      const double nlo = lo + step * (double)t;
      const double nhi = (t < TRI_THREADS) ? lo + step * (double)(t + 1) : hi;
      lo = nlo;
      hi = nhi;
    }
  }
  const double e = 0.5 * (lo + hi);
  // Eigenvector of T - e I by the twisted factorisation: the top-down pivots
  // dp (T - e I = L D+ L^T, multipliers lq) and the bottom-up pivots dm
  // (= U D- U^T, multipliers uq) on two warps at once; the twist index r
  // minimises |gamma_k| = |dp_k + dm_k - (a_k - e)| (gamma_k^-1 is the k-th
  // diagonal entry of (T - e I)^-1, largest where the eigenvector is); then
  // z_r = 1, z_i = -lq_i z_(i+1) above r and z_(i+1) = -uq_i z_i below it, the
  // two product chains again on two warps. A zero pivot becomes a tiny one of
  // the same sign.
  const double tiny = 1e-300 + 1e-18 * tn;
  if (tid == 0) {
    double d = a[0] - e;
    for (int i = 0; i + 1 < m; ++i) {
      if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
      dd[i] = d;
      const double l = b[i] / d;
      ml[i] = l;
      d = (a[i + 1] - e) - l * b[i];
    }
    if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
    dd[m - 1] = d;
  } else if (tid == 32) {
    double d = a[m - 1] - e;
    for (int i = m - 2; i >= 0; --i) {
      if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
      du[i + 1] = d;
      const double u = b[i] / d;
      rd[i] = u;
      d = (a[i] - e) - u * b[i];
    }
    if (fabs(d) < tiny) d = d < 0.0 ? -tiny : tiny;
    du[0] = d;
  }
  __syncthreads();
  // twist index: smallest |gamma|, ties to the smallest index
  double gbest = 1e308;
  int rbest = 0;
  for (int k = tid; k < m; k += TRI_THREADS) {
    const double g = fabs(dd[k] + du[k] - (a[k] - e));
    if (g < gbest) {
      gbest = g;
      rbest = k;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double go = __shfl_xor_sync(0xffffffffu, gbest, o);
    const int ro = __shfl_xor_sync(0xffffffffu, rbest, o);
    if (go < gbest || (go == gbest && ro < rbest)) {
      gbest = go;
      rbest = ro;
    }
  }
  if (lane == 0) {
    red[0][warp] = gbest;
    sh4[warp] = rbest;
  }
  __syncthreads();
  int r = sh4[0];
  double gr = red[0][0];
  for (int w = 1; w < TRI_THREADS / 32; ++w)
    if (red[0][w] < gr || (red[0][w] == gr && sh4[w] < r)) {
      gr = red[0][w];
      r = sh4[w];
    }
  __syncthreads();  // red / sh4 are reused below
  if (tid == 0) {
    x[r] = 1.0;
    for (int i = r - 1; i >= 0; --i) x[i] = -ml[i] * x[i + 1];
  } else if (tid == 32) {
    for (int i = r; i + 1 < m; ++i) x[i + 1] = -rd[i] * (i == r ? 1.0 : x[i]);
  }
  __syncthreads();
  // normalise (fixed-order block sum)
  double ss = 0.0;
  for (int i = tid; i < m; i += TRI_THREADS) ss = fma(x[i], x[i], ss);
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[1][warp] = ss;
  __syncthreads();
  double nrm2 = 0.0;
  for (int w = 0; w < TRI_THREADS / 32; ++w) nrm2 += red[1][w];
  const bool vec_ok = nrm2 > 0.0 && isfinite(nrm2);
  const double inv_nrm = vec_ok ? 1.0 / sqrt(nrm2) : 0.0;
  for (int i = tid; i < m; i += TRI_THREADS) {
    x[i] = vec_ok ? x[i] * inv_nrm : (i == 0 ? 1.0 : 0.0);
    sc[OFF_S + i] = x[i];
  }
  __syncthreads();
  if (tid == 0) {
    const double res = b[j] * fabs(x[m - 1]);
    sc[OFF_MISC + 0] = e;
    sc[OFF_MISC + 1] = res;
    sc[OFF_MISC + 2] = b[j];
    int stop = STOP_NONE;
    if (!isfinite(e) || !isfinite(res))
      stop = STOP_NONFINITE;
    else if (res <= tol || b[j] == 0.0 || (long long)m == n)
      stop = STOP_CONVERGED;
    else if (m >= max_iter)
      stop = STOP_CAP;
    st[ST_M] = m;
    st[ST_STOP] = stop;
    if (stop == STOP_NONE) st[ST_J] = j + 1;
    if (set_cond) cudaGraphSetConditional(cond, stop == STOP_NONE ? 1u : 0u);
  }
}

// Next Krylov vector V[J] = w / beta_{J-1} after a step that did not stop
// (the same arithmetic as vec_scale_by_inv), also into x when it is set: the
// fixed input buffer of the matrix-vector product recorded in the step graph.
__global__ void k_next_vector(double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                              int64_t n, const double* __restrict__ sc, double* __restrict__ x) {
  const int* st = lz_state(sc);
  if (st[ST_STOP] != STOP_NONE) return;
  const int jn = st[ST_J];
  const double f = 1.0 / sc[OFF_BETA + jn - 1];
  double* y = V + (int64_t)jn * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w[i] * f;
    y[i] = v;
    if (x) x[i] = v;
  }
}

// First node of the step graph: enter the loop only if the step run before
// the graph did not stop.
__global__ void k_loop_init(const double* __restrict__ sc, cudaGraphConditionalHandle cond) {
  cudaGraphSetConditional(cond, lz_state(sc)[ST_STOP] == STOP_NONE ? 1u : 0u);
}

// Element chunks for k_multidot: about two element pairs per thread, and no
// more chunks than fit on the GPU in one wave (3 blocks per SM at its
// register use); the vector groups multiply the blocks.
int dot_blocks(int64_t n, int sm_count) {
  int64_t b = cdiv(n, DOT_THREADS * 4);
  const int64_t wave = 3 * (int64_t)(sm_count > 0 ? sm_count : 1);
  if (b > wave) b = wave;
  if (b > DOT_MAX_BLOCKS) b = DOT_MAX_BLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

// k_combine (128 threads): one element pair per thread up to 8192 blocks,
// then grid-stride.
int combine_blocks(int64_t n) {
  int64_t b = cdiv(n >> 1, 128);
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

// The second Gram-Schmidt pass is needed only where the first removed most
// of w (Daniel-Gragg-Kaufman-Stewart test, eta = 1/sqrt 2): with orthonormal
// Krylov vectors the projected norm is ||w'||^2 = ||w||^2 - sum_i c_i^2, so
// the pass is skipped (flag = 1) when sum_i c_i^2 <= ||w||^2 / 2 for the
// first pass's coefficients c (i <= jcur[0]); w2 = ||w||^2 before it.
__global__ void k_reorth_decide(const double* __restrict__ c, const double* __restrict__ w2,
                                const int* __restrict__ jcur, int* __restrict__ flag) {
  const int nv = jcur[0] + 1;
  double sq = 0.0;
  for (int i = threadIdx.x; i < nv; i += 32) sq = fma(c[i], c[i], sq);
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (threadIdx.x == 0) *flag = (isfinite(sq) && sq <= 0.5 * w2[0]) ? 1 : 0;
}

int ew_blocks(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

// w -= V^T-projection of w onto the nv stored Krylov vectors (rows of V with
// an even stride ld, 16-byte aligned like w), coefficients to coef. With
// jcur set, the kernels take nv = jcur[0] + 1 from the device and nv only
// bounds it (the blocks of the final reduction).
osmps_status project(osmps_ctx* ctx, const double* V, int64_t ld, int64_t n, int nv, double* w,
                     double* part, double* coef, cudaStream_t s, const int* jcur = nullptr,
                     const int* skip = nullptr) {
  const int nb = dot_blocks(n, ctx->sm_count);
  const dim3 dgrid(nb, (unsigned)cdiv(nv, DOT_GROUP));
  { k_multidot<<<dgrid, DOT_THREADS, 0, s>>>(V, ld, nv, w, n, part, jcur, skip); note_launch(); }
  { k_multidot_final<<<nv, 256, 0, s>>>(part, nb, coef, jcur, skip); note_launch(); }
  if (n < ((int64_t)1 << 20)) {
    k_combine<4><<<combine_blocks(n), 128, 0, s>>>(V, ld, nv, coef, w, n, 0, jcur, skip);
  } else {
    k_combine<1><<<ew_blocks(n), 256, 0, s>>>(V, ld, nv, coef, w, n, 0, jcur, skip);
  }
  note_launch();
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

// OSMPS_LANCZOS_AUTO: the graph for small Krylov vectors, except on the
// batch scheduler's worker threads, where many streams run at once and the
// host loop measured faster (64-chain batch, 8 workers: 2.29 sweeps/s with
// the host loop, 1.79 with graphs).
bool use_step_graph(const osmps_ctx* ctx, int64_t n, int max_iter) {
  if (ctx->prof_on || max_iter < 2) return false;
  if (ctx->lanczos_mode == OSMPS_LANCZOS_HOST) return false;
  if (ctx->lanczos_mode == OSMPS_LANCZOS_GRAPH) return true;
  return n <= ((int64_t)1 << 20) && !is_batch_worker();
}

using StepRecorder = std::function<osmps_status(cudaStream_t, cudaGraphConditionalHandle)>;
using LzGraph = osmps_ctx::LzGraph;
constexpr size_t LZ_GRAPHS_KEPT = 16;

void destroy_graph(LzGraph& gr) {
  if (gr.e) cudaGraphExecDestroy(gr.e);
  if (gr.g) cudaGraphDestroy(gr.g);
  gr.e = nullptr;
  gr.g = nullptr;
}

// A graph recorded for one call only, destroyed when the call returns (after
// the stream has drained: SyncOnExit is declared after it).
struct OneShotGraph {
  LzGraph gr;
  ~OneShotGraph() { destroy_graph(gr); }
};
struct SyncOnExit {
  cudaStream_t s = nullptr;
  bool armed = false;
  ~SyncOnExit() {
    if (armed) cudaStreamSynchronize(s);
  }
};

// Record [k_loop_init] -> while (cond) { step } and instantiate it. The step
// is recorded by stream capture on the context's capture stream; workspace
// growth is an error while the capture is open. gr.body_launches: kernels
// one step launches (the capture's own count is taken back: recording
// launches nothing).
osmps_status record_step_graph(osmps_ctx* ctx, const double* sc, const StepRecorder& record,
                               LzGraph& gr) {
  if (!ctx->capture_stream)
    OSMPS_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = ctx->capture_stream;
  OSMPS_CUDA(cudaGraphCreate(&gr.g, 0));
  cudaGraphConditionalHandle cond;
  OSMPS_CUDA(cudaGraphConditionalHandleCreate(&cond, gr.g, 0, cudaGraphCondAssignDefault));
  cudaKernelNodeParams kn = {};
  void* args[2] = {(void*)&sc, (void*)&cond};
  kn.func = (void*)k_loop_init;
  kn.gridDim = dim3(1);
  kn.blockDim = dim3(1);
  kn.sharedMemBytes = 0;
  kn.kernelParams = args;
  kn.extra = nullptr;
  cudaGraphNode_t init = nullptr, loop = nullptr;
  OSMPS_CUDA(cudaGraphAddKernelNode(&init, gr.g, nullptr, 0, &kn));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  OSMPS_CUDA(cudaGraphAddNode(&loop, gr.g, &init, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const long long before = thread_launch_count();
  OSMPS_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
  ctx->capturing = true;
  const osmps_status st = record(cs, cond);
  ctx->capturing = false;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
  gr.body_launches = thread_launch_count() - before;
  note_launches(-gr.body_launches);
  if (st != OSMPS_OK) return st;
  if (ce != cudaSuccess)
    return set_error(OSMPS_ECUDA, "lanczos: recording the step graph failed: %s",
                     cudaGetErrorString(ce));
  OSMPS_CUDA(cudaGraphInstantiate(&gr.e, gr.g, 0));
  return OSMPS_OK;
}

}  // namespace


osmps_status lanczos_core(osmps_ctx* ctx, int64_t n, double* theta, int max_iter, double tol,
                          const Matvec& matvec, double* energy, int* iters, double* resid,
                          cudaStream_t s, const double* P, int64_t ldp, int kp,
                          const long long* mkey, int nmkey) {
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
  const bool graph = use_step_graph(ctx, n, max_iter);
  double* X = nullptr;
  if (graph) {
    X = (double*)ws_get(ctx, SLOT_LZ_X, (size_t)n * 8, s, &st);
    if (!X) return st;
  }
  OSMPS_TRY(pinned_reserve(ctx, 16));
  int* state = lz_state(sc);

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
  OSMPS_CUDA(cudaMemsetAsync(state, 0, 4 * sizeof(int), s));

  // One step on stream q: w = H_eff V[J] (x is V[J] itself, or the buffer X
  // that the previous step's k_next_vector filled), projected out of the
  // projector rows and twice out of V[0..J], its norm, the tridiagonal solve
  // with the stopping decision, and V[J+1] (and its copy in X, when there is
  // one). final_blocks bounds J + 1.
  // Krylov vectors of 2^16 entries and more take the second Gram-Schmidt
  // pass only when the first asks for it; smaller ones, where the launches
  // and not the vector traffic cost, always take both.
  const bool twice_if_needed = n >= ((int64_t)1 << 16);
  auto step = [&](cudaStream_t q, const double* x, int final_blocks,
                  cudaGraphConditionalHandle cond, int set_cond) -> osmps_status {
    OSMPS_TRY(matvec(x, w, q));
    if (kp > 0) {  // the operator restricted to the complement: w <- (1 - P^T P) H v_j
      OSMPS_TRY(project(ctx, P, ldp, n, kp, w, part, sc + OFF_PROJ, q));
      OSMPS_TRY(project(ctx, P, ldp, n, kp, w, part, sc + OFF_PROJ + MAX_PROJ, q));
    }
    if (twice_if_needed) {  // the second pass only where the first removed most of w
      int* skip = reinterpret_cast<int*>(sc + OFF_MISC + 6);
      OSMPS_TRY(vec_norm2(ctx, w, n, sc + OFF_MISC + 5, q));
      OSMPS_TRY(project(ctx, V, ld, n, final_blocks, w, part, sc + OFF_C1, q, state));
      { k_reorth_decide<<<1, 32, 0, q>>>(sc + OFF_C1, sc + OFF_MISC + 5, state, skip); note_launch(); }
      OSMPS_TRY(project(ctx, V, ld, n, final_blocks, w, part, sc + OFF_C2, q, state, skip));
    } else {
      OSMPS_TRY(project(ctx, V, ld, n, final_blocks, w, part, sc + OFF_C1, q, state));
      OSMPS_TRY(project(ctx, V, ld, n, final_blocks, w, part, sc + OFF_C2, q, state));
    }
    OSMPS_TRY(vec_norm2(ctx, w, n, sc + OFF_MISC + 3, q));
    { k_tridiag<<<1, TRI_THREADS, 0, q>>>(sc, max_iter, tol, (long long)n, cond, set_cond); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    { k_next_vector<<<ew_blocks(n), 256, 0, q>>>(V, ld, w, n, sc, X); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    return OSMPS_OK;
  };

  OneShotGraph once;
  SyncOnExit drain;
  long long body_launches = 0;
  if (!graph) {
    for (int j = 0; j < max_iter; ++j) {
      OSMPS_TRY(step(s, V + (int64_t)j * ld, j + 1, 0, 0));
      OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC, MISC_READ * 8,
                                 cudaMemcpyDeviceToHost, s));
      OSMPS_CUDA(cudaStreamSynchronize(s));
      if (lz_state_in_misc(ctx->host_pinned)[ST_STOP] != STOP_NONE) break;
    }
  } else {
    // Step 0 runs directly: it sizes every workspace slot a step uses, so
    // nothing grows while the step is recorded. The other steps run in the
    // graph loop, recorded now or replayed from the context's cache.
    OSMPS_TRY(step(s, V, 1, 0, 0));
    std::vector<long long> key(mkey, mkey + (mkey ? nmkey : 0));
    long long tol_bits;
    memcpy(&tol_bits, &tol, sizeof tol_bits);
    for (long long k : {(long long)n, (long long)max_iter, tol_bits, (long long)kp, (long long)ldp,
                        (long long)(intptr_t)P, (long long)ctx->ws_epoch})
      key.push_back(k);
    LzGraph* gr = nullptr;
    if (mkey && nmkey > 0)
      for (auto& c : ctx->lz_graphs)
        if (c.key == key) gr = &c;
    if (!gr) {
      const StepRecorder rec = [&](cudaStream_t q, cudaGraphConditionalHandle cond) {
        return step(q, X, max_iter, cond, 1);
      };
      LzGraph fresh;
      fresh.key = key;
      const osmps_status rs = record_step_graph(ctx, sc, rec, fresh);
      if (rs != OSMPS_OK) {
        destroy_graph(fresh);
        return rs;
      }
      if (mkey && nmkey > 0) {
        if (ctx->lz_graphs.size() >= LZ_GRAPHS_KEPT) {  // every earlier call has drained
          size_t lru = 0;
          for (size_t i = 1; i < ctx->lz_graphs.size(); ++i)
            if (ctx->lz_graphs[i].last_use < ctx->lz_graphs[lru].last_use) lru = i;
          destroy_graph(ctx->lz_graphs[lru]);
          ctx->lz_graphs.erase(ctx->lz_graphs.begin() + lru);
        }
        ctx->lz_graphs.push_back(fresh);
        gr = &ctx->lz_graphs.back();
      } else {
        once.gr = fresh;
        gr = &once.gr;
      }
    }
    gr->last_use = ++ctx->lz_clock;
    body_launches = gr->body_launches;
    drain.s = s;
    drain.armed = true;
    OSMPS_CUDA(cudaGraphLaunch(gr->e, s));
    note_launch();  // k_loop_init
  }
  // Ritz vector theta = sum_i s_i v_i, normalised
  { k_combine_scalar<<<ew_blocks(n), 256, 0, s>>>(V, ld, sc, theta, n); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  OSMPS_TRY(vec_norm2(ctx, theta, n, sc + OFF_MISC + 4, s));
  OSMPS_TRY(vec_scale_by_inv_sqrt(theta, n, sc + OFF_MISC + 4, s));
  int* hflag = reinterpret_cast<int*>(ctx->host_pinned + MISC_READ);
  OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC, MISC_READ * 8,
                             cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaMemcpyAsync(hflag, ctx->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  const double e = ctx->host_pinned[0], res = ctx->host_pinned[1];
  const int* hs = lz_state_in_misc(ctx->host_pinned);
  const int stop = hs[ST_STOP], m = hs[ST_M];
  if (graph) note_launches(body_launches * (long long)(m - 1));  // the loop ran m - 1 steps
  if (*hflag & 1) {
    cudaMemsetAsync(ctx->dev_flags, 0, sizeof(int), s);
    return set_error(OSMPS_ETIMEOUT, "lanczos: a bounded device wait gave up");
  }
  if (stop == STOP_NONFINITE)
    return set_error(OSMPS_ENAN, "lanczos: non-finite Ritz value at step %d", m - 1);
  *energy = e;
  *iters = m;
  if (resid) *resid = res;
  if (stop != STOP_CONVERGED)
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
  const Matvec mv = [&](const double* x, double* y, cudaStream_t q) {
    return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, x, y, chi_l, d1, d2, chi_r,
                           wl, wm, wr, precision, q, true);
  };
  const long long key[9] = {1, chi_l, d1, d2, chi_r, wl, wm, wr, precision};
  return lanczos_core(ctx, chi_l * d1 * d2 * chi_r, theta, max_iter, tol, mv, energy, iters,
                      resid, s, nullptr, 0, 0, key, 9);
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
  const Matvec mv = [&](const double* x, double* y, cudaStream_t q) {
    return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, x, y, chi_l, d1, d2, chi_r,
                           wl, wm, wr, precision, q, true);
  };
  const long long key[9] = {1, chi_l, d1, d2, chi_r, wl, wm, wr, precision};
  return lanczos_core(ctx, n, theta_inout, max_iter, tol, mv, energy_out, iters_out, resid_out, s,
                      Q, ld, k, key, 9);
}


// ---------------------------------------------------------------------------
// Krylov propagator exp(-i tau H_eff) theta (Sec. 5.2, Eq. propSE and
// Eq. krylov:approx), the local step of the two-site TDVP (Sec. 5.4).
//
// Complex tensors enter as interleaved (re, im) float64 pairs and are worked
// on in the real 2x2 embedding z = x + iy -> [[x, -y], [y, x]] applied to
// every bond index pair: a complex tensor X[r, w, c] becomes the real
// X~[(p, r), w, (q, c)] with the (p, q) block of each element. The embedding
// turns products into products, so the real H_eff.theta of the ground-state
// search, given L~ = emb(L), R~ = emb(conj R) and theta~ = emb(theta) at
// bond dimensions 2 chi_l, 2 chi_r, computes emb(H_eff theta) exactly. Real
// Lanczos on embedded vectors reproduces the complex Lanczos recurrence (its
// alpha and beta are real for a Hermitian H_eff), so the Krylov basis, the
// reorthogonalisation and the tridiagonal T are the ground-state path's
// kernels. Multiplying by i is the map J(B) = B [[0, -1], [1, 0]] on the q
// blocks, used once in the final combination.
// ---------------------------------------------------------------------------
namespace osmps {
namespace {

constexpr int EXPM_THREADS = 128;
constexpr int EXPM_MAXIT = EXPM_THREADS;  // one thread per Krylov coordinate
constexpr int EXPM_TAYLOR = 18;  // terms per substep with |h| ||T|| <= 1: remainder below 1/19!
constexpr int EXPM_MAX_SUBSTEPS = 1 << 16;

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  for (int k = 1; k < EXPM_THREADS / 32; ++k) r = fmax(r, red[k]);
  return r;
}

// Step j = state J of the propagator: record alpha_j and beta_j as the
// ground-state kernel does, then u = exp(-i tau T_m) e_1 for the leading
// m = j + 1 rows of T. u comes from the Taylor series applied to e_1 in s
// substeps of length h = tau / s, s the smallest count with |h| g <= 1 for
// the Gershgorin bound g of T_m, EXPM_TAYLOR terms each; one thread per
// coordinate, each term one tridiagonal product. (The float64 eigensolver
// chains are long on this GPU: a dependent float64 operation takes 64
// cycles, a division 628.) The weight leaving the space is estimated as
// beta_j |u_{m-1}|; the space counts as exhausted when beta_j <= 1e-14 times
// max|alpha| + max|beta| of T_m. u goes to OFF_URE / OFF_UIM, the estimate
// to OFF_MISC + 1, and the stop decision to the state.
__global__ void __launch_bounds__(EXPM_THREADS) k_expm_tridiag(double* __restrict__ sc,
                                                               int max_iter, double tol,
                                                               double tau, long long n) {
  __shared__ double a[EXPM_MAXIT], b[EXPM_MAXIT], tr[EXPM_MAXIT], ti[EXPM_MAXIT];
  __shared__ double red[EXPM_THREADS / 32];
  int* st = lz_state(sc);
  const int j = st[ST_J];
  const int i = threadIdx.x;
  if (j < 0 || j >= max_iter || j >= EXPM_MAXIT) {  // not reachable from the driver below
    if (i == 0) {
      st[ST_STOP] = STOP_NONFINITE;
      st[ST_M] = 1;
    }
    return;
  }
  const int m = j + 1;
  if (i == 0) {
    sc[OFF_ALPHA + j] = sc[OFF_C1 + j] + sc[OFF_C2 + j];
    sc[OFF_BETA + j] = sqrt(sc[OFF_MISC + 3]);
  }
  __syncthreads();
  const bool act = i < m;
  if (act) {
    a[i] = sc[OFF_ALPHA + i];
    b[i] = sc[OFF_BETA + i];  // b[i] couples i and i+1; b[m-1] = beta_j is the residual
  }
  __syncthreads();
  double gi = 0.0, ai = 0.0, bi = 0.0;
  if (act) {
    ai = fabs(a[i]);
    bi = (i < m - 1) ? fabs(b[i]) : 0.0;
    gi = ai + bi + (i > 0 ? fabs(b[i - 1]) : 0.0);
  }
  const double g = block_max(gi, red);
  const double amax = block_max(ai, red);
  const double bmax = block_max(bi, red);
  const double bj = b[m - 1];
  const double steps = ceil(fabs(tau) * g);
  if (!isfinite(g) || !isfinite(bj) || !(steps <= (double)EXPM_MAX_SUBSTEPS)) {
    if (i == 0) {
      st[ST_STOP] = STOP_NONFINITE;
      st[ST_M] = m;
    }
    return;
  }
  const int nsub = steps < 1.0 ? 1 : (int)steps;
  const double h = tau / nsub;
  // u = e_1, then nsub times u <- sum_k (-i h T)^k u / k!
  double yr = (i == 0) ? 1.0 : 0.0, yi = 0.0;
  const double al = act ? a[i] : 0.0;
  const double bl = (act && i > 0) ? b[i - 1] : 0.0;
  const double br = (act && i < m - 1) ? b[i] : 0.0;
  for (int sub = 0; sub < nsub; ++sub) {
    if (act) {
      tr[i] = yr;
      ti[i] = yi;
    }
    __syncthreads();
#pragma unroll
    for (int k = 1; k <= EXPM_TAYLOR; ++k) {
      double pr = 0.0, pi = 0.0;  // (T t)_i
      if (act) {
        pr = al * tr[i];
        pi = al * ti[i];
        if (i > 0) {
          pr = fma(bl, tr[i - 1], pr);
          pi = fma(bl, ti[i - 1], pi);
        }
        if (i < m - 1) {
          pr = fma(br, tr[i + 1], pr);
          pi = fma(br, ti[i + 1], pi);
        }
      }
      __syncthreads();
      // (-i h T)(t_r + i t_i) / k = (h T t_i - i h T t_r) / k
      const double hk = h * (1.0 / (double)k);
      if (act) {
        const double nr = hk * pi, ni = -hk * pr;
        tr[i] = nr;
        ti[i] = ni;
        yr += nr;
        yi += ni;
      }
      __syncthreads();
    }
  }
  if (act) {
    sc[OFF_URE + i] = yr;
    sc[OFF_UIM + i] = yi;
    tr[i] = yr;
    ti[i] = yi;
  }
  __syncthreads();
  if (i == 0) {
    const double ul = sqrt(tr[m - 1] * tr[m - 1] + ti[m - 1] * ti[m - 1]);
    const bool exhausted = bj <= 1e-14 * fmax(amax + bmax, 1e-300);
    const double err = exhausted ? 0.0 : bj * ul;
    sc[OFF_MISC + 1] = err;
    sc[OFF_MISC + 2] = bj;
    int stop = STOP_NONE;
    if (!isfinite(err) || !isfinite(tr[0]) || !isfinite(ti[0]))
      stop = STOP_NONFINITE;
    else if (exhausted || err <= tol || (long long)m == n)
      stop = STOP_CONVERGED;
    else if (m >= max_iter)
      stop = STOP_CAP;
    st[ST_M] = m;
    st[ST_STOP] = stop;
    if (stop == STOP_NONE) st[ST_J] = j + 1;
  }
}

// out = ||theta~|| sum_i u_i v_i, read back from the embedding: with B the
// (p, q) blocks of the real basis vector v_i at one complex element,
// sum_i Re(u_i) B + Im(u_i) J(B) averaged over its duplicate blocks. out is
// interleaved complex [chi_l, D, chi_r], or with emb set the embedded
// [(p, a), D, (q, c)] form of the vectors themselves. Nothing is written
// when the iteration stopped on a non-finite value.
__global__ void k_expm_combine(const double* __restrict__ V, int64_t ld,
                               const double* __restrict__ sc, double* __restrict__ out,
                               int64_t chi_l, int64_t D, int64_t chi_r, int emb) {
  __shared__ double ur[EXPM_MAXIT], ui[EXPM_MAXIT];
  const int* st = lz_state(sc);
  if (st[ST_STOP] == STOP_NONFINITE) return;
  const int m = st[ST_M];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    ur[i] = sc[OFF_URE + i];
    ui[i] = sc[OFF_UIM + i];
  }
  __syncthreads();
  const double scale = 0.5 * sqrt(sc[OFF_MISC + 4]);
  const int64_t dc = D * chi_r, nc = chi_l * dc, row = 2 * chi_r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / dc, rem = e - a * dc, s = rem / chi_r, c = rem - s * chi_r;
    const int64_t o00 = (a * D + s) * row + c, o10 = ((chi_l + a) * D + s) * row + c;
    double xr = 0.0, xi = 0.0;
    for (int i = 0; i < m; ++i) {
      const double* v = V + (int64_t)i * ld;
      const double b00 = v[o00], b01 = v[o00 + chi_r], b10 = v[o10], b11 = v[o10 + chi_r];
      xr = fma(ur[i], b00 + b11, fma(ui[i], b01 - b10, xr));
      xi = fma(ur[i], b10 - b01, fma(ui[i], b00 + b11, xi));
    }
    if (emb) {
      out[o00] = scale * xr;
      out[o00 + chi_r] = -scale * xi;
      out[o10] = scale * xi;
      out[o10 + chi_r] = scale * xr;
    } else {
      out[2 * e] = scale * xr;
      out[2 * e + 1] = scale * xi;
    }
  }
}

}  // namespace

namespace {

// out[((p r + i) w + k) 2c + q c + j] = (p, q) block of z[i, k, j] (or of
// its conjugate): blocks (0,0) = (1,1) = Re, (1,0) = Im, (0,1) = -Im.
__global__ void k_embed3(const double* __restrict__ z, double* __restrict__ out, int64_t r,
                         int64_t w, int64_t c, int conj) {
  const int64_t wc = w * c, n = r * wc, row = 2 * c, plane = r * w * row;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / wc, rem = e - i * wc, k = rem / c, jj = rem - k * c;
    const double re = z[2 * e], im = conj ? -z[2 * e + 1] : z[2 * e + 1];
    const int64_t o = (i * w + k) * row + jj;
    out[o] = re;
    out[o + c] = -im;
    out[plane + o] = im;
    out[plane + o + c] = re;
  }
}

}  // namespace

osmps_status embed_complex(const double* z, double* out, int64_t r, int64_t w, int64_t c,
                           bool conj, cudaStream_t s) {
  { k_embed3<<<ew_blocks(r * w * c), 256, 0, s>>>(z, out, r, w, c, conj ? 1 : 0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

// theta_out = exp(-i tau H) theta~, interleaved complex, or embedded (and
// then free to alias theta_emb) with out_embedded; theta_emb is the embedded
// start vector of length 4 n_c, matvec the embedded operator.
osmps_status expm_core(osmps_ctx* ctx, int64_t n_c, const double* theta_emb, double* theta_out,
                       int64_t chi_l, int64_t D, int64_t chi_r, double tau, int max_iter,
                       double tol, const Matvec& matvec, int* iters, double* err, cudaStream_t s,
                       bool out_embedded) {
  osmps_status st = OSMPS_OK;
  const int64_t n = 4 * n_c;
  const int64_t ld = n;  // a multiple of 4: 16-byte aligned rows
  if (max_iter > n_c) max_iter = (int)n_c;
  double* V = (double*)ws_get(ctx, SLOT_LZ_BASIS, (size_t)max_iter * ld * 8, s, &st);
  if (!V) return st;
  double* w = (double*)ws_get(ctx, SLOT_LZ_W, (size_t)n * 8, s, &st);
  if (!w) return st;
  double* sc = (double*)ws_get(ctx, SLOT_LZ_SCAL, SCAL_COUNT * 8, s, &st);
  if (!sc) return st;
  double* part = (double*)ws_get(ctx, SLOT_LZ_PART, (size_t)MAXIT * DOT_MAX_BLOCKS * 8, s, &st);
  if (!part) return st;
  OSMPS_TRY(pinned_reserve(ctx, 16));
  int* state = lz_state(sc);

  OSMPS_TRY(vec_norm2(ctx, theta_emb, n, sc + OFF_MISC + 4, s));
  OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC + 4, 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (!(ctx->host_pinned[0] > 0.0) || !std::isfinite(ctx->host_pinned[0]))
    return set_error(ctx->host_pinned[0] == 0.0 ? OSMPS_EINVAL : OSMPS_ENAN,
                     "heff_expm: start vector has norm^2 %g", ctx->host_pinned[0] / 2);
  OSMPS_CUDA(cudaMemcpyAsync(V, theta_emb, n * 8, cudaMemcpyDeviceToDevice, s));
  OSMPS_TRY(vec_scale_by_inv_sqrt(V, n, sc + OFF_MISC + 4, s));
  OSMPS_CUDA(cudaMemsetAsync(state, 0, 4 * sizeof(int), s));
  for (int j = 0; j < max_iter; ++j) {
    OSMPS_TRY(matvec(V + (int64_t)j * ld, w, s));
    OSMPS_TRY(project(ctx, V, ld, n, j + 1, w, part, sc + OFF_C1, s, state));
    OSMPS_TRY(project(ctx, V, ld, n, j + 1, w, part, sc + OFF_C2, s, state));
    OSMPS_TRY(vec_norm2(ctx, w, n, sc + OFF_MISC + 3, s));
    { k_expm_tridiag<<<1, EXPM_THREADS, 0, s>>>(sc, max_iter, tol, tau, (long long)n_c); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    { k_next_vector<<<ew_blocks(n), 256, 0, s>>>(V, ld, w, n, sc, nullptr); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, sc + OFF_MISC, MISC_READ * 8,
                               cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
    if (lz_state_in_misc(ctx->host_pinned)[ST_STOP] != STOP_NONE) break;
  }
  { k_expm_combine<<<ew_blocks(n_c), 256, 0, s>>>(V, ld, sc, theta_out, chi_l, D, chi_r, out_embedded ? 1 : 0); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  OSMPS_CUDA(cudaStreamSynchronize(s));
  const int* hs = lz_state_in_misc(ctx->host_pinned);
  const int stop = hs[ST_STOP], m = hs[ST_M];
  const double e = ctx->host_pinned[1];
  if (stop == STOP_NONFINITE)
    return set_error(OSMPS_ENAN, "heff_expm: non-finite Krylov data at step %d", m - 1);
  *iters = m;
  if (err) *err = e;
  if (stop != STOP_CONVERGED)
    return set_error(OSMPS_ENOCONV, "heff_expm: error estimate %.3e above tol %.3e after %d vectors",
                     e, tol, m);
  return OSMPS_OK;
}

// Embedded operands of a complex H_eff: L~ = emb(L), R~ = emb(conj R),
// prepared for the real H_eff.theta at bond dimensions 2 chi_l, 2 chi_r.
osmps_status heff_prepare_complex(osmps_ctx* ctx, const double* L, const double* W1,
                                  const double* W2, const double* R, int64_t chi_l, int64_t d1,
                                  int64_t d2, int64_t chi_r, int64_t wl, int64_t wm, int64_t wr,
                                  int precision, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  double* Le = (double*)ws_get(ctx, SLOT_CX_L, (size_t)4 * chi_l * wl * chi_l * 8, s, &st);
  if (!Le) return st;
  double* Re = (double*)ws_get(ctx, SLOT_CX_R, (size_t)4 * chi_r * wr * chi_r * 8, s, &st);
  if (!Re) return st;
  OSMPS_TRY(embed_complex(L, Le, chi_l, wl, chi_l, false, s));
  OSMPS_TRY(embed_complex(R, Re, chi_r, wr, chi_r, true, s));
  return heff_prepare(ctx, Le, W1, W2, Re, 2 * chi_l, d1, d2, 2 * chi_r, wl, wm, wr, precision, s);
}

}  // namespace osmps

extern "C" osmps_status osmps_heff_expm(osmps_ctx* ctx, const double* L, const double* W1,
                                        const double* W2, const double* R, double* theta_inout,
                                        int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                        int64_t wl, int64_t wm, int64_t wr, double tau,
                                        int max_iter, double tol, int precision, int* iters_out,
                                        double* err_out, void* stream) {
  clear_error();
  if (!ctx || !L || !W1 || !W2 || !R || !theta_inout || !iters_out)
    return set_error(OSMPS_EINVAL, "osmps_heff_expm: null argument");
  if (max_iter < 1 || max_iter > EXPM_MAXIT)
    return set_error(OSMPS_EINVAL, "osmps_heff_expm: max_iter %d outside [1, %d]", max_iter,
                     EXPM_MAXIT);
  if (!(tol >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_heff_expm: tol %g", tol);
  if (!std::isfinite(tau)) return set_error(OSMPS_EINVAL, "osmps_heff_expm: tau %g", tau);
  if (!valid_precision(precision))
    return set_error(OSMPS_EINVAL, "osmps_heff_expm: precision %d", precision);
  for (int64_t x : {chi_l, d1, d2, chi_r, wl, wm, wr})
    if (x <= 0 || x > ((int64_t)1 << 30))
      return set_error(OSMPS_ESHAPE, "osmps_heff_expm: non-positive or oversized dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  const int64_t n_c = chi_l * d1 * d2 * chi_r;
  double* th = (double*)ws_get(ctx, SLOT_CX_THETA, (size_t)4 * n_c * 8, s, &st);
  if (!th) return st;
  OSMPS_TRY(heff_prepare_complex(ctx, L, W1, W2, R, chi_l, d1, d2, chi_r, wl, wm, wr, precision, s));
  OSMPS_TRY(embed_complex(theta_inout, th, chi_l, d1 * d2, chi_r, false, s));
  const Matvec mv = [&](const double* x, double* y, cudaStream_t q) {
    return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, x, y, 2 * chi_l, d1, d2,
                           2 * chi_r, wl, wm, wr, precision, q, true);
  };
  return expm_core(ctx, n_c, th, theta_inout, chi_l, d1 * d2, chi_r, tau, max_iter, tol, mv,
                   iters_out, err_out, s, false);
}
