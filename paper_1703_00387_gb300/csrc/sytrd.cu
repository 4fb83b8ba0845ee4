// Householder reduction of a symmetric matrix to tridiagonal form,
// T = Q^T A Q (the first step of the float64 eigendecomposition used by the
// split, Sec. 2 Eq. AAD_ULLUD), with the reflectors stored as LAPACK's dsytrd
// (lower) stores them: Q = H(0) ... H(n-2), H(j) = I - tau_j v_j v_j^T,
// v_j = (0, .., 0, 1 at j+1, A[j+2.., j]).
//
// Blocked as in LAPACK's dlatrd: panels of NB columns. Inside a panel, column
// j is first brought up to date with the panel's earlier reflectors
// (A - V W^T - W V^T), its reflector is formed, and
//   w = tau (A22 v - W (V^T v) - V (W^T v)),  w -= (tau/2)(w^T v) v
// with A22 the trailing matrix as it stood at the start of the panel. The
// product A22 v (a symmetric matrix-vector product over the trailing block)
// is the float64 work; it runs on every SM. A cooperative kernel does one
// panel with three grid-wide reductions per column (the norm of the updated
// column; A22 v and V^T v, W^T v; w^T v). After each panel the trailing
// block is updated, A22 -= V W^T + W V^T, by the float64-accurate emulated
// tensor-core GEMM. The matrix is kept full (both triangles), so row r of
// the trailing block is contiguous; the reflectors overwrite column j below
// the subdiagonal (row j of the row-major view), which later columns never read.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace osmps {
namespace {

constexpr int NB = 32;            // panel width
constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int RCHUNK = 8;         // rows per ownership chunk (chunk c -> block c % G)

struct SytrdArgs {
  double* A;        // n x n, full symmetric (row r contiguous)
  int n, k0, nbp;   // panel [k0, k0 + nbp)
  double* d;        // diagonal of T
  double* e;        // off-diagonal of T
  double* tau;      // reflector scalars
  double* Vp;       // panel reflectors, column-major NB x n: Vp[q * n + r]
  double* Wp;       // panel w vectors, same layout
  double* col;      // updated column (n)
  double* t;        // A22 v (n)
  double* wraw;     // A22 v - W (V^T v) - V (W^T v) (n)
  double* part;     // per-block partial sums: G x (2 NB + 4)
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < ST_WARPS; ++w) s += sh[w];
  return s;  // valid in thread 0
}

// Sum over the G blocks' partials part[b * PW + off] by one warp (lanes over
// blocks, fixed order, then a fixed shuffle tree): the same value in every
// block. Returned in all lanes of the calling warp.
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part, int G, int pw,
                                                 int off) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < G; b += 32) s += part[(size_t)b * pw + off];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Rows owned by this block: chunks c = blockIdx.x, blockIdx.x + G, ... of
// RCHUNK consecutive rows, thread threadIdx.x < RCHUNK of the block taking
// row c RCHUNK + threadIdx.x in every per-row phase, so a row's entries of
// V and W are written and read by the same thread.
__global__ void __launch_bounds__(ST_THREADS) k_sytrd_panel(SytrdArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sv[];   // v over rows [0, n) (entries up to j are 0)
  __shared__ double sh[ST_WARPS];
  __shared__ double sy[2 * NB];    // V^T v, W^T v of the current column
  __shared__ double sc[4];         // tau, 1/(alpha - beta), alpha2, W entry of row j
  const int n = a.n, G = gridDim.x;
  const int nchunks = (n + RCHUNK - 1) / RCHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int PW = 2 * NB + 4;
  double* part = a.part + (size_t)blockIdx.x * PW;
  double tau_prev = 0.0, alpha2_prev = 0.0;

  for (int jj = 0; jj < a.nbp; ++jj) {
    const int j = a.k0 + jj;
    // W's entry of the previous column at row j: tau w_raw[j] + alpha2 v[j],
    // v[j] = 1 (j is the row after the previous column); formed by every block
    // instead of read back from the block that owns row j.
    const double wj_prev = jj > 0 ? fma(tau_prev, a.wraw[j], alpha2_prev) : 0.0;
    // ---- A: column j brought up to date with the panel's earlier reflectors
    double ssq = 0.0;
    for (int c = blockIdx.x; c < nchunks; c += G) {
      const int r = c * RCHUNK + threadIdx.x;
      if (threadIdx.x < RCHUNK && r < n && r >= j) {
        double x = a.A[(size_t)j * n + r];
        for (int q = 0; q < jj; ++q) {
          const double wjq = q == jj - 1 ? wj_prev : a.Wp[(size_t)q * n + j];
          x -= a.Vp[(size_t)q * n + r] * wjq + a.Wp[(size_t)q * n + r] * a.Vp[(size_t)q * n + j];
        }
        a.col[r] = x;
        if (r >= j + 2) ssq = fma(x, x, ssq);
      }
    }
    {
      const double s = block_sum(ssq, sh);
      if (threadIdx.x == 0) part[0] = s;
    }
    grid.sync();
    // ---- B: the reflector (every block the same), v staged in shared memory
    if (warp == 0) {
      const double sigma = warp_sum_parts(a.part, G, PW, 0);
      if (lane == 0) {
      double tau = 0.0, inv = 0.0, beta = 0.0;
      if (j < n - 1) {
        const double alpha = a.col[j + 1];
        if (sigma == 0.0) {
          beta = alpha;  // nothing below the subdiagonal: H = I
        } else {
          const double nrm = sqrt(fma(alpha, alpha, sigma));
          beta = alpha >= 0.0 ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          inv = 1.0 / (alpha - beta);
        }
      }
      sc[0] = tau;
      sc[1] = inv;
      if (blockIdx.x == 0) {
        a.d[j] = a.col[j];
        if (j < n - 1) {
          a.e[j] = beta;
          a.tau[j] = tau;
        }
      }
      }
    }
    __syncthreads();
    const double tau = sc[0], inv = sc[1];
    for (int r = threadIdx.x; r < n; r += ST_THREADS)
      sv[r] = r == j + 1 ? 1.0 : (r > j + 1 ? a.col[r] * inv : 0.0);
    __syncthreads();
    // reflector storage (row j of the row-major view) and the panel's V column
    for (int c = blockIdx.x; c < nchunks; c += G) {
      const int r = c * RCHUNK + threadIdx.x;
      if (threadIdx.x < RCHUNK && r < n) {
        if (r >= j + 2) a.A[(size_t)j * n + r] = sv[r];
        a.Vp[(size_t)jj * n + r] = sv[r];
      }
    }
    // t = A22 v on owned rows, one warp per row
    if (j < n - 1) {
      for (int c = blockIdx.x; c < nchunks; c += G) {
        for (int rr = warp; rr < RCHUNK; rr += ST_WARPS) {
          const int r = c * RCHUNK + rr;
          if (r >= n || r < j + 1) continue;
          const double* row = a.A + (size_t)r * n;
          double acc = 0.0;
          for (int k = j + 1 + lane; k < n; k += 32) acc = fma(row[k], sv[k], acc);
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) a.t[r] = acc;
        }
      }
    }
    // partial V^T v and W^T v over the owned rows: thread q < 2 jj takes one
    if (threadIdx.x < 2 * NB) {
      const int q = threadIdx.x % NB;
      const double* X = threadIdx.x < NB ? a.Vp : a.Wp;
      double acc = 0.0;
      if (q < jj && j < n - 1)
        for (int c = blockIdx.x; c < nchunks; c += G)
          for (int rr = 0; rr < RCHUNK; ++rr) {
            const int r = c * RCHUNK + rr;
            if (r < n && r >= j + 1) acc = fma(X[(size_t)q * n + r], sv[r], acc);
          }
      part[1 + threadIdx.x] = acc;
    }
    grid.sync();
    // ---- C: w_raw = t - W (V^T v) - V (W^T v), partial w^T v
    for (int q = warp; q < 2 * NB; q += ST_WARPS) {  // one warp per coefficient
      const double s = (q % NB) < jj ? warp_sum_parts(a.part, G, PW, 1 + q) : 0.0;
      if (lane == 0) sy[q] = s;
    }
    __syncthreads();
    double pwv = 0.0;
    if (j < n - 1) {
      for (int c = blockIdx.x; c < nchunks; c += G) {
        const int r = c * RCHUNK + threadIdx.x;
        if (threadIdx.x < RCHUNK && r < n && r >= j + 1) {
          double x = a.t[r];
          for (int q = 0; q < jj; ++q)
            x -= a.Wp[(size_t)q * n + r] * sy[q] + a.Vp[(size_t)q * n + r] * sy[NB + q];
          a.wraw[r] = x;
          pwv = fma(tau * x, sv[r], pwv);
        }
      }
    }
    {
      const double s = block_sum(pwv, sh);
      if (threadIdx.x == 0) part[2 * NB + 1] = s;
    }
    grid.sync();
    // ---- D: w = tau w_raw + alpha2 v, alpha2 = -(tau/2) (tau w_raw)^T v
    if (warp == 0) {
      const double s = warp_sum_parts(a.part, G, PW, 2 * NB + 1);
      if (lane == 0) sc[2] = -0.5 * tau * s;
    }
    __syncthreads();
    const double alpha2 = sc[2];
    for (int c = blockIdx.x; c < nchunks; c += G) {
      const int r = c * RCHUNK + threadIdx.x;
      if (threadIdx.x < RCHUNK && r < n)
        a.Wp[(size_t)jj * n + r] =
            (j < n - 1 && r >= j + 1) ? fma(alpha2, sv[r], tau * a.wraw[r]) : 0.0;
    }
    tau_prev = tau;
    alpha2_prev = alpha2;
    __syncthreads();  // sc and sv are rewritten by the next column
  }
}

// A[k + r][k + c] -= C[r][c] for the trailing m x m block (C row-major m x m).
__global__ void k_sub_trailing(double* __restrict__ A, int64_t n, int64_t k,
                               const double* __restrict__ C, int64_t m) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / m, c = e - r * m;
    A[(k + r) * n + (k + c)] -= C[e];
  }
}

// [V | W] and [W | V] as m x 2 NB row-major operands for the trailing update
// (rows k.. of the panel's column-major V, W).
__global__ void k_pack_vw(const double* __restrict__ Vp, const double* __restrict__ Wp,
                          int64_t n, int64_t k, int64_t m, int nbp, double* __restrict__ X,
                          double* __restrict__ Y) {
  const int64_t w = 2 * NB;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / w, q = e - r * w;
    const int64_t qq = q % NB;
    double vx = 0.0, vy = 0.0;
    if (qq < nbp) {
      const double v = Vp[qq * n + k + r], ww = Wp[qq * n + k + r];
      vx = q < NB ? v : ww;
      vy = q < NB ? ww : v;
    }
    X[e] = vx;
    Y[e] = vy;
  }
}

int grid_1d(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 16384)); }

}  // namespace

bool sytrd_supported(int64_t n) { return n >= 2 && n <= 8192; }

// A (n x n, symmetric, full) -> reflectors in A (lower, dsytrd layout), d, e, tau.
osmps_status sytrd_tc(osmps_ctx* ctx, double* A, int64_t n, double* d, double* e, double* tau,
                      cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  if (!sytrd_supported(n)) return set_error(OSMPS_EUNSUPPORTED, "sytrd: n=%lld", (long long)n);
  const size_t smem = (size_t)n * 8;
  static const cudaError_t cfg = cudaFuncSetAttribute(
      k_sytrd_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
  OSMPS_CUDA(cfg);
  int per_sm = 0;
  OSMPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sytrd_panel, ST_THREADS, smem));
  if (per_sm < 1) return set_error(OSMPS_EUNSUPPORTED, "sytrd: panel kernel does not fit an SM");
  const int nchunks = (int)cdiv(n, RCHUNK);
  const int G = std::max(1, std::min(ctx->sm_count * std::min(per_sm, 1), nchunks));
  double* buf = (double*)ws_get(ctx, SLOT_TRD, (size_t)(2 * NB * n + 3 * n + (size_t)G * (2 * NB + 4) +
                                                        2 * n * 2 * NB + (size_t)n * n + 64) * 8, s, &st);
  if (!buf) return st;
  double* Vp = buf;
  double* Wp = Vp + NB * n;
  double* col = Wp + NB * n;
  double* t = col + n;
  double* wraw = t + n;
  double* part = wraw + n;
  double* X = part + (size_t)G * (2 * NB + 4);
  double* Y = X + 2 * NB * n;
  double* C = Y + 2 * NB * n;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nbp = (int)std::min<int64_t>(NB, n - k0);
    SytrdArgs a;
    a.A = A; a.n = (int)n; a.k0 = (int)k0; a.nbp = nbp;
    a.d = d; a.e = e; a.tau = tau; a.Vp = Vp; a.Wp = Wp;
    a.col = col; a.t = t; a.wraw = wraw; a.part = part;
    void* args[] = {&a};
    OSMPS_CUDA(cudaLaunchCooperativeKernel((void*)k_sytrd_panel, dim3(G), dim3(ST_THREADS), args,
                                           smem, s));
    note_launch();
    const int64_t k = k0 + nbp, m = n - k;
    if (m <= 0) break;
    { k_pack_vw<<<grid_1d(m * 2 * NB), 256, 0, s>>>(Vp, Wp, n, k, m, nbp, X, Y); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    // C = [V W] [W V]^T = V W^T + W V^T on the trailing block
    SplitView xv; xv.src = X; xv.rows = m; xv.K = 2 * NB; xv.s0 = 2 * NB; xv.sk = 1;
    SplitView yv; yv.src = Y; yv.rows = m; yv.K = 2 * NB; yv.s0 = 2 * NB; yv.sk = 1;
    OSMPS_TRY(gemm_emu(ctx, xv, yv, m, m, 2 * NB, C, m, s));
    { k_sub_trailing<<<grid_1d(m * m), 256, 0, s>>>(A, n, k, C, m); note_launch(); }
    OSMPS_LAUNCH_CHECK();
  }
  return OSMPS_OK;
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_sytrd(osmps_ctx* ctx, double* A, int64_t n, double* d, double* e,
                                    double* tau, void* stream) {
  clear_error();
  if (!ctx || !A || !d || !e || !tau) return set_error(OSMPS_EINVAL, "osmps_sytrd: null argument");
  if (!sytrd_supported(n)) return set_error(OSMPS_ESHAPE, "osmps_sytrd: n=%lld outside [2, 8192]", (long long)n);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return sytrd_tc(ctx, A, n, d, e, tau, (cudaStream_t)stream);
}
