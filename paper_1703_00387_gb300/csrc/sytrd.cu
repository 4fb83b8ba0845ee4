// Householder reduction of a symmetric matrix to tridiagonal form,
// T = Q^T A Q (the first step of the float64 eigendecomposition used by the
// split, Sec. 2 Eq. AAD_ULLUD), with the reflectors stored as LAPACK's dsytrd
// (lower) stores them: Q = H(0) ... H(n-2), H(j) = I - tau_j v_j v_j^T,
// v_j = (0, .., 0, 1 at j+1, A[j+2.., j]).
//
// Blocked as in LAPACK's dlatrd: panels of NB columns. Inside a panel, column
// j is first brought up to date with the panel's earlier reflectors
// (A - V W^T - W V^T), its reflector is formed, and
//   w = tau (A22 v - W y - V z) + alpha2 v,   y = V^T v,  z = W^T v,
//   alpha2 = -(tau/2) tau (A22 v - W y - V z)^T v
// with A22 the trailing matrix as it stood at the start of the panel. Since
// y and z are V^T v and W^T v, (W y + V z)^T v = 2 y^T z, so the scalar
// needs only t^T v (t = A22 v) besides y and z: it comes out of the same
// reduction as y and z, and a column costs two grid-wide reductions:
//   1. the squared norm of the updated column below the subdiagonal;
//   2. t = A22 v on every row (the float64 work, spread over all SMs), with
//      the partial sums of y, z and t^T v.
// The kernel is one cooperative launch per panel; its grid barriers are a
// counter in global memory with bounded waits (after ~2 s a block records
// the failure in the error flag and leaves). Rows are dealt to the blocks
// round robin (row r to block r mod G), and each block keeps its rows of V
// and W in shared memory, so only v (every block needs all of it) and the
// reductions cross the grid. After each panel the trailing block is updated,
// A22 -= V W^T + W V^T, by the float64-accurate emulated tensor-core GEMM,
// subtracting in its epilogue. The matrix is kept full (both triangles), so
// row r of the trailing block is contiguous; the reflectors overwrite column
// j below the subdiagonal (row j of the row-major view), which later
// columns never read.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "gridsync.cuh"

namespace osmps {
namespace {

constexpr int NB = 32;            // panel width (one lane per earlier reflector)
constexpr int ST_THREADS = 256;
constexpr int ST_WARPS = ST_THREADS / 32;
constexpr int MAXLOC = 64;        // rows per block at most
constexpr int PW = 2 * NB + 2;    // partial sums per block: y | z | t^T v | ssq
constexpr int P_TV = 2 * NB, P_SSQ = 2 * NB + 1;

struct SytrdArgs {
  double* A;         // n x n, full symmetric (row r contiguous)
  int n, k0, nbp;    // panel [k0, k0 + nbp)
  double* d;         // diagonal of T
  double* e;         // off-diagonal of T
  double* tau;       // reflector scalars
  double* Vp;        // panel reflectors, column-major NB x n: Vp[q * n + r]
  double* Wp;        // panel w vectors, same layout
  double* col;       // updated column (n)
  double* t;         // A22 v, only row j+1 is read by other blocks
  double* part;      // per-block partial sums: G x PW
  unsigned* bar;     // grid barrier counter
  unsigned bar_base; // counter value at the start of this launch
  int* err;          // bit 0: a barrier wait gave up
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the G blocks' partials part[b * PW + off] by one warp (lanes over
// blocks, fixed order, then a fixed shuffle tree): the same value in every
// block and every lane.
__device__ __forceinline__ double sum_parts(const double* __restrict__ part, int G, int off) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int b = lane; b < G; b += 32) s += part[(size_t)b * PW + off];
  return warp_sum(s);
}

// Four threads of a quad share one row: sum over q < jj with q = sub (mod 4)
// of a[q] bs[q] + c[q] ds[q] in two interleaved partial sums, then two xor
// shuffles, so every thread of the quad gets the total. GB300's float64
// pipe is narrow: a warp-wide tree would spend five additions of 32 lanes on
// each row's sum, the quad two of four. Every lane of the warp must call it.
__device__ __forceinline__ double quad_dot2(const double* __restrict__ a,
                                            const double* __restrict__ bs,
                                            const double* __restrict__ c,
                                            const double* __restrict__ ds, int jj, int sub) {
  double p0 = 0.0, p1 = 0.0;
  int q = sub;
  for (; q + 4 < jj; q += 8) {
    p0 = fma(a[q], bs[q], fma(c[q], ds[q], p0));
    p1 = fma(a[q + 4], bs[q + 4], fma(c[q + 4], ds[q + 4], p1));
  }
  if (q < jj) p0 = fma(a[q], bs[q], fma(c[q], ds[q], p0));
  double x = p0 + p1;
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  return x;
}

__global__ void __launch_bounds__(ST_THREADS, 1) k_sytrd_panel(SytrdArgs a) {
  extern __shared__ double sv[];            // v over rows [0, n) (entries up to j are 0)
  __shared__ double sV[MAXLOC][NB];         // this block's rows of V and W
  __shared__ double sW[MAXLOC][NB];
  __shared__ double st[MAXLOC];             // this block's rows of t = A22 v
  __shared__ double sVs[NB], sWs[NB];       // V_q[j], W_q[j] of the current column
  __shared__ double scoef[2 * NB + 1];      // y | z | t^T v of the current column
  __shared__ double sq[MAXLOC];             // squares of this block's column entries
  __shared__ double sc[4];                  // tau, 1/(alpha - beta), alpha2, row j+1 sum
  __shared__ int s_ok;
  const int n = a.n, G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cnt = b < n ? (n - b + G - 1) / G : 0;  // rows b, b + G, ...
  double* part = a.part + (size_t)b * PW;
  unsigned target = a.bar_base;
  // per-row work: the quad of threads 4 loc .. 4 loc + 3 takes row r = b + G loc
  const int qloc = threadIdx.x >> 2, qsub = threadIdx.x & 3;
  const int qrow = b + G * qloc;
  const bool qmine = qloc < cnt;
  // A[j][qrow], loaded one column ahead by the quad's first thread (row j of A
  // is not written before column j reads it)
  auto load_arow = [&](int jrow) {
    return (qsub == 0 && qmine && jrow < n) ? a.A[(size_t)jrow * n + qrow] : 0.0;
  };
  double arow = load_arow(a.k0);

  for (int jj = 0; jj < a.nbp; ++jj) {
    const int j = a.k0 + jj;
    // ---- A: column j brought up to date with the panel's earlier reflectors
    // x_r = A[j][r] - sum_q (V_q[r] W_q[j] + W_q[r] V_q[j])
    {
      double sq_r = 0.0;
      if (warp * 8 < cnt) {  // warps without rows keep off the float64 pipe
        const double x = quad_dot2(&sV[qloc][0], sWs, &sW[qloc][0], sVs, jj, qsub);
        if (qsub == 0 && qmine && qrow >= j) {
          const double xv = arow - x;
          a.col[qrow] = xv;
          if (qrow == j) a.d[j] = xv;
          if (qrow >= j + 2) sq_r = xv * xv;
        }
      }
      if (qsub == 0) sq[qloc] = sq_r;
    }
    __syncthreads();
    if (warp == 0) {
      const double s = warp_sum(sq[lane] + sq[lane + 32]);
      if (lane == 0) part[P_SSQ] = s;
    }
    target += G;
    if (!grid_barrier(a.bar, target, a.err, &s_ok)) return;

    // ---- B: the reflector (every block the same), v staged in shared memory
    if (warp == 0) {
      const double sigma = sum_parts(a.part, G, P_SSQ);
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
          if (b == 0) {
            a.e[j] = beta;
            a.tau[j] = tau;
          }
        }
        sc[0] = tau;
        sc[1] = inv;
      }
    }
    for (int r = threadIdx.x; r < n; r += ST_THREADS)
      sv[r] = r > j + 1 ? a.col[r] : (r == j + 1 ? 1.0 : 0.0);
    __syncthreads();
    const double tau = sc[0], inv = sc[1];
    for (int r = j + 2 + threadIdx.x; r < n; r += ST_THREADS) sv[r] *= inv;
    __syncthreads();
    // reflector storage (row j of the row-major view) and this block's V rows
    for (int loc = threadIdx.x; loc < cnt; loc += ST_THREADS) {
      const int r = b + G * loc;
      const double v = sv[r];
      if (r >= j + 2) a.A[(size_t)j * n + r] = v;
      a.Vp[(size_t)jj * n + r] = v;
      sV[loc][jj] = v;
    }
    // t = A22 v on this block's rows, one warp per row. The row is read from
    // L2 in 16-byte pairs, eight per lane in flight (the loop is bound by the
    // latency of these loads, not by the float64 pipe): element j+1 alone when
    // its address is not 16-byte aligned, then pairs, then a last odd element.
    if (j < n - 1) {
      for (int loc = warp; loc < cnt; loc += ST_WARPS) {
        const int r = b + G * loc;
        if (r < j + 1) continue;
        const double* row = a.A + (size_t)r * n;
        const int k1 = j + 1;
        const int ka = k1 + (int)((reinterpret_cast<uintptr_t>(row + k1) >> 3) & 1);  // 16-byte aligned
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        if (lane == 0 && ka > k1) s0 = row[k1] * sv[k1];
        const int np2 = ka < n ? (n - ka) >> 1 : 0;  // pairs (ka + 2p, ka + 2p + 1)
        const double2* row2 = reinterpret_cast<const double2*>(row + ka);
        const double* svp = sv + ka;
        int p = lane;
        for (; p + 224 < np2; p += 256) {
          double2 x[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) x[u] = row2[p + 32 * u];
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            const int k = 2 * (p + 32 * u);
            s0 = fma(x[u].x, svp[k], s0);
            s1 = fma(x[u].y, svp[k + 1], s1);
            s2 = fma(x[u + 1].x, svp[k + 64], s2);
            s3 = fma(x[u + 1].y, svp[k + 65], s3);
          }
        }
        for (; p < np2; p += 32) {
          const double2 x = row2[p];
          s0 = fma(x.x, svp[2 * p], s0);
          s1 = fma(x.y, svp[2 * p + 1], s1);
        }
        if (lane == 1 && ka < n && ((n - ka) & 1)) s2 = fma(row[n - 1], sv[n - 1], s2);
        const double tr = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) {
          st[loc] = tr;
          if (r == j + 1) a.t[r] = tr;
        }
      }
    }
    __syncthreads();
    // partial y_q = V_q^T v, z_q = W_q^T v (q < jj) and t^T v over this block's rows
    if (threadIdx.x < 2 * NB + 1) {
      const int c = threadIdx.x;
      double p0 = 0.0, p1 = 0.0;
      if (j < n - 1 && (c == 2 * NB || (c % NB) < jj)) {
        const int q = c % NB;
        int loc = 0;
        for (; loc < cnt; ++loc) {
          const int r = b + G * loc;
          if (r < j + 1) continue;
          const double x = c == 2 * NB ? st[loc] : (c < NB ? sV[loc][q] : sW[loc][q]);
          if (loc & 1) p1 = fma(x, sv[r], p1);
          else p0 = fma(x, sv[r], p0);
        }
      }
      part[c] = p0 + p1;
    }
    target += G;
    if (!grid_barrier(a.bar, target, a.err, &s_ok)) return;

    // ---- C: y, z, t^T v summed over the blocks; w on this block's rows
    // (loads that do not depend on the sums are issued first)
    double vq_next = 0.0, wq_next = 0.0;  // V_q[j+1], W_q[j+1] for the next column
    if (warp == 1 && j + 1 < n && lane < jj) {
      vq_next = a.Vp[(size_t)lane * n + j + 1];
      wq_next = a.Wp[(size_t)lane * n + j + 1];
    }
    arow = load_arow(j + 1);
    double t_next = 0.0;  // t[j+1], written before the barrier by its owner
    if (warp == 0 && lane == 0 && j + 1 < n) t_next = a.t[j + 1];
    {
      // y_q, z_q: warp w sums coefficients 8w .. 8w+7 (y for w < 4, z after)
      // over the blocks: lane l loads them (two 16-byte loads per four) from
      // blocks l, l + 32, ...; the lanes then combine by a butterfly that
      // halves the live values at each of the first three steps, so lane l
      // ends with coefficient (l >> 2) & 7 summed over all lanes. Warp 0 also
      // sums t^T v. Every load is issued before the first addition.
      const int c0 = 8 * warp;
      const bool live = j < n - 1 && (c0 % NB) < jj;   // this warp's coefficients
      const bool with_tv = warp == 0 && j < n - 1;      // t^T v is needed from jj = 0 on
      if (live || with_tv) {
        constexpr int MAXB = 5;  // blocks per lane: G <= 160
        double2 v[MAXB][4];
        double tvp[MAXB];
#pragma unroll
        for (int i = 0; i < MAXB; ++i) {
          const int bb = lane + 32 * i;
          const bool ok = bb < G;
          const double2* src = reinterpret_cast<const double2*>(a.part + (size_t)bb * PW + c0);
#pragma unroll
          for (int u = 0; u < 4; ++u) v[i][u] = (ok && live) ? src[u] : make_double2(0.0, 0.0);
          tvp[i] = (ok && with_tv) ? a.part[(size_t)bb * PW + P_TV] : 0.0;
        }
        double acc[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[2 * u] = v[0][u].x;
          acc[2 * u + 1] = v[0][u].y;
        }
#pragma unroll
        for (int i = 1; i < MAXB; ++i)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            acc[2 * u] += v[i][u].x;
            acc[2 * u + 1] += v[i][u].y;
          }
        // butterfly: keep the half of the values selected by the lane bit
        double h4[4], h2[2], h1;
        {
          const bool up = lane & 16;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double send = up ? acc[i] : acc[i + 4];
            const double keep = up ? acc[i + 4] : acc[i];
            h4[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
          }
        }
        {
          const bool up = lane & 8;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const double send = up ? h4[i] : h4[i + 2];
            const double keep = up ? h4[i + 2] : h4[i];
            h2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
          }
        }
        {
          const bool up = lane & 4;
          const double send = up ? h2[0] : h2[1];
          const double keep = up ? h2[1] : h2[0];
          h1 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
        h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
        if ((lane & 3) == 0)
          scoef[c0 + ((lane & 16) ? 4 : 0) + ((lane & 8) ? 2 : 0) + ((lane & 4) ? 1 : 0)] = h1;
        if (with_tv) {
          double tv = tvp[0];
#pragma unroll
          for (int i = 1; i < MAXB; ++i) tv += tvp[i];
          tv = warp_sum(tv);
          if (lane == 0) scoef[P_TV] = tv;
        }
      } else {
        if (lane < 8) scoef[c0 + lane] = 0.0;
        if (warp == 0 && lane == 0) scoef[P_TV] = 0.0;
      }
      if (warp == 1 && lane < jj) {
        sVs[lane] = vq_next;
        sWs[lane] = wq_next;
      }
    }
    __syncthreads();
    if (warp == 0) {
      // alpha2 = -(tau/2) tau (t^T v - 2 y^T z)
      double yz = lane < jj ? scoef[lane] * scoef[NB + lane] : 0.0;
      yz = warp_sum(yz);
      if (lane == 0) sc[2] = -0.5 * tau * (tau * (scoef[P_TV] - 2.0 * yz));
    } else if (warp == 1) {
      // the quad sum of row j+1 exactly as its owner's quad forms it below
      const double x = quad_dot2(sWs, scoef, sVs, scoef + NB, jj, lane & 3);
      if (lane == 0) sc[3] = x;
    }
    __syncthreads();
    const double alpha2 = sc[2];
    if (threadIdx.x == 0 && j + 1 < n) {  // the next column's V_jj[j+1], W_jj[j+1]
      sVs[jj] = 1.0;
      sWs[jj] = j < n - 1 ? fma(tau, t_next - sc[3], alpha2) : 0.0;
    }
    if (warp * 8 < cnt) {
      const double x = quad_dot2(&sW[qloc][0], scoef, &sV[qloc][0], scoef + NB, jj, qsub);
      if (qsub == 0 && qmine) {
        double w = 0.0;
        if (j < n - 1 && qrow >= j + 1) w = fma(tau, st[qloc] - x, alpha2 * sv[qrow]);
        sW[qloc][jj] = w;
        a.Wp[(size_t)jj * n + qrow] = w;
      }
    }
    __syncthreads();  // sv, sc and the shared scalars are rewritten by the next column
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
  // about 8 rows per block, at most one block per SM (all blocks co-resident)
  const int G = (int)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(ctx->sm_count, 160), cdiv(n, 8)));
  if (cdiv(n, G) > MAXLOC)
    return set_error(OSMPS_EUNSUPPORTED, "sytrd: n=%lld needs more than %d rows per block",
                     (long long)n, MAXLOC);
  double* buf = (double*)ws_get(ctx, SLOT_TRD, (size_t)(2 * NB * n + 2 * n + (size_t)G * PW +
                                                        2 * n * 2 * NB + 64) * 8, s, &st);
  if (!buf) return st;
  double* Vp = buf;
  double* Wp = Vp + NB * n;
  double* col = Wp + NB * n;
  double* t = col + n;
  double* part = t + n;
  double* X = part + (size_t)G * PW;
  double* Y = X + 2 * NB * n;
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->dev_flags + 8);
  int* err = ctx->dev_flags + 3;
  OSMPS_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), s));
  unsigned base = 0;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nbp = (int)std::min<int64_t>(NB, n - k0);
    SytrdArgs a;
    a.A = A; a.n = (int)n; a.k0 = (int)k0; a.nbp = nbp;
    a.d = d; a.e = e; a.tau = tau; a.Vp = Vp; a.Wp = Wp;
    a.col = col; a.t = t; a.part = part;
    a.bar = bar; a.bar_base = base; a.err = err;
    void* args[] = {&a};
    // algorithmic float64 work of the panel: per column j (i columns of the
    // panel before it, m = n - j - 1 trailing rows) the product A22 v
    // (2 m^2) and the corrections V (W^T v) + W (V^T v) (8 m i)
    double pf = 0.0;
    for (int i = 0; i < nbp; ++i) {
      const double mm = (double)(n - (k0 + i) - 1);
      pf += 2.0 * mm * mm + 8.0 * mm * i;
    }
    const int ph = prof_begin(s);
    OSMPS_CUDA(cudaLaunchCooperativeKernel((void*)k_sytrd_panel, dim3(G), dim3(ST_THREADS), args,
                                           smem, s));
    note_launch();
    prof_end(ph, s, OSMPS_KERNEL_SYTRD_PANEL, pf, 0.0);
    base += 2u * (unsigned)nbp * (unsigned)G;
    const int64_t k = k0 + nbp, m = n - k;
    if (m <= 0) break;
    { k_pack_vw<<<grid_1d(m * 2 * NB), 256, 0, s>>>(Vp, Wp, n, k, m, nbp, X, Y); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    // A22 -= [V W] [W V]^T = V W^T + W V^T on the trailing block
    SplitView xv; xv.src = X; xv.rows = m; xv.K = 2 * NB; xv.s0 = 2 * NB; xv.sk = 1;
    SplitView yv; yv.src = Y; yv.rows = m; yv.K = 2 * NB; yv.s0 = 2 * NB; yv.sk = 1;
    OSMPS_TRY(gemm_emu(ctx, xv, yv, m, m, 2 * NB, A + k * n + k, n, s, true));
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
  cudaStream_t s = (cudaStream_t)stream;
  OSMPS_TRY(sytrd_tc(ctx, A, n, d, e, tau, s));
  int flag = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&flag, ctx->dev_flags + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (flag) {
    cudaMemsetAsync(ctx->dev_flags + 3, 0, sizeof(int), s);
    return set_error(OSMPS_ETIMEOUT, "osmps_sytrd: a grid barrier wait gave up");
  }
  return OSMPS_OK;
}
