// Float64 strided batched GEMM on the FP64 tensor path (mma.sync m8n8k4 f64).
//
// Used for the plain float64 contractions (Sec. 3.4 matvec and environment
// updates at OSMPS_PREC_FP64), the Gram matrices and projections of the
// eigendecomposition split (Sec. 2, Eq. AAD_ULLUD), theta formation and the
// QR shifts. Arbitrary element strides let one kernel express every
// transpose and index grouping the contractions need without copies.
//
// Tiling: 64x64 output tile per CTA, K step 16, 8 warps (2 x 4), each warp
// owns a 32x16 sub-tile = 4 x 2 fragments of 8x8. Global loads go through
// registers into a double-buffered shared tile.
#include "common.cuh"

namespace osmps {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 4, THREADS = 256;

struct Args {
  int64_t M, N, K;
  const double* A;
  int64_t sam, sak, sab;
  const double* B;
  int64_t sbk, sbn, sbb;
  double* C;
  int64_t scm, scn, scb;
  double alpha, beta;
};

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

template <bool A_KFAST, bool B_NFAST>
__global__ void __launch_bounds__(THREADS) k_gemm_f64(Args p) {
  __shared__ double As[2][BK][BM + PAD];
  __shared__ double Bs[2][BK][BN + PAD];

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 2) * 32, wn = (warp & 3) * 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t bz = blockIdx.z;
  const double* A = p.A + bz * p.sab;
  const double* B = p.B + bz * p.sbb;

  double ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * THREADS;
      int mm, kk;
      if (A_KFAST) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      ra[r] = (gm < p.M && gk < p.K) ? A[gm * p.sam + gk * p.sak] : 0.0;
      int nn;
      if (B_NFAST) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      int64_t gn = n0 + nn;
      gk = k0 + kk;
      rb[r] = (gn < p.N && gk < p.K) ? B[gk * p.sbk + gn * p.sbn] : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + r * THREADS;
      int mm, kk;
      if (A_KFAST) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      As[buf][kk][mm] = ra[r];
      int nn;
      if (B_NFAST) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      Bs[buf][kk][nn] = rb[r];
    }
  };

  double acc[4][2][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  const int64_t nk = cdiv(p.K, BK);
  if (nk > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int k4 = 0; k4 < BK; k4 += 4) {
      double a[4], b[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][k4 + tq][wm + i * 8 + g];
#pragma unroll
      for (int j = 0; j < 2; ++j) b[j] = Bs[buf][k4 + tq][wn + j * 8 + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) dmma(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
    if (kt + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }

  double* C = p.C + bz * p.scb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        int64_t gm = m0 + wm + i * 8 + g;
        int64_t gn = n0 + wn + j * 8 + tq * 2 + r;
        if (gm < p.M && gn < p.N) {
          double* c = C + gm * p.scm + gn * p.scn;
          double v = p.alpha * acc[i][j][r];
          if (p.beta != 0.0) v = fma(p.beta, *c, v);
          *c = v;
        }
      }
}

}  // namespace

osmps_status gemm_f64(const GemmF64& g, cudaStream_t stream) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return OSMPS_OK;
  if (g.K <= 0) {
    return set_error(OSMPS_ESHAPE, "gemm_f64: K=%lld", (long long)g.K);
  }
  if (cdiv(g.M, BM) > 65535 || g.batch > 65535)
    return set_error(OSMPS_ESHAPE, "gemm_f64: M=%lld batch=%lld exceed the grid limits",
                     (long long)g.M, (long long)g.batch);
  Args a{g.M, g.N, g.K, g.A, g.sam, g.sak, g.sab, g.B, g.sbk, g.sbn, g.sbb,
         g.C, g.scm, g.scn, g.scb, g.alpha, g.beta};
  dim3 grid((unsigned)cdiv(g.N, BN), (unsigned)cdiv(g.M, BM), (unsigned)g.batch);
  bool akf = (g.sak == 1), bnf = (g.sbn == 1);
  const int ph = prof_begin(stream);
  if (akf && bnf) { k_gemm_f64<true, true><<<grid, THREADS, 0, stream>>>(a); note_launch(); }
  else if (akf) { k_gemm_f64<true, false><<<grid, THREADS, 0, stream>>>(a); note_launch(); }
  else if (bnf) { k_gemm_f64<false, true><<<grid, THREADS, 0, stream>>>(a); note_launch(); }
  else { k_gemm_f64<false, false><<<grid, THREADS, 0, stream>>>(a); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  const double f = 2.0 * (double)g.M * (double)g.N * (double)g.K * (double)g.batch;
  prof_end(ph, stream, OSMPS_KERNEL_GEMM_F64, f, f);
  return OSMPS_OK;
}

}  // namespace osmps
