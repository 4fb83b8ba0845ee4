// Gradients for the differentiation workload (Sec. 3.4 operators, Eq. mpo).
//
// H_eff.theta is linear in theta, W1 and W2 (Fig. LanczosMPS), and the MPO
// energy <psi|H|psi> / <psi|psi> at a fixed state is linear in every MPO
// site tensor, so every cotangent is a full contraction of the incoming
// cotangent with all other factors:
//   g_theta = H_eff^T gy: the same four-stage product with bra and ket
//             swapped in L, W1, W2 and R;
//   g_W1[w,t1,s1,w1] = sum T1[a2,w,s1,s2,c] P[a2,t1,w1,s2,c], with
//             T1 = L theta (stage 1), Q = gy R (over c2), P = Q W2 (over t2, w2);
//   g_W2[w1,t2,s2,w2] = sum T2[a2,t1,w1,s2,c] Q[a2,t1,t2,w2,c], T2 = T1 W1;
//   dE/dW_k[w,t,s,w2] = sum L_k[a2,w,a] A[a2,t,b2] A[a,s,b] R_{k+1}[b2,w2,b] / <psi|psi>.
// The weight-gradient contractions (a sum over all fibers of the outer
// product of two short vectors) run in a shared-memory-tiled reduction; the
// large contractions are GEMMs (float64 DMMA or the float64-accurate
// emulated tensor-core GEMM). The chain rule from dE/dW to Hamiltonian
// couplings is a sparse gather with the affine coupling basis dW/dp.
#include <algorithm>

#include "common.cuh"

namespace osmps {

namespace {

constexpr int WG_THREADS = 256;
constexpr int WG_TILE = 32;    // fibers per shared-memory tile (consecutive c)
constexpr int WG_MAXP = 64;
constexpr int WG_PAIRS = 16;   // (i, o) pairs per thread: P * Q <= 16 * 256

// part[b][i*Q + o] = sum over block b's fibers of X[fiber, i] * Y[fiber, o]
__global__ void __launch_bounds__(WG_THREADS) k_fiber_wgrad(Fiber f, const double* __restrict__ X,
                                                            const double* __restrict__ Y,
                                                            double* __restrict__ part) {
  __shared__ double xs[WG_MAXP][WG_TILE + 1];
  __shared__ double ys[WG_MAXP][WG_TILE + 1];
  const int P = (int)f.P, Q = (int)f.Q, PQ = P * Q;
  double acc[WG_PAIRS];
#pragma unroll
  for (int u = 0; u < WG_PAIRS; ++u) acc[u] = 0.0;
  const int64_t ctiles = cdiv(f.nc, WG_TILE);
  const int64_t ntiles = f.n_o1 * f.n_o2 * ctiles;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t ct = tile % ctiles, o12 = tile / ctiles;
    const int64_t o2 = o12 % f.n_o2, o1 = o12 / f.n_o2;
    const int64_t c0 = ct * WG_TILE;
    const double* xb = X + o1 * f.is1 + o2 * f.is2 + c0;
    const double* yb = Y + o1 * f.os1 + o2 * f.os2 + c0;
    for (int e = threadIdx.x; e < (P + Q) * WG_TILE; e += WG_THREADS) {
      const int row = e / WG_TILE, cc = e - row * WG_TILE;
      const bool in = c0 + cc < f.nc;
      if (row < P) xs[row][cc] = in ? xb[(int64_t)row * f.istride + cc] : 0.0;
      else ys[row - P][cc] = in ? yb[(int64_t)(row - P) * f.ostride + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < WG_PAIRS; ++u) {
      const int pq = threadIdx.x + u * WG_THREADS;
      if (pq < PQ) {
        const int i = pq / Q, o = pq - i * Q;
        double a = acc[u];
        for (int cc = 0; cc < WG_TILE; ++cc) a = fma(xs[i][cc], ys[o][cc], a);
        acc[u] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < WG_PAIRS; ++u) {
    const int pq = threadIdx.x + u * WG_THREADS;
    if (pq < PQ) part[(int64_t)blockIdx.x * PQ + pq] = acc[u];
  }
}

// Block partials summed in a fixed order (deterministic).
__global__ void k_sum_parts(const double* __restrict__ part, int nb, int PQ, double* __restrict__ out) {
  for (int pq = blockIdx.x * blockDim.x + threadIdx.x; pq < PQ; pq += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += part[(int64_t)b * PQ + pq];
    out[pq] = a;
  }
}

// gW[w,t,s,w2] = scale * G[i][o] with i = (w, s), o = (t, w2): the inverse of
// the W reorder WORD_IN_W_S__OUT_T_W2.
__global__ void k_w_unreorder(const double* __restrict__ G, int64_t dw, int64_t d, int64_t dw2,
                              double scale, double* __restrict__ gW) {
  const int64_t total = dw * d * d * dw2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t w2 = e % dw2, r = e / dw2;
    const int64_t s = r % d;
    r /= d;
    const int64_t t = r % d, w = r / d;
    gW[e] = scale * G[(w * d + s) * (d * dw2) + (t * dw2 + w2)];
  }
}

// out[x, w, y] = in[y, w, x]: bra and ket of an environment swapped
__global__ void k_env_transpose(const double* __restrict__ in, int64_t chi, int64_t w,
                                double* __restrict__ out) {
  const int64_t total = chi * w * chi;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = e % chi, r = e / chi;
    const int64_t ww = r % w, x = r / w;
    out[e] = in[(y * w + ww) * chi + x];
  }
}

// out[w, x, y, w2] = in[w, y, x, w2]: bra and ket of an MPO tensor swapped
__global__ void k_w_transpose(const double* __restrict__ in, int64_t dw, int64_t d, int64_t dw2,
                              double* __restrict__ out) {
  const int64_t total = dw * d * d * dw2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t w2 = e % dw2, r = e / dw2;
    const int64_t y = r % d;
    r /= d;
    const int64_t x = r % d, w = r / d;
    out[e] = in[((w * d + y) * d + x) * dw2 + w2];
  }
}

// g_par[p] = sum_{j in [row_ptr[p], row_ptr[p+1])} val[j] * g[col[j]]: one warp
// per parameter, fixed-order shuffle reduction. An index outside [0, n_g) or a
// bad row pointer is recorded in *bad and contributes nothing.
__global__ void k_csr_gather(int64_t n_par, const int64_t* __restrict__ row_ptr,
                             const int64_t* __restrict__ col, const double* __restrict__ val,
                             const double* __restrict__ g, int64_t n_g, int64_t nnz,
                             double* __restrict__ out, int* bad) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < n_par; p += nwarps) {
    int64_t j0 = row_ptr[p], j1 = row_ptr[p + 1];
    if (j0 < 0 || j1 < j0 || j1 > nnz) {
      if (lane == 0) atomicOr(bad, 1);
      j0 = j1 = 0;  // treated as an empty row
    }
    double a = 0.0;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
      const int64_t c = col[j];
      if (c >= 0 && c < n_g) a = fma(val[j], g[c], a);
      else atomicOr(bad, 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[p] = a;
  }
}

int nblk(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), 8192)); }

bool wgrad_fits(int64_t P, int64_t Q) {
  return P <= WG_MAXP && Q <= WG_MAXP && P * Q <= (int64_t)WG_PAIRS * WG_THREADS;
}

// Float64-accurate GEMM on views: emulated tensor cores, or DMMA for FP64.
osmps_status gemm_views(osmps_ctx* ctx, int precision, const SplitView& a, const SplitView& b,
                        int64_t M, int64_t N, int64_t K, double* C, int64_t ldc, cudaStream_t s) {
  if (precision != OSMPS_PREC_FP64) return gemm_emu(ctx, a, b, M, N, K, C, ldc, s);
  if (a.n1 != 1 || b.n1 != 1)
    return set_error(OSMPS_EUNSUPPORTED, "gradient GEMM: two-level views need the emulated path");
  GemmF64 g;
  g.M = M; g.N = N; g.K = K;
  g.A = (const double*)a.src; g.sam = a.s0; g.sak = a.sk;
  g.B = (const double*)b.src; g.sbk = b.sk; g.sbn = b.s0;
  g.C = C; g.scm = ldc; g.scn = 1;
  return gemm_f64(g, s);
}

}  // namespace

osmps_status fiber_weight_grad(osmps_ctx* ctx, const Fiber& f, const double* X, const double* Y,
                               double* dMat, cudaStream_t s) {
  if (!wgrad_fits(f.P, f.Q))
    return set_error(OSMPS_EUNSUPPORTED, "weight gradient: MPO block %lld x %lld too large",
                     (long long)f.P, (long long)f.Q);
  osmps_status st = OSMPS_OK;
  const int64_t ntiles = f.n_o1 * f.n_o2 * cdiv(f.nc, WG_TILE);
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, 4 * (int64_t)ctx->sm_count));
  const int PQ = (int)(f.P * f.Q);
  double* part = (double*)ws_get(ctx, SLOT_GRAD_PART, (size_t)nb * PQ * 8, s, &st);
  if (!part) return st;
  { k_fiber_wgrad<<<nb, WG_THREADS, 0, s>>>(f, X, Y, part); note_launch(); }
  { k_sum_parts<<<nblk(PQ), 256, 0, s>>>(part, nb, PQ, dMat); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

static osmps_status heff_backward_impl(osmps_ctx* ctx, const double* L, const double* W1,
                                       const double* W2, const double* R, const double* theta,
                                       const double* gy, double* gtheta, double* gW1, double* gW2,
                                       int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r,
                                       int64_t wl, int64_t wm, int64_t wr, int precision,
                                       cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  if (gtheta) {
    // H_eff^T: bra and ket swapped in every factor, then the forward product
    const size_t nL = (size_t)chi_l * wl * chi_l, nR = (size_t)chi_r * wr * chi_r;
    const size_t n1 = (size_t)wl * d1 * d1 * wm, n2 = (size_t)wm * d2 * d2 * wr;
    double* buf = (double*)ws_get(ctx, SLOT_GRAD_T, (nL + nR + n1 + n2) * 8, s, &st);
    if (!buf) return st;
    double* Lt = buf;
    double* Rt = Lt + nL;
    double* W1t = Rt + nR;
    double* W2t = W1t + n1;
    { k_env_transpose<<<nblk(nL), 256, 0, s>>>(L, chi_l, wl, Lt); note_launch(); }
    { k_env_transpose<<<nblk(nR), 256, 0, s>>>(R, chi_r, wr, Rt); note_launch(); }
    { k_w_transpose<<<nblk(n1), 256, 0, s>>>(W1, wl, d1, wm, W1t); note_launch(); }
    { k_w_transpose<<<nblk(n2), 256, 0, s>>>(W2, wm, d2, wr, W2t); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    OSMPS_TRY(heff_apply_impl(ctx, Lt, W1t, W2t, Rt, gy, gtheta, chi_l, d1, d2, chi_r, wl, wm, wr,
                              precision, s, false));
  }
  if (!gW1 && !gW2) return OSMPS_OK;
  // The weight gradients are float64-accurate in every precision.
  const int gp = precision == OSMPS_PREC_FP64 ? OSMPS_PREC_FP64 : OSMPS_PREC_FP64_EMU;
  const int64_t N1 = d1 * d2 * chi_r;
  double* T1 = (double*)ws_get(ctx, SLOT_GRAD_A, (size_t)chi_l * wl * N1 * 8, s, &st);
  if (!T1) return st;
  double* Q = (double*)ws_get(ctx, SLOT_GRAD_B, (size_t)chi_l * d1 * d2 * wr * chi_r * 8, s, &st);
  if (!Q) return st;
  double* PT = (double*)ws_get(ctx, SLOT_GRAD_C, (size_t)chi_l * d1 * wm * d2 * chi_r * 8, s, &st);
  if (!PT) return st;
  double* mats = (double*)ws_get(ctx, SLOT_GRAD_M, (size_t)2 * WG_MAXP * WG_MAXP * 8, s, &st);
  if (!mats) return st;
  double* wmat = mats;                       // a reordered MPO tensor
  double* dmat = mats + WG_MAXP * WG_MAXP;   // a weight gradient before the inverse reorder
  // T1[(a2,w), (s1,s2,c)] = sum_a L[(a2,w), a] theta[a, (s1,s2,c)]
  SplitView la; la.src = L; la.rows = chi_l * wl; la.K = chi_l; la.s0 = chi_l; la.sk = 1;
  SplitView tt; tt.src = theta; tt.rows = N1; tt.K = chi_l; tt.s0 = 1; tt.sk = N1;
  OSMPS_TRY(gemm_views(ctx, gp, la, tt, chi_l * wl, N1, chi_l, T1, N1, s));
  // Q[(a2,t1,t2), (w2,c)] = sum_c2 gy[(a2,t1,t2), c2] R[c2, (w2,c)]
  const int64_t M4 = chi_l * d1 * d2, K4 = wr * chi_r;
  SplitView gv; gv.src = gy; gv.rows = M4; gv.K = chi_r; gv.s0 = chi_r; gv.sk = 1;
  SplitView rv; rv.src = R; rv.rows = K4; rv.K = chi_r; rv.s0 = 1; rv.sk = K4;
  OSMPS_TRY(gemm_views(ctx, gp, gv, rv, M4, K4, chi_r, Q, K4, s));
  Fiber f2;  // stage-2 layout: outer (a2, s2), i = (w, s1), o = (t1, w1), inner c
  f2.P = wl * d1; f2.Q = d1 * wm; f2.n_o1 = chi_l; f2.n_o2 = d2; f2.nc = chi_r;
  f2.is1 = wl * d1 * d2 * chi_r; f2.is2 = chi_r; f2.istride = d2 * chi_r;
  f2.os1 = d1 * wm * d2 * chi_r; f2.os2 = chi_r; f2.ostride = d2 * chi_r;
  Fiber f3;  // stage-3 layout: outer (a2, t1), i = (w1, s2), o = (t2, w2), inner c
  f3.P = wm * d2; f3.Q = d2 * wr; f3.n_o1 = chi_l * d1; f3.n_o2 = 1; f3.nc = chi_r;
  f3.is1 = wm * d2 * chi_r; f3.istride = chi_r; f3.os1 = d2 * wr * chi_r; f3.ostride = chi_r;
  if (gW1) {
    // P[a2,t1,(w1,s2),c] = sum_{(t2,w2)} Q[a2,t1,(t2,w2),c] W2[w1,t2,s2,w2]: stage 3 run backwards
    OSMPS_TRY(w_reorder(W2, wm, d2, wr, WORD_IN_T_W2__OUT_W_S, wmat, s));
    Fiber fb;
    fb.P = d2 * wr; fb.Q = wm * d2; fb.n_o1 = chi_l * d1; fb.n_o2 = 1; fb.nc = chi_r;
    fb.is1 = d2 * wr * chi_r; fb.istride = chi_r; fb.os1 = wm * d2 * chi_r; fb.ostride = chi_r;
    OSMPS_TRY(fiber_contract_f64(fb, wmat, Q, PT, s));
    OSMPS_TRY(fiber_weight_grad(ctx, f2, T1, PT, dmat, s));
    { k_w_unreorder<<<nblk(wl * d1 * d1 * wm), 256, 0, s>>>(dmat, wl, d1, wm, 1.0, gW1); note_launch(); }
    OSMPS_LAUNCH_CHECK();
  }
  if (gW2) {
    // T2 = T1 W1 (stage 2), then g_W2 = sum over the stage-3 fibers of T2 (x) Q
    OSMPS_TRY(w_reorder(W1, wl, d1, wm, WORD_IN_W_S__OUT_T_W2, wmat, s));
    OSMPS_TRY(fiber_contract_f64(f2, wmat, T1, PT, s));
    OSMPS_TRY(fiber_weight_grad(ctx, f3, PT, Q, dmat, s));
    { k_w_unreorder<<<nblk(wm * d2 * d2 * wr), 256, 0, s>>>(dmat, wm, d2, wr, 1.0, gW2); note_launch(); }
    OSMPS_LAUNCH_CHECK();
  }
  return OSMPS_OK;
}

osmps_status site_energy_grad(osmps_ctx* ctx, const double* Lenv, const double* A,
                              const double* Renv, double* gW, int64_t chi_l, int64_t d,
                              int64_t chi_r, int64_t wl, int64_t wr, double scale, int precision,
                              cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  double* X = (double*)ws_get(ctx, SLOT_GRAD_A, (size_t)chi_l * wl * d * chi_r * 8, s, &st);
  if (!X) return st;
  double* Y = (double*)ws_get(ctx, SLOT_GRAD_B, (size_t)chi_l * d * wr * chi_r * 8, s, &st);
  if (!Y) return st;
  double* dmat = (double*)ws_get(ctx, SLOT_GRAD_M, (size_t)2 * WG_MAXP * WG_MAXP * 8, s, &st);
  if (!dmat) return st;
  // X[(a2, w), (s, b)] = sum_a L[(a2, w), a] A[a, (s, b)]
  SplitView lv; lv.src = Lenv; lv.rows = chi_l * wl; lv.K = chi_l; lv.s0 = chi_l; lv.sk = 1;
  SplitView at; at.src = A; at.rows = d * chi_r; at.K = chi_l; at.s0 = 1; at.sk = d * chi_r;
  OSMPS_TRY(gemm_views(ctx, precision, lv, at, chi_l * wl, d * chi_r, chi_l, X, d * chi_r, s));
  // Y[(a2, t), (w2, b)] = sum_b2 A[(a2, t), b2] R[b2, (w2, b)]
  SplitView av; av.src = A; av.rows = chi_l * d; av.K = chi_r; av.s0 = chi_r; av.sk = 1;
  SplitView rv; rv.src = Renv; rv.rows = wr * chi_r; rv.K = chi_r; rv.s0 = 1; rv.sk = wr * chi_r;
  OSMPS_TRY(gemm_views(ctx, precision, av, rv, chi_l * d, wr * chi_r, chi_r, Y, wr * chi_r, s));
  Fiber f;  // fibers (a2, b): i = (w, s) in X, o = (t, w2) in Y
  f.P = wl * d; f.Q = d * wr; f.n_o1 = chi_l; f.n_o2 = 1; f.nc = chi_r;
  f.is1 = wl * d * chi_r; f.istride = chi_r; f.os1 = d * wr * chi_r; f.ostride = chi_r;
  OSMPS_TRY(fiber_weight_grad(ctx, f, X, Y, dmat, s));
  { k_w_unreorder<<<nblk(wl * d * d * wr), 256, 0, s>>>(dmat, wl, d, wr, scale, gW); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

}  // namespace osmps

using namespace osmps;

extern "C" {

osmps_status osmps_heff_backward(osmps_ctx* ctx, const double* L, const double* W1,
                                 const double* W2, const double* R, const double* theta,
                                 const double* gy, double* gtheta, double* gW1, double* gW2,
                                 int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int64_t wl,
                                 int64_t wm, int64_t wr, int precision, void* stream) {
  clear_error();
  if (!ctx || !L || !W1 || !W2 || !R || !gy || (!theta && (gW1 || gW2)))
    return set_error(OSMPS_EINVAL, "osmps_heff_backward: null argument");
  if (gtheta && (gtheta == gy || gtheta == theta))
    return set_error(OSMPS_EINVAL, "osmps_heff_backward: g_theta aliases an input");
  if (!valid_precision(precision))
    return set_error(OSMPS_EINVAL, "osmps_heff_backward: precision %d", precision);
  for (int64_t x : {chi_l, d1, d2, chi_r, wl, wm, wr})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_heff_backward: non-positive or oversized dimension");
  if ((gW1 || gW2) && !(wgrad_fits(wl * d1, d1 * wm) && wgrad_fits(wm * d2, d2 * wr) &&
                        wgrad_fits(d2 * wr, wm * d2)))
    return set_error(OSMPS_EUNSUPPORTED, "osmps_heff_backward: MPO blocks too large for the weight gradient");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  return heff_backward_impl(ctx, L, W1, W2, R, theta, gy, gtheta, gW1, gW2, chi_l, d1, d2, chi_r,
                            wl, wm, wr, precision, (cudaStream_t)stream);
}

osmps_status osmps_coupling_grad(osmps_ctx* ctx, int64_t n_par, const int64_t* row_ptr,
                                 const int64_t* col, const double* val, int64_t nnz,
                                 const double* gW, int64_t n_w, double* g_par, void* stream) {
  clear_error();
  if (!ctx || (n_par > 0 && (!row_ptr || !g_par)) || (nnz > 0 && (!col || !val || !gW)))
    return set_error(OSMPS_EINVAL, "osmps_coupling_grad: null argument");
  if (n_par < 0 || nnz < 0 || n_w < 0)
    return set_error(OSMPS_ESHAPE, "osmps_coupling_grad: negative size");
  if (n_par == 0) return OSMPS_OK;
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  int* bad = ctx->dev_flags + 2;
  OSMPS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n_par, 8), 4096));
  { k_csr_gather<<<blocks, 256, 0, s>>>(n_par, row_ptr, col, val, gW, n_w, nnz, g_par, bad); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  int h = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (h) return set_error(OSMPS_EINVAL, "osmps_coupling_grad: basis index out of range");
  return OSMPS_OK;
}

}  // extern "C"
