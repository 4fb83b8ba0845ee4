// Two-site time-dependent variational principle (Sec. 5.4): real-time
// evolution |psi(t + dt)> = exp(-i H dt) |psi(t)> (Eq. propSE) projected onto
// MPS of bounded bond dimension, with the local propagators of Sec. 5.2
// (Eq. krylov:approx) applied to the centre tensor only.
//
// One time step dt is the symmetric second-order scheme: a left-to-right
// half sweep with dt/2, then a right-to-left half sweep with dt/2. At the
// pair (k, k+1), left to right: theta = A_k A_{k+1};
// theta <- exp(-i H_eff dt/2) theta; theta = U S V^dagger truncated as in the
// ground-state search; A_k = U; grow L; unless k+1 is the last site,
// C = S V^dagger <- exp(+i H1_eff dt/2) C with the one-site H_eff of site
// k+1; A_{k+1} = C. Right to left mirrored (A_{k+1} = V^dagger, grow R,
// C = U S evolved backwards at site k unless k = 0).
//
// Complex tensors live on the device in the real 2x2 embedding of the
// Krylov propagator (lanczos.cu): X[r, w, c] -> X~[(p, r), w, (q, c)].
// Products of embedded tensors are embedded products, so theta formation,
// H_eff.theta and the environment updates are the real kernels of the
// ground-state search at doubled bond dimensions. The left environments are
// emb(L); the right ones come out as emb(conj R), which is the form the real
// H_eff.theta needs. The split forms the complex Hermitian Gram matrix from
// the embedded one, takes its eigenpairs from cuSOLVER zheevd (Eq. AAD_ULLUD,
// the eigendecomposition route of the ground-state split), truncates by the
// same rule, and re-embeds the kept vectors.
#include <cuComplex.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

namespace osmps {

namespace {

__device__ __forceinline__ int64_t emb_index(int64_t i, int q, int64_t bw) {
  // position of (q, i) in an embedded index whose complex index i = (g, r),
  // r < bw, is laid out as (g, q, r)
  const int64_t g = i / bw;
  return g * 2 * bw + q * bw + (i - g * bw);
}

// Complex Hermitian Gram matrix (column-major nz x nz) from its real
// embedding Gt (2nz x 2nz, row-major): entry (i, j) = Gt[(0,i),(0,j)] +
// i Gt[(1,i),(0,j)], the embedded index of (q, i) given by emb_index with
// block width bw.
__global__ void k_gram_to_complex(const double* __restrict__ Gt, cuDoubleComplex* __restrict__ Z,
                                  int64_t nz, int64_t bw) {
  const int64_t n2 = 2 * nz, total = nz * nz;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / nz, i = e - j * nz;
    const int64_t c0 = emb_index(j, 0, bw);
    Z[e] = make_cuDoubleComplex(Gt[emb_index(i, 0, bw) * n2 + c0], Gt[emb_index(i, 1, bw) * n2 + c0]);
  }
}

// Left-to-right: A1~ = emb(U_kept) as (2m) x (2 keep), rows (p, i), columns
// (q, j), with U[i, k] = Z[k m + i] (zheevd's column-major eigenvectors).
__global__ void k_embed_kept_cols(const cuDoubleComplex* __restrict__ Z, const int* __restrict__ idx,
                                  double* __restrict__ out, int64_t m, int64_t keep) {
  const int64_t total = m * keep, row = 2 * keep;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / keep, j = e - i * keep;
    const cuDoubleComplex v = Z[(int64_t)idx[j] * m + i];
    const int64_t o0 = i * row + j, o1 = (m + i) * row + j;
    out[o0] = v.x;
    out[o0 + keep] = -v.y;
    out[o1] = v.y;  // (1,0) block: Im
    out[o1 + keep] = v.x;
  }
}

// Right-to-left: B~ = emb(V_kept^dagger) as (2 keep) x (d2, 2 chi_r), rows
// (p, j), columns (s2, q, c), with V[i, k] = Z[k n + i], i = (s2, c).
__global__ void k_embed_kept_rows_conj(const cuDoubleComplex* __restrict__ Z,
                                       const int* __restrict__ idx, double* __restrict__ out,
                                       int64_t n, int64_t keep, int64_t chi_r) {
  const int64_t total = keep * n, row = 2 * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const cuDoubleComplex v = Z[(int64_t)idx[j] * n + i];
    const double re = v.x, im = -v.y;  // conjugate
    const int64_t c0 = emb_index(i, 0, chi_r), c1 = emb_index(i, 1, chi_r);
    out[j * row + c0] = re;
    out[j * row + c1] = -im;
    out[(keep + j) * row + c0] = im;
    out[(keep + j) * row + c1] = re;
  }
}

// x <- x sqrt(2 / ||x||^2): unit complex norm for an embedded tensor (whose
// real norm^2 is twice the complex one).
__global__ void k_unit_embedded(double* __restrict__ x, int64_t n, const double* __restrict__ nrm2) {
  const double f = sqrt(2.0 / nrm2[0]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

// z[i, k, j] = emb^{-1}(out): the average of the duplicate blocks,
// re = (B00 + B11) / 2, im = (B10 - B01) / 2; z interleaved complex.
__global__ void k_extract3(const double* __restrict__ emb, double* __restrict__ z, int64_t r,
                           int64_t w, int64_t c) {
  const int64_t wc = w * c, n = r * wc, row = 2 * c, plane = r * w * row;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / wc, rem = e - i * wc, k = rem / c, jj = rem - k * c;
    const int64_t o = (i * w + k) * row + jj;
    z[2 * e] = 0.5 * (emb[o] + emb[plane + o + c]);
    z[2 * e + 1] = 0.5 * (emb[plane + o] - emb[o + c]);
  }
}

// out[0] = x . y, out[1] = x . x, one block, fixed order.
__global__ void k_dot2(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                       double* __restrict__ out) {
  __shared__ double sh[2][8];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    a = fma(x[i], y[i], a);
    b = fma(x[i], x[i], b);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = a;
    sh[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s0 += sh[0][k];
      s1 += sh[1][k];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

int grid_for(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 8192) b = 8192;
  return (int)b;
}

}  // namespace

// Split of an embedded two-site tensor th~ = emb(theta), theta as the complex
// (chi_l d1) x (d2 chi_r) matrix M, with truncation (Sec. 2, Eq. AAD_ULLUD):
//   move_right: G = M M^dagger = U lambda^2 U^dagger; A1 = U_kept
//               (left-canonical), A2 = U_kept^dagger M renormalised;
//   otherwise:  G = M^dagger M = V lambda^2 V^dagger; A2 = V_kept^dagger
//               (right-canonical), A1 = M V_kept renormalised.
// A1~ (2 chi_l, d1, 2 keep) and A2~ (2 keep, d2, 2 chi_r) are written
// embedded. The Gram matrix and the projection are float64 GEMMs on the
// embedded tensors (DMMA for OSMPS_PREC_FP64, the emulated float64 GEMM
// otherwise); the eigenpairs come from cuSOLVER (zheevdx for the largest
// min(chi_max, rank) only, zheevd when that is all of them); chi' and the
// discarded weight follow truncate_spectrum with tr = ||theta||^2.
osmps_status split_embedded(osmps_ctx* ctx, const double* th, double* A1, double* A2,
                            int64_t chi_l, int64_t d1, int64_t d2, int64_t chi_r, int move_right,
                            int64_t chi_max, double eps_local, int precision, int64_t* chi_new,
                            double* discarded, double* entropy, double* lam2_out, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  const int64_t m = chi_l * d1, n = d2 * chi_r, m2 = 2 * m, n2 = 2 * n;
  const int64_t nz = move_right ? m : n, g2 = 2 * nz;
  if (nz > 23170) return set_error(OSMPS_ESHAPE, "split: Gram dimension %lld too large", (long long)nz);
  const bool emu = precision != OSMPS_PREC_FP64;
  double* Gt = (double*)ws_get(ctx, SLOT_SPLIT_G, (size_t)g2 * g2 * 8, s, &st);
  if (!Gt) return st;
  cuDoubleComplex* Z = (cuDoubleComplex*)ws_get(ctx, SLOT_SPLIT_TMP2, (size_t)nz * nz * 16, s, &st);
  if (!Z) return st;
  double* ev = (double*)ws_get(ctx, SLOT_SPLIT_EV, (size_t)(nz + 8) * 8, s, &st);
  if (!ev) return st;
  double* tr_dev = ev + nz;  // ||th~||^2 = 2 ||theta||^2
  OSMPS_TRY(vec_norm2(ctx, th, m2 * n2, tr_dev, s));
  // embedded Gram: Gt = M~ M~^T (rows (p, a, s1)) or M~^T M~ (index (s2, q, c))
  if (emu) {
    SplitView mv;
    mv.src = th;
    if (move_right) { mv.rows = m2; mv.K = n2; mv.s0 = n2; mv.sk = 1; }
    else { mv.rows = n2; mv.K = m2; mv.s0 = 1; mv.sk = n2; }
    OSMPS_TRY(gemm_emu(ctx, mv, mv, g2, g2, mv.K, Gt, g2, s));
  } else {
    GemmF64 g;
    if (move_right) {
      g.M = m2; g.N = m2; g.K = n2;
      g.A = th; g.sam = n2; g.sak = 1;
      g.B = th; g.sbk = 1; g.sbn = n2;
    } else {
      g.M = n2; g.N = n2; g.K = m2;
      g.A = th; g.sam = 1; g.sak = n2;
      g.B = th; g.sbk = n2; g.sbn = 1;
    }
    g.C = Gt; g.scm = g2; g.scn = 1;
    OSMPS_TRY(gemm_f64(g, s));
  }
  { k_gram_to_complex<<<grid_for(nz * nz), 256, 0, s>>>(Gt, Z, nz, move_right ? m : chi_r); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  // Only the largest min(chi_max, rank) eigenpairs can be kept: compute just
  // those when that is fewer than all (zheevdx, range by index).
  const int64_t nev = std::min<int64_t>(nz, std::min<int64_t>(chi_max, std::min(m, n)));
  OSMPS_SOLVER(cusolverDnSetStream(ctx->solver, s));
  int lwork = 0, found = (int)nz;
  if (nev == nz) {
    OSMPS_SOLVER(cusolverDnZheevd_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                             CUBLAS_FILL_MODE_LOWER, (int)nz, Z, (int)nz, ev, &lwork));
    cuDoubleComplex* work =
        (cuDoubleComplex*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 16, s, &st);
    if (!work) return st;
    OSMPS_SOLVER(cusolverDnZheevd(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                                  (int)nz, Z, (int)nz, ev, work, lwork, ctx->dev_info));
  } else {
    const int il = (int)(nz - nev + 1), iu = (int)nz;
    OSMPS_SOLVER(cusolverDnZheevdx_bufferSize(ctx->solver, CUSOLVER_EIG_MODE_VECTOR,
                                              CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, (int)nz,
                                              Z, (int)nz, 0.0, 0.0, il, iu, &found, ev, &lwork));
    cuDoubleComplex* work =
        (cuDoubleComplex*)ws_get(ctx, SLOT_SPLIT_WORK, (size_t)std::max(lwork, 1) * 16, s, &st);
    if (!work) return st;
    OSMPS_SOLVER(cusolverDnZheevdx(ctx->solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                   CUBLAS_FILL_MODE_LOWER, (int)nz, Z, (int)nz, 0.0, 0.0, il, iu,
                                   &found, ev, work, lwork, ctx->dev_info));
  }
  OSMPS_TRY(pinned_reserve(ctx, (size_t)nz + 16));
  double* h = ctx->host_pinned;
  int info = 0;
  OSMPS_CUDA(cudaMemcpyAsync(h, ev, (size_t)(nz + 1) * 8, cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaMemcpyAsync(&info, ctx->dev_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (info != 0) return set_error(OSMPS_ECUDA, "split: zheevd info %d", info);
  if (found < 1 || found > nz) return set_error(OSMPS_ECUDA, "split: zheevdx found %d eigenpairs", found);
  const double trace = 0.5 * h[nz];
  // the selected eigenvectors occupy the first `found` columns of Z
  std::vector<double> ev_host(h, h + found);
  Trunc t;
  OSMPS_TRY(truncate_spectrum(ev_host.data(), found, trace, std::min(m, n), chi_max, eps_local, &t));
  const int64_t keep = t.keep;
  if (lam2_out)
    for (int64_t i = 0; i < std::min(m, n); ++i) lam2_out[i] = i < found ? t.lam2[i] : 0.0;
  *chi_new = keep;
  *discarded = t.discarded;
  *entropy = t.entropy;
  int* idx = (int*)ws_get(ctx, SLOT_QR_TAU, (size_t)keep * sizeof(int) + 256, s, &st);
  if (!idx) return st;
  OSMPS_CUDA(cudaMemcpyAsync(idx, t.order.data(), (size_t)keep * sizeof(int), cudaMemcpyHostToDevice, s));
  double* nrm = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);
  if (!nrm) return st;
  const int64_t k2 = 2 * keep;
  if (move_right) {
    { k_embed_kept_cols<<<grid_for(m * keep), 256, 0, s>>>(Z, idx, A1, m, keep); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    // A2~ = A1~^T M~: (2 keep) x (2n)
    if (emu) {
      SplitView a; a.src = A1; a.rows = k2; a.K = m2; a.s0 = 1; a.sk = k2;
      SplitView b; b.src = th; b.rows = n2; b.K = m2; b.s0 = 1; b.sk = n2;
      OSMPS_TRY(gemm_emu(ctx, a, b, k2, n2, m2, A2, n2, s));
    } else {
      GemmF64 p;
      p.M = k2; p.N = n2; p.K = m2;
      p.A = A1; p.sam = 1; p.sak = k2;
      p.B = th; p.sbk = n2; p.sbn = 1;
      p.C = A2; p.scm = n2; p.scn = 1;
      OSMPS_TRY(gemm_f64(p, s));
    }
    OSMPS_TRY(vec_norm2(ctx, A2, k2 * n2, nrm, s));
    { k_unit_embedded<<<grid_for(k2 * n2), 256, 0, s>>>(A2, k2 * n2, nrm); note_launch(); }
  } else {
    { k_embed_kept_rows_conj<<<grid_for(keep * n), 256, 0, s>>>(Z, idx, A2, n, keep, chi_r); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    // A1~ = M~ A2~^T: (2m) x (2 keep)
    if (emu) {
      SplitView a; a.src = th; a.rows = m2; a.K = n2; a.s0 = n2; a.sk = 1;
      SplitView b; b.src = A2; b.rows = k2; b.K = n2; b.s0 = n2; b.sk = 1;
      OSMPS_TRY(gemm_emu(ctx, a, b, m2, k2, n2, A1, k2, s));
    } else {
      GemmF64 p;
      p.M = m2; p.N = k2; p.K = n2;
      p.A = th; p.sam = n2; p.sak = 1;
      p.B = A2; p.sbk = 1; p.sbn = n2;
      p.C = A1; p.scm = k2; p.scn = 1;
      OSMPS_TRY(gemm_f64(p, s));
    }
    OSMPS_TRY(vec_norm2(ctx, A1, m2 * k2, nrm, s));
    { k_unit_embedded<<<grid_for(m2 * k2), 256, 0, s>>>(A1, m2 * k2, nrm); note_launch(); }
  }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

namespace {

// Device buffers of one evolution, freed on every exit path.
struct DevBufs {
  std::vector<double*> ptrs;
  ~DevBufs() {
    for (double* p : ptrs)
      if (p) cudaFree(p);
  }
  double* get(size_t doubles) {
    double* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(doubles, 1) * 8) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return p;
  }
};

__global__ void k_identity_bond(double* __restrict__ W, int64_t w) {
  // W[a, 0, 0, b] = delta(a, b): the one-site H_eff as a two-site one with d2 = 1
  for (int64_t e = threadIdx.x; e < w * w; e += blockDim.x) W[e] = (e / w == e % w) ? 1.0 : 0.0;
}

__global__ void k_boundary_env(double* __restrict__ E) {
  // emb of the boundary environment ones(1,1,1): the 2 x 1 x 2 identity
  if (threadIdx.x < 4) E[threadIdx.x] = (threadIdx.x == 0 || threadIdx.x == 3) ? 1.0 : 0.0;
}

}  // namespace

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_split_complex(osmps_ctx* ctx, const double* theta, double* A1,
                                            double* A2, int64_t chi_l, int64_t d1, int64_t d2,
                                            int64_t chi_r, int move_right, int64_t chi_max,
                                            double eps_local, int64_t* chi_new_out,
                                            double* discarded_out, double* entropy_out,
                                            double* lam2_out, int precision, void* stream) {
  clear_error();
  if (!ctx || !theta || !A1 || !A2 || !chi_new_out || !discarded_out || !entropy_out)
    return set_error(OSMPS_EINVAL, "osmps_split_complex: null argument");
  if (A1 == theta || A2 == theta || A1 == A2)
    return set_error(OSMPS_EINVAL, "osmps_split_complex: outputs alias each other or theta");
  if (move_right != 0 && move_right != 1)
    return set_error(OSMPS_EINVAL, "osmps_split_complex: move_right %d", move_right);
  if (chi_max < 1) return set_error(OSMPS_EINVAL, "osmps_split_complex: chi_max %lld", (long long)chi_max);
  if (!valid_precision(precision))
    return set_error(OSMPS_EINVAL, "osmps_split_complex: precision %d", precision);
  if (!(eps_local >= 0.0)) return set_error(OSMPS_EINVAL, "osmps_split_complex: eps_local %g", eps_local);
  for (int64_t x : {chi_l, d1, d2, chi_r})
    if (x <= 0 || x > ((int64_t)1 << 30))
      return set_error(OSMPS_ESHAPE, "osmps_split_complex: non-positive or oversized dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  const int64_t m = chi_l * d1, n = d2 * chi_r, kmax = std::min(chi_max, std::min(m, n));
  double* th = (double*)ws_get(ctx, SLOT_CX_THETA, (size_t)4 * m * n * 8, s, &st);
  if (!th) return st;
  double* e1 = (double*)ws_get(ctx, SLOT_CX_L, (size_t)4 * m * kmax * 8, s, &st);
  if (!e1) return st;
  double* e2 = (double*)ws_get(ctx, SLOT_CX_R, (size_t)4 * kmax * n * 8, s, &st);
  if (!e2) return st;
  OSMPS_TRY(embed_complex(theta, th, chi_l, d1 * d2, chi_r, false, s));
  OSMPS_TRY(split_embedded(ctx, th, e1, e2, chi_l, d1, d2, chi_r, move_right, chi_max, eps_local,
                           precision, chi_new_out, discarded_out, entropy_out, lam2_out, s));
  const int64_t keep = *chi_new_out;
  { k_extract3<<<grid_for(chi_l * d1 * keep), 256, 0, s>>>(e1, A1, chi_l, d1, keep); note_launch(); }
  { k_extract3<<<grid_for(keep * d2 * chi_r), 256, 0, s>>>(e2, A2, keep, d2, chi_r); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  OSMPS_CUDA(cudaStreamSynchronize(s));
  return OSMPS_OK;
}

extern "C" osmps_status osmps_tdvp_evolve(osmps_ctx* ctx, const osmps_mpo* mpo,
                                          const int64_t* chi_in, const double* const* host_in,
                                          const osmps_tdvp_params* p, int64_t* chi_out,
                                          double* const* host_out, osmps_tdvp_stats* stats,
                                          void* stream) {
  clear_error();
  if (!ctx || !mpo || !chi_in || !host_in || !p || !chi_out || !host_out)
    return set_error(OSMPS_EINVAL, "osmps_tdvp_evolve: null argument");
  if (mpo->ctx != ctx) return set_error(OSMPS_EINVAL, "osmps_tdvp_evolve: MPO of another context");
  const int64_t L = mpo->L;
  if (!std::isfinite(p->dt) || p->n_steps < 0 || p->chi_max < 1 || !(p->eps_local >= 0.0) ||
      !(p->krylov_tol >= 0.0) || p->krylov_max_iter < 1 || p->krylov_max_iter > 128 ||
      !valid_precision(p->precision))
    return set_error(OSMPS_EINVAL, "osmps_tdvp_evolve: bad parameters");
  if (chi_in[0] != 1 || chi_in[L] != 1)
    return set_error(OSMPS_ESHAPE, "osmps_tdvp_evolve: boundary bonds must be 1");
  // bond capacities: the exact bound min(prod d left, prod d right) and chi_max
  std::vector<int64_t> cap(L + 1), chi(chi_in, chi_in + L + 1);
  {
    std::vector<int64_t> left(L + 1, 1), right(L + 1, 1);
    for (int64_t k = 0; k < L; ++k) left[k + 1] = std::min<int64_t>(left[k] * mpo->d[k], 1 << 30);
    for (int64_t k = L - 1; k >= 0; --k) right[k] = std::min<int64_t>(right[k + 1] * mpo->d[k], 1 << 30);
    for (int64_t k = 0; k <= L; ++k) {
      cap[k] = std::min(p->chi_max, std::min(left[k], right[k]));
      if (chi[k] < 1 || chi[k] > cap[k] || !(k == L || host_in[k]))
        return set_error(OSMPS_ESHAPE, "osmps_tdvp_evolve: bond %lld has dimension %lld (at most %lld)",
                         (long long)k, (long long)chi[k], (long long)cap[k]);
    }
  }
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const auto t_start = std::chrono::steady_clock::now();
  const int prec = p->precision;
  const std::vector<int64_t>& d = mpo->d;
  const std::vector<int64_t>& w = mpo->w;
  DevBufs mem;
  std::vector<double*> At(L), Lt(L + 1, nullptr), Rt(L + 1, nullptr), Wid(L + 1, nullptr);
  size_t th_max = 1, site_max = 1;
  for (int64_t k = 0; k < L; ++k) {
    site_max = std::max<size_t>(site_max, (size_t)4 * cap[k] * d[k] * cap[k + 1]);
    if (k + 1 < L)
      th_max = std::max<size_t>(th_max, (size_t)4 * cap[k] * d[k] * d[k + 1] * cap[k + 2]);
  }
  for (int64_t k = 0; k < L; ++k)
    if (!(At[k] = mem.get((size_t)4 * cap[k] * d[k] * cap[k + 1])))
      return set_error(OSMPS_ENOMEM, "osmps_tdvp_evolve: out of device memory");
  for (int64_t k = 0; k <= L; ++k) {
    const size_t env = (size_t)4 * cap[k] * w[k] * cap[k];
    if (!(Lt[k] = mem.get(env)) || !(Rt[k] = mem.get(env)) || !(Wid[k] = mem.get((size_t)w[k] * w[k])))
      return set_error(OSMPS_ENOMEM, "osmps_tdvp_evolve: out of device memory");
    { k_identity_bond<<<1, 256, 0, s>>>(Wid[k], w[k]); note_launch(); }
  }
  double* TH = mem.get(th_max);
  double* Y = mem.get(site_max);
  double* Zc = mem.get(site_max / 2);
  double* dots = mem.get(2);
  if (!TH || !Y || !Zc || !dots) return set_error(OSMPS_ENOMEM, "osmps_tdvp_evolve: out of device memory");
  { k_boundary_env<<<1, 32, 0, s>>>(Lt[0]); note_launch(); }
  { k_boundary_env<<<1, 32, 0, s>>>(Rt[L]); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  // upload and embed the state; unit norm at the centre (site 0)
  for (int64_t k = 0; k < L; ++k) {
    const size_t nc = (size_t)chi[k] * d[k] * chi[k + 1];
    OSMPS_CUDA(cudaMemcpyAsync(Zc, host_in[k], nc * 16, cudaMemcpyHostToDevice, s));
    OSMPS_TRY(embed_complex(Zc, At[k], chi[k], d[k], chi[k + 1], false, s));
  }
  osmps_status st = OSMPS_OK;
  double* nrm = (double*)ws_get(ctx, SLOT_NORM, 64, s, &st);
  if (!nrm) return st;
  OSMPS_TRY(vec_norm2(ctx, At[0], 4 * chi[0] * d[0] * chi[1], nrm, s));
  { k_unit_embedded<<<grid_for(4 * chi[0] * d[0] * chi[1]), 256, 0, s>>>(At[0], 4 * chi[0] * d[0] * chi[1], nrm); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  for (int64_t k = L - 1; k >= 2; --k)
    OSMPS_TRY(env_update_impl(ctx, 1, Rt[k + 1], At[k], mpo->W[k], Rt[k], 2 * chi[k], d[k],
                              2 * chi[k + 1], w[k + 1], w[k], prec, s));

  osmps_tdvp_stats acc = {};
  if (stats) {
    acc.energy = stats->energy;
    acc.norm = stats->norm;
  }
  const double half = 0.5 * p->dt;
  auto propagate = [&](const double* Lenv, const double* W1, const double* W2, const double* Renv,
                       double* x, int64_t chl, int64_t d1, int64_t d2, int64_t chr, int64_t wl,
                       int64_t wm, int64_t wr, double tau) -> osmps_status {
    OSMPS_TRY(heff_prepare(ctx, Lenv, W1, W2, Renv, 2 * chl, d1, d2, 2 * chr, wl, wm, wr, prec, s));
    const Matvec mv = [&](const double* xv, double* yv, cudaStream_t q) {
      return heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, xv, yv, 2 * chl, d1, d2,
                             2 * chr, wl, wm, wr, prec, q, true);
    };
    int it = 0;
    double err = 0.0;
    const osmps_status es = expm_core(ctx, chl * d1 * d2 * chr, x, x, chl, d1 * d2, chr, tau,
                                      p->krylov_max_iter, p->krylov_tol, mv, &it, &err, s, true);
    if (es != OSMPS_OK && es != OSMPS_ENOCONV) return es;
    if (es == OSMPS_ENOCONV) ++acc.nonconverged;
    clear_error();
    acc.krylov_calls += 1;
    acc.krylov_vectors += it;
    acc.max_krylov = std::max(acc.max_krylov, it);
    return OSMPS_OK;
  };
  auto pair = [&](int64_t k, bool right) -> osmps_status {
    const int64_t chl = chi[k], chm = chi[k + 1], chr = chi[k + 2], d1 = d[k], d2 = d[k + 1];
    if (prec == OSMPS_PREC_FP64)
      OSMPS_TRY(theta_form_impl(At[k], At[k + 1], TH, 2 * chl, d1, 2 * chm, d2, 2 * chr, s));
    else
      OSMPS_TRY(theta_form_tc(ctx, At[k], At[k + 1], TH, 2 * chl, d1, 2 * chm, d2, 2 * chr, prec, s));
    OSMPS_TRY(propagate(Lt[k], mpo->W[k], mpo->W[k + 1], Rt[k + 2], TH, chl, d1, d2, chr, w[k],
                        w[k + 1], w[k + 2], half));
    int64_t keep = 0;
    double disc = 0.0, ent = 0.0;
    OSMPS_TRY(split_embedded(ctx, TH, At[k], At[k + 1], chl, d1, d2, chr, right ? 1 : 0,
                             cap[k + 1], p->eps_local, prec, &keep, &disc, &ent, nullptr, s));
    chi[k + 1] = keep;
    acc.max_discarded = std::max(acc.max_discarded, disc);
    acc.max_chi = std::max(acc.max_chi, keep);
    if (right) {
      OSMPS_TRY(env_update_impl(ctx, 0, Lt[k], At[k], mpo->W[k], Lt[k + 1], 2 * chl, d1, 2 * keep,
                                w[k], w[k + 1], prec, s));
      if (k + 1 < L - 1)
        OSMPS_TRY(propagate(Lt[k + 1], mpo->W[k + 1], Wid[k + 2], Rt[k + 2], At[k + 1], keep, d2, 1,
                            chr, w[k + 1], w[k + 2], w[k + 2], -half));
    } else {
      OSMPS_TRY(env_update_impl(ctx, 1, Rt[k + 2], At[k + 1], mpo->W[k + 1], Rt[k + 1], 2 * keep,
                                d2, 2 * chr, w[k + 2], w[k + 1], prec, s));
      if (k > 0)
        OSMPS_TRY(propagate(Lt[k], mpo->W[k], Wid[k + 1], Rt[k + 1], At[k], chl, d1, 1, keep, w[k],
                            w[k + 1], w[k + 1], -half));
    }
    return OSMPS_OK;
  };
  OSMPS_TRY(pinned_reserve(ctx, 16));
  for (int step = 0; step < p->n_steps; ++step) {
    for (int64_t k = 0; k + 1 < L; ++k) OSMPS_TRY(pair(k, true));
    for (int64_t k = L - 2; k >= 0; --k) OSMPS_TRY(pair(k, false));
    if (acc.energy || acc.norm) {
      // <H> and <psi|psi> at the centre (site 0) through the one-site H_eff
      const int64_t n0 = 4 * chi[0] * d[0] * chi[1];
      OSMPS_TRY(heff_prepare(ctx, Lt[0], mpo->W[0], Wid[1], Rt[1], 2 * chi[0], d[0], 1, 2 * chi[1],
                             w[0], w[1], w[1], prec, s));
      OSMPS_TRY(heff_apply_impl(ctx, nullptr, nullptr, nullptr, nullptr, At[0], Y, 2 * chi[0], d[0],
                                1, 2 * chi[1], w[0], w[1], w[1], prec, s, true));
      { k_dot2<<<1, 256, 0, s>>>(At[0], Y, n0, dots); note_launch(); }
      OSMPS_LAUNCH_CHECK();
      OSMPS_CUDA(cudaMemcpyAsync(ctx->host_pinned, dots, 16, cudaMemcpyDeviceToHost, s));
      OSMPS_CUDA(cudaStreamSynchronize(s));
      const double xy = ctx->host_pinned[0], xx = ctx->host_pinned[1];
      if (acc.energy) acc.energy[step] = xy / xx;
      if (acc.norm) acc.norm[step] = 0.5 * xx;
    }
  }
  // read the state back
  for (int64_t k = 0; k < L; ++k) {
    const int64_t nc = chi[k] * d[k] * chi[k + 1];
    { k_extract3<<<grid_for(nc), 256, 0, s>>>(At[k], Zc, chi[k], d[k], chi[k + 1]); note_launch(); }
    OSMPS_LAUNCH_CHECK();
    OSMPS_CUDA(cudaMemcpyAsync(host_out[k], Zc, (size_t)nc * 16, cudaMemcpyDeviceToHost, s));
    OSMPS_CUDA(cudaStreamSynchronize(s));
  }
  for (int64_t k = 0; k <= L; ++k) chi_out[k] = chi[k];
  acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = acc;
  return OSMPS_OK;
}
