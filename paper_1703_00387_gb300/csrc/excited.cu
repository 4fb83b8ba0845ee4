// Building blocks of the excited-state search (Sec. 4.1, eMPS, Eq.
// emps_lagrange): the overlap <psi|phi> of the state being optimised with a
// lower eigenstate, carried as left and right overlap environments, and the
// lower state's two-site block seen in the current basis, which the local
// Lanczos must stay orthogonal to. All products are float64 DMMA GEMMs.
#include "common.cuh"

namespace osmps {
namespace {

osmps_status gemm_rm(double* C, const double* A, const double* B, int64_t M, int64_t N, int64_t K,
                     int64_t sam, int64_t sak, int64_t sbk, int64_t sbn, cudaStream_t s) {
  GemmF64 g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.sam = sam; g.sak = sak;
  g.B = B; g.sbk = sbk; g.sbn = sbn;
  g.C = C; g.scm = N; g.scn = 1;
  return gemm_f64(g, s);
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" {

osmps_status osmps_overlap_env_update(osmps_ctx* ctx, int side, const double* env_in,
                                      const double* A, const double* Bk, double* env_out,
                                      int64_t chi_l, int64_t d, int64_t chi_r, int64_t chik_l,
                                      int64_t chik_r, void* stream) {
  clear_error();
  if (!ctx || !env_in || !A || !Bk || !env_out)
    return set_error(OSMPS_EINVAL, "osmps_overlap_env_update: null argument");
  if (side != 0 && side != 1) return set_error(OSMPS_EINVAL, "osmps_overlap_env_update: side %d", side);
  for (int64_t x : {chi_l, d, chi_r, chik_l, chik_r})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_overlap_env_update: bad dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  if (side == 0) {
    // X[a2, (t, bk)] = sum_ak O[a2, ak] Bk[ak, (t, bk)];  O'[b2, bk] = sum_(a2, t) A[(a2, t), b2] X[(a2, t), bk]
    double* X = (double*)ws_get(ctx, SLOT_OV_X, (size_t)chi_l * d * chik_r * 8, s, &st);
    if (!X) return st;
    OSMPS_TRY(gemm_rm(X, env_in, Bk, chi_l, d * chik_r, chik_l, chik_l, 1, d * chik_r, 1, s));
    return gemm_rm(env_out, A, X, chi_r, chik_r, chi_l * d, 1, chi_r, chik_r, 1, s);
  }
  // X[(ak, t), b2] = sum_bk Bk[(ak, t), bk] O[b2, bk];  O'[a2, ak] = sum_(t, b2) A[a2, (t, b2)] X[ak, (t, b2)]
  double* X = (double*)ws_get(ctx, SLOT_OV_X, (size_t)chik_l * d * chi_r * 8, s, &st);
  if (!X) return st;
  OSMPS_TRY(gemm_rm(X, Bk, env_in, chik_l * d, chi_r, chik_r, chik_r, 1, 1, chik_r, s));
  return gemm_rm(env_out, A, X, chi_l, chik_l, d * chi_r, d * chi_r, 1, 1, d * chi_r, s);
}

osmps_status osmps_projected_state(osmps_ctx* ctx, const double* OL, const double* B1,
                                   const double* B2, const double* OR, double* v, int64_t chi_l,
                                   int64_t d1, int64_t d2, int64_t chi_r, int64_t chik_l,
                                   int64_t chik_m, int64_t chik_r, void* stream) {
  clear_error();
  if (!ctx || !OL || !B1 || !B2 || !OR || !v)
    return set_error(OSMPS_EINVAL, "osmps_projected_state: null argument");
  for (int64_t x : {chi_l, d1, d2, chi_r, chik_l, chik_m, chik_r})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_projected_state: bad dimension");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  osmps_status st = OSMPS_OK;
  const size_t nth = (size_t)chik_l * d1 * d2 * chik_r, ny = (size_t)chik_l * d1 * d2 * chi_r;
  double* buf = (double*)ws_get(ctx, SLOT_OV_X, (nth + ny) * 8, s, &st);
  if (!buf) return st;
  double* thk = buf;
  double* Y = buf + nth;
  // theta_k = B1 B2;  Y[(ak, s1, s2), c] = sum_ck theta_k[(ak s1 s2), ck] OR[c, ck];
  // v[a, (s1 s2 c)] = sum_ak OL[a, ak] Y[ak, (s1 s2 c)]
  OSMPS_TRY(gemm_rm(thk, B1, B2, chik_l * d1, d2 * chik_r, chik_m, chik_m, 1, d2 * chik_r, 1, s));
  OSMPS_TRY(gemm_rm(Y, thk, OR, chik_l * d1 * d2, chi_r, chik_r, chik_r, 1, 1, chik_r, s));
  return gemm_rm(v, OL, Y, chi_l, d1 * d2 * chi_r, chik_l, chik_l, 1, d1 * d2 * chi_r, 1, s);
}

}  // extern "C"
