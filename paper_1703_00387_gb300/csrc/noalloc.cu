// H_eff . theta without any device allocation.
//
// Same float64 product as osmps_heff_apply(..., OSMPS_PREC_FP64, ...), but the
// intermediates live in a fixed array compiled into the library instead of
// a context workspace, so the call needs no osmps_ctx and never calls
// cudaMalloc/cudaFree. The array costs NOALLOC_SCRATCH_BYTES of device memory
// on every GPU where the library is used, held until the process exits.
#include <initializer_list>
#include <mutex>

#include "common.cuh"

namespace osmps {

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_heff_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_heff_scratch per device. In host code the symbol name
// is only a host-side stand-in, so the address is looked up once per device
// with that device current.
void* g_scratch_addr[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

osmps_status scratch_address(void** out) {
  int dev = 0;
  OSMPS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES)
    return set_error(OSMPS_EUNSUPPORTED, "heff_apply_noalloc: device %d beyond %d", dev, MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_heff_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return set_error(OSMPS_ECUDA, "heff_apply_noalloc: cudaGetSymbolAddress failed on device %d: %s",
                       dev, cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return OSMPS_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bytes of a float64 array with the given extents, 256-byte aligned, or
// false when the product overflows or alone exceeds the fixed scratch (each
// factor is at most 2^31, so a product of five or six of them can wrap).
bool region_bytes(std::initializer_list<int64_t> dims, size_t* out) {
  uint64_t b = 8;
  for (int64_t x : dims) {
    uint64_t r = 0;
    if (__builtin_mul_overflow(b, (uint64_t)x, &r) || r > NOALLOC_SCRATCH_BYTES) return false;
    b = r;
  }
  *out = align256((size_t)b);
  return true;
}

}  // namespace

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_heff_apply_noalloc(const double* L, const double* W1,
                                                 const double* W2, const double* R,
                                                 const double* theta, double* y, int64_t chi_l,
                                                 int64_t d1, int64_t d2, int64_t chi_r, int64_t wl,
                                                 int64_t wm, int64_t wr, void* stream) {
  clear_error();
  if (!L || !W1 || !W2 || !R || !theta || !y)
    return set_error(OSMPS_EINVAL, "osmps_heff_apply_noalloc: null argument");
  if ((const void*)y == (const void*)theta)
    return set_error(OSMPS_EINVAL, "osmps_heff_apply_noalloc: y aliases theta");
  for (int64_t x : {chi_l, d1, d2, chi_r, wl, wm, wr})
    if (x <= 0 || x > ((int64_t)1 << 31))
      return set_error(OSMPS_ESHAPE, "osmps_heff_apply_noalloc: non-positive or oversized dimension");
  size_t b_mat1 = 0, b_mat2 = 0, b_t1 = 0, b_t2 = 0, b_t3 = 0;
  const bool fits = region_bytes({wl, d1, d1, wm}, &b_mat1) && region_bytes({wm, d2, d2, wr}, &b_mat2) &&
                    region_bytes({chi_l, wl, d1, d2, chi_r}, &b_t1) &&
                    region_bytes({chi_l, d1, wm, d2, chi_r}, &b_t2) &&
                    region_bytes({chi_l, d1, d2, wr, chi_r}, &b_t3);
  if (!fits)
    return set_error(OSMPS_ESHAPE,
                     "osmps_heff_apply_noalloc: an intermediate of these dimensions alone exceeds "
                     "the fixed scratch of %zu bytes (use osmps_heff_apply with a context instead)",
                     NOALLOC_SCRATCH_BYTES);
  const int64_t N1 = d1 * d2 * chi_r;
  const int64_t P1 = wl * d1, Q1 = d1 * wm, P2 = wm * d2, Q2 = d2 * wr;
  const size_t need = b_mat1 + b_mat2 + b_t1 + b_t2 + b_t3;  // each term <= 32 MiB + 255
  if (need > NOALLOC_SCRATCH_BYTES)
    return set_error(OSMPS_ESHAPE,
                     "osmps_heff_apply_noalloc: these dimensions need %zu bytes of scratch; the "
                     "fixed scratch holds %zu (use osmps_heff_apply with a context instead)",
                     need, NOALLOC_SCRATCH_BYTES);
  void* base = nullptr;
  OSMPS_TRY(scratch_address(&base));
  unsigned char* p = static_cast<unsigned char*>(base);
  double* mat1 = reinterpret_cast<double*>(p);
  double* mat2 = reinterpret_cast<double*>(p + b_mat1);
  double* T1 = reinterpret_cast<double*>(p + b_mat1 + b_mat2);
  double* T2 = reinterpret_cast<double*>(p + b_mat1 + b_mat2 + b_t1);
  double* T3 = reinterpret_cast<double*>(p + b_mat1 + b_mat2 + b_t1 + b_t2);
  cudaStream_t s = (cudaStream_t)stream;

  // Every scratch region below is fully written before it is read, so the
  // previous call's contents never leak into this one.
  OSMPS_TRY(w_reorder(W1, wl, d1, wm, WORD_IN_W_S__OUT_T_W2, mat1, s));
  OSMPS_TRY(w_reorder(W2, wm, d2, wr, WORD_IN_W_S__OUT_T_W2, mat2, s));
  GemmF64 g1;  // T1[(a2,w),(s1,s2,c)] = L[(a2,w),a] theta[a,(s1,s2,c)]
  g1.M = chi_l * wl; g1.N = N1; g1.K = chi_l;
  g1.A = L; g1.sam = chi_l; g1.sak = 1;
  g1.B = theta; g1.sbk = N1; g1.sbn = 1;
  g1.C = T1; g1.scm = N1; g1.scn = 1;
  OSMPS_TRY(gemm_f64(g1, s));
  Fiber f2;  // W1 step
  f2.P = P1; f2.Q = Q1; f2.n_o1 = chi_l; f2.n_o2 = d2; f2.nc = chi_r;
  f2.is1 = wl * d1 * d2 * chi_r; f2.is2 = chi_r; f2.istride = d2 * chi_r;
  f2.os1 = d1 * wm * d2 * chi_r; f2.os2 = chi_r; f2.ostride = d2 * chi_r;
  OSMPS_TRY(fiber_contract_f64(f2, mat1, T1, T2, s));
  Fiber f3;  // W2 step
  f3.P = P2; f3.Q = Q2; f3.n_o1 = chi_l * d1; f3.n_o2 = 1; f3.nc = chi_r;
  f3.is1 = wm * d2 * chi_r; f3.istride = chi_r; f3.os1 = d2 * wr * chi_r; f3.ostride = chi_r;
  OSMPS_TRY(fiber_contract_f64(f3, mat2, T2, T3, s));
  GemmF64 g4;  // y[(a2,t1,t2),c2] = T3[(a2,t1,t2),(w2,c)] R[c2,(w2,c)]
  g4.M = chi_l * d1 * d2; g4.N = chi_r; g4.K = wr * chi_r;
  g4.A = T3; g4.sam = wr * chi_r; g4.sak = 1;
  g4.B = R; g4.sbk = 1; g4.sbn = wr * chi_r;
  g4.C = y; g4.scm = chi_r; g4.scn = 1;
  return gemm_f64(g4, s);
}
