// Operand preparation and MPO contraction steps.
//
// * split_operand: float64/float32 -> [hi | lo] rows in bf16 or tf32 for the
//   tensor-core GEMM (x = hi + lo + O(2^-17 |x|) for bf16, O(2^-22 |x|) for tf32).
//   Rows are written K-major; a source whose K index is not contiguous is read
//   through a 32 x 32 shared-memory transpose so both sides stay coalesced.
// * fiber contractions: the W-steps of Sec. 3.4, where the MPO tensors
//   M^[k] (few entries, Eq. MPOdef) act on the small (w, s) index pair of an
//   intermediate, for every (outer, inner) fiber. These are bandwidth-bound:
//   one coalesced pass over the input and the output.
#include <cuda_bf16.h>

#include "common.cuh"

namespace osmps {

namespace {

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

template <int KIND>
__device__ __forceinline__ void split_store(void* dst, int64_t off_hi, int64_t Kp, double x) {
  if (KIND == TC_BF16) {
    __nv_bfloat16 h = __double2bfloat16(x);
    __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi] = h;
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi + Kp] = l;
  } else {
    uint32_t h = to_tf32((float)x);
    uint32_t l = to_tf32((float)(x - (double)__uint_as_float(h)));
    reinterpret_cast<uint32_t*>(dst)[off_hi] = h;
    reinterpret_cast<uint32_t*>(dst)[off_hi + Kp] = l;
  }
}

// The same split for a float32 value with float32 arithmetic only (the
// float64 pipe is narrow on this GPU). x - hi is exact in float32 (hi keeps
// the leading bits of x), so the result equals split_store's bit for bit.
template <int KIND>
__device__ __forceinline__ void split_store_f32(void* dst, int64_t off_hi, int64_t Kp, float x) {
  if (KIND == TC_BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi] = h;
    reinterpret_cast<__nv_bfloat16*>(dst)[off_hi + Kp] = l;
  } else {
    const uint32_t h = to_tf32(x);
    const uint32_t l = to_tf32(x - __uint_as_float(h));
    reinterpret_cast<uint32_t*>(dst)[off_hi] = h;
    reinterpret_cast<uint32_t*>(dst)[off_hi + Kp] = l;
  }
}

// Two consecutive values (off_hi even, so the pair is 4- or 8-byte aligned).
template <int KIND>
__device__ __forceinline__ void split_store2_f32(void* dst, int64_t off_hi, int64_t Kp, float a, float b) {
  if (KIND == TC_BF16) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    __nv_bfloat162 h2, l2;
    h2.x = ha; h2.y = hb;
    l2.x = la; l2.y = lb;
    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(dst) + off_hi) = h2;
    *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(dst) + off_hi + Kp) = l2;
  } else {
    const uint32_t ha = to_tf32(a), hb = to_tf32(b);
    const uint32_t la = to_tf32(a - __uint_as_float(ha)), lb = to_tf32(b - __uint_as_float(hb));
    *reinterpret_cast<uint2*>(reinterpret_cast<uint32_t*>(dst) + off_hi) = make_uint2(ha, hb);
    *reinterpret_cast<uint2*>(reinterpret_cast<uint32_t*>(dst) + off_hi + Kp) = make_uint2(la, lb);
  }
}

__device__ __forceinline__ double load_src(const void* src, bool f32, int64_t off) {
  return f32 ? (double)reinterpret_cast<const float*>(src)[off]
             : reinterpret_cast<const double*>(src)[off];
}

// K contiguous in the source: thread per (row, k), k fastest.
template <int KIND>
__global__ void k_split_direct(SplitView v, void* __restrict__ dst, int64_t Kp) {
  const int64_t total = v.rows * Kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kp, k = e - r * Kp;
    double x = 0.0;
    if (k < v.K) {
      const int64_t r0 = r / v.n1, r1 = r - r0 * v.n1;
      x = load_src(v.src, v.src_f32, r0 * v.s0 + r1 * v.s1 + k * v.sk);
    }
    split_store<KIND>(dst, r * 2 * Kp + k, Kp, x);
  }
}

// K strided in the source: 32x32 tiles transposed through shared memory.
template <int KIND>
__global__ void k_split_transpose(SplitView v, void* __restrict__ dst, int64_t Kp) {
  __shared__ double tile[32][33];
  const int64_t r_base = (int64_t)blockIdx.x * 32;
  const int64_t k_base = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int64_t k = k_base + j, r = r_base + tx;  // rows fastest while reading
    double x = 0.0;
    if (k < v.K && r < v.rows) {
      const int64_t r0 = r / v.n1, r1 = r - r0 * v.n1;
      x = load_src(v.src, v.src_f32, r0 * v.s0 + r1 * v.s1 + k * v.sk);
    }
    tile[j][tx] = x;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r_base + j, k = k_base + tx;  // k fastest while writing
    if (r < v.rows && k < Kp) split_store<KIND>(dst, r * 2 * Kp + k, Kp, tile[tx][j]);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = cdiv(n, threads);
  if (b < 1) b = 1;
  if (b > 65536) b = 65536;
  return (int)b;
}

template <typename T, int QMAX, int MODE>  // MODE 0: plain output, 1/2: split bf16/tf32
__global__ void k_fiber(Fiber f, const double* __restrict__ Mat, const T* __restrict__ in,
                        T* __restrict__ out, void* __restrict__ sdst, int64_t Kcols, int64_t Kp) {
  extern __shared__ uint8_t fsm[];
  T* Ms = reinterpret_cast<T*>(fsm);
  const int P = (int)f.P, Q = (int)f.Q;
  for (int i = threadIdx.x; i < P * Q; i += blockDim.x) Ms[i] = (T)Mat[i];
  __syncthreads();
  const int64_t total = f.n_o1 * f.n_o2 * f.nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % f.nc;
    const int64_t o12 = e / f.nc;
    const int64_t o2 = o12 % f.n_o2, o1 = o12 / f.n_o2;
    const T* src = in + o1 * f.is1 + o2 * f.is2 + c;
    T acc[QMAX];
#pragma unroll
    for (int o = 0; o < QMAX; ++o) acc[o] = (T)0;
    for (int i = 0; i < P; ++i) {
      const T x = src[(int64_t)i * f.istride];
      const T* mrow = Ms + i * Q;
#pragma unroll
      for (int o = 0; o < QMAX; ++o)
        if (o < Q) acc[o] = fma(mrow[o], x, acc[o]);
    }
    const int64_t ob = o1 * f.os1 + o2 * f.os2 + c;
#pragma unroll
    for (int o = 0; o < QMAX; ++o) {
      if (o < Q) {
        const int64_t off = ob + (int64_t)o * f.ostride;
        if (MODE == 0) {
          out[off] = acc[o];
        } else {
          const int64_t row = off / Kcols, col = off - row * Kcols;
          split_store_f32<MODE == 1 ? TC_BF16 : TC_TF32>(sdst, row * 2 * Kp + col, Kp, (float)acc[o]);
        }
      }
    }
  }
}

template <typename T, int MODE>
osmps_status fiber_dispatch(const Fiber& f, const double* Mat, const T* in, T* out, void* sdst,
                            int64_t Kcols, int64_t Kp, cudaStream_t s) {
  if (f.P <= 0 || f.Q <= 0 || f.nc <= 0 || f.n_o1 <= 0 || f.n_o2 <= 0) return OSMPS_OK;
  const size_t sm = (size_t)f.P * f.Q * sizeof(T);
  if (sm > 96 * 1024)
    return set_error(OSMPS_EUNSUPPORTED, "W-step: MPO block %lld x %lld too large",
                     (long long)f.P, (long long)f.Q);
  const int64_t total = f.n_o1 * f.n_o2 * f.nc;
  const int threads = 256;
  const int blocks = grid_for(total, threads);
  if (f.Q <= 8) {
    auto k = k_fiber<T, 8, MODE>;
    if (sm > 48 * 1024) OSMPS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { k<<<blocks, threads, sm, s>>>(f, Mat, in, out, sdst, Kcols, Kp); note_launch(); }
  } else if (f.Q <= 16) {
    auto k = k_fiber<T, 16, MODE>;
    if (sm > 48 * 1024) OSMPS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { k<<<blocks, threads, sm, s>>>(f, Mat, in, out, sdst, Kcols, Kp); note_launch(); }
  } else if (f.Q <= 32) {
    auto k = k_fiber<T, 32, MODE>;
    if (sm > 48 * 1024) OSMPS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { k<<<blocks, threads, sm, s>>>(f, Mat, in, out, sdst, Kcols, Kp); note_launch(); }
  } else if (f.Q <= 64) {
    auto k = k_fiber<T, 64, MODE>;
    if (sm > 48 * 1024) OSMPS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    { k<<<blocks, threads, sm, s>>>(f, Mat, in, out, sdst, Kcols, Kp); note_launch(); }
  } else {
    return set_error(OSMPS_EUNSUPPORTED, "W-step: output block %lld > 64", (long long)f.Q);
  }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

template <int KIND>
__global__ void k_zero_pad(void* dst, int64_t rows, int64_t Kcols, int64_t Kp) {
  const int64_t w = Kp - Kcols;
  const int64_t total = rows * w;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / w, k = Kcols + (e - r * w);
    split_store_f32<KIND>(dst, r * 2 * Kp + k, Kp, 0.0f);
  }
}

__global__ void k_w_reorder(const double* __restrict__ W, int64_t dw, int64_t d, int64_t dw2,
                            int order, double* __restrict__ Mat) {
  const int64_t total = dw * d * d * dw2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    // e enumerates W[w, t, s, w2] in row-major order
    int64_t w2 = e % dw2, r = e / dw2;
    int64_t s = r % d;
    r /= d;
    int64_t t = r % d, w = r / d;
    int64_t i, o, Q;
    if (order == WORD_IN_W_S__OUT_T_W2) {
      i = w * d + s;
      o = t * dw2 + w2;
      Q = d * dw2;
    } else if (order == WORD_IN_T_W2__OUT_W_S) {
      i = t * dw2 + w2;
      o = w * d + s;
      Q = dw * d;
    } else {
      i = s * dw2 + w2;
      o = w * d + t;
      Q = dw * d;
    }
    Mat[i * Q + o] = W[e];
  }
}

// Both W-steps of H_eff.theta in one pass, for the spin-1/2 chains (d = 2)
// whose MPO bond dimensions are fixed at compile time: for every fiber
// (a2, c) the wl*d*d values T1[a2, w, s1, s2, c] are contracted with W1 and
// then W2 in registers and written straight into the split operand
// T3[(a2, t1, t2), (w2, c)]; the intermediate T2 never touches memory.
// Identity environment channels (skip_l, skip_r >= 0): L[:, skip_l, :] = 1,
// so T1's channel skip_l is theta itself and the stage-1 GEMM leaves it out
// (T1 holds the other WL - 1 channels in order); R[:, skip_r, :] = 1, so
// output channel skip_r needs no stage-4 GEMM: it goes as float32 to yid
// (row (a2, t1, t2), column c2), which the stage-4 epilogue adds, and the
// split operand holds the other WR - 1 channels in order.
// SL, SR: the identity channels fixed at compile time (-1: none), or
// SKIP_RUNTIME to take skip_l / skip_r from the arguments. Compile-time
// values let the channel loops fold: with runtime tests in the load loop the
// kernel measured 58 instead of 38 us at chi = 1024.
constexpr int SKIP_RUNTIME = -2;
template <int D, int WL, int WM, int WR, int KIND, int V, int SL, int SR>
__global__ void __launch_bounds__(256, 2) k_fused_wsteps(const float* __restrict__ T1,
                                                         const double* __restrict__ Mat1,
                                                         const double* __restrict__ Mat2,
                                                         void* __restrict__ dst, int64_t chi_l,
                                                         int64_t chi_r, int64_t Kp,
                                                         const double* __restrict__ theta,
                                                         int skip_l_arg, int skip_r_arg,
                                                         float* __restrict__ yid) {
  const int skip_l = SL == SKIP_RUNTIME ? skip_l_arg : SL;
  const int skip_r = SR == SKIP_RUNTIME ? skip_r_arg : SR;
  constexpr int P1 = WL * D, Q1 = D * WM, P2 = WM * D, Q2 = D * WR;
  static_assert(P1 <= 32 && P2 <= 32, "input masks are 32-bit");
  __shared__ float sm1[P1 * Q1], sm2[P2 * Q2];
  __shared__ unsigned nz1[Q1], nz2[Q2];  // per output: which inputs have a nonzero W entry
  for (int i = threadIdx.x; i < P1 * Q1; i += blockDim.x) sm1[i] = (float)Mat1[i];
  for (int i = threadIdx.x; i < P2 * Q2; i += blockDim.x) sm2[i] = (float)Mat2[i];
  if (threadIdx.x < Q1) nz1[threadIdx.x] = 0u;
  if (threadIdx.x < Q2) nz2[threadIdx.x] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < P1 * Q1; i += blockDim.x)
    if (sm1[i] != 0.0f) atomicOr(&nz1[i % Q1], 1u << (i / Q1));
  for (int i = threadIdx.x; i < P2 * Q2; i += blockDim.x)
    if (sm2[i] != 0.0f) atomicOr(&nz2[i % Q2], 1u << (i / Q2));
  __syncthreads();
  // MPO tensors are mostly zeros (an identity in two corners and a few local
  // operators): every multiply-add is guarded by the output's nonzero mask,
  // a branch that is uniform over the grid, and the W entry is read from
  // shared memory only where it is nonzero (kept in registers the ~200
  // entries would leave one block per SM, too few loads in flight for HBM)
  const volatile float* m1 = sm1;
  const volatile float* m2 = sm2;
  // V consecutive fibers c per thread (V = 2: 8-byte loads, paired stores;
  // chi_r even)
  const int64_t cv = chi_r / V;
  const int64_t total = chi_l * cv;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a2 = e / cv, c = (e - a2 * cv) * V;
    const int wlt = skip_l >= 0 ? WL - 1 : WL;  // channels held in T1
    const float* src = T1 + a2 * (wlt * D * D) * chi_r + c;
    float x[WL][D][D][V];
#pragma unroll
    for (int w = 0; w < WL; ++w)
#pragma unroll
      for (int s1 = 0; s1 < D; ++s1)
#pragma unroll
        for (int s2 = 0; s2 < D; ++s2) {
          if (w == skip_l) {  // uniform branch: the identity channel is theta
            const double* q = theta + ((a2 * D + s1) * D + s2) * chi_r + c;
            if (V == 2) {
              const double2 f = *reinterpret_cast<const double2*>(q);
              x[w][s1][s2][0] = (float)f.x;
              x[w][s1][s2][V - 1] = (float)f.y;
            } else {
              x[w][s1][s2][0] = (float)q[0];
            }
            continue;
          }
          const int wt = (skip_l >= 0 && w > skip_l) ? w - 1 : w;
          const float* p = src + ((wt * D + s1) * D + s2) * chi_r;
          if (V == 2) {
            const float2 f = *reinterpret_cast<const float2*>(p);
            x[w][s1][s2][0] = f.x;
            x[w][s1][s2][V - 1] = f.y;
          } else {
            x[w][s1][s2][0] = p[0];
          }
        }
    float mid[D][WM][D][V];  // T2[t1, w1, s2]
#pragma unroll
    for (int t1 = 0; t1 < D; ++t1)
#pragma unroll
      for (int w1 = 0; w1 < WM; ++w1) {
        const unsigned mask = nz1[t1 * WM + w1];
        float acc[D][V];
#pragma unroll
        for (int s2 = 0; s2 < D; ++s2)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[s2][v] = 0.0f;
#pragma unroll
        for (int w = 0; w < WL; ++w)
#pragma unroll
          for (int s1 = 0; s1 < D; ++s1)
            if (mask & (1u << (w * D + s1))) {
              const float m = m1[(w * D + s1) * Q1 + t1 * WM + w1];
#pragma unroll
              for (int s2 = 0; s2 < D; ++s2)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[s2][v] = fmaf(m, x[w][s1][s2][v], acc[s2][v]);
            }
#pragma unroll
        for (int s2 = 0; s2 < D; ++s2)
#pragma unroll
          for (int v = 0; v < V; ++v) mid[t1][w1][s2][v] = acc[s2][v];
      }
#pragma unroll
    for (int t2 = 0; t2 < D; ++t2)
#pragma unroll
      for (int w2 = 0; w2 < WR; ++w2) {
        const unsigned mask = nz2[t2 * WR + w2];
        float acc[D][V];
#pragma unroll
        for (int t1 = 0; t1 < D; ++t1)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[t1][v] = 0.0f;
#pragma unroll
        for (int w1 = 0; w1 < WM; ++w1)
#pragma unroll
          for (int s2 = 0; s2 < D; ++s2)
            if (mask & (1u << (w1 * D + s2))) {
              const float m = m2[(w1 * D + s2) * Q2 + t2 * WR + w2];
#pragma unroll
              for (int t1 = 0; t1 < D; ++t1)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[t1][v] = fmaf(m, mid[t1][w1][s2][v], acc[t1][v]);
            }
#pragma unroll
        for (int t1 = 0; t1 < D; ++t1) {
          const int64_t row = (a2 * D + t1) * D + t2;
          if (w2 == skip_r) {
            float* q = yid + row * chi_r + c;
            if (V == 2) *reinterpret_cast<float2*>(q) = make_float2(acc[t1][0], acc[t1][V - 1]);
            else q[0] = acc[t1][0];
            continue;
          }
          const int w2t = (skip_r >= 0 && w2 > skip_r) ? w2 - 1 : w2;
          const int64_t off = row * 2 * Kp + (int64_t)w2t * chi_r + c;
          if (V == 2) split_store2_f32<KIND>(dst, off, Kp, acc[t1][0], acc[t1][V - 1]);
          else split_store_f32<KIND>(dst, off, Kp, acc[t1][0]);
        }
      }
  }
}

template <int D, int WL, int WM, int WR>
bool try_fused(int64_t d, int64_t wl, int64_t wm, int64_t wr, int kind, const float* T1,
               const double* m1, const double* m2, void* dst, int64_t chi_l, int64_t chi_r,
               int64_t Kp, const WStepIdentity& id, cudaStream_t s, bool launch) {
  if (d != D || wl != WL || wm != WM || wr != WR) return false;
  if (!launch) return true;  // shape query only
  const double* th = id.theta;
  const int sl = id.skip_l, sr = id.skip_r;
  float* yid = id.yid;
  // two resident blocks per SM, each striding over many fibers (the
  // per-block set-up of the W tables is then paid a few hundred times only)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 152;
  // pairs of fibers: 8-byte loads of T1, 16-byte loads of theta (identity
  // channel) and paired stores, so chi_r even and theta 16-byte aligned
  const bool pair = chi_r % 2 == 0 && (sl < 0 || (reinterpret_cast<uintptr_t>(th) & 15) == 0);
  const int blocks = (int)std::min<int64_t>(grid_for(chi_l * (pair ? chi_r / 2 : chi_r), 256), 2 * (int64_t)sms);
  // compile-time identity channels for the cases a sweep meets (none; L's
  // last and/or R's first channel), the runtime form for the rest
  const int combo = (sl == -1 && sr == -1) ? 0 : (sl == WL - 1 && sr == 0) ? 1
                  : (sl == WL - 1 && sr == -1) ? 2 : (sl == -1 && sr == 0) ? 3 : 4;
#define OSMPS_FUSED(K, V, L_, R_) \
  k_fused_wsteps<D, WL, WM, WR, K, V, L_, R_><<<blocks, 256, 0, s>>>(T1, m1, m2, dst, chi_l, chi_r, Kp, th, sl, sr, yid)
#define OSMPS_FUSED_KIND(K)                                                   \
  if (!pair) OSMPS_FUSED(K, 1, SKIP_RUNTIME, SKIP_RUNTIME);                    \
  else if (combo == 0) OSMPS_FUSED(K, 2, -1, -1);                             \
  else if (combo == 1) OSMPS_FUSED(K, 2, WL - 1, 0);                          \
  else if (combo == 2) OSMPS_FUSED(K, 2, WL - 1, -1);                         \
  else if (combo == 3) OSMPS_FUSED(K, 2, -1, 0);                              \
  else OSMPS_FUSED(K, 2, SKIP_RUNTIME, SKIP_RUNTIME);
  if (kind == TC_BF16) {
    OSMPS_FUSED_KIND(TC_BF16)
  } else {
    OSMPS_FUSED_KIND(TC_TF32)
  }
#undef OSMPS_FUSED_KIND
#undef OSMPS_FUSED
  note_launch();
  return true;
}

}  // namespace

osmps_status split_operand(const SplitView& v, int kind, void* dst, int64_t Kp, cudaStream_t s) {
  if (v.rows <= 0) return OSMPS_OK;
  if (Kp < v.K || Kp % 64 != 0) return set_error(OSMPS_ESHAPE, "split_operand: bad Kp");
  if (v.sk == 1 || v.K == 1) {
    const int blocks = grid_for(v.rows * Kp, 256);
    if (kind == TC_BF16) { k_split_direct<TC_BF16><<<blocks, 256, 0, s>>>(v, dst, Kp); note_launch(); }
    else { k_split_direct<TC_TF32><<<blocks, 256, 0, s>>>(v, dst, Kp); note_launch(); }
  } else {
    if (cdiv(Kp, 32) > 65535) return set_error(OSMPS_ESHAPE, "split_operand: K too large");
    dim3 grid((unsigned)cdiv(v.rows, 32), (unsigned)cdiv(Kp, 32));
    dim3 block(32, 8);
    if (kind == TC_BF16) { k_split_transpose<TC_BF16><<<grid, block, 0, s>>>(v, dst, Kp); note_launch(); }
    else { k_split_transpose<TC_TF32><<<grid, block, 0, s>>>(v, dst, Kp); note_launch(); }
  }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

osmps_status fiber_contract_f64(const Fiber& f, const double* Mat, const double* in, double* out,
                                cudaStream_t s) {
  return fiber_dispatch<double, 0>(f, Mat, in, out, nullptr, 1, 0, s);
}

osmps_status fiber_contract_f32(const Fiber& f, const double* Mat, const float* in, float* out,
                                cudaStream_t s) {
  return fiber_dispatch<float, 0>(f, Mat, in, out, nullptr, 1, 0, s);
}

osmps_status fiber_contract_f32_split(const Fiber& f, const double* Mat, const float* in,
                                      void* dst, int kind, int64_t Kcols, int64_t Kp,
                                      cudaStream_t s) {
  if (kind == TC_BF16) return fiber_dispatch<float, 1>(f, Mat, in, nullptr, dst, Kcols, Kp, s);
  return fiber_dispatch<float, 2>(f, Mat, in, nullptr, dst, Kcols, Kp, s);
}

// max over (a, b) of |E[a, w, b] - delta_ab| for w = 0 (blockIdx.y = 0) and
// w = w_count - 1 (blockIdx.y = 1), as the bit patterns of non-negative
// doubles (ordered like the values) combined by atomicMax
__global__ void k_identity_deviation(const double* __restrict__ E, int64_t chi, int64_t w_count,
                                     unsigned long long* __restrict__ out) {
  const int64_t w = blockIdx.y == 0 ? 0 : w_count - 1;
  const int64_t total = chi * chi;
  double m = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / chi, b = e - a * chi;
    const double v = E[(a * w_count + w) * chi + b] - (a == b ? 1.0 : 0.0);
    const double av = fabs(v);
    m = (av > m || av != av) ? (av != av ? INFINITY : av) : m;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&out[blockIdx.y], (unsigned long long)__double_as_longlong(m));
}

static bool fused_dispatch(int64_t d1, int64_t d2, int64_t wl, int64_t wm, int64_t wr, int kind,
                           const float* T1, const double* Mat1, const double* Mat2, void* dst,
                           int64_t chi_l, int64_t chi_r, int64_t Kp, const WStepIdentity& id,
                           cudaStream_t s, bool launch) {
  if (d1 != d2) return false;
  const int64_t d = d1;
#define OSMPS_TRY_FUSED(a, b, c, e) \
  try_fused<a, b, c, e>(d, wl, wm, wr, kind, T1, Mat1, Mat2, dst, chi_l, chi_r, Kp, id, s, launch)
  return OSMPS_TRY_FUSED(2, 5, 5, 5) || OSMPS_TRY_FUSED(2, 1, 5, 5) || OSMPS_TRY_FUSED(2, 5, 5, 1) ||
         OSMPS_TRY_FUSED(2, 3, 3, 3) || OSMPS_TRY_FUSED(2, 1, 3, 3) || OSMPS_TRY_FUSED(2, 3, 3, 1);
#undef OSMPS_TRY_FUSED
}

osmps_status identity_channel_deviation(const double* E, int64_t chi, int64_t w_count,
                                        double* dev_out, cudaStream_t s) {
  OSMPS_CUDA(cudaMemsetAsync(dev_out, 0, 2 * sizeof(double), s));
  if (chi <= 0 || w_count <= 0) return OSMPS_OK;
  const int bx = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(chi * chi, 256 * 8), 1024));
  k_identity_deviation<<<dim3(bx, 2), 256, 0, s>>>(E, chi, w_count,
                                                  reinterpret_cast<unsigned long long*>(dev_out));
  note_launch();
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

bool fused_wsteps_supported(int64_t d1, int64_t d2, int64_t wl, int64_t wm, int64_t wr) {
  return fused_dispatch(d1, d2, wl, wm, wr, TC_BF16, nullptr, nullptr, nullptr, nullptr, 0, 0, 0,
                        WStepIdentity{}, nullptr, false);
}

osmps_status fused_wsteps_f32_split(const float* T1, const double* Mat1, const double* Mat2,
                                    void* dst, int kind, int64_t chi_l, int64_t d1, int64_t d2,
                                    int64_t chi_r, int64_t wl, int64_t wm, int64_t wr, int64_t Kp,
                                    const WStepIdentity& id, cudaStream_t s, bool* done) {
  *done = false;
  if ((id.skip_l >= 0 && !id.theta) || (id.skip_r >= 0 && !id.yid))
    return set_error(OSMPS_EINVAL, "fused W-steps: identity channel without its buffer");
  if (!fused_dispatch(d1, d2, wl, wm, wr, kind, T1, Mat1, Mat2, dst, chi_l, chi_r, Kp, id, s, true))
    return OSMPS_OK;
  OSMPS_LAUNCH_CHECK();
  *done = true;
  return OSMPS_OK;
}

osmps_status zero_pad_columns(void* dst, int kind, int64_t rows, int64_t Kcols, int64_t Kp,
                              cudaStream_t s) {
  if (Kp <= Kcols || rows <= 0) return OSMPS_OK;
  const int blocks = grid_for(rows * (Kp - Kcols), 256);
  if (kind == TC_BF16) { k_zero_pad<TC_BF16><<<blocks, 256, 0, s>>>(dst, rows, Kcols, Kp); note_launch(); }
  else { k_zero_pad<TC_TF32><<<blocks, 256, 0, s>>>(dst, rows, Kcols, Kp); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

osmps_status w_reorder(const double* W, int64_t dw, int64_t d, int64_t dw2, int order, double* Mat,
                       cudaStream_t s) {
  const int64_t total = dw * d * d * dw2;
  { k_w_reorder<<<grid_for(total, 256), 256, 0, s>>>(W, dw, d, dw2, order, Mat); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

}  // namespace osmps
