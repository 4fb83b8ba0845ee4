// Float64-accurate GEMM on the bf16 tensor cores (error-free slicing).
//
// GB300's float64 units are slow; its bf16 tensor cores are about a
// thousand times faster. A float64 GEMM is emulated on them exactly in the
// manner of Ozaki's error-free transformation of matrix products:
//   * every row of A (and of B, both K-major) is scaled by a power of two
//     2^-e so that its entries lie in (-1, 1), rounded to 56 fractional bits
//     and cut into S = 8 balanced base-128 digits q_p (|q_p| <= 128), so
//     x = 2^e sum_p q_p 2^(-7(p+1)); the slices hold the integers q_p, exact
//     in bf16 (all of this with integer arithmetic on the IEEE bits);
//   * a slice pair (i, j) gives integer products q_i q_j of at most 2^14,
//     so a run of 1024 of them sums to at most 2^24: exact in the float32
//     TMEM accumulator, integers being exact there up to 2^24 (tested with
//     every top digit at 128);
//   * the epilogue converts those exact integers and adds them per slice diagonal
//     i + j (same unit 2^(-7(i+j+2))), over the 36 pairs with i + j <= 7
//     (the dropped pairs are below 2^-56 of the row scales);
//   * pairs on one diagonal share the unit, so a TMEM partial sum runs over
//     up to 16 K blocks of 64 across the pairs of a diagonal (at K = 64 the
//     36 pairs take 8 epilogue rounds, not 36);
//   * the diagonals are combined exactly in int64, Horner fashion in steps
//     of 2^7, within groups of consecutive diagonals (two groups of four
//     while K <= 2^17, whose sums stay below 2^53); each group sum becomes
//     a float64 by integer operations on the IEEE bits, the row and column
//     scales 2^(e_A + e_B) folded into its exponent, and the group values
//     are added in float64 in a second TMEM region. One float64 addition per
//     output element and tile remains: GB300's float64 pipe is what limits
//     this kind of kernel otherwise. The result is stored, or subtracted
//     from C.
// The kernel reuses the persistent, warp-specialised structure of gemm_tc:
// 128 x 128 tiles, a 6-stage TMA ring, two 128-column TMEM buffers, 16
// epilogue warps each holding 32 float64 accumulators per row.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tcgen05.cuh"

namespace osmps {

namespace {

using namespace tc;

constexpr int SLICES = 8;
constexpr int SLICE_BITS = 7;
constexpr int EBM = 128, EBN = 128;
constexpr int ESTAGES = 6;
constexpr int E_A_STAGE = EBM * 128, E_B_STAGE = EBN * 128;
constexpr int E_STAGE = E_A_STAGE + E_B_STAGE;
constexpr int E_EPI_WARPS = 16;
constexpr int E_EPI_COLS = EBN / 4;
constexpr int E_THREADS = 64 + 32 * E_EPI_WARPS;
// 64-element K slices per exact partial sum: products are at most 2^14 (the
// pair of top digits, |d_0| <= 128), so 16 slices (1024 products) stay
// within 2^24. (Diagonals other than 0 could run 32 slices, their products
// being at most 2^13; measured slightly slower, the epilogue then drains in
// longer, fewer bursts.)
constexpr int E_CHUNK = 16;
constexpr uint32_t E_TMEM_COLS = 512;   // 2 x 128 accumulator columns, then the float64 sums
constexpr uint32_t E_ACC_COL0 = 256;    // float64 group sums: two 32-bit columns per tile column
constexpr size_t E_SMEM = (size_t)ESTAGES * E_STAGE + 1024 + 256;

struct PairList {
  int n;
  unsigned char a[64], b[64];
};

// x 2^k as a float64 for an integer |x| < 2^53, built from the IEEE-754 bit
// layout (sign, biased exponent, 52 fraction bits) with integer operations
// only; exact whenever the result is a normal number, else left to scalbn.
__device__ __forceinline__ double i64_ldexp(long long x, int k) {
  if (x == 0) return 0.0;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int e = 63 - __clzll((long long)a);  // a in [2^e, 2^(e+1)), e <= 52
  const int E = e + k + 1023;
  if (E <= 0 || E >= 2047) return scalbn((double)x, k);
  const unsigned long long frac = (a << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(((unsigned long long)(x < 0) << 63) |
                                          ((unsigned long long)E << 52) | frac));
}

// Tile t -> (m0, n0) in groups of E_GROUP_M tile rows, columns walked within
// a group: the tiles that run at the same time then share E_GROUP_M A row
// slabs and fewer B column slabs than a row-major walk, so more of the slice
// operands stay in L2 between the pairs' passes.
constexpr int E_GROUP_M = 8;
__device__ __forceinline__ void emu_tile(int tile, int tiles_m, int tiles_n, int& m0, int& n0) {
  const int per_group = E_GROUP_M * tiles_n;
  const int g = tile / per_group, first = g * E_GROUP_M;
  const int rows = min(tiles_m - first, E_GROUP_M);
  const int local = tile - g * per_group;
  m0 = (first + local % rows) * EBM;
  n0 = (local / rows) * EBN;
}

// Close a diagonal group of the epilogue: its sums H (the last diagonal `cur`
// at weight 1) become float64 with the scales folded in and are added to the
// float64 sums of the earlier groups kept in TMEM (acc_t); after the last
// group the total is stored to C (or subtracted from it). H is zeroed.
__device__ __forceinline__ void close_group(long long (&H)[E_EPI_COLS], int& groups, bool last,
                                            uint32_t acc_t, int cur, int ea,
                                            const int* __restrict__ eB, int64_t col0, int64_t N,
                                            int64_t row, int64_t M, double* __restrict__ C,
                                            int64_t ldc, int subtract) {
  const int k0 = -SLICE_BITS * (cur + 2) + ea;
#pragma unroll
  for (int h = 0; h < E_EPI_COLS / 8; ++h) {  // 8 values = 16 TMEM words at a time
    uint32_t w[16];
    if (groups > 0) tmem_ld16(acc_t + 16 * h, w);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = 8 * h + i;
      const int eb = (col0 + j < N) ? eB[col0 + j] : 0;
      double v = i64_ldexp(H[j], k0 + eb);
      if (groups > 0) v += __hiloint2double((int)w[2 * i + 1], (int)w[2 * i]);
      if (last) {
        if (row < M && col0 + j < N) {
          double* dst = C + row * ldc + col0 + j;
          if (subtract) *dst -= v;
          else *dst = v;
        }
      } else {
        w[2 * i] = (uint32_t)__double2loint(v);
        w[2 * i + 1] = (uint32_t)__double2hiint(v);
      }
      H[j] = 0;
    }
    if (!last) tmem_st16(acc_t + 16 * h, w);
  }
  if (!last) tmem_st_wait();
  ++groups;
}

__global__ void __launch_bounds__(E_THREADS, 1)
    k_gemm_emu(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               double* __restrict__ C, int64_t M, int64_t N, int64_t ldc, int nkb, int Kp,
               int tiles_n, int n_tiles, const int* __restrict__ eA, const int* __restrict__ eB,
               const __grid_constant__ PairList pl, int* __restrict__ err, int subtract,
               int group_diags) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + ESTAGES * E_A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ESTAGES * E_STAGE);
  uint64_t* empty = full + ESTAGES;
  uint64_t* tfull = empty + ESTAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ESTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], E_EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(E_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int npairs = pl.n;
  // the K block kb of pair q is the last of its TMEM partial sum when the
  // sum holds E_CHUNK blocks or the next block belongs to another diagonal
  auto chunk_ends = [&](int q, int kb, int inchunk) {
    return inchunk == E_CHUNK ||
           (kb == nkb - 1 && (q == npairs - 1 || pl.a[q + 1] + pl.b[q + 1] != pl.a[q] + pl.b[q]));
  };

  if (warp == 0 && lane == 0) {
    uint32_t g = 0, issued = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int m0, n0;
      emu_tile(tile, n_tiles / tiles_n, tiles_n, m0, n0);
      for (int q = 0; q < npairs && ok; ++q) {
        const int xa = pl.a[q] * Kp, xb = pl.b[q] * Kp;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = g % ESTAGES;
          if (!mbar_wait(&empty[s], ((g / ESTAGES) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], E_STAGE);
          tma_load_2d(sA + s * E_A_STAGE, &tmA, xa + kb * 64, m0, &full[s]);
          tma_load_2d(sB + s * E_B_STAGE, &tmB, xb + kb * 64, n0, &full[s]);
          issued = g + 1;
        }
      }
    }
    if (!ok) atomicOr(err, 1);
    for (uint32_t q = (issued > ESTAGES ? issued - ESTAGES : 0); q < issued; ++q)
      if (!mbar_wait(&full[q % ESTAGES], (q / ESTAGES) & 1u)) atomicOr(err, 1);
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc<TC_BF16, EBM, EBN>();
    uint32_t g = 0, gc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int inchunk = 0;
      for (int q = 0; q < npairs && ok; ++q) {
        for (int kb = 0; kb < nkb && ok; ++kb, ++g) {
          const bool first = inchunk == 0;
          const uint32_t buf = gc & 1u;
          if (first) {
            if (!mbar_wait(&tempty[buf], ((gc >> 1) & 1u) ^ 1u)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const int s = g % ESTAGES;
          if (!mbar_wait(&full[s], (g / ESTAGES) & 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = sdesc(smem_u32(sA + s * E_A_STAGE));
          const uint64_t bd = sdesc(smem_u32(sB + s * E_B_STAGE));
          const uint32_t dt = tmem + buf * (uint32_t)EBN;
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma<TC_BF16>(dt, ad + 2u * k, bd + 2u * k, id, (!first || k > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
          if (chunk_ends(q, kb, ++inchunk)) {
            umma_commit(&tfull[buf]);
            ++gc;
            inchunk = 0;
          }
        }
      }
    }
    if (!ok) atomicOr(err, 1);
    if (gc > 0 && !mbar_wait(&tfull[(gc - 1) & 1u], ((gc - 1) >> 1) & 1u)) atomicOr(err, 1);
  } else if (warp >= 2) {
    const int qd = warp & 3;
    const int part = (warp - 2) >> 2;
    // this thread's float64 group sums: TMEM lane of its row, two columns per value
    const uint32_t acc_t = tmem + ((uint32_t)(qd * 32) << 16) + E_ACC_COL0 + part * 2 * E_EPI_COLS;
    uint32_t gc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int m0, n0;
      emu_tile(tile, n_tiles / tiles_n, tiles_n, m0, n0);
      const int64_t row = (int64_t)m0 + qd * 32 + lane;
      const int64_t col0 = (int64_t)n0 + part * E_EPI_COLS;
      const int ea = row < M ? eA[row] : 0;
      long long H[E_EPI_COLS];  // exact group sum, the current diagonal at weight 1
#pragma unroll
      for (int j = 0; j < E_EPI_COLS; ++j) H[j] = 0;
      int cur = pl.a[0] + pl.b[0];
      int inchunk = 0, groups = 0;
      for (int q = 0; q < npairs && ok; ++q) {
        const int diag = pl.a[q] + pl.b[q];
        for (int kb = 0; kb < nkb && ok; ++kb) {
          if (!chunk_ends(q, kb, ++inchunk)) continue;
          inchunk = 0;
          if (diag != cur) {
            if (diag / group_diags != cur / group_diags) {
              close_group(H, groups, false, acc_t, cur, ea, eB, col0, N, row, M, C, ldc,
                          subtract);
            } else {
              const int sh = SLICE_BITS * (diag - cur);
#pragma unroll
              for (int j = 0; j < E_EPI_COLS; ++j) H[j] <<= sh;
            }
            cur = diag;
          }
          const uint32_t buf = gc & 1u;
          if (!mbar_wait(&tfull[buf], (gc >> 1) & 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base =
              tmem + ((uint32_t)(qd * 32) << 16) + buf * (uint32_t)EBN + part * E_EPI_COLS;
#pragma unroll
          for (int j = 0; j < E_EPI_COLS / 16; ++j) {
            uint32_t r[16];
            tmem_ld16(base + 16 * j, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              // an exact integer of magnitude <= 2^24: converted exactly
              H[16 * j + i] += (long long)__float2int_rn(__uint_as_float(r[i]));
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
          ++gc;
        }
      }
      if (!ok) break;
      close_group(H, groups, true, acc_t, cur, ea, eB, col0, N, row, M, C, ldc, subtract);
    }
    if (!ok) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(E_TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------
// Slicing
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_view(const SplitView& v, int64_t r, int64_t k) {
  const int64_t r0 = r / v.n1, r1 = r - r0 * v.n1;
  const int64_t off = r0 * v.s0 + r1 * v.s1 + k * v.sk;
  return v.src_f32 ? (double)reinterpret_cast<const float*>(v.src)[off]
                   : reinterpret_cast<const double*>(v.src)[off];
}

// Biased exponent field of |x| (0 for zero and subnormals): comparing the
// magnitude bits as integers orders doubles by size.
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int exponent_of_max(unsigned long long mbits) {
  const int E = (int)(mbits >> 52);
  return E == 0 ? 0 : E - 1022;  // |x| < 2^(E - 1022) for every x of the row
}

// e[r] for rows whose K index is contiguous: one block per row.
__global__ void k_rowexp_contig(SplitView v, int* __restrict__ e) {
  __shared__ unsigned long long sh[8];
  const int64_t r = blockIdx.x;
  unsigned long long m = 0;
  for (int64_t k = threadIdx.x; k < v.K; k += blockDim.x) m = max(m, mag_bits(load_view(v, r, k)));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = max(m, sh[i]);
    e[r] = exponent_of_max(max(m, sh[0]));
  }
}

// Row maxima (of the magnitude bits) for rows that are adjacent in memory (K
// strided): 32 rows x a chunk of K per block, threads along the rows read
// neighbouring addresses; partial maxima combined with atomicMax into m[r].
constexpr int ROWMAX_KCHUNK = 256;
__global__ void k_rowmax_strided(SplitView v, unsigned long long* __restrict__ m) {
  __shared__ unsigned long long sh[8][33];
  const int64_t r = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * ROWMAX_KCHUNK;
  const int64_t k1 = min(k0 + (int64_t)ROWMAX_KCHUNK, v.K);
  unsigned long long a = 0;
  if (r < v.rows)
    for (int64_t k = k0 + threadIdx.y; k < k1; k += 8) a = max(a, mag_bits(load_view(v, r, k)));
  sh[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && r < v.rows) {
    for (int i = 1; i < 8; ++i) a = max(a, sh[i][threadIdx.x]);
    atomicMax(&m[r], a);
  }
}

__global__ void k_exp_from_max(const unsigned long long* __restrict__ m, int64_t rows,
                               int* __restrict__ e) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    e[r] = exponent_of_max(m[r]);
}

// x * 2^(56 - e) rounded to the nearest integer, from the IEEE bits (integer
// arithmetic only). |x| < 2^e, so |X| <= 2^56. Subnormal inputs count as 0.
__device__ __forceinline__ long long fixed56(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long mant = (bits & 0xFFFFFFFFFFFFFll) | (1ll << 52);
  const int sh = E - 1075 + 56 - e;  // value = mant * 2^(E - 1075)
  long long X;
  if (sh >= 0) X = mant << sh;  // sh <= 3 since |x| < 2^e
  else if (sh < -62) X = 0;
  else X = (mant + (1ll << (-sh - 1))) >> (-sh);
  return bits < 0 ? -X : X;
}

// Balanced base-128 digits of X: X = sum_p d_p 128^(7 - p); d_1..d_7 in
// [-64, 63], d_0 in [-128, 128]; slice p of the operand is the integer d_p
// (exact in bf16) and stands for d_p 2^(-7 (p + 1)) 2^e.
__device__ __forceinline__ void store_slices(__nv_bfloat16* dst, int64_t base, int64_t Kp, double x,
                                             int e) {
  long long X = fixed56(x, e);
  int d[SLICES];
#pragma unroll
  for (int p = SLICES - 1; p > 0; --p) {
    const int dig = (int)(((X + 64) & 127) - 64);
    d[p] = dig;
    X = (X - dig) >> SLICE_BITS;
  }
  d[0] = (int)X;
#pragma unroll
  for (int p = 0; p < SLICES; ++p) dst[base + (int64_t)p * Kp] = __float2bfloat16_rn((float)d[p]);
}

__global__ void k_slice_direct(SplitView v, const int* __restrict__ e, __nv_bfloat16* __restrict__ dst,
                               int64_t Kp) {
  const int64_t total = v.rows * Kp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / Kp, k = t - r * Kp;
    const double x = (k < v.K) ? load_view(v, r, k) : 0.0;
    store_slices(dst, r * SLICES * Kp + k, Kp, x, e[r]);
  }
}

__global__ void k_slice_transpose(SplitView v, const int* __restrict__ e,
                                  __nv_bfloat16* __restrict__ dst, int64_t Kp) {
  __shared__ double tile[32][33];
  const int64_t r_base = (int64_t)blockIdx.x * 32, k_base = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t k = k_base + j, r = r_base + tx;
    tile[j][tx] = (k < v.K && r < v.rows) ? load_view(v, r, k) : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r_base + j, k = k_base + tx;
    if (r < v.rows && k < Kp) store_slices(dst, r * SLICES * Kp + k, Kp, tile[tx][j], e[r]);
  }
}

int blocks_1d(int64_t n, int t) {
  int64_t b = cdiv(n, t);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65536));
}

osmps_status slice_operand(osmps_ctx* ctx, const SplitView& v, int64_t Kp, int* e,
                           __nv_bfloat16* dst, cudaStream_t s) {
  if (v.rows <= 0) return OSMPS_OK;
  const bool contig = (v.sk == 1);
  if (contig) {
    if (v.rows > 2147483647ll) return set_error(OSMPS_ESHAPE, "emulated GEMM: too many rows");
    { k_rowexp_contig<<<(unsigned)v.rows, 256, 0, s>>>(v, e); note_launch(); }
    { k_slice_direct<<<blocks_1d(v.rows * Kp, 256), 256, 0, s>>>(v, e, dst, Kp); note_launch(); }
  } else {
    if (cdiv(Kp, 32) > 65535 || cdiv(v.K, ROWMAX_KCHUNK) > 65535)
      return set_error(OSMPS_ESHAPE, "emulated GEMM: K too large");
    osmps_status st = OSMPS_OK;
    auto* mx = (unsigned long long*)ws_get(ctx, SLOT_EMU_MAX, (size_t)v.rows * 8, s, &st);
    if (!mx) return st;
    OSMPS_CUDA(cudaMemsetAsync(mx, 0, (size_t)v.rows * 8, s));
    dim3 g1((unsigned)cdiv(v.rows, 32), (unsigned)std::max<int64_t>(1, cdiv(v.K, ROWMAX_KCHUNK)));
    { k_rowmax_strided<<<g1, dim3(32, 8), 0, s>>>(v, mx); note_launch(); }
    { k_exp_from_max<<<blocks_1d(v.rows, 256), 256, 0, s>>>(mx, v.rows, e); note_launch(); }
    dim3 grid((unsigned)cdiv(v.rows, 32), (unsigned)cdiv(Kp, 32));
    { k_slice_transpose<<<grid, dim3(32, 8), 0, s>>>(v, e, dst, Kp); note_launch(); }
  }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

PairList make_pairs() {
  PairList pl{};
  pl.n = 0;
  for (int sum = 0; sum < SLICES; ++sum)
    for (int i = 0; i <= sum; ++i) {
      pl.a[pl.n] = (unsigned char)i;
      pl.b[pl.n] = (unsigned char)(sum - i);
      ++pl.n;
    }
  return pl;
}

}  // namespace

osmps_status gemm_emu(osmps_ctx* ctx, const SplitView& a, const SplitView& b, int64_t M,
                      int64_t N, int64_t K, double* C, int64_t ldc, cudaStream_t s,
                      bool subtract, bool small_on_dmma) {
  if (M <= 0 || N <= 0) return OSMPS_OK;
  if (K <= 0 || a.rows != M || b.rows != N || a.K != K || b.K != K)
    return set_error(OSMPS_ESHAPE, "gemm_emu: inconsistent operand views");
  // Small products go to the float64 DMMA kernel, which is float64-accurate
  // too: the emulation costs about 56 us even for one tile (slicing passes,
  // 36 slice pairs), while the DMMA kernel spreads its 64 x 64 tiles over the
  // SMs at about 8 GFLOP/s each. Taken when that estimate is under 40 us.
  const double dmma_tiles =
      std::min<double>((double)cdiv(M, 64) * (double)cdiv(N, 64), (double)ctx->sm_count);
  const double dmma_us = 2.0 * (double)M * (double)N * (double)K / (dmma_tiles * 8e3);
  if (small_on_dmma && a.n1 == 1 && b.n1 == 1 && !a.src_f32 && !b.src_f32 && dmma_us < 40.0) {
    GemmF64 g;
    g.M = M; g.N = N; g.K = K;
    g.A = static_cast<const double*>(a.src); g.sam = a.s0; g.sak = a.sk;
    g.B = static_cast<const double*>(b.src); g.sbk = b.sk; g.sbn = b.s0;
    g.C = C; g.scm = ldc; g.scn = 1;
    if (subtract) {
      g.alpha = -1.0;
      g.beta = 1.0;
    }
    return gemm_f64(g, s);
  }
  const int64_t Kp = round_up(K, 64);
  if (SLICES * Kp > ((int64_t)1 << 31) || cdiv(M, EBM) * cdiv(N, EBN) > ((int64_t)1 << 31))
    return set_error(OSMPS_ESHAPE, "gemm_emu: dimensions exceed the supported range");
  osmps_status st = OSMPS_OK;
  auto* sa = (__nv_bfloat16*)ws_get(ctx, SLOT_EMU_A, (size_t)M * SLICES * Kp * 2, s, &st);
  if (!sa) return st;
  auto* sb = (__nv_bfloat16*)ws_get(ctx, SLOT_EMU_B, (size_t)N * SLICES * Kp * 2, s, &st);
  if (!sb) return st;
  int* ex = (int*)ws_get(ctx, SLOT_EMU_EXP, (size_t)(M + N + 64) * sizeof(int), s, &st);
  if (!ex) return st;
  int* eA = ex;
  int* eB = ex + ((M + 63) / 64) * 64;
  OSMPS_TRY(slice_operand(ctx, a, Kp, eA, sa, s));
  OSMPS_TRY(slice_operand(ctx, b, Kp, eB, sb, s));
  CUtensorMap ma, mb;
  OSMPS_TRY(tc_make_map(&ma, sa, TC_BF16, M, SLICES * Kp, EBM));
  OSMPS_TRY(tc_make_map(&mb, sb, TC_BF16, N, SLICES * Kp, EBN));
  // thread-safe one-time setup (function-local static initialisation)
  static const cudaError_t configured =
      cudaFuncSetAttribute(k_gemm_emu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E_SMEM);
  OSMPS_CUDA(configured);
  static const PairList pl = make_pairs();
  const int tiles_n = (int)cdiv(N, EBN);
  const int n_tiles = tiles_n * (int)cdiv(M, EBM);
  const int grid = std::min(n_tiles, ctx->sm_count);
  const int nkb = (int)(Kp / 64);
  // diagonals per exact int64 group: four while a group sum stays below 2^53
  // (|I_d| < (d + 1) K 2^14 with slice digits of at most 2^7 and 2^6), else two
  const int group_diags = Kp <= ((int64_t)1 << 17) ? 4 : 2;
  const int ph = prof_begin(s);
  {
    k_gemm_emu<<<grid, E_THREADS, E_SMEM, s>>>(ma, mb, C, M, N, ldc, nkb, (int)Kp, tiles_n,
                                               n_tiles, eA, eB, pl, ctx->dev_flags,
                                               subtract ? 1 : 0, group_diags);
    note_launch();
  }
  OSMPS_LAUNCH_CHECK();
  const double logical = 2.0 * (double)M * (double)N * (double)K;
  prof_end(ph, s, OSMPS_KERNEL_GEMM_EMU, logical, (double)pl.n * logical);
  return OSMPS_OK;
}

}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_dgemm_emu(osmps_ctx* ctx, const double* A, const double* B, double* C,
                                        int64_t M, int64_t N, int64_t K, void* stream) {
  clear_error();
  if (!ctx || !A || !B || !C) return set_error(OSMPS_EINVAL, "osmps_dgemm_emu: null argument");
  if (C == A || C == B) return set_error(OSMPS_EINVAL, "osmps_dgemm_emu: C aliases an input");
  if (M <= 0 || N <= 0 || K <= 0) return set_error(OSMPS_ESHAPE, "osmps_dgemm_emu: dimensions");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  SplitView a;
  a.src = A; a.rows = M; a.K = K; a.s0 = K; a.sk = 1;
  SplitView b;  // row n of the B operand = column n of B
  b.src = B; b.rows = N; b.K = K; b.s0 = 1; b.sk = N;
  return gemm_emu(ctx, a, b, M, N, K, C, N, (cudaStream_t)stream, false, false);
}
