// Split-precision GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The dense contractions of the effective Hamiltonian (Sec. 3.4,
// Fig. LanczosMPS) and of the environment updates are GEMMs
//   C[M,N] = sum_k A[m,k] B[n,k]
// with float64 data. Each float64 operand x is stored as x_hi + x_lo, both in
// the tensor-core type (bf16 or tf32), and the product is accumulated in
// float32 as A_hi B_hi + A_hi B_lo + A_lo B_hi (the A_lo B_lo term is below
// the accumulator's resolution). Each operand row holds [hi | lo], Kp columns
// each, so a product is just a K-range of the same two TMA tensors.
//
// Kernel structure (persistent, 128 x 256 output tiles, 576 threads):
//   warp 0, one lane : TMA producer, 4-stage ring of 128B-swizzled tiles
//   warp 1           : allocates all 512 TMEM columns; one lane issues the
//                      MMAs (M=128, N=256, 4 instructions per 128-byte K slice),
//                      commits each stage back to the producer and each
//                      16-MMA partial sum to the epilogue
//   warps 2..17      : epilogue, TMEM partial sums -> float32 registers
//                      (round-to-nearest adds) -> shared-memory staging ->
//                      row-contiguous global stores (f32 or f64)
// Every mbarrier wait is bounded by %globaltimer (2 s); on expiry the kernel
// records bit 0 in the context's error flag, drains its own copies (bounded),
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "ieee.cuh"
#include "tcgen05.cuh"

namespace osmps {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int KSLICE_BYTES = 128;  // K bytes per stage row = one 128B swizzle span
constexpr int A_STAGE = BM * KSLICE_BYTES;  // 16 KB
constexpr int EPI_WARPS = 16;                // 4 lane quarters x 4 column quarters
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr int CHUNK = 4;                     // K slices (x 4 MMAs) per TMEM partial sum
// epilogue staging: per epilogue warp 32 rows x 16 columns of float32
constexpr int STG_COLS = 16;
constexpr int STG_BYTES = EPI_WARPS * 32 * STG_COLS * 4;  // 32 KB

// Tile width BN (256, 128 or 64 output columns): the B stage, the ring depth
// (about 192 KB of stages), the epilogue columns per thread and the two TMEM
// accumulator buffers follow from it. The arithmetic per output element
// (K order, partial sums, promotion) does not depend on BN, so every width
// gives the same bits.
template <int BN>
struct TcTile {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  static constexpr int B_STAGE = BN * KSLICE_BYTES;
  static constexpr int STAGE_BYTES = A_STAGE + B_STAGE;
  static constexpr int STAGES = (192 * 1024) / STAGE_BYTES;  // 4 / 6 / 8
  static constexpr int EPI_COLS = BN / 4;                     // columns per epilogue thread
  static constexpr uint32_t TMEM_COLS = 2 * BN;               // two accumulator buffers
  static constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024 + 256 + STG_BYTES;
};

// One epilogue warp's 32 x 64 results (lane = row, acc = its 64 columns) to
// global memory, through its 32 x 16 float32 staging block in 4 passes: the
// lanes write their rows (float4 groups XOR-swizzled by row), then each
// half-warp stores 16 consecutive columns of one row, so a store instruction
// covers 2 rows x 16 columns (4 full sectors for float32, 8 for float64)
// instead of touching 32 rows.
template <int OUT, int EPI_COLS>
__device__ __forceinline__ void store_tile_rows(void* C, int64_t row0, int64_t col0, int64_t M,
                                                int64_t N, int64_t ldc, const float (&acc)[EPI_COLS],
                                                float* __restrict__ stg, int lane,
                                                const float* __restrict__ addend) {
#pragma unroll
  for (int pass = 0; pass < EPI_COLS / STG_COLS; ++pass) {
#pragma unroll
    for (int v = 0; v < STG_COLS / 4; ++v) {
      const int g = v ^ (lane & 3);
      reinterpret_cast<float4*>(stg + lane * STG_COLS)[g] =
          make_float4(acc[STG_COLS * pass + 4 * v], acc[STG_COLS * pass + 4 * v + 1],
                      acc[STG_COLS * pass + 4 * v + 2], acc[STG_COLS * pass + 4 * v + 3]);
    }
    __syncwarp();
    const int cc = lane & 15;
    const int64_t col = col0 + STG_COLS * pass + cc;
    if (OUT != TC_OUT_F32 && addend) {
      // the addend's values of eight rows are requested before the first of
      // their stores, so their latency is paid twice per pass, not per row;
      // the sum is formed in float32 (both terms are float32 results) and
      // widened by integer fields (the float64 pipe is narrow)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float add[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t row = row0 + 2 * (8 * h + i) + (lane >> 4);
          add[i] = (row < M && col < N) ? addend[row * ldc + col] : 0.0f;
        }
#pragma unroll 4
        for (int i = 0; i < 8; ++i) {
          const int rr = 2 * (8 * h + i) + (lane >> 4);
          const float val = stg[rr * STG_COLS + (((cc >> 2) ^ (rr & 3)) << 2) + (cc & 3)];
          const int64_t row = row0 + rr;
          if (row < M && col < N) reinterpret_cast<double*>(C)[row * ldc + col] = f32_to_f64(val + add[i]);
        }
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < 16; ++i) {
        const int rr = 2 * i + (lane >> 4);
        const float val = stg[rr * STG_COLS + (((cc >> 2) ^ (rr & 3)) << 2) + (cc & 3)];
        const int64_t row = row0 + rr;
        if (row < M && col < N) {
          if (OUT == TC_OUT_F32)
            reinterpret_cast<float*>(C)[row * ldc + col] = val;
          else
            reinterpret_cast<double*>(C)[row * ldc + col] = (double)val;
        }
      }
    }
    __syncwarp();  // the next pass overwrites the staging block
  }
}

// Persistent kernel: CTA b handles tiles b, b + gridDim.x, ... (N-tile index
// fastest, so neighbouring CTAs share A rows in L2). The K loop is cut into
// chunks of CHUNK slices (16 MMAs); each chunk accumulates into one of two
// 256-column TMEM buffers, and the epilogue warps add the chunk into float32
// registers with round-to-nearest. This keeps the tensor core's own
// accumulation to 16 additions per partial sum, so its truncating
// accumulator does not build a bias over long K.
// One output tile: where its operand rows start, its K-slice count and where
// its results go. Plain GEMM: one problem. Grouped GEMM: tile -> problem by
// binary search over the problems' first tiles (GroupProblem table).
struct TileJob {
  int a_row, b_row, nkb;
  int64_t row0, col0, M, N, ldc;
  void* C;
};

template <int OUT, int BN>
__device__ __forceinline__ TileJob tile_job(int tile, void* C, int64_t M, int64_t N, int64_t ldc,
                                            int nkb, int tiles_n,
                                            const GroupProblem* __restrict__ probs, int n_prob) {
  TileJob j;
  if (probs == nullptr) {
    j.row0 = (int64_t)(tile / tiles_n) * BM;
    j.col0 = (int64_t)(tile % tiles_n) * BN;
    j.a_row = (int)j.row0;
    j.b_row = (int)j.col0;
    j.nkb = nkb;
    j.M = M;
    j.N = N;
    j.ldc = ldc;
    j.C = C;
    return j;
  }
  int lo = 0, hi = n_prob - 1;  // last problem with tile0 <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  const GroupProblem& p = probs[lo];
  const int local = tile - p.tile0;
  j.row0 = (int64_t)(local / p.tiles_n) * BM;
  j.col0 = (int64_t)(local % p.tiles_n) * BN;
  j.a_row = p.a_row0 + (int)j.row0;
  j.b_row = p.b_row0 + (int)j.col0;
  j.nkb = p.nkb;
  j.M = p.M;
  j.N = p.N;
  j.ldc = p.ldc;
  j.C = reinterpret_cast<uint8_t*>(C) + p.c_off * (OUT == TC_OUT_F32 ? 4 : 8);
  return j;
}

template <int KIND, int OUT, int BN>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              void* __restrict__ C, int64_t M, int64_t N, int64_t ldc, int nkb, int kelem,
              int Kp, int tiles_n, int n_tiles, int* __restrict__ err,
              const GroupProblem* __restrict__ probs, int n_prob, const float* __restrict__ addend) {
  using T = TcTile<BN>;
  constexpr int STAGES = T::STAGES, B_STAGE = T::B_STAGE, STAGE_BYTES = T::STAGE_BYTES;
  constexpr int EPI_COLS = T::EPI_COLS;
  constexpr uint32_t TMEM_COLS = T::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;   // 2: chunk in TMEM buffer ready
  uint64_t* tempty = tfull + 2;       // 2: TMEM buffer drained by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // Producer. Slice it of a tile covers K slice kb = it / 3 of product
    // p = it % 3: p = 0 (hi, hi), 1 (hi, lo), 2 (lo, hi).
    uint32_t g = 0;  // slices issued by this CTA (ring position)
    uint32_t issued = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const TileJob job = tile_job<OUT, BN>(tile, C, M, N, ldc, nkb, tiles_n, probs, n_prob);
      const int total = 3 * job.nkb;  // K slices over the three products
      for (int it = 0; it < total; ++it, ++g) {
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u)) {
          ok = false;
          break;
        }
        const int kb = it / 3, p = it % 3;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(sA + s * A_STAGE, &tmA, kb * kelem + (p == 2 ? Kp : 0), job.a_row, &full[s]);
        tma_load_2d(sB + s * B_STAGE, &tmB, kb * kelem + (p == 1 ? Kp : 0), job.b_row, &full[s]);
        issued = g + 1;
      }
    }
    if (!ok) atomicOr(err, 1);
    // Drain: the last copy issued into each stage has landed before exit.
    for (uint32_t q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
      if (!mbar_wait(&full[q % STAGES], (q / STAGES) & 1u)) atomicOr(err, 1);
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc<KIND, BM, BN>();
    uint32_t g = 0, gc = 0;  // slices / chunks consumed by this CTA
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const int total = 3 * tile_job<OUT, BN>(tile, C, M, N, ldc, nkb, tiles_n, probs, n_prob).nkb;
      for (int it = 0; it < total && ok; ++it, ++g) {
        const bool first = (it % CHUNK) == 0;
        const uint32_t buf = gc & 1u;
        if (first) {
          if (!mbar_wait(&tempty[buf], ((gc >> 1) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const int s = g % STAGES;
        if (!mbar_wait(&full[s], (g / STAGES) & 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t ad = sdesc(smem_u32(sA + s * A_STAGE));
        const uint64_t bd = sdesc(smem_u32(sB + s * B_STAGE));
        const uint32_t dt = tmem + buf * (uint32_t)BN;
#pragma unroll
        for (int k = 0; k < KSLICE_BYTES / 32; ++k)  // 32 bytes of K per MMA: +2 in the address field
          umma<KIND>(dt, ad + 2u * k, bd + 2u * k, id, (!first || k > 0) ? 1u : 0u);
        umma_commit(&empty[s]);
        if ((it % CHUNK) == CHUNK - 1 || it == total - 1) {
          umma_commit(&tfull[buf]);
          ++gc;
        }
      }
    }
    if (!ok) atomicOr(err, 1);
    // No MMA may still be running when TMEM is released: wait for the last chunk.
    if (gc > 0 && !mbar_wait(&tfull[(gc - 1) & 1u], ((gc - 1) >> 1) & 1u)) atomicOr(err, 1);
  } else if (warp >= 2) {
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int part = (warp - 2) >> 2;       // which 64-column quarter of the tile
    uint32_t gc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      const int nchunk =
          (3 * tile_job<OUT, BN>(tile, C, M, N, ldc, nkb, tiles_n, probs, n_prob).nkb + CHUNK - 1) / CHUNK;
      float acc[EPI_COLS];
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) acc[j] = 0.0f;
      for (int c = 0; c < nchunk; ++c, ++gc) {
        const uint32_t buf = gc & 1u;
        if (!mbar_wait(&tfull[buf], (gc >> 1) & 1u)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + buf * (uint32_t)BN + part * EPI_COLS;
#pragma unroll
        for (int j = 0; j < EPI_COLS / 16; ++j) {
          uint32_t r[16];
          tmem_ld16(base + 16 * j, r);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[16 * j + i] += __uint_as_float(r[i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      if (!ok) break;
      // decoded again after the K loop so its fields are not live during it
      const TileJob job = tile_job<OUT, BN>(tile, C, M, N, ldc, nkb, tiles_n, probs, n_prob);
      float* stg = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES + 256) + (warp - 2) * 32 * STG_COLS;
      store_tile_rows<OUT, EPI_COLS>(job.C, job.row0 + q * 32, job.col0 + part * EPI_COLS, job.M, job.N,
                           job.ldc, acc, stg, lane, addend);
    }
    if (!ok) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

osmps_status tc_make_map(CUtensorMap* map, const void* base, int kind, int64_t rows, int64_t cols,
                         int box_rows) {
  auto fn = encode_fn();
  if (!fn) return set_error(OSMPS_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  const size_t es = tc_elem_bytes(kind);
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return set_error(OSMPS_EINVAL, "tensor-core operand base not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * es)};
  cuuint32_t box[2] = {(cuuint32_t)(KSLICE_BYTES / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, kind == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(OSMPS_ECUDA, "cuTensorMapEncodeTiled failed (%d): rows=%lld cols=%lld", (int)r,
                     (long long)rows, (long long)cols);
  return OSMPS_OK;
}

namespace {

template <int KIND, int OUT, int BN>
osmps_status launch(const CUtensorMap& a, const CUtensorMap& b, const GemmTc& g, int* err,
                    int sm_count, cudaStream_t stream) {
  using T = TcTile<BN>;
  // thread-safe one-time setup (function-local static initialisation)
  static const cudaError_t configured = cudaFuncSetAttribute(
      k_gemm_tc<KIND, OUT, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM_BYTES);
  OSMPS_CUDA(configured);
  const int kelem = KSLICE_BYTES / (int)tc_elem_bytes(KIND);
  const int nkb = (int)(g.Kp / kelem);
  const int tiles_n = (int)cdiv(g.N, BN);
  const int n_tiles = tiles_n * (int)cdiv(g.M, BM);
  const int grid = std::min(n_tiles, sm_count);
  const int ph = prof_begin(stream);
  { k_gemm_tc<KIND, OUT, BN><<<grid, THREADS, T::SMEM_BYTES, stream>>>(
        a, b, g.C, g.M, g.N, g.ldc, nkb, kelem, (int)g.Kp, tiles_n, n_tiles, err, nullptr, 0,
        OUT == TC_OUT_F64 ? g.addend : nullptr); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  const double logical = 2.0 * (double)g.M * (double)g.N * (double)(g.K > 0 ? g.K : g.Kp);
  prof_end(ph, stream, OSMPS_KERNEL_GEMM_TC, logical, 3.0 * logical);
  return OSMPS_OK;
}

template <int KIND, int OUT>
osmps_status launch_bn(int bn, const CUtensorMap& a, const CUtensorMap& b, const GemmTc& g, int* err,
                       int sm_count, cudaStream_t stream) {
  if (bn == 64) return launch<KIND, OUT, 64>(a, b, g, err, sm_count, stream);
  if (bn == 128) return launch<KIND, OUT, 128>(a, b, g, err, sm_count, stream);
  return launch<KIND, OUT, 256>(a, b, g, err, sm_count, stream);
}

osmps_status launch_any(int bn, const CUtensorMap& a, const CUtensorMap& b, const GemmTc& g, int* err,
                        int sm_count, cudaStream_t stream) {
  if (g.kind == TC_BF16) {
    if (g.out == TC_OUT_F32) return launch_bn<TC_BF16, TC_OUT_F32>(bn, a, b, g, err, sm_count, stream);
    return launch_bn<TC_BF16, TC_OUT_F64>(bn, a, b, g, err, sm_count, stream);
  }
  if (g.out == TC_OUT_F32) return launch_bn<TC_TF32, TC_OUT_F32>(bn, a, b, g, err, sm_count, stream);
  return launch_bn<TC_TF32, TC_OUT_F64>(bn, a, b, g, err, sm_count, stream);
}

template <int KIND, int OUT, int BN>
osmps_status launch_grouped(const CUtensorMap& ma, const CUtensorMap& mb, const GemmTcGrouped& g,
                            int64_t n_tiles, int* err, int sm_count, cudaStream_t stream) {
  using T = TcTile<BN>;
  static const cudaError_t cfg = cudaFuncSetAttribute(
      k_gemm_tc<KIND, OUT, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::SMEM_BYTES);
  OSMPS_CUDA(cfg);
  const int kelem = KSLICE_BYTES / (int)tc_elem_bytes(KIND);
  const int grid = (int)std::min<int64_t>(n_tiles, sm_count);
  k_gemm_tc<KIND, OUT, BN><<<grid, THREADS, T::SMEM_BYTES, stream>>>(
      ma, mb, g.C, 0, 0, 0, 0, kelem, (int)g.Kpl, 1, (int)n_tiles, err, g.probs, g.n_prob, nullptr);
  note_launch();
  return OSMPS_OK;
}

template <int KIND, int OUT>
osmps_status launch_grouped_bn(int bn, const CUtensorMap& ma, const CUtensorMap& mb,
                               const GemmTcGrouped& g, int64_t n_tiles, int* err, int sm_count,
                               cudaStream_t stream) {
  if (bn == 64) return launch_grouped<KIND, OUT, 64>(ma, mb, g, n_tiles, err, sm_count, stream);
  if (bn == 128) return launch_grouped<KIND, OUT, 128>(ma, mb, g, n_tiles, err, sm_count, stream);
  return launch_grouped<KIND, OUT, 256>(ma, mb, g, n_tiles, err, sm_count, stream);
}

}  // namespace

bool tc_tile_width_ok(int bn) { return bn == 64 || bn == 128 || bn == 256; }

int64_t group_tiles(GroupProblem* probs, int n_prob, int bn) {
  int64_t t = 0;
  for (int i = 0; i < n_prob; ++i) {
    probs[i].tiles_n = (int)cdiv(probs[i].N, bn);
    probs[i].tile0 = (int)t;
    t += (int64_t)probs[i].tiles_n * cdiv(probs[i].M, BM);
  }
  return t;
}

osmps_status gemm_tc_grouped(osmps_ctx* ctx, const GemmTcGrouped& g, cudaStream_t stream) {
  if (g.n_prob <= 0 || g.n_tiles <= 0) return OSMPS_OK;
  if (g.Kpl <= 0 || g.Kpl % 64 != 0 || 2 * g.Kpl > (int64_t)1 << 31 || g.n_tiles > ((int64_t)1 << 31) ||
      g.rowsA > ((int64_t)1 << 31) || g.rowsB > ((int64_t)1 << 31))
    return set_error(OSMPS_ESHAPE, "gemm_tc_grouped: bad packed operand shape");
  if (!tc_tile_width_ok(g.bn)) return set_error(OSMPS_EINVAL, "gemm_tc_grouped: tile width %d", g.bn);
  CUtensorMap ma, mb;
  OSMPS_TRY(tc_make_map(&ma, g.A, g.kind, g.rowsA, 2 * g.Kpl, BM));
  OSMPS_TRY(tc_make_map(&mb, g.B, g.kind, g.rowsB, 2 * g.Kpl, g.bn));
  const int ph = prof_begin(stream);
  int* err = ctx->dev_flags;
  if (g.kind == TC_BF16) {
    if (g.out == TC_OUT_F32)
      OSMPS_TRY((launch_grouped_bn<TC_BF16, TC_OUT_F32>(g.bn, ma, mb, g, g.n_tiles, err, ctx->sm_count, stream)));
    else
      OSMPS_TRY((launch_grouped_bn<TC_BF16, TC_OUT_F64>(g.bn, ma, mb, g, g.n_tiles, err, ctx->sm_count, stream)));
  } else {
    if (g.out == TC_OUT_F32)
      OSMPS_TRY((launch_grouped_bn<TC_TF32, TC_OUT_F32>(g.bn, ma, mb, g, g.n_tiles, err, ctx->sm_count, stream)));
    else
      OSMPS_TRY((launch_grouped_bn<TC_TF32, TC_OUT_F64>(g.bn, ma, mb, g, g.n_tiles, err, ctx->sm_count, stream)));
  }
  OSMPS_LAUNCH_CHECK();
  prof_end(ph, stream, OSMPS_KERNEL_GEMM_TC, g.logical_flops, 3.0 * g.logical_flops);
  return OSMPS_OK;
}

osmps_status gemm_tc(osmps_ctx* ctx, const GemmTc& g, cudaStream_t stream) {
  if (g.M <= 0 || g.N <= 0) return OSMPS_OK;
  if (g.Kp <= 0 || g.Kp % 64 != 0)
    return set_error(OSMPS_ESHAPE, "gemm_tc: Kp=%lld must be a positive multiple of 64",
                     (long long)g.Kp);
  if (2 * g.Kp > (int64_t)1 << 31 || cdiv(g.M, BM) > 65535 || g.M > ((int64_t)1 << 31) ||
      g.N > ((int64_t)1 << 31))
    return set_error(OSMPS_ESHAPE, "gemm_tc: dimensions exceed the supported range");
  int* err = ctx->dev_flags;
  CUtensorMap ma;
  OSMPS_TRY(tc_make_map(&ma, g.A, g.kind, g.M, 2 * g.Kp, BM));
  const TcKey key = tc_key(0, g.kind, g.out, cdiv(g.M, BM), cdiv(g.N, 64), cdiv(g.Kp, 512));
  int bn = tc_tuned_width(ctx, key);
  if (bn == 0 && tc_may_tune(ctx)) {
    // Autotuning: the first product of a size class is run at every tile
    // width, each timed on the stream after one untimed run (the outputs are
    // the same bits); the fastest width is kept for the class.
    float us[3] = {0.f, 0.f, 0.f};
    const int widths[3] = {256, 128, 64};
    for (int w = 0; w < 3; ++w) {
      CUtensorMap mb;
      OSMPS_TRY(tc_make_map(&mb, g.B, g.kind, g.N, 2 * g.Kp, widths[w]));
      OSMPS_TRY(launch_any(widths[w], ma, mb, g, err, ctx->sm_count, stream));
      OSMPS_TRY(tc_time_launches(ctx, stream, 2, &us[w], [&](cudaStream_t s) {
        return launch_any(widths[w], ma, mb, g, err, ctx->sm_count, s);
      }));
    }
    bn = tc_record_tuning(ctx, key, widths, us);
    return OSMPS_OK;  // the last timed run left the product in C
  }
  if (bn == 0) bn = 256;
  CUtensorMap mb;
  OSMPS_TRY(tc_make_map(&mb, g.B, g.kind, g.N, 2 * g.Kp, bn));
  return launch_any(bn, ma, mb, g, err, ctx->sm_count, stream);
}

}  // namespace osmps
