// Failure-path self-test of the bounded device waits. Every wait in this
// library's kernels on a flag, a barrier or an mbarrier gives up after a time
// limit, records the failure in the context's error flags, releases what the
// kernel holds and returns, so a lost arrival becomes OSMPS_ETIMEOUT instead
// of a hung GPU. These kernels make such a wait run out on purpose, with a
// short limit, on a barrier that nothing completes:
//   which = 0: one CTA allocates tensor memory (TMEM) as the tcgen05 kernels
//              do, waits on an mbarrier no thread arrives at, frees the TMEM;
//   which = 1: a cooperative grid whose last block leaves without arriving at
//              the grid barrier the others wait at.
// Nothing faults, traps or spins without a bound; the context stays usable.
#include "common.cuh"
#include "gridsync.cuh"
#include "ieee.cuh"
#include "tcgen05.cuh"

namespace osmps {
namespace {

constexpr int SELFTEST_FLAG = 12;  // dev_flags slot of these kernels

__global__ void __launch_bounds__(64, 1) k_selftest_mbarrier(uint64_t limit_ns, int* __restrict__ err) {
  using namespace tc;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(32u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 32) {  // phase 0 never completes: nobody arrives
    if (!mbar_wait(&bar, 0u, limit_ns)) atomicOr(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u));
  }
}

__global__ void k_selftest_grid(unsigned* bar, uint64_t limit_ns, int* __restrict__ err) {
  __shared__ int s_ok;
  if (blockIdx.x == gridDim.x - 1) return;  // this block never arrives
  grid_barrier(bar, gridDim.x, err, &s_ok, limit_ns);
}

__global__ void k_selftest_convert(const double* __restrict__ x64, float* __restrict__ y32,
                                   const float* __restrict__ x32, double* __restrict__ y64, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    y32[i] = f64_to_f32_rn(x64[i]);
    y64[i] = f32_to_f64(x32[i]);
  }
}

__global__ void k_selftest_bf16(const double* __restrict__ x, uint16_t* __restrict__ y_int,
                                uint16_t* __restrict__ y_hw, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    y_int[i] = __bfloat16_as_ushort(f64_to_bf16_rn(x[i]));
    y_hw[i] = __bfloat16_as_ushort(__double2bfloat16(x[i]));
  }
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_selftest_bf16(osmps_ctx* ctx, const double* x, uint16_t* y_int,
                                            uint16_t* y_hw, int64_t n, void* stream) {
  clear_error();
  if (!ctx || (n > 0 && (!x || !y_int || !y_hw)))
    return set_error(OSMPS_EINVAL, "osmps_selftest_bf16: null argument");
  if (n < 0) return set_error(OSMPS_EINVAL, "osmps_selftest_bf16: n=%lld", (long long)n);
  if (n == 0) return OSMPS_OK;
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_selftest_bf16<<<blocks, 256, 0, s>>>(x, y_int, y_hw, n);
  note_launch();
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

extern "C" osmps_status osmps_selftest_convert(osmps_ctx* ctx, const double* x64, float* y32,
                                               const float* x32, double* y64, int64_t n, void* stream) {
  clear_error();
  if (!ctx || (n > 0 && (!x64 || !y32 || !x32 || !y64)))
    return set_error(OSMPS_EINVAL, "osmps_selftest_convert: null argument");
  if (n < 0) return set_error(OSMPS_EINVAL, "osmps_selftest_convert: n=%lld", (long long)n);
  if (n == 0) return OSMPS_OK;
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_selftest_convert<<<blocks, 256, 0, s>>>(x64, y32, x32, y64, n);
  note_launch();
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

extern "C" osmps_status osmps_selftest_wait_timeout(osmps_ctx* ctx, int which, double limit_us,
                                                    void* stream) {
  clear_error();
  if (!ctx) return set_error(OSMPS_EINVAL, "osmps_selftest_wait_timeout: null context");
  if (which != 0 && which != 1)
    return set_error(OSMPS_EINVAL, "osmps_selftest_wait_timeout: which %d", which);
  if (!(limit_us >= 1.0 && limit_us <= 1e6))
    return set_error(OSMPS_EINVAL, "osmps_selftest_wait_timeout: limit %g us outside [1, 1e6]", limit_us);
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  CtxScope scope_(ctx);
  cudaStream_t s = (cudaStream_t)stream;
  int* flag = ctx->dev_flags + SELFTEST_FLAG;
  unsigned* bar = reinterpret_cast<unsigned*>(ctx->dev_flags + SELFTEST_FLAG + 1);
  OSMPS_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), s));
  const uint64_t limit_ns = (uint64_t)(limit_us * 1e3);
  if (which == 0) {
    k_selftest_mbarrier<<<1, 64, 0, s>>>(limit_ns, flag);
    note_launch();
    OSMPS_LAUNCH_CHECK();
  } else {
    const int G = std::max(2, std::min(ctx->sm_count, 8));
    void* args[] = {&bar, (void*)&limit_ns, &flag};
    OSMPS_CUDA(cudaLaunchCooperativeKernel((void*)k_selftest_grid, dim3(G), dim3(64), args, 0, s));
    note_launch();
  }
  int h = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  if (h & 1)
    return set_error(OSMPS_ETIMEOUT, "osmps_selftest_wait_timeout: the %s wait gave up after %g us",
                     which == 0 ? "mbarrier" : "grid barrier", limit_us);
  return OSMPS_OK;
}
