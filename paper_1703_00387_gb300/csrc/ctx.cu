// Context, error reporting, workspace and float64 vector primitives.
#include <atomic>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace osmps {

static thread_local char g_err[1024] = "";

osmps_status set_error(osmps_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

void clear_error() { g_err[0] = 0; }

void* ws_get(osmps_ctx* ctx, Slot slot, size_t bytes, cudaStream_t stream, osmps_status* st) {
  Buffer& b = ctx->slots[slot];
  if (bytes == 0) bytes = 256;
  if (b.bytes >= bytes) return b.ptr;
  if (ctx->capturing) {
    *st = set_error(OSMPS_EUNSUPPORTED, "workspace slot %d would grow inside a CUDA graph capture",
                    (int)slot);
    return nullptr;
  }
  size_t want = bytes + bytes / 8;
  want = (want + 255) & ~size_t(255);
  if (b.ptr) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      *st = set_error(OSMPS_ECUDA, "workspace grow: stream sync failed: %s", cudaGetErrorString(e));
      return nullptr;
    }
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *st = set_error(OSMPS_ENOMEM, "workspace slot %d: cudaMalloc(%zu) failed: %s", (int)slot, want,
                    cudaGetErrorString(e));
    return nullptr;
  }
  b.ptr = p;
  b.bytes = want;
  ++ctx->ws_epoch;
  return p;
}

static thread_local osmps_ctx* g_cur = nullptr;
static std::atomic<long long> g_launches{0};

static thread_local long long t_launches = 0;
static thread_local bool t_batch_worker = false;

void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void note_launches(long long k) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  t_launches += k;
}
long long thread_launch_count() { return t_launches; }
void set_batch_worker(bool on) { t_batch_worker = on; }
bool is_batch_worker() { return t_batch_worker; }

CtxScope::CtxScope(osmps_ctx* c) : prev(g_cur) { g_cur = c; }
CtxScope::~CtxScope() { g_cur = prev; }
osmps_ctx* current_ctx() { return g_cur; }

static cudaEvent_t pool_event(osmps_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

int prof_begin(cudaStream_t stream) {
  osmps_ctx* c = g_cur;
  if (!c || !c->prof_on) return -1;
  osmps_ctx::ProfRec r{};
  r.a = pool_event(c);
  r.b = pool_event(c);
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, stream);
  c->prof.push_back(r);
  return (int)c->prof.size() - 1;
}

void prof_end(int h, cudaStream_t stream, int kernel, double flops, double tensor_flops) {
  osmps_ctx* c = g_cur;
  if (!c || h < 0 || h >= (int)c->prof.size()) return;
  auto& r = c->prof[h];
  cudaEventRecord(r.b, stream);
  r.kernel = kernel;
  r.flops = flops;
  r.tensor_flops = tensor_flops;
}

osmps_status pinned_reserve(osmps_ctx* ctx, size_t count) {
  if (ctx->host_pinned_count >= count) return OSMPS_OK;
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  ctx->host_pinned = nullptr;
  ctx->host_pinned_count = 0;
  size_t n = count < 4096 ? 4096 : count;
  OSMPS_CUDA(cudaMallocHost((void**)&ctx->host_pinned, n * sizeof(double)));
  ctx->host_pinned_count = n;
  return OSMPS_OK;
}

// ---------------------------------------------------------------------------
// Reductions: fixed-order two-stage sums (deterministic run to run).
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RED_THREADS / 32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < RED_THREADS / 32) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;
}

__global__ void k_sumsq_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = x[i];
    acc = fma(v, v, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

static int red_blocks(int64_t n) {
  int64_t b = cdiv(n, RED_THREADS * 4);
  if (b < 1) b = 1;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)b;
}

osmps_status vec_norm2(osmps_ctx* ctx, const double* x, int64_t n, double* dev_out, cudaStream_t s) {
  osmps_status st = OSMPS_OK;
  double* part = (double*)ws_get(ctx, SLOT_RED, RED_MAX_BLOCKS * sizeof(double), s, &st);
  if (!part) return st;
  int nb = red_blocks(n);
  { k_sumsq_partial<<<nb, RED_THREADS, 0, s>>>(x, n, part); note_launch(); }
  { k_sum_final<<<1, RED_THREADS, 0, s>>>(part, nb, dev_out); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

__global__ void k_scale_inv_sqrt(double* __restrict__ x, int64_t n, const double* __restrict__ nrm2) {
  double f = 1.0 / sqrt(*nrm2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

__global__ void k_scale_inv(double* __restrict__ y, const double* __restrict__ x, int64_t n,
                            const double* __restrict__ div) {
  double f = 1.0 / (*div);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

static int ew_blocks(int64_t n) {
  int64_t b = cdiv(n, 256 * 4);
  if (b < 1) b = 1;
  if (b > 65536) b = 65536;
  return (int)b;
}

osmps_status vec_scale_by_inv_sqrt(double* x, int64_t n, const double* dev_norm2, cudaStream_t s) {
  { k_scale_inv_sqrt<<<ew_blocks(n), 256, 0, s>>>(x, n, dev_norm2); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

osmps_status vec_scale_by_inv(double* y, const double* x, int64_t n, const double* dev_div,
                              cudaStream_t s) {
  { k_scale_inv<<<ew_blocks(n), 256, 0, s>>>(y, x, n, dev_div); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  return OSMPS_OK;
}

__global__ void k_nonfinite(const double* __restrict__ x, int64_t n, int* __restrict__ flag) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 4);
}

osmps_status check_finite(osmps_ctx* ctx, const double* x, int64_t n, cudaStream_t s, bool* ok) {
  OSMPS_CUDA(cudaMemsetAsync(ctx->dev_flags + 1, 0, sizeof(int), s));
  { k_nonfinite<<<ew_blocks(n), 256, 0, s>>>(x, n, ctx->dev_flags + 1); note_launch(); }
  OSMPS_LAUNCH_CHECK();
  int h = 0;
  OSMPS_CUDA(cudaMemcpyAsync(&h, ctx->dev_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  OSMPS_CUDA(cudaStreamSynchronize(s));
  *ok = (h == 0);
  return OSMPS_OK;
}

}  // namespace osmps

using namespace osmps;

extern "C" {

const char* osmps_last_error(void) { return g_err; }

const char* osmps_status_string(osmps_status s) {
  switch (s) {
    case OSMPS_OK: return "OSMPS_OK";
    case OSMPS_EINVAL: return "OSMPS_EINVAL";
    case OSMPS_ESHAPE: return "OSMPS_ESHAPE";
    case OSMPS_ENOMEM: return "OSMPS_ENOMEM";
    case OSMPS_ECUDA: return "OSMPS_ECUDA";
    case OSMPS_ENOCONV: return "OSMPS_ENOCONV";
    case OSMPS_ETIMEOUT: return "OSMPS_ETIMEOUT";
    case OSMPS_ENAN: return "OSMPS_ENAN";
    case OSMPS_EUNSUPPORTED: return "OSMPS_EUNSUPPORTED";
  }
  return "OSMPS_UNKNOWN";
}

osmps_status osmps_ctx_create(int device, size_t ws_bytes, osmps_ctx** out) {
  clear_error();
  if (!out) return set_error(OSMPS_EINVAL, "osmps_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_error(OSMPS_ECUDA, "osmps_ctx_create: no CUDA device (%s)", cudaGetErrorString(e));
  }
  if (device < 0 || device >= ndev)
    return set_error(OSMPS_EINVAL, "osmps_ctx_create: device %d out of range [0,%d)", device, ndev);
  OSMPS_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  OSMPS_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major < 10)
    return set_error(OSMPS_EUNSUPPORTED, "osmps_ctx_create: device %d is sm_%d%d; sm_103 required",
                     device, prop.major, prop.minor);
  osmps_ctx* ctx = new osmps_ctx();
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  if (cudaMalloc(&ctx->dev_flags, 16 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->dev_info, 16 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    osmps_ctx_destroy(ctx);
    return set_error(OSMPS_ENOMEM, "osmps_ctx_create: flag allocation failed");
  }
  cudaMemset(ctx->dev_flags, 0, 16 * sizeof(int));
  cudaMemset(ctx->dev_info, 0, 16 * sizeof(int));
  if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS) {
    osmps_ctx_destroy(ctx);
    return set_error(OSMPS_ECUDA, "osmps_ctx_create: cusolverDnCreate failed");
  }
  if (ws_bytes > 0) {
    osmps_status st = OSMPS_OK;
    if (!ws_get(ctx, SLOT_HEFF_T1, ws_bytes, 0, &st)) {
      osmps_ctx_destroy(ctx);
      return st;
    }
  }
  osmps_status st = pinned_reserve(ctx, 4096);
  if (st != OSMPS_OK) {
    osmps_ctx_destroy(ctx);
    return st;
  }
  *out = ctx;
  return OSMPS_OK;
}

osmps_status osmps_ctx_destroy(osmps_ctx* ctx) {
  if (!ctx) return OSMPS_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& r : ctx->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < SLOT_COUNT; ++i)
    if (ctx->slots[i].ptr) cudaFree(ctx->slots[i].ptr);
  if (ctx->dev_flags) cudaFree(ctx->dev_flags);
  if (ctx->dev_info) cudaFree(ctx->dev_info);
  if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
  if (ctx->solver) cusolverDnDestroy(ctx->solver);
  for (auto& gr : ctx->lz_graphs) {
    if (gr.e) cudaGraphExecDestroy(gr.e);
    if (gr.g) cudaGraphDestroy(gr.g);
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
  return OSMPS_OK;
}

osmps_status osmps_profile_enable(osmps_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) return set_error(OSMPS_EINVAL, "osmps_profile_enable: null context");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  OSMPS_CUDA(cudaDeviceSynchronize());
  for (auto& r : ctx->prof) {
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof.clear();
  ctx->prof_on = enable != 0;
  return OSMPS_OK;
}

osmps_status osmps_profile_read(osmps_ctx* ctx, int kernel, int64_t* launches, double* total_ms,
                                double* flops, double* tensor_flops) {
  clear_error();
  if (!ctx || !launches || !total_ms || !flops || !tensor_flops)
    return set_error(OSMPS_EINVAL, "osmps_profile_read: null argument");
  OSMPS_CUDA(cudaSetDevice(ctx->device));
  OSMPS_CUDA(cudaDeviceSynchronize());
  int64_t n = 0;
  double ms = 0.0, f = 0.0, tf = 0.0;
  for (auto& r : ctx->prof) {
    if (r.kernel != kernel) continue;
    float t = 0.0f;
    OSMPS_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    ++n;
    ms += t;
    f += r.flops;
    tf += r.tensor_flops;
  }
  *launches = n;
  *total_ms = ms;
  *flops = f;
  *tensor_flops = tf;
  return OSMPS_OK;
}

int64_t osmps_kernel_launches(void) { return (int64_t)g_launches.load(); }

size_t osmps_ctx_workspace_bytes(const osmps_ctx* ctx) {
  if (!ctx) return 0;
  size_t t = 0;
  for (int i = 0; i < SLOT_COUNT; ++i) t += ctx->slots[i].bytes;
  return t;
}

}  // extern "C"

extern "C" osmps_status osmps_ctx_set_eig_solver(osmps_ctx* ctx, int solver) {
  osmps::clear_error();
  if (!ctx) return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_eig_solver: null context");
  if (solver < OSMPS_EIG_AUTO || solver > OSMPS_EIG_TRIDIAG)
    return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_eig_solver: solver %d", solver);
  ctx->eig_solver = solver;
  return OSMPS_OK;
}

extern "C" osmps_status osmps_ctx_set_identity_skip(osmps_ctx* ctx, int mode) {
  osmps::clear_error();
  if (!ctx) return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_identity_skip: null context");
  if (mode < OSMPS_IDENTITY_OFF || mode > OSMPS_IDENTITY_ALWAYS)
    return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_identity_skip: mode %d", mode);
  ctx->identity_skip = mode;
  return OSMPS_OK;
}

extern "C" osmps_status osmps_ctx_set_lanczos_mode(osmps_ctx* ctx, int mode) {
  osmps::clear_error();
  if (!ctx) return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_lanczos_mode: null context");
  if (mode < OSMPS_LANCZOS_AUTO || mode > OSMPS_LANCZOS_GRAPH)
    return osmps::set_error(OSMPS_EINVAL, "osmps_ctx_set_lanczos_mode: mode %d", mode);
  ctx->lanczos_mode = mode;
  return OSMPS_OK;
}
