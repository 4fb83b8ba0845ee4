// Many independent chains on one GPU: the paper's data parallelism over
// independent simulations (appendix "Convenient features", the MPI item: a
// master hands jobs to workers one by one, largest systems first, so that no
// worker is left with a long job at the end).
//
// A native work queue: n_workers host threads, each owning one context
// (workspace, cuSOLVER handle) and one non-blocking stream, take chains in
// decreasing order of estimated cost and run the full sweep schedule of each
// (osmps_sweep). The GPU overlaps the chains' kernels across streams, which
// hides the per-step host synchronisations and fills the SMs that a single
// small chain leaves idle.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "handles.cuh"

namespace osmps {
namespace {

// Work estimate of one chain: sum over bonds of chi_max(bond)^3 (the H_eff
// and split cost per step), times the number of sweeps.
double chain_cost(const osmps_mps* m, const osmps_sweep_params& p) {
  double c = 0.0;
  for (int64_t k = 1; k < m->L; ++k) {
    const double x = (double)std::min<int64_t>(m->cap[k], p.chi_max);
    c += x * x * x;
  }
  return c * (double)std::max(1, p.n_sweeps + p.refine_sweeps);
}

}  // namespace
}  // namespace osmps

using namespace osmps;

extern "C" osmps_status osmps_sweep_batch(osmps_ctx* const* ctxs, int n_workers,
                                          osmps_mps* const* mps, const osmps_mpo* const* mpo,
                                          const osmps_sweep_params* params, int64_t n_chains,
                                          osmps_sweep_stats* stats, osmps_status* chain_status) {
  clear_error();
  if (!ctxs || n_workers < 1 || n_chains < 0 || (n_chains > 0 && (!mps || !mpo || !params)))
    return set_error(OSMPS_EINVAL, "osmps_sweep_batch: null argument or no worker");
  for (int w = 0; w < n_workers; ++w) {
    if (!ctxs[w]) return set_error(OSMPS_EINVAL, "osmps_sweep_batch: context %d is NULL", w);
    if (ctxs[w]->device != ctxs[0]->device)
      return set_error(OSMPS_EINVAL, "osmps_sweep_batch: contexts on different devices");
    for (int v = 0; v < w; ++v)
      if (ctxs[v] == ctxs[w])
        return set_error(OSMPS_EINVAL, "osmps_sweep_batch: context %d used by two workers", w);
  }
  for (int64_t i = 0; i < n_chains; ++i) {
    if (!mps[i] || !mpo[i]) return set_error(OSMPS_EINVAL, "osmps_sweep_batch: chain %lld is NULL", (long long)i);
    for (int64_t j = 0; j < i; ++j)
      if (mps[j] == mps[i])
        return set_error(OSMPS_EINVAL, "osmps_sweep_batch: chains %lld and %lld share an MPS",
                         (long long)j, (long long)i);
  }
  if (chain_status)
    for (int64_t i = 0; i < n_chains; ++i) chain_status[i] = (osmps_status)-1;  // not started
  if (n_chains == 0) return OSMPS_OK;

  std::vector<int64_t> order(n_chains);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(n_chains);
  for (int64_t i = 0; i < n_chains; ++i) cost[i] = chain_cost(mps[i], params[i]);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });

  std::atomic<int64_t> next{0};
  std::atomic<bool> abort{false};
  std::mutex err_mu;
  osmps_status first = OSMPS_OK;
  std::string first_msg;
  const int nw = (int)std::min<int64_t>(n_workers, n_chains);

  auto worker = [&](int w) {
    osmps_ctx* ctx = ctxs[w];
    auto fail = [&](osmps_status st, const char* msg) {
      std::lock_guard<std::mutex> g(err_mu);
      if (first == OSMPS_OK) {
        first = st;
        first_msg = msg;
      }
      abort = true;
    };
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      fail(OSMPS_ECUDA, "osmps_sweep_batch: cudaSetDevice failed in a worker");
      return;
    }
    set_batch_worker(true);  // Lanczos in OSMPS_LANCZOS_AUTO keeps the host loop here
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      fail(OSMPS_ECUDA, "osmps_sweep_batch: stream creation failed");
      return;
    }
    for (;;) {
      if (abort.load()) break;
      const int64_t q = next.fetch_add(1);
      if (q >= n_chains) break;
      const int64_t i = order[q];
      osmps_sweep_stats local;
      std::memset(&local, 0, sizeof(local));
      osmps_sweep_stats* out = stats ? &stats[i] : &local;
      const osmps_status st = osmps_sweep(ctx, mps[i], mpo[i], &params[i], out, (void*)s);
      if (chain_status) chain_status[i] = st;
      if (st != OSMPS_OK) {
        char buf[1200];
        std::snprintf(buf, sizeof(buf), "chain %lld: %s", (long long)i, osmps_last_error());
        fail(st, buf);
      }
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };

  std::vector<std::thread> pool;
  pool.reserve(nw);
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w);
  for (auto& t : pool) t.join();
  if (first != OSMPS_OK) return set_error(first, "osmps_sweep_batch: %s", first_msg.c_str());
  return OSMPS_OK;
}
