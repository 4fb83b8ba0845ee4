// Device-resident chain handles (osmps_mps, osmps_mpo), shared by the sweep
// and the batch scheduler.
#pragma once

#include <vector>

#include "common.cuh"

struct osmps_mps {
  osmps_ctx* ctx = nullptr;
  int64_t L = 0;
  std::vector<int64_t> d, chi, cap;
  std::vector<double*> A;
  std::vector<double*> Lenv, Renv;  // bond k: (cap[k], w[k], cap[k])
  std::vector<int64_t> env_w;       // MPO bond dims the environments were sized for
  std::vector<char> lvalid, rvalid;
  int64_t center = -1;
};

struct osmps_mpo {
  osmps_ctx* ctx = nullptr;
  int64_t L = 0;
  std::vector<int64_t> d, w;
  std::vector<double*> W;
  std::vector<double*> ident;  // per site: identity operator (1, d, d, 1) for norms
};
