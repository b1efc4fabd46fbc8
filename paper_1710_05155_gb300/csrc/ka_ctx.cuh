// ka_ctx.cuh -- the context behind the opaque ka_ctx handle of include/ka.h.
#pragma once

#include <string>
#include <vector>

#include "ka_internal.cuh"

struct ka_ctx {
  ka_params prm;
  int topo = 0, d = 0, L = 0, z = 0, m = 0, R = 0;
  int64_t N = 0, nclass = 0, nbonds = 0;
  bool pencil = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool owns = false;
  void* buf = nullptr;
  size_t bytes = 0;
  ka::Planes pl{};
  ka::InitScratch is{};
  unsigned long long* counts_dev = nullptr;
  int* err_dev = nullptr;  // device error word of bounded device waits (0 = none)
  uint64_t* stage = nullptr;
  ka::GraphDev g{};
  ka::Topology host;  // class offsets (graphs) and tables for inspection
  bool initialized = false;
  int64_t sweep = 0, K = -1;
  uint64_t seed = 0;
  ka::RoundKeys rk{};
  std::string err;
  // kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_dir;  // direction of every recorded event pair
  size_t ev_used = 0;
  double prof_ms[4] = {0.0, 0.0, 0.0, 0.0};  // by direction mu (graph classes: 0)
  int64_t prof_launches[4] = {0, 0, 0, 0};
};

namespace ka {
// Creates a context in a caller-provided (or owned) device buffer; defined in ka_api.cu.
ka_status create_context(const ka_params* params, void* buf, size_t bytes, bool owns, ka_ctx** out);
// Device bytes a context needs; defined in ka_api.cu.
ka_status context_bytes(const ka_params* params, size_t* bytes);
}  // namespace ka
