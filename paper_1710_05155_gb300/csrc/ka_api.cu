// ka_api.cu -- the C ABI declared in include/ka.h.
//
// A context owns (or borrows) one device buffer carved into: the three state
// planes n, n0, p; the per-replica observable counters; the init scratch;
// and, on the edge-gather path, the neighbour list and the class-ordered
// bond arrays.  All work is issued on the context stream in call order.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ka_ctx.cuh"


namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t n, n0, p, stage, counts, hist, pre_key, pre_idx, krem, unresolved, err, nbr, bu, bv, bid,
      perm, inv, total;
};

struct Shape {
  int topo, d, L, z, m, R, W, V, P, xs;
  int64_t N, E;
  bool pencil;
};

const char* check_params(const ka_params* p, Shape& s) {
  if (!p) return "params is NULL";
  s.topo = p->topo;
  s.m = p->m;
  s.R = p->replicas;
  if (s.R <= 0 || s.R % 64 || s.R > 65536) return "replicas must be a positive multiple of 64, at most 65536";
  s.W = s.R / 64;
  s.V = (s.W % 2 == 0) ? 2 : 1;  // refined below for the cubic pencil kernel
  if (p->topo == KA_CUBIC) {
    s.d = p->d;
    s.L = p->L;
    if (s.d < 1 || s.d > 4) return "cubic: d must be in [1, 4]";
    if (s.L < 4 || s.L % 4) return "cubic: L must be a multiple of 4, at least 4";
    int64_t N = 1;
    for (int k = 0; k < s.d; ++k) {
      N *= s.L;
      if (N >= ((int64_t)1 << 31)) return "cubic: L^d must be below 2^31";
    }
    s.N = N;
    s.z = 2 * s.d;
    s.E = (int64_t)s.d * N;
    s.pencil = !(p->flags & KA_FLAG_GENERIC) && s.L <= 128;
  } else if (p->topo == KA_RRG || p->topo == KA_GRAPH) {
    s.d = 0;
    s.L = 0;
    s.N = p->N;
    s.z = p->z;
    if (s.N < 2 || s.z < 1 || s.z > 8 || s.z >= s.N) return "graph: need N >= 2, 1 <= z <= 8, z < N";
    if ((s.N * s.z) % 2) return "graph: N z must be even";
    if (s.N * s.z > 0xFFFFFFFFLL) return "graph: N z must be below 2^32";
    if (p->topo == KA_GRAPH && !p->nbr) return "KA_GRAPH needs nbr";
    s.E = s.N * s.z / 2;
    s.pencil = false;
  } else {
    return "unknown topology";
  }
  if (s.m < 0 || s.m > s.z - 1) return "m must be in [0, z-1]";
  // words per site and plane: a whole 32-byte sector per site when 4 words
  // fit (the edge-gather kernel's random accesses move whole sectors anyway).
  // Cubic lattices of dimension >= 2 on the pencil kernels keep one word per
  // site and plane in split-row order: a plane's n and p (16 bytes per site)
  // then stay resident in the L2 across the sweeps of that plane, and a
  // group's active sites are whole sectors.
  if (s.W % 4 == 0) s.V = 4;
  s.xs = 0;
  if (s.topo == KA_CUBIC && s.pencil && s.d >= 2) {
    s.V = 1;
    s.xs = ka::split_side(s.d, s.L);
  }
  s.P = s.W / s.V;
  return nullptr;
}

Layout layout_of(const Shape& s) {
  Layout l{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  const size_t plane = (size_t)s.N * s.W * sizeof(uint64_t);
  l.n = take(plane);
  l.n0 = take(plane);
  l.p = take(plane);
  // layout conversion of get/set_state (graphs: breadth-first storage order)
  l.stage = (s.V > 1 || s.xs || s.topo != KA_CUBIC) ? take(plane) : 0;
  l.counts = take((size_t)s.R * 4 * sizeof(unsigned long long));
  l.hist = take((size_t)s.R * 256 * sizeof(uint32_t));
  l.pre_key = take((size_t)s.R * sizeof(uint64_t));
  l.pre_idx = take((size_t)s.R * sizeof(uint32_t));
  l.krem = take((size_t)s.R * sizeof(int64_t));
  l.unresolved = take(sizeof(int32_t));
  l.err = take(sizeof(int32_t));
  if (!s.pencil) {
    l.nbr = take((size_t)s.N * s.z * sizeof(int32_t));
    l.bu = take((size_t)s.E * sizeof(int32_t));
    l.bv = take((size_t)s.E * sizeof(int32_t));
    l.bid = take((size_t)s.E * sizeof(uint32_t));
  }
  if (s.topo != KA_CUBIC) {
    l.perm = take((size_t)s.N * sizeof(int32_t));
    l.inv = take((size_t)s.N * sizeof(int32_t));
  }
  l.total = off;
  return l;
}

ka_status fail(ka_ctx* c, ka_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ka_status cuda_fail(ka_ctx* c, cudaError_t e, const char* what) {
  return fail(c, KA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ka_status create_common(const ka_params* params, void* buf, size_t bytes, bool owns, ka_ctx** out) {
  Shape s{};
  if (const char* e = check_params(params, s)) return KA_EINVAL;
  ka_ctx* c = new ka_ctx();
  c->prm = *params;
  c->prm.nbr = nullptr;
  c->topo = s.topo;
  c->d = s.d;
  c->L = s.L;
  c->z = s.z;
  c->m = s.m;
  c->R = s.R;
  c->N = s.N;
  c->pencil = s.pencil;
  c->stream = (cudaStream_t)params->stream;
  c->device = params->device;
  c->owns = owns;
  c->buf = buf;
  c->bytes = bytes;
  const Layout l = layout_of(s);
  char* base = (char*)buf;
  c->pl.n = (uint64_t*)(base + l.n);
  c->pl.n0 = (uint64_t*)(base + l.n0);
  c->pl.p = (uint64_t*)(base + l.p);
  c->pl.N = s.N;
  c->pl.W = s.W;
  c->pl.V = s.V;
  c->pl.P = s.P;
  c->pl.xs = s.xs;
  c->err_dev = (int*)(base + l.err);
  c->counts_dev = (unsigned long long*)(base + l.counts);
  c->stage = (s.V > 1 || s.xs || s.topo != KA_CUBIC) ? (uint64_t*)(base + l.stage) : nullptr;
  c->is.hist = (uint32_t*)(base + l.hist);
  c->is.pre_key = (uint64_t*)(base + l.pre_key);
  c->is.pre_idx = (uint32_t*)(base + l.pre_idx);
  c->is.krem = (int64_t*)(base + l.krem);
  c->is.unresolved = (int32_t*)(base + l.unresolved);
  c->is.cand = c->stage ? (uint32_t*)c->stage : nullptr;  // idle during init
  c->is.cand_bytes = c->stage ? (size_t)s.N * s.W * sizeof(uint64_t) : 0;

  {
    const cudaError_t ez = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
    if (ez || cudaStreamSynchronize(c->stream)) {
      if (owns) cudaFree(buf);
      delete c;
      return KA_ECUDA;
    }
  }
  std::string msg;
  if (s.topo == KA_CUBIC) {
    c->nclass = (s.d == 1) ? 4 : 8 * s.d;
    c->nbonds = s.E;
    if (!s.pencil) msg = ka::build_cubic_tables(s.d, s.L, c->host);
  } else if (s.topo == KA_RRG) {
    msg = ka::build_rrg(s.N, s.z, params->graph_seed, c->host);
  } else {
    msg = ka::build_graph(s.N, s.z, params->nbr, c->host);
  }
  if (!msg.empty()) {
    if (owns) cudaFree(buf);
    delete c;
    return KA_EINVAL;
  }
  if (!s.pencil) {
    c->nclass = c->host.nclass();
    c->nbonds = (int64_t)c->host.bu.size();
    c->g.nbr = (const int32_t*)(base + l.nbr);
    c->g.bu = (const int32_t*)(base + l.bu);
    c->g.bv = (const int32_t*)(base + l.bv);
    c->g.bid = (const uint32_t*)(base + l.bid);
    c->g.z = s.z;
    c->g.m = s.m;
    c->g.cubic_L = (s.topo == KA_CUBIC) ? s.L : 0;
    // Device tables.  Graphs keep their sites in breadth-first order: the
    // neighbour rows, the bonds (sorted by position inside each class) and
    // the planes use storage positions; bond ids, classes and the state
    // layout of the ABI stay canonical.  Cubic lattices on this path keep
    // index order.
    std::vector<int32_t> perm, inv, nbr_d, bu_d, bv_d;
    std::vector<uint32_t> bid_d;
    if (s.topo != KA_CUBIC) {
      ka::bfs_order(s.N, s.z, c->host.nbr.data(), perm, inv);
      ka::relabel_tables(c->host, s.z, perm, nbr_d, bu_d, bv_d, bid_d);
      c->g.perm = (const int32_t*)(base + l.perm);
      c->pl.inv = (const int32_t*)(base + l.inv);
    } else {
      nbr_d = c->host.nbr;
      bu_d = c->host.bu;
      bv_d = c->host.bv;
      bid_d.assign(c->host.bid.begin(), c->host.bid.end());
    }
    cudaError_t e = cudaMemcpyAsync((void*)c->g.nbr, nbr_d.data(), nbr_d.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync((void*)c->g.bu, bu_d.data(), bu_d.size() * 4,
                                cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync((void*)c->g.bv, bv_d.data(), bv_d.size() * 4,
                                cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync((void*)c->g.bid, bid_d.data(), bid_d.size() * 4,
                                cudaMemcpyHostToDevice, c->stream);
    if (!e && c->g.perm)
      e = cudaMemcpyAsync((void*)c->g.perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice,
                          c->stream);
    if (!e && c->pl.inv)
      e = cudaMemcpyAsync((void*)c->pl.inv, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice,
                          c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
      if (owns) cudaFree(buf);
      delete c;
      return KA_ECUDA;
    }
  }
  *out = c;
  return KA_OK;
}

cudaEvent_t next_event(ka_ctx* c) {
  if (c->ev_used == c->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev.push_back(e);
  }
  return c->ev[c->ev_used++];
}

// Start timing one sweep-kernel launch of direction dir when profiling is
// on: records the first event of a pair and returns the second (nullptr when
// off), which the caller records after the launch.
cudaEvent_t prof_begin(ka_ctx* c, int dir) {
  if (!c->prof) return nullptr;
  cudaEvent_t e0 = next_event(c), e1 = next_event(c);
  if (!e0 || !e1) return nullptr;
  c->ev_dir.push_back(dir);
  cudaEventRecord(e0, c->stream);
  return e1;
}

// accumulate the elapsed time of recorded event pairs by direction
ka_status drain_profile(ka_ctx* c) {
  if (c->ev_used == 0) return KA_OK;
  cudaError_t e = cudaEventSynchronize(c->ev[c->ev_used - 1]);
  if (e) return cuda_fail(c, e, "profile sync");
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
    if (e) return cuda_fail(c, e, "profile elapsed");
    const int dir = c->ev_dir[k / 2];
    c->prof_ms[dir] += ms;
    c->prof_launches[dir]++;
  }
  c->ev_used = 0;
  c->ev_dir.clear();
  return KA_OK;
}

// Read (and clear) the device error word of the bounded waits; synchronises
// the context stream.  KA_ETIMEOUT when a wait ran out since the last check.
ka_status check_device_error(ka_ctx* c) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "sync");
  if (h) {
    e = cudaMemsetAsync(c->err_dev, 0, sizeof(int), c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "sync");
    return fail(c, KA_ETIMEOUT,
                std::string("a bounded device wait ran out (code ") +
                    std::to_string(h) + "); the state of this context is not valid");
  }
  return KA_OK;
}

}  // namespace

namespace ka {
ka_status create_context(const ka_params* params, void* buf, size_t bytes, bool owns, ka_ctx** out) {
  return create_common(params, buf, bytes, owns, out);
}
ka_status context_bytes(const ka_params* params, size_t* bytes) {
  Shape s{};
  if (!bytes || check_params(params, s)) return KA_EINVAL;
  *bytes = layout_of(s).total;
  return KA_OK;
}
}  // namespace ka

extern "C" {

const char* ka_status_name(ka_status s) {
  switch (s) {
    case KA_OK: return "KA_OK";
    case KA_EINVAL: return "KA_EINVAL";
    case KA_ENOMEM: return "KA_ENOMEM";
    case KA_ECUDA: return "KA_ECUDA";
    case KA_ETIMEOUT: return "KA_ETIMEOUT";
    case KA_EBUSY: return "KA_EBUSY";
    case KA_ESTATE: return "KA_ESTATE";
  }
  return "KA_UNKNOWN";
}

ka_status ka_required_bytes(const ka_params* params, size_t* bytes) {
  Shape s{};
  if (!bytes || check_params(params, s)) return KA_EINVAL;
  *bytes = layout_of(s).total;
  return KA_OK;
}

ka_status ka_create(const ka_params* params, ka_ctx** out) {
  if (!out) return KA_EINVAL;
  *out = nullptr;
  Shape s{};
  if (check_params(params, s)) return KA_EINVAL;
  DeviceGuard dg(params->device);
  const size_t bytes = layout_of(s).total;
  void* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return KA_ENOMEM;
  }
  return create_common(params, buf, bytes, true, out);
}

ka_status ka_create_in(const ka_params* params, void* device_buffer, size_t bytes, ka_ctx** out) {
  if (!out) return KA_EINVAL;
  *out = nullptr;
  Shape s{};
  if (check_params(params, s) || !device_buffer) return KA_EINVAL;
  if ((uintptr_t)device_buffer % kAlign) return KA_EINVAL;
  if (bytes < layout_of(s).total) return KA_ENOMEM;
  DeviceGuard dg(params->device);
  return create_common(params, device_buffer, bytes, false, out);
}

ka_status ka_init(ka_ctx* c, uint64_t seed, double rho) {
  ka::NvtxRange nvtx_range("ka_init");
  if (!c) return KA_EINVAL;
  if (!(rho >= 0.0 && rho <= 1.0)) return fail(c, KA_EINVAL, "rho must be in [0, 1]");
  DeviceGuard dg(c->device);
  const int64_t K = (int64_t)floor(rho * (double)c->N + 0.5);
  c->seed = seed;
  c->rk = ka::round_keys(seed);
  cudaError_t e = ka::launch_init(c->pl, c->is, c->R, K, c->rk, c->stream);
  if (e) return cuda_fail(c, e, "init");
  c->K = K;
  c->sweep = 0;
  c->initialized = true;
  return KA_OK;
}

ka_status ka_sweep(ka_ctx* c, int64_t n) {
  ka::NvtxRange nvtx_range("ka_sweep");
  if (!c || n < 0) return c ? fail(c, KA_EINVAL, "n must be >= 0") : KA_EINVAL;
  if (!c->initialized) return fail(c, KA_ESTATE, "sweep before init or set_state");
  if (c->sweep + n > ((int64_t)1 << 32)) return fail(c, KA_EINVAL, "sweep counter would pass 2^32");
  if (n == 0) return KA_OK;
  DeviceGuard dg(c->device);
  cudaError_t e = cudaSuccess;
  if (c->pencil && ka::stream_preferred(c->d, c->L, c->pl.P)) {
    // plane-outer order keeps the planes of one launch resident in the L2
    // across sweeps
    const int nq = ka::stream_planes_per_launch(c->L, c->pl.P);
    for (int q0 = 0; q0 < c->pl.P && !e; q0 += nq) {
      const int cnt = std::min(nq, c->pl.P - q0);
      for (int64_t s = 0; s < n && !e; ++s)
        for (int mu = 0; mu < 3 && !e; ++mu)
          for (int par = 0; par < 2 && !e; ++par) {
            cudaEvent_t e1 = prof_begin(c, mu);
            e = ka::launch_stream_group(c->pl, q0, cnt, c->L, c->m, mu, par,
                                        (uint32_t)(c->sweep + s), c->rk, c->stream);
            if (e1) cudaEventRecord(e1, c->stream);
          }
    }
  } else if (c->pencil) {
    const ka::CubicShape sh{c->d, c->L, c->m};
    const int npar = (c->d == 1) ? 1 : 2;
    // plane-outer order keeps one plane's n and p resident in L2 across sweeps
    for (int q = 0; q < c->pl.P && !e; ++q)
      for (int64_t s = 0; s < n && !e; ++s)
        for (int mu = 0; mu < c->d && !e; ++mu)
          for (int par = 0; par < npar && !e; ++par) {
            cudaEvent_t e1 = prof_begin(c, mu);
            e = ka::launch_cubic_group(c->pl, q, sh, mu, par, (uint32_t)(c->sweep + s), c->rk,
                                       c->stream);
            if (e1) cudaEventRecord(e1, c->stream);
          }
  } else {
    for (int64_t s = 0; s < n && !e; ++s)
      for (int64_t cl = 0; cl < c->nclass && !e; ++cl) {
        cudaEvent_t e1 = prof_begin(c, 0);
        const int64_t off = c->host.class_off[cl];
        e = ka::launch_graph_class(c->pl, c->g, off, c->host.class_off[cl + 1] - off,
                                   (uint32_t)cl, (uint32_t)(c->sweep + s), c->rk, c->stream);
        if (e1) cudaEventRecord(e1, c->stream);
      }
  }
  if (e) return cuda_fail(c, e, "sweep launch");
  c->sweep += n;
  return KA_OK;
}

ka_status ka_observe_device(ka_ctx* c, int64_t* counts_device) {
  ka::NvtxRange nvtx_range("ka_observe");
  if (!c || !counts_device) return KA_EINVAL;
  if (!c->initialized) return fail(c, KA_ESTATE, "observe before init or set_state");
  DeviceGuard dg(c->device);
  cudaError_t e = ka::launch_observe(c->pl, c->R, (unsigned long long*)counts_device, c->stream);
  if (e) return cuda_fail(c, e, "observe");
  return KA_OK;
}

ka_status ka_observe(ka_ctx* c, int64_t* sweep_out, int64_t* counts) {
  ka::NvtxRange nvtx_range("ka_observe");
  if (!c || !counts) return KA_EINVAL;
  if (!c->initialized) return fail(c, KA_ESTATE, "observe before init or set_state");
  DeviceGuard dg(c->device);
  cudaError_t e = ka::launch_observe(c->pl, c->R, c->counts_dev, c->stream);
  if (!e) e = cudaMemcpyAsync(counts, c->counts_dev, (size_t)c->R * 4 * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, c->stream);
  if (e) return cuda_fail(c, e, "observe");
  if (ka_status st = check_device_error(c)) return st;
  if (sweep_out) *sweep_out = c->sweep;
  return KA_OK;
}

ka_status ka_get_state(ka_ctx* c, uint64_t* n, uint64_t* n0, uint64_t* p) {
  ka::NvtxRange nvtx_range("ka_get_state");
  if (!c) return KA_EINVAL;
  DeviceGuard dg(c->device);
  const size_t bytes = (size_t)c->pl.P * c->pl.plane_elems() * sizeof(uint64_t);
  uint64_t* dst[3] = {n, n0, p};
  const uint64_t* src[3] = {c->pl.n, c->pl.n0, c->pl.p};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && !e; ++k) {
    if (!dst[k]) continue;
    const uint64_t* from = src[k];
    if (c->stage) {
      e = ka::launch_to_canonical(src[k], c->stage, c->N, c->pl.P, c->pl.V, c->pl.xs, c->pl.inv,
                                  c->stream);
      from = c->stage;
    }
    // stream order keeps the next conversion from overwriting the staging
    // plane before this copy has read it
    if (!e) e = cudaMemcpyAsync(dst[k], from, bytes, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e) return cuda_fail(c, e, "get_state");
  return check_device_error(c);
}

}  // extern "C"

namespace {

// Queue the copies of a canonical-layout state onto the context's stream;
// synchronises when sync.
ka_status set_state_impl(ka_ctx* c, const uint64_t* n, const uint64_t* n0, const uint64_t* p,
                         int64_t sweep, uint64_t seed, bool sync) {
  if (!c || !n || !n0 || !p || sweep < 0 || sweep >= ((int64_t)1 << 32)) return KA_EINVAL;
  DeviceGuard dg(c->device);
  const size_t bytes = (size_t)c->pl.P * c->pl.plane_elems() * sizeof(uint64_t);
  const uint64_t* src[3] = {n, n0, p};
  uint64_t* dst[3] = {c->pl.n, c->pl.n0, c->pl.p};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && !e; ++k) {
    if (c->stage) {
      // stream order keeps the next copy from overwriting the staging plane
      // before the conversion has read it
      e = cudaMemcpyAsync(c->stage, src[k], bytes, cudaMemcpyHostToDevice, c->stream);
      if (!e)
        e = ka::launch_to_device(c->stage, dst[k], c->N, c->pl.P, c->pl.V, c->pl.xs, c->pl.inv,
                                 c->stream);
    } else {
      e = cudaMemcpyAsync(dst[k], src[k], bytes, cudaMemcpyHostToDevice, c->stream);
    }
  }
  if (!e && sync) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "set_state");
  c->sweep = sweep;
  c->seed = seed;
  c->rk = ka::round_keys(seed);
  c->K = -1;
  c->initialized = true;
  return KA_OK;
}

}  // namespace

extern "C" {

ka_status ka_set_state(ka_ctx* c, const uint64_t* n, const uint64_t* n0, const uint64_t* p,
                       int64_t sweep, uint64_t seed) {
  ka::NvtxRange nvtx_range("ka_set_state");
  return set_state_impl(c, n, n0, p, sweep, seed, true);
}

ka_status ka_set_state_async(ka_ctx* c, const uint64_t* n, const uint64_t* n0, const uint64_t* p,
                             int64_t sweep, uint64_t seed) {
  ka::NvtxRange nvtx_range("ka_set_state_async");
  return set_state_impl(c, n, n0, p, sweep, seed, false);
}

ka_status ka_sync(ka_ctx* c) {
  if (!c) return KA_EINVAL;
  DeviceGuard dg(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "sync");
  return check_device_error(c);
}

ka_status ka_info(const ka_ctx* c, ka_info_t* out) {
  if (!c || !out) return KA_EINVAL;
  out->N = c->N;
  out->z = c->z;
  out->m = c->m;
  out->replicas = c->R;
  out->words = c->R / 64;
  out->nclass = c->nclass;
  out->nbonds = c->nbonds;
  out->sweep = c->sweep;
  out->K = c->K;
  out->seed = c->seed;
  out->kernel = !c->pencil ? 1 : ka::stream_preferred(c->d, c->L, c->pl.P) ? 3 : 0;
  out->rrg_attempts = c->host.attempts;
  out->device_bytes = c->bytes;
  out->planes = c->pl.P;
  out->plane_words = c->pl.V;
  out->planes_per_launch =
      (c->pencil && ka::stream_preferred(c->d, c->L, c->pl.P)) ? ka::stream_planes_per_launch(c->L, c->pl.P)
                                                                : 1;
  return KA_OK;
}

ka_status ka_graph_tables(const ka_ctx* c, int32_t* nbr, int64_t* class_off, int32_t* bu,
                          int32_t* bv, int64_t* bid) {
  if (!c) return KA_EINVAL;
  ka::Topology local;
  const ka::Topology* t = &c->host;
  if (c->pencil) {
    if (!ka::build_cubic_tables(c->d, c->L, local).empty()) return KA_EINVAL;
    t = &local;
  }
  if (nbr) std::memcpy(nbr, t->nbr.data(), t->nbr.size() * sizeof(int32_t));
  if (class_off) std::memcpy(class_off, t->class_off.data(), t->class_off.size() * sizeof(int64_t));
  if (bu) std::memcpy(bu, t->bu.data(), t->bu.size() * sizeof(int32_t));
  if (bv) std::memcpy(bv, t->bv.data(), t->bv.size() * sizeof(int32_t));
  if (bid) std::memcpy(bid, t->bid.data(), t->bid.size() * sizeof(int64_t));
  return KA_OK;
}

ka_status ka_build_topology(const ka_params* params, int64_t* nclass, int64_t* nbonds, int32_t* nbr,
                      int64_t* class_off, int32_t* bu, int32_t* bv, int64_t* bid) {
  Shape s{};
  if (check_params(params, s)) return KA_EINVAL;
  ka::Topology t;
  std::string msg;
  if (s.topo == KA_CUBIC)
    msg = ka::build_cubic_tables(s.d, s.L, t);
  else if (s.topo == KA_RRG)
    msg = ka::build_rrg(s.N, s.z, params->graph_seed, t);
  else
    msg = ka::build_graph(s.N, s.z, params->nbr, t);
  if (!msg.empty()) return KA_EINVAL;
  if (nclass) *nclass = t.nclass();
  if (nbonds) *nbonds = (int64_t)t.bu.size();
  if (nbr) std::memcpy(nbr, t.nbr.data(), t.nbr.size() * sizeof(int32_t));
  if (class_off) std::memcpy(class_off, t.class_off.data(), t.class_off.size() * sizeof(int64_t));
  if (bu) std::memcpy(bu, t.bu.data(), t.bu.size() * sizeof(int32_t));
  if (bv) std::memcpy(bv, t.bv.data(), t.bv.size() * sizeof(int32_t));
  if (bid) std::memcpy(bid, t.bid.data(), t.bid.size() * sizeof(int64_t));
  return KA_OK;
}

ka_status ka_profile_enable(ka_ctx* c, int32_t enable) {
  if (!c) return KA_EINVAL;
  if (!enable) {
    ka_status s = drain_profile(c);
    if (s) return s;
  }
  c->prof = enable != 0;
  return KA_OK;
}

ka_status ka_profile_read(ka_ctx* c, double* kernel_ms, int64_t* launches) {
  if (!c) return KA_EINVAL;
  DeviceGuard dg(c->device);
  ka_status s = drain_profile(c);
  if (s) return s;
  double ms = 0.0;
  int64_t nl = 0;
  for (int k = 0; k < 4; ++k) {
    ms += c->prof_ms[k];
    nl += c->prof_launches[k];
    c->prof_ms[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  if (kernel_ms) *kernel_ms = ms;
  if (launches) *launches = nl;
  return KA_OK;
}

ka_status ka_profile_read_dirs(ka_ctx* c, double* kernel_ms, int64_t* launches) {
  if (!c) return KA_EINVAL;
  DeviceGuard dg(c->device);
  ka_status s = drain_profile(c);
  if (s) return s;
  for (int k = 0; k < 4; ++k) {
    if (kernel_ms) kernel_ms[k] = c->prof_ms[k];
    if (launches) launches[k] = c->prof_launches[k];
    c->prof_ms[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  return KA_OK;
}

ka_status ka_destroy(ka_ctx* c) {
  if (!c) return KA_OK;
  DeviceGuard dg(c->device);
  ka_status st = KA_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) st = KA_ECUDA;
  else st = check_device_error(c);
  for (cudaEvent_t ev : c->ev) cudaEventDestroy(ev);
  if (c->owns && c->buf) cudaFree(c->buf);
  delete c;
  return st;
}

const char* ka_last_error(const ka_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

}  // extern "C"
