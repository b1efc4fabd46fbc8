// ka_batch.cu -- many independent jobs advanced together (include/ka.h, batch API).
//
// Every job is an ordinary context (own device buffer, topology, seed,
// density, replica count) plus a device buffer of observations.  A round
// advances all unfinished jobs by up to k sweeps: for every sweep offset s
// and every bond-class group, ONE launch covers all work units (job planes)
// of a shape class: the group kernels of three-dimensional lattices for the
// units of one side and m (d = 3), the general pencil kernel for the cubic
// units of one (d, V, m) otherwise; and ONE launch of the edge-gather kernel
// covers class c of all graph units of a shape class (V, m).  Units carry their own sweep counter t_base and stop counter t_end
// in a device table, so a job that reaches its next observation point (or
// its target) inside the round simply idles.  The round's launch sequence
// can be captured in a CUDA graph and replayed while the job set and the
// round length stay the same (the unit tables are refreshed by a copy before
// every replay).
#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ka_ctx.cuh"

namespace {

struct Job {
  int64_t id = 0;
  ka_ctx* ctx = nullptr;
  void* buf = nullptr;
  size_t bytes = 0;
  int64_t target = 0, every = 1, t = 0;
  int64_t n_obs = 0, cap = 0;
  int64_t* obs_dev = nullptr;  // [cap][R][4]
  std::vector<int64_t> obs_t;
  bool finished = false;
  bool batched = true;  // false: runs with its own (single-instance) launches inside each round
};

struct CubicClass {
  int d = 0, V = 0, m = 0;
  std::vector<ka::CubicUnit> units;
  std::vector<Job*> owner;
  ka::CubicUnit* dev = nullptr;
  uint32_t* tile_unit_dev[2] = {nullptr, nullptr};  // unit of every global tile, per kind
  uint32_t ntiles[2] = {0, 0};
  int PSmax = 0;
};

// Jobs on three-dimensional lattices of one side L and activation number m:
// one entry of the group kernels' unit table per plane (ka_cubic_stream.cuh).
struct StreamClass {
  int L = 0, m = 0;
  std::vector<unsigned char> units;  // host copy, stream_unit_bytes() per unit
  std::vector<Job*> owner;
  std::vector<int> plane;
  void* dev = nullptr;
  size_t count() const { return owner.size(); }
};

struct GraphClass {
  int V = 0, m = 0, cmax = 0;
  std::vector<ka::GraphUnit> units;
  std::vector<Job*> owner;
  std::vector<int64_t> prefix, first, total;  // per class: [cmax][n+1], [cmax][n], [cmax]
  ka::GraphUnit* dev = nullptr;
  int64_t* prefix_dev = nullptr;
  int64_t* first_dev = nullptr;
};

uint32_t cubic_tiles(int d, int L, int V, bool x) {
  const int tp = ka::kCubicWarps / V, win = 2 * tp;
  int64_t np = 1;
  for (int k = 0; k < d - 1; ++k) np *= L;
  if (d >= 2) np /= 2;
  if (x) return (uint32_t)((np + tp - 1) / tp);
  int64_t t = (L + win - 1) / win;
  for (int k = 0; k < d - 2; ++k) t *= L;
  return (uint32_t)t;
}

}  // namespace

struct ka_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0, used = 0;
  int32_t flags = 0;
  int64_t next_id = 1;
  std::map<int64_t, Job*> jobs;
  bool dirty = true;         // jobs were added: the tables must be rebuilt
  int64_t units = 0;         // units in the tables
  int64_t idle_units = 0;    // of which belong to finished or removed jobs
  std::vector<CubicClass> cubic;
  std::vector<StreamClass> sclass;  // three-dimensional lattices: the group kernels
  std::vector<GraphClass> graph;
  std::vector<void*> table_mem;  // device tables of the current job set
  bool own_stream = false;
  cudaGraphExec_t exec = nullptr;
  int64_t exec_k = 0;
  int64_t last_k = 0;  // a round length is captured the second time it is used
  int64_t tuned_k = 16;
  int64_t wave_tiles = 304;  // tiles one persistent launch of the pencil kernel runs at once
  // cubic jobs whose groups have at least this many tiles of the batched
  // pencil kernel run with their own launches (0: one wave, wave_tiles)
  int64_t own_tiles = 0;
  std::string err;
};

namespace {

ka_status cuda_err(ka_batch* b, cudaError_t e, const char* what) {
  b->err = std::string(what) + ": " + cudaGetErrorString(e);
  return KA_ECUDA;
}

void free_tables(ka_batch* b) {
  for (void* p : b->table_mem) cudaFree(p);
  b->table_mem.clear();
  b->cubic.clear();
  b->sclass.clear();
  b->graph.clear();
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->exec_k = 0;
}

template <typename T>
cudaError_t dev_alloc(ka_batch* b, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) b->table_mem.push_back((void*)*p);
  return e;
}

// Group the unfinished batched jobs into shape classes and build the unit
// tables (host copies; device copies are allocated here and filled per round).
cudaError_t rebuild(ka_batch* b) {
  free_tables(b);
  for (auto& kv : b->jobs) {
    Job* j = kv.second;
    if (j->finished || !j->batched) continue;
    ka_ctx* c = j->ctx;
    const int V = c->pl.V;
    for (int q = 0; q < c->pl.P; ++q) {
      uint64_t* n = c->pl.n + (size_t)q * c->pl.plane_elems();
      uint64_t* p = c->pl.p + (size_t)q * c->pl.plane_elems();
      if (c->topo == KA_CUBIC && c->d == 3 && ka::stream_supported(3, c->L) && V == 1 &&
          c->pl.xs == c->L) {
        // three-dimensional lattices: the group kernels, one unit per plane
        StreamClass* sc = nullptr;
        for (auto& x : b->sclass)
          if (x.L == c->L && x.m == c->m) sc = &x;
        if (!sc) {
          b->sclass.push_back(StreamClass{});
          sc = &b->sclass.back();
          sc->L = c->L;
          sc->m = c->m;
        }
        sc->owner.push_back(j);
        sc->plane.push_back(q);
        sc->units.resize(sc->units.size() + ka::stream_unit_bytes());
      } else if (c->topo == KA_CUBIC) {
        CubicClass* cc = nullptr;
        for (auto& x : b->cubic)
          if (x.d == c->d && x.V == V && x.m == c->m) cc = &x;
        if (!cc) {
          b->cubic.push_back(CubicClass{});
          cc = &b->cubic.back();
          cc->d = c->d;
          cc->V = V;
          cc->m = c->m;
        }
        ka::CubicUnit u{};
        u.n = n;
        u.p = p;
        u.d = c->d;
        u.L = c->L;
        u.word0 = (uint32_t)(q * V);
        u.tile0[0] = cc->ntiles[0];
        u.tile0[1] = cc->ntiles[1];
        cc->ntiles[0] += cubic_tiles(c->d, c->L, V, true);
        cc->ntiles[1] += cubic_tiles(c->d, c->L, V, false);
        u.rk = c->rk;
        cc->PSmax = std::max(cc->PSmax, ((c->L + 15) / 16) * 16 + 1);
        cc->units.push_back(u);
        cc->owner.push_back(j);
      } else {
        GraphClass* gc = nullptr;
        for (auto& x : b->graph)
          if (x.V == V && x.m == c->m) gc = &x;
        if (!gc) {
          b->graph.push_back(GraphClass{});
          gc = &b->graph.back();
          gc->V = V;
          gc->m = c->m;
        }
        ka::GraphUnit u{};
        u.n = n;
        u.p = p;
        u.nbr = c->g.nbr;
        u.bu = c->g.bu;
        u.bv = c->g.bv;
        u.bid = c->g.bid;
        u.z = c->z;
        u.word0 = (uint32_t)(q * V);
        u.rk = c->rk;
        gc->units.push_back(u);
        gc->owner.push_back(j);
        gc->cmax = std::max<int>(gc->cmax, (int)c->nclass);
      }
    }
  }
  cudaError_t e = cudaSuccess;
  for (auto& cc : b->cubic) {
    if ((e = dev_alloc(b, &cc.dev, cc.units.size()))) return e;
    for (int mode = 0; mode < 2; ++mode) {
      std::vector<uint32_t> owner(cc.ntiles[mode]);
      for (size_t u = 0; u < cc.units.size(); ++u) {
        const uint32_t end = (u + 1 < cc.units.size()) ? cc.units[u + 1].tile0[mode] : cc.ntiles[mode];
        for (uint32_t g = cc.units[u].tile0[mode]; g < end; ++g) owner[g] = (uint32_t)u;
      }
      if ((e = dev_alloc(b, &cc.tile_unit_dev[mode], owner.size()))) return e;
      if (!owner.empty() &&
          (e = cudaMemcpyAsync(cc.tile_unit_dev[mode], owner.data(), owner.size() * sizeof(uint32_t),
                               cudaMemcpyHostToDevice, b->stream)))
        return e;
      // the host vector must outlive the copy
      if ((e = cudaStreamSynchronize(b->stream))) return e;
    }
  }
  for (auto& sc : b->sclass) {
    unsigned char* d = nullptr;
    if ((e = dev_alloc(b, &d, sc.units.size()))) return e;
    sc.dev = d;
  }
  for (auto& gc : b->graph) {
    const int n = (int)gc.units.size();
    gc.prefix.assign((size_t)gc.cmax * (n + 1), 0);
    gc.first.assign((size_t)gc.cmax * n, 0);
    gc.total.assign(gc.cmax, 0);
    for (int c = 0; c < gc.cmax; ++c) {
      int64_t acc = 0;
      for (int u = 0; u < n; ++u) {
        const ka_ctx* x = gc.owner[u]->ctx;
        int64_t cnt = 0, f = 0;
        if (c < x->nclass) {
          f = x->host.class_off[c];
          cnt = x->host.class_off[c + 1] - f;
        }
        gc.prefix[(size_t)c * (n + 1) + u] = acc;
        gc.first[(size_t)c * n + u] = f;
        acc += cnt;
      }
      gc.prefix[(size_t)c * (n + 1) + n] = acc;
      gc.total[c] = acc;
    }
    if ((e = dev_alloc(b, &gc.dev, gc.units.size()))) return e;
    if ((e = dev_alloc(b, &gc.prefix_dev, gc.prefix.size()))) return e;
    if ((e = dev_alloc(b, &gc.first_dev, gc.first.size()))) return e;
    e = cudaMemcpyAsync(gc.prefix_dev, gc.prefix.data(), gc.prefix.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice, b->stream);
    if (!e) e = cudaMemcpyAsync(gc.first_dev, gc.first.data(), gc.first.size() * sizeof(int64_t),
                                cudaMemcpyHostToDevice, b->stream);
    if (e) return e;
  }
  b->dirty = false;
  b->last_k = 0;
  b->units = 0;
  for (auto& cc : b->cubic) b->units += (int64_t)cc.units.size();
  for (auto& sc : b->sclass) b->units += (int64_t)sc.count();
  for (auto& gc : b->graph) b->units += (int64_t)gc.units.size();
  b->idle_units = 0;
  return cudaStreamSynchronize(b->stream);
}

// Whether a job shares the batched launches: graphs always; a cubic lattice
// on the pencil kernels unless its groups have own_tiles tiles or more (it
// then runs with its own launches inside each round: the group kernels of
// three-dimensional lattices or the single-instance pencil kernel, arguments
// in the constant bank); a cubic lattice on the edge-gather path never.
bool shares_launches(const ka_batch* b, const ka_ctx* ctx) {
  if (ctx->topo != KA_CUBIC) return true;
  if (!ctx->pencil) return false;
  int64_t pencils = 1;
  for (int k = 0; k < ctx->d - 1; ++k) pencils *= ctx->L;
  if (ctx->d >= 2) pencils /= 2;
  const int64_t tiles = (pencils + ka::kCubicWarps / ctx->pl.V - 1) / (ka::kCubicWarps / ctx->pl.V);
  return tiles < (b->own_tiles > 0 ? b->own_tiles : b->wave_tiles);
}

// sweeps job j may run in a round of length k: up to its next observation or its target
int64_t allowance(const Job* j, int64_t k) {
  const int64_t next_obs = (j->t / j->every + 1) * j->every;
  const int64_t stop = std::min(next_obs, j->target);
  return std::max<int64_t>(0, std::min(k, stop - j->t));
}

// The launches of one round of length k (captured or run directly).
cudaError_t issue_round(ka_batch* b, int64_t k) {
  cudaError_t e = cudaSuccess;
  for (int64_t s = 0; s < k && !e; ++s) {
    for (auto& cc : b->cubic) {
      const int npar = (cc.d == 1) ? 1 : 2;
      for (int mu = 0; mu < cc.d && !e; ++mu)
        for (int par = 0; par < npar && !e; ++par) {
          const bool x = (mu == 0) || cc.d == 1;
          e = ka::launch_cubic_group_batch(cc.dev, cc.tile_unit_dev[x ? 0 : 1],
                                           (int)cc.units.size(), cc.ntiles[x ? 0 : 1],
                                           cc.PSmax, cc.d, cc.V, cc.m, mu, par, (uint32_t)s,
                                           b->stream);
        }
    }
    for (auto& sc : b->sclass)
      for (int mu = 0; mu < 3 && !e; ++mu)
        for (int par = 0; par < 2 && !e; ++par)
          e = ka::launch_stream_batch(sc.dev, (int)sc.count(), sc.L, sc.m, mu, par, (uint32_t)s,
                                      b->stream);
    for (auto& gc : b->graph) {
      const int n = (int)gc.units.size();
      for (int c = 0; c < gc.cmax && !e; ++c)
        e = ka::launch_graph_class_batch(gc.dev, gc.prefix_dev + (size_t)c * (n + 1),
                                         gc.first_dev + (size_t)c * n, n, gc.total[c], gc.V, gc.m,
                                         (uint32_t)c, (uint32_t)s, b->stream);
    }
  }
  return e;
}

ka_status observe_job(ka_batch* b, Job* j) {
  if (j->n_obs >= j->cap) {
    b->err = "observation buffer full";
    return KA_ESTATE;
  }
  const int R = j->ctx->R;
  cudaError_t e = ka::launch_observe(j->ctx->pl, R,
                                     (unsigned long long*)(j->obs_dev + j->n_obs * R * 4),
                                     b->stream);
  if (e) return cuda_err(b, e, "observe");
  j->obs_t.push_back(j->t);
  j->n_obs++;
  return KA_OK;
}

ka_status run_round(ka_batch* b, int64_t k_req, int64_t* ran) {
  // finished and removed jobs stay in the tables as idle units (their
  // launches skip them) until they are half of all units; new jobs need a
  // rebuild at once
  if (b->dirty || 2 * b->idle_units > b->units) {
    cudaError_t e = rebuild(b);
    if (e) return cuda_err(b, e, "batch tables");
  }
  // the round's length: the requested k, but no longer than any job may go
  int64_t k = 0;
  for (auto& kv : b->jobs) {
    Job* j = kv.second;
    if (!j->finished) k = std::max(k, allowance(j, k_req));
  }
  if (ran) *ran = k;
  if (k == 0) return KA_OK;
  cudaError_t e = cudaSuccess;
  if (b->flags & KA_BATCH_PLAIN) {
    // the unbatched reference: every job with its own launches
    for (auto& kv : b->jobs) {
      Job* j = kv.second;
      if (j->finished) continue;
      ka_status st = ka_sweep(j->ctx, allowance(j, k));
      if (st) return st;
    }
  } else {
    // unit tables: this round's start and stop sweeps
    for (auto& cc : b->cubic) {
      for (size_t u = 0; u < cc.units.size(); ++u) {
        const Job* j = cc.owner[u];
        const bool live = j && !j->finished;
        cc.units[u].t_base = live ? (uint32_t)j->t : 0u;
        cc.units[u].t_end = live ? (uint32_t)(j->t + allowance(j, k)) : 0u;
      }
      if ((e = cudaMemcpyAsync(cc.dev, cc.units.data(), cc.units.size() * sizeof(ka::CubicUnit),
                               cudaMemcpyHostToDevice, b->stream)))
        return cuda_err(b, e, "unit table");
    }
    for (auto& sc : b->sclass) {
      const size_t ub = ka::stream_unit_bytes();
      for (size_t u = 0; u < sc.count(); ++u) {
        const Job* j = sc.owner[u];
        const bool live = j && !j->finished;
        const ka_ctx* c = j ? j->ctx : nullptr;
        const int q = sc.plane[u];
        ka::stream_unit_fill(sc.units.data() + u * ub,
                             c ? c->pl.n + (size_t)q * c->pl.plane_elems() : nullptr,
                             c ? c->pl.p + (size_t)q * c->pl.plane_elems() : nullptr,
                             (uint32_t)(q * (c ? c->pl.V : 1)), live ? (uint32_t)j->t : 0u,
                             live ? (uint32_t)(j->t + allowance(j, k)) : 0u,
                             c ? c->rk : ka::RoundKeys{});
      }
      if ((e = cudaMemcpyAsync(sc.dev, sc.units.data(), sc.units.size(), cudaMemcpyHostToDevice,
                               b->stream)))
        return cuda_err(b, e, "unit table");
    }
    for (auto& gc : b->graph) {
      for (size_t u = 0; u < gc.units.size(); ++u) {
        const Job* j = gc.owner[u];
        const bool live = j && !j->finished;
        gc.units[u].t_base = live ? (uint32_t)j->t : 0u;
        gc.units[u].t_end = live ? (uint32_t)(j->t + allowance(j, k)) : 0u;
      }
      if ((e = cudaMemcpyAsync(gc.dev, gc.units.data(), gc.units.size() * sizeof(ka::GraphUnit),
                               cudaMemcpyHostToDevice, b->stream)))
        return cuda_err(b, e, "unit table");
    }
    const bool replay = (b->flags & KA_BATCH_GRAPH) && k == b->last_k;
    b->last_k = k;
    if (replay) {
      if (!b->exec || b->exec_k != k) {
        if (b->exec) {
          cudaGraphExecDestroy(b->exec);
          b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (!e) {
          const cudaError_t ei = issue_round(b, k);
          e = cudaStreamEndCapture(b->stream, &g);
          if (!e) e = ei;
        }
        if (!e) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e) return cuda_err(b, e, "round graph");
        b->exec_k = k;
      }
      e = cudaGraphLaunch(b->exec, b->stream);
    } else {
      e = issue_round(b, k);
    }
    if (e) return cuda_err(b, e, "round");
    // jobs not in the tables (large lattices, the edge-gather path) run with their own launches
    for (auto& kv : b->jobs) {
      Job* j = kv.second;
      if (j->finished || j->batched) continue;
      ka_status st = ka_sweep(j->ctx, allowance(j, k));
      if (st) return st;
    }
  }
  // advance the counters, record due observations, retire finished jobs
  for (auto& kv : b->jobs) {
    Job* j = kv.second;
    if (j->finished) continue;
    const int64_t a = allowance(j, k);
    if (a == 0) continue;
    j->t += a;
    if (!(b->flags & KA_BATCH_PLAIN) && j->batched) j->ctx->sweep = j->t;
    if (j->t % j->every == 0 || j->t == j->target) {
      ka_status st = observe_job(b, j);
      if (st) return st;
    }
    if (j->t >= j->target) {
      j->finished = true;
      if (j->batched) b->idle_units += j->ctx->pl.P;  // idles in the tables until rebuilt
    }
  }
  e = cudaStreamSynchronize(b->stream);
  if (e) return cuda_err(b, e, "round sync");
  return KA_OK;
}

size_t obs_bytes(const ka_job_spec* spec, int64_t replicas) {
  const int64_t cap = spec->sweeps / spec->observe_every + 2;
  return (size_t)cap * (size_t)replicas * 4 * sizeof(int64_t);
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
      cudaSetDevice(dev);
    else
      prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Make an initialised context (owning its buffer) a job of the batch: move
// it onto the batch's stream, allocate its observation buffer and record
// the first observation.  On failure the context is left to the caller.
ka_status enrol(ka_batch* b, ka_ctx* ctx, const ka_job_spec* spec, int64_t* job_id) {
  const size_t ob = obs_bytes(spec, ctx->R);
  Job* j = new Job();
  if (cudaMalloc((void**)&j->obs_dev, ob) != cudaSuccess) {
    cudaGetLastError();
    delete j;
    return KA_ENOMEM;
  }
  ctx->stream = b->stream;
  ctx->prm.stream = b->stream;
  j->ctx = ctx;
  j->buf = ctx->buf;
  j->t = ctx->sweep;
  j->target = spec->sweeps;
  j->every = spec->observe_every;
  j->cap = spec->sweeps / spec->observe_every + 2;
  // small jobs share the batched launches (shares_launches)
  j->batched = shares_launches(b, ctx);
  const ka_status st = observe_job(b, j);
  if (st) {
    cudaFree(j->obs_dev);
    delete j;
    return st;
  }
  j->id = b->next_id++;
  j->bytes = ctx->bytes + ob;
  if (j->t >= j->target) j->finished = true;
  b->jobs[j->id] = j;
  b->used += j->bytes;
  b->dirty = true;
  if (job_id) *job_id = j->id;
  return KA_OK;
}

}  // namespace

namespace {

// Site-word-sweeps one round of length k would run (the unfinished jobs).
double round_work(const ka_batch* b, int64_t k) {
  double work = 0.0;
  for (auto& kv : b->jobs) {
    const Job* j = kv.second;
    if (!j->finished) work += (double)j->ctx->N * (j->ctx->R / 64) * (double)allowance(j, k);
  }
  return work;
}

// Site-word-sweeps per ms of rounds of length k in the batch's present
// configuration: warm-up rounds first (the first builds the tables; in graph
// mode the second captures the round, a length being captured on its second
// use), then one timed round.  All rounds do real work.  Returns < 0 when no
// job is left to run.
double time_rounds(ka_batch* b, int64_t k, cudaEvent_t e0, cudaEvent_t e1, ka_status* st) {
  int64_t ran = 0;
  const int warm = (b->flags & KA_BATCH_GRAPH) ? 2 : 1;
  for (int w = 0; w < warm && !*st; ++w) *st = run_round(b, k, &ran);
  if (*st || ran == 0) return -1.0;
  const double work = round_work(b, k);
  if (work == 0.0) return -1.0;
  cudaEventRecord(e0, b->stream);
  *st = run_round(b, k, &ran);
  cudaEventRecord(e1, b->stream);
  cudaEventSynchronize(e1);
  if (*st) return -1.0;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return work / (ms > 0.f ? ms : 1e-3f);
}

// Put every unfinished cubic job on its own or the shared launches for the
// threshold own_tiles; the tables are rebuilt before the next round if any
// job moved.
void apply_own_tiles(ka_batch* b, int64_t own_tiles) {
  b->own_tiles = own_tiles;
  for (auto& kv : b->jobs) {
    Job* j = kv.second;
    if (j->finished) continue;
    const bool shared = shares_launches(b, j->ctx);
    if (shared != j->batched) {
      j->batched = shared;
      b->dirty = true;
    }
  }
}

}  // namespace

extern "C" {

ka_status ka_batch_create(int32_t device, void* stream, size_t hbm_budget, int32_t flags,
                          ka_batch** out) {
  if (!out) return KA_EINVAL;
  *out = nullptr;
  ka_batch* b = new ka_batch();
  b->device = device;
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {  // stream capture needs a stream other than the legacy default one
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    const cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      delete b;
      return KA_ECUDA;
    }
    b->own_stream = true;
  }
  b->budget = hbm_budget;
  b->flags = flags;
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
      b->wave_tiles = 2 * (int64_t)sms;  // two CTAs of the pencil kernel per SM
  }
  *out = b;
  return KA_OK;
}

ka_status ka_job_bytes(const ka_params* params, const ka_job_spec* spec, size_t* bytes) {
  if (!params || !spec || !bytes || spec->sweeps < 0 || spec->observe_every < 1) return KA_EINVAL;
  size_t ctx_bytes = 0;
  const ka_status st = ka::context_bytes(params, &ctx_bytes);
  if (st) return st;
  *bytes = ctx_bytes + obs_bytes(spec, params->replicas);
  return KA_OK;
}

ka_status ka_batch_add(ka_batch* b, const ka_params* params, const ka_job_spec* spec,
                       int64_t* job_id) {
  ka::NvtxRange nvtx_range("ka_batch_admit");
  if (!b || !params || !spec || spec->sweeps < 0 || spec->observe_every < 1) return KA_EINVAL;
  if (spec->sweeps >= ((int64_t)1 << 32)) return KA_EINVAL;
  ka_params prm = *params;
  prm.device = b->device;
  prm.stream = b->stream;
  size_t bytes = 0;
  ka_status st = ka::context_bytes(&prm, &bytes);
  if (st) return st;
  if (b->used + bytes + obs_bytes(spec, prm.replicas) > b->budget) return KA_EBUSY;
  DeviceScope scope(b->device);
  void* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return KA_ENOMEM;
  }
  ka_ctx* ctx = nullptr;
  st = ka::create_context(&prm, buf, bytes, true, &ctx);
  if (st) {
    cudaFree(buf);
    return st;
  }
  st = ka_init(ctx, spec->seed, spec->rho);
  if (!st) st = enrol(b, ctx, spec, job_id);
  if (st) ka_destroy(ctx);
  return st;
}

ka_status ka_batch_adopt(ka_batch* b, ka_ctx* ctx, const ka_job_spec* spec, int64_t* job_id) {
  ka::NvtxRange nvtx_range("ka_batch_admit");
  if (!b || !ctx || !spec || spec->observe_every < 1) return KA_EINVAL;
  if (spec->sweeps < ctx->sweep || spec->sweeps >= ((int64_t)1 << 32)) return KA_EINVAL;
  if (!ctx->owns || ctx->device != b->device) return KA_EINVAL;
  if (!ctx->initialized) return KA_ESTATE;
  if (b->used + ctx->bytes + obs_bytes(spec, ctx->R) > b->budget) return KA_EBUSY;
  DeviceScope scope(b->device);
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e) return cuda_err(b, e, "adopted context");
  return enrol(b, ctx, spec, job_id);
}

ka_status ka_batch_step(ka_batch* b, int64_t max_sweeps, int64_t* sweeps_run) {
  ka::NvtxRange nvtx_range("ka_batch_round");
  if (!b || max_sweeps < 0) return KA_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  const ka_status st = run_round(b, max_sweeps ? max_sweeps : b->tuned_k, sweeps_run);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

ka_status ka_batch_autotune(ka_batch* b, int64_t* best_round) {
  ka::NvtxRange nvtx_range("ka_batch_autotune");
  if (!b) return KA_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ka_status st = KA_OK;
  // (1) which cubic jobs run with their own launches: the tile threshold, at
  // the present round length (one wave of tiles, half, a quarter, an eighth,
  // or no job on its own launches)
  if (!(b->flags & KA_BATCH_PLAIN)) {
    const int64_t w = b->wave_tiles;
    const int64_t cand[] = {w, w / 2, w / 4, w / 8, INT64_MAX};
    double best = -1.0;
    int64_t best_t = b->own_tiles > 0 ? b->own_tiles : w;
    for (int64_t t : cand) {
      apply_own_tiles(b, t);
      const double rate = time_rounds(b, b->tuned_k, e0, e1, &st);
      if (st || rate < 0.0) break;
      if (rate > best) {
        best = rate;
        best_t = t;
      }
    }
    if (!st) apply_own_tiles(b, best_t);
  }
  // (2) the round length, with that threshold
  const int64_t cand_k[] = {4, 16, 64};
  double best = -1.0;
  int64_t best_k = b->tuned_k;
  for (int64_t k : cand_k) {
    if (st) break;
    const double rate = time_rounds(b, k, e0, e1, &st);
    if (st || rate < 0.0) break;
    if (rate > best) {
      best = rate;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tuned_k = best_k;
  if (best_round) *best_round = best_k;
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

ka_status ka_batch_tuning(const ka_batch* b, int64_t* round_sweeps, int64_t* own_tiles) {
  if (!b) return KA_EINVAL;
  if (round_sweeps) *round_sweeps = b->tuned_k;
  if (own_tiles) *own_tiles = b->own_tiles > 0 ? b->own_tiles : b->wave_tiles;
  return KA_OK;
}

ka_status ka_batch_poll(const ka_batch* b, int64_t job_id, int64_t* sweep, int32_t* finished) {
  if (!b) return KA_EINVAL;
  auto it = b->jobs.find(job_id);
  if (it == b->jobs.end()) return KA_EINVAL;
  if (sweep) *sweep = it->second->t;
  if (finished) *finished = it->second->finished ? 1 : 0;
  return KA_OK;
}

ka_status ka_batch_observations(const ka_batch* b, int64_t job_id, int64_t* n_obs,
                                int64_t* obs_sweeps, int64_t* counts) {
  if (!b) return KA_EINVAL;
  auto it = b->jobs.find(job_id);
  if (it == b->jobs.end()) return KA_EINVAL;
  const Job* j = it->second;
  if (n_obs) *n_obs = j->n_obs;
  if (obs_sweeps) std::memcpy(obs_sweeps, j->obs_t.data(), j->obs_t.size() * sizeof(int64_t));
  if (counts && j->n_obs > 0) {
    cudaError_t e = cudaMemcpyAsync(counts, j->obs_dev,
                                    (size_t)j->n_obs * j->ctx->R * 4 * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, b->stream);
    if (!e) e = cudaStreamSynchronize(b->stream);
    if (e) return KA_ECUDA;
  }
  return KA_OK;
}

ka_status ka_batch_state(ka_batch* b, int64_t job_id, uint64_t* n, uint64_t* n0, uint64_t* p) {
  if (!b) return KA_EINVAL;
  auto it = b->jobs.find(job_id);
  if (it == b->jobs.end()) return KA_EINVAL;
  DeviceScope scope(b->device);
  // the job's context runs on the batch stream: ka_get_state waits for it
  return ka_get_state(it->second->ctx, n, n0, p);
}

ka_status ka_batch_remove(ka_batch* b, int64_t job_id) {
  if (!b) return KA_EINVAL;
  auto it = b->jobs.find(job_id);
  if (it == b->jobs.end()) return KA_EINVAL;
  Job* j = it->second;
  cudaStreamSynchronize(b->stream);
  // its units (if any) stay in the tables as idle units, with no owner
  int64_t in_tables = 0;
  for (auto& cc : b->cubic)
    for (auto& o : cc.owner)
      if (o == j) {
        o = nullptr;
        ++in_tables;
      }
  for (auto& sc : b->sclass)
    for (auto& o : sc.owner)
      if (o == j) {
        o = nullptr;
        ++in_tables;
      }
  for (auto& gc : b->graph)
    for (auto& o : gc.owner)
      if (o == j) {
        o = nullptr;
        ++in_tables;
      }
  if (!j->finished) b->idle_units += in_tables;
  const ka_status st = ka_destroy(j->ctx);  // frees the context's buffer
  cudaFree(j->obs_dev);
  b->used -= j->bytes;
  b->jobs.erase(it);
  delete j;
  return st;
}

ka_status ka_batch_info(const ka_batch* b, size_t* used_bytes, int64_t* jobs, int64_t* active) {
  if (!b) return KA_EINVAL;
  int64_t a = 0;
  for (auto& kv : b->jobs) a += kv.second->finished ? 0 : 1;
  if (used_bytes) *used_bytes = b->used;
  if (jobs) *jobs = (int64_t)b->jobs.size();
  if (active) *active = a;
  return KA_OK;
}

ka_status ka_batch_destroy(ka_batch* b) {
  if (!b) return KA_OK;
  cudaStreamSynchronize(b->stream);
  ka_status st = KA_OK;
  for (auto& kv : b->jobs) {
    Job* j = kv.second;
    if (ka_destroy(j->ctx)) st = KA_ECUDA;
    cudaFree(j->obs_dev);
    delete j;
  }
  free_tables(b);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return st;
}

}  // extern "C"
