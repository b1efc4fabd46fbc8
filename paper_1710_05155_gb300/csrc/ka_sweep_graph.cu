// ka_sweep_graph.cu -- edge-gather sweep kernel for one bond class.
//
// One thread per (bond of the class, plane).  The bond (u, v) gathers the
// words of u, v and of their other neighbours from the int32 neighbour
// list, counts the occupied neighbours of u other than v and of v other
// than u with bit-sliced adders (64 replicas per word), and applies the
// exchange rule of section 2.1 (rules (a)-(c)) under the replica's Philox
// gate bit.  Bonds of a class form a strong matching, so threads never
// touch each other's sites.
//
// A plane holds V = 1, 2 or 4 words per site, so a site's words share one
// 32-byte sector: every gather is a random access, and the sector is the
// unit the memory system moves.  The partner's word is not gathered twice,
// and p is never read: the bits of p that a swap clears are cleared by an
// atomic AND in the L2.
// A thread first loads what depends only on static tables (its bond, the
// two neighbour rows) and computes the gate words, then gathers the state.
// Single-instance class launches are chained with programmatic dependent
// launch, so that this prologue overlaps the previous class's tail (small
// graphs are bound by launch latency); batched launches are not, since a
// grid waiting on the SMs slows the one it waits for.
#include "ka_internal.cuh"

namespace ka {
namespace {

struct ClassArgs {
  uint64_t* n;
  uint64_t* p;
  const int32_t* nbr;
  const int32_t* bu;
  const int32_t* bv;
  const uint32_t* bid;
  size_t plane_elems;
  int64_t count;
  int z;
  uint32_t t, cls;
  uint32_t pair_stride;  // cubic lattices: stride of the bond direction, 0 on graphs
  RoundKeys rk;
};

// (c2 c1 c0) += x, bit-sliced; the count stays below 8 (at most 7 inputs)
__device__ __forceinline__ void add3(uint64_t& c2, uint64_t& c1, uint64_t& c0, uint64_t x) {
  const uint64_t k0 = c0 & x;
  c0 ^= x;
  const uint64_t k1 = c1 & k0;
  c1 ^= k0;
  c2 |= k1;
}

template <int T>
__device__ __forceinline__ uint64_t le3(uint64_t b2, uint64_t b1, uint64_t b0) {
  if constexpr (T < 0) {
    return 0ull;
  } else if constexpr (T >= 7) {
    return ~0ull;
  } else {
    const uint64_t g0 = (T & 1) ? 0ull : b0;
    const uint64_t g1 = (T & 2) ? (b1 & g0) : (b1 | g0);
    const uint64_t g2 = (T & 4) ? (b2 & g1) : (b2 | g1);
    return ~g2;
  }
}

// the V words of site i (16-byte vectors for V >= 2; a site's words are
// 8 V-byte aligned)
template <int V>
__device__ __forceinline__ void ld(const uint64_t* base, int64_t i, uint64_t (&o)[V]) {
  if constexpr (V == 1) {
    o[0] = base[i];
  } else {
#pragma unroll
    for (int h = 0; h < V; h += 2) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(base + V * i + h);
      o[h] = v.x;
      o[h + 1] = v.y;
    }
  }
}

template <int V>
__device__ __forceinline__ void st(uint64_t* base, int64_t i, const uint64_t (&o)[V]) {
  if constexpr (V == 1) {
    base[i] = o[0];
  } else {
#pragma unroll
    for (int h = 0; h < V; h += 2)
      *reinterpret_cast<ulonglong2*>(base + V * i + h) = make_ulonglong2(o[h], o[h + 1]);
  }
}

constexpr int kMaxZ = 8;

// neighbour row of x (z <= 8); z = 4 rows are one 16-byte load
__device__ __forceinline__ void load_row(const int32_t* nbr, int z, int32_t x,
                                         int32_t (&r)[kMaxZ]) {
  if (z == 4) {
    const int4 q = *reinterpret_cast<const int4*>(nbr + (int64_t)x * 4);
    r[0] = q.x;
    r[1] = q.y;
    r[2] = q.z;
    r[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < kMaxZ; ++k)
      if (k < z) r[k] = nbr[(int64_t)x * z + k];
  }
}

// Graph gate stream: word w of bond id takes half w mod 2 of the block
// (t, class, id, w / 2).  Planes start at an even word when V >= 2.
template <int V>
__device__ __forceinline__ void graph_gates(uint32_t t, uint32_t cls, uint32_t id, uint32_t w0,
                                            const RoundKeys& rk, uint64_t (&g)[V]) {
  if constexpr (V == 1) {
    const uint4 b = philox(make_uint4(t, cls, id, w0 >> 1), rk);
    g[0] = (w0 & 1u) ? hi64(b) : lo64(b);
  } else {
#pragma unroll
    for (int h = 0; h < V; h += 2) {
      const uint4 b = philox(make_uint4(t, cls, id, (w0 + h) >> 1), rk);
      g[h] = lo64(b);
      g[h + 1] = hi64(b);
    }
  }
}

// The exchange on bond (u, v), V words: counts of the other neighbours of
// u and of v, the rule, the gated swap, and the persistence update.
template <int V, int M>
__device__ __forceinline__ void exchange(uint64_t* np, uint64_t* pp, int z, int32_t u, int32_t v,
                                         const int32_t (&ru)[kMaxZ], const int32_t (&rv)[kMaxZ],
                                         const uint64_t (&g)[V]) {
  uint64_t nu[V], nv[V];
  ld<V>(np, u, nu);
  ld<V>(np, v, nv);
  uint64_t cu2[V], cu1[V], cu0[V], cv2[V], cv1[V], cv0[V];
#pragma unroll
  for (int h = 0; h < V; ++h) cu2[h] = cu1[h] = cu0[h] = cv2[h] = cv1[h] = cv0[h] = 0;
#pragma unroll
  for (int k = 0; k < kMaxZ; ++k) {
    if (k < z) {
      if (ru[k] != v) {  // the partner is not one of the "other" neighbours
        uint64_t x[V];
        ld<V>(np, ru[k], x);
#pragma unroll
        for (int h = 0; h < V; ++h) add3(cu2[h], cu1[h], cu0[h], x[h]);
      }
      if (rv[k] != u) {
        uint64_t x[V];
        ld<V>(np, rv[k], x);
#pragma unroll
        for (int h = 0; h < V; ++h) add3(cv2[h], cv1[h], cv0[h], x[h]);
      }
    }
  }
  uint64_t sw[V];
  bool any = false;
#pragma unroll
  for (int h = 0; h < V; ++h) {
    const uint64_t ok = le3<M>(cu2[h], cu1[h], cu0[h]) & le3<M>(cv2[h], cv1[h], cv0[h]);
    sw[h] = (nu[h] ^ nv[h]) & g[h] & ok;
    nu[h] ^= sw[h];
    nv[h] ^= sw[h];
    any |= (sw[h] != 0);
  }
  if (any) {
    st<V>(np, u, nu);
    st<V>(np, v, nv);
    // Persistence: an atomic AND performed in the L2 (no reply), not a load
    // of p after the swap is known and a store: random gathers are bound by
    // the misses an SM keeps in flight, and this removes two of them per bond
    // and a dependent round trip.
    unsigned long long* pw = reinterpret_cast<unsigned long long*>(pp);
#pragma unroll
    for (int h = 0; h < V; ++h) {
      if (sw[h]) {
        atomicAnd(pw + (size_t)V * u + h, (unsigned long long)~sw[h]);
        atomicAnd(pw + (size_t)V * v + h, (unsigned long long)~sw[h]);
      }
    }
  }
}

template <int V, int M>
__global__ void __launch_bounds__(256) k_graph_class(const __grid_constant__ ClassArgs a) {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count) return;
  const int q = blockIdx.y;
  uint64_t* np = a.n + (size_t)q * a.plane_elems;
  uint64_t* pp = a.p + (size_t)q * a.plane_elems;
  const int32_t u = a.bu[e], v = a.bv[e];
  const uint32_t id = a.bid[e];
  int32_t ru[kMaxZ], rv[kMaxZ];
  load_row(a.nbr, a.z, u, ru);
  load_row(a.nbr, a.z, v, rv);
  // gate words.  Graphs: the graph stream.  Cubic lattices on this path:
  // bonds of classes 4g+2b and 4g+2b+1 that start at neighbouring pencil
  // positions share the block (t, 4g+2b, base site of the first, word),
  // half = class parity.
  uint64_t g[V];
  const uint32_t w0 = (uint32_t)(q * V);
  if (a.pair_stride != 0) {
    const uint32_t odd = a.cls & 1u;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      const uint4 b = philox(make_uint4(a.t, a.cls - odd, id - odd * a.pair_stride, w0 + h), a.rk);
      g[h] = odd ? hi64(b) : lo64(b);
    }
  } else {
    graph_gates<V>(a.t, a.cls, id, w0, a.rk, g);
  }
  asm volatile("griddepcontrol.wait;\n" ::: "memory");  // the previous class is complete
  exchange<V, M>(np, pp, a.z, u, v, ru, rv, g);
}

// Batched form: one launch runs class c of every graph unit (one state plane
// of one job); edges of all units are numbered consecutively, unit u owning
// [prefix[u], prefix[u+1]) of them, which start at edge first[u] of its
// class-ordered edge arrays.  Units whose sweep counter reached t_end skip.
template <int V, int M>
__global__ void __launch_bounds__(256) k_graph_class_batch(const GraphUnit* __restrict__ units,
                                                           const int64_t* __restrict__ prefix,
                                                           const int64_t* __restrict__ first,
                                                           int nunits, uint32_t cls,
                                                           uint32_t sweep_offset) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= prefix[nunits]) return;
  int lo = 0, hi = nunits - 1;  // last unit with prefix <= e
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= e) lo = mid; else hi = mid - 1;
  }
  const GraphUnit& gu = units[lo];
  const uint32_t t = gu.t_base + sweep_offset;
  if (t >= gu.t_end) return;
  const int64_t k = first[lo] + (e - prefix[lo]);
  const int32_t u = gu.bu[k], v = gu.bv[k];
  const uint32_t id = gu.bid[k];
  const int z = gu.z;
  int32_t ru[kMaxZ], rv[kMaxZ];
  load_row(gu.nbr, z, u, ru);
  load_row(gu.nbr, z, v, rv);
  uint64_t g[V];
  graph_gates<V>(t, cls, id, gu.word0, gu.rk, g);
  exchange<V, M>(gu.n, gu.p, z, u, v, ru, rv, g);
}

// single-instance launch with programmatic stream serialisation
template <typename Kern>
cudaError_t launch_pdl(Kern kern, dim3 grid, cudaStream_t s, const ClassArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int V>
cudaError_t launch_v(const ClassArgs& a, int m, dim3 grid, cudaStream_t s) {
  switch (m < 7 ? m : 7) {
#define KA_CASE(MM) \
  case MM:          \
    return launch_pdl(k_graph_class<V, MM>, grid, s, a);
    KA_CASE(0)
    KA_CASE(1)
    KA_CASE(2)
    KA_CASE(3)
    KA_CASE(4)
    KA_CASE(5)
    KA_CASE(6)
    KA_CASE(7)
#undef KA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int V>
cudaError_t launch_batch_v(const GraphUnit* units, const int64_t* prefix, const int64_t* first,
                           int nunits, int m, uint32_t cls, uint32_t off, dim3 grid,
                           cudaStream_t s) {
  switch (m < 7 ? m : 7) {
#define KA_CASE(MM)                                                                     \
  case MM:                                                                              \
    k_graph_class_batch<V, MM><<<grid, 256, 0, s>>>(units, prefix, first, nunits, cls, off); \
    return cudaGetLastError();
    KA_CASE(0)
    KA_CASE(1)
    KA_CASE(2)
    KA_CASE(3)
    KA_CASE(4)
    KA_CASE(5)
    KA_CASE(6)
    KA_CASE(7)
#undef KA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_graph_class_batch(const GraphUnit* units_dev, const int64_t* prefix_dev,
                                     const int64_t* first_dev, int nunits, int64_t total_edges,
                                     int V, int m, uint32_t cls, uint32_t sweep_offset,
                                     cudaStream_t s) {
  if (nunits <= 0 || total_edges <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((total_edges + 255) / 256));
  if (V == 4)
    return launch_batch_v<4>(units_dev, prefix_dev, first_dev, nunits, m, cls, sweep_offset, grid, s);
  if (V == 2)
    return launch_batch_v<2>(units_dev, prefix_dev, first_dev, nunits, m, cls, sweep_offset, grid, s);
  if (V == 1)
    return launch_batch_v<1>(units_dev, prefix_dev, first_dev, nunits, m, cls, sweep_offset, grid, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_graph_class(const Planes& pl, const GraphDev& g, int64_t off, int64_t count,
                               uint32_t cls, uint32_t t, const RoundKeys& rk, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  ClassArgs a;
  a.n = pl.n;
  a.p = pl.p;
  a.nbr = g.nbr;
  a.bu = g.bu + off;
  a.bv = g.bv + off;
  a.bid = g.bid + off;
  a.plane_elems = pl.plane_elems();
  a.count = count;
  a.z = g.z;
  a.t = t;
  a.cls = cls;
  a.pair_stride = 0;
  if (g.cubic_L > 0) {
    uint32_t s = 1;
    for (uint32_t k = 0; k < cls / 8; ++k) s *= (uint32_t)g.cubic_L;
    a.pair_stride = s;
  }
  a.rk = rk;
  const dim3 grid((unsigned)((count + 255) / 256), (unsigned)pl.P);
  if (pl.V == 4) return launch_v<4>(a, g.m, grid, s);
  if (pl.V == 2) return launch_v<2>(a, g.m, grid, s);
  return launch_v<1>(a, g.m, grid, s);
}

}  // namespace ka
