// ka_sweep_graph.cu -- edge-gather sweep kernel for one bond class.
//
// One thread per (bond of the class, plane).  The bond (u, v) gathers the
// words of u, v and of their neighbours from the int32 neighbour list, counts
// the occupied neighbours of u other than v and of v other than u with
// bit-sliced adders (64 replicas per word), and applies the exchange rule of
// section 2.1 (rules (a)-(c)) under the replica's Philox gate bit.  Bonds of
// a class form a strong matching, so threads never touch each other's sites.
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

template <int V>
__device__ __forceinline__ void ld(const uint64_t* base, int64_t i, uint64_t (&o)[V]) {
  if constexpr (V == 2) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(base + 2 * i);
    o[0] = v.x;
    o[1] = v.y;
  } else {
    o[0] = base[i];
  }
}

template <int V>
__device__ __forceinline__ void st(uint64_t* base, int64_t i, const uint64_t (&o)[V]) {
  if constexpr (V == 2) {
    *reinterpret_cast<ulonglong2*>(base + 2 * i) = make_ulonglong2(o[0], o[1]);
  } else {
    base[i] = o[0];
  }
}

template <int V, int M>
__global__ void __launch_bounds__(256) k_graph_class(const ClassArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.count) return;
  const int q = blockIdx.y;
  uint64_t* np = a.n + (size_t)q * a.plane_elems;
  uint64_t* pp = a.p + (size_t)q * a.plane_elems;
  const int32_t u = a.bu[e], v = a.bv[e];
  const uint32_t id = a.bid[e];
  const int z = a.z;

  uint64_t nu[V], nv[V];
  ld<V>(np, u, nu);
  ld<V>(np, v, nv);
  uint64_t cu2[V], cu1[V], cu0[V], cv2[V], cv1[V], cv0[V];
#pragma unroll
  for (int h = 0; h < V; ++h) cu2[h] = cu1[h] = cu0[h] = cv2[h] = cv1[h] = cv0[h] = 0;
  for (int k = 0; k < z; ++k) {
    const int32_t wu = a.nbr[(int64_t)u * z + k];
    const int32_t wv = a.nbr[(int64_t)v * z + k];
    uint64_t xu[V], xv[V];
    ld<V>(np, wu, xu);
    ld<V>(np, wv, xv);
    const uint64_t keep_u = (wu != v) ? ~0ull : 0ull;  // skip the partner
    const uint64_t keep_v = (wv != u) ? ~0ull : 0ull;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      add3(cu2[h], cu1[h], cu0[h], xu[h] & keep_u);
      add3(cv2[h], cv1[h], cv0[h], xv[h] & keep_v);
    }
  }
  // gate words.  Graphs: block (t, class, edge, word pair), half = word
  // parity.  Cubic lattices (one-word planes): bonds of classes 4g+2b and
  // 4g+2b+1 that start at neighbouring pencil positions share the block
  // (t, 4g+2b, base site of the first, word), half = class parity.
  uint64_t g[V];
  if (a.pair_stride != 0) {
    const uint32_t odd = a.cls & 1u;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      const uint4 b = philox(
          make_uint4(a.t, a.cls - odd, id - odd * a.pair_stride, (uint32_t)(q * V + h)), a.rk);
      g[h] = odd ? hi64(b) : lo64(b);
    }
  } else {
    uint32_t c3, half;
    if constexpr (V == 2) {
      c3 = (uint32_t)q;
      half = 0;
    } else {
      c3 = (uint32_t)(q >> 1);
      half = (uint32_t)(q & 1);
    }
    const uint4 b = philox(make_uint4(a.t, a.cls, id, c3), a.rk);
    if constexpr (V == 2) {
      g[0] = lo64(b);
      g[1] = hi64(b);
    } else {
      g[0] = half ? hi64(b) : lo64(b);
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
    uint64_t pu[V], pv[V];
    ld<V>(pp, u, pu);
    ld<V>(pp, v, pv);
#pragma unroll
    for (int h = 0; h < V; ++h) {
      pu[h] &= ~sw[h];
      pv[h] &= ~sw[h];
    }
    st<V>(pp, u, pu);
    st<V>(pp, v, pv);
  }
}

template <int V>
cudaError_t launch_v(const ClassArgs& a, int m, dim3 grid, cudaStream_t s) {
  const int mm = m < 7 ? m : 7;
  switch (mm) {
#define KA_CASE(MM)                                                   \
  case MM:                                                            \
    k_graph_class<V, MM><<<grid, 256, 0, s>>>(a);                     \
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
  uint64_t* np = gu.n;
  uint64_t* pp = gu.p;
  const int32_t u = gu.bu[k], v = gu.bv[k];
  const uint32_t id = gu.bid[k];
  const int z = gu.z;
  uint64_t nu[V], nv[V];
  ld<V>(np, u, nu);
  ld<V>(np, v, nv);
  uint64_t cu2[V], cu1[V], cu0[V], cv2[V], cv1[V], cv0[V];
#pragma unroll
  for (int h = 0; h < V; ++h) cu2[h] = cu1[h] = cu0[h] = cv2[h] = cv1[h] = cv0[h] = 0;
  for (int q = 0; q < z; ++q) {
    const int32_t wu = gu.nbr[(int64_t)u * z + q];
    const int32_t wv = gu.nbr[(int64_t)v * z + q];
    uint64_t xu[V], xv[V];
    ld<V>(np, wu, xu);
    ld<V>(np, wv, xv);
    const uint64_t keep_u = (wu != v) ? ~0ull : 0ull;
    const uint64_t keep_v = (wv != u) ? ~0ull : 0ull;
#pragma unroll
    for (int h = 0; h < V; ++h) {
      add3(cu2[h], cu1[h], cu0[h], xu[h] & keep_u);
      add3(cv2[h], cv1[h], cv0[h], xv[h] & keep_v);
    }
  }
  // graph gate stream: block (t, class, edge, word pair), half = word parity
  uint64_t g[V];
  const uint32_t w0 = gu.word0;
  if constexpr (V == 2) {
    const uint4 b = philox(make_uint4(t, cls, id, w0 >> 1), gu.rk);
    g[0] = lo64(b);
    g[1] = hi64(b);
  } else {
    const uint4 b = philox(make_uint4(t, cls, id, w0 >> 1), gu.rk);
    g[0] = (w0 & 1u) ? hi64(b) : lo64(b);
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
    uint64_t pu[V], pv[V];
    ld<V>(pp, u, pu);
    ld<V>(pp, v, pv);
#pragma unroll
    for (int h = 0; h < V; ++h) {
      pu[h] &= ~sw[h];
      pv[h] &= ~sw[h];
    }
    st<V>(pp, u, pu);
    st<V>(pp, v, pv);
  }
}

}  // namespace

cudaError_t launch_graph_class_batch(const GraphUnit* units_dev, const int64_t* prefix_dev,
                                     const int64_t* first_dev, int nunits, int64_t total_edges,
                                     int V, int m, uint32_t cls, uint32_t sweep_offset,
                                     cudaStream_t s) {
  if (nunits <= 0 || total_edges <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((total_edges + 255) / 256);
  const int mm = m < 7 ? m : 7;
#define KA_CASE(VV, MM)                                                                  \
  if (V == VV && mm == MM) {                                                             \
    k_graph_class_batch<VV, MM><<<grid, 256, 0, s>>>(units_dev, prefix_dev, first_dev,   \
                                                     nunits, cls, sweep_offset);         \
    return cudaGetLastError();                                                           \
  }
  KA_CASE(1, 0) KA_CASE(1, 1) KA_CASE(1, 2) KA_CASE(1, 3) KA_CASE(1, 4) KA_CASE(1, 5)
  KA_CASE(1, 6) KA_CASE(1, 7)
  KA_CASE(2, 0) KA_CASE(2, 1) KA_CASE(2, 2) KA_CASE(2, 3) KA_CASE(2, 4) KA_CASE(2, 5)
  KA_CASE(2, 6) KA_CASE(2, 7)
#undef KA_CASE
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
  dim3 grid((unsigned)((count + 255) / 256), (unsigned)pl.P);
  return pl.V == 2 ? launch_v<2>(a, g.m, grid, s) : launch_v<1>(a, g.m, grid, s);
}

}  // namespace ka
