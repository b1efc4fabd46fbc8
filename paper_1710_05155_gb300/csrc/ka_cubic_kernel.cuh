// ka_cubic_kernel.cuh -- cubic-lattice sweep kernel (one bond-class group per launch).
//
// A group (mu, par) is the four classes c = 4(2 mu + par) + a, a = 0..3: all
// bonds along direction mu on the pencils (lines along mu) whose
// perpendicular coordinates sum to par mod 2.  Inside a group only those
// "active" pencils are written; their perpendicular neighbours lie on
// pencils of the other parity and stay fixed, so each site's count of
// occupied perpendicular neighbours is computed once per group.  Along a
// pencil the four classes are the bonds (4k+a, 4k+a+1), run in order.
//
// Exchange rule (section 2.1, rules (a)-(c); section 3.2 Table 1 with a
// random gate): on bond (i, j) the replicas with n_i != n_j, gate bit 1, at
// most m occupied among the other z-1 neighbours of i, and at most m among
// those of j, swap n_i and n_j; both sites lose their persistence bit.
// Everything is bit-sliced over the 64 replicas of one word.  A launch works
// on one state plane holding V words per site (V = 4, 2 or 1, the largest
// that divides the word count): with V = 4 every site is one full 32-byte
// sector.  Phase B runs one warp per (pencil, word).
//
// Gates: the bonds at pencil positions 4k+2b and 4k+2b+1 (classes 4g+2b and
// 4g+2b+1) take the two 64-bit halves of the Philox4x32-10 block at counter
// (sweep, 4g+2b, base site of the first, word).
//
// A persistent CTA walks tiles of 8 / V active pencils; while it computes one
// tile, the copies of its next tile are in flight (two staging buffers).
// Per tile it works in three phases:
//  A. memory-order pass: asynchronous copies (cp.async) of each active
//     site's word, its persistence word and its 2(d-1) perpendicular
//     neighbours into shared memory -- many copies in flight, no registers;
//  B. pencil order: one warp per (pencil, word), one lane per four-site segment;
//     the lane turns the staged neighbours into the masks A = [c <= m-1],
//     B = [c <= m] of its sites, runs the four classes, trading the
//     along-pencil neighbours with warp shuffles, and leaves n and p in
//     shared memory;
//  C. memory-order write-back of n and p.
// For mu = 0 the pencils are rows of memory; for mu > 0 a CTA takes the
// active pencils of a (16 / V)-column window along x, so a memory-order item
// walks along x.  Shared memory keeps one plane per word, with XOR-swizzled
// slots so the segment-order reads of phase B are free of bank conflicts.
//
// The kernel has one instance per (d, words per site, m, direction kind,
// batched or not); the instances are compiled in several translation units
// (ka_cubic_d*.cu), one per (d, batched), so that they build in parallel.
#pragma once

#include <mutex>

#include "ka_internal.cuh"

namespace ka {
namespace cubic {

#ifndef KA_CUBIC_MIN_BLOCKS
#define KA_CUBIC_MIN_BLOCKS 4
#endif
constexpr int kWarps = kCubicWarps;
constexpr int kThreads = 32 * kWarps;
// active pencils per CTA: 8 / V (mu = 0), or the active half of a
// (16 / V)-column window along x (mu > 0)
template <int V>
__host__ __device__ constexpr int tp_of() { return kWarps / V; }
template <int V>
__host__ __device__ constexpr int log2_of() { return V == 4 ? 2 : (V == 2 ? 1 : 0); }

struct GroupArgs {
  uint64_t* n;  // word plane
  uint64_t* p;
  int L, S, PW;   // pencil length, segments per pencil, pencils per warp (phase B)
  int mu, par;
  int64_t NP;     // active pencils (mu = 0)
  int nwin;       // x windows (mu > 0)
  int64_t st[4];  // strides L^k
  int pd[3];      // perpendicular dimensions, ascending
  int PS;         // shared-memory entries per pencil (odd, >= the swizzled slots)
  uint32_t ntiles;  // tiles (CTA work items) of the launch
  uint32_t t, cls0, word0;  // word0: global index of the plane's first word
  RoundKeys rk;
};

// Launch one group over the instance of dimension D (batched if B): V words
// per site, x = pencils along memory rows; returns the launch error.
template <int D, bool B>
cudaError_t launch_d(int V, bool x, const GroupArgs& a, const BatchArgs& ba, int m, unsigned blocks,
                     size_t smem, cudaStream_t st);

#define KA_CUBIC_EXTERN(DD)                                                                   \
  extern template cudaError_t launch_d<DD, false>(int, bool, const GroupArgs&, const BatchArgs&, \
                                                  int, unsigned, size_t, cudaStream_t);       \
  extern template cudaError_t launch_d<DD, true>(int, bool, const GroupArgs&, const BatchArgs&,  \
                                                 int, unsigned, size_t, cudaStream_t);
KA_CUBIC_EXTERN(1)
KA_CUBIC_EXTERN(2)
KA_CUBIC_EXTERN(3)
KA_CUBIC_EXTERN(4)
#undef KA_CUBIC_EXTERN

#ifdef KA_CUBIC_INSTANCES
namespace {


__device__ __forceinline__ uint64_t maj3(uint64_t a, uint64_t b, uint64_t c) {
  return (a & b) | (c & (a | b));
}

// [count <= T] for a bit-sliced 3-bit count (b2 b1 b0); T is a compile-time constant
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
    return ~g2;  // not (count > T)
  }
}

// bit-sliced count of K perpendicular neighbour words (K = 0, 2, 4 or 6)
template <int K>
__device__ __forceinline__ void count_perp(const uint64_t* x, uint64_t& b2, uint64_t& b1,
                                           uint64_t& b0) {
  if constexpr (K == 0) {
    b2 = b1 = b0 = 0;
  } else if constexpr (K == 2) {
    b0 = x[0] ^ x[1];
    b1 = x[0] & x[1];
    b2 = 0;
  } else if constexpr (K == 4) {
    const uint64_t s = x[0] ^ x[1] ^ x[2], c = maj3(x[0], x[1], x[2]);
    b0 = s ^ x[3];
    const uint64_t k = s & x[3];
    b1 = c ^ k;
    b2 = c & k;
  } else {
    const uint64_t s1 = x[0] ^ x[1] ^ x[2], c1 = maj3(x[0], x[1], x[2]);
    const uint64_t s2 = x[3] ^ x[4] ^ x[5], c2 = maj3(x[3], x[4], x[5]);
    b0 = s1 ^ s2;
    const uint64_t k = s1 & s2;
    b1 = c1 ^ c2 ^ k;
    b2 = maj3(c1, c2, k);
  }
}

// swizzled shared-memory slot of position t along a pencil (one word per
// entry): lanes reading positions 4l + k, or 32i + l, hit distinct banks
__device__ __forceinline__ int slot(int t) { return t ^ ((t >> 2) & 15); }

// asynchronous 8-byte global -> shared copy
__device__ __forceinline__ void cp_async8(uint64_t* s, const uint64_t* g) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(g) : "memory");
}

// L2 eviction priority for the persistence plane p.  A group touches p only
// on its active sites and the next group does not read those lines again,
// while it does read the n lines (its active pencils were this group's
// neighbours and the other way round); marking p's lines evict-first keeps
// more of n in L2 from one launch to the next.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}

// cp_async8 with an L2 cache policy
__device__ __forceinline__ void cp_async8_hint(uint64_t* s, const uint64_t* g, uint64_t pol) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(g),
               "l"(pol)
               : "memory");
}

// 8-byte global store with an L2 cache policy
__device__ __forceinline__ void st_hint(uint64_t* g, uint64_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;\n" ::"l"(g), "l"(v), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Which active pencils a CTA owns.
template <int D, int V, bool X>
struct PencilMap {
  static constexpr int kTP = tp_of<V>();
  static constexpr int kWin = 2 * tp_of<V>();
  uint32_t b0;  // first active pencil (mu = 0)
  int count;    // active pencils in this CTA
  int x0;       // x window start (mu > 0)
  int off;      // parity offset of the active x columns (mu > 0)
  int yo[2];    // coordinates of the other perpendicular dims (mu > 0)

  __device__ __forceinline__ void init(const GroupArgs& a, uint32_t tile) {
    yo[0] = yo[1] = 0;
    if constexpr (X) {
      b0 = tile * (uint32_t)kTP;
      const int64_t left = a.NP - (int64_t)b0;
      count = left < kTP ? (int)left : kTP;
      x0 = off = 0;
    } else {
      const int w = (int)(tile % (unsigned)a.nwin);
      uint32_t rest = tile / (unsigned)a.nwin;
      int s = 0;
#pragma unroll
      for (int k = 0; k < D - 2; ++k) {
        const uint32_t q = rest / (uint32_t)a.L;
        yo[k] = (int)(rest - q * (uint32_t)a.L);
        rest = q;
        s += yo[k];
      }
      x0 = w * kWin;
      const int width = (a.L - x0) < kWin ? (a.L - x0) : kWin;
      count = width / 2;
      off = (a.par + s) & 1;
      b0 = 0;
    }
  }

  // perpendicular coordinates y[k] (along dims pd[k]) of pencil j; returns
  // the site index of its position 0
  __device__ __forceinline__ uint32_t coords(const GroupArgs& a, int j, int* y) const {
    uint32_t base = 0;
    if constexpr (D >= 2) {
      if constexpr (X) {
        const uint32_t pi = b0 + (uint32_t)j;
        const uint32_t half = (uint32_t)a.L >> 1;
        uint32_t rest = pi / half;
        const int r0 = (int)(pi - rest * half);
        int hi = 0;
#pragma unroll
        for (int k = 1; k < D - 1; ++k) {
          const uint32_t q = rest / (uint32_t)a.L;
          y[k] = (int)(rest - q * (uint32_t)a.L);
          rest = q;
          hi += y[k];
        }
        y[0] = 2 * r0 + ((a.par + hi) & 1);
      } else {
        y[0] = x0 + 2 * j + off;
#pragma unroll
        for (int k = 1; k < D - 1; ++k) y[k] = yo[k - 1];
      }
#pragma unroll
      for (int k = 0; k < D - 1; ++k) base += (uint32_t)y[k] * (uint32_t)a.st[a.pd[k]];
    }
    return base;
  }
};

// Per-pencil table of a CTA, built once in shared memory: the position of
// the pencil's site 0 in the plane, the signed offsets to the perpendicular
// neighbours (with the periodic wrap folded in), both in the plane's site
// order, and the canonical index of site 0 (the gate counters).
template <int D>
struct PencilInfo {
  uint32_t base;
  uint32_t cbase;
  int32_t nb[2 * (D - 1) > 0 ? 2 * (D - 1) : 1];
};

// offset of x within its row in the split-row order of a plane (d >= 2):
// even x first, then odd x
__device__ __forceinline__ int32_t xoff(int x, int L) { return (x & 1) * (L >> 1) + (x >> 1); }

template <int D, int V, bool X>
__device__ __forceinline__ void build_info(const GroupArgs& a, const PencilMap<D, V, X>& pm, int j,
                                           PencilInfo<D>& out) {
  int y[3] = {0, 0, 0};
  out.cbase = pm.coords(a, j, y);
  out.base = out.cbase;
#pragma unroll
  for (int k = 0; k < D - 1; ++k) {
    const int32_t s = (int32_t)a.st[a.pd[k]];
    out.nb[2 * k] = (y[k] == a.L - 1) ? -(a.L - 1) * s : s;
    out.nb[2 * k + 1] = (y[k] == 0) ? (a.L - 1) * s : -s;
  }
  if constexpr (D >= 2 && !X) {
    // the pencil sits at x = y[0] (dimension 0 is perpendicular); its x
    // neighbours are in the other half of the row
    const int L = a.L, x = y[0];
    out.base = out.cbase - (uint32_t)x + (uint32_t)xoff(x, L);
    out.nb[0] = xoff(x == L - 1 ? 0 : x + 1, L) - xoff(x, L);
    out.nb[1] = xoff(x == 0 ? L - 1 : x - 1, L) - xoff(x, L);
  }
}

// position in the plane of site t of a pencil whose site 0 is at `base`
template <int D, bool X>
__device__ __forceinline__ uint32_t pencil_pos(uint32_t base, int t, uint32_t smu, int L) {
  if constexpr (X && D >= 2) {
    return base + (uint32_t)xoff(t, L);  // rows in split-row order
  } else {
    return base + (uint32_t)t * smu;
  }
}

// Memory-order walk of phases A and C over the tile's elements (site, word h).
// A thread keeps one pencil j and visits elements f = f0, f0 + step, ...
//   mu = 0: a pencil is a row of L sites x V words; V warps share pencil
//           warp % TP and their lanes walk consecutive elements of the row.
//   mu > 0: the TP pencils of a window sit at x0 + 2j + off; the E = TP V
//           elements (j, h) of one row are lanes lane % E, and a warp covers
//           32 / E rows (positions t = lane / E + (32 / E) warp, step 32 / E
//           times the warps).
// Returns the position t and word h of element f.
template <int V, bool X>
__device__ __forceinline__ void elem_start(int warp, int lane, int& j, int& h, int& f0,
                                           int& step) {
  constexpr int TP = tp_of<V>();
  if constexpr (X) {
    j = warp % TP;
    h = 0;
    f0 = lane + 32 * (warp / TP);
    step = 32 * V;
  } else {
    constexpr int E = TP * V;  // elements (pencil, word) of one row: one lane each
    j = (lane % E) / V;
    h = (lane % E) % V;
    f0 = lane / E + (32 / E) * warp;
    step = (32 / E) * kWarps;
  }
}

// Fill the arguments of one unit for group (mu, par) of its current sweep;
// sets ntiles = 0 when the unit has finished its sweeps.
template <int V>
__device__ void unit_args(const CubicUnit& u, const BatchArgs& ba, GroupArgs& a) {
  a.n = u.n;
  a.p = u.p;
  a.L = u.L;
  a.S = u.L / 4;
  a.PW = 32 / a.S;
  a.mu = ba.mu;
  a.par = ba.par;
  a.st[0] = 1;
  for (int k = 1; k < 4; ++k) a.st[k] = a.st[k - 1] * u.L;
  int j = 0;
  for (int k = 0; k < u.d; ++k)
    if (k != ba.mu) a.pd[j++] = k;
  for (; j < 3; ++j) a.pd[j] = 0;
  a.NP = 1;
  for (int k = 0; k < u.d - 1; ++k) a.NP *= u.L;
  if (u.d >= 2) a.NP /= 2;
  const int win = 2 * tp_of<V>();
  a.nwin = (u.L + win - 1) / win;
  a.PS = ((u.L + 15) / 16) * 16 + 1;
  const uint32_t t = u.t_base + ba.sweep_offset;
  a.t = t;
  a.cls0 = (uint32_t)(4 * (2 * ba.mu + ba.par));
  a.word0 = u.word0;
  a.rk = u.rk;
  const bool x = (ba.mu == 0) || u.d == 1;
  int64_t tiles;
  if (x) {
    tiles = (a.NP + tp_of<V>() - 1) / tp_of<V>();
  } else {
    tiles = a.nwin;
    for (int k = 0; k < u.d - 2; ++k) tiles *= u.L;
  }
  a.ntiles = (t < u.t_end) ? (uint32_t)tiles : 0u;
}

// Resolve global tile g of a batched launch: the arguments of the unit that
// owns it and its tile index within that unit.
template <int V, bool X>
__device__ void resolve(const BatchArgs& ba, uint32_t g, GroupArgs& a, uint32_t& local) {
  const int mode = X ? 0 : 1;
  const uint32_t u = ba.tile_unit[g];
  unit_args<V>(ba.units[u], ba, a);
  local = g - ba.units[u].tile0[mode];
  if (local >= a.ntiles) a.ntiles = 0;  // finished unit: no work in this tile
}

// B selects the batched form: the arguments of every tile come from the unit
// table (through shared memory) instead of the launch's own parameters.
template <int D, int V, int M, bool X, bool B>
__global__ void __launch_bounds__(kThreads, KA_CUBIC_MIN_BLOCKS)
    k_cubic_group(const __grid_constant__ GroupArgs la, const __grid_constant__ BatchArgs ba) {
  constexpr int KP = 2 * (D - 1);
  constexpr int TP = tp_of<V>();
  extern __shared__ __align__(16) uint64_t smem[];
  // two staging buffers; each holds n, p, then the KP neighbour arrays, one
  // plane of [TP][PSmax] words per array and word
  const int PSmax = B ? ba.PSmax : la.PS;
  const uint32_t ntiles = B ? ba.ntiles : la.ntiles;
  const int plane = TP * PSmax;
  const int bufsize = (2 + KP) * V * plane;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t pol_p = l2_evict_first_policy();
  __shared__ PencilInfo<D> info[2][TP];
  __shared__ GroupArgs sargs[B ? 2 : 1];
  __shared__ uint32_t slocal[B ? 2 : 1];
  // the arguments of buffer b's tile: the unit's (batched) or the launch's
#define KA_TILE_ARGS(b) (B ? sargs[(b)] : la)

  // shared memory of buffer b: array a (0 = n, 1 = p, 2.. = neighbours), word
  // h is the plane [(a V + h)][TP][PSmax]
  auto splane = [&](int b, int arr, int h) -> uint64_t* {
    return smem + b * bufsize + (arr * V + h) * plane;
  };

  // asynchronous copies of one tile into buffer b (memory order)
  auto issue = [&](const GroupArgs& a, const PencilMap<D, V, X>& pm, int b) {
    const int L = a.L, PS = a.PS;
    const uint32_t smu = (uint32_t)a.st[a.mu];
    int j, h, f0, step;
    elem_start<V, X>(warp, lane, j, h, f0, step);
    if (j < pm.count) {
      const uint32_t base = info[b][j].base;
      int32_t nb[KP > 0 ? KP : 1];
#pragma unroll
      for (int k = 0; k < KP; ++k) nb[k] = info[b][j].nb[k];
      const int lim = X ? L * V : L;
      for (int f = f0; f < lim; f += step) {
        int t, hh;
        if constexpr (X) {
          t = f >> log2_of<V>();
          hh = f & (V - 1);
        } else {
          t = f;
          hh = h;
        }
        const uint32_t site = pencil_pos<D, X>(base, t, smu, L);
        const int e = j * PS + slot(t);
        cp_async8(splane(b, 0, hh) + e, a.n + (size_t)site * V + hh);
        cp_async8_hint(splane(b, 1, hh) + e, a.p + (size_t)site * V + hh, pol_p);
#pragma unroll
        for (int k = 0; k < KP; ++k)
          cp_async8(splane(b, 2 + k, hh) + e, a.n + (size_t)(site + (uint32_t)nb[k]) * V + hh);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // set up buffer b for global tile g: arguments, pencil map and pencil table
  auto prepare = [&](uint32_t g, int b, PencilMap<D, V, X>& pm) {
    uint32_t local = g;
    if constexpr (B) {
      if (threadIdx.x == 0) resolve<V, X>(ba, g, sargs[b], slocal[b]);
      __syncthreads();
      if (sargs[b].ntiles == 0) {
        pm.count = 0;
        return;
      }
      local = slocal[b];
    }
    const GroupArgs& a = KA_TILE_ARGS(b);
    pm.init(a, local);
    if (threadIdx.x < pm.count) build_info<D, V, X>(a, pm, threadIdx.x, info[b][threadIdx.x]);
  };

  // prologue: the CTA's first tile.  Single-instance launches are chained
  // with programmatic dependent launch: the next group may start as soon as
  // every CTA of this one runs, and this one prepares its first tile (static
  // tables only) before waiting for the previous group to finish writing the
  // state.  Without that launch attribute the wait returns at once.  The
  // batched form never lets a dependent start early: a waiting grid would
  // share the SMs with this one for its whole run.
  if constexpr (!B) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  uint32_t tile = blockIdx.x;
  PencilMap<D, V, X> pm;
  prepare(tile, 0, pm);
  __syncthreads();
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  issue(KA_TILE_ARGS(0), pm, 0);

  for (int it = 0; tile < ntiles; ++it) {
    const int b = it & 1;
    const uint32_t nxt = tile + gridDim.x;
    const bool more = nxt < ntiles;
    PencilMap<D, V, X> pn;
    pn.count = 0;
    if (more) prepare(nxt, b ^ 1, pn);
    __syncthreads();
    // start the next tile's copies, then wait for this tile's
    if (more) {
      issue(KA_TILE_ARGS(b ^ 1), pn, b ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();

    const GroupArgs& a = KA_TILE_ARGS(b);
    const int L = a.L, PS = a.PS;
    const uint32_t smu = (uint32_t)a.st[a.mu];
    const int count = pm.count;

  // ---- phase B: pencil order, one warp per (pencil group, word)
  {
    const int S = a.S, PW = a.PW;
    const int h = warp % V;
    const int gj = lane / S, seg = lane - gj * S;
    const int groups = (count + PW - 1) / PW;
    const uint32_t word = a.word0 + (uint32_t)h;
    uint64_t* sN = splane(b, 0, h);
    uint64_t* sP = splane(b, 1, h);
    for (int g = warp / V; g < groups; g += kWarps / V) {
      const int j = g * PW + gj;
      const bool valid = gj < PW && j < count;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const int prev = gj * S + (seg == 0 ? S - 1 : seg - 1);
        const int next = gj * S + (seg == S - 1 ? 0 : seg + 1);
        const uint32_t s0 = info[b][j].cbase + (uint32_t)(4 * seg) * smu;
        // gate blocks: classes (0, 1) share one, (2, 3) the other; they do not
        // depend on the state, so start them first
        const uint4 g01 = philox(make_uint4(a.t, a.cls0, s0, word), a.rk);
        const uint4 g23 = philox(make_uint4(a.t, a.cls0 + 2, s0 + 2 * smu, word), a.rk);
        int e[4];
        uint64_t nn[4], mA[4], mB[4], fl[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          e[k] = j * PS + slot(4 * seg + k);
          nn[k] = sN[e[k]];
          uint64_t xs[KP > 0 ? KP : 1];
#pragma unroll
          for (int q = 0; q < KP; ++q) xs[q] = splane(b, 2 + q, h)[e[k]];
          uint64_t b2, b1, b0;
          count_perp<KP>(xs, b2, b1, b0);
          mA[k] = le3<M - 1>(b2, b1, b0);
          mB[k] = le3<M>(b2, b1, b0);
          fl[k] = 0;
        }
        // class 0: bond (s0, s1); s0's other along-neighbour is the previous
        // segment's s3 (still at its group-start value), s1's is s2
        {
          const uint64_t left = __shfl_sync(act, nn[3], prev);
          const uint64_t ok0 = (left & mA[0]) | (~left & mB[0]);
          const uint64_t ok1 = (nn[2] & mA[1]) | (~nn[2] & mB[1]);
          const uint64_t sw = (nn[0] ^ nn[1]) & lo64(g01) & ok0 & ok1;
          nn[0] ^= sw;
          nn[1] ^= sw;
          fl[0] |= sw;
          fl[1] |= sw;
        }
        // class 1: bond (s1, s2); other along-neighbours s0 and s3
        {
          const uint64_t ok1 = (nn[0] & mA[1]) | (~nn[0] & mB[1]);
          const uint64_t ok2 = (nn[3] & mA[2]) | (~nn[3] & mB[2]);
          const uint64_t sw = (nn[1] ^ nn[2]) & hi64(g01) & ok1 & ok2;
          nn[1] ^= sw;
          nn[2] ^= sw;
          fl[1] |= sw;
          fl[2] |= sw;
        }
        // class 2: bond (s2, s3); s3's other along-neighbour is the next
        // segment's s0, which only class 0 has written so far
        const uint64_t right = __shfl_sync(act, nn[0], next);
        {
          const uint64_t ok2 = (nn[1] & mA[2]) | (~nn[1] & mB[2]);
          const uint64_t ok3 = (right & mA[3]) | (~right & mB[3]);
          const uint64_t sw = (nn[2] ^ nn[3]) & lo64(g23) & ok2 & ok3;
          nn[2] ^= sw;
          nn[3] ^= sw;
          fl[2] |= sw;
          fl[3] |= sw;
        }
        // class 3: bond (s3, next s0); the owner of next s0 evaluates that
        // site's condition (its other along-neighbour is its s1) and sends it
        {
          const uint64_t mine = (nn[1] & mA[0]) | (~nn[1] & mB[0]);
          const uint64_t okn = __shfl_sync(act, mine, next);
          const uint64_t ok3 = (nn[2] & mA[3]) | (~nn[2] & mB[3]);
          const uint64_t sw = (nn[3] ^ right) & hi64(g23) & ok3 & okn;
          nn[3] ^= sw;
          fl[3] |= sw;
          const uint64_t in = __shfl_sync(act, sw, prev);
          nn[0] ^= in;
          fl[0] |= in;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          sN[e[k]] = nn[k];
          sP[e[k]] &= ~fl[k];
        }
      }
    }
  }
  __syncthreads();

  // ---- phase C: memory-order write-back of n and p
  {
    int j, h, f0, step;
    elem_start<V, X>(warp, lane, j, h, f0, step);
    if (j < count) {
      const uint32_t base = info[b][j].base;
      const int lim = X ? L * V : L;
#pragma unroll 2
      for (int f = f0; f < lim; f += step) {
        int t, hh;
        if constexpr (X) {
          t = f >> log2_of<V>();
          hh = f & (V - 1);
        } else {
          t = f;
          hh = h;
        }
        const uint32_t site = pencil_pos<D, X>(base, t, smu, L);
        const int e = j * PS + slot(t);
        a.n[(size_t)site * V + hh] = splane(b, 0, hh)[e];
        st_hint(a.p + (size_t)site * V + hh, splane(b, 1, hh)[e], pol_p);
      }
    }
  }
    __syncthreads();  // buffer b and info[b] are free again
    pm = pn;
    tile = nxt;
  }
}

#undef KA_TILE_ARGS

// Per kernel instance and device: the dynamic shared memory granted so far
// and the resident CTAs per SM at the last shared-memory size.  Guarded, as
// contexts may be created and swept from several host threads.
struct LaunchCache {
  static constexpr int kDevices = 16;
  std::mutex mu;
  size_t granted[kDevices] = {}, occ_smem[kDevices] = {};
  int per_sm[kDevices] = {}, sms[kDevices] = {};
};

// Launch a persistent grid (at most as many CTAs as fit on the device at
// once), with programmatic stream serialisation if pdl.  Single-instance
// sweeps use it (a group's first tile is prepared while the previous group
// drains); batched rounds do not, where it measured slower.
template <typename Kern>
cudaError_t launch_persistent(Kern kern, LaunchCache& lc, const GroupArgs& a, const BatchArgs& ba,
                              unsigned blocks, size_t smem, cudaStream_t st, bool pdl) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= LaunchCache::kDevices) return cudaErrorInvalidDevice;
  unsigned cap;
  {
    std::lock_guard<std::mutex> lock(lc.mu);
    if (smem > lc.granted[dev]) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      lc.granted[dev] = smem;
    }
    if (lc.per_sm[dev] == 0 || lc.occ_smem[dev] != smem) {
      int per_sm = 0, sms = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
      lc.per_sm[dev] = per_sm < 1 ? 1 : per_sm;
      lc.sms[dev] = sms < 1 ? 1 : sms;
      lc.occ_smem[dev] = smem;
    }
    cap = (unsigned)(lc.per_sm[dev] * lc.sms[dev]);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks < cap ? blocks : cap);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, ba);
}

template <int D, int V, bool X, bool B>
cudaError_t launch_dx(const GroupArgs& a, const BatchArgs& ba, int m, unsigned blocks, size_t smem,
                      cudaStream_t st) {
  constexpr int Z = 2 * D;
  const int mm = m < Z - 1 ? m : Z - 1;
  switch (mm) {
#define KA_CASE(MM)                                                                    \
  case MM:                                                                             \
    if constexpr (MM <= Z - 1) {                                                       \
      static LaunchCache lc;                                                           \
      return launch_persistent(k_cubic_group<D, V, MM, X, B>, lc, a, ba, blocks, smem, \
                               st, !B);                                                \
    }                                                                                  \
    break;
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
      break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace

template <int D, bool B>
cudaError_t launch_d(int V, bool x, const GroupArgs& a, const BatchArgs& ba, int m, unsigned blocks,
                     size_t smem, cudaStream_t st) {
  if constexpr (D == 1) {
    if (V == 4) return launch_dx<1, 4, true, B>(a, ba, m, blocks, smem, st);
    return V == 2 ? launch_dx<1, 2, true, B>(a, ba, m, blocks, smem, st)
                  : launch_dx<1, 1, true, B>(a, ba, m, blocks, smem, st);
  } else {
    if (V == 4)
      return x ? launch_dx<D, 4, true, B>(a, ba, m, blocks, smem, st)
               : launch_dx<D, 4, false, B>(a, ba, m, blocks, smem, st);
    if (V == 2)
      return x ? launch_dx<D, 2, true, B>(a, ba, m, blocks, smem, st)
               : launch_dx<D, 2, false, B>(a, ba, m, blocks, smem, st);
    return x ? launch_dx<D, 1, true, B>(a, ba, m, blocks, smem, st)
             : launch_dx<D, 1, false, B>(a, ba, m, blocks, smem, st);
  }
}
#endif  // KA_CUBIC_INSTANCES

}  // namespace cubic
}  // namespace ka
