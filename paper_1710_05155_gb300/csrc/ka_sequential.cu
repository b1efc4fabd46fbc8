// ka_sequential.cu -- the random-sequential schedule of section 3.2.
//
// The paper's own update: each step picks one bond at random, shared by all
// replicas packed in a word, and exchanges the two sites in every replica
// where the rule of section 2.1 allows it (no per-replica gate).  N attempts
// make a sweep (the time unit of section 2.1).  Attempt k of sweep t of word
// w draws r uniform in [0, N z) by Lemire's method on the low 64 bits of the
// Philox block at counter (t, 0xFFFFFFFC - draw, k, w), key = seed, and takes
// site i = r / z and its neighbour in slot r mod z (slots 2 mu and 2 mu + 1
// are the up and down neighbours along mu on a cubic lattice; on a graph the
// slots follow the neighbour row, kept in ascending order).
//
// The attempts of one word form a chain; one warp runs one word and applies
// its attempts 32 at a time, one per lane, with the result of the chain in
// order.  An attempt reads n on its read set R = {i, j} and the neighbours
// of i and of j, and writes n and p on W = {i, j}.  Attempts k and l
// conflict when W_k meets R_l or W_l meets R_k.  The neighbour relation is
// symmetric (cubic lattices by construction, graphs are checked when the
// context is made), so the two are the same condition: a site of W_k equals
// a site of W_l or neighbours one.  Every attempt sets its lane bit in a
// shared-memory stamp word of both sites of W, then ORs the stamps over R
// (sites share a stamp modulo the table size when N is larger; a shared
// stamp can only add conflicts).  The warp applies the
// pending attempts in rounds: in each, every pending attempt that conflicts
// with no earlier pending attempt (a set that always holds the earliest)
// reads, decides and writes.  Such an attempt sees exactly the state the
// chain would give it: no earlier attempt still pending writes what it
// reads, and it writes nothing that an earlier pending attempt has yet to
// read; attempts applied in one round touch disjoint sites.  The word's n
// and p planes sit in shared memory when they fit, else in global memory.
#include <algorithm>
#include <string>

#include "ka_ctx.cuh"

namespace ka {
namespace {

constexpr uint32_t kTagSequential = 0xFFFFFFFCu;
constexpr int kSmemWords = 20480;  // n and p of up to 10240 sites in shared memory
constexpr uint32_t kStampsGlobal = 32768;  // stamp words when the planes stay in global memory

struct SeqArgs {
  uint64_t* n;
  uint64_t* p;
  const int32_t* nbr;  // [N][z], or null: periodic cubic lattice from coordinates
  int64_t N;
  int z, d, L, V;
  int xs;  // split-row order of the planes (0: index order)
  const int32_t* perm;  // graphs: storage position of every canonical site (nbr in positions)
  size_t plane_elems;
  uint32_t t0;
  int nsweeps;
  uint32_t hmask;  // stamp words - 1 (a power of two)
  RoundKeys rk;
};

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

// the bond draw of attempt k: r uniform in [0, range)
__device__ __forceinline__ uint64_t draw_bond(const RoundKeys& rk, uint32_t t, uint32_t k,
                                              uint32_t w, uint64_t range) {
  uint32_t draw = 0;
  uint64_t x = lo64(philox(make_uint4(t, kTagSequential, k, w), rk));
  uint64_t low = x * range;
  if (low < range) {
    const uint64_t threshold = (0ull - range) % range;
    while (low < threshold) {
      ++draw;
      x = lo64(philox(make_uint4(t, kTagSequential - draw, k, w), rk));
      low = x * range;
    }
  }
  return __umul64hi(x, range);
}

// the 2d neighbours of site i of a periodic cubic lattice, slot 2 mu up and
// 2 mu + 1 down along mu (32-bit arithmetic: N z < 2^32)
__device__ __forceinline__ void cubic_neighbours(const SeqArgs& a, uint32_t i, uint32_t (&out)[8]) {
  uint32_t rest = i, stride = 1;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    if (mu >= a.d) break;
    const uint32_t L = (uint32_t)a.L, q = rest / L, x = rest - q * L;
    rest = q;
    out[2 * mu] = (x == L - 1) ? i - (L - 1) * stride : i + stride;
    out[2 * mu + 1] = (x == 0) ? i + (L - 1) * stride : i - stride;
    stride *= L;
  }
}

// the z neighbours of site i
__device__ __forceinline__ void neighbours(const SeqArgs& a, uint32_t i, uint32_t (&out)[8]) {
  if (a.nbr) {
#pragma unroll
    for (int s = 0; s < 8; ++s)
      if (s < a.z) out[s] = (uint32_t)a.nbr[(int64_t)i * a.z + s];
  } else {
    cubic_neighbours(a, i, out);
  }
}

// one warp per word; n and p of the word at stride `st` (V in global memory,
// 1 in shared memory)
template <int M, bool SMEM>
__global__ void __launch_bounds__(32) k_sequential(const __grid_constant__ SeqArgs a) {
  extern __shared__ uint64_t sm[];
  const int lane = threadIdx.x;
  const uint32_t w = blockIdx.x;  // word index
  const int q = (int)(w / (uint32_t)a.V), h = (int)(w % (uint32_t)a.V);
  uint64_t* gn = a.n + (size_t)q * a.plane_elems + h;
  uint64_t* gp = a.p + (size_t)q * a.plane_elems + h;
  uint64_t* n = gn;
  uint64_t* p = gp;
  int64_t st = a.V;
  if constexpr (SMEM) {
    // shared memory holds the word's planes in site index order
    // (graphs: storage order, the labels the neighbour table uses)
    for (int64_t i = lane; i < a.N; i += 32) {
      const int64_t g = (a.perm ? i : dev_site(a.xs, i)) * a.V;
      sm[i] = gn[g];
      sm[a.N + i] = gp[g];
    }
    __syncwarp();
    n = sm;
    p = sm + a.N;
    st = 1;
  }
  // element of site i in n and p
  auto at = [&](uint32_t i) -> int64_t {
    return SMEM ? (int64_t)i : (a.perm ? (int64_t)i : dev_site(a.xs, i)) * st;
  };
  uint32_t* stamp = reinterpret_cast<uint32_t*>(sm + (SMEM ? 2 * a.N : 0));
  const uint32_t hm = a.hmask;
  for (uint32_t b = lane; b <= hm; b += 32) stamp[b] = 0;
  __syncwarp();
  const uint64_t range = (uint64_t)a.N * (uint64_t)a.z;
  const uint32_t earlier = (1u << lane) - 1u;  // lanes of the earlier attempts
  for (int s = 0; s < a.nsweeps; ++s) {
    const uint32_t t = a.t0 + (uint32_t)s;
    for (int64_t k0 = 0; k0 < a.N; k0 += 32) {
      const int64_t k = k0 + lane;
      const bool live = k < a.N;
      const uint64_t r = live ? draw_bond(a.rk, t, (uint32_t)k, w, range) : 0ull;
      // this lane's bond (i, j) and the neighbours of both: drawn by
      // canonical site and slot, then (graphs) followed in storage positions
      uint32_t i = (uint32_t)(r / (uint64_t)a.z);
      if (a.perm && live) i = (uint32_t)a.perm[i];
      const int sel = (int)(r % (uint64_t)a.z);
      uint32_t ni_[8], nj_[8];
      neighbours(a, i, ni_);
      uint32_t j = 0;
#pragma unroll
      for (int s2 = 0; s2 < 8; ++s2)
        if (s2 == sel) j = ni_[s2];
      neighbours(a, j, nj_);
      // bit o of conf: attempt o writes a site this attempt reads (or one
      // sharing its stamp)
      if (live) {
        atomicOr(&stamp[i & hm], 1u << lane);
        atomicOr(&stamp[j & hm], 1u << lane);
      }
      __syncwarp();
      uint32_t conf = stamp[i & hm] | stamp[j & hm];
#pragma unroll
      for (int slot = 0; slot < 8; ++slot) {
        if (slot >= a.z) break;
        conf |= stamp[ni_[slot] & hm] | stamp[nj_[slot] & hm];
      }
      __syncwarp();
      if (live) {
        stamp[i & hm] = 0;
        stamp[j & hm] = 0;
      }
      __syncwarp();
      uint32_t pending = __ballot_sync(0xffffffffu, live);
      while (pending) {
        const bool ready = ((pending >> lane) & 1u) && !(conf & pending & earlier);
        if (ready) {
          const uint64_t vi = n[at(i)], vj = n[at(j)];
          uint64_t ci2 = 0, ci1 = 0, ci0 = 0, cj2 = 0, cj1 = 0, cj0 = 0;
#pragma unroll
          for (int slot = 0; slot < 8; ++slot) {
            if (slot >= a.z) break;
            if (ni_[slot] != j) add3(ci2, ci1, ci0, n[at(ni_[slot])]);
            if (nj_[slot] != i) add3(cj2, cj1, cj0, n[at(nj_[slot])]);
          }
          // at most m occupied among the other neighbours of i and of j
          const uint64_t ok = le3<M>(ci2, ci1, ci0) & le3<M>(cj2, cj1, cj0);
          const uint64_t sw = (vi ^ vj) & ok;
          if (sw) {
            n[at(i)] = vi ^ sw;
            n[at(j)] = vj ^ sw;
            p[at(i)] &= ~sw;
            p[at(j)] &= ~sw;
          }
        }
        pending &= ~__ballot_sync(0xffffffffu, ready);
        __syncwarp();
      }
    }
  }
  if constexpr (SMEM) {
    __syncwarp();
    for (int64_t i = lane; i < a.N; i += 32) {
      const int64_t g = (a.perm ? i : dev_site(a.xs, i)) * a.V;
      gn[g] = sm[i];
      gp[g] = sm[a.N + i];
    }
  }
}

template <bool SMEM>
cudaError_t launch_m(const SeqArgs& a, int m, unsigned words, size_t smem, cudaStream_t st) {
  switch (m < 7 ? m : 7) {
#define KA_CASE(MM)                                                                        \
  case MM: {                                                                               \
    auto kern = k_sequential<MM, SMEM>;                                                    \
    if (smem > 48 * 1024) {                                                                \
      const cudaError_t e =                                                                \
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                      \
    }                                                                                      \
    kern<<<words, 32, smem, st>>>(a);                                                      \
    return cudaGetLastError();                                                             \
  }
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
}  // namespace ka

extern "C" ka_status ka_sweep_sequential(ka_ctx* c, int64_t nsweeps) {
  ka::NvtxRange nvtx_range("ka_sweep_sequential");
  using namespace ka;
  if (!c || nsweeps < 0) return KA_EINVAL;
  if (!c->initialized) {
    c->err = "sequential sweep before init or set_state";
    return KA_ESTATE;
  }
  if (c->sweep + nsweeps > ((int64_t)1 << 32)) {
    c->err = "sweep counter would pass 2^32";
    return KA_EINVAL;
  }
  if ((uint64_t)c->N * (uint64_t)c->z > 0xFFFFFFFFull) {
    c->err = "N z must stay below 2^32";
    return KA_EINVAL;
  }
  if (nsweeps == 0) return KA_OK;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || prev == c->device) prev = -1;
  if (prev >= 0) cudaSetDevice(c->device);
  SeqArgs a{};
  a.n = c->pl.n;
  a.p = c->pl.p;
  a.nbr = c->pencil ? nullptr : c->g.nbr;
  a.N = c->N;
  a.z = c->z;
  a.d = c->d;
  a.L = c->L;
  a.V = c->pl.V;
  a.xs = c->pl.xs;
  a.perm = c->g.perm;
  a.plane_elems = c->pl.plane_elems();
  a.rk = c->rk;
  const unsigned words = (unsigned)(c->R / 64);
  const bool smem = 2 * c->N <= kSmemWords;
  // stamp table: one word per site when the planes are in shared memory
  // (exact), else kStampsGlobal words shared modulo their count
  uint32_t H = 32;
  if (smem) {
    while ((int64_t)H < c->N) H <<= 1;
  } else {
    H = kStampsGlobal;
  }
  a.hmask = H - 1;
  const size_t smem_bytes = (smem ? (size_t)2 * c->N * sizeof(uint64_t) : 0) + (size_t)H * 4;
  if (smem_bytes > (size_t)227 * 1024) {
    if (prev >= 0) cudaSetDevice(prev);
    c->err = "sequential sweep: shared memory plan too large";
    return KA_EINVAL;
  }
  // launches of at most about 2^20 attempts each
  const int64_t chunk = std::max<int64_t>(1, ((int64_t)1 << 20) / c->N);
  cudaError_t e = cudaSuccess;
  for (int64_t done = 0; done < nsweeps && !e; done += chunk) {
    a.t0 = (uint32_t)(c->sweep + done);
    a.nsweeps = (int)std::min<int64_t>(chunk, nsweeps - done);
    e = smem ? launch_m<true>(a, c->m, words, smem_bytes, c->stream)
             : launch_m<false>(a, c->m, words, smem_bytes, c->stream);
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (e) {
    c->err = std::string("sequential sweep: ") + cudaGetErrorString(e);
    return KA_ECUDA;
  }
  c->sweep += nsweeps;
  return KA_OK;
}
