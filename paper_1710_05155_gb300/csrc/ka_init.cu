// ka_init.cu -- initial state: exactly K particles per replica, uniform.
//
// Section 3.1 draws the initial configurations at fixed density at random.
// Replica r occupies the K sites with the smallest composite key
// (key_r(i), i), where key_r(i) is half (r mod 2) of the Philox block at
// counter (r / 2, 0xFFFFFFFF, i, 0): the first K entries of a uniformly
// random permutation, so every K-subset is equally likely.
//
// The K-th smallest composite key of every replica is found exactly by a
// most-significant-digit radix select over 8-bit digits: eight passes over
// the 64-bit key, then (only if some replica's threshold key is tied)
// passes over the site index.  Keys are recomputed instead of stored, which
// keeps the scratch at R x 256 counters.  When the context has room (its
// staging plane, idle during init), the sites whose key shares the threshold's
// top byte -- about N / 256 per replica -- are collected into per-replica
// lists after the first pass, and the later passes evaluate only those; a list
// that would overflow its capacity sends the later passes back to scanning
// all sites.  A final pass writes the bit planes: n = [composite <=
// threshold], n0 = n, p = all ones.
#include <algorithm>
#include <vector>

#include "ka_internal.cuh"

namespace ka {
namespace {

constexpr int kSitesPerThread = 32;

struct InitArgs {
  uint32_t* hist;
  uint32_t* cand_n;  // [R] candidates collected per replica
  uint32_t* cand;    // [R][cap] their site indices
  int64_t cap;
  uint64_t* pre_key;
  uint32_t* pre_idx;
  int64_t* krem;
  int32_t* unresolved;
  int64_t N;
  int idx_bits;  // bits of the site index digits (a multiple of 8)
  int pass;      // 0..7 key bytes from the top, then index bytes from the top
  RoundKeys rk;
};

// does the composite (key, i) agree with the decided digits of the threshold
// of replica r, and which digit does it have in this pass?
__device__ __forceinline__ bool digit_of(const InitArgs& a, uint64_t key, uint32_t i,
                                         uint64_t pk, uint32_t pi, int& digit) {
  const int p = a.pass;
  if (p < 8) {
    if (p > 0 && (key >> (64 - 8 * p)) != (pk >> (64 - 8 * p))) return false;
    digit = (int)((key >> (56 - 8 * p)) & 0xFF);
    return true;
  }
  if (key != pk) return false;
  const int ip = p - 8;  // index byte from the top
  const int top = a.idx_bits - 8 * ip;
  if (ip > 0 && (i >> top) != (pi >> top)) return false;
  digit = (int)((i >> (top - 8)) & 0xFF);
  return true;
}

// grid: x over site chunks, y over replica pairs
__global__ void __launch_bounds__(256) k_init_hist(const InitArgs a) {
  __shared__ uint32_t sh[2][256];
  const int rp = blockIdx.y;
  if (a.pass >= 8 && *a.unresolved == 0) return;  // uniform early exit
  for (int k = threadIdx.x; k < 512; k += blockDim.x) (&sh[0][0])[k] = 0;
  __syncthreads();
  const int r0 = 2 * rp;
  const bool live0 = a.krem[r0] > 0, live1 = a.krem[r0 + 1] > 0;
  if (live0 || live1) {
    const uint64_t pk0 = a.pre_key[r0], pk1 = a.pre_key[r0 + 1];
    const uint32_t pi0 = a.pre_idx[r0], pi1 = a.pre_idx[r0 + 1];
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kSitesPerThread + threadIdx.x;
    for (int s = 0; s < kSitesPerThread; ++s) {
      const int64_t i = i0 + (int64_t)s * blockDim.x;
      if (i >= a.N) break;
      const uint4 b = philox(make_uint4((uint32_t)rp, kTagInit, (uint32_t)i, 0u), a.rk);
      int dg;
      if (live0 && digit_of(a, lo64(b), (uint32_t)i, pk0, pi0, dg)) atomicAdd(&sh[0][dg], 1u);
      if (live1 && digit_of(a, hi64(b), (uint32_t)i, pk1, pi1, dg)) atomicAdd(&sh[1][dg], 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 512; k += blockDim.x) {
    const uint32_t c = (&sh[0][0])[k];
    if (c) atomicAdd(&a.hist[(size_t)(r0 + (k >> 8)) * 256 + (k & 255)], c);
  }
}

// After pass 0: collect the sites whose key has the threshold's top byte
// (the only ones later passes can count), per replica.
__global__ void __launch_bounds__(256) k_init_collect(const InitArgs a) {
  const int rp = blockIdx.y;
  const int r0 = 2 * rp;
  const bool live0 = a.krem[r0] > 0, live1 = a.krem[r0 + 1] > 0;
  if (!live0 && !live1) return;
  const uint64_t top0 = a.pre_key[r0] >> 56, top1 = a.pre_key[r0 + 1] >> 56;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kSitesPerThread + threadIdx.x;
  for (int s = 0; s < kSitesPerThread; ++s) {
    const int64_t i = i0 + (int64_t)s * blockDim.x;
    if (i >= a.N) break;
    const uint4 b = philox(make_uint4((uint32_t)rp, kTagInit, (uint32_t)i, 0u), a.rk);
    if (live0 && (lo64(b) >> 56) == top0) {
      const uint32_t k = atomicAdd(&a.cand_n[r0], 1u);
      if (k < (uint64_t)a.cap) a.cand[(size_t)r0 * a.cap + k] = (uint32_t)i;
    }
    if (live1 && (hi64(b) >> 56) == top1) {
      const uint32_t k = atomicAdd(&a.cand_n[r0 + 1], 1u);
      if (k < (uint64_t)a.cap) a.cand[(size_t)(r0 + 1) * a.cap + k] = (uint32_t)i;
    }
  }
}

// a histogram pass over the candidate list of each replica (grid: x over
// list chunks, y over replicas)
__global__ void __launch_bounds__(256) k_init_hist_cand(const InitArgs a) {
  __shared__ uint32_t sh[256];
  const int r = blockIdx.y;
  if (a.pass >= 8 && *a.unresolved == 0) return;  // uniform early exit
  if (a.krem[r] <= 0) return;
  for (int k = threadIdx.x; k < 256; k += blockDim.x) sh[k] = 0;
  __syncthreads();
  const int64_t n = a.cand_n[r];
  const uint64_t pk = a.pre_key[r];
  const uint32_t pi = a.pre_idx[r];
  const int64_t c0 = (int64_t)blockIdx.x * blockDim.x * kSitesPerThread + threadIdx.x;
  for (int s = 0; s < kSitesPerThread; ++s) {
    const int64_t c = c0 + (int64_t)s * blockDim.x;
    if (c >= n) break;
    const uint32_t i = a.cand[(size_t)r * a.cap + c];
    const uint4 b = philox(make_uint4((uint32_t)(r >> 1), kTagInit, i, 0u), a.rk);
    int dg;
    if (digit_of(a, (r & 1) ? hi64(b) : lo64(b), i, pk, pi, dg)) atomicAdd(&sh[dg], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 256; k += blockDim.x) {
    const uint32_t v = sh[k];
    if (v) atomicAdd(&a.hist[(size_t)r * 256 + k], v);
  }
}

// one warp per replica: pick the bucket holding rank krem, fix that digit
__global__ void k_init_select(const InitArgs a, int R) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= R) return;
  if (a.pass >= 8 && *a.unresolved == 0) return;
  const int64_t want = a.krem[r];
  uint32_t* h = a.hist + (size_t)r * 256;
  if (want <= 0) {  // resolved replica: only clear the counters
    for (int k = lane; k < 256; k += 32) h[k] = 0;
    return;
  }
  // lane l owns buckets 8l .. 8l+7
  uint32_t c[8];
  int64_t mine = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j] = h[8 * lane + j];
    mine += c[j];
  }
  int64_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int64_t excl = incl - mine;
  const bool here = (excl < want) && (want <= incl);
  const unsigned who = __ballot_sync(0xffffffffu, here);
  const int src = __ffs(who) - 1;
  if (lane == src) {
    int64_t before = excl;
    int dg = 8 * lane;
    for (int j = 0; j < 8; ++j) {
      if (before + c[j] >= want) {
        dg = 8 * lane + j;
        break;
      }
      before += c[j];
    }
    const int64_t in_bucket = c[dg - 8 * lane];
    const int64_t rank = want - before;  // 1-based rank inside the bucket
    const int p = a.pass;
    if (p < 8) {
      a.pre_key[r] |= (uint64_t)dg << (56 - 8 * p);
      if (p == 7) {
        if (rank == in_bucket) {
          // every key equal to the threshold is taken: no index passes
          a.pre_idx[r] = 0xFFFFFFFFu;
          a.krem[r] = 0;
        } else {
          a.krem[r] = rank;
          atomicOr(a.unresolved, 1);
        }
      } else {
        a.krem[r] = rank;
      }
    } else {
      const int top = a.idx_bits - 8 * (p - 8);
      a.pre_idx[r] |= (uint32_t)dg << (top - 8);
      a.krem[r] = (top - 8 == 0) ? 0 : rank;
    }
  }
  __syncwarp();
  for (int k = lane; k < 256; k += 32) h[k] = 0;
}

__global__ void k_init_rank(int64_t* krem, int R, int64_t K) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) krem[r] = K;
}

// one thread per (site position, word of a plane element): write n, n0, p
template <int V>
__global__ void __launch_bounds__(256) k_init_mark(const InitArgs a, Planes pl) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (e >= a.N * V) return;
  const int64_t i = canon_pos(pl.inv, pl.xs, e / V);  // canonical site held at this position
  const int w = q * V + (int)(e % V);  // word index, replicas 64w .. 64w+63
  uint64_t word = 0;
  for (int j = 0; j < 32; ++j) {
    const int r = 64 * w + 2 * j;
    const uint4 b = philox(make_uint4((uint32_t)(r >> 1), kTagInit, (uint32_t)i, 0u), a.rk);
    const uint64_t k0 = lo64(b), k1 = hi64(b);
    const uint64_t t0 = a.pre_key[r], t1 = a.pre_key[r + 1];
    const uint32_t x0 = a.pre_idx[r], x1 = a.pre_idx[r + 1];
    const bool in0 = (k0 < t0) || (k0 == t0 && (uint32_t)i <= x0);
    const bool in1 = (k1 < t1) || (k1 == t1 && (uint32_t)i <= x1);
    word |= (uint64_t)in0 << (2 * j);
    word |= (uint64_t)in1 << (2 * j + 1);
  }
  const size_t off = (size_t)q * pl.plane_elems() + (size_t)e;
  pl.n[off] = word;
  pl.n0[off] = word;
  pl.p[off] = ~0ull;
}

}  // namespace

cudaError_t launch_init(const Planes& pl, const InitScratch& s, int R, int64_t K,
                        const RoundKeys& rk, cudaStream_t st) {
  const size_t bytes = (size_t)pl.P * pl.plane_elems() * sizeof(uint64_t);
  cudaError_t err;
  if (K <= 0 || K >= pl.N) {
    const int fill = (K <= 0) ? 0x00 : 0xFF;
    if ((err = cudaMemsetAsync(pl.n, fill, bytes, st)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(pl.n0, fill, bytes, st)) != cudaSuccess) return err;
    return cudaMemsetAsync(pl.p, 0xFF, bytes, st);
  }
  InitArgs a;
  a.hist = s.hist;
  a.pre_key = s.pre_key;
  a.pre_idx = s.pre_idx;
  a.krem = s.krem;
  a.unresolved = s.unresolved;
  a.N = pl.N;
  int bits = 1;
  while (bits < 32 && ((int64_t)1 << bits) < pl.N) ++bits;
  a.idx_bits = ((bits + 7) / 8) * 8;
  a.rk = rk;
  // threshold state: rank K, nothing decided
  if ((err = cudaMemsetAsync(s.hist, 0, (size_t)R * 256 * sizeof(uint32_t), st))) return err;
  if ((err = cudaMemsetAsync(s.pre_key, 0, (size_t)R * sizeof(uint64_t), st))) return err;
  if ((err = cudaMemsetAsync(s.pre_idx, 0, (size_t)R * sizeof(uint32_t), st))) return err;
  if ((err = cudaMemsetAsync(s.unresolved, 0, sizeof(int32_t), st))) return err;
  k_init_rank<<<(R + 255) / 256, 256, 0, st>>>(s.krem, R, K);
  if ((err = cudaGetLastError())) return err;

  const int64_t chunk = 256LL * kSitesPerThread;
  dim3 hgrid((unsigned)((pl.N + chunk - 1) / chunk), (unsigned)(R / 2));
  const int passes = 8 + a.idx_bits / 8;
  // candidate lists: about N / 256 entries expected per replica; take them
  // when the room holds N / 128 + 1024 (a list longer than that falls back)
  a.cand_n = nullptr;
  a.cand = nullptr;
  a.cap = 0;
  bool lists = false;
  if (s.cand && pl.N >= 65536) {
    const int64_t room = (int64_t)(s.cand_bytes / sizeof(uint32_t)) - R;
    const int64_t cap = room / R;
    if (cap >= pl.N / 128 + 1024) {
      a.cand_n = s.cand;
      a.cand = s.cand + R;
      a.cap = cap;
      lists = true;
    }
  }
  for (int p = 0; p < passes; ++p) {
    a.pass = p;
    if (lists && p == 1) {
      // collect the candidates of every replica, then check the lists fit
      if ((err = cudaMemsetAsync(a.cand_n, 0, (size_t)R * sizeof(uint32_t), st))) return err;
      k_init_collect<<<hgrid, 256, 0, st>>>(a);
      if ((err = cudaGetLastError())) return err;
      std::vector<uint32_t> counts(R);
      if ((err = cudaMemcpyAsync(counts.data(), a.cand_n, (size_t)R * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, st)))
        return err;
      if ((err = cudaStreamSynchronize(st))) return err;
      int64_t longest = 0;
      for (uint32_t c : counts) longest = std::max<int64_t>(longest, c);
      lists = longest <= a.cap;
    }
    if (lists && p >= 1) {
      const int64_t cchunk = 256LL * kSitesPerThread;
      const unsigned cx = (unsigned)std::max<int64_t>(1, (a.cap + cchunk - 1) / cchunk);
      // the grid covers the capacity; blocks past a replica's count return at once
      k_init_hist_cand<<<dim3(cx, (unsigned)R), 256, 0, st>>>(a);
    } else {
      k_init_hist<<<hgrid, 256, 0, st>>>(a);
    }
    if ((err = cudaGetLastError())) return err;
    k_init_select<<<(R + 7) / 8, 256, 0, st>>>(a, R);
    if ((err = cudaGetLastError())) return err;
  }
  dim3 mgrid((unsigned)((pl.N * pl.V + 255) / 256), (unsigned)pl.P);
  if (pl.V == 4)
    k_init_mark<4><<<mgrid, 256, 0, st>>>(a, pl);
  else if (pl.V == 2)
    k_init_mark<2><<<mgrid, 256, 0, st>>>(a, pl);
  else
    k_init_mark<1><<<mgrid, 256, 0, st>>>(a, pl);
  return cudaGetLastError();
}

}  // namespace ka
