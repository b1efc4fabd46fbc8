// ka_four_point.cu -- four-point correlations on cubic lattices.
//
// Section 2.2 defines the space-dependent susceptibility g_4(r, t) from the
// overlaps q_i = n_i(t) n_i(0) of pairs of sites at distance r, and section
// 3.3 computes its numerator Phi(r, t) as popcounts of n_i(t) & n_i(0) &
// n_j(t) & n_j(0) summed over pairs.  Here every ordered pair (i, j) is
// counted once, at the representative of its displacement with every
// component in [-L/2, L/2), in the shell s = |delta|^2:
//   phi[r][s] = sum over pairs in shell s of q_i q_j          (replica r)
//   psi[s]    = sum over pairs in shell s of M_i M_j,  M_i = sum_r q_i^r
// (psi gives the <q_i><q_j> term of g_4).
//
// phi: one launch per shell; a thread takes a few site-words (site i, word
// h of plane q) and all vectors of the shell, and adds q_i & q_{i+delta}
// into bit-sliced counters (all 64 replicas of the word at once); lanes of
// the same word position are summed by warp shuffles, then per block in
// shared memory, then one atomic per (replica, shell).  psi: the per-site
// counts M_i are computed once, then a thread per site sums M_i M_{i+delta}
// over the shell's vectors.
#include <algorithm>
#include <string>
#include <vector>

#include "ka_ctx.cuh"

namespace ka {
namespace {

constexpr int kSlices = 8;            // per-thread counters hold up to 255
constexpr int kWide = kSlices + 5;    // after summing 32 lanes
constexpr int kMaxVectors = 1 << 16;  // displacement vectors per call

struct Vec {
  int16_t dx[4];
};

struct Geometry {
  int d, L;
  int64_t st[4];  // L^k
};

__device__ __forceinline__ void ripple_add(uint64_t (&c)[kSlices], uint64_t x) {
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const uint64_t k = c[s] & x;
    c[s] ^= x;
    x = k;
  }
}

__device__ __forceinline__ void shfl_add(uint64_t (&c)[kWide], int off) {
  uint64_t carry = 0;
#pragma unroll
  for (int s = 0; s < kWide; ++s) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, c[s], off);
    const uint64_t sum = c[s] ^ o ^ carry;
    carry = (c[s] & o) | (carry & (c[s] | o));
    c[s] = sum;
  }
}

// site index of (coordinates of i) + delta, periodic
__device__ __forceinline__ int64_t shifted(const Geometry& g, const int (&x)[4], const Vec& v) {
  int64_t j = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k < g.d) {
      int y = x[k] + v.dx[k];
      y += (y < 0) ? g.L : 0;
      y -= (y >= g.L) ? g.L : 0;
      j += (int64_t)y * g.st[k];
    }
  }
  return j;
}

__device__ __forceinline__ void coords(const Geometry& g, int64_t i, int (&x)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = 0;
    if (k < g.d) {
      x[k] = (int)(i % g.L);
      i /= g.L;
    }
  }
}

// phi of one shell: vectors [v0, v1) of the table, `spt` site-words per
// thread, plane blockIdx.y
template <int V>
__global__ void __launch_bounds__(256) k_phi(Planes pl, Geometry g, const Vec* __restrict__ vec,
                                             int v0, int v1, int spt, int shell, int nshell,
                                             unsigned long long* phi) {
  __shared__ unsigned int acc[64 * V];
  for (int k = threadIdx.x; k < 64 * V; k += blockDim.x) acc[k] = 0;
  __syncthreads();
  const int q = blockIdx.y;
  const size_t E = pl.plane_elems();
  const uint64_t* n = pl.n + (size_t)q * E;
  const uint64_t* n0 = pl.n0 + (size_t)q * E;
  uint64_t c[kSlices];
#pragma unroll
  for (int s = 0; s < kSlices; ++s) c[s] = 0;
  // element e = site * V + h; the stride (blockDim) is a multiple of V, so
  // a thread always sees the same word position h
  const size_t e0 = (size_t)blockIdx.x * blockDim.x * spt + threadIdx.x;
  for (int k = 0; k < spt; ++k) {
    const size_t e = e0 + (size_t)k * blockDim.x;
    if (e >= E) break;
    const int64_t i = canon_site(pl.xs, (int64_t)(e / V));  // the site held at element e
    const int h = (int)(e % V);
    const uint64_t qi = n[e] & n0[e];
    if (qi == 0) continue;
    int x[4];
    coords(g, i, x);
    for (int t = v0; t < v1; ++t) {
      const int64_t j = shifted(g, x, vec[t]);
      const size_t f = (size_t)dev_site(pl.xs, j) * V + h;
      ripple_add(c, qi & n[f] & n0[f]);
    }
  }
  const int lane = threadIdx.x & 31;
  uint64_t w[kWide];
#pragma unroll
  for (int s = 0; s < kWide; ++s) w[s] = (s < kSlices) ? c[s] : 0;
#pragma unroll
  for (int off = 16; off >= V; off >>= 1) shfl_add(w, off);
  // lanes 0 .. V-1 hold the warp totals of word positions 0 .. V-1; every
  // lane extracts replicas (bits) lane and lane + 32 of each
#pragma unroll
  for (int hh = 0; hh < V; ++hh) {
    unsigned int lo = 0, hi = 0;
#pragma unroll
    for (int s = 0; s < kWide; ++s) {
      const uint64_t t = __shfl_sync(0xffffffffu, w[s], hh);
      lo |= (unsigned int)((t >> lane) & 1u) << s;
      hi |= (unsigned int)((t >> (lane + 32)) & 1u) << s;
    }
    if (lo) atomicAdd(&acc[hh * 64 + lane], lo);
    if (hi) atomicAdd(&acc[hh * 64 + lane + 32], hi);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 64 * V; k += blockDim.x) {
    const unsigned int v = acc[k];
    if (v) {
      const int r = (q * V + k / 64) * 64 + (k % 64);
      atomicAdd(&phi[(size_t)r * nshell + shell], (unsigned long long)v);
    }
  }
}

// M_i = number of replicas with q_i = 1
template <int V>
__global__ void k_site_counts(Planes pl, uint32_t* M) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pl.N) return;
  const size_t E = pl.plane_elems();
  uint32_t m = 0;
  for (int q = 0; q < pl.P; ++q)
#pragma unroll
    for (int h = 0; h < V; ++h) {
      const size_t e = (size_t)q * E + (size_t)dev_site(pl.xs, i) * V + h;
      m += (uint32_t)__popcll(pl.n[e] & pl.n0[e]);
    }
  M[i] = m;
}

// psi of one shell: a thread per site, all vectors of the shell
__global__ void __launch_bounds__(256) k_psi(Geometry g, int64_t N, const uint32_t* __restrict__ M,
                                             const Vec* __restrict__ vec, int v0, int v1,
                                             unsigned long long* psi_s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long acc = 0;
  if (i < N && M[i] != 0) {
    int x[4];
    coords(g, i, x);
    unsigned long long sum = 0;
    for (int t = v0; t < v1; ++t) sum += M[shifted(g, x, vec[t])];
    acc = sum * M[i];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ unsigned long long part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    if (s) atomicAdd(psi_s, s);
  }
}

}  // namespace
}  // namespace ka

namespace {

struct Scope {
  int prev = -1;
  explicit Scope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
      cudaSetDevice(dev);
    else
      prev = -1;
  }
  ~Scope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

ka_status four_point_fail(ka_ctx* c, ka_status st, const std::string& msg) {
  c->err = msg;
  return st;
}

}  // namespace

extern "C" ka_status ka_four_point(ka_ctx* c, int32_t smax, int64_t* phi, int64_t* psi) {
  ka::NvtxRange nvtx_range("ka_four_point");
  using namespace ka;
  if (!c) return KA_EINVAL;
  if (!phi || smax < 0) return four_point_fail(c, KA_EINVAL, "phi must be non-NULL, smax >= 0");
  if (c->topo != KA_CUBIC)
    return four_point_fail(c, KA_EINVAL, "four-point correlations need a cubic lattice");
  if (!c->initialized) return four_point_fail(c, KA_ESTATE, "four-point before init or set_state");
  const int d = c->d, L = c->L, half = L / 2;
  if ((int64_t)smax > (int64_t)d * half * half)
    return four_point_fail(c, KA_EINVAL, "smax above d (L/2)^2, the largest shell");
  // representative displacement vectors (components in [-L/2, L/2)) by shell
  int rad = 0;
  while ((int64_t)(rad + 1) * (rad + 1) <= smax) ++rad;
  const int lo = -std::min(rad, half), hi = std::min(rad, half - 1);
  const int S = smax + 1;
  std::vector<std::vector<Vec>> shell(S);
  int64_t nvec = 0;
  int x[4] = {lo, lo, lo, lo};
  for (int k = d; k < 4; ++k) x[k] = 0;
  for (;;) {
    int64_t s2 = 0;
    for (int k = 0; k < d; ++k) s2 += (int64_t)x[k] * x[k];
    if (s2 <= smax) {
      Vec v{};
      for (int k = 0; k < 4; ++k) v.dx[k] = (int16_t)x[k];
      shell[s2].push_back(v);
      if (++nvec > kMaxVectors)
        return four_point_fail(c, KA_EINVAL, "more than 65536 displacement vectors: lower smax");
    }
    int k = 0;
    while (k < d && x[k] == hi) x[k++] = lo;
    if (k == d) break;
    ++x[k];
  }
  std::vector<Vec> table;
  std::vector<int> off(S + 1, 0);
  for (int s2 = 0; s2 < S; ++s2) {
    off[s2] = (int)table.size();
    table.insert(table.end(), shell[s2].begin(), shell[s2].end());
  }
  off[S] = (int)table.size();

  Scope scope(c->device);
  const cudaStream_t st = c->stream;
  const int R = c->R;
  const size_t phi_bytes = (size_t)R * S * sizeof(unsigned long long);
  const size_t psi_bytes = (size_t)S * sizeof(unsigned long long);
  const size_t m_bytes = psi ? (size_t)c->N * sizeof(uint32_t) : 0;
  const size_t v_bytes = std::max<size_t>(table.size(), 1) * sizeof(Vec);
  const size_t a = 256;
  auto up = [&](size_t b) { return (b + a - 1) / a * a; };
  const size_t total = up(phi_bytes) + up(psi_bytes) + up(m_bytes) + up(v_bytes);
  char* mem = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&mem, total, st);
  if (e) return four_point_fail(c, KA_ENOMEM, std::string("scratch: ") + cudaGetErrorString(e));
  unsigned long long* phi_dev = (unsigned long long*)mem;
  unsigned long long* psi_dev = (unsigned long long*)(mem + up(phi_bytes));
  uint32_t* M = (uint32_t*)(mem + up(phi_bytes) + up(psi_bytes));
  Vec* vec = (Vec*)(mem + up(phi_bytes) + up(psi_bytes) + up(m_bytes));
  e = cudaMemsetAsync(mem, 0, up(phi_bytes) + up(psi_bytes), st);
  if (!e && !table.empty())
    e = cudaMemcpyAsync(vec, table.data(), table.size() * sizeof(Vec), cudaMemcpyHostToDevice, st);
  Geometry g{};
  g.d = d;
  g.L = L;
  g.st[0] = 1;
  for (int k = 1; k < 4; ++k) g.st[k] = g.st[k - 1] * L;
  const Planes& pl = c->pl;
  const size_t E = pl.plane_elems();
  if (!e && psi) {
    const unsigned blocks = (unsigned)((c->N + 255) / 256);
    if (pl.V == 4)
      k_site_counts<4><<<blocks, 256, 0, st>>>(pl, M);
    else if (pl.V == 2)
      k_site_counts<2><<<blocks, 256, 0, st>>>(pl, M);
    else
      k_site_counts<1><<<blocks, 256, 0, st>>>(pl, M);
    e = cudaGetLastError();
  }
  for (int s2 = 0; s2 < S && !e; ++s2) {
    // chunks of at most 255 vectors keep every per-thread counter below 256
    for (int v0 = off[s2]; v0 < off[s2 + 1] && !e; v0 += 255) {
      const int v1 = std::min(v0 + 255, off[s2 + 1]);
      const int spt = std::max(1, std::min(32, 255 / (v1 - v0)));
      const dim3 grid((unsigned)((E + (size_t)256 * spt - 1) / ((size_t)256 * spt)), (unsigned)pl.P);
      if (pl.V == 4)
        k_phi<4><<<grid, 256, 0, st>>>(pl, g, vec, v0, v1, spt, s2, S, phi_dev);
      else if (pl.V == 2)
        k_phi<2><<<grid, 256, 0, st>>>(pl, g, vec, v0, v1, spt, s2, S, phi_dev);
      else
        k_phi<1><<<grid, 256, 0, st>>>(pl, g, vec, v0, v1, spt, s2, S, phi_dev);
      e = cudaGetLastError();
      if (!e && psi) {
        k_psi<<<(unsigned)((c->N + 255) / 256), 256, 0, st>>>(g, c->N, M, vec, v0, v1,
                                                              psi_dev + s2);
        e = cudaGetLastError();
      }
    }
  }
  if (!e) e = cudaMemcpyAsync(phi, phi_dev, phi_bytes, cudaMemcpyDeviceToHost, st);
  if (!e && psi) e = cudaMemcpyAsync(psi, psi_dev, psi_bytes, cudaMemcpyDeviceToHost, st);
  const cudaError_t ef = cudaFreeAsync(mem, st);
  if (!e) e = ef;
  const cudaError_t es = cudaStreamSynchronize(st);
  if (!e) e = es;
  if (e) return four_point_fail(c, KA_ECUDA, std::string("four-point: ") + cudaGetErrorString(e));
  return KA_OK;
}
