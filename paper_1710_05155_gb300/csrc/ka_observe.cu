// ka_observe.cu -- per-replica observables by vertical popcounts.
//
// Section 3.3 computes overlaps as bitwise ANDs of multispin words and
// counts their ones.  Here the counts are needed per replica, i.e. per bit
// position, summed over sites: for every replica r
//   particles   = sum_i n_i
//   overlap     = sum_i n_i & n0_i        (the q_i(t) = n_i(t) n_i(0) of section 2.2)
//   persist_occ = sum_i n0_i & p_i
//   persist_all = sum_i p_i
//
// Each thread adds up to 63 words into bit-sliced counters (6 slices: one
// uint64 per binary digit, so all 64 replicas count in parallel with a
// ripple adder); the words per thread are chosen so that the grid fills the
// device, four independent loads in flight per thread.  Lanes holding the same word position are then summed in
// bit-sliced form through warp shuffles, the warp total is turned into one
// integer per replica, and blocks accumulate in shared memory before one
// 64-bit atomic per counter goes to global memory.
#include <mutex>
#include "ka_internal.cuh"

namespace ka {
namespace {

constexpr int kSlices = 6;        // per-thread counters hold up to 63
constexpr int kPerThread = 63;    // most words per thread
constexpr int kWide = kSlices + 5;  // after summing 32 lanes

__device__ __forceinline__ void ripple_add(uint64_t (&c)[kSlices], uint64_t x) {
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    const uint64_t k = c[s] & x;
    c[s] ^= x;
    x = k;
  }
}

// add the counter of lane (lane ^ off) into this lane's, bit-sliced
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

template <int V>
__global__ void __launch_bounds__(256, 2) k_observe(Planes pl, unsigned long long* counts,
                                                 int per_thread) {
  __shared__ unsigned int acc[4][64 * V];
  const int q = blockIdx.y;
  for (int k = threadIdx.x; k < 4 * 64 * V; k += blockDim.x) (&acc[0][0])[k] = 0;
  __syncthreads();

  const size_t E = pl.plane_elems();
  const size_t base = (size_t)q * E;
  // element e of the plane holds word h = e % V of site e / V; blockDim and
  // the stride are even, so a thread always sees the same h
  const size_t e0 = (size_t)blockIdx.x * blockDim.x * per_thread + threadIdx.x;
  uint64_t c[4][kSlices];
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int s = 0; s < kSlices; ++s) c[o][s] = 0;
  for (int k = 0; k < per_thread; k += 4) {
    uint64_t n[4], n0[4], p[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t e = e0 + (size_t)(k + u) * blockDim.x;
      const bool in = (k + u < per_thread) && e < E;
      n[u] = in ? pl.n[base + e] : 0ull;
      n0[u] = in ? pl.n0[base + e] : 0ull;
      p[u] = in ? pl.p[base + e] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      ripple_add(c[0], n[u]);
      ripple_add(c[1], n[u] & n0[u]);
      ripple_add(c[2], n0[u] & p[u]);
      ripple_add(c[3], p[u]);
    }
  }

  const int lane = threadIdx.x & 31;
  const int h = lane % V;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    uint64_t w[kWide];
#pragma unroll
    for (int s = 0; s < kWide; ++s) w[s] = (s < kSlices) ? c[o][s] : 0;
    // sum lanes with the same word position (stride V)
#pragma unroll
    for (int off = 16; off >= V; off >>= 1) shfl_add(w, off);
    // lanes 0 .. V-1 hold the totals of word positions 0 .. V-1; every lane
    // extracts replicas (bit positions) lane and lane + 32 of each
#pragma unroll
    for (int hh = 0; hh < V; ++hh) {
      unsigned int lo = 0, hi = 0;
#pragma unroll
      for (int s = 0; s < kWide; ++s) {
        const uint64_t t = __shfl_sync(0xffffffffu, w[s], hh);
        lo |= (unsigned int)((t >> lane) & 1u) << s;
        hi |= (unsigned int)((t >> (lane + 32)) & 1u) << s;
      }
      if (lo) atomicAdd(&acc[o][hh * 64 + lane], lo);
      if (hi) atomicAdd(&acc[o][hh * 64 + lane + 32], hi);
    }
  }
  (void)h;
  __syncthreads();
  for (int k = threadIdx.x; k < 4 * 64 * V; k += blockDim.x) {
    const int o = k / (64 * V), rb = k % (64 * V);  // rb = h * 64 + bit
    const unsigned int v = acc[o][rb];
    if (v) {
      const int r = (q * V + rb / 64) * 64 + (rb % 64);
      atomicAdd(&counts[(size_t)r * 4 + o], (unsigned long long)v);
    }
  }
}

}  // namespace

cudaError_t launch_observe(const Planes& pl, int R, unsigned long long* counts_dev,
                           cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(counts_dev, 0, (size_t)R * 4 * sizeof(unsigned long long), st);
  if (err != cudaSuccess) return err;
  // words per thread: enough blocks for four per SM, at most kPerThread
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t E = pl.plane_elems();
  const size_t want = (size_t)256 * 4 * (size_t)(sms > 0 ? sms : 148);
  int per_thread = (int)((E + want - 1) / want);
  per_thread = per_thread < 4 ? 4 : (per_thread > kPerThread ? kPerThread : per_thread);
  const size_t per_block = (size_t)256 * per_thread;
  dim3 grid((unsigned)((E + per_block - 1) / per_block), (unsigned)pl.P);
  if (pl.V == 4)
    k_observe<4><<<grid, 256, 0, st>>>(pl, counts_dev, per_thread);
  else if (pl.V == 2)
    k_observe<2><<<grid, 256, 0, st>>>(pl, counts_dev, per_thread);
  else
    k_observe<1><<<grid, 256, 0, st>>>(pl, counts_dev, per_thread);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant (ka_observe_static): the per-replica accumulators
// live in a file-scope device array instead of memory the caller or the
// library allocates.  Every GPU that loads the library holds this array
// until the process exits.
// ---------------------------------------------------------------------------

constexpr int kStaticMaxReplicas = 4096;  // 4096 x 4 x 8 bytes = 128 KiB per device
static __device__ __align__(256) unsigned long long g_static_counts[kStaticMaxReplicas * 4];

namespace {
constexpr int kMaxDevices = 64;

// The array's device address on one device, looked up once: std::call_once
// orders the lookup before every use from any host thread.
struct StaticSlot {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned long long* ptr = nullptr;
};
StaticSlot g_static_slot[kMaxDevices];
}  // namespace

// Device address of the array on the current device.  In host code the
// symbol itself is only a host-side stand-in, so its address is looked up
// (with that device current) by the first call on each device and cached;
// a failed lookup is returned to every later call on that device.
cudaError_t static_counts_ptr(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  StaticSlot& s = g_static_slot[dev];
  std::call_once(s.once, [&s] {
    void* ptr = nullptr;
    s.err = cudaGetSymbolAddress(&ptr, g_static_counts);
    s.ptr = (unsigned long long*)ptr;
  });
  if (s.err != cudaSuccess) return s.err;
  *out = s.ptr;
  return cudaSuccess;
}

}  // namespace ka

extern "C" ka_status ka_observe_static(const uint64_t* n, const uint64_t* n0, const uint64_t* p,
                                       int64_t N, int32_t replicas, int64_t* counts,
                                       void* stream) {
  if (!n || !n0 || !p || !counts || N < 1 || replicas <= 0 || replicas % 64 ||
      replicas > ka::kStaticMaxReplicas)
    return KA_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (st) {
    // the array whose address is used is the current device's: the stream
    // must belong to that device
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess)
      return KA_ECUDA;
    if (sdev != cur) return KA_EINVAL;
  }
  unsigned long long* scratch = nullptr;
  cudaError_t e = ka::static_counts_ptr(&scratch);
  if (e != cudaSuccess) return KA_ECUDA;
  // the canonical layout [R/64][N] is the device layout with one word per plane
  ka::Planes pl{};
  pl.n = const_cast<uint64_t*>(n);
  pl.n0 = const_cast<uint64_t*>(n0);
  pl.p = const_cast<uint64_t*>(p);
  pl.N = N;
  pl.W = replicas / 64;
  pl.V = 1;
  pl.P = pl.W;
  e = ka::launch_observe(pl, replicas, scratch, st);  // clears the scratch, then accumulates
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(counts, scratch, (size_t)replicas * 4 * sizeof(int64_t),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? KA_OK : KA_ECUDA;
}
