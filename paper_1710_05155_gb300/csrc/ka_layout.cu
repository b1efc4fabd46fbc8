// ka_layout.cu -- conversion between the canonical state layout of the ABI
// ([W][N] uint64, word-plane major) and the device layout ([P][N][V], word w
// of site i in plane w / V at element dev_site(xs, i) * V + w % V, or, for
// graphs, at the breadth-first position of i: inv gives the canonical site of
// every position).  With V = 1, xs = 0 and no inv both layouts coincide.
#include "ka_internal.cuh"

namespace ka {
namespace {

// canonical -> device, one thread per (plane, site position, word)
__global__ void k_to_device(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                            int64_t N, int P, int V, int xs, const int32_t* __restrict__ inv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // device element
  if (e >= (int64_t)P * N * V) return;
  const int64_t q = e / (N * V), r = e - q * N * V;
  const int64_t pos = r / V, h = r - pos * V;
  dst[e] = src[(q * V + h) * N + canon_pos(inv, xs, pos)];
}

// device -> canonical
__global__ void k_to_canonical(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                               int64_t N, int P, int V, int xs, const int32_t* __restrict__ inv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)P * N * V) return;
  const int64_t q = e / (N * V), r = e - q * N * V;
  const int64_t pos = r / V, h = r - pos * V;
  dst[(q * V + h) * N + canon_pos(inv, xs, pos)] = src[e];
}

}  // namespace

cudaError_t launch_to_device(const uint64_t* canonical, uint64_t* device_layout, int64_t N, int P,
                             int V, int xs, const int32_t* inv, cudaStream_t st) {
  const int64_t n = (int64_t)P * N * V;
  k_to_device<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(canonical, device_layout, N, P, V, xs,
                                                           inv);
  return cudaGetLastError();
}

cudaError_t launch_to_canonical(const uint64_t* device_layout, uint64_t* canonical, int64_t N,
                                int P, int V, int xs, const int32_t* inv, cudaStream_t st) {
  const int64_t n = (int64_t)P * N * V;
  k_to_canonical<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(device_layout, canonical, N, P, V,
                                                               xs, inv);
  return cudaGetLastError();
}

}  // namespace ka
