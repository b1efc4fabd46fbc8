// ka_layout.cu -- conversion between the canonical state layout of the ABI
// ([W][N] uint64, word-plane major) and the device layout ([P][N][V]).
// Only needed when V = 2; with V = 1 both layouts coincide.
#include "ka_internal.cuh"

namespace ka {
namespace {

// canonical -> device: dst[q][i][h] = src[2q + h][i]
__global__ void k_to_device(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                            int64_t N, int P) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over P * N sites
  if (e >= (int64_t)P * N) return;
  const int64_t q = e / N, i = e - q * N;
  const ulonglong2 v = make_ulonglong2(src[(2 * q) * N + i], src[(2 * q + 1) * N + i]);
  reinterpret_cast<ulonglong2*>(dst)[q * N + i] = v;
}

// device -> canonical
__global__ void k_to_canonical(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                               int64_t N, int P) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)P * N) return;
  const int64_t q = e / N, i = e - q * N;
  const ulonglong2 v = reinterpret_cast<const ulonglong2*>(src)[q * N + i];
  dst[(2 * q) * N + i] = v.x;
  dst[(2 * q + 1) * N + i] = v.y;
}

}  // namespace

cudaError_t launch_to_device(const uint64_t* canonical, uint64_t* device_layout, int64_t N, int P,
                             cudaStream_t st) {
  const int64_t n = (int64_t)P * N;
  k_to_device<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(canonical, device_layout, N, P);
  return cudaGetLastError();
}

cudaError_t launch_to_canonical(const uint64_t* device_layout, uint64_t* canonical, int64_t N,
                                int P, cudaStream_t st) {
  const int64_t n = (int64_t)P * N;
  k_to_canonical<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(device_layout, canonical, N, P);
  return cudaGetLastError();
}

}  // namespace ka
