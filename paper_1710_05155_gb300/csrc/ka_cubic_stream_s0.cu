// ka_cubic_stream_s0.cu -- instances of the group kernels' general form for the
// sides 4, 8, 12, 16 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<4>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<8>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<12>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<16>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
