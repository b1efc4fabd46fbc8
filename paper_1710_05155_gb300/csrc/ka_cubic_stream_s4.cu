// ka_cubic_stream_s4.cu -- instances of the group kernels' general form for the
// sides 76, 80, 84, 88 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<76>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<80>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<84>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<88>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
