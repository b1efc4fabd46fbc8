// ka_cubic_stream_s3.cu -- instances of the group kernels' general form for the
// sides 56, 60, 68, 72 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<56>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<60>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<68>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<72>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
