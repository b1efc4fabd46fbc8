// ka_cubic_stream_s5.cu -- instances of the group kernels' general form for the
// sides 92, 96, 100, 104 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<92>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<96>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<100>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<104>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
