// ka_cubic_stream_s1.cu -- instances of the group kernels' general form for the
// sides 20, 24, 28, 36 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<20>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<24>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<28>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<36>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
