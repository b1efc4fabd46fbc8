// ka_cubic_stream_s6.cu -- instances of the group kernels' general form for the
// sides 108, 112, 116, 120 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<108>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<112>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<116>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<120>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
