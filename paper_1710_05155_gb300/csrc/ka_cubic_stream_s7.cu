// ka_cubic_stream_s7.cu -- instances of the group kernels' general form for the
// sides 124 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<124>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
