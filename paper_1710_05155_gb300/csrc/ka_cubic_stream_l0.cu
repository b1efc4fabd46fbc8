// ka_cubic_stream_l0.cu -- instances of the group kernels that read the side L
// from their arguments (every side but 32, 64 and 128; one translation unit
// per instance set, so that they compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<0>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
