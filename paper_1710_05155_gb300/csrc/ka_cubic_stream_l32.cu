// ka_cubic_stream_l32.cu -- instances of the streaming group kernel for L = 32
// (one translation unit per side, so that they compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<32>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
