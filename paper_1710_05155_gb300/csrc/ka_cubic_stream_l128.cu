// ka_cubic_stream_l128.cu -- instances of the streaming group kernel for L = 128
// (one translation unit per side, so that they compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<128>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
