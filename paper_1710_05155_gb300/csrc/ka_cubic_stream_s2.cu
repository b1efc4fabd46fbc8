// ka_cubic_stream_s2.cu -- instances of the group kernels' general form for the
// sides 40, 44, 48, 52 (a few sides per translation unit, so that the
// instances compile in parallel).
#define KA_STREAM_INSTANCES
#include "ka_cubic_stream.cuh"

namespace ka {
namespace stream {
template cudaError_t launch_l<40>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<44>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<48>(const Args&, int, cudaStream_t);
template cudaError_t launch_l<52>(const Args&, int, cudaStream_t);
}  // namespace stream
}  // namespace ka
