// ka_cubic_d3.cu -- the single-instance cubic kernels of dimension 3.
#define KA_CUBIC_INSTANCES
#include "ka_cubic_kernel.cuh"

namespace ka {
namespace cubic {
template cudaError_t launch_d<3, false>(int, bool, const GroupArgs&, const BatchArgs&, int,
                                          unsigned, size_t, cudaStream_t);
}  // namespace cubic
}  // namespace ka
