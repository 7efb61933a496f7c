// Streaming contraction kernels, FP32 instantiations (see stream_impl.cuh and
// reduce_impl.cuh).
#define TN_STREAM_HOST_DEFS
#include "stream_impl.cuh"
#include "reduce_impl.cuh"

namespace tn {
template void launch_absorb<float>(const ADesc &, int, cudaStream_t);
template void launch_reduce<float>(const RDesc &, void *, cudaStream_t);
}  // namespace tn
