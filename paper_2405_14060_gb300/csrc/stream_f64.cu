// Streaming contraction kernels, FP64 instantiations (see stream_impl.cuh and
// reduce_impl.cuh).
#include "stream_impl.cuh"
#include "reduce_impl.cuh"

namespace tn {
template void launch_absorb<double>(const ADesc &, int, cudaStream_t);
template void launch_reduce<double>(const RDesc &, void *, cudaStream_t);
}  // namespace tn
