// FP32-storage instantiations of the streaming temporal-blocked kernel.
#include "k_stream.cuh"

namespace cpb {
cudaError_t launch_stream_f32(const StreamPass& p, int k, cudaStream_t s) {
  return launch_stream_any<false>(p, k, s);
}
}  // namespace cpb
