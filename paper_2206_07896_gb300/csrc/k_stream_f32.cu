// FP32-storage instantiations of the streaming temporal-blocked kernels.
#include "k_stream.cuh"

namespace cpb {
cudaError_t launch_stream_f32(const StreamPass& p, int k, cudaStream_t s) {
  return launch_stream_any<false>(p, k, s);
}
cudaError_t read_stream_status_f32(int* out) { return read_stream_status(out); }
cudaError_t read_bounds_stream_f32(int* out) { return read_bounds_word(out); }
}  // namespace cpb
