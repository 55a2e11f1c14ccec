// BF16-Kahan-storage instantiations of the streaming temporal-blocked kernels
// that round into storage only the rows a pass stores (CPB_BF16_KAHAN_BLOCK).
#include "k_stream.cuh"

namespace cpb {
cudaError_t launch_stream_bf16k_block(const StreamPass& p, int k, cudaStream_t s) {
  return launch_stream_any<true, false>(p, k, s);
}
cudaError_t read_stream_status_bf16k_block(int* out) { return read_stream_status(out); }
cudaError_t read_bounds_stream_bf16k_block(int* out) { return read_bounds_word(out); }
}  // namespace cpb
