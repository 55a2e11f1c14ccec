// Host-side launchers shared between the translation units of libcpb.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace cpb {

// Parameters of one pass of the streaming temporal-blocked kernel.
struct StreamPass {
  const void* u_in;
  void* u_out;
  const void* kappa;
  const void* src;
  int nx, ny;
  float dt, hdt;
  int bc;
  int vec;          // 1: 128-bit access path (nx % 4 == 0, aligned pointers)
  int chunk_rows;   // output rows per warp item
  int warps_per_block;
};

// Number of output columns per warp strip for temporal depth k (128 columns
// per warp minus a halo of k rounded up to a multiple of 4 on each side).
inline int strip_out_width(int k) { return 128 - 2 * ((k + 3) & ~3); }

// One pass of depth k (1..8) over the whole grid.  Returns the launch error.
cudaError_t launch_stream_f32(const StreamPass& p, int k, cudaStream_t s);
cudaError_t launch_stream_bf16k(const StreamPass& p, int k, cudaStream_t s);

// The tiled one-step kernel (bx x by threads, one cell each).
cudaError_t launch_tile_f32(const float* u_in, float* u_out, const float* kappa, const float* src,
                            int nx, int ny, float dt, int bc, dim3 grid, dim3 block, size_t shm,
                            cudaStream_t s);

// FP64 heat sum: partial pass + final pass.
int heat_sum_blocks(long long n);
cudaError_t launch_heat_sum(const void* u, long long n, int dtype, double* d_out, double* partials,
                            int nblocks, cudaStream_t s);

cudaError_t launch_bf16_round(const float* x, uint16_t* out, long long n, cudaStream_t s);
cudaError_t launch_bf16k_pack(const float* u, uint32_t* st, long long n, cudaStream_t s);
cudaError_t launch_bf16k_unpack(const uint32_t* st, float* u, long long n, cudaStream_t s);

}  // namespace cpb
