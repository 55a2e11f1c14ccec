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
  int depth;        // time steps of this pass (<= the instantiated depth K)
  int variant;      // 0: register prefetch, 1: TMA bulk-copy ring
  int stages;       // variant 1: ring slots per warp (power of two, 2..16)
  int wait_limit;   // variant 1: mbarrier polls before a wait gives up
  int inject_on;    // variant 1, tests only: 1 = the copies of row inject_row never complete
  int inject_row;
  // Depth 4, FP32, variant 1 only: also store level t (1..depth-1) of the
  // pass to levels[t - 1] (each an nx*ny field), so one pass yields depth
  // consecutive states.
  int store_levels = 0;
  float* levels[7] = {};
};

// Number of output columns per warp strip for temporal depth k (128 columns
// per warp minus a halo of k rounded up to a multiple of 4 on each side).
inline int strip_out_width(int k) { return 128 - 2 * ((k + 3) & ~3); }

// Variant 1 ring geometry: cells per slot row and the column alignment
// (in cells) that keeps every bulk copy on 16-byte boundaries.
inline int bulk_slot_cells(bool bf16) { return bf16 ? 136 : 128; }
inline int bulk_align_cells(bool bf16) { return bf16 ? 8 : 4; }
inline size_t bulk_smem_bytes(bool bf16, int warps, int stages) {
  const size_t slot = (size_t)bulk_slot_cells(bf16) * (bf16 ? 4 + 2 + 2 : 4 + 4 + 4);
  return (size_t)warps * stages * (slot + sizeof(uint64_t));
}

// Dynamic shared memory of one CTA of the stream kernels: per warp a ring of
// (k + 2) & ~1 rows (k + 1 rounded up to even) of per-row face terms
// (3 x 32 float4), plus the variant-1 row ring.
inline size_t stream_smem_bytes(bool bf16, int k, int warps, int variant, int stages) {
  return (size_t)warps * ((k + 2) & ~1) * 3 * 32 * 16 +
         (variant == 1 ? bulk_smem_bytes(bf16, warps, stages) : 0);
}

// One pass of instantiated depth k (1..8) over the whole grid.
cudaError_t launch_stream_f32(const StreamPass& p, int k, cudaStream_t s);
cudaError_t launch_stream_bf16k(const StreamPass& p, int k, cudaStream_t s);
cudaError_t launch_stream_bf16k_block(const StreamPass& p, int k, cudaStream_t s);
// Read and clear the device status word of the f32 / bf16 / bf16-block stream kernels.
cudaError_t read_stream_status_f32(int* out);
cudaError_t read_stream_status_bf16k(int* out);
cudaError_t read_stream_status_bf16k_block(int* out);

// Read and clear the first out-of-range source line recorded by each
// translation unit's kernels (bounds-checked build; 0 otherwise).
cudaError_t read_bounds_stream_f32(int* out);
cudaError_t read_bounds_stream_bf16k(int* out);
cudaError_t read_bounds_stream_bf16k_block(int* out);
cudaError_t read_bounds_batch(int* out);
cudaError_t read_bounds_adjoint(int* out);
cudaError_t read_bounds_vol(int* out);
cudaError_t read_bounds_tile(int* out);
cudaError_t read_bounds_sum(int* out);

// The shared-memory temporal-blocked tiled kernel (k_tile.cu): d steps per
// launch, bx x by threads, four (bx + 2d) x (by + 2d) float tiles.
size_t tile_blocked_smem_bytes(int bx, int by, int d);
cudaError_t launch_tile_blocked_f32(const float* u_in, float* u_out, const float* kappa, const float* src,
                                    int nx, int ny, float dt, int bc, int d, dim3 grid, dim3 block,
                                    cudaStream_t s);

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

#include "../../include/cpb.h"
namespace cpb {
// Batched persistent launch (k_batch.cu).
// Largest CTA of the batched kernel at temporal depth `depth` (4 or 8; 0 for
// any other depth).
int batch_threads_max(int depth);
cudaError_t batch_blocks_per_sm(int depth, int threads, int* out);
// Bounded-wait limit of the TMA row ring and the test-only missing-bytes
// injection (see StreamPass), passed to the batched kernel by value.
struct BatchDebug {
  int wait_limit;
  int inject_on;
  int inject_row;
};
// Multi-warp teams for the small-grid queue: team_warps <= 1 (one warp per
// grid) or a divisor of the CTA's warps with at most 15 teams per CTA.
bool batch_team_ok(int threads, int team_warps);
cudaError_t launch_batch(int depth, const cpb_grid_desc* descs, const int* order, int ngrids, int n_large, int bc,
                         int grain, int blocks, int threads, int team_warps, const BatchDebug& dbg, int* work,
                         cudaStream_t s);
}  // namespace cpb

namespace cpb {
// One adjoint step (k_adjoint.cu): lam_out = lam + dt D lam; gk += face terms.
cudaError_t launch_adjoint_step(const float* lam, float* lam_out, const float* u, const float* k,
                                float* gk, int nx, int ny, float dt, int bc, cudaStream_t s);
// `depth` adjoint steps in one pass (k_adjoint.cu), lam = lambda_m ->
// lam_out = lambda_{m-depth}; u[t - 1] = u_{m-t}.  nx % 4 == 0, 16-byte
// aligned fields, depth 1..4; the same bits as `depth` one-step launches.
cudaError_t launch_adjoint_pass(const float* lam, float* lam_out, const float* const* u, int depth, const float* k,
                                float* gk, int nx, int ny, float dt, int bc, int chunk_rows, cudaStream_t s);
}  // namespace cpb

namespace cpb {
// 3-D 7-point z-marching kernel (k_vol.cu): one launch per step, block
// (32, by), grid (ceil(nx / 128), ceil(ny / by), z-chunks).
size_t vol_smem_bytes(int by);
cudaError_t launch_vol_f32(const float* u_in, float* u_out, const float* kappa, const float* src, int nx,
                           int ny, int nz, float dt, int bc, int vec, dim3 grid, int by, cudaStream_t s);
}  // namespace cpb

namespace cpb {
// Heat sum with partials in a file-scope device array (k_sum.cu).
long long heat_sum_noalloc_max_cells();
cudaError_t launch_heat_sum_noalloc(const void* u, long long n, int dtype, double* d_out,
                                    cudaStream_t s);
}  // namespace cpb
