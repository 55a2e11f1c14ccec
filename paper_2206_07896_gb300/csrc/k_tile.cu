// The tiled one-step stencil kernel: one thread per cell, a (bx+2) x (by+2)
// shared tile of u and of kappa with a one-cell halo, one __syncthreads.
//
// This is the kernel class the paper translates for CPUs (Sec. III-B): its
// two barrier-free regions -- stage the tile, then update from the tile --
// are what the CPU executor turns into two thread loops ("loop fission").
// Launch geometry is the caller's (<<<grid, block, shm>>>), one launch per step.
#include "common.cuh"
#include "internal.h"

namespace cpb {
namespace {

// Stage the value seen at grid position (gi, gj) into tile slot `slot`:
// inside the grid the cell itself; outside, the boundary rule (Dirichlet:
// u = 0 and kappa of the nearest in-grid cell, which is the kappa of the cell
// across the face; periodic: wrap).
__device__ __forceinline__ void stage(const float* __restrict__ u, const float* __restrict__ k,
                                      int nx, int ny, int bc, int gi, int gj, float* su, float* sk,
                                      int slot) {
  if (bc == BC_PERIODIC) {
    size_t g = (size_t)wrap_index(gj, ny) * nx + wrap_index(gi, nx);
    su[slot] = u[g];
    sk[slot] = k[g];
  } else {
    bool inside = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    su[slot] = inside ? u[(size_t)gj * nx + gi] : 0.0f;
    sk[slot] = k[(size_t)clamp_index(gj, ny) * nx + clamp_index(gi, nx)];
  }
}

__global__ void tile_step_f32(const float* __restrict__ u, float* __restrict__ uo,
                              const float* __restrict__ k, const float* __restrict__ s, int nx,
                              int ny, float dt, float hdt, int bc) {
  extern __shared__ float tile[];
  const int BX = blockDim.x, BY = blockDim.y, TW = BX + 2;
  float* su = tile;
  float* sk = tile + TW * (BY + 2);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gi = blockIdx.x * BX + tx, gj = blockIdx.y * BY + ty;

  // Region 0: stage own cell, edge threads stage the halo in their direction.
  stage(u, k, nx, ny, bc, gi, gj, su, sk, (ty + 1) * TW + (tx + 1));
  if (tx == 0) stage(u, k, nx, ny, bc, gi - 1, gj, su, sk, (ty + 1) * TW);
  if (tx == BX - 1) stage(u, k, nx, ny, bc, gi + 1, gj, su, sk, (ty + 1) * TW + BX + 1);
  if (ty == 0) stage(u, k, nx, ny, bc, gi, gj - 1, su, sk, tx + 1);
  if (ty == BY - 1) stage(u, k, nx, ny, bc, gi, gj + 1, su, sk, (BY + 1) * TW + tx + 1);
  __syncthreads();
  // Region 1: update in-grid cells from the tile.
  if (gi < nx && gj < ny) {
    const int c = (ty + 1) * TW + (tx + 1);
    const size_t g = (size_t)gj * nx + gi;
    const float kc = sk[c];
    uo[g] = cell_update(su[c], su[c - 1], su[c + 1], su[c - TW], su[c + TW], kc + sk[c - 1],
                        kc + sk[c + 1], kc + sk[c - TW], kc + sk[c + TW], dt * s[g], hdt);
  }
}

}  // namespace

cudaError_t launch_tile_f32(const float* u_in, float* u_out, const float* kappa, const float* src,
                            int nx, int ny, float dt, int bc, dim3 grid, dim3 block, size_t shm,
                            cudaStream_t s) {
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  tile_step_f32<<<grid, block, shm, s>>>(u_in, u_out, kappa, src, nx, ny, dt, 0.5f * dt, bc);
  return cudaGetLastError();
}

}  // namespace cpb
