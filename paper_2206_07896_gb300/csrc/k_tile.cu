// The tiled one-step stencil kernel: one thread per cell, a (bx+2) x (by+2)
// shared tile of u and of kappa with a one-cell halo, one __syncthreads.
//
// This is the kernel class the paper translates for CPUs (Sec. III "SPMD to MPMD"): its
// two barrier-free regions -- stage the tile, then update from the tile --
// are what the CPU executor turns into two thread loops ("loop fission").
// Launch geometry is the caller's (<<<grid, block, shm>>>), one launch per step.
#include "common.cuh"
#include "internal.h"

namespace cpb {
namespace {

// Periodic wrap of a tile position, which lies within one period of [0, n)
// unless the grid is smaller than the tile's halo: compares instead of an
// integer division in the common case.
__device__ __forceinline__ int wrap_tile(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  return wrap_index(i, n);
}

// Stage the value seen at grid position (gi, gj) into tile slot `slot`:
// inside the grid the cell itself; outside, the boundary rule (Dirichlet:
// u = 0 and kappa of the nearest in-grid cell, which is the kappa of the cell
// across the face; periodic: wrap).
__device__ __forceinline__ void stage(const float* __restrict__ u, const float* __restrict__ k,
                                      int nx, int ny, int bc, int gi, int gj, float* su, float* sk,
                                      int slot) {
  const size_t n = (size_t)nx * ny;
  if (bc == BC_PERIODIC) {
    size_t g = CPB_CHK((size_t)wrap_tile(gj, ny) * nx + wrap_tile(gi, nx), 1, n);
    su[slot] = u[g];
    sk[slot] = k[g];
  } else {
    bool inside = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    su[slot] = inside ? u[CPB_CHK((size_t)gj * nx + gi, 1, n)] : 0.0f;
    sk[slot] = k[CPB_CHK((size_t)clamp_index(gj, ny) * nx + clamp_index(gi, nx), 1, n)];
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
    const size_t g = CPB_CHK((size_t)gj * nx + gi, 1, (size_t)nx * ny);
    const float kc = sk[c];
    uo[g] = cell_update(su[c], su[c - 1], su[c + 1], su[c - TW], su[c + TW], kc + sk[c - 1],
                        kc + sk[c + 1], kc + sk[c - TW], kc + sk[c + TW], dt * s[g], hdt);
  }
}

// The shared-memory temporal-blocked tiled kernel: `d` steps per launch and
// d + 1 barriers, d of them inside the time loop -- the multi-barrier kernel
// class (the paper's srad has nine block synchronisations, Sec. V) whose CPU
// translation needs loop fission with the time loop kept.  A block of
// BX x BY threads stages a (BX + 2d) x (BY + 2d) tile of u, kappa and s
// (tile origin (bx BX - d, by BY - d); boundary rule as in stage()), then for
// t = 1 .. d updates the shrinking region [t, TW - t) x [t, TH - t) from level
// t - 1 into level t (two u tiles, alternating), a barrier after each level,
// and writes level d of its BX x BY interior.  Each thread covers the tile
// positions (tx + i BX, ty + j BY).  Every cell update is the canonical
// per-cell expression, so the result does not depend on d or the geometry.
__global__ void tile_blocked_f32(const float* __restrict__ u, float* __restrict__ uo,
                                 const float* __restrict__ k, const float* __restrict__ s, int nx,
                                 int ny, float dt, float hdt, int bc, int d) {
  extern __shared__ float tb[];
  const int BX = blockDim.x, BY = blockDim.y, TW = BX + 2 * d, TH = BY + 2 * d, NT = TW * TH;
  float* lev0 = tb;
  float* lev1 = tb + NT;
  float* kt = tb + 2 * NT;
  float* st = tb + 3 * NT;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx0 = blockIdx.x * BX - d, gy0 = blockIdx.y * BY - d;
  const bool periodic = bc == BC_PERIODIC;
  // Region 0: stage the tile.
  for (int tj = ty; tj < TH; tj += BY)
    for (int ti = tx; ti < TW; ti += BX) {
      const int gi = gx0 + ti, gj = gy0 + tj, c = tj * TW + ti;
      stage(u, k, nx, ny, bc, gi, gj, lev0, kt, c);
      float sv = 0.0f;
      if (s) {
        if (periodic)
          sv = s[CPB_CHK((size_t)wrap_tile(gj, ny) * nx + wrap_tile(gi, nx), 1, (size_t)nx * ny)];
        else if (gi >= 0 && gi < nx && gj >= 0 && gj < ny)
          sv = s[CPB_CHK((size_t)gj * nx + gi, 1, (size_t)nx * ny)];
      }
      st[c] = sv;
    }
  __syncthreads();
  // Regions 1 .. d: one time level each.
  for (int t = 1; t <= d; ++t) {
    const float* a = (t & 1) ? lev0 : lev1;
    float* b = (t & 1) ? lev1 : lev0;
    for (int tj = t + ty; tj < TH - t; tj += BY)
      for (int ti = t + tx; ti < TW - t; ti += BX) {
        const int c = tj * TW + ti;
        if (!periodic) {
          const int gi = gx0 + ti, gj = gy0 + tj;
          if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) {  // Dirichlet ghosts stay at zero
            b[c] = 0.0f;
            continue;
          }
        }
        const float kc = kt[c];
        b[c] = cell_update(a[c], a[c - 1], a[c + 1], a[c - TW], a[c + TW], kc + kt[c - 1], kc + kt[c + 1],
                           kc + kt[c - TW], kc + kt[c + TW], dt * st[c], hdt);
      }
    __syncthreads();
  }
  // Region d + 1: write the interior.
  const float* a = (d & 1) ? lev1 : lev0;
  const int gi = blockIdx.x * BX + tx, gj = blockIdx.y * BY + ty;
  if (gi < nx && gj < ny) uo[CPB_CHK((size_t)gj * nx + gi, 1, (size_t)nx * ny)] = a[(ty + d) * TW + tx + d];
}

unsigned g_tile_blocked_optin;  // devices on which the shared-memory opt-in was set

}  // namespace

size_t tile_blocked_smem_bytes(int bx, int by, int d) {
  return (size_t)4 * sizeof(float) * (size_t)(bx + 2 * d) * (size_t)(by + 2 * d);
}

cudaError_t launch_tile_blocked_f32(const float* u_in, float* u_out, const float* kappa, const float* src,
                                    int nx, int ny, float dt, int bc, int d, dim3 grid, dim3 block,
                                    cudaStream_t s) {
  const size_t shm = tile_blocked_smem_bytes((int)block.x, (int)block.y, d);
  if (shm > 48 * 1024) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(dev < 32 && (g_tile_blocked_optin & (1u << dev)))) {
      int optin = 0;
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess) return e;
      if (shm > (size_t)optin) return cudaErrorInvalidValue;
      e = cudaFuncSetAttribute((const void*)tile_blocked_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
      if (e != cudaSuccess) return e;
      if (dev < 32) g_tile_blocked_optin |= 1u << dev;
    }
  }
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  tile_blocked_f32<<<grid, block, shm, s>>>(u_in, u_out, kappa, src, nx, ny, dt, 0.5f * dt, bc, d);
  return cudaGetLastError();
}

cudaError_t launch_tile_f32(const float* u_in, float* u_out, const float* kappa, const float* src,
                            int nx, int ny, float dt, int bc, dim3 grid, dim3 block, size_t shm,
                            cudaStream_t s) {
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  tile_step_f32<<<grid, block, shm, s>>>(u_in, u_out, kappa, src, nx, ny, dt, 0.5f * dt, bc);
  return cudaGetLastError();
}

cudaError_t read_bounds_tile(int* out) { return read_bounds_word(out); }

}  // namespace cpb
