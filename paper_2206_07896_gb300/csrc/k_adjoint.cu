// Discrete adjoint of the N-step stencil (FP32 storage and arithmetic).
//
// Forward step: u_{n+1} = u_n + dt D(kappa) u_n + dt s, D symmetric (face
// coefficients (kc+kn)/2 shared by both cells; Dirichlet ghosts at 0).  For
// L = loss(u_T) with lambda_T = dL/du_T:
//   lambda_n = lambda_{n+1} + dt D(kappa) lambda_{n+1}     (the update, s = 0)
//   dL/dkappa_c += sum over faces f of c, with u = u_n, lambda = lambda_{n+1}:
//     interior face:            hdt * (u_f - u_c) * (lambda_c - lambda_f)
//     Dirichlet boundary face:  dt * (0 - u_c) * lambda_c
//   dL/du_0 = lambda_0.
// One kernel does both for one step: each thread owns one cell (so the
// kappa-gradient accumulation has no race), reads lambda, u and kappa at the
// cell and its 4 neighbours through L1/L2, writes lambda_n and adds to
// grad_kappa.  The driver (api.cu) recomputes each checkpoint segment's states
// with the forward kernels and then sweeps the segment backwards.
#include "common.cuh"
#include "internal.h"

namespace cpb {
namespace {

constexpr int ADJ_BX = 32, ADJ_BY = 8;

__global__ void __launch_bounds__(ADJ_BX* ADJ_BY)
    adjoint_step(const float* __restrict__ lam, float* __restrict__ lam_out,
                 const float* __restrict__ u, const float* __restrict__ k,
                 float* __restrict__ gk, int nx, int ny, float dt, float hdt, int bc) {
  const int i = blockIdx.x * ADJ_BX + threadIdx.x;
  const int j = blockIdx.y * ADJ_BY + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const bool periodic = bc == BC_PERIODIC;
  const size_t c = (size_t)j * nx + i;
  const float lc = lam[c], uc = u[c], kc = k[c];
  // neighbour values across the faces W, E, S, N
  float ln[4], un[4], kn[4];
  bool inside[4];
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    int ii = i + di[f], jj = j + dj[f];
    if (periodic) {
      ii = wrap_index(ii, nx);
      jj = wrap_index(jj, ny);
      inside[f] = true;
    } else {
      inside[f] = ii >= 0 && ii < nx && jj >= 0 && jj < ny;
    }
    if (inside[f]) {
      const size_t g = (size_t)jj * nx + ii;
      ln[f] = lam[g];
      un[f] = u[g];
      kn[f] = k[g];
    } else {
      ln[f] = 0.0f;
      un[f] = 0.0f;
      kn[f] = kc;
    }
  }
  lam_out[c] = cell_update(lc, ln[0], ln[1], ln[2], ln[3], kc + kn[0], kc + kn[1], kc + kn[2],
                           kc + kn[3], 0.0f, hdt);
  float g[4];
#pragma unroll
  for (int f = 0; f < 4; ++f)
    g[f] = inside[f] ? hdt * (un[f] - uc) * (lc - ln[f]) : dt * (0.0f - uc) * lc;
  gk[c] += (g[0] + g[1]) + (g[2] + g[3]);
}

}  // namespace

cudaError_t launch_adjoint_step(const float* lam, float* lam_out, const float* u, const float* k,
                                float* gk, int nx, int ny, float dt, int bc, cudaStream_t s) {
  dim3 block(ADJ_BX, ADJ_BY);
  dim3 grid((nx + ADJ_BX - 1) / ADJ_BX, (ny + ADJ_BY - 1) / ADJ_BY);
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  adjoint_step<<<grid, block, 0, s>>>(lam, lam_out, u, k, gk, nx, ny, dt, 0.5f * dt, bc);
  return cudaGetLastError();
}

}  // namespace cpb
