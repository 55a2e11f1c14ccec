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
// One kernel does both for one step, each cell owned by one thread (so the
// kappa-gradient accumulation has no race): a per-cell form for any width,
// and a row-marching form with 16-byte accesses for nx % 4 == 0.  The driver (api.cu) recomputes each checkpoint segment's states
// with the forward kernels and then sweeps the segment backwards.
#include <algorithm>

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

// Row-marching form of the same step, for nx % 4 == 0 and 16-byte aligned
// fields: a warp owns a strip of 128 columns (4 per lane, 16-byte accesses)
// and a chunk of `rows` rows, and keeps rows j-1, j, j+1 of lambda, u and
// kappa in registers while it marches down, so each value is read once per
// step (the per-cell kernel reads every value five times).  x-neighbours come
// by shuffle; the strip's edge columns from lanes 0 and 31.  Every cell is
// computed with the per-cell kernel's expressions in the same order.  The
// chunk height is chosen at launch so the items fill about one wave of
// resident warps (the result does not depend on it).
constexpr int ADJ_WARPS = 4;

struct Row3 {
  float4 l, u, k;
};

__device__ __forceinline__ float4 ldg4(const float* p, size_t i) {
  return __ldg(reinterpret_cast<const float4*>(p + i));
}

__device__ __forceinline__ float comp(const float4& v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

__global__ void __launch_bounds__(32 * ADJ_WARPS)
    adjoint_rows(const float* __restrict__ lam, float* __restrict__ lam_out, const float* __restrict__ u,
                 const float* __restrict__ k, float* __restrict__ gk, int nx, int ny, float dt, float hdt,
                 int bc, int n_strips, int n_items, int rows) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
  if (item >= n_items) return;  // warp-uniform; no block-level barrier is used
  const int strip = item % n_strips, chunk = item / n_strips;
  const int xs = strip * 128, x0 = xs + 4 * lane;
  const int y0 = chunk * rows, y1 = min(ny, y0 + rows);
  const bool periodic = bc == BC_PERIODIC;
  const int xv = periodic ? wrap_index(x0, nx) : (x0 < nx ? x0 : nx - 4);  // a valid 16-byte column
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_row = [&](int r) -> Row3 {
    Row3 R{z4, z4, z4};
    if (periodic || (r >= 0 && r < ny)) {
      const size_t g = (size_t)(periodic ? wrap_index(r, ny) : r) * nx + xv;
      R.l = ldg4(lam, g);
      R.u = ldg4(u, g);
      R.k = ldg4(k, g);
    }
    return R;
  };
  // x-halo column of lanes 0 and 31 (west of the strip, east of the strip)
  const int xh = lane == 0 ? xs - 1 : xs + 128;
  const bool hin = periodic || (xh >= 0 && xh < nx);
  const int xhc = periodic ? wrap_index(xh, nx) : (xh < 0 ? 0 : (xh >= nx ? nx - 1 : xh));
  // Row j's gradient accumulator and x-halo values, loaded one row ahead
  // like the rows of lambda, u and kappa, so no load is waited for at its use.
  auto load_gk = [&](int r) -> float4 {
    return (r < y1 && x0 < nx) ? *reinterpret_cast<const float4*>(gk + (size_t)r * nx + x0) : z4;
  };
  auto load_halo = [&](int r, float& hl, float& hu, float& hk) {
    hl = hu = hk = 0.f;
    if ((lane == 0 || lane == 31) && hin && r < y1) {
      const size_t g = (size_t)r * nx + xhc;
      hl = __ldg(lam + g);
      hu = __ldg(u + g);
      hk = __ldg(k + g);
    }
  };
  Row3 S = load_row(y0 - 1), C = load_row(y0), N = load_row(y0 + 1);
  float4 g_cur = load_gk(y0);
  float hl, hu, hk;
  load_halo(y0, hl, hu, hk);
  for (int j = y0; j < y1; ++j) {
    const Row3 NN = (j + 1 < y1) ? load_row(j + 2) : Row3{z4, z4, z4};
    const float4 g_next = load_gk(j + 1);
    float hl_n, hu_n, hk_n;
    load_halo(j + 1, hl_n, hu_n, hk_n);
    const float lW1 = __shfl_up_sync(0xffffffffu, C.l.w, 1), lE1 = __shfl_down_sync(0xffffffffu, C.l.x, 1);
    const float uW1 = __shfl_up_sync(0xffffffffu, C.u.w, 1), uE1 = __shfl_down_sync(0xffffffffu, C.u.x, 1);
    const float kW1 = __shfl_up_sync(0xffffffffu, C.k.w, 1), kE1 = __shfl_down_sync(0xffffffffu, C.k.x, 1);
    if (x0 < nx) {
      const size_t c0 = (size_t)j * nx + x0;
      const float4 g_old = g_cur;
      const bool iS = periodic || j - 1 >= 0, iN = periodic || j + 1 < ny;
      float lo[4], go[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + e;
        const float lc = comp(C.l, e), uc = comp(C.u, e), kc = comp(C.k, e);
        float ln[4], un[4], kn[4];
        bool in[4];
        // W, E, S, N (same order as the per-cell kernel)
        in[0] = periodic || x - 1 >= 0;
        in[1] = periodic || x + 1 < nx;
        in[2] = iS;
        in[3] = iN;
        ln[0] = e > 0 ? comp(C.l, e - 1) : (lane == 0 ? hl : lW1);
        un[0] = e > 0 ? comp(C.u, e - 1) : (lane == 0 ? hu : uW1);
        kn[0] = e > 0 ? comp(C.k, e - 1) : (lane == 0 ? hk : kW1);
        ln[1] = e < 3 ? comp(C.l, e + 1) : (lane == 31 ? hl : lE1);
        un[1] = e < 3 ? comp(C.u, e + 1) : (lane == 31 ? hu : uE1);
        kn[1] = e < 3 ? comp(C.k, e + 1) : (lane == 31 ? hk : kE1);
        ln[2] = comp(S.l, e);
        un[2] = comp(S.u, e);
        kn[2] = comp(S.k, e);
        ln[3] = comp(N.l, e);
        un[3] = comp(N.u, e);
        kn[3] = comp(N.k, e);
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (!in[f]) {
            ln[f] = 0.0f;
            un[f] = 0.0f;
            kn[f] = kc;
          }
        lo[e] = cell_update(lc, ln[0], ln[1], ln[2], ln[3], kc + kn[0], kc + kn[1], kc + kn[2], kc + kn[3],
                            0.0f, hdt);
        float g[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) g[f] = in[f] ? hdt * (un[f] - uc) * (lc - ln[f]) : dt * (0.0f - uc) * lc;
        go[e] = comp(g_old, e) + ((g[0] + g[1]) + (g[2] + g[3]));
      }
      *reinterpret_cast<float4*>(lam_out + c0) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      *reinterpret_cast<float4*>(gk + c0) = make_float4(go[0], go[1], go[2], go[3]);
    }
    S = C;
    C = N;
    N = NN;
    g_cur = g_next;
    hl = hl_n;
    hu = hu_n;
    hk = hk_n;
  }
}

// Warps of adjoint_rows resident on the whole device, once per device
// (ordinal < 32; others are queried on every call).
int g_adj_resident[32];

cudaError_t resident_warps(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && g_adj_resident[dev] > 0) {
    *out = g_adj_resident[dev];
    return cudaSuccess;
  }
  int sms = 0, per_sm = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_rows, 32 * ADJ_WARPS, 0);
  if (e != cudaSuccess) return e;
  const int w = std::max(1, sms * std::max(1, per_sm) * ADJ_WARPS);
  if (dev < 32) g_adj_resident[dev] = w;
  *out = w;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_adjoint_step(const float* lam, float* lam_out, const float* u, const float* k,
                                float* gk, int nx, int ny, float dt, int bc, cudaStream_t s) {
  const uintptr_t al = reinterpret_cast<uintptr_t>(lam) | reinterpret_cast<uintptr_t>(lam_out) |
                       reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(k) |
                       reinterpret_cast<uintptr_t>(gk);
  if (nx % 4 == 0 && al % 16 == 0) {
    const int n_strips = (nx + 127) / 128;
    int warps = 0;
    cudaError_t e = resident_warps(&warps);
    if (e != cudaSuccess) return e;
    // rows per item: the items come to about one wave of resident warps;
    // at least 4 rows (the two halo rows are re-read per item)
    const long long want = ((long long)n_strips * ny + warps - 1) / warps;
    const int rows = (int)std::max(4LL, std::min(want, 1024LL));
    const long long items = (long long)n_strips * ((ny + rows - 1) / rows);
    if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((items + ADJ_WARPS - 1) / ADJ_WARPS);
    (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
    adjoint_rows<<<blocks, 32 * ADJ_WARPS, 0, s>>>(lam, lam_out, u, k, gk, nx, ny, dt, 0.5f * dt, bc, n_strips,
                                                   (int)items, rows);
    return cudaGetLastError();
  }
  dim3 block(ADJ_BX, ADJ_BY);
  dim3 grid((nx + ADJ_BX - 1) / ADJ_BX, (ny + ADJ_BY - 1) / ADJ_BY);
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  adjoint_step<<<grid, block, 0, s>>>(lam, lam_out, u, k, gk, nx, ny, dt, 0.5f * dt, bc);
  return cudaGetLastError();
}

}  // namespace cpb
