// The 3-D 7-point stencil (the class of the paper's hotspot3D benchmark):
// a z-marching tiled kernel with a __syncthreads inside its plane loop.
//
// Update (the 2-D flux-form step with a third pair of faces, rounded in
// exactly this order): D = plane below, U = plane above,
//   f   = (kc + kn) * (un - c)                for n in W, E, S, N, D, U
//   acc = ((fW + fE) + (fS + fN)) + (fD + fU)
//   u'  = c + (hdt * acc + dt * s)
// Boundaries as in 2-D: a Dirichlet ghost has u = 0 and the kappa of the
// nearest in-grid cell (so a boundary face conducts with 2 kc); periodic
// wraps every axis.  Layout u[z][y][x], x fastest.
//
// Work decomposition.  A CTA of 32 x BY threads owns a tile of 128 columns x
// BY rows and a run of planes [z0, z1) (grid.z chunks of ceil(nz / grid.z)
// planes).  Lane l of warp ty holds the 4 cells x0 + 4l .. x0 + 4l + 3 of row
// y, so every row access is one 16-byte load or store per lane.  Per plane z:
//   issue the loads of the next plane (the lane's u, kappa of plane z + 2 and
//   s of plane z + 1; the first and last warp also the y-halo rows of plane
//   z + 1, lanes 0 and 31 the x-halo cell beyond the tile's edge), so every
//   load has one plane of work to arrive;
//   stage u and kappa of plane z, with its y-halo rows, into the shared tile
//   (double-buffered by plane parity);
//   __syncthreads()
//   x-neighbours of the lane's edge cells by warp shuffle (the x-halo at the
//   tile edges), y-neighbours from the tile, z-neighbours from the registers
//   holding planes z - 1 and z + 1; store u'.
// With two tile buffers one barrier per plane suffices (a warp cannot reach
// the buffer of plane z again before all warps have passed the barrier of
// plane z + 1).  HBM traffic per cell-update: u, kappa, s read once and u
// written once (16 B); the y-halo rows and the z-chunk's two extra planes are
// re-reads, mostly from L2.
#include "common.cuh"
#include "internal.h"

namespace cpb {
namespace {

struct VolArgs {
  const float* u;
  float* uo;
  const float* k;
  const float* s;
  int nx, ny, nz;
  float dt, hdt;
  int bc;
  int vec;  // 16-byte accesses: nx % 4 == 0 and 16-byte aligned fields
  int pz;   // planes per z-chunk
};

#define CPB_FULL_MASK 0xffffffffu

__device__ __forceinline__ size_t vidx(const VolArgs& a, int x, int y, int z) {
  return ((size_t)z * a.ny + y) * a.nx + x;
}

// u and kappa of one cell under the boundary rule.
__device__ __forceinline__ void cell_at(const VolArgs& a, int x, int y, int z, float& uv, float& kv) {
  if (a.bc == BC_PERIODIC) {
    const size_t g = vidx(a, wrap_index(x, a.nx), wrap_index(y, a.ny), wrap_index(z, a.nz));
    uv = __ldg(a.u + g);
    kv = __ldg(a.k + g);
  } else {
    const bool in = x >= 0 && x < a.nx && y >= 0 && y < a.ny && z >= 0 && z < a.nz;
    const size_t g = vidx(a, clamp_index(x, a.nx), clamp_index(y, a.ny), clamp_index(z, a.nz));
    kv = __ldg(a.k + g);
    uv = in ? __ldg(a.u + g) : 0.0f;
  }
}

// u and kappa of the 4 cells x0 .. x0+3 (x0 % 4 == 0) of row (y, z).
__device__ __forceinline__ void row4(const VolArgs& a, int x0, int y, int z, float4& u4, float4& k4) {
  if (a.vec) {
    if (a.bc == BC_PERIODIC) {
      const size_t g = vidx(a, wrap_index(x0, a.nx), wrap_index(y, a.ny), wrap_index(z, a.nz));
      u4 = __ldg(reinterpret_cast<const float4*>(a.u + g));
      k4 = __ldg(reinterpret_cast<const float4*>(a.k + g));
    } else {
      // nx % 4 == 0: the 4 cells are all inside or all outside in x
      const bool xin = x0 < a.nx;
      const bool in = xin && y >= 0 && y < a.ny && z >= 0 && z < a.nz;
      const size_t g = vidx(a, xin ? x0 : a.nx - 4, clamp_index(y, a.ny), clamp_index(z, a.nz));
      k4 = __ldg(reinterpret_cast<const float4*>(a.k + g));
      if (!xin) k4 = make_float4(k4.w, k4.w, k4.w, k4.w);  // ghost columns: kappa of column nx-1
      u4 = in ? __ldg(reinterpret_cast<const float4*>(a.u + g)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
    cell_at(a, x0, y, z, u4.x, k4.x);
    cell_at(a, x0 + 1, y, z, u4.y, k4.y);
    cell_at(a, x0 + 2, y, z, u4.z, k4.z);
    cell_at(a, x0 + 3, y, z, u4.w, k4.w);
  }
}

// s of the 4 cells (0 outside the grid or without a source).
__device__ __forceinline__ float4 src4(const VolArgs& a, int x0, int y, int z) {
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!a.s || y >= a.ny || z >= a.nz) return r;
  if (a.vec) {
    if (x0 < a.nx) r = __ldg(reinterpret_cast<const float4*>(a.s + vidx(a, x0, y, z)));
  } else {
    if (x0 < a.nx) r.x = __ldg(a.s + vidx(a, x0, y, z));
    if (x0 + 1 < a.nx) r.y = __ldg(a.s + vidx(a, x0 + 1, y, z));
    if (x0 + 2 < a.nx) r.z = __ldg(a.s + vidx(a, x0 + 2, y, z));
    if (x0 + 3 < a.nx) r.w = __ldg(a.s + vidx(a, x0 + 3, y, z));
  }
  return r;
}

__device__ __forceinline__ float update7(float c, float uW, float uE, float uS, float uN, float uD, float uU,
                                         float kc, float kW, float kE, float kS, float kN, float kD, float kU,
                                         float s, float dt, float hdt) {
  const float fW = (kc + kW) * (uW - c);
  const float fE = (kc + kE) * (uE - c);
  const float fS = (kc + kS) * (uS - c);
  const float fN = (kc + kN) * (uN - c);
  const float fD = (kc + kD) * (uD - c);
  const float fU = (kc + kU) * (uU - c);
  const float acc = ((fW + fE) + (fS + fN)) + (fD + fU);
  return c + (hdt * acc + dt * s);
}

__global__ void __launch_bounds__(256) vol_kernel(const VolArgs a) {
  extern __shared__ __align__(16) float4 tile[];
  const int lane = threadIdx.x, ty = threadIdx.y, BY = blockDim.y;
  const int TS = (BY + 2) * 32;  // float4s per field and buffer
  const int xt = blockIdx.x * 128, x0 = xt + 4 * lane;
  const int y = blockIdx.y * BY + ty;
  const int z0 = blockIdx.z * a.pz, z1 = min(a.nz, z0 + a.pz);
  if (z0 >= z1) return;  // uniform over the CTA
  const bool store = y < a.ny && x0 < a.nx;
  const bool south = ty == 0, north = ty == BY - 1, xedge = lane == 0 || lane == 31;
  const int xh = lane == 0 ? xt - 1 : xt + 128;  // the x-halo column of lanes 0 and 31

  // Registers: the lane's u, kappa of planes z-1, z, z+1, s of plane z, and
  // the halo values of plane z; each is loaded one plane ahead.
  float4 um, km, uc, kc, up, kp;
  row4(a, x0, y, z0 - 1, um, km);
  row4(a, x0, y, z0, uc, kc);
  row4(a, x0, y, z0 + 1, up, kp);
  float4 sc = src4(a, x0, y, z0);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 hsu = zero4, hsk = zero4, hnu = zero4, hnk = zero4;
  float hxu = 0.f, hxk = 0.f;
  if (south) row4(a, x0, y - 1, z0, hsu, hsk);
  if (north) row4(a, x0, y + 1, z0, hnu, hnk);
  if (xedge) cell_at(a, xh, y, z0, hxu, hxk);
  for (int z = z0; z < z1; ++z) {
    // issue the loads of the next plane (used from the next iteration on)
    float4 un = zero4, kn = zero4, sn = zero4, hsu_n = zero4, hsk_n = zero4, hnu_n = zero4, hnk_n = zero4;
    float hxu_n = 0.f, hxk_n = 0.f;
    if (z + 1 < z1) {
      row4(a, x0, y, z + 2, un, kn);
      sn = src4(a, x0, y, z + 1);
      if (south) row4(a, x0, y - 1, z + 1, hsu_n, hsk_n);
      if (north) row4(a, x0, y + 1, z + 1, hnu_n, hnk_n);
      if (xedge) cell_at(a, xh, y, z + 1, hxu_n, hxk_n);
    }
    // stage plane z into buffer z & 1: rows 0 and BY+1 are the y-halo rows
    float4* su = tile + (z & 1) * 2 * TS;
    float4* sk = su + TS;
    su[(ty + 1) * 32 + lane] = uc;
    sk[(ty + 1) * 32 + lane] = kc;
    if (south) {
      su[lane] = hsu;
      sk[lane] = hsk;
    }
    if (north) {
      su[(BY + 1) * 32 + lane] = hnu;
      sk[(BY + 1) * 32 + lane] = hnk;
    }
    // One barrier per plane: the tile is double-buffered, and a warp cannot
    // write this buffer again (plane z + 2) before every warp has passed the
    // barrier of plane z + 1, i.e. finished reading it.
    __syncthreads();
    const float4 uS = su[ty * 32 + lane], uN = su[(ty + 2) * 32 + lane];
    const float4 kS = sk[ty * 32 + lane], kN = sk[(ty + 2) * 32 + lane];
    float uWl = __shfl_up_sync(CPB_FULL_MASK, uc.w, 1), kWl = __shfl_up_sync(CPB_FULL_MASK, kc.w, 1);
    float uEl = __shfl_down_sync(CPB_FULL_MASK, uc.x, 1), kEl = __shfl_down_sync(CPB_FULL_MASK, kc.x, 1);
    if (lane == 0) {
      uWl = hxu;
      kWl = hxk;
    }
    if (lane == 31) {
      uEl = hxu;
      kEl = hxk;
    }
    if (store) {
      const float dt = a.dt, hdt = a.hdt;
      float4 o;
      o.x = update7(uc.x, uWl, uc.y, uS.x, uN.x, um.x, up.x, kc.x, kWl, kc.y, kS.x, kN.x, km.x, kp.x, sc.x,
                    dt, hdt);
      o.y = update7(uc.y, uc.x, uc.z, uS.y, uN.y, um.y, up.y, kc.y, kc.x, kc.z, kS.y, kN.y, km.y, kp.y, sc.y,
                    dt, hdt);
      o.z = update7(uc.z, uc.y, uc.w, uS.z, uN.z, um.z, up.z, kc.z, kc.y, kc.w, kS.z, kN.z, km.z, kp.z, sc.z,
                    dt, hdt);
      o.w = update7(uc.w, uc.z, uEl, uS.w, uN.w, um.w, up.w, kc.w, kc.z, kEl, kS.w, kN.w, km.w, kp.w, sc.w,
                    dt, hdt);
      float* dst = a.uo + vidx(a, x0, y, z);
      if (a.vec) {
        *reinterpret_cast<float4*>(dst) = o;
      } else {
        dst[0] = o.x;
        if (x0 + 1 < a.nx) dst[1] = o.y;
        if (x0 + 2 < a.nx) dst[2] = o.z;
        if (x0 + 3 < a.nx) dst[3] = o.w;
      }
    }
    um = uc;
    km = kc;
    uc = up;
    kc = kp;
    up = un;
    kp = kn;
    sc = sn;
    hsu = hsu_n;
    hsk = hsk_n;
    hnu = hnu_n;
    hnk = hnk_n;
    hxu = hxu_n;
    hxk = hxk_n;
  }
}

}  // namespace

size_t vol_smem_bytes(int by) { return (size_t)4 * (by + 2) * 32 * sizeof(float4); }

cudaError_t launch_vol_f32(const float* u_in, float* u_out, const float* kappa, const float* src, int nx,
                           int ny, int nz, float dt, int bc, int vec, dim3 grid, int by, cudaStream_t s) {
  VolArgs a;
  a.u = u_in;
  a.uo = u_out;
  a.k = kappa;
  a.s = src;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.dt = dt;
  a.hdt = 0.5f * dt;
  a.bc = bc;
  a.vec = vec;
  a.pz = (nz + (int)grid.z - 1) / (int)grid.z;
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  vol_kernel<<<grid, dim3(32, by, 1), vol_smem_bytes(by), s>>>(a);
  return cudaGetLastError();
}

}  // namespace cpb
