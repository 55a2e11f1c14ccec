// Streaming temporal-blocked stencil kernel (the tuned path of libcpb).
//
// Work decomposition
//   A warp owns a strip of 128 columns (4 consecutive columns per lane, so a
//   row of the strip is one 128-bit access per lane) and a chunk of output
//   rows [y0, y1).  It streams rows y0-K .. y1+K-1 of u, kappa and s from HBM
//   once and advances them K time steps in registers: level t (1..K) produces
//   row r_in - t from level t-1's rows r_in-t-1 .. r_in-t+1 as soon as input
//   row r_in has arrived.  Level t is valid on columns [x0+t, x0+128-t), so the
//   strip writes its inner 128 - 2*HALO columns (HALO = K rounded up to a
//   multiple of 4, which keeps stores 16-byte aligned); neighbouring strips
//   overlap by 2*HALO columns.  West/east neighbours of a lane's first/last
//   column come from the adjacent lanes by warp shuffle.
//   Face conductivity sums (kc + kE, kc + kN) and dt*s are time-invariant:
//   they are formed once per row and reused by all K levels.
//   Warps are independent (no shared memory, no block barrier); items are
//   numbered strip-fastest so neighbouring warps read overlapping halo columns
//   close together in time and the overlap hits L2.
//
// Boundaries
//   Dirichlet: cells outside the grid are ghosts held at u = 0; kappa of a
//   ghost is the kappa of the in-grid cell it touches (clamped index), so a
//   boundary face conducts with 2 kc.  Ghost values computed at any level are
//   reset to 0 before the next level reads them.  Periodic: indices wrap.
//
// Storage
//   A null source pointer means s = 0.
//   F32: u, kappa, s float.  BF16-Kahan: u as (hi | cmp << 16) words, kappa and
//   s bf16; every level rounds its result into (hi, cmp) and continues from
//   the represented value hi - cmp, exactly as if each step were stored.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace cpb {

struct StreamArgs {
  const void* u_in;
  void* u_out;
  const void* kappa;
  const void* src;
  int nx, ny;
  float dt, hdt;
  int bc, vec, chunk_rows;
  int n_strips, n_items;
};

#define CPB_FULL 0xffffffffu

template <bool BF>
struct Io;

template <>
struct Io<false> {
  static __device__ __forceinline__ float4 u4(const void* p, size_t i) {
    return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + i));
  }
  static __device__ __forceinline__ float4 k4(const void* p, size_t i) { return u4(p, i); }
  static __device__ __forceinline__ float u1(const void* p, size_t i) {
    return __ldg(static_cast<const float*>(p) + i);
  }
  static __device__ __forceinline__ float k1(const void* p, size_t i) { return u1(p, i); }
};

template <>
struct Io<true> {
  static __device__ __forceinline__ float4 u4(const void* p, size_t i) {
    uint4 w = __ldg(reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(p) + i));
    return make_float4(kahan_value(w.x), kahan_value(w.y), kahan_value(w.z), kahan_value(w.w));
  }
  static __device__ __forceinline__ float4 k4(const void* p, size_t i) {
    uint2 w = __ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(p) + i));
    return make_float4(bf16_bits_to_f32(w.x & 0xffffu), bf16_bits_to_f32(w.x >> 16),
                       bf16_bits_to_f32(w.y & 0xffffu), bf16_bits_to_f32(w.y >> 16));
  }
  static __device__ __forceinline__ float u1(const void* p, size_t i) {
    return kahan_value(__ldg(static_cast<const uint32_t*>(p) + i));
  }
  static __device__ __forceinline__ float k1(const void* p, size_t i) {
    return bf16_bits_to_f32(__ldg(static_cast<const unsigned short*>(p) + i));
  }
};

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }

template <int K, bool BF>
__global__ void __launch_bounds__(256) stream_kernel(const StreamArgs a) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  using IO = Io<BF>;
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items) return;  // warp-uniform
  const int nx = a.nx, ny = a.ny;
  const bool periodic = a.bc == BC_PERIODIC;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int xo = strip * OW;
  const int xs = xo - HALO + 4 * lane;
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, ny);
  const float dt = a.dt, hdt = a.hdt;

  // Column addressing of this lane's 4 cells.
  int xv = 0, kb = 0;      // vector path: load column, kappa broadcast (1: .x, 2: .w)
  bool cin4 = true;        // vector path, Dirichlet: the 4 columns are in the grid
  int xe[4];               // scalar path: per-cell column index
  bool ine[4];             // per-cell "column inside the grid" (Dirichlet ghost mask)
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int x = xs + e;
    ine[e] = periodic || (x >= 0 && x < nx);
    xe[e] = periodic ? wrap_index(x, nx) : clamp_index(x, nx);
  }
  if (a.vec) {
    if (periodic) {
      xv = wrap_index(xs, nx);
    } else {
      cin4 = xs >= 0 && xs < nx;
      xv = xs < 0 ? 0 : (xs > nx - 4 ? nx - 4 : xs);
      kb = xs < 0 ? 1 : (xs >= nx ? 2 : 0);
    }
  }
  // Output columns of this lane: inside [xo, xo+OW) and inside the grid.
  const bool lane_out = lane >= HALO / 4 && lane < (HALO + OW) / 4;

  auto load_row = [&](int r, float4& U, float4& Kp, float4& S) {
    bool rin = periodic || (r >= 0 && r < ny);
    int rr = periodic ? wrap_index(r, ny) : clamp_index(r, ny);
    size_t row = (size_t)rr * nx;
    if (a.vec) {
      float4 k4 = IO::k4(a.kappa, row + xv);
      if (kb == 1) k4 = f4(k4.x);
      if (kb == 2) k4 = f4(k4.w);
      Kp = k4;
      if (rin && cin4) {
        U = IO::u4(a.u_in, row + xv);
        S = a.src ? IO::k4(a.src, row + xv) : f4(0.0f);
      } else {
        U = f4(0.0f);
        S = f4(0.0f);
      }
    } else {
      float uu[4], kk[4], ss[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        kk[e] = IO::k1(a.kappa, row + xe[e]);
        bool in = rin && ine[e];
        uu[e] = in ? IO::u1(a.u_in, row + xe[e]) : 0.0f;
        ss[e] = (in && a.src) ? IO::k1(a.src, row + xe[e]) : 0.0f;
      }
      U = make_float4(uu[0], uu[1], uu[2], uu[3]);
      Kp = make_float4(kk[0], kk[1], kk[2], kk[3]);
      S = make_float4(ss[0], ss[1], ss[2], ss[3]);
    }
  };

  // Rings (see header): at the start of iteration r_in
  //   W[t][0], W[t][1] = level-t rows r_in-t-2, r_in-t-1   (t = 0..K-1)
  //   FE[q] = faceE(r_in-1-q), DS[q] = dt*s(r_in-1-q), FN[q] = faceN(r_in-2-q)
  //   kprev = kappa(r_in-1)
  float4 W[K][2], FE[K], DS[K], FN[K], kprev = f4(0.0f);
#pragma unroll
  for (int t = 0; t < K; ++t) {
    W[t][0] = W[t][1] = FE[t] = DS[t] = FN[t] = f4(0.0f);
  }

  int r_in = y0 - K;
  const int r_end = y1 + K;
  float4 pu, pk, ps;
  load_row(r_in, pu, pk, ps);
  for (; r_in < r_end; ++r_in) {
    const float4 un = pu, kn = pk, sn = ps;
    if (r_in + 1 < r_end) load_row(r_in + 1, pu, pk, ps);

    // Per-row time-invariant terms for row r_in (and faceN of row r_in-1).
    const float4 fn_new = make_float4(kprev.x + kn.x, kprev.y + kn.y, kprev.z + kn.z, kprev.w + kn.w);
    const float kx_e = __shfl_down_sync(CPB_FULL, kn.x, 1);
    const float4 fe_new = make_float4(kn.x + kn.y, kn.y + kn.z, kn.z + kn.w, kn.w + kx_e);
    const float4 ds_new = make_float4(dt * sn.x, dt * sn.y, dt * sn.z, dt * sn.w);

    float4 nw = un;  // the row level t-1 produced in this iteration
    uint4 packed = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      const int rho = r_in - t;
      const float4 C = W[t - 1][1], S = W[t - 1][0], N = nw;
      const float4 fe = FE[t - 1], ds = DS[t - 1], fs = FN[t - 1];
      const float4 fn = (t == 1) ? fn_new : FN[t - 2];
      const float uWx = __shfl_up_sync(CPB_FULL, C.w, 1);
      const float uEw = __shfl_down_sync(CPB_FULL, C.x, 1);
      const float fWx = __shfl_up_sync(CPB_FULL, fe.w, 1);
      float4 v;
      v.x = cell_update(C.x, uWx, C.y, S.x, N.x, fWx, fe.x, fs.x, fn.x, ds.x, hdt);
      v.y = cell_update(C.y, C.x, C.z, S.y, N.y, fe.x, fe.y, fs.y, fn.y, ds.y, hdt);
      v.z = cell_update(C.z, C.y, C.w, S.z, N.z, fe.y, fe.z, fs.z, fn.z, ds.z, hdt);
      v.w = cell_update(C.w, C.z, uEw, S.w, N.w, fe.z, fe.w, fs.w, fn.w, ds.w, hdt);
      if (BF) {
        float e0, e1, e2, e3;
        packed = make_uint4(kahan_round(v.x, e0), kahan_round(v.y, e1), kahan_round(v.z, e2),
                            kahan_round(v.w, e3));
        v = make_float4(e0, e1, e2, e3);
      }
      if (!periodic) {  // Dirichlet ghosts stay at zero
        if (rho < 0 || rho >= ny) v = f4(0.0f);
        v.x = ine[0] ? v.x : 0.0f;
        v.y = ine[1] ? v.y : 0.0f;
        v.z = ine[2] ? v.z : 0.0f;
        v.w = ine[3] ? v.w : 0.0f;
      }
      W[t - 1][0] = W[t - 1][1];
      W[t - 1][1] = nw;
      nw = v;
    }

    // Store level K's row.
    const int ro = r_in - K;
    if (ro >= y0 && lane_out) {
      const size_t row = (size_t)ro * nx;
      if (a.vec) {
        if (xs < nx) {
          if (BF)
            *reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.u_out) + row + xs) = packed;
          else
            *reinterpret_cast<float4*>(static_cast<float*>(a.u_out) + row + xs) = nw;
        }
      } else {
        const float vv[4] = {nw.x, nw.y, nw.z, nw.w};
        const uint32_t pw[4] = {packed.x, packed.y, packed.z, packed.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (xs + e < nx) {
            if (BF)
              static_cast<uint32_t*>(a.u_out)[row + xs + e] = pw[e];
            else
              static_cast<float*>(a.u_out)[row + xs + e] = vv[e];
          }
        }
      }
    }

    // Advance the rings.
#pragma unroll
    for (int q = K - 1; q > 0; --q) {
      FE[q] = FE[q - 1];
      DS[q] = DS[q - 1];
      FN[q] = FN[q - 1];
    }
    FE[0] = fe_new;
    DS[0] = ds_new;
    FN[0] = fn_new;
    kprev = kn;
  }
}

template <int K, bool BF>
cudaError_t launch_stream_k(const StreamPass& p, cudaStream_t s) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  StreamArgs a;
  a.u_in = p.u_in;
  a.u_out = p.u_out;
  a.kappa = p.kappa;
  a.src = p.src;
  a.nx = p.nx;
  a.ny = p.ny;
  a.dt = p.dt;
  a.hdt = p.hdt;
  a.bc = p.bc;
  a.vec = p.vec;
  a.chunk_rows = p.chunk_rows;
  a.n_strips = (p.nx + OW - 1) / OW;
  const long long n_chunks = (p.ny + p.chunk_rows - 1) / p.chunk_rows;
  const long long items = (long long)a.n_strips * n_chunks;
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  a.n_items = (int)items;
  const int wpb = p.warps_per_block;
  const long long blocks = (items + wpb - 1) / wpb;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  stream_kernel<K, BF><<<(unsigned)blocks, 32 * wpb, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool BF>
cudaError_t launch_stream_any(const StreamPass& p, int k, cudaStream_t s) {
  switch (k) {
    case 1: return launch_stream_k<1, BF>(p, s);
    case 2: return launch_stream_k<2, BF>(p, s);
    case 3: return launch_stream_k<3, BF>(p, s);
    case 4: return launch_stream_k<4, BF>(p, s);
    case 5: return launch_stream_k<5, BF>(p, s);
    case 6: return launch_stream_k<6, BF>(p, s);
    case 7: return launch_stream_k<7, BF>(p, s);
    case 8: return launch_stream_k<8, BF>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cpb
