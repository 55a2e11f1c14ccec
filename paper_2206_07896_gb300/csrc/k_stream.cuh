// Streaming temporal-blocked stencil kernels (the tuned path of libcpb).
//
// Work decomposition
//   A warp owns a strip of 128 columns (4 consecutive columns per lane, so a
//   row of the strip is one 128-bit access per lane) and a chunk of output
//   rows [y0, y1).  It streams rows y0-d .. y1+d-1 of u, kappa and s from HBM
//   once and advances them d <= K time steps in registers: level t (1..d)
//   produces row r_in - t from level t-1's rows r_in-t-1 .. r_in-t+1 as soon as
//   input row r_in has arrived.  Level t is valid on columns [x0+t, x0+128-t),
//   so the strip writes its inner 128 - 2*HALO columns (HALO = K rounded up to
//   a multiple of 4, which keeps stores 16-byte aligned); neighbouring strips
//   overlap by 2*HALO columns.  West/east neighbours of a lane's first/last
//   column come from the adjacent lanes by warp shuffle.  Face conductivity
//   sums (kc + kE, kc + kN) and dt*s are time-invariant: they are formed once
//   per row and reused by every level.  Items are numbered strip-fastest so
//   neighbouring warps read overlapping halo columns close together in time.
//
// Two ways to bring rows in (same arithmetic, same results):
//   variant 0  each lane loads its 16 bytes of the next row into registers
//              one row ahead (any nx, any alignment);
//   variant 1  per warp, a ring of `stages` shared-memory row slots filled by
//              TMA bulk copies (cp.async.bulk, completion on one mbarrier per
//              slot): many rows in flight per warp without spending registers.
//              Needs 16-byte aligned fields, nx a multiple of 4 (FP32) or 8
//              (BF16-Kahan) and nx >= 128 (FP32) or 136 (BF16-Kahan).
//   Every mbarrier wait is bounded; on expiry the kernel records
//   CPB_ERR_TIMEOUT in a device status word (read by cpb_device_status),
//   drains its own copies (bounded) and returns.
//
// Boundaries
//   Dirichlet: cells outside the grid are ghosts held at u = 0; kappa of a
//   ghost is the kappa of the in-grid cell it touches (clamped index), so a
//   boundary face conducts with 2 kc.  Ghost values computed at any level are
//   reset to 0 before the next level reads them.  Periodic: indices wrap.
//
// Storage
//   F32: u, kappa, s float.  BF16-Kahan: u as (hi | cmp << 16) words, kappa and
//   s bf16; every level rounds its result into (hi, cmp) and continues from the
//   represented value hi - cmp, exactly as if each step were stored.  A null
//   source pointer means s = 0.
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
  int depth;       // time steps of this pass, 1..K
  int stages;      // variant 1: ring slots per warp (power of two)
  int wait_limit;  // variant 1: bounded mbarrier wait, in try_wait polls
  int inject_on;   // variant 1, tests only: 1 = the copies of row inject_row never complete
  int inject_row;
};

#define CPB_FULL 0xffffffffu

// Device status word of this translation unit (CPB_ERR_TIMEOUT after a wait
// gave up).  Read and cleared by the host through cpb_device_status.
static __device__ int g_stream_status;

template <bool BF>
struct Io;

template <>
struct Io<false> {
  static constexpr int U_BYTES = 4, KS_BYTES = 4;
  static __device__ __forceinline__ float4 u4(const void* p, size_t i) {
    return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + i));
  }
  static __device__ __forceinline__ float4 k4(const void* p, size_t i) { return u4(p, i); }
  static __device__ __forceinline__ float u1(const void* p, size_t i) {
    return __ldg(static_cast<const float*>(p) + i);
  }
  static __device__ __forceinline__ float k1(const void* p, size_t i) { return u1(p, i); }
  static __device__ __forceinline__ float4 u4_cg(const void* p, size_t i) {
    return __ldcg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + i));
  }
  static __device__ __forceinline__ float u1_cg(const void* p, size_t i) {
    return __ldcg(static_cast<const float*>(p) + i);
  }
  // shared-memory row slot readers (offset in cells)
  static __device__ __forceinline__ float4 su4(const unsigned char* row, int o) {
    return *reinterpret_cast<const float4*>(row + 4 * o);
  }
  static __device__ __forceinline__ float4 sk4(const unsigned char* row, int o) { return su4(row, o); }
};

template <>
struct Io<true> {
  static constexpr int U_BYTES = 4, KS_BYTES = 2;
  static __device__ __forceinline__ float4 unpack_u(uint4 w) {
    return make_float4(kahan_value(w.x), kahan_value(w.y), kahan_value(w.z), kahan_value(w.w));
  }
  static __device__ __forceinline__ float4 unpack_k(uint2 w) {
    return make_float4(bf16_bits_to_f32(w.x & 0xffffu), bf16_bits_to_f32(w.x >> 16),
                       bf16_bits_to_f32(w.y & 0xffffu), bf16_bits_to_f32(w.y >> 16));
  }
  static __device__ __forceinline__ float4 u4(const void* p, size_t i) {
    return unpack_u(__ldg(reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(p) + i)));
  }
  static __device__ __forceinline__ float4 k4(const void* p, size_t i) {
    return unpack_k(__ldg(reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(p) + i)));
  }
  static __device__ __forceinline__ float u1(const void* p, size_t i) {
    return kahan_value(__ldg(static_cast<const uint32_t*>(p) + i));
  }
  static __device__ __forceinline__ float k1(const void* p, size_t i) {
    return bf16_bits_to_f32(__ldg(static_cast<const unsigned short*>(p) + i));
  }
  static __device__ __forceinline__ float4 u4_cg(const void* p, size_t i) {
    return unpack_u(__ldcg(reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(p) + i)));
  }
  static __device__ __forceinline__ float u1_cg(const void* p, size_t i) {
    return kahan_value(__ldcg(static_cast<const uint32_t*>(p) + i));
  }
  static __device__ __forceinline__ float4 su4(const unsigned char* row, int o) {
    return unpack_u(*reinterpret_cast<const uint4*>(row + 4 * o));
  }
  static __device__ __forceinline__ float4 sk4(const unsigned char* row, int o) {
    return unpack_k(*reinterpret_cast<const uint2*>(row + 2 * o));
  }
};

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }

// Column geometry of one lane's 4 cells inside its strip.
struct LaneCols {
  int xs;       // first column (unwrapped), multiple of 4
  int xv;       // vector path: column of the 16-byte access (wrapped / clamped)
  int kb;       // Dirichlet ghost lane: broadcast kappa .x (1) or .w (2) of the edge access
  bool cin4;    // the 4 columns are inside the grid (vector path)
  bool ine[4];  // per-cell inside flag (Dirichlet ghost mask)
  int xe[4];    // scalar path: per-cell wrapped / clamped column
};

__device__ __forceinline__ LaneCols lane_cols(int xs, int nx, bool periodic) {
  LaneCols c;
  c.xs = xs;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int x = xs + e;
    c.ine[e] = periodic || (x >= 0 && x < nx);
    c.xe[e] = periodic ? wrap_index(x, nx) : clamp_index(x, nx);
  }
  if (periodic) {
    c.xv = wrap_index(xs, nx);
    c.cin4 = true;
    c.kb = 0;
  } else {
    c.cin4 = xs >= 0 && xs < nx;
    c.xv = xs < 0 ? 0 : (xs > nx - 4 ? nx - 4 : xs);
    c.kb = xs < 0 ? 1 : (xs >= nx ? 2 : 0);
  }
  return c;
}

// The K-level register pipeline of one warp strip.  At the start of the
// iteration that receives input row r_in:
//   W[t][0], W[t][1] = level-t rows r_in-t-2, r_in-t-1   (t = 0..K-1)
//   FE[q] = faceE(r_in-1-q), DS[q] = dt*s(r_in-1-q), FN[q] = faceN(r_in-2-q)
//   kprev = kappa(r_in-1)
template <int K, bool BF>
struct Pipe {
  float4 W[K][2], FE[K], DS[K], FN[K], kprev;

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int t = 0; t < K; ++t) W[t][0] = W[t][1] = FE[t] = DS[t] = FN[t] = f4(0.0f);
    kprev = f4(0.0f);
  }

  // Consume input row r_in; leaves level d's row r_in - d in `out` (and, for
  // BF16-Kahan storage, its packed words in `packed`).
  __device__ __forceinline__ void step(int r_in, int d, int ny, bool periodic, const LaneCols& lc,
                                       float dt, float hdt, float4 un, float4 kn, float4 sn,
                                       float4& out, uint4& packed) {
    const float4 fn_new = make_float4(kprev.x + kn.x, kprev.y + kn.y, kprev.z + kn.z, kprev.w + kn.w);
    const float kx_e = __shfl_down_sync(CPB_FULL, kn.x, 1);
    const float4 fe_new = make_float4(kn.x + kn.y, kn.y + kn.z, kn.z + kn.w, kn.w + kx_e);
    const float4 ds_new = make_float4(dt * sn.x, dt * sn.y, dt * sn.z, dt * sn.w);

    float4 nw = un;  // the row level t-1 produced in this iteration
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      if (t <= d) {
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
          v.x = lc.ine[0] ? v.x : 0.0f;
          v.y = lc.ine[1] ? v.y : 0.0f;
          v.z = lc.ine[2] ? v.z : 0.0f;
          v.w = lc.ine[3] ? v.w : 0.0f;
        }
        W[t - 1][0] = W[t - 1][1];
        W[t - 1][1] = nw;
        nw = v;
      }
    }
    out = nw;
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
};

// Store one output row of a lane (only columns this strip owns).
template <bool BF>
__device__ __forceinline__ void store_row(void* u_out, size_t row, int xs, int nx, bool vec,
                                          float4 v, uint4 packed) {
  if (vec) {
    if (xs < nx) {
      if (BF)
        *reinterpret_cast<uint4*>(static_cast<uint32_t*>(u_out) + row + xs) = packed;
      else
        *reinterpret_cast<float4*>(static_cast<float*>(u_out) + row + xs) = v;
    }
  } else {
    const float vv[4] = {v.x, v.y, v.z, v.w};
    const uint32_t pw[4] = {packed.x, packed.y, packed.z, packed.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (xs + e < nx) {
        if (BF)
          static_cast<uint32_t*>(u_out)[row + xs + e] = pw[e];
        else
          static_cast<float*>(u_out)[row + xs + e] = vv[e];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// variant 0: register prefetch, one row ahead
// ---------------------------------------------------------------------------
// One warp item (strip, chunk) of one pass.  COH: read u through L2 only
// (ld.global.cg), for callers that read, in the same launch, a buffer they
// wrote earlier (the batched persistent kernel); otherwise the read-only path.
// FULL: the pass depth is K (known at compile time, so the per-level depth
// guards fold away); otherwise the depth a.depth <= K is read at run time.
template <int K, bool BF, bool COH, bool FULL = false>
__device__ __forceinline__ void stream_item(const StreamArgs& a, int item, int lane) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  using IO = Io<BF>;
  const int nx = a.nx, ny = a.ny, d = FULL ? K : a.depth;
  const bool periodic = a.bc == BC_PERIODIC;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int xo = strip * OW;
  const LaneCols lc = lane_cols(xo - HALO + 4 * lane, nx, periodic);
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, ny);
  const bool lane_out = lane >= HALO / 4 && lane < (HALO + OW) / 4;

  auto load_row = [&](int r, float4& U, float4& Kp, float4& S) {
    bool rin = periodic || (r >= 0 && r < ny);
    int rr = periodic ? wrap_index(r, ny) : clamp_index(r, ny);
    size_t row = (size_t)rr * nx;
    if (a.vec) {
      float4 k4 = IO::k4(a.kappa, row + lc.xv);
      if (lc.kb == 1) k4 = f4(k4.x);
      if (lc.kb == 2) k4 = f4(k4.w);
      Kp = k4;
      if (rin && lc.cin4) {
        U = COH ? IO::u4_cg(a.u_in, row + lc.xv) : IO::u4(a.u_in, row + lc.xv);
        S = a.src ? IO::k4(a.src, row + lc.xv) : f4(0.0f);
      } else {
        U = f4(0.0f);
        S = f4(0.0f);
      }
    } else {
      float uu[4], kk[4], ss[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        kk[e] = IO::k1(a.kappa, row + lc.xe[e]);
        bool in = rin && lc.ine[e];
        uu[e] = in ? (COH ? IO::u1_cg(a.u_in, row + lc.xe[e]) : IO::u1(a.u_in, row + lc.xe[e]))
                   : 0.0f;
        ss[e] = (in && a.src) ? IO::k1(a.src, row + lc.xe[e]) : 0.0f;
      }
      U = make_float4(uu[0], uu[1], uu[2], uu[3]);
      Kp = make_float4(kk[0], kk[1], kk[2], kk[3]);
      S = make_float4(ss[0], ss[1], ss[2], ss[3]);
    }
  };

  Pipe<K, BF> pipe;
  pipe.init();
  int r_in = y0 - d;
  const int r_end = y1 + d;
  float4 pu, pk, ps;
  load_row(r_in, pu, pk, ps);
  for (; r_in < r_end; ++r_in) {
    const float4 un = pu, kn = pk, sn = ps;
    if (r_in + 1 < r_end) load_row(r_in + 1, pu, pk, ps);
    float4 out;
    uint4 packed = make_uint4(0, 0, 0, 0);
    pipe.step(r_in, d, ny, periodic, lc, a.dt, a.hdt, un, kn, sn, out, packed);
    const int ro = r_in - d;
    if (ro >= y0 && lane_out) store_row<BF>(a.u_out, (size_t)ro * nx, lc.xs, nx, a.vec, out, packed);
  }
}

template <int K, bool BF>
__global__ void __launch_bounds__(256) stream_kernel(const StreamArgs a) {
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items) return;  // warp-uniform
  if (a.depth == K)
    stream_item<K, BF, false, true>(a, item, threadIdx.x & 31);
  else
    stream_item<K, BF, false, false>(a, item, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// variant 1: TMA bulk copies into a per-warp shared-memory ring
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier.  Returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One TMA bulk copy global -> this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Ring slot geometry.  A slot holds SW cells of u, kappa and s of one row,
// starting at column x0a = x0 rounded down to ALIGN cells, so that every
// bulk copy starts and ends on a 16-byte boundary (ALIGN cells of the
// narrowest field = 16 bytes when nx % ALIGN == 0).
template <bool BF>
struct Slot {
  static constexpr int ALIGN = BF ? 8 : 4;
  static constexpr int SW = BF ? 136 : 128;
  static constexpr int UB = Io<BF>::U_BYTES, KB = Io<BF>::KS_BYTES;
  static constexpr int BYTES = SW * (UB + 2 * KB);
  static constexpr int K_OFF = SW * UB;
  static constexpr int S_OFF = SW * (UB + KB);
};

// Issue the copies of input row r into a slot (all completing on one
// mbarrier); extra_bytes > 0 (tests only) expects bytes that never arrive.
// Columns: Dirichlet copies the in-grid part of [x0a, x0a+SW) (ghost cells
// are masked by the reader); periodic wraps, which takes two copies when the
// window crosses an edge (nx >= SW guarantees at most two).  u and s are
// skipped on a Dirichlet ghost row; kappa comes from the clamped row.
template <bool BF>
__device__ __forceinline__ void issue_row(const StreamArgs& a, int r, int x0a, unsigned char* slot,
                                          uint64_t* bar, uint32_t extra_bytes) {
  using SL = Slot<BF>;
  const int nx = a.nx, ny = a.ny;
  const bool periodic = a.bc == BC_PERIODIC;
  const bool rin = periodic || (r >= 0 && r < ny);
  const int rr = periodic ? wrap_index(r, ny) : clamp_index(r, ny);
  const size_t row = (size_t)rr * nx;
  int pc[2], pw[2], po[2], np;
  if (periodic) {
    const int c = wrap_index(x0a, nx);
    const int w1 = min(SL::SW, nx - c);
    pc[0] = c, pw[0] = w1, po[0] = 0, np = 1;
    if (w1 < SL::SW) pc[1] = 0, pw[1] = SL::SW - w1, po[1] = w1, np = 2;
  } else {
    const int lo = max(x0a, 0), hi = min(x0a + SL::SW, nx);
    pc[0] = lo, pw[0] = hi - lo, po[0] = lo - x0a, np = 1;
  }
  const uint32_t per_cell = SL::KB + (rin ? SL::UB + (a.src ? SL::KB : 0) : 0);
  uint32_t total = 0;
  for (int i = 0; i < np; ++i) total += (uint32_t)pw[i] * per_cell;
  mbar_arrive_expect_tx(bar, total + extra_bytes);
  for (int i = 0; i < np; ++i) {
    const size_t g = row + pc[i];
    bulk_g2s(slot + SL::K_OFF + po[i] * SL::KB,
             static_cast<const unsigned char*>(a.kappa) + g * SL::KB, pw[i] * SL::KB, bar);
    if (rin) {
      bulk_g2s(slot + po[i] * SL::UB, static_cast<const unsigned char*>(a.u_in) + g * SL::UB,
               pw[i] * SL::UB, bar);
      if (a.src)
        bulk_g2s(slot + SL::S_OFF + po[i] * SL::KB,
                 static_cast<const unsigned char*>(a.src) + g * SL::KB, pw[i] * SL::KB, bar);
    }
  }
}

template <int K, bool BF, bool FULL>
__device__ __forceinline__ void bulk_item(const StreamArgs& a, unsigned char* smem) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  using SL = Slot<BF>;
  using IO = Io<BF>;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int R = a.stages;
  unsigned char* ring = smem + (size_t)wib * R * SL::BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)(blockDim.x >> 5) * R * SL::BYTES) + wib * R;
  const int item = blockIdx.x * (blockDim.x >> 5) + wib;
  const int nx = a.nx, ny = a.ny, d = FULL ? K : a.depth;
  const bool periodic = a.bc == BC_PERIODIC;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int x0 = strip * OW - HALO;
  const int x0a = x0 & ~(SL::ALIGN - 1);  // floor to ALIGN (x0 may be negative)
  const LaneCols lc = lane_cols(x0 + 4 * lane, nx, periodic);
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, ny);
  const bool lane_out = lane >= HALO / 4 && lane < (HALO + OW) / 4;
  const int r_first = y0 - d, r_end = y1 + d, nrows = r_end - r_first;
  // Slot offsets (cells) of this lane's 4 cells and of the edge access that
  // supplies kappa to a Dirichlet ghost lane.
  const int own = x0 - x0a + 4 * lane;
  const int kofs = lc.kb ? lc.xv - x0a : own;

  if (lane == 0) {
    for (int i = 0; i < R; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < R && i < nrows; ++i)
      issue_row<BF>(a, r_first + i, x0a, ring + (size_t)i * SL::BYTES, &bars[i],
                    (a.inject_on && r_first + i == a.inject_row) ? 16u : 0u);
  }
  __syncwarp();

  Pipe<K, BF> pipe;
  pipe.init();
  int failed_at = -1;
  for (int i = 0; i < nrows; ++i) {
    const int r_in = r_first + i;
    const int slot = i & (R - 1);
    if (!mbar_wait_bounded(&bars[slot], (uint32_t)(i / R) & 1u, a.wait_limit)) {
      failed_at = i;
      break;
    }
    const unsigned char* srow = ring + (size_t)slot * SL::BYTES;
    const bool rin = periodic || (r_in >= 0 && r_in < ny);
    float4 kn = IO::sk4(srow + SL::K_OFF, kofs);
    if (lc.kb == 1) kn = f4(kn.x);
    if (lc.kb == 2) kn = f4(kn.w);
    float4 un = f4(0.0f), sn = f4(0.0f);
    if (rin && lc.cin4) {
      un = IO::su4(srow, own);
      if (a.src) sn = IO::sk4(srow + SL::S_OFF, own);
    }
    __syncwarp();
    // Every lane has read the slot: refill it with row r_in + R.
    if (lane == 0 && i + R < nrows) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_row<BF>(a, r_in + R, x0a, ring + (size_t)slot * SL::BYTES, &bars[slot],
                    (a.inject_on && r_in + R == a.inject_row) ? 16u : 0u);
    }
    float4 out;
    uint4 packed = make_uint4(0, 0, 0, 0);
    pipe.step(r_in, d, ny, periodic, lc, a.dt, a.hdt, un, kn, sn, out, packed);
    const int ro = r_in - d;
    if (ro >= y0 && lane_out) store_row<BF>(a.u_out, (size_t)ro * nx, lc.xs, nx, true, out, packed);
  }
  if (failed_at >= 0) {
    // Record the timeout, then give every row still in flight (issued but not
    // consumed) one more bounded wait so no copy targets this CTA's shared
    // memory after it exits.
    if (lane == 0) atomicExch(&g_stream_status, (int)CPB_ERR_TIMEOUT);
    const int last = min(nrows, failed_at + R);
    for (int j = failed_at; j < last; ++j)
      mbar_wait_bounded(&bars[j & (R - 1)], (uint32_t)(j / R) & 1u, a.wait_limit);
    __syncwarp();
  }
}

template <int K, bool BF>
__global__ void __launch_bounds__(256) stream_bulk_kernel(const StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= a.n_items) return;  // warp-uniform; no block-level barrier is used
  if (a.depth == K)
    bulk_item<K, BF, true>(a, smem);
  else
    bulk_item<K, BF, false>(a, smem);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
namespace {
// Per (storage, depth) kernel: devices on which the shared-memory opt-in was set.
unsigned g_bulk_attr_done[2][9];
}  // namespace

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
  a.depth = p.depth;
  a.stages = p.stages;
  a.wait_limit = p.wait_limit;
  a.inject_on = p.inject_on;
  a.inject_row = p.inject_row;
  a.n_strips = (p.nx + OW - 1) / OW;
  const long long n_chunks = (p.ny + p.chunk_rows - 1) / p.chunk_rows;
  const long long items = (long long)a.n_strips * n_chunks;
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  a.n_items = (int)items;
  const int wpb = p.warps_per_block;
  const long long blocks = (items + wpb - 1) / wpb;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (p.variant == 1) {
    const size_t shm = bulk_smem_bytes(BF, wpb, p.stages);
    // Opt in to more than 48 KB of dynamic shared memory, once per device.
    // The flag has internal linkage (one per translation unit and library):
    // a function-local static of a template would be merged across every
    // shared object loaded in the process.
    unsigned& attr_done = g_bulk_attr_done[BF ? 1 : 0][K];  // bit per device ordinal (< 32)
    int dev = 0;
    cudaGetDevice(&dev);
    if (shm > 48 * 1024 && (dev >= 32 || !(attr_done & (1u << dev)))) {
      int optin = 0;
      cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(stream_bulk_kernel<K, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin);
      if (e != cudaSuccess) return e;
      if (dev < 32) attr_done |= 1u << dev;
    }
    stream_bulk_kernel<K, BF><<<(unsigned)blocks, 32 * wpb, shm, s>>>(a);
  } else {
    stream_kernel<K, BF><<<(unsigned)blocks, 32 * wpb, 0, s>>>(a);
  }
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

// Read and clear this translation unit's device status word.
inline cudaError_t read_stream_status(int* out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_stream_status, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_stream_status, &zero, sizeof(int));
}

}  // namespace cpb
