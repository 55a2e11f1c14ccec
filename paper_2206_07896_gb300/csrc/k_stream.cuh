// Streaming temporal-blocked stencil kernels (the tuned path of libcpb).
//
// Work decomposition
//   A warp owns a strip of 128 columns (4 consecutive columns per lane, so a
//   row of the strip is one 128-bit access per lane) and a chunk of output
//   rows [y0, y1).  It streams rows y0-d .. y1+d-1 of u, kappa and s from HBM
//   once and advances them d <= K time steps in registers: level t (1..d)
//   produces row r_in - t from level t-1's rows r_in-t-1 .. r_in-t+1 as soon as
//   input row r_in has arrived (see Pipe for the flux form of the update).
//   Level t is valid on columns [x0+t, x0+128-t),
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
//   s bf16.  RE = true (CPB_BF16_KAHAN): every level rounds its result into
//   (hi, cmp) and continues from the represented value hi - cmp, exactly as if
//   each step were stored.  RE = false (CPB_BF16_KAHAN_BLOCK): the levels of a
//   pass run in FP32 and only the row a pass stores is rounded into (hi, cmp).
//   A null source pointer means s = 0.
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
  int inject_on;   // variant 1, tests only: 1 = the copies of row inject_row are never issued
  int inject_row;
};

// Level-storing kernel only: the rows of level t (1..depth-1) of a pass go to
// p[t - 1] (each an nx x ny field).
struct LevelOut {
  float* p[7];
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

// Periodic wrap of an index that is usually within one period of [0, n):
// a compare or two instead of an integer division.
__device__ __forceinline__ int wrap_near(int i, int n) {
  if (i >= 0 && i < n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i < 2 * n) return i - n;
  return wrap_index(i, n);
}

template <int V>
struct Int {
  static constexpr int value = V;
};

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

// Per-lane ring of the time-invariant per-row terms, in shared memory: for
// each of `rf` row slots, the lane's faceE (kc + kE of its 4 cells), faceN
// (kc + kN) and dt*s, as float4s.  Each lane reads only what it wrote itself,
// so program order is the only ordering needed.  Layout per warp:
// [slot][field][lane] float4, field 0 = faceE, 1 = faceN, 2 = dt*s.
constexpr int FACE_FE = 0, FACE_FN = 1, FACE_DS = 2;
constexpr int FACE_SLOT_F4 = 3 * 32;  // float4 units per slot
constexpr int FACE_SLOT_BYTES = FACE_SLOT_F4 * 16;

// Rows of the face ring for depth k: level k reads row r_in - k and the
// newest row written is r_in, so k + 1 rows are needed; rounded up to even so
// that a row loop unrolled by the ring length keeps both the register parity
// and every face-ring slot a compile-time constant.
__host__ __device__ constexpr int face_ring_rows(int k) { return (k + 2) & ~1; }

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// BF16-Kahan rounding of two step results at once: hi = rn(v), cmp =
// rn(hi - v), value hi - cmp; the same operations as kahan_round, with packed
// conversions and differences.  words: (hi | cmp << 16) per cell.
__device__ __forceinline__ float2 kahan_round2(float2 v, uint2& words) {
  const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
  const float2 hif = __bfloat1622float2(hi);
  const float2 r = sub2(hif, v);  // hi - v, both components in one packed operation
  const __nv_bfloat162 cm = __floats2bfloat162_rn(r.x, r.y);
  const float2 cmf = __bfloat1622float2(cm);
  const unsigned hb = *reinterpret_cast<const unsigned*>(&hi), cb = *reinterpret_cast<const unsigned*>(&cm);
  words = make_uint2(__byte_perm(hb, cb, 0x5410), __byte_perm(hb, cb, 0x7632));
  return sub2(hif, cmf);  // hi - cmp
}

// The K-level pipeline of one warp strip, in flux form.
//
// Iteration r_in (input row r_in) lets level t (1..K) produce row
// rho = r_in - t from level t-1's rows rho (C, finished last iteration) and
// rho+1 (N, finished this iteration by level t-1).  The update is evaluated
// through face fluxes: F = (kc + kE)(uE - c) on each east face and
// G = (kc + kN)(uN - c) on each north face.  The west term of a cell is
// exactly -F of its west neighbour and the south term exactly -G of the row
// below at the same level (negation and the commuted sums are exact), so
//   acc = (fW + fE) + (fS + fN) = (F_i - F_{i-1}) + (G - G_below)
// gives the canonical rounding sequence bit for bit while each flux is formed
// once.  F_{i-1} of a lane's first cell comes from the lane to the west
// (shuffle); G_below is this level's G of the previous iteration, carried in
// registers.  The row-wise work (vertical fluxes and the combination) runs on
// packed FP32 pairs.
//
// Registers: U[t][p] holds level t's row written at iteration parity p (t = 0
// is the input), G[t][p] level t+1's north fluxes; with the row loop unrolled
// by 2 every index is a compile-time constant and no copies are needed.
template <int K, bool BF, bool RE = true>
struct Pipe {
  float4 U[K][2];
  float4 G[K][2];
  float4 kprev;
  float4* ring;  // this lane's slice: ring[slot * FACE_SLOT_F4 + field * 32]
  int slot_in;   // face-ring slot of the current input row

  static constexpr int RF = face_ring_rows(K);

  __device__ __forceinline__ void init(float4* warp_ring, int lane) {
#pragma unroll
    for (int t = 0; t < K; ++t) U[t][0] = U[t][1] = G[t][0] = G[t][1] = f4(0.0f);
    kprev = f4(0.0f);
    ring = warp_ring + lane;
    slot_in = 0;
    for (int i = 0; i < 3 * RF; ++i) ring[i * 32] = f4(0.0f);
  }

  __device__ __forceinline__ float4& at(int slot, int field) { return ring[slot * FACE_SLOT_F4 + field * 32]; }

  // Face-ring slot of the row n rows above the input row.  SLOT >= 0: the
  // input row's slot is the compile-time constant SLOT (the caller's row loop
  // is unrolled by RF and leaves slot_in untouched); SLOT < 0: slot_in.
  template <int SLOT>
  __device__ __forceinline__ int back(int n) const {
    if (SLOT >= 0) return (SLOT - n + 2 * RF) % RF;
    const int sl = slot_in - n;
    return sl < 0 ? sl + RF : sl;
  }

  // Consume input row r_in at iteration parity P.  Leaves level d's row
  // r_in - d in `out` (and, for BF16-Kahan storage, its packed words in
  // `packed`).  FULL: d == K.  SLOT: see back().
  template <int P, bool FULL, int SLOT = -1>
  __device__ __forceinline__ void step(int r_in, int d, int ny, bool periodic, const LaneCols& lc,
                                       float dt, float hdt, float4 un, float4 kn, float4 sn,
                                       float4& out, uint4& packed) {
    constexpr int Q = 1 - P;
    const float kx_e = __shfl_down_sync(CPB_FULL, kn.x, 1);
    at(back<SLOT>(0), FACE_FE) = make_float4(kn.x + kn.y, kn.y + kn.z, kn.z + kn.w, kn.w + kx_e);
    at(back<SLOT>(0), FACE_DS) = make_float4(dt * sn.x, dt * sn.y, dt * sn.z, dt * sn.w);
    at(back<SLOT>(1), FACE_FN) =
        make_float4(kprev.x + kn.x, kprev.y + kn.y, kprev.z + kn.z, kprev.w + kn.w);
    kprev = kn;
    U[0][P] = un;
    const float2 h2 = make_float2(hdt, hdt);

    float4 nw = un;
#pragma unroll
    for (int t = 1; t <= K; ++t) {
      if (FULL || t <= d) {
        const int rho = r_in - t;
        const float4 C = U[t - 1][Q], N = U[t - 1][P];
        const int sl = back<SLOT>(t);
        const float4 fe = at(sl, FACE_FE), fn = at(sl, FACE_FN), ds = at(sl, FACE_DS);
        const float uEw = __shfl_down_sync(CPB_FULL, C.x, 1);
        float4 F;
        F.x = fe.x * (C.y - C.x);
        F.y = fe.y * (C.z - C.y);
        F.z = fe.z * (C.w - C.z);
        F.w = fe.w * (uEw - C.w);
        const float Fm1 = __shfl_up_sync(CPB_FULL, F.w, 1);
        const float4 hsum = make_float4(F.x - Fm1, F.y - F.x, F.z - F.y, F.w - F.z);  // fW + fE
        // north-face fluxes and the combination, on packed pairs
        const float2 gl = mul2(lo2(fn), sub2(lo2(N), lo2(C)));
        const float2 gh = mul2(hi2(fn), sub2(hi2(N), hi2(C)));
        G[t - 1][P] = cat4(gl, gh);
        const float4 Gb = G[t - 1][Q];  // north fluxes of row rho-1: minus the south terms
        const float2 accl = add2(lo2(hsum), sub2(gl, lo2(Gb)));
        const float2 acch = add2(hi2(hsum), sub2(gh, hi2(Gb)));
        float4 v = cat4(add2(lo2(C), madd2(h2, accl, lo2(ds))), add2(hi2(C), madd2(h2, acch, hi2(ds))));
        uint4 pk = make_uint4(0, 0, 0, 0);
        if (BF && RE) {  // round every level into storage and continue from the stored value
          uint2 wl, wh;
          const float2 el = kahan_round2(lo2(v), wl), eh = kahan_round2(hi2(v), wh);
          pk = make_uint4(wl.x, wl.y, wh.x, wh.y);
          v = cat4(el, eh);
        } else if (BF && (FULL ? t == K : t == d)) {  // round only the row the pass stores
          uint2 wl, wh;
          kahan_round2(lo2(v), wl);
          kahan_round2(hi2(v), wh);
          pk = make_uint4(wl.x, wl.y, wh.x, wh.y);
        }
        if (!periodic) {  // Dirichlet ghosts stay at zero
          if (rho < 0 || rho >= ny) v = f4(0.0f);
          v.x = lc.ine[0] ? v.x : 0.0f;
          v.y = lc.ine[1] ? v.y : 0.0f;
          v.z = lc.ine[2] ? v.z : 0.0f;
          v.w = lc.ine[3] ? v.w : 0.0f;
        }
        if (t < K) U[t][P] = v;
        nw = v;
        packed = pk;
      }
    }
    out = nw;
    if (SLOT < 0) slot_in = (slot_in + 1 == RF) ? 0 : slot_in + 1;
  }
};

// Store one output row of a lane (only columns this strip owns) into a
// field of n cells.
template <bool BF>
__device__ __forceinline__ void store_row(void* u_out, size_t row, int xs, int nx, size_t n, bool vec,
                                          float4 v, uint4 packed) {
  if (vec) {
    if (xs < nx) {
      const size_t i = CPB_CHK(row + xs, 4, n);
      if (BF)
        *reinterpret_cast<uint4*>(static_cast<uint32_t*>(u_out) + i) = packed;
      else
        *reinterpret_cast<float4*>(static_cast<float*>(u_out) + i) = v;
    }
  } else {
    const float vv[4] = {v.x, v.y, v.z, v.w};
    const uint32_t pw[4] = {packed.x, packed.y, packed.z, packed.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (xs + e < nx) {
        const size_t i = CPB_CHK(row + xs + e, 1, n);
        if (BF)
          static_cast<uint32_t*>(u_out)[i] = pw[e];
        else
          static_cast<float*>(u_out)[i] = vv[e];
      }
    }
  }
}

template <int K, bool BF>
__device__ __forceinline__ bool item_interior(const StreamArgs& a, int item);

// ---------------------------------------------------------------------------
// variant 0: register prefetch, one row ahead
// ---------------------------------------------------------------------------
// One warp item (strip, chunk) of one pass.  COH: read u through L2 only
// (ld.global.cg), for callers that read, in the same launch, a buffer they
// wrote earlier (the batched persistent kernel); otherwise the read-only path.
// FULL: the pass depth is K (known at compile time, so the per-level depth
// guards fold away); otherwise the depth a.depth <= K is read at run time.
// INTERIOR: a Dirichlet item that touches no edge (item_interior) runs with
// the periodic flag, which skips the ghost masks (a run-time branch here, so
// no second copy of the loop body).
template <int K, bool BF, bool COH, bool FULL = false, bool RE = true, bool INTERIOR = false>
__device__ __forceinline__ void stream_item(const StreamArgs& a, int item, int lane, float4* face_ring) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  using IO = Io<BF>;
  const int nx = a.nx, ny = a.ny, d = FULL ? K : a.depth;
  const bool periodic = a.bc == BC_PERIODIC || (INTERIOR && item_interior<K, BF>(a, item));
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int xo = strip * OW;
  const LaneCols lc = lane_cols(xo - HALO + 4 * lane, nx, periodic);
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, ny);
  const bool lane_out = lane >= HALO / 4 && lane < (HALO + OW) / 4;
  const size_t ncell = (size_t)nx * ny;

  auto load_row = [&](int r, float4& U, float4& Kp, float4& S) {
    bool rin = periodic || (r >= 0 && r < ny);
    int rr = periodic ? wrap_near(r, ny) : clamp_index(r, ny);
    size_t row = (size_t)rr * nx;
    if (a.vec) {
      const size_t iv = CPB_CHK(row + lc.xv, 4, ncell);
      float4 k4 = IO::k4(a.kappa, iv);
      if (!periodic) {  // Dirichlet ghost lanes take kappa of the edge cell
        if (lc.kb == 1) k4 = f4(k4.x);
        if (lc.kb == 2) k4 = f4(k4.w);
      }
      Kp = k4;
      if (rin && lc.cin4) {
        U = COH ? IO::u4_cg(a.u_in, iv) : IO::u4(a.u_in, iv);
        S = a.src ? IO::k4(a.src, iv) : f4(0.0f);
      } else {
        U = f4(0.0f);
        S = f4(0.0f);
      }
    } else {
      float uu[4], kk[4], ss[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const size_t ie = CPB_CHK(row + lc.xe[e], 1, ncell);
        kk[e] = IO::k1(a.kappa, ie);
        bool in = rin && lc.ine[e];
        uu[e] = in ? (COH ? IO::u1_cg(a.u_in, ie) : IO::u1(a.u_in, ie)) : 0.0f;
        ss[e] = (in && a.src) ? IO::k1(a.src, ie) : 0.0f;
      }
      U = make_float4(uu[0], uu[1], uu[2], uu[3]);
      Kp = make_float4(kk[0], kk[1], kk[2], kk[3]);
      S = make_float4(ss[0], ss[1], ss[2], ss[3]);
    }
  };

  Pipe<K, BF, RE> pipe;
  pipe.init(face_ring, lane);
  const int r_end = y1 + d;
  float4 pu, pk, ps;
  load_row(y0 - d, pu, pk, ps);
  auto body = [&](auto parity, int r_in) {
    const float4 un = pu, kn = pk, sn = ps;
    if (r_in + 1 < r_end) load_row(r_in + 1, pu, pk, ps);
    float4 out;
    uint4 packed = make_uint4(0, 0, 0, 0);
    pipe.template step<decltype(parity)::value, FULL>(r_in, d, ny, periodic, lc, a.dt, a.hdt, un, kn,
                                                      sn, out, packed);
    const int ro = r_in - d;
    if (ro >= y0 && lane_out) store_row<BF>(a.u_out, (size_t)ro * nx, lc.xs, nx, ncell, a.vec, out, packed);
  };
  int r_in = y0 - d;
  for (; r_in + 1 < r_end; r_in += 2) {  // unrolled by 2: register slots alternate by parity
    body(Int<0>{}, r_in);
    body(Int<1>{}, r_in + 1);
  }
  if (r_in < r_end) body(Int<0>{}, r_in);
}

template <int K, bool BF, bool RE>
__global__ void __launch_bounds__(256) stream_kernel(const StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int wib = threadIdx.x >> 5;
  const int item = blockIdx.x * (blockDim.x >> 5) + wib;
  if (item >= a.n_items) return;  // warp-uniform
  float4* face = reinterpret_cast<float4*>(smem + (size_t)wib * face_ring_rows(K) * FACE_SLOT_BYTES);
  if (a.depth == K)
    stream_item<K, BF, false, true, RE>(a, item, threadIdx.x & 31, face);
  else
    stream_item<K, BF, false, false, RE>(a, item, threadIdx.x & 31, face);
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

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The helpers below take shared-memory addresses (32-bit, shared window);
// the pointer forms convert once.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  mbar_arrive_expect_tx(smem_addr(bar), bytes);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier.  Returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  return mbar_wait_bounded(smem_addr(bar), parity, limit);
}

// One TMA bulk copy global -> this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  bulk_g2s(smem_addr(dst), src, bytes, smem_addr(bar));
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

// Per-lane part of the copy plan of a strip's rows.  A row takes up to six
// bulk copies (kappa, u, s) x (one or two column pieces); lane j < 6 owns copy
// j: field j % 3 (0 = kappa, 1 = u, 2 = s), piece j / 3.  Columns: Dirichlet
// copies the in-grid part of [x0a, x0a+SW) (ghost cells are masked by the
// reader); periodic wraps, which takes two pieces when the window crosses an
// edge (nx >= SW guarantees at most two).  The row-independent part is
// computed once per item.
struct CopyPlan {
  bool active;          // this lane owns a copy (piece exists, field present)
  int field;            // 0 kappa, 1 u, 2 s
  const unsigned char* src_base;
  int col;              // first grid column of the piece
  int dst_off;          // byte offset in the slot
  uint32_t bytes;       // bytes of this copy
  uint32_t kappa_bytes, us_bytes;  // per row: kappa bytes, u+s bytes (for expect_tx)
};

template <bool BF>
__device__ __forceinline__ CopyPlan make_copy_plan(const StreamArgs& a, int x0a, int lane) {
  using SL = Slot<BF>;
  const int nx = a.nx;
  int pc[2], pw[2], po[2], np;
  if (a.bc == BC_PERIODIC) {
    const int c = wrap_index(x0a, nx);
    const int w1 = min(SL::SW, nx - c);
    pc[0] = c, pw[0] = w1, po[0] = 0, np = 1;
    pc[1] = 0, pw[1] = SL::SW - w1, po[1] = w1;
    if (w1 < SL::SW) np = 2;
  } else {
    const int lo = max(x0a, 0), hi = min(x0a + SL::SW, nx);
    pc[0] = lo, pw[0] = hi - lo, po[0] = lo - x0a, np = 1;
    pc[1] = pw[1] = po[1] = 0;
  }
  CopyPlan p;
  const int piece = lane / 3;
  p.field = lane % 3;
  p.active = lane < 6 && piece < np && !(p.field == 2 && a.src == nullptr);
  const int pcs = piece < 2 ? piece : 0;
  const int eb = p.field == 1 ? SL::UB : SL::KB;
  p.src_base = static_cast<const unsigned char*>(p.field == 0 ? a.kappa : (p.field == 1 ? a.u_in : a.src));
  p.col = pc[pcs];
  p.dst_off = (p.field == 0 ? SL::K_OFF : (p.field == 1 ? 0 : SL::S_OFF)) + po[pcs] * eb;
  p.bytes = (uint32_t)pw[pcs] * eb;
  const uint32_t cells = (uint32_t)pw[0] + (np == 2 ? (uint32_t)pw[1] : 0u);
  p.kappa_bytes = cells * SL::KB;
  p.us_bytes = cells * (SL::UB + (a.src ? SL::KB : 0));
  return p;
}

// Issue the copies of input row r into a slot, all completing on one mbarrier
// (lane 0 posts the expected byte count; a complete_tx that lands before it is
// allowed, the phase cannot finish before lane 0 arrives).  u and s are
// skipped on a Dirichlet ghost row; kappa comes from the clamped row.
// withhold (tests only): post the byte count but issue none of the copies, so
// the slot's phase never completes and no copy into it is in flight.
template <bool BF>
__device__ __forceinline__ void issue_row(const StreamArgs& a, const CopyPlan& cp, int r, int lane,
                                          unsigned char* slot, uint64_t* bar, bool withhold) {
  const bool periodic = a.bc == BC_PERIODIC;
  const bool rin = periodic || (r >= 0 && r < a.ny);
  if (lane == 0) mbar_arrive_expect_tx(bar, cp.kappa_bytes + (rin ? cp.us_bytes : 0u));
  if (cp.active && (rin || cp.field == 0) && !withhold) {
    const int rr = periodic ? wrap_near(r, a.ny) : clamp_index(r, a.ny);
    const size_t eb = cp.field == 1 ? Io<BF>::U_BYTES : Io<BF>::KS_BYTES;
    const size_t g = CPB_CHK((size_t)rr * a.nx + cp.col, cp.bytes / eb, (size_t)a.nx * a.ny);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk_g2s(slot + cp.dst_off, cp.src_base + g * eb, cp.bytes, bar);
  }
}

// Rows J .. N-1 of an unrolled group, in order, stopping at the first that
// fails: f(parity, slot, i) with both constants known at compile time.
template <int J, int N, class F>
__device__ __forceinline__ bool rows_unrolled(F& f, int i) {
  if constexpr (J == N) {
    return true;
  } else {
    if (!f(Int<J & 1>{}, Int<J>{}, i + J)) return false;
    return rows_unrolled<J + 1, N>(f, i);
  }
}

// Rows J, J + 2, .. < N of an unrolled group as pairs f(_, slot, i) with
// the slot a compile-time constant, stopping at the first that fails.
template <int J, int N, class F>
__device__ __forceinline__ bool pairs_unrolled(F& f, int i) {
  if constexpr (J >= N) {
    return true;
  } else {
    if (!f(Int<0>{}, Int<J>{}, i + J)) return false;
    return pairs_unrolled<J + 2, N>(f, i);
  }
}

// Depths at which the row loop takes rows in pairs: there the level
// registers already limit a multiprocessor to 8-10 warps, so the extra
// registers of a pair cost no occupancy and the overlap of two rows hides
// latency (measured on GB300 at 8192^2: depth 8, 444 -> 390 us per pass); at
// depth <= 5 a pair needs more than 128 registers and loses 16 -> 11 warps.
__host__ __device__ constexpr bool rows_in_pairs(int k) { return k >= 6; }

// One warp item of one pass through this warp's row ring (`ring`, a.stages
// slots), its mbarriers (`bars`) and face ring (`face`), for one boundary
// rule.  Returns false if a bounded wait expired: *status is set to
// CPB_ERR_TIMEOUT (if still 0), the ring is drained and its mbarriers are left
// as they are (the caller must not use the ring again).  On success the
// mbarriers are invalidated, so the next item may initialise them afresh.
//
// The row loop is unrolled by the face-ring length RF (even), so register
// parities and face-ring slots are constants; the last nrows % RF rows take
// the same body with run-time face slots.  Periodic refills walk a per-lane
// source pointer row by row (one compare for the wrap) and expect a constant
// byte count; Dirichlet refills go through issue_row (ghost rows).
template <int K, bool BF, bool FULL, bool PERIODIC, bool LV, bool RE, bool UNROLL = true>
__device__ __forceinline__ bool bulk_item_bc(const StreamArgs& a, int item, int lane, unsigned char* ring,
                                             uint64_t* bars, float4* face, int* status, const LevelOut* lv) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  constexpr bool periodic = PERIODIC;
  using SL = Slot<BF>;
  using IO = Io<BF>;
  constexpr int RF = Pipe<K, BF>::RF;
  const int R = a.stages;
  const int lgR = __ffs(R) - 1;  // R is a power of two
  const int nx = a.nx, ny = a.ny, d = FULL ? K : a.depth;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int x0 = strip * OW - HALO;
  const int x0a = x0 & ~(SL::ALIGN - 1);  // floor to ALIGN (x0 may be negative)
  const LaneCols lc = lane_cols(x0 + 4 * lane, nx, periodic);
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, ny);
  // Lanes that store: inside the strip's output columns and the grid.
  const bool lane_store = lane >= HALO / 4 && lane < (HALO + OW) / 4 && lc.xs < nx;
  const size_t ncell = (size_t)nx * ny;
  const int r_first = y0 - d, r_end = y1 + d, nrows = r_end - r_first;
  // Slot offsets (cells) of this lane's 4 cells and of the edge access that
  // supplies kappa to a Dirichlet ghost lane.
  const int own = x0 - x0a + 4 * lane;
  const int kofs = lc.kb ? lc.xv - x0a : own;
  const CopyPlan cp = make_copy_plan<BF>(a, x0a, lane);
  const uint32_t ring_s = smem_addr(ring), bars_s = smem_addr(bars);
  // Refill at iteration i issues row r_first + i + R; the test hook's row
  // (if any) is refilled at iteration inject_i.
  const int inject_i = a.inject_on ? a.inject_row - r_first - R : -0x7fffffff;

  if (lane == 0) {
    for (int i = 0; i < R; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  for (int i = 0; i < R && i < nrows; ++i)
    issue_row<BF>(a, cp, r_first + i, lane, ring + (size_t)i * SL::BYTES, &bars[i],
                  a.inject_on && r_first + i == a.inject_row);
  // Periodic refill cursor of this lane's copy: wrapped row and its source.
  const size_t row_bytes = (size_t)nx * (cp.field == 1 ? SL::UB : SL::KB);
  int next_row = 0;
  const unsigned char* next_src = nullptr;
  if (periodic) {
    next_row = wrap_index(r_first + R, ny);
    next_src = cp.src_base + (size_t)next_row * row_bytes + (size_t)cp.col * (cp.field == 1 ? SL::UB : SL::KB);
  }
  const uint32_t tx_periodic = cp.kappa_bytes + cp.us_bytes;

  Pipe<K, BF, RE> pipe;
  pipe.init(face, lane);
  int failed_at = -1;
  // Wait for input row i (slot i mod R) and read the lane's kappa, u and s.
  // The lanes poll converged (one try_wait per poll for the whole warp), so
  // they reach the same verdict; a warp vote here would make that explicit
  // but costs registers the pipeline needs (measured: -9%).
  auto fetch = [&](int i, float4& kn, float4& un, float4& sn) -> bool {
    const int r_in = r_first + i;
    const int slot = i & (R - 1);
    if (!mbar_wait_bounded(bars_s + 8u * slot, (uint32_t)(i >> lgR) & 1u, a.wait_limit)) return false;
    const unsigned char* srow = ring + (size_t)slot * SL::BYTES;
    const bool rin = periodic || (r_in >= 0 && r_in < ny);
    kn = IO::sk4(srow + SL::K_OFF, kofs);
    if (!periodic) {  // Dirichlet ghost lanes take kappa of the edge cell
      if (lc.kb == 1) kn = f4(kn.x);
      if (lc.kb == 2) kn = f4(kn.w);
    }
    un = f4(0.0f);
    sn = f4(0.0f);
    if (rin && lc.cin4) {
      un = IO::su4(srow, own);
      if (a.src) sn = IO::sk4(srow + SL::S_OFF, own);
    }
    return true;
  };
  // Every lane has read slot i mod R: refill it with row r_first + i + R.
  auto refill = [&](int i) {
    if (i + R >= nrows) return;
    const int slot = i & (R - 1);
    if (periodic) {
      const uint32_t bar = bars_s + 8u * slot;
      if (lane == 0) mbar_arrive_expect_tx(bar, tx_periodic);
      if (cp.active && i != inject_i) {
        const unsigned char* src = next_src;
#ifdef CPB_BOUNDS_CHECK
        const size_t eb = cp.field == 1 ? SL::UB : SL::KB;
        src = cp.src_base + CPB_CHK((size_t)(next_src - cp.src_base) / eb, cp.bytes / eb, (size_t)nx * ny) * eb;
#endif
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bulk_g2s(ring_s + (uint32_t)(slot * SL::BYTES + cp.dst_off), src, cp.bytes, bar);
      }
      next_src += row_bytes;
      if (++next_row == ny) {
        next_row = 0;
        next_src -= (size_t)ny * row_bytes;
      }
    } else {
      issue_row<BF>(a, cp, r_first + i + R, lane, ring + (size_t)slot * SL::BYTES, &bars[slot],
                    i == inject_i);
    }
  };
  // Advance the pipeline by input row i and store the finished row.
  auto compute = [&](auto parity, auto slot_c, int i, float4 kn, float4 un, float4 sn) {
    constexpr int SLOT = decltype(slot_c)::value;
    const int r_in = r_first + i;
    float4 out;
    uint4 packed = make_uint4(0, 0, 0, 0);
    pipe.template step<decltype(parity)::value, FULL, SLOT>(r_in, d, ny, periodic, lc, a.dt, a.hdt, un,
                                                            kn, sn, out, packed);
    if (i >= 2 * d && lane_store)  // output row r_in - d >= y0
      store_row<BF>(a.u_out, (size_t)(r_in - d) * nx, lc.xs, nx, ncell, true, out, packed);
    if constexpr (LV) {  // also the rows of levels 1..d-1 that fall in this chunk
#pragma unroll
      for (int t = 1; t < K; ++t) {
        const int rho = r_in - t;
        if (t < d && rho >= y0 && rho < y1 && lane_store)
          store_row<BF>(lv->p[t - 1], (size_t)rho * nx, lc.xs, nx, ncell, true,
                        pipe.U[t][decltype(parity)::value], packed);
      }
    }
  };
  auto body = [&](auto parity, auto slot_c, int i) -> bool {
    float4 kn, un, sn;
    if (!fetch(i, kn, un, sn)) {
      failed_at = i;
      return false;
    }
    __syncwarp();
    refill(i);
    compute(parity, slot_c, i, kn, un, sn);
    return true;
  };
  // Rows i and i + 1 (i even): both waits first, then one straight-line block
  // advancing both rows, in which row i + 1's lower levels can overlap row i's
  // upper levels (the spin-wait loop of a single row ends the scheduler's
  // block).  A failed wait consumed nothing that the drain below misses.
  auto pair = [&](auto, auto slot_c, int i) -> bool {
    constexpr int S0 = decltype(slot_c)::value;
    float4 k0, u0, s0, k1, u1, s1;
    if (!fetch(i, k0, u0, s0) || !fetch(i + 1, k1, u1, s1)) {
      failed_at = i;
      return false;
    }
    __syncwarp();
    refill(i);
    refill(i + 1);
    compute(Int<0>{}, Int<S0>{}, i, k0, u0, s0);
    compute(Int<1>{}, Int<S0 + 1>{}, i + 1, k1, u1, s1);
    return true;
  };
  int i = 0;
  if constexpr (UNROLL && rows_in_pairs(K)) {
    for (; i + RF <= nrows; i += RF)
      if (!pairs_unrolled<0, RF>(pair, i)) break;
  } else if constexpr (UNROLL) {
    for (; i + RF <= nrows; i += RF)
      if (!rows_unrolled<0, RF>(body, i)) break;
  }
  if (failed_at < 0) {
    // pipe.slot_in is still 0 = i mod RF: the run-time slots take over here
    for (; i + 1 < nrows; i += 2) {
      if (!body(Int<0>{}, Int<-1>{}, i)) break;
      if (!body(Int<1>{}, Int<-1>{}, i + 1)) break;
    }
    if (failed_at < 0 && i < nrows) body(Int<0>{}, Int<-1>{}, i);
  }
  if (failed_at >= 0) {
    // Record the timeout, then give every row still in flight (issued but not
    // consumed) one more bounded wait so no copy targets this CTA's shared
    // memory after it exits (a withheld row has no copy in flight).
    if (lane == 0) atomicCAS(status, 0, (int)CPB_ERR_TIMEOUT);
    const int last = min(nrows, failed_at + R);
    for (int j = failed_at; j < last; ++j)
      mbar_wait_bounded(&bars[j & (R - 1)], (uint32_t)(j >> lgR) & 1u, a.wait_limit);
    __syncwarp();
    return false;
  }
  // Every issued row was consumed, so no copy is in flight.
  __syncwarp();
  if (lane == 0)
    for (int j = 0; j < R; ++j) mbar_inval(&bars[j]);
  __syncwarp();
  return true;
}

// True if every cell and row the item touches lies inside the grid (the
// strip's columns and its TMA window, rows y0 - depth .. y1 + depth - 1).  A
// Dirichlet item of that kind computes exactly what the periodic code
// computes (nothing wraps, no ghost), so it can run that code without the
// ghost masks.
template <int K, bool BF>
__device__ __forceinline__ bool item_interior(const StreamArgs& a, int item) {
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const int x0 = strip * OW - HALO;
  const int x0a = x0 & ~(Slot<BF>::ALIGN - 1);
  const int y0 = chunk * a.chunk_rows;
  const int y1 = min(y0 + a.chunk_rows, a.ny);
  return x0a >= 0 && x0a + Slot<BF>::SW <= a.nx && x0 + 128 <= a.nx && y0 - a.depth >= 0 &&
         y1 + a.depth <= a.ny;
}

// EDGES (single-grid kernels, depth <= 6): the items of a Dirichlet grid
// that touch no edge run the periodic body (unrolled, no masks); the edge
// items run the masked body with its row loop not unrolled, so that one large
// loop body is live on a multiprocessor (two unrolled bodies executing side
// by side cost more in instruction fetch than the masks they save: measured
// at 8192^2, depth 8, 505 -> 652 us per pass).  Measured per pass on GB300:
// 16384^2 Dirichlet depth 4 915 -> 865 us, depth 6 1708 -> 1515 us.  At depth
// 8 the changed register allocation slowed the periodic body itself (8192^2:
// 385 -> 433 us), so depth 8, and the batched kernel (whose small grids are
// mostly edge items), keep the masked unrolled body for every Dirichlet item.
template <int K, bool BF, bool FULL, bool LV = false, bool RE = true, bool EDGES = false>
__device__ __forceinline__ bool bulk_item(const StreamArgs& a, int item, int lane, unsigned char* ring,
                                          uint64_t* bars, float4* face, int* status,
                                          const LevelOut* lv = nullptr) {
  constexpr bool SPLIT = EDGES && K <= 6;
  if (a.bc == BC_PERIODIC || (SPLIT && item_interior<K, BF>(a, item)))
    return bulk_item_bc<K, BF, FULL, true, LV, RE>(a, item, lane, ring, bars, face, status, lv);
  return bulk_item_bc<K, BF, FULL, false, LV, RE, !SPLIT>(a, item, lane, ring, bars, face, status, lv);
}

// Shared memory of a CTA of `nwarps` warps using the row ring:
// [row rings of all warps][mbarriers of all warps][face rings of all warps].
template <int K, bool BF>
struct BulkSmem {
  unsigned char* ring;
  uint64_t* bars;
  float4* face;
  __device__ __forceinline__ BulkSmem(unsigned char* smem, int wib, int nwarps, int R) {
    using SL = Slot<BF>;
    ring = smem + (size_t)wib * R * SL::BYTES;
    unsigned char* bar_base = smem + (size_t)nwarps * R * SL::BYTES;
    bars = reinterpret_cast<uint64_t*>(bar_base) + wib * R;
    face = reinterpret_cast<float4*>(bar_base + (size_t)nwarps * R * sizeof(uint64_t) +
                                     (size_t)wib * face_ring_rows(K) * FACE_SLOT_BYTES);
  }
};

template <int K, bool BF, bool RE>
__global__ void __launch_bounds__(256) stream_bulk_kernel(const StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int item = blockIdx.x * nwarps + wib;
  if (item >= a.n_items) return;  // warp-uniform; no block-level barrier is used
  const BulkSmem<K, BF> sm(smem, wib, nwarps, a.stages);
  if (a.depth == K)
    bulk_item<K, BF, true, false, RE, true>(a, item, threadIdx.x & 31, sm.ring, sm.bars, sm.face,
                                            &g_stream_status);
  else
    bulk_item<K, BF, false, false, RE, true>(a, item, threadIdx.x & 31, sm.ring, sm.bars, sm.face,
                                             &g_stream_status);
}

// The same pass, also storing the rows of every intermediate level, so that a
// pass of depth d yields d consecutive states (the adjoint's segment
// recompute).  FP32 storage, TMA row ring.
template <int K>
__global__ void __launch_bounds__(256) stream_bulk_levels_kernel(const StreamArgs a, const LevelOut lv) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int wib = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int item = blockIdx.x * nwarps + wib;
  if (item >= a.n_items) return;  // warp-uniform; no block-level barrier is used
  const BulkSmem<K, false> sm(smem, wib, nwarps, a.stages);
  if (a.depth == K)
    bulk_item<K, false, true, true>(a, item, threadIdx.x & 31, sm.ring, sm.bars, sm.face, &g_stream_status, &lv);
  else
    bulk_item<K, false, false, true>(a, item, threadIdx.x & 31, sm.ring, sm.bars, sm.face, &g_stream_status, &lv);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
namespace {
// Per (variant, storage, depth) kernel: devices (bit per ordinal < 32) on which
// the shared-memory opt-in was set.  Storage: 0 FP32, 1 BF16-Kahan rounded
// every level, 2 BF16-Kahan rounded where stored.  Internal linkage: one per translation
// unit and library (a function-local static of a template would be merged
// across every shared object loaded in the process).
unsigned g_smem_attr_done[2][3][9];
unsigned g_smem_attr_levels_done;  // the level-storing kernel (depth 4, FP32)

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per device.
inline cudaError_t ensure_smem_optin(const void* fn, unsigned& done, size_t shm) {
  if (shm <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (done & (1u << dev))) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  const int dyn_max = optin - (int)fa.sharedSizeBytes;  // static + dynamic <= opt-in limit
  if (shm > (size_t)dyn_max) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  if (e == cudaSuccess && dev < 32) done |= 1u << dev;
  return e;
}
}  // namespace

template <int K, bool BF, bool RE>
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
  const size_t face = (size_t)wpb * face_ring_rows(K) * FACE_SLOT_BYTES;
  const bool bulk = p.variant == 1;
  const size_t shm = face + (bulk ? bulk_smem_bytes(BF, wpb, p.stages) : 0);
  if (p.store_levels) {  // built for depth 4, FP32, TMA row ring only
    if constexpr (K == 4 && !BF) {
      if (!bulk) return cudaErrorInvalidValue;
      cudaError_t e = ensure_smem_optin((const void*)stream_bulk_levels_kernel<4>, g_smem_attr_levels_done, shm);
      if (e != cudaSuccess) return e;
      LevelOut lv;
      for (int j = 0; j < 7; ++j) lv.p[j] = p.levels[j];
      (void)cudaGetLastError();
      stream_bulk_levels_kernel<4><<<(unsigned)blocks, 32 * wpb, shm, s>>>(a, lv);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  cudaError_t e = ensure_smem_optin(bulk ? (const void*)stream_bulk_kernel<K, BF, RE>
                                         : (const void*)stream_kernel<K, BF, RE>,
                                    g_smem_attr_done[bulk ? 1 : 0][BF ? (RE ? 1 : 2) : 0][K], shm);
  if (e != cudaSuccess) return e;
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  if (bulk)
    stream_bulk_kernel<K, BF, RE><<<(unsigned)blocks, 32 * wpb, shm, s>>>(a);
  else
    stream_kernel<K, BF, RE><<<(unsigned)blocks, 32 * wpb, shm, s>>>(a);
  return cudaGetLastError();
}

template <bool BF, bool RE = true>
cudaError_t launch_stream_any(const StreamPass& p, int k, cudaStream_t s) {
  switch (k) {
    case 1: return launch_stream_k<1, BF, RE>(p, s);
    case 2: return launch_stream_k<2, BF, RE>(p, s);
    case 3: return launch_stream_k<3, BF, RE>(p, s);
    case 4: return launch_stream_k<4, BF, RE>(p, s);
    case 5: return launch_stream_k<5, BF, RE>(p, s);
    case 6: return launch_stream_k<6, BF, RE>(p, s);
    case 7: return launch_stream_k<7, BF, RE>(p, s);
    case 8: return launch_stream_k<8, BF, RE>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

// Read and clear this translation unit's device status word.
static inline cudaError_t read_stream_status(int* out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_stream_status, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_stream_status, &zero, sizeof(int));
}

}  // namespace cpb
