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
#include "k_stream.cuh"

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
  const size_t n = (size_t)nx * ny;
  const size_t c = CPB_CHK((size_t)j * nx + i, 1, n);
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
      const size_t g = CPB_CHK((size_t)jj * nx + ii, 1, n);
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
  const size_t n = (size_t)nx * ny;
  auto load_row = [&](int r) -> Row3 {
    Row3 R{z4, z4, z4};
    if (periodic || (r >= 0 && r < ny)) {
      const size_t g = CPB_CHK((size_t)(periodic ? wrap_index(r, ny) : r) * nx + xv, 4, n);
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
    return (r < y1 && x0 < nx) ? *reinterpret_cast<const float4*>(gk + CPB_CHK((size_t)r * nx + x0, 4, n)) : z4;
  };
  auto load_halo = [&](int r, float& hl, float& hu, float& hk) {
    hl = hu = hk = 0.f;
    if ((lane == 0 || lane == 31) && hin && r < y1) {
      const size_t g = CPB_CHK((size_t)r * nx + xhc, 1, n);
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
      const size_t c0 = CPB_CHK((size_t)j * nx + x0, 4, n);
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

// ---------------------------------------------------------------------------
// Temporally blocked adjoint: D steps per pass
// ---------------------------------------------------------------------------
// One pass advances lambda D steps backwards, lambda_{m} -> lambda_{m-D}, and
// adds the D steps' kappa-gradient terms, so lambda, kappa and the gradient
// cross memory once per D steps instead of once per step (each level still
// reads its own forward state u_{m-t}).  The lambda recursion is the forward
// update with no source, so it runs on the streaming kernel's register
// pipeline (Pipe, flux form): a warp owns a 128-column strip and a chunk of
// rows, level t makes row rho = r_in - t of lambda_{m-t} from level t-1's rows.
// Next to it, level t forms the gradient terms of the same row from the
// level's input rows (lambda_{m-t+1}) and the rows rho, rho + 1 of u_{m-t}:
// the face product hdt (u_f - u_c)(lambda_c - lambda_f) of an interior face
// is the same number seen from either cell (both factors change sign
// exactly), so each east and north face is formed once, the west face comes
// from the lane to the west (shuffle) and the south face is the north face of
// the row below at the same level, carried in registers; a Dirichlet boundary
// face takes dt (0 - u_c) lambda_c.  A row's accumulator is loaded from the
// gradient buffer when the row enters level 1 and receives the terms of
// levels 1, 2, .. D in that order, the order in which the one-step kernel
// adds them: the pass gives the one-step kernels' bits, whatever D.
// nx % 4 == 0 and 16-byte aligned fields; D = 1..4 (instantiated).
constexpr int ADJ_TB_WARPS = 1;
constexpr int ADJ_STAGES = 4;  // rows in the per-lane copy ring (ADJ_STAGES - 1 ahead)

struct AdjPassArgs {
  const float* lam;
  float* lam_out;
  const float* k;
  float* gk;
  const float* u[4];  // u[t - 1]: the forward state of level t (u_{m-t})
  int nx, ny;
  float dt, hdt;
  int bc, chunk_rows, n_strips, n_items;
};

__device__ __forceinline__ float4 face_term(float hdt, float4 uf, float4 uc, float4 lc, float4 lf) {
  return make_float4(hdt * (uf.x - uc.x) * (lc.x - lf.x), hdt * (uf.y - uc.y) * (lc.y - lf.y),
                     hdt * (uf.z - uc.z) * (lc.z - lf.z), hdt * (uf.w - uc.w) * (lc.w - lf.w));
}

// The same face terms on packed pairs, for operands that sit in the same
// columns (north faces): each component rounds exactly as face_term's.
__device__ __forceinline__ float4 face_term2(float hdt, float4 uf, float4 uc, float4 lc, float4 lf) {
  const float2 h = make_float2(hdt, hdt);
  return cat4(mul2(mul2(h, sub2(lo2(uf), lo2(uc))), sub2(lo2(lc), lo2(lf))),
              mul2(mul2(h, sub2(hi2(uf), hi2(uc))), sub2(hi2(lc), hi2(lf))));
}

// Dirichlet boundary-face term dt (0 - u_c) lambda_c, on packed pairs.
__device__ __forceinline__ float4 boundary_term2(float dt, float4 uc, float4 lc) {
  const float2 d = make_float2(dt, dt), z = make_float2(0.0f, 0.0f);
  return cat4(mul2(mul2(d, sub2(z, lo2(uc))), lo2(lc)), mul2(mul2(d, sub2(z, hi2(uc))), hi2(lc)));
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return cat4(add2(lo2(a), lo2(b)), add2(hi2(a), hi2(b)));
}

template <int D>
__global__ void __launch_bounds__(32 * ADJ_TB_WARPS) adjoint_pass(const AdjPassArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int HALO = (D + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * ADJ_TB_WARPS + wib;
  if (item >= a.n_items) return;  // warp-uniform; no block-level barrier is used
  float4* face = reinterpret_cast<float4*>(smem + (size_t)wib * face_ring_rows(D) * FACE_SLOT_BYTES);
  const int nx = a.nx, ny = a.ny;
  const bool periodic = a.bc == BC_PERIODIC;
  const int strip = item % a.n_strips, chunk = item / a.n_strips;
  const LaneCols lc = lane_cols(strip * OW - HALO + 4 * lane, nx, periodic);
  const int y0 = chunk * a.chunk_rows, y1 = min(y0 + a.chunk_rows, ny);
  const bool lane_out = lane >= HALO / 4 && lane < (HALO + OW) / 4 && lc.xs < nx;
  // Dirichlet boundary faces of this lane's cells (west of x = 0, east of x = nx - 1)
  const bool bW0 = !periodic && lc.xs == 0;
  bool bE[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) bE[e] = !periodic && lc.xs + e == nx - 1;
  const float4 z4 = f4(0.0f);

  // Input rows reach shared memory through a per-lane ring of ADJ_STAGES
  // slots filled by asynchronous 16-byte copies, ADJ_STAGES - 1 rows ahead
  // (each lane copies and reads only its own 16 bytes of each field, so the
  // lane's own wait orders them).  Slot of input row r: fields lambda row r,
  // kappa row r, gradient row r - 1, and u_{m-t} row r - t + 1 for t = 1..D.
  // Ghost rows (Dirichlet): zero-filled copies; kappa from the clamped row.
  float4* ring = reinterpret_cast<float4*>(smem + (size_t)ADJ_TB_WARPS * face_ring_rows(D) * FACE_SLOT_BYTES) +
                 (size_t)wib * ADJ_STAGES * (D + 3) * 32 + lane;
  auto row_of = [&](int r, bool& in) -> size_t {
    in = periodic || (r >= 0 && r < ny);
    const int rr = periodic ? wrap_near(r, ny) : clamp_index(r, ny);
    return CPB_CHK((size_t)rr * nx + lc.xv, 4, (size_t)nx * ny);
  };
  auto issue = [&](int r, int slot) {
    float4* d = ring + (size_t)slot * (D + 3) * 32;
    bool in;
    size_t g = row_of(r, in);
    cp_async16(d, a.lam + g, (in && lc.cin4) ? 16 : 0);
    cp_async16(d + 32, a.k + g, 16);
    g = row_of(r - 1, in);
    cp_async16(d + 64, a.gk + g, (in && lc.cin4) ? 16 : 0);
#pragma unroll
    for (int t = 1; t <= D; ++t) {
      g = row_of(r - t + 1, in);
      cp_async16(d + 32 * (2 + t), a.u[t - 1] + g, (in && lc.cin4) ? 16 : 0);
    }
  };

  Pipe<D, false> pipe;
  pipe.init(face, lane);
  float4 Urow[D];  // level t: row rho of u_{m-t} (carried from the previous iteration)
  float4 PN[D];    // level t: north-face terms of the previous row (its south faces)
  float4 A[D];     // A[t]: gradient accumulator of the row at level t (1 .. D-1)
#pragma unroll
  for (int t = 0; t < D; ++t) Urow[t] = PN[t] = A[t] = z4;
  const int r_first = y0 - D, r_end = y1 + D;
#pragma unroll
  for (int j = 0; j < ADJ_STAGES - 1; ++j) {
    if (r_first + j < r_end) issue(r_first + j, j);
    cp_async_commit();
  }
  auto body = [&](auto parity, int r_in) {
    constexpr int P = decltype(parity)::value, Q = 1 - P;
    const int i = r_in - r_first;
    // refill the slot read last iteration, then wait for this row's copies
    if (r_in + ADJ_STAGES - 1 < r_end) issue(r_in + ADJ_STAGES - 1, (i + ADJ_STAGES - 1) % ADJ_STAGES);
    cp_async_commit();
    cp_async_wait<ADJ_STAGES - 1>();
    const float4* sl = ring + (size_t)(i % ADJ_STAGES) * (D + 3) * 32;
    const float4 ln = sl[0], g_init = sl[64];
    float4 kn = sl[32];
    if (!periodic) {  // Dirichlet ghost lanes take kappa of the edge cell
      if (lc.kb == 1) kn = f4(kn.x);
      if (lc.kb == 2) kn = f4(kn.w);
    }
    float4 un[D];
#pragma unroll
    for (int t = 0; t < D; ++t) un[t] = sl[32 * (3 + t)];
    float4 out;
    uint4 packed;
    pipe.template step<P, true>(r_in, D, ny, periodic, lc, a.dt, a.hdt, ln, kn, z4, out, packed);
    // gradient terms of level t at row rho = r_in - t, from the level's input
    // rows (pipe.U[t-1][Q]: row rho, pipe.U[t-1][P]: row rho + 1)
    float4 c[D];
#pragma unroll
    for (int t = 1; t <= D; ++t) {
      const int rho = r_in - t;
      const float4 lC = pipe.U[t - 1][Q], lN = pipe.U[t - 1][P];
      const float4 uC = Urow[t - 1], uN = un[t - 1];
      Urow[t - 1] = uN;
      const float uE3 = __shfl_down_sync(CPB_FULL, uC.x, 1), lE3 = __shfl_down_sync(CPB_FULL, lC.x, 1);
      float4 pE = face_term(a.hdt, make_float4(uC.y, uC.z, uC.w, uE3), uC, lC, make_float4(lC.y, lC.z, lC.w, lE3));
      // Dirichlet boundary faces take dt (0 - u_c) lambda_c instead (selected
      // without branches, so the levels stay one straight-line block)
      const float4 bt = boundary_term2(a.dt, uC, lC);
      pE.x = bE[0] ? bt.x : pE.x;
      pE.y = bE[1] ? bt.y : pE.y;
      pE.z = bE[2] ? bt.z : pE.z;
      pE.w = bE[3] ? bt.w : pE.w;
      // west faces: the east terms of the cells to the west (the lane's first
      // cell: the last of the lane to the west)
      const float pW0 = __shfl_up_sync(CPB_FULL, pE.w, 1);
      const float4 pW = make_float4(bW0 ? bt.x : pW0, pE.x, pE.y, pE.z);
      // north faces: same columns, so on packed pairs
      float4 pN = face_term2(a.hdt, uN, uC, lC, lN);
      if (!periodic && rho + 1 >= ny) pN = bt;
      float4 pS = PN[t - 1];
      if (!periodic && rho - 1 < 0) pS = bt;
      PN[t - 1] = pN;
      const float4 we = make_float4(pW.x + pE.x, pW.y + pE.y, pW.z + pE.z, pW.w + pE.w);
      c[t - 1] = add4(we, add4(pS, pN));
    }
    // accumulate: the row at level D leaves, the others move up one level
    float4 g_out;
    if constexpr (D == 1) {
      g_out = add4(g_init, c[0]);
    } else {
      g_out = add4(A[D - 2], c[D - 1]);
#pragma unroll
      for (int t = D - 2; t >= 1; --t) A[t] = add4(A[t - 1], c[t]);
      A[0] = add4(g_init, c[0]);
    }
    const int ro = r_in - D;
    if (ro >= y0 && lane_out) {
      const size_t g = CPB_CHK((size_t)ro * nx + lc.xs, 4, (size_t)nx * ny);
      *reinterpret_cast<float4*>(a.lam_out + g) = out;
      *reinterpret_cast<float4*>(a.gk + g) = g_out;
    }
  };
  int r_in = r_first;
  for (; r_in + 1 < r_end; r_in += 2) {
    body(Int<0>{}, r_in);
    body(Int<1>{}, r_in + 1);
  }
  if (r_in < r_end) body(Int<0>{}, r_in);
  cp_async_wait<0>();  // no copy may target this CTA's shared memory after it exits
}

// Shared-memory opt-in above 48 KB, once per depth and device (ordinal < 32).
unsigned g_adj_attr_done[5];
cudaError_t ensure_smem_optin_adj(int depth, size_t shm) {
  const void* fn = depth == 1 ? (const void*)adjoint_pass<1>
                   : depth == 2 ? (const void*)adjoint_pass<2>
                   : depth == 3 ? (const void*)adjoint_pass<3>
                                : (const void*)adjoint_pass<4>;
  return ensure_smem_optin(fn, g_adj_attr_done[depth], shm);
}

size_t adjoint_pass_smem(int depth) {
  return (size_t)ADJ_TB_WARPS * (face_ring_rows(depth) * FACE_SLOT_BYTES + ADJ_STAGES * (depth + 3) * 32 * 16);
}

}  // namespace

cudaError_t launch_adjoint_pass(const float* lam, float* lam_out, const float* const* u, int depth, const float* k,
                                float* gk, int nx, int ny, float dt, int bc, int chunk_rows, cudaStream_t s) {
  if (depth < 1 || depth > 4) return cudaErrorInvalidValue;
  if (chunk_rows < 1) {
    // chunks sized so the items come to about one wave of resident warps
    // (at least 16 rows: each chunk recomputes 2 x 4 halo rows)
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_pass<4>, 32 * ADJ_TB_WARPS,
                                                        adjoint_pass_smem(4));
    if (e != cudaSuccess) return e;
    const long long warps = std::max(1LL, (long long)sms * std::max(1, per_sm) * ADJ_TB_WARPS);
    const long long strips = (nx + strip_out_width(4) - 1) / strip_out_width(4);
    chunk_rows = (int)std::max(16LL, std::min((strips * ny + warps - 1) / warps, 1024LL));
  }
  AdjPassArgs a;
  a.lam = lam;
  a.lam_out = lam_out;
  a.k = k;
  a.gk = gk;
  for (int t = 0; t < 4; ++t) a.u[t] = t < depth ? u[t] : nullptr;
  a.nx = nx;
  a.ny = ny;
  a.dt = dt;
  a.hdt = 0.5f * dt;
  a.bc = bc;
  a.chunk_rows = chunk_rows;
  const int ow = strip_out_width(4);  // HALO = 4 for every depth 1..4
  a.n_strips = (nx + ow - 1) / ow;
  const long long items = (long long)a.n_strips * ((ny + chunk_rows - 1) / chunk_rows);
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  a.n_items = (int)items;
  const unsigned blocks = (unsigned)((items + ADJ_TB_WARPS - 1) / ADJ_TB_WARPS);
  const size_t shm = adjoint_pass_smem(depth);
  cudaError_t e = ensure_smem_optin_adj(depth, shm);
  if (e != cudaSuccess) return e;
  (void)cudaGetLastError();
  switch (depth) {
    case 1: adjoint_pass<1><<<blocks, 32 * ADJ_TB_WARPS, shm, s>>>(a); break;
    case 2: adjoint_pass<2><<<blocks, 32 * ADJ_TB_WARPS, shm, s>>>(a); break;
    case 3: adjoint_pass<3><<<blocks, 32 * ADJ_TB_WARPS, shm, s>>>(a); break;
    default: adjoint_pass<4><<<blocks, 32 * ADJ_TB_WARPS, shm, s>>>(a); break;
  }
  return cudaGetLastError();
}

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

cudaError_t read_bounds_adjoint(int* out) { return read_bounds_word(out); }

}  // namespace cpb
