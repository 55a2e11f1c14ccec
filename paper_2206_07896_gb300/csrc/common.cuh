// Device-side building blocks shared by the stencil kernels of libcpb.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cpb.h"

namespace cpb {

enum { BC_DIRICHLET = 0, BC_PERIODIC = 1 };

// One step of the canonical flux-form update for one cell, from precomputed
// face conductivity sums (kc + kn) and the precomputed source increment
// dt * s.  Both are time-invariant and their values are identical to forming
// them inline, so the rounding sequence is exactly
//   c + (hdt * (((kc+kW)*(uW-c) + (kc+kE)*(uE-c)) + ((kc+kS)*(uS-c) + (kc+kN)*(uN-c))) + dt*s).
__device__ __forceinline__ float cell_update(float c, float uW, float uE, float uS, float uN,
                                             float fkW, float fkE, float fkS, float fkN, float dts,
                                             float hdt) {
  float fW = fkW * (uW - c);
  float fE = fkE * (uE - c);
  float fS = fkS * (uS - c);
  float fN = fkN * (uN - c);
  float acc = (fW + fE) + (fS + fN);
  return c + (hdt * acc + dts);
}

// Packed FP32 pair arithmetic (sm_100+): each component is rounded exactly as
// the scalar operation.  b - a is formed as fma(a, -1, b), which is exact in
// the product and rounds once, i.e. the same bits as the subtraction.
__device__ __forceinline__ float2 sub2(float2 b, float2 a) {
  return __ffma2_rn(a, make_float2(-1.0f, -1.0f), b);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// In the build that reproduces the canonical order bit for bit, every packed
// product is made opaque before it is used, so the compiler cannot fuse it
// into a following addition (it does so for packed pairs even under
// --fmad=false); the default build lets it fuse.
__device__ __forceinline__ float2 round_product(float2 p) {
#ifdef CPB_EXACT_ARITH
  unsigned long long b = (unsigned long long)__float_as_uint(p.x) |
                         ((unsigned long long)__float_as_uint(p.y) << 32);
  asm volatile("" : "+l"(b));
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
#else
  return p;
#endif
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return round_product(__fmul2_rn(a, b)); }
// h * acc + ds: fused in the default build; two roundings (product, then
// sum) in the exact build.
__device__ __forceinline__ float2 madd2(float2 h, float2 acc, float2 ds) {
#ifdef CPB_EXACT_ARITH
  return __fadd2_rn(mul2(h, acc), ds);
#else
  return __ffma2_rn(h, acc, ds);
#endif
}

__device__ __forceinline__ int wrap_index(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ int clamp_index(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// BF16-Kahan state word: bits 0..15 hi, bits 16..31 cmp.
__device__ __forceinline__ float bf16_bits_to_f32(uint32_t h16) {
  return __uint_as_float(h16 << 16);
}

__device__ __forceinline__ float kahan_value(uint32_t w) {
  return bf16_bits_to_f32(w & 0xffffu) - bf16_bits_to_f32(w >> 16);
}

__device__ __forceinline__ uint32_t f32_to_bf16_bits(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Round an FP32 step result into BF16-Kahan storage; returns the packed word
// and (through eff) the effective value the stored state represents.
__device__ __forceinline__ uint32_t kahan_round(float v, float& eff) {
  uint32_t hi = f32_to_bf16_bits(v);
  float hif = bf16_bits_to_f32(hi);
  uint32_t cm = f32_to_bf16_bits(hif - v);
  eff = hif - bf16_bits_to_f32(cm);
  return hi | (cm << 16);
}

// Bounds-checked build (CPB_BOUNDS_CHECK, the library's third build): every
// element range [i, i + count) a kernel reads from or writes to a field of n
// elements passes through CPB_CHK(i, count, n).  Outside the field it
// records the source line in this translation unit's g_bounds_line (the
// first one wins) and returns a clamped index, so the access stays inside the
// field; the other builds return i unchanged and compile no check.
#ifdef CPB_BOUNDS_CHECK
static __device__ int g_bounds_line;
#endif
__device__ __forceinline__ size_t chk_range(size_t i, size_t count, size_t n, int line) {
#ifdef CPB_BOUNDS_CHECK
  if (i > n || count > n - i) {
    atomicCAS(&g_bounds_line, 0, line);
    return n >= count ? n - count : 0;
  }
#endif
  (void)count;
  (void)n;
  (void)line;
  return i;
}
#define CPB_CHK(i, count, n) ::cpb::chk_range((size_t)(i), (size_t)(count), (size_t)(n), __LINE__)

// Host side: read and clear this translation unit's g_bounds_line (0 in the
// builds without checks).
static inline cudaError_t read_bounds_word(int* out) {
#ifdef CPB_BOUNDS_CHECK
  const int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_line, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_bounds_line, &zero, sizeof(int));
#else
  *out = 0;
  return cudaSuccess;
#endif
}

// Per-thread asynchronous copies global -> shared (cp.async): 16 or 4 bytes,
// src_bytes = 0 fills the destination with zeros (the source address must
// still be a valid one).  One commit group per call of cp_async_commit;
// cp_async_wait<N> returns once at most N of this thread's groups are pending.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace cpb
