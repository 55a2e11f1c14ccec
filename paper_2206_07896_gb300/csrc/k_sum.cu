// FP64 heat sum and BF16 conversion kernels.
//
// Heat sum: sum over all cells of the cell value in FP64 (FP32 storage: the
// float widened; BF16-Kahan: (double)hi - (double)cmp, which is exact).  Two
// passes with a fixed reduction order (grid-stride per thread, warp shuffle
// tree, block tree, then one block over the per-block partials), so the same
// input gives the same bits on the same device.  This is the only FP64
// arithmetic on the GPU path.

#include "common.cuh"
#include "internal.h"

namespace cpb {
namespace {

constexpr int SUM_THREADS = 256;
constexpr int SUM_MAX_BLOCKS = 1024;

__device__ __forceinline__ double cell_value(const uint32_t* u, long long i) {
  uint32_t w = u[i];
  return (double)bf16_bits_to_f32(w & 0xffffu) - (double)bf16_bits_to_f32(w >> 16);
}

__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double part[SUM_THREADS / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  v = 0.0;
  if (warp == 0) {
    v = lane < SUM_THREADS / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  }
  return v;
}

// Pass 1, FP32 storage: 128-bit loads over the 16-byte-aligned body, scalar
// loads for the head/tail.
__global__ void __launch_bounds__(SUM_THREADS) heat_partial_f32(const float* __restrict__ u,
                                                                long long n, long long head,
                                                                double* __restrict__ partials) {
  double acc = 0.0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long nvec = (n - head) / 4;
  for (long long i = tid; i < nvec; i += nthreads) {
    const size_t j = CPB_CHK(head + 4 * i, 4, n);
    float4 v = __ldcs(reinterpret_cast<const float4*>(u + j));
    acc += (double)v.x;
    acc += (double)v.y;
    acc += (double)v.z;
    acc += (double)v.w;
  }
  for (long long i = tid; i < head; i += nthreads) acc += (double)u[CPB_CHK(i, 1, n)];
  for (long long i = head + 4 * nvec + tid; i < n; i += nthreads) acc += (double)u[CPB_CHK(i, 1, n)];
  acc = block_reduce(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(SUM_THREADS) heat_partial_bf16k(const uint32_t* __restrict__ u,
                                                                  long long n,
                                                                  double* __restrict__ partials) {
  double acc = 0.0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < n; i += nthreads) acc += cell_value(u, CPB_CHK(i, 1, n));
  acc = block_reduce(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(SUM_THREADS) heat_final(const double* __restrict__ partials,
                                                          int nblocks, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[i];
  acc = block_reduce(acc);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void bf16_round_kernel(const float* __restrict__ x, uint16_t* __restrict__ out,
                                  long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (uint16_t)f32_to_bf16_bits(x[i]);
}

__global__ void bf16k_pack_kernel(const float* __restrict__ u, uint32_t* __restrict__ st,
                                  long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float eff;
    st[i] = kahan_round(u[i], eff);
  }
}

__global__ void bf16k_unpack_kernel(const uint32_t* __restrict__ st, float* __restrict__ u,
                                    long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = kahan_value(st[i]);
}

int elementwise_blocks(long long n) {
  (void)cudaGetLastError();  // called right before each launch: drop a stale non-sticky error
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

int heat_sum_blocks(long long n) {
  long long b = (n + SUM_THREADS * 16 - 1) / (SUM_THREADS * 16);
  return (int)(b < 1 ? 1 : (b > SUM_MAX_BLOCKS ? SUM_MAX_BLOCKS : b));
}

cudaError_t launch_heat_sum(const void* u, long long n, int dtype, double* d_out, double* partials,
                            int nblocks, cudaStream_t s) {
  (void)cudaGetLastError();  // drop a stale non-sticky error so the checks below are these launches'
  if (dtype == CPB_F32) {
    const float* f = static_cast<const float*>(u);
    long long mis = (long long)(reinterpret_cast<uintptr_t>(f) & 15) / 4;
    long long head = mis ? 4 - mis : 0;
    if (head > n) head = n;
    heat_partial_f32<<<nblocks, SUM_THREADS, 0, s>>>(f, n, head, partials);
  } else {
    heat_partial_bf16k<<<nblocks, SUM_THREADS, 0, s>>>(static_cast<const uint32_t*>(u), n, partials);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  heat_final<<<1, SUM_THREADS, 0, s>>>(partials, nblocks, d_out);
  return cudaGetLastError();
}

cudaError_t launch_bf16_round(const float* x, uint16_t* out, long long n, cudaStream_t s) {
  bf16_round_kernel<<<elementwise_blocks(n), 256, 0, s>>>(x, out, n);
  return cudaGetLastError();
}

cudaError_t launch_bf16k_pack(const float* u, uint32_t* st, long long n, cudaStream_t s) {
  bf16k_pack_kernel<<<elementwise_blocks(n), 256, 0, s>>>(u, st, n);
  return cudaGetLastError();
}

cudaError_t launch_bf16k_unpack(const uint32_t* st, float* u, long long n, cudaStream_t s) {
  bf16k_unpack_kernel<<<elementwise_blocks(n), 256, 0, s>>>(st, u, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Heat sum that allocates nothing (cpb_heat_sum_noalloc)
// ---------------------------------------------------------------------------
// For callers that cannot allocate device memory: the per-block partial sums
// of the two-pass reduction live in a file-scope device array instead of a
// caller workspace.  Every GPU that loads the library holds this array (32 KB)
// until the process exits.  One partial per block of NOALLOC_CELLS_PER_BLOCK
// cells, so grids of up to NOALLOC_MAX_PARTIALS * NOALLOC_CELLS_PER_BLOCK
// = 2^26 cells are accepted; larger grids are rejected before any launch.
// All calls share the array and it keeps the previous call's contents; every
// partial that is read is first written by the same call, so nothing needs
// clearing.  Calls whose executions overlap on the GPU (different streams,
// no ordering between them) race on the array.
namespace {
constexpr int NOALLOC_MAX_PARTIALS = 4096;
constexpr long long NOALLOC_CELLS_PER_BLOCK = 16384;
}  // namespace

static __device__ __align__(256) double g_heat_sum_scratch[NOALLOC_MAX_PARTIALS];

namespace {
// The host-side name of a __device__ array is not a device address: ask the
// runtime for it, with the device current, on every call.  The lookup
// allocates nothing and does not synchronise; asking each time (instead of
// caching per device) keeps the address right after a cudaDeviceReset, which
// reloads the module at a new address.
cudaError_t noalloc_scratch(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_heat_sum_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}
}  // namespace

long long heat_sum_noalloc_max_cells() { return NOALLOC_MAX_PARTIALS * NOALLOC_CELLS_PER_BLOCK; }

cudaError_t launch_heat_sum_noalloc(const void* u, long long n, int dtype, double* d_out,
                                    cudaStream_t s) {
  double* partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) return e;
  const int nblocks = (int)((n + NOALLOC_CELLS_PER_BLOCK - 1) / NOALLOC_CELLS_PER_BLOCK);
  return launch_heat_sum(u, n, dtype, d_out, partials, nblocks, s);
}

cudaError_t read_bounds_sum(int* out) { return read_bounds_word(out); }

}  // namespace cpb
