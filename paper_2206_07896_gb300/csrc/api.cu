// libcpb C ABI: validation, pass scheduling, tuning cache, autotuner, heat
// sum, BF16 conversions, host end-to-end call and CUDA-graph capture.
//
// A launch call is the host half of the paper's launch model (Sec. IV, "Push
// task queue"): it checks the arguments, decides the sequence of kernel
// passes, enqueues them on the caller's stream and returns without waiting.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <unistd.h>

#include "common.cuh"
#include "internal.h"

using namespace cpb;

namespace {

thread_local std::string g_last_error;

cpb_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CPB_SUCCESS;
  g_last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources)
    return CPB_ERR_LAUNCH;
  return CPB_ERR_CUDA;
}

#define CPB_TRY(expr)                            \
  do {                                           \
    cpb_status _st = from_cuda(expr);            \
    if (_st != CPB_SUCCESS) return _st;          \
  } while (0)

bool aligned(const void* p, size_t a) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) % a) == 0; }

size_t u_bytes(cpb_dtype) { return 4; }                    // f32 or (hi, cmp) word
size_t ks_bytes(cpb_dtype d) { return d == CPB_F32 ? 4 : 2; }  // kappa / source element
bool dtype_ok(int d) { return d == CPB_F32 || d == CPB_BF16_KAHAN || d == CPB_BF16_KAHAN_BLOCK; }

bool overlap(const void* a, const void* b, size_t n) {
  if (!a || !b) return false;
  uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + n && y < x + n;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return sms > 0 ? sms : 148;
}

// ---------------------------------------------------------------------------
// Tuning cache
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, cpb_tuning> g_tune;

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

bool tuning_valid(const cpb_tuning& t) {
  if (t.k < 1 || t.k > 8 || t.chunk_rows < 1 || t.warps_per_block < 1 || t.warps_per_block > 8)
    return false;
  if (t.variant == 0) return stream_smem_bytes(true, t.k, t.warps_per_block, 0, 0) <= 227 * 1024;
  return t.variant == 1 && pow2(t.stages) && t.stages >= 2 && t.stages <= 16 &&
         stream_smem_bytes(false, t.k, t.warps_per_block, 1, t.stages) <= 227 * 1024;
}

// Variant 1 (TMA bulk-copy ring) needs aligned rows; otherwise variant 0 runs.
bool bulk_eligible(int nx, cpb_dtype d, bool vec, const void* kappa, const void* src) {
  const bool bf = d != CPB_F32;
  return vec && nx % bulk_align_cells(bf) == 0 && nx >= bulk_slot_cells(bf) && aligned(kappa, 16) &&
         aligned(src, 16);
}

// Built-in default (the autotuner's winner on GB300 at 8192^2 and 16384^2):
// depth 4, TMA ring of 2 stages, one warp per CTA, and chunks sized so the
// grid yields about one resident wave of warp items (16 per SM).
cpb_tuning default_tuning(int nx, int ny, cpb_dtype) {
  cpb_tuning t;
  t.k = 4;
  t.warps_per_block = 1;
  t.variant = 1;
  t.stages = 2;
  const long long strips = (nx + strip_out_width(t.k) - 1) / strip_out_width(t.k);
  const long long target = (long long)device_sm_count() * 16;
  long long rows = (strips * ny + target - 1) / target;
  t.chunk_rows = (int)std::max(16LL, std::min(rows, 1024LL));
  return t;
}

// Debug knobs (tests only): mbarrier wait limit and an injected row whose
// copies never complete.
int g_wait_limit = 1 << 20;
int g_inject_on = 0;
int g_inject_row = 0;

cpb_tuning lookup_tuning(int nx, int ny, cpb_dtype d, cpb_boundary bc) {
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune.find(TuneKey(nx, ny, (int)d, (int)bc));
  if (it != g_tune.end()) return it->second;
  return default_tuning(nx, ny, d);
}

// ---------------------------------------------------------------------------
// Pass schedule
// ---------------------------------------------------------------------------
// Depths of the passes for `steps` steps at depth k.  Without scratch the
// passes alternate u_in -> u_out -> u_in ..., so the result lands in u_out
// only for an odd number of passes: an even count is made odd by splitting a
// pass of depth >= 2 in two; if every pass has depth 1, the result is copied
// from u_in at the end (*copy_at_end).
std::vector<int> pass_depths(int steps, int k, bool have_scratch, bool* copy_at_end) {
  std::vector<int> d(steps / k, k);
  if (steps % k) d.push_back(steps % k);
  *copy_at_end = false;
  if (!have_scratch && d.size() % 2 == 0 && !d.empty()) {
    int idx = -1;
    for (int i = (int)d.size() - 1; i >= 0; --i)
      if (d[i] >= 2) {
        idx = i;
        break;
      }
    if (idx >= 0) {
      int a = d[idx] - d[idx] / 2, b = d[idx] / 2;
      d[idx] = a;
      d.insert(d.begin() + idx + 1, b);
    } else {
      *copy_at_end = true;
    }
  }
  return d;
}

struct Fields {
  void* u_in;
  void* u_out;
  const void* kappa;
  const void* src;
  void* scratch;
};

cpb_status check_common(const Fields& f, int nx, int ny, int steps, float dt, cpb_boundary bc,
                        cpb_dtype dtype) {
  if (nx < 1 || ny < 1 || steps < 0) return CPB_ERR_INVALID_VALUE;
  if (!(dt > 0.0f) || !std::isfinite(dt)) return CPB_ERR_INVALID_VALUE;
  if (bc != CPB_DIRICHLET0 && bc != CPB_PERIODIC) return CPB_ERR_INVALID_VALUE;
  if (!dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  if (!f.u_in || !f.u_out || !f.kappa) return CPB_ERR_INVALID_VALUE;
  const size_t n = (size_t)nx * (size_t)ny;
  if (n > (size_t)1 << 40) return CPB_ERR_INVALID_VALUE;
  const size_t ub = n * u_bytes(dtype);
  if (overlap(f.u_in, f.u_out, ub) || overlap(f.u_in, f.scratch, ub) ||
      overlap(f.u_out, f.scratch, ub))
    return CPB_ERR_INVALID_VALUE;
  const size_t ua = u_bytes(dtype), ka = ks_bytes(dtype);
  if (!aligned(f.u_in, ua) || !aligned(f.u_out, ua) || !aligned(f.scratch, ua) ||
      !aligned(f.kappa, ka) || !aligned(f.src, ka))
    return CPB_ERR_INVALID_VALUE;
  return CPB_SUCCESS;
}

cpb_status enqueue_tuned(const Fields& f, int nx, int ny, int steps, float dt, cpb_boundary bc,
                         cpb_dtype dtype, const cpb_tuning& t, cudaStream_t s) {
  const size_t ub = (size_t)nx * ny * u_bytes(dtype);
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(f.u_out, f.u_in, ub, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  const int ow = strip_out_width(t.k);
  const long long items = (long long)((nx + ow - 1) / ow) * ((ny + t.chunk_rows - 1) / t.chunk_rows);
  if ((items + t.warps_per_block - 1) / t.warps_per_block > 0x7fffffffLL) return CPB_ERR_LAUNCH;

  const size_t ka = dtype == CPB_F32 ? 16 : 8;
  StreamPass p;
  p.kappa = f.kappa;
  p.src = f.src;
  p.nx = nx;
  p.ny = ny;
  p.dt = dt;
  p.hdt = 0.5f * dt;
  p.bc = (int)bc;
  p.vec = (nx % 4 == 0) && aligned(f.u_in, 16) && aligned(f.u_out, 16) && aligned(f.scratch, 16) &&
          aligned(f.kappa, ka) && aligned(f.src, ka);
  p.chunk_rows = t.chunk_rows;
  p.warps_per_block = t.warps_per_block;
  p.variant = (t.variant == 1 && bulk_eligible(nx, dtype, p.vec != 0, f.kappa, f.src)) ? 1 : 0;
  p.stages = t.stages;
  p.wait_limit = g_wait_limit;
  p.inject_on = g_inject_on;
  p.inject_row = g_inject_row;

  bool copy_at_end = false;
  std::vector<int> depths = pass_depths(steps, t.k, f.scratch != nullptr, &copy_at_end);
  const int P = (int)depths.size();
  const void* src_buf = f.u_in;
  void* dst = nullptr;
  for (int i = 0; i < P; ++i) {
    if (f.scratch)
      dst = ((P - 1 - i) % 2 == 0) ? f.u_out : f.scratch;
    else if (!copy_at_end)
      dst = ((P - 1 - i) % 2 == 0) ? f.u_out : f.u_in;
    else
      dst = (i % 2 == 0) ? f.u_out : f.u_in;
    p.u_in = src_buf;
    p.u_out = dst;
    p.depth = depths[i];
    cudaError_t e = dtype == CPB_F32          ? launch_stream_f32(p, t.k, s)
                    : dtype == CPB_BF16_KAHAN ? launch_stream_bf16k(p, t.k, s)
                                              : launch_stream_bf16k_block(p, t.k, s);
    CPB_TRY(e);
    src_buf = dst;
  }
  if (copy_at_end) CPB_TRY(cudaMemcpyAsync(f.u_out, f.u_in, ub, cudaMemcpyDeviceToDevice, s));
  return CPB_SUCCESS;
}

cpb_status enqueue_tile(const Fields& f, int nx, int ny, int steps, float dt, cpb_boundary bc,
                        cpb_dim3 grid, cpb_dim3 block, size_t shared_bytes, cudaStream_t s) {
  const long long bx = block.x, by = block.y;
  if (block.z != 1 || bx < 1 || by < 1 || bx * by > 1024) return CPB_ERR_UNSUPPORTED_CONFIG;
  if ((long long)grid.x != (nx + bx - 1) / bx || (long long)grid.y != (ny + by - 1) / by || grid.z != 1)
    return CPB_ERR_INVALID_VALUE;
  const size_t need = 2 * sizeof(float) * (size_t)(bx + 2) * (size_t)(by + 2);
  if (shared_bytes < need) return CPB_ERR_SHARED_MEM;
  const size_t ub = (size_t)nx * ny * sizeof(float);
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(f.u_out, f.u_in, ub, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  bool copy_at_end = false;
  std::vector<int> depths = pass_depths(steps, 1, f.scratch != nullptr, &copy_at_end);
  const int P = (int)depths.size();
  const void* src_buf = f.u_in;
  for (int i = 0; i < P; ++i) {
    void* dst;
    if (f.scratch)
      dst = ((P - 1 - i) % 2 == 0) ? f.u_out : f.scratch;
    else if (!copy_at_end)
      dst = ((P - 1 - i) % 2 == 0) ? f.u_out : f.u_in;
    else
      dst = (i % 2 == 0) ? f.u_out : f.u_in;
    CPB_TRY(launch_tile_f32(static_cast<const float*>(src_buf), static_cast<float*>(dst),
                            static_cast<const float*>(f.kappa), static_cast<const float*>(f.src),
                            nx, ny, dt, (int)bc, dim3(grid.x, grid.y, 1), dim3(block.x, block.y, 1),
                            need, s));
    src_buf = dst;
  }
  if (copy_at_end) CPB_TRY(cudaMemcpyAsync(f.u_out, f.u_in, ub, cudaMemcpyDeviceToDevice, s));
  return CPB_SUCCESS;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

#define CPB_TRY_STATUS(expr)             \
  do {                                   \
    cpb_status _s = (expr);              \
    if (_s != CPB_SUCCESS) return _s;    \
  } while (0)

// Device tag of the tuning file: the given name, or the current device's
// name, with blanks replaced by '_'.
cpb_status device_tag(const char* device, std::string* out) {
  std::string d;
  if (device) {
    d = device;
  } else {
    int dev = 0;
    cudaDeviceProp prop;
    CPB_TRY(cudaGetDevice(&dev));
    CPB_TRY(cudaGetDeviceProperties(&prop, dev));
    d = prop.name;
  }
  if (d.empty()) return CPB_ERR_INVALID_VALUE;
  for (char& c : d)
    if (c == ' ' || c == '\t' || c == '\n') c = '_';
  *out = d;
  return CPB_SUCCESS;
}

}  // namespace

struct cpb_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" {

int cpb_version(void) { return 1; }

const char* cpb_status_string(cpb_status st) {
  switch (st) {
    case CPB_SUCCESS: return "success";
    case CPB_ERR_INVALID_VALUE: return "invalid value";
    case CPB_ERR_UNSUPPORTED_CONFIG: return "unsupported configuration";
    case CPB_ERR_SHARED_MEM: return "shared memory too small";
    case CPB_ERR_LAUNCH: return "launch failed";
    case CPB_ERR_TIMEOUT: return "device wait timed out";
    case CPB_ERR_CUDA: return "CUDA error";
    case CPB_ERR_WORKSPACE: return "workspace missing or too small";
  }
  return "unknown status";
}

const char* cpb_last_error_detail(void) { return g_last_error.c_str(); }

cpb_status cpb_device_info(int* sm_count, int* l2_bytes, int* smem_optin_bytes) {
  int dev = 0;
  CPB_TRY(cudaGetDevice(&dev));
  if (sm_count) CPB_TRY(cudaDeviceGetAttribute(sm_count, cudaDevAttrMultiProcessorCount, dev));
  if (l2_bytes) CPB_TRY(cudaDeviceGetAttribute(l2_bytes, cudaDevAttrL2CacheSize, dev));
  if (smem_optin_bytes)
    CPB_TRY(cudaDeviceGetAttribute(smem_optin_bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return CPB_SUCCESS;
}

cpb_status cpb_stencil_launch(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                              int ny, int steps, float dt, cpb_boundary bc, cpb_dtype dtype,
                              cpb_dim3 grid, cpb_dim3 block, size_t shared_bytes, void* scratch,
                              cpb_stream_t stream) {
  Fields f{u_in, u_out, kappa, src, scratch};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (block.x == 0 && block.y == 0 && block.z == 0)
    return enqueue_tuned(f, nx, ny, steps, dt, bc, dtype, lookup_tuning(nx, ny, dtype, bc), s);
  if (dtype != CPB_F32) return CPB_ERR_UNSUPPORTED_CONFIG;
  if (!src) return CPB_ERR_INVALID_VALUE;
  return enqueue_tile(f, nx, ny, steps, dt, bc, grid, block, shared_bytes, s);
}

size_t cpb_tile_blocked_shared_bytes(int bx, int by, int depth) {
  if (bx < 1 || by < 1 || (long long)bx * by > 1024 || depth < 1 || depth > 16) return 0;
  return tile_blocked_smem_bytes(bx, by, depth);
}

cpb_status cpb_stencil_tile_blocked(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                                    int ny, int steps, int depth, float dt, cpb_boundary bc, cpb_dim3 grid,
                                    cpb_dim3 block, size_t shared_bytes, void* scratch,
                                    cpb_stream_t stream) {
  Fields f{u_in, u_out, kappa, src, scratch};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, CPB_F32);
  if (st != CPB_SUCCESS) return st;
  if (depth < 1 || depth > 16) return CPB_ERR_INVALID_VALUE;
  const long long bx = block.x, by = block.y;
  if (block.z != 1 || bx < 1 || by < 1 || bx * by > 1024) return CPB_ERR_UNSUPPORTED_CONFIG;
  if ((long long)grid.x != (nx + bx - 1) / bx || (long long)grid.y != (ny + by - 1) / by || grid.z != 1)
    return CPB_ERR_INVALID_VALUE;
  const size_t need = tile_blocked_smem_bytes((int)bx, (int)by, depth);
  if (need > 227 * 1024) return CPB_ERR_UNSUPPORTED_CONFIG;
  if (shared_bytes < need) return CPB_ERR_SHARED_MEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t ub = (size_t)nx * ny * sizeof(float);
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(u_out, u_in, ub, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  bool copy_at_end = false;
  std::vector<int> depths = pass_depths(steps, depth, scratch != nullptr, &copy_at_end);
  const int P = (int)depths.size();
  const void* src_buf = u_in;
  for (int i = 0; i < P; ++i) {
    void* dst;
    if (scratch)
      dst = ((P - 1 - i) % 2 == 0) ? u_out : scratch;
    else if (!copy_at_end)
      dst = ((P - 1 - i) % 2 == 0) ? u_out : u_in;
    else
      dst = (i % 2 == 0) ? u_out : u_in;
    CPB_TRY(launch_tile_blocked_f32(static_cast<const float*>(src_buf), static_cast<float*>(dst),
                                    static_cast<const float*>(kappa), static_cast<const float*>(src), nx, ny,
                                    dt, (int)bc, depths[i], dim3(grid.x, grid.y, 1), dim3(block.x, block.y, 1),
                                    s));
    src_buf = dst;
  }
  if (copy_at_end) CPB_TRY(cudaMemcpyAsync(u_out, u_in, ub, cudaMemcpyDeviceToDevice, s));
  return CPB_SUCCESS;
}

size_t cpb_stencil3d_shared_bytes(int by) { return (by >= 1 && by <= 8) ? vol_smem_bytes(by) : 0; }

cpb_status cpb_stencil3d_launch(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                                int ny, int nz, int steps, float dt, cpb_boundary bc, cpb_dim3 grid,
                                cpb_dim3 block, size_t shared_bytes, void* scratch, cpb_stream_t stream) {
  if (nx < 1 || ny < 1 || nz < 1 || steps < 0) return CPB_ERR_INVALID_VALUE;
  if ((long long)ny * nz > 0x7fffffffLL) return CPB_ERR_INVALID_VALUE;
  Fields f{u_in, u_out, kappa, src, scratch};
  // the checks of the 2-D call on the same bytes (nx x (ny*nz) cells)
  cpb_status st = check_common(f, nx, ny * nz, steps, dt, bc, CPB_F32);
  if (st != CPB_SUCCESS) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int gx = (nx + 127) / 128;
  int by = 8, gz = 0;
  if (block.x == 0 && block.y == 0 && block.z == 0) {
    // default: 32 x 8 threads, z-chunks of about 32 planes (measured at 512^3
    // on GB300 over by = 1..8 and 8..64-plane chunks: by = 8 with 32-64
    // planes is fastest; each chunk re-reads two planes)
    gz = std::max(1, (nz + 31) / 32);
  } else {
    if (block.x != 32 || block.y < 1 || block.y > 8 || block.z != 1) return CPB_ERR_UNSUPPORTED_CONFIG;
    by = (int)block.y;
    if ((long long)grid.x != gx || (long long)grid.y != (ny + by - 1) / by || grid.z < 1 ||
        (long long)grid.z > nz)
      return CPB_ERR_INVALID_VALUE;
    if (shared_bytes < vol_smem_bytes(by)) return CPB_ERR_SHARED_MEM;
    gz = (int)grid.z;
  }
  const dim3 g3((unsigned)gx, (unsigned)((ny + by - 1) / by), (unsigned)gz);
  const int vec = (nx % 4 == 0) && aligned(u_in, 16) && aligned(u_out, 16) && aligned(scratch, 16) &&
                  aligned(kappa, 16) && aligned(src, 16);
  const size_t ub = (size_t)nx * ny * nz * sizeof(float);
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(u_out, u_in, ub, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  bool copy_at_end = false;
  std::vector<int> depths = pass_depths(steps, 1, scratch != nullptr, &copy_at_end);
  const int P = (int)depths.size();
  const void* src_buf = u_in;
  for (int i = 0; i < P; ++i) {
    void* dst;
    if (scratch)
      dst = ((P - 1 - i) % 2 == 0) ? u_out : scratch;
    else if (!copy_at_end)
      dst = ((P - 1 - i) % 2 == 0) ? u_out : u_in;
    else
      dst = (i % 2 == 0) ? u_out : u_in;
    CPB_TRY(launch_vol_f32(static_cast<const float*>(src_buf), static_cast<float*>(dst),
                           static_cast<const float*>(kappa), static_cast<const float*>(src), nx, ny, nz, dt,
                           (int)bc, vec, g3, by, s));
    src_buf = dst;
  }
  if (copy_at_end) CPB_TRY(cudaMemcpyAsync(u_out, u_in, ub, cudaMemcpyDeviceToDevice, s));
  return CPB_SUCCESS;
}

cpb_status cpb_stencil_launch_tuned(void* u_in, void* u_out, const void* kappa, const void* src,
                                    int nx, int ny, int steps, float dt, cpb_boundary bc,
                                    cpb_dtype dtype, const cpb_tuning* tuning, void* scratch,
                                    cpb_stream_t stream) {
  Fields f{u_in, u_out, kappa, src, scratch};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cpb_tuning t = tuning ? *tuning : lookup_tuning(nx, ny, dtype, bc);
  if (!tuning_valid(t)) return CPB_ERR_UNSUPPORTED_CONFIG;
  return enqueue_tuned(f, nx, ny, steps, dt, bc, dtype, t, reinterpret_cast<cudaStream_t>(stream));
}

cpb_status cpb_set_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, const cpb_tuning* t) {
  if (!t || !tuning_valid(*t) || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune[TuneKey(nx, ny, (int)dtype, (int)bc)] = *t;
  return CPB_SUCCESS;
}

cpb_status cpb_get_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, cpb_tuning* t) {
  if (!t || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  *t = lookup_tuning(nx, ny, dtype, bc);
  return CPB_SUCCESS;
}

cpb_status cpb_lookup_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, cpb_tuning* t,
                             int* found) {
  if (!t || !found || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  auto it = g_tune.find(TuneKey(nx, ny, (int)dtype, (int)bc));
  *found = it != g_tune.end() ? 1 : 0;
  if (*found) *t = it->second;
  return CPB_SUCCESS;
}

cpb_status cpb_tuning_save(const char* path, const char* device) {
  if (!path) return CPB_ERR_INVALID_VALUE;
  std::string dev;
  CPB_TRY_STATUS(device_tag(device, &dev));
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) {
    g_last_error = "cannot write " + tmp;
    return CPB_ERR_INVALID_VALUE;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    for (const auto& kv : g_tune) {
      const cpb_tuning& t = kv.second;
      std::fprintf(f, "cpb-tuning 1 %s %d %d %d %d %d %d %d %d %d\n", dev.c_str(), std::get<0>(kv.first),
                   std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first), t.k, t.chunk_rows,
                   t.warps_per_block, t.variant, t.stages);
    }
  }
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    g_last_error = std::string("cannot replace ") + path;
    return CPB_ERR_INVALID_VALUE;
  }
  return CPB_SUCCESS;
}

cpb_status cpb_tuning_load(const char* path, const char* device, int* loaded) {
  if (loaded) *loaded = 0;
  if (!path) return CPB_ERR_INVALID_VALUE;
  std::string dev;
  CPB_TRY_STATUS(device_tag(device, &dev));
  FILE* f = std::fopen(path, "r");
  if (!f) {
    g_last_error = std::string("cannot open ") + path;
    return CPB_ERR_INVALID_VALUE;
  }
  char line[512];
  int n = 0;
  cpb_status st = CPB_SUCCESS;
  while (std::fgets(line, sizeof line, f)) {
    char name[256];
    int ver, nx, ny, dt, bc;
    cpb_tuning t;
    char tail = 0;
    const int got = std::sscanf(line, "cpb-tuning %d %255s %d %d %d %d %d %d %d %d %d %c", &ver, name, &nx, &ny,
                                &dt, &bc, &t.k, &t.chunk_rows, &t.warps_per_block, &t.variant, &t.stages, &tail);
    if (got != 11 || ver != 1 || nx < 1 || ny < 1 || !dtype_ok(dt) ||
        (bc != CPB_DIRICHLET0 && bc != CPB_PERIODIC) || !tuning_valid(t)) {
      g_last_error = std::string("bad tuning line: ") + line;
      st = CPB_ERR_INVALID_VALUE;
      break;
    }
    if (dev != name) continue;
    {
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      g_tune[TuneKey(nx, ny, dt, bc)] = t;
    }
    ++n;
  }
  std::fclose(f);
  if (loaded) *loaded = n;
  return st;
}

cpb_status cpb_autotune(void* u_a, void* u_b, const void* kappa, const void* src, int nx, int ny,
                        int steps, float dt, cpb_boundary bc, cpb_dtype dtype, cpb_stream_t stream,
                        cpb_tuning* best) {
  Fields f{u_a, u_b, kappa, src, nullptr};
  cpb_status st = check_common(f, nx, ny, steps < 1 ? 1 : steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ks[] = {1, 2, 3, 4, 5, 6, 8};
  // short chunks give small grids a full wave of warp items
  const int chunks[] = {16, 32, 64, 96, 128, 192, 256, 512};
  const int wpbs[] = {1, 2, 4};
  const int variants[] = {0, 1};
  const int stages_list[] = {2, 4, 8};
  cudaEvent_t e0, e1;
  CPB_TRY(cudaEventCreate(&e0));
  CPB_TRY(cudaEventCreate(&e1));
  const int probe = steps >= 1 ? steps : 16;
  // Time `reps` runs of a probe after one timed warm-up run; returns cell
  // updates per second.  The probe is an odd number of passes of depth k
  // near `probe` steps, so every pass has depth k (an even count would split
  // one pass in two); a run shorter than 1 ms is repeated until the timed
  // region reaches about 1 ms, so small grids are not timed on noise.
  auto time_runs = [&](const cpb_tuning& t, int n, int reps, float* ms) -> bool {
    if (cudaEventRecord(e0, s) != cudaSuccess) return false;
    for (int rep = 0; rep < reps; ++rep)
      if (enqueue_tuned(f, nx, ny, n, dt, bc, dtype, t, s) != CPB_SUCCESS) return false;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return false;
    return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess && *ms > 0.0f;
  };
  auto rate_of = [&](const cpb_tuning& t, int reps) -> double {
    const int n = t.k * (std::max(1, probe / t.k) | 1);
    float ms = 0.0f;
    if (!time_runs(t, n, 1, &ms)) return -1.0;  // warm-up, and the length of one run
    reps = std::max(reps, std::min(64, (int)std::ceil(1.0f / ms)));
    if (!time_runs(t, n, reps, &ms)) return -1.0;
    return (double)reps * n * (double)nx * ny / (ms * 1e-3);
  };
  // Phase 1: screen every candidate (the better of two single runs, so one
  // disturbed run does not drop a candidate).  Phase 2: re-time the best
  // twelve with more repetitions and keep the fastest.
  std::vector<std::pair<double, cpb_tuning>> screened;
  for (int k : ks)
    for (int c : chunks)
      for (int w : wpbs)
        for (int v : variants)
          for (int st : stages_list) {
            if (c > 2 * ny && c != chunks[0]) continue;
            if (v == 0 && st != stages_list[0]) continue;
            cpb_tuning t{k, c, w, v, st};
            if (!tuning_valid(t)) continue;
            const double r = std::max(rate_of(t, 1), rate_of(t, 1));
            if (r > 0.0) screened.push_back({r, t});
          }
  {  // the built-in default (its chunk height is sized for one wave) competes too
    const cpb_tuning t = default_tuning(nx, ny, dtype);
    const double r = std::max(rate_of(t, 1), rate_of(t, 1));
    if (r > 0.0) screened.push_back({r, t});
  }
  std::sort(screened.begin(), screened.end(),
            [](const std::pair<double, cpb_tuning>& x, const std::pair<double, cpb_tuning>& y) {
              return x.first > y.first;
            });
  cpb_tuning bt = default_tuning(nx, ny, dtype);
  double best_rate = -1.0;
  for (size_t i = 0; i < screened.size() && i < 12; ++i) {
    const double r = rate_of(screened[i].second, 4);
    if (r > best_rate) {
      best_rate = r;
      bt = screened[i].second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  (void)cudaGetLastError();
  cpb_set_tuning(nx, ny, dtype, bc, &bt);
  if (best) *best = bt;
  return CPB_SUCCESS;
}

cpb_status cpb_device_status(int* status) {
  if (!status) return CPB_ERR_INVALID_VALUE;
  CPB_TRY(cudaDeviceSynchronize());
  int a = 0, b = 0, c = 0;
  CPB_TRY(read_stream_status_f32(&a));
  CPB_TRY(read_stream_status_bf16k(&b));
  CPB_TRY(read_stream_status_bf16k_block(&c));
  *status = a ? a : (b ? b : c);
  return CPB_SUCCESS;
}

cpb_status cpb_bounds_status(int* unit, int* line) {
  if (!unit || !line) return CPB_ERR_INVALID_VALUE;
  CPB_TRY(cudaDeviceSynchronize());
  cudaError_t (*const readers[])(int*) = {read_bounds_stream_f32, read_bounds_stream_bf16k,
                                          read_bounds_stream_bf16k_block, read_bounds_batch,
                                          read_bounds_adjoint, read_bounds_vol, read_bounds_tile,
                                          read_bounds_sum};
  *unit = 0;
  *line = 0;
  for (int u = 0; u < (int)(sizeof(readers) / sizeof(readers[0])); ++u) {
    int l = 0;
    CPB_TRY(readers[u](&l));
    if (l != 0 && *line == 0) {
      *unit = u + 1;
      *line = l;
    }
  }
#ifdef CPB_BOUNDS_CHECK
  return CPB_SUCCESS;
#else
  return CPB_ERR_UNSUPPORTED_CONFIG;
#endif
}

cpb_status cpb_debug_set(int wait_limit, int inject_row) {
  g_wait_limit = wait_limit > 0 ? wait_limit : (1 << 20);
  g_inject_on = inject_row >= 0 ? 1 : 0;
  g_inject_row = inject_row;
  return CPB_SUCCESS;
}

size_t cpb_heat_sum_workspace_bytes(int nx, int ny) {
  if (nx < 1 || ny < 1) return 0;
  return sizeof(double) * (size_t)heat_sum_blocks((long long)nx * ny);
}

cpb_status cpb_heat_sum(const void* u, int nx, int ny, cpb_dtype dtype, double* d_out,
                        void* workspace, size_t ws_bytes, cpb_stream_t stream) {
  if (!u || !d_out || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  if (!dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  if (!aligned(u, 4) || !aligned(d_out, 8)) return CPB_ERR_INVALID_VALUE;
  const long long n = (long long)nx * ny;
  const int nb = heat_sum_blocks(n);
  if (!workspace || !aligned(workspace, 8) || ws_bytes < sizeof(double) * (size_t)nb)
    return CPB_ERR_WORKSPACE;
  return from_cuda(launch_heat_sum(u, n, (int)dtype, d_out, static_cast<double*>(workspace), nb,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_heat_sum_noalloc(const void* u, int nx, int ny, cpb_dtype dtype, double* d_out,
                                cpb_stream_t stream) {
  if (!u || !d_out || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  if (!dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  if (!aligned(u, 4) || !aligned(d_out, 8)) return CPB_ERR_INVALID_VALUE;
  const long long n = (long long)nx * ny;
  if (n > heat_sum_noalloc_max_cells()) {
    g_last_error = "grid larger than the built-in heat-sum scratch allows (" +
                   std::to_string(heat_sum_noalloc_max_cells()) + " cells); use cpb_heat_sum";
    return CPB_ERR_WORKSPACE;
  }
  return from_cuda(launch_heat_sum_noalloc(u, n, (int)dtype, d_out,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_bf16_round(const float* x, uint16_t* out, long long n, cpb_stream_t stream) {
  if (n < 0 || (n > 0 && (!x || !out))) return CPB_ERR_INVALID_VALUE;
  if (n == 0) return CPB_SUCCESS;
  return from_cuda(launch_bf16_round(x, out, n, reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_bf16k_pack(const float* u, uint32_t* state, long long n, cpb_stream_t stream) {
  if (n < 0 || (n > 0 && (!u || !state))) return CPB_ERR_INVALID_VALUE;
  if (n == 0) return CPB_SUCCESS;
  return from_cuda(launch_bf16k_pack(u, state, n, reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_bf16k_unpack(const uint32_t* state, float* u, long long n, cpb_stream_t stream) {
  if (n < 0 || (n > 0 && (!u || !state))) return CPB_ERR_INVALID_VALUE;
  if (n == 0) return CPB_SUCCESS;
  return from_cuda(launch_bf16k_unpack(state, u, n, reinterpret_cast<cudaStream_t>(stream)));
}

size_t cpb_host_workspace_bytes(int nx, int ny, cpb_dtype dtype) {
  if (nx < 1 || ny < 1) return 0;
  const size_t n = (size_t)nx * ny;
  return 2 * align256(n * u_bytes(dtype)) + 2 * align256(n * ks_bytes(dtype));
}

cpb_status cpb_stencil_host(const void* u0_host, const void* kappa_host, const void* src_host,
                            void* u_out_host, int nx, int ny, int steps, float dt, cpb_boundary bc,
                            cpb_dtype dtype, void* d_workspace, size_t ws_bytes,
                            cpb_stream_t stream) {
  if (!u0_host || !kappa_host || !u_out_host || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  if (!dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  const size_t need = cpb_host_workspace_bytes(nx, ny, dtype);
  if (!d_workspace || ws_bytes < need || !aligned(d_workspace, 256)) return CPB_ERR_WORKSPACE;
  const size_t n = (size_t)nx * ny;
  const size_t ub = n * u_bytes(dtype), kb = n * ks_bytes(dtype);
  char* base = static_cast<char*>(d_workspace);
  void* ua = base;
  void* ubuf = base + align256(ub);
  void* kd = base + 2 * align256(ub);
  void* sd = src_host ? base + 2 * align256(ub) + align256(kb) : nullptr;
  Fields f{ua, ubuf, kd, sd, nullptr};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CPB_TRY(cudaMemcpyAsync(ua, u0_host, ub, cudaMemcpyHostToDevice, s));
  CPB_TRY(cudaMemcpyAsync(kd, kappa_host, kb, cudaMemcpyHostToDevice, s));
  if (sd) CPB_TRY(cudaMemcpyAsync(sd, src_host, kb, cudaMemcpyHostToDevice, s));
  st = enqueue_tuned(f, nx, ny, steps, dt, bc, dtype, lookup_tuning(nx, ny, dtype, bc), s);
  if (st != CPB_SUCCESS) return st;
  CPB_TRY(cudaMemcpyAsync(u_out_host, ubuf, ub, cudaMemcpyDeviceToHost, s));
  CPB_TRY(cudaStreamSynchronize(s));
  return CPB_SUCCESS;
}

cpb_status cpb_stencil_host_async(const void* u0_host, const void* kappa_host, const void* src_host,
                                  void* u_out_host, int nx, int ny, int steps, float dt, cpb_boundary bc,
                                  cpb_dtype dtype, void* d_workspace, size_t ws_bytes, cpb_stream_t h2d,
                                  cpb_stream_t compute, cpb_stream_t d2h) {
  if (!u0_host || !kappa_host || !u_out_host || nx < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  if (!dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  if (h2d == compute || compute == d2h || h2d == d2h) return CPB_ERR_INVALID_VALUE;
  const size_t need = cpb_host_workspace_bytes(nx, ny, dtype);
  if (!d_workspace || ws_bytes < need || !aligned(d_workspace, 256)) return CPB_ERR_WORKSPACE;
  const size_t n = (size_t)nx * ny;
  const size_t ub = n * u_bytes(dtype), kb = n * ks_bytes(dtype);
  char* base = static_cast<char*>(d_workspace);
  void* ua = base;
  void* ubuf = base + align256(ub);
  void* kd = base + 2 * align256(ub);
  void* sd = src_host ? base + 2 * align256(ub) + align256(kb) : nullptr;
  Fields f{ua, ubuf, kd, sd, nullptr};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cudaStream_t sin = reinterpret_cast<cudaStream_t>(h2d), sc = reinterpret_cast<cudaStream_t>(compute),
               sout = reinterpret_cast<cudaStream_t>(d2h);
  // Two events per call, released by cudaEventDestroy once they complete.
  cudaEvent_t in_done, run_done;
  CPB_TRY(cudaEventCreateWithFlags(&in_done, cudaEventDisableTiming));
  const cudaError_t e = cudaEventCreateWithFlags(&run_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaEventDestroy(in_done);
    return from_cuda(e);
  }
  auto finish = [&](cpb_status r) {
    cudaEventDestroy(in_done);
    cudaEventDestroy(run_done);
    return r;
  };
  cpb_status r = from_cuda(cudaMemcpyAsync(ua, u0_host, ub, cudaMemcpyHostToDevice, sin));
  if (r == CPB_SUCCESS) r = from_cuda(cudaMemcpyAsync(kd, kappa_host, kb, cudaMemcpyHostToDevice, sin));
  if (r == CPB_SUCCESS && sd) r = from_cuda(cudaMemcpyAsync(sd, src_host, kb, cudaMemcpyHostToDevice, sin));
  if (r == CPB_SUCCESS) r = from_cuda(cudaEventRecord(in_done, sin));
  if (r == CPB_SUCCESS) r = from_cuda(cudaStreamWaitEvent(sc, in_done, 0));
  if (r == CPB_SUCCESS) r = enqueue_tuned(f, nx, ny, steps, dt, bc, dtype, lookup_tuning(nx, ny, dtype, bc), sc);
  if (r == CPB_SUCCESS) r = from_cuda(cudaEventRecord(run_done, sc));
  if (r == CPB_SUCCESS) r = from_cuda(cudaStreamWaitEvent(sout, run_done, 0));
  if (r == CPB_SUCCESS) r = from_cuda(cudaMemcpyAsync(u_out_host, ubuf, ub, cudaMemcpyDeviceToHost, sout));
  return finish(r);
}

cpb_status cpb_batch_plan_default(cpb_batch_plan* plan) {
  if (!plan) return CPB_ERR_INVALID_VALUE;
  plan->grain = 1;
  plan->blocks = 0;
  plan->depth = 4;
  plan->threads = batch_threads_max(plan->depth);
  // Measured on the 4096-grid set (sides 32..1024): a whole CTA per grid down
  // to 32 x 32 beats one warp per small grid (a long small grid on one warp
  // becomes the critical path): 154 ms at 1024 vs 231 ms at 65536.
  plan->team_cells = 1024;
  plan->team_warps = 1;
  return CPB_SUCCESS;
}

namespace {
bool host_desc_ok(const cpb_grid_desc& g) {
  return g.nx >= 1 && g.ny >= 1 && g.steps >= 0 && g.u_in && g.u_out && g.kappa &&
         g.u_in != g.u_out && g.dt > 0.0f && std::isfinite(g.dt) &&
         (long long)g.nx * g.ny <= (1LL << 31) && aligned(g.u_in, 4) && aligned(g.u_out, 4) &&
         aligned(g.kappa, 4) && aligned(g.src, 4);
}

bool plan_ok(const cpb_batch_plan& p) {
  return p.grain >= 1 && p.threads >= 32 && p.threads % 32 == 0 && batch_threads_max(p.depth) > 0 &&
         p.threads <= batch_threads_max(p.depth) && p.team_cells >= 1 && batch_team_ok(p.threads, p.team_warps);
}
}  // namespace

cpb_status cpb_batch_order(const cpb_grid_desc* h_descs, int ngrids, const cpb_batch_plan* plan,
                           int* h_order, int* n_large) {
  if (!h_descs || !h_order || !n_large || ngrids < 0) return CPB_ERR_INVALID_VALUE;
  cpb_batch_plan p;
  cpb_batch_plan_default(&p);
  if (plan) p = *plan;
  if (!plan_ok(p)) return CPB_ERR_INVALID_VALUE;
  std::vector<int> large, small;
  for (int i = 0; i < ngrids; ++i) {
    if (!host_desc_ok(h_descs[i])) return CPB_ERR_INVALID_VALUE;
    ((long long)h_descs[i].nx * h_descs[i].ny >= p.team_cells ? large : small).push_back(i);
  }
  auto cost = [&](int i) { return (double)h_descs[i].nx * h_descs[i].ny * (double)h_descs[i].steps; };
  auto lpt = [&](int a, int b) { return cost(a) > cost(b) || (cost(a) == cost(b) && a < b); };
  std::sort(large.begin(), large.end(), lpt);
  std::sort(small.begin(), small.end(), lpt);
  int o = 0;
  for (int i : large) h_order[o++] = i;
  for (int i : small) h_order[o++] = i;
  *n_large = (int)large.size();
  return CPB_SUCCESS;
}

size_t cpb_batch_work_bytes(void) { return 4 * sizeof(int); }

cpb_status cpb_stencil_batched(const cpb_grid_desc* d_descs, const int* d_order, int ngrids,
                               int n_large, cpb_dtype dtype, cpb_boundary bc,
                               const cpb_batch_plan* plan, int* d_work, cpb_stream_t stream) {
  if (ngrids < 0 || n_large < 0 || n_large > ngrids) return CPB_ERR_INVALID_VALUE;
  if (bc != CPB_DIRICHLET0 && bc != CPB_PERIODIC) return CPB_ERR_INVALID_VALUE;
  if (dtype != CPB_F32) return CPB_ERR_UNSUPPORTED_CONFIG;
  if (!d_work || !aligned(d_work, 4)) return CPB_ERR_WORKSPACE;
  if (ngrids > 0 && (!d_descs || !d_order)) return CPB_ERR_INVALID_VALUE;
  cpb_batch_plan p;
  cpb_batch_plan_default(&p);
  if (plan) p = *plan;
  if (!plan_ok(p)) return CPB_ERR_INVALID_VALUE;
  int blocks = p.blocks;
  if (blocks <= 0) {
    int per_sm = 0;
    CPB_TRY(batch_blocks_per_sm(p.depth, p.threads, &per_sm));
    blocks = std::max(1, per_sm) * device_sm_count();
  }
  const BatchDebug dbg{g_wait_limit, g_inject_on, g_inject_row};
  return from_cuda(launch_batch(p.depth, d_descs, d_order, ngrids, n_large, (int)bc, p.grain, blocks, p.threads,
                                p.team_warps, dbg, d_work, reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_batch_status(const int* d_work, int* status, cpb_stream_t stream) {
  if (!d_work || !status) return CPB_ERR_INVALID_VALUE;
  int w[4] = {0, 0, 0, 0};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CPB_TRY(cudaMemcpyAsync(w, d_work, sizeof(w), cudaMemcpyDeviceToHost, s));
  CPB_TRY(cudaStreamSynchronize(s));
  *status = w[2];
  return CPB_SUCCESS;
}

cpb_status cpb_batch_autotune(const cpb_grid_desc* d_descs, const int* d_order, int ngrids,
                              int n_large, cpb_dtype dtype, cpb_boundary bc, int* d_work,
                              cpb_stream_t stream, cpb_batch_plan* plan, float* ms_table) {
  if (!plan || !plan_ok(*plan)) return CPB_ERR_INVALID_VALUE;
  static const int depths[CPB_BATCH_TUNE_DEPTHS] = {4, 8};
  static const int grains[CPB_BATCH_TUNE_GRAINS] = {1, 2, 4, 8, 16};
  static const int threads[CPB_BATCH_TUNE_THREADS] = {128, 256, 384};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  CPB_TRY(cudaEventCreate(&e0));
  CPB_TRY(cudaEventCreate(&e1));
  cpb_status result = CPB_SUCCESS;
  // Time `reps` back-to-back runs of plan p; -1 if the launch is rejected.
  auto time_plan = [&](const cpb_batch_plan& p, int reps) -> float {
    if (cudaEventRecord(e0, s) != cudaSuccess) return -1.0f;
    for (int r = 0; r < reps; ++r) {
      const cpb_status st = cpb_stencil_batched(d_descs, d_order, ngrids, n_large, dtype, bc, &p, d_work, stream);
      if (st != CPB_SUCCESS) {
        if (result == CPB_SUCCESS && st != CPB_ERR_LAUNCH && st != CPB_ERR_CUDA) result = st;
        return -1.0f;
      }
    }
    float ms = -1.0f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return -1.0f;
    int status = 0;
    if (cpb_batch_status(d_work, &status, stream) != CPB_SUCCESS || status != CPB_SUCCESS) {
      if (result == CPB_SUCCESS) result = status != CPB_SUCCESS ? (cpb_status)status : CPB_ERR_CUDA;
      return -1.0f;
    }
    return ms / reps;
  };
  std::vector<std::pair<float, cpb_batch_plan>> timed;
  cpb_batch_plan p = *plan;
  p.blocks = 0;
  time_plan(p, 1);  // warm-up (first launch sets the shared-memory opt-in)
  for (int di = 0; di < CPB_BATCH_TUNE_DEPTHS; ++di)
    for (int gi = 0; gi < CPB_BATCH_TUNE_GRAINS; ++gi)
      for (int ti = 0; ti < CPB_BATCH_TUNE_THREADS; ++ti) {
        p.depth = depths[di];
        p.grain = grains[gi];
        p.threads = threads[ti];
        // a CTA size the depth cannot run is skipped (-1 in the table)
        const float ms = (result == CPB_SUCCESS && plan_ok(p)) ? time_plan(p, 1) : -1.0f;
        if (ms_table) ms_table[(di * CPB_BATCH_TUNE_GRAINS + gi) * CPB_BATCH_TUNE_THREADS + ti] = ms;
        if (ms > 0.0f) timed.push_back({ms, p});
      }
  std::sort(timed.begin(), timed.end(),
            [](const std::pair<float, cpb_batch_plan>& a, const std::pair<float, cpb_batch_plan>& b) {
              return a.first < b.first;
            });
  float best = -1.0f;
  cpb_batch_plan bp = *plan;
  for (size_t i = 0; i < timed.size() && i < 3 && result == CPB_SUCCESS; ++i) {
    const float ms = time_plan(timed[i].second, 2);
    if (ms > 0.0f && (best < 0.0f || ms < best)) {
      best = ms;
      bp = timed[i].second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != CPB_SUCCESS) return result;
  if (best < 0.0f) return CPB_ERR_LAUNCH;
  *plan = bp;
  return CPB_SUCCESS;
}

// ---------------------------------------------------------------------------
// Adjoint with checkpointing
// ---------------------------------------------------------------------------
namespace {
struct AdjointLayout {
  size_t slot;  // bytes per field slot (256-aligned)
  int nseg;     // checkpoints (states at m * ckpt)
  int nsegbuf;  // recompute slots per segment (ckpt - 1)
  size_t bytes;
  float* ckpt(void* ws, int m) const { return reinterpret_cast<float*>(static_cast<char*>(ws) + m * slot); }
  float* seg(void* ws, int q) const { return ckpt(ws, nseg + q); }
  float* lam(void* ws, int i) const { return ckpt(ws, nseg + nsegbuf + i); }
  float* tmp(void* ws) const { return ckpt(ws, nseg + nsegbuf + 2); }
};

AdjointLayout adjoint_layout(int nx, int ny, int steps, int ckpt) {
  AdjointLayout L;
  L.slot = align256((size_t)nx * ny * sizeof(float));
  L.nseg = steps > 0 ? (steps + ckpt - 1) / ckpt : 0;
  L.nsegbuf = std::max(0, std::min(ckpt, steps) - 1);
  L.bytes = L.slot * (size_t)(std::max(L.nseg, 1) + L.nsegbuf + 3);
  return L;
}

cpb_status adjoint_check(int nx, int ny, int steps, float dt, cpb_boundary bc, int ckpt, void* ws,
                         size_t ws_bytes) {
  if (nx < 1 || ny < 1 || steps < 0 || ckpt < 1) return CPB_ERR_INVALID_VALUE;
  if (!(dt > 0.0f) || !std::isfinite(dt)) return CPB_ERR_INVALID_VALUE;
  if (bc != CPB_DIRICHLET0 && bc != CPB_PERIODIC) return CPB_ERR_INVALID_VALUE;
  if (!ws || !aligned(ws, 256) || ws_bytes < adjoint_layout(nx, ny, steps, ckpt).bytes)
    return CPB_ERR_WORKSPACE;
  return CPB_SUCCESS;
}
}  // namespace

size_t cpb_adjoint_workspace_bytes(int nx, int ny, int steps, int ckpt_every) {
  if (nx < 1 || ny < 1 || steps < 0 || ckpt_every < 1) return 0;
  return adjoint_layout(nx, ny, steps, ckpt_every).bytes;
}

cpb_status cpb_adjoint_forward(const float* u0, const float* kappa, const float* src, int nx, int ny,
                               int steps, float dt, cpb_boundary bc, int ckpt_every, float* u_T,
                               void* workspace, size_t ws_bytes, cpb_stream_t stream) {
  cpb_status st = adjoint_check(nx, ny, steps, dt, bc, ckpt_every, workspace, ws_bytes);
  if (st != CPB_SUCCESS) return st;
  if (!u0 || !kappa || !u_T || !aligned(u0, 4) || !aligned(kappa, 4) || !aligned(src, 4))
    return CPB_ERR_INVALID_VALUE;
  const AdjointLayout L = adjoint_layout(nx, ny, steps, ckpt_every);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)nx * ny * sizeof(float);
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(u_T, u0, nb, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  const cpb_tuning t = lookup_tuning(nx, ny, CPB_F32, bc);
  CPB_TRY(cudaMemcpyAsync(L.ckpt(workspace, 0), u0, nb, cudaMemcpyDeviceToDevice, s));
  for (int m = 0; m < L.nseg; ++m) {
    const int len = std::min(ckpt_every, steps - m * ckpt_every);
    float* dst = (m == L.nseg - 1) ? u_T : L.ckpt(workspace, m + 1);
    Fields f{L.ckpt(workspace, m), dst, kappa, src, L.tmp(workspace)};
    st = enqueue_tuned(f, nx, ny, len, dt, bc, CPB_F32, t, s);
    if (st != CPB_SUCCESS) return st;
  }
  return CPB_SUCCESS;
}

cpb_status cpb_adjoint_backward(const float* kappa, const float* src, const float* lambda_T, int nx,
                                int ny, int steps, float dt, cpb_boundary bc, int ckpt_every,
                                float* grad_u0, float* grad_kappa, void* workspace, size_t ws_bytes,
                                cpb_stream_t stream) {
  cpb_status st = adjoint_check(nx, ny, steps, dt, bc, ckpt_every, workspace, ws_bytes);
  if (st != CPB_SUCCESS) return st;
  if (!kappa || !lambda_T || !grad_u0 || !grad_kappa) return CPB_ERR_INVALID_VALUE;
  const AdjointLayout L = adjoint_layout(nx, ny, steps, ckpt_every);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t nb = (size_t)nx * ny * sizeof(float);
  CPB_TRY(cudaMemsetAsync(grad_kappa, 0, nb, s));
  if (steps == 0) {
    CPB_TRY(cudaMemcpyAsync(grad_u0, lambda_T, nb, cudaMemcpyDeviceToDevice, s));
    return CPB_SUCCESS;
  }
  cpb_tuning t1 = lookup_tuning(nx, ny, CPB_F32, bc);
  t1.k = 1;  // recompute one step per state
  // Where the TMA row ring applies, a segment is recomputed by depth-4 passes
  // that also store their intermediate levels: one pass reads the fields once
  // and yields four consecutive states (12/4 + 4 B per cell and state instead
  // of 16).  Slots are 256-byte aligned, so only the caller's fields decide.
  const bool levels = bulk_eligible(nx, CPB_F32, nx % 4 == 0 && aligned(kappa, 16) && aligned(src, 16), kappa,
                                    src);
  StreamPass lp;
  if (levels) {
    // depth 4, TMA ring, chunks sized for one wave (the built-in default;
    // measured on the 2048^2 workload: the geometry of a deeper tuning made
    // the recompute slower)
    const cpb_tuning t4 = default_tuning(nx, ny, CPB_F32);
    lp.kappa = kappa;
    lp.src = src;
    lp.nx = nx;
    lp.ny = ny;
    lp.dt = dt;
    lp.hdt = 0.5f * dt;
    lp.bc = (int)bc;
    lp.vec = 1;
    lp.chunk_rows = t4.chunk_rows;
    lp.warps_per_block = t4.warps_per_block;
    lp.variant = 1;
    lp.stages = t4.stages;
    lp.wait_limit = g_wait_limit;
    lp.inject_on = 0;
    lp.inject_row = 0;
    lp.store_levels = 1;
  }
  // Temporally blocked adjoint passes need the 16-byte row path of every
  // field they touch (workspace slots are 256-byte aligned).
  const bool blocked = nx % 4 == 0 && aligned(lambda_T, 16) && aligned(kappa, 16) && aligned(grad_kappa, 16) &&
                       aligned(grad_u0, 16);
  const float* lam_cur = lambda_T;
  int flip = 0;
  for (int m = L.nseg - 1; m >= 0; --m) {
    const int len = std::min(ckpt_every, steps - m * ckpt_every);
    // states u_{a}, u_{a+1}, ..., u_{a+len-1}: the checkpoint, then recompute
    // (state q of the segment goes to slot seg(q - 1))
    if (levels) {
      for (int q = 1; q < len;) {
        const int d = std::min(4, len - q);  // this pass yields states q .. q + d - 1
        lp.u_in = q == 1 ? (const void*)L.ckpt(workspace, m) : (const void*)L.seg(workspace, q - 2);
        for (int t = 1; t < d; ++t) lp.levels[t - 1] = L.seg(workspace, q + t - 2);
        lp.u_out = L.seg(workspace, q + d - 2);
        lp.depth = d;
        CPB_TRY(launch_stream_f32(lp, 4, s));
        q += d;
      }
    } else {
      for (int q = 1; q < len; ++q) {
        void* prev = q == 1 ? (void*)L.ckpt(workspace, m) : (void*)L.seg(workspace, q - 2);
        Fields f{prev, L.seg(workspace, q - 1), kappa, src, L.tmp(workspace)};
        st = enqueue_tuned(f, nx, ny, 1, dt, bc, CPB_F32, t1, s);
        if (st != CPB_SUCCESS) return st;
      }
    }
    // Backward sweep of the segment: lambda_{a+q+1} -> lambda_{a+q} for q =
    // len-1 .. 0 uses state u_{a+q}.  Where the 16-byte row path applies, in
    // passes of up to 4 steps (the same bits as one launch per step).
    auto state = [&](int q) -> const float* { return q == 0 ? L.ckpt(workspace, m) : L.seg(workspace, q - 1); };
    for (int q = len - 1; q >= 0;) {
      const int d = blocked ? std::min(4, q + 1) : 1;  // steps q, q-1, .. q-d+1
      float* out = (m == 0 && q - d + 1 == 0) ? grad_u0 : L.lam(workspace, flip);
      if (blocked) {
        const float* us[4] = {nullptr, nullptr, nullptr, nullptr};
        for (int t = 1; t <= d; ++t) us[t - 1] = state(q - t + 1);
        CPB_TRY(launch_adjoint_pass(lam_cur, out, us, d, kappa, grad_kappa, nx, ny, dt, (int)bc, 0, s));
      } else {
        CPB_TRY(launch_adjoint_step(lam_cur, out, state(q), kappa, grad_kappa, nx, ny, dt, (int)bc, s));
      }
      lam_cur = out;
      flip ^= 1;
      q -= d;
    }
  }
  return CPB_SUCCESS;
}

cpb_status cpb_stencil_adjoint(const float* u0, const float* kappa, const float* src,
                               const float* lambda_T, int nx, int ny, int steps, float dt,
                               cpb_boundary bc, int ckpt_every, float* grad_u0, float* grad_kappa,
                               void* workspace, size_t ws_bytes, cpb_stream_t stream) {
  cpb_status st = adjoint_check(nx, ny, steps, dt, bc, ckpt_every, workspace, ws_bytes);
  if (st != CPB_SUCCESS) return st;
  const AdjointLayout L = adjoint_layout(nx, ny, steps, ckpt_every);
  // u_T is not needed by the backward sweep: park it in a lambda slot.
  st = cpb_adjoint_forward(u0, kappa, src, nx, ny, steps, dt, bc, ckpt_every, L.lam(workspace, 1),
                           workspace, ws_bytes, stream);
  if (st != CPB_SUCCESS) return st;
  return cpb_adjoint_backward(kappa, src, lambda_T, nx, ny, steps, dt, bc, ckpt_every, grad_u0,
                              grad_kappa, workspace, ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// Slab decomposition (one rank per GPU)
// ---------------------------------------------------------------------------
cpb_status cpb_slab_rows(int ny, int world, int rank, int depth, cpb_boundary bc, int* row_lo, int* row_hi,
                         int* halo_lo, int* halo_hi) {
  if (world < 1 || rank < 0 || rank >= world || depth < 1 || ny < 1) return CPB_ERR_INVALID_VALUE;
  if (bc != CPB_DIRICHLET0 && bc != CPB_PERIODIC) return CPB_ERR_INVALID_VALUE;
  if ((long long)world * depth > ny) return CPB_ERR_INVALID_VALUE;
  const int base = ny / world, extra = ny % world;
  const int lo = rank * base + std::min(rank, extra);
  const int hi = lo + base + (rank < extra ? 1 : 0);
  const bool periodic = bc == CPB_PERIODIC;
  if (row_lo) *row_lo = lo;
  if (row_hi) *row_hi = hi;
  if (halo_lo) *halo_lo = (periodic || rank > 0) ? depth : 0;
  if (halo_hi) *halo_hi = (periodic || rank < world - 1) ? depth : 0;
  return CPB_SUCCESS;
}

cpb_status cpb_slab_exchange_rows(void* slab, size_t row_bytes, int n_own, int halo_lo, int halo_hi,
                                  const void* below, int below_halo_lo, int below_n_own, const void* above,
                                  int above_halo_lo, int above_n_own, cpb_stream_t stream) {
  if (!slab || row_bytes < 1 || n_own < 1) return CPB_ERR_INVALID_VALUE;
  if (halo_lo < 0 || halo_hi < 0 || halo_lo > n_own || halo_hi > n_own) return CPB_ERR_INVALID_VALUE;
  if (halo_lo > 0 && (!below || below_halo_lo < 0 || below_n_own < halo_lo)) return CPB_ERR_INVALID_VALUE;
  if (halo_hi > 0 && (!above || above_halo_lo < 0 || above_n_own < halo_hi)) return CPB_ERR_INVALID_VALUE;
  const size_t row = row_bytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* dst = static_cast<char*>(slab);
  if (halo_lo > 0) {
    const char* src = static_cast<const char*>(below) + (size_t)(below_halo_lo + below_n_own - halo_lo) * row;
    CPB_TRY(cudaMemcpyAsync(dst, src, (size_t)halo_lo * row, cudaMemcpyDefault, s));
  }
  if (halo_hi > 0) {
    const char* src = static_cast<const char*>(above) + (size_t)above_halo_lo * row;
    CPB_TRY(cudaMemcpyAsync(dst + (size_t)(halo_lo + n_own) * row, src, (size_t)halo_hi * row,
                            cudaMemcpyDefault, s));
  }
  return CPB_SUCCESS;
}

cpb_status cpb_slab_exchange(void* slab, int nx, int n_own, int halo_lo, int halo_hi, const void* below,
                             int below_halo_lo, int below_n_own, const void* above, int above_halo_lo,
                             int above_n_own, cpb_dtype dtype, cpb_stream_t stream) {
  if (nx < 1 || !dtype_ok(dtype)) return CPB_ERR_INVALID_VALUE;
  return cpb_slab_exchange_rows(slab, (size_t)nx * u_bytes(dtype), n_own, halo_lo, halo_hi, below, below_halo_lo,
                                below_n_own, above, above_halo_lo, above_n_own, stream);
}

cpb_status cpb_slab_step(const void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                         int rows_total, int halo_lo, int halo_hi, int steps, float dt, cpb_boundary bc,
                         cpb_dtype dtype, const cpb_tuning* tuning, cpb_stream_t stream) {
  if (halo_lo < 0 || halo_hi < 0 || (long long)halo_lo + halo_hi >= rows_total) return CPB_ERR_INVALID_VALUE;
  if (steps < 1 || steps > 8 || (halo_lo > 0 && steps > halo_lo) || (halo_hi > 0 && steps > halo_hi))
    return CPB_ERR_INVALID_VALUE;
  // One pass (steps <= the tuning's depth): it reads u_in and writes u_out,
  // so u_in is left as it was.
  Fields f{const_cast<void*>(u_in), u_out, kappa, src, nullptr};
  cpb_status st = check_common(f, nx, rows_total, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cpb_tuning t = tuning ? *tuning : lookup_tuning(nx, rows_total, dtype, bc);
  if (t.k < steps) t.k = steps;
  if (!tuning_valid(t)) return CPB_ERR_UNSUPPORTED_CONFIG;
  return enqueue_tuned(f, nx, rows_total, steps, dt, bc, dtype, t, reinterpret_cast<cudaStream_t>(stream));
}

cpb_status cpb_graph_create(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                            int ny, int steps, float dt, cpb_boundary bc, cpb_dtype dtype,
                            const cpb_tuning* tuning, void* scratch, cpb_graph_t* graph) {
  if (!graph) return CPB_ERR_INVALID_VALUE;
  *graph = nullptr;
  Fields f{u_in, u_out, kappa, src, scratch};
  cpb_status st = check_common(f, nx, ny, steps, dt, bc, dtype);
  if (st != CPB_SUCCESS) return st;
  cpb_tuning t = tuning ? *tuning : lookup_tuning(nx, ny, dtype, bc);
  if (!tuning_valid(t)) return CPB_ERR_UNSUPPORTED_CONFIG;
  cudaStream_t cs;
  CPB_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = enqueue_tuned(f, nx, ny, steps, dt, bc, dtype, t, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  cudaStreamDestroy(cs);
  if (st != CPB_SUCCESS) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  CPB_TRY(e);
  cudaGraphExec_t ex;
  e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return from_cuda(e);
  }
  cpb_graph_s* h = new cpb_graph_s{g, ex};
  *graph = h;
  return CPB_SUCCESS;
}

cpb_status cpb_graph_launch(cpb_graph_t graph, cpb_stream_t stream) {
  if (!graph) return CPB_ERR_INVALID_VALUE;
  return from_cuda(cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)));
}

cpb_status cpb_graph_destroy(cpb_graph_t graph) {
  if (!graph) return CPB_ERR_INVALID_VALUE;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return CPB_SUCCESS;
}

}  // extern "C"
