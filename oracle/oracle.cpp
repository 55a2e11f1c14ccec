// CPU oracle for the barrier-tiled heat stencil.  TEST INFRASTRUCTURE ONLY:
// it is loaded by tests/, by __graft_entry__.smoke() and by bench.py's CPU
// baseline leg, never by the product path.  It shares no code, header, table
// or helper with the CUDA library.
//
// What it computes
// ----------------
// 1. A direct serial loop of the canonical 5-point update (the stencil's
//    definition; the paper contains no stencil, so the update, its boundary
//    rules and its rounding order are this project's stated readings):
//        fW = (kc + kW) * (uW - c)      fE = (kc + kE) * (uE - c)
//        fS = (kc + kS) * (uS - c)      fN = (kc + kN) * (uN - c)
//        acc = (fW + fE) + (fS + fN)
//        u'  = c + (hdt * acc + dt * s)         with hdt = 0.5 * dt
//    every operation rounded in the working precision, in exactly that order.
//    Dirichlet: a neighbour outside the grid has u = 0 and kappa = kc.
//    Periodic: indices wrap.
// 2. The same kernel executed the way the paper defines CUDA execution on a
//    CPU: the tiled SPMD kernel (one thread per cell, a shared (BX+2)x(BY+2)
//    halo tile of u and kappa, one __syncthreads) is turned into an explicit
//    loop over the threads of a block, split into one loop per barrier-free
//    region ("SPMD to MPMD", Sec. III), with launch geometry held in
//    explicitly inserted variables (Sec. III, "Extra variable insertion"),
//    parameters packed into a void** (Sec. III, "Parameter packing",
//    Listing 5), and blocks run by a pthread pool fed by a mutex-protected
//    task queue of kernel structures (Sec. IV, Listing 6) with average
//    coarse-grained fetching, ceil(gridSize / poolSize) blocks per fetch
//    (Sec. IV, "Runtime Optimizations").
// 3. BF16-Kahan storage: state (hi, cmp) in bf16, effective value
//    (float)hi - (float)cmp, FP32 compute, hi' = rn(v), cmp' = rn(hi' - v).
// 4. An FP64 heat sum, an FP64 discrete adjoint (gradient of
//    L = 0.5 ||u_T - target||^2 with respect to u_0 and kappa), and a
//    dependency-cone evaluator for sampled cells of a large run.
// 5. A shuffle-based, temporal-blocked strip kernel (a warp per 128-column
//    strip, K time levels per pass) executed the way the paper runs kernels
//    with warp-level functions: nested loops over the warps of a block and
//    the 32 lanes of a warp, split at every shuffle (Sec. III "SPMD to MPMD").
// 6. The 3-D 7-point variant: a direct loop and a z-marching tiled kernel
//    with two barriers inside its plane loop, run with loop fission.
// 7. A shared-memory temporal-blocked tiled kernel (K steps per launch,
//    K + 1 barriers, K of them inside its time loop), run with loop fission.
//
// Build: g++ -O3 -ffp-contract=off (no FMA contraction: GCC contracts a*b+c
// by default on aarch64, which would change the rounding order above).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Runtime: kernel structure, thread pool, task queue (Sec. IV)
// ---------------------------------------------------------------------------
struct Dim3 {
  int x, y, z;
};

// The kernel structure of Listing 6: entry point, packed arguments, launch
// geometry, dynamic shared size, and the queue bookkeeping (totalBlocks,
// curr_blockId, block_per_fetch).  done_blocks / error / fetches are this
// oracle's additions: the host waits for completion (CUDA stream semantics;
// the paper pops a task at its last fetch and leaves kernel-to-kernel
// ordering unstated) and kernel errors are reported, not lost.
struct KernelTask {
  int (*start_routine)(void** args);
  void** args;
  Dim3 gridDim;
  Dim3 blockDim;
  size_t dynamic_shared_mem_size;
  int totalBlocks;
  int curr_blockId;
  int block_per_fetch;
  int done_blocks;
  int error;
  int fetches;
};

// Per-worker launch context, assigned by the runtime before each block runs
// (Sec. III "Extra variable insertion", Listing 7).  The paper's listing
// assigns the block *size* from totalBlocks; the reading taken here is the
// block dimension.
thread_local int block_index;
thread_local Dim3 block_size;
thread_local Dim3 grid_size;
thread_local void* dynamic_shared_memory;

class ThreadPool {
 public:
  explicit ThreadPool(int n) : size_(n) {
    for (int i = 0; i < n; ++i) workers_.emplace_back([this] { worker_loop(); });
  }
  ~ThreadPool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    wake_pool_.notify_all();
    for (auto& t : workers_) t.join();
  }
  int size() const { return size_; }

  // Push task queue: enqueue under the lock, then broadcast wake_pool.
  void push(KernelTask* k) {
    {
      std::lock_guard<std::mutex> lk(m_);
      queue_.push_back(k);
    }
    wake_pool_.notify_all();
  }

  // Host-side synchronisation: wait until every block of k has finished.
  int synchronize(KernelTask* k) {
    std::unique_lock<std::mutex> lk(m_);
    finished_.wait(lk, [&] { return k->done_blocks == k->totalBlocks; });
    return k->error;
  }

 private:
  void worker_loop() {
    // This worker's dynamic shared memory, reused across blocks (the paper
    // mallocs one per block and never frees it; that leak is not copied).
    std::vector<unsigned char> shm;
    for (;;) {
      KernelTask* k = nullptr;
      int first = 0, count = 0;
      {
        // Fetch task queue: under the lock, take block_per_fetch blocks from
        // the front task and pop it once curr_blockId reaches totalBlocks.
        std::unique_lock<std::mutex> lk(m_);
        wake_pool_.wait(lk, [&] { return stop_ || !queue_.empty(); });
        if (queue_.empty()) return;  // stop requested and nothing left
        k = queue_.front();
        first = k->curr_blockId;
        count = std::min(k->block_per_fetch, k->totalBlocks - first);
        k->curr_blockId += count;
        k->fetches += 1;
        if (k->curr_blockId >= k->totalBlocks) queue_.pop_front();
      }
      // Execute fetched blocks outside the lock (Listing 7).
      if (shm.size() < k->dynamic_shared_mem_size) shm.resize(k->dynamic_shared_mem_size);
      int err = 0;
      for (int s = 0; s < count; ++s) {
        block_index = first + s;
        block_size = k->blockDim;
        grid_size = k->gridDim;
        // Shared memory is uninitialised on a GPU; fill it with 0xFF bytes
        // (NaN for float/double) so a read of an unstaged slot is visible.
        if (k->dynamic_shared_mem_size) std::memset(shm.data(), 0xFF, k->dynamic_shared_mem_size);
        dynamic_shared_memory = shm.data();
        int rc = k->start_routine(k->args);
        if (rc != 0 && err == 0) err = rc;
      }
      {
        std::lock_guard<std::mutex> lk(m_);
        k->done_blocks += count;
        if (err != 0 && k->error == 0) k->error = err;
        if (k->done_blocks == k->totalBlocks) finished_.notify_all();
      }
    }
  }

  int size_;
  std::mutex m_;
  std::condition_variable wake_pool_;
  std::condition_variable finished_;
  std::deque<KernelTask*> queue_;
  std::vector<std::thread> workers_;
  bool stop_ = false;
};

// The pool is created once and reused for the whole program (Sec. IV); a
// request for a different size replaces it.
std::mutex g_pool_mutex;
std::unique_ptr<ThreadPool> g_pool;

ThreadPool& pool_of(int n) {
  if (n < 1) n = 1;
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  if (!g_pool || g_pool->size() != n) {
    g_pool.reset();
    g_pool.reset(new ThreadPool(n));
  }
  return *g_pool;
}

// Launch = build a kernel structure, push it, and (stream semantics) wait for
// it.  block_per_fetch <= 0 selects average coarse-grained fetching,
// ceil(totalBlocks / poolSize).
int launch(int (*fn)(void**), void** args, Dim3 grid, Dim3 block, size_t shm, int pool,
           int block_per_fetch, int* fetches_out = nullptr) {
  KernelTask k{};
  k.start_routine = fn;
  k.args = args;
  k.gridDim = grid;
  k.blockDim = block;
  k.dynamic_shared_mem_size = shm;
  k.totalBlocks = grid.x * grid.y * grid.z;
  k.curr_blockId = 0;
  ThreadPool& p = pool_of(pool);
  k.block_per_fetch = block_per_fetch > 0 ? block_per_fetch
                                          : (k.totalBlocks + p.size() - 1) / p.size();
  if (k.block_per_fetch < 1) k.block_per_fetch = 1;
  if (k.totalBlocks == 0) {
    if (fetches_out) *fetches_out = 0;
    return 0;
  }
  p.push(&k);
  int rc = p.synchronize(&k);
  if (fetches_out) *fetches_out = k.fetches;
  return rc;
}

// ---------------------------------------------------------------------------
// The canonical cell update and boundary rule (stated readings; see header)
// ---------------------------------------------------------------------------
template <class T>
inline T cell_update(T c, T uW, T uE, T uS, T uN, T kc, T kW, T kE, T kS, T kN, T s, T dt,
                     T hdt) {
  T fW = (kc + kW) * (uW - c);
  T fE = (kc + kE) * (uE - c);
  T fS = (kc + kS) * (uS - c);
  T fN = (kc + kN) * (uN - c);
  T acc = (fW + fE) + (fS + fN);
  return c + (hdt * acc + dt * s);
}

inline int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

enum { BC_DIRICHLET = 0, BC_PERIODIC = 1 };

// Value of u and kappa seen across the face from cell (i, j) towards (ii, jj).
template <class T>
inline void neighbour(const T* u, const T* k, int nx, int ny, int bc, int ii, int jj, T kc, T& un,
                      T& kn) {
  if (bc == BC_PERIODIC) {
    int w = wrap(ii, nx), h = wrap(jj, ny);
    un = u[(size_t)h * nx + w];
    kn = k[(size_t)h * nx + w];
  } else if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) {
    un = T(0);
    kn = kc;
  } else {
    un = u[(size_t)jj * nx + ii];
    kn = k[(size_t)jj * nx + ii];
  }
}

template <class T>
void direct_rows(const T* u, T* uo, const T* k, const T* s, int nx, int ny, T dt, T hdt, int bc,
                 int j0, int j1) {
  for (int j = j0; j < j1; ++j) {
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      T kc = k[c], uW, kW, uE, kE, uS, kS, uN, kN;
      neighbour(u, k, nx, ny, bc, i - 1, j, kc, uW, kW);
      neighbour(u, k, nx, ny, bc, i + 1, j, kc, uE, kE);
      neighbour(u, k, nx, ny, bc, i, j - 1, kc, uS, kS);
      neighbour(u, k, nx, ny, bc, i, j + 1, kc, uN, kN);
      uo[c] = cell_update<T>(u[c], uW, uE, uS, uN, kc, kW, kE, kS, kN, s[c], dt, hdt);
    }
  }
}

// The direct loop as a plain row-band kernel for the pool (no tiling, no
// barrier): block b updates rows [b*band, (b+1)*band).
template <class T>
int direct_band_mpmd(void** p) {
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  int nx = *(int*)p[4], ny = *(int*)p[5];
  T dt = *(T*)p[6], hdt = *(T*)p[7];
  int bc = *(int*)p[8], band = *(int*)p[9];
  int j0 = block_index * band, j1 = std::min(ny, j0 + band);
  direct_rows<T>(u, uo, k, s, nx, ny, dt, hdt, bc, j0, j1);
  return 0;
}

// Runs `steps` steps, ping-ponging between two buffers; the result is written
// to out.  pool <= 1 runs the serial loop; otherwise row bands go through the
// runtime (bit-identical: every cell is computed by the same expression).
template <class T>
int run_direct(const T* u0, const T* k, const T* s, int nx, int ny, int steps, T dt, int bc,
               int pool, T* out) {
  size_t n = (size_t)nx * ny;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  for (int t = 0; t < steps; ++t) {
    if (pool <= 1) {
      direct_rows<T>(a.data(), b.data(), k, s, nx, ny, dt, hdt, bc, 0, ny);
    } else {
      const T* ua = a.data();
      T* ub = b.data();
      int band = std::max(1, (ny + 4 * pool - 1) / (4 * pool));
      void* args[10] = {&ua, &ub, &k, &s, &nx, &ny, &dt, &hdt, &bc, &band};
      int rc = launch(direct_band_mpmd<T>, args, Dim3{(ny + band - 1) / band, 1, 1}, Dim3{1, 1, 1},
                      0, pool, 0);
      if (rc) return rc;
    }
    a.swap(b);
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// ---------------------------------------------------------------------------
// The tiled SPMD kernel, translated to MPMD with loop fission at its barrier
// ---------------------------------------------------------------------------
// Original SPMD kernel (one thread per cell, blockDim = (BX, BY), dynamic
// shared memory = two (BX+2)*(BY+2) tiles of T):
//   R0: stage own cell into the tile; edge threads also stage the halo cell
//       in their direction; any staged position outside the grid takes the
//       boundary rule (Dirichlet: u = 0, kappa = kappa of the nearest
//       in-grid cell, which is the neighbouring cell's own kappa; periodic:
//       wrap).
//   __syncthreads();
//   R1: if the cell is inside the grid, apply the update from the tile.
// Values live across the barrier (tx, ty, gi, gj) are recomputed in each
// region from the thread index (the paper leaves this unstated).
template <class T>
inline void stage(const T* u, const T* k, int nx, int ny, int bc, int gi, int gj, T* su, T* sk,
                  int slot) {
  if (bc == BC_PERIODIC) {
    size_t g = (size_t)wrap(gj, ny) * nx + wrap(gi, nx);
    su[slot] = u[g];
    sk[slot] = k[g];
  } else {
    bool inside = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    int ci = std::min(std::max(gi, 0), nx - 1), cj = std::min(std::max(gj, 0), ny - 1);
    su[slot] = inside ? u[(size_t)gj * nx + gi] : T(0);
    sk[slot] = k[(size_t)cj * nx + ci];
  }
}

template <class T>
int stencil_tile_mpmd(void** p) {
  // Unpacking prologue (Sec. III, "Parameter packing").
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  int nx = *(int*)p[4], ny = *(int*)p[5];
  T dt = *(T*)p[6], hdt = *(T*)p[7];
  int bc = *(int*)p[8];
  // Launch context from the inserted variables.
  const int BX = block_size.x, BY = block_size.y, TW = BX + 2, TH = BY + 2;
  const int bx = block_index % grid_size.x, by = block_index / grid_size.x;
  T* su = (T*)dynamic_shared_memory;
  T* sk = su + (size_t)TW * TH;
  const int nthreads = BX * BY;

  // Region R0 (loop over the block's threads).
  for (int tid = 0; tid < nthreads; ++tid) {
    int tx = tid % BX, ty = tid / BX;
    int gi = bx * BX + tx, gj = by * BY + ty;
    stage(u, k, nx, ny, bc, gi, gj, su, sk, (ty + 1) * TW + (tx + 1));
    if (tx == 0) stage(u, k, nx, ny, bc, gi - 1, gj, su, sk, (ty + 1) * TW + 0);
    if (tx == BX - 1) stage(u, k, nx, ny, bc, gi + 1, gj, su, sk, (ty + 1) * TW + (BX + 1));
    if (ty == 0) stage(u, k, nx, ny, bc, gi, gj - 1, su, sk, 0 * TW + (tx + 1));
    if (ty == BY - 1) stage(u, k, nx, ny, bc, gi, gj + 1, su, sk, (BY + 1) * TW + (tx + 1));
  }
  // __syncthreads(): the fission point.
  // Region R1.
  for (int tid = 0; tid < nthreads; ++tid) {
    int tx = tid % BX, ty = tid / BX;
    int gi = bx * BX + tx, gj = by * BY + ty;
    if (gi < nx && gj < ny) {
      int c = (ty + 1) * TW + (tx + 1);
      size_t g = (size_t)gj * nx + gi;
      uo[g] = cell_update<T>(su[c], su[c - 1], su[c + 1], su[c - TW], su[c + TW], sk[c],
                             sk[c - 1], sk[c + 1], sk[c - TW], sk[c + TW], s[g], dt, hdt);
    }
  }
  return 0;
}

template <class T>
int run_fission(const T* u0, const T* k, const T* s, int nx, int ny, int steps, T dt, int bc,
                int bx, int by, int pool, int block_per_fetch, T* out) {
  size_t n = (size_t)nx * ny;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  Dim3 grid{(nx + bx - 1) / bx, (ny + by - 1) / by, 1};
  size_t shm = 2 * sizeof(T) * (size_t)(bx + 2) * (by + 2);
  for (int t = 0; t < steps; ++t) {
    const T* ua = a.data();
    T* ub = b.data();
    // Packing prologue: every argument's address in a void* array.
    void* args[9] = {&ua, &ub, &k, &s, &nx, &ny, &dt, &hdt, &bc};
    int rc = launch(stencil_tile_mpmd<T>, args, grid, Dim3{bx, by, 1}, shm, pool, block_per_fetch);
    if (rc) return rc;
    a.swap(b);
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// ---------------------------------------------------------------------------
// The shared-memory temporal-blocked tiled kernel: K steps per launch, K + 1
// barriers, K of them inside the time loop (the multi-barrier class of the
// paper's srad, Sec. V), translated with loop fission
// ---------------------------------------------------------------------------
// SPMD kernel (blockDim = (BX, BY); dynamic shared memory = four
// (BX + 2K) x (BY + 2K) tiles of T: two u levels, kappa, s):
//   R0:  the block's threads stage, in a strided loop over the tile, u, kappa
//        and s of every tile position (tile origin (bx BX - K, by BY - K);
//        boundary rule as in the one-step kernel, s = 0 on a Dirichlet ghost)
//   __syncthreads();
//   for t = 1 .. K:
//     Rt: the threads update, in a strided loop, every position of the
//         shrinking region [t, TW - t) x [t, TH - t) from level t - 1 into
//         level t (the other u tile); a Dirichlet ghost position stays 0
//     __syncthreads();
//   RK+1: the threads write level K of the BX x BY interior (in-grid cells).
// MPMD: the time loop is kept, and each barrier-free region -- R0, each Rt,
// RK+1 -- becomes one loop over the block's threads.  fission = 0 runs all
// regions of a thread before the next thread starts (barriers ignored), for
// the test that shows the split is needed.
template <class T>
int stencil_tilek_mpmd(void** p) {
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  const int nx = *(int*)p[4], ny = *(int*)p[5];
  const T dt = *(T*)p[6], hdt = *(T*)p[7];
  const int bc = *(int*)p[8], K = *(int*)p[9], fission = *(int*)p[10];
  const int BX = block_size.x, BY = block_size.y, TW = BX + 2 * K, TH = BY + 2 * K;
  const int nthreads = BX * BY, ntile = TW * TH;
  const int bx = block_index % grid_size.x, by = block_index / grid_size.x;
  const int gx0 = bx * BX - K, gy0 = by * BY - K;
  const bool periodic = bc == BC_PERIODIC;
  T* lev[2] = {(T*)dynamic_shared_memory, (T*)dynamic_shared_memory + ntile};
  T* kt = lev[1] + ntile;
  T* st = kt + ntile;
  auto in_grid = [&](int gi, int gj) { return gi >= 0 && gi < nx && gj >= 0 && gj < ny; };
  // region bodies for one thread
  auto r0 = [&](int tid) {
    for (int c = tid; c < ntile; c += nthreads) {
      const int gi = gx0 + c % TW, gj = gy0 + c / TW;
      stage(u, k, nx, ny, bc, gi, gj, lev[0], kt, c);
      if (periodic)
        st[c] = s[(size_t)wrap(gj, ny) * nx + wrap(gi, nx)];
      else
        st[c] = in_grid(gi, gj) ? s[(size_t)gj * nx + gi] : T(0);
    }
  };
  auto rt = [&](int tid, int t) {
    const T* a = lev[(t - 1) & 1];
    T* b = lev[t & 1];
    const int w = TW - 2 * t, h = TH - 2 * t;
    for (int q = tid; q < w * h; q += nthreads) {
      const int ti = t + q % w, tj = t + q / w, c = tj * TW + ti;
      if (!periodic && !in_grid(gx0 + ti, gy0 + tj)) {
        b[c] = T(0);
        continue;
      }
      b[c] = cell_update<T>(a[c], a[c - 1], a[c + 1], a[c - TW], a[c + TW], kt[c], kt[c - 1], kt[c + 1],
                            kt[c - TW], kt[c + TW], st[c], dt, hdt);
    }
  };
  auto rlast = [&](int tid) {
    const T* a = lev[K & 1];
    for (int q = tid; q < nthreads; q += nthreads) {
      const int ti = K + q % BX, tj = K + q / BX;
      const int gi = gx0 + ti, gj = gy0 + tj;
      if (gi < nx && gj < ny) uo[(size_t)gj * nx + gi] = a[tj * TW + ti];
    }
  };
  if (fission) {
    for (int tid = 0; tid < nthreads; ++tid) r0(tid);
    // __syncthreads()
    for (int t = 1; t <= K; ++t) {
      for (int tid = 0; tid < nthreads; ++tid) rt(tid, t);
      // __syncthreads()
    }
    for (int tid = 0; tid < nthreads; ++tid) rlast(tid);
  } else {
    for (int tid = 0; tid < nthreads; ++tid) {
      r0(tid);
      for (int t = 1; t <= K; ++t) rt(tid, t);
      rlast(tid);
    }
  }
  return 0;
}

// Passes of depth `depth` (the last takes the rest), one launch each.
template <class T>
int run_tilek(const T* u0, const T* k, const T* s, int nx, int ny, int steps, T dt, int bc, int depth,
              int bx, int by, int pool, int fission, T* out) {
  if (depth < 1 || bx < 1 || by < 1) return 1;
  size_t n = (size_t)nx * ny;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  Dim3 grid{(nx + bx - 1) / bx, (ny + by - 1) / by, 1};
  for (int done = 0; done < steps;) {
    int d = std::min(depth, steps - done);
    size_t shm = 4 * sizeof(T) * (size_t)(bx + 2 * d) * (by + 2 * d);
    const T* ua = a.data();
    T* ub = b.data();
    void* args[11] = {&ua, &ub, &k, &s, &nx, &ny, &dt, &hdt, &bc, &d, &fission};
    int rc = launch(stencil_tilek_mpmd<T>, args, grid, Dim3{bx, by, 1}, shm, pool, 0);
    if (rc) return rc;
    a.swap(b);
    done += d;
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// ---------------------------------------------------------------------------
// BF16-Kahan storage
// ---------------------------------------------------------------------------
// IEEE round-to-nearest-even of a binary32 value to bfloat16 (the upper 16
// bits of binary32), written from the definition: keep the upper half, and
// round up when the discarded lower half exceeds half an ulp, or equals it and
// the kept half is odd.  A carry into the exponent field is the correct
// result (next binade or infinity).  NaN stays NaN (quiet bit set).
inline uint16_t bf16_rn(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu)) return (uint16_t)((b >> 16) | 0x0040u);
  uint32_t hi = b >> 16, lo = b & 0xffffu;
  if (lo > 0x8000u || (lo == 0x8000u && (hi & 1u))) hi += 1u;
  return (uint16_t)hi;
}

inline float bf16_f32(uint16_t h) {
  uint32_t b = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// State word: bits 0..15 = hi, bits 16..31 = cmp; effective value hi - cmp.
inline float eff(uint32_t w) { return bf16_f32((uint16_t)(w & 0xffffu)) - bf16_f32((uint16_t)(w >> 16)); }

// compensate = 0 is the diagnostic without compensation (cmp forced to 0).
void bf16k_rows(const uint32_t* st, uint32_t* so, const uint16_t* k, const uint16_t* s, int nx, int ny,
                float dt, float hdt, int bc, int compensate, int j0, int j1) {
  auto nb = [&](int ii, int jj, float kc, float& un, float& kn) {
    if (bc == BC_PERIODIC) {
      size_t g = (size_t)wrap(jj, ny) * nx + wrap(ii, nx);
      un = eff(st[g]);
      kn = bf16_f32(k[g]);
    } else if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) {
      un = 0.0f;
      kn = kc;
    } else {
      size_t g = (size_t)jj * nx + ii;
      un = eff(st[g]);
      kn = bf16_f32(k[g]);
    }
  };
  for (int j = j0; j < j1; ++j) {
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      float kc = bf16_f32(k[c]), uW, kW, uE, kE, uS, kS, uN, kN;
      nb(i - 1, j, kc, uW, kW);
      nb(i + 1, j, kc, uE, kE);
      nb(i, j - 1, kc, uS, kS);
      nb(i, j + 1, kc, uN, kN);
      float v = cell_update<float>(eff(st[c]), uW, uE, uS, uN, kc, kW, kE, kS, kN, bf16_f32(s[c]),
                                   dt, hdt);
      uint16_t hi = bf16_rn(v);
      uint16_t cm = compensate ? bf16_rn(bf16_f32(hi) - v) : (uint16_t)0;
      so[c] = (uint32_t)hi | ((uint32_t)cm << 16);
    }
  }
}

int bf16k_band_mpmd(void** p) {
  const uint32_t* st = *(const uint32_t**)p[0];
  uint32_t* so = *(uint32_t**)p[1];
  const uint16_t* k = *(const uint16_t**)p[2];
  const uint16_t* s = *(const uint16_t**)p[3];
  int nx = *(int*)p[4], ny = *(int*)p[5];
  float dt = *(float*)p[6], hdt = *(float*)p[7];
  int bc = *(int*)p[8], band = *(int*)p[9], compensate = *(int*)p[10];
  int j0 = block_index * band, j1 = std::min(ny, j0 + band);
  bf16k_rows(st, so, k, s, nx, ny, dt, hdt, bc, compensate, j0, j1);
  return 0;
}

// ---------------------------------------------------------------------------
// Executor self-tests: the paper's two example kernels
// ---------------------------------------------------------------------------
// vecAdd (Listings 1-2): c[id] = a[id] + b[id], id = blockIdx * blockDim + tid.
// A bounds guard (id < n) is added so a ragged last block is allowed.
int vecadd_mpmd(void** p) {
  const double* a = *(const double**)p[0];
  const double* b = *(const double**)p[1];
  double* c = *(double**)p[2];
  int n = *(int*)p[3];
  for (int tid = 0; tid < block_size.x; ++tid) {
    int id = block_index * block_size.x + tid;
    if (id < n) c[id] = a[id] + b[id];
  }
  return 0;
}

// dynamicReverse (Listing 3): s[t] = d[t]; __syncthreads(); d[t] = s[n-t-1].
// Fissioned: one thread loop per region.  Unfissioned: each thread runs both
// regions before the next thread starts, which ignores the barrier.
int reverse_fission_mpmd(void** p) {
  int* d = *(int**)p[0];
  int n = *(int*)p[1];
  int* s = (int*)dynamic_shared_memory;
  for (int t = 0; t < block_size.x; ++t) s[t] = d[t];
  for (int t = 0; t < block_size.x; ++t) d[t] = s[n - t - 1];
  return 0;
}

int reverse_nofission_mpmd(void** p) {
  int* d = *(int**)p[0];
  int n = *(int*)p[1];
  int* s = (int*)dynamic_shared_memory;
  for (int t = 0; t < block_size.x; ++t) {
    s[t] = d[t];
    d[t] = s[n - t - 1];
  }
  return 0;
}

// Accounting kernel: counts how often each block runs; optionally fails.
int count_mpmd(void** p) {
  int* counts = *(int**)p[0];
  int fail_block = *(int*)p[1];
  __atomic_fetch_add(&counts[block_index], 1, __ATOMIC_RELAXED);
  return block_index == fail_block ? 7 : 0;
}

// ---------------------------------------------------------------------------
// Warp-level kernel: a shuffle-based, temporal-blocked strip kernel executed
// with nested loops split at every warp function (Sec. III "SPMD to MPMD": a kernel that
// uses warp-level features is wrapped in an outer loop over the
// ceil(block_size / 32) warps of a block and an inner loop over the 32 lanes
// of a warp, one such nest per code section between warp functions)
// ---------------------------------------------------------------------------
// The SPMD kernel, one warp per (strip, chunk) item, blockDim.x = 32 * W:
//   H = K rounded up to a multiple of 4, OW = 128 - 2H.  The warp's strip
//   covers the 128 columns x0 .. x0 + 127 with x0 = strip * OW - H; lane l
//   holds the 4 columns x0 + 4l .. x0 + 4l + 3.  The item's output rows are
//   [y0, y1) (chunks of `chunk` rows); its input rows y0 - d .. y1 + d - 1.
//   For each input row r:
//     load u, kappa, s of the lane's 4 cells of row r.  Periodic: wrap.
//       Dirichlet: a cell outside the grid is a ghost with u = 0, s = 0 and
//       the kappa of the nearest in-grid cell.
//     kW = shfl_up(kappa[3]), kE = shfl_down(kappa[0])          [warp function]
//     for t = 1 .. d (level t produces row rho = r - t):
//       uW = shfl_up(L[t-1](rho)[3]), uE = shfl_down(L[t-1](rho)[0])
//                                                               [warp function]
//       each of the 4 cells: the canonical update from level t-1's rows
//       rho - 1, rho, rho + 1; Dirichlet ghost cells stay 0
//     level d's row r - d is stored where it lies in [y0, y1), in the grid
//     and in the strip's output columns [x0 + H, x0 + 128 - H).
//   shfl_up / shfl_down with delta 1 over the full warp: a lane with no
//   source lane keeps its own value.  Level t of a strip is exact on the
//   columns [x0 + t, x0 + 128 - t), which contain the output columns.
// MPMD form: the per-lane values that live across a warp function (the level
// rows, the kappa and source rows) are replicated into per-lane arrays; the
// values a warp function exchanges pass through a per-warp array of 32 slots.
// fission = 0 runs every lane's write and read of an exchange in one lane
// loop (the warp function ignored), for the test that shows the split is
// needed.
template <class T>
struct WarpLane {
  // rings indexed by row mod 3 (levels 0 .. K) and row mod (K + 2) (inputs)
  T lev[9][3][4];
  T kap[10][6];  // kW, k0..k3, kE of a row
  T src[10][4];
};

template <class T>
int strip_warp_mpmd(void** p) {
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  const int nx = *(int*)p[4], ny = *(int*)p[5];
  const T dt = *(T*)p[6], hdt = *(T*)p[7];
  const int bc = *(int*)p[8], K = *(int*)p[9], d = *(int*)p[10], chunk = *(int*)p[11];
  const int n_items = *(int*)p[12], fission = *(int*)p[13];
  const int H = (K + 3) & ~3, OW = 128 - 2 * H;
  const int n_strips = (nx + OW - 1) / OW;
  const int n_warps = (block_size.x + 31) / 32;
  const bool periodic = bc == BC_PERIODIC;
  const int RK = K + 2;
  std::vector<WarpLane<T>> lanes(32);
  T x_a[32], x_b[32];  // exchange slots of one warp function

  // Exchange through the per-warp slots.  fission: every lane writes, then
  // every lane reads (two lane loops).  Otherwise one lane loop does both,
  // so a lane reads its east neighbour's slot before that lane has written.
  auto exchange = [&](auto&& put_a, auto&& put_b, auto&& take) {
    if (fission) {
      for (int l = 0; l < 32; ++l) {
        x_a[l] = put_a(l);
        x_b[l] = put_b(l);
      }
      for (int l = 0; l < 32; ++l) take(l, x_a[l > 0 ? l - 1 : l], x_b[l < 31 ? l + 1 : l]);
    } else {
      for (int l = 0; l < 32; ++l) {
        x_a[l] = put_a(l);
        x_b[l] = put_b(l);
        take(l, x_a[l > 0 ? l - 1 : l], x_b[l < 31 ? l + 1 : l]);
      }
    }
  };

  for (int w = 0; w < n_warps; ++w) {  // outer loop: warps of the block
    const int item = block_index * n_warps + w;
    if (item >= n_items) continue;
    const int strip = item % n_strips, ch = item / n_strips;
    const int x0 = strip * OW - H;
    const int y0 = ch * chunk, y1 = std::min(y0 + chunk, ny);
    // Exchange slots start as NaN so a read of an unwritten slot shows.
    for (int l = 0; l < 32; ++l) x_a[l] = x_b[l] = std::numeric_limits<T>::quiet_NaN();
    for (int l = 0; l < 32; ++l)
      for (int t = 0; t < 9; ++t)
        for (int q = 0; q < 3; ++q)
          for (int e = 0; e < 4; ++e) lanes[l].lev[t][q][e] = T(0);

    auto col_in = [&](int x) { return periodic || (x >= 0 && x < nx); };
    auto row_in = [&](int y) { return periodic || (y >= 0 && y < ny); };
    auto mod = [](int a, int m) { int r = a % m; return r < 0 ? r + m : r; };

    for (int r = y0 - d; r < y1 + d; ++r) {
      const int slot = mod(r, RK);
      // Section 1 (lane loop) + kappa exchange: load the input row, then
      // kW / kE from the lanes to the west / east.
      auto load = [&](int l) {
        WarpLane<T>& L = lanes[l];
        const int rr = periodic ? mod(r, ny) : std::min(std::max(r, 0), ny - 1);
        for (int e = 0; e < 4; ++e) {
          const int x = x0 + 4 * l + e;
          const int xx = periodic ? mod(x, nx) : std::min(std::max(x, 0), nx - 1);
          const size_t g = (size_t)rr * nx + xx;
          const bool in = col_in(x) && row_in(r);
          L.kap[slot][1 + e] = k[g];
          L.src[slot][e] = in ? s[g] : T(0);
          L.lev[0][mod(r, 3)][e] = in ? u[g] : T(0);
        }
        return T(0);
      };
      for (int l = 0; l < 32; ++l) load(l);
      exchange([&](int l) { return lanes[l].kap[slot][4]; }, [&](int l) { return lanes[l].kap[slot][1]; },
               [&](int l, T west, T east) {
                 lanes[l].kap[slot][0] = west;
                 lanes[l].kap[slot][5] = east;
               });
      for (int t = 1; t <= d; ++t) {
        const int rho = r - t;
        const int cs = mod(rho, 3), ss = mod(rho - 1, 3), ns = mod(rho + 1, 3);
        const int ks = mod(rho, RK), kss = mod(rho - 1, RK), kns = mod(rho + 1, RK);
        // u exchange of level t-1's row rho, then the update (section t).
        exchange([&](int l) { return lanes[l].lev[t - 1][cs][3]; },
                 [&](int l) { return lanes[l].lev[t - 1][cs][0]; },
                 [&](int l, T uWl, T uEl) {
                   WarpLane<T>& L = lanes[l];
                   T out[4];
                   for (int e = 0; e < 4; ++e) {
                     const int x = x0 + 4 * l + e;
                     if (!col_in(x) || !row_in(rho)) {
                       out[e] = T(0);
                       continue;
                     }
                     const T c = L.lev[t - 1][cs][e];
                     const T kc = L.kap[ks][1 + e];
                     const T uW = e > 0 ? L.lev[t - 1][cs][e - 1] : uWl;
                     const T uE = e < 3 ? L.lev[t - 1][cs][e + 1] : uEl;
                     const T kW = L.kap[ks][e], kE = L.kap[ks][e + 2];
                     const T uS = L.lev[t - 1][ss][e], uN = L.lev[t - 1][ns][e];
                     const T kS = L.kap[kss][1 + e], kN = L.kap[kns][1 + e];
                     out[e] = cell_update<T>(c, uW, uE, uS, uN, kc, kW, kE, kS, kN, L.src[ks][e], dt, hdt);
                   }
                   for (int e = 0; e < 4; ++e) L.lev[t][cs][e] = out[e];
                 });
      }
      // Section d+1: store level d's row r - d.
      const int ro = r - d;
      if (ro >= y0 && ro < y1) {
        for (int l = 0; l < 32; ++l) {
          for (int e = 0; e < 4; ++e) {
            const int x = x0 + 4 * l + e;
            if (x >= x0 + H && x < x0 + 128 - H && x >= 0 && x < nx)
              uo[(size_t)ro * nx + x] = lanes[l].lev[d][mod(ro, 3)][e];
          }
        }
      }
    }
  }
  return 0;
}

// Runs `steps` steps in passes of depth K (the last pass takes the rest),
// one launch of the strip kernel per pass, W warps per block.
template <class T>
int run_strip_warp(const T* u0, const T* k, const T* s, int nx, int ny, int steps, T dt, int bc, int K,
                   int chunk, int W, int pool, int fission, T* out) {
  if (K < 1 || K > 8 || chunk < 1 || W < 1 || W > 32) return 1;
  size_t n = (size_t)nx * ny;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  const int H = (K + 3) & ~3, OW = 128 - 2 * H;
  const int n_items = ((nx + OW - 1) / OW) * ((ny + chunk - 1) / chunk);
  for (int done = 0; done < steps;) {
    int d = std::min(K, steps - done);
    const T* ua = a.data();
    T* ub = b.data();
    void* args[14] = {&ua, &ub, &k, &s, &nx, &ny, &dt, &hdt, &bc, &K, &d, &chunk, (void*)&n_items, &fission};
    int rc = launch(strip_warp_mpmd<T>, args, Dim3{(n_items + W - 1) / W, 1, 1}, Dim3{32 * W, 1, 1}, 0, pool, 0);
    if (rc) return rc;
    a.swap(b);
    done += d;
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// ---------------------------------------------------------------------------
// 3-D 7-point variant (the paper's hotspot3D class) and its z-marching tiled
// kernel with two barriers inside a loop
// ---------------------------------------------------------------------------
// Canonical 3-D update (a stated reading, the 2-D update with a third pair of
// faces): D = (i, j, k-1), U = (i, j, k+1),
//   acc = ((fW + fE) + (fS + fN)) + (fD + fU),   u' = c + (hdt * acc + dt * s)
// with the same face fluxes and boundary rules as in 2-D.  Layout
// u[k][j][i], x fastest.
template <class T>
inline T cell_update3(T c, const T un[6], const T kn[6], T kc, T s, T dt, T hdt) {
  T f[6];
  for (int q = 0; q < 6; ++q) f[q] = (kc + kn[q]) * (un[q] - c);
  T acc = ((f[0] + f[1]) + (f[2] + f[3])) + (f[4] + f[5]);
  return c + (hdt * acc + dt * s);
}

// u and kappa seen across the face from a cell towards (ii, jj, kk).
template <class T>
inline void neighbour3(const T* u, const T* k, int nx, int ny, int nz, int bc, int ii, int jj, int kk,
                       T kc, T& un, T& kn) {
  if (bc == BC_PERIODIC) {
    size_t g = ((size_t)wrap(kk, nz) * ny + wrap(jj, ny)) * nx + wrap(ii, nx);
    un = u[g];
    kn = k[g];
  } else if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) {
    un = T(0);
    kn = kc;
  } else {
    size_t g = ((size_t)kk * ny + jj) * nx + ii;
    un = u[g];
    kn = k[g];
  }
}

template <class T>
void direct3_planes(const T* u, T* uo, const T* k, const T* s, int nx, int ny, int nz, T dt, T hdt,
                    int bc, int k0, int k1) {
  const int di[6] = {-1, 1, 0, 0, 0, 0}, dj[6] = {0, 0, -1, 1, 0, 0}, dk[6] = {0, 0, 0, 0, -1, 1};
  for (int kk = k0; kk < k1; ++kk)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t c = ((size_t)kk * ny + j) * nx + i;
        T kc = k[c], un[6], kn[6];
        for (int q = 0; q < 6; ++q)
          neighbour3(u, k, nx, ny, nz, bc, i + di[q], j + dj[q], kk + dk[q], kc, un[q], kn[q]);
        uo[c] = cell_update3<T>(u[c], un, kn, kc, s[c], dt, hdt);
      }
}

template <class T>
int direct3_band_mpmd(void** p) {
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  int nx = *(int*)p[4], ny = *(int*)p[5], nz = *(int*)p[6];
  T dt = *(T*)p[7], hdt = *(T*)p[8];
  int bc = *(int*)p[9], band = *(int*)p[10];
  int k0 = block_index * band, k1 = std::min(nz, k0 + band);
  direct3_planes<T>(u, uo, k, s, nx, ny, nz, dt, hdt, bc, k0, k1);
  return 0;
}

template <class T>
int run_direct3(const T* u0, const T* k, const T* s, int nx, int ny, int nz, int steps, T dt, int bc,
                int pool, T* out) {
  size_t n = (size_t)nx * ny * nz;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  for (int t = 0; t < steps; ++t) {
    if (pool <= 1) {
      direct3_planes<T>(a.data(), b.data(), k, s, nx, ny, nz, dt, hdt, bc, 0, nz);
    } else {
      const T* ua = a.data();
      T* ub = b.data();
      int band = std::max(1, (nz + 2 * pool - 1) / (2 * pool));
      void* args[11] = {&ua, &ub, &k, &s, &nx, &ny, &nz, &dt, &hdt, &bc, &band};
      int rc = launch(direct3_band_mpmd<T>, args, Dim3{(nz + band - 1) / band, 1, 1}, Dim3{1, 1, 1}, 0,
                      pool, 0);
      if (rc) return rc;
    }
    a.swap(b);
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// The z-marching tiled SPMD kernel (blockDim = (BX, BY), grid = (ceil(nx/BX),
// ceil(ny/BY), ZC); block (bx, by, bz) owns the column tile and the planes
// [bz*PZ, min(nz, (bz+1)*PZ)), PZ = ceil(nz / ZC); dynamic shared memory =
// two (BX+2)*(BY+2) tiles of T).  Each thread keeps its cell's u and kappa of
// planes k-1, k, k+1 and s of plane k in registers:
//   prologue: load planes z0 - 1 and z0 (boundary rule for planes outside).
//   for k = z0 .. z1-1:
//     R0: load plane k+1 into registers; stage plane k of u and kappa into
//         the tiles (edge threads also stage the in-plane halo cell in their
//         direction, boundary rule as in 2-D)
//     __syncthreads();
//     R1: if the cell is in the grid: the update from the tile (in-plane
//         neighbours) and the registers (planes k-1, k+1); write u_out;
//         rotate the register planes (k-1 <- k <- k+1)
//     __syncthreads();
// MPMD: both barriers sit inside the k loop, so the loop over k is kept and
// each of its two barrier-free regions becomes one loop over the block's
// threads; the per-thread register planes live across the barriers and are
// replicated into per-thread arrays.
template <class T>
int stencil3_tile_mpmd(void** p) {
  const T* u = *(const T**)p[0];
  T* uo = *(T**)p[1];
  const T* k = *(const T**)p[2];
  const T* s = *(const T**)p[3];
  const int nx = *(int*)p[4], ny = *(int*)p[5], nz = *(int*)p[6];
  const T dt = *(T*)p[7], hdt = *(T*)p[8];
  const int bc = *(int*)p[9];
  const int BX = block_size.x, BY = block_size.y, TW = BX + 2, TH = BY + 2;
  const int gx = grid_size.x, gy = grid_size.y, ZC = grid_size.z;
  const int bx = block_index % gx, by = (block_index / gx) % gy, bz = block_index / (gx * gy);
  const int PZ = (nz + ZC - 1) / ZC, z0 = bz * PZ, z1 = std::min(nz, z0 + PZ);
  if (z0 >= z1) return 0;
  T* su = (T*)dynamic_shared_memory;
  T* sk = su + (size_t)TW * TH;
  const int nthreads = BX * BY;
  const bool periodic = bc == BC_PERIODIC;
  // per-thread register planes: u and kappa of planes k-1, k, k+1
  std::vector<T> um(nthreads), uc(nthreads), up(nthreads), km(nthreads), kc(nthreads), kp(nthreads);
  // Value of (gi, gj, kk) under the boundary rule: Dirichlet ghosts have u = 0
  // and kappa of the nearest in-grid cell.
  auto fetch = [&](int gi, int gj, int kk, T& uv, T& kv) {
    if (periodic) {
      size_t g = ((size_t)wrap(kk, nz) * ny + wrap(gj, ny)) * nx + wrap(gi, nx);
      uv = u[g];
      kv = k[g];
    } else {
      bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny && kk >= 0 && kk < nz;
      int ci = std::min(std::max(gi, 0), nx - 1), cj = std::min(std::max(gj, 0), ny - 1);
      int ck = std::min(std::max(kk, 0), nz - 1);
      uv = in ? u[((size_t)kk * ny + gj) * nx + gi] : T(0);
      kv = k[((size_t)ck * ny + cj) * nx + ci];
    }
  };
  auto stage = [&](int gi, int gj, int kk, int slot) { fetch(gi, gj, kk, su[slot], sk[slot]); };
  // prologue (one region, no barrier yet)
  for (int tid = 0; tid < nthreads; ++tid) {
    int gi = bx * BX + tid % BX, gj = by * BY + tid / BX;
    fetch(gi, gj, z0 - 1, um[tid], km[tid]);
    fetch(gi, gj, z0, uc[tid], kc[tid]);
  }
  for (int kk = z0; kk < z1; ++kk) {
    // R0
    for (int tid = 0; tid < nthreads; ++tid) {
      int tx = tid % BX, ty = tid / BX;
      int gi = bx * BX + tx, gj = by * BY + ty;
      fetch(gi, gj, kk + 1, up[tid], kp[tid]);
      int c = (ty + 1) * TW + (tx + 1);
      su[c] = uc[tid];
      sk[c] = kc[tid];
      if (tx == 0) stage(gi - 1, gj, kk, c - 1);
      if (tx == BX - 1) stage(gi + 1, gj, kk, c + 1);
      if (ty == 0) stage(gi, gj - 1, kk, c - TW);
      if (ty == BY - 1) stage(gi, gj + 1, kk, c + TW);
    }
    // __syncthreads()
    // R1
    for (int tid = 0; tid < nthreads; ++tid) {
      int tx = tid % BX, ty = tid / BX;
      int gi = bx * BX + tx, gj = by * BY + ty;
      if (gi < nx && gj < ny) {
        int c = (ty + 1) * TW + (tx + 1);
        size_t g = ((size_t)kk * ny + gj) * nx + gi;
        const T un[6] = {su[c - 1], su[c + 1], su[c - TW], su[c + TW], um[tid], up[tid]};
        const T kn[6] = {sk[c - 1], sk[c + 1], sk[c - TW], sk[c + TW], km[tid], kp[tid]};
        uo[g] = cell_update3<T>(su[c], un, kn, sk[c], s[g], dt, hdt);
      }
      um[tid] = uc[tid];
      km[tid] = kc[tid];
      uc[tid] = up[tid];
      kc[tid] = kp[tid];
    }
    // __syncthreads(): the next R0 overwrites the tiles
  }
  return 0;
}

template <class T>
int run_fission3(const T* u0, const T* k, const T* s, int nx, int ny, int nz, int steps, T dt, int bc,
                 int bx, int by, int zc, int pool, T* out) {
  size_t n = (size_t)nx * ny * nz;
  T hdt = T(0.5) * dt;
  std::vector<T> a(u0, u0 + n), b(n);
  Dim3 grid{(nx + bx - 1) / bx, (ny + by - 1) / by, zc};
  size_t shm = 2 * sizeof(T) * (size_t)(bx + 2) * (by + 2);
  for (int t = 0; t < steps; ++t) {
    const T* ua = a.data();
    T* ub = b.data();
    void* args[10] = {&ua, &ub, &k, &s, &nx, &ny, &nz, &dt, &hdt, &bc};
    int rc = launch(stencil3_tile_mpmd<T>, args, grid, Dim3{bx, by, 1}, shm, pool, 0);
    if (rc) return rc;
    a.swap(b);
  }
  std::memcpy(out, a.data(), n * sizeof(T));
  return 0;
}

// ---------------------------------------------------------------------------
// Adjoint (FP64)
// ---------------------------------------------------------------------------
// Step: u_{n+1} = u_n + dt * D(kappa) u_n + dt * s with D symmetric, so
// lambda_n = lambda_{n+1} + dt * D(kappa) lambda_{n+1} (the same update with
// s = 0), dL/du_0 = lambda_0, and per face (c, f) and step:
//   interior face: dL/dkappa_c += hdt * (u_f - u_c) * (lambda_c - lambda_f)
//   Dirichlet boundary face (conductivity 2 kappa_c): dL/dkappa_c += dt * (0 - u_c) * lambda_c
// with u = u_n and lambda = lambda_{n+1}.
void kappa_grad_step(const double* u, const double* lam, double* gk, int nx, int ny, double dt, int bc) {
  double hdt = 0.5 * dt;
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      size_t c = (size_t)j * nx + i;
      double g = 0.0;
      for (int d = 0; d < 4; ++d) {
        int ii = i + di[d], jj = j + dj[d];
        if (bc == BC_PERIODIC) {
          size_t f = (size_t)wrap(jj, ny) * nx + wrap(ii, nx);
          g += hdt * (u[f] - u[c]) * (lam[c] - lam[f]);
        } else if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) {
          g += dt * (0.0 - u[c]) * lam[c];
        } else {
          size_t f = (size_t)jj * nx + ii;
          g += hdt * (u[f] - u[c]) * (lam[c] - lam[f]);
        }
      }
      gk[c] += g;
    }
  }
}

}  // namespace

extern "C" {

int orc_version(void) { return 1; }

// Direct loop.  pool <= 1: serial; else row bands on the thread pool.
int orc_direct_f64(const double* u0, const double* k, const double* s, int nx, int ny, int steps,
                   double dt, int bc, int pool, double* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_direct<double>(u0, k, s, nx, ny, steps, dt, bc, pool, out);
}

int orc_direct_f32(const float* u0, const float* k, const float* s, int nx, int ny, int steps,
                   float dt, int bc, int pool, float* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_direct<float>(u0, k, s, nx, ny, steps, dt, bc, pool, out);
}

// The tiled kernel executed block by block with loop fission at the barrier.
int orc_fission_f64(const double* u0, const double* k, const double* s, int nx, int ny, int steps,
                    double dt, int bc, int bx, int by, int pool, int block_per_fetch, double* out) {
  if (nx < 1 || ny < 1 || steps < 0 || bx < 1 || by < 1) return 1;
  return run_fission<double>(u0, k, s, nx, ny, steps, dt, bc, bx, by, pool, block_per_fetch, out);
}

int orc_fission_f32(const float* u0, const float* k, const float* s, int nx, int ny, int steps,
                    float dt, int bc, int bx, int by, int pool, int block_per_fetch, float* out) {
  if (nx < 1 || ny < 1 || steps < 0 || bx < 1 || by < 1) return 1;
  return run_fission<float>(u0, k, s, nx, ny, steps, dt, bc, bx, by, pool, block_per_fetch, out);
}

// BF16-Kahan direct loop.  state: nx*ny words (hi | cmp << 16).
int orc_direct_bf16k(const uint32_t* st0, const uint16_t* k, const uint16_t* s, int nx, int ny,
                     int steps, float dt, int bc, int compensate, int pool, uint32_t* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  size_t n = (size_t)nx * ny;
  float hdt = 0.5f * dt;
  std::vector<uint32_t> a(st0, st0 + n), b(n);
  for (int t = 0; t < steps; ++t) {
    if (pool <= 1) {
      bf16k_rows(a.data(), b.data(), k, s, nx, ny, dt, hdt, bc, compensate, 0, ny);
    } else {
      const uint32_t* ua = a.data();
      uint32_t* ub = b.data();
      int band = std::max(1, (ny + 4 * pool - 1) / (4 * pool));
      void* args[11] = {&ua, &ub, &k, &s, &nx, &ny, &dt, &hdt, &bc, &band, &compensate};
      int rc = launch(bf16k_band_mpmd, args, Dim3{(ny + band - 1) / band, 1, 1}, Dim3{1, 1, 1}, 0,
                      pool, 0);
      if (rc) return rc;
    }
    a.swap(b);
  }
  std::memcpy(out, a.data(), n * sizeof(uint32_t));
  return 0;
}

void orc_bf16_round(const float* x, uint16_t* out, long long n) {
  for (long long i = 0; i < n; ++i) out[i] = bf16_rn(x[i]);
}

// Heat sums: plain sequential FP64 accumulation.
double orc_heat_sum_f32(const float* u, long long n) {
  double acc = 0.0;
  for (long long i = 0; i < n; ++i) acc += (double)u[i];
  return acc;
}

double orc_heat_sum_f64(const double* u, long long n) {
  double acc = 0.0;
  for (long long i = 0; i < n; ++i) acc += u[i];
  return acc;
}

// BF16-Kahan: the exact per-cell value (double)hi - (double)cmp, summed in FP64.
double orc_heat_sum_bf16k(const uint32_t* st, long long n) {
  double acc = 0.0;
  for (long long i = 0; i < n; ++i)
    acc += (double)bf16_f32((uint16_t)(st[i] & 0xffffu)) - (double)bf16_f32((uint16_t)(st[i] >> 16));
  return acc;
}

}  // extern "C"

namespace {
// Value after `steps` steps of each sampled cell, computed on its dependency
// cone only (a (2*steps+1)^2 window around the cell), FP32 arithmetic.
// idx: flat indices j*nx + i.  Same per-cell expression and boundary rule as
// the direct loop, so the result is bit-identical to the full-grid run.
template <class T>
int sample_cone(const T* u0, const T* k, const T* s, int nx, int ny, int steps, T dt, int bc,
                const long long* idx, int nidx, T* out) {
  const int R = steps, W = 2 * R + 1;
  T hdt = T(0.5) * dt;
  std::vector<T> a((size_t)W * W), b((size_t)W * W), kw((size_t)W * W), sw((size_t)W * W);
  std::vector<unsigned char> in((size_t)W * W);
  for (int q = 0; q < nidx; ++q) {
    int i0 = (int)(idx[q] % nx), j0 = (int)(idx[q] / nx);
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx) {
        size_t w = (size_t)(dy + R) * W + (dx + R);
        int gi = i0 + dx, gj = j0 + dy;
        bool inside = bc == BC_PERIODIC || (gi >= 0 && gi < nx && gj >= 0 && gj < ny);
        in[w] = inside;
        if (inside) {
          size_t g = (size_t)wrap(gj, ny) * nx + wrap(gi, nx);
          a[w] = u0[g];
          kw[w] = k[g];
          sw[w] = s[g];
        } else {
          a[w] = T(0);
          kw[w] = T(0);
          sw[w] = T(0);
        }
      }
    for (int t = 1; t <= R; ++t) {
      int r = R - t;
      for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) {
          size_t w = (size_t)(dy + R) * W + (dx + R);
          if (!in[w]) {
            b[w] = T(0);
            continue;
          }
          T kc = kw[w];
          auto nbv = [&](size_t v, T& un, T& kn) {
            if (in[v]) {
              un = a[v];
              kn = kw[v];
            } else {
              un = T(0);
              kn = kc;
            }
          };
          T uW, kW, uE, kE, uS, kS, uN, kN;
          nbv(w - 1, uW, kW);
          nbv(w + 1, uE, kE);
          nbv(w - W, uS, kS);
          nbv(w + W, uN, kN);
          b[w] = cell_update<T>(a[w], uW, uE, uS, uN, kc, kW, kE, kS, kN, sw[w], dt, hdt);
        }
      a.swap(b);
    }
    out[q] = a[(size_t)R * W + R];
  }
  return 0;
}

}  // namespace

extern "C" {

int orc_sample_f32(const float* u0, const float* k, const float* s, int nx, int ny, int steps,
                   float dt, int bc, const long long* idx, int nidx, float* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return sample_cone<float>(u0, k, s, nx, ny, steps, dt, bc, idx, nidx, out);
}

int orc_sample_f64(const double* u0, const double* k, const double* s, int nx, int ny, int steps,
                   double dt, int bc, const long long* idx, int nidx, double* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return sample_cone<double>(u0, k, s, nx, ny, steps, dt, bc, idx, nidx, out);
}

// FP64 adjoint with checkpoints every `ckpt` steps (segments recomputed in
// the backward sweep).  Returns the loss 0.5 ||u_T - target||^2 in *loss.
int orc_adjoint_f64(const double* u0, const double* k, const double* s, const double* target, int nx,
                    int ny, int steps, double dt, int bc, int ckpt, int pool, double* grad_u0,
                    double* grad_k, double* loss) {
  if (nx < 1 || ny < 1 || steps < 0 || ckpt < 1) return 1;
  size_t n = (size_t)nx * ny;
  int nseg = (steps + ckpt - 1) / ckpt;
  std::vector<std::vector<double>> cks(std::max(nseg, 1));
  std::vector<double> cur(u0, u0 + n), nxt(n);
  for (int m = 0; m < nseg; ++m) {
    cks[m] = cur;
    int len = std::min(ckpt, steps - m * ckpt);
    int rc = run_direct<double>(cur.data(), k, s, nx, ny, len, dt, bc, pool, nxt.data());
    if (rc) return rc;
    cur.swap(nxt);
  }
  double L = 0.0;
  std::vector<double> lam(n), lam2(n), zero(n, 0.0);
  for (size_t c = 0; c < n; ++c) {
    double r = cur[c] - target[c];
    L += 0.5 * r * r;
    lam[c] = r;
  }
  std::fill(grad_k, grad_k + n, 0.0);
  std::vector<std::vector<double>> seg;
  for (int m = nseg - 1; m >= 0; --m) {
    int a = m * ckpt, len = std::min(ckpt, steps - a);
    seg.assign(len, std::vector<double>());
    seg[0] = cks[m];
    for (int q = 1; q < len; ++q) {
      seg[q].resize(n);
      int rc = run_direct<double>(seg[q - 1].data(), k, s, nx, ny, 1, dt, bc, pool, seg[q].data());
      if (rc) return rc;
    }
    for (int q = len - 1; q >= 0; --q) {
      kappa_grad_step(seg[q].data(), lam.data(), grad_k, nx, ny, dt, bc);
      int rc = run_direct<double>(lam.data(), k, zero.data(), nx, ny, 1, dt, bc, pool, lam2.data());
      if (rc) return rc;
      lam.swap(lam2);
    }
  }
  std::memcpy(grad_u0, lam.data(), n * sizeof(double));
  *loss = L;
  return 0;
}

// The warp-level strip kernel (K <= 8, the depths of the GPU path).
int orc_strip_warp_f32(const float* u0, const float* k, const float* s, int nx, int ny, int steps,
                       float dt, int bc, int K, int chunk, int warps, int pool, int fission, float* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_strip_warp<float>(u0, k, s, nx, ny, steps, dt, bc, K, chunk, warps, pool, fission, out);
}

int orc_strip_warp_f64(const double* u0, const double* k, const double* s, int nx, int ny, int steps,
                       double dt, int bc, int K, int chunk, int warps, int pool, int fission, double* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_strip_warp<double>(u0, k, s, nx, ny, steps, dt, bc, K, chunk, warps, pool, fission, out);
}

// The shared-memory temporal-blocked tiled kernel (multi-barrier).
int orc_tilek_f32(const float* u0, const float* k, const float* s, int nx, int ny, int steps, float dt,
                  int bc, int depth, int bx, int by, int pool, int fission, float* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_tilek<float>(u0, k, s, nx, ny, steps, dt, bc, depth, bx, by, pool, fission, out);
}

int orc_tilek_f64(const double* u0, const double* k, const double* s, int nx, int ny, int steps, double dt,
                  int bc, int depth, int bx, int by, int pool, int fission, double* out) {
  if (nx < 1 || ny < 1 || steps < 0) return 1;
  return run_tilek<double>(u0, k, s, nx, ny, steps, dt, bc, depth, bx, by, pool, fission, out);
}

// 3-D 7-point variant.
int orc_direct3_f32(const float* u0, const float* k, const float* s, int nx, int ny, int nz, int steps,
                    float dt, int bc, int pool, float* out) {
  if (nx < 1 || ny < 1 || nz < 1 || steps < 0) return 1;
  return run_direct3<float>(u0, k, s, nx, ny, nz, steps, dt, bc, pool, out);
}

int orc_direct3_f64(const double* u0, const double* k, const double* s, int nx, int ny, int nz,
                    int steps, double dt, int bc, int pool, double* out) {
  if (nx < 1 || ny < 1 || nz < 1 || steps < 0) return 1;
  return run_direct3<double>(u0, k, s, nx, ny, nz, steps, dt, bc, pool, out);
}

int orc_fission3_f32(const float* u0, const float* k, const float* s, int nx, int ny, int nz, int steps,
                     float dt, int bc, int bx, int by, int zc, int pool, float* out) {
  if (nx < 1 || ny < 1 || nz < 1 || steps < 0 || bx < 1 || by < 1 || zc < 1) return 1;
  return run_fission3<float>(u0, k, s, nx, ny, nz, steps, dt, bc, bx, by, zc, pool, out);
}

int orc_fission3_f64(const double* u0, const double* k, const double* s, int nx, int ny, int nz,
                     int steps, double dt, int bc, int bx, int by, int zc, int pool, double* out) {
  if (nx < 1 || ny < 1 || nz < 1 || steps < 0 || bx < 1 || by < 1 || zc < 1) return 1;
  return run_fission3<double>(u0, k, s, nx, ny, nz, steps, dt, bc, bx, by, zc, pool, out);
}

// Executor self-tests.
int orc_vecadd(const double* a, const double* b, double* c, int n, int grid, int block, int pool) {
  void* args[4] = {&a, &b, &c, &n};
  return launch(vecadd_mpmd, args, Dim3{grid, 1, 1}, Dim3{block, 1, 1}, 0, pool, 0);
}

int orc_dynamic_reverse(int* d, int n, int fission) {
  void* args[2] = {&d, &n};
  return launch(fission ? reverse_fission_mpmd : reverse_nofission_mpmd, args, Dim3{1, 1, 1},
                Dim3{n, 1, 1}, (size_t)n * sizeof(int), 1, 0);
}

// Runs the accounting kernel over `grid` blocks; counts[b] = times block b
// ran; *fetches = number of queue fetches.  Returns the kernel's error code
// (7 if fail_block >= 0 was reached).
int orc_fetch_accounting(int grid, int pool, int block_per_fetch, int fail_block, int* counts,
                         int* fetches) {
  std::fill(counts, counts + grid, 0);
  void* args[2] = {&counts, &fail_block};
  return launch(count_mpmd, args, Dim3{grid, 1, 1}, Dim3{1, 1, 1}, 0, pool, block_per_fetch, fetches);
}

}  // extern "C"
