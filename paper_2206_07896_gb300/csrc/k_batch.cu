// Batched persistent stencil: thousands of independent grids of uneven sizes
// and step counts in ONE launch.
//
// The launch is the GPU counterpart of the paper's runtime (Sec. IV): instead
// of a host thread pool fetching blocks from a mutex-protected task queue in
// grains of block_per_fetch ("coarse-grained fetching"), resident CTAs fetch
// grids from a device work queue with one atomicAdd per grain of `grain`
// grids.  The host orders the queue longest-first (LPT) so the expensive grids
// start early.  Two queues:
//   large grids (cells >= team_cells): a whole CTA per grid; its warps split the
//     (strip, chunk) items of each pass and meet at __syncthreads between
//     passes;
//   small grids: one warp per grid, passes separated by __syncwarp.
// Each pass is the streaming temporal-blocked routine of the single-grid path
// (stream_item) with u read through L2 (.cg), because a grid's buffers are
// rewritten by later passes of the same launch.  A grid's u_in is its
// ping-pong partner (clobbered), and the pass count is made odd so the result
// lands in u_out.  No CTA ever waits on another CTA, so there is no inter-CTA
// wait to bound.  Invalid descriptors are skipped and reported in the status
// word (work[2] = CPB_ERR_INVALID_VALUE).
#include "k_stream.cuh"

namespace cpb {
namespace {

constexpr int BATCH_STAGES = 2;  // TMA ring slots per warp
constexpr int BATCH_MAX_TEAMS = 15;  // named barriers 1..15 for multi-warp teams

// Temporal depths the batched kernel is built for, and the largest CTA of
// each: one CTA per SM, and the registers of depth 8 (rows in pairs) allow
// at most 256 threads.
template <int K>
struct BatchDepth {
  static constexpr int MAX_THREADS = K <= 4 ? 384 : 256;
};

// Depth of pass i of a grid with S steps at depth K, with the pass count made
// odd (split the last pass, or, if it has depth 1, the one before it).
__device__ __forceinline__ int npasses(int S, int K) {
  const int P = (S + K - 1) / K;
  return (P % 2 == 0) ? P + 1 : P;
}

__device__ __forceinline__ int pass_depth(int i, int S, int K) {
  const int P = (S + K - 1) / K;
  const int dl = S - (P - 1) * K;  // depth of the last regular pass
  if (P % 2 == 1) return i < P - 1 ? K : dl;
  if (dl >= 2) {  // split the last pass
    if (i < P - 1) return K;
    return i == P - 1 ? dl - dl / 2 : dl / 2;
  }
  // dl == 1: split pass P-2 (depth K >= 2)
  if (i < P - 2) return K;
  if (i == P - 2) return K - K / 2;
  if (i == P - 1) return K / 2;
  return 1;
}

__device__ __forceinline__ bool desc_ok(const cpb_grid_desc& g) {
  return g.nx >= 1 && g.ny >= 1 && g.steps >= 0 && g.u_in && g.u_out && g.kappa &&
         g.u_in != g.u_out && g.dt > 0.0f;
}

// Chunk height for a team of nw warps: choose the number of chunks that best
// balances items over warps, discounting the 2*d halo rows each chunk re-reads.
__device__ __forceinline__ int team_chunk_rows(int ny, int strips, int nw, int d) {
  if (nw == 1) return ny;
  int best = ny;
  float best_eff = -1.0f;
  for (int c = 1; c <= 8; ++c) {
    int chunks = (c * nw + strips - 1) / strips;
    if (chunks > ny) chunks = ny;
    const int rows = (ny + chunks - 1) / chunks;
    const int items = strips * ((ny + rows - 1) / rows);
    const int rounds = (items + nw - 1) / nw;
    const float eff = (float)items / (float)(rounds * nw) * (float)rows / (float)(rows + 2 * d);
    if (eff > best_eff + 1e-4f) {
      best_eff = eff;
      best = rows;
    }
  }
  return best;
}

// A team of warps that works on one grid at a time: the whole CTA (bar 0,
// __syncthreads), one warp (__syncwarp), or `threads / 32` consecutive warps
// of a CTA that meet at named barrier `bar` (1 + the team's index).  Every
// warp of a team takes the same path through a grid, so each barrier is
// reached by exactly `threads` threads.
struct Team {
  int bar;
  int threads;
};

__device__ __forceinline__ void team_sync(const Team& t) {
  if (t.threads == 32)
    __syncwarp();
  else if (t.bar == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(t.bar), "r"(t.threads) : "memory");
}

// Run all steps of one grid with a team of nw warps (wib: this warp's index in
// the team).  sm: this warp's row ring, mbarriers and face ring; tma_ok: the
// warp's ring is usable (cleared for the rest of the launch if a bounded wait
// expired).
template <int K>
__device__ void run_grid(const cpb_grid_desc& g, int bc, int wib, int nw, int lane, int* status,
                         const BulkSmem<K, false>& sm, bool& tma_ok, const BatchDebug& dbg, const Team& team) {
  if (!desc_ok(g)) {
    if (lane == 0 && wib == 0) atomicExch(status, (int)CPB_ERR_INVALID_VALUE);
    return;
  }
  const int nx = g.nx, ny = g.ny, S = g.steps;
  const size_t n = (size_t)nx * ny;
  if (S == 0) {
    const int tid = wib * 32 + lane, nt = nw * 32;
    for (size_t i = tid; i < n; i += nt) {
      const size_t j = CPB_CHK(i, 1, n);
      static_cast<float*>(g.u_out)[j] = __ldcg(static_cast<const float*>(g.u_in) + j);
    }
    team_sync(team);
    return;
  }
  constexpr int HALO = (K + 3) & ~3;
  constexpr int OW = 128 - 2 * HALO;
  StreamArgs a;
  a.kappa = g.kappa;
  a.src = g.src;
  a.nx = nx;
  a.ny = ny;
  a.dt = g.dt;
  a.hdt = 0.5f * g.dt;
  a.bc = bc;
  const uintptr_t al = reinterpret_cast<uintptr_t>(g.u_in) | reinterpret_cast<uintptr_t>(g.u_out) |
                       reinterpret_cast<uintptr_t>(g.kappa) | reinterpret_cast<uintptr_t>(g.src);
  a.vec = (nx % 4 == 0) && (al % 16 == 0);
  a.n_strips = (nx + OW - 1) / OW;
  a.stages = BATCH_STAGES;
  a.wait_limit = dbg.wait_limit;
  a.inject_on = dbg.inject_on;
  a.inject_row = dbg.inject_row;
  // Rows through the TMA ring when the grid allows it (see bulk_eligible in
  // api.cu); otherwise each lane loads its row slices itself.
  const bool bulk = a.vec && nx >= 128;
  const int P = npasses(S, K);
  const void* src_buf = g.u_in;
  for (int i = 0; i < P; ++i) {
    void* dst = ((P - 1 - i) % 2 == 0) ? g.u_out : g.u_in;
    a.u_in = src_buf;
    a.u_out = dst;
    a.depth = pass_depth(i, S, K);
    a.chunk_rows = team_chunk_rows(ny, a.n_strips, nw, a.depth);
    a.n_items = a.n_strips * ((ny + a.chunk_rows - 1) / a.chunk_rows);
    for (int it = wib; it < a.n_items; it += nw) {
      if (bulk && tma_ok) {
        tma_ok = bulk_item<K, false, false>(a, it, lane, sm.ring, sm.bars, sm.face, status);
        if (!tma_ok)  // a wait expired (status set): redo this item without the ring
          stream_item<K, false, true, false, true, true>(a, it, lane, sm.face);
      } else {
        stream_item<K, false, true, false, true, true>(a, it, lane, sm.face);
      }
    }
    // This pass's ordinary stores must be visible to the next pass's bulk
    // copies (async proxy) before the team moves on.
    asm volatile("fence.proxy.async.global;" ::: "memory");
    team_sync(team);
    src_buf = dst;
  }
}

template <int K>
__global__ void __launch_bounds__(BatchDepth<K>::MAX_THREADS, 1)
    batch_kernel(const cpb_grid_desc* __restrict__ descs, const int* __restrict__ order, int ngrids,
                 int n_large, int bc, int grain, int team_warps, BatchDebug dbg, int* work) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ int s_first;
  __shared__ int s_team_first[BATCH_MAX_TEAMS];
  extern __shared__ __align__(128) unsigned char smem[];
  // this warp's row ring, mbarriers and ring of per-row face terms (k_stream.cuh)
  const BulkSmem<K, false> sm(smem, wib, nw, BATCH_STAGES);
  bool tma_ok = true;
  // Phase 1: large grids, one CTA per grid, fetched `grain` at a time.
  for (;;) {
    if (threadIdx.x == 0) s_first = atomicAdd(&work[0], grain);
    __syncthreads();
    const int first = s_first;
    __syncthreads();
    if (first >= n_large) break;
    const int last = min(first + grain, n_large);
    for (int q = first; q < last; ++q) {
      const cpb_grid_desc g = descs[CPB_CHK(order[q], 1, ngrids)];
      run_grid<K>(g, bc, wib, nw, lane, &work[2], sm, tma_ok, dbg, Team{0, (int)blockDim.x});
    }
  }
  // Phase 2: small grids, one team of team_warps warps per grid (one warp,
  // or a few warps meeting at a named barrier; the host checks that the
  // teams tile the CTA).  A team's first thread fetches from the queue.
  const int n_small = ngrids - n_large;
  if (team_warps <= 1) {
    for (;;) {
      int first = 0;
      if (lane == 0) first = atomicAdd(&work[1], grain);
      first = __shfl_sync(0xffffffffu, first, 0);
      if (first >= n_small) break;
      const int last = min(first + grain, n_small);
      for (int q = first; q < last; ++q) {
        const cpb_grid_desc g = descs[CPB_CHK(order[n_large + q], 1, ngrids)];
        run_grid<K>(g, bc, 0, 1, lane, &work[2], sm, tma_ok, dbg, Team{0, 32});
      }
    }
  } else {
    const int tix = wib / team_warps, twib = wib % team_warps;
    const Team team{1 + tix, 32 * team_warps};
    for (;;) {
      if (twib == 0 && lane == 0) s_team_first[tix] = atomicAdd(&work[1], grain);
      team_sync(team);
      const int first = s_team_first[tix];
      team_sync(team);  // every warp of the team has read it before the next fetch
      if (first >= n_small) break;
      const int last = min(first + grain, n_small);
      for (int q = first; q < last; ++q) {
        const cpb_grid_desc g = descs[CPB_CHK(order[n_large + q], 1, ngrids)];
        run_grid<K>(g, bc, twib, team_warps, lane, &work[2], sm, tma_ok, dbg, team);
      }
    }
  }
}

}  // namespace

bool batch_team_ok(int threads, int team_warps) {
  if (team_warps <= 1) return true;
  const int nw = threads / 32;
  return team_warps <= nw && nw % team_warps == 0 && nw / team_warps <= BATCH_MAX_TEAMS;
}

int batch_threads_max(int depth) {
  return depth == 4 ? BatchDepth<4>::MAX_THREADS : (depth == 8 ? BatchDepth<8>::MAX_THREADS : 0);
}

namespace {
unsigned g_batch_attr_done[2];  // per depth (4, 8): devices with the shared-memory opt-in set
size_t batch_smem(int depth, int threads) {
  return stream_smem_bytes(false, depth, threads / 32, 1, BATCH_STAGES);
}
const void* batch_fn(int depth) {
  return depth == 8 ? (const void*)batch_kernel<8> : (const void*)batch_kernel<4>;
}
}  // namespace

cudaError_t batch_blocks_per_sm(int depth, int threads, int* out) {
  if (batch_threads_max(depth) == 0) return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem_optin(batch_fn(depth), g_batch_attr_done[depth == 8], batch_smem(depth, threads));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, batch_fn(depth), threads, batch_smem(depth, threads));
}

cudaError_t launch_batch(int depth, const cpb_grid_desc* descs, const int* order, int ngrids, int n_large,
                         int bc, int grain, int blocks, int threads, int team_warps, const BatchDebug& dbg,
                         int* work, cudaStream_t s) {
  if (batch_threads_max(depth) == 0 || threads > batch_threads_max(depth)) return cudaErrorInvalidValue;
  if (!batch_team_ok(threads, team_warps)) return cudaErrorInvalidValue;
  const size_t shm = batch_smem(depth, threads);
  cudaError_t e = ensure_smem_optin(batch_fn(depth), g_batch_attr_done[depth == 8], shm);
  if (e != cudaSuccess) return e;
  (void)cudaGetLastError();  // drop a stale non-sticky error so the check below is this launch's
  e = cudaMemsetAsync(work, 0, 3 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (depth == 8)
    batch_kernel<8><<<blocks, threads, shm, s>>>(descs, order, ngrids, n_large, bc, grain, team_warps, dbg, work);
  else
    batch_kernel<4><<<blocks, threads, shm, s>>>(descs, order, ngrids, n_large, bc, grain, team_warps, dbg, work);
  return cudaGetLastError();
}

cudaError_t read_bounds_batch(int* out) { return read_bounds_word(out); }

}  // namespace cpb
