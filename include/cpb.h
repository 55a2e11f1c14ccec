/* cpb.h — C ABI of libcpb: a barrier-tiled 2-D heat-diffusion stencil for
 * NVIDIA GB300 (sm_103a).
 *
 * The stencil
 * -----------
 * Grid: ny rows x nx columns, row-major, x fastest; cell (i, j), 0 <= i < nx,
 * 0 <= j < ny.  Neighbours W=(i-1,j), E=(i+1,j), S=(i,j-1), N=(i,j+1).
 * One step of the explicit flux-form update with conductivity kappa and
 * source s (hdt = 0.5f * dt; every operation rounded in FP32, in this order):
 *     fW = (kc + kW) * (uW - c)      fE = (kc + kE) * (uE - c)
 *     fS = (kc + kS) * (uS - c)      fN = (kc + kN) * (uN - c)
 *     u' = c + (hdt * ((fW + fE) + (fS + fN)) + dt * s)
 * Boundary CPB_DIRICHLET0: a neighbour outside the grid has u = 0 and
 * kappa = kc (the boundary face conducts with 2 kc).  CPB_PERIODIC: wrap.
 * The paper (CuPBoP, arXiv 2206.07896) contains no stencil: the update, its
 * boundary rule and its rounding order are this library's definition.  The
 * library built with --fmad=false (libcpb_nofma.so) reproduces that order
 * bit for bit; the default build (libcpb.so) lets the compiler contract
 * multiply-adds into FMAs.
 *
 * Launch model
 * ------------
 * Calls follow the CUDA launch model the paper executes on CPUs (Sec. II,
 * Sec. IV "Push task queue"): the caller supplies launch geometry (grid,
 * block, dynamic shared bytes) as in <<<grid, block, shm>>> and the fields of
 * the paper's kernel structure (Listing 6); every call only enqueues work on
 * the caller's stream and returns (asynchronous launch, Sec. III "Implicit
 * barrier insertion": the caller synchronises before reading results on the
 * host).  Errors are status codes, never exceptions.
 *
 * Memory
 * ------
 * All field pointers are device memory owned by the caller; the library never
 * allocates or frees them.  Storage formats:
 *   CPB_F32         u, kappa, s: float, nx*ny each.
 *   CPB_BF16_KAHAN  u: one 32-bit word per cell, bits 0..15 = hi (bf16),
 *                   bits 16..31 = cmp (bf16), value = (float)hi - (float)cmp;
 *                   kappa, s: bf16 (uint16 bit patterns), nx*ny each.
 *                   Each step computes v in FP32 from the effective values,
 *                   then hi' = rn_bf16(v), cmp' = rn_bf16((float)hi' - v).
 *   CPB_BF16_KAHAN_BLOCK  the same storage format; the steps of one pass of
 *                   the temporal-blocked kernel (its depth k, see cpb_tuning)
 *                   run in FP32 from the effective values, and only the
 *                   result the pass stores is rounded into (hi, cmp) as
 *                   above.  The result depends on the pass schedule: passes
 *                   of depth k, a last pass of steps % k, and (with no
 *                   scratch buffer) one pass of depth d >= 2 split into
 *                   d - d/2 and d/2 when the pass count is even.  The
 *                   reading of "BF16 storage, FP32 compute" in which storage
 *                   happens where the kernel stores; CPB_BF16_KAHAN rounds
 *                   every step as if each were stored.
 * Streams are CUDA stream handles (cudaStream_t); NULL is the legacy default
 * stream.
 *
 * Validation happens before any launch: a failed check returns its code and
 * enqueues nothing.  A CUDA error from an enqueue returns CPB_ERR_CUDA
 * (details: cpb_last_error_detail()).
 */
#ifndef CPB_H
#define CPB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cpb_stream_t; /* == cudaStream_t */

typedef enum {
  CPB_SUCCESS = 0,
  CPB_ERR_INVALID_VALUE = 1,      /* bad size, null pointer, bad enum, in-place call   */
  CPB_ERR_UNSUPPORTED_CONFIG = 2, /* launch geometry / dtype with no compiled variant  */
  CPB_ERR_SHARED_MEM = 3,         /* shared_bytes below what the variant needs         */
  CPB_ERR_LAUNCH = 4,             /* kernel launch rejected (geometry beyond limits)   */
  CPB_ERR_TIMEOUT = 5,            /* a bounded device-side wait gave up                */
  CPB_ERR_CUDA = 6,               /* any other CUDA runtime error                      */
  CPB_ERR_WORKSPACE = 7           /* workspace missing or smaller than required        */
} cpb_status;

typedef enum { CPB_F32 = 0, CPB_BF16_KAHAN = 1, CPB_BF16_KAHAN_BLOCK = 2 } cpb_dtype;
typedef enum { CPB_DIRICHLET0 = 0, CPB_PERIODIC = 1 } cpb_boundary;

typedef struct {
  unsigned x, y, z;
} cpb_dim3;

/* Parameters of the streaming temporal-blocked kernel (the tuned path).
 *   k               time steps fused per pass over HBM (temporal block depth), 1..8
 *   chunk_rows      output rows per warp work item (>= 1)
 *   warps_per_block warps per CTA (1..8)
 *   variant         0 = each lane loads its 128-bit slice of the next row into
 *                       registers (any size, any alignment);
 *                   1 = per-warp ring of shared-memory row slots filled by TMA
 *                       bulk copies (cp.async.bulk + mbarrier).  Used when the
 *                       fields are 16-byte aligned, nx % 4 == 0 and nx >= 128
 *                       (BF16-Kahan: nx % 8 == 0, nx >= 136); otherwise
 *                       variant 0 runs with the same results.
 *   stages          variant 1: ring slots per warp, a power of two in 2..16 */
typedef struct {
  int k;
  int chunk_rows;
  int warps_per_block;
  int variant;
  int stages;
} cpb_tuning;

int cpb_version(void);
const char* cpb_status_string(cpb_status status);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* cpb_last_error_detail(void);

/* Device facts used for launch sizing (current device). */
cpb_status cpb_device_info(int* sm_count, int* l2_bytes, int* smem_optin_bytes);

/* Advance `steps` steps; the result is ALWAYS in u_out.
 *
 * u_in is read.  When scratch == NULL, u_in is also the ping-pong buffer and
 * is clobbered (steps >= 2); when scratch != NULL (nx*ny cells of the storage
 * format) u_in is left untouched.  u_in, u_out and scratch must not overlap.
 * steps == 0 copies u_in to u_out.
 *
 * Geometry (the paper's <<<grid, block, shm>>>):
 *  - block = {bx, by, 1} with 1 <= bx*by <= 1024: the tiled one-step kernel,
 *    one thread per cell, a (bx+2)x(by+2) shared tile of u and of kappa, one
 *    __syncthreads; grid must be {ceil(nx/bx), ceil(ny/by), 1} and
 *    shared_bytes >= 2*(bx+2)*(by+2)*4.  CPB_F32 only.  One launch per step.
 *  - block = {0, 0, 0}: the tuned streaming kernel (grid and shared_bytes are
 *    ignored); its parameters come from cpb_set_tuning / cpb_autotune for
 *    this (nx, ny, dtype, bc), else from the built-in default.
 * dt > 0 and finite.  Alignment: 16-byte aligned fields with nx % 4 == 0 use
 * 128-bit accesses; anything else uses the scalar-access path (same results). */
cpb_status cpb_stencil_launch(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                              int ny, int steps, float dt, cpb_boundary bc, cpb_dtype dtype,
                              cpb_dim3 grid, cpb_dim3 block, size_t shared_bytes, void* scratch,
                              cpb_stream_t stream);

/* Same as cpb_stencil_launch with block = {0,0,0} but with explicit tuning. */
cpb_status cpb_stencil_launch_tuned(void* u_in, void* u_out, const void* kappa, const void* src,
                                    int nx, int ny, int steps, float dt, cpb_boundary bc,
                                    cpb_dtype dtype, const cpb_tuning* tuning, void* scratch,
                                    cpb_stream_t stream);

/* Tuning cache (process-wide, keyed by nx, ny, dtype, bc).  The paper's
 * nearest counterpart is the per-kernel block_per_fetch its runtime sets
 * (Sec. IV "Runtime Optimizations"); here a tuning fixes the temporal depth
 * and the work shape of the tuned path.  cpb_get_tuning returns the cached
 * tuning or the built-in default; cpb_lookup_tuning sets *found to 1 and *t
 * only when a tuning is cached for the key.  Errors: null pointers or
 * nx, ny < 1 give CPB_ERR_INVALID_VALUE; an invalid tuning given to
 * cpb_set_tuning gives CPB_ERR_INVALID_VALUE. */
cpb_status cpb_set_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, const cpb_tuning* t);
cpb_status cpb_get_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, cpb_tuning* t);
cpb_status cpb_lookup_tuning(int nx, int ny, cpb_dtype dtype, cpb_boundary bc, cpb_tuning* t,
                             int* found);

/* Persistent tuning cache (no counterpart in the paper): a tuning is a
 * measurement on one device for one grid shape, worth keeping between
 * processes (autotuning a large grid takes seconds).  Text file, one tuning
 * per line:
 *   cpb-tuning 1 <device> <nx> <ny> <dtype> <bc> <k> <chunk_rows> <warps_per_block> <variant> <stages>
 * where <device> is the device name with every blank replaced by '_'.
 * cpb_tuning_save writes every tuning cached in this process under `device`
 * (NULL: the current device's name), replacing the file (written to a
 * temporary name, then renamed).  cpb_tuning_load caches every line whose
 * device equals `device` (NULL: the current device's name) and writes how
 * many in *loaded (may be NULL); lines of other devices are skipped.  A line
 * that does not parse or holds an invalid tuning, or a file that cannot be
 * opened, gives CPB_ERR_INVALID_VALUE (lines before a bad one stay loaded).
 * With `device` given, neither call touches the GPU. */
cpb_status cpb_tuning_save(const char* path, const char* device);
cpb_status cpb_tuning_load(const char* path, const char* device, int* loaded);

/* Time candidate tunings on the caller's buffers (u_a and u_b are
 * clobbered; kappa, src read) for `steps` steps each, store the fastest in the
 * cache and return it in *best.  Synchronises `stream`.  The paper leaves the
 * choice of its grain size to heuristics per kernel (Sec. IV "Runtime
 * Optimizations"); this measures instead.  Candidates: depth 1..6 and 8,
 * chunk 16..512 rows, 1..4 warps per CTA, both row-load variants, 2..8 ring
 * stages, and the built-in default; each timed twice (the better run counts), the best twelve again
 * four times.  A timed run is an odd number of passes of the candidate's
 * depth near `steps` steps, repeated to at least about 1 ms.  Arguments are
 * validated as for cpb_stencil_launch. */
cpb_status cpb_autotune(void* u_a, void* u_b, const void* kappa, const void* src, int nx, int ny,
                        int steps, float dt, cpb_boundary bc, cpb_dtype dtype, cpb_stream_t stream,
                        cpb_tuning* best);

/* Device status word of the stream kernels: synchronises the device, returns
 * in *status CPB_SUCCESS or CPB_ERR_TIMEOUT (a bounded mbarrier wait in a
 * variant-1 kernel gave up; that kernel's output is invalid), and clears it. */
cpb_status cpb_device_status(int* status);

/* Bounds-checked build (libcpb_check.so: --fmad=false arithmetic plus a range
 * check on every global element range the stencil, batched, adjoint, 3-D,
 * tiled and heat-sum kernels read or write; the element-wise conversion
 * kernels index i < n directly; the paper has no counterpart, this stands in
 * for a memory checker).  Synchronises the
 * device, then returns in *line the source line of the first access found
 * outside its field since the last call (0: none) and in *unit its
 * translation unit (1 stream FP32, 2 stream BF16-Kahan, 3 stream BF16-Kahan
 * per pass, 4 batched, 5 adjoint, 6 3-D, 7 tiled, 8 heat sum; 0: none), and
 * clears them.  The checked kernel clamped the access into its field, so
 * nothing outside it was touched, but its result is invalid.  In the other
 * builds *unit = *line = 0 and the call returns CPB_ERR_UNSUPPORTED_CONFIG. */
cpb_status cpb_bounds_status(int* unit, int* line);

/* Test hook: mbarrier wait limit in polls (<= 0: default, about 1M polls) and
 * a row index whose TMA copies are withheld (-1: off): its ring slot is told
 * the row's byte count but no copy is issued, so the wait for that slot runs
 * out and nothing is left in flight.  Applies to subsequent launches of this
 * process.  Used to exercise the timeout path. */
cpb_status cpb_debug_set(int wait_limit, int inject_row);

/* FP64 sum of the field (CPB_F32: sum of (double)u; CPB_BF16_KAHAN: sum of
 * (double)hi - (double)cmp), written to *d_out (device pointer).  Two
 * deterministic passes (per-block partials in `workspace`, then one block in
 * a fixed order): the same input gives the same bits on the same device.
 * workspace: device memory of at least cpb_heat_sum_workspace_bytes(). */
size_t cpb_heat_sum_workspace_bytes(int nx, int ny);
cpb_status cpb_heat_sum(const void* u, int nx, int ny, cpb_dtype dtype, double* d_out,
                        void* workspace, size_t ws_bytes, cpb_stream_t stream);

/* cpb_heat_sum without a workspace: the same FP64 heat sum, for callers that
 * cannot allocate device memory — code that runs where cudaMalloc is not
 * available to it (a host framework that owns all device memory through its
 * own pool, an embedding that forbids new allocations after start-up) or
 * where the implicit device synchronisation of cudaMalloc/cudaFree is not
 * acceptable (latency-critical loops).  There is no counterpart in the paper.
 *
 * The per-block partial sums live in a 32 KB array inside the library (one
 * per GPU that loads it, held until the process exits).  Grids of more than
 * 2^26 cells (67,108,864) are rejected with CPB_ERR_WORKSPACE before any
 * launch; use cpb_heat_sum for those.  The call allocates nothing.  Every
 * call looks up the array's device address on the current device
 * (cudaGetSymbolAddress: no allocation, no synchronisation), so the address
 * stays right across a cudaDeviceReset; the first call on a device may load
 * the library's device code, so make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's partial
 * sums; every partial a call reads it has written itself, so nothing needs
 * clearing.  Calls whose executions overlap on the GPU (unordered streams)
 * race on the array and may return wrong sums: order them on one stream.
 * The blocking differs from cpb_heat_sum, so the two may differ in the last
 * bits when the sum is not exact in FP64 (it is exact, and the two equal,
 * for FP32 values that are multiples of 2^-24 in [0, 1)). */
cpb_status cpb_heat_sum_noalloc(const void* u, int nx, int ny, cpb_dtype dtype, double* d_out,
                                cpb_stream_t stream);

/* BF16 conversions on the device (IEEE round to nearest even), for moving
 * fields in and out of the CPB_BF16_KAHAN storage format.  The paper has no
 * reduced-precision storage; the format is this library's (one 32-bit word
 * per cell: the bf16 value hi in the low half, the bf16 compensation cmp in
 * the high half, represented value hi - cmp).
 * cpb_bf16_round: out[i] = rn_bf16(x[i]) (bf16 bit patterns).
 * cpb_bf16k_pack: state[i] = hi | cmp << 16 with hi = rn(u), cmp = rn(hi - u).
 * cpb_bf16k_unpack: u[i] = (float)hi - (float)cmp.
 * n elements; all pointers caller-owned device memory, 4-byte (2-byte for
 * out) aligned.  n < 0, or n > 0 with a null pointer: CPB_ERR_INVALID_VALUE;
 * n == 0 does nothing.  Asynchronous on `stream`. */
cpb_status cpb_bf16_round(const float* x, uint16_t* out, long long n, cpb_stream_t stream);
cpb_status cpb_bf16k_pack(const float* u, uint32_t* state, long long n, cpb_stream_t stream);
cpb_status cpb_bf16k_unpack(const uint32_t* state, float* u, long long n, cpb_stream_t stream);

/* End-to-end call on HOST buffers (the paper's timings include the
 * host <-> device transfers, Sec. V "Performance"): copies u0, kappa, src in (pinned host
 * memory gives asynchronous copies), runs `steps` steps on the tuned path,
 * copies the result to u_out_host and synchronises `stream` before it
 * returns.  Host buffers: caller-owned, nx * ny elements of the storage
 * format (u as for cpb_stencil_launch, kappa and src float for CPB_F32 and
 * bf16 for CPB_BF16_KAHAN), read or written only during the call; src may be
 * NULL (s = 0).  d_workspace: caller-owned device memory, 256-byte aligned,
 * of at least cpb_host_workspace_bytes(nx, ny, dtype) bytes (0 for invalid
 * sizes), else CPB_ERR_WORKSPACE.  Null host pointers, sizes below 1, an
 * unknown dtype and the argument errors of cpb_stencil_launch_tuned:
 * CPB_ERR_INVALID_VALUE. */
size_t cpb_host_workspace_bytes(int nx, int ny, cpb_dtype dtype);
cpb_status cpb_stencil_host(const void* u0_host, const void* kappa_host, const void* src_host,
                            void* u_out_host, int nx, int ny, int steps, float dt, cpb_boundary bc,
                            cpb_dtype dtype, void* d_workspace, size_t ws_bytes,
                            cpb_stream_t stream);

/* The same run as cpb_stencil_host, enqueued on three streams and returned
 * from at once, so that consecutive problems overlap their transfers with
 * each other's compute (the copy engines and the SMs work side by side; on
 * the GB300 machine a step's 1 GB of transfers costs about 5 ms over the host
 * link).  h2d: the copies of u0, kappa, src into the workspace; compute
 * (waits for them): the tuned passes; d2h (waits for those): the copy of the
 * result to u_out_host.  The streams must be distinct.  The host buffers
 * must stay valid, and the workspace unused by anything else, until the
 * d2h stream has passed this call's copy (the caller synchronises d2h, or
 * records an event on it, before reading u_out_host).  Consecutive calls
 * that alternate two workspaces overlap; a call on the workspace of an
 * unfinished earlier call races with it unless the caller orders them.
 * Host buffers should be pinned (pageable memory makes the copies
 * synchronous).  Validation and errors as for cpb_stencil_host. */
cpb_status cpb_stencil_host_async(const void* u0_host, const void* kappa_host, const void* src_host,
                                  void* u_out_host, int nx, int ny, int steps, float dt, cpb_boundary bc,
                                  cpb_dtype dtype, void* d_workspace, size_t ws_bytes, cpb_stream_t h2d,
                                  cpb_stream_t compute, cpb_stream_t d2h);

/* Shared-memory temporal blocking with the caller's geometry: the
 * multi-barrier kernel class (the paper's srad has nine block
 * synchronisations, Sec. V; its CPU translation needs loop fission with the
 * time loop kept, Sec. III "SPMD to MPMD").  One launch advances `depth` steps (1..16): a
 * block of block.x x block.y threads stages a (bx + 2 depth) x
 * (by + 2 depth) tile of u, kappa and s, __syncthreads, then per step
 * updates the shrinking region of the tile in shared memory and
 * __syncthreads again, and finally writes its bx x by interior.  Same update,
 * boundary rules, ping-pong and scratch semantics as cpb_stencil_launch
 * (result always in u_out); CPB_F32 only; src may be NULL (s = 0).
 * Geometry: block = (bx, by, 1) with bx * by <= 1024, else
 * CPB_ERR_UNSUPPORTED_CONFIG; grid = (ceil(nx / bx), ceil(ny / by), 1), else
 * CPB_ERR_INVALID_VALUE; shared_bytes >= cpb_tile_blocked_shared_bytes(bx,
 * by, depth) (16 (bx + 2 depth)(by + 2 depth) bytes), else CPB_ERR_SHARED_MEM
 * (more than 227 KB: CPB_ERR_UNSUPPORTED_CONFIG); depth outside 1..16:
 * CPB_ERR_INVALID_VALUE.  Asynchronous on `stream`. */
size_t cpb_tile_blocked_shared_bytes(int bx, int by, int depth); /* 0 if invalid */
cpb_status cpb_stencil_tile_blocked(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                                    int ny, int steps, int depth, float dt, cpb_boundary bc, cpb_dim3 grid,
                                    cpb_dim3 block, size_t shared_bytes, void* scratch,
                                    cpb_stream_t stream);

/* 3-D 7-point variant (the class of the paper's hotspot3D benchmark,
 * Sec. V): u'(x,y,z) from its six face neighbours, with the faces D (z-1)
 * and U (z+1) added to the 2-D update and rounded in the order
 *   acc = ((fW + fE) + (fS + fN)) + (fD + fU),  u' = c + (hdt*acc + dt*s),
 * f = (kc + kn)(un - c); Dirichlet ghosts u = 0, kappa = kc; periodic wraps
 * every axis.  CPB_F32 only.  Fields are nz x ny x nx, x fastest, caller-owned
 * device memory; src may be NULL (s = 0).  Steps run one launch each of the
 * z-marching tiled kernel (a CTA of 32 x by threads owns 128 columns x by
 * rows and a run of ceil(nz / grid.z) planes, with a __syncthreads inside its
 * plane loop), ping-ponging as cpb_stencil_launch does (result always in u_out;
 * u_in clobbered unless scratch is given).  The caller's launch geometry:
 * block = (32, by, 1) with 1 <= by <= 8, else CPB_ERR_UNSUPPORTED_CONFIG;
 * grid = (ceil(nx / 128), ceil(ny / by), zc) with 1 <= zc <= nz, else
 * CPB_ERR_INVALID_VALUE; shared_bytes >= cpb_stencil3d_shared_bytes(by),
 * else CPB_ERR_SHARED_MEM.  With nx % 4 == 0 and 16-byte aligned fields the
 * planes stream through an 8-slot shared-memory ring filled by asynchronous
 * copies several planes ahead; otherwise each thread loads the next plane
 * into registers.  block = {0,0,0} selects by = 8 and z-chunks of about
 * 32 planes.  Validation and errors as for cpb_stencil_launch; asynchronous
 * on `stream`. */
size_t cpb_stencil3d_shared_bytes(int by); /* 0 if by is outside 1..8 */
cpb_status cpb_stencil3d_launch(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                                int ny, int nz, int steps, float dt, cpb_boundary bc, cpb_dim3 grid,
                                cpb_dim3 block, size_t shared_bytes, void* scratch, cpb_stream_t stream);

/* Batched persistent stencil: many independent grids (uneven sizes and step
 * counts, CPB_F32 storage, one boundary rule) advanced in ONE kernel launch.
 * Resident CTAs fetch grids from a device work queue, `grain` grids per atomic
 * fetch (the GPU counterpart of the paper's task queue with block_per_fetch,
 * Sec. IV "Fetch task queue" and "Runtime Optimizations").  Grids with at
 * least team_cells cells run on a whole CTA, smaller ones on teams of
 * plan->team_warps warps (one warp by default).
 * Each grid's result is written to its u_out; its u_in is clobbered (used as
 * the ping-pong buffer).  Every grid advances plan->depth (4 or 8) time
 * steps per pass; at depth 8 the row loop takes rows in pairs, as in the
 * single-grid kernel.  Grids
 * whose u_in, u_out, kappa and src are 16-byte aligned with nx % 4 == 0 and
 * nx >= 128 stream their rows through a per-warp TMA ring (bounded waits, as
 * in the variant-1 single-grid kernel); the others load rows with ordinary
 * 128-bit or scalar loads.
 *
 * cpb_batch_order (host): validates the host copy of the descriptors and
 * writes the queue order into h_order[ngrids]: large grids first, each class
 * longest-first (LPT by cells x steps), and *n_large.  Invalid descriptor ->
 * CPB_ERR_INVALID_VALUE.
 * cpb_stencil_batched: d_descs / d_order are device copies; d_work is device
 * memory of cpb_batch_work_bytes() bytes (queue counters + status word), reset
 * by the call itself (the call is one memset + one kernel launch, so it can be
 * captured in a CUDA graph).  plan == NULL or plan->blocks <= 0 fills the GPU.
 * cpb_batch_status: synchronises `stream` and returns the status word:
 * CPB_SUCCESS; CPB_ERR_INVALID_VALUE if a device descriptor was invalid (that
 * grid is skipped, the others are complete); or CPB_ERR_TIMEOUT if a TMA-ring
 * wait expired in some warp (that warp redid the item with ordinary loads and
 * left the ring for the rest of the launch: every output is still complete).
 * The first error recorded wins. */
typedef struct {
  void* u_in;
  void* u_out;
  const void* kappa;
  const void* src; /* may be NULL: no source */
  int nx, ny, steps;
  float dt;
} cpb_grid_desc;

typedef struct {
  int grain;      /* grids per queue fetch (>= 1) */
  int blocks;     /* persistent CTAs (<= 0: one wave filling the GPU) */
  int threads;    /* threads per CTA, a multiple of 32, <= 384 at depth 4, <= 256 at depth 8 */
  int team_cells; /* grids with nx*ny >= team_cells run on a whole CTA */
  int depth;      /* time steps per pass over a grid: 4 or 8 */
  int team_warps; /* warps per team for the other grids: <= 1 one warp per grid;
                     otherwise a divisor of threads / 32 with at most 15 teams
                     per CTA, the teams of a CTA taking grids independently
                     once the whole-CTA grids are done */
} cpb_batch_plan;

cpb_status cpb_batch_plan_default(cpb_batch_plan* plan);
cpb_status cpb_batch_order(const cpb_grid_desc* h_descs, int ngrids, const cpb_batch_plan* plan,
                           int* h_order, int* n_large);
size_t cpb_batch_work_bytes(void);
cpb_status cpb_stencil_batched(const cpb_grid_desc* d_descs, const int* d_order, int ngrids,
                               int n_large, cpb_dtype dtype, cpb_boundary bc,
                               const cpb_batch_plan* plan, int* d_work, cpb_stream_t stream);
cpb_status cpb_batch_status(const int* d_work, int* status, cpb_stream_t stream);

/* Grain-size selection for the batched launch, the GPU counterpart of the
 * paper's trade-off between average and aggressive coarse-grained fetching
 * (Sec. IV "Runtime Optimizations", evaluated in Sec. V "aggressive
 * coarse-grained fetching"): more grids per atomic fetch means fewer fetches
 * but a coarser balance of work over the resident CTAs, so the best grain
 * depends on the batch.  The call times the batch once for every candidate
 * (depth, grain, threads) in CPB_BATCH_TUNE_DEPTHS x CPB_BATCH_TUNE_GRAINS x
 * CPB_BATCH_TUNE_THREADS, in that nesting, with plan->team_cells and one
 * wave of CTAs, re-times the three fastest twice and writes the fastest plan
 * to *plan (blocks = 0).  ms_table (optional, host,
 * CPB_BATCH_TUNE_CANDIDATES floats) receives the single-run time of every
 * candidate in milliseconds (-1 where the plan is not valid, e.g. 384
 * threads at depth 8, or the launch was rejected).  Arguments as for cpb_stencil_batched, with d_order built
 * for plan->team_cells.  The batch runs several times: every grid's u_in
 * and u_out are overwritten, so tune on copies of the fields.  Synchronises
 * `stream`.  A status word other than CPB_SUCCESS after a run is returned
 * (the plan is then left unchanged). */
#define CPB_BATCH_TUNE_DEPTHS 2   /* 4, 8 */
#define CPB_BATCH_TUNE_GRAINS 5   /* 1, 2, 4, 8, 16 */
#define CPB_BATCH_TUNE_THREADS 3  /* 128, 256, 384 */
#define CPB_BATCH_TUNE_CANDIDATES \
  (CPB_BATCH_TUNE_DEPTHS * CPB_BATCH_TUNE_GRAINS * CPB_BATCH_TUNE_THREADS)
cpb_status cpb_batch_autotune(const cpb_grid_desc* d_descs, const int* d_order, int ngrids,
                              int n_large, cpb_dtype dtype, cpb_boundary bc, int* d_work,
                              cpb_stream_t stream, cpb_batch_plan* plan, float* ms_table);

/* Discrete adjoint of the N-step stencil (CPB_F32), for gradients of a loss
 * L(u_T) with respect to u_0 and kappa.  With lambda_T = dL/du_T (given):
 *   lambda_n = lambda_{n+1} + dt D(kappa) lambda_{n+1}   (D symmetric: the
 *              same update with s = 0), dL/du_0 = lambda_0,
 *   dL/dkappa_c = sum over steps and faces f of c, with u = u_n and
 *              lambda = lambda_{n+1}: hdt (u_f - u_c)(lambda_c - lambda_f) for
 *              an interior face, dt (0 - u_c) lambda_c for a Dirichlet
 *              boundary face.
 * The paper has no adjoint; this is the derivative of the update defined
 * above.  States are checkpointed every ckpt_every steps by the forward call
 * and each segment is recomputed during the backward sweep: where the fields
 * allow the TMA row path (nx % 4 == 0, nx >= 128, 16-byte aligned kappa and
 * src), by depth-4 passes that store every intermediate state, otherwise one
 * step per pass; either way the states equal those of a one-step run.
 *
 * workspace: device memory of cpb_adjoint_workspace_bytes() bytes, 256-byte
 * aligned, holding the checkpoints between cpb_adjoint_forward and
 * cpb_adjoint_backward (same nx, ny, steps, dt, bc, ckpt_every, kappa, src).
 * cpb_adjoint_forward writes u_T.  cpb_adjoint_backward overwrites grad_u0
 * and grad_kappa.  cpb_stencil_adjoint runs both (u_T is not returned).
 * src may be NULL (no source).  All asynchronous on `stream`. */
size_t cpb_adjoint_workspace_bytes(int nx, int ny, int steps, int ckpt_every);
cpb_status cpb_adjoint_forward(const float* u0, const float* kappa, const float* src, int nx, int ny,
                               int steps, float dt, cpb_boundary bc, int ckpt_every, float* u_T,
                               void* workspace, size_t ws_bytes, cpb_stream_t stream);
cpb_status cpb_adjoint_backward(const float* kappa, const float* src, const float* lambda_T, int nx,
                                int ny, int steps, float dt, cpb_boundary bc, int ckpt_every,
                                float* grad_u0, float* grad_kappa, void* workspace, size_t ws_bytes,
                                cpb_stream_t stream);
cpb_status cpb_stencil_adjoint(const float* u0, const float* kappa, const float* src,
                               const float* lambda_T, int nx, int ny, int steps, float dt,
                               cpb_boundary bc, int ckpt_every, float* grad_u0, float* grad_kappa,
                               void* workspace, size_t ws_bytes, cpb_stream_t stream);

/* CUDA graph of a whole multi-step run (the launch sequence captured once and
 * replayed; Sec. VI of the paper measures launch + sync overhead of many
 * launches).  The pointers are baked into the graph.  tuning == NULL uses the
 * cached / default tuning. */
typedef struct cpb_graph_s* cpb_graph_t;
cpb_status cpb_graph_create(void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                            int ny, int steps, float dt, cpb_boundary bc, cpb_dtype dtype,
                            const cpb_tuning* tuning, void* scratch, cpb_graph_t* graph);
cpb_status cpb_graph_launch(cpb_graph_t graph, cpb_stream_t stream);
cpb_status cpb_graph_destroy(cpb_graph_t graph);

/* Slab decomposition across ranks (one rank per GPU).  The paper has no
 * multi-device runtime; this is the decomposition the stencil takes when it
 * is spread over several GPUs, each running the single-GPU path on its slab.
 * Rank r of `world` owns the contiguous rows [row_lo, row_hi) of the
 * ny x nx grid (full width; sizes differ by at most one row) and keeps
 * `depth` halo rows on each side that has a neighbouring rank (both sides
 * for a periodic grid, a ring; none past a Dirichlet edge, where the slab's
 * edge is the grid's).  A slab buffer holds halo_lo + (row_hi - row_lo) +
 * halo_hi rows of nx cells, own rows starting at row halo_lo.  One round:
 * cpb_slab_exchange fills the halos from the neighbours' own rows, then
 * cpb_slab_step advances up to `depth` steps; the error of the cut edges
 * moves inward one row per step, so the own rows are exact after it.
 *
 * cpb_slab_rows: host only.  world >= 1, 0 <= rank < world, depth >= 1,
 * every rank must own at least `depth` rows (ny >= world * depth), else
 * CPB_ERR_INVALID_VALUE.  Any output pointer may be NULL. */
cpb_status cpb_slab_rows(int ny, int world, int rank, int depth, cpb_boundary bc, int* row_lo, int* row_hi,
                         int* halo_lo, int* halo_hi);

/* Fill this slab's halo rows: rows [0, halo_lo) from the lower neighbour's
 * last halo_lo own rows, rows [halo_lo + n_own, + halo_hi) from the upper
 * neighbour's first halo_hi own rows.  `below` / `above`: the neighbours'
 * slab buffers (own rows starting at their row below_halo_lo / above_halo_lo;
 * the lower neighbour owns below_n_own rows), device memory of this or a
 * peer device (one cudaMemcpyAsync per side, cudaMemcpyDefault, on
 * `stream`: device to device, or peer to peer through unified addressing).
 * A side with halo 0 is skipped and its pointer may be NULL.  With one rank
 * and a periodic grid, below and above are the slab itself.  Element size
 * from dtype: the u field (4 bytes for every storage format).  The caller orders the
 * exchange after the neighbours' last step (stream order or events).
 * Validation: nx, n_own >= 1, halos in [0, n_own] and not above the
 * neighbours' own row counts, non-null buffers for non-empty sides; else
 * CPB_ERR_INVALID_VALUE.  Not measured on a machine with more than one GPU. */
cpb_status cpb_slab_exchange(void* slab, int nx, int n_own, int halo_lo, int halo_hi, const void* below,
                             int below_halo_lo, int below_n_own, const void* above, int above_halo_lo,
                             int above_n_own, cpb_dtype dtype, cpb_stream_t stream);

/* The same exchange for a field of any element size, row_bytes = nx x the
 * element size: the kappa and source fields of the BF16-Kahan formats are
 * 2-byte fields (row_bytes = 2 nx), every other field 4-byte.  A slab's
 * kappa and source halos are filled once, before its first step.  Validation
 * as for cpb_slab_exchange (row_bytes >= 1). */
cpb_status cpb_slab_exchange_rows(void* slab, size_t row_bytes, int n_own, int halo_lo, int halo_hi,
                                  const void* below, int below_halo_lo, int below_n_own, const void* above,
                                  int above_halo_lo, int above_n_own, cpb_stream_t stream);

/* One pass of `steps` (1 <= steps <= min of the non-zero halos, and <= 8)
 * steps over the whole slab buffer (rows_total = halo_lo + n_own + halo_hi)
 * under the grid's boundary rule, u_in -> u_out (u_in untouched), kappa and
 * src slab buffers of the same shape whose halos hold the neighbours' rows
 * (they never change: exchange them once).  The tuned streaming path with
 * depth = steps, one launch; tuning NULL: the cached / default tuning of the
 * slab's shape.  Only the own rows of u_out are valid afterwards. */
cpb_status cpb_slab_step(const void* u_in, void* u_out, const void* kappa, const void* src, int nx,
                         int rows_total, int halo_lo, int halo_hi, int steps, float dt, cpb_boundary bc,
                         cpb_dtype dtype, const cpb_tuning* tuning, cpb_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CPB_H */
