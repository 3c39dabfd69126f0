/*
 * rti.h -- C ABI of the GB300 (sm_103a) RTi tsunami time-stepping library.
 *
 * The library advances the nonlinear shallow-water equations on 1:3 nested
 * staggered grids (Takahashi et al., Sec. II-A, Eqs. 1-3) with one dt on all
 * levels (Sec. V-A), in the order of the time-integration loop of Sec. IV-A /
 * Fig. 2: mass update, child-to-parent water level (Sec. IV-C-2, Listing 5),
 * momentum update, parent-to-child fluxes, output update (maximum level and
 * inundation depth, arrival), buffer swap. All arithmetic runs in CUDA kernels;
 * there is no CPU fallback.
 *
 * Conventions for every call:
 *  - Return 0 (RTI_OK) on success or a negative RTI_ERR_* code. Nothing aborts,
 *    throws or exits across this boundary. rti_last_error() gives a message.
 *  - Grids are row-major with x fastest. A block of nx*ny cells has eta and
 *    outputs as nx*ny arrays, M (x-faces) as ny*(nx+1) and N (y-faces) as
 *    (ny+1)*nx. Face f of row j of M lies between cells f-1 and f.
 *  - h > 0 is still-water depth (sea), h <= 0 is land elevation (negated).
 *  - Host pointers are read (inputs, copied) or written (outputs) during the
 *    call only; the caller owns them. Device memory belongs to the library
 *    unless the caller passes its own arena to rti_create.
 *  - Calls on one handle or batch are not thread-safe; different handles may
 *    be used from different threads.
 */
#ifndef RTI_H
#define RTI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTI_OK 0
#define RTI_ERR_INVALID_ARG -1 /* null pointer, bad size or index, bad params */
#define RTI_ERR_CFL -2         /* Eq. 4 violated: dx/dt < sqrt(2 g h_max) on a block */
#define RTI_ERR_NESTING -3     /* child not 1:3, not inside its parent with a 3-cell margin, overlapping siblings, parents not listed first */
#define RTI_ERR_OOM -4         /* device memory exhausted or caller arena too small */
#define RTI_ERR_NONFINITE -5   /* a non-finite water level appeared on the device */
#define RTI_ERR_TIMEOUT -6     /* a bounded device wait ran out (the device-wide barrier between
                                  steps, or a strip's wait for the strips it depends on); the
                                  state is undefined until rti_set_initial_uplift or
                                  rti_set_state sets it again (the condition is cleared when
                                  it is reported) */
#define RTI_ERR_CUDA -7        /* a CUDA runtime call failed (message in rti_last_error) */
#define RTI_ERR_STATE -8       /* call not allowed in the current state (e.g. handle in a batch) */

#define RTI_BC_WALL 0      /* zero normal flux */
#define RTI_BC_RADIATION 1 /* outward flux sqrt(g h) * eta of the edge cell (root blocks only) */

#define RTI_FP64 0 /* all state and arithmetic in binary64 */
#define RTI_FP32 1 /* state and arithmetic in binary32; eta is the deviation from still water;
                      the volume budget and the nesting sums accumulate in binary64 */

/* Fine-to-coarse feedback (Sec. IV-C-2, "JNZSND"): which parent cells take the mean of
 * their 3x3 child cells (the mean of the wet ones, floored at the parent's ground). */
#define RTI_NEST_RING 0 /* the boundary cells: the inner ring of the child's footprint */
#define RTI_NEST_FULL 1 /* every parent cell the child covers (full two-way nesting); all
                           levels exchange at once, so a cell above a grandchild gets the
                           child's own level, and the grandchild's mean one step later */
/* Coarse-to-fine boundary flux ("JNQ"): how a child edge face takes the parent flux. */
#define RTI_FLUX_LINEAR 0   /* linear along the edge: 2/3, 1/3 weights at the outer fine faces */
#define RTI_FLUX_CONSTANT 1 /* each fine face takes its coarse face's flux (the edge carries
                               exactly the coarse discharge) */

#define RTI_SCHED_PERSISTENT 0 /* one cooperative launch per chunk of steps: device-wide barriers
                                  between steps, or with full feedback one dataflow in which
                                  each strip waits only for the strips it depends on */
#define RTI_SCHED_PER_PASS 1   /* one ordinary launch per step (no device-wide barrier) */

/* One rectangular block of a grid level (Sec. II-A "blocks"). */
typedef struct {
  int level;  /* 1 for the root level, parent level + 1 otherwise */
  int parent; /* index of the parent block in the same array, -1 for a root */
  int nx, ny; /* cells, 3 .. 2^20 each and (nx + 9 rounded up to 32) x (ny + 5) < 2^31;
                 multiples of 3 for a child */
  int i0, j0; /* child origin in parent cells; the child covers nx/3 x ny/3 parent cells */
  double dx;  /* cell size in metres; a child has exactly its parent's dx / 3 */
  int bc[4];  /* west, east, south, north edge of a root block: RTI_BC_*; ignored for children */
} rti_block;

typedef struct {
  double dt;          /* seconds, shared by all levels (Sec. V-A) */
  double g;           /* gravity, m/s^2 (9.81) */
  double dry_eps;     /* a cell is wet when h + eta > dry_eps (m; 1e-3) */
  double arrival_thr; /* arrival: max eta first >= this (m; 0.01) */
  int precision;      /* RTI_FP64 or RTI_FP32 */
  int schedule;       /* RTI_SCHED_* */
  int tile_x;         /* strip width in cells: 0 or 28 (a warp's 32 lanes less a 2-cell halo
                         on each side); other values are RTI_ERR_INVALID_ARG */
  int tile_y;         /* strip height in cells, a multiple of 8; 0 = 64 */
  int track_velocity; /* 1: keep the maximum water velocity (one more plane per block and a
                         read of it per cell-step); 0: off. Not for rti_step_noalloc. */
  int nest_feedback;  /* RTI_NEST_RING (0, the default) or RTI_NEST_FULL */
  int nest_flux;      /* RTI_FLUX_LINEAR (0, the default) or RTI_FLUX_CONSTANT */
  int ctas_per_sm;    /* resident CTAs per SM of the step kernel's grid: 0 = as many as fit
                         (the occupancy limit), else at most this many (a tuning knob; the
                         results do not depend on it) */
  double velocity_limit; /* m/s; 0 = off (the default). On, every interior face's flux is
                         also held to |flux| <= velocity_limit x its face depth, after the
                         front's outflow limit: a velocity limiter that binds only near
                         wet/dry fronts, where face depths are small. */
} rti_params;

typedef struct rti_handle rti_handle;
typedef struct rti_batch rti_batch;

/* Device bytes rti_create needs for this hierarchy (the arena size for a caller-owned
 * arena): the planes of every block of the nested grid system (Sec. II-A, Fig. 1's levels
 * and blocks) in the state precision. Validates the descriptors like rti_create (the
 * 1:3 inclusive nesting of Sec. II-A) but reads no bathymetry. */
int rti_footprint(const rti_block* blocks, int nblocks, const rti_params* params, size_t* bytes);

/* Build a hierarchy on the current CUDA device. bathy[b] (nx*ny doubles) and manning[b]
 * (nx*ny floats) are copied. Checks Eq. 4 per block with that block's h_max and the
 * nesting rules. device_mem == NULL: the library allocates and frees the arena;
 * otherwise device_mem (256-byte aligned, device_bytes >= rti_footprint) is used and
 * must outlive the handle. The state starts at rest (eta = 0 on sea, -h on land). */
int rti_create(const rti_block* blocks, int nblocks, const double* const* bathy,
               const float* const* manning, const rti_params* params, void* device_mem,
               size_t device_bytes, rti_handle** out);

/* Initial condition of one block: eta0 = max(dz, -h) on sea cells, -h on land, both
 * fluxes zero, maxima and arrival reset (cells with eta0 >= arrival_thr arrive at t = 0),
 * the block's budget terms reset, and the handle's step counter reset to 0.
 * dz: nx*ny doubles (NULL = sea at rest). */
int rti_set_initial_uplift(rti_handle* h, int block, const double* dz);

/* Enqueue nsteps time steps of the whole hierarchy on `stream` (a cudaStream_t, NULL =
 * the legacy default stream) and return without waiting. One step is the time-integration
 * loop body of Sec. IV-A / Fig. 2 on every block with one dt (Sec. V-A): mass (Eq. 1),
 * fine-to-coarse level (Sec. IV-C-2, Listing 5), momentum (Eqs. 2-3), coarse-to-fine
 * fluxes, output update, buffer swap. Device errors (non-finite level, a bounded wait
 * that ran out) are reported by the next call that waits. */
int rti_step(rti_handle* h, int nsteps, void* stream);

/* Wait for the handle's enqueued work and return its device status. */
int rti_sync(rti_handle* h);
/* Host watchdog: wait at most `seconds` for the handle's enqueued work, polling without a
 * blocking device call. RTI_ERR_TIMEOUT if it has not finished by then (the work stays
 * enqueued; a later wait picks it up), else what rti_sync returns. */
int rti_sync_timeout(rti_handle* h, double seconds);

/* Outputs of one block, nx*ny doubles into caller memory; each waits for enqueued work.
 * max depth = h + max eta over wet instants (0 if never wet); max height = max eta over
 * wet instants (NaN if never wet); arrival = seconds, -1 if never. */
int rti_get_max_depth(rti_handle* h, int block, double* out);
int rti_get_max_height(rti_handle* h, int block, double* out);
int rti_get_arrival_time(rti_handle* h, int block, double* out);
/* Maximum water velocity (Sec. IV-A names it among the outputs of the time loop; the
 * formula is this library's reading): the largest cell-centre speed sqrt(u^2 + v^2) over
 * the initial state and every state a step finished with, on wet cells
 * (h + eta > dry_eps), m/s, 0 if never wet. u = (Mw/Dw + Me/De)/2 and v = (Ns/Ds +
 * Nn/Dn)/2 average the velocities of the cell's four faces, each its flux over its own
 * depth D_f = (h1 + h2)/2 + (eta1 + eta2)/2 (the edge cell's depth on a block edge;
 * velocity 0 where D_f <= dry_eps).
 * Needs track_velocity = 1 at create; otherwise RTI_ERR_STATE. */
int rti_get_max_velocity(rti_handle* h, int block, double* out);

/* State access: current eta (nx*ny), M (ny*(nx+1)), N ((ny+1)*nx) of one block, the
 * variables of Eqs. 1-3 on the staggered grid (eta at cell centres, M and N on the x and
 * y faces), in binary64; a child's edge fluxes are those the next step takes from its
 * parent. NULL skips one. rti_set_state leaves maxima, arrival, budget terms and the step
 * counter unchanged. */
int rti_get_state(rti_handle* h, int block, double* eta, double* M, double* N);
int rti_set_state(rti_handle* h, int block, const double* eta, const double* M,
                  const double* N);

/* Checkpoint and resume of the whole handle, bit for bit: the current level of every
 * block's eta, M and N, its maximum level, arrival steps, speed maximum (when tracked),
 * budget terms, and the step counter, as raw device bytes in the state precision.
 * rti_checkpoint_bytes gives the size of the caller's host buffer; rti_checkpoint_save
 * fills it (waiting for enqueued work); rti_checkpoint_load restores it into a handle
 * created with the same blocks and params (RTI_ERR_INVALID_ARG otherwise), after which
 * stepping continues exactly as the saved handle would have. */
size_t rti_checkpoint_bytes(const rti_handle* h);
int rti_checkpoint_save(rti_handle* h, void* host_buf, size_t bytes);
int rti_checkpoint_load(rti_handle* h, const void* host_buf, size_t bytes);

/* Volume budget of one block (binary64): out[0] = water volume sum (h + eta) dx^2,
 * out[1] = cumulative volume that left through the block's boundary faces, out[2] =
 * cumulative volume added by the dry clip, out[3] = cumulative change from the
 * fine-to-coarse ring replacement. V(t) = V(0) - out[1] + out[2] + out[3]. */
int rti_get_budget(rti_handle* h, int block, double out[4]);

/* Volume budget of the whole domain (binary64), over the root blocks, whose cells hold
 * the water of the regions their children refine as well (the fine-to-coarse feedback
 * keeps them consistent): volume = sum of out[0], boundary_outflow = volume that left
 * through the domain's edges (radiation faces), clip_volume = volume the dry clip
 * added, feedback_volume = change from the fine-to-coarse feedback, so that
 * volume(t) = volume(0) - boundary_outflow + clip_volume + feedback_volume. Any output
 * may be NULL. Waits for enqueued work. */
int rti_volume(rti_handle* h, double* volume, double* boundary_outflow, double* clip_volume,
               double* feedback_volume);

/* Host<->device bytes this handle's calls have copied so far (inputs, initial state,
 * outputs, checkpoints). */
int rti_get_transfer_bytes(const rti_handle* h, long long* h2d, long long* d2h);

/* Steps completed (after the enqueued work finishes). */
long long rti_steps_done(rti_handle* h);
int rti_num_blocks(const rti_handle* h);
long long rti_num_cells(const rti_handle* h);

void rti_destroy(rti_handle* h);
/* message of the handle's last failure; with NULL, of the last failed rti_create or
 * rti_step_noalloc on the calling thread */
const char* rti_last_error(const rti_handle* h);
const char* rti_error_string(int code);

/* ---- Allocation-free stepping of one grid ----
 * The paper has no counterpart to this call. It serves callers that cannot call
 * cudaMalloc: a process whose device memory is handed in full to its own pool allocator
 * (a forecast service that reserves HBM for its scenario slots at start-up), and code
 * that must not allocate because an allocation can fail once that reservation is made
 * or can synchronise the device and stall the other streams of a real-time service.
 * rti_create allocates its arena, tables and events; this call allocates nothing: the
 * caller owns the state arrays and the call takes its scratch (block descriptor, tile
 * list, counters, device barrier, status words, budget partials) from one file-scope
 * device array of about 200 KB that every GPU which loads the library holds until the
 * process exits. Limit: a single root grid (parent -1) of at most 4096 strips (2048 x 2048
 * cells make 2368 of the default 28 x 64 strips); larger grids return RTI_ERR_INVALID_ARG and
 * rti_last_error(NULL) says why.
 *
 * State layout (element type double for RTI_FP64, float for RTI_FP32; manning is always
 * float and arrival_step int): every array starts on a 16-byte boundary and has `pitch`
 * elements per row with pitch >= nx + 9 and a multiple of 4, and ny + 5 rows, with
 * pitch x (ny + 5) < 2^31; element
 * (column c, row r) lives at
 * (r + 2) * pitch + (c + 4). Cells use columns 0..nx-1 and rows 0..ny-1, M uses columns
 * 0..nx, N rows 0..ny. eta/M/N come in two time levels: level (steps_done & 1) is the
 * current one on entry, level ((steps_done + nsteps) & 1) on return. max_eta starts at
 * eta0 on wet cells and -1e30 elsewhere; arrival_step at 0 where eta0 >= arrival_thr on
 * wet cells and -1 elsewhere. steps_done numbers the steps for the arrival record.
 *
 * The call steps nsteps times on `stream` (a cudaStream_t, NULL = legacy default), reads
 * the status words on that stream, synchronises the stream (it returns only when its
 * work has finished) and returns the device status (RTI_ERR_NONFINITE, RTI_ERR_TIMEOUT). Its
 * first call on a device looks up the scratch address; make that first call before any
 * stream capture. Every call shares the one scratch array, which keeps the previous
 * call's contents (the call clears what must start at zero); calls that overlap on the
 * GPU, from several threads or streams, race on it. It does not check Eq. 4 (it reads no
 * bathymetry on the host). */
typedef struct {
  void* eta[2];
  void* M[2];
  void* N[2];
  const void* h;
  const float* manning;
  void* max_eta;
  int* arrival_step;
  int pitch; /* elements per row of every array */
} rti_noalloc_state;

int rti_step_noalloc(const rti_block* grid, const rti_params* params,
                     const rti_noalloc_state* state, long long steps_done, int nsteps,
                     void* stream);

/* ---- Batches: many hierarchies stepped together in one persistent launch ----
 * The paper steps one hierarchy per run (Sec. IV-A) and launches a kernel per block on
 * asynchronous queues (Sec. IV-B); a batch steps the blocks of many independent
 * hierarchies (earthquake scenarios) through the same loop body in one launch, each
 * hierarchy exactly as rti_step would. All handles of a batch share one precision. A
 * handle in a batch is stepped only by rti_batch_step (rti_step returns RTI_ERR_STATE).
 * Adding or removing members patches the device-resident tile list; the captured CUDA
 * graph is reused. */
int rti_batch_create(int precision, int schedule, int chunk_steps, rti_batch** out);
/* The same with the strip height and CTA cap of the batch (members must be created with
 * the same tile_y); rti_batch_create uses tile_y 64 and no cap. */
typedef struct {
  int precision;   /* RTI_FP64 or RTI_FP32 */
  int schedule;    /* RTI_SCHED_* */
  int chunk_steps; /* steps per rti_batch_step */
  int tile_y;      /* strip height, a multiple of 8; 0 = 64 */
  int ctas_per_sm; /* as in rti_params */
} rti_batch_config;
int rti_batch_create_ex(const rti_batch_config* cfg, rti_batch** out);
/* add a member that will take `nsteps` more steps, then stop */
int rti_batch_add(rti_batch* b, rti_handle* h, long long nsteps);
int rti_batch_remove(rti_batch* b, rti_handle* h);
/* Enqueue one chunk (chunk_steps steps; members with fewer remaining steps stop early). */
int rti_batch_step(rti_batch* b, void* stream);
/* steps a member still has to take, as of the enqueued work */
long long rti_batch_remaining(rti_batch* b, rti_handle* h);
int rti_batch_sync(rti_batch* b);
/* rti_batch_sync with the host watchdog of rti_sync_timeout */
int rti_batch_sync_timeout(rti_batch* b, double seconds);
void rti_batch_destroy(rti_batch* b);

#ifdef __cplusplus
}
#endif
#endif
