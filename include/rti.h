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
#define RTI_ERR_TIMEOUT -6     /* a device-wide barrier wait ran out; the state is undefined */
#define RTI_ERR_CUDA -7        /* a CUDA runtime call failed (message in rti_last_error) */
#define RTI_ERR_STATE -8       /* call not allowed in the current state (e.g. handle in a batch) */

#define RTI_BC_WALL 0      /* zero normal flux */
#define RTI_BC_RADIATION 1 /* outward flux sqrt(g h) * eta of the edge cell (root blocks only) */

#define RTI_FP64 0 /* all state and arithmetic in binary64 */
#define RTI_FP32 1 /* state and arithmetic in binary32; eta is the deviation from still water;
                      the volume budget and the nesting sums accumulate in binary64 */

#define RTI_SCHED_PERSISTENT 0 /* one cooperative launch per chunk of steps, device-wide barriers */
#define RTI_SCHED_PER_PASS 1   /* two launches per step (mass pass, momentum pass) */

/* One rectangular block of a grid level (Sec. II-A "blocks"). */
typedef struct {
  int level;  /* 1 for the root level, parent level + 1 otherwise */
  int parent; /* index of the parent block in the same array, -1 for a root */
  int nx, ny; /* cells; multiples of 3 for a child */
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
  int tile_x, tile_y; /* tile shape in cells, 0 = library default */
} rti_params;

typedef struct rti_handle rti_handle;
typedef struct rti_batch rti_batch;

/* Device bytes rti_create needs for this hierarchy (the arena size for a caller-owned
 * arena). Validates the descriptors like rti_create but reads no bathymetry. */
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
 * the legacy default stream) and return without waiting. Device errors (non-finite
 * level, barrier timeout) are reported by the next call that waits. */
int rti_step(rti_handle* h, int nsteps, void* stream);

/* Wait for the handle's enqueued work and return its device status. */
int rti_sync(rti_handle* h);

/* Outputs of one block, nx*ny doubles into caller memory; each waits for enqueued work.
 * max depth = h + max eta over wet instants (0 if never wet); max height = max eta over
 * wet instants (NaN if never wet); arrival = seconds, -1 if never. */
int rti_get_max_depth(rti_handle* h, int block, double* out);
int rti_get_max_height(rti_handle* h, int block, double* out);
int rti_get_arrival_time(rti_handle* h, int block, double* out);

/* Checkpoint access: current eta (nx*ny), M (ny*(nx+1)), N ((ny+1)*nx); NULL skips one.
 * rti_set_state leaves maxima, arrival, budget terms and the step counter unchanged. */
int rti_get_state(rti_handle* h, int block, double* eta, double* M, double* N);
int rti_set_state(rti_handle* h, int block, const double* eta, const double* M,
                  const double* N);

/* Volume budget of one block (binary64): out[0] = water volume sum (h + eta) dx^2,
 * out[1] = cumulative volume that left through the block's boundary faces, out[2] =
 * cumulative volume added by the dry clip, out[3] = cumulative change from the
 * fine-to-coarse ring replacement. V(t) = V(0) - out[1] + out[2] + out[3]. */
int rti_get_budget(rti_handle* h, int block, double out[4]);

/* Host<->device bytes this handle's calls have copied so far (inputs, initial state,
 * outputs, checkpoints). */
int rti_get_transfer_bytes(const rti_handle* h, long long* h2d, long long* d2h);

/* Steps completed (after the enqueued work finishes). */
long long rti_steps_done(rti_handle* h);
int rti_num_blocks(const rti_handle* h);
long long rti_num_cells(const rti_handle* h);

void rti_destroy(rti_handle* h);
const char* rti_last_error(const rti_handle* h);
const char* rti_error_string(int code);

/* ---- Batches: many hierarchies stepped together in one persistent launch ----
 * All handles of a batch share one precision. A handle in a batch is stepped only by
 * rti_batch_step (rti_step returns RTI_ERR_STATE). Adding or removing members patches
 * the device-resident tile list; the captured CUDA graph is reused. */
int rti_batch_create(int precision, int schedule, int chunk_steps, rti_batch** out);
/* add a member that will take `nsteps` more steps, then stop */
int rti_batch_add(rti_batch* b, rti_handle* h, long long nsteps);
int rti_batch_remove(rti_batch* b, rti_handle* h);
/* Enqueue one chunk (chunk_steps steps; members with fewer remaining steps stop early). */
int rti_batch_step(rti_batch* b, void* stream);
/* steps a member still has to take, as of the enqueued work */
long long rti_batch_remaining(rti_batch* b, rti_handle* h);
int rti_batch_sync(rti_batch* b);
void rti_batch_destroy(rti_batch* b);

#ifdef __cplusplus
}
#endif
#endif
