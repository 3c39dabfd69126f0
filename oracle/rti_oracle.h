/*
 * rti_oracle.h -- plain FP64 CPU oracle for the RTi / TUNAMI-N2 time step.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this library. The product path (the CUDA library
 * under paper_2408_07609_gb300/) never includes, links or calls it, and it
 * shares no code with that path.
 *
 * What it computes: one leap-frog step on staggered grids of the nonlinear
 * shallow-water equations (Takahashi et al., Sec. II-A, Eqs. 1-3) on 1:3
 * nested blocks (Sec. II-A, inclusive nesting, single dt on all levels,
 * Sec. V-A), in the order of the time-integration loop of Sec. IV-A / Fig. 2:
 * mass -> child-to-parent eta -> momentum -> parent-to-child flux -> output
 * update -> buffer swap. The paper gives the PDEs only; every discrete choice
 * made here is a stated reading (R1..R11 in the comments of rti_oracle.c).
 */
#ifndef RTI_ORACLE_H
#define RTI_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BC_WALL 0
#define ORC_BC_RADIATION 1

#define ORC_OK 0
#define ORC_ERR_INVALID_ARG -1
#define ORC_ERR_CFL -2
#define ORC_ERR_NESTING -3
#define ORC_ERR_OOM -4

typedef struct {
  int level;   /* 1 = root */
  int parent;  /* index of the parent block, -1 for a root block */
  int nx, ny;  /* cells */
  int i0, j0;  /* origin of a child, in parent cells */
  double dx;   /* cell size (m); a child has parent dx / 3 */
  int bc[4];   /* west, east, south, north: ORC_BC_WALL or ORC_BC_RADIATION (roots only) */
} orc_block;

#define ORC_NEST_RING 0     /* fine->coarse: the parent cells on the footprint's inner ring */
#define ORC_NEST_FULL 1     /* fine->coarse: every parent cell the child covers */
#define ORC_FLUX_LINEAR 0   /* coarse->fine: flux interpolated linearly along the edge */
#define ORC_FLUX_CONSTANT 1 /* coarse->fine: each fine face takes its coarse face's flux */

typedef struct {
  double dt;          /* s, same on every level */
  double g;           /* m/s^2 */
  double dry_eps;     /* m: a cell is wet when h + eta > dry_eps */
  double arrival_thr; /* m: arrival when max eta first reaches this */
  int nest_feedback;  /* ORC_NEST_RING or ORC_NEST_FULL */
  int nest_flux;      /* ORC_FLUX_LINEAR or ORC_FLUX_CONSTANT */
  double vel_limit;   /* m/s: |flux| <= vel_limit * face depth at every interior face
                         (R12); 0 = no limit */
} orc_params;

typedef struct orc_state orc_state;

/* bathy[b]: nx*ny doubles, h > 0 sea depth, h <= 0 land; manning[b]: nx*ny floats.
 * Row-major, x fastest. Inputs are copied. Returns NULL and sets *err on failure. */
orc_state* orc_create(const orc_block* blocks, int nblocks, const double* const* bathy,
                      const float* const* manning, const orc_params* p, int* err);
void orc_destroy(orc_state* s);

/* eta0 = max(dz, -h) on sea cells, -h on land; M = N = 0; maxima, arrival and the
 * block's budget terms reset; step counter of the whole state reset to 0. */
int orc_set_initial_uplift(orc_state* s, int block, const double* dz);
int orc_step(orc_state* s, int nsteps);
long orc_steps_done(const orc_state* s);

/* eta: nx*ny, M: ny*(nx+1) (face f of row j at j*(nx+1)+f), N: (ny+1)*nx. */
int orc_get_state(const orc_state* s, int block, double* eta, double* M, double* N);
int orc_set_state(orc_state* s, int block, const double* eta, const double* M, const double* N);
/* max eta over wet instants (NaN if never wet) */
int orc_get_max_height(const orc_state* s, int block, double* out);
/* max total depth h + eta over wet instants (0 if never wet) */
int orc_get_max_depth(const orc_state* s, int block, double* out);
/* seconds, -1 if max eta never reached the threshold */
int orc_get_arrival_time(const orc_state* s, int block, double* out);
/* R11: max over the initial state and every finished step of the cell-centre speed
 * sqrt(u^2 + v^2), u = (Mw/Dw + Me/De)/2, v = (Ns/Ds + Nn/Dn)/2 with D_f the depth of each
 * face (0 velocity on a face without water), on wet cells, m/s (0 if never wet) */
int orc_get_max_velocity(const orc_state* s, int block, double* out);
/* out[0] = water volume sum (h+eta) dx^2, out[1] = cumulative volume that left through
 * the block boundary, out[2] = cumulative volume added by the dry clip, out[3] = cumulative
 * volume changed by the fine-to-coarse replacement of parent cells (R8). */
int orc_get_budget(const orc_state* s, int block, double* out);
/* the cube root the friction term uses (a stated Newton iteration; see rti_oracle.c) */
double orc_cube_root(double x);

/* One step in phases, for a hierarchy whose blocks are split over several ranks (each
 * rank holds a state of the whole hierarchy and steps its own blocks). Per step:
 *   1. orc_phase_mass for each own block;
 *   2. orc_pack_means for each own child (orc_means_count values) -> the parent's rank;
 *   3. orc_unpack_means for each child of an own parent, in decreasing block order;
 *   4. orc_phase_momentum for each own block;
 *   5. orc_get_edge_fluxes on the parent's rank (orc_edge_count values) -> the child's
 *      rank, orc_set_edge_fluxes there; orc_phase_edges for each own child;
 *   6. orc_phase_swap for each own block, orc_end_step once.
 * On one rank with every block this performs orc_step's operations in its order. */
int orc_phase_mass(orc_state* s, int block);
int orc_means_count(const orc_state* s, int child);
int orc_pack_means(const orc_state* s, int child, double* out);
int orc_unpack_means(orc_state* s, int child, const double* in);
int orc_phase_momentum(orc_state* s, int block);
int orc_edge_count(const orc_state* s, int child);
int orc_get_edge_fluxes(const orc_state* s, int child, double* out);
int orc_set_edge_fluxes(orc_state* s, int child, const double* in);
int orc_phase_edges(orc_state* s, int child);
int orc_phase_swap(orc_state* s, int block);
int orc_end_step(orc_state* s);

#ifdef __cplusplus
}
#endif
#endif
