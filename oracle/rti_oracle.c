/*
 * rti_oracle.c -- plain FP64 CPU oracle of the RTi / TUNAMI-N2 time step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline). Slow on purpose: one plain loop per rule, no blocking, no fusion,
 * no reordering beyond what the rules below state. Build with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * The same source builds single-threaded and, with -fopenmp, with the rows of
 * each loop shared among threads. Every cell's arithmetic is the same in both,
 * and the one sum over cells inside a step (the clip volume of R5) is formed
 * per row and then added row by row in order, so both builds give identical
 * bits.
 *
 * Source: Takahashi et al., "Modernizing an Operational Real-time Tsunami
 * Simulator to Support Diverse Hardware Platforms".
 *   Eq. 1 (Sec. II-A)  continuity  d(eta)/dt + dM/dx + dN/dy = 0
 *   Eq. 2, Eq. 3       momentum with advection, g D grad(eta) and Manning friction
 *                      g n^2 D^(-7/3) M sqrt(M^2+N^2); D = h + eta
 *   Eq. 4              CFL  dx/dt >= sqrt(2 g h_max)
 *   Sec. II-A          leap-frog in time, staggered grid, 1:3 inclusive nesting
 *   Sec. IV-A, Fig. 2  loop order: mass, child->parent eta, momentum,
 *                      parent->child fluxes, output update, buffer swap
 *   Sec. IV-C-2, Listing 5  child->parent eta = (sum of a 3x3 child patch) * (1/9)
 *   Sec. V-A           one dt on all levels
 * The paper gives no discrete stencil. The readings used here:
 *   R1  mass: eta1 = eta - ((dt/dx)(Me - Mw) + (dt/dx)(Nn - Ns)), every cell.
 *   R2  x-momentum at interior faces: D_f = (hL+hR)/2 + (etaL+etaR)/2 from the new
 *       eta; first-order upwind advection on the sign of M (x) and of the 4-point mean
 *       N (y), each flux over its own face depth; centred when the sign is zero;
 *       dropped when a face it needs is a block-boundary face or has D <= dry_eps;
 *       pressure g D_f (dt/dx)(etaR - etaL); semi-implicit Manning friction
 *       F = (dt/2) g n_f^2 sqrt(M^2 + Nbar^2) / (D_f^2 cbrt(D_f)), n_f = max(nL, nR);
 *       M1 = ((1 - F) M - dt Adv - P) / (1 + F). The cube root is the stated Newton
 *       iteration of cube_root() below, not a math library's cbrt: every other operation
 *       of the step is an IEEE-rounded +, -, *, / or sqrt, so with it a binary64
 *       implementation that performs the same operations in the same order reproduces
 *       this oracle bit for bit, at any run length.
 *   R3  y-momentum: R2 with x and y exchanged, same operation order.
 *   R4  wet/dry front: a cell is wet when h + eta > dry_eps. Both wet: R2. One wet and
 *       its level above the dry cell's ground: D_f = eta_wet + h_dry, gradient against
 *       the dry ground level, no advection. Otherwise, or when D_f <= dry_eps, zero.
 *   R5  clip after R1: if h + eta < 0 then eta = -h; the added volume is counted.
 *   R6  root-block edges: wall = zero flux; radiation = outward sqrt(g max(h,0)) eta of
 *       the adjacent cell when that cell is wet, else zero.
 *   R7  coarse->fine: each child edge face takes the parent flux on the coarse face it
 *       lies on, linearly interpolated along the edge (weights 2/3, 1/3 at the outer fine
 *       faces, neighbour clamped at the segment ends); no time interpolation.
 *       Option ORC_FLUX_CONSTANT: the three fine faces of a coarse face all take its
 *       flux unchanged (piecewise constant, so the edge carries exactly the coarse
 *       face's discharge).
 *   R8  fine->coarse: parent cells on the inner ring of the child footprint take the
 *       Listing 5 mean of their 3x3 child cells (x outer, y inner, FP64 sum, times 1/9).
 *       Only wet child cells enter the mean (sum times 1/count; all nine wet gives the
 *       listing's formula exactly); the result is floored at the parent's ground level
 *       -h; a patch with no wet cell leaves the parent's own value. Averaging dry land
 *       levels into a sea cell would break the lake at rest.
 *       Option ORC_NEST_FULL: every parent cell the child covers takes that mean (full
 *       two-way nesting). The exchange is simultaneous, as a pack-then-unpack of every
 *       level's messages: all means are formed from the levels the mass step left,
 *       before any block receives. A parent cell above a grandchild therefore gets the
 *       child's own level there; the grandchild's mean reaches it one step later. With
 *       the ring option the order does not matter: the 3-cell nesting margin keeps a
 *       ring's patches away from the cells the child itself receives.
 *   R9  after R8: on wet cells, etamax = max(etamax, eta); the arrival step is recorded
 *       when etamax first reaches the threshold (>=).
 *   R10 initial state: eta0 = max(dz, -h) on sea cells, -h on land, fluxes zero.
 *   R11 maximum water velocity (the output update of Sec. IV-A names it; no formula is
 *       given): cell-centre velocity of a state as the mean of its faces' velocities,
 *       u = (Mw/Dw + Me/De)/2, v = (Ns/Ds + Nn/Dn)/2, where a face's velocity is its flux
 *       over its depth D_f = (h1 + h2)/2 + (eta1 + eta2)/2 (the two cells it separates;
 *       on a block edge the edge cell's own depth), and 0 where D_f <= dry_eps; kept as
 *       the square u^2 + v^2 on wet cells (D = h + eta > dry_eps). Dividing each face's
 *       flux by its own depth keeps the speed of a film barely above the wet threshold
 *       that a neighbour floods at the speed of the flow through its faces; dividing the
 *       mean flux by the film's depth gave hundreds of m/s. It is taken from the state
 *       each step starts from (the state the previous iteration finished with), and the
 *       read adds the current state, so the result is the maximum over the initial state
 *       and every state a step finished with; 0 if never wet.
 *   R12 velocity limit (option vel_limit, off by default): after R4's outflow limit, an
 *       interior face's flux is also held to |flux| <= vel_limit * D_f with D_f the face
 *       depth of its update (R2, or R4's front depth). In open water it never binds
 *       (tsunami currents are a few m/s); near a front, where D_f is small, it caps the
 *       flux that floods or drains a thin layer.
 */
#include "rti_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NEVER_WET (-1.0e30)

typedef struct {
  orc_block d;
  int nx, ny;
  double dx, dtdx;
  double* h;    /* nx*ny */
  double* n;    /* nx*ny, Manning n (input floats, exactly widened) */
  double* eta;  /* eta^n */
  double* eta1; /* eta^{n+1} */
  double* M;    /* ny*(nx+1) */
  double* M1;
  double* N;    /* (ny+1)*nx */
  double* N1;
  double* emax;
  long* arr;     /* arrival step, -1 if never */
  double* vmax2; /* R11: max squared cell-centre speed on wet instants (0 if never) */
  double* rowsum; /* ny: the clip volume of each row in the current step */
  double outflow, clip, ring;
} oblk;

struct orc_state {
  int nb;
  oblk* b;
  orc_params p;
  long step;
};

/* index helpers: cell (i,j), x-face (f,j), y-face (i,g) */
#define C(b, i, j) ((size_t)(j) * (size_t)(b)->nx + (size_t)(i))
#define FX(b, f, j) ((size_t)(j) * (size_t)((b)->nx + 1) + (size_t)(f))
#define FY(b, i, g) ((size_t)(g) * (size_t)(b)->nx + (size_t)(i))

static void free_blk(oblk* b) {
  free(b->h); free(b->n); free(b->eta); free(b->eta1); free(b->M); free(b->M1);
  free(b->N); free(b->N1); free(b->emax); free(b->arr); free(b->vmax2); free(b->rowsum);
}

void orc_destroy(orc_state* s) {
  if (!s) return;
  for (int k = 0; k < s->nb; ++k) free_blk(&s->b[k]);
  free(s->b);
  free(s);
}

static int check_blocks(const orc_block* bl, int nb, const double* const* bathy,
                        const orc_params* p) {
  for (int k = 0; k < nb; ++k) {
    const orc_block* d = &bl[k];
    if (d->nx < 3 || d->ny < 3 || !(d->dx > 0)) return ORC_ERR_INVALID_ARG;
    /* Eq. 4: dx / dt >= sqrt(2 g h_max) on every block */
    double hmax = 0;
    for (size_t c = 0; c < (size_t)d->nx * d->ny; ++c)
      if (bathy[k][c] > hmax) hmax = bathy[k][c];
    if (d->dx / p->dt < sqrt(2.0 * p->g * hmax)) return ORC_ERR_CFL;
    if (d->parent < 0) {
      if (d->level != 1) return ORC_ERR_NESTING;
      continue;
    }
    if (d->parent >= k) return ORC_ERR_NESTING; /* parents come first */
    const orc_block* P = &bl[d->parent];
    if (d->level != P->level + 1) return ORC_ERR_NESTING;
    if (d->nx % 3 || d->ny % 3) return ORC_ERR_NESTING;
    if (fabs(d->dx * 3.0 - P->dx) > 1e-9 * P->dx) return ORC_ERR_NESTING;
    /* inclusive nesting with a 3-cell margin inside the parent */
    if (d->i0 < 3 || d->j0 < 3 || d->i0 + d->nx / 3 > P->nx - 3 || d->j0 + d->ny / 3 > P->ny - 3)
      return ORC_ERR_NESTING;
    for (int q = 0; q < k; ++q) { /* siblings may touch but not overlap */
      const orc_block* o = &bl[q];
      if (o->parent != d->parent) continue;
      int ox = d->i0 < o->i0 + o->nx / 3 && o->i0 < d->i0 + d->nx / 3;
      int oy = d->j0 < o->j0 + o->ny / 3 && o->j0 < d->j0 + d->ny / 3;
      if (ox && oy) return ORC_ERR_NESTING;
    }
  }
  return ORC_OK;
}

orc_state* orc_create(const orc_block* blocks, int nblocks, const double* const* bathy,
                      const float* const* manning, const orc_params* p, int* err) {
  int e = ORC_OK;
  if (!blocks || nblocks <= 0 || !bathy || !manning || !p || !(p->dt > 0) || !(p->g > 0) ||
      (p->nest_feedback != ORC_NEST_RING && p->nest_feedback != ORC_NEST_FULL) ||
      (p->nest_flux != ORC_FLUX_LINEAR && p->nest_flux != ORC_FLUX_CONSTANT) ||
      !(p->vel_limit >= 0))
    e = ORC_ERR_INVALID_ARG;
  for (int k = 0; e == ORC_OK && k < nblocks; ++k)
    if (!bathy[k] || !manning[k]) e = ORC_ERR_INVALID_ARG;
  if (e == ORC_OK) e = check_blocks(blocks, nblocks, bathy, p);
  if (e != ORC_OK) {
    if (err) *err = e;
    return NULL;
  }
  orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
  if (!s) goto oom;
  s->b = (oblk*)calloc((size_t)nblocks, sizeof(oblk));
  if (!s->b) goto oom;
  s->nb = nblocks;
  s->p = *p;
  for (int k = 0; k < nblocks; ++k) {
    oblk* b = &s->b[k];
    b->d = blocks[k];
    b->nx = blocks[k].nx;
    b->ny = blocks[k].ny;
    b->dx = blocks[k].dx;
    b->dtdx = p->dt / b->dx;
    size_t nc = (size_t)b->nx * b->ny;
    size_t nfx = (size_t)(b->nx + 1) * b->ny;
    size_t nfy = (size_t)b->nx * (b->ny + 1);
    b->h = (double*)malloc(nc * sizeof(double));
    b->n = (double*)malloc(nc * sizeof(double));
    b->eta = (double*)calloc(nc, sizeof(double));
    b->eta1 = (double*)calloc(nc, sizeof(double));
    b->M = (double*)calloc(nfx, sizeof(double));
    b->M1 = (double*)calloc(nfx, sizeof(double));
    b->N = (double*)calloc(nfy, sizeof(double));
    b->N1 = (double*)calloc(nfy, sizeof(double));
    b->emax = (double*)malloc(nc * sizeof(double));
    b->arr = (long*)malloc(nc * sizeof(long));
    b->vmax2 = (double*)calloc(nc, sizeof(double));
    b->rowsum = (double*)calloc((size_t)b->ny, sizeof(double));
    if (!b->h || !b->n || !b->eta || !b->eta1 || !b->M || !b->M1 || !b->N || !b->N1 ||
        !b->emax || !b->arr || !b->vmax2 || !b->rowsum)
      goto oom;
    for (size_t c = 0; c < nc; ++c) {
      b->h[c] = bathy[k][c];
      b->n[c] = (double)manning[k][c];
    }
  }
  for (int k = 0; k < nblocks; ++k) orc_set_initial_uplift(s, k, NULL);
  if (err) *err = ORC_OK;
  return s;
oom:
  orc_destroy(s);
  if (err) *err = ORC_ERR_OOM;
  return NULL;
}

/* R9: output update of one cell, after R8 */
static void track_cell(oblk* b, size_t c, long step, const orc_params* p) {
  double e = b->eta1[c];
  if (b->h[c] + e > p->dry_eps && e > b->emax[c]) {
    if (b->emax[c] < p->arrival_thr && e >= p->arrival_thr) b->arr[c] = step;
    b->emax[c] = e;
  }
}

/* R11: depth of the face between cells a and b of the state eta (a == b on a block edge) */
static double face_depth(const oblk* b, const double* eta, size_t ca, size_t cb) {
  return 0.5 * (b->h[ca] + b->h[cb]) + 0.5 * (eta[ca] + eta[cb]);
}

/* R11: velocity across a face of flux q and depth D (0 on a face without water) */
static double face_velocity(double q, double D, double eps) { return D > eps ? q / D : 0.0; }

/* R11: squared cell-centre speed of cell (i, j) in the state (eta, M, N); -1 if dry */
static double speed2(const oblk* b, const double* eta, const double* M, const double* N, int i,
                     int j, const orc_params* p) {
  const size_t c = C(b, i, j);
  double D = b->h[c] + eta[c];
  if (!(D > p->dry_eps)) return -1.0;
  const double eps = p->dry_eps;
  double Dw = face_depth(b, eta, i > 0 ? C(b, i - 1, j) : c, c);
  double De = face_depth(b, eta, c, i < b->nx - 1 ? C(b, i + 1, j) : c);
  double Ds = face_depth(b, eta, j > 0 ? C(b, i, j - 1) : c, c);
  double Dn = face_depth(b, eta, c, j < b->ny - 1 ? C(b, i, j + 1) : c);
  double u = 0.5 * (face_velocity(M[FX(b, i, j)], Dw, eps) + face_velocity(M[FX(b, i + 1, j)], De, eps));
  double v = 0.5 * (face_velocity(N[FY(b, i, j)], Ds, eps) + face_velocity(N[FY(b, i, j + 1)], Dn, eps));
  return u * u + v * v;
}

/* R11 output update: the state a step starts from */
static void track_speed(oblk* b, const orc_params* p) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < b->ny; ++j)
    for (int i = 0; i < b->nx; ++i) {
      double s2 = speed2(b, b->eta, b->M, b->N, i, j, p);
      if (s2 > b->vmax2[C(b, i, j)]) b->vmax2[C(b, i, j)] = s2;
    }
}

/* R10 (dz == NULL: sea at rest) */
int orc_set_initial_uplift(orc_state* s, int k, const double* dz) {
  if (!s || k < 0 || k >= s->nb) return ORC_ERR_INVALID_ARG;
  oblk* b = &s->b[k];
  size_t nc = (size_t)b->nx * b->ny;
  for (size_t c = 0; c < nc; ++c) {
    double h = b->h[c];
    double e;
    if (h > 0) {
      e = dz ? dz[c] : 0.0;
      if (e < -h) e = -h;
    } else {
      e = -h;
    }
    b->eta[c] = e;
    b->eta1[c] = e;
    b->emax[c] = NEVER_WET;
    b->arr[c] = -1;
    b->vmax2[c] = 0.0;
    track_cell(b, c, 0, &s->p);
  }
  memset(b->M, 0, (size_t)(b->nx + 1) * b->ny * sizeof(double));
  memset(b->M1, 0, (size_t)(b->nx + 1) * b->ny * sizeof(double));
  memset(b->N, 0, (size_t)b->nx * (b->ny + 1) * sizeof(double));
  memset(b->N1, 0, (size_t)b->nx * (b->ny + 1) * sizeof(double));
  b->outflow = 0;
  b->clip = 0;
  b->ring = 0;
  s->step = 0;
  return ORC_OK;
}

/* ---- R1 + R5: mass (Eq. 1) over one block, with boundary outflow bookkeeping ---- */
static void mass_block(oblk* b, const orc_params* p) {
  const double dtdx = b->dtdx, dx2 = b->dx * b->dx, vol = p->dt * b->dx;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < b->ny; ++j) {
    double clip_row = 0.0;
    for (int i = 0; i < b->nx; ++i) {
      double Mw = b->M[FX(b, i, j)], Me = b->M[FX(b, i + 1, j)];
      double Ns = b->N[FY(b, i, j)], Nn = b->N[FY(b, i, j + 1)];
      size_t c = C(b, i, j);
      double e = b->eta[c] - (dtdx * (Me - Mw) + dtdx * (Nn - Ns));
      if (b->h[c] + e < 0) {
        clip_row += (-b->h[c] - e) * dx2;
        e = -b->h[c];
      }
      b->eta1[c] = e;
    }
    b->rowsum[j] = clip_row;
  }
  for (int j = 0; j < b->ny; ++j) b->clip += b->rowsum[j];
  /* volume that left through the block's own boundary faces this step */
  for (int j = 0; j < b->ny; ++j) {
    b->outflow += vol * (-b->M[FX(b, 0, j)]);
    b->outflow += vol * b->M[FX(b, b->nx, j)];
  }
  for (int i = 0; i < b->nx; ++i) {
    b->outflow += vol * (-b->N[FY(b, i, 0)]);
    b->outflow += vol * b->N[FY(b, i, b->ny)];
  }
}

/* ---- R8: fine->coarse (Listing 5) ---- */
/* does parent cell (I, J) of a child footprint a x bb cells receive the child's mean? */
static int receives(const orc_params* p, int I, int J, int a, int bb) {
  if (p->nest_feedback == ORC_NEST_FULL) return 1;
  return I == 0 || I == a - 1 || J == 0 || J == bb - 1; /* the inner ring */
}

/* pack: the mean of the wet child cells of every receiving parent cell of child k, from
 * the child's eta^{n+1}, into out[J * a + I]; NAN where the patch has no wet cell or
 * the cell does not receive */
static void pack_child(const orc_state* s, int k, double* out) {
  const oblk* c = &s->b[k];
  int a = c->nx / 3, bb = c->ny / 3;
#pragma omp parallel for schedule(static)
  for (int J = 0; J < bb; ++J) {
    for (int I = 0; I < a; ++I) {
      out[(size_t)J * a + I] = NAN;
      if (!receives(&s->p, I, J, a, bb)) continue;
      double sum = 0.0;
      int wet = 0;
      for (int x = 3 * I; x < 3 * I + 3; ++x) {   /* outer: x (the paper's J) */
        for (int y = 3 * J; y < 3 * J + 3; ++y) { /* inner: y (the paper's I) */
          size_t q = C(c, x, y);
          if (c->h[q] + c->eta1[q] > s->p.dry_eps) {
            sum = sum + c->eta1[q];
            wet = wet + 1;
          }
        }
      }
      if (wet == 0) continue;                  /* dry patch: the parent keeps its value */
      out[(size_t)J * a + I] = sum * (1.0 / (double)wet); /* all 9 wet: SUMZ * (1.0/9.0) */
    }
  }
}

/* unpack: the parent of child k takes the packed means, floored at its ground level */
static void unpack_child(orc_state* s, int k, const double* in) {
  const oblk* c = &s->b[k];
  oblk* P = &s->b[c->d.parent];
  int a = c->nx / 3, bb = c->ny / 3;
  double dx2 = P->dx * P->dx;
  for (int J = 0; J < bb; ++J) {
    for (int I = 0; I < a; ++I) {
      double avg = in[(size_t)J * a + I];
      if (isnan(avg)) continue;
      size_t pc = C(P, c->d.i0 + I, c->d.j0 + J);
      if (avg < -P->h[pc]) avg = -P->h[pc];
      P->ring += (avg - P->eta1[pc]) * dx2;
      P->eta1[pc] = avg;
    }
  }
}

/* every child packs, then every parent unpacks (finest children first) */
static void fine_to_coarse(orc_state* s) {
  double** buf = (double**)calloc((size_t)s->nb, sizeof(double*));
  if (!buf) abort();
  for (int k = 0; k < s->nb; ++k) {
    const oblk* c = &s->b[k];
    if (c->d.parent < 0) continue;
    buf[k] = (double*)malloc((size_t)(c->nx / 3) * (size_t)(c->ny / 3) * sizeof(double));
    if (!buf[k]) abort();
    pack_child(s, k, buf[k]);
  }
  for (int k = s->nb - 1; k >= 0; --k)
    if (buf[k]) unpack_child(s, k, buf[k]);
  for (int k = 0; k < s->nb; ++k) free(buf[k]);
  free(buf);
}

/* ---- R2/R3 helpers. x-faces (f,j) separate cells (f-1,j) and (f,j). ---- */
static double dep_x(const oblk* b, int f, int j) {
  size_t L = C(b, f - 1, j), R = C(b, f, j);
  return 0.5 * (b->h[L] + b->h[R]) + 0.5 * (b->eta1[L] + b->eta1[R]);
}
static double dep_y(const oblk* b, int i, int g) {
  size_t S = C(b, i, g - 1), Nc = C(b, i, g);
  return 0.5 * (b->h[S] + b->h[Nc]) + 0.5 * (b->eta1[S] + b->eta1[Nc]);
}
/* interior x-face usable by advection */
static int ok_x(const oblk* b, int f, int j, double eps) {
  return f >= 1 && f <= b->nx - 1 && j >= 0 && j <= b->ny - 1 && dep_x(b, f, j) > eps;
}
static int ok_y(const oblk* b, int i, int g, double eps) {
  return g >= 1 && g <= b->ny - 1 && i >= 0 && i <= b->nx - 1 && dep_y(b, i, g) > eps;
}
/* 4-point mean of N around x-face (f,j), pairs taken along x */
static double nbar_x(const oblk* b, int f, int j) {
  return 0.25 * ((b->N[FY(b, f - 1, j)] + b->N[FY(b, f, j)]) +
                 (b->N[FY(b, f - 1, j + 1)] + b->N[FY(b, f, j + 1)]));
}
/* 4-point mean of M around y-face (i,g), pairs taken along y */
static double mbar_y(const oblk* b, int i, int g) {
  return 0.25 * ((b->M[FX(b, i, g - 1)] + b->M[FX(b, i, g)]) +
                 (b->M[FX(b, i + 1, g - 1)] + b->M[FX(b, i + 1, g)]));
}

/* first-order upwind difference of a face flux phi on the sign of the carrier w:
 * w > 0: phi0 - phim, w < 0: phip - phi0, w == 0: (phip - phim) / 2.
 * okm/okp say whether the lower/upper neighbour face is usable. */
static double upwind(double w, double phim, double phi0, double phip, int okm, int okp) {
  if (w > 0) return okm ? phi0 - phim : 0.0;
  if (w < 0) return okp ? phip - phi0 : 0.0;
  return (okm && okp) ? 0.5 * (phip - phim) : 0.0;
}

/* M^2/D at x-face (f,j) and M*Nbar/D at x-face (f,j) */
static double qx(const oblk* b, int f, int j) {
  double m = b->M[FX(b, f, j)];
  return (m * m) / dep_x(b, f, j);
}
static double rx(const oblk* b, int f, int j) {
  return (b->M[FX(b, f, j)] * nbar_x(b, f, j)) / dep_x(b, f, j);
}
static double qy(const oblk* b, int i, int g) {
  double v = b->N[FY(b, i, g)];
  return (v * v) / dep_y(b, i, g);
}
static double ry(const oblk* b, int i, int g) {
  return (b->N[FY(b, i, g)] * mbar_y(b, i, g)) / dep_y(b, i, g);
}

/* Cube root of a positive normal number (the D^(7/3) of Eq. 2's friction term), by
 * Newton-Raphson iteration for the reciprocal cube root, which needs no division:
 *   x = m 2^e with m in [0.5, 1), e = 3q + r with r in {0, 1, 2}, a = m 2^r in [0.5, 4);
 *   y0 = (c0 + m (c1 + m c2)) s_r, a least-squares quadratic start for m^(-1/3) on
 *        [0.5, 1) (relative error 3.2e-3) times s_r ~ 2^(-r/3);
 *   three steps y <- y + y (1 - a y^3) / 3 (the error e goes to about 2 e^2);
 *   cbrt(x) = (a y) y 2^q, where the power of two is exact.
 * Within 4 ulp of the correctly rounded cube root on [1e-3, 1e5] (pinned). */
double orc_cube_root(double x) {
  uint64_t bits, mbits, pbits;
  memcpy(&bits, &x, sizeof bits);
  int e = (int)((bits >> 52) & 0x7ff) - 1022;
  mbits = (bits & 0x800fffffffffffffULL) | ((uint64_t)1022 << 52);
  double m;
  memcpy(&m, &mbits, sizeof m);
  int q = e >= 0 ? e / 3 : -((2 - e) / 3);
  int r = e - 3 * q;
  double a = r == 0 ? m : (r == 1 ? m * 2.0 : m * 4.0);
  double s = r == 0 ? 1.0 : (r == 1 ? 0.7937005259840998 : 0.6299605249474366);
  double y = (1.7375834500937248 + m * (-1.1916185163999664 + m * 0.4564206970782672)) * s;
  for (int k = 0; k < 3; ++k) {
    double t = y * y;
    t = t * y;
    t = a * t;
    t = 1.0 - t;
    t = y * t;
    t = t * 0.3333333333333333;
    y = y + t;
  }
  double c = a * y;
  c = c * y;
  pbits = (uint64_t)(q + 1023) << 52;
  double p2;
  memcpy(&p2, &pbits, sizeof p2);
  return c * p2;
}

/* common tail of R2/R3: pressure, friction, semi-implicit update */
static double flux_update(double m, double across, double Df, double grad, double adv, double nf,
                          double dtdx, const orc_params* p) {
  double P = p->g * Df * dtdx * grad;
  double F = 0.5 * p->dt * p->g * nf * nf * sqrt(m * m + across * across) /
             (Df * Df * orc_cube_root(Df));
  return ((1.0 - F) * m - adv - P) / (1.0 + F);
}

/* R4: a face may carry out of its upwind cell at most a quarter of that cell's water
 * per step (|flux| <= D_src dx / (4 dt)), so four faces cannot drain a cell below dry.
 * R12 (option): nor more than vel_limit times its face depth Df (a velocity limit). */
static double limit_outflow(double m, double Dlo, double Dhi, double Df, double dx, double dt,
                            double vel_limit) {
  double cap = (m > 0 ? Dlo : Dhi) * dx / (4.0 * dt);
  if (vel_limit > 0) {
    double vc = vel_limit * Df;
    if (vc < cap) cap = vc;
  }
  if (m > cap) return cap;
  if (m < -cap) return -cap;
  return m;
}

/* R2 + R4 at interior x-face (f,j), 1 <= f <= nx-1 */
static double xmom(const oblk* b, int f, int j, const orc_params* p) {
  const double eps = p->dry_eps;
  size_t L = C(b, f - 1, j), R = C(b, f, j);
  double eL = b->eta1[L], eR = b->eta1[R], hL = b->h[L], hR = b->h[R];
  int wL = hL + eL > eps, wR = hR + eR > eps;
  double m = b->M[FX(b, f, j)];
  double Df, grad, adv;
  if (wL && wR) {
    Df = 0.5 * (hL + hR) + 0.5 * (eL + eR);
    grad = eR - eL;
    double ax = upwind(m, ok_x(b, f - 1, j, eps) ? qx(b, f - 1, j) : 0.0, qx(b, f, j),
                       ok_x(b, f + 1, j, eps) ? qx(b, f + 1, j) : 0.0, ok_x(b, f - 1, j, eps),
                       ok_x(b, f + 1, j, eps));
    double nb = nbar_x(b, f, j);
    double ay = upwind(nb, ok_x(b, f, j - 1, eps) ? rx(b, f, j - 1) : 0.0, rx(b, f, j),
                       ok_x(b, f, j + 1, eps) ? rx(b, f, j + 1) : 0.0, ok_x(b, f, j - 1, eps),
                       ok_x(b, f, j + 1, eps));
    adv = b->dtdx * (ax + ay);
  } else if (wL && !wR && eL > -hR) {
    Df = eL + hR;
    grad = -hR - eL;
    adv = 0.0;
  } else if (wR && !wL && eR > -hL) {
    Df = eR + hL;
    grad = eR + hL;
    adv = 0.0;
  } else {
    return 0.0;
  }
  if (!(Df > eps)) return 0.0;
  double nf = b->n[L] > b->n[R] ? b->n[L] : b->n[R];
  double m1 = flux_update(m, nbar_x(b, f, j), Df, grad, adv, nf, b->dtdx, p);
  if (!(wL && wR) && (wL ? m1 < 0.0 : m1 > 0.0)) return 0.0; /* no flow out of a dry cell */
  return limit_outflow(m1, hL + eL, hR + eR, Df, b->dx, p->dt, p->vel_limit);
}

/* R3 + R4 at interior y-face (i,g), 1 <= g <= ny-1: R2 with x and y exchanged */
static double ymom(const oblk* b, int i, int g, const orc_params* p) {
  const double eps = p->dry_eps;
  size_t S = C(b, i, g - 1), Nc = C(b, i, g);
  double eS = b->eta1[S], eN = b->eta1[Nc], hS = b->h[S], hN = b->h[Nc];
  int wS = hS + eS > eps, wN = hN + eN > eps;
  double v = b->N[FY(b, i, g)];
  double Df, grad, adv;
  if (wS && wN) {
    Df = 0.5 * (hS + hN) + 0.5 * (eS + eN);
    grad = eN - eS;
    double ay = upwind(v, ok_y(b, i, g - 1, eps) ? qy(b, i, g - 1) : 0.0, qy(b, i, g),
                       ok_y(b, i, g + 1, eps) ? qy(b, i, g + 1) : 0.0, ok_y(b, i, g - 1, eps),
                       ok_y(b, i, g + 1, eps));
    double mb = mbar_y(b, i, g);
    double ax = upwind(mb, ok_y(b, i - 1, g, eps) ? ry(b, i - 1, g) : 0.0, ry(b, i, g),
                       ok_y(b, i + 1, g, eps) ? ry(b, i + 1, g) : 0.0, ok_y(b, i - 1, g, eps),
                       ok_y(b, i + 1, g, eps));
    adv = b->dtdx * (ay + ax);
  } else if (wS && !wN && eS > -hN) {
    Df = eS + hN;
    grad = -hN - eS;
    adv = 0.0;
  } else if (wN && !wS && eN > -hS) {
    Df = eN + hS;
    grad = eN + hS;
    adv = 0.0;
  } else {
    return 0.0;
  }
  if (!(Df > eps)) return 0.0;
  double nf = b->n[S] > b->n[Nc] ? b->n[S] : b->n[Nc];
  double v1 = flux_update(v, mbar_y(b, i, g), Df, grad, adv, nf, b->dtdx, p);
  if (!(wS && wN) && (wS ? v1 < 0.0 : v1 > 0.0)) return 0.0; /* no flow out of a dry cell */
  return limit_outflow(v1, hS + eS, hN + eN, Df, b->dx, p->dt, p->vel_limit);
}

/* R6: radiation flux leaving through an edge next to cell c (sign: +1 east/north) */
static double radiate(const oblk* b, size_t c, double sign, const orc_params* p) {
  double h = b->h[c], e = b->eta1[c];
  if (!(h + e > p->dry_eps)) return 0.0;
  return sign * (sqrt(p->g * (h > 0 ? h : 0.0)) * e);
}

/* ---- R2-R4 + R6: momentum (Eqs. 2-3) over one block ---- */
static void momentum_block(oblk* b, const orc_params* p) {
  const int nx = b->nx, ny = b->ny;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int f = 1; f <= nx - 1; ++f) b->M1[FX(b, f, j)] = xmom(b, f, j, p);
#pragma omp parallel for schedule(static)
  for (int g = 1; g <= ny - 1; ++g)
    for (int i = 0; i < nx; ++i) b->N1[FY(b, i, g)] = ymom(b, i, g, p);
  if (b->d.parent >= 0) { /* child edges are set by R7 after all blocks */
    for (int j = 0; j < ny; ++j) {
      b->M1[FX(b, 0, j)] = b->M[FX(b, 0, j)];
      b->M1[FX(b, nx, j)] = b->M[FX(b, nx, j)];
    }
    for (int i = 0; i < nx; ++i) {
      b->N1[FY(b, i, 0)] = b->N[FY(b, i, 0)];
      b->N1[FY(b, i, ny)] = b->N[FY(b, i, ny)];
    }
    return;
  }
  for (int j = 0; j < ny; ++j) {
    b->M1[FX(b, 0, j)] =
        b->d.bc[0] == ORC_BC_RADIATION ? radiate(b, C(b, 0, j), -1.0, p) : 0.0;
    b->M1[FX(b, nx, j)] =
        b->d.bc[1] == ORC_BC_RADIATION ? radiate(b, C(b, nx - 1, j), 1.0, p) : 0.0;
  }
  for (int i = 0; i < nx; ++i) {
    b->N1[FY(b, i, 0)] =
        b->d.bc[2] == ORC_BC_RADIATION ? radiate(b, C(b, i, 0), -1.0, p) : 0.0;
    b->N1[FY(b, i, ny)] =
        b->d.bc[3] == ORC_BC_RADIATION ? radiate(b, C(b, i, ny - 1), 1.0, p) : 0.0;
  }
}

/* ---- R7: coarse->fine edge fluxes ---- */
/* value for fine face number t along an edge whose coarse faces are v(k), k = 0..K-1 */
static double interp_edge(const double* v, int K, int t, int constant) {
  int k = t / 3, sub = t % 3;
  if (sub == 1 || constant) return v[k];
  int kn = sub == 0 ? k - 1 : k + 1;
  if (kn < 0) kn = 0;
  if (kn > K - 1) kn = K - 1;
  return (2.0 * v[k] + v[kn]) / 3.0;
}

static void edges_child(orc_state* s, int k) {
  oblk* c = &s->b[k];
  const oblk* P = &s->b[c->d.parent];
  int a = c->nx / 3, bb = c->ny / 3, i0 = c->d.i0, j0 = c->d.j0;
  int cst = s->p.nest_flux == ORC_FLUX_CONSTANT;
  double* v = (double*)malloc((size_t)(a > bb ? a : bb) * sizeof(double));
  if (!v) abort();
  /* west and east: parent x-faces i0 and i0+a, parent rows j0..j0+bb-1 */
  for (int side = 0; side < 2; ++side) {
    int F = side == 0 ? i0 : i0 + a, f = side == 0 ? 0 : c->nx;
    for (int t = 0; t < bb; ++t) v[t] = P->M1[FX(P, F, j0 + t)];
    for (int j = 0; j < c->ny; ++j) c->M1[FX(c, f, j)] = interp_edge(v, bb, j, cst);
  }
  /* south and north: parent y-faces j0 and j0+bb, parent columns i0..i0+a-1 */
  for (int side = 0; side < 2; ++side) {
    int G = side == 0 ? j0 : j0 + bb, g = side == 0 ? 0 : c->ny;
    for (int t = 0; t < a; ++t) v[t] = P->N1[FY(P, i0 + t, G)];
    for (int i = 0; i < c->nx; ++i) c->N1[FY(c, i, g)] = interp_edge(v, a, i, cst);
  }
  free(v);
}

static void swap_ptr(double** a, double** b) {
  double* t = *a;
  *a = *b;
  *b = t;
}

int orc_step(orc_state* s, int nsteps) {
  if (!s || nsteps < 0) return ORC_ERR_INVALID_ARG;
  for (int it = 0; it < nsteps; ++it) {
    long step = s->step + 1;
    for (int k = 0; k < s->nb; ++k) track_speed(&s->b[k], &s->p);
    for (int k = 0; k < s->nb; ++k) mass_block(&s->b[k], &s->p);
    fine_to_coarse(s);
    for (int k = 0; k < s->nb; ++k) {
      oblk* b = &s->b[k];
      const long nc = (long)b->nx * b->ny;
#pragma omp parallel for schedule(static)
      for (long c = 0; c < nc; ++c) track_cell(b, (size_t)c, step, &s->p);
    }
    for (int k = 0; k < s->nb; ++k) momentum_block(&s->b[k], &s->p);
    for (int k = 0; k < s->nb; ++k)
      if (s->b[k].d.parent >= 0) edges_child(s, k);
    for (int k = 0; k < s->nb; ++k) {
      oblk* b = &s->b[k];
      swap_ptr(&b->eta, &b->eta1);
      swap_ptr(&b->M, &b->M1);
      swap_ptr(&b->N, &b->N1);
    }
    s->step = step;
  }
  return ORC_OK;
}

long orc_steps_done(const orc_state* s) { return s ? s->step : -1; }

/* ---- one step in phases, for the blocks of one hierarchy split over several ranks ----
 * orc_step above, taken apart at the points where a block decomposition exchanges data
 * (Sec. IV-C: the child's means go to the parent after the mass step, the parent's new
 * fluxes on the footprint edge go to the child after the momentum step). Each rank keeps
 * a state of the whole hierarchy but steps only its own blocks; the phases below read
 * and write only the block they are given, except the exchange calls, which move exactly
 * the values of one message. Called for every block on one rank, in the order the
 * header gives, they perform orc_step's operations in its order. */
static int valid_block(const orc_state* s, int k) { return s && k >= 0 && k < s->nb; }
static int valid_child(const orc_state* s, int k) {
  return valid_block(s, k) && s->b[k].d.parent >= 0;
}

int orc_phase_mass(orc_state* s, int k) {
  if (!valid_block(s, k)) return ORC_ERR_INVALID_ARG;
  track_speed(&s->b[k], &s->p);
  mass_block(&s->b[k], &s->p);
  return ORC_OK;
}

/* parent cells of child k that receive its mean (its footprint's inner ring, or all of
 * it with full feedback), in rows J, then columns I */
int orc_means_count(const orc_state* s, int k) {
  if (!valid_child(s, k)) return ORC_ERR_INVALID_ARG;
  int a = s->b[k].nx / 3, bb = s->b[k].ny / 3, n = 0;
  for (int J = 0; J < bb; ++J)
    for (int I = 0; I < a; ++I) n += receives(&s->p, I, J, a, bb);
  return n;
}

int orc_pack_means(const orc_state* s, int k, double* out) {
  if (!valid_child(s, k) || !out) return ORC_ERR_INVALID_ARG;
  int a = s->b[k].nx / 3, bb = s->b[k].ny / 3, n = 0;
  double* all = (double*)malloc((size_t)a * (size_t)bb * sizeof(double));
  if (!all) abort();
  pack_child(s, k, all);
  for (int J = 0; J < bb; ++J)
    for (int I = 0; I < a; ++I)
      if (receives(&s->p, I, J, a, bb)) out[n++] = all[(size_t)J * a + I];
  free(all);
  return ORC_OK;
}

int orc_unpack_means(orc_state* s, int k, const double* in) {
  if (!valid_child(s, k) || !in) return ORC_ERR_INVALID_ARG;
  int a = s->b[k].nx / 3, bb = s->b[k].ny / 3, n = 0;
  double* all = (double*)malloc((size_t)a * (size_t)bb * sizeof(double));
  if (!all) abort();
  for (int J = 0; J < bb; ++J)
    for (int I = 0; I < a; ++I)
      all[(size_t)J * a + I] = receives(&s->p, I, J, a, bb) ? in[n++] : NAN;
  unpack_child(s, k, all);
  free(all);
  return ORC_OK;
}

int orc_phase_momentum(orc_state* s, int k) {
  if (!valid_block(s, k)) return ORC_ERR_INVALID_ARG;
  oblk* b = &s->b[k];
  const long nc = (long)b->nx * b->ny;
  const long step = s->step + 1;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < nc; ++c) track_cell(b, (size_t)c, step, &s->p);
  momentum_block(b, &s->p);
  return ORC_OK;
}

/* the parent's new fluxes on child k's footprint edge: west and east x-faces over the
 * footprint's rows, then south and north y-faces over its columns (2 ny/3 + 2 nx/3) */
int orc_edge_count(const orc_state* s, int k) {
  if (!valid_child(s, k)) return ORC_ERR_INVALID_ARG;
  return 2 * (s->b[k].ny / 3) + 2 * (s->b[k].nx / 3);
}

static void edge_values(orc_state* s, int k, double* v, int set) {
  const oblk* c = &s->b[k];
  oblk* P = &s->b[c->d.parent];
  int a = c->nx / 3, bb = c->ny / 3, i0 = c->d.i0, j0 = c->d.j0, n = 0;
  for (int side = 0; side < 2; ++side) {
    int F = side == 0 ? i0 : i0 + a;
    for (int t = 0; t < bb; ++t, ++n) {
      double* q = &P->M1[FX(P, F, j0 + t)];
      if (set) *q = v[n];
      else v[n] = *q;
    }
  }
  for (int side = 0; side < 2; ++side) {
    int G = side == 0 ? j0 : j0 + bb;
    for (int t = 0; t < a; ++t, ++n) {
      double* q = &P->N1[FY(P, i0 + t, G)];
      if (set) *q = v[n];
      else v[n] = *q;
    }
  }
}

int orc_get_edge_fluxes(const orc_state* s, int k, double* out) {
  if (!valid_child(s, k) || !out) return ORC_ERR_INVALID_ARG;
  edge_values((orc_state*)s, k, out, 0);
  return ORC_OK;
}

int orc_set_edge_fluxes(orc_state* s, int k, const double* in) {
  if (!valid_child(s, k) || !in) return ORC_ERR_INVALID_ARG;
  edge_values(s, k, (double*)in, 1);
  return ORC_OK;
}

int orc_phase_edges(orc_state* s, int k) {
  if (!valid_child(s, k)) return ORC_ERR_INVALID_ARG;
  edges_child(s, k);
  return ORC_OK;
}

int orc_phase_swap(orc_state* s, int k) {
  if (!valid_block(s, k)) return ORC_ERR_INVALID_ARG;
  oblk* b = &s->b[k];
  swap_ptr(&b->eta, &b->eta1);
  swap_ptr(&b->M, &b->M1);
  swap_ptr(&b->N, &b->N1);
  return ORC_OK;
}

int orc_end_step(orc_state* s) {
  if (!s) return ORC_ERR_INVALID_ARG;
  s->step += 1;
  return ORC_OK;
}

int orc_get_state(const orc_state* s, int k, double* eta, double* M, double* N) {
  if (!s || k < 0 || k >= s->nb) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  if (eta) memcpy(eta, b->eta, (size_t)b->nx * b->ny * sizeof(double));
  if (M) memcpy(M, b->M, (size_t)(b->nx + 1) * b->ny * sizeof(double));
  if (N) memcpy(N, b->N, (size_t)b->nx * (b->ny + 1) * sizeof(double));
  return ORC_OK;
}

int orc_set_state(orc_state* s, int k, const double* eta, const double* M, const double* N) {
  if (!s || k < 0 || k >= s->nb) return ORC_ERR_INVALID_ARG;
  oblk* b = &s->b[k];
  if (eta) memcpy(b->eta, eta, (size_t)b->nx * b->ny * sizeof(double));
  if (M) memcpy(b->M, M, (size_t)(b->nx + 1) * b->ny * sizeof(double));
  if (N) memcpy(b->N, N, (size_t)b->nx * (b->ny + 1) * sizeof(double));
  return ORC_OK;
}

int orc_get_max_height(const orc_state* s, int k, double* out) {
  if (!s || k < 0 || k >= s->nb || !out) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  for (size_t c = 0; c < (size_t)b->nx * b->ny; ++c)
    out[c] = b->emax[c] == NEVER_WET ? NAN : b->emax[c];
  return ORC_OK;
}

int orc_get_max_depth(const orc_state* s, int k, double* out) {
  if (!s || k < 0 || k >= s->nb || !out) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  for (size_t c = 0; c < (size_t)b->nx * b->ny; ++c)
    out[c] = b->emax[c] == NEVER_WET ? 0.0 : b->h[c] + b->emax[c];
  return ORC_OK;
}

int orc_get_max_velocity(const orc_state* s, int k, double* out) {
  if (!s || k < 0 || k >= s->nb || !out) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  for (int j = 0; j < b->ny; ++j)
    for (int i = 0; i < b->nx; ++i) {
      double m = b->vmax2[C(b, i, j)];
      double s2 = speed2(b, b->eta, b->M, b->N, i, j, &s->p);
      if (s2 > m) m = s2;
      out[C(b, i, j)] = sqrt(m);
    }
  return ORC_OK;
}

int orc_get_arrival_time(const orc_state* s, int k, double* out) {
  if (!s || k < 0 || k >= s->nb || !out) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  for (size_t c = 0; c < (size_t)b->nx * b->ny; ++c)
    out[c] = b->arr[c] < 0 ? -1.0 : (double)b->arr[c] * s->p.dt;
  return ORC_OK;
}

int orc_get_budget(const orc_state* s, int k, double* out) {
  if (!s || k < 0 || k >= s->nb || !out) return ORC_ERR_INVALID_ARG;
  const oblk* b = &s->b[k];
  double v = 0.0;
  for (size_t c = 0; c < (size_t)b->nx * b->ny; ++c) v += b->h[c] + b->eta[c];
  out[0] = v * (b->dx * b->dx);
  out[1] = b->outflow;
  out[2] = b->clip;
  out[3] = b->ring;
  return ORC_OK;
}
