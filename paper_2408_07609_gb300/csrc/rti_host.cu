// rti_host.cu -- the C ABI (include/rti.h): hierarchy validation, the device arena of a
// handle, the tile work list of a group of handles, chunk launches and CUDA graphs,
// batches, and host<->device transfers. No arithmetic of the time step runs here.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "rti.h"
#include "rti_launch.h"
#include "rti_layout.h"
#include "rti_schedule.h"

using namespace rti;

namespace rti {
__global__ void k_advance(ScenDev* sc, const int* nscen, int nsteps);
__global__ void k_set_scen(ScenDev* sc, int idx, long long base, long long remaining);
#ifdef RTI_CHECKED
cudaError_t debug_check_fp32(int* out8);
cudaError_t debug_check_fp64(int* out8);
#endif
}  // namespace rti

// message of the last rti_create or rti_step_noalloc that failed on this thread
static thread_local std::string t_create_err;

namespace {

constexpr int kDefaultTx = kStripW, kDefaultTy = 64;
// grid of the host-transfer kernels: 8 CTAs of 256 per SM of 152
constexpr int kIoThreads = 256, kIoBlocks = 1216;
constexpr long long kSpinCycles = 4000000000LL;  // ~2 s at the maximum SM clock

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct BlkMem {
  size_t eta[2], M[2], N[2], h, emax, man, arr, budget;
  size_t ring;  // fine-to-coarse overrides of a block with children (0 = none)
  size_t vmax;  // running max of the squared speed (0 = not tracked)
  int pitch;
  long long rows;
  int tiles_x, tiles_y;
};

size_t esize(int prec) { return prec == RTI_FP32 ? 4 : 8; }

// Layout of one handle's arena; returns the total size.
size_t plan_layout(const rti_block* b, int nb, int prec, int tx, int ty, std::vector<BlkMem>* mem,
                   size_t* off_status, size_t* off_io = nullptr, bool velocity = false) {
  size_t off = 0;
  const size_t es = esize(prec);
  if (mem) mem->resize(nb);
  for (int k = 0; k < nb; ++k) {
    BlkMem m;
    m.pitch = pitch_for(b[k].nx);
    m.rows = rows_for(b[k].ny);
    const size_t plane = (size_t)m.pitch * (size_t)m.rows;
    auto take = [&](size_t bytes) {
      size_t o = off;
      off = align256(off + bytes);
      return o;
    };
    for (int s = 0; s < 2; ++s) m.eta[s] = take(plane * es);
    for (int s = 0; s < 2; ++s) m.M[s] = take(plane * es);
    for (int s = 0; s < 2; ++s) m.N[s] = take(plane * es);
    m.h = take(plane * es);
    m.emax = take(plane * es);
    m.man = take(plane * 4);
    m.arr = take(plane * 4);
    bool parent_of_some = false;
    for (int c = 0; c < nb; ++c) parent_of_some |= b[c].parent == k;
    m.ring = parent_of_some ? take(plane * es) : 0;
    m.vmax = velocity ? take(plane * es) : 0;
    m.tiles_x = (b[k].nx + tx - 1) / tx;
    m.tiles_y = (b[k].ny + ty - 1) / ty;
    m.budget = take((size_t)m.tiles_x * m.tiles_y * 4 * sizeof(double));
    if (mem) (*mem)[k] = m;
  }
  size_t st = off;
  off = align256(off + 64);
  if (off_status) *off_status = st;
  // binary64 staging of host reads and writes: one dense plane of the largest block
  size_t io_elems = kIoBlocks;  // at least the partial sums of plane_sum
  for (int k = 0; k < nb; ++k)
    io_elems = std::max(io_elems, (size_t)(b[k].nx + 1) * (size_t)(b[k].ny + 1));
  if (off_io) *off_io = off;
  off = align256(off + io_elems * sizeof(double));
  return off;
}

int validate(const rti_block* bl, int nb, const rti_params* p, std::string* why) {
  if (!bl || nb <= 0 || !p) {
    *why = "null descriptor or no blocks";
    return RTI_ERR_INVALID_ARG;
  }
  if (!(p->dt > 0) || !(p->g > 0) || !(p->dry_eps >= 0) ||
      (p->precision != RTI_FP32 && p->precision != RTI_FP64) ||
      (p->schedule != RTI_SCHED_PERSISTENT && p->schedule != RTI_SCHED_PER_PASS) ||
      (p->tile_x != 0 && p->tile_x != kStripW) || p->tile_y < 0 || p->tile_y % 8 ||
      p->ctas_per_sm < 0 || !(p->velocity_limit >= 0) ||
      (p->track_velocity != 0 && p->track_velocity != 1) ||
      (p->nest_feedback != RTI_NEST_RING && p->nest_feedback != RTI_NEST_FULL) ||
      (p->nest_flux != RTI_FLUX_LINEAR && p->nest_flux != RTI_FLUX_CONSTANT)) {
    *why = "bad params (dt, g, dry_eps, precision, schedule, tile shape, track_velocity "
           "or nesting options)";
    return RTI_ERR_INVALID_ARG;
  }
  for (int k = 0; k < nb; ++k) {
    const rti_block* d = &bl[k];
    if (d->nx < 3 || d->ny < 3 || !(d->dx > 0) || d->nx > (1 << 20) || d->ny > (1 << 20)) {
      *why = "block " + std::to_string(k) + ": bad size or dx";
      return RTI_ERR_INVALID_ARG;
    }
    // the kernels index a plane with 32-bit element offsets
    if ((long long)pitch_for(d->nx) * rows_for(d->ny) >= (1LL << 31)) {
      *why = "block " + std::to_string(k) + ": more than 2^31 elements per plane";
      return RTI_ERR_INVALID_ARG;
    }
    if (d->parent < 0) {
      if (d->level != 1) {
        *why = "block " + std::to_string(k) + ": a root must have level 1";
        return RTI_ERR_NESTING;
      }
      for (int s = 0; s < 4; ++s)
        if (d->bc[s] != RTI_BC_WALL && d->bc[s] != RTI_BC_RADIATION) {
          *why = "block " + std::to_string(k) + ": bad boundary kind";
          return RTI_ERR_INVALID_ARG;
        }
      continue;
    }
    auto bad = [&](const char* m) {
      *why = "block " + std::to_string(k) + ": " + m;
      return RTI_ERR_NESTING;
    };
    if (d->parent >= k) return bad("parents must be listed before their children");
    const rti_block* P = &bl[d->parent];
    if (d->level != P->level + 1) return bad("level must be parent level + 1");
    if (d->nx % 3 || d->ny % 3) return bad("child size must be a multiple of 3");
    if (std::fabs(d->dx * 3.0 - P->dx) > 1e-9 * P->dx) return bad("child dx must be parent dx / 3");
    if (d->i0 < 3 || d->j0 < 3 || d->i0 + d->nx / 3 > P->nx - 3 || d->j0 + d->ny / 3 > P->ny - 3)
      return bad("child must lie inside its parent with a 3-cell margin");
    for (int q = 0; q < k; ++q) {
      const rti_block* o = &bl[q];
      if (o->parent != d->parent) continue;
      bool ox = d->i0 < o->i0 + o->nx / 3 && o->i0 < d->i0 + d->nx / 3;
      bool oy = d->j0 < o->j0 + o->ny / 3 && o->j0 < d->j0 + d->ny / 3;
      if (ox && oy) return bad("overlaps a sibling");
    }
  }
  return RTI_OK;
}

const char* cuda_name(cudaError_t e) { return cudaGetErrorString(e); }

}  // namespace

// ------------------------------------------------------------------------------ groups
struct Group {
  int prec = RTI_FP64, sched = RTI_SCHED_PERSISTENT, tx = kDefaultTx, ty = kDefaultTy;
  int chunk = 1;
  std::vector<rti_handle*> members;
  std::vector<long long> remaining;  // host mirror of ScenDev.remaining (as enqueued)
  // device tables
  char* d_blk = nullptr;
  size_t cap_blk = 0;  // bytes
  int* d_kids = nullptr;
  size_t cap_kids = 0;
  Tile* d_tiles = nullptr;
  size_t cap_tiles = 0;
  int* d_counts = nullptr;  // [0] = ntiles, [1] = nscen
  unsigned long long* d_done = nullptr;  // per strip: the last step it has ended
  size_t cap_done = 0;      // bytes
  int* d_dep = nullptr;     // dataflow dependencies: offsets (ntiles + 1), then indices
  size_t cap_dep = 0;       // bytes
  ScenDev* d_scen = nullptr;
  size_t cap_scen = 0;
  int* d_status = nullptr;
  Bar* d_bar = nullptr;
  int grid = 0;                  // co-resident grid of the plain variant
  int grids[kStepModes] = {};    // of every variant (0: not computed yet)
  int cap = 0;                   // CTAs per SM cap (0 = none)
  bool track = false;            // some member keeps the maximum velocity
  bool limit = false;            // some member keeps the velocity limit
  bool full = false;             // some member has full feedback (finer levels listed first)
  long long spin_cycles = kSpinCycles;
  // pinned staging for table uploads
  char* h_stage = nullptr;
  size_t cap_stage = 0;
  cudaEvent_t staged = nullptr;
  // graph of one chunk
  cudaGraphExec_t gexec = nullptr;
  bool graph_tried = false;
  cudaStream_t cap_stream = nullptr;
  int ntiles = 0, nblk = 0, nkids = 0;
  long long cells = 0;
  bool dirty = true;
};

struct rti_handle {
  int prec = RTI_FP64;
  rti_params params{};
  std::vector<rti_block> blocks;
  std::vector<BlkMem> mem;
  std::vector<double> sum_h;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own = false;
  size_t off_status = 0;
  size_t off_io = 0;   // binary64 staging plane for host reads and writes
  long long base = 0;  // steps completed including enqueued work
  std::string err;
  rti_batch* batch = nullptr;
  Group* self = nullptr;
  cudaEvent_t done = nullptr;
  long long cells = 0;
  long long h2d = 0, d2h = 0;  // bytes moved by this handle's calls
};

struct rti_batch {
  Group g;
  std::string err;
  cudaEvent_t done = nullptr;
};

namespace {

int set_err(std::string* dst, int code, const std::string& msg) {
  if (dst) *dst = msg;
  return code;
}

int cuda_err(std::string* dst, cudaError_t e, const char* what) {
  if (dst) *dst = std::string(what) + ": " + cuda_name(e);
  return RTI_ERR_CUDA;
}

template <class T>
Blk<T> make_blk(rti_handle* h, int k, int base_index, int scen, int child_first, int child_count,
                int tx) {
  const rti_block& d = h->blocks[k];
  const BlkMem& m = h->mem[k];
  const rti_params& p = h->params;
  Blk<T> b;
  std::memset(&b, 0, sizeof(b));
  char* A = h->arena;
  for (int s = 0; s < 2; ++s) {
    b.eta[s] = (T*)(A + m.eta[s]);
    b.M[s] = (T*)(A + m.M[s]);
    b.N[s] = (T*)(A + m.N[s]);
  }
  b.h = (const T*)(A + m.h);
  b.man = (const float*)(A + m.man);
  b.emax = (T*)(A + m.emax);
  b.arr = (int*)(A + m.arr);
  b.ring = m.ring ? (T*)(A + m.ring) : nullptr;
  b.vmax = m.vmax ? (T*)(A + m.vmax) : nullptr;
  b.nx = d.nx;
  b.ny = d.ny;
  b.pitch = m.pitch;
  b.parent = d.parent < 0 ? -1 : base_index + d.parent;
  b.i0 = d.i0;
  b.j0 = d.j0;
  b.child_first = child_first;
  b.child_count = child_count;
  for (int s = 0; s < 4; ++s) b.bc[s] = d.bc[s];
  b.scen = scen;
  b.is_child = d.parent >= 0;
  b.tiles_x = (d.nx + tx - 1) / tx;
  b.nest = (p.nest_feedback == RTI_NEST_FULL ? kNestFull : 0) |
           (p.nest_flux == RTI_FLUX_CONSTANT ? kNestConst : 0);
  b.budget = (double*)(A + m.budget);
  b.status = (int*)(A + h->off_status);
  const double dt = p.dt, dx = d.dx;
  b.dtdx = (T)(dt / dx);
  b.dt = (T)dt;
  b.g = (T)p.g;
  b.cfric = (T)(0.5 * dt * p.g);
  b.eps = (T)p.dry_eps;
  b.thr = (T)p.arrival_thr;
  b.dx = (T)dx;
  b.q4dt = (T)(4.0 * dt);
  b.vlim = p.velocity_limit > 0 ? (T)p.velocity_limit : (T)INFINITY;
  b.dx2 = dx * dx;
  b.vol = dt * dx;
  b.eps_d = p.dry_eps;
#ifdef RTI_CHECKED
  b.lo = h->arena;
  b.hi = h->arena + h->arena_bytes;
#endif
  return b;
}

void free_group_dev(Group* g) {
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  g->gexec = nullptr;
  g->graph_tried = false;
  cudaFree(g->d_blk);
  cudaFree(g->d_kids);
  cudaFree(g->d_tiles);
  cudaFree(g->d_counts);
  cudaFree(g->d_done);
  cudaFree(g->d_dep);
  cudaFree(g->d_scen);
  cudaFree(g->d_status);
  cudaFree(g->d_bar);
  if (g->h_stage) cudaFreeHost(g->h_stage);
  if (g->staged) cudaEventDestroy(g->staged);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  g->d_blk = nullptr;
  g->d_kids = nullptr;
  g->d_tiles = nullptr;
  g->d_counts = nullptr;
  g->d_done = nullptr;
  g->d_dep = nullptr;
  g->d_scen = nullptr;
  g->d_status = nullptr;
  g->d_bar = nullptr;
  g->h_stage = nullptr;
  g->staged = nullptr;
  g->cap_stream = nullptr;
}

int group_init(Group* g, int prec, int sched, int tx, int ty, int chunk, int cap,
               std::string* err) {
  g->prec = prec;
  g->sched = sched;
  g->tx = tx;
  g->ty = ty;
  g->chunk = chunk;
  cudaError_t e = cudaMalloc(&g->d_counts, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_bar, sizeof(Bar));
  if (e == cudaSuccess) e = cudaMemset(g->d_counts, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(g->d_bar, 0, sizeof(Bar));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming);
  // RTI_BARRIER_SPIN_CYCLES shortens the bounded barrier wait (used to test the timeout path)
  if (const char* v = std::getenv("RTI_BARRIER_SPIN_CYCLES")) {
    long long c = std::atoll(v);
    if (c > 0) g->spin_cycles = c;
  }
  g->cap = cap;
  if (e == cudaSuccess)
    e = prec == RTI_FP32 ? persistent_grid<float>(&g->grid, tx, ty, kStepPlain, cap)
                         : persistent_grid<double>(&g->grid, tx, ty, kStepPlain, cap);
  if (e != cudaSuccess) return cuda_err(err, e, "group setup");
  return RTI_OK;
}

template <class T>
KParams<T> kparams(Group* g, int nsteps) {
  KParams<T> kp;
  kp.blk = (const Blk<T>*)g->d_blk;
  kp.kids = g->d_kids;
  kp.tiles = g->d_tiles;
  kp.ntiles = g->d_counts;
  kp.done = g->d_done;
  kp.ndone = (int)(g->cap_done / sizeof(*g->d_done));
  kp.dep_off = g->full ? g->d_dep : nullptr;
  kp.scen = g->d_scen;
  kp.status = g->d_status;
  kp.bar = g->d_bar;
  kp.nsteps = nsteps;
  kp.track = g->track ? 1 : 0;
  kp.limit = g->limit ? 1 : 0;
  kp.full = g->full ? 1 : 0;
  kp.tx = g->tx;
  kp.ty = g->ty;
  kp.spin_cycles = g->spin_cycles;
#ifdef RTI_CHECKED
  kp.nblk = g->nblk;
  kp.nkids = g->nkids;
#endif
  return kp;
}

template <class T>
cudaError_t grow(T** ptr, size_t* cap, size_t need_bytes, bool* moved) {
  if (need_bytes <= *cap && *ptr) return cudaSuccess;
  size_t n = std::max(need_bytes, *cap * 2);
  n = std::max<size_t>(n, 256);
  cudaFree(*ptr);
  *ptr = nullptr;
  cudaError_t e = cudaMalloc((void**)ptr, n);
  if (e == cudaSuccess) {
    *cap = n;
    *moved = true;
  }
  return e;
}

// Rebuild and upload the block table, child lists and tile list of a group (stream-ordered).
template <class T>
int group_upload(Group* g, cudaStream_t st, std::string* err) {
  std::vector<Blk<T>> blks;
  std::vector<int> kids;
  std::vector<Tile> tiles;
  int nflags = 0;  // strips of the group (one flag each)
  long long cells = 0;
  bool track = false, limit = false, full_any = false;
  for (size_t mi = 0; mi < g->members.size(); ++mi) {
    rti_handle* h = g->members[mi];
    track = track || h->params.track_velocity != 0;
    limit = limit || h->params.velocity_limit > 0;
    full_any = full_any || h->params.nest_feedback == RTI_NEST_FULL;
    const int base = (int)blks.size();
    const int nb = (int)h->blocks.size();
    std::vector<std::vector<int>> ch(nb);
    for (int k = 0; k < nb; ++k)
      if (h->blocks[k].parent >= 0) ch[h->blocks[k].parent].push_back(k);
    for (int k = 0; k < nb; ++k) {
      const int cf = (int)kids.size();
      for (int c : ch[k]) kids.push_back(base + c);
      blks.push_back(make_blk<T>(h, k, base, (int)mi, cf, (int)ch[k].size(), g->tx));
      blks.back().strip0 = nflags;
      nflags += h->mem[k].tiles_x * h->mem[k].tiles_y;
    }
    for (int k = 0; k < nb; ++k) {
      const rti_block& d = h->blocks[k];
      cells += (long long)d.nx * d.ny;
      for (int ty = 0; ty < h->mem[k].tiles_y; ++ty) {
        for (int tx = 0; tx < h->mem[k].tiles_x; ++tx) {
          Tile t;
          t.blk = base + k;
          t.x0 = tx * g->tx;
          t.y0 = ty * g->ty;
          t.flags = 0;
          if (t.x0 == 0) t.flags |= kTfWest;
          if (t.x0 + g->tx >= d.nx) t.flags |= kTfEast;
          if (t.y0 == 0) t.flags |= kTfSouth;
          if (t.y0 + g->ty >= d.ny) t.flags |= kTfNorth;
          // the strip recomputes eta^{n+1} on a 2-cell halo: flag it when that halo
          // meets the inner ring of a child footprint (any of it with full feedback)
          const int hx0 = t.x0 - 2, hy0 = t.y0 - 2, hx1 = t.x0 + g->tx + 2, hy1 = t.y0 + g->ty + 2;
          const bool full = h->params.nest_feedback == RTI_NEST_FULL;
          for (int c : ch[k]) {
            const rti_block& cd = h->blocks[c];
            int a0 = cd.i0, a1 = cd.i0 + cd.nx / 3, b0 = cd.j0, b1 = cd.j0 + cd.ny / 3;
            bool meets = hx0 < a1 && a0 < hx1 && hy0 < b1 && b0 < hy1;
            bool inner = hx0 >= a0 + 1 && hx1 <= a1 - 1 && hy0 >= b0 + 1 && hy1 <= b1 - 1;
            if (meets && (full || !inner)) t.flags |= kTfRing;
          }
          tiles.push_back(t);
        }
      }
    }
  }
  // The step kernel hands strips out in list order, the slow ones first. With full
  // feedback a parent's ring strip reads the means its children's strips formed this step
  // and waits for the flags of the child strips under its region: the list then follows
  // a simulated schedule (full_feedback_order) in which a strip comes after every strip it
  // waits for, so that it waits only on running warps, which wait on nothing later in the
  // list (no cycle).
  if (!full_any) {
    // longest first: a strip weighs its cells, 2.1 times for a ring strip (its prepass
    // recomputes the child levels of the ring) and 1.05 for a child's edge strip (the
    // pulled fluxes), as their measured durations go; the small strips at the blocks'
    // far edges then come last and fill the end of the step (+2.2 % on the 46.65 M-cell
    // case against heavy strips first in block order)
    auto weight = [&](const Tile& t) {
      const Blk<T>& b = blks[t.blk];
      const bool edge = b.is_child && (t.x0 == 0 || t.x0 + g->tx + 2 >= b.nx || t.y0 == 0 ||
                                       t.y0 + g->ty + 2 >= b.ny);
      const int cells = std::min(g->tx, b.nx - t.x0) * std::min(g->ty, b.ny - t.y0);
      return ((t.flags & kTfRing) ? 2.1 : edge ? 1.05 : 1.0) * cells;
    };
    std::stable_sort(tiles.begin(), tiles.end(),
                     [&](const Tile& a, const Tile& b) { return weight(a) > weight(b); });
  } else {
    const int mode = (track ? kStepTrack : kStepPlain) | (limit ? kStepLimit : 0) | kStepFull;
    int grid = 0;
    if (persistent_grid<T>(&grid, g->tx, g->ty, mode, g->cap) != cudaSuccess || grid <= 0)
      grid = g->grid;
    tiles = full_feedback_order<T>(blks, kids, tiles, g->tx, g->ty, grid * kWarps);
  }
  std::vector<int> dep_off, dep_idx;  // the dataflow of full-feedback chunks
  if (full_any) dataflow_deps<T>(blks, tiles, g->tx, g->ty, &dep_off, &dep_idx);
  bool moved = false;
  cudaError_t e = grow(&g->d_blk, &g->cap_blk, blks.size() * sizeof(Blk<T>) + 64, &moved);
  if (e == cudaSuccess) e = grow(&g->d_kids, &g->cap_kids, kids.size() * sizeof(int) + 64, &moved);
  if (e == cudaSuccess) e = grow(&g->d_tiles, &g->cap_tiles, tiles.size() * sizeof(Tile) + 64, &moved);
  if (e == cudaSuccess)
    e = grow(&g->d_scen, &g->cap_scen, g->members.size() * sizeof(ScenDev) + 64, &moved);
  if (e == cudaSuccess)
    e = grow(&g->d_done, &g->cap_done, (size_t)nflags * sizeof(*g->d_done), &moved);
  if (e == cudaSuccess)
    e = grow(&g->d_dep, &g->cap_dep, (dep_off.size() + dep_idx.size()) * sizeof(int), &moved);
  if (e != cudaSuccess) return cuda_err(err, e, "device tables");
  // the captured graph holds the old pointers and sizes, or the other kernel variant
  if ((moved || track != g->track || limit != g->limit || full_any != g->full) && g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    g->graph_tried = false;
  }
  const size_t nb_blk = blks.size() * sizeof(Blk<T>);
  const size_t nb_kids = kids.size() * sizeof(int);
  const size_t nb_tiles = tiles.size() * sizeof(Tile);
  const size_t nb_scen = g->members.size() * sizeof(ScenDev);
  const size_t nb_dep = (dep_off.size() + dep_idx.size()) * sizeof(int);
  const size_t need = align256(nb_blk) + align256(nb_kids) + align256(nb_tiles) +
                      align256(nb_scen) + align256(nb_dep) + 256;
  // the previous upload must have left the staging buffer before it is rewritten
  e = cudaEventSynchronize(g->staged);
  if (e != cudaSuccess) return cuda_err(err, e, "staging wait");
  if (need > g->cap_stage) {
    if (g->h_stage) cudaFreeHost(g->h_stage);
    g->h_stage = nullptr;
    e = cudaMallocHost((void**)&g->h_stage, need * 2);
    if (e != cudaSuccess) return cuda_err(err, e, "pinned staging");
    g->cap_stage = need * 2;
  }
  char* s = g->h_stage;
  size_t o = 0;
  auto put = [&](const void* src, size_t n, void* dst) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    std::memcpy(s + o, src, n);
    cudaError_t r = cudaMemcpyAsync(dst, s + o, n, cudaMemcpyHostToDevice, st);
    o += align256(n);
    return r;
  };
  std::vector<ScenDev> sc(g->members.size());
  for (size_t mi = 0; mi < g->members.size(); ++mi) {
    sc[mi].base = g->members[mi]->base;
    sc[mi].remaining = g->remaining[mi];
  }
  int counts[2] = {(int)tiles.size(), (int)g->members.size()};
  e = put(blks.data(), nb_blk, g->d_blk);
  if (e == cudaSuccess) e = put(kids.data(), nb_kids, g->d_kids);
  if (e == cudaSuccess) e = put(tiles.data(), nb_tiles, g->d_tiles);
  if (e == cudaSuccess) e = put(sc.data(), nb_scen, g->d_scen);
  std::vector<int> dep(dep_off);
  dep.insert(dep.end(), dep_idx.begin(), dep_idx.end());
  if (e == cudaSuccess) e = put(dep.data(), nb_dep, g->d_dep);
  if (e == cudaSuccess) e = put(counts, sizeof(counts), g->d_counts);
  if (e == cudaSuccess) e = cudaEventRecord(g->staged, st);
  if (e != cudaSuccess) return cuda_err(err, e, "table upload");
  g->ntiles = (int)tiles.size();
  g->nblk = (int)blks.size();
  g->nkids = (int)kids.size();
  g->cells = cells;
  g->track = track;
  g->limit = limit;
  g->full = full_any;
  g->dirty = false;
  return RTI_OK;
}

int group_upload_any(Group* g, cudaStream_t st, std::string* err) {
  return g->prec == RTI_FP32 ? group_upload<float>(g, st, err) : group_upload<double>(g, st, err);
}

// grid of the variant a chunk of this group launches, computed on first use
int launch_grid(Group* g) {
  const int mode = (g->track ? kStepTrack : kStepPlain) | (g->limit ? kStepLimit : 0) |
                   (g->full ? kStepFull : 0);
  if (!g->grids[mode]) {
    int grid = 0;
    const cudaError_t e =
        g->prec == RTI_FP32 ? persistent_grid<float>(&grid, g->tx, g->ty, mode, g->cap)
                            : persistent_grid<double>(&grid, g->tx, g->ty, mode, g->cap);
    g->grids[mode] = e == cudaSuccess && grid > 0 ? grid : g->grid;
  }
  return g->grids[mode];
}

int launch_any(Group* g, int nsteps, cudaStream_t st, std::string* err) {
  cudaError_t e;
  if (g->prec == RTI_FP32)
    e = launch_chunk<float>(kparams<float>(g, nsteps), g->sched, launch_grid(g), g->d_counts + 1,
                            st);
  else
    e = launch_chunk<double>(kparams<double>(g, nsteps), g->sched, launch_grid(g),
                             g->d_counts + 1, st);
  if (e != cudaSuccess) return cuda_err(err, e, "chunk launch");
  return RTI_OK;
}

int snapshot_any(Group* g, cudaStream_t st, std::string* err) {
  cudaError_t e = g->prec == RTI_FP32 ? launch_snapshot<float>(kparams<float>(g, 0), g->grid, st)
                                      : launch_snapshot<double>(kparams<double>(g, 0), g->grid, st);
  if (e != cudaSuccess) return cuda_err(err, e, "snapshot");
  return RTI_OK;
}

// One chunk of a group, through a captured CUDA graph when the capture works.
int group_chunk(Group* g, cudaStream_t st, std::string* err) {
  if (!g->graph_tried) {
    g->graph_tried = true;
    cudaError_t e = cudaSuccess;
    if (!g->cap_stream) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      std::string lerr;
      launch_any(g, g->chunk, g->cap_stream, &lerr);
      e = cudaStreamEndCapture(g->cap_stream, &graph);
    }
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {  // capture unsupported here: launch directly from now on
      g->gexec = nullptr;
      cudaGetLastError();
    }
  }
  if (g->gexec) {
    cudaError_t e = cudaGraphLaunch(g->gexec, st);
    if (e != cudaSuccess) return cuda_err(err, e, "graph launch");
    return RTI_OK;
  }
  return launch_any(g, g->chunk, st, err);
}

void advance_mirror(Group* g, int nsteps) {
  for (size_t mi = 0; mi < g->members.size(); ++mi) {
    long long d = std::min<long long>(g->remaining[mi], nsteps);
    if (d < 0) d = 0;
    g->members[mi]->base += d;
    g->remaining[mi] -= d;
  }
}

// The device status of a handle (and of the group that steps it). A barrier timeout is
// reported once: the group's status word is cleared with the report, so that every later
// launch of the group does not stop at its first barrier; the state stays undefined until
// the caller sets a new one.
int read_status(Group* g, rti_handle* h, std::string* err) {
  int st_h = 0, st_g = 0;
  cudaError_t e = cudaMemcpy(&st_h, h->arena + h->off_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && g) e = cudaMemcpy(&st_g, g->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(err, e, "status read");
  if ((st_h | st_g) & kStTimeout) {
    if (g) e = cudaMemset(g->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_err(err, e, "status reset");
    return set_err(err, RTI_ERR_TIMEOUT,
                   "device barrier wait timed out; state undefined until it is set again");
  }
  if (st_h & kStNonFinite) return set_err(err, RTI_ERR_NONFINITE, "non-finite water level");
  return RTI_OK;
}

bool bad_block(const rti_handle* h, int k) { return !h || k < 0 || k >= (int)h->blocks.size(); }

// ---- host transfers: binary64 host arrays <-> pitched planes in the state precision.
// A host array is copied whole into the handle's binary64 staging plane, and a kernel
// converts it into (or out of) the pitched layout, so the host does no per-cell work.

template <class T>
__global__ void k_plane_from_dense(const double* in, T* plane, int nx, int ny, int pitch) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    plane[(size_t)(r + kYOff) * pitch + (c + kXOff)] = (T)in[i];
  }
}

template <class T>
__global__ void k_dense_from_plane(const T* plane, int nx, int ny, int pitch, double* out) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    out[i] = (double)plane[(size_t)(r + kYOff) * pitch + (c + kXOff)];
  }
}

// R11: velocity across a face of flux q and depth D (0 on a face without water)
template <class T>
__device__ __forceinline__ T face_velocity(T q, T D, T eps) {
  return D > eps ? q / D : T(0);
}

// maximum water velocity of a block: the running maximum, with the current state added
// (R11: the mean of the four face velocities, each flux over its face's depth; a block
// edge's face has the edge cell's depth)
template <class T>
__global__ void k_max_velocity(const T* vmax, const T* eta, const T* M, const T* N, const T* hpl,
                               int nx, int ny, int pitch, T eps, double* out) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    const size_t o = (size_t)(r + kYOff) * pitch + (c + kXOff);
    T m = vmax[o];
    const T h = hpl[o], e = eta[o], D = h + e;
    if (D > eps) {
      const size_t w = c > 0 ? o - 1 : o, ea = c < nx - 1 ? o + 1 : o;
      const size_t s = r > 0 ? o - pitch : o, no = r < ny - 1 ? o + pitch : o;
      const T Dw = T(0.5) * (hpl[w] + h) + T(0.5) * (eta[w] + e);
      const T De = T(0.5) * (h + hpl[ea]) + T(0.5) * (e + eta[ea]);
      const T Ds = T(0.5) * (hpl[s] + h) + T(0.5) * (eta[s] + e);
      const T Dn = T(0.5) * (h + hpl[no]) + T(0.5) * (e + eta[no]);
      const T u = T(0.5) * (face_velocity(M[o], Dw, eps) + face_velocity(M[o + 1], De, eps));
      const T v = T(0.5) * (face_velocity(N[o], Ds, eps) + face_velocity(N[o + pitch], Dn, eps));
      const T s2 = u * u + v * v;
      if (s2 > m) m = s2;
    }
    out[i] = sqrt((double)m);
  }
}

// forecast outputs of a block: 0 max depth (0 where never wet), 1 max height (NaN where
// never wet; the marker is kNeverWet rounded to the state precision, tested by range),
// 2 arrival time in seconds (-1 where the level never reached the threshold)
template <class T>
__global__ void k_output(int kind, const T* emax, const T* hpl, const int* arr, int nx, int ny,
                         int pitch, double dt, double* out) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    const size_t o = (size_t)(r + kYOff) * pitch + (c + kXOff);
    if (kind == 2) {
      const int a = arr[o];
      out[i] = a < 0 ? -1.0 : (double)a * dt;
    } else {
      const double em = (double)emax[o];
      const bool never = em < 0.5 * kNeverWet;
      out[i] = kind == 1 ? (never ? nan("") : em) : (never ? 0.0 : (double)hpl[o] + em);
    }
  }
}

// Initial state of a block (R10): eta0 = dz on sea cells (h > 0), floored at -h; the dry
// land level -h elsewhere; max eta and arrival step from the initial level.
template <class T>
__global__ void k_init_block(const double* dz, const T* hpl, T* eta, T* emax, int* arr, int nx,
                             int ny, int pitch, T eps, T thr) {
  const long long n = (long long)nx * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    const size_t o = (size_t)(r + kYOff) * pitch + (c + kXOff);
    const double hh = (double)hpl[o];
    double e0;
    if (hh > 0) {
      e0 = dz ? dz[i] : 0.0;
      if (e0 < -hh) e0 = -hh;
    } else {
      e0 = -hh;
    }
    const T e = (T)e0, ht = (T)hh;
    T em = (T)kNeverWet;
    int a = -1;
    if (ht + e > eps && e > em) {
      if (em < thr && e >= thr) a = 0;
      em = e;
    }
    eta[o] = e;
    emax[o] = em;
    arr[o] = a;
  }
}

// binary64 sum of a block's plane in a fixed order: kIoBlocks partial sums, summed on the host
template <class T>
__global__ void k_sum_plane(const T* plane, int nx, int ny, int pitch, double* part) {
  __shared__ double red[kIoThreads / 32];
  const long long n = (long long)nx * ny;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nx), c = (int)(i - (long long)r * nx);
    acc += (double)plane[(size_t)(r + kYOff) * pitch + (c + kXOff)];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kIoThreads / 32; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

double* io_plane(rti_handle* h) { return reinterpret_cast<double*>(h->arena + h->off_io); }

// download a pitched plane (ncols x nrows starting at column/row 0) into a host double array
int download(rti_handle* h, size_t off, int ncols, int nrows, int pitch, bool is_state,
             double* out, std::string* err) {
  const size_t n = (size_t)ncols * nrows;
  double* io = io_plane(h);
  if (!is_state)
    k_dense_from_plane<float><<<kIoBlocks, kIoThreads>>>((const float*)(h->arena + off), ncols,
                                                          nrows, pitch, io);
  else if (h->prec == RTI_FP32)
    k_dense_from_plane<float><<<kIoBlocks, kIoThreads>>>((const float*)(h->arena + off), ncols,
                                                          nrows, pitch, io);
  else
    k_dense_from_plane<double><<<kIoBlocks, kIoThreads>>>((const double*)(h->arena + off),
                                                           ncols, nrows, pitch, io);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, io, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(err, e, "download");
  h->d2h += (long long)(n * sizeof(double));
  return RTI_OK;
}

int upload(rti_handle* h, size_t off, int ncols, int nrows, int pitch, const double* in,
           std::string* err) {
  const size_t n = (size_t)ncols * nrows;
  double* io = io_plane(h);
  cudaError_t e = cudaMemcpy(io, in, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (h->prec == RTI_FP32)
      k_plane_from_dense<float><<<kIoBlocks, kIoThreads>>>(io, (float*)(h->arena + off), ncols,
                                                            nrows, pitch);
    else
      k_plane_from_dense<double><<<kIoBlocks, kIoThreads>>>(io, (double*)(h->arena + off), ncols,
                                                             nrows, pitch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(err, e, "upload");
  h->h2d += (long long)(n * sizeof(double));
  return RTI_OK;
}

// binary64 sum of the state-precision plane at `off` (block k)
int plane_sum(rti_handle* h, size_t off, int nx, int ny, int pitch, double* sum, std::string* err) {
  double* io = io_plane(h);
  if (h->prec == RTI_FP32)
    k_sum_plane<float><<<kIoBlocks, kIoThreads>>>((const float*)(h->arena + off), nx, ny, pitch, io);
  else
    k_sum_plane<double><<<kIoBlocks, kIoThreads>>>((const double*)(h->arena + off), nx, ny, pitch,
                                                    io);
  std::vector<double> part(kIoBlocks);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(part.data(), io, kIoBlocks * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(err, e, "plane sum");
  double t = 0.0;
  for (double v : part) t += v;
  *sum = t;
  return RTI_OK;
}

int wait_handle(rti_handle* h) {
  cudaError_t e = cudaEventSynchronize(h->done);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "wait");
  return RTI_OK;
}

// Poll an event until it completes or `seconds` pass (no blocking device call):
// RTI_OK, RTI_ERR_TIMEOUT, or RTI_ERR_CUDA.
int poll_event(cudaEvent_t ev, double seconds, std::string* err) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return RTI_OK;
    if (e != cudaErrorNotReady) return cuda_err(err, e, "wait");
    const double dt =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt >= seconds)
      return set_err(err, RTI_ERR_TIMEOUT, "host watchdog: the enqueued work has not finished");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// initial level and outputs of block k (dz: host binary64 uplift, or null for rest)
template <class T>
int init_block_t(rti_handle* h, int k, const double* dz) {
  const rti_block& d = h->blocks[k];
  const BlkMem& m = h->mem[k];
  const size_t n = (size_t)d.nx * d.ny;
  cudaError_t e = cudaSuccess;
  double* io = io_plane(h);
  if (dz) {
    e = cudaMemcpy(io, dz, n * sizeof(double), cudaMemcpyHostToDevice);
    h->h2d += (long long)(n * sizeof(double));
  }
  if (e == cudaSuccess) {
    k_init_block<T><<<kIoBlocks, kIoThreads>>>(
        dz ? io : nullptr, (const T*)(h->arena + m.h), (T*)(h->arena + m.eta[0]),
        (T*)(h->arena + m.emax), (int*)(h->arena + m.arr), d.nx, d.ny, m.pitch,
        (T)h->params.dry_eps, (T)h->params.arrival_thr);
    e = cudaGetLastError();
  }
  const size_t plane = (size_t)m.pitch * m.rows, es = sizeof(T);
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) e = cudaMemset(h->arena + m.M[s], 0, plane * es);
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) e = cudaMemset(h->arena + m.N[s], 0, plane * es);
  if (e == cudaSuccess)
    e = cudaMemset(h->arena + m.budget, 0, (size_t)m.tiles_x * m.tiles_y * 4 * sizeof(double));
  if (e == cudaSuccess && m.vmax) e = cudaMemset(h->arena + m.vmax, 0, plane * es);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "initial state");
  return RTI_OK;
}

}  // namespace

// ============================================================================== C ABI
extern "C" {

const char* rti_error_string(int code) {
  switch (code) {
    case RTI_OK: return "ok";
    case RTI_ERR_INVALID_ARG: return "invalid argument";
    case RTI_ERR_CFL: return "CFL condition violated (Eq. 4)";
    case RTI_ERR_NESTING: return "invalid nesting";
    case RTI_ERR_OOM: return "out of device memory";
    case RTI_ERR_NONFINITE: return "non-finite water level";
    case RTI_ERR_TIMEOUT: return "device barrier timeout";
    case RTI_ERR_CUDA: return "CUDA error";
    case RTI_ERR_STATE: return "call not allowed in this state";
    default: return "unknown error";
  }
}

const char* rti_last_error(const rti_handle* h) { return h ? h->err.c_str() : t_create_err.c_str(); }

int rti_footprint(const rti_block* blocks, int nblocks, const rti_params* params, size_t* bytes) {
  std::string why;
  if (!bytes) return RTI_ERR_INVALID_ARG;
  int rc = validate(blocks, nblocks, params, &why);
  if (rc) return rc;
  const int tx = params->tile_x ? params->tile_x : kDefaultTx;
  const int ty = params->tile_y ? params->tile_y : kDefaultTy;
  *bytes = plan_layout(blocks, nblocks, params->precision, tx, ty, nullptr, nullptr, nullptr,
                       params->track_velocity != 0);
  return RTI_OK;
}

namespace {

// Scan of the host inputs before any device call: every bathymetry and Manning value
// finite, and Eq. 4 per block with that block's h_max. The scan reads every input byte
// once (0.56 GB for the 46.65 M-cell hierarchy, tens of milliseconds on one core), so
// large inputs are split into chunks of 2^20 cells taken by up to 16 host threads.
int scan_inputs(const rti_block* blocks, int nblocks, const double* const* bathy,
                const float* const* manning, const rti_params* p) {
  constexpr size_t kChunk = size_t(1) << 20;
  struct Unit {
    int k;
    size_t a, b;
    double hmax;
    bool bad;
  };
  std::vector<Unit> units;
  size_t total = 0;
  for (int k = 0; k < nblocks; ++k) {
    const size_t n = (size_t)blocks[k].nx * blocks[k].ny;
    total += n;
    for (size_t a = 0; a < n; a += kChunk) units.push_back(Unit{k, a, std::min(n, a + kChunk), 0.0, false});
  }
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t u = next.fetch_add(1); u < units.size(); u = next.fetch_add(1)) {
      Unit& w = units[u];
      const double* hb = bathy[w.k];
      const float* mn = manning[w.k];
      double hm = 0.0;
      bool bad = false;
      for (size_t c = w.a; c < w.b; ++c) {
        bad = bad || !std::isfinite(hb[c]) || !std::isfinite(mn[c]);
        hm = std::max(hm, hb[c]);
      }
      w.hmax = hm;
      w.bad = bad;
    }
  };
  std::vector<std::thread> pool;
  if (total > 4 * kChunk) {
    const unsigned hw = std::thread::hardware_concurrency();
    const unsigned nt = std::min<unsigned>(16, std::max(1u, hw)) - 1;
    try {
      for (unsigned i = 0; i < nt && i + 1 < units.size(); ++i) pool.emplace_back(work);
    } catch (...) {  // no more threads: the ones running and this one finish the scan
    }
  }
  work();
  for (std::thread& t : pool) t.join();
  std::vector<double> hmax(nblocks, 0.0);
  std::vector<char> bad(nblocks, 0);
  for (const Unit& w : units) {
    hmax[w.k] = std::max(hmax[w.k], w.hmax);
    bad[w.k] = bad[w.k] || w.bad;
  }
  for (int k = 0; k < nblocks; ++k) {  // first offending block decides, as a serial scan
    if (bad[k]) return RTI_ERR_INVALID_ARG;
    if (blocks[k].dx / p->dt < std::sqrt(2.0 * p->g * hmax[k])) return RTI_ERR_CFL;
  }
  return RTI_OK;
}

}  // namespace

int rti_create(const rti_block* blocks, int nblocks, const double* const* bathy,
               const float* const* manning, const rti_params* params, void* device_mem,
               size_t device_bytes, rti_handle** out) {
  if (!out) return RTI_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  int rc = validate(blocks, nblocks, params, &why);
  if (rc) return rc;
  if (!bathy || !manning) return RTI_ERR_INVALID_ARG;
  for (int k = 0; k < nblocks; ++k)
    if (!bathy[k] || !manning[k]) return RTI_ERR_INVALID_ARG;
  rc = scan_inputs(blocks, nblocks, bathy, manning, params);  // Eq. 4 with each block's h_max
  if (rc) return rc;
  if (device_mem && ((uintptr_t)device_mem & 255)) return RTI_ERR_INVALID_ARG;
  rti_handle* h = new (std::nothrow) rti_handle();
  if (!h) return RTI_ERR_OOM;
  h->prec = params->precision;
  h->params = *params;
  h->params.tile_x = params->tile_x ? params->tile_x : kDefaultTx;
  h->params.tile_y = params->tile_y ? params->tile_y : kDefaultTy;
  h->blocks.assign(blocks, blocks + nblocks);
  h->arena_bytes = plan_layout(blocks, nblocks, h->prec, h->params.tile_x, h->params.tile_y,
                               &h->mem, &h->off_status, &h->off_io,
                               h->params.track_velocity != 0);
  for (int k = 0; k < nblocks; ++k) h->cells += (long long)blocks[k].nx * blocks[k].ny;
  cudaError_t e = cudaSuccess;
  if (device_mem) {
    if (device_bytes < h->arena_bytes) {
      delete h;
      return RTI_ERR_OOM;
    }
    h->arena = (char*)device_mem;
  } else {
    e = cudaMalloc((void**)&h->arena, h->arena_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return e == cudaErrorMemoryAllocation ? RTI_ERR_OOM : RTI_ERR_CUDA;
    }
    h->own = true;
  }
  auto fail = [&](int code) {
    cudaError_t last = cudaGetLastError();
    t_create_err = h->err.empty() ? std::string("rti_create: ") + cuda_name(last) : h->err;
    rti_destroy(h);
    return code;
  };
  e = cudaMemset(h->arena, 0, h->arena_bytes);
  for (int k = 0; k < nblocks && e == cudaSuccess; ++k) {  // ring overrides start unset
    const BlkMem& m = h->mem[k];
    if (m.ring) e = cudaMemset(h->arena + m.ring, 0xFF, (size_t)m.pitch * m.rows * esize(h->prec));
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cuda_err(&h->err, e, "arena setup");
    return fail(RTI_ERR_CUDA);
  }
  // bathymetry and Manning n into the pitched arrays; sum of h per block for the budget
  h->sum_h.assign(nblocks, 0.0);
  for (int k = 0; k < nblocks; ++k) {
    const rti_block& d = blocks[k];
    const BlkMem& m = h->mem[k];
    const size_t n = (size_t)d.nx * d.ny;
    rc = upload(h, m.h, d.nx, d.ny, m.pitch, bathy[k], &h->err);
    if (rc) return fail(rc);
    rc = plane_sum(h, m.h, d.nx, d.ny, m.pitch, &h->sum_h[k], &h->err);
    if (rc) return fail(rc);
    char* dst = h->arena + m.man + ((size_t)kYOff * m.pitch + kXOff) * 4;
    e = cudaMemcpy2D(dst, (size_t)m.pitch * 4, manning[k], (size_t)d.nx * 4, (size_t)d.nx * 4,
                     (size_t)d.ny, cudaMemcpyHostToDevice);
    h->h2d += (long long)n * 4;
    if (e != cudaSuccess) {
      cuda_err(&h->err, e, "manning upload");
      return fail(RTI_ERR_CUDA);
    }
  }
  h->self = new (std::nothrow) Group();
  if (!h->self) return fail(RTI_ERR_OOM);
  rc = group_init(h->self, h->prec, params->schedule, h->params.tile_x, h->params.tile_y, 1,
                  params->ctas_per_sm, &h->err);
  if (rc) return fail(rc);
  h->self->members.push_back(h);
  h->self->remaining.push_back(0);
  rc = group_upload_any(h->self, 0, &h->err);
  if (rc) return fail(rc);
  for (int k = 0; k < nblocks; ++k) {
    rc = h->prec == RTI_FP32 ? init_block_t<float>(h, k, nullptr)
                             : init_block_t<double>(h, k, nullptr);
    if (rc) return fail(rc);
  }
  rc = snapshot_any(h->self, 0, &h->err);
  if (rc) return fail(rc);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cuda_err(&h->err, e, "create sync");
    return fail(RTI_ERR_CUDA);
  }
  *out = h;
  return RTI_OK;
}

int rti_set_initial_uplift(rti_handle* h, int block, const double* dz) {
  if (bad_block(h, block)) return RTI_ERR_INVALID_ARG;
  if (h->batch) return set_err(&h->err, RTI_ERR_STATE, "handle is in a batch");
  int rc = wait_handle(h);
  if (rc) return rc;
  const size_t es = esize(h->prec);
  if (h->base & 1) {  // move the other blocks' current level to parity 0
    for (size_t k = 0; k < h->blocks.size(); ++k) {
      const BlkMem& m = h->mem[k];
      const size_t plane = (size_t)m.pitch * m.rows * es;
      cudaError_t e = cudaMemcpy(h->arena + m.eta[0], h->arena + m.eta[1], plane, cudaMemcpyDeviceToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(h->arena + m.M[0], h->arena + m.M[1], plane, cudaMemcpyDeviceToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(h->arena + m.N[0], h->arena + m.N[1], plane, cudaMemcpyDeviceToDevice);
      if (e != cudaSuccess) return cuda_err(&h->err, e, "parity reset");
    }
  }
  h->base = 0;
  rc = h->prec == RTI_FP32 ? init_block_t<float>(h, block, dz)
                           : init_block_t<double>(h, block, dz);
  if (rc) return rc;
  cudaError_t e = cudaMemset(h->arena + h->off_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->self->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_err(&h->err, e, "status reset");
  h->self->remaining[0] = 0;
  h->self->dirty = true;
  rc = group_upload_any(h->self, 0, &h->err);
  if (rc) return rc;
  rc = snapshot_any(h->self, 0, &h->err);
  if (rc) return rc;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(&h->err, e, "initial condition");
  return RTI_OK;
}

int rti_step(rti_handle* h, int nsteps, void* stream) {
  if (!h || nsteps < 0) return RTI_ERR_INVALID_ARG;
  if (h->batch) return set_err(&h->err, RTI_ERR_STATE, "handle is stepped by its batch");
  if (nsteps == 0) return RTI_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Group* g = h->self;
  k_set_scen<<<1, 1, 0, st>>>(g->d_scen, 0, h->base, nsteps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(&h->err, e, "step setup");
  g->remaining[0] = nsteps;
  int rc = launch_any(g, nsteps, st, &h->err);
  if (rc) return rc;
  advance_mirror(g, nsteps);
  e = cudaEventRecord(h->done, st);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "event");
  return RTI_OK;
}

int rti_sync(rti_handle* h) {
  if (!h) return RTI_ERR_INVALID_ARG;
  int rc = wait_handle(h);
  if (rc) return rc;
  if (h->batch) {
    cudaError_t e = cudaEventSynchronize(h->batch->done);
    if (e != cudaSuccess) return cuda_err(&h->err, e, "wait");
    return read_status(&h->batch->g, h, &h->err);
  }
  return read_status(h->self, h, &h->err);
}

int rti_sync_timeout(rti_handle* h, double seconds) {
  if (!h || !(seconds >= 0)) return RTI_ERR_INVALID_ARG;
  int rc = poll_event(h->done, seconds, &h->err);
  if (rc) return rc;
  if (h->batch) {
    rc = poll_event(h->batch->done, seconds, &h->err);
    if (rc) return rc;
    return read_status(&h->batch->g, h, &h->err);
  }
  return read_status(h->self, h, &h->err);
}

static int sync_for_read(rti_handle* h) {
  int rc = wait_handle(h);
  if (rc) return rc;
  if (h->batch) {
    cudaError_t e = cudaEventSynchronize(h->batch->done);
    if (e != cudaSuccess) return cuda_err(&h->err, e, "wait");
  }
  return RTI_OK;
}

int rti_get_state(rti_handle* h, int block, double* eta, double* M, double* N) {
  if (bad_block(h, block)) return RTI_ERR_INVALID_ARG;
  int rc = sync_for_read(h);
  if (rc) return rc;
  const rti_block& d = h->blocks[block];
  const BlkMem& m = h->mem[block];
  const int p = (int)(h->base & 1);
  if (d.parent >= 0 && (M || N)) {  // a child's edge fluxes are defined by its parent
    Group* g = h->self;
    cudaError_t e = g->prec == RTI_FP32
                        ? launch_fill_edges<float>(kparams<float>(g, 0), g->grid, p, 0)
                        : launch_fill_edges<double>(kparams<double>(g, 0), g->grid, p, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_err(&h->err, e, "edge fluxes");
  }
  if (eta && (rc = download(h, m.eta[p], d.nx, d.ny, m.pitch, true, eta, &h->err))) return rc;
  if (M && (rc = download(h, m.M[p], d.nx + 1, d.ny, m.pitch, true, M, &h->err))) return rc;
  if (N && (rc = download(h, m.N[p], d.nx, d.ny + 1, m.pitch, true, N, &h->err))) return rc;
  return RTI_OK;
}

int rti_set_state(rti_handle* h, int block, const double* eta, const double* M, const double* N) {
  if (bad_block(h, block)) return RTI_ERR_INVALID_ARG;
  if (h->batch) return set_err(&h->err, RTI_ERR_STATE, "handle is in a batch");
  int rc = wait_handle(h);
  if (rc) return rc;
  const rti_block& d = h->blocks[block];
  const BlkMem& m = h->mem[block];
  const int p = (int)(h->base & 1);
  if (eta && (rc = upload(h, m.eta[p], d.nx, d.ny, m.pitch, eta, &h->err))) return rc;
  if (M && (rc = upload(h, m.M[p], d.nx + 1, d.ny, m.pitch, M, &h->err))) return rc;
  if (N && (rc = upload(h, m.N[p], d.nx, d.ny + 1, m.pitch, N, &h->err))) return rc;
  rc = snapshot_any(h->self, 0, &h->err);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(&h->err, e, "set state");
  return RTI_OK;
}

static int get_out(rti_handle* h, int block, double* out, int kind) {
  if (bad_block(h, block) || !out) return RTI_ERR_INVALID_ARG;
  int rc = sync_for_read(h);
  if (rc) return rc;
  const rti_block& d = h->blocks[block];
  const BlkMem& m = h->mem[block];
  const size_t n = (size_t)d.nx * d.ny;
  double* io = io_plane(h);
  const int* arr = (const int*)(h->arena + m.arr);
  if (h->prec == RTI_FP32)
    k_output<float><<<kIoBlocks, kIoThreads>>>(kind, (const float*)(h->arena + m.emax),
                                                (const float*)(h->arena + m.h), arr, d.nx, d.ny,
                                                m.pitch, h->params.dt, io);
  else
    k_output<double><<<kIoBlocks, kIoThreads>>>(kind, (const double*)(h->arena + m.emax),
                                                 (const double*)(h->arena + m.h), arr, d.nx, d.ny,
                                                 m.pitch, h->params.dt, io);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(out, io, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "outputs");
  h->d2h += (long long)(n * sizeof(double));
  return RTI_OK;
}

int rti_get_max_velocity(rti_handle* h, int block, double* out) {
  if (bad_block(h, block) || !out) return RTI_ERR_INVALID_ARG;
  const BlkMem& m = h->mem[block];
  if (!m.vmax)
    return set_err(&h->err, RTI_ERR_STATE, "the handle was created without track_velocity");
  int rc = sync_for_read(h);
  if (rc) return rc;
  const rti_block& d = h->blocks[block];
  const int p = (int)(h->base & 1);
  cudaError_t e = cudaSuccess;
  if (d.parent >= 0) {  // the current state's edge fluxes are defined by the parent
    Group* g = h->self;
    e = g->prec == RTI_FP32 ? launch_fill_edges<float>(kparams<float>(g, 0), g->grid, p, 0)
                            : launch_fill_edges<double>(kparams<double>(g, 0), g->grid, p, 0);
  }
  double* io = io_plane(h);
  char* A = h->arena;
  if (e == cudaSuccess) {
    if (h->prec == RTI_FP32)
      k_max_velocity<float><<<kIoBlocks, kIoThreads>>>(
          (const float*)(A + m.vmax), (const float*)(A + m.eta[p]), (const float*)(A + m.M[p]),
          (const float*)(A + m.N[p]), (const float*)(A + m.h), d.nx, d.ny, m.pitch,
          (float)h->params.dry_eps, io);
    else
      k_max_velocity<double><<<kIoBlocks, kIoThreads>>>(
          (const double*)(A + m.vmax), (const double*)(A + m.eta[p]), (const double*)(A + m.M[p]),
          (const double*)(A + m.N[p]), (const double*)(A + m.h), d.nx, d.ny, m.pitch,
          h->params.dry_eps, io);
    e = cudaGetLastError();
  }
  const size_t n = (size_t)d.nx * d.ny;
  if (e == cudaSuccess) e = cudaMemcpy(out, io, n * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "max velocity");
  h->d2h += (long long)(n * sizeof(double));
  return RTI_OK;
}

int rti_get_max_depth(rti_handle* h, int block, double* out) { return get_out(h, block, out, 0); }
int rti_get_max_height(rti_handle* h, int block, double* out) { return get_out(h, block, out, 1); }
int rti_get_arrival_time(rti_handle* h, int block, double* out) { return get_out(h, block, out, 2); }

// ---- checkpoints: a header, then per block the raw planes of the current level
namespace {
struct CkptHeader {
  unsigned long long magic;  // 'RTICKPT1'
  int prec, nblocks, track, pad;
  long long base;
  unsigned long long bytes;  // whole checkpoint
};
constexpr unsigned long long kCkptMagic = 0x3154504b43495452ULL;

// the (offset, bytes) ranges of block k's checkpointed planes at level p
void ckpt_ranges(const rti_handle* h, int k, int p, std::vector<std::pair<size_t, size_t>>* out) {
  const BlkMem& m = h->mem[k];
  const size_t plane = (size_t)m.pitch * (size_t)m.rows, es = esize(h->prec);
  out->push_back({m.eta[p], plane * es});
  out->push_back({m.M[p], plane * es});
  out->push_back({m.N[p], plane * es});
  out->push_back({m.emax, plane * es});
  out->push_back({m.arr, plane * 4});
  if (m.vmax) out->push_back({m.vmax, plane * es});
  out->push_back({m.budget, (size_t)m.tiles_x * m.tiles_y * 4 * sizeof(double)});
}

size_t ckpt_size(const rti_handle* h) {
  size_t n = sizeof(CkptHeader);
  std::vector<std::pair<size_t, size_t>> r;
  for (size_t k = 0; k < h->blocks.size(); ++k) ckpt_ranges(h, (int)k, 0, &r);
  for (auto& x : r) n += x.second;
  return n;
}
}  // namespace

size_t rti_checkpoint_bytes(const rti_handle* h) { return h ? ckpt_size(h) : 0; }

int rti_checkpoint_save(rti_handle* h, void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < ckpt_size(h)) return RTI_ERR_INVALID_ARG;
  int rc = sync_for_read(h);
  if (rc) return rc;
  CkptHeader hd = {kCkptMagic, h->prec, (int)h->blocks.size(), h->params.track_velocity, 0,
                   h->base, (unsigned long long)ckpt_size(h)};
  char* out = static_cast<char*>(host_buf);
  std::memcpy(out, &hd, sizeof hd);
  size_t o = sizeof hd;
  const int p = (int)(h->base & 1);
  std::vector<std::pair<size_t, size_t>> r;
  for (size_t k = 0; k < h->blocks.size(); ++k) ckpt_ranges(h, (int)k, p, &r);
  for (auto& x : r) {
    cudaError_t e = cudaMemcpy(out + o, h->arena + x.first, x.second, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(&h->err, e, "checkpoint save");
    o += x.second;
    h->d2h += (long long)x.second;
  }
  return RTI_OK;
}

int rti_checkpoint_load(rti_handle* h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf || bytes < sizeof(CkptHeader)) return RTI_ERR_INVALID_ARG;
  if (h->batch) return set_err(&h->err, RTI_ERR_STATE, "handle is in a batch");
  CkptHeader hd;
  std::memcpy(&hd, host_buf, sizeof hd);
  if (hd.magic != kCkptMagic || hd.prec != h->prec || hd.nblocks != (int)h->blocks.size() ||
      hd.track != h->params.track_velocity || hd.bytes != ckpt_size(h) || bytes < hd.bytes ||
      hd.base < 0)
    return set_err(&h->err, RTI_ERR_INVALID_ARG, "checkpoint of another hierarchy or params");
  int rc = wait_handle(h);
  if (rc) return rc;
  const char* in = static_cast<const char*>(host_buf);
  size_t o = sizeof hd;
  const int p = (int)(hd.base & 1);
  std::vector<std::pair<size_t, size_t>> r;
  for (size_t k = 0; k < h->blocks.size(); ++k) ckpt_ranges(h, (int)k, p, &r);
  for (auto& x : r) {
    cudaError_t e = cudaMemcpy(h->arena + x.first, in + o, x.second, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(&h->err, e, "checkpoint load");
    o += x.second;
    h->h2d += (long long)x.second;
  }
  h->base = hd.base;
  cudaError_t e = cudaMemset(h->arena + h->off_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->self->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_err(&h->err, e, "status reset");
  h->self->remaining[0] = 0;
  h->self->dirty = true;
  rc = group_upload_any(h->self, 0, &h->err);
  if (rc) return rc;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(&h->err, e, "checkpoint load");
  return RTI_OK;
}

int rti_get_budget(rti_handle* h, int block, double out[4]) {
  if (bad_block(h, block) || !out) return RTI_ERR_INVALID_ARG;
  int rc = sync_for_read(h);
  if (rc) return rc;
  const BlkMem& m = h->mem[block];
  const size_t nt = (size_t)m.tiles_x * m.tiles_y;
  std::vector<double> s(nt * 4);
  cudaError_t e = cudaMemcpy(s.data(), h->arena + m.budget, nt * 4 * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(&h->err, e, "budget");
  double acc[4] = {0, 0, 0, 0};
  for (size_t t = 0; t < nt; ++t)
    for (int q = 0; q < 4; ++q) acc[q] += s[4 * t + q];
  const double dx = h->blocks[block].dx;
  out[0] = (h->sum_h[block] + acc[0]) * (dx * dx);
  out[1] = acc[2];
  out[2] = acc[1];
  out[3] = acc[3];
  return RTI_OK;
}

int rti_volume(rti_handle* h, double* volume, double* boundary_outflow, double* clip_volume,
               double* feedback_volume) {
  if (!h) return RTI_ERR_INVALID_ARG;
  double acc[4] = {0, 0, 0, 0};
  for (int k = 0; k < (int)h->blocks.size(); ++k) {
    if (h->blocks[k].parent >= 0) continue;
    double b[4];
    const int rc = rti_get_budget(h, k, b);
    if (rc) return rc;
    for (int q = 0; q < 4; ++q) acc[q] += b[q];
  }
  if (volume) *volume = acc[0];
  if (boundary_outflow) *boundary_outflow = acc[1];
  if (clip_volume) *clip_volume = acc[2];
  if (feedback_volume) *feedback_volume = acc[3];
  return RTI_OK;
}

int rti_get_transfer_bytes(const rti_handle* h, long long* h2d, long long* d2h) {
  if (!h || !h2d || !d2h) return RTI_ERR_INVALID_ARG;
  *h2d = h->h2d;
  *d2h = h->d2h;
  return RTI_OK;
}

#ifdef RTI_CHECKED
// Checked builds only: the first out-of-range kernel access of the binary64 module
// (out8[0..7]) and of the binary32 module (out8[8..15]): code, index, extent, ..., CTA.
extern "C" int rti_debug_check(int* out16) {
  cudaError_t e = rti::debug_check_fp64(out16);
  if (e == cudaSuccess) e = rti::debug_check_fp32(out16 + 8);
  return e == cudaSuccess ? RTI_OK : RTI_ERR_CUDA;
}
#endif

long long rti_steps_done(rti_handle* h) {
  if (!h) return -1;
  if (sync_for_read(h)) return -1;
  return h->base;
}
int rti_num_blocks(const rti_handle* h) { return h ? (int)h->blocks.size() : 0; }
long long rti_num_cells(const rti_handle* h) { return h ? h->cells : 0; }

void rti_destroy(rti_handle* h) {
  if (!h) return;
  if (h->batch) rti_batch_remove(h->batch, h);
  if (h->done) cudaEventSynchronize(h->done);
  if (h->self) {
    free_group_dev(h->self);
    delete h->self;
  }
  if (h->done) cudaEventDestroy(h->done);
  if (h->own && h->arena) cudaFree(h->arena);
  delete h;
}

// ------------------------------------------------------------------------------ batches
int rti_batch_create(int precision, int schedule, int chunk_steps, rti_batch** out) {
  const rti_batch_config cfg = {precision, schedule, chunk_steps, 0, 0};
  return rti_batch_create_ex(&cfg, out);
}

int rti_batch_create_ex(const rti_batch_config* cfg, rti_batch** out) {
  if (!out || !cfg || cfg->chunk_steps <= 0 ||
      (cfg->precision != RTI_FP32 && cfg->precision != RTI_FP64) ||
      (cfg->schedule != RTI_SCHED_PERSISTENT && cfg->schedule != RTI_SCHED_PER_PASS) ||
      cfg->tile_y < 0 || cfg->tile_y % 8 || cfg->ctas_per_sm < 0)
    return RTI_ERR_INVALID_ARG;
  rti_batch* b = new (std::nothrow) rti_batch();
  if (!b) return RTI_ERR_OOM;
  int rc = group_init(&b->g, cfg->precision, cfg->schedule, kDefaultTx,
                      cfg->tile_y ? cfg->tile_y : kDefaultTy, cfg->chunk_steps, cfg->ctas_per_sm,
                      &b->err);
  if (rc == RTI_OK && cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
    rc = RTI_ERR_CUDA;
  if (rc) {
    free_group_dev(&b->g);
    delete b;
    return rc;
  }
  *out = b;
  return RTI_OK;
}

int rti_batch_add(rti_batch* b, rti_handle* h, long long nsteps) {
  if (!b || !h || nsteps < 0) return RTI_ERR_INVALID_ARG;
  if (h->batch) return set_err(&h->err, RTI_ERR_STATE, "handle already in a batch");
  if (h->prec != b->g.prec || h->params.tile_x != b->g.tx || h->params.tile_y != b->g.ty)
    return set_err(&h->err, RTI_ERR_INVALID_ARG, "precision or tile shape differs from the batch");
  int rc = wait_handle(h);
  if (rc) return rc;
  b->g.members.push_back(h);
  b->g.remaining.push_back(nsteps);
  b->g.dirty = true;
  h->batch = b;
  return RTI_OK;
}

int rti_batch_remove(rti_batch* b, rti_handle* h) {
  if (!b || !h || h->batch != b) return RTI_ERR_INVALID_ARG;
  cudaEventSynchronize(b->done);  // the member's kernels must be finished
  for (size_t i = 0; i < b->g.members.size(); ++i) {
    if (b->g.members[i] == h) {
      b->g.members.erase(b->g.members.begin() + i);
      b->g.remaining.erase(b->g.remaining.begin() + i);
      break;
    }
  }
  h->batch = nullptr;
  b->g.dirty = true;
  // the handle's own group keeps stepping it from where the batch left it
  h->self->remaining[0] = 0;
  return RTI_OK;
}

int rti_batch_step(rti_batch* b, void* stream) {
  if (!b) return RTI_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->g.dirty) {
    int rc = group_upload_any(&b->g, st, &b->err);
    if (rc) return rc;
  }
  if (b->g.members.empty()) return RTI_OK;
  int rc = group_chunk(&b->g, st, &b->err);
  if (rc) return rc;
  advance_mirror(&b->g, b->g.chunk);
  cudaError_t e = cudaEventRecord(b->done, st);
  if (e != cudaSuccess) return cuda_err(&b->err, e, "event");
  return RTI_OK;
}

long long rti_batch_remaining(rti_batch* b, rti_handle* h) {
  if (!b) return -1;
  for (size_t i = 0; i < b->g.members.size(); ++i)
    if (b->g.members[i] == h) return b->g.remaining[i];
  return -1;
}

int rti_batch_sync(rti_batch* b) {
  if (!b) return RTI_ERR_INVALID_ARG;
  cudaError_t e = cudaEventSynchronize(b->done);
  if (e != cudaSuccess) return cuda_err(&b->err, e, "wait");
  for (rti_handle* h : b->g.members) {
    int rc = read_status(&b->g, h, &h->err);
    if (rc) return rc;
  }
  return RTI_OK;
}

int rti_batch_sync_timeout(rti_batch* b, double seconds) {
  if (!b || !(seconds >= 0)) return RTI_ERR_INVALID_ARG;
  int rc = poll_event(b->done, seconds, &b->err);
  if (rc) return rc;
  for (rti_handle* h : b->g.members) {
    rc = read_status(&b->g, h, &h->err);
    if (rc) return rc;
  }
  return RTI_OK;
}

void rti_batch_destroy(rti_batch* b) {
  if (!b) return;
  cudaEventSynchronize(b->done);
  for (rti_handle* h : b->g.members) h->batch = nullptr;
  free_group_dev(&b->g);
  if (b->done) cudaEventDestroy(b->done);
  delete b;
}

}  // extern "C"

// ===================================================================== allocation-free step
// rti_step_noalloc: one root grid stepped with the library's kernels, every piece of
// scratch (block descriptor, tile list, scenario counters, device barrier, status words,
// per-tile budget partials) taken from one file-scope device array instead of cudaMalloc.
namespace {

constexpr int kNoAllocMaxTiles = 4096;  // e.g. 2048 x 2048 cells in 28 x 64 strips (2368)

struct NoAllocScratch {
  Blk<double> blk;  // holds a Blk<float> or a Blk<double>
  int counts[2];    // tiles, scenarios
  int status_group;
  int status_grid;
  ScenDev scen;
  Bar bar;
  int kids[4];
  unsigned long long done[4];  // strip flags of full feedback (unused by a lone root)
  Tile tiles[kNoAllocMaxTiles];
  double budget[4 * kNoAllocMaxTiles];
};

}  // namespace

// The scratch itself: ~200 KB, resident on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256];  // device address of the scratch, per device ordinal

// Writes the tile list, the descriptor and the counters, and clears the barrier, the
// status words and the budget partials (the array keeps the previous call's contents).
template <class T>
__global__ void k_noalloc_setup(NoAllocScratch* s, Blk<T> b, int tx, int ty, int tiles_x,
                                int tiles_y, long long steps_done, long long nsteps) {
  const int nt = tiles_x * tiles_y;
  for (int k = threadIdx.x; k < nt; k += blockDim.x) {
    Tile t;
    t.blk = 0;
    t.x0 = (k % tiles_x) * tx;
    t.y0 = (k / tiles_x) * ty;
    t.flags = (t.x0 == 0 ? kTfWest : 0) | (t.x0 + tx >= b.nx ? kTfEast : 0) |
              (t.y0 == 0 ? kTfSouth : 0) | (t.y0 + ty >= b.ny ? kTfNorth : 0);
    s->tiles[k] = t;
    for (int q = 0; q < 4; ++q) s->budget[4 * k + q] = 0.0;
  }
  if (threadIdx.x == 0) {
    *reinterpret_cast<Blk<T>*>(&s->blk) = b;
    s->counts[0] = nt;
    s->counts[1] = 1;
    s->status_group = 0;
    s->status_grid = 0;
    s->scen.base = steps_done;
    s->scen.remaining = nsteps;
    s->bar.count = 0;
    s->bar.gen = 0;
    s->bar.next[0] = s->bar.next[1] = 0;
  }
}

template <class T>
int noalloc_run(NoAllocScratch* s, const rti_block* g, const rti_params* p,
                const rti_noalloc_state* st, long long steps_done, int nsteps, cudaStream_t stream) {
  const int tx = p->tile_x ? p->tile_x : kDefaultTx, ty = p->tile_y ? p->tile_y : kDefaultTy;
  const int tiles_x = (g->nx + tx - 1) / tx, tiles_y = (g->ny + ty - 1) / ty;
  Blk<T> b;
  std::memset(&b, 0, sizeof(b));
  for (int q = 0; q < 2; ++q) {
    b.eta[q] = (T*)st->eta[q];
    b.M[q] = (T*)st->M[q];
    b.N[q] = (T*)st->N[q];
  }
  b.h = (const T*)st->h;
  b.man = st->manning;
  b.emax = (T*)st->max_eta;
  b.arr = st->arrival_step;
  b.nx = g->nx;
  b.ny = g->ny;
  b.pitch = st->pitch;
  b.parent = -1;
  for (int q = 0; q < 4; ++q) b.bc[q] = g->bc[q];
  b.tiles_x = tiles_x;
  b.budget = s->budget;
  b.status = &s->status_grid;
  b.dtdx = (T)(p->dt / g->dx);
  b.dt = (T)p->dt;
  b.g = (T)p->g;
  b.cfric = (T)(0.5 * p->dt * p->g);
  b.eps = (T)p->dry_eps;
  b.thr = (T)p->arrival_thr;
  b.dx = (T)g->dx;
  b.q4dt = (T)(4.0 * p->dt);
  b.vlim = p->velocity_limit > 0 ? (T)p->velocity_limit : (T)INFINITY;
  b.dx2 = g->dx * g->dx;
  b.vol = p->dt * g->dx;
  b.eps_d = p->dry_eps;
#ifdef RTI_CHECKED
  b.lo = nullptr;
  b.hi = reinterpret_cast<const char*>(~0ull);
#endif
  k_noalloc_setup<T><<<1, 256, 0, stream>>>(s, b, tx, ty, tiles_x, tiles_y, steps_done, nsteps);
  cudaError_t e = cudaGetLastError();
  int grid = 0;
  const int mode = kStepPlain | (p->velocity_limit > 0 ? kStepLimit : 0);
  if (e == cudaSuccess) e = persistent_grid<T>(&grid, tx, ty, mode, p->ctas_per_sm);
  if (e == cudaSuccess) {
    KParams<T> kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.blk = reinterpret_cast<const Blk<T>*>(&s->blk);
    kp.kids = s->kids;
    kp.tiles = s->tiles;
    kp.ntiles = &s->counts[0];
    kp.scen = &s->scen;
    kp.status = &s->status_group;
    kp.bar = &s->bar;
    kp.done = s->done;
    kp.ndone = 1;
    kp.nsteps = nsteps;
    kp.tx = tx;
    kp.ty = ty;
    kp.spin_cycles = kSpinCycles;
    kp.limit = p->velocity_limit > 0 ? 1 : 0;
#ifdef RTI_CHECKED
    kp.nblk = 1;
    kp.nkids = 0;
#endif
    e = launch_chunk<T>(kp, p->schedule, grid, &s->counts[1], stream);
  }
  // the two status words, read on the caller's stream behind the steps; the one wait
  // below covers the steps and the copy
  int words[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(words, &s->status_group, sizeof(words), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    t_create_err = std::string("rti_step_noalloc: ") + cudaGetErrorString(e);
    return RTI_ERR_CUDA;
  }
  if ((words[0] | words[1]) & kStTimeout) return RTI_ERR_TIMEOUT;
  if (words[1] & kStNonFinite) return RTI_ERR_NONFINITE;
  return RTI_OK;
}

}  // namespace

extern "C" int rti_step_noalloc(const rti_block* grid, const rti_params* params,
                                const rti_noalloc_state* state, long long steps_done, int nsteps,
                                void* stream) {
  t_create_err.clear();
  std::string why;
  if (!grid || !params || !state || steps_done < 0 || nsteps < 0) return RTI_ERR_INVALID_ARG;
  int rc = validate(grid, 1, params, &why);
  if (rc) {
    t_create_err = "rti_step_noalloc: " + why;
    return rc;
  }
  if (params->track_velocity) {
    t_create_err = "rti_step_noalloc: track_velocity needs a plane the state does not have";
    return RTI_ERR_INVALID_ARG;
  }
  const int tx = params->tile_x ? params->tile_x : kDefaultTx;
  const int ty = params->tile_y ? params->tile_y : kDefaultTy;
  const long long tiles = (long long)((grid->nx + tx - 1) / tx) * ((grid->ny + ty - 1) / ty);
  if (tiles > kNoAllocMaxTiles) {
    t_create_err = "rti_step_noalloc: grid of " + std::to_string(tiles) + " tiles exceeds the " +
                    std::to_string(kNoAllocMaxTiles) + "-tile scratch";
    return RTI_ERR_INVALID_ARG;
  }
  for (int q = 0; q < 2; ++q)
    if (!state->eta[q] || !state->M[q] || !state->N[q]) return RTI_ERR_INVALID_ARG;
  if (!state->h || !state->manning || !state->max_eta || !state->arrival_step ||
      state->pitch < grid->nx + 9 || state->pitch % 4 ||
      (long long)state->pitch * rows_for(grid->ny) >= (1LL << 31)) {
    t_create_err = "rti_step_noalloc: null state array, or pitch below nx + 9, not a multiple of 4 "
                   "or too large (pitch x (ny + 5) must stay below 2^31)";
    return RTI_ERR_INVALID_ARG;
  }
  if (nsteps == 0) return RTI_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) return RTI_ERR_CUDA;
  {  // every array must be memory the device can address (no launch on a stray pointer)
    const void* arr[10] = {state->eta[0], state->eta[1], state->M[0],       state->M[1],
                           state->N[0],   state->N[1],   state->h,          state->manning,
                           state->max_eta, state->arrival_step};
    for (const void* a : arr) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, a) != cudaSuccess || at.devicePointer == nullptr ||
          (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        t_create_err = "rti_step_noalloc: a state array is not device memory";
        return RTI_ERR_INVALID_ARG;
      }
      if (reinterpret_cast<uintptr_t>(a) % 16) {
        t_create_err = "rti_step_noalloc: a state array is not 16-byte aligned";
        return RTI_ERR_INVALID_ARG;
      }
    }
  }
  void* addr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {  // once per device, with that device current
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) {
        t_create_err = std::string("rti_step_noalloc: scratch address: ") + cudaGetErrorString(e);
        return RTI_ERR_CUDA;
      }
      g_noalloc_addr[dev] = addr;
    }
    addr = g_noalloc_addr[dev];
  }
  NoAllocScratch* s = static_cast<NoAllocScratch*>(addr);
  cudaStream_t st = (cudaStream_t)stream;
  return params->precision == RTI_FP32 ? noalloc_run<float>(s, grid, params, state, steps_done, nsteps, st)
                                       : noalloc_run<double>(s, grid, params, state, steps_done, nsteps, st);
}
