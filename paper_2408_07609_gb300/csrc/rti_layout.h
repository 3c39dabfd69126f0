// rti_layout.h -- device data layout shared by the host library and the kernels.
//
// Every field of a block lives in its own pitched 2-D array with a margin: element
// (column c, row r) is at (r + kYOff) * pitch + (c + kXOff). Cells use columns
// 0..nx-1 and rows 0..ny-1; x-faces (M) columns 0..nx; y-faces (N) rows 0..ny.
// The margin keeps every stencil read of the kernels inside the allocation; the
// kernels still test indices for the numerics. Rows start on 128-byte boundaries.
#pragma once

#include <stdint.h>

namespace rti {

constexpr int kXOff = 4;       // margin columns before column 0
constexpr int kYOff = 2;       // margin rows before row 0 and after row ny
constexpr int kPitchAlign = 32; // elements
constexpr int kWarps = 4;      // warps per CTA of the step kernel
constexpr int kStripW = 28;    // owned columns of a strip: a warp's 32 lanes less a 2-column halo each side
constexpr double kNeverWet = -1.0e30;

enum : int { kBcWall = 0, kBcRadiation = 1 };
enum : int { kStNonFinite = 1, kStTimeout = 2 };
// tile flags
enum : int { kTfWest = 1, kTfEast = 2, kTfSouth = 4, kTfNorth = 8, kTfRing = 16 };

inline int pitch_for(int nx) {
  int w = kXOff + nx + 1 + 4;
  return (w + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
}
inline long long rows_for(int ny) { return (long long)ny + 1 + 2 * kYOff; }

// Per-block descriptor in device memory. T is the state precision.
template <class T>
struct Blk {
  T* eta[2];  // ping-pong water level (deviation from still water)
  T* M[2];    // ping-pong x-fluxes
  T* N[2];    // ping-pong y-fluxes
  const T* h; // still-water depth
  const float* man;
  T* emax;    // max eta over wet instants (kNeverWet until wet)
  int* arr;   // arrival step, -1 if never
  T* ring;    // a parent's fine-to-coarse eta^{n+1} on ring cells, all-ones bits elsewhere
              // (written each step by the strips that read it); null without children
  T* vmax;    // running max of the squared cell-centre speed; null when not tracked
  int nx, ny, pitch, parent; // parent: index in the batch block table, -1 for a root
  int i0, j0;                // child origin in parent cells
  int child_first, child_count; // children: kids[child_first .. +child_count)
  int bc[4];
  int scen;   // scenario slot (ScenDev index)
  int is_child;
  int tiles_x;     // tiles along x (tile slot = ty_index * tiles_x + tx_index)
  int strip0;      // first of this block's strip flags in the group's flag array (slot
                   // = strip0 + ty_index * tiles_x + tx_index)
  int nest;        // kNest* bits of the owning handle's nesting options
  double* budget;  // 4 doubles per tile of this block: sum(eta) snapshot, clip, outflow, ring
  int* status;     // the owning handle's device status word
  // constants in the state precision (all exactly the values the oracle uses in FP64)
  T dtdx, dt, g, cfric /* 0.5*dt*g */, eps, thr, dx, q4dt /* 4*dt */;
  T vlim;  // velocity limit of the fluxes (m/s), +inf when off
  // binary64 constants for the nesting sums and the budget
  double dx2, vol /* dt*dx */, eps_d;
#ifdef RTI_CHECKED
  const char* lo;  // the owning handle's arena, for the range-checked build
  const char* hi;
#endif
};

// variants of the step kernel
constexpr int kStepPlain = 0;  // no block keeps the maximum velocity
constexpr int kStepTrack = 1;  // some block keeps it
constexpr int kStepLimit = 2;  // flag added to a variant: some block keeps the velocity limit
constexpr int kStepFull = 4;   // flag added to a variant: some block has full feedback
constexpr int kStepModes = 8;  // mode values 0 .. 7

// Flag of a strip with full feedback: (s << 32) | kDoneAll once the strip has ended step s
// of the chunk (its patch means stored). Flags only grow within a chunk.
constexpr unsigned long long kDoneAll = 0xffffffffull;

// nesting options of a block (Blk::nest)
constexpr int kNestFull = 1;   // fine-to-coarse feedback on every covered parent cell
constexpr int kNestConst = 2;  // piecewise-constant coarse-to-fine edge flux

struct ScenDev {
  long long base;    // steps completed before this chunk
  long long remaining; // steps left as of the start of this chunk
};

struct Bar {
  unsigned int count;
  unsigned int gen;
  unsigned int next[2];  // strip counters of the step kernel (step parity)
};

// One tile: cells [x0, x0+tx) x [y0, y0+ty) of block `blk`.
struct Tile {
  int blk, x0, y0, flags;
};

template <class T>
struct KParams {
  const Blk<T>* blk;
  const int* kids;
  const Tile* tiles;
  const int* ntiles;   // device-resident tile count (patched between chunks)
  unsigned long long* done;  // per strip: the last step it has ended (kDoneAll)
  int ndone;                 // entries of `done` (cleared at the start of every chunk)
  const int* dep_off;        // dataflow: strips (flag indices) work-list entry t waits on at
                             // its previous step are idx[dep_off[t] .. dep_off[t+1]), with
                             // idx = dep_off + ntiles + 1; null: steps separated by barriers
  ScenDev* scen;
  int* status;         // group status (barrier timeout)
  Bar* bar;
  int nsteps;
  int track;           // some block keeps the maximum velocity (selects the kernel variant)
  int limit;           // some block keeps the velocity limit (selects the kernel variant)
  int full;            // some block has full feedback (selects the kernel variant)
  int tx, ty;          // tile shape in cells
  long long spin_cycles;
#ifdef RTI_CHECKED
  int nblk, nkids;     // table sizes, for the range-checked build
#endif
};

}  // namespace rti
