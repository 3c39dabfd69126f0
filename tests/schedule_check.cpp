// Host-side check of the work-list schedule (rti_schedule.h), built and run by
// tests/test_schedule.py with the host compiler (no CUDA).
//
// Input (stdin): tx ty workers full steps nblocks, then per block: nx ny parent i0 j0.
// It builds the block descriptors and strips as the library's group upload does (strips
// row by row per block; the ring flag where the strip's 2-cell halo meets a child
// footprint's inner ring, or any of it with full feedback), orders them (longest first,
// or with full feedback full_feedback_order), lists the dataflow dependencies, and
// checks:
//   1. the order is a permutation of the strips;
//   2. a ring strip of a parent with full feedback comes after every child strip whose
//      flag it waits for in the same step (the kernel's ranges);
//   3. every strip's dependencies include its 3 x 3 neighbourhood of strips, itself
//      included, and the nest dependencies are symmetric;
//   4. over `steps` steps handed out step by step in list order, every strip any item
//      waits for (the previous step's dependencies, the same step's children for full
//      feedback) was handed out before that item: a waiting warp waits only on strips
//      held by warps that started earlier, so no wait can close a cycle.
// Prints "OK <strips> <dependencies>" or the first violation, and exits non-zero then.
#include <cstdio>
#include <cstring>
#include <vector>

#include "rti_schedule.h"

using namespace rti;

static int fail(const char* what, int a, int b) {
  std::printf("FAIL %s %d %d\n", what, a, b);
  return 1;
}

int main() {
  int tx, ty, workers, full, steps, nb;
  if (std::scanf("%d %d %d %d %d %d", &tx, &ty, &workers, &full, &steps, &nb) != 6) return 2;
  std::vector<Blk<float>> blks(nb);
  std::vector<std::vector<int>> ch(nb);
  for (int k = 0; k < nb; ++k) {
    Blk<float>& b = blks[k];
    std::memset(&b, 0, sizeof(b));
    if (std::scanf("%d %d %d %d %d", &b.nx, &b.ny, &b.parent, &b.i0, &b.j0) != 5) return 2;
    b.is_child = b.parent >= 0;
    b.nest = full ? kNestFull : 0;
    b.tiles_x = (b.nx + tx - 1) / tx;
    if (b.parent >= 0) ch[b.parent].push_back(k);
  }
  std::vector<int> kids;
  int nflags = 0;
  for (int k = 0; k < nb; ++k) {
    blks[k].child_first = (int)kids.size();
    blks[k].child_count = (int)ch[k].size();
    for (int c : ch[k]) kids.push_back(c);
    blks[k].strip0 = nflags;
    nflags += blks[k].tiles_x * ((blks[k].ny + ty - 1) / ty);
  }
  std::vector<Tile> tiles;
  for (int k = 0; k < nb; ++k) {
    const Blk<float>& b = blks[k];
    for (int y0 = 0; y0 < b.ny; y0 += ty)
      for (int x0 = 0; x0 < b.nx; x0 += tx) {
        Tile t{k, x0, y0, 0};
        const int hx0 = x0 - 2, hy0 = y0 - 2, hx1 = x0 + tx + 2, hy1 = y0 + ty + 2;
        for (int c : ch[k]) {
          const Blk<float>& cd = blks[c];
          const int a0 = cd.i0, a1 = cd.i0 + cd.nx / 3, b0 = cd.j0, b1 = cd.j0 + cd.ny / 3;
          const bool meets = hx0 < a1 && a0 < hx1 && hy0 < b1 && b0 < hy1;
          const bool inner = hx0 >= a0 + 1 && hx1 <= a1 - 1 && hy0 >= b0 + 1 && hy1 <= b1 - 1;
          if (meets && (full || !inner)) t.flags |= kTfRing;
        }
        tiles.push_back(t);
      }
  }
  const int n = (int)tiles.size();
  auto flag_of = [&](const Tile& t) {
    const Blk<float>& b = blks[t.blk];
    return b.strip0 + (t.y0 / ty) * b.tiles_x + t.x0 / tx;
  };
  std::vector<Tile> order = full ? full_feedback_order<float>(blks, kids, tiles, tx, ty, workers)
                                 : tiles;
  // 1. a permutation
  if ((int)order.size() != n) return fail("size", (int)order.size(), n);
  std::vector<int> pos(nflags, -1);
  for (int i = 0; i < n; ++i) {
    const int f = flag_of(order[i]);
    if (pos[f] >= 0) return fail("duplicate", f, i);
    pos[f] = i;
  }
  // the child strips a full-feedback ring strip waits for in its step (the kernel's ranges)
  auto same_step = [&](const Tile& td, std::vector<int>* out) {
    out->clear();
    const Blk<float>& b = blks[td.blk];
    if (!full || !(td.flags & kTfRing)) return;
    const int ye = std::min(td.y0 + ty, b.ny);
    const int c0 = std::max(td.x0 - 2, 0), c1 = std::min(td.x0 + kStripW + 2, b.nx);
    const int r0 = std::max(td.y0 - 2, 0), r1 = std::min(ye + 1, b.ny);
    for (int q = 0; q < b.child_count; ++q) {
      const Blk<float>& c = blks[kids[b.child_first + q]];
      const int a0 = c.i0, a1 = c.i0 + c.nx / 3, b0 = c.j0, b1 = c.j0 + c.ny / 3;
      const int u0 = std::max(c0, a0) - a0, u1 = std::min(c1, a1) - a0;
      const int v0 = std::max(r0, b0) - b0, v1 = std::min(r1, b1) - b0;
      if (u0 >= u1 || v0 >= v1) continue;
      for (int sy = (3 * v0 + 2) / ty; sy <= (3 * (v1 - 1) + 2) / ty; ++sy)
        for (int sx = (3 * u0 + 2) / tx; sx <= (3 * (u1 - 1) + 2) / tx; ++sx)
          out->push_back(c.strip0 + sy * c.tiles_x + sx);
    }
  };
  // 2. children before the ring strips that wait for them
  std::vector<int> w;
  for (int i = 0; i < n; ++i) {
    same_step(order[i], &w);
    for (int f : w)
      if (pos[f] >= i) return fail("child after its ring strip", pos[f], i);
  }
  // 3. neighbourhood and symmetry of the dataflow dependencies
  std::vector<int> off, idx;
  dataflow_deps<float>(blks, order, tx, ty, &off, &idx);
  if ((int)off.size() != n + 1) return fail("offsets", (int)off.size(), n + 1);
  auto has = [&](int i, int f) {
    for (int k = off[i]; k < off[i + 1]; ++k)
      if (idx[k] == f) return true;
    return false;
  };
  for (int i = 0; i < n; ++i) {
    const Tile& t = order[i];
    const Blk<float>& b = blks[t.blk];
    const int tiles_y = (b.ny + ty - 1) / ty, sx = t.x0 / tx, sy = t.y0 / ty;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = sx + dx, y = sy + dy;
        if (x >= 0 && x < b.tiles_x && y >= 0 && y < tiles_y &&
            !has(i, b.strip0 + y * b.tiles_x + x))
          return fail("neighbour missing", i, b.strip0 + y * b.tiles_x + x);
      }
    for (int k = off[i]; k < off[i + 1]; ++k) {
      const int j = pos[idx[k]];
      if (order[j].blk != t.blk && !has(j, flag_of(t)))
        return fail("nest dependency not symmetric", i, j);
    }
  }
  // 4. every wait is on a strip handed out earlier (global sequence step-major)
  for (int s = 0; s < steps; ++s)
    for (int i = 0; i < n; ++i) {
      const long long me = (long long)s * n + i;
      if (s > 0)
        for (int k = off[i]; k < off[i + 1]; ++k)
          if ((long long)(s - 1) * n + pos[idx[k]] >= me) return fail("late dependency", i, k);
      same_step(order[i], &w);
      for (int f : w)
        if ((long long)s * n + pos[f] >= me) return fail("late child", i, f);
    }
  std::printf("OK %d %d\n", n, (int)idx.size());
  return 0;
}
