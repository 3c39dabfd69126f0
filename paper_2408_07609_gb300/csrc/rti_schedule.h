// rti_schedule.h -- host-side scheduling of a group's work list (no CUDA): the order of
// a full-feedback group's strips and the dependencies of a chunk run as one dataflow.
// Kept apart from the host library so that the CPU tests can check their properties
// (every strip comes after the strips it waits for; the dependencies cover each
// strip's neighbourhood and nest partners).
#pragma once

#include <algorithm>
#include <queue>
#include <utility>
#include <vector>

#include "rti_layout.h"

namespace rti {

// Order of the work list of a group with full feedback (list scheduling on the critical
// path). A parent's ring strip with full feedback waits for the child strips that own
// the patches under its region (the ranges the kernel waits for, wait_ring_means). Each
// strip weighs its cells, a ring strip 1.3 times (it also reads the ring plane); its rank
// is its weight plus the largest rank among the strips that wait for it, i.e. the
// longest chain of waits it starts. A simulation of `workers` warps, each taking, as it
// frees up, the highest-ranked strip whose dependencies have ended, gives the handout
// order: deep chains start first, the rest fills in around them, and every strip comes
// after the strips it waits for (so a waiting warp waits only on strips already handed
// out). `tiles` holds each block's strips from index strip0 on, row by row.
template <class T>
std::vector<Tile> full_feedback_order(const std::vector<Blk<T>>& blks,
                                      const std::vector<int>& kids,
                                      const std::vector<Tile>& tiles, int tx, int ty,
                                      int workers) {
  const int n = (int)tiles.size();
  std::vector<double> w(n), rank(n);
  std::vector<std::vector<int>> deps(n), users(n);
  for (int t = 0; t < n; ++t) {
    const Tile& td = tiles[t];
    const Blk<T>& b = blks[td.blk];
    const int cols = std::min(tx, b.nx - td.x0), rows = std::min(ty, b.ny - td.y0);
    w[t] = (double)cols * rows * ((td.flags & kTfRing) ? 1.3 : 1.0);
    if (!(td.flags & kTfRing) || !(b.nest & kNestFull)) continue;
    const int ye = std::min(td.y0 + ty, b.ny);
    const int c0 = std::max(td.x0 - 2, 0), c1 = std::min(td.x0 + tx + 2, b.nx);
    const int r0 = std::max(td.y0 - 2, 0), r1 = std::min(ye + 1, b.ny);
    for (int q = 0; q < b.child_count; ++q) {
      const Blk<T>& c = blks[kids[b.child_first + q]];
      const int a0 = c.i0, a1 = c.i0 + c.nx / 3, b0 = c.j0, b1 = c.j0 + c.ny / 3;
      const int u0 = std::max(c0, a0) - a0, u1 = std::min(c1, a1) - a0;
      const int v0 = std::max(r0, b0) - b0, v1 = std::min(r1, b1) - b0;
      if (u0 >= u1 || v0 >= v1) continue;
      for (int sy = (3 * v0 + 2) / ty; sy <= (3 * (v1 - 1) + 2) / ty; ++sy)
        for (int sx = (3 * u0 + 2) / tx; sx <= (3 * (u1 - 1) + 2) / tx; ++sx)
          deps[t].push_back(c.strip0 + sy * c.tiles_x + sx);
    }
    for (int d : deps[t]) users[d].push_back(t);
  }
  // ranks, coarse levels first (a strip's waiters sit one level up)
  std::vector<int> level(blks.size(), 0);
  for (size_t k = 0; k < blks.size(); ++k)
    for (int a = blks[k].parent; a >= 0; a = blks[a].parent) ++level[k];
  std::vector<int> by_level(n);
  for (int t = 0; t < n; ++t) by_level[t] = t;
  std::stable_sort(by_level.begin(), by_level.end(), [&](int a, int b) {
    return level[tiles[a].blk] < level[tiles[b].blk];
  });
  for (int t : by_level) {
    double up = 0.0;
    for (int u : users[t]) up = std::max(up, rank[u]);
    rank[t] = w[t] + up;
  }
  // the simulated handout
  std::vector<int> left(n);
  std::priority_queue<std::pair<double, int>> ready;  // (rank, -index): lowest index on ties
  std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>,
                      std::greater<std::pair<double, int>>>
      running;  // (finish time, index)
  for (int t = 0; t < n; ++t) {
    left[t] = (int)deps[t].size();
    if (!left[t]) ready.push({rank[t], -t});
  }
  std::vector<Tile> out;
  std::vector<char> taken(n, 0);
  out.reserve(n);
  double now = 0.0;
  int idle = std::max(workers, 1);
  while ((int)out.size() < n) {
    while (idle > 0 && !ready.empty()) {
      const int t = -ready.top().second;
      ready.pop();
      out.push_back(tiles[t]);
      taken[t] = 1;
      running.push({now + w[t], t});
      --idle;
    }
    if (running.empty()) break;  // nothing left that can start (no dependency cycle exists)
    const std::pair<double, int> f = running.top();
    running.pop();
    now = f.first;
    ++idle;
    for (int u : users[f.second])
      if (--left[u] == 0) ready.push({rank[u], -u});
  }
  for (int t = 0; t < n; ++t)
    if (!taken[t]) out.push_back(tiles[t]);
  return out;
}

// Dependencies of the steps of a chunk run as one dataflow (no device-wide barrier):
// strip X's step s may start once these strips (as flag indices, strip0 + slot) have
// ended step s - 1. A strip reads, at step s, cells and faces up to 4 columns and 2 rows
// beyond its own (its 3 x 3 neighbourhood of strips, itself included, wrote them at step
// s - 1) and overwrites at step s what they read at step s - 1 (the ping-pong buffers).
// Across levels the conservative rule: a child strip and a parent strip depend on each
// other both ways when the child strip's region, in parent cells and one cell wider,
// meets the parent strip's region (the child pulls the parent's edge fluxes, the
// parent's ring strip recomputes or reads the child's levels, and each overwrites at the
// next step what the other read). Returns CSR lists by work-list position: deps of list
// entry t are idx[off[t] .. off[t+1]).
template <class T>
void dataflow_deps(const std::vector<Blk<T>>& blks, const std::vector<Tile>& tiles, int tx,
                   int ty, std::vector<int>* off, std::vector<int>* idx) {
  const int n = (int)tiles.size();
  std::vector<std::vector<int>> deps(n);
  std::vector<int> pos;  // flag index -> work-list position
  for (const Blk<T>& b : blks) pos.resize(std::max<size_t>(pos.size(), (size_t)b.strip0 +
                                                            b.tiles_x * ((b.ny + ty - 1) / ty)));
  auto flag_of = [&](const Tile& t) {
    const Blk<T>& b = blks[t.blk];
    return b.strip0 + (t.y0 / ty) * b.tiles_x + t.x0 / tx;
  };
  for (int t = 0; t < n; ++t) pos[flag_of(tiles[t])] = t;
  auto floor_div = [](int a, int d) { return a >= 0 ? a / d : -((-a + d - 1) / d); };
  for (int t = 0; t < n; ++t) {
    const Tile& td = tiles[t];
    const Blk<T>& b = blks[td.blk];
    const int tiles_y = (b.ny + ty - 1) / ty, sx = td.x0 / tx, sy = td.y0 / ty;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = sx + dx, y = sy + dy;
        if (x >= 0 && x < b.tiles_x && y >= 0 && y < tiles_y)
          deps[t].push_back(b.strip0 + y * b.tiles_x + x);
      }
    if (!b.is_child) continue;
    // this child strip's region in parent cells, one cell wider
    const Blk<T>& P = blks[b.parent];
    const int ye = std::min(td.y0 + ty, b.ny);
    const int pc0 = b.i0 + floor_div(td.x0 - 4, 3) - 1, pc1 = b.i0 + (td.x0 + tx + 4 + 2) / 3 + 1;
    const int pr0 = b.j0 + floor_div(td.y0 - 2, 3) - 1, pr1 = b.j0 + (ye + 2 + 2) / 3 + 1;
    const int ptiles_y = (P.ny + ty - 1) / ty;
    for (int y = std::max(0, floor_div(pr0 - ty - 2, ty)); y < ptiles_y && y * ty - 2 < pr1; ++y)
      for (int x = std::max(0, floor_div(pc0 - tx - 4, tx)); x < P.tiles_x && x * tx - 4 < pc1;
           ++x) {
        const int px0 = x * tx - 4, px1 = x * tx + tx + 4;
        const int py0 = y * ty - 2, py1 = std::min(y * ty + ty, P.ny) + 2;
        if (px0 >= pc1 || pc0 >= px1 || py0 >= pr1 || pr0 >= py1) continue;
        const int pf = P.strip0 + y * P.tiles_x + x;
        deps[t].push_back(pf);                     // the child strip waits on the parent's
        deps[pos[pf]].push_back(flag_of(td));      // and the parent strip on the child's
      }
  }
  off->assign(1, 0);
  idx->clear();
  for (int t = 0; t < n; ++t) {
    std::sort(deps[t].begin(), deps[t].end());
    deps[t].erase(std::unique(deps[t].begin(), deps[t].end()), deps[t].end());
    idx->insert(idx->end(), deps[t].begin(), deps[t].end());
    off->push_back((int)idx->size());
  }
}

}  // namespace rti
