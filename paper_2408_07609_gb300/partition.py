"""Decomposition of one nested-grid hierarchy over several GPUs (ranks): the block-to-rank
partitioner and the nest-exchange plan. Host logic only.

Partitioner (the paper's Sec. IV-D, Eq. 5 and Alg. 1). Each rank takes a run of
consecutive blocks of the hierarchy's block list; the runs are set by separators. The
predicted time of a rank is the sum over its blocks of a linear per-block cost,
alpha * cells + beta (Eq. 5 fits alpha = 1.09e-4 us per cell and beta = 46.2 us per
block to its kernel; here the constants are arguments, e.g. the autotuner's per-strip
fit scaled to blocks). Hill climbing improves the separators: pick one at random, move it
to a random position between its neighbours, keep the move only if the score does not
get worse; the score is first the variance of the ranks' predicted times (which every
move changes), then their maximum (which is what a step waits for). Keeping moves that
leave the score unchanged lets the search cross the plateaus of the maximum, where most
moves do not touch the slowest rank; with strictly improving moves only it stalled 20-40 %
above the balanced time on blocks of equal cost.

Exchange plan. Blocks on one rank exchange nothing across ranks with each other; a child
and its parent on different ranks exchange two messages per step (Sec. IV-C):
  - coarse-to-fine ("JNQ"): the parent's new fluxes on the coarse faces along the
    child's footprint edge, nx/3 faces on the south and north edges and ny/3 on the west
    and east, sent to the child's rank after the parent's momentum update;
  - fine-to-coarse ("JNZ"): the child's 3x3 means on the parent cells of the footprint's
    inner ring (every covered cell with full feedback), sent to the parent's rank before
    the parent's next mass update.
Sibling blocks do not exchange (each takes its edge fluxes from the parent), so there
is no same-level halo exchange when whole blocks are assigned.
"""
from __future__ import annotations

import random
from dataclasses import dataclass, field

ALPHA_US, BETA_US = 1.09e-4, 46.2  # Eq. 5 constants (A100, the paper's kernel)


def block_cost(cells, alpha=ALPHA_US, beta=BETA_US):
    return alpha * cells + beta


def rank_times(costs, seps):
    """Predicted time of every rank for separators seps (ascending block indices where a
    new rank starts; len(seps) = ranks - 1)."""
    bounds = [0] + list(seps) + [len(costs)]
    return [sum(costs[bounds[k]:bounds[k + 1]]) for k in range(len(bounds) - 1)]


def _variance(t):
    m = sum(t) / len(t)
    return sum((x - m) ** 2 for x in t) / len(t)


def equal_cells(cells, ranks):
    """The baseline split that equalises cells (the decomposition the paper starts from):
    rank k starts after the block where the running cell count first reaches k / ranks of
    the total, keeping at least one block for every remaining rank."""
    n, total = len(cells), float(sum(cells))
    seps, run = [], 0.0
    for i in range(n - 1):
        run += cells[i]
        k = len(seps) + 1
        if k >= ranks:
            break
        if run >= k * total / ranks or n - (i + 1) == ranks - k:
            seps.append(i + 1)
    return seps


def hill_climb(costs, ranks, iters=20000, seed=0, phase_split=0.5):
    """Alg. 1: separators of `ranks` runs of consecutive blocks minimising first the
    variance, then the maximum of the predicted rank times. Every rank keeps at least
    one block. Returns (separators, rank times)."""
    n = len(costs)
    if ranks < 1 or ranks > n:
        raise ValueError(f"{ranks} ranks for {n} blocks")
    rng = random.Random(seed)
    seps = sorted(rng.sample(range(1, n), ranks - 1)) if ranks > 1 else []
    score = _variance
    best = score(rank_times(costs, seps))
    for it in range(iters):
        if it == int(iters * phase_split):
            score = max
            best = score(rank_times(costs, seps))
        if not seps:
            break
        k = rng.randrange(len(seps))
        lo = seps[k - 1] + 1 if k > 0 else 1
        hi = seps[k + 1] - 1 if k + 1 < len(seps) else n - 1
        if hi < lo:
            continue
        old = seps[k]
        seps[k] = rng.randint(lo, hi)
        s = score(rank_times(costs, seps))
        if s <= best:  # a move that leaves the score unchanged is kept as well
            best = s
        else:
            seps[k] = old
    return seps, rank_times(costs, seps)


def assignment(nblocks, seps):
    """Rank of every block for separators seps."""
    out, r = [], 0
    bounds = list(seps) + [nblocks]
    for i in range(nblocks):
        while i >= bounds[r]:
            r += 1
        out.append(r)
    return out


@dataclass
class Message:
    kind: str   # "JNQ" (parent fluxes to the child) or "JNZ" (child means to the parent)
    src: int    # sending rank
    dst: int    # receiving rank
    child: int  # block index of the child the message concerns
    count: int  # values per step


@dataclass
class Plan:
    ranks: int
    owner: list
    times: list
    messages: list = field(default_factory=list)

    def sends(self, rank):
        return [m for m in self.messages if m.src == rank]

    def receives(self, rank):
        return [m for m in self.messages if m.dst == rank]


def exchange_plan(blocks, owner, full_feedback=False):
    """The cross-rank messages of one step for a block-to-rank map `owner`."""
    msgs = []
    for k, b in enumerate(blocks):
        p = b["parent"]
        if p < 0 or owner[p] == owner[k]:
            continue
        a, bb = b["nx"] // 3, b["ny"] // 3
        msgs.append(Message("JNQ", owner[p], owner[k], k, 2 * a + 2 * bb))
        ring = a * bb if full_feedback else (a * bb - max(a - 2, 0) * max(bb - 2, 0))
        msgs.append(Message("JNZ", owner[k], owner[p], k, ring))
    return msgs


def partition(blocks, ranks, alpha=ALPHA_US, beta=BETA_US, iters=20000, seed=0,
              full_feedback=False):
    """Block-to-rank map of a hierarchy (list of block dicts, parents first) over `ranks`
    GPUs by Alg. 1, with its predicted rank times and its exchange plan."""
    costs = [block_cost(b["nx"] * b["ny"], alpha, beta) for b in blocks]
    seps, times = hill_climb(costs, ranks, iters=iters, seed=seed)
    owner = assignment(len(blocks), seps)
    return Plan(ranks, owner, times, exchange_plan(blocks, owner, full_feedback))
