"""Decomposition of one hierarchy over several ranks (host logic, CPU): the Alg. 1
partitioner against the equal-cells split it replaces, the exchange plan's messages, and
a two-rank gloo run that sends every planned message and checks what arrives."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2408_07609_gb300 import partition as P


def c4_blocks():
    root = dict(level=1, parent=-1, nx=2400, ny=2000)
    bl = [root]
    for lev, count, nx, ny in ((2, 3, 900, 900), (3, 6, 900, 900), (4, 12, 1200, 1200),
                               (5, 16, 1200, 900)):
        for k in range(count):
            par = [i for i, b in enumerate(bl) if b["level"] == lev - 1]
            bl.append(dict(level=lev, parent=par[k % len(par)], nx=nx, ny=ny))
    return bl


def test_separators_are_ordered_and_every_rank_has_a_block():
    costs = [P.block_cost(b["nx"] * b["ny"]) for b in c4_blocks()]
    for ranks in (1, 2, 3, 8, 16, 38):
        seps, times = P.hill_climb(costs, ranks, iters=3000, seed=ranks)
        assert len(seps) == ranks - 1 and all(a < b for a, b in zip(seps, seps[1:]))
        assert all(0 < s < len(costs) for s in seps)
        assert len(times) == ranks and abs(sum(times) - sum(costs)) < 1e-6 * sum(costs)
        owner = P.assignment(len(costs), seps)
        assert sorted(set(owner)) == list(range(ranks)) and owner == sorted(owner)
    with pytest.raises(ValueError):
        P.hill_climb(costs, len(costs) + 1)


def test_hill_climbing_beats_the_equal_cells_split():
    """With a fixed cost per block (Eq. 5's beta) the equal-cells split overloads the
    ranks that hold many small blocks; Alg. 1 balances the predicted times."""
    bl = c4_blocks()
    cells = [b["nx"] * b["ny"] for b in bl]
    for alpha, beta in ((1.09e-4, 46.2), (1e-6, 500.0)):
        costs = [P.block_cost(c, alpha, beta) for c in cells]
        base = max(P.rank_times(costs, P.equal_cells(cells, 8)))
        seps, times = P.hill_climb(costs, 8, iters=20000, seed=1)
        assert max(times) <= base
        assert max(times) <= 1.25 * sum(costs) / 8 + max(costs)
    # block costs dominated by beta: hill climbing evens out the block counts
    costs = [P.block_cost(c, 1e-9, 100.0) for c in cells]
    seps, times = P.hill_climb(costs, 8, iters=20000, seed=2)
    assert max(times) <= 5 * 100.0 + 0.1  # 38 near-equal blocks over 8 ranks: 5 at most


def test_exchange_plan_counts():
    """Root, two children, a grandchild in the second child: owners 0, 1, 0, 1."""
    bl = [dict(level=1, parent=-1, nx=90, ny=60), dict(level=2, parent=0, nx=30, ny=24),
          dict(level=2, parent=0, nx=60, ny=45), dict(level=3, parent=2, nx=18, ny=27)]
    msgs = P.exchange_plan(bl, [0, 1, 0, 1])
    got = {(m.kind, m.src, m.dst, m.child): m.count for m in msgs}
    # child 1: footprint 10 x 8 parent cells: 36 edge faces, ring 80 - 48 = 32 cells
    # child 3: footprint 6 x 9: 30 edge faces, ring 54 - 28 = 26 cells; child 2 is local
    assert got == {("JNQ", 0, 1, 1): 36, ("JNZ", 1, 0, 1): 32,
                   ("JNQ", 0, 1, 3): 30, ("JNZ", 1, 0, 3): 26}
    full = {(m.kind, m.child): m.count for m in P.exchange_plan(bl, [0, 1, 0, 1], True)}
    assert full[("JNZ", 1)] == 80 and full[("JNZ", 3)] == 54
    assert P.exchange_plan(bl, [0, 0, 0, 0]) == []


def _payload(m, step):
    return torch.arange(m.count, dtype=torch.float64) + 1000.0 * m.child + (0.5 if m.kind == "JNQ" else 0.25) + 1e6 * step


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = P.partition(c4_blocks(), world, iters=5000, seed=3)
    ok = True
    for step in range(3):  # the two exchanges of a step, in the step's order
        for kind in ("JNZ", "JNQ"):
            reqs, bufs = [], []
            for m in plan.messages:
                if m.kind != kind:
                    continue
                if m.src == rank:
                    reqs.append(dist.isend(_payload(m, step), dst=m.dst, tag=m.child))
                elif m.dst == rank:
                    b = torch.empty(m.count, dtype=torch.float64)
                    reqs.append(dist.irecv(b, src=m.src, tag=m.child))
                    bufs.append((m, b))
            for r in reqs:
                r.wait()
            for m, b in bufs:
                ok = ok and bool(torch.equal(b, _payload(m, step)))
        dist.barrier()
    out[rank] = (ok, len(plan.sends(rank)), len(plan.receives(rank)))
    dist.destroy_process_group()


def test_two_rank_exchange_over_gloo():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    plan = P.partition(c4_blocks(), 2, iters=5000, seed=3)
    assert plan.messages, "the split must cut at least one parent-child pair"
    for r in range(2):
        ok, ns, nr = out[r]
        assert ok and ns == len(plan.sends(r)) and nr == len(plan.receives(r))
