"""A nested hierarchy split over two CPU ranks (gloo) by the block partitioner, stepped by
the oracle's phases with exactly the messages of the exchange plan between the ranks,
ends bitwise where the same hierarchy stepped on one rank ends (Sec. IV-B/IV-C: the
child's 3x3 means go to the parent's rank after the mass step, the parent's new fluxes on
the footprint edge go to the child's rank after the momentum step; Alg. 1 places the
blocks). Every cross-rank value travels through torch.distributed send/recv; a rank holds
a state of the whole hierarchy but steps only its own blocks, so a missing or misrouted
message changes the result.

Host logic only: the split numerics are the oracle's (the CUDA library runs one hierarchy
on one GPU)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2408_07609_gb300 import partition as P  # noqa: E402
from paper_2408_07609_gb300 import scenarios as S  # noqa: E402

STEPS = 40


def nest():
    """3 levels (root 200 x 120 at 810 m, a 216 x 135 child, a 135 x 90 grandchild), a
    Gaussian source over the child: both links carry non-zero means and fluxes."""
    return S.coastal_hierarchy(
        "3-level nest, wide child", 9, (200, 120, 810.0), [(1, 216, 135), (1, 135, 90)],
        dt=0.5, steps=STEPS, shelf_w=15e3, slope_w=20e3, wiggle=2e3, coast_frac=0.6,
        land_frac=0.4, source=dict(kind="gauss", sigma=8e3, peak=2.0))


def cases(blocks):
    alg1 = P.partition(blocks, 2, iters=2000, seed=1).owner
    # (owner map, full feedback, constant edge flux); [0, 1, 0] cuts both links
    return [(alg1, False, False), ([0, 1, 0], True, False), ([0, 0, 1], False, True)]


def split_run(o, blocks, owner, plan, rank, steps):
    """Step oracle state `o` on `rank`, exchanging the plan's messages; returns the largest
    |value| each message kind carried."""
    own = [k for k in range(len(blocks)) if owner[k] == rank]
    children = [k for k in range(len(blocks)) if blocks[k]["parent"] >= 0]
    carried = {"JNZ": 0.0, "JNQ": 0.0}
    for _ in range(steps):
        for k in own:
            o.phase_mass(k)
        # fine to coarse: every own child's means, to the parent's rank when remote
        packs, reqs = {}, []
        for k in children:
            if owner[k] == rank:
                packs[k] = o.pack_means(k)
        for m in plan.sends(rank):
            if m.kind == "JNZ":
                v = packs[m.child]
                assert v.size == m.count
                carried["JNZ"] = max(carried["JNZ"], float(np.nanmax(np.abs(v))))
                reqs.append(dist.isend(torch.from_numpy(v), m.dst, tag=2 * m.child))
        for m in plan.receives(rank):
            if m.kind == "JNZ":
                buf = torch.empty(m.count, dtype=torch.float64)
                dist.recv(buf, m.src, tag=2 * m.child)
                packs[m.child] = buf.numpy()
        for r in reqs:
            r.wait()
        for k in sorted(packs, reverse=True):  # the oracle's unpack order
            if owner[blocks[k]["parent"]] == rank:
                o.unpack_means(k, packs[k])
        for k in own:
            o.phase_momentum(k)
        # coarse to fine: the parent's new edge fluxes, to the child's rank when remote
        reqs = []
        for m in plan.sends(rank):
            if m.kind == "JNQ":
                v = o.edge_fluxes(m.child)
                assert v.size == m.count
                carried["JNQ"] = max(carried["JNQ"], float(np.abs(v).max()))
                reqs.append(dist.isend(torch.from_numpy(v), m.dst, tag=2 * m.child + 1))
        for m in plan.receives(rank):
            if m.kind == "JNQ":
                buf = torch.empty(m.count, dtype=torch.float64)
                dist.recv(buf, m.src, tag=2 * m.child + 1)
                o.set_edge_fluxes(m.child, buf.numpy())
        for r in reqs:
            r.wait()
        for k in children:
            if owner[k] == rank:
                o.phase_edges(k)
        for k in own:
            o.phase_swap(k)
        o.end_step()
    return carried


def same(o, ref, k):
    ok = all(np.array_equal(a, b) for a, b in zip(o.get_state(k), ref.get_state(k)))
    ok = ok and np.array_equal(o.max_height(k), ref.max_height(k), equal_nan=True)
    ok = ok and np.array_equal(o.arrival_time(k), ref.arrival_time(k))
    return ok and o.budget(k) == ref.budget(k)


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O

    sc = nest()
    res = []
    for owner, full, const in cases(sc.blocks):
        kw = dict(nest_feedback=int(full), nest_flux=int(const))
        plan = P.Plan(2, owner, [], P.exchange_plan(sc.blocks, owner, full_feedback=full))
        o = O.from_scenario(sc, **kw)
        carried = split_run(o, sc.blocks, owner, plan, rank, STEPS)
        ref = O.from_scenario(sc, **kw)
        ref.step(STEPS)
        ok = all(same(o, ref, k) for k in range(len(sc.blocks)) if owner[k] == rank)
        res.append((ok, len(plan.sends(rank)), len(plan.receives(rank)), carried))
        dist.barrier()
    out[rank] = res
    dist.destroy_process_group()


def test_split_over_two_ranks_matches_one_rank_bitwise():
    pytest.importorskip("torch.distributed")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    blocks = nest().blocks
    for i, (owner, full, const) in enumerate(cases(blocks)):
        plan = P.exchange_plan(blocks, owner, full_feedback=full)
        assert plan, "every case cuts at least one parent-child link"
        moved = {"JNZ": 0.0, "JNQ": 0.0}
        for r in range(2):
            ok, ns, nr, carried = out[r][i]
            assert ok, (owner, full, const, r)
            assert ns == sum(m.src == r for m in plan) and nr == sum(m.dst == r for m in plan)
            for kind in moved:
                moved[kind] = max(moved[kind], carried[kind])
        # the messages carried the nest's live data, not zeros (the grandchild link's
        # levels and fluxes are small this early, but not zero)
        assert moved["JNZ"] > 1e-5 and moved["JNQ"] > 1e-5, moved
