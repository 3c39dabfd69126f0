"""The multi-rank path of bench.py on CPU: two gloo ranks (world_size 2).

bench.py runs one independent hierarchy per rank (replicas, no collective in the data
path). The only cross-rank calls are the barrier around the timed region and the
max-over-ranks of the timed durations; the whole-job rate is
world x cells x steps / (max duration). The reference arm's rank 1 exits without work.
"""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK="0",
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    r, w, _ = bench.dist_setup(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    ms = 10.0 * (rank + 1)  # rank 1 is the slower one
    worst = bench.max_over_ranks(ms, w)
    rate = bench.whole_job_rate(cells=1000, steps=5, ms=worst, world=w)
    out = io.StringIO()

    class A:
        steps, cpu_steps = 1, 1

    if rank == 1:  # the reference arm prints nothing and does no work on rank 1
        with redirect_stdout(out):
            bench.run_reference(A())
    bench.barrier(w)
    import torch.distributed as dist

    dist.destroy_process_group()
    q.put((rank, worst, rate, out.getvalue()))


def test_two_gloo_ranks_take_the_max_duration_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [20.0, 20.0]
    # 2 ranks x 1000 cells x 5 steps in 20 ms
    assert all(abs(x[2] - 2 * 1000 * 5 / 0.020 / 1e9) < 1e-15 for x in res)
    assert res[1][3] == ""
    json.dumps(res)  # plain values only
