"""The N>1 path of bench.py, on CPU: replicas are independent processes with
no data-path collective; they share only a barrier and the max/sum of their
timings and work (torch.distributed, gloo here).  Two ranks each plan and run
the out-of-core launch sequence in a dry-run context (planner, dependency
tracker and memory manager, no device) with the host pool bench.py gives a
rank, and combine their results the way bench.py does."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import types

    import bench
    from paper_2202_05549_gb300 import _lib as L
    from paper_2202_05549_gb300 import lightning as lt

    r, w, local = bench.env_dist()
    grp = bench.Group(w, local)
    try:
        # bench.py sizes each replica's pinned pool from its share of host memory
        args = types.SimpleNamespace(rows=4096, cols=4096, band=512, tb=1, hbm_gib=0.0)
        pl = bench.plan_ooc(args, w)
        # each replica runs its own workload: here a streaming launch sequence
        # planned and bookkept without a device
        band = 512
        cb = (band + 2) * 4096 * 4
        with lt.Context(hbm_budget=5 * cb, host_pool=14 * cb, flags=L.LT_FLAG_DRYRUN) as ctx:
            U = ctx.array(lt.F32, (4096, 4096), lt.Dist.rows(band, halo=1))
            V = ctx.array(lt.F32, (4096, 4096), lt.Dist.rows(band, halo=1))
            U.fill(L.LT_INIT_UNIFORM, seed=2204, stream=0)
            k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                           [("U", lt.F32), ("V", lt.F32)])
            for _ in range(4):
                k.launch(grid=(4096, 4096), block=(128, 4), superblock=(4096, band), args=[U, V])
                U, V = V, U
            ctx.synchronize()
            st = ctx.stats()
        grp.barrier()
        t = 1.0 + r  # this rank's "time"
        q.put({"rank": r, "world": w, "host": pl["host"], "budget": pl["budget"], "fetches": st["fetches"],
               "evictions": st["evictions"], "max_t": grp.max(t), "sum_work": grp.sum(10.0 * (r + 1))})
    finally:
        grp.close()


def test_two_replicas_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in range(world)), key=lambda d: d["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [d["world"] for d in out] == [2, 2]
    # max over ranks of the timings, sum over ranks of the work
    assert all(d["max_t"] == 2.0 and d["sum_work"] == 30.0 for d in out)
    # identical replicas: same plan, same memory traffic, same pools
    assert out[0]["host"] == out[1]["host"] and out[0]["budget"] == out[1]["budget"]
    assert out[0]["fetches"] == out[1]["fetches"] > 0
    assert out[0]["evictions"] == out[1]["evictions"] > 0
