"""K-Means built-ins (the K-Means benchmark of Sec. 4): assignment with a
reduce(+) of per-centre fp64 sums and counts, and the centre update, checked
bit for bit against the oracle over several iterations.  Uniform features
are multiples of 2^-24 in [0, 1), so every fp64 sum is exact whatever the
order of its additions."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

ASSIGN = "global i => read X[4*i:4*i+3], read C[:], reduce(+) S[:]"
UPDATE = "global j => read S[5*j:5*j+4], read C[4*j:4*j+3], write C2[4*j:4*j+3]"
SEED = 2209


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def kernels(ctx):
    ka = ctx.kernel(lt.KMEANS_ASSIGN, ASSIGN, [("X", lt.F32), ("C", lt.F32), ("S", lt.F64), ("k", lt.U32, False)])
    ku = ctx.kernel(lt.KMEANS_UPDATE, UPDATE, [("S", lt.F64), ("C", lt.F32), ("C2", lt.F32)])
    return ka, ku


def test_kmeans_plan_maps_records_to_features():
    with lt.Context(hbm_budget=1 << 30, flags=L.LT_FLAG_DRYRUN) as ctx:
        n, k = 1000, 8
        X = ctx.array(lt.F32, (4 * n,), lt.Dist.rows(4 * 300))      # chunks of 300 whole records
        Xp = ctx.array(lt.F32, (4 * n,), lt.Dist.rows(4 * 300 + 2))  # chunks that split records
        C = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        S = ctx.array(lt.F64, (5 * k,), lt.Dist.block())
        ka, _ = kernels(ctx)
        plan = ka.explain(grid=(n,), block=(100,), superblock=(300,), args=[X, C, S, k])
        sb = plan["superblocks"][1]
        assert sb["args"][0]["region"] == {"lo": [1200], "hi": [2399]}
        assert [a["kind"] for a in sb["args"]] == ["direct", "direct", "reduce", "value"]
        plan = ka.explain(grid=(n,), block=(100,), superblock=(300,), args=[Xp, C, S, k])
        assert plan["superblocks"][1]["args"][0]["kind"] == "pack"


def run_kmeans(n, k, xdist, sb, iters, far=None):
    x = oracle.gen_uniform_f32(SEED, 0, 0, 4 * n).reshape(n, 4)
    c = x[:k].copy()
    if far is not None:
        c[far] = 100.0
    got_s, got_c, want_s, want_c = [], [], [], []
    with lt.Context() as ctx:
        X = ctx.array(lt.F32, (4 * n,), xdist)
        C = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        C2 = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        S = ctx.array(lt.F64, (5 * k,), lt.Dist.block())
        X.fill(L.LT_INIT_UNIFORM, seed=SEED, stream=0)
        C.write(c.reshape(-1))
        ka, ku = kernels(ctx)
        for _ in range(iters):
            ka.launch(grid=(n,), block=(256,), superblock=(sb,), args=[X, C, S, k])
            ku.launch(grid=(k,), block=(64,), superblock=(0,), args=[S, C, C2])
            got_s.append(S.read().reshape(k, 5))
            got_c.append(C2.read().reshape(k, 4))
            C, C2 = C2, C
    ci = c
    for _ in range(iters):
        s, _ = oracle.kmeans_assign(x, ci)
        ci = oracle.kmeans_update(s, ci)
        want_s.append(s)
        want_c.append(ci)
    return got_s, got_c, want_s, want_c


@pytest.mark.gpu
@pytest.mark.parametrize("xdist_name", ["records", "split_records"])
def test_kmeans_iterations_bit_exact(xdist_name):
    n, k, iters = 100_003, 40, 5
    xdist = {"records": lt.Dist.rows(4 * 25_000), "split_records": lt.Dist.rows(4 * 25_000 + 2)}[xdist_name]
    got_s, got_c, want_s, want_c = run_kmeans(n, k, xdist, 30_000, iters)
    for it in range(iters):
        assert np.array_equal(got_s[it], want_s[it]), f"sums differ at iteration {it}"
        assert np.array_equal(got_c[it], want_c[it]), f"centres differ at iteration {it}"
    assert got_s[-1][:, 4].sum() == n


@pytest.mark.gpu
def test_kmeans_empty_cluster_keeps_its_centre():
    n, k = 20_000, 10
    got_s, got_c, want_s, want_c = run_kmeans(n, k, lt.Dist.rows(4 * 5000), 7000, 3, far=k - 1)
    for it in range(3):
        assert got_s[it][k - 1, 4] == 0 and np.all(got_c[it][k - 1] == 100.0)
        assert np.array_equal(got_s[it], want_s[it]) and np.array_equal(got_c[it], want_c[it])


@pytest.mark.gpu
def test_kmeans_fp64_fallback_path_bit_exact():
    # features in [1, 2) are not multiples of 2^-24 in [0, 1): they take the
    # fp64 atomics; as multiples of 2^-23 their fp64 sums are still exact
    n, k, iters = 30_011, 16, 3
    x = (oracle.gen_uniform_f32(SEED, 3, 0, 4 * n) + np.float32(1.0)).reshape(n, 4)
    c = x[:k].copy()
    with lt.Context() as ctx:
        X = ctx.array(lt.F32, (4 * n,), lt.Dist.rows(4 * 8_000))
        C = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        C2 = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        S = ctx.array(lt.F64, (5 * k,), lt.Dist.block())
        X.write(x.reshape(-1))
        C.write(c.reshape(-1))
        ka, ku = kernels(ctx)
        want_c = c
        for _ in range(iters):
            ka.launch(grid=(n,), block=(256,), superblock=(8_000,), args=[X, C, S, k])
            ku.launch(grid=(k,), block=(64,), superblock=(0,), args=[S, C, C2])
            s, _ = oracle.kmeans_assign(x, want_c)
            want_c = oracle.kmeans_update(s, want_c)
            assert np.array_equal(S.read().reshape(k, 5), s)
            assert np.array_equal(C2.read().reshape(k, 4), want_c)
            C, C2 = C2, C


def _slice_sums(part):
    """Oracle sums and counts of records [lo, hi) of the seeded records
    (runs in a spawned worker process)."""
    lo, hi, c = part
    oracle.set_threads(1)
    x = oracle.gen_uniform_f32(SEED, 0, 4 * lo, 4 * (hi - lo)).reshape(-1, 4)
    return oracle.kmeans_assign(x, c)[0]


@pytest.mark.gpu
def test_kmeans_full_size_bit_exact():
    """The launch configuration of the K-Means benchmark: 1e9 records (16 GB),
    k = 40, 25M records per chunk and superblock, the first k records as
    centres; one Lloyd iteration.  The oracle assigns slices of the records
    in worker processes and adds their fp64 sums: every sum is a multiple of
    2^-24 below 2^29, so it is exact whatever the order of the additions."""
    n, k, per = 1_000_000_000, 40, 25_000_000
    c = oracle.gen_uniform_f32(SEED, 0, 0, 4 * k).reshape(k, 4)
    with lt.Context() as ctx:
        X = ctx.array(lt.F32, (4 * n,), lt.Dist.rows(4 * per))
        C = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        C2 = ctx.array(lt.F32, (4 * k,), lt.Dist.block())
        S = ctx.array(lt.F64, (5 * k,), lt.Dist.block())
        X.fill(L.LT_INIT_UNIFORM, seed=SEED, stream=0)
        C.write(c.reshape(-1))
        ka, ku = kernels(ctx)
        ka.launch(grid=(n,), block=(64,), superblock=(per,), args=[X, C, S, k])
        ku.launch(grid=(k,), block=(64,), superblock=(0,), args=[S, C, C2])
        got_s = S.read().reshape(k, 5)
        got_c = C2.read().reshape(k, 4)
        assert ctx.stats()["bytes_d2d"] == 0  # every superblock reads its own chunk in place
    step = 15_625_000
    parts = [(lo, min(lo + step, n), c) for lo in range(0, n, step)]
    workers = max(1, min(16, len(os.sched_getaffinity(0))))
    # spawned, not forked: this process holds a CUDA context
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        want_s = np.sum(list(pool.map(_slice_sums, parts)), axis=0)
    assert want_s[:, 4].sum() == n
    assert np.array_equal(got_s, want_s)
    assert np.array_equal(got_c, oracle.kmeans_update(want_s, c))
