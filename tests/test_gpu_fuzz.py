"""Seeded random configurations of the stencil launches (shapes, chunkings,
halos, superblocks, blocks, HBM budgets small enough to spill), each checked
bit for bit against the oracle: edge cases no hand-written case names."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu
ANN2 = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"
ANN3 = "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _dist(rng, shape):
    nd = len(shape)
    kind = rng.integers(0, 4)
    halo = int(rng.integers(0, 2))
    if kind == 0:
        return lt.Dist.block()
    if kind == 1:
        return lt.Dist.rows(int(rng.integers(1, shape[0] + 1)), halo=halo)
    tile = tuple(int(rng.integers(1, s + 1)) for s in shape)
    return lt.Dist.tiles(tile, halo=(halo,) * nd)


@pytest.mark.parametrize("case", range(24))
def test_jacobi2d_random_configurations(case):
    rng = np.random.default_rng(9000 + case)
    ny, nx = int(rng.integers(1, 700)), int(rng.integers(1, 900))
    iters = int(rng.integers(1, 4))
    u0 = si.uniform_field(2203, 300 + case, ny, nx)
    bx = int(rng.choice([1, 4, 32, 64, 128]))
    by = int(rng.choice([1, 2, 4, 8]))
    sb = (int(rng.integers(1, nx + 1)), int(rng.integers(1, ny + 1))) if rng.random() < 0.8 else (0, 0)
    dist = _dist(rng, (ny, nx))
    spill = rng.random() < 0.3
    cells = (ny + 2) * (nx + 64) * 4
    kw = dict(hbm_budget=max(cells, 1 << 20) * 2, host_pool=cells * 8 + (8 << 20)) if spill else {}
    with lt.Context(**kw) as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN2, [("U", lt.F32), ("V", lt.F32)])
        try:
            for _ in range(iters):
                k.launch(grid=(nx, ny), block=(bx, by), superblock=sb, args=[U, V])
                U, V = V, U
            if rng.random() < 0.5:
                V.discard()
            ctx.synchronize()
        except lt.LightningError as e:
            # a budget below one superblock's footprint is reported, not run
            assert spill and e.code == L.LT_ERR_OOM_DEVICE, e
            return
        got = U.read()
    want = oracle.jacobi2d(u0, iters)
    assert np.array_equal(got, want), (ny, nx, sb, f"{np.sum(got != want)} cells differ")


@pytest.mark.parametrize("case", range(12))
def test_jacobi3d_random_configurations(case):
    rng = np.random.default_rng(9500 + case)
    shape = (int(rng.integers(1, 40)), int(rng.integers(1, 70)), int(rng.integers(1, 300)))
    iters = int(rng.integers(1, 3))
    idx = np.arange(int(np.prod(shape)), dtype=np.uint64)
    u0 = si.gen_uniform_f32(2203, 400 + case, idx).reshape(shape)
    sb = tuple(int(rng.integers(1, s + 1)) for s in shape[::-1]) if rng.random() < 0.8 else (0, 0, 0)
    bx = int(rng.choice([1, 4, 32, 128]))
    with lt.Context() as ctx:
        dist = _dist(rng, shape)
        U = ctx.array(lt.F32, shape, dist)
        V = ctx.array(lt.F32, shape, dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN3, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=shape[::-1], block=(bx, 2, 1), superblock=sb, args=[U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    want = oracle.jacobi3d(u0, iters)
    assert np.array_equal(got, want), (shape, sb, f"{np.sum(got != want)} cells differ")


def _source_case(case):
    """A random source-kernel launch configuration.  Half of the cases align
    the superblocks with the chunks (chunks a whole number of blocks), so that
    writes go straight into chunks with halo replicas to update; the others
    take random superblocks (reads packed, writes through temporaries)."""
    rng = np.random.default_rng(9500 + case)
    ny, nx = int(rng.integers(1, 600)), int(rng.integers(1, 800))
    iters = int(rng.integers(1, 4))
    bx = int(rng.choice([1, 16, 32, 64]))
    by = int(rng.choice([1, 2, 4, 8]))
    if rng.random() < 0.5:
        cy = by * int(rng.integers(1, max(2, ny // by + 1)))
        cx = bx * int(rng.integers(1, max(2, nx // bx + 1)))
        halo = int(rng.integers(0, 2)) if rng.random() < 0.3 else 1
        if rng.random() < 0.5:
            dist, sb = lt.Dist.rows(cy, halo=halo), (nx, cy)
        else:
            dist, sb = lt.Dist.tiles((cy, cx), halo=(halo, halo)), (cx, cy)
    else:
        sb = (int(rng.integers(1, nx + 1)), int(rng.integers(1, ny + 1))) if rng.random() < 0.8 else (0, 0)
        dist = _dist(rng, (ny, nx))
    flags = L.LT_FLAG_NO_FUSED_REPLICAS if rng.random() < 0.3 else 0
    spill = rng.random() < 0.25
    return ny, nx, iters, (bx, by), sb, dist, flags, spill


@pytest.mark.parametrize("case", range(20))
def test_source_kernel_random_configurations(case):
    # the one-cell-per-thread source kernel (runtime-compiled) under random
    # shapes, chunkings, superblocks and blocks: replicas updated inside the
    # launch or by a copy kernel, reads packed across chunks, sometimes
    # spilling; inputs and results through the asynchronous host copies
    import bench
    ny, nx, iters, block, sb, dist, flags, spill = _source_case(case)
    u0 = si.uniform_field(2203, 500 + case, ny, nx)
    cells = (ny + 2) * (nx + 64) * 4
    kw = dict(hbm_budget=max(cells, 1 << 20) * 2, host_pool=cells * 8 + (8 << 20)) if spill else {}
    h = np.ascontiguousarray(u0)
    with lt.Context(flags=flags, **kw) as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write_async(h)
        k = ctx.kernel_from_source(bench.USER_JACOBI, "jacobi", ANN2, [("ny", lt.U32, False), ("nx", lt.U32, False),
                                                                        ("U", lt.F32), ("V", lt.F32)])
        try:
            for _ in range(iters):
                k.launch(grid=(nx, ny), block=block, superblock=sb, args=[ny, nx, U, V])
                U, V = V, U
            out = np.empty((ny, nx), np.float32)
            U.read_async(out)
            ctx.synchronize()
        except lt.LightningError as e:
            assert spill and e.code == L.LT_ERR_OOM_DEVICE, e
            return
    want = oracle.jacobi2d(u0, iters)
    assert np.array_equal(out, want), (ny, nx, sb, block, f"{np.sum(out != want)} cells differ")
