"""GPU parity of the stencil path through the C ABI against the CPU oracle.

Bar: bit-exact (same per-cell f32 operation order) for chunked and unchunked
runs, every distribution, the spill path, and the full 4096^2 x 10 config.
"""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu

ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def variants(ctx):
    """Kernel variants the Execute tasks logged since logging was enabled:
    1 register strips, 0 scalar."""
    return {t["variant"] for t in ctx.log() if t["kind"] == "execute"}


def run_jacobi(ctx, u0, dist, iters, block=(128, 4), superblock=(0, 0), fill_seed=None):
    ny, nx = u0.shape
    U = ctx.array(lt.F32, (ny, nx), dist)
    V = ctx.array(lt.F32, (ny, nx), dist)
    if fill_seed is None:
        U.write(u0)
    else:
        U.fill(L.LT_INIT_UNIFORM, seed=fill_seed, stream=0)
    k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
    for _ in range(iters):
        k.launch(grid=(nx, ny), block=block, superblock=superblock, args=[U, V])
        U, V = V, U
    ctx.synchronize()
    out = U.read()
    U.destroy()
    V.destroy()
    return out


def test_fill_generators_match_input_module():
    with lt.Context() as ctx:
        n = 1 << 20
        a = ctx.array(lt.F32, (n,), lt.Dist.rows(300_000, halo=3))
        a.fill(L.LT_INIT_UNIFORM, seed=2204, stream=0)
        assert np.array_equal(a.read(), si.gen_uniform_f32(2204, 0, np.arange(n)))
        a.fill(L.LT_INIT_KAPPA, seed=2207, stream=1)
        assert np.array_equal(a.read(), si.gen_kappa_f32(2207, 1, np.arange(n)))
        b = ctx.array(lt.U8, (1000, 1000), lt.Dist.tiles((333, 500)))
        b.fill(L.LT_INIT_U8, seed=2206, stream=10003)
        assert np.array_equal(b.read().ravel(), si.gen_u8(2206, 10003, np.arange(10**6)))
        c = ctx.array(lt.BF16, (512, 768), lt.Dist.cols(256))
        c.fill(L.LT_INIT_NORMAL_BF16, seed=2205, stream=1, scale=1 / 256)
        want = si.gen_normal_bf16_bits(2205, 1, np.arange(512 * 768), 1 / 256).reshape(512, 768)
        # fp64 log/cos of two libraries may differ in the last ulp; a bf16
        # rounding decision flips only if that ulp straddles a tie
        assert np.mean(c.read() != want) < 1e-5


def test_paper_host_example_1d_stencil():
    # host code of Sec. 3.6: n = 1e6 ones, StencilDist(64000, 1), BlockDist(64000), 10 launches
    n = 1_000_000
    x = np.ones(n, np.float32)
    want = x
    for _ in range(10):
        want = oracle.stencil1d_paper(want)
    with lt.Context() as ctx:
        dist = lt.Dist.rows(64_000, halo=1)
        inp = ctx.array(lt.F32, (n,), dist)
        out = ctx.array(lt.F32, (n,), dist)
        inp.fill(L.LT_INIT_CONST, value=1.0)
        k = ctx.kernel(lt.STENCIL1D, "global i => read input[i-1:i+1], write output[i]",
                       [("output", lt.F32), ("input", lt.F32)])
        for _ in range(10):
            k.launch(grid=(n,), block=(16,), superblock=(64_000,), args=[out, inp])
            inp, out = out, inp
        ctx.synchronize()
        got = inp.read()
    assert np.array_equal(got, want)


DISTS = {
    "block": lt.Dist.block(),
    "rows_halo": lt.Dist.rows(64, halo=1),
    "cols_halo": lt.Dist.cols(96, halo=1),
    "tiles_halo": lt.Dist.tiles((64, 128), halo=(1, 1)),
    "tiles_nohalo": lt.Dist.tiles((64, 128)),     # reads span chunks: pack path
    "rows_nohalo": lt.Dist.rows(50),              # ragged bands, pack path
    "tiles_wide_halo": lt.Dist.tiles((100, 100), halo=(3, 2)),
}


@pytest.mark.parametrize("name", sorted(DISTS))
@pytest.mark.parametrize("sbshape", [(0, 0), (128, 64), (96, 32)])
def test_jacobi_all_distributions_bit_exact(name, sbshape):
    ny, nx, iters = 301, 517, 4           # several tiles and ragged tails
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 0, ny, nx)
    want = oracle.jacobi2d(u0, iters)
    block = (32, 4) if sbshape == (96, 32) else (128, 4)
    with lt.Context() as ctx:
        ctx.log_enable()
        got = run_jacobi(ctx, u0, DISTS[name], iters, block=block, superblock=sbshape)
        ran = variants(ctx)
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"
    assert ran == {1}  # every superblock starts on a multiple of 4 columns


def test_jacobi_degenerate_shapes():
    with lt.Context() as ctx:
        ctx.log_enable()
        for (ny, nx) in [(1, 1), (1, 7), (9, 1), (2, 3), (5, 129)]:
            u0 = si.uniform_field(2203, 5, ny, nx)
            for dist in (lt.Dist.block(), lt.Dist.tiles((2, 2), halo=(1, 1)), lt.Dist.tiles((1, 2))):
                got = run_jacobi(ctx, u0, dist, 3, block=(1, 1), superblock=(2, 2))
                assert np.array_equal(got, oracle.jacobi2d(u0, 3)), (ny, nx)
        # superblocks two columns wide: single-superblock launches take the
        # strip kernel, the others the scalar one
        assert variants(ctx) == {0, 1}


@pytest.mark.parametrize("block", [(64, 4), (1, 4)])
def test_jacobi_write_through_replicas_many_chunks(block):
    # 8 x 16 = 128 chunks with 1-cell halos: every launch writes ~900
    # replica boxes (edges and corners) from the replica CTAs appended to the
    # strip kernel's grid (block (64, 4)) or the scalar kernel's ((1, 4): odd
    # superblock columns)
    ny, nx = 256, 1024
    u0 = si.uniform_field(2203, 13, ny, nx)
    sb = (64, 32) if block[0] == 64 else (63, 32)
    with lt.Context() as ctx:
        ctx.log_enable()
        got = run_jacobi(ctx, u0, lt.Dist.tiles((32, 64), halo=(1, 1)), 3, block=block, superblock=sb)
        ran = variants(ctx)
        st = ctx.stats()
        unpacks = [t for t in ctx.log() if t["kind"] == "unpack"]
    assert np.array_equal(got, oracle.jacobi2d(u0, 3))
    assert ran == ({1} if block[0] == 64 else {0})
    assert st["bytes_replica_wt"] > 0
    if block[0] == 64:
        assert not unpacks  # superblocks equal the chunks: every write is direct


def test_jacobi_grid_larger_than_array_and_superblock_order():
    ny, nx = 130, 260
    u0 = si.uniform_field(2203, 9, ny, nx)
    want = oracle.jacobi2d(u0, 2)
    with lt.Context(flags=L.LT_FLAG_FIXED_SWEEP) as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(32, halo=1))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(32, halo=1))
        U.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        k.launch(grid=(512, 256), block=(128, 4), superblock=(512, 32), args=[U, V])
        k.launch(grid=(512, 256), block=(128, 4), superblock=(512, 32), args=[V, U])
        ctx.synchronize()
        assert np.array_equal(U.read(), want)


def test_spill_through_host_memory_bit_exact():
    # 16 bands of 64 x 2048 f32; HBM budget of 6 bands: every launch streams
    ny, nx, band, iters = 1024, 2048, 64, 5
    cb = (band + 2) * nx * 4
    u0 = si.uniform_field(si.SEED_JACOBI_OOC, 0, ny, nx)
    want = oracle.jacobi2d(u0, iters)
    # 2 arrays x 16 bands = 32 chunks: 6 in HBM, the rest (and slack) in host memory
    with lt.Context(hbm_budget=6 * cb + (1 << 20), host_pool=30 * cb) as ctx:
        got = run_jacobi(ctx, u0, lt.Dist.rows(band, halo=1), iters, superblock=(nx, band),
                         fill_seed=si.SEED_JACOBI_OOC)
        s = ctx.stats()
    assert s["evictions"] > 0 and s["fetches"] > 0 and s["dead_skips"] > 0
    assert np.array_equal(got, want)


def test_full_size_incore_1_chunk_and_4x4_tiles():
    n, iters = 4096, 10
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 0, n, n)
    want = oracle.jacobi2d(u0, iters)
    with lt.Context() as ctx:
        one = run_jacobi(ctx, u0, lt.Dist.block(), iters, superblock=(0, 0), fill_seed=si.SEED_JACOBI_INCORE)
        tiled = run_jacobi(ctx, u0, lt.Dist.tiles((1024, 1024), halo=(1, 1)), iters, superblock=(1024, 1024),
                           fill_seed=si.SEED_JACOBI_INCORE)
        s = ctx.stats()
    assert np.array_equal(one, tiled)
    assert np.array_equal(one, want)
    # the repeated launches planned once per shape and reused their device tables
    assert s["plans_reused"] >= 2 * iters - 4
    assert s["tables_resident"] > 0


def test_out_of_core_lightcone_samples_small():
    # the out-of-core launch shape (row bands + 1-row halo, budget < data) on a
    # grid the oracle checks cell by cell through its light cone
    NY, NX, band, iters = 4096, 4096, 512, 20
    cb = (band + 2) * NX * 4
    with lt.Context(hbm_budget=5 * cb, host_pool=14 * cb) as ctx:
        U = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        V = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=si.SEED_JACOBI_OOC, stream=0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(NX, NY), block=(128, 4), superblock=(NX, band), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    si_, sj_ = si.sample_cells(2204, NY, NX, 512, seams_every=band)
    want = oracle.jacobi2d_lightcone(NY, NX, si.SEED_JACOBI_OOC, 0, iters, si_, sj_)
    assert np.array_equal(got[si_, sj_], want)


def test_out_of_core_16384x8192_every_cell_vs_unchunked_oracle():
    # the out-of-core launch shape at a size the oracle runs unchunked in a
    # few seconds: 16384 x 8192 f32 in 1000-row bands + 1-row halo (17 bands,
    # the last one 384 rows), an HBM budget of 5 bands for two 512 MiB
    # arrays, 20 iterations; every cell compared
    NY, NX, band, iters = 16384, 8192, 1000, 20
    cb = (band + 2) * NX * 4
    u0 = si.uniform_field(si.SEED_JACOBI_OOC, 0, NY, NX)
    with lt.Context(hbm_budget=5 * cb + (1 << 20), host_pool=40 * cb) as ctx:
        U = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        V = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        U.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(NX, NY), block=(128, 4), superblock=(NX, band), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        s = ctx.stats()
        got = U.read()
    assert s["evictions"] > 0 and s["fetches"] > 0
    want = oracle.jacobi2d(u0, iters)
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


def test_discard_of_the_stale_buffer_keeps_results_exact():
    # out of core (budget 5 bands of 16 + 16): runs of 3 iterations, each
    # ending with the stale ping-pong buffer discarded before the synchronize;
    # the result stays bit-exact and the closing write-back shrinks
    ny, nx, band = 2048, 2048, 128
    cb = (band + 2) * nx * 4
    u0 = si.uniform_field(si.SEED_JACOBI_OOC, 3, ny, nx)
    d2h = []
    for discard in (False, True):
        with lt.Context(hbm_budget=5 * cb + (1 << 20), host_pool=40 * cb) as ctx:
            U = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(band, halo=1))
            V = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(band, halo=1))
            U.write(u0)
            k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
            ctx.synchronize()
            ctx.reset_stats()
            for run in range(2):
                for _ in range(3):
                    k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
                    U, V = V, U
                if discard:
                    V.discard()
                ctx.synchronize()
                assert np.array_equal(U.read(), oracle.jacobi2d(u0, 3 * (run + 1))), (discard, run)
            d2h.append(ctx.stats()["bytes_d2h"])
    assert d2h[1] < d2h[0]


def test_out_of_core_full_size_lightcone_samples():
    # the out-of-core configuration at full size, as bench.py runs it: 262144 x
    # 131072 f32 (128 GiB per buffer), 8192-row bands + 1-row halo, the HBM
    # budget and pinned host pool bench.py sizes, one run of 20 iterations;
    # 4096 cells (edges and band seams included) against the oracle's light cone
    import types

    import bench
    NY, NX, band, iters = 262144, 131072, 8192, 20
    pl = bench.plan_ooc(types.SimpleNamespace(rows=NY, cols=NX, band=band, tb=1, hbm_gib=0.0), 1)
    si_, sj_ = si.sample_cells(2204, NY, NX, 4096, seams_every=band)
    with lt.Context(hbm_budget=pl["budget"], host_pool=pl["host"]) as ctx:
        U = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        V = ctx.array(lt.F32, (NY, NX), lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=si.SEED_JACOBI_OOC, stream=0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(NX, NY), block=(128, 4), superblock=(NX, band), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        s = ctx.stats()
        got = np.array([U.read_box((i, j), (i, j))[0, 0] for i, j in zip(si_, sj_)], np.float32)
    assert s["evictions"] > 0  # the run does not fit: the synchronize writes back what does not
    want = oracle.jacobi2d_lightcone(NY, NX, si.SEED_JACOBI_OOC, 0, iters, si_, sj_)
    assert np.array_equal(got, want), f"{np.sum(got != want)} of {len(want)} sampled cells differ"


MANN = "global [i, j] => read U[i-{k}:i+{k}, j-{k}:j+{k}], write V[i, j]"


@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("dist_name", ["block", "rows_halo_k", "tiles_halo_k", "rows_halo_1_pack"])
def test_multi_step_jacobi_bit_exact(k, dist_name):
    ny, nx, launches = 301, 517, 3
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 7, ny, nx)
    want = oracle.jacobi2d(u0, k * launches)
    dist, sb = {"block": (lt.Dist.block(), (0, 0)),
                "rows_halo_k": (lt.Dist.rows(64, halo=k), (nx, 64)),
                "tiles_halo_k": (lt.Dist.tiles((64, 128), halo=(k, k)), (128, 64)),
                "rows_halo_1_pack": (lt.Dist.rows(64, halo=1), (nx, 64))}[dist_name]
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        km = ctx.kernel(lt.JACOBI2D_MULTI, MANN.format(k=k), [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        for _ in range(launches):
            km.launch(grid=(nx, ny), block=(128, 4), superblock=sb, args=[U, V, k])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


@pytest.mark.parametrize("k", [3, 10, 16])
@pytest.mark.parametrize("dist_name", ["block", "rows_halo_k"])
def test_multi_step_tall_grid_bit_exact(k, dist_name):
    # more rows than one warp segment (512) and columns that end mid-window
    ny, nx, launches = 1500, 700, 3
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 8, ny, nx)
    want = oracle.jacobi2d(u0, k * launches)
    dist, sb = {"block": (lt.Dist.block(), (0, 0)),
                "rows_halo_k": (lt.Dist.rows(400, halo=k), (nx, 400))}[dist_name]
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        km = ctx.kernel(lt.JACOBI2D_MULTI, MANN.format(k=k), [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        for _ in range(launches):
            km.launch(grid=(nx, ny), block=(128, 4), superblock=sb, args=[U, V, k])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


def test_multi_step_unaligned_superblocks_bit_exact():
    # superblocks that start at columns not divisible by 4 take the shared-memory variant
    ny, nx, k, launches = 200, 390, 3, 2
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 9, ny, nx)
    want = oracle.jacobi2d(u0, k * launches)
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.block())
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.block())
        U.write(u0)
        km = ctx.kernel(lt.JACOBI2D_MULTI, MANN.format(k=k), [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        for _ in range(launches):
            km.launch(grid=(nx, ny), block=(2, 2), superblock=(130, 66), args=[U, V, k])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


def test_multi_step_out_of_core_spill_bit_exact():
    ny, nx, band, k, launches = 1024, 2048, 64, 4, 3
    cb = (band + 2 * k) * nx * 4
    u0 = si.uniform_field(si.SEED_JACOBI_OOC, 0, ny, nx)
    want = oracle.jacobi2d(u0, k * launches)
    # 16 bands per array, 10 chunk slots: less than one array, so every launch streams
    with lt.Context(hbm_budget=10 * cb + (64 << 10), host_pool=30 * cb) as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(band, halo=k))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(band, halo=k))
        U.fill(L.LT_INIT_UNIFORM, seed=si.SEED_JACOBI_OOC, stream=0)
        km = ctx.kernel(lt.JACOBI2D_MULTI, MANN.format(k=k), [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        for _ in range(launches):
            km.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V, k])
            U, V = V, U
        ctx.synchronize()
        s = ctx.stats()
        got = U.read()
    assert s["evictions"] > 0 and s["fetches"] > 0
    assert np.array_equal(got, want)


@pytest.mark.parametrize("flags", [0, L.LT_FLAG_NO_PDL])
def test_dependent_launches_and_deferred_fences_stay_exact(flags):
    # In-place launches run as programmatic dependents with their fence
    # events deferred.  A fill that needs the memory then evicts the results
    # (the eviction on the copy stream must wait for the deferred kernels),
    # and the next launches fetch them back.
    ny, nx, iters = 1536, 2048, 9
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 5, ny, nx)
    want = oracle.jacobi2d(u0, 2 * iters)
    dist = lt.Dist.tiles((512, 512), halo=(1, 1))
    field = 4 * ny * nx
    with lt.Context(hbm_budget=int(2.6 * field), host_pool=4 * field, flags=flags) as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        W = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(512, 512), args=[U, V])
            U, V = V, U
        W.fill(L.LT_INIT_UNIFORM, seed=9, stream=0)   # evicts chunks written by the launches above
        for _ in range(iters):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(512, 512), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        assert ctx.stats()["evictions"] > 0
        assert np.array_equal(U.read(), want)


@pytest.mark.parametrize("flags", [0, L.LT_FLAG_NO_STAGED])
@pytest.mark.parametrize("shape,dist,sb", [
    ((301, 517), lt.Dist.tiles((64, 128)), (0, 0)),          # odd row pitch: unaligned heads and tails
    ((301, 517), lt.Dist.tiles((64, 128)), (96, 160)),       # superblocks across chunks: packs and write-backs
    ((200, 4100), lt.Dist.tiles((40, 3000)), (0, 0)),        # rows of 12 KB: several rows per stage
    ((130, 1024), lt.Dist.rows(50), (0, 0)),                 # aligned rows, ragged bands
    ((257, 600), lt.Dist.cols(200), (0, 0)),                 # one-column packs (narrow pieces)
])
def test_pack_through_shared_memory_and_registers_bit_exact(flags, shape, dist, sb):
    # Packs and write-backs of whole aligned rows move through shared memory
    # with bulk asynchronous copies; LT_FLAG_NO_STAGED keeps them on the
    # register path.  Both are exact copies.
    ny, nx = shape
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 7, ny, nx)
    want = oracle.jacobi2d(u0, 3)
    with lt.Context(flags=flags) as ctx:
        ctx.log_enable()
        got = run_jacobi(ctx, u0, dist, 3, block=(32, 4), superblock=sb)
        kinds = {t["kind"] for t in ctx.log()}
    assert "pack" in kinds
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


@pytest.mark.parametrize("dist", [lt.Dist.rows(100, halo=1), lt.Dist.tiles((128, 256), halo=(1, 1)),
                                  lt.Dist.rows(100)])
def test_async_host_copies_round_trip_through_one_buffer(dist):
    # the end-to-end loop with asynchronous copies: upload from a pinned
    # buffer, three launches, read the result back into the same buffer,
    # upload it again, three more launches; the copies of one step overlap
    # those of the next only where their host rows do not
    import torch
    ny, nx = 700, 1100
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 9, ny, nx)
    h = torch.empty((ny, nx), dtype=torch.float32, pin_memory=True).numpy()
    h[...] = u0
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(2):
            U.write_async(h)
            for _ in range(3):
                k.launch(grid=(nx, ny), block=(128, 4), superblock=(0, 0), args=[U, V])
                U, V = V, U
            U.read_async(h)
        ctx.synchronize()
    assert np.array_equal(h, oracle.jacobi2d(u0, 6))


def _with_special_values(u, seed):
    # about one cell in eight replaced by a value the fast division path
    # must hand to the IEEE division (zeros of both signs, subnormals, sums
    # that cancel below 1e-30, huge values whose sums overflow, infinities,
    # NaN) or that sits at the edge of its range
    rng = np.random.default_rng(seed)
    special = np.array([0.0, -0.0, 1e-40, -1e-42, 1e-35, -1e-35, 3e38, -3e38, np.inf, -np.inf, np.nan,
                        1e30, -1e30, 5e-30, 1e-30, 2.5e29], dtype=np.float32)
    u = u.copy()
    mask = rng.random(u.shape) < 0.125
    u[mask] = rng.choice(special, size=int(mask.sum()))
    return u


def _same(got, want):
    # bit for bit, any two NaNs equal (their payloads are not specified)
    return (got.view(np.uint32) == want.view(np.uint32)) | (np.isnan(got) & np.isnan(want))


@pytest.mark.parametrize("kind", ["strips_tiles_halo", "strips_block", "multi_step_rows_halo"])
def test_jacobi_special_values_match_the_oracle(kind):
    # the strips divide four sums with one range test and fall back to the
    # IEEE division for all four when one is out of range; the multi-step
    # kernel does the same: both must match the oracle's float division
    ny, nx = 203, 390
    u0 = _with_special_values(si.uniform_field(si.SEED_JACOBI_INCORE, 40, ny, nx), 40)
    with np.errstate(all="ignore"):
        if kind == "multi_step_rows_halo":
            k, launches = 3, 2
            want = oracle.jacobi2d(u0, k * launches)
        else:
            launches = 3
            want = oracle.jacobi2d(u0, launches)
    with lt.Context() as ctx:
        if kind == "multi_step_rows_halo":
            dist, sb = lt.Dist.rows(64, halo=k), (nx, 64)
        elif kind == "strips_tiles_halo":
            dist, sb = lt.Dist.tiles((64, 128), halo=(1, 1)), (128, 64)
        else:
            dist, sb = lt.Dist.block(), (0, 0)
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        if kind == "multi_step_rows_halo":
            kern = ctx.kernel(lt.JACOBI2D_MULTI, MANN.format(k=k), [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
            extra = [k]
        else:
            kern = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
            extra = []
        for _ in range(launches):
            kern.launch(grid=(nx, ny), block=(128, 4), superblock=sb, args=[U, V] + extra)
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    same = _same(got, want)
    assert np.isnan(want).any() and np.isinf(want).any() and (want == 0).any()
    assert same.all(), f"{int((~same).sum())} cells differ, e.g. got {got[~same][:4]} want {want[~same][:4]}"
