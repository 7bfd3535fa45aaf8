"""GPU parity of the 3-D 7-point Jacobi built-in against the CPU oracle
(bit-exact: same f32 operation order) over several distributions, including
the 3-D pack path (tiles without halo) and ragged shapes."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu
ANN = "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def field3(nz, ny, nx, stream=0):
    idx = np.arange(nz * ny * nx, dtype=np.uint64)
    return si.gen_uniform_f32(2203, 20 + stream, idx).reshape(nz, ny, nx)


# distribution, block, superblock (x, y, z; rounded up to whole blocks), and
# the kernel variant the launch takes: 2 = TMA plane ring (every superblock's
# columns start 16-byte aligned), 0 = scalar (some do not)
DISTS = {
    "block": (lt.Dist.block(), (64, 4, 1), (0, 0, 0), 2),
    "tiles_halo": (lt.Dist.tiles((16, 24, 64), halo=(1, 1, 1)), (64, 4, 1), (64, 24, 16), 2),
    "tiles_nohalo": (lt.Dist.tiles((16, 24, 64)), (64, 4, 1), (64, 24, 16), 2),
    "zbands_halo": (lt.Dist.rows(10, halo=1), (64, 4, 1), (0, 0, 10), 2),
    "odd_sb_rounded": (lt.Dist.tiles((13, 30, 70), halo=(1, 1, 1)), (64, 4, 1), (35, 15, 13), 2),
    "odd_sb": (lt.Dist.tiles((13, 30, 70), halo=(1, 1, 1)), (5, 3, 1), (35, 15, 13), 0),
}


def variants(ctx):
    return {t["variant"] for t in ctx.log() if t["kind"] == "execute"}


@pytest.mark.parametrize("name", sorted(DISTS))
def test_jacobi3d_bit_exact(name):
    # 37 x 50 x 133: ragged against the staged kernel's 16-plane units,
    # 32-row and 128-column tiles (the last column tile is 5 wide)
    nz, ny, nx, iters = 37, 50, 133, 3
    u0 = field3(nz, ny, nx)
    want = oracle.jacobi3d(u0, iters)
    dist, block, sb, variant = DISTS[name]
    with lt.Context() as ctx:
        ctx.log_enable()
        U = ctx.array(lt.F32, (nz, ny, nx), dist)
        V = ctx.array(lt.F32, (nz, ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny, nz), block=block, superblock=sb, args=[U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
        ran = variants(ctx)
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"
    assert ran == {variant}


def test_jacobi3d_many_chunks_take_the_register_kernel():
    # 512 chunks in one launch: more than the staged kernel's tensor maps, so
    # the register-strip kernel runs
    shape = (8, 64, 256)
    u0 = field3(*shape, stream=3)
    with lt.Context() as ctx:
        ctx.log_enable()
        dist = lt.Dist.tiles((1, 8, 32), halo=(1, 1, 1))
        U = ctx.array(lt.F32, shape, dist)
        V = ctx.array(lt.F32, shape, dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(2):
            k.launch(grid=shape[::-1], block=(32, 4, 1), superblock=(32, 8, 1), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi3d(u0, 2))
        assert variants(ctx) == {1}


def test_jacobi3d_units_outnumber_ctas():
    # 40 x 300 x 1000 in 8-plane slabs: 5 tasks x 8 x 10 tiles x 1 unit = 400
    # units, more than the resident CTAs, so CTAs stream several units and the
    # plane ring carries loads across unit boundaries
    shape = (40, 300, 1000)
    u0 = field3(*shape, stream=4)
    with lt.Context() as ctx:
        ctx.log_enable()
        U = ctx.array(lt.F32, shape, lt.Dist.rows(8, halo=1))
        V = ctx.array(lt.F32, shape, lt.Dist.rows(8, halo=1))
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(3):
            k.launch(grid=shape[::-1], block=(128, 4, 1), superblock=(1000, 300, 8), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi3d(u0, 3))
        assert variants(ctx) == {2}


def test_jacobi3d_full_size_lightcone_samples():
    # the configuration bench.py times: 1024^3 f32 in 128-plane z-slabs with
    # a 1-plane halo, one run of 10 iterations; 192 cells (corners, faces,
    # slab seams, unit and tile seams) against the oracle's light cone
    n, slab, iters = 1024, 128, 10
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n - 1, 0), (n - 1, 0, n - 1), (n // 2, 0, n // 2),
           (n // 2, n - 1, 5), (7, 9, n - 1), (n - 1, 300, 0)]
    for z in (slab - 1, slab, 31, 32, 3 * slab - 1, 3 * slab):
        for y, x in ((31, 127), (32, 128), (500, 511), (0, 640), (n - 1, 129)):
            pts.append((z, y, x))
    r = si.gen_u64(2208, 79, np.arange(3 * 154, dtype=np.uint64))
    pts += [(int(r[3 * m] % np.uint64(n)), int(r[3 * m + 1] % np.uint64(n)), int(r[3 * m + 2] % np.uint64(n)))
            for m in range(192 - len(pts))]
    sk, si_, sj = (np.array(c, np.int64) for c in zip(*pts))
    with lt.Context() as ctx:
        ctx.log_enable()
        U = ctx.array(lt.F32, (n, n, n), lt.Dist.rows(slab, halo=1))
        V = ctx.array(lt.F32, (n, n, n), lt.Dist.rows(slab, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=2208, stream=0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(n, n, n), block=(128, 4, 1), superblock=(n, n, slab), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        assert variants(ctx) == {2}
        got = np.array([U.read_box((a, b, c), (a, b, c))[0, 0, 0] for a, b, c in pts], np.float32)
    want = oracle.jacobi3d_lightcone((n, n, n), 2208, 0, iters, sk, si_, sj)
    assert np.array_equal(got, want), f"{np.sum(got != want)} of {len(want)} sampled cells differ"


def test_jacobi3d_degenerate_and_larger():
    with lt.Context() as ctx:
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for shape in [(1, 1, 1), (1, 3, 5), (70, 1, 9), (5, 6, 1)]:
            u0 = field3(*shape, stream=1)
            U = ctx.array(lt.F32, shape, lt.Dist.tiles((2, 2, 2), halo=(1, 1, 1)))
            V = ctx.array(lt.F32, shape, lt.Dist.tiles((2, 2, 2), halo=(1, 1, 1)))
            U.write(u0)
            k.launch(grid=shape[::-1], block=(1, 1, 1), superblock=(2, 2, 2), args=[U, V])
            ctx.synchronize()
            assert np.array_equal(V.read(), oracle.jacobi3d(u0, 1)), shape
        u0 = field3(128, 256, 256, stream=2)
        U = ctx.array(lt.F32, u0.shape, lt.Dist.rows(32, halo=1))
        V = ctx.array(lt.F32, u0.shape, lt.Dist.rows(32, halo=1))
        U.write(u0)
        for _ in range(2):
            k.launch(grid=(256, 256, 128), block=(128, 2, 1), superblock=(256, 256, 32), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi3d(u0, 2))


@pytest.mark.parametrize("name", ["tiles_halo", "odd_sb", "many_chunks"])
def test_jacobi3d_special_values_match_the_oracle(name):
    # one cell in eight a zero of either sign, a subnormal, a value whose
    # sums overflow or cancel below 1e-30, an infinity or NaN: the division
    # by 7 must fall back to the IEEE division exactly where the oracle's
    # float division differs from the fast path (any two NaNs count as equal)
    nz, ny, nx, iters = 21, 40, 133, 2
    rng = np.random.default_rng(41)
    special = np.array([0.0, -0.0, 1e-40, -1e-42, 1e-35, 3e38, -3e38, np.inf, -np.inf, np.nan, 1e30, 5e-30],
                       dtype=np.float32)
    u0 = field3(nz, ny, nx, stream=5)
    mask = rng.random(u0.shape) < 0.125
    u0[mask] = rng.choice(special, size=int(mask.sum()))
    with np.errstate(all="ignore"):
        want = oracle.jacobi3d(u0, iters)
    if name == "many_chunks":
        dist, block, sb = lt.Dist.tiles((1, 8, 32), halo=(1, 1, 1)), (32, 4, 1), (32, 8, 1)
    else:
        dist, block, sb, _ = DISTS[name]
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (nz, ny, nx), dist)
        V = ctx.array(lt.F32, (nz, ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny, nz), block=block, superblock=sb, args=[U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    same = (got.view(np.uint32) == want.view(np.uint32)) | (np.isnan(got) & np.isnan(want))
    assert np.isnan(want).any() and np.isinf(want).any()
    assert same.all(), f"{int((~same).sum())} cells differ"
