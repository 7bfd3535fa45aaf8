"""GPU parity of the 3-D 7-point Jacobi built-in against the CPU oracle
(bit-exact: same f32 operation order) over several distributions, including
the 3-D pack path (tiles without halo) and ragged shapes."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
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


DISTS = {
    "block": (lt.Dist.block(), (0, 0, 0)),
    "tiles_halo": (lt.Dist.tiles((16, 24, 64), halo=(1, 1, 1)), (64, 24, 16)),
    "tiles_nohalo": (lt.Dist.tiles((16, 24, 64)), (64, 24, 16)),
    "zbands_halo": (lt.Dist.rows(10, halo=1), (0, 0, 10)),
    "odd_sb": (lt.Dist.tiles((13, 30, 70), halo=(1, 1, 1)), (35, 15, 13)),
}


@pytest.mark.parametrize("name", sorted(DISTS))
def test_jacobi3d_bit_exact(name):
    nz, ny, nx, iters = 37, 50, 133, 3
    u0 = field3(nz, ny, nx)
    want = oracle.jacobi3d(u0, iters)
    dist, sb = DISTS[name]
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (nz, ny, nx), dist)
        V = ctx.array(lt.F32, (nz, ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI3D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny, nz), block=(64, 4, 1), superblock=sb, args=[U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


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
