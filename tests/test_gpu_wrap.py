"""Zero-copy import of CUDA tensors (lt_array_wrap_device): launches read
and write the tensors' memory in place, bit for bit equal to the oracle."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_wrapped_tensors_in_and_out():
    ny, nx, iters = 700, 1030, 5
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 21, ny, nx)
    tu = torch.from_numpy(u0).cuda()
    tv = torch.zeros_like(tu)
    with lt.Context() as ctx:
        U, V = ctx.wrap(tu), ctx.wrap(tv)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        a, b = U, V
        for _ in range(iters):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(512, 256), args=[a, b])
            a, b = b, a
        ctx.synchronize()
        U.destroy()
        V.destroy()
    got = (tv if iters % 2 else tu).cpu().numpy()
    assert np.array_equal(got, oracle.jacobi2d(u0, iters))


def test_wrapped_input_feeds_chunked_array_with_pitch():
    # a padded tensor (row pitch > width) as input, a tiled library array with halos as output
    ny, nx, pitch = 300, 517, 640
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 22, ny, nx)
    big = torch.zeros((ny, pitch), dtype=torch.float32, device="cuda")
    big[:, :nx] = torch.from_numpy(u0).cuda()
    tu = big[:, :nx]
    with lt.Context() as ctx:
        U = ctx.wrap(tu)
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((128, 256), halo=(1, 1)))
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(256, 128), args=[U, V])
        ctx.synchronize()
        got = V.read()
    assert np.array_equal(got, oracle.jacobi2d(u0, 1))


def test_zero_fill_of_a_wrapped_view_leaves_its_row_padding():
    # a zero fill writes the box rows only: the columns past the view's width
    # (another tensor's data in the caller's allocation) keep their values
    ny, nx, pitch = 129, 517, 640
    big = torch.full((ny, pitch), 5.0, dtype=torch.float32, device="cuda")
    with lt.Context() as ctx:
        A = ctx.wrap(big[:, :nx])
        A.fill(L.LT_INIT_ZERO)
        ctx.synchronize()
        A.destroy()
    got = big.cpu().numpy()
    assert not got[:, :nx].any()
    assert (got[:, nx:] == 5.0).all()
