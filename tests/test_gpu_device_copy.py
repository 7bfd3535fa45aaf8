"""Copies between a chunked array and a dense device buffer
(lt_array_write_device / lt_array_read_device).

When every chunk fits in device memory at once, one box-copy kernel moves
all of them; otherwise (a chunk in the host pool, a budget too small) the
copies go chunk by chunk.  Both paths must give the buffer back bit for bit,
fill the halos a write covers, read a never-written array as zeros, and
order themselves after the launches that produce or use the chunks.  A zero
fill (a strided memset of each chunk's box) clears halos as well."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"

DISTS = {
    "block": lt.Dist.block(),
    "rows_halo": lt.Dist.rows(37, halo=1),
    "cols_halo2": lt.Dist.cols(50, halo=2),
    "tiles_halo": lt.Dist.tiles((64, 96), halo=(1, 1)),
    "tiles": lt.Dist.tiles((64, 96)),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("name", sorted(DISTS))
def test_round_trip_and_halos_feed_a_launch(name):
    ny, nx = 200, 333
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 31, ny, nx)
    src = torch.from_numpy(u0).cuda()
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), DISTS[name])
        V = ctx.array(lt.F32, (ny, nx), DISTS[name])
        U.write_device(src.data_ptr(), src.numel() * 4)
        assert np.array_equal(U.read(), u0)
        back = torch.empty_like(src)
        U.read_device(back.data_ptr(), back.numel() * 4)
        assert np.array_equal(back.cpu().numpy(), u0)
        # the write filled the halo copies too: a stencil launch over the
        # chunks reads them and must match the unchunked oracle
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(96, 64), args=[U, V])
        out = torch.empty_like(src)
        V.read_device(out.data_ptr(), out.numel() * 4)   # waits for the launch that writes V
        assert np.array_equal(out.cpu().numpy(), oracle.jacobi2d(u0, 1))


def test_never_written_array_reads_as_zeros_and_f64_3d():
    with lt.Context() as ctx:
        Z = ctx.array(lt.F32, (70, 90), lt.Dist.tiles((32, 32), halo=(1, 1)))
        buf = torch.full((70, 90), 7.0, dtype=torch.float32, device="cuda")
        Z.read_device(buf.data_ptr(), buf.numel() * 4)
        assert torch.count_nonzero(buf).item() == 0
        x = torch.arange(5 * 40 * 33, dtype=torch.float64, device="cuda").reshape(5, 40, 33) * 0.5
        A = ctx.array(lt.F64, (5, 40, 33), lt.Dist.tiles((2, 16, 16), halo=(1, 1, 1)))
        A.write_device(x.data_ptr(), x.numel() * 8)
        y = torch.empty_like(x)
        A.read_device(y.data_ptr(), y.numel() * 8)
        assert torch.equal(x, y)


def test_write_waits_for_launches_that_still_read_the_chunks():
    # a launch reads U; the write of new contents into U must come after it
    ny, nx = 256, 384
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 32, ny, nx)
    u1 = si.uniform_field(si.SEED_JACOBI_INCORE, 33, ny, nx)
    t0, t1 = torch.from_numpy(u0).cuda(), torch.from_numpy(u1).cuda()
    with lt.Context() as ctx:
        d = lt.Dist.tiles((128, 128), halo=(1, 1))
        U, V = ctx.array(lt.F32, (ny, nx), d), ctx.array(lt.F32, (ny, nx), d)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        U.write_device(t0.data_ptr(), t0.numel() * 4)
        for _ in range(3):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(128, 128), args=[U, V])
            U.write_device(t1.data_ptr(), t1.numel() * 4)   # overwrites what the launch reads
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(128, 128), args=[U, V])
            U.write_device(t0.data_ptr(), t0.numel() * 4)
        out = torch.empty_like(t0)
        V.read_device(out.data_ptr(), out.numel() * 4)
        assert np.array_equal(out.cpu().numpy(), oracle.jacobi2d(u1, 1))


def test_chunks_that_do_not_fit_together_go_one_by_one():
    # two 4 MiB arrays of 64 tiles under a 2 MiB budget: the launches stream
    # superblocks through the host pool, chunks lie there when the copies
    # run, and the copies take the chunk-by-chunk path
    ny, nx = 1024, 1024
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 34, ny, nx)
    src = torch.from_numpy(u0).cuda()
    with lt.Context(hbm_budget=2 << 20, host_pool=32 << 20) as ctx:
        d = lt.Dist.tiles((128, 128), halo=(1, 1))
        U, V = ctx.array(lt.F32, (ny, nx), d), ctx.array(lt.F32, (ny, nx), d)
        U.write_device(src.data_ptr(), src.numel() * 4)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        a, b = U, V
        for _ in range(4):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(128, 128), args=[a, b])
            a, b = b, a
        out = torch.empty_like(src)
        a.read_device(out.data_ptr(), out.numel() * 4)
        assert ctx.stats()["evictions"] > 0
    assert np.array_equal(out.cpu().numpy(), oracle.jacobi2d(u0, 4))


def test_zero_fill_clears_owned_cells_and_halos():
    ny, nx = 300, 250
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 35, ny, nx)
    with lt.Context() as ctx:
        d = lt.Dist.tiles((64, 64), halo=(1, 1))
        U, V = ctx.array(lt.F32, (ny, nx), d), ctx.array(lt.F32, (ny, nx), d)
        U.write(u0)
        U.fill(L.LT_INIT_ZERO)
        assert not U.read().any()
        # the halo copies are zero too: a stencil over the chunks gives zeros
        V.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(64, 64), args=[U, V])
        assert not V.read().any()
