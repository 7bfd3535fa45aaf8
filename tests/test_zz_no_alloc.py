"""The allocation-free Jacobi entry point against the engine's own launch.

lt_jacobi2d_packed_noalloc is for callers that cannot allocate device memory
(they run under another framework's allocator or a fixed device budget): it
keeps its scratch in a static device array instead of the engine's pool.
This test calls it through the C ABI on device buffers the test owns, twice
in a row (the second call reads the first call's output, so stale scratch
from the first call would show), and compares both results with an
annotated lt_launch over tiles without halo, which packs the same regions
through the engine's pool.  Jacobi results are bit-exact in this project.
"""
import ctypes as C

import numpy as np
import pytest

import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu

ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def engine_steps(u0, tile, iters):
    ny, nx = u0.shape
    out = []
    with lt.Context() as ctx:
        dist = lt.Dist.tiles(tile)                     # no halo: the pack path
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(tile[1], tile[0]), args=[U, V])
            U, V = V, U
            ctx.synchronize()
            out.append(U.read())
    return out


@pytest.mark.parametrize("ny,nx,tile", [(1000, 1500, (128, 256)), (4096, 4096, (2048, 4096)), (77, 130, (16, 20))])
def test_noalloc_matches_engine_launch_two_calls(ny, nx, tile):
    torch = pytest.importorskip("torch")
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 3, ny, nx)
    want = engine_steps(u0, tile, 2)
    lib = L.load()
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    rc = lib.lt_jacobi2d_packed_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), ny, nx, nx, nx,
                                        tile[0], tile[1], None)
    assert rc == L.LT_OK, lib.lt_last_error()
    rc = lib.lt_jacobi2d_packed_noalloc(C.c_void_p(b.data_ptr()), C.c_void_p(a.data_ptr()), ny, nx, nx, nx,
                                        tile[0], tile[1], None)
    assert rc == L.LT_OK, lib.lt_last_error()
    torch.cuda.synchronize()
    got1 = b.cpu().numpy()
    got2 = a.cpu().numpy()
    assert np.array_equal(got1, want[0])
    assert np.array_equal(got2, want[1])


def test_noalloc_rejects_tiles_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    lib = L.load()
    a = torch.zeros((16, 8), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    # 5000 x 5000 f32 tile: about 100 MB > 64 MiB scratch
    rc = lib.lt_jacobi2d_packed_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), 10000, 10000, 10000,
                                        10000, 5000, 5000, None)
    assert rc == L.LT_ERR_INVALID_ARG
    assert b"scratch" in lib.lt_last_error()
    rc = lib.lt_jacobi2d_packed_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), 16, 8, 8, 8, 4, 4, None)
    assert rc == L.LT_ERR_INVALID_ARG
