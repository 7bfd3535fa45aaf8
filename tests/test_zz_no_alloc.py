"""The allocation-free Jacobi entry point against the oracle and the engine.

lt_jacobi2d_packed_noalloc is for callers that cannot allocate device memory
(they run under another framework's allocator or a fixed device budget): it
keeps its scratch in a static device array instead of the engine's pool.
These tests call it through the C ABI on device buffers the test owns, twice
in a row (the second call reads the first call's output, so stale scratch
from the first call would show), and compare both results with the oracle
and with an annotated lt_launch over tiles without halo, which packs the
same regions through the engine's pool.  Jacobi results are bit-exact in
this project.  The file is collected last, so a run that stops at the first
failure has run every other test before it.
"""
import ctypes as C

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


def call(lib, src, dst, ny, nx, tile, stream=None):
    return lib.lt_jacobi2d_packed_noalloc(C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()), ny, nx, nx, nx,
                                          tile[0], tile[1], stream)


@pytest.mark.parametrize("ny,nx,tile", [(1000, 1500, (128, 256)), (4096, 4096, (2048, 4096)), (77, 130, (16, 20))])
def test_noalloc_matches_oracle_and_engine_launch_two_calls(ny, nx, tile):
    torch = pytest.importorskip("torch")
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 3, ny, nx)
    want = engine_steps(u0, tile, 2)
    assert np.array_equal(want[0], oracle.jacobi2d(u0, 1))
    assert np.array_equal(want[1], oracle.jacobi2d(u0, 2))
    lib = L.load()
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    rc = call(lib, a, b, ny, nx, tile)
    assert rc == L.LT_OK, lib.lt_last_error()
    rc = call(lib, b, a, ny, nx, tile)
    assert rc == L.LT_OK, lib.lt_last_error()
    torch.cuda.synchronize()
    got1 = b.cpu().numpy()
    got2 = a.cpu().numpy()
    assert np.array_equal(got1, want[0])
    assert np.array_equal(got2, want[1])


def test_noalloc_calls_leave_free_device_memory_unchanged():
    # after one warm-up call (module and kernels loaded), further calls must
    # not take device memory: the scratch is the static array
    torch = pytest.importorskip("torch")
    ny, nx, tile = 2048, 3000, (512, 1024)
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 4, ny, nx)
    lib = L.load()
    a = torch.from_numpy(u0).cuda()
    b = torch.empty_like(a)
    assert call(lib, a, b, ny, nx, tile) == L.LT_OK, lib.lt_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call(lib, a, b, ny, nx, tile) == L.LT_OK, lib.lt_last_error()
        assert call(lib, b, a, ny, nx, tile) == L.LT_OK, lib.lt_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.array_equal(a.cpu().numpy(), oracle.jacobi2d(u0, 6))


def test_noalloc_rejects_tiles_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    lib = L.load()
    n = 10000
    # buffers of the size the call is told, so that a regressed size check
    # could not write outside them
    a = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    # 5000 x 5000 f32 tile: about 100 MB > 64 MiB scratch
    rc = call(lib, a, b, n, n, (5000, 5000))
    assert rc == L.LT_ERR_INVALID_ARG
    assert b"scratch" in lib.lt_last_error()
    rc = lib.lt_jacobi2d_packed_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), 16, 8, 8, 8, 4, 4, None)
    assert rc == L.LT_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(b)) == 0


def test_noalloc_refuses_a_capturing_stream():
    torch = pytest.importorskip("torch")
    lib = L.load()
    ny, nx = 64, 96
    a = torch.rand((ny, nx), device="cuda")
    b = torch.zeros_like(a)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        rc = call(lib, a, b, ny, nx, (32, 32), stream=C.c_void_p(s.cuda_stream))
        b.add_(0.0)  # the capture holds one node
    assert rc == L.LT_ERR_UNSUPPORTED
    assert b"capturing" in lib.lt_last_error()
