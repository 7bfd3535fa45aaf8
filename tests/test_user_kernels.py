"""Runtime-compiled user kernels (Sec. 3.5): a __device__ function in the
paper's convention (virtual block index + view types), wrapped, compiled by
NVRTC for sm_103a and launched through the planner.  The kernel bodies here
are this project's own code, written for the computations the paper
describes.  CPU tests compile in a dry-run context; GPU tests check results
against the oracle."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

AVG3 = r"""
__device__ void avg3(dim3 vb, int64_t len, lightning::Vector<float> dst, lightning::Vector<float> src) {
    const int64_t g = (int64_t)vb.x * blockDim.x + threadIdx.x;
    if (g >= len) return;
    float acc = g > 0 ? src[g - 1] : 0.0f;
    acc = acc + src[g];
    acc = acc + (g + 1 < len ? src[g + 1] : 0.0f);
    dst[g] = (float)((double)acc / 3.0);
}
"""

MATMUL = r"""
__device__ void mm(dim3 vb, int64_t M, int64_t N, int64_t K,
                   lightning::Matrix<float> A, lightning::Matrix<float> B, lightning::Matrix<float> C) {
    const int64_t col = (int64_t)vb.x * blockDim.x + threadIdx.x;
    const int64_t row = (int64_t)vb.y * blockDim.y + threadIdx.y;
    if (row >= M || col >= N) return;
    float s = 0.0f;
    for (int64_t k = 0; k < K; ++k) s = s + A(row, k) * B[k][col];
    C(row, col) = s;
}
"""

JAC_BLOCK_LOCAL = r"""
__device__ void jac(dim3 vb, int64_t ny, int64_t nx, lightning::Matrix<float> U, lightning::Matrix<float> V) {
    const int64_t i = (int64_t)vb.y * 8 + threadIdx.y, j = (int64_t)vb.x * 32 + threadIdx.x;
    if (i >= ny || j >= nx) return;
    float a = U(i, j);
    a = a + (i > 0 ? U(i - 1, j) : 0.0f);
    a = a + (i + 1 < ny ? U(i + 1, j) : 0.0f);
    a = a + (j > 0 ? U(i, j - 1) : 0.0f);
    a = a + (j + 1 < nx ? U(i, j + 1) : 0.0f);
    V(i, j) = a / 5.0f;
}
"""


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def dry():
    return lt.Context(hbm_budget=1 << 30, flags=L.LT_FLAG_DRYRUN)


def test_source_kernel_compiles_and_plans_in_dry_run():
    with dry() as ctx:
        A = ctx.array(lt.F32, (1000,), lt.Dist.rows(300, halo=1))
        B = ctx.array(lt.F32, (1000,), lt.Dist.rows(300, halo=1))
        k = ctx.kernel_from_source(AVG3, "avg3", "global i => read src[i-1:i+1], write dst[i]",
                                   [("len", lt.U32, False), ("dst", lt.F32), ("src", lt.F32)])
        plan = k.explain(grid=(1000,), block=(100,), superblock=(300,), args=[1000, B, A])
        assert [a["kind"] for a in plan["superblocks"][1]["args"]] == ["value", "direct", "direct"]
        # a superblock that straddles two chunks writes a temporary and reads a packed copy
        plan = k.explain(grid=(1000,), block=(64,), superblock=(320,), args=[1000, B, A])
        assert [a["kind"] for a in plan["superblocks"][1]["args"]] == ["value", "temp_write", "pack"]
        k.launch(grid=(1000,), block=(64,), superblock=(320,), args=[1000, B, A])
        ctx.synchronize()


def test_source_kernel_rejects_oversized_blocks():
    with dry() as ctx:
        A = ctx.array(lt.F32, (1000,), lt.Dist.rows(500, halo=1))
        B = ctx.array(lt.F32, (1000,), lt.Dist.rows(500, halo=1))
        k = ctx.kernel_from_source(AVG3, "avg3", "global i => read src[i-1:i+1], write dst[i]",
                                   [("len", lt.U32, False), ("dst", lt.F32), ("src", lt.F32)])
        with pytest.raises(lt.LightningError) as e:
            k.launch(grid=(1000,), block=(2048,), superblock=(2048,), args=[1000, B, A])
        assert e.value.code == L.LT_ERR_INVALID_ARG


def test_source_kernel_compile_error_reports_the_log():
    with dry() as ctx:
        with pytest.raises(lt.LightningError) as e:
            ctx.kernel_from_source("__device__ void bad(dim3 vb, lightning::Vector<float> x) { x[0] = undefined_name; }",
                                   "bad", "global i => write x[i]", [("x", lt.F32)])
        assert e.value.code == L.LT_ERR_COMPILE
        assert "undefined_name" in str(e.value)


@pytest.mark.gpu
def test_user_kernel_paper_example_bit_exact():
    n = 1_000_000
    want = np.ones(n, np.float32)
    for _ in range(10):
        want = oracle.stencil1d_paper(want)
    with lt.Context() as ctx:
        dist = lt.Dist.rows(64_000, halo=1)
        src = ctx.array(lt.F32, (n,), dist)
        dst = ctx.array(lt.F32, (n,), dist)
        src.fill(L.LT_INIT_CONST, value=1.0)
        k = ctx.kernel_from_source(AVG3, "avg3", "global i => read src[i-1:i+1], write dst[i]",
                                   [("len", lt.U32, False), ("dst", lt.F32), ("src", lt.F32)])
        for _ in range(10):
            k.launch(grid=(n,), block=(16,), superblock=(64_000,), args=[n, dst, src])
            src, dst = dst, src
        ctx.synchronize()
        assert np.array_equal(src.read(), want)


@pytest.mark.gpu
@pytest.mark.parametrize("adist", ["rows", "tiles_pack"])
def test_user_kernel_matmul_annotation(adist):
    M, N, K = 96, 80, 70
    rng = np.random.default_rng(5)
    a = rng.standard_normal((M, K)).astype(np.float32)
    b = rng.standard_normal((K, N)).astype(np.float32)
    want = oracle.gemm_f64(a.astype(np.float64), b.astype(np.float64))
    with lt.Context() as ctx:
        A = ctx.array(lt.F32, (M, K), lt.Dist.rows(32) if adist == "rows" else lt.Dist.tiles((32, 30)))
        B = ctx.array(lt.F32, (K, N), lt.Dist.cols(48))
        Cm = ctx.array(lt.F32, (M, N), lt.Dist.tiles((32, 48)))
        A.write(a)
        B.write(b)
        k = ctx.kernel_from_source(MATMUL, "mm", "global [i, j] => read A[i, :], read B[:, j], write C[i, j]",
                                   [("M", lt.U32, False), ("N", lt.U32, False), ("K", lt.U32, False),
                                    ("A", lt.F32), ("B", lt.F32), ("C", lt.F32)])
        k.launch(grid=(N, M), block=(16, 16), superblock=(48, 32), args=[M, N, K, A, B, Cm])
        ctx.synchronize()
        got = Cm.read().astype(np.float64)
    bound = K * 2.0**-23 * (np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)))
    assert np.all(np.abs(got - want) <= bound)


@pytest.mark.gpu
def test_user_kernel_block_local_bindings_bit_exact():
    ny, nx = 200, 300
    u0 = si.uniform_field(2203, 11, ny, nx)
    ann = ("block [bi, bj], local [li, lj] => "
           "read U[8*bi + li - 1 : 8*bi + li + 1, 32*bj + lj - 1 : 32*bj + lj + 1], write V[8*bi + li, 32*bj + lj]")
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((64, 96), halo=(1, 1)))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((64, 96), halo=(1, 1)))
        U.write(u0)
        k = ctx.kernel_from_source(JAC_BLOCK_LOCAL, "jac", ann,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        for _ in range(3):
            k.launch(grid=(nx, ny), block=(32, 8), superblock=(96, 64), args=[ny, nx, U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi2d(u0, 3))


# A body that stages its block's cells and the two halo cells in shared
# memory and waits at a barrier before it reads them: the persistent wrapper
# must keep every virtual block's shared memory apart from the next one's.
AVG3_SHARED = r"""
__device__ void avg3s(dim3 vb, int64_t len, lightning::Vector<float> dst, lightning::Vector<float> src) {
    __shared__ float tile[258];
    const int64_t g = (int64_t)vb.x * blockDim.x + threadIdx.x;
    const int t = threadIdx.x + 1;
    tile[t] = g < len ? src[g] : 0.0f;
    if (threadIdx.x == 0) tile[0] = g > 0 && g - 1 < len ? src[g - 1] : 0.0f;
    if (threadIdx.x == blockDim.x - 1) tile[t + 1] = g + 1 < len ? src[g + 1] : 0.0f;
    __syncthreads();
    if (g >= len) return;
    float acc = tile[t - 1];
    acc = acc + tile[t];
    acc = acc + tile[t + 1];
    dst[g] = (float)((double)acc / 3.0);
}
"""


@pytest.mark.gpu
def test_user_kernel_with_shared_memory_and_barrier_bit_exact():
    n = 3_000_017
    x0 = si.uniform_field(2203, 12, 1, n).ravel()
    want = x0.copy()
    for _ in range(4):
        want = oracle.stencil1d_paper(want)
    with lt.Context() as ctx:
        dist = lt.Dist.rows(500_000, halo=1)
        src = ctx.array(lt.F32, (n,), dist)
        dst = ctx.array(lt.F32, (n,), dist)
        src.write(x0)
        k = ctx.kernel_from_source(AVG3_SHARED, "avg3s", "global i => read src[i-1:i+1], write dst[i]",
                                   [("len", lt.U32, False), ("dst", lt.F32), ("src", lt.F32)])
        for _ in range(4):
            k.launch(grid=(n,), block=(256,), superblock=(500_000,), args=[n, dst, src])
            src, dst = dst, src
        ctx.synchronize()
        assert np.array_equal(src.read(), want)


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [0, L.LT_FLAG_NO_FUSED_REPLICAS])
@pytest.mark.parametrize("dist_kind", ["tiles_halo", "block", "rows_halo"])
def test_user_kernel_four_cells_per_thread_bit_exact(dist_kind, flags):
    # the benchmark's vector body: four columns per thread from float4 rows,
    # annotated "read U[i-1:i+1, 4*j-1:4*j+4], write V[i, 4*j:4*j+3]"; a ragged
    # width (not a multiple of 4) exercises the masked edge
    import bench
    ny, nx, iters = 300, 517, 3
    u0 = si.uniform_field(2203, 13, ny, nx)
    dist, sb = {"tiles_halo": (lt.Dist.tiles((128, 256), halo=(1, 1)), (64, 128)),
                "block": (lt.Dist.block(), (0, 0)),
                "rows_halo": (lt.Dist.rows(100, halo=1), ((nx + 3) // 4, 100))}[dist_kind]
    with lt.Context(flags=flags) as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel_from_source(bench.USER_JACOBI_VEC, "jacobi4", bench.USER_JACOBI_VEC_ANN,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=((nx + 3) // 4, ny), block=(64, 4), superblock=sb, args=[ny, nx, U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi2d(u0, iters))


HSUM_F64 = r"""
__device__ void hsum(dim3 vb, int64_t ny, int64_t nx, lightning::Matrix<double> U, lightning::Matrix<double> V) {
    const int64_t i = (int64_t)vb.y * blockDim.y + threadIdx.y, j = (int64_t)vb.x * blockDim.x + threadIdx.x;
    if (i >= ny || j >= nx) return;
    double a = j > 0 ? U(i, j - 1) : 0.0;
    a = a + U(i, j);
    a = a + (j + 1 < nx ? U(i, j + 1) : 0.0);
    V(i, j) = a;
}
"""


@pytest.mark.gpu
@pytest.mark.parametrize("halo,flags", [(0, 0), (1, 0), (1, L.LT_FLAG_NO_FUSED_REPLICAS)])
def test_user_kernel_f64_column_bands_pack_and_replicas_exact(halo, flags):
    # f64 arrays in column bands: without a halo every band's read region
    # takes one column from each neighbour (8-byte one-column pack pieces);
    # with a 1-column halo the written columns update the neighbours'
    # replicas (8-byte one-column copies).  The sum of three doubles in this
    # order is exact to compare: the same operations as the numpy expression.
    ny, nx, iters = 2500, 700, 3
    rng = np.random.default_rng(2203)
    u0 = rng.standard_normal((ny, nx))
    want = u0.copy()
    for _ in range(iters):
        left = np.zeros_like(want)
        right = np.zeros_like(want)
        left[:, 1:] = want[:, :-1]
        right[:, :-1] = want[:, 1:]
        want = (left + want) + right
    with lt.Context(flags=flags) as ctx:
        ctx.log_enable()
        dist = lt.Dist.cols(96, halo=halo) if halo else lt.Dist.cols(96)
        U = ctx.array(lt.F64, (ny, nx), dist)
        V = ctx.array(lt.F64, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel_from_source(HSUM_F64, "hsum", "global [i, j] => read U[i, j-1:j+1], write V[i, j]",
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F64), ("V", lt.F64)])
        for _ in range(iters):
            k.launch(grid=(nx, ny), block=(32, 8), superblock=(96, ny), args=[ny, nx, U, V])
            U, V = V, U
        ctx.synchronize()
        kinds = {t["kind"] for t in ctx.log()}
        got = U.read()
    if not halo:
        assert "pack" in kinds
    else:  # the wrapper copies the replicas itself unless told not to
        assert ("unpack" in kinds) == bool(flags & L.LT_FLAG_NO_FUSED_REPLICAS)
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


def test_source_kernel_replicas_fused_into_the_launch_in_dry_run():
    # a source kernel writing tiles with halos: no copy step follows its
    # launch (the wrapper updates the replicas after a grid-wide barrier);
    # with LT_FLAG_NO_FUSED_REPLICAS an unpack step does, for the same bytes
    import bench
    got = {}
    for fl in (0, L.LT_FLAG_NO_FUSED_REPLICAS):
        with lt.Context(hbm_budget=1 << 30, flags=L.LT_FLAG_DRYRUN | fl) as ctx:
            k = ctx.kernel_from_source(bench.USER_JACOBI_VEC, "jacobi4", bench.USER_JACOBI_VEC_ANN,
                                       [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
            ctx.log_enable()
            dist = lt.Dist.tiles((1024, 1024), halo=(1, 1))
            U = ctx.array(lt.F32, (4096, 4096), dist)
            V = ctx.array(lt.F32, (4096, 4096), dist)
            k.launch(grid=(1024, 4096), block=(64, 4), superblock=(256, 1024), args=[4096, 4096, U, V])
            ctx.synchronize()
            st = ctx.stats()
            got[fl] = ({t["kind"] for t in ctx.log()}, st["bytes_replica_wt"], st["bytes_d2d"])
    # 4 x 4 tiles of 1024^2: 24 inner edges, each copied both ways (1024 cells), and at each of the
    # 9 inner corner points the 4 tiles' corner cells, each to its diagonal neighbour's corner halo
    edge_bytes = 4 * (24 * 2 * 1024 + 9 * 4)
    assert got[0] == ({"zero", "execute"}, edge_bytes, 0)
    assert got[L.LT_FLAG_NO_FUSED_REPLICAS] == ({"zero", "execute", "unpack"}, 0, edge_bytes)


@pytest.mark.gpu
def test_source_kernel_replica_barrier_timeout_reports_and_context_survives():
    # failure detection without a fault: the test flag makes the wrapper's
    # grid barrier wait for one CTA more than the launch has, so its bounded
    # wait (2 s) runs out; the replicas are left as they were, the host reads
    # LT_ERR_TIMEOUT, and the same context then runs a launch without
    # replicas (one chunk) correctly
    import bench
    ny, nx = 300, 517
    u0 = si.uniform_field(2203, 17, ny, nx)
    with lt.Context(flags=L.LT_FLAG_TEST_REPLICA_STALL) as ctx:
        k = ctx.kernel_from_source(bench.USER_JACOBI_VEC, "jacobi4", bench.USER_JACOBI_VEC_ANN,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((128, 256), halo=(1, 1)))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((128, 256), halo=(1, 1)))
        U.write(u0)
        k.launch(grid=((nx + 3) // 4, ny), block=(64, 4), superblock=(64, 128), args=[ny, nx, U, V])
        with pytest.raises(lt.LightningError) as e:
            ctx.synchronize()
        assert e.value.code == L.LT_ERR_TIMEOUT
        A = ctx.array(lt.F32, (ny, nx), lt.Dist.block())
        B = ctx.array(lt.F32, (ny, nx), lt.Dist.block())
        A.write(u0)
        k.launch(grid=((nx + 3) // 4, ny), block=(64, 4), superblock=(0, 0), args=[ny, nx, A, B])
        ctx.synchronize()
        assert np.array_equal(B.read(), oracle.jacobi2d(u0, 1))


JAC3 = r"""
__device__ void jac3(dim3 vb, int64_t nz, int64_t ny, int64_t nx, lightning::Tensor<float> U, lightning::Tensor<float> V) {
    const int64_t k = (int64_t)vb.z * blockDim.z + threadIdx.z;
    const int64_t i = (int64_t)vb.y * blockDim.y + threadIdx.y;
    const int64_t j = (int64_t)vb.x * blockDim.x + threadIdx.x;
    if (k >= nz || i >= ny || j >= nx) return;
    float a = U(k, i, j);
    a = a + (k > 0 ? U(k - 1, i, j) : 0.0f);
    a = a + (k + 1 < nz ? U(k + 1, i, j) : 0.0f);
    a = a + (i > 0 ? U(k, i - 1, j) : 0.0f);
    a = a + (i + 1 < ny ? U(k, i + 1, j) : 0.0f);
    a = a + (j > 0 ? U(k, i, j - 1) : 0.0f);
    a = a + (j + 1 < nx ? U(k, i, j + 1) : 0.0f);
    V(k, i, j) = a / 7.0f;
}
"""


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [0, L.LT_FLAG_NO_FUSED_REPLICAS])
@pytest.mark.parametrize("block,sb", [((32, 4, 1), (64, 24, 13)), ((32, 4, 2), (64, 24, 14))])
def test_user_kernel_3d_tiles_with_halos_replicas_bit_exact(flags, block, sb):
    # a 7-point body over 3-D tiles with 1-cell halos: every launch updates
    # face, edge and corner replicas of the written array (inside the launch
    # by default); the same operation order as the oracle's 3-D Jacobi.
    # Superblocks of one chunk each, or 14 planes deep across 13-plane chunks
    # (packed reads, writes through temporaries and replicas together)
    nz, ny, nx, iters = 37, 50, 133, 3
    idx = np.arange(nz * ny * nx, dtype=np.uint64)
    u0 = si.gen_uniform_f32(2203, 23, idx).reshape(nz, ny, nx)
    dist = lt.Dist.tiles((13, 24, 64), halo=(1, 1, 1))
    with lt.Context(flags=flags) as ctx:
        ctx.log_enable()
        U = ctx.array(lt.F32, (nz, ny, nx), dist)
        V = ctx.array(lt.F32, (nz, ny, nx), dist)
        U.write(u0)
        k = ctx.kernel_from_source(JAC3, "jac3", "global [k, i, j] => read U[k-1:k+1, i-1:i+1, j-1:j+1], write V[k, i, j]",
                                   [("nz", lt.U32, False), ("ny", lt.U32, False), ("nx", lt.U32, False),
                                    ("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(nx, ny, nz), block=block, superblock=sb, args=[nz, ny, nx, U, V])
            U, V = V, U
        ctx.synchronize()
        kinds = {t["kind"] for t in ctx.log()}
        got = U.read()
    if sb[2] == 13:
        assert ("unpack" in kinds) == bool(flags & L.LT_FLAG_NO_FUSED_REPLICAS)
    want = oracle.jacobi3d(u0, iters)
    assert np.array_equal(got, want), f"{np.sum(got != want)} cells differ"


@pytest.mark.gpu
def test_user_kernel_full_size_incore_4x4_as_benchmarked_bit_exact():
    # the benchmark's source-kernel configuration: 4096^2 in 4 x 4 tiles of
    # 1024^2 + halo, superblocks of 256 x 1024 threads (1024 columns), 10
    # iterations, replicas updated inside each launch; every cell compared
    import bench
    n, iters = 4096, 10
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 0, n, n)
    dist = lt.Dist.tiles((1024, 1024), halo=(1, 1))
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (n, n), dist)
        V = ctx.array(lt.F32, (n, n), dist)
        U.write(u0)
        k = ctx.kernel_from_source(bench.USER_JACOBI_VEC, "jacobi4", bench.USER_JACOBI_VEC_ANN,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(n // 4, n), block=(64, 4), superblock=(256, 1024), args=[n, n, U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, oracle.jacobi2d(u0, iters))


@pytest.mark.gpu
@pytest.mark.parametrize("flags", [0, L.LT_FLAG_NO_FUSED_REPLICAS])
@pytest.mark.parametrize("dist_kind", ["tiles_halo", "block", "rows_halo", "cols_halo", "tiles_nohalo"])
def test_user_kernel_sixteen_cells_per_thread_bit_exact(dist_kind, flags):
    # the benchmark's body with four rows of four cells per thread, annotated
    # "read U[4*i-1:4*i+4, 4*j-1:4*j+4], write V[4*i:4*i+3, 4*j:4*j+3]"; a
    # height and width that are not multiples of 4 exercise the masked edges,
    # tiles without halo the pack and temporary-write paths
    import bench
    ny, nx, iters = 301, 517, 3
    u0 = si.uniform_field(2203, 14, ny, nx)
    dist, sb = {"tiles_halo": (lt.Dist.tiles((128, 256), halo=(1, 1)), (64, 32)),
                "block": (lt.Dist.block(), (0, 0)),
                "rows_halo": (lt.Dist.rows(100, halo=1), ((nx + 3) // 4, 25)),
                "cols_halo": (lt.Dist.cols(128, halo=1), (32, (ny + 3) // 4)),
                "tiles_nohalo": (lt.Dist.tiles((128, 256), halo=(0, 0)), (64, 32))}[dist_kind]
    with lt.Context(flags=flags) as ctx:
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        U.write(u0)
        k = ctx.kernel_from_source(bench.USER_JACOBI_VEC4, "jacobi16", bench.USER_JACOBI_VEC4_ANN,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=((nx + 3) // 4, (ny + 3) // 4), block=(64, 4), superblock=sb, args=[ny, nx, U, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi2d(u0, iters))


@pytest.mark.gpu
def test_user_kernel_sixteen_cells_full_size_incore_4x4_bit_exact():
    # the benchmarked configuration of that body: 4096^2 in 4 x 4 tiles of
    # 1024^2 + halo, superblocks of 256 x 256 threads, 10 iterations
    import bench
    n, iters = 4096, 10
    u0 = si.uniform_field(si.SEED_JACOBI_INCORE, 0, n, n)
    dist = lt.Dist.tiles((1024, 1024), halo=(1, 1))
    with lt.Context() as ctx:
        U = ctx.array(lt.F32, (n, n), dist)
        V = ctx.array(lt.F32, (n, n), dist)
        U.write(u0)
        k = ctx.kernel_from_source(bench.USER_JACOBI_VEC4, "jacobi16", bench.USER_JACOBI_VEC4_ANN,
                                   [("ny", lt.U32, False), ("nx", lt.U32, False), ("U", lt.F32), ("V", lt.F32)])
        for _ in range(iters):
            k.launch(grid=(n // 4, n // 4), block=(64, 4), superblock=(256, 256), args=[n, n, U, V])
            U, V = V, U
        ctx.synchronize()
        got = U.read()
    assert np.array_equal(got, oracle.jacobi2d(u0, iters))


DIV_HELPERS = r"""
__device__ void div1(dim3 vb, int64_t n, lightning::Vector<float> q, lightning::Vector<float> a) {
    const int64_t g = (int64_t)vb.x * blockDim.x + threadIdx.x;
    if (g < n) q[g] = lightning::div_rn<5>(a[g]);
}
__device__ void div4(dim3 vb, int64_t n4, lightning::Vector<float> q, lightning::Vector<float> a) {
    const int64_t g = (int64_t)vb.x * blockDim.x + threadIdx.x;
    if (g >= n4) return;
    const float4 r = lightning::div4_rn<7>(make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]));
    q[4 * g] = r.x; q[4 * g + 1] = r.y; q[4 * g + 2] = r.z; q[4 * g + 3] = r.w;
}
"""


def _division_inputs():
    # random bit patterns (NaNs, infinities, subnormals and all) plus the
    # edges of the fast path's range, each special value in every one of
    # the four positions of a group, next to ordinary values
    rng = np.random.default_rng(2202)
    bits = rng.integers(0, 2 ** 32, size=1 << 16, dtype=np.uint64).astype(np.uint32)
    special = np.array([0.0, -0.0, 1e-30, -1e-30, 9.99e-31, 1e30, -1e30, 1.01e30, 1e-45, -1e-45, 1.17549435e-38,
                        3.4028235e38, np.inf, -np.inf, np.nan, 1.0, 5.0, 7.0, 0.2, 1.0 / 3.0], dtype=np.float32)
    groups = []
    for v in special:
        for pos in range(4):
            g = np.array([0.75, 1.5, 3.25, 6.0], dtype=np.float32)
            g[pos] = v
            groups.append(g)
    return np.concatenate([bits.view(np.float32), np.concatenate(groups)])


@pytest.mark.gpu
def test_source_kernel_division_helpers_match_ieee_division():
    a = _division_inputs()
    n = a.size
    assert n % 4 == 0
    with lt.Context() as ctx:
        A = ctx.array(lt.F32, (n,), lt.Dist.rows(n // 3 // 4 * 4, halo=0))
        Q = ctx.array(lt.F32, (n,), lt.Dist.rows(n // 3 // 4 * 4, halo=0))
        A.write(a)
        k1 = ctx.kernel_from_source(DIV_HELPERS, "div1", "global i => read a[i], write q[i]",
                                    [("n", lt.U32, False), ("q", lt.F32), ("a", lt.F32)])
        k1.launch(grid=(n,), block=(128,), superblock=(n // 3 // 4 * 4,), args=[n, Q, A])
        got5 = Q.read()
        k4 = ctx.kernel_from_source(DIV_HELPERS, "div4", "global i => read a[4*i:4*i+3], write q[4*i:4*i+3]",
                                    [("n4", lt.U32, False), ("q", lt.F32), ("a", lt.F32)])
        k4.launch(grid=(n // 4,), block=(128,), superblock=(n // 3 // 16 * 4,), args=[n // 4, Q, A])
        got7 = Q.read()
    with np.errstate(all="ignore"):
        for got, c in ((got5, 5), (got7, 7)):
            want = a / np.float32(c)
            same = (got.view(np.uint32) == want.view(np.uint32)) | (np.isnan(got) & np.isnan(want))
            assert same.all(), (c, a[~same][:8], got[~same][:8], want[~same][:8])
