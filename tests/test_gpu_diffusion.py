"""GPU parity of the diffusion forward launch and its chunked adjoint.

Bars: forward f32 vs fp64 oracle <= 1e-5 relative (and chunked == unchunked
bit for bit); gradients (adjoint with checkpoints + recomputation) vs the
fp64 oracle gradient <= 1e-4 relative L2, and vs central finite differences
of the fp64 forward (exact up to rounding: J is quadratic in u0).
"""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu
FWD = "global [i, j] => read U[i-1:i+1, j-1:j+1], read K[i, j], write V[i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def fields(ny, nx):
    return (si.uniform_field(si.SEED_DIFFUSION, si.STREAM_U, ny, nx),
            si.kappa_field(si.SEED_DIFFUSION, si.STREAM_KAPPA, ny, nx))


def test_forward_chunked_bit_exact_and_vs_fp64():
    ny, nx, T = 300, 517, 6
    u0, k = fields(ny, nx)
    want = oracle.diffusion_forward(u0.astype(np.float64), k.astype(np.float64), T)
    outs = []
    with lt.Context() as ctx:
        kf = ctx.kernel(lt.DIFFUSION2D, FWD, [("U", lt.F32), ("K", lt.F32), ("V", lt.F32)])
        for dist, sb in [(lt.Dist.block(), (0, 0)), (lt.Dist.tiles((64, 128), halo=(1, 1)), (128, 64)),
                         (lt.Dist.rows(50, halo=1), (517, 50)), (lt.Dist.tiles((64, 64)), (64, 64))]:
            U = ctx.array(lt.F32, (ny, nx), dist)
            V = ctx.array(lt.F32, (ny, nx), dist)
            K = ctx.array(lt.F32, (ny, nx), dist)
            U.write(u0)
            K.write(k)
            for _ in range(T):
                kf.launch(grid=(nx, ny), block=(128, 2), superblock=sb, args=[U, K, V])
                U, V = V, U
            ctx.synchronize()
            outs.append(U.read())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert rel(outs[0], want) < 1e-5


@pytest.mark.parametrize("chunk,ckpt", [(0, 10), (16, 10), (24, 7)])
def test_adjoint_64x64_vs_fp64_gradient_and_fd(chunk, ckpt):
    torch = pytest.importorskip("torch")
    from paper_2202_05549_gb300.autograd import DiffusionChunked

    n, T = 64, 50
    u0, k = fields(n, n)
    u = torch.from_numpy(u0).cuda().requires_grad_(True)
    kt = torch.from_numpy(k).cuda().requires_grad_(True)
    sb = (chunk, chunk) if chunk else (0, 0)
    uT = DiffusionChunked.apply(u, kt, T, ckpt, chunk, sb)
    J = (uT.double() ** 2).sum()
    J.backward()
    J64, du0, dk = oracle.diffusion_grad(u0.astype(np.float64), k.astype(np.float64), T)
    assert abs(J.item() - J64) / J64 < 1e-5
    assert rel(u.grad.cpu().numpy(), du0) < 1e-4
    assert rel(kt.grad.cpu().numpy(), dk) < 1e-4
    # central finite differences of the fp64 forward
    g = u.grad.cpu().numpy()
    for (i, j) in [(0, 0), (31, 17), (63, 63), (5, 62)]:
        h = 1e-3
        up = u0.astype(np.float64).copy(); up[i, j] += h
        dn = u0.astype(np.float64).copy(); dn[i, j] -= h
        fd = (np.sum(oracle.diffusion_forward(up, k.astype(np.float64), T) ** 2)
              - np.sum(oracle.diffusion_forward(dn, k.astype(np.float64), T) ** 2)) / (2 * h)
        assert abs(g[i, j] - fd) <= 1e-4 * max(abs(fd), 1e-3)


def test_adjoint_full_size_16384_sampled_vs_lightcone():
    torch = pytest.importorskip("torch")
    from paper_2202_05549_gb300.autograd import DiffusionPlan

    n, T, ck, chunk = 16384, 50, 10, 4096
    field = n * n * 4
    with lt.Context(hbm_budget=int(26 * field * 1.1)) as ctx:
        plan = DiffusionPlan(ctx, n, n, T, ck, lt.Dist.tiles((chunk, chunk), halo=(1, 1)), (chunk, chunk))
        plan.K.fill(L.LT_INIT_KAPPA, seed=si.SEED_DIFFUSION, stream=si.STREAM_KAPPA)
        plan.ck[0].fill(L.LT_INIT_UNIFORM, seed=si.SEED_DIFFUSION, stream=si.STREAM_U)
        plan.forward()
        uT = torch.empty((n, n), dtype=torch.float32, device="cuda")
        plan.ck[-1].read_device(uT.data_ptr(), field)
        lamT = (2.0 * uT).contiguous()
        torch.cuda.synchronize()
        plan.lam[0].write_device(lamT.data_ptr(), field)
        lam0 = plan.backward()
        ii, jj = si.sample_cells(2207, n, n, 16, seams_every=chunk)
        g_u = np.array([lam0.read_box((a, b), (a, b))[0, 0] for a, b in zip(ii, jj)])
        g_k = np.array([plan.G.read_box((a, b), (a, b))[0, 0] for a, b in zip(ii, jj)])
        u_T = np.array([plan.ck[-1].read_box((a, b), (a, b))[0, 0] for a, b in zip(ii, jj)])
    wu, wdu, wdk = oracle.diffusion_lightcone(n, n, si.SEED_DIFFUSION, si.STREAM_U, si.STREAM_KAPPA, T, ii, jj)
    assert rel(u_T, wu) < 1e-5
    assert rel(g_u, wdu) < 1e-4
    assert rel(g_k, wdk) < 1e-4


@pytest.mark.parametrize("dist_name", ["tiles_halo", "block"])
def test_adjoint_staged_and_register_kernels_agree_bit_for_bit(dist_name):
    # the adjoint launch through the cp.async-staged kernel (default) and the
    # register kernel (LT_FLAG_NO_STAGED): same operations, same results;
    # 300 x 520 is ragged against the 32 x 128 tiles and the 4-column groups
    torch = pytest.importorskip("torch")
    from paper_2202_05549_gb300.autograd import DiffusionPlan

    ny, nx, T, ck = 300, 520, 6, 3
    dist, sb = {"tiles_halo": (lt.Dist.tiles((100, 256), halo=(1, 1)), (256, 100)),
                "block": (lt.Dist.block(), (0, 0))}[dist_name]
    u0, k = fields(ny, nx)
    out = []
    for flags in (0, L.LT_FLAG_NO_STAGED):
        with lt.Context(flags=flags) as ctx:
            ctx.log_enable()
            plan = DiffusionPlan(ctx, ny, nx, T, ck, dist, sb)
            plan.K.write(k)
            plan.ck[0].write(u0)
            plan.forward()
            uT = plan.ck[-1].read()
            plan.lam[0].write((2.0 * uT).astype(np.float32))
            lam0 = plan.backward()
            ctx.synchronize()
            variants = {t["variant"] for t in ctx.log() if t["kind"] == "execute"}
            out.append((lam0.read(), plan.G.read(), variants))
    assert 2 in out[0][2] and 2 not in out[1][2]
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    _, du0, dk = oracle.diffusion_grad(u0.astype(np.float64), k.astype(np.float64), T)
    assert rel(out[0][0], du0) < 1e-4 and rel(out[0][1], dk) < 1e-4


def _unfused_grad(u0, kap, T, chunk):
    """Forward and gradient of J = sum u_T^2 as separate element-wise and
    Laplacian launches, every state kept (the unfused form of the step)."""
    n = u0.shape[0]
    with lt.Context() as ctx:
        dist = lt.Dist.tiles((chunk, chunk), halo=(1, 1))
        mk = lambda: ctx.array(lt.F32, (n, n), dist)  # noqa: E731
        K, H, W, G, DK = mk(), mk(), mk(), mk(), mk()
        S = [mk() for _ in range(T + 1)]
        lam = [mk(), mk()]
        K.write(kap)
        S[0].write(u0)
        kl = ctx.kernel(lt.LAPLACE2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write G[i, j]",
                        [("U", lt.F32), ("G", lt.F32)])
        ke = ctx.kernel(lt.EWISE2D, "global [i, j] => read A[i, j], read B[i, j], write C[i, j]",
                        [("A", lt.F32), ("B", lt.F32), ("C", lt.F32), ("op", lt.U32, False)])
        km = ctx.kernel(lt.MULADD2D, "global [i, j] => read A[i, j], read B[i, j], readwrite C[i, j]",
                        [("A", lt.F32), ("B", lt.F32), ("C", lt.F32)])
        g = dict(grid=(n, n), block=(128, 2), superblock=(chunk, chunk))
        for t in range(T):
            kl.launch(**g, args=[S[t], H])
            ke.launch(**g, args=[K, H, W, 1])
            ke.launch(**g, args=[S[t], W, S[t + 1], 0])
        ke.launch(**g, args=[S[T], S[T], lam[0], 0])
        DK.fill(L.LT_INIT_ZERO)
        for t in reversed(range(T)):
            ke.launch(**g, args=[K, lam[0], W, 1])
            kl.launch(**g, args=[W, G])
            ke.launch(**g, args=[lam[0], G, lam[1], 0])
            kl.launch(**g, args=[S[t], H])
            km.launch(**g, args=[lam[0], H, DK])
            lam.reverse()
        ctx.synchronize()
        return S[T].read(), lam[0].read(), DK.read()


def test_unfused_laplace_and_elementwise_launches_match_numpy():
    n = 300
    a = si.uniform_field(2207, 20, n, n)
    b = si.kappa_field(2207, 21, n, n)
    c = si.uniform_field(2207, 22, n, n)
    p = np.pad(a, 1)
    lap = ((((p[:-2, 1:-1] + p[2:, 1:-1]) + p[1:-1, :-2]) + p[1:-1, 2:]) - np.float32(4.0) * a).astype(np.float32)
    with lt.Context() as ctx:
        dist = lt.Dist.tiles((128, 96), halo=(1, 1))
        A, B, C, D = (ctx.array(lt.F32, (n, n), dist) for _ in range(4))
        A.write(a)
        B.write(b)
        C.write(c)
        kl = ctx.kernel(lt.LAPLACE2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write G[i, j]",
                        [("U", lt.F32), ("G", lt.F32)])
        ke = ctx.kernel(lt.EWISE2D, "global [i, j] => read A[i, j], read B[i, j], write C[i, j]",
                        [("A", lt.F32), ("B", lt.F32), ("C", lt.F32), ("op", lt.U32, False)])
        km = ctx.kernel(lt.MULADD2D, "global [i, j] => read A[i, j], read B[i, j], readwrite C[i, j]",
                        [("A", lt.F32), ("B", lt.F32), ("C", lt.F32)])
        g = dict(grid=(n, n), block=(128, 2), superblock=(96, 128))
        kl.launch(**g, args=[A, D])
        ctx.synchronize()
        assert np.array_equal(D.read(), lap)
        ke.launch(**g, args=[A, B, D, 0])
        ctx.synchronize()
        assert np.array_equal(D.read(), a + b)
        ke.launch(**g, args=[A, B, D, 1])
        ctx.synchronize()
        assert np.array_equal(D.read(), a * b)
        km.launch(**g, args=[A, B, C])
        ctx.synchronize()
        assert np.array_equal(C.read(), c + a * b)


def test_unfused_gradient_matches_the_fp64_oracle_and_the_fused_adjoint():
    n, T = 64, 12
    u0 = si.uniform_field(si.SEED_DIFFUSION, si.STREAM_U, n, n)
    kap = si.kappa_field(si.SEED_DIFFUSION, si.STREAM_KAPPA, n, n)
    uT, du, dk = _unfused_grad(u0, kap, T, 32)
    J, du_o, dk_o = oracle.diffusion_grad(u0, kap, T)
    rel = lambda x, y: float(np.linalg.norm(x - y) / np.linalg.norm(y))  # noqa: E731
    assert rel(du, du_o) <= 1e-4 and rel(dk, dk_o) <= 1e-4
    # the forward steps as three launches each round like the fused step: the same states
    with lt.Context() as ctx:
        kf = ctx.kernel(lt.DIFFUSION2D, FWD, [("U", lt.F32), ("K", lt.F32), ("V", lt.F32)])
        dist = lt.Dist.tiles((32, 32), halo=(1, 1))
        U, V, K = (ctx.array(lt.F32, (n, n), dist) for _ in range(3))
        U.write(u0)
        K.write(kap)
        for _ in range(T):
            kf.launch(grid=(n, n), block=(128, 2), superblock=(32, 32), args=[U, K, V])
            U, V = V, U
        ctx.synchronize()
        assert np.array_equal(uT, U.read())
