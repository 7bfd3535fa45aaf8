"""GPU parity of the tcgen05 BF16 GEMM built-in (annotation
"global [i, j] => read A[i, :], read B[:, j], write C[i, j]") against the
fp64 oracle.  Bar (the benchmark spec): <= 1e-2 relative Frobenius error against
fp64 of the unrounded inputs; against fp64 of the bf16-rounded inputs only
the f32 accumulation differs, checked at <= 1e-4.
"""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu
ANN = "global [i, j] => read A[i, :], read B[:, j], write C[i, j]"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def bf16_inputs(M, N, K, seed=si.SEED_GEMM, scale=None):
    scale = scale if scale is not None else 1.0 / np.sqrt(K)
    a = si.gen_normal_bf16_bits(seed, si.STREAM_A, np.arange(M * K), scale).reshape(M, K)
    b = si.gen_normal_bf16_bits(seed, si.STREAM_B, np.arange(K * N), scale).reshape(K, N)
    return a, b, scale


def relfro(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def run_gemm(ctx, a_bits, b_bits, adist, bdist, cdist, sb, fill=None):
    M, K = a_bits.shape
    N = b_bits.shape[1]
    A = ctx.array(lt.BF16, (M, K), adist)
    B = ctx.array(lt.BF16, (K, N), bdist)
    Cm = ctx.array(lt.F32, (M, N), cdist)
    A.write(a_bits)
    B.write(b_bits)
    k = ctx.kernel(lt.GEMM_BF16, ANN, [("A", lt.BF16), ("B", lt.BF16), ("C", lt.F32)])
    k.launch(grid=(N, M), block=(256, 1), superblock=sb, args=[A, B, Cm])
    ctx.synchronize()
    return Cm.read()


@pytest.mark.parametrize("M,N,K,ch", [(512, 512, 512, (256, 256)), (256, 768, 1024, (128, 256)),
                                      (300, 520, 200, (150, 260)), (129, 257, 72, (129, 257))])
def test_gemm_small_and_ragged_vs_fp64(M, N, K, ch):
    a, b, _ = bf16_inputs(M, N, K)
    af = si.bf16_bits_to_f32(a).astype(np.float64)
    bf = si.bf16_bits_to_f32(b).astype(np.float64)
    ref = oracle.gemm_f64(af, bf)
    with lt.Context() as ctx:
        got = run_gemm(ctx, a, b, lt.Dist.rows(ch[0]), lt.Dist.cols(ch[1], order=L.LT_ORDER_COL),
                       lt.Dist.tiles(ch), (ch[1], ch[0]))
    err = relfro(got.astype(np.float64), ref)
    assert err < 1e-5, err
    # elementwise: f32 accumulation bound
    bound = 1e-5 * (np.abs(af) @ np.abs(bf)) + 1e-30
    assert np.all(np.abs(got - ref) <= bound)


def test_gemm_identity_and_unsupported_layout():
    M = K = N = 256
    a, _, _ = bf16_inputs(M, N, K)
    eye = np.zeros((K, N), np.uint16)
    eye[np.arange(K), np.arange(N)] = 0x3F80          # bf16 1.0
    with lt.Context() as ctx:
        got = run_gemm(ctx, a, eye, lt.Dist.rows(128), lt.Dist.cols(256, order=L.LT_ORDER_COL),
                       lt.Dist.tiles((128, 256)), (256, 128))
        assert np.array_equal(got, si.bf16_bits_to_f32(a))   # exact: one nonzero product per entry
        A = ctx.array(lt.BF16, (M, K), lt.Dist.rows(128))
        B = ctx.array(lt.BF16, (K, N), lt.Dist.cols(256))    # row-major B: not K-contiguous
        Cm = ctx.array(lt.F32, (M, N), lt.Dist.tiles((128, 256)))
        k = ctx.kernel(lt.GEMM_BF16, ANN, [("A", lt.BF16), ("B", lt.BF16), ("C", lt.F32)])
        with pytest.raises(lt.LightningError) as e:
            k.launch(grid=(N, M), block=(256, 1), superblock=(256, 128), args=[A, B, Cm])
            ctx.synchronize()
        assert e.value.code == L.LT_ERR_UNSUPPORTED


def test_gemm_full_size_sampled_vs_fp64():
    M = N = K = 65536
    T = 8192
    scale = 1.0 / 256
    with lt.Context() as ctx:
        A = ctx.array(lt.BF16, (M, K), lt.Dist.rows(T))
        B = ctx.array(lt.BF16, (K, N), lt.Dist.cols(T, order=L.LT_ORDER_COL))
        Cm = ctx.array(lt.F32, (M, N), lt.Dist.tiles((T, T)))
        A.fill(L.LT_INIT_NORMAL_BF16, seed=si.SEED_GEMM, stream=si.STREAM_A, scale=scale)
        B.fill(L.LT_INIT_NORMAL_BF16, seed=si.SEED_GEMM, stream=si.STREAM_B, scale=scale)
        k = ctx.kernel(lt.GEMM_BF16, ANN, [("A", lt.BF16), ("B", lt.BF16), ("C", lt.F32)])
        k.launch(grid=(N, M), block=(256, 1), superblock=(T, T), args=[A, B, Cm])
        ctx.synchronize()
        rows, cols = si.sample_cells(2205, M, N, 32)
        rows = np.unique(np.concatenate([rows, [0, M - 1]]))[:32]
        cols = np.unique(np.concatenate([cols, [0, N - 1]]))[:32]
        got = np.stack([Cm.read_box((r, 0), (r, N - 1))[0][cols] for r in rows]).astype(np.float64)
    ref_r, ref_u = oracle.gemm_sample(M, N, K, si.SEED_GEMM, si.STREAM_A, si.STREAM_B, scale, rows, cols)
    assert relfro(got, ref_u) < 1e-2
    assert relfro(got, ref_r) < 1e-4
