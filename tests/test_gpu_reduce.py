"""GPU parity of the reduce(f) access mode with every operator, through the
paper's own row-reduction annotation "global [i, j] => read A[i, j],
reduce(f) sum[i]" (Sec. 2.3), against the fp64 oracle: min and max exact,
+ and * within f32 accumulation error.  Partials of superblocks that share
rows are combined in superblock order (deterministic)."""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("op", ["+", "*", "min", "max"])
@pytest.mark.parametrize("adist,sb", [(lt.Dist.block(), (0, 0)), (lt.Dist.tiles((64, 128)), (128, 64)),
                                      (lt.Dist.rows(100), (160, 32)), (lt.Dist.cols(200, halo=2), (96, 48))])
def test_rowreduce_all_ops(op, adist, sb):
    ny, nx = 301, 517
    u = si.uniform_field(2206, 300, ny, nx)
    a = (1.0 + (u - 0.5) * 0.02).astype(np.float32) if op == "*" else (u - 0.5).astype(np.float32)
    want = oracle.rowreduce(a.astype(np.float64), op)
    with lt.Context() as ctx:
        A = ctx.array(lt.F32, (ny, nx), adist)
        S = ctx.array(lt.F32, (ny,), lt.Dist.rows(64))
        A.write(a)
        k = ctx.kernel(lt.ROWREDUCE, f"global [i, j] => read A[i, j], reduce({op}) sum[i]",
                       [("A", lt.F32), ("sum", lt.F32)])
        k.launch(grid=(nx, ny), block=(32, 8), superblock=sb, args=[A, S])
        ctx.synchronize()
        got = S.read().astype(np.float64)
    if op in ("min", "max"):
        assert np.array_equal(got, want)
    elif op == "+":
        # f32 summation error bound: n * eps * sum |a| (rows cancel, so |sum| is no scale)
        scale = np.abs(a.astype(np.float64)).sum(axis=1)
        assert np.all(np.abs(got - want) <= nx * 2.0**-24 * scale)
    else:
        assert np.max(np.abs(got - want) / np.abs(want)) < nx * 2.0**-24
