"""GPU parity of the batched form: many uneven Jacobi launches and
histograms run as one persistent kernel (replayed from a CUDA graph), bit
for bit equal to the CPU oracle and to the same launches issued one by one.
"""
import numpy as np
import pytest

import oracle
import synth_inputs as si
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

pytestmark = pytest.mark.gpu
ANN = "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]"
HANN = "global i => read X[i], reduce(+) H[:]"
SHAPES = [(1, 1), (2, 3), (63, 65), (64, 64), (37, 129), (130, 130), (300, 517), (1024, 768)]
LENS = [1, 15, 16, 4097, 100003, 3 * 65536 + 7]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def make(ctx, reps):
    kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
    kh = ctx.kernel(lt.HIST256, HANN, [("X", lt.U8), ("H", lt.U32)])
    launches, jac, hist = [], [], []
    for q, (ny, nx) in enumerate(SHAPES):
        u0 = si.uniform_field(si.SEED_BATCH, si.STREAM_BATCH_JACOBI0 + q, ny, nx)
        U = ctx.array(lt.F32, (ny, nx))
        V = ctx.array(lt.F32, (ny, nx))
        U.write(u0)
        jac.append((u0, U, V))
        launches.append((kj, (nx, ny), (128, 4), (0, 0), [U, V], reps))
    for h, n in enumerate(LENS + [70000]):
        x = si.u8_array(si.SEED_BATCH, si.STREAM_BATCH_HIST0 + h, n) if h < len(LENS) else np.full(n, 7, np.uint8)
        X = ctx.array(lt.U8, (n,))
        H = ctx.array(lt.U32, (256,))
        X.write(x)
        hist.append((x, X, H))
        launches.append((kh, (n,), (256,), (0,), [X, H], 1))
    return launches, jac, hist


def check(jac, hist, done):
    for u0, U, V in jac:
        a, b = (U, V) if done % 2 == 0 else (V, U)
        assert np.array_equal(a.read(), oracle.jacobi2d(u0, done))          # newest state
        assert np.array_equal(b.read(), oracle.jacobi2d(u0, done - 1))      # the one before
    for x, X, H in hist:
        assert np.array_equal(H.read(), oracle.hist256(x))


@pytest.mark.parametrize("flags", [0, L.LT_BATCH_NO_GRAPH, L.LT_BATCH_PLAIN])
def test_batch_bit_exact_and_replay(flags):
    with lt.Context() as ctx:
        launches, jac, hist = make(ctx, 4)
        ctx.launch_batch(launches, flags)
        ctx.synchronize()
        check(jac, hist, 4)
        ctx.launch_batch(launches, flags)     # same batch again: graph replay
        ctx.synchronize()
        check(jac, hist, 8)
        s = ctx.stats()
        if flags == L.LT_BATCH_PLAIN:
            assert s["batches_plain"] == 2
        else:
            assert s["batches_fused"] == 2 and s["tuned_tile_rows"] in (16, 32, 64, 128)
            if flags == 0:
                assert s["graph_replays"] == 1


def test_batch_replay_skips_the_checks_but_a_changed_launch_is_checked():
    with lt.Context() as ctx:
        launches, jac, hist = make(ctx, 2)
        ctx.launch_batch(launches, 0)
        reused = ctx.stats()["plans_reused"]
        ctx.launch_batch(launches, 0)  # the same batch: its launches were checked already
        ctx.synchronize()
        check(jac, hist, 4)
        assert ctx.stats()["plans_reused"] == reused
        # a kernel whose annotation misses the halo the Jacobi body reads, in
        # superblocks of 8 rows (one superblock would cover the whole array)
        narrow = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i, j], write V[i, j]",
                            [("U", lt.F32), ("V", lt.F32)])
        q = SHAPES.index((37, 129))
        bad = list(launches)
        bad[q] = (narrow, launches[q][1], launches[q][2], (129, 8), launches[q][4], launches[q][5])
        with pytest.raises(lt.LightningError, match="does not contain"):
            ctx.launch_batch(bad, 0)
        ctx.launch_batch(launches, 0)  # checked again, then run
        ctx.synchronize()
        check(jac, hist, 6)


@pytest.mark.parametrize("graph", [0, L.LT_BATCH_NO_GRAPH, L.LT_BATCH_TEST_TILE_COLS])
def test_batch_of_chunked_instances_with_halos_is_fused_and_exact(graph):
    # chunked instances in the device-side queue: row bands, 2-D tiles with
    # halos (superblocks smaller than the chunks, and a ragged edge) next to
    # one-chunk instances and histograms; the batch kernel keeps the halo
    # replicas itself, so every iteration is bit-exact against the oracle
    with lt.Context() as ctx:
        kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        kh = ctx.kernel(lt.HIST256, HANN, [("X", lt.U8), ("H", lt.U32)])
        cases = [((200, 300), lt.Dist.rows(64, halo=1), (300, 64)),
                 ((333, 517), lt.Dist.tiles((128, 256), halo=(1, 1)), (256, 128)),
                 ((512, 1024), lt.Dist.tiles((256, 512), halo=(1, 1)), (256, 128)),
                 ((130, 130), None, (0, 0)),
                 ((100, 2500), lt.Dist.rows(40, halo=1), (2500, 40))]    # parts wider than 1024 columns
        launches, jac = [], []
        for q, ((ny, nx), dist, sb) in enumerate(cases):
            u0 = si.uniform_field(si.SEED_BATCH, si.STREAM_BATCH_JACOBI0 + 50 + q, ny, nx)
            U = ctx.array(lt.F32, (ny, nx), dist)
            V = ctx.array(lt.F32, (ny, nx), dist)
            U.write(u0)
            jac.append((u0, U, V))
            launches.append((kj, (nx, ny), (128, 4), sb, [U, V], 5))
        x = si.u8_array(si.SEED_BATCH, si.STREAM_BATCH_HIST0 + 50, 123457)
        X = ctx.array(lt.U8, (x.size,))
        H = ctx.array(lt.U32, (256,))
        X.write(x)
        launches.append((kh, (x.size,), (256,), (0,), [X, H], 1))
        for rep in range(2):
            ctx.launch_batch(launches, graph)
            ctx.synchronize()
            done = 5 * (rep + 1)
            for u0, U, V in jac:
                assert np.array_equal(V.read(), oracle.jacobi2d(u0, done))      # odd count: the result is in V
                assert np.array_equal(U.read(), oracle.jacobi2d(u0, done - 1))
            assert np.array_equal(H.read(), oracle.hist256(x))
            # the next batch continues from V: the buffers swap roles
            launches = [(k, g, b, sb, [a[1], a[0]] if k is kj else a, r) for (k, g, b, sb, a, r) in launches]
            jac = [(u0, V, U) for (u0, U, V) in jac]
        s = ctx.stats()
        assert s["batches_fused"] == 2 and s["batches_plain"] == 0
        assert s["tuned_tile_cols"] in (0, 1024)
        if graph == L.LT_BATCH_TEST_TILE_COLS:
            assert s["tuned_tile_cols"] == 1024


def test_batch_of_chunked_instances_without_halo_falls_back_to_plain():
    # without a halo every superblock packs its read region first: the plain form
    with lt.Context() as ctx:
        kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        u0 = si.uniform_field(2206, 5, 200, 300)
        U = ctx.array(lt.F32, (200, 300), lt.Dist.rows(64))
        V = ctx.array(lt.F32, (200, 300), lt.Dist.rows(64))
        U.write(u0)
        ctx.launch_batch([(kj, (300, 200), (128, 4), (300, 64), [U, V], 4)])
        ctx.synchronize()
        assert ctx.stats()["batches_plain"] == 1
        assert np.array_equal(U.read(), oracle.jacobi2d(u0, 4))


def test_histogram_plain_launch_reduce_partials():
    # the plain reduce(+) path: superblock partials summed in order
    with lt.Context() as ctx:
        kh = ctx.kernel(lt.HIST256, HANN, [("X", lt.U8), ("H", lt.U32)])
        for n, dist, sb in [(1_000_003, lt.Dist.rows(300_000), (250_000,)), (777, lt.Dist.block(), (100,)),
                            (5_000_000, lt.Dist.rows(1 << 20, halo=5), (0,))]:
            x = si.u8_array(2206, 10001, n)
            X = ctx.array(lt.U8, (n,), dist)
            H = ctx.array(lt.U32, (256,))
            X.write(x)
            kh.launch(grid=(n,), block=(256,), superblock=sb, args=[X, H])
            ctx.synchronize()
            assert np.array_equal(H.read(), oracle.hist256(x))


def test_bounded_wait_expires_reports_timeout_and_context_survives():
    # failure detection without a fault: the queue's first iteration is left
    # out, so every later item's bounded dependency wait runs out (~2 s); the
    # kernel records the error and returns, the host reads LT_ERR_TIMEOUT,
    # and the same context then runs a normal batch correctly
    with lt.Context() as ctx:
        kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        u0 = si.uniform_field(2206, 9, 96, 160)
        U = ctx.array(lt.F32, (96, 160))
        V = ctx.array(lt.F32, (96, 160))
        U.write(u0)
        ctx.launch_batch([(kj, (160, 96), (128, 4), (0, 0), [U, V], 2)], L.LT_BATCH_TEST_STALL)
        with pytest.raises(lt.LightningError) as e:
            ctx.synchronize()
        assert e.value.code == L.LT_ERR_TIMEOUT
        U.write(u0)
        ctx.launch_batch([(kj, (160, 96), (128, 4), (0, 0), [U, V], 2)])
        ctx.synchronize()
        assert np.array_equal(U.read(), oracle.jacobi2d(u0, 2))


def test_batch_full_size_sampled_vs_oracle():
    # the batched configuration at full size, as bench.py builds it: 4096
    # Jacobi instances (sides log-uniform 64..4096, 8 iterations) and 1024
    # histograms (lengths log-uniform 1e4..1e7), one fused batch; 8 instances
    # across the size range and every histogram against the oracle
    r = si.BatchRecipe()
    sides, lens = [int(x) for x in r.sides()], [int(x) for x in r.hist_lengths()]
    with lt.Context() as ctx:
        kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        kh = ctx.kernel(lt.HIST256, HANN, [("X", lt.U8), ("H", lt.U32)])
        launches, Us, Hs = [], [], []
        for q, s_ in enumerate(sides):
            U = ctx.array(lt.F32, (s_, s_))
            V = ctx.array(lt.F32, (s_, s_))
            U.fill(L.LT_INIT_UNIFORM, seed=si.SEED_BATCH, stream=si.STREAM_BATCH_JACOBI0 + q)
            launches.append((kj, (s_, s_), (128, 4), (0, 0), [U, V], r.iters))
            Us.append(U)
        for h, n in enumerate(lens):
            X = ctx.array(lt.U8, (n,))
            H = ctx.array(lt.U32, (256,))
            X.fill(L.LT_INIT_U8, seed=si.SEED_BATCH, stream=si.STREAM_BATCH_HIST0 + h)
            launches.append((kh, (n,), (256,), (0,), [X, H], 1))
            Hs.append(H)
        ctx.launch_batch(launches, 0)
        ctx.synchronize()
        assert ctx.stats()["batches_fused"] == 1
        order = sorted(range(len(sides)), key=lambda q: sides[q])
        pick = sorted({order[0], order[-1]} | {order[len(order) * f // 6] for f in range(1, 6)} | {1})
        got_u = {q: Us[q].read() for q in pick}
        got_h = [H.read() for H in Hs]
    assert r.iters % 2 == 0  # the newest state is back in U
    for q in pick:
        s_ = sides[q]
        u0 = oracle.gen_uniform_f32(si.SEED_BATCH, si.STREAM_BATCH_JACOBI0 + q, 0, s_ * s_).reshape(s_, s_)
        assert np.array_equal(got_u[q], oracle.jacobi2d(u0, r.iters)), f"instance {q} ({s_}^2) differs"
    for h, n in enumerate(lens):
        x = oracle.gen_u8(si.SEED_BATCH, si.STREAM_BATCH_HIST0 + h, 0, n)
        assert np.array_equal(got_h[h], oracle.hist256(x)), f"histogram {h} differs"


def test_batch_special_values_match_the_oracle():
    # the fused kernel's strips on instances where one cell in eight is a
    # zero of either sign, a subnormal, a value whose sums overflow or cancel
    # below 1e-30, an infinity or NaN (any two NaNs count as equal)
    rng = np.random.default_rng(42)
    special = np.array([0.0, -0.0, 1e-40, -1e-42, 1e-35, 3e38, -3e38, np.inf, -np.inf, np.nan, 1e30, 5e-30],
                       dtype=np.float32)
    with lt.Context() as ctx:
        kj = ctx.kernel(lt.JACOBI2D, ANN, [("U", lt.F32), ("V", lt.F32)])
        launches, jac = [], []
        for q, (ny, nx) in enumerate([(63, 65), (130, 130), (300, 517)]):
            u0 = si.uniform_field(si.SEED_BATCH, si.STREAM_BATCH_JACOBI0 + 60 + q, ny, nx)
            mask = rng.random(u0.shape) < 0.125
            u0[mask] = rng.choice(special, size=int(mask.sum()))
            U = ctx.array(lt.F32, (ny, nx))
            V = ctx.array(lt.F32, (ny, nx))
            U.write(u0)
            jac.append((u0, U, V))
            launches.append((kj, (nx, ny), (128, 4), (0, 0), [U, V], 3))
        ctx.launch_batch(launches, 0)
        ctx.synchronize()
        assert ctx.stats()["batches_fused"] == 1
        for u0, U, V in jac:
            with np.errstate(all="ignore"):
                want = oracle.jacobi2d(u0, 3)
            got = V.read()  # three iterations: the newest state is in V
            same = (got.view(np.uint32) == want.view(np.uint32)) | (np.isnan(got) & np.isnan(want))
            assert same.all(), f"{int((~same).sum())} cells differ"
