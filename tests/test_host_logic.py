"""Host logic of the engine, run without a GPU (dry-run contexts).

Covers: the C ABI exports, the annotation parser, access regions against the
oracle's brute-force enumeration, the chunk decisions of the planner
(direct / pack / temp-write / reduce, replica copies), dependency edges
between launches and the memory manager's spill bookkeeping.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2202_05549_gb300 import _lib as L
from paper_2202_05549_gb300 import lightning as lt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def dry(budget=1 << 30, host=0, flags=0):
    return lt.Context(hbm_budget=budget, host_pool=host, flags=L.LT_FLAG_DRYRUN | flags)


# ----------------------------------------------------------------- ABI
def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "lightning.h")).read()
    names = set(re.findall(r"^\s*(?:lt_status|const char \*)\s*(lt_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 18
    lib = C.CDLL(L.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(L.SIGNATURES), names ^ set(L.SIGNATURES)


# ----------------------------------------------------------------- parser
@pytest.mark.parametrize("bad", [
    "global i => read A[i*i]",            # not affine
    "global i => read A[k]",              # unknown variable
    "global i => peek A[i]",              # unknown mode
    "global i => reduce(/) A[i]",         # unknown reduction
    "global i read A[i]",                 # missing arrow
    "global [i, i] => read A[i]",         # bound twice
    "global i => read A[i], write A[i]",  # same array twice
    "global i => read A[i,i,i,i]",        # rank > 3
])
def test_parse_errors(bad):
    with dry() as ctx:
        ctx.array(lt.F32, (10,))
        with pytest.raises(lt.LightningError) as e:
            ctx.kernel(lt.PLAN_ONLY, bad, [("A", lt.F32)])
        assert e.value.code == L.LT_ERR_PARSE


def test_annotation_must_name_every_array():
    with dry() as ctx:
        with pytest.raises(lt.LightningError) as e:
            ctx.kernel(lt.PLAN_ONLY, "global i => read A[i]", [("A", lt.F32), ("B", lt.F32)])
        assert e.value.code == L.LT_ERR_INVALID_ARG


# ----------------------------------------------------------------- regions vs brute force
def _brute(tlo, thi, acc, shape):
    box = [(tlo[d], thi[d]) for d in range(len(tlo))]
    return oracle.access_region_bruteforce(box, acc, shape)


def _region(a):
    r = a["region"]
    return list(zip(r["lo"], r["hi"]))


def test_paper_stencil_regions_and_wrapper_offsets():
    g = {}
    for line in open(os.path.join(GOLDEN, "paper_wrapper_offsets.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(" ", 1)
            g[k] = v.strip()
    n = 1_000_000
    with dry() as ctx:
        out = ctx.array(lt.F32, (n,), lt.Dist.rows(64_000, halo=1))
        inp = ctx.array(lt.F32, (n,), lt.Dist.rows(64_000, halo=1))
        k = ctx.kernel(lt.STENCIL1D, g["annotation"], [("output", lt.F32), ("input", lt.F32)])
        first = int(g["first_thread"])
        # superblocks of `first` threads (blocks of 16), like BlockDist
        plan = k.explain(grid=(n,), block=(16,), superblock=(first,), args=[out, inp])
        sb = plan["superblocks"][1]
        assert sb["threads"]["lo"][0] == first
        a_out, a_in = sb["args"]
        assert a_in["region"]["lo"][0] == int(g["input_offset"])
        assert a_out["region"]["lo"][0] == int(g["output_offset"])
        # every superblock's regions equal the enumeration of its threads
        for sb in plan["superblocks"][:3] + plan["superblocks"][-2:]:
            lo, hi = sb["threads"]["lo"][0], sb["threads"]["hi"][0]
            assert _region(sb["args"][1]) == _brute([lo], [hi], lambda i: [(i - 1,), (i,), (i + 1,)], (n,))
            assert _region(sb["args"][0]) == _brute([lo], [hi], lambda i: [(i,)], (n,))
            assert sb["args"][0]["kind"] == "direct" and sb["args"][1]["kind"] == "direct"


def test_paper_matmul_and_rowsum_regions_vs_bruteforce():
    M, N, K = 12, 10, 7
    with dry() as ctx:
        A = ctx.array(lt.F32, (M, K), lt.Dist.rows(4))
        B = ctx.array(lt.F32, (K, N), lt.Dist.cols(5))
        Cm = ctx.array(lt.F32, (M, N), lt.Dist.tiles((4, 5)))
        k = ctx.kernel(lt.PLAN_ONLY, "global [i, j] => read A[i,:], read B[:,j], write C[i,j]",
                       [("A", lt.F32), ("B", lt.F32), ("C", lt.F32)])
        plan = k.explain(grid=(N, M), block=(5, 4), superblock=(5, 4), args=[A, B, Cm])
        assert len(plan["superblocks"]) == 6
        for sb in plan["superblocks"]:
            (x0, y0, _), (x1, y1, _) = sb["threads"]["lo"], sb["threads"]["hi"]
            # "global [i, j]": j is x (columns), i is y (rows)
            acc_a = lambda i, j: [(i, k2) for k2 in range(K)]
            acc_b = lambda i, j: [(k2, j) for k2 in range(K)]
            acc_c = lambda i, j: [(i, j)]
            assert _region(sb["args"][0]) == _brute([y0, x0], [y1, x1], acc_a, (M, K))
            assert _region(sb["args"][1]) == _brute([y0, x0], [y1, x1], acc_b, (K, N))
            assert _region(sb["args"][2]) == _brute([y0, x0], [y1, x1], acc_c, (M, N))
            assert [a["kind"] for a in sb["args"]] == ["direct", "direct", "direct"]
        S = ctx.array(lt.F32, (M,), lt.Dist.rows(6))
        k2 = ctx.kernel(lt.PLAN_ONLY, "global [i, j] => read A[i,j], reduce(+) sum[i]",
                        [("A", lt.F32), ("sum", lt.F32)])
        plan = k2.explain(grid=(K, M), block=(7, 4), superblock=(7, 4), args=[A, S])
        for sb in plan["superblocks"]:
            (x0, y0, _), (x1, y1, _) = sb["threads"]["lo"], sb["threads"]["hi"]
            assert _region(sb["args"][1]) == _brute([y0, x0], [y1, x1], lambda i, j: [(i,)], (M,))
            assert sb["args"][1]["kind"] == "reduce"


def test_block_and_local_bindings_regions():
    # thread (b, l) of block size 8 touches A[8*b + l - 2 : 8*b + l]
    n = 100
    with dry() as ctx:
        A = ctx.array(lt.F32, (n,), lt.Dist.rows(25))
        k = ctx.kernel(lt.PLAN_ONLY, "block b, local l => read A[8*b + l - 2 : 8*b + l]", [("A", lt.F32)])
        plan = k.explain(grid=(n,), block=(8,), superblock=(24,), args=[A])
        for sb in plan["superblocks"]:
            t0, t1 = sb["threads"]["lo"][0], sb["threads"]["hi"][0]
            want = _brute([t0], [t1], lambda t: [(t + d,) for d in (-2, -1, 0)], (n,))
            assert _region(sb["args"][0]) == want


def test_jacobi_regions_all_superblocks_vs_bruteforce():
    ny, nx = 37, 53
    with dry() as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((16, 16), halo=(1, 1)))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((16, 16), halo=(1, 1)))
        k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])
        plan = k.explain(grid=(nx, ny), block=(8, 4), superblock=(16, 16), args=[U, V])
        assert len(plan["superblocks"]) == 4 * 3
        for sb in plan["superblocks"]:
            (x0, y0, _), (x1, y1, _) = sb["threads"]["lo"], sb["threads"]["hi"]
            acc = lambda i, j: [(i + a, j + b) for a in (-1, 0, 1) for b in (-1, 0, 1)]
            assert _region(sb["args"][0]) == _brute([y0, x0], [min(y1, ny - 1), min(x1, nx - 1)], acc, (ny, nx))
            assert sb["args"][0]["kind"] == "direct"


def test_pack_pieces_partition_the_read_region():
    ny, nx = 40, 40
    with dry() as ctx:
        U = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((10, 10)))   # no halo: reads span chunks
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.tiles((10, 10)))
        k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])
        plan = k.explain(grid=(nx, ny), block=(10, 10), superblock=(10, 10), args=[U, V])
        for sb in plan["superblocks"]:
            a = sb["args"][0]
            assert a["kind"] == "pack"
            reg = np.zeros((ny, nx), np.int32)
            for p in a["pieces"]:
                (r0, c0), (r1, c1) = p["box"]["lo"], p["box"]["hi"]
                reg[r0:r1 + 1, c0:c1 + 1] += 1
            (r0, c0), (r1, c1) = a["region"]["lo"], a["region"]["hi"]
            want = np.zeros_like(reg)
            want[r0:r1 + 1, c0:c1 + 1] = 1
            assert np.array_equal(reg, want)       # exact partition, no double copy
            assert sb["args"][1]["kind"] == "direct" and not sb["args"][1]["replicas"]


def test_replicas_cover_neighbour_halos_exactly():
    ny, nx = 30, 30
    with dry() as ctx:
        dist = lt.Dist.tiles((10, 10), halo=(1, 1))
        U = ctx.array(lt.F32, (ny, nx), dist)
        V = ctx.array(lt.F32, (ny, nx), dist)
        chunks = V.chunks()
        k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])
        plan = k.explain(grid=(nx, ny), block=(10, 10), superblock=(10, 10), args=[U, V])
        # every halo cell of every chunk is refreshed by exactly one replica copy
        copies = {c: np.zeros((ny, nx), np.int32) for c in range(len(chunks))}
        for sb in plan["superblocks"]:
            w = sb["args"][1]
            assert w["kind"] == "direct"
            for r in w["replicas"]:
                (r0, c0), (r1, c1) = r["box"]["lo"], r["box"]["hi"]
                copies[r["chunk"]][r0:r1 + 1, c0:c1 + 1] += 1
        for c, (lo, hi, _) in enumerate(chunks):
            cell = np.zeros((ny, nx), np.int32)
            cell[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1] = 1
            own = np.zeros_like(cell)
            tr, tc = divmod(c, 3)
            own[tr * 10:tr * 10 + 10, tc * 10:tc * 10 + 10] = 1
            assert np.array_equal(copies[c], cell - own), c


def test_annotation_must_contain_the_kernels_accesses():
    with dry() as ctx:
        U = ctx.array(lt.F32, (32, 32), lt.Dist.tiles((16, 16), halo=(1, 1)))
        V = ctx.array(lt.F32, (32, 32), lt.Dist.tiles((16, 16), halo=(1, 1)))
        k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])
        with pytest.raises(lt.LightningError) as e:
            k.launch(grid=(32, 32), block=(16, 16), superblock=(16, 16), args=[U, V])
        assert e.value.code == L.LT_ERR_INVALID_ARG
        with pytest.raises(lt.LightningError):
            ctx.kernel(lt.JACOBI2D, "global [i, j] => write U[i-1:i+1, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])


# ----------------------------------------------------------------- dependencies
def _jacobi_ctx(ctx, ny, nx, dist):
    U = ctx.array(lt.F32, (ny, nx), dist)
    V = ctx.array(lt.F32, (ny, nx), dist)
    k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                   [("U", lt.F32), ("V", lt.F32)])
    return U, V, k


def _ooc_run(discard):
    # 8 row bands of 64 x 1024 f32 per array; the HBM budget holds 6 bands,
    # so both arrays cannot stay resident: 4 launches, then a synchronize
    ny, nx, band = 512, 1024, 64
    cb = (band + 2) * nx * 4
    with dry(budget=6 * cb + 4096, host=16 * cb) as ctx:
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=3)
        ctx.synchronize()
        ctx.reset_stats()
        for _ in range(4):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
            U, V = V, U
        if discard:
            V.discard()  # the last launch's input: stale once U holds the result
        ctx.synchronize()
        s = ctx.stats()
        # the result is still complete: one more launch reads it and
        # overwrites the discarded array
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
        ctx.synchronize()
        return s


def test_discarded_array_is_dropped_not_written_back():
    keep, drop = _ooc_run(False), _ooc_run(True)
    # without the discard the last launch writes back the input bands it
    # evicts to make room for its output; with it they are dropped
    assert drop["bytes_d2h"] < keep["bytes_d2h"]
    assert drop["dead_skips"] > keep["dead_skips"]
    assert drop["bytes_h2d"] == keep["bytes_h2d"]  # the launches read the same inputs


def test_discard_waits_for_the_pending_launch_and_writes_revive():
    # the pending launch still reads the discarded array: its chunks may be
    # dropped only after that launch has used them, and a fill makes them live
    ny, nx, band = 512, 1024, 64
    cb = (band + 2) * nx * 4
    with dry(budget=6 * cb + 4096, host=16 * cb, flags=L.LT_FLAG_FIXED_SWEEP) as ctx:
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=3)
        on_host = ctx.stats()["evictions"]  # U bands the fill moved to host memory
        ctx.reset_stats()
        ctx.log_enable()
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
        U.discard()
        ctx.synchronize()
        log = ctx.log()
        ex = [t for t in log if t["kind"] == "execute"]
        assert len(ex) == 8  # one band per group: every band of U was read
        # U is the context's first array (id 1).  The budget is too small for
        # the launch itself, so bands it still needs are written back and
        # fetched again; a band past its last use is dropped, never written back
        ev = [t for t in log if t["kind"] == "evict" and t.get("array") == 1]
        fe = [t for t in log if t["kind"] == "fetch" and t.get("array") == 1]
        assert on_host > 0 and len(fe) >= on_host
        for t in ev:
            assert any(f["chunk"] == t["chunk"] and f["id"] > t["id"] for f in fe), t
        assert ctx.stats()["dead_skips"] > 0
        U.fill(L.LT_INIT_UNIFORM, seed=4)
        k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
        ctx.synchronize()


def test_dependencies_between_successive_launches():
    with dry(flags=L.LT_FLAG_FIXED_SWEEP) as ctx:
        U, V, k = _jacobi_ctx(ctx, 64, 64, lt.Dist.rows(16, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=1)
        ctx.log_enable()
        k.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[U, V])   # reads U, writes V
        k.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[V, U])   # reads V (RAW), writes U (WAR)
        log = ctx.log()
        ex = [t for t in log if t["kind"] == "execute"]
        un = [t for t in log if t["kind"] == "unpack"]
        # the Jacobi kernel writes the halo replicas of its output itself: no copy step
        assert len(ex) == 2 and not un
        assert ex[0]["replicas"] == 6 and ex[1]["replicas"] == 6  # 4 bands: 3 seams x 2 sides
        l1, l2 = ex[0]["launch"], ex[1]["launch"]
        assert l2 > l1
        # launch 2 must wait for launch 1's writes of V (its outputs and replicas)
        # and its write of U (read by launch 1) must come after launch 1's reads
        assert ex[0]["id"] in ex[1]["deps"]
        s = ctx.stats()
        assert s["bytes_replica_wt"] == 2 * 6 * 64 * 4


def test_replica_copies_remain_for_kernels_that_do_not_write_through():
    # the multi-step stencil keeps the copy step for its k-row halo replicas
    with dry(flags=L.LT_FLAG_FIXED_SWEEP) as ctx:
        dist = lt.Dist.rows(16, halo=2)
        U = ctx.array(lt.F32, (64, 64), dist)
        V = ctx.array(lt.F32, (64, 64), dist)
        U.fill(L.LT_INIT_UNIFORM, seed=1)
        km = ctx.kernel(lt.JACOBI2D_MULTI, "global [i, j] => read U[i-2:i+2, j-2:j+2], write V[i, j]",
                        [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        ctx.log_enable()
        km.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[U, V, 2])
        log = ctx.log()
        ex = [t for t in log if t["kind"] == "execute"]
        un = [t for t in log if t["kind"] == "unpack"]
        assert len(ex) == 1 and ex[0]["replicas"] == 0 and len(un) == 1
        assert un[0]["id"] > ex[0]["id"] and ex[0]["id"] in un[0]["deps"]


def test_write_only_chunks_are_not_fetched_and_spill_roundtrip():
    # 8 row bands of 64 x 1024 f32 (256 KiB each); budget = 6 chunks, host = 16 chunks
    ny, nx = 512, 1024
    band = 64
    cb = (band + 2) * nx * 4
    with dry(budget=6 * cb + 4096, host=16 * cb) as ctx:
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=3)
        s = ctx.stats()
        assert s["evictions"] >= 8 - 6          # filling 8 bands through a 6-band budget spills
        for it in range(4):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        s = ctx.stats()
        assert s["fetches"] > 0 and s["evictions"] > 0
        assert s["dead_skips"] > 0               # output bands are never fetched
        assert s["hbm_peak"] <= 6 * cb + 4096
        assert s["tasks_execute"] == 4 * 8


def test_out_of_memory_is_reported():
    ny, nx, band = 256, 1024, 64
    cb = (band + 2) * nx * 4
    with dry(budget=2 * cb, host=cb) as ctx:       # 2 device slots, 1 host slot: cannot run
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        with pytest.raises(lt.LightningError) as e:
            U.fill(L.LT_INIT_UNIFORM, seed=3)
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
        assert e.value.code in (L.LT_ERR_OOM_HOST, L.LT_ERR_OOM_DEVICE)


def test_alternating_sweep_reuses_resident_chunks():
    ny, nx, band = 1024, 256, 64
    cb = (band + 2) * nx * 4
    res = {}
    # 16 bands per array: the live data (one array) exceeds the 10-chunk budget
    for flags in (0, L.LT_FLAG_FIXED_SWEEP):
        with dry(budget=10 * cb, host=40 * cb, flags=flags) as ctx:
            U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
            U.fill(L.LT_INIT_UNIFORM, seed=3)
            ctx.reset_stats()
            for it in range(6):
                k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
                U, V = V, U
            s = ctx.stats()
            res[flags] = s["bytes_h2d"] + s["bytes_d2h"]
    assert res[0] < res[L.LT_FLAG_FIXED_SWEEP]


def test_reduce_plan_pieces():
    with dry() as ctx:
        X = ctx.array(lt.U8, (1000,), lt.Dist.rows(300))
        H = ctx.array(lt.U32, (256,))
        k = ctx.kernel(lt.PLAN_ONLY, "global i => read X[i], reduce(+) H[:]", [("X", lt.U8), ("H", lt.U32)])
        plan = k.explain(grid=(1000,), block=(100,), superblock=(300,), args=[X, H])
        assert len(plan["superblocks"]) == 4
        for sb in plan["superblocks"]:
            assert sb["args"][1]["kind"] == "reduce"
            assert sb["args"][1]["region"] == {"lo": [0], "hi": [255]}
        ctx.log_enable()
        k.launch(grid=(1000,), block=(100,), superblock=(300,), args=[X, H])
        kinds = [t["kind"] for t in ctx.log()]
        assert kinds.count("reduce") == 1 and "reduce_init" in kinds


def test_lookahead_skips_writeback_of_data_the_next_launch_overwrites():
    # ping-pong Jacobi through a budget of 6 of 16 bands: with one launch of
    # lookahead, bands read in launch t and overwritten unread in t+1 are
    # dropped on eviction instead of written back
    ny, nx, band = 1024, 512, 64
    cb = (band + 2) * nx * 4
    out = {}
    for lookahead in (True, False):
        with dry(budget=6 * cb + 8192, host=30 * cb) as ctx:
            U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
            U.fill(L.LT_INIT_UNIFORM, seed=3)
            ctx.synchronize()
            ctx.reset_stats()
            for it in range(6):
                k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
                U, V = V, U
                if not lookahead:
                    ctx.synchronize()        # flushes each launch before the next is seen
            ctx.synchronize()
            out[lookahead] = ctx.stats()
    assert out[True]["tasks_execute"] == out[False]["tasks_execute"] == 6 * 16
    assert out[True]["bytes_d2h"] < 0.8 * out[False]["bytes_d2h"]
    assert out[True]["bytes_h2d"] <= out[False]["bytes_h2d"]


def test_batch_in_dry_run_is_the_plain_sequence():
    with dry() as ctx:
        U, V, k = _jacobi_ctx(ctx, 64, 64, lt.Dist.block())
        X = ctx.array(lt.U8, (1000,))
        H = ctx.array(lt.U32, (256,))
        kh = ctx.kernel(lt.HIST256, "global i => read X[i], reduce(+) H[:]", [("X", lt.U8), ("H", lt.U32)])
        ctx.log_enable()
        ctx.launch_batch([(k, (64, 64), (64, 4), (0, 0), [U, V], 5), (kh, (1000,), (256,), (0,), [X, H], 1)])
        s = ctx.stats()
        assert s["launches"] == 6 and s["batches_plain"] == 1 and s["batches_fused"] == 0
        ex = [t for t in ctx.log() if t["kind"] == "execute"]
        assert len(ex) == 6
        # iteration t+1 depends on iteration t (ping-pong through U and V)
        for a, b in zip(ex[:4], ex[1:5]):
            assert a["id"] in b["deps"]


def test_prepared_batch_is_the_same_sequence_as_the_list():
    with dry() as ctx:
        U, V, k = _jacobi_ctx(ctx, 64, 64, lt.Dist.block())
        X = ctx.array(lt.U8, (1000,))
        H = ctx.array(lt.U32, (256,))
        kh = ctx.kernel(lt.HIST256, "global i => read X[i], reduce(+) H[:]", [("X", lt.U8), ("H", lt.U32)])
        b = ctx.prepare_batch([(k, (64, 64), (64, 4), (0, 0), [U, V], 3), (kh, (1000,), (256,), (0,), [X, H], 1)])
        assert b.n == 2 and b.descs[0].repeat == 3 and b.descs[1].nargs == 2
        ctx.launch_batch(b)
        ctx.launch_batch(b)
        s = ctx.stats()
        assert s["launches"] == 8 and s["batches_plain"] == 2


def test_multi_step_annotation_must_cover_k_rings():
    with dry() as ctx:
        U = ctx.array(lt.F32, (64, 64), lt.Dist.rows(16, halo=3))
        V = ctx.array(lt.F32, (64, 64), lt.Dist.rows(16, halo=3))
        km = ctx.kernel(lt.JACOBI2D_MULTI, "global [i, j] => read U[i-2:i+2, j-2:j+2], write V[i, j]",
                        [("U", lt.F32), ("V", lt.F32), ("k", lt.U32, False)])
        km.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[U, V, 2])   # k = 2: covered
        with pytest.raises(lt.LightningError) as e:
            km.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[U, V, 3])  # k = 3: not covered
        assert e.value.code == L.LT_ERR_INVALID_ARG
        with pytest.raises(lt.LightningError):
            km.launch(grid=(64, 64), block=(64, 4), superblock=(64, 16), args=[U, V, 0])   # k out of range


def test_plan_cache_reuses_plans_of_the_same_shape_only():
    # the plan depends on grid, block, superblock and the arrays' geometry
    # and aliasing, not on which arrays of that geometry are passed
    with dry() as ctx:
        U, V, k = _jacobi_ctx(ctx, 96, 128, lt.Dist.tiles((32, 64), halo=(1, 1)))
        W = ctx.array(lt.F32, (96, 128), lt.Dist.rows(32, halo=1))
        launch = dict(grid=(128, 96), block=(64, 4), superblock=(64, 32))
        plan_uv = k.explain(args=[U, V], **launch)
        ctx.reset_stats()
        k.launch(args=[U, V], **launch)
        k.launch(args=[V, U], **launch)                 # swapped arrays: same plan
        assert ctx.stats()["plans_reused"] == 2          # both launches hit the cached plan
        assert k.explain(args=[V, U], **launch) == plan_uv
        ctx.reset_stats()
        k.launch(args=[U, W], **launch)                 # other geometry for V
        k.launch(grid=(128, 96), block=(64, 4), superblock=(64, 16), args=[U, V])  # other superblock
        assert ctx.stats()["plans_reused"] == 0
        plan_uw = k.explain(args=[U, W], **launch)
        assert plan_uw != plan_uv
        ctx.synchronize()


def test_plan_cache_keeps_4096_shapes_and_drops_the_least_recent():
    with dry() as ctx:
        A = ctx.array(lt.F32, (8192,), lt.Dist.block())
        B = ctx.array(lt.F32, (8192,), lt.Dist.block())
        k = ctx.kernel(lt.STENCIL1D, "global i => read input[i-1:i+1], write output[i]",
                       [("n", lt.U32, False), ("output", lt.F32), ("input", lt.F32)])
        for g in range(1, 4098):  # 4097 grids: the first one no longer fits
            k.launch(grid=(g,), block=(1,), superblock=(0,), args=[8192, B, A])
        ctx.reset_stats()
        k.launch(grid=(4097,), block=(1,), superblock=(0,), args=[8192, B, A])
        k.launch(grid=(2,), block=(1,), superblock=(0,), args=[8192, B, A])
        assert ctx.stats()["plans_reused"] == 2
        k.launch(grid=(1,), block=(1,), superblock=(0,), args=[8192, B, A])  # dropped: planned again
        assert ctx.stats()["plans_reused"] == 2
        ctx.synchronize()


def test_plan_cache_tells_aliased_arguments_apart():
    # passing one array twice is a different plan input (the dead-data analysis
    # differs), so it must not reuse the plan of two distinct arrays
    with dry() as ctx:
        A = ctx.array(lt.F32, (64,), lt.Dist.rows(16, halo=1))
        B = ctx.array(lt.F32, (64,), lt.Dist.rows(16, halo=1))
        k = ctx.kernel(lt.STENCIL1D, "global i => read input[i-1:i+1], write output[i]",
                       [("n", lt.U32, False), ("output", lt.F32), ("input", lt.F32)])
        ctx.reset_stats()
        k.launch(grid=(64,), block=(16,), superblock=(16,), args=[64, B, A])
        k.launch(grid=(64,), block=(16,), superblock=(16,), args=[64, A, A])
        assert ctx.stats()["plans_reused"] == 0
        k.launch(grid=(64,), block=(16,), superblock=(16,), args=[64, A, B])
        assert ctx.stats()["plans_reused"] == 1
        ctx.synchronize()


def test_eviction_prefers_dead_and_finished_chunks():
    # Two arrays of 16 bands, 20 chunk slots: one array (the live data of an
    # iterative U -> V -> U loop) fits.  With the one-launch lookahead every
    # band a launch has read is dead (the next launch overwrites it), so the
    # steady state moves nothing over the host link.  The last launch, flushed
    # without a successor, must write back what does not fit, but it never
    # evicts an input it has yet to read (no fetches).
    ny, nx, band = 1024, 256, 64
    cb = (band + 2) * nx * 4
    with dry(budget=20 * cb, host=40 * cb) as ctx:
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=3)
        ctx.synchronize()
        ctx.log_enable()
        for it in range(8):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=[U, V])
            U, V = V, U
        ctx.synchronize()
        log = ctx.log()
        launches = sorted({t["launch"] for t in log if t["kind"] == "execute"})
        assert len(launches) == 8
        last = launches[-1]
        moved = [(t["launch"], t["kind"]) for t in log if t["kind"] in ("fetch", "evict")]
        assert all(l == last for l, _ in moved), moved          # nothing in the steady state
        assert not any(kind == "fetch" for _, kind in moved)   # the flush only writes back
        # both arrays are live after the flush: 32 chunks in 20 slots, so exactly 12 go to host
        assert sum(1 for _, kind in moved if kind == "evict") == 32 - 20


def test_reduce_partials_in_place_when_regions_are_chunk_boxes():
    # the adjoint's reduce(+) over a superblock and its ring equals the box of
    # the superblock's own chunk (tiles with a one-cell halo): every partial
    # accumulates in its chunk; a reduce into one small array takes only the
    # first superblock's partial in place
    n, t = 256, 64
    with dry() as ctx:
        dist = lt.Dist.tiles((t, t), halo=(1, 1))
        arrs = [ctx.array(lt.F32, (n, n), dist) for _ in range(5)]
        ka = ctx.kernel(lt.DIFFUSION2D_ADJ, "global [i, j] => read L1[i, j], read K[i, j], read U[i-1:i+1, j-1:j+1], "
                        "readwrite G[i, j], reduce(+) L0[i-1:i+1, j-1:j+1]",
                        [("L1", lt.F32), ("K", lt.F32), ("U", lt.F32), ("G", lt.F32), ("L0", lt.F32)])
        ctx.reset_stats()
        ka.launch(grid=(n, n), block=(64, 2), superblock=(t, t), args=arrs)
        ctx.synchronize()
        assert ctx.stats()["reduce_inplace"] == (n // t) ** 2
        x = ctx.array(lt.U8, (10_000,), lt.Dist.rows(2_500))
        h = ctx.array(lt.U32, (256,), lt.Dist.block())
        kh = ctx.kernel(lt.HIST256, "global i => read X[i], reduce(+) H[:]", [("X", lt.U8), ("H", lt.U32)])
        ctx.reset_stats()
        kh.launch(grid=(10_000,), block=(256,), superblock=(2_500,), args=[x, h])
        ctx.synchronize()
        assert ctx.stats()["reduce_inplace"] == 1


def test_wrapped_device_memory_is_never_moved():
    # a wrapped array's one chunk is the caller's memory: always resident,
    # never evicted (even under a budget that forces the other array to
    # spill), never freed by the library; launches use it directly
    ny, nx = 512, 256
    cb = (64 + 2) * nx * 4
    with dry(budget=6 * cb, host=40 * cb) as ctx:
        fake = 0x7F0000000000  # dry run: never dereferenced
        U = lt.Array(ctx, lt.F32, (ny, nx), None, wrap=(fake, (nx, 1), None))
        V = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(64, halo=1))
        k = ctx.kernel(lt.JACOBI2D, "global [i, j] => read U[i-1:i+1, j-1:j+1], write V[i, j]",
                       [("U", lt.F32), ("V", lt.F32)])
        plan = k.explain(grid=(nx, ny), block=(128, 4), superblock=(nx, 64), args=[U, V])
        assert all(sb["args"][0]["kind"] == "direct" for sb in plan["superblocks"])
        ctx.log_enable()
        for _ in range(3):
            k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, 64), args=[U, V])
        ctx.synchronize()
        u_id = [t for t in ctx.log() if t["kind"] == "execute"]
        assert u_id
        assert not any(t["kind"] in ("evict", "fetch") and t.get("array") == 1 for t in ctx.log())
        U.destroy()
        with pytest.raises(lt.LightningError):
            lt.Array(ctx, lt.F32, (4, 4), None, wrap=(fake, (1, 4), None))  # innermost stride must be 1


def _reduce_then_pressure(discard):
    ny, nx = 256, 1024
    cb = 64 * nx * 4
    with dry(budget=5 * cb, host=16 * cb) as ctx:
        A = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(64))
        B = ctx.array(lt.F32, (ny, nx), lt.Dist.rows(64))
        S = ctx.array(lt.F32, (ny,), lt.Dist.block())
        T = ctx.array(lt.F32, (ny,), lt.Dist.block())
        A.fill(L.LT_INIT_UNIFORM, seed=1)
        S.fill(L.LT_INIT_ZERO)
        if discard:
            S.discard()
        k = ctx.kernel(lt.ROWREDUCE, "global [i, j] => read A[i, j], reduce(+) sum[i]",
                       [("A", lt.F32), ("sum", lt.F32)])
        k.launch(grid=(nx, ny), block=(32, 8), superblock=(nx, 64), args=[A, S])
        ctx.synchronize()
        B.fill(L.LT_INIT_UNIFORM, seed=2)  # needs every slot: A and S must leave HBM
        k.launch(grid=(nx, ny), block=(32, 8), superblock=(nx, 64), args=[B, T])
        ctx.synchronize()
        return ctx.stats()


def test_reduce_into_a_discarded_array_makes_it_live():
    # S is discarded, then a launch reduces into it: from then on it is live,
    # so memory pressure treats it exactly as if it had never been discarded
    # (written back, not dropped)
    a, b = _reduce_then_pressure(False), _reduce_then_pressure(True)
    for key in ("evictions", "dead_skips", "bytes_d2h", "fetches"):
        assert a[key] == b[key], key
    assert a["evictions"] > 0


def test_streaming_plan_of_the_full_out_of_core_grid_fits_its_pools(monkeypatch):
    # the benchmark's streaming regime: the 262144 x 131072 grid (two 128 GiB
    # arrays) through a 64 GiB HBM budget; the pinned pool is sized from the
    # live set (one array plus bands in flight), not from both arrays
    import sys
    import bench
    monkeypatch.setattr(bench, "mem_available", lambda: 209 * 10**9)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "spill"])
    args = bench.parse()
    pl = bench.plan_ooc(args, 1, hbm_gib=64)
    assert pl["host"] < 0.65 * 209 * 10**9 and pl["budget"] < 64 * 2**30
    ny, nx, band = pl["ny"], pl["nx"], pl["band"]
    with dry(budget=pl["budget"], host=pl["host"]) as ctx:
        U, V, k = _jacobi_ctx(ctx, ny, nx, lt.Dist.rows(band, halo=1))
        U.fill(L.LT_INIT_UNIFORM, seed=3)
        bufs = [U, V]
        for _ in range(2):
            for _ in range(20):
                k.launch(grid=(nx, ny), block=(128, 4), superblock=(nx, band), args=bufs)
                bufs.reverse()
            bufs[1].discard()
            ctx.synchronize()
        s = ctx.stats()
        assert s["fetches"] > 0 and s["evictions"] > 0
        assert s["hbm_peak"] <= pl["budget"]
        assert s["tasks_execute"] == 2 * 20 * (ny // band)


def test_async_host_copies_order_overlapping_host_regions():
    # lt_array_write_async reads a chunk's whole box (halo rows included) from
    # the buffer, lt_array_read_async writes the chunk's owned rows into it:
    # a write of band b waits for the reads of bands b-1..b+1 (their owned
    # rows lie in its box) and a read of band b for the earlier writes of
    # b-1..b+1; copies run on the H2D / D2H streams (dry run: no device)
    import numpy as np
    with lt.Context(hbm_budget=1 << 30, flags=L.LT_FLAG_DRYRUN) as ctx:
        ctx.log_enable()
        U = ctx.array(lt.F32, (64, 32), lt.Dist.rows(16, halo=1))
        h = np.zeros((64, 32), np.float32)
        U.write_async(h)
        U.read_async(h)
        U.write_async(h)
        ctx.synchronize()
        log = ctx.log()
    w1 = [t for t in log if t["kind"] == "write" and t["launch"] == 1]
    rd = [t for t in log if t["kind"] == "read"]
    w2 = [t for t in log if t["kind"] == "write" and t["launch"] == 2]
    assert len(w1) == len(rd) == len(w2) == 4
    assert {t["stream"] for t in w1 + w2} == {1} and {t["stream"] for t in rd} == {2}
    # fences keep the newest operation per stream: the newest overlapping one
    for b in range(4):
        assert rd[b]["deps"] == [w1[min(b + 1, 3)]["id"]]
        assert w2[b]["deps"] == [w1[b]["id"], rd[min(b + 1, 3)]["id"]]
