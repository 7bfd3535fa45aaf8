"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties one oracle function to a published value, a closed form, an
invariant, a brute-force enumeration or an independent library routine, so
that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ inputs
# SplitMix64 seeded with 1234567: the first five outputs as published with
# the reference implementation of the generator (Steele, Lea & Flood 2014;
# the same sequence is used as a test vector by common PRNG libraries).
SPLITMIX_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                    4593380528125082431, 16408922859458223821]


def test_splitmix64_published_vector_oracle():
    st = 1234567
    got = []
    for _ in range(5):
        x, st = oracle.splitmix64_next(st)
        got.append(x)
    assert got == SPLITMIX_1234567


def test_splitmix64_published_vector_inputs_module():
    assert si.splitmix64_sequence(1234567, 5) == SPLITMIX_1234567


def test_counter_form_equals_sequential_form():
    # element idx of a stream is the (idx+1)-th sequential output from its key
    key = si.stream_key(2203, 0)
    seq = si.splitmix64_sequence(key, 6)
    assert list(oracle.gen_u64(2203, 0, 0, 6)) == seq
    assert list(si.gen_u64(2203, 0, np.arange(6))) == seq


@pytest.mark.parametrize("seed,stream", [(2203, 0), (2207, 1), (2206, 10017)])
def test_oracle_and_input_module_generators_agree(seed, stream):
    idx0, n = 123456789, 4099
    idx = np.arange(idx0, idx0 + n, dtype=np.uint64)
    assert np.array_equal(oracle.gen_u64(seed, stream, idx0, n), si.gen_u64(seed, stream, idx))
    assert np.array_equal(oracle.gen_uniform_f32(seed, stream, idx0, n), si.gen_uniform_f32(seed, stream, idx))
    assert np.array_equal(oracle.gen_u8(seed, stream, idx0, n), si.gen_u8(seed, stream, idx))
    assert np.array_equal(oracle.gen_kappa_f32(seed, stream, idx0, n), si.gen_kappa_f32(seed, stream, idx))
    a = oracle.gen_normal_bf16_bits(seed, stream, idx0, n, 1.0 / 256)
    b = si.gen_normal_bf16_bits(seed, stream, idx, 1.0 / 256)
    assert np.array_equal(a, b)


def test_uniform_is_exact_24bit_grid_in_unit_interval():
    u = oracle.gen_uniform_f32(2204, 0, 0, 1 << 16).astype(np.float64)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2**24 == np.floor(u * 2**24))
    assert abs(u.mean() - 0.5) < 0.01


def test_normal_moments_and_bf16_representable():
    bits = oracle.gen_normal_bf16_bits(2205, 0, 0, 1 << 18, 1.0)
    z = si.bf16_bits_to_f32(bits).astype(np.float64)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.02
    assert abs(np.mean(np.abs(z) < 1.0) - 0.6827) < 0.01


def test_kappa_range():
    k = oracle.gen_kappa_f32(2207, 1, 0, 1 << 16)
    assert k.min() >= np.float32(0.05) and k.max() <= np.float32(0.2)


def test_batch_recipe_means():
    r = si.BatchRecipe()
    s = r.sides()
    assert s.min() >= 64 and s.max() <= 4096 and s.size == 4096
    assert abs(np.mean(s.astype(np.float64) ** 2) / si.expected_batch_cells() - 1) < 0.08
    assert abs(np.mean(s <= 256) - 1 / 3) < 0.04
    L = r.hist_lengths()
    assert L.min() >= 10_000 and L.max() <= 10_000_000


# ------------------------------------------------------------------ 1-D worked example
def test_paper_1d_stencil_first_step_by_hand():
    # Listing 1 on ones: the ends see one zero ghost, (1+1+0)/3.0 = 2/3
    x = np.ones(8, np.float32)
    y = oracle.stencil1d_paper(x)
    assert y[0] == np.float32(2.0 / 3.0) and y[-1] == np.float32(2.0 / 3.0)
    assert np.all(y[1:-1] == 1.0)
    assert oracle.stencil1d_paper(np.array([3.0], np.float32))[0] == np.float32(1.0)


def test_paper_1d_stencil_ten_launches_vs_exact_rationals():
    # host code of Sec. 3.6: ones input, ten launches with swap
    n = 7
    x = np.ones(n, np.float32)
    ex = [Fraction(1)] * n
    for _ in range(10):
        x = oracle.stencil1d_paper(x)
        ex = [((ex[i - 1] if i else 0) + ex[i] + (ex[i + 1] if i + 1 < n else 0)) / 3 for i in range(n)]
    assert np.allclose(x, [float(v) for v in ex], rtol=2e-6, atol=0)


# ------------------------------------------------------------------ 2-D Jacobi
def test_jacobi_brute_force_tiny_grids():
    # 1x1: (u + 4 zero ghosts)/5
    assert oracle.jacobi2d(np.array([[2.5]], np.float32), 1)[0, 0] == np.float32(0.5)
    # 1x3 [1,2,3]: (1+2)/5, (2+1+3)/5, (3+2)/5
    got = oracle.jacobi2d(np.array([[1, 2, 3]], np.float32), 1)[0]
    assert list(got) == [np.float32(3 / 5), np.float32(6 / 5), np.float32(1.0)]
    # 3x3 with a single 5 in the middle: a plus shape of ones
    u = np.zeros((3, 3), np.float32)
    u[1, 1] = 5
    want = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], np.float32)
    assert np.array_equal(oracle.jacobi2d(u, 1), want)
    # 2x3 corner: only two real neighbours
    u = np.arange(6, dtype=np.float32).reshape(2, 3)
    got = oracle.jacobi2d(u, 1)
    assert got[0, 0] == np.float32((0 + 3 + 1) / 5)
    assert got[1, 2] == np.float32((5 + 2 + 4) / 5)
    assert got[0, 1] == np.float32((1 + 4 + 0 + 2) / 5)



def test_jacobi_f32_sum_order_is_centre_north_south_west_east():
    # The sum order ((((c + n) + s) + w) + e) / 5 in f32, pinned by values
    # whose rounded sums depend on it (worked by hand): c = 2^24, n = s = 1,
    # w = -2^24, e = 0.5.  In that order c + n = 2^24 + 1 is a tie and rounds
    # to the even 2^24, so does (c + n) + s, + w gives 0 and + e gives 0.5:
    # the centre becomes 0.5f / 5 = f32(0.1).  Summing n + s first would give
    # 2 + 2^24 (exact), then 2, 2.5 and 0.5; any order that adds w to c before
    # n and s gives 2.5 as well.
    u = np.zeros((3, 3), np.float32)
    u[1, 1] = 2.0 ** 24
    u[0, 1] = u[2, 1] = 1.0
    u[1, 0] = -(2.0 ** 24)
    u[1, 2] = 0.5
    got = oracle.jacobi2d(u, 1)
    assert got[1, 1] == np.float32(0.1)
    assert got[1, 1] != np.float32(0.5)

def _sine_mode(ny, nx, k, l):
    i = np.arange(ny)[:, None]
    j = np.arange(nx)[None, :]
    return np.sin(np.pi * k * (i + 1) / (ny + 1)) * np.sin(np.pi * l * (j + 1) / (nx + 1))


@pytest.mark.parametrize("ny,nx,k,l,T", [(13, 17, 2, 3, 7), (9, 6, 1, 5, 12)])
def test_jacobi_sine_modes_closed_form(ny, nx, k, l, T):
    mode = _sine_mode(ny, nx, k, l)
    lam = (1 + 2 * math.cos(math.pi * k / (ny + 1)) + 2 * math.cos(math.pi * l / (nx + 1))) / 5
    p = np.zeros((ny + 2, nx + 2))
    p[1:-1, 1:-1] = mode
    got = oracle.jacobi2d_ring_f64(p, T)[1:-1, 1:-1]
    assert np.max(np.abs(got - lam**T * mode)) < 1e-12
    # the f32 product-semantics function follows the same mode
    g32 = oracle.jacobi2d(mode.astype(np.float32), T).astype(np.float64)
    assert np.max(np.abs(g32 - lam**T * mode)) < 2e-6


def test_jacobi_constant_ghost_steady_state():
    c = 0.75
    p = np.full((10, 10), c)
    p[1:-1, 1:-1] = np.random.default_rng(0).random((8, 8))
    got = oracle.jacobi2d_ring_f64(p, 900)
    assert np.max(np.abs(got - c)) < 1e-10


def test_jacobi_linear_field_is_fixed_point():
    i = np.arange(12)[:, None]
    j = np.arange(9)[None, :]
    p = 0.5 * i - 0.25 * j + 3.0
    got = oracle.jacobi2d_ring_f64(p, 5)
    assert np.array_equal(got, p)


def test_jacobi_periodic_conserves_sum():
    p = np.zeros((18, 22))
    p[1:-1, 1:-1] = np.random.default_rng(1).random((16, 20))
    s0 = p[1:-1, 1:-1].sum()
    got = oracle.jacobi2d_ring_f64(p, 25, periodic=True)
    assert abs(got[1:-1, 1:-1].sum() - s0) / s0 < 1e-12


def test_jacobi_f32_agrees_with_f64_on_random_data():
    u = si.uniform_field(2203, 0, 37, 53)
    p = np.zeros((39, 55))
    p[1:-1, 1:-1] = u
    r64 = oracle.jacobi2d_ring_f64(p, 10)[1:-1, 1:-1]
    r32 = oracle.jacobi2d(u, 10).astype(np.float64)
    assert np.max(np.abs(r32 - r64)) < 1e-6


def test_jacobi_lightcone_equals_full_run():
    NY, NX, T = 40, 52, 5
    full = oracle.jacobi2d(si.uniform_field(2204, 0, NY, NX), T)
    ii, jj = np.meshgrid(np.arange(NY), np.arange(NX), indexing="ij")
    got = oracle.jacobi2d_lightcone(NY, NX, 2204, 0, T, ii.ravel(), jj.ravel())
    assert np.array_equal(got.reshape(NY, NX), full)


def test_jacobi3d_lightcone_equals_full_run():
    shape, T = (9, 11, 13), 3
    idx = np.arange(9 * 11 * 13, dtype=np.uint64)
    full = oracle.jacobi3d(si.gen_uniform_f32(2208, 0, idx).reshape(shape), T)
    kk, ii, jj = np.meshgrid(*[np.arange(e) for e in shape], indexing="ij")
    got = oracle.jacobi3d_lightcone(shape, 2208, 0, T, kk.ravel(), ii.ravel(), jj.ravel())
    assert np.array_equal(got.reshape(shape), full)


def test_jacobi3d_sine_mode_closed_form_and_f32():
    nz, ny, nx, T = 5, 7, 9, 6
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    a, b, c = 1, 2, 3
    mode = (np.sin(np.pi * a * (z + 1) / (nz + 1)) * np.sin(np.pi * b * (y + 1) / (ny + 1))
            * np.sin(np.pi * c * (x + 1) / (nx + 1)))
    lam = (1 + 2 * math.cos(math.pi * a / (nz + 1)) + 2 * math.cos(math.pi * b / (ny + 1))
           + 2 * math.cos(math.pi * c / (nx + 1))) / 7
    assert np.max(np.abs(oracle.jacobi3d_f64(mode, T) - lam**T * mode)) < 1e-12
    g32 = oracle.jacobi3d(mode.astype(np.float32), T).astype(np.float64)
    assert np.max(np.abs(g32 - lam**T * mode)) < 2e-6


# ------------------------------------------------------------------ GEMM
def test_gemm_f64_matches_library_and_exact_cases():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((33, 47))
    B = rng.standard_normal((47, 29))
    assert np.allclose(oracle.gemm_f64(A, B), A @ B, rtol=1e-12, atol=1e-12)
    # identity and permutation are exact
    assert np.array_equal(oracle.gemm_f64(A, np.eye(47)), A)
    P = np.eye(47)[rng.permutation(47)]
    assert np.array_equal(oracle.gemm_f64(A, P), A @ P)
    # K = 1: outer product, exact
    u = rng.standard_normal((20, 1))
    v = rng.standard_normal((1, 30))
    assert np.array_equal(oracle.gemm_f64(u, v), u * v)


def test_gemm_sample_matches_full_product_at_256():
    M = N = K = 256
    scale = 1.0 / 16
    A = si.bf16_bits_to_f32(si.gen_normal_bf16_bits(2205, 0, np.arange(M * K), scale)).reshape(M, K)
    B = si.bf16_bits_to_f32(si.gen_normal_bf16_bits(2205, 1, np.arange(K * N), scale)).reshape(K, N)
    full = A.astype(np.float64) @ B.astype(np.float64)
    rows = np.array([0, 17, 128, 255])
    cols = np.array([0, 3, 200, 254, 255])
    cr, cu = oracle.gemm_sample(M, N, K, 2205, 0, 1, scale, rows, cols)
    assert np.allclose(cr, full[np.ix_(rows, cols)], rtol=1e-12, atol=1e-14)
    # unrounded inputs differ from bf16-rounded ones by ~2^-9 relative
    rel = np.linalg.norm(cu - cr) / np.linalg.norm(cu)
    assert 1e-4 < rel < 1e-2


# ------------------------------------------------------------------ histogram
def test_hist256_invariants_and_library():
    x = si.u8_array(2206, 10000, 100_003)
    h = oracle.hist256(x)
    assert int(h.sum()) == x.size
    assert np.array_equal(h, np.bincount(x, minlength=256).astype(np.uint32))
    c = np.full(5000, 201, np.uint8)
    hc = oracle.hist256(c)
    assert hc[201] == 5000 and hc.sum() == 5000
    assert oracle.hist256(np.zeros(0, np.uint8)).sum() == 0
    tiny = np.array([0, 255, 255, 7], np.uint8)
    ht = oracle.hist256(tiny)
    assert ht[0] == 1 and ht[255] == 2 and ht[7] == 1 and ht.sum() == 4


# ------------------------------------------------------------------ diffusion and adjoint
def _diff_fields(n, m, seed=2207):
    u0 = si.uniform_field(seed, 0, n, m).astype(np.float64)
    k = si.kappa_field(seed, 1, n, m).astype(np.float64)
    return u0, k


def test_diffusion_gradient_u0_central_differences_exact():
    u0, k = _diff_fields(12, 10)
    T = 6
    J, du0, dk = oracle.diffusion_grad(u0, k, T)
    assert abs(J - np.sum(oracle.diffusion_forward(u0, k, T) ** 2)) < 1e-12 * J
    # J is quadratic in u0: central differences are exact up to rounding
    for (i, j) in [(0, 0), (5, 4), (11, 9), (3, 9)]:
        h = 1e-3
        up = u0.copy(); up[i, j] += h
        dn = u0.copy(); dn[i, j] -= h
        fd = (np.sum(oracle.diffusion_forward(up, k, T) ** 2)
              - np.sum(oracle.diffusion_forward(dn, k, T) ** 2)) / (2 * h)
        assert abs(fd - du0[i, j]) < 1e-9 * max(1.0, abs(du0[i, j]))


def test_diffusion_gradient_kappa_central_differences():
    u0, k = _diff_fields(9, 11)
    T = 5
    J, du0, dk = oracle.diffusion_grad(u0, k, T)
    for (i, j) in [(0, 0), (4, 5), (8, 10), (2, 7)]:
        h = 1e-6
        kp = k.copy(); kp[i, j] += h
        km = k.copy(); km[i, j] -= h
        fd = (np.sum(oracle.diffusion_forward(u0, kp, T) ** 2)
              - np.sum(oracle.diffusion_forward(u0, km, T) ** 2)) / (2 * h)
        assert abs(fd - dk[i, j]) < 1e-6 * max(1.0, abs(dk[i, j]))


def test_diffusion_constant_kappa_sine_mode_closed_form():
    ny, nx, kk, ll, T, c = 14, 11, 3, 2, 9, 0.13
    v = _sine_mode(ny, nx, kk, ll)
    sk = math.sin(math.pi * kk / (2 * (ny + 1))) ** 2
    sl = math.sin(math.pi * ll / (2 * (nx + 1))) ** 2
    mu = 1 - 4 * c * (sk + sl)
    J, du0, dk = oracle.diffusion_grad(v, np.full((ny, nx), c), T)
    nv2 = float(np.sum(v * v))
    assert abs(J - mu ** (2 * T) * nv2) < 1e-12 * nv2
    assert np.max(np.abs(du0 - 2 * mu ** (2 * T) * v)) < 1e-12
    dmu = -4 * (sk + sl)
    assert abs(dk.sum() - 2 * T * mu ** (2 * T - 1) * dmu * nv2) < 1e-10 * nv2


def test_diffusion_lightcone_equals_full_run():
    NY, NX, T = 30, 26, 4
    u0, k = _diff_fields(NY, NX)
    J, du0, dk = oracle.diffusion_grad(u0, k, T)
    uT = oracle.diffusion_forward(u0, k, T)
    ii, jj = np.meshgrid(np.arange(NY), np.arange(NX), indexing="ij")
    a, b, c = oracle.diffusion_lightcone(NY, NX, 2207, 0, 1, T, ii.ravel(), jj.ravel())
    assert np.allclose(a.reshape(NY, NX), uT, rtol=1e-13, atol=1e-15)
    assert np.allclose(b.reshape(NY, NX), du0, rtol=1e-12, atol=1e-14)
    assert np.allclose(c.reshape(NY, NX), dk, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ planner regions
def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split(" ", 1)
            vals[key] = val.strip()
    return vals


def test_region_bruteforce_reproduces_paper_wrapper_offsets():
    g = _read_golden("paper_wrapper_offsets.txt")
    first = int(g["first_thread"])
    n = 1_000_000
    box = [(first, first + 63)]       # a few threads suffice for the lower bounds
    rin = oracle.access_region_bruteforce(box, lambda i: [(i - 1,), (i,), (i + 1,)], (n,))
    rout = oracle.access_region_bruteforce(box, lambda i: [(i,)], (n,))
    assert rin[0][0] == int(g["input_offset"])
    assert rout[0][0] == int(g["output_offset"])


def test_region_bruteforce_clips_to_domain():
    r = oracle.access_region_bruteforce([(0, 3), (0, 3)],
                                        lambda i, j: [(i + a, j + b) for a in (-1, 0, 1) for b in (-1, 0, 1)],
                                        (4, 10))
    assert r == [(0, 3), (0, 4)]


# ------------------------------------------------------------------ row reduction (reduce modes)
def test_rowreduce_closed_forms_and_brute_force():
    c = np.full((3, 7), 1.5)
    assert np.allclose(oracle.rowreduce(c, "+"), 10.5)
    assert np.allclose(oracle.rowreduce(c, "*"), 1.5 ** 7)
    assert np.array_equal(oracle.rowreduce(c, "min"), [1.5] * 3)
    a = np.array([[3.0, -1.0, 4.0, 1.0], [-5.0, 9.0, 2.0, -6.0]])
    assert list(oracle.rowreduce(a, "+")) == [7.0, 0.0]
    assert list(oracle.rowreduce(a, "*")) == [-12.0, 540.0]
    assert list(oracle.rowreduce(a, "min")) == [-1.0, -6.0]
    assert list(oracle.rowreduce(a, "max")) == [4.0, 9.0]
    one = np.array([[2.5], [-0.5]])
    for op in ("+", "*", "min", "max"):
        assert list(oracle.rowreduce(one, op)) == [2.5, -0.5]


# ------------------------------------------------------------------ K-Means
def test_kmeans_constructed_clusters_exact_means():
    # three well separated centres; every record is its centre plus an offset
    # that is a multiple of 2^-10 below 0.1, so the labels are known by
    # construction and the new centres are exact rational means rounded to f32
    rng = np.random.default_rng(11)
    true_c = np.array([[1, 1, 1, 1], [5, 1, 1, 1], [1, 5, 5, 1]], np.float32)
    n = 300
    lab_true = rng.integers(0, 3, n)
    off = rng.integers(-100, 101, (n, 4)) / 1024.0
    x = (true_c[lab_true] + off).astype(np.float32)
    start = true_c + np.float32(0.25)
    s, lab = oracle.kmeans_assign(x, start)
    assert np.array_equal(lab, lab_true)
    for j in range(3):
        members = x[lab_true == j].astype(np.float64)
        assert s[j, 4] == len(members)
        for f in range(4):
            exact = sum(Fraction(float(v)) for v in members[:, f])
            assert Fraction(s[j, f]) == exact                     # fp64 sums of 2^-10 multiples are exact
    c1 = oracle.kmeans_update(s, start)
    for j in range(3):
        members = x[lab_true == j]
        for f in range(4):
            mean = sum(Fraction(float(v)) for v in members[:, f]) / len(members)
            assert c1[j, f] == np.float32(float(mean))


def test_kmeans_ties_go_to_the_lowest_centre():
    x = np.zeros((1, 4), np.float32)
    c = np.array([[2, 0, 0, 0], [-1, 0, 0, 0], [1, 0, 0, 0]], np.float32)  # centres 1 and 2 equidistant
    s, lab = oracle.kmeans_assign(x, c)
    assert lab[0] == 1 and s[1, 4] == 1 and s[0, 4] == 0 and s[2, 4] == 0


def test_kmeans_invariants_and_optimal_assignment():
    # uniform features (multiples of 2^-24 in [0, 1)): counts add up to n, the
    # sums are conserved exactly, and each record's centre is nearest in fp64
    # up to f32 rounding of the distances
    n, k = 5000, 40
    x = si.uniform_field(2209, 0, n, 4)
    c = x[:k].copy()
    s, lab = oracle.kmeans_assign(x, c)
    assert s[:, 4].sum() == n and np.array_equal(np.bincount(lab, minlength=k), s[:, 4].astype(np.int64))
    for f in range(4):
        assert math.fsum(s[:, f]) == math.fsum(x[:, f].astype(np.float64))
    d = ((x.astype(np.float64)[:, None, :] - c.astype(np.float64)[None, :, :]) ** 2).sum(axis=2)
    chosen = d[np.arange(n), lab]
    assert np.all(chosen <= d.min(axis=1) * (1 + 4 * 2.0**-23) + 1e-12)


def test_kmeans_lloyd_objective_never_increases_and_empty_cluster_keeps_centre():
    n, k = 4000, 12
    x = si.uniform_field(2209, 1, n, 4)
    c = x[:k].copy()
    c[-1] = 50.0  # no record comes near this centre
    prev = math.inf
    for _ in range(6):
        s, lab = oracle.kmeans_assign(x, c)
        obj = float(((x.astype(np.float64) - c.astype(np.float64)[lab]) ** 2).sum())
        assert obj <= prev * (1 + 1e-6)
        prev = obj
        assert s[k - 1, 4] == 0
        c_new = oracle.kmeans_update(s, c)
        assert np.array_equal(c_new[k - 1], c[k - 1])
        c = c_new
