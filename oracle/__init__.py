"""CPU oracle: plain, slow, obviously correct definitions of every workload.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA path (``oracle.c`` is plain
C, compiled by gcc with ``-O2 -ffp-contract=off``); the only thing both
sides share is the seeded input recipe in ``synth_inputs``.

Functions and the passages they follow:

* ``stencil1d_paper`` -- the paper's worked example (Listings 1-2 and the
  host code of Sec. 3.6): ``(in[i-1] + in[i] + in[i+1]) / 3.0`` with zero
  out-of-range reads.
* ``jacobi2d`` / ``jacobi2d_lightcone`` -- the 2-D 5-point Jacobi that
  stands in for HotSpot (Sec. 4.2), f32, zero ghosts, fixed sum order.
* ``jacobi2d_ring_f64`` -- the same update in fp64 with arbitrary fixed or
  periodic ghost rings, used only to pin the definition.
* ``jacobi3d`` / ``jacobi3d_lightcone`` -- 3-D 7-point variant.
* ``gemm_f64`` / ``gemm_sample`` -- C = A B (Sec. 4.2 "GEMM") in fp64.
* ``hist256`` -- the reduce(+) access mode (Sec. 2.3) as a 256-bin count.
* ``diffusion_*`` -- variable-coefficient diffusion, its loss and its
  adjoint gradient in fp64 (an extension beyond the paper).
* ``access_region_bruteforce`` -- the access region of a superblock
  (Sec. 2.3: the dense box of all elements its threads touch), found by
  enumerating every thread's accesses.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = C.c_int64
_u64 = C.c_uint64
_p = C.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no nvcc, no CUDA) if missing or stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            sig = {
                "orc_splitmix64_next": (_u64, [C.POINTER(_u64)]),
                "orc_stream_key": (_u64, [_u64, _u64]),
                "orc_gen_u64": (None, [_u64, _u64, _u64, _i64, _p]),
                "orc_gen_uniform_f32": (None, [_u64, _u64, _u64, _i64, _p]),
                "orc_gen_u8": (None, [_u64, _u64, _u64, _i64, _p]),
                "orc_gen_kappa_f32": (None, [_u64, _u64, _u64, _i64, _p]),
                "orc_gen_normal_bf16": (None, [_u64, _u64, _u64, _i64, C.c_double, _p]),
                "orc_max_threads": (C.c_int, []),
                "orc_set_threads": (None, [C.c_int]),
                "orc_stencil1d_paper": (None, [_i64, _p, _p]),
                "orc_jacobi2d_f32": (C.c_int, [_i64, _i64, _p, _p, C.c_int]),
                "orc_jacobi2d_f64_ring": (C.c_int, [_i64, _i64, _p, C.c_int, C.c_int]),
                "orc_jacobi2d_f32_lightcone": (C.c_int, [_i64, _i64, _u64, _u64, C.c_int, _i64, _p, _p, _p]),
                "orc_jacobi3d_f32": (C.c_int, [_i64, _i64, _i64, _p, _p, C.c_int]),
                "orc_kmeans_assign": (None, [_i64, _i64, _p, _p, _p, _p]),
                "orc_kmeans_update": (None, [_i64, _p, _p, _p]),
                "orc_jacobi3d_f64": (C.c_int, [_i64, _i64, _i64, _p, C.c_int]),
                "orc_gemm_f64": (None, [_i64, _i64, _i64, _p, _p, _p]),
                "orc_gemm_sample_f64": (C.c_int, [_i64, _i64, _i64, _u64, _u64, _u64, C.c_double,
                                                  _i64, _p, _i64, _p, _p, _p]),
                "orc_gemm_bf16_corner_f32": (C.c_int, [_i64, _i64, _i64, _i64, _i64, _u64, _u64, _u64,
                                                       C.c_double, _p]),
                "orc_hist256": (None, [_i64, _p, _p]),
                "orc_rowreduce_f64": (None, [_i64, _i64, _p, C.c_int, _p]),
                "orc_diff_forward_f64": (C.c_int, [_i64, _i64, _p, _p, C.c_int, _p]),
                "orc_diff_grad_f64": (C.c_int, [_i64, _i64, _p, _p, C.c_int, _p, _p, _p]),
                "orc_diff_lightcone_f64": (C.c_int, [_i64, _i64, _u64, _u64, _u64, C.c_int, _i64, _p, _p,
                                                     _p, _p, _p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise MemoryError(f"oracle {what} failed (rc={rc})")


# ---------------------------------------------------------------- inputs
def splitmix64_next(state: int) -> tuple[int, int]:
    s = _u64(state)
    out = lib().orc_splitmix64_next(C.byref(s))
    return int(out), int(s.value)


def gen_u64(seed, stream, idx0, n):
    out = np.empty(n, np.uint64)
    lib().orc_gen_u64(seed, stream, idx0, n, _ptr(out))
    return out


def gen_uniform_f32(seed, stream, idx0, n):
    out = np.empty(n, np.float32)
    lib().orc_gen_uniform_f32(seed, stream, idx0, n, _ptr(out))
    return out


def gen_u8(seed, stream, idx0, n):
    out = np.empty(n, np.uint8)
    lib().orc_gen_u8(seed, stream, idx0, n, _ptr(out))
    return out


def gen_kappa_f32(seed, stream, idx0, n):
    out = np.empty(n, np.float32)
    lib().orc_gen_kappa_f32(seed, stream, idx0, n, _ptr(out))
    return out


def gen_normal_bf16_bits(seed, stream, idx0, n, scale):
    out = np.empty(n, np.uint16)
    lib().orc_gen_normal_bf16(seed, stream, idx0, n, scale, _ptr(out))
    return out


def max_threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int):
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- stencils
def stencil1d_paper(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(x)
    lib().orc_stencil1d_paper(x.size, _ptr(x), _ptr(out))
    return out


def jacobi2d(u: np.ndarray, iters: int) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float32)
    out = np.empty_like(u)
    _check(lib().orc_jacobi2d_f32(u.shape[0], u.shape[1], _ptr(u), _ptr(out), iters), "jacobi2d")
    return out


def jacobi2d_ring_f64(padded: np.ndarray, iters: int, periodic: bool = False) -> np.ndarray:
    p = np.array(padded, dtype=np.float64, copy=True, order="C")
    _check(lib().orc_jacobi2d_f64_ring(p.shape[0] - 2, p.shape[1] - 2, _ptr(p), iters, int(periodic)),
           "jacobi2d_ring_f64")
    return p


def jacobi2d_lightcone(NY, NX, seed, stream, iters, si, sj) -> np.ndarray:
    si = np.ascontiguousarray(si, np.int64)
    sj = np.ascontiguousarray(sj, np.int64)
    out = np.empty(si.size, np.float32)
    _check(lib().orc_jacobi2d_f32_lightcone(NY, NX, seed, stream, iters, si.size, _ptr(si), _ptr(sj),
                                            _ptr(out)), "jacobi2d_lightcone")
    return out


def jacobi3d(u: np.ndarray, iters: int) -> np.ndarray:
    u = np.ascontiguousarray(u, np.float32)
    out = np.empty_like(u)
    _check(lib().orc_jacobi3d_f32(*u.shape, _ptr(u), _ptr(out), iters), "jacobi3d")
    return out


def jacobi3d_lightcone(shape, seed, stream, iters, sk, si, sj) -> np.ndarray:
    """Cells (sk, si, sj) of ``iters`` 3-D Jacobi steps from the seeded
    uniform field of ``shape``, each from its light cone alone: a cell after
    n steps depends only on initial cells within n steps along every axis, so
    the box [p - n, p + n] (clipped to the domain, where the zero ghosts are
    the true ones) run through ``jacobi3d`` gives it exactly; the wrong zeros
    beyond the box's inner faces move one cell per step and never reach p."""
    import synth_inputs as si_mod

    NZ, NY, NX = shape
    out = np.empty(len(sk), np.float32)
    for n, (k, i, j) in enumerate(zip(sk, si, sj)):
        lo = [max(0, int(c) - iters) for c in (k, i, j)]
        hi = [min(e - 1, int(c) + iters) for c, e in zip((k, i, j), shape)]
        kk, ii, jj = np.meshgrid(*[np.arange(a, b + 1, dtype=np.uint64) for a, b in zip(lo, hi)], indexing="ij")
        idx = (kk * np.uint64(NY) + ii) * np.uint64(NX) + jj
        box = si_mod.gen_uniform_f32(seed, stream, idx.ravel()).reshape(kk.shape)
        out[n] = jacobi3d(box, iters)[int(k) - lo[0], int(i) - lo[1], int(j) - lo[2]]
    return out


def jacobi3d_f64(u: np.ndarray, iters: int) -> np.ndarray:
    p = np.array(u, dtype=np.float64, copy=True, order="C")
    _check(lib().orc_jacobi3d_f64(*p.shape, _ptr(p), iters), "jacobi3d_f64")
    return p


# ---------------------------------------------------------------- GEMM
def gemm_f64(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    Cm = np.empty((M, N), np.float64)
    lib().orc_gemm_f64(M, N, K, _ptr(A), _ptr(B), _ptr(Cm))
    return Cm


def gemm_sample(M, N, K, seed, streamA, streamB, scale, rows, cols):
    rows = np.ascontiguousarray(rows, np.int64)
    cols = np.ascontiguousarray(cols, np.int64)
    cr = np.empty((rows.size, cols.size), np.float64)
    cu = np.empty_like(cr)
    _check(lib().orc_gemm_sample_f64(M, N, K, seed, streamA, streamB, scale, rows.size, _ptr(rows),
                                     cols.size, _ptr(cols), _ptr(cr), _ptr(cu)), "gemm_sample")
    return cr, cu


def gemm_bf16_corner_f32(M, N, K, ldN, ldK, seed, streamA, streamB, scale):
    out = np.empty((M, N), np.float32)
    _check(lib().orc_gemm_bf16_corner_f32(M, N, K, ldN, ldK, seed, streamA, streamB, scale, _ptr(out)),
           "gemm_bf16_corner_f32")
    return out


# ---------------------------------------------------------------- histogram
def hist256(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.uint8)
    h = np.empty(256, np.uint32)
    lib().orc_hist256(x.size, _ptr(x), _ptr(h))
    return h


def rowreduce(a: np.ndarray, op: str) -> np.ndarray:
    """out[i] = a[i,0] op a[i,1] op ... (fp64, left to right); op in + * min max."""
    a = np.ascontiguousarray(a, np.float64)
    out = np.empty(a.shape[0], np.float64)
    lib().orc_rowreduce_f64(a.shape[0], a.shape[1], _ptr(a), {"+": 0, "*": 1, "min": 2, "max": 3}[op], _ptr(out))
    return out


# ---------------------------------------------------------------- diffusion
def diffusion_forward(u0, kappa, T):
    u0 = np.ascontiguousarray(u0, np.float64)
    kappa = np.ascontiguousarray(kappa, np.float64)
    out = np.empty_like(u0)
    _check(lib().orc_diff_forward_f64(u0.shape[0], u0.shape[1], _ptr(u0), _ptr(kappa), T, _ptr(out)),
           "diffusion_forward")
    return out


def diffusion_grad(u0, kappa, T):
    u0 = np.ascontiguousarray(u0, np.float64)
    kappa = np.ascontiguousarray(kappa, np.float64)
    du0 = np.empty_like(u0)
    dk = np.empty_like(u0)
    J = np.zeros(1, np.float64)
    _check(lib().orc_diff_grad_f64(u0.shape[0], u0.shape[1], _ptr(u0), _ptr(kappa), T, _ptr(J), _ptr(du0),
                                   _ptr(dk)), "diffusion_grad")
    return float(J[0]), du0, dk


def diffusion_lightcone(NY, NX, seed, stream_u, stream_k, T, si, sj):
    si = np.ascontiguousarray(si, np.int64)
    sj = np.ascontiguousarray(sj, np.int64)
    uT = np.empty(si.size, np.float64)
    du = np.empty(si.size, np.float64)
    dk = np.empty(si.size, np.float64)
    _check(lib().orc_diff_lightcone_f64(NY, NX, seed, stream_u, stream_k, T, si.size, _ptr(si), _ptr(sj),
                                        _ptr(uT), _ptr(du), _ptr(dk)), "diffusion_lightcone")
    return uT, du, dk


# ---------------------------------------------------------------- planner
def kmeans_assign(x: np.ndarray, c: np.ndarray):
    """One K-Means assignment (Sec. 4 K-Means benchmark): x (n, 4) f32 records,
    c (k, 4) f32 centres -> (s (k, 5) fp64 feature sums and counts, labels (n,))."""
    x = np.ascontiguousarray(x, np.float32)
    c = np.ascontiguousarray(c, np.float32)
    n, k = x.shape[0], c.shape[0]
    s = np.zeros((k, 5), np.float64)
    lab = np.zeros(n, np.int32)
    lib().orc_kmeans_assign(n, k, _ptr(x), _ptr(c), _ptr(s), _ptr(lab))
    return s, lab


def kmeans_update(s: np.ndarray, c: np.ndarray) -> np.ndarray:
    """New centres from the sums and counts of kmeans_assign (empty clusters keep theirs)."""
    s = np.ascontiguousarray(s, np.float64)
    c = np.ascontiguousarray(c, np.float32)
    out = np.empty_like(c)
    lib().orc_kmeans_update(c.shape[0], _ptr(s), _ptr(c), _ptr(out))
    return out


def access_region_bruteforce(thread_box, accesses, shape):
    """Access region of one superblock for one array, by enumeration.

    ``thread_box`` is a list of (lo, hi) inclusive ranges, one per bound
    variable; ``accesses(*vars)`` returns the list of index tuples one thread
    touches; ``shape`` clips the region to the array domain (Sec. 2.3 defines
    the region as the dense box of elements the superblock's threads access).
    Returns (lo, hi) inclusive per axis, or None if nothing is touched.
    Pure Python: tiny grids only.
    """
    import itertools

    lo = [None] * len(shape)
    hi = [None] * len(shape)
    ranges = [range(a, b + 1) for a, b in thread_box]
    for v in itertools.product(*ranges):
        for idx in accesses(*v):
            if any(x < 0 or x >= n for x, n in zip(idx, shape)):
                continue
            for d, x in enumerate(idx):
                lo[d] = x if lo[d] is None else min(lo[d], x)
                hi[d] = x if hi[d] is None else max(hi[d], x)
    if lo[0] is None:
        return None
    return list(zip(lo, hi))
