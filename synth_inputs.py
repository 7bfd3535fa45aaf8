"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds only the input recipe: a counter-based SplitMix64 stream
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) and the maps from its 64-bit outputs to the value
distributions of the workloads.  It computes none of the method's
arithmetic.  The CUDA fill kernel and the C oracle each implement the same
published generator independently; all three must agree bit for bit.

Recipe (the paper fixes no input data; its workloads are only described):

* key(seed, stream) = first SplitMix64 output from state
  ``seed XOR (stream << 32)``.
* element ``idx`` of a stream = SplitMix64 mix of ``key + (idx + 1) * GAMMA``
  (mod 2^64), i.e. the (idx+1)-th output of a generator seeded with ``key``.
  Any chunk can therefore regenerate its own elements from global indices.
* uniform f32 in [0, 1): ``(x >> 40) * 2^-24`` (exact in f32).
* uint8: ``x >> 56``.
* diffusion coefficient kappa: ``float(0.05 + 0.15 * double(u))``, u the
  uniform f32 of the same element, i.e. uniform in [0.05, 0.2).
* N(0,1) * scale, rounded to bf16: Box-Muller in fp64 from counters
  ``2*idx`` and ``2*idx+1`` (u1 = ((x1 >> 11) + 1) * 2^-53 in (0, 1],
  u2 = (x2 >> 11) * 2^-53), times ``scale``, rounded to f32 (RNE) then
  to bf16 (RNE).
* Seeds are ``2202 + config_id``; stream ids are per array (below).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

# seeds (2202 + config id) and stream ids of every array in the workloads
SEED_JACOBI_INCORE = 2203      # 4096^2 Jacobi, 10 iterations
SEED_JACOBI_OOC = 2204         # 262144 x 131072 out-of-core Jacobi
SEED_GEMM = 2205               # 65536^3 BF16 GEMM
SEED_BATCH = 2206              # 4096 uneven Jacobi + 1024 histograms
SEED_DIFFUSION = 2207          # 16384^2 variable-coefficient diffusion

STREAM_U = 0
STREAM_A = 0
STREAM_B = 1
STREAM_KAPPA = 1
STREAM_BATCH_SIDES = 100
STREAM_BATCH_HISTLEN = 101
STREAM_BATCH_JACOBI0 = 1000    # instance q uses stream 1000 + q
STREAM_BATCH_HIST0 = 10000     # histogram h uses stream 10000 + h


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_sequence(seed: int, n: int) -> list[int]:
    """First ``n`` outputs of a SplitMix64 generator seeded with ``seed``
    (the sequential published form: state += GAMMA; output mix(state))."""
    with np.errstate(over="ignore"):
        st = np.uint64(seed & MASK64)
        out = []
        for _ in range(n):
            st = np.uint64((int(st) + int(GAMMA)) & MASK64)
            out.append(int(_mix(np.array([st], dtype=np.uint64))[0]))
    return out


def stream_key(seed: int, stream: int) -> int:
    return splitmix64_sequence((seed ^ (stream << 32)) & MASK64, 1)[0]


def gen_u64(seed: int, stream: int, idx) -> np.ndarray:
    """Raw 64-bit outputs for the global element indices ``idx``."""
    idx = np.asarray(idx, dtype=np.uint64)
    key = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        st = key + (idx + np.uint64(1)) * GAMMA
        return _mix(st)


def gen_uniform_f32(seed: int, stream: int, idx) -> np.ndarray:
    x = gen_u64(seed, stream, idx)
    return ((x >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def gen_u8(seed: int, stream: int, idx) -> np.ndarray:
    return (gen_u64(seed, stream, idx) >> np.uint64(56)).astype(np.uint8)


def gen_kappa_f32(seed: int, stream: int, idx) -> np.ndarray:
    u = gen_uniform_f32(seed, stream, idx).astype(np.float64)
    return (0.05 + 0.15 * u).astype(np.float32)


def _f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f32(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def gen_normal_bf16_bits(seed: int, stream: int, idx, scale: float) -> np.ndarray:
    """bf16 bit patterns of N(0,1)*scale (recipe above)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x1 = gen_u64(seed, stream, idx * np.uint64(2))
        x2 = gen_u64(seed, stream, idx * np.uint64(2) + np.uint64(1))
    u1 = ((x1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (x2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)
    return _f32_to_bf16_bits((z * scale).astype(np.float32))


def uniform_field(seed: int, stream: int, ny: int, nx: int) -> np.ndarray:
    """Row-major ny x nx f32 field; element (i, j) has global index i*nx+j."""
    idx = np.arange(ny * nx, dtype=np.uint64)
    return gen_uniform_f32(seed, stream, idx).reshape(ny, nx)


def kappa_field(seed: int, stream: int, ny: int, nx: int) -> np.ndarray:
    idx = np.arange(ny * nx, dtype=np.uint64)
    return gen_kappa_f32(seed, stream, idx).reshape(ny, nx)


def u8_array(seed: int, stream: int, n: int) -> np.ndarray:
    return gen_u8(seed, stream, np.arange(n, dtype=np.uint64))


def _uniform_f64(seed: int, stream: int, n: int) -> np.ndarray:
    x = gen_u64(seed, stream, np.arange(n, dtype=np.uint64))
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


@dataclass(frozen=True)
class BatchRecipe:
    """Shapes of the batched uneven workload: square Jacobi instances with
    side ``min(4096, floor(64 * 64**u))`` (log-uniform in [64, 4096]) and
    uint8 arrays of length ``min(1e7, floor(1e4 * 1000**u))``."""
    n_jacobi: int = 4096
    n_hist: int = 1024
    iters: int = 8
    seed: int = SEED_BATCH

    def sides(self) -> np.ndarray:
        u = _uniform_f64(self.seed, STREAM_BATCH_SIDES, self.n_jacobi)
        return np.minimum(4096, np.floor(64.0 * np.power(64.0, u))).astype(np.int64)

    def hist_lengths(self) -> np.ndarray:
        u = _uniform_f64(self.seed, STREAM_BATCH_HISTLEN, self.n_hist)
        return np.minimum(10_000_000, np.floor(1e4 * np.power(1000.0, u))).astype(np.int64)


def log_uniform_int(seed: int, stream: int, n: int, lo: float, ratio: float, cap: int) -> np.ndarray:
    """``min(cap, floor(lo * ratio**u))`` for n uniform u (for scaled-down batches)."""
    u = _uniform_f64(seed, stream, n)
    return np.minimum(cap, np.floor(lo * np.power(ratio, u))).astype(np.int64)


def sample_cells(seed: int, ny: int, nx: int, n: int, seams_every: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Deterministic sample of cell coordinates: the four corners, edge
    midpoints, cells on both sides of every ``seams_every``-row seam (if
    given, up to n/4 of them) and the rest uniform from a dedicated stream."""
    pts = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1),
           (0, nx // 2), (ny - 1, nx // 2), (ny // 2, 0), (ny // 2, nx - 1)]
    if seams_every:
        seams = list(range(seams_every, ny, seams_every))
        x = gen_u64(seed, 77, np.arange(2 * len(seams), dtype=np.uint64))
        for k, s in enumerate(seams[: max(1, n // 8)]):
            j = int(x[2 * k] % np.uint64(nx))
            pts += [(s - 1, j), (s, j)]
    rest = max(0, n - len(pts))
    x = gen_u64(seed, 78, np.arange(2 * rest, dtype=np.uint64))
    for k in range(rest):
        pts.append((int(x[2 * k] % np.uint64(ny)), int(x[2 * k + 1] % np.uint64(nx))))
    pts = pts[:n]
    return (np.array([p[0] for p in pts], dtype=np.int64),
            np.array([p[1] for p in pts], dtype=np.int64))


def expected_batch_cells() -> float:
    """E[s^2] for s = 64 * 64**u, u ~ U[0,1): 4096 * 4095 / ln 4096."""
    return 4096.0 * 4095.0 / math.log(4096.0)
