"""Python helper over the C ABI: contexts, distributed arrays, annotated
kernels and launches, mirroring the host API of the paper (Sec. 3.6:
``CudaKernelDef ... .annotate(...)``, ``context.zeros(n, dist)``,
``kernel.launch(grid, block, work_dist, args)``, ``context.synchronize()``).
Argument marshalling only; every step runs in liblightning.so.
"""
from __future__ import annotations

import ctypes as C
import json

import numpy as np

from . import _lib as L

F32, BF16, U8, U32, F64 = L.LT_F32, L.LT_BF16, L.LT_U8, L.LT_U32, L.LT_F64
STENCIL1D, JACOBI2D, JACOBI3D, GEMM_BF16, HIST256 = (L.LT_K_STENCIL1D, L.LT_K_JACOBI2D, L.LT_K_JACOBI3D,
                                                     L.LT_K_GEMM_BF16, L.LT_K_HIST256)
DIFFUSION2D, DIFFUSION2D_ADJ = L.LT_K_DIFFUSION2D, L.LT_K_DIFFUSION2D_ADJ
PLAN_ONLY = L.LT_K_PLAN_ONLY
ROWREDUCE = L.LT_K_ROWREDUCE
JACOBI2D_MULTI = L.LT_K_JACOBI2D_MULTI
KMEANS_ASSIGN = L.LT_K_KMEANS_ASSIGN
KMEANS_UPDATE = L.LT_K_KMEANS_UPDATE
LAPLACE2D, EWISE2D, MULADD2D = L.LT_K_LAPLACE2D, L.LT_K_EWISE2D, L.LT_K_MULADD2D

_NP = {F32: np.float32, BF16: np.uint16, U8: np.uint8, U32: np.uint32, F64: np.float64}


class LightningError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lightning error {code}: {msg}")
        self.code = code


def check(rc: int):
    if rc != L.LT_OK:
        msg = L.load().lt_last_error()
        raise LightningError(rc, msg.decode() if msg else "")


class Dist:
    """Distribution policy (Sec. 2.2): chunk extents per axis and halo."""

    def __init__(self, kind, chunk=(0, 0, 0), halo=(0, 0, 0), order=L.LT_ORDER_ROW):
        self.kind = kind
        self.chunk = tuple(chunk) + (0,) * (3 - len(chunk))
        self.halo = tuple(halo) + (0,) * (3 - len(halo))
        self.order = order

    @staticmethod
    def block():
        return Dist(L.LT_DIST_BLOCK)

    @staticmethod
    def rows(n, halo=0):
        return Dist(L.LT_DIST_ROWS, (n, 0, 0), (halo, 0, 0))

    @staticmethod
    def cols(n, halo=0, order=L.LT_ORDER_ROW):
        return Dist(L.LT_DIST_COLS, (0, n, 0), (0, halo, 0), order)

    @staticmethod
    def tiles(chunk, halo=(0, 0, 0), order=L.LT_ORDER_ROW):
        return Dist(L.LT_DIST_TILES, chunk, halo, order)

    def c(self):
        d = L.lt_dist()
        d.kind = self.kind
        d.order = self.order
        for i in range(3):
            d.chunk[i] = self.chunk[i]
            d.halo[i] = self.halo[i]
        return d


class Array:
    def __init__(self, ctx: "Context", dtype: int, shape, dist: Dist | None, wrap=None):
        """wrap: (device pointer, element strides, owner) for a zero-copy
        import of caller memory (lt_array_wrap_device); owner is kept alive."""
        self.ctx = ctx
        self.dtype = dtype
        self.shape = tuple(int(s) for s in shape)
        sh = (C.c_int64 * 3)(*(list(self.shape) + [1] * (3 - len(self.shape))))
        h = C.c_void_p()
        self._owner = None
        if wrap is not None:
            ptr, strides, self._owner = wrap
            st = (C.c_int64 * 3)(*(list(strides) + [1] * (3 - len(strides))))
            check(L.load().lt_array_wrap_device(ctx.h, dtype, len(self.shape), sh, st, C.c_void_p(ptr), C.byref(h)))
        else:
            d = dist.c()
            check(L.load().lt_array_create(ctx.h, dtype, len(self.shape), sh, C.byref(d), C.byref(h)))
        self.h = h

    @property
    def nbytes(self):
        return int(np.prod(self.shape)) * np.dtype(_NP[self.dtype]).itemsize

    def write(self, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=_NP[self.dtype])
        assert a.shape == self.shape, (a.shape, self.shape)
        check(L.load().lt_array_write(self.ctx.h, self.h, a.ctypes.data_as(C.c_void_p), a.nbytes))

    def write_async(self, a: np.ndarray):
        """Enqueue the copy from `a` (C-contiguous, this shape and dtype;
        pinned memory for the copy to overlap) and return
        (lt_array_write_async); the context keeps `a` until its next
        synchronize, and the caller must not change it before then."""
        assert a.shape == self.shape and a.dtype == _NP[self.dtype] and a.flags.c_contiguous
        check(L.load().lt_array_write_async(self.ctx.h, self.h, a.ctypes.data_as(C.c_void_p), a.nbytes))
        self.ctx._held.append(a)

    def read_async(self, out: np.ndarray) -> np.ndarray:
        """Enqueue the copy into `out` and return (lt_array_read_async); the
        values are there after the context's next synchronize."""
        assert out.shape == self.shape and out.dtype == _NP[self.dtype] and out.flags.c_contiguous
        check(L.load().lt_array_read_async(self.ctx.h, self.h, out.ctypes.data_as(C.c_void_p), out.nbytes))
        self.ctx._held.append(out)
        return out

    def discard(self):
        """Declare the contents dead: dropped instead of written back when
        memory is needed (lt_array_discard)."""
        check(L.load().lt_array_discard(self.ctx.h, self.h))

    def read(self, out: np.ndarray | None = None) -> np.ndarray:
        """The whole array, into `out` if given (C-contiguous, this shape and
        dtype; a pinned buffer makes the copy a direct DMA)."""
        if out is None:
            out = np.empty(self.shape, dtype=_NP[self.dtype])
        assert out.shape == self.shape and out.dtype == _NP[self.dtype] and out.flags.c_contiguous
        check(L.load().lt_array_read(self.ctx.h, self.h, out.ctypes.data_as(C.c_void_p), out.nbytes))
        return out

    def write_device(self, ptr: int, nbytes: int):
        """Copy from a dense row-major device buffer (e.g. tensor.data_ptr())."""
        check(L.load().lt_array_write_device(self.ctx.h, self.h, C.c_void_p(ptr), nbytes))

    def read_device(self, ptr: int, nbytes: int):
        check(L.load().lt_array_read_device(self.ctx.h, self.h, C.c_void_p(ptr), nbytes))

    def read_box(self, lo, hi) -> np.ndarray:
        nd = len(self.shape)
        shp = tuple(int(h) - int(l) + 1 for l, h in zip(lo, hi))
        out = np.empty(shp, dtype=_NP[self.dtype])
        clo = (C.c_int64 * 3)(*(list(lo) + [0] * (3 - nd)))
        chi = (C.c_int64 * 3)(*(list(hi) + [0] * (3 - nd)))
        check(L.load().lt_array_read_box(self.ctx.h, self.h, clo, chi, out.ctypes.data_as(C.c_void_p), out.nbytes))
        return out

    def fill(self, kind: int, seed: int = 0, stream: int = 0, value: float = 0.0, scale: float = 1.0):
        init = L.lt_init(kind, seed, stream, value, scale)
        check(L.load().lt_array_fill(self.ctx.h, self.h, C.byref(init)))

    def chunks(self):
        n = C.c_int64()
        check(L.load().lt_array_num_chunks(self.ctx.h, self.h, C.byref(n)))
        out = []
        for i in range(n.value):
            lo = (C.c_int64 * 3)()
            hi = (C.c_int64 * 3)()
            loc = C.c_int32()
            check(L.load().lt_array_chunk_info(self.ctx.h, self.h, i, lo, hi, C.byref(loc)))
            nd = len(self.shape)
            out.append((tuple(lo[:nd]), tuple(hi[:nd]), loc.value))
        return out

    def destroy(self):
        if self.h:
            check(L.load().lt_array_destroy(self.ctx.h, self.h))
            self.h = None


def _dim3(t):
    t = tuple(t) + (1,) * (3 - len(t))
    return L.lt_dim3(*t)


class Kernel:
    def __init__(self, ctx: "Context", builtin: int, annotation: str, params, source: str | None = None,
                 name: str | None = None):
        self.ctx = ctx
        self.params = []
        for p in params:
            pname, dtype = p[0], p[1]
            is_array = p[2] if len(p) > 2 else True
            self.params.append((pname, dtype, is_array))
        arr = (L.lt_param * len(self.params))()
        self._names = [n.encode() for n, _, _ in self.params]
        for i, (n, d, a) in enumerate(self.params):
            arr[i] = L.lt_param(self._names[i], 1 if a else 0, d)
        h = C.c_void_p()
        if source is not None:
            check(L.load().lt_kernel_register_source(ctx.h, source.encode(), name.encode(), annotation.encode(), arr,
                                                     len(self.params), C.byref(h)))
        else:
            check(L.load().lt_kernel_register(ctx.h, builtin, annotation.encode(), arr, len(self.params),
                                              C.byref(h)))
        self.h = h

    def destroy(self):
        if self.h:
            check(L.load().lt_kernel_destroy(self.ctx.h, self.h))
            self.h = None

    def _args(self, args):
        assert len(args) == len(self.params)
        a = (L.lt_arg * len(args))()
        for i, v in enumerate(args):
            if self.params[i][2]:
                a[i].array = v.h
            elif self.params[i][1] == F32:
                a[i].f = float(v)
            else:
                a[i].i = int(v)
        return a

    def launch(self, grid, block, superblock=(0, 0, 0), args=()):
        wd = L.lt_workdist((C.c_int64 * 3)(*(tuple(superblock) + (0,) * (3 - len(superblock)))))
        a = self._args(args)
        check(L.load().lt_launch(self.ctx.h, self.h, _dim3(grid), _dim3(block), C.byref(wd), a, len(args)))

    def explain(self, grid, block, superblock=(0, 0, 0), args=()):
        wd = L.lt_workdist((C.c_int64 * 3)(*(tuple(superblock) + (0,) * (3 - len(superblock)))))
        a = self._args(args)
        need = C.c_size_t()
        check(L.load().lt_plan_explain(self.ctx.h, self.h, _dim3(grid), _dim3(block), C.byref(wd), a, len(args),
                                       None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        check(L.load().lt_plan_explain(self.ctx.h, self.h, _dim3(grid), _dim3(block), C.byref(wd), a, len(args),
                                       buf, need.value, None))
        return json.loads(buf.value.decode())



class Batch:
    """The lt_launch_desc array of a batch of launches, built once.  It holds
    the launches (and so their arrays and argument tables) alive; descriptors
    are rebuilt only by preparing a new Batch."""

    def __init__(self, launches):
        self.launches = list(launches)
        self.n = len(self.launches)
        self.descs = (L.lt_launch_desc * self.n)()
        self._args = []
        for i, (k, grid, block, sb, args, rep) in enumerate(self.launches):
            a = k._args(args)
            self._args.append(a)
            d = self.descs[i]
            d.kernel = k.h
            d.grid = _dim3(grid)
            d.block = _dim3(block)
            d.wd = L.lt_workdist((C.c_int64 * 3)(*(tuple(sb) + (0,) * (3 - len(sb)))))
            d.args = C.cast(a, C.POINTER(L.lt_arg))
            d.nargs = len(args)
            d.repeat = rep


class Context:
    def __init__(self, device=0, hbm_budget=0, host_pool=0, staging_cap=0, flags=0):
        cfg = L.lt_config(hbm_budget, host_pool, staging_cap, device, flags)
        h = C.c_void_p()
        check(L.load().lt_ctx_create(C.byref(cfg), C.byref(h)))
        self.h = h
        self._held = []  # host buffers of asynchronous copies, kept until the next synchronize

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.h:
            L.load().lt_ctx_destroy(self.h)
            self.h = None
        self._held = []

    def array(self, dtype, shape, dist: Dist | None = None) -> Array:
        return Array(self, dtype, shape, dist or Dist.block())

    def kernel(self, builtin, annotation, params) -> Kernel:
        return Kernel(self, builtin, annotation, params)

    def wrap(self, tensor) -> Array:
        """Zero-copy array over a CUDA tensor's memory (one chunk, never moved
        or freed by the library).  The tensor's pending work is waited for
        first; the tensor holds every launch's results after synchronize()."""
        import torch
        dt = {torch.float32: F32, torch.float64: F64, torch.uint8: U8, torch.bfloat16: BF16, torch.int32: U32}
        if not tensor.is_cuda or tensor.dtype not in dt:
            raise ValueError("wrap needs a CUDA tensor of float32, float64, uint8, bfloat16 or int32")
        torch.cuda.current_stream(tensor.device).synchronize()
        return Array(self, dt[tensor.dtype], tuple(tensor.shape), None,
                     wrap=(tensor.data_ptr(), tuple(tensor.stride()), tensor))

    def kernel_from_source(self, source: str, name: str, annotation: str, params) -> Kernel:
        """Runtime-compiled user kernel (the paper's CudaKernelDef ... compile())."""
        return Kernel(self, L.LT_K_USER, annotation, params, source=source, name=name)

    def prepare_batch(self, launches) -> "Batch":
        """Marshal a batch once, for repeated launch_batch calls."""
        return Batch(launches)

    def launch_batch(self, launches, flags=0):
        """launches: a Batch, or a list of (kernel, grid, block, superblock, args, repeat)."""
        b = launches if isinstance(launches, Batch) else Batch(launches)
        check(L.load().lt_launch_batch(self.h, C.cast(b.descs, C.c_void_p), b.n, flags))

    def synchronize(self):
        check(L.load().lt_synchronize(self.h))
        self._held.clear()

    def timer_start(self):
        check(L.load().lt_timer_start(self.h))

    def timer_stop(self) -> float:
        ms = C.c_double()
        check(L.load().lt_timer_stop(self.h, C.byref(ms)))
        return ms.value

    def op_timing(self, on: bool = True):
        check(L.load().lt_op_timing(self.h, 1 if on else 0))

    def stats(self) -> dict:
        s = L.lt_stats()
        check(L.load().lt_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.lt_stats._fields_}

    def reset_stats(self):
        check(L.load().lt_stats_reset(self.h))

    def log_enable(self, on=True):
        check(L.load().lt_debug_log_enable(self.h, 1 if on else 0))

    def timeline(self):
        """Start and end times (ms) of the operations timed while the log was on."""
        need = C.c_size_t()
        check(L.load().lt_debug_timeline(self.h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        check(L.load().lt_debug_timeline(self.h, buf, need.value, None))
        return json.loads(buf.value.decode())

    def log(self):
        need = C.c_size_t()
        check(L.load().lt_debug_log(self.h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value)
        check(L.load().lt_debug_log(self.h, buf, need.value, None))
        return json.loads(buf.value.decode())
