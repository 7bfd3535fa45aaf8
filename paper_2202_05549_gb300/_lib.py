"""ctypes declarations of the C ABI in include/lightning.h (same names).

Argument marshalling only: every step of a launch runs in the native
library.  Importing this module loads liblightning.so and fails loudly if
it is missing -- there is no CPU fallback.
"""
import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblightning.so")

# status codes
LT_OK = 0
LT_ERR_INVALID_ARG = -1
LT_ERR_PARSE = -2
LT_ERR_OOM_DEVICE = -3
LT_ERR_OOM_HOST = -4
LT_ERR_CUDA = -5
LT_ERR_TIMEOUT = -6
LT_ERR_BUSY = -7
LT_ERR_UNSUPPORTED = -8
LT_ERR_DEVICE_CHECK = -9
LT_ERR_COMPILE = -10

# dtypes
LT_F32, LT_BF16, LT_U8, LT_U32, LT_F64 = 0, 1, 2, 3, 4
# distributions
LT_DIST_BLOCK, LT_DIST_ROWS, LT_DIST_COLS, LT_DIST_TILES = 0, 1, 2, 3
LT_ORDER_ROW, LT_ORDER_COL = 0, 1
# flags
LT_FLAG_TIMING, LT_FLAG_DRYRUN, LT_FLAG_FIXED_SWEEP, LT_FLAG_NO_STAGED, LT_FLAG_NO_LINK_QUARANTINE = 1, 2, 4, 8, 16
LT_FLAG_NO_PDL = 32
LT_FLAG_NO_FUSED_REPLICAS = 64
LT_FLAG_TEST_REPLICA_STALL = 128
# fills
(LT_INIT_ZERO, LT_INIT_CONST, LT_INIT_UNIFORM, LT_INIT_KAPPA, LT_INIT_NORMAL_BF16,
 LT_INIT_U8) = range(6)
# built-ins
LT_K_PLAN_ONLY = 0
LT_K_USER = 100
LT_K_STENCIL1D, LT_K_JACOBI2D, LT_K_JACOBI3D, LT_K_GEMM_BF16, LT_K_HIST256 = 1, 2, 3, 4, 5
LT_K_DIFFUSION2D, LT_K_DIFFUSION2D_ADJ, LT_K_ROWREDUCE, LT_K_JACOBI2D_MULTI = 6, 7, 8, 9
LT_K_KMEANS_ASSIGN, LT_K_KMEANS_UPDATE = 10, 11
LT_K_LAPLACE2D, LT_K_EWISE2D, LT_K_MULADD2D = 12, 13, 14


class lt_dist(C.Structure):
    _fields_ = [("kind", C.c_int32), ("order", C.c_int32), ("chunk", C.c_int64 * 3), ("halo", C.c_int64 * 3)]


class lt_config(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("host_pool_bytes", C.c_size_t),
                ("staging_cap_bytes", C.c_size_t), ("device", C.c_int32), ("flags", C.c_int32)]


class lt_init(C.Structure):
    _fields_ = [("kind", C.c_int32), ("seed", C.c_uint64), ("stream", C.c_uint64), ("value", C.c_double),
                ("scale", C.c_double)]


class lt_param(C.Structure):
    _fields_ = [("name", C.c_char_p), ("is_array", C.c_int32), ("dtype", C.c_int32)]


class lt_dim3(C.Structure):
    _fields_ = [("x", C.c_uint64), ("y", C.c_uint64), ("z", C.c_uint64)]


class lt_workdist(C.Structure):
    _fields_ = [("superblock", C.c_int64 * 3)]


class lt_arg(C.Structure):
    _fields_ = [("array", C.c_void_p), ("f", C.c_double), ("i", C.c_int64)]


class lt_stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "launches", "tasks_execute", "tasks_copy", "tasks_reduce", "deps", "fetches", "evictions", "dead_skips",
        "bytes_h2d", "bytes_d2h", "bytes_d2d", "kernels", "hbm_in_use", "hbm_peak", "host_in_use")] + [
        ("ms_execute", C.c_double), ("n_execute_kernels", C.c_uint64), ("ms_copy_kernels", C.c_double),
        ("n_copy_kernels", C.c_uint64), ("ms_h2d", C.c_double), ("ms_d2h", C.c_double), ("ms_fill", C.c_double),
        ("batches_fused", C.c_uint64), ("batches_plain", C.c_uint64), ("graph_replays", C.c_uint64),
        ("tuned_tile_rows", C.c_int64), ("tuned_hist_slice", C.c_int64), ("tables_resident", C.c_uint64),
        ("plans_reused", C.c_uint64), ("reduce_inplace", C.c_uint64), ("bytes_replica_wt", C.c_uint64),
        ("ms_span", C.c_double), ("ms_link_busy", C.c_double), ("ms_link_both", C.c_double),
        ("ms_exec_hidden", C.c_double), ("host_withheld_bytes", C.c_uint64),
        ("host_quarantined", C.c_uint64), ("tuned_tile_cols", C.c_int64)]


class lt_launch_desc(C.Structure):
    _fields_ = [("kernel", C.c_void_p), ("grid", lt_dim3), ("block", lt_dim3), ("wd", lt_workdist),
                ("args", C.POINTER(lt_arg)), ("nargs", C.c_int32), ("repeat", C.c_int32)]


LT_BATCH_PLAIN, LT_BATCH_NO_GRAPH, LT_BATCH_RETUNE, LT_BATCH_TEST_STALL = 1, 2, 4, 256
LT_BATCH_TEST_TILE_COLS = 512


_vp = C.c_void_p
_st = C.c_int32
SIGNATURES = {
    "lt_ctx_create": (_st, [C.POINTER(lt_config), C.POINTER(_vp)]),
    "lt_ctx_destroy": (_st, [_vp]),
    "lt_last_error": (C.c_char_p, []),
    "lt_array_create": (_st, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(lt_dist),
                              C.POINTER(_vp)]),
    "lt_array_wrap_device": (_st, [_vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp,
                                   C.POINTER(_vp)]),
    "lt_array_destroy": (_st, [_vp, _vp]),
    "lt_array_write": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_read": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_write_async": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_read_async": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_write_device": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_read_device": (_st, [_vp, _vp, _vp, C.c_size_t]),
    "lt_array_read_box": (_st, [_vp, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp, C.c_size_t]),
    "lt_array_fill": (_st, [_vp, _vp, C.POINTER(lt_init)]),
    "lt_array_num_chunks": (_st, [_vp, _vp, C.POINTER(C.c_int64)]),
    "lt_array_chunk_info": (_st, [_vp, _vp, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int32)]),
    "lt_kernel_register": (_st, [_vp, C.c_int32, C.c_char_p, C.POINTER(lt_param), C.c_int32, C.POINTER(_vp)]),
    "lt_kernel_destroy": (_st, [_vp, _vp]),
    "lt_kernel_register_source": (_st, [_vp, C.c_char_p, C.c_char_p, C.c_char_p, C.POINTER(lt_param), C.c_int32,
                                        C.POINTER(_vp)]),
    "lt_launch": (_st, [_vp, _vp, lt_dim3, lt_dim3, C.POINTER(lt_workdist), C.POINTER(lt_arg), C.c_int32]),
    "lt_synchronize": (_st, [_vp]),
    "lt_launch_batch": (_st, [_vp, C.c_void_p, C.c_int32, C.c_int32]),
    "lt_timer_start": (_st, [_vp]),
    "lt_timer_stop": (_st, [_vp, C.POINTER(C.c_double)]),
    "lt_op_timing": (_st, [_vp, C.c_int32]),
    "lt_array_discard": (_st, [_vp, _vp]),
    "lt_stats_get": (_st, [_vp, C.POINTER(lt_stats)]),
    "lt_stats_reset": (_st, [_vp]),
    "lt_plan_explain": (_st, [_vp, _vp, lt_dim3, lt_dim3, C.POINTER(lt_workdist), C.POINTER(lt_arg), C.c_int32,
                              C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "lt_debug_log_enable": (_st, [_vp, C.c_int32]),
    "lt_debug_log": (_st, [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "lt_debug_timeline": (_st, [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "lt_jacobi2d_packed_noalloc": (_st, [_vp, _vp, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                         C.c_int64, _vp]),
    "lt_selftest_div_const": (_st, [C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]),
}

_lib = None


def load():
    """Load liblightning.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first; "
                              "there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
