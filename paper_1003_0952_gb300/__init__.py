"""Python binding of the GB300 CSRC library (include/csrc.h).

The binding only marshals arguments. Every step of a product runs in the
library's CUDA kernels in ``lib/libcsrc_gb300.so``, which this module builds in-tree
on first import when it is missing or stale, then loads.
PyTorch supplies device memory and streams: tensors are passed by
``data_ptr()``, streams by ``cuda_stream``. If the shared library is missing,
the import fails. There is no fallback path.

The functions keep the C names and argument order. Handles are ``int``
(opaque pointers). A status other than ``CSRC_OK`` raises ``CsrcError``.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcsrc_gb300.so")

# status codes (csrc_status)
CSRC_OK = 0
CSRC_ERR_INVALID_ARG = 1
CSRC_ERR_NOT_STRUCT_SYMMETRIC = 2
CSRC_ERR_INDEX_RANGE = 3
CSRC_ERR_DUPLICATE = 4
CSRC_ERR_ALIAS = 5
CSRC_ERR_NOT_PARTITIONED = 6
CSRC_ERR_NOT_COLORED = 7
CSRC_ERR_OUT_OF_MEMORY = 8
CSRC_ERR_CUDA = 9
CSRC_ERR_DEVICE_TIMEOUT = 10
CSRC_ERR_DEVICE_BOUNDS = 11
CSRC_ERR_RANGE = 12
CSRC_ERR_MISMATCH = 13
CSRC_ERR_NOT_NUM_SYMMETRIC = 14
CSRC_ERR_NOT_CONVERGED = 15
CSRC_ERR_BREAKDOWN = 16
CSRC_ERR_NOT_FOUND = 17
CSRC_ERR_IO = 18

# storage (csrc_dtype)
CSRC_F64, CSRC_F32, CSRC_BF16 = 0, 1, 2
# strategies (csrc_strategy)
CSRC_STRAT_AUTO, CSRC_STRAT_WINDOW, CSRC_STRAT_COLOR, CSRC_STRAT_ATOMIC, CSRC_STRAT_WINDOW_ATOMIC = 0, 1, 2, 3, 4
# flags
CSRC_FLAG_PAD_PATTERN, CSRC_FLAG_ONE_BASED, CSRC_FLAG_FP64_ARITH, CSRC_FLAG_NODE_BLOCKS = 1, 2, 4, 8
CSRC_FLAG_SYMMETRIC_VALUES = 16
CSRC_FLAG_COMPRESS_INDICES = 32
CSRC_FLAG_DF32_ARITH = 64

STRATEGIES = {"auto": CSRC_STRAT_AUTO, "window": CSRC_STRAT_WINDOW, "color": CSRC_STRAT_COLOR,
              "atomic": CSRC_STRAT_ATOMIC, "window_atomic": CSRC_STRAT_WINDOW_ATOMIC}
STORAGE = {"f64": CSRC_F64, "f32": CSRC_F32, "bf16": CSRC_BF16}


class CsrcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {csrc_status_string(status)} (status {status})")


class csrc_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("pairs", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("storage", ctypes.c_int32), ("arith", ctypes.c_int32), ("model_bytes", ctypes.c_int64),
        ("nbands", ctypes.c_int32), ("page_rows", ctypes.c_int32), ("spill_entries", ctypes.c_int64),
        ("spill_rows", ctypes.c_int64), ("accum_bytes", ctypes.c_int64), ("max_window_slots", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32), ("ncolors", ctypes.c_int32), ("tuned_strategy", ctypes.c_int32),
        ("tuned_rk", ctypes.c_int32), ("group", ctypes.c_int32), ("nstages", ctypes.c_int64),
        ("block", ctypes.c_int32), ("m", ctypes.c_int64), ("rect_nnz", ctypes.c_int64),
        ("list_entries", ctypes.c_int64), ("list_slices", ctypes.c_int64), ("list_lane_steps", ctypes.c_int64),
        ("list_bytes", ctypes.c_int64), ("stream_nbands", ctypes.c_int32), ("stream_spill_entries", ctypes.c_int64),
        ("precision", ctypes.c_int32), ("error_bound", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class csrc_tune_key(ctypes.Structure):
    _fields_ = [("pattern_hash", ctypes.c_uint64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("storage", ctypes.c_int32), ("flags", ctypes.c_uint32), ("device", ctypes.c_char * 64)]


CSRC_TUNE_STRATEGY, CSRC_TUNE_KTILE, CSRC_TUNE_PRECISION = 0, 1, 2

# kernel kinds (csrc_kernel_times)
CSRC_KERNEL_PRODUCT, CSRC_KERNEL_ACCUMULATE, CSRC_KERNEL_OTHER, CSRC_KERNEL_KINDS = 0, 1, 2, 3
KERNEL_KINDS = ("product", "accumulate", "other")


class csrc_kernel_times(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * CSRC_KERNEL_KINDS), ("ms", ctypes.c_double * CSRC_KERNEL_KINDS)]


# Every entry point of include/csrc.h: name -> (restype, argtypes)
_VP = ctypes.c_void_p
_P = ctypes.POINTER
SIGNATURES = {
    "csrc_create_from_csr": (ctypes.c_int, [_P(_VP), ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int, ctypes.c_uint32, _VP]),
    "csrc_create_from_coo": (ctypes.c_int, [_P(_VP), ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, ctypes.c_int,
                                            ctypes.c_uint32, _VP]),
    "csrc_create_rect_from_csr": (ctypes.c_int, [_P(_VP), ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int,
                                                 ctypes.c_uint32, _VP]),
    "csrc_partition": (ctypes.c_int, [_VP, ctypes.c_int32, _VP]),
    "csrc_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int64]),
    "csrc_bicg": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int32, ctypes.c_int, _P(ctypes.c_int32),
                                 _P(ctypes.c_double), _VP]),
    "csrc_color": (ctypes.c_int, [_VP, ctypes.c_uint64, _P(ctypes.c_int32), _VP]),
    "csrc_color_stride": (ctypes.c_int, [_VP, ctypes.c_int64, _P(ctypes.c_int32), _VP]),
    "csrc_spmv": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "csrc_spmv_t": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "csrc_spmm_batched": (ctypes.c_int, [_P(_VP), ctypes.c_int32, _P(_VP), _P(_VP), ctypes.c_int32, ctypes.c_int32,
                                         _VP]),
    "csrc_spmv_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP]),
    "csrc_autotune": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "csrc_autotune_spmm": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP]),
    "csrc_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "csrc_get_kernel_times": (ctypes.c_int, [_VP, _P(csrc_kernel_times)]),
    "csrc_get_info": (ctypes.c_int, [_VP, _P(csrc_info)]),
    "csrc_get_last_device_error": (ctypes.c_int, [_VP]),
    "csrc_destroy": (ctypes.c_int, [_VP]),
    "csrc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "csrc_set_precision": (ctypes.c_int, [_VP, ctypes.c_int]),
    "csrc_autotune_precision": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_double, _P(ctypes.c_int32),
                                               _P(ctypes.c_double), _VP]),
    "csrc_get_tune_key": (ctypes.c_int, [_VP, _P(csrc_tune_key)]),
    "csrc_tune_cache_lookup": (ctypes.c_int, [_P(csrc_tune_key), ctypes.c_int32, ctypes.c_double,
                                              _P(ctypes.c_int32)]),
    "csrc_tune_cache_store": (ctypes.c_int, [_P(csrc_tune_key), ctypes.c_int32, ctypes.c_double,
                                             _P(ctypes.c_int32)]),
}


def _load():
    # build in-tree when the library is missing or older than its sources
    from . import build as _build

    try:
        _build.build()
    except Exception as e:  # no nvcc, compile error, ...
        raise ImportError(f"cannot build {LIB_PATH}: {e} (there is no CPU fallback)") from e
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def csrc_status_string(status: int) -> str:
    return _lib.csrc_status_string(status).decode()


def _check(status: int, where: str) -> None:
    if status != CSRC_OK:
        raise CsrcError(status, where)


def _ptr(a) -> int | None:
    """Address of a torch tensor, numpy array or raw integer pointer."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        return a.ctypes.data
    raise TypeError(f"cannot take the address of {type(a)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def csrc_create_from_csr(n, row_ptr, col, val, storage=CSRC_F64, flags=0, stream=None) -> int:
    """row_ptr int64[n+1], col int32[nnz], val float64[nnz]: host numpy arrays."""
    import numpy as np
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = _VP()
    _check(_lib.csrc_create_from_csr(ctypes.byref(h), int(n), _ptr(row_ptr), _ptr(col), _ptr(val), int(storage),
                                     int(flags), _stream(stream)), "csrc_create_from_csr")
    return h.value


def csrc_create_rect_from_csr(n, m, row_ptr, col, val, storage=CSRC_F64, flags=0, stream=None) -> int:
    """Rectangular n-by-m matrix (m >= n): row_ptr int64[n+1], col int32[nnz] in [0, m),
    val float64[nnz], host numpy arrays. Products read x of m entries (A x) or n (A^T x)."""
    import numpy as np
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = _VP()
    _check(_lib.csrc_create_rect_from_csr(ctypes.byref(h), int(n), int(m), _ptr(row_ptr), _ptr(col), _ptr(val),
                                          int(storage), int(flags), _stream(stream)), "csrc_create_rect_from_csr")
    return h.value


def csrc_create_from_coo(n, nnz, row, col, val, storage=CSRC_F64, flags=0, stream=None) -> int:
    import numpy as np
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = _VP()
    _check(_lib.csrc_create_from_coo(ctypes.byref(h), int(n), int(nnz), _ptr(row), _ptr(col), _ptr(val),
                                     int(storage), int(flags), _stream(stream)), "csrc_create_from_coo")
    return h.value


def csrc_partition(h, nbands=0, band_ptr_out=None) -> None:
    _check(_lib.csrc_partition(h, int(nbands), _ptr(band_ptr_out)), "csrc_partition")


def csrc_color(h, seed, colors_out=None) -> int:
    nc = ctypes.c_int32(0)
    _check(_lib.csrc_color(h, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), ctypes.byref(nc), _ptr(colors_out)),
           "csrc_color")
    return nc.value


def csrc_color_stride(h, stride, colors_out=None) -> int:
    """Stride-bounded colouring (ascending rows, class gaps of at most stride; 0 = unbounded)."""
    nc = ctypes.c_int32(0)
    _check(_lib.csrc_color_stride(h, int(stride), ctypes.byref(nc), _ptr(colors_out)), "csrc_color_stride")
    return nc.value


def csrc_spmv(h, x, y, strategy=CSRC_STRAT_AUTO, stream=None) -> None:
    _check(_lib.csrc_spmv(h, _ptr(x), _ptr(y), int(strategy), _stream(stream)), "csrc_spmv")


def csrc_spmv_t(h, x, y, strategy=CSRC_STRAT_AUTO, stream=None) -> None:
    _check(_lib.csrc_spmv_t(h, _ptr(x), _ptr(y), int(strategy), _stream(stream)), "csrc_spmv_t")


def csrc_spmm_batched(hs, X, Y, nrhs, transpose=False, stream=None) -> None:
    b = len(hs)
    harr = (_VP * max(b, 1))(*hs)
    xarr = (_VP * max(b, 1))(*[_ptr(x) for x in X])
    yarr = (_VP * max(b, 1))(*[_ptr(y) for y in Y])
    _check(_lib.csrc_spmm_batched(harr, b, xarr, yarr, int(nrhs), int(bool(transpose)), _stream(stream)),
           "csrc_spmm_batched")


CSRC_NOALLOC_MAX_SPILL_ENTRIES = 1 << 21


def csrc_spmv_noalloc(h, x, y, transpose=False, stream=None) -> None:
    """Window-strategy product that allocates nothing (spill in the library's static array)."""
    _check(_lib.csrc_spmv_noalloc(h, _ptr(x), _ptr(y), int(bool(transpose)), _stream(stream)), "csrc_spmv_noalloc")


def csrc_bicg(h, b, x, rtol=1e-10, maxit=1000, strategy=CSRC_STRAT_AUTO, stream=None) -> dict:
    """Solve A x = b by BiCG on the device (x: initial guess in, solution out). Returns
    {"status", "iters", "relres"}; NOT_CONVERGED and BREAKDOWN are reported there, other
    errors raise CsrcError."""
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = _lib.csrc_bicg(h, _ptr(b), _ptr(x), float(rtol), int(maxit), int(strategy), ctypes.byref(it),
                        ctypes.byref(rr), _stream(stream))
    if st not in (CSRC_OK, CSRC_ERR_NOT_CONVERGED, CSRC_ERR_BREAKDOWN):
        _check(st, "csrc_bicg")
    return {"status": st, "iters": it.value, "relres": rr.value}


def csrc_selftest_bounded_wait(cycles=2_000_000) -> int:
    """Run the bounded-wait self-test; returns the status (CSRC_ERR_DEVICE_TIMEOUT expected)."""
    return _lib.csrc_selftest_bounded_wait(int(cycles))


def csrc_autotune(h, x, y, stream=None) -> None:
    _check(_lib.csrc_autotune(h, _ptr(x), _ptr(y), _stream(stream)), "csrc_autotune")


def csrc_set_profiling(h, enable=True) -> None:
    _check(_lib.csrc_set_profiling(h, int(bool(enable))), "csrc_set_profiling")


def csrc_get_kernel_times(h) -> dict:
    """{kind: (launches, milliseconds)} for the launches recorded since profiling was turned on."""
    t = csrc_kernel_times()
    _check(_lib.csrc_get_kernel_times(h, ctypes.byref(t)), "csrc_get_kernel_times")
    return {k: (int(t.launches[i]), float(t.ms[i])) for i, k in enumerate(KERNEL_KINDS)}


def csrc_autotune_spmm(h, X, Y, nrhs, stream=None) -> None:
    _check(_lib.csrc_autotune_spmm(h, _ptr(X), _ptr(Y), int(nrhs), _stream(stream)), "csrc_autotune_spmm")


def csrc_get_info(h) -> dict:
    info = csrc_info()
    _check(_lib.csrc_get_info(h, ctypes.byref(info)), "csrc_get_info")
    return info.as_dict()


def csrc_get_last_device_error(h) -> int:
    """Returns the status code (does not raise)."""
    return _lib.csrc_get_last_device_error(h)


def csrc_destroy(h) -> None:
    _check(_lib.csrc_destroy(h), "csrc_destroy")


def csrc_set_precision(h, precision) -> None:
    """Precision of the window strategy's values (CSRC_F64, CSRC_F32 or CSRC_BF16)."""
    _check(_lib.csrc_set_precision(h, int(precision)), "csrc_set_precision")


def csrc_autotune_precision(h, x, y, max_rel_err, stream=None) -> tuple[int, float]:
    """Pick the fastest precision whose error bound meets max_rel_err; returns (precision, bound)."""
    p = ctypes.c_int32(0)
    b = ctypes.c_double(0.0)
    _check(_lib.csrc_autotune_precision(h, _ptr(x), _ptr(y), float(max_rel_err), ctypes.byref(p), ctypes.byref(b),
                                        _stream(stream)), "csrc_autotune_precision")
    return p.value, b.value


def csrc_get_tune_key(h) -> csrc_tune_key:
    k = csrc_tune_key()
    _check(_lib.csrc_get_tune_key(h, ctypes.byref(k)), "csrc_get_tune_key")
    return k


def csrc_tune_cache_lookup(key, kind, param=0.0):
    """The recorded values (4 ints) for key / kind / param, or None on a miss."""
    v = (ctypes.c_int32 * 4)()
    st = _lib.csrc_tune_cache_lookup(ctypes.byref(key), int(kind), float(param), v)
    if st == CSRC_ERR_NOT_FOUND:
        return None
    _check(st, "csrc_tune_cache_lookup")
    return list(v)


def csrc_tune_cache_store(key, kind, param, values) -> None:
    v = (ctypes.c_int32 * 4)(*[int(a) for a in (list(values) + [0, 0, 0, 0])[:4]])
    _check(_lib.csrc_tune_cache_store(ctypes.byref(key), int(kind), float(param), v), "csrc_tune_cache_store")
