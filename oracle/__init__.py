"""CPU oracle for CSRC SpMV (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline``
/ ``--impl reference`` legs import this package. The library
(``paper_1003_0952_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``csrc_oracle.c``: plain single-threaded FP64 C built
with ``-O2 -ffp-contract=off``. This module marshals numpy arrays and adds
two independent checks written with numpy: a dense brute-force product and a
partition invariant checker.

Every function cites the paper passage it implements (arXiv:1003.0952):
- ``csr_to_csrc``: Section 2 (the CSRC layout).
- ``csrc_spmv``: Fig. 2(a) and Section 2.2.
- ``csrc_spmv_t``: Section 5 (swap al and au).
- ``csr_to_csrcr``, ``csrcr_spmv`` and ``csrcr_spmv_t``: Section 2.1 and Fig. 2(b) (rectangular
  matrices: CSRC square part plus an auxiliary CSR).
- ``csr_spmv``: Section 1 (the CSR product).
- ``bicg``: the biconjugate gradient method (Fletcher 1976, as written in Saad, Iterative Methods for
  Sparse Linear Systems, 2nd ed., Algorithm 7.3), the kind of oblique-projection solver that Section 1
  says benefits from CSRC's implicit transpose; its products are ``csrc_spmv`` and ``csrc_spmv_t``.
- ``partition``: Section 3.1 (non-zero guided bands).
- ``greedy_color`` and ``check_coloring``: Section 3.2 (conflict graph colouring).
- ``working_set_bytes``: Table 1 (ws column).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

I64P = ctypes.POINTER(ctypes.c_int64)
I32P = ctypes.POINTER(ctypes.c_int32)
F64P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_count_lower.restype = ctypes.c_int64
            lib.oracle_count_lower.argtypes = [ctypes.c_int64, I64P, I32P]
            lib.oracle_csr_to_csrc.restype = ctypes.c_int
            lib.oracle_csr_to_csrc.argtypes = [ctypes.c_int64, I64P, I32P, F64P, I64P, I32P, F64P, F64P, F64P]
            for f in (lib.oracle_csrc_spmv, lib.oracle_csrc_spmv_t):
                f.restype = None
                f.argtypes = [ctypes.c_int64, I64P, I32P, F64P, F64P, F64P, F64P, ctypes.c_int64, F64P,
                              ctypes.c_int64]
            lib.oracle_csrcr_spmv.restype = None
            lib.oracle_csrcr_spmv.argtypes = [ctypes.c_int64, I64P, I32P, F64P, F64P, F64P, I64P, I32P, F64P, F64P,
                                              F64P]
            lib.oracle_csrcr_spmv_t.restype = None
            lib.oracle_csrcr_spmv_t.argtypes = [ctypes.c_int64, ctypes.c_int64, I64P, I32P, F64P, F64P, F64P, I64P,
                                                I32P, F64P, F64P, F64P]
            lib.oracle_csrc_spmm.restype = None
            lib.oracle_csrc_spmm.argtypes = [ctypes.c_int64, I64P, I32P, F64P, F64P, F64P, ctypes.c_int64, F64P,
                                             F64P, ctypes.c_int]
            lib.oracle_csr_spmv.restype = None
            lib.oracle_csr_spmv.argtypes = [ctypes.c_int64, I64P, I32P, F64P, F64P, ctypes.c_int64, F64P,
                                            ctypes.c_int64]
            lib.oracle_csr_spmv_rows.restype = None
            lib.oracle_csr_spmv_rows.argtypes = [I64P, I32P, F64P, F64P, ctypes.c_int64, I64P, F64P]
            lib.oracle_max_rel_err.restype = ctypes.c_double
            lib.oracle_max_rel_err.argtypes = [ctypes.c_int64, I64P, I32P, F64P, F64P, ctypes.c_int64, F64P, F64P,
                                               ctypes.c_int64, ctypes.c_int]
            for f in (lib.oracle_round_f32, lib.oracle_round_bf16):
                f.restype = None
                f.argtypes = [F64P, F64P, ctypes.c_int64]
            lib.oracle_partition.restype = None
            lib.oracle_partition.argtypes = [ctypes.c_int64, I64P, ctypes.c_int64, I64P]
            lib.oracle_priority.restype = ctypes.c_uint64
            lib.oracle_priority.argtypes = [ctypes.c_uint64, ctypes.c_int64]
            lib.oracle_priority_order.restype = ctypes.c_int
            lib.oracle_priority_order.argtypes = [ctypes.c_int64, ctypes.c_uint64, I64P]
            lib.oracle_greedy_color.restype = ctypes.c_int64
            lib.oracle_greedy_color.argtypes = [ctypes.c_int64, I64P, I32P, I64P, I32P]
            lib.oracle_greedy_color_stride.restype = ctypes.c_int64
            lib.oracle_greedy_color_stride.argtypes = [ctypes.c_int64, I64P, I32P, ctypes.c_int64, I32P]
            lib.oracle_check_coloring.restype = ctypes.c_int
            lib.oracle_check_coloring.argtypes = [ctypes.c_int64, I64P, I32P, I32P, ctypes.c_int64]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class CSRC:
    """CSRC arrays built by the oracle (Section 2)."""

    def __init__(self, n, ia, ja, al, au, ad):
        self.n, self.ia, self.ja, self.al, self.au, self.ad = n, ia, ja, al, au, ad

    @property
    def pairs(self):
        return int(self.ia[-1])


class OracleError(ValueError):
    pass


def csr_to_csrc(n, row_ptr, col, val) -> CSRC:
    """Section 2: split a full CSR matrix into ad / ia / ja / al / au."""
    lib = _load()
    rp, c, v = _i64(row_ptr), _i32(col), _f64(val)
    h = lib.oracle_count_lower(n, _p(rp, I64P), _p(c, I32P))
    ia = np.empty(n + 1, np.int64)
    ja = np.empty(max(h, 1), np.int32)
    al = np.empty(max(h, 1), np.float64)
    au = np.empty(max(h, 1), np.float64)
    ad = np.empty(max(n, 1), np.float64)
    rc = lib.oracle_csr_to_csrc(n, _p(rp, I64P), _p(c, I32P), _p(v, F64P), _p(ia, I64P), _p(ja, I32P),
                                _p(al, F64P), _p(au, F64P), _p(ad, F64P))
    if rc != 0:
        raise OracleError({1: "pattern not structurally symmetric", 2: "column index out of range",
                           3: "columns not strictly ascending"}[rc])
    return CSRC(n, ia, ja[:h], al[:h], au[:h], ad[:n])


def from_matrix(m) -> CSRC:
    return csr_to_csrc(m.n, m.row_ptr, m.col, m.val)


def _spmv(fn, c: CSRC, x, al=None, au=None, ad=None):
    lib = _load()
    x = _f64(x)
    al = _f64(c.al if al is None else al)
    au = _f64(c.au if au is None else au)
    ad = _f64(c.ad if ad is None else ad)
    ia, ja = _i64(c.ia), _i32(c.ja)
    y = np.full(max(c.n, 1), np.nan)  # Fig. 2(a) needs no initialisation of y
    getattr(lib, fn)(c.n, _p(ia, I64P), _p(ja, I32P), _p(al, F64P), _p(au, F64P), _p(ad, F64P), _p(x, F64P), 1,
                     _p(y, F64P), 1)
    return y[:c.n]


def csrc_spmv(c: CSRC, x, al=None, au=None, ad=None) -> np.ndarray:
    """Fig. 2(a): y = A x in FP64 (optionally with replacement value arrays)."""
    return _spmv("oracle_csrc_spmv", c, x, al, au, ad)


def csrc_spmv_t(c: CSRC, x, al=None, au=None, ad=None) -> np.ndarray:
    """Section 5: y = A^T x, Fig. 2(a) with al and au swapped."""
    return _spmv("oracle_csrc_spmv_t", c, x, al, au, ad)


def csrc_spmm(c: CSRC, X, transpose=False, al=None, au=None, ad=None) -> np.ndarray:
    """Y = A X (or A^T X) for X n-by-r row-major, one Fig. 2(a) product per column."""
    lib = _load()
    X = _f64(X)
    n, r = X.shape
    assert n == c.n
    Y = np.full((max(n, 1), r), np.nan)
    al = _f64(c.al if al is None else al)
    au = _f64(c.au if au is None else au)
    ad = _f64(c.ad if ad is None else ad)
    ia, ja = _i64(c.ia), _i32(c.ja)
    lib.oracle_csrc_spmm(n, _p(ia, I64P), _p(ja, I32P), _p(al, F64P), _p(au, F64P), _p(ad, F64P), r,
                         _p(X, F64P), _p(Y, F64P), int(bool(transpose)))
    return Y[:n]


class CSRCR:
    """Rectangular CSRC (Section 2.1): the square CSRC part and the auxiliary CSR."""

    def __init__(self, n, m, square: CSRC, iar, jar, ar):
        self.n, self.m, self.square, self.iar, self.jar, self.ar = n, m, square, iar, jar, ar


def csr_to_csrcr(n, m, row_ptr, col, val) -> CSRCR:
    """Section 2.1: an n-by-m CSR matrix (m >= n) as A_S + A_R. Columns below n form the
    structurally symmetric square part A_S (stored as CSRC); columns n..m-1 go to the
    auxiliary CSR, which keeps their column numbers."""
    rp, c, v = _i64(row_ptr), _i32(col), _f64(val)
    if m < n:
        raise OracleError("a rectangular CSRC matrix needs m >= n")
    if len(c) and (c.min() < 0 or c.max() >= m):
        raise OracleError("column index out of range")
    rows = np.repeat(np.arange(n), np.diff(rp))
    sq = c < n
    sq_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows[sq], minlength=n), out=sq_ptr[1:])
    ar_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows[~sq], minlength=n), out=ar_ptr[1:])
    square = csr_to_csrc(n, sq_ptr, c[sq], v[sq])
    return CSRCR(n, m, square, ar_ptr, _i32(c[~sq]), _f64(v[~sq]))


def csrcr_spmv(r: CSRCR, x) -> np.ndarray:
    """Fig. 2(b): y = A x for the rectangular matrix (x has m entries, y has n)."""
    lib = _load()
    c = r.square
    x = _f64(x)
    assert len(x) == r.m
    y = np.full(max(r.n, 1), np.nan)
    ia, ja = _i64(c.ia), _i32(c.ja)
    al, au, ad = _f64(c.al), _f64(c.au), _f64(c.ad)
    iar, jar, ar = _i64(r.iar), _i32(r.jar), _f64(r.ar)
    lib.oracle_csrcr_spmv(r.n, _p(ia, I64P), _p(ja, I32P), _p(al, F64P), _p(au, F64P), _p(ad, F64P),
                          _p(iar, I64P), _p(jar, I32P), _p(ar, F64P), _p(x, F64P), _p(y, F64P))
    return y[:r.n]


def csrcr_spmv_t(r: CSRCR, x) -> np.ndarray:
    """y = A^T x for the rectangular matrix (x has n entries, y has m)."""
    lib = _load()
    c = r.square
    x = _f64(x)
    assert len(x) == r.n
    y = np.full(max(r.m, 1), np.nan)
    ia, ja = _i64(c.ia), _i32(c.ja)
    al, au, ad = _f64(c.al), _f64(c.au), _f64(c.ad)
    iar, jar, ar = _i64(r.iar), _i32(r.jar), _f64(r.ar)
    lib.oracle_csrcr_spmv_t(r.n, r.m, _p(ia, I64P), _p(ja, I32P), _p(al, F64P), _p(au, F64P), _p(ad, F64P),
                            _p(iar, I64P), _p(jar, I32P), _p(ar, F64P), _p(x, F64P), _p(y, F64P))
    return y[:r.m]


def max_rel_err_rect(n, m, row_ptr, col, val, x, y, yref, transpose=False) -> float:
    """The error metric of ``max_rel_err`` for an n-by-m matrix: per output entry,
    |y - yref| / sum |a||x| over its row of A (over its column of A for A^T)."""
    rp, c, v = _i64(row_ptr), _i32(col), np.abs(_f64(val))
    rows = np.repeat(np.arange(n), np.diff(rp))
    x = np.abs(_f64(x))
    if transpose:
        den = np.zeros(m)
        np.add.at(den, c, v * x[rows])
    else:
        den = np.zeros(n)
        np.add.at(den, rows, v * x[c])
    d = np.abs(_f64(y) - _f64(yref))
    if np.isnan(d).any():
        return float("nan")
    e = np.where(den > 0, d / np.where(den > 0, den, 1.0), d)
    return float(e.max()) if len(e) else 0.0


def dense_rect(n, m, row_ptr, col, val) -> np.ndarray:
    """Brute force: the dense n-by-m matrix built entry by entry."""
    a = np.zeros((n, m))
    for i in range(n):
        for p in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            a[i, int(col[p])] += float(val[p])
    return a


class SolveResult:
    def __init__(self, x, iters, relres, status):
        self.x, self.iters, self.relres, self.status = x, iters, relres, status


def bicg(c: CSRC, b, x0=None, rtol=1e-10, maxit=1000) -> SolveResult:
    """Biconjugate gradients for A x = b (Saad, Algorithm 7.3, with the shadow residual
    r*_0 = r_0). Every iteration takes one product with A (Fig. 2(a)) and one with A^T
    (Section 5: al and au swapped). Stops when ||r||_2 <= rtol ||b||_2; status "converged",
    "maxit" or "breakdown" (a zero (r, r*) or (A p, p*))."""
    b = _f64(b)
    x = np.zeros(c.n) if x0 is None else _f64(x0).copy()
    r = b - csrc_spmv(c, x)
    rs = r.copy()
    p, ps = r.copy(), rs.copy()
    rho = float(r @ rs)
    bnorm = float(np.sqrt(b @ b))
    tol = rtol * bnorm
    nrm = float(np.sqrt(r @ r))
    if nrm <= tol:
        return SolveResult(x, 0, nrm / bnorm if bnorm > 0 else 0.0, "converged")
    for it in range(1, maxit + 1):
        q = csrc_spmv(c, p)
        qs = csrc_spmv_t(c, ps)
        sigma = float(q @ ps)
        if rho == 0.0 or sigma == 0.0:
            return SolveResult(x, it - 1, nrm / bnorm, "breakdown")
        alpha = rho / sigma
        x = x + alpha * p
        r = r - alpha * q
        rs = rs - alpha * qs
        nrm = float(np.sqrt(r @ r))
        if nrm <= tol:
            return SolveResult(x, it, nrm / bnorm, "converged")
        rho_new = float(r @ rs)
        beta = rho_new / rho
        rho = rho_new
        p = r + beta * p
        ps = rs + beta * ps
    return SolveResult(x, maxit, nrm / bnorm, "maxit")


def csr_spmv(n, row_ptr, col, val, x) -> np.ndarray:
    """Section 1: the plain CSR product on the original full matrix."""
    lib = _load()
    rp, c, v, x = _i64(row_ptr), _i32(col), _f64(val), _f64(x)
    y = np.empty(max(n, 1))
    lib.oracle_csr_spmv(n, _p(rp, I64P), _p(c, I32P), _p(v, F64P), _p(x, F64P), 1, _p(y, F64P), 1)
    return y[:n]


def csr_spmv_rows(row_ptr, col, val, x, rows) -> np.ndarray:
    """Selected rows of the CSR product (sampled checks at full size)."""
    lib = _load()
    rp, c, v, x, rows = _i64(row_ptr), _i32(col), _f64(val), _f64(x), _i64(rows)
    y = np.empty(max(len(rows), 1))
    lib.oracle_csr_spmv_rows(_p(rp, I64P), _p(c, I32P), _p(v, F64P), _p(x, F64P), len(rows), _p(rows, I64P),
                             _p(y, F64P))
    return y[:len(rows)]


def dense_spmv(n, row_ptr, col, val, x) -> np.ndarray:
    """Brute force: build the dense matrix entry by entry and multiply (numpy matmul)."""
    a = np.zeros((n, n))
    for i in range(n):
        for p in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            a[i, int(col[p])] += float(val[p])
    return a @ np.asarray(x, dtype=np.float64)


def max_rel_err(m, x, y, yref, transpose=False) -> float:
    """max_i |y_i - yref_i| / sum_j |a_ij||x_j| (original FP64 values; column sums for A^T)."""
    lib = _load()
    x = _f64(x).reshape(m.n, -1)
    y = _f64(y).reshape(m.n, -1)
    yref = _f64(yref).reshape(m.n, -1)
    r = x.shape[1]
    rp, c, v = _i64(m.row_ptr), _i32(m.col), _f64(m.val)
    worst = 0.0
    for k in range(r):
        xk, yk, rk = _f64(x[:, k]), _f64(y[:, k]), _f64(yref[:, k])
        e = lib.oracle_max_rel_err(m.n, _p(rp, I64P), _p(c, I32P), _p(v, F64P), _p(xk, F64P), 1, _p(yk, F64P),
                                   _p(rk, F64P), 1, int(bool(transpose)))
        if e != e:
            return float("nan")
        worst = max(worst, e)
    return worst


def round_f32(a) -> np.ndarray:
    """FP64 -> FP32 (nearest, ties to even), returned widened to FP64."""
    lib = _load()
    a = _f64(a)
    out = np.empty_like(a)
    lib.oracle_round_f32(_p(a, F64P), _p(out, F64P), a.size)
    return out


def round_bf16(a) -> np.ndarray:
    """FP64 -> BF16 directly (8 significant bits, nearest, ties to even), widened to FP64."""
    lib = _load()
    a = _f64(a)
    out = np.empty_like(a)
    lib.oracle_round_bf16(_p(a, F64P), _p(out, F64P), a.size)
    return out


def quantised(c: CSRC, storage: str):
    """(al, au, ad) as stored by a reduced-precision handle, widened to FP64."""
    f = {"f64": lambda a: _f64(a), "f32": round_f32, "bf16": round_bf16}[storage]
    return f(c.al), f(c.au), f(c.ad)


def partition(c: CSRC, nbands: int) -> np.ndarray:
    """Section 3.1: non-zero guided contiguous row bands (boundaries b_0..b_B)."""
    lib = _load()
    ia = _i64(c.ia)
    out = np.empty(nbands + 1, np.int64)
    lib.oracle_partition(c.n, _p(ia, I64P), nbands, _p(out, I64P))
    return out


def check_partition(ia, nbands, band_ptr) -> None:
    """Invariants of the Section 3.1 partition, computed independently with numpy.

    For each 0 < t < B: P(b_t) * B >= t*nnz and P(b_t - 1) * B < t*nnz (b_t is the
    first row boundary that reaches the t-th share); b_0 = 0, b_B = n, and the
    boundaries are non-decreasing.
    """
    ia = np.asarray(ia, dtype=np.int64)
    n = len(ia) - 1
    w = 1 + 2 * np.diff(ia)
    P = np.zeros(n + 1, dtype=object)
    P[1:] = np.cumsum(w).astype(object)
    nnz = int(P[n]) if n > 0 else 0
    b = [int(v) for v in band_ptr]
    if len(b) != nbands + 1:
        raise AssertionError("wrong number of boundaries")
    if b[0] != 0 or b[-1] != n:
        raise AssertionError("endpoints")
    for t in range(1, nbands):
        if b[t] < b[t - 1]:
            raise AssertionError("not monotone")
        if P[b[t]] * nbands < t * nnz:
            raise AssertionError(f"boundary {t} short of its share")
        if b[t] > 0 and P[b[t] - 1] * nbands >= t * nnz:
            raise AssertionError(f"boundary {t} not the first to reach its share")


def priority(seed: int, i: int) -> int:
    """Jones-Plassmann priority of row i: SplitMix64(seed XOR i)."""
    return int(_load().oracle_priority(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), i))


def priority_order(n: int, seed: int) -> np.ndarray:
    lib = _load()
    out = np.empty(max(n, 1), np.int64)
    lib.oracle_priority_order(n, ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _p(out, I64P))
    return out[:n]


def greedy_color(c: CSRC, order) -> tuple[int, np.ndarray]:
    """Section 3.2: greedy colouring of the write-conflict graph in the given order."""
    lib = _load()
    ia, ja, order = _i64(c.ia), _i32(c.ja), _i64(order)
    colors = np.empty(max(c.n, 1), np.int32)
    k = lib.oracle_greedy_color(c.n, _p(ia, I64P), _p(ja if len(ja) else np.zeros(1, np.int32), I32P),
                                _p(order, I64P), _p(colors, I32P))
    if k < 0:
        raise MemoryError
    return int(k), colors[:c.n]


def greedy_color_stride(c: CSRC, stride: int) -> tuple[int, np.ndarray]:
    """Stride-bounded greedy colouring (the future work of Section 6), in ascending row order:
    first fit among the colours without a conflict whose last member lies at most `stride`
    rows back; stride <= 0 means no bound."""
    lib = _load()
    ia, ja = _i64(c.ia), _i32(c.ja)
    colors = np.empty(max(c.n, 1), np.int32)
    k = lib.oracle_greedy_color_stride(c.n, _p(ia, I64P), _p(ja if len(ja) else np.zeros(1, np.int32), I32P),
                                       int(stride), _p(colors, I32P))
    if k < 0:
        raise MemoryError
    return int(k), colors[:c.n]


def max_class_gap(colors, ncolors: int) -> int:
    """Largest distance between consecutive rows of one colour class (0 for classes of one row)."""
    colors = np.asarray(colors)
    worst = 0
    for k in range(ncolors):
        rows = np.nonzero(colors == k)[0]
        if len(rows) > 1:
            worst = max(worst, int(np.diff(rows).max()))
    return worst


def jp_color(c: CSRC, seed: int) -> tuple[int, np.ndarray]:
    """The colouring Jones-Plassmann reaches: greedy in decreasing SplitMix64 priority."""
    return greedy_color(c, priority_order(c.n, seed))


def check_coloring(c: CSRC, colors, ncolors: int) -> int:
    """0 if every colour class has pairwise disjoint write sets, else non-zero."""
    lib = _load()
    ia, ja, colors = _i64(c.ia), _i32(c.ja), _i32(colors)
    return int(lib.oracle_check_coloring(c.n, _p(ia, I64P), _p(ja if len(ja) else np.zeros(1, np.int32), I32P),
                                         _p(colors, I32P), ncolors))


def working_set_bytes(n: int, pairs: int, symmetric: bool = False, value_bytes: int = 8, index_bytes: int = 4,
                      x_bytes: int = 8, y_bytes: int = 8) -> int:
    """Bytes of the arrays one CSRC product touches (Table 1's ws): ia, ja, al, [au], ad, x, y.

    A numerically symmetric matrix stores no au (Section 2.2).
    """
    ia = index_bytes * (n + 1)
    ja = index_bytes * pairs
    vals = value_bytes * pairs * (1 if symmetric else 2)
    ad = value_bytes * n
    return ia + ja + vals + ad + x_bytes * n + y_bytes * n
