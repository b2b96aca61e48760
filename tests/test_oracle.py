"""Pins for the CPU oracle against facts that the paper and the mathematics fix.

Nothing here compares the oracle with itself. Each test checks it against a
brute-force definition, an exact integer result, a closed form, an identity,
or the paper's printed Table 1. So a dropped term, a wrong sign, a swapped
al/au or a wrong index fails at least one test.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import fe_inputs as fe
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mat(n, rp, c, val, name="t"):
    return fe.FEMatrix(n, rp, c, val, name)


def _random_matrix(n, density, seed, empty_rows=True):
    rp, c = fe.random_symmetric_pattern(n, density, seed, empty_rows=empty_rows)
    return _mat(n, rp, c, fe.random_fe_values(rp, c, seed + 7))


SMALL = [(1, 0.0, 1), (2, 1.0, 2), (5, 0.5, 3), (9, 0.4, 4), (17, 0.3, 5), (33, 0.2, 6), (64, 0.1, 7),
         (64, 0.9, 8), (40, 0.02, 9)]


# --------------------------------------------------------------------------- Section 2 / Fig. 2(a)
@pytest.mark.parametrize("n,density,seed", SMALL)
def test_csrc_spmv_matches_dense_brute_force(n, density, seed):
    m = _random_matrix(n, density, seed)
    c = oracle.from_matrix(m)
    assert c.pairs == (m.nnz - n) // 2
    x = fe.source_vector(n, seed)
    y = oracle.csrc_spmv(c, x)
    yd = oracle.dense_spmv(n, m.row_ptr, m.col, m.val, x)
    assert oracle.max_rel_err(m, x, y, yd) <= 1e-15
    ycsr = oracle.csr_spmv(n, m.row_ptr, m.col, m.val, x)
    assert oracle.max_rel_err(m, x, ycsr, yd) <= 1e-15


@pytest.mark.parametrize("n,density,seed", SMALL)
def test_integer_values_are_exact(n, density, seed):
    rp, c = fe.random_symmetric_pattern(n, density, seed)
    m = _mat(n, rp, c, fe.integer_values(rp, c, seed))
    cc = oracle.from_matrix(m)
    x = fe.integer_vector(n, seed)
    yd = oracle.dense_spmv(n, rp, c, m.val, x)
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, x), yd)
    np.testing.assert_array_equal(oracle.csr_spmv(n, rp, c, m.val, x), yd)
    # transpose against the explicit transpose built by scipy
    at = sp.csr_matrix((m.val, c, rp), shape=(n, n)).T.tocsr()
    ydt = oracle.dense_spmv(n, at.indptr, at.indices, at.data, x)
    np.testing.assert_array_equal(oracle.csrc_spmv_t(cc, x), ydt)


def test_conversion_layout_small_hand_example():
    # A 4x4 matrix written out by hand:
    #   [10  1  0  2]
    #   [ 3 20  4  0]
    #   [ 0  5 30  6]
    #   [ 7  0  8 40]
    dense = np.array([[10, 1, 0, 2], [3, 20, 4, 0], [0, 5, 30, 6], [7, 0, 8, 40]], dtype=float)
    a = sp.csr_matrix(dense)
    c = oracle.csr_to_csrc(4, a.indptr, a.indices, a.data)
    # lower entries row by row: (1,0)=3, (2,1)=5, (3,0)=7, (3,2)=8; au holds the mirrors a_ji
    np.testing.assert_array_equal(c.ia, [0, 0, 1, 2, 4])
    np.testing.assert_array_equal(c.ja, [0, 1, 0, 2])
    np.testing.assert_array_equal(c.al, [3, 5, 7, 8])
    np.testing.assert_array_equal(c.au, [1, 4, 2, 6])
    np.testing.assert_array_equal(c.ad, [10, 20, 30, 40])
    x = np.array([1.0, -2.0, 3.0, 0.5])
    np.testing.assert_array_equal(oracle.csrc_spmv(c, x), dense @ x)
    np.testing.assert_array_equal(oracle.csrc_spmv_t(c, x), dense.T @ x)


def test_conversion_rejects_bad_input():
    # a_01 present without a_10
    rp = np.array([0, 2, 3]); col = np.array([0, 1, 1]); val = np.ones(3)
    with pytest.raises(oracle.OracleError, match="symmetric"):
        oracle.csr_to_csrc(2, rp, col, val)
    rp = np.array([0, 2, 4]); col = np.array([1, 0, 0, 1]); val = np.ones(4)
    with pytest.raises(oracle.OracleError, match="ascending"):
        oracle.csr_to_csrc(2, rp, col, val)
    rp = np.array([0, 1, 2]); col = np.array([0, 5]); val = np.ones(2)
    with pytest.raises(oracle.OracleError, match="range"):
        oracle.csr_to_csrc(2, rp, col, val)


# --------------------------------------------------------------------------- Section 5 (transpose)
@pytest.mark.parametrize("n,density,seed", SMALL[1:])
def test_transpose_matches_explicit_transpose_and_bilinear_identity(n, density, seed):
    m = _random_matrix(n, density, seed)
    c = oracle.from_matrix(m)
    x = fe.source_vector(n, seed + 1)
    y = fe.source_vector(n, seed + 2)
    at = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(n, n)).T.tocsr()
    mt = _mat(n, at.indptr, at.indices, at.data)
    yt = oracle.csrc_spmv_t(c, x)
    ref = oracle.csr_spmv(n, at.indptr, at.indices, at.data, x)
    assert oracle.max_rel_err(mt, x, yt, ref) <= 1e-15
    # y^T (A x) == x^T (A^T y)
    lhs = float(y @ oracle.csrc_spmv(c, x))
    rhs = float(x @ oracle.csrc_spmv_t(c, y))
    scale = float(np.abs(y) @ (abs(sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(n, n))) @ np.abs(x)))
    assert abs(lhs - rhs) <= 1e-14 * max(scale, 1.0)


def test_symmetric_values_transpose_is_bitwise_identical():
    rp, c = fe.q1_hex27_pattern(6, 5, 4)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    lo, hi = np.minimum(rows, c), np.maximum(rows, c)
    val = fe.hash_uniform(11, lo, hi)  # a_ij == a_ji
    m = _mat(n, rp, c, val)
    cc = oracle.from_matrix(m)
    np.testing.assert_array_equal(cc.al, cc.au)
    x = fe.source_vector(n, 3)
    y1 = oracle.csrc_spmv(cc, x)
    np.testing.assert_array_equal(y1, oracle.csrc_spmv_t(cc, x))
    assert oracle.max_rel_err(m, x, y1, oracle.dense_spmv(n, rp, c, val, x)) <= 1e-15


# --------------------------------------------------------------------------- closed forms
def _grid_coords(nx, ny, nz):
    ids = np.arange(nx * ny * nz)
    return ids % nx, (ids // nx) % ny, ids // (nx * ny)


def test_27_point_laplacian_closed_forms():
    nx, ny, nz = 9, 8, 7
    rp, c = fe.q1_hex27_pattern(nx, ny, nz)
    n = len(rp) - 1
    val = fe.laplacian_values(rp, c)
    cc = oracle.from_matrix(_mat(n, rp, c, val))
    ix, iy, iz = _grid_coords(nx, ny, nz)
    interior = (ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1) & (iz > 0) & (iz < nz - 1)
    # A 1 = 0 on every row (zero row sums)
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, np.ones(n)), np.zeros(n))
    # discrete Laplacian of a linear field vanishes in the interior
    f = 3.0 * ix - 2.0 * iy + 5.0 * iz + 1.0
    y = oracle.csrc_spmv(cc, f)
    np.testing.assert_array_equal(y[interior], 0.0)
    # f = ix^2: sum over the 26 neighbours of (ix^2 - (ix+dx)^2) = -sum dx^2 = -18
    y = oracle.csrc_spmv(cc, ix.astype(float) ** 2)
    np.testing.assert_array_equal(y[interior], -18.0)


def test_convection_diffusion_closed_forms_distinguish_a_and_at():
    nx, ny, nz = 8, 7, 6
    rp, c = fe.q1_hex27_pattern(nx, ny, nz)
    n = len(rp) - 1
    ix, iy, iz = _grid_coords(nx, ny, nz)
    beta = 0.25
    val = fe.convection_values(rp, c, ix.astype(float), beta)
    cc = oracle.from_matrix(_mat(n, rp, c, val))
    interior = (ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1) & (iz > 0) & (iz < nz - 1)
    f = ix.astype(float)
    # (A f)_i = sum_j (1 + beta dx)(f_i - f_j) = -beta * sum dx^2 = -18 beta
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, f)[interior], -18 * beta)
    # (A^T f)_i = +18 beta: an al/au swap flips the sign
    np.testing.assert_array_equal(oracle.csrc_spmv_t(cc, f)[interior], 18 * beta)
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, np.ones(n)), 0.0)


def test_p1_triangle_stiffness_closed_forms():
    nx, ny = 12, 9
    ei, ej = fe.p1_triangle_grid_edges(nx, ny)
    rp, c = fe.pattern_from_edges(nx * ny, ei, ej)
    n = nx * ny
    rows = np.repeat(np.arange(n), np.diff(rp))
    # P1 Laplace stiffness on right triangles: -1 on axis edges, 0 on the diagonals
    # (kept in the pattern as explicit zeros), and zero row sums.
    d = c - rows
    axis = (np.abs(d) == 1) | (np.abs(d) == nx)
    val = np.where(rows == c, 0.0, np.where(axis, -1.0, 0.0))
    deg = np.bincount(rows[axis], minlength=n).astype(float)
    val[rows == c] = deg
    cc = oracle.from_matrix(_mat(n, rp, c, val))
    ix, iy = np.arange(n) % nx, np.arange(n) // nx
    interior = (ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1)
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, 2.0 * ix + 3.0 * iy)[interior], 0.0)
    np.testing.assert_array_equal(oracle.csrc_spmv(cc, ix.astype(float) ** 2)[interior], -2.0)


# --------------------------------------------------------------------------- several right-hand sides
# --------------------------------------------------------------------------- Section 2.1 / Fig. 2(b)
def _random_rect(n, extra, density, seed, integer=False):
    """Square symmetric pattern plus random entries in `extra` extra columns."""
    rp, c = fe.random_symmetric_pattern(n, density, seed)
    rng = np.random.default_rng(seed + 100)
    rows = [list(c[rp[i]:rp[i + 1]]) for i in range(n)]
    for i in range(n):
        if extra:
            k = int(rng.integers(0, min(extra, 4) + 1))
            rows[i] += sorted(set(int(v) for v in n + rng.integers(0, extra, size=k)))
    ptr = np.zeros(n + 1, np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([v for r in rows for v in r], dtype=np.int32)
    if integer:
        val = rng.integers(-8, 9, size=len(col)).astype(np.float64)
    else:
        val = rng.uniform(-1.0, 1.0, size=len(col))
    return fe.RectMatrix(n, n + extra, ptr, col, val)


RECT = [(1, 0, 0.0, 1), (1, 3, 0.0, 2), (5, 2, 0.5, 3), (9, 7, 0.4, 4), (33, 5, 0.2, 5), (64, 40, 0.1, 6)]


@pytest.mark.parametrize("n,extra,density,seed", RECT)
def test_rectangular_product_matches_dense_brute_force(n, extra, density, seed):
    a = _random_rect(n, extra, density, seed)
    r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
    d = oracle.dense_rect(a.n, a.m, a.row_ptr, a.col, a.val)
    x = fe.source_vector(a.m, seed)
    np.testing.assert_allclose(oracle.csrcr_spmv(r, x), d @ x, rtol=1e-13, atol=1e-13)
    xt = fe.source_vector(a.n, seed + 1)
    np.testing.assert_allclose(oracle.csrcr_spmv_t(r, xt), d.T @ xt, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n,extra,density,seed", RECT)
def test_rectangular_integer_values_exact_and_bilinear(n, extra, density, seed):
    a = _random_rect(n, extra, density, seed, integer=True)
    r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
    d = oracle.dense_rect(a.n, a.m, a.row_ptr, a.col, a.val)
    x = fe.integer_vector(a.m, seed)
    u = fe.integer_vector(a.n, seed + 2)
    y = oracle.csrcr_spmv(r, x)
    np.testing.assert_array_equal(y, d @ x)
    # the CSR product of the whole n-by-m matrix (Section 1) gives the same rows
    np.testing.assert_array_equal(y, oracle.csr_spmv(a.n, a.row_ptr, a.col, a.val, x))
    yt = oracle.csrcr_spmv_t(r, u)
    np.testing.assert_array_equal(yt, d.T @ u)
    assert float(u @ y) == float(yt @ x)  # u^T (A x) = (A^T u)^T x, exact in integers


def test_rectangular_without_extra_columns_is_the_square_product():
    m = _random_matrix(33, 0.3, 11)
    r = oracle.csr_to_csrcr(m.n, m.n, m.row_ptr, m.col, m.val)
    c = oracle.from_matrix(m)
    x = fe.source_vector(m.n, 12)
    np.testing.assert_array_equal(oracle.csrcr_spmv(r, x), oracle.csrc_spmv(c, x))
    np.testing.assert_array_equal(oracle.csrcr_spmv_t(r, x), oracle.csrc_spmv_t(c, x))


def test_overlap_subdomain_rows_equal_the_global_product():
    # one subdomain of an overlapping decomposition: its rows of the global product, with x
    # zero outside the subdomain and its overlap
    g = fe.q1_hex(6, 3, 13)
    a = fe.overlap_subdomain(g, g.n // 2)
    assert a.m > a.n
    r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
    xs = fe.integer_vector(a.m, 14)
    xg = np.zeros(g.n)
    xg[:a.n] = xs[:a.n]
    xg[a.meta["overlap"]] = xs[a.n:]
    yg = oracle.csrc_spmv(oracle.from_matrix(fe.FEMatrix(g.n, g.row_ptr, g.col,
                                                         np.round(g.val * 8.0))), xg)
    ar = fe.RectMatrix(a.n, a.m, a.row_ptr, a.col, np.round(a.val * 8.0))
    rr = oracle.csr_to_csrcr(ar.n, ar.m, ar.row_ptr, ar.col, ar.val)
    np.testing.assert_array_equal(oracle.csrcr_spmv(rr, xs), yg[:a.n])
    # the square part is the global matrix's leading principal block
    sq = sp.csr_matrix((g.val, g.col, g.row_ptr), shape=(g.n, g.n))[:a.n, :a.n].tocsr()
    sq.sort_indices()
    np.testing.assert_array_equal(r.square.ad, sq.diagonal())


def test_rectangular_error_metric_and_rejections():
    a = _random_rect(9, 7, 0.4, 21)
    r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
    x = fe.source_vector(a.m, 22)
    y = oracle.csrcr_spmv(r, x)
    assert oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, x, y, y) == 0.0
    # dropping one auxiliary term is seen at the level of that term
    i = int(np.argmax(np.diff(r.iar)))
    k = int(r.iar[i])
    bad = y.copy()
    bad[i] -= r.ar[k] * x[r.jar[k]]
    assert oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, x, bad, y) > 1e-3
    with pytest.raises(oracle.OracleError):
        oracle.csr_to_csrcr(a.n, a.n - 1, a.row_ptr, a.col, a.val)


# --------------------------------------------------------------------------- BiCG (Section 1's oblique-projection solvers)
@pytest.mark.parametrize("n,density,seed", [(5, 0.5, 91), (40, 0.2, 92), (120, 0.05, 93)])
def test_bicg_solves_against_dense_direct_solution(n, density, seed):
    m = _random_matrix(n, density, seed, empty_rows=False)  # diagonally dominant (ad = 1 + sum |a|)
    c = oracle.from_matrix(m)
    xt = fe.source_vector(n, seed + 1)
    b = oracle.dense_spmv(n, m.row_ptr, m.col, m.val, xt)
    res = oracle.bicg(c, b, rtol=1e-13, maxit=10 * n)
    assert res.status == "converged"
    a = np.zeros((n, n))
    for i in range(n):
        a[i, m.col[m.row_ptr[i]:m.row_ptr[i + 1]]] = m.val[m.row_ptr[i]:m.row_ptr[i + 1]]
    np.testing.assert_allclose(res.x, np.linalg.solve(a, b), rtol=1e-9, atol=1e-11)
    # the true residual (CSR product, Section 1) meets the tolerance up to the rounding drift of
    # the recursively updated one
    r = b - oracle.csr_spmv(n, m.row_ptr, m.col, m.val, res.x)
    assert np.linalg.norm(r) <= max(1e-13, res.relres) * 10.0 * np.linalg.norm(b)


def test_bicg_on_symmetric_spd_matches_conjugate_gradients():
    # with a = a^T and r*_0 = r_0 BiCG's iterates are those of CG (Saad, Section 7.3.1)
    rp, c = fe.q1_hex27_pattern(6, 6, 6)
    n = len(rp) - 1
    m = fe.FEMatrix(n, rp, c, fe.laplacian_values(rp, c) + 0.0)
    diag = np.repeat(np.arange(n), np.diff(rp)) == c
    m.val[diag] += 1.0  # 27-point Laplacian plus identity: SPD
    cc = oracle.from_matrix(m)
    b = fe.source_vector(n, 94)
    res = oracle.bicg(cc, b, rtol=1e-12, maxit=500)
    # plain CG written out here with scipy's sparse product (an independent product)
    a = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(n, n))
    x = np.zeros(n)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    it = 0
    while np.sqrt(rr) > 1e-12 * np.linalg.norm(b):
        q = a @ p
        al = rr / (p @ q)
        x += al * p
        r -= al * q
        rr2 = r @ r
        p = r + (rr2 / rr) * p
        rr = rr2
        it += 1
    assert res.status == "converged"
    assert abs(res.iters - it) <= 1
    np.testing.assert_allclose(res.x, x, rtol=1e-9, atol=1e-12)


def test_bicg_reports_maxit_and_zero_rhs():
    m = _random_matrix(30, 0.2, 95, empty_rows=False)
    c = oracle.from_matrix(m)
    b = fe.source_vector(30, 96)
    res = oracle.bicg(c, b, rtol=1e-14, maxit=2)
    assert res.status == "maxit" and res.iters == 2 and res.relres > 1e-14
    res = oracle.bicg(c, np.zeros(30), rtol=1e-10)
    assert res.status == "converged" and res.iters == 0 and np.all(res.x == 0)


def test_spmm_columns_match_dense():
    m = _random_matrix(30, 0.2, 21)
    c = oracle.from_matrix(m)
    X = fe.source_vector(30, 5, nrhs=7)
    Y = oracle.csrc_spmm(c, X)
    dense = np.zeros((30, 30))
    for i in range(30):
        for p in range(m.row_ptr[i], m.row_ptr[i + 1]):
            dense[i, m.col[p]] = m.val[p]
    assert np.max(np.abs(Y - dense @ X)) <= 1e-14 * np.max(np.abs(dense) @ np.abs(X))
    Yt = oracle.csrc_spmm(c, X, transpose=True)
    assert np.max(np.abs(Yt - dense.T @ X)) <= 1e-14 * np.max(np.abs(dense.T) @ np.abs(X))


# --------------------------------------------------------------------------- error metric
def test_error_metric_detects_a_dropped_term():
    m = _random_matrix(20, 0.3, 31)
    c = oracle.from_matrix(m)
    x = fe.source_vector(20, 31)
    y = oracle.csrc_spmv(c, x)
    # plant a mistake in the oracle's arrays: drop the scatter of one pair
    au_bad = c.au.copy()
    au_bad[len(au_bad) // 2] = 0.0
    y_bad = oracle.csrc_spmv(c, x, au=au_bad)
    assert oracle.max_rel_err(m, x, y_bad, y) > 1e-6
    assert oracle.max_rel_err(m, x, y, y) == 0.0


def _lopsided(n, density, seed):
    """A random structurally symmetric matrix whose upper-triangle values are 1000 times
    larger than the lower ones, so that the row sums and the column sums of |A| differ."""
    m = _random_matrix(n, density, seed)
    rows = np.repeat(np.arange(n), np.diff(m.row_ptr))
    val = np.where(m.col > rows, 1000.0, 1.0) * m.val
    return fe.FEMatrix(n, m.row_ptr, m.col, val)


@pytest.mark.parametrize("transpose", [False, True])
def test_error_metric_denominator_brute_force(transpose):
    # the metric of A x divides by the row sums of |A||x|, that of A^T x by the column sums
    # (the rows of A^T): one perturbed entry at a time, against a dense brute force
    n = 24
    m = _lopsided(n, 0.3, 41)
    x = fe.source_vector(n, 42)
    dense = np.abs(oracle.dense_rect(n, n, m.row_ptr, m.col, m.val))
    den = (dense.T if transpose else dense) @ np.abs(x)
    other = (dense if transpose else dense.T) @ np.abs(x)
    yref = fe.source_vector(n, 43)
    checked = 0
    for i in range(n):
        if den[i] == 0.0:
            continue
        y = yref.copy()
        y[i] += 1e-3 * den[i]
        e = oracle.max_rel_err(m, x, y, yref, transpose=transpose)
        assert e == pytest.approx(1e-3, rel=1e-9)
        # a denominator of the wrong orientation gives a visibly different value here
        if abs(other[i] - den[i]) > 0.5 * den[i]:
            assert abs(1e-3 * den[i] / other[i] - e) > 1e-4
            checked += 1
    assert checked > n // 3


@pytest.mark.parametrize("transpose", [False, True])
def test_rect_error_metric_denominator_brute_force(transpose):
    # the n-by-m form: A x over rows of A, A^T x over columns of A (m outputs)
    n, mm = 15, 21
    rng = np.random.default_rng(44)
    dense = np.where(rng.random((n, mm)) < 0.35, rng.uniform(-1, 1, (n, mm)), 0.0)
    dense[:, 16] = 0.0  # an empty column: the metric takes the absolute difference there
    dense *= np.where(np.arange(mm)[None, :] >= n, 1000.0, 1.0)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum((dense != 0).sum(axis=1), out=rp[1:])
    col = np.nonzero(dense)[1].astype(np.int32)
    val = dense[dense != 0]
    xlen, ylen = (n, mm) if transpose else (mm, n)
    x = fe.source_vector(xlen, 45)
    den = (np.abs(dense).T if transpose else np.abs(dense)) @ np.abs(x)
    yref = fe.source_vector(ylen, 46)
    for i in range(ylen):
        y = yref.copy()
        y[i] += 2e-3 * max(den[i], 1.0)
        e = oracle.max_rel_err_rect(n, mm, rp, col, val, x, y, yref, transpose=transpose)
        want = 2e-3 * max(den[i], 1.0) / den[i] if den[i] > 0 else 2e-3
        assert e == pytest.approx(want, rel=1e-9), (i, e, want)


def test_error_metric_transpose_detects_a_dropped_term():
    # a planted mistake in the transposed product: the metric with column sums flags it
    m = _lopsided(30, 0.25, 47)
    c = oracle.from_matrix(m)
    x = fe.source_vector(30, 48)
    yt = oracle.csrc_spmv_t(c, x)
    al_bad = c.al.copy()
    al_bad[len(al_bad) // 3] = 0.0  # A^T x scatters with al: drop one of its terms
    yt_bad = oracle.csrc_spmv_t(c, x, al=al_bad)
    assert oracle.max_rel_err(m, x, yt_bad, yt, transpose=True) > 1e-6
    assert oracle.max_rel_err(m, x, yt, yt, transpose=True) == 0.0


# --------------------------------------------------------------------------- Table 1 working sets
def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_working_sets.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            name, sym, n, nnz, _, ws = ln.split()
            rows.append((name, sym == "yes", int(n), int(nnz), int(ws)))
    return rows


def test_table1_working_sets():
    rows = _table1()
    assert len(rows) == 60
    checked = 0
    for name, sym, n, nnz, ws in rows:
        if name.endswith("_o32"):
            continue  # rectangular: m is not given in the text
        if sym:
            pairs = nnz - n  # nnz counts the lower triangle with the diagonal
            b = oracle.working_set_bytes(n, pairs, symmetric=True)
        else:
            assert (nnz - n) % 2 == 0, name
            b = oracle.working_set_bytes(n, (nnz - n) // 2)
        assert b // 1024 == ws, (name, b / 1024, ws)
        checked += 1
    assert checked == 57


# --------------------------------------------------------------------------- reduced precision
def test_round_f32_matches_ieee_conversion():
    v = np.concatenate([fe.source_vector(10000, 1) * 10.0 ** np.arange(-20, 20, 0.004), [0.0, -0.0, 1.0]])
    np.testing.assert_array_equal(oracle.round_f32(v), v.astype(np.float32).astype(np.float64))


def _bf16_neighbours(v):
    """The two BF16 numbers around v, found by stepping FP32 encodings with low 16 bits zero."""
    f = np.float32(v)
    bits = np.array([f]).view(np.uint32)[0] & np.uint32(0xFFFF0000)
    a = np.array([bits], dtype=np.uint32).view(np.float32)[0]
    step = np.uint32(0x10000)
    b = np.array([bits + step], dtype=np.uint32).view(np.float32)[0]
    c = np.array([bits - step], dtype=np.uint32).view(np.float32)[0]
    return [float(a), float(b), float(c)], int(bits)


def test_round_bf16_is_nearest_even_without_double_rounding():
    rng = np.random.default_rng(5)
    v = rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-60, 60, 20000)
    r = oracle.round_bf16(v)
    for vi, ri in zip(v[:3000], r[:3000]):
        cands, _ = _bf16_neighbours(vi)
        best = min(abs(cc - vi) for cc in cands)
        assert abs(ri - vi) == best
        # result is a BF16 number: its FP32 encoding has zero low half
        assert (np.array([np.float32(ri)]).view(np.uint32)[0] & 0xFFFF) == 0
        assert float(np.float32(ri)) == ri
    # ties go to the even neighbour
    assert oracle.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert oracle.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    # rounded once from FP64: just above the tie rounds up, whereas FP64->FP32->BF16
    # would land on the tie and round down to even
    v = 1.0 + 2.0 ** -8 + 2.0 ** -40
    assert oracle.round_bf16(np.array([v]))[0] == 1.0 + 2.0 ** -7
    assert float(np.float32(v)) == 1.0 + 2.0 ** -8
    # integers up to 256 are exact
    ints = np.arange(-256, 257, dtype=float)
    np.testing.assert_array_equal(oracle.round_bf16(ints), ints)


# --------------------------------------------------------------------------- Section 3.1 partition
@pytest.mark.parametrize("nbands", [1, 2, 3, 7, 16, 100, 152])
def test_partition_invariants(nbands):
    for m in (fe.p1_grid(20, 13), _random_matrix(64, 0.1, 3), _random_matrix(50, 0.9, 4)):
        c = oracle.from_matrix(m)
        b = oracle.partition(c, nbands)
        oracle.check_partition(c.ia, nbands, b)
        # each band's weight is within one row weight of its share nnz/B
        w = 1 + 2 * np.diff(c.ia)
        P = np.concatenate([[0], np.cumsum(w)])
        for t in range(1, nbands):
            assert abs(P[b[t]] - t * m.nnz / nbands) <= w.max()


def test_partition_brute_force_definition():
    m = _random_matrix(40, 0.2, 8)
    c = oracle.from_matrix(m)
    w = [1 + 2 * int(c.ia[i + 1] - c.ia[i]) for i in range(m.n)]
    for B in (1, 3, 5, 11):
        want = []
        for t in range(B + 1):
            acc, r = 0, 0
            while r < m.n and acc * B < t * m.nnz:
                acc += w[r]
                r += 1
            want.append(r)
        np.testing.assert_array_equal(oracle.partition(c, B), want)


def test_partition_checker_rejects_a_shifted_boundary():
    m = _random_matrix(64, 0.3, 9)
    c = oracle.from_matrix(m)
    b = oracle.partition(c, 4).copy()
    b[2] += 1
    with pytest.raises(AssertionError):
        oracle.check_partition(c.ia, 4, b)


# --------------------------------------------------------------------------- Section 3.2 colouring
def _write_sets(c):
    return [set([i]) | set(int(j) for j in c.ja[c.ia[i]:c.ia[i + 1]]) for i in range(c.n)]


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_jp_colouring_is_valid_and_first_fit(seed):
    m = _random_matrix(48, 0.1, 40 + seed)
    c = oracle.from_matrix(m)
    k, col = oracle.jp_color(c, seed)
    assert oracle.check_coloring(c, col, k) == 0
    assert col.max() == k - 1
    W = _write_sets(c)
    pri = [oracle.priority(seed, i) for i in range(c.n)]
    for u in range(c.n):
        nbrs = [v for v in range(c.n) if v != u and W[u] & W[v]]
        assert all(col[v] != col[u] for v in nbrs)
        # first fit in decreasing-priority order: every smaller colour is taken by a
        # conflicting row of higher priority
        higher = {int(col[v]) for v in nbrs if pri[v] > pri[u]}
        assert all(cc in higher for cc in range(col[u]))


def test_colouring_special_cases():
    # diagonal matrix: no conflicts, one colour
    n = 10
    rp, c = fe.pattern_from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64))
    cc = oracle.from_matrix(_mat(n, rp, c, np.ones(n)))
    assert oracle.greedy_color(cc, np.arange(n))[0] == 1
    # path (tridiagonal): W(i) = {i, i-1}; natural order gives 2 colours
    rp, c = fe.pattern_from_edges(n, np.arange(1, n), np.arange(0, n - 1))
    cc = oracle.from_matrix(_mat(n, rp, c, np.ones(len(c))))
    k, col = oracle.greedy_color(cc, np.arange(n))
    assert k == 2
    np.testing.assert_array_equal(col, np.arange(n) % 2)
    # dense pattern: every pair of rows conflicts, n colours
    ii, jj = np.triu_indices(n, 1)
    rp, c = fe.pattern_from_edges(n, ii, jj)
    cc = oracle.from_matrix(_mat(n, rp, c, np.ones(len(c))))
    k, col = oracle.jp_color(cc, 7)
    assert k == n and sorted(col) == list(range(n))


def test_colouring_lower_bound_and_direct_conflicts():
    m = fe.p1_grid(15, 11)
    c = oracle.from_matrix(m)
    k, col = oracle.jp_color(c, 99)
    up = np.bincount(c.ja, minlength=c.n)
    assert k >= 1 + up.max()  # row t and every row of A_U column t write y(t)
    # the direct conflicts of row i are exactly ja(ia(i)..ia(i+1)-1): h of them in total
    assert len(c.ja) == (m.nnz - m.n) // 2


def test_colouring_checker_detects_planted_conflict():
    m = fe.p1_grid(8, 8)
    c = oracle.from_matrix(m)
    k, col = oracle.jp_color(c, 3)
    bad = col.copy()
    # give a row the colour of one of its direct conflicts
    i = 20
    bad[i] = bad[c.ja[c.ia[i]]]
    assert oracle.check_coloring(c, bad, k) == 1


# --------------------------------------------------------------------------- configurations
def test_config_sizes():
    m = fe.p1_grid()
    assert (m.n, m.nnz, m.pairs) == (10_000, 69_202, 29_601)
    rp, c = fe.q1_hex27_pattern(96, 96, 96)
    assert (len(rp) - 1, rp[-1]) == (884_736, 23_393_656)
    # 3 DOFs with dense 3x3 node blocks multiply nnz by 9
    small = fe.q1_hex(5, 3, 1)
    rp5, _ = fe.q1_hex27_pattern(5, 5, 5)
    assert small.n == 375 and small.nnz == 9 * rp5[-1]
    cc = oracle.from_matrix(small)
    assert cc.pairs == (small.nnz - small.n) // 2


# --------------------------------------------------------------------------- stride-bounded colouring
def _write_sets(c):
    """W(i) = {i} U ja(row i): the y entries row i writes (Section 3.2 conflicts)."""
    return [{i} | {int(j) for j in c.ja[c.ia[i]:c.ia[i + 1]]} for i in range(c.n)]


def _stride_greedy_brute_force(c, stride):
    """The stride-bounded reading written out directly: ascending rows, first fit among the
    colours whose members never share a written y entry with the row and whose last member is
    at most `stride` rows back (no bound for stride <= 0); a new colour otherwise."""
    W = _write_sets(c)
    classes = []  # list of member lists, ascending
    colors = [-1] * c.n
    for i in range(c.n):
        chosen = None
        for k, members in enumerate(classes):
            if any(W[i] & W[r] for r in members):
                continue
            if stride > 0 and i - members[-1] > stride:
                continue
            chosen = k
            break
        if chosen is None:
            classes.append([])
            chosen = len(classes) - 1
        classes[chosen].append(i)
        colors[i] = chosen
    return len(classes), np.array(colors, np.int32)


@pytest.mark.parametrize("n,density,seed", SMALL + [(120, 0.05, 10), (200, 0.02, 11)])
@pytest.mark.parametrize("stride", [0, 1, 3, 8, 40])
def test_stride_colouring_matches_brute_force(n, density, seed, stride):
    c = oracle.from_matrix(_random_matrix(n, density, seed))
    k, colors = oracle.greedy_color_stride(c, stride)
    k_ref, colors_ref = _stride_greedy_brute_force(c, stride)
    assert k == k_ref
    np.testing.assert_array_equal(colors, colors_ref)


@pytest.mark.parametrize("stride", [1, 2, 16, 64, 500])
def test_stride_colouring_invariants_on_meshes(stride):
    for m in (fe.p1_grid(30, 20, 3), fe.q1_hex(7, 3, 4), fe.tet_mesh(1500, 5, method="kuhn")):
        c = oracle.from_matrix(m)
        k, colors = oracle.greedy_color_stride(c, stride)
        assert oracle.check_coloring(c, colors, k) == 0  # valid: no two rows of a class conflict
        assert oracle.max_class_gap(colors, k) <= stride  # the stride bound inside every class


def test_unbounded_stride_is_ascending_greedy():
    # stride <= 0: plain sequential greedy colouring in the matrix's own order (Section 3.2)
    for m in (fe.p1_grid(25, 19, 6), fe.q1_hex(6, 3, 7), _random_matrix(300, 0.03, 8)):
        c = oracle.from_matrix(m)
        k, colors = oracle.greedy_color_stride(c, 0)
        k2, colors2 = oracle.greedy_color(c, np.arange(m.n))
        assert k == k2
        np.testing.assert_array_equal(colors, colors2)
        # and a stride as long as the matrix binds nothing
        k3, colors3 = oracle.greedy_color_stride(c, m.n)
        np.testing.assert_array_equal(colors3, colors)


def test_stride_of_one_forces_consecutive_members():
    # stride 1: a class is a run of consecutive rows that pairwise do not conflict; on a
    # tridiagonal pattern every row conflicts with its neighbour, so every class is one row
    # until the class of row i - 2 can no longer be reached
    n = 12
    ei, ej = np.arange(1, n), np.arange(0, n - 1)
    rp, col = fe.pattern_from_edges(n, ei, ej)
    c = oracle.from_matrix(fe.FEMatrix(n, rp, col, np.ones(len(col))))
    k, colors = oracle.greedy_color_stride(c, 1)
    assert k == n
    assert oracle.max_class_gap(colors, k) == 0


def test_class_gap_checker_detects_a_planted_violation():
    colors = np.array([0, 1, 0, 1, 1, 0, 2], np.int32)  # class 0: rows 0, 2, 5 -> gap 3
    assert oracle.max_class_gap(colors, 3) == 3
    colors[5] = 1  # class 0: rows 0, 2 -> gap 2; class 1: rows 1, 3, 4, 5 -> gap 2
    assert oracle.max_class_gap(colors, 3) == 2
