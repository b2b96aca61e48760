"""GPU parity for rectangular CSRC (Section 2.1, Fig. 2(b)) against the CPU oracle.

A rectangular handle is one subdomain of an overlapping decomposition: its own
unknowns (the structurally symmetric square part, CSRC) and the overlap columns
(the auxiliary CSR). y = A x reads m entries of x and writes n; y = A^T x reads n
and writes m. Tolerances as for square matrices, relative to sum |a||x| per output.
"""
import numpy as np
import pytest

import fe_inputs as fe
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _subdomains():
    g = fe.q1_hex(10, 3, 31)  # 3 DOF per node, RCM order: 3000 rows
    p = fe.p1_grid(40, 40, 32)  # scalar 2D triangles, natural order
    return [fe.overlap_subdomain(g, g.n // 2), fe.overlap_subdomain(g, 700), fe.overlap_subdomain(p, 900)]


def _run(cs, h, a, x, storage, strategy, transpose):
    dt = torch.float64 if storage == "f64" else torch.float32
    xd = torch.as_tensor(np.asarray(x), dtype=dt).cuda()
    yd = torch.full((a.m if transpose else a.n,), float("nan"), dtype=dt, device="cuda")
    (cs.csrc_spmv_t if transpose else cs.csrc_spmv)(h, xd, yd, cs.STRATEGIES[strategy], torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
    return yd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_rectangular_products_match_oracle(cs, storage):
    for a in _subdomains():
        r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
        x = fe.source_vector(a.m, 33)
        xt = fe.source_vector(a.n, 34)
        if storage != "f64":
            x = x.astype(np.float32).astype(np.float64)
            xt = xt.astype(np.float32).astype(np.float64)
        y_ref, yt_ref = oracle.csrcr_spmv(r, x), oracle.csrcr_spmv_t(r, xt)
        h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.STORAGE[storage])
        try:
            info = cs.csrc_get_info(h)
            assert info["m"] == a.m and info["n"] == a.n
            assert info["rect_nnz"] == len(r.jar) > 0
            cs.csrc_color(h, 7)
            for strategy in ("window", "window_atomic", "atomic", "color"):
                y = _run(cs, h, a, x, storage, strategy, False)
                e = oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, x, y, y_ref)
                assert e <= TOL[storage], (a.name, strategy, e)
                yt = _run(cs, h, a, xt, storage, strategy, True)
                e = oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, xt, yt, yt_ref, transpose=True)
                assert e <= TOL[storage], (a.name, strategy, "T", e)
        finally:
            cs.csrc_destroy(h)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_rectangular_integer_values_bit_exact(cs, storage):
    a = _subdomains()[0]
    # integers in [-8, 8]: exact in every storage type, sums exact in FP32
    ai = fe.RectMatrix(a.n, a.m, a.row_ptr, a.col, fe.integer_values(a.row_ptr, a.col, 35))
    r = oracle.csr_to_csrcr(ai.n, ai.m, ai.row_ptr, ai.col, ai.val)
    x, xt = fe.integer_vector(ai.m, 35), fe.integer_vector(ai.n, 36)
    h = cs.csrc_create_rect_from_csr(ai.n, ai.m, ai.row_ptr, ai.col, ai.val, cs.STORAGE[storage])
    try:
        for nbands in (0, 5, 200):
            cs.csrc_partition(h, nbands)
            for strategy in ("window", "window_atomic", "atomic"):
                np.testing.assert_array_equal(_run(cs, h, ai, x, storage, strategy, False), oracle.csrcr_spmv(r, x))
                np.testing.assert_array_equal(_run(cs, h, ai, xt, storage, strategy, True),
                                              oracle.csrcr_spmv_t(r, xt))
    finally:
        cs.csrc_destroy(h)


def test_rectangular_host_vectors_and_autotune(cs):
    a = _subdomains()[1]
    r = oracle.csr_to_csrcr(a.n, a.m, a.row_ptr, a.col, a.val)
    h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
    try:
        x = fe.source_vector(a.m, 37)
        y = np.full(a.n, np.nan)
        cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_AUTO, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, x, y, oracle.csrcr_spmv(r, x)) <= 1e-12
        xt = fe.source_vector(a.n, 38)
        yt = np.full(a.m, np.nan)
        cs.csrc_spmv_t(h, xt, yt, cs.CSRC_STRAT_AUTO, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, xt, yt, oracle.csrcr_spmv_t(r, xt),
                                       transpose=True) <= 1e-12
        xd = torch.as_tensor(x).cuda()
        yd = torch.empty(a.n, dtype=torch.float64, device="cuda")
        cs.csrc_autotune(h, xd, yd, torch.cuda.current_stream())
        yd.fill_(float("nan"))
        cs.csrc_spmv(h, xd, yd, cs.CSRC_STRAT_AUTO, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert oracle.max_rel_err_rect(a.n, a.m, a.row_ptr, a.col, a.val, x, yd.cpu().numpy(),
                                       oracle.csrcr_spmv(r, x)) <= 1e-12
    finally:
        cs.csrc_destroy(h)


def test_rectangular_degenerate_shapes(cs):
    # m == n: a square matrix through the rectangular entry point
    g = fe.q1_hex(5, 1, 39)
    h = cs.csrc_create_rect_from_csr(g.n, g.n, g.row_ptr, g.col, g.val, cs.CSRC_F64)
    try:
        x = fe.source_vector(g.n, 40)
        y = _run(cs, h, fe.RectMatrix(g.n, g.n, g.row_ptr, g.col, g.val), x, "f64", "window", False)
        assert oracle.max_rel_err(g, x, y, oracle.csrc_spmv(oracle.from_matrix(g), x)) <= 1e-12
        assert cs.csrc_get_info(h)["rect_nnz"] == 0
    finally:
        cs.csrc_destroy(h)
    # n == 0 rows: A^T x is all zeros, A x is empty
    h = cs.csrc_create_rect_from_csr(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), cs.CSRC_F64)
    try:
        xt = torch.zeros(1, dtype=torch.float64, device="cuda")
        yt = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        cs.csrc_spmv_t(h, xt, yt, cs.CSRC_STRAT_AUTO, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.all(yt == 0)
    finally:
        cs.csrc_destroy(h)
    # rows whose only entries are in the overlap (no square-part entries, no diagonal)
    rp = np.array([0, 1, 2, 4], np.int64)
    col = np.array([3, 4, 3, 4], np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0])
    a = fe.RectMatrix(3, 5, rp, col, val)
    r = oracle.csr_to_csrcr(3, 5, rp, col, val)
    h = cs.csrc_create_rect_from_csr(3, 5, rp, col, val, cs.CSRC_F64)
    try:
        x = np.arange(1.0, 6.0)
        np.testing.assert_array_equal(_run(cs, h, a, x, "f64", "window", False), oracle.csrcr_spmv(r, x))
        np.testing.assert_array_equal(_run(cs, h, a, x[:3], "f64", "atomic", True), oracle.csrcr_spmv_t(r, x[:3]))
    finally:
        cs.csrc_destroy(h)


def test_rectangular_interface_errors(cs):
    a = _subdomains()[2]
    with pytest.raises(cs.CsrcError) as e:
        cs.csrc_create_rect_from_csr(a.n, a.n - 1, a.row_ptr, a.col, a.val, cs.CSRC_F64)
    assert e.value.status == cs.CSRC_ERR_INVALID_ARG
    bad = a.col.copy()
    bad[-1] = a.m
    with pytest.raises(cs.CsrcError) as e:
        cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, bad, a.val, cs.CSRC_F64)
    assert e.value.status == cs.CSRC_ERR_INDEX_RANGE
    h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
    try:
        X = torch.zeros((a.m, 4), dtype=torch.float64, device="cuda")
        Y = torch.zeros((a.m, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmm_batched([h], [X], [Y], 4, False, torch.cuda.current_stream())
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
    finally:
        cs.csrc_destroy(h)
