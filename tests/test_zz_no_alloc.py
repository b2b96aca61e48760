"""csrc_spmv_noalloc: the product for callers that may not allocate device memory.

Some callers cannot call cudaMalloc while they compute: their GPU memory belongs to
another allocator's pool, or their host thread must not block on the device
synchronisation that allocation can cause. They create and partition a handle once,
then call csrc_spmv_noalloc, whose spill buffer is a fixed array in the library's
static device memory. These tests call it through the C ABI and check that two calls
in a row give what csrc_spmv / csrc_spmv_t give with the window strategy, and what the
CPU oracle gives, within the tolerances of the parity tests (relative to
sum_j |a_ij||x_j| per row: 1e-12 for FP64 storage, 1e-5 for FP32, 1e-2 for BF16).

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import fe_inputs as fe
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _transpose(m):
    at = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(m.n, m.n)).T.tocsr()
    return fe.FEMatrix(m.n, at.indptr.astype(np.int64), at.indices.astype(np.int32), at.data)


def _create(cs, m, storage="f64"):
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
    cs.csrc_partition(h, 0)
    return h


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_two_calls_match_the_window_product(cs, storage):
    m = fe.q1_hex(14, 3, 21)  # n = 8232, RCM order: several bands, spilled rows
    h = _create(cs, m, storage)
    tol = {"f64": TOL, "f32": 1e-5, "bf16": 1e-2}[storage]
    dt = torch.float64 if storage == "f64" else torch.float32
    c = oracle.from_matrix(m)
    try:
        info = cs.csrc_get_info(h)
        assert 0 < info["spill_entries"] <= cs.CSRC_NOALLOC_MAX_SPILL_ENTRIES
        s = torch.cuda.current_stream()
        xs = [fe.source_vector(m.n, 31), fe.source_vector(m.n, 32)]
        if storage != "f64":  # the vectors the product sees are FP32
            xs = [v.astype(np.float32).astype(np.float64) for v in xs]
        x1, x2 = (torch.as_tensor(v, dtype=dt).cuda() for v in xs)
        y = torch.full_like(x1, float("nan"))
        yref = torch.full_like(x1, float("nan"))
        mt = _transpose(m)
        # two calls in a row, with different inputs and directions: the second finds the
        # first call's partial sums in the shared array and must not be affected by them
        for x, tr in ((x1, False), (x2, True), (x1, True), (x2, False)):
            (cs.csrc_spmv_t if tr else cs.csrc_spmv)(h, x, yref, cs.CSRC_STRAT_WINDOW, s)
            y.fill_(float("nan"))
            cs.csrc_spmv_noalloc(h, x, y, tr, s)
            torch.cuda.synchronize()
            assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
            xn = x.cpu().numpy().astype(np.float64)
            yn = y.cpu().numpy().astype(np.float64)
            err = oracle.max_rel_err(mt if tr else m, xn, yn, yref.cpu().numpy().astype(np.float64))
            assert err <= tol, (tr, err)
            # and against the CPU oracle itself, so that a fault shared by both GPU paths shows
            ref = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(c, xn)
            err = oracle.max_rel_err(mt if tr else m, xn, yn, ref)
            assert err <= tol, (tr, "oracle", err)
    finally:
        cs.csrc_destroy(h)


def test_two_handles_share_the_array(cs):
    a = fe.p1_grid(70, 40, 5)
    b = fe.q1_hex(10, 1, 6)
    ha, hb = _create(cs, a), _create(cs, b)
    try:
        s = torch.cuda.current_stream()
        for m, h, seed in ((a, ha, 1), (b, hb, 2), (a, ha, 3)):
            x = torch.from_numpy(fe.source_vector(m.n, seed)).cuda()
            yref = torch.empty_like(x)
            y = torch.empty_like(x)
            cs.csrc_spmv(h, x, yref, cs.CSRC_STRAT_WINDOW, s)
            cs.csrc_spmv_noalloc(h, x, y, False, s)
            torch.cuda.synchronize()
            err = oracle.max_rel_err(m, x.cpu().numpy(), y.cpu().numpy(), yref.cpu().numpy())
            assert err <= TOL, err
    finally:
        cs.csrc_destroy(ha)
        cs.csrc_destroy(hb)


def test_rejections(cs):
    m = fe.p1_grid(30, 30, 7)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        x = torch.from_numpy(fe.source_vector(m.n, 8)).cuda()
        y = torch.empty_like(x)
        # no plan yet: the entry point does not build one (that would allocate)
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv_noalloc(h, x, y)
        assert e.value.status == cs.CSRC_ERR_NOT_PARTITIONED
        cs.csrc_partition(h, 0)
        # host vectors would need staging buffers
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv_noalloc(h, x.cpu().numpy(), y.cpu().numpy())
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv_noalloc(h, x, x)
        assert e.value.status == cs.CSRC_ERR_ALIAS
    finally:
        cs.csrc_destroy(h)
    # a plan whose spill exceeds the fixed array: one row per band spills every stored pair
    m = fe.q1_hex(40, 3, 9)
    assert m.pairs > cs.CSRC_NOALLOC_MAX_SPILL_ENTRIES
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        cs.csrc_partition(h, m.n)
        assert cs.csrc_get_info(h)["spill_entries"] > cs.CSRC_NOALLOC_MAX_SPILL_ENTRIES
        x = torch.from_numpy(fe.source_vector(m.n, 10)).cuda()
        y = torch.empty_like(x)
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv_noalloc(h, x, y)
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
    finally:
        cs.csrc_destroy(h)


def test_rectangular_handle_is_rejected(cs):
    g = fe.q1_hex(6, 1, 41)
    a = fe.overlap_subdomain(g, g.n // 2)
    h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
    try:
        cs.csrc_partition(h, 0)
        x = torch.zeros(a.m, dtype=torch.float64, device="cuda")
        y = torch.zeros(a.m, dtype=torch.float64, device="cuda")
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv_noalloc(h, x, y, False, torch.cuda.current_stream())
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
    finally:
        cs.csrc_destroy(h)
