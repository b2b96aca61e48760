"""GPU BiCG (csrc_bicg) against the oracle's BiCG and against the true residual.

BiCG (Saad, Algorithm 7.3) runs one A p and one A^T p* per iteration through the
library's own products, so it exercises the implicit transpose the paper points to
for oblique-projection solvers (Section 1). Rounding differs between the GPU path
(double-float scatter, atomics) and the oracle, so the checks are: convergence, an
iteration count close to the oracle's, the true residual b - A x (through the
oracle's independent CSR product) within a small multiple of the tolerance, and the
solution close to the oracle's.
"""
import numpy as np
import pytest

import fe_inputs as fe
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _true_relres(m, x, b):
    r = b - oracle.csr_spmv(m.n, m.row_ptr, m.col, m.val, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def _solve(cs, h, b, storage, rtol, maxit, strategy="window", x0=None):
    dt = torch.float64 if storage == "f64" else torch.float32
    bd = torch.as_tensor(b, dtype=dt).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.as_tensor(x0, dtype=dt).cuda()
    res = cs.csrc_bicg(h, bd, xd, rtol, maxit, cs.STRATEGIES[strategy], torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
    return res, xd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("strategy", ["window", "window_atomic", "atomic", "color"])
def test_bicg_fp64_matches_oracle(cs, strategy):
    for m in (fe.q1_hex(10, 3, 101), fe.tet_mesh(6000, 102, method="kuhn")):
        c = oracle.from_matrix(m)
        b = fe.source_vector(m.n, 103)
        ref = oracle.bicg(c, b, rtol=1e-10, maxit=400)
        assert ref.status == "converged"
        h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
        try:
            cs.csrc_color(h, 9)
            res, x = _solve(cs, h, b, "f64", 1e-10, 400, strategy)
            assert res["status"] == cs.CSRC_OK, res
            assert abs(res["iters"] - ref.iters) <= 2, (res, ref.iters)
            assert res["relres"] <= 1e-10
            assert _true_relres(m, x, b) <= 1e-9
            assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        finally:
            cs.csrc_destroy(h)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_bicg_reduced_precision_storage(cs, storage):
    # FP32 vectors and accumulation on the stored (rounded) matrix: the true residual against
    # the FP64 matrix is bounded by the storage rounding, not by the iteration
    m = fe.q1_hex(10, 3, 104)
    b = fe.source_vector(m.n, 105).astype(np.float32).astype(np.float64)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
    try:
        res, x = _solve(cs, h, b, storage, 1e-5, 400)
        assert res["status"] == cs.CSRC_OK, res
        assert _true_relres(m, x, b) <= {"f32": 1e-4, "bf16": 3e-2}[storage]
    finally:
        cs.csrc_destroy(h)


def test_bicg_symmetric_storage_and_initial_guess(cs):
    base = fe.q1_hex(8, 3, 106)
    rows = np.repeat(np.arange(base.n), np.diff(base.row_ptr))
    v = fe.hash_uniform(107, np.minimum(rows, base.col), np.maximum(rows, base.col))
    diag = rows == base.col
    v[diag] = 0.0
    v[diag] = 1.0 + np.bincount(rows, weights=np.abs(v), minlength=base.n)
    m = fe.FEMatrix(base.n, base.row_ptr, base.col, v)
    b = fe.source_vector(m.n, 108)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64, cs.CSRC_FLAG_SYMMETRIC_VALUES)
    try:
        res, x = _solve(cs, h, b, "f64", 1e-11, 400)
        assert res["status"] == cs.CSRC_OK and _true_relres(m, x, b) <= 1e-10
        # starting from the solution: converged before the first iteration
        res2, x2 = _solve(cs, h, b, "f64", 1e-9, 400, x0=x)
        assert res2["status"] == cs.CSRC_OK and res2["iters"] == 0
        np.testing.assert_array_equal(x2, x)
    finally:
        cs.csrc_destroy(h)


def test_bicg_limits_and_errors(cs):
    m = fe.q1_hex(6, 1, 109)
    b = fe.source_vector(m.n, 110)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        res, _ = _solve(cs, h, b, "f64", 1e-14, 2)
        assert res["status"] == cs.CSRC_ERR_NOT_CONVERGED and res["iters"] == 2 and res["relres"] > 1e-14
        res, x = _solve(cs, h, np.zeros(m.n), "f64", 1e-10, 10)
        assert res["status"] == cs.CSRC_OK and res["iters"] == 0 and not np.any(x)
        with pytest.raises(cs.CsrcError) as e:  # host vectors are not accepted
            cs.csrc_bicg(h, b, np.zeros(m.n), 1e-10, 10)
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
        bd = torch.as_tensor(b).cuda()
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_bicg(h, bd, bd, 1e-10, 10)
        assert e.value.status == cs.CSRC_ERR_ALIAS
    finally:
        cs.csrc_destroy(h)
    a = fe.overlap_subdomain(m, m.n // 2)
    h = cs.csrc_create_rect_from_csr(a.n, a.m, a.row_ptr, a.col, a.val, cs.CSRC_F64)
    try:
        bd = torch.zeros(a.n, dtype=torch.float64, device="cuda")
        xd = torch.zeros(a.m, dtype=torch.float64, device="cuda")
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_bicg(h, bd, xd, 1e-10, 10)
        assert e.value.status == cs.CSRC_ERR_INVALID_ARG
    finally:
        cs.csrc_destroy(h)
