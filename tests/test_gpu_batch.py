"""GPU parity of the batched products and of the per-matrix precision of the window strategy.

A batch mixes members of every storage type and precision in one csrc_spmm_batched call
(one owner-kernel launch per mode and columns-per-pass group, one accumulation launch per
mode, all in one CUDA graph), for one and several right-hand sides; members tuned to another
strategy run their own launches. Every member is checked against the CPU oracle at its own
tolerance, relative to sum_j |a_ij||x_j| per row: 1e-12 for FP64, 1e-5 for FP32 values and
1e-2 for BF16 values (the bound of csrc_autotune_precision is checked too).
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


@pytest.fixture()
def tune_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("CSRC_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.setenv("CSRC_TUNE", "cache")
    return tmp_path / "tune.txt"


def _transpose(m):
    at = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(m.n, m.n)).T.tocsr()
    return fe.FEMatrix(m.n, at.indptr.astype(np.int64), at.indices.astype(np.int32), at.data)


# (storage, precision): the handle's storage type and its window strategy's precision
MEMBER_KINDS = [("f64", "f64"), ("f32", "f32"), ("bf16", "bf16"), ("f64", "f32"), ("f64", "bf16")]


def _members(cs):
    mats = [fe.p1_grid(37, 21, 1), fe.q1_hex(9, 3, 2), fe.tet_mesh(3000, 3, method="kuhn"), fe.q1_hex(11, 1, 4),
            fe.p1_grid(90, 70, 5), fe.q1_hex(7, 3, 6), fe.tet_mesh(900, 7, method="kuhn")]
    out = []
    for i, m in enumerate(mats):
        storage, prec = MEMBER_KINDS[i % len(MEMBER_KINDS)]
        h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
        if prec != storage:
            cs.csrc_set_precision(h, cs.STORAGE[prec])
        out.append((m, h, storage, prec))
    return out


@pytest.mark.parametrize("nrhs", [1, 3, 8, 13])
def test_mixed_batch_matches_oracle(cs, nrhs):
    members = _members(cs)
    try:
        Xs, Xd, Yd = [], [], []
        for i, (m, h, storage, prec) in enumerate(members):
            X = fe.source_vector(m.n, 20 + i, nrhs=nrhs if nrhs > 1 else None)
            dt = torch.float64 if storage == "f64" else torch.float32
            if storage != "f64":  # the vectors the product sees are FP32
                X = X.astype(np.float32).astype(np.float64)
            Xs.append(X)
            Xd.append(torch.as_tensor(X, dtype=dt).cuda().contiguous())
            Yd.append(torch.full_like(Xd[-1], float("nan")))
        for rep in range(2):  # the second call replays the graph
            for tr in (False, True):
                for y in Yd:
                    y.fill_(float("nan"))
                cs.csrc_spmm_batched([mm[1] for mm in members], Xd, Yd, nrhs, tr, torch.cuda.current_stream())
                torch.cuda.synchronize()
                for (m, h, storage, prec), X, Y in zip(members, Xs, Yd):
                    c = oracle.from_matrix(m)
                    ref = oracle.csrc_spmm(c, X.reshape(m.n, -1), transpose=tr).reshape(X.shape)
                    err = oracle.max_rel_err(m, X, Y.cpu().numpy().astype(np.float64), ref, transpose=tr)
                    assert err <= TOL[prec], (m.name, storage, prec, nrhs, tr, err)
                    assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
    finally:
        for _, h, _, _ in members:
            cs.csrc_destroy(h)


def test_reduced_precision_single_products(cs):
    # an FP64 handle at FP32 / BF16 precision: double vectors in and out, errors within the
    # tolerance and the bound, and visibly above FP64 rounding (the values really are rounded)
    m = fe.q1_hex(14, 3, 31)
    x = fe.source_vector(m.n, 32)
    c = oracle.from_matrix(m)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        for prec, tol in (("f32", 1e-5), ("bf16", 1e-2), ("f64", 1e-12)):
            cs.csrc_set_precision(h, cs.STORAGE[prec])
            for tr in (False, True):
                (cs.csrc_spmv_t if tr else cs.csrc_spmv)(h, xd, yd, cs.CSRC_STRAT_WINDOW)
                torch.cuda.synchronize()
                ref = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(c, x)
                err = oracle.max_rel_err(m, x, yd.cpu().numpy(), ref, transpose=tr)
                info = cs.csrc_get_info(h)
                assert info["precision"] == cs.STORAGE[prec]
                assert err <= min(tol, info["error_bound"]), (prec, tr, err, info["error_bound"])
                if prec != "f64":
                    assert err > 1e-12
        with pytest.raises(cs.CsrcError):
            cs.csrc_set_precision(h, 7)
    finally:
        cs.csrc_destroy(h)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F32)
    try:
        with pytest.raises(cs.CsrcError):  # a float handle cannot run in FP64
            cs.csrc_set_precision(h, cs.CSRC_F64)
    finally:
        cs.csrc_destroy(h)


def test_autotune_precision_meets_the_budget(cs, tune_cache):
    m = fe.q1_hex(16, 3, 41)
    x = fe.source_vector(m.n, 42)
    c = oracle.from_matrix(m)
    ref = oracle.csrc_spmv(c, x)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        for budget in (1e-2, 1e-5, 1e-12):
            p, bound = cs.csrc_autotune_precision(h, xd, yd, budget)
            assert bound <= budget
            if budget == 1e-12:
                assert p == cs.CSRC_F64  # the FP32 bound is far above 1e-12
            cs.csrc_spmv(h, xd, yd, cs.CSRC_STRAT_AUTO)
            torch.cuda.synchronize()
            assert oracle.max_rel_err(m, x, yd.cpu().numpy(), ref) <= bound
        with pytest.raises(cs.CsrcError):  # nothing reaches 1e-20
            cs.csrc_autotune_precision(h, xd, yd, 1e-20)
        key = cs.csrc_get_tune_key(h)
        assert cs.csrc_tune_cache_lookup(key, cs.CSRC_TUNE_PRECISION, 1e-5) is not None
    finally:
        cs.csrc_destroy(h)


def test_tuning_cache_is_reused(cs, tune_cache, monkeypatch):
    m = fe.q1_hex(12, 3, 51)
    x = fe.source_vector(m.n, 52)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    h1 = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    h2 = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        cs.csrc_autotune(h1, xd, yd)
        i1 = cs.csrc_get_info(h1)
        key = cs.csrc_get_tune_key(h1)
        rec = cs.csrc_tune_cache_lookup(key, cs.CSRC_TUNE_STRATEGY)
        assert rec is not None and rec[0] == i1["tuned_strategy"]
        # a second handle of the same matrix takes the recorded decision without timing
        cs.csrc_autotune(h2, xd, yd)
        i2 = cs.csrc_get_info(h2)
        assert i2["tuned_strategy"] == i1["tuned_strategy"]
        # a recorded decision is honoured: force the atomic strategy through the cache
        cs.csrc_tune_cache_store(key, cs.CSRC_TUNE_STRATEGY, 0.0, [cs.CSRC_STRAT_ATOMIC, 0])
        cs.csrc_autotune(h2, xd, yd)
        assert cs.csrc_get_info(h2)["tuned_strategy"] == cs.CSRC_STRAT_ATOMIC
        cs.csrc_spmv(h2, xd, yd, cs.CSRC_STRAT_AUTO)
        torch.cuda.synchronize()
        ref = oracle.csrc_spmv(oracle.from_matrix(m), x)
        assert oracle.max_rel_err(m, x, yd.cpu().numpy(), ref) <= 1e-12
        # CSRC_TUNE=full times again and records its own decision
        monkeypatch.setenv("CSRC_TUNE", "full")
        cs.csrc_autotune(h2, xd, yd)
        assert cs.csrc_tune_cache_lookup(key, cs.CSRC_TUNE_STRATEGY)[0] == cs.csrc_get_info(h2)["tuned_strategy"]
    finally:
        cs.csrc_destroy(h1)
        cs.csrc_destroy(h2)


def test_batch_keeps_members_tuned_strategies(cs, tune_cache):
    # members tuned (through recorded decisions) to the colour and atomic strategies run their own
    # launches next to the graph of the window members; integer values: every result exact
    mats = [fe.p1_grid(30, 20, 61), fe.q1_hex(8, 3, 62), fe.tet_mesh(2000, 63, method="kuhn")]
    ims = [fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 64 + i)) for i, m in enumerate(mats)]
    hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64) for m in ims]
    try:
        cs.csrc_color(hs[0], 5)
        xs = [fe.integer_vector(m.n, 70 + i) for i, m in enumerate(ims)]
        Xd = [torch.from_numpy(x).cuda() for x in xs]
        Yd = [torch.empty_like(x) for x in Xd]
        for h, strat in zip(hs[:2], (cs.CSRC_STRAT_COLOR, cs.CSRC_STRAT_ATOMIC)):
            cs.csrc_tune_cache_store(cs.csrc_get_tune_key(h), cs.CSRC_TUNE_STRATEGY, 0.0, [strat, 0])
        for h, x, y in zip(hs, Xd, Yd):
            cs.csrc_autotune(h, x, y)
        assert cs.csrc_get_info(hs[0])["tuned_strategy"] == cs.CSRC_STRAT_COLOR
        assert cs.csrc_get_info(hs[1])["tuned_strategy"] == cs.CSRC_STRAT_ATOMIC
        for tr in (False, True):
            for y in Yd:
                y.fill_(float("nan"))
            cs.csrc_spmm_batched(hs, Xd, Yd, 1, tr, torch.cuda.current_stream())
            torch.cuda.synchronize()
            for m, x, y in zip(ims, xs, Yd):
                ref = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(oracle.from_matrix(m), x)
                np.testing.assert_array_equal(y.cpu().numpy(), ref)
    finally:
        for h in hs:
            cs.csrc_destroy(h)
