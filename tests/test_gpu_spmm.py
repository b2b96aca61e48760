"""GPU parity of the several-right-hand-side product Y = A X (and A^T X), X n-by-r row-major.

The oracle applies Fig. 2(a) to each column. Tolerances per row and column are those of
the single-vector product: 1e-12 (FP64 storage), 1e-5 (FP32), 1e-2 (BF16), relative to
sum_j |a_ij||x_jc|. Integer-valued inputs are exact in every storage type, so there the
results must match bit for bit.
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


def _transpose(m):
    at = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(m.n, m.n)).T.tocsr()
    return fe.FEMatrix(m.n, at.indptr.astype(np.int64), at.indices.astype(np.int32), at.data)


def _run(cs, h, X, storage, transpose):
    dt = torch.float64 if storage == "f64" else torch.float32
    Xd = torch.as_tensor(X, dtype=dt).cuda().contiguous()
    Yd = torch.full_like(Xd, float("nan"))
    cs.csrc_spmm_batched([h], [Xd], [Yd], X.shape[1], transpose, torch.cuda.current_stream())
    torch.cuda.synchronize()
    st = cs.csrc_get_last_device_error(h)
    assert st == cs.CSRC_OK, cs.csrc_status_string(st)
    return Yd.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("nrhs", [1, 3, 4, 8, 13, 32])
def test_spmm_matches_oracle(cs, storage, nrhs):
    m = fe.q1_hex(12, 1, 31)  # scalar Q1, RCM order, n = 1728
    c = oracle.from_matrix(m)
    X = fe.source_vector(m.n, 41, nrhs=nrhs)
    if storage != "f64":
        X = X.astype(np.float32).astype(np.float64)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage])
    try:
        cs.csrc_partition(h, 0)
        for tr in (False, True):
            Y = _run(cs, h, X, storage, tr)
            Yref = oracle.csrc_spmm(c, X, transpose=tr)
            mm = _transpose(m) if tr else m
            err = oracle.max_rel_err(mm, X, Y, Yref)
            assert err <= TOL[storage], (tr, err)
    finally:
        cs.csrc_destroy(h)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_spmm_integer_values_bit_exact(cs, storage):
    for m in (fe.q1_hex(7, 3, 5), fe.p1_grid(23, 17, 6), fe.tet_mesh(2000, 7, method="kuhn")):
        im = fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 77))
        c = oracle.from_matrix(im)
        X = fe.integer_vector(m.n, 78, nrhs=6)
        h = cs.csrc_create_from_csr(im.n, im.row_ptr, im.col, im.val, cs.STORAGE[storage])
        try:
            cs.csrc_partition(h, 7)
            for tr in (False, True):
                np.testing.assert_array_equal(_run(cs, h, X, storage, tr), oracle.csrc_spmm(c, X, transpose=tr))
        finally:
            cs.csrc_destroy(h)


def test_spmm_columns_equal_single_vector_products(cs):
    # a one-column block is the single-vector product, and every column of a block is one
    m = fe.q1_hex(10, 3, 8)
    X = fe.source_vector(m.n, 9, nrhs=4)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        Y = _run(cs, h, X, "f64", False)
        for col in range(4):
            xd = torch.from_numpy(np.ascontiguousarray(X[:, col])).cuda()
            yd = torch.empty_like(xd)
            cs.csrc_spmv(h, xd, yd, cs.CSRC_STRAT_WINDOW)
            torch.cuda.synchronize()
            assert oracle.max_rel_err(m, X[:, col], Y[:, col], yd.cpu().numpy()) <= 1e-12
    finally:
        cs.csrc_destroy(h)


def test_spmm_batch_of_uneven_members(cs):
    ms = [fe.p1_grid(9, 7, 1), fe.q1_hex(6, 3, 2), fe.tet_mesh(900, 3, method="kuhn"), fe.p1_grid(40, 3, 4)]
    hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64) for m in ms]
    try:
        Xs = [fe.source_vector(m.n, 10 + i, nrhs=5) for i, m in enumerate(ms)]
        Xd = [torch.from_numpy(x).cuda() for x in Xs]
        Yd = [torch.full_like(x, float("nan")) for x in Xd]
        cs.csrc_spmm_batched(hs, Xd, Yd, 5, False, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for m, X, Y in zip(ms, Xs, Yd):
            err = oracle.max_rel_err(m, X, Y.cpu().numpy(), oracle.csrc_spmm(oracle.from_matrix(m), X))
            assert err <= 1e-12
    finally:
        for h in hs:
            cs.csrc_destroy(h)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batched_single_vectors_graph_replay(cs, storage):
    # one persistent launch over all members' bands, captured in a CUDA graph and replayed
    ms = fe.batch_meshes(12, 77, nmin=50, nmax=30000)
    hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage]) for m in ms]
    dt = torch.float64 if storage == "f64" else torch.float32
    try:
        xs = [fe.source_vector(m.n, 100 + i) for i, m in enumerate(ms)]
        if storage != "f64":
            xs = [x.astype(np.float32).astype(np.float64) for x in xs]
        Xd = [torch.from_numpy(x).to(dt).cuda() for x in xs]
        Yd = [torch.full_like(x, float("nan")) for x in Xd]
        tol = 1e-12 if storage == "f64" else 1e-5
        for rep in range(3):  # first call builds the graph, the others replay it
            for tr in (False, True):
                for y in Yd:
                    y.fill_(float("nan"))
                cs.csrc_spmm_batched(hs, Xd, Yd, 1, tr, torch.cuda.current_stream())
                torch.cuda.synchronize()
                for m, x, y, h in zip(ms, xs, Yd, hs):
                    c = oracle.from_matrix(m)
                    yref = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(c, x)
                    mm = _transpose(m) if tr else m
                    assert oracle.max_rel_err(mm, x, y.cpu().numpy().astype(np.float64), yref) <= tol
                    assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
        # new output buffers: a new graph
        Yd2 = [torch.empty_like(x) for x in Xd]
        cs.csrc_spmm_batched(hs, Xd, Yd2, 1, False, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for m, x, y in zip(ms, xs, Yd2):
            yref = oracle.csrc_spmv(oracle.from_matrix(m), x)
            assert oracle.max_rel_err(m, x, y.cpu().numpy().astype(np.float64), yref) <= tol
    finally:
        for h in hs:
            cs.csrc_destroy(h)


def test_batched_integer_exact_and_mixed_storage(cs):
    ms = [fe.p1_grid(11, 9, 1), fe.q1_hex(5, 3, 2), fe.tet_mesh(1500, 3, method="kuhn")]
    ims = [fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 5)) for m in ms]
    hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64) for m in ims]
    try:
        xs = [fe.integer_vector(m.n, 6 + i) for i, m in enumerate(ims)]
        Xd = [torch.from_numpy(x).cuda() for x in xs]
        Yd = [torch.empty_like(x) for x in Xd]
        cs.csrc_spmm_batched(hs, Xd, Yd, 1, False, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for m, x, y in zip(ims, xs, Yd):
            np.testing.assert_array_equal(y.cpu().numpy(), oracle.csrc_spmv(oracle.from_matrix(m), x))
        # members of different storage types share one batch (each with its own vector type)
        h32 = cs.csrc_create_from_csr(ims[0].n, ims[0].row_ptr, ims[0].col, ims[0].val, cs.CSRC_F32)
        try:
            x32 = Xd[0].float()
            y32 = torch.empty_like(x32)
            cs.csrc_spmm_batched([hs[0], h32], [Xd[0], x32], [Yd[0], y32], 1, False)
            torch.cuda.synchronize()
            ref = oracle.csrc_spmv(oracle.from_matrix(ims[0]), xs[0])
            np.testing.assert_array_equal(Yd[0].cpu().numpy(), ref)
            np.testing.assert_array_equal(y32.cpu().numpy().astype(np.float64), ref)
        finally:
            cs.csrc_destroy(h32)
    finally:
        for h in hs:
            cs.csrc_destroy(h)


def test_batched_member_with_a_wide_row(cs):
    # the last row couples to one row in each of 400 window pages of 64 rows: a wide window,
    # next to small members; integer values make every result exact
    n = 64 * 400
    ei = np.concatenate([np.arange(1, n), np.full(400, n - 1)])
    ej = np.concatenate([np.arange(0, n - 1), np.arange(0, n - 1, 64)])  # 400 rows, one per page
    rp, col = fe.pattern_from_edges(n, ei, ej)
    wide = fe.FEMatrix(n, rp, col, fe.integer_values(rp, col, 11))
    g = fe.p1_grid(20, 15, 12)
    small = fe.FEMatrix(g.n, g.row_ptr, g.col, fe.integer_values(g.row_ptr, g.col, 13))
    ms = [small, wide, small]
    for storage in ("f64", "f32"):
        hs = [cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage]) for m in ms]
        dt = torch.float64 if storage == "f64" else torch.float32
        try:
            xs = [fe.integer_vector(m.n, 14 + i) for i, m in enumerate(ms)]
            Xd = [torch.from_numpy(x).to(dt).cuda() for x in xs]
            Yd = [torch.full_like(x, float("nan")) for x in Xd]
            for tr in (False, True):
                cs.csrc_spmm_batched(hs, Xd, Yd, 1, tr, torch.cuda.current_stream())
                torch.cuda.synchronize()
                for m, x, y, h in zip(ms, xs, Yd, hs):
                    c = oracle.from_matrix(m)
                    yref = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(c, x)
                    np.testing.assert_array_equal(y.cpu().numpy().astype(np.float64), yref)
                    assert cs.csrc_get_last_device_error(h) == cs.CSRC_OK
        finally:
            for h in hs:
                cs.csrc_destroy(h)


def test_autotune_spmm_k_tile(cs):
    m = fe.q1_hex(11, 1, 12)
    c = oracle.from_matrix(m)
    X = fe.source_vector(m.n, 13, nrhs=16)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        cs.csrc_autotune_spmm(h, Xd, Yd, 16, torch.cuda.current_stream())
        assert cs.csrc_get_info(h)["tuned_rk"] in (1, 2, 4, 8)
        Y = _run(cs, h, X, "f64", False)
        assert oracle.max_rel_err(m, X, Y, oracle.csrc_spmm(c, X)) <= 1e-12
    finally:
        cs.csrc_destroy(h)
