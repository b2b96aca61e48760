"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances, per row i, relative to sum_j |a_ij||x_j| (original FP64 values):
1e-12 for FP64 storage, 1e-5 for FP32 storage, 1e-2 for BF16 storage. Integer-valued
inputs are exact in every storage type and strategy, so there the results
must match bit for bit. Partitions and colourings must match exactly.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import fe_inputs as fe
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-2}
STRATS = ("window", "window_atomic", "atomic", "color")


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


class Handle:
    def __init__(self, cs, m, storage="f64", flags=0, seed=None):
        self.cs = cs
        self.m = m
        self.storage = storage
        self.h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.STORAGE[storage], flags)
        self.ncolors = None
        if seed is not None:
            self.ncolors = cs.csrc_color(self.h, seed)

    def run(self, x, strategy="window", transpose=False, nbands=None):
        cs = self.cs
        if nbands is not None:
            cs.csrc_partition(self.h, nbands)
        if strategy == "color" and self.ncolors is None:
            self.ncolors = cs.csrc_color(self.h, 12345)
        dt = torch.float64 if self.storage == "f64" else torch.float32
        xd = torch.as_tensor(np.asarray(x), dtype=dt).cuda()
        yd = torch.full_like(xd, float("nan"))
        fn = cs.csrc_spmv_t if transpose else cs.csrc_spmv
        fn(self.h, xd, yd, cs.STRATEGIES[strategy], torch.cuda.current_stream())
        torch.cuda.synchronize()
        st = cs.csrc_get_last_device_error(self.h)
        assert st == cs.CSRC_OK, cs.csrc_status_string(st)
        return yd.cpu().numpy().astype(np.float64)

    def close(self):
        self.cs.csrc_destroy(self.h)


def _transpose(m):
    at = sp.csr_matrix((m.val, m.col, m.row_ptr), shape=(m.n, m.n)).T.tocsr()
    return fe.FEMatrix(m.n, at.indptr.astype(np.int64), at.indices.astype(np.int32), at.data)


def _ref(m, x, transpose=False):
    c = oracle.from_matrix(m)
    return oracle.csrc_spmv_t(c, x) if transpose else oracle.csrc_spmv(c, x)


def _check(m, x, y, transpose, tol):
    mm = _transpose(m) if transpose else m
    err = oracle.max_rel_err(mm, x, y, _ref(m, x, transpose))
    assert err <= tol, f"max rel err {err:.3e} > {tol:.0e}"
    return err


# --------------------------------------------------------------------------- config 1: P1 100x100, FP64
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("transpose", [False, True])
def test_p1_grid_fp64(cs, strategy, transpose):
    m = fe.p1_grid(100, 100, 1001)
    x = fe.source_vector(m.n, 2001)
    h = Handle(cs, m)
    try:
        _check(m, x, h.run(x, strategy, transpose), transpose, TOL["f64"])
    finally:
        h.close()


@pytest.mark.parametrize("strategy", ["window", "window_atomic", "atomic"])
@pytest.mark.parametrize("flags", ["default", "fp64", "df32"])
def test_arithmetic_flags(cs, strategy, flags):
    # FP64 storage computes on the FP64 pipe unless double-float is asked for, which only the
    # stream-order strategies use
    m = fe.p1_grid(60, 50, 11)
    x = fe.source_vector(m.n, 12)
    f = {"default": 0, "fp64": cs.CSRC_FLAG_FP64_ARITH, "df32": cs.CSRC_FLAG_DF32_ARITH}[flags]
    h = Handle(cs, m, flags=f)
    try:
        assert cs.csrc_get_info(h.h)["arith"] == (0 if flags == "df32" else 1)
        for tr in (False, True):
            _check(m, x, h.run(x, strategy, tr), tr, TOL["f64"])
    finally:
        h.close()


def test_window_strategy_is_bitwise_reproducible(cs):
    # every window row is summed by one lane in a fixed order: repeated products agree bit
    # for bit, for every storage type and for A x and A^T x
    m = fe.q1_hex(12, 3, 91)
    x = fe.source_vector(m.n, 92)
    for storage in ("f64", "f32", "bf16"):
        h = Handle(cs, m, storage)
        try:
            for tr in (False, True):
                y0 = h.run(x, "window", tr)
                for _ in range(3):
                    np.testing.assert_array_equal(h.run(x, "window", tr), y0)
        finally:
            h.close()


def test_window_lists_cover_every_entry(cs):
    # the lists hold every stored value once (n diagonal entries and both values of each pair)
    for m in (fe.q1_hex(12, 3, 93), fe.p1_grid(70, 40, 94), fe.tet_mesh(5000, 95, method="kuhn")):
        x = fe.source_vector(m.n, 96)
        h = Handle(cs, m)
        try:
            for nb in (None, 1, 5, 300):
                h.run(x, "window", False, nbands=nb)
                info = cs.csrc_get_info(h.h)
                assert info["list_entries"] == m.nnz
                assert info["list_lane_steps"] >= info["list_entries"]
                assert info["list_slices"] * 32 >= m.n + info["spill_entries"]
        finally:
            h.close()


# --------------------------------------------------------------------------- exact integer cases
def _integer_cases():
    cases = []
    for n, d, s in ((1, 0.0, 1), (2, 1.0, 2), (17, 0.3, 3), (300, 0.02, 4), (1000, 0.005, 5), (777, 0.01, 6)):
        rp, c = fe.random_symmetric_pattern(n, d, s)
        cases.append((f"rand{n}", rp, c))
    ei, ej = fe.p1_triangle_grid_edges(13, 7)
    rp, c = fe.pattern_from_edges(91, ei, ej)
    cases.append(("p1_13x7", rp, c))
    q = fe.q1_hex(7, 3, 5)
    cases.append(("q1v_7", q.row_ptr, q.col))
    return cases


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("strategy", STRATS)
def test_integer_values_bit_exact(cs, storage, strategy):
    for name, rp, c in _integer_cases():
        n = len(rp) - 1
        m = fe.FEMatrix(n, rp, c, fe.integer_values(rp, c, 77))
        x = fe.integer_vector(n, 78)
        h = Handle(cs, m, storage)
        try:
            for tr in (False, True):
                y = h.run(x, strategy, tr)
                np.testing.assert_array_equal(y, _ref(m, x, tr), err_msg=f"{name} {storage} {strategy} T={tr}")
        finally:
            h.close()


# --------------------------------------------------------------------------- several bands, ragged tails
@pytest.mark.parametrize("nbands", [1, 3, 152, 1000])
def test_q1_vector_many_bands(cs, nbands):
    m = fe.q1_hex(14, 3, 21)  # n = 8232, RCM order
    x = fe.source_vector(m.n, 22)
    h = Handle(cs, m)
    try:
        for strategy in ("window", "window_atomic", "atomic"):
            for tr in (False, True):
                _check(m, x, h.run(x, strategy, tr, nbands=nbands), tr, TOL["f64"])
        info = cs.csrc_get_info(h.h)
        assert info["nbands"] >= min(nbands, m.n)
    finally:
        h.close()


def test_partition_matches_oracle(cs):
    for m in (fe.p1_grid(30, 20, 3), fe.q1_hex(9, 3, 4), fe.tet_mesh(3000, 5, method="kuhn")):
        c = oracle.from_matrix(m)
        h = Handle(cs, m)
        try:
            for nb in (1, 2, 7, 152, 500):
                out = np.zeros(nb + 1, np.int32)
                cs.csrc_partition(h.h, nb, out)
                np.testing.assert_array_equal(out, oracle.partition(c, nb))
                oracle.check_partition(c.ia, nb, out)
        finally:
            h.close()


def test_colouring_matches_oracle_greedy(cs):
    for m, seed in ((fe.p1_grid(40, 25, 3), 1), (fe.q1_hex(8, 3, 4), 99), (fe.tet_mesh(4000, 6, method="kuhn"), 7)):
        c = oracle.from_matrix(m)
        h = Handle(cs, m)
        try:
            colors = np.zeros(m.n, np.int32)
            k = cs.csrc_color(h.h, seed, colors)
            k_ref, colors_ref = oracle.jp_color(c, seed)
            assert k == k_ref
            np.testing.assert_array_equal(colors, colors_ref)
            assert oracle.check_coloring(c, colors, k) == 0
        finally:
            h.close()


# --------------------------------------------------------------------------- mixed precision
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("strategy", STRATS)
def test_mixed_precision_error(cs, storage, strategy):
    m = fe.tet_mesh(20000, 1003, method="kuhn")
    x = fe.source_vector(m.n, 2003).astype(np.float32).astype(np.float64)
    h = Handle(cs, m, storage)
    try:
        for tr in (False, True):
            y = h.run(x, strategy, tr)
            err = _check(m, x, y, tr, TOL[storage])
            # against the exact product of the stored (rounded) matrix: FP32 accumulation only
            c = oracle.from_matrix(m)
            al, au, ad = oracle.quantised(c, storage)
            yq = (oracle.csrc_spmv_t if tr else oracle.csrc_spmv)(c, x, al=al, au=au, ad=ad)
            mm = _transpose(m) if tr else m
            assert oracle.max_rel_err(mm, x, y, yq) <= 2e-6, err
    finally:
        h.close()


# --------------------------------------------------------------------------- long rows: 16 lanes per row
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_long_rows_run_sixteen_lanes(cs, storage):
    # 3 DOF per node on a 14^3 grid: about 34 pairs per row, taken by 16 lanes in a
    # 1024-thread CTA (three pairs per lane per pass, so rows of up to 48 pairs in one pass)
    m = fe.q1_hex(14, 3, 23)
    x = fe.source_vector(m.n, 24)
    if storage != "f64":
        x = x.astype(np.float32).astype(np.float64)
    mi = fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 25))
    xi = fe.integer_vector(m.n, 26)
    h, hi = Handle(cs, m, storage), Handle(cs, mi, storage)
    try:
        for nbands in (None, 7, 300):
            for strategy in ("window", "window_atomic", "atomic"):
                for tr in (False, True):
                    _check(m, x, h.run(x, strategy, tr, nbands=nbands), tr, TOL[storage])
                    np.testing.assert_array_equal(hi.run(xi, strategy, tr, nbands=nbands), _ref(mi, xi, tr))
        assert cs.csrc_get_info(h.h)["group"] == 16
        assert cs.csrc_get_info(hi.h)["group"] == 16
    finally:
        h.close()
        hi.close()


# --------------------------------------------------------------------------- symmetric values
def test_symmetric_values(cs):
    rp, c = fe.q1_hex27_pattern(10, 9, 8)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    val = fe.hash_uniform(5, np.minimum(rows, c), np.maximum(rows, c))
    m = fe.FEMatrix(n, rp, c, val)
    x = fe.source_vector(n, 6)
    h = Handle(cs, m, seed=3)
    try:
        # colour-ordered rows have a fixed update order: A x and A^T x agree bit for bit
        np.testing.assert_array_equal(h.run(x, "color", False), h.run(x, "color", True))
        # so do the window strategy's lists (one lane per row, a fixed order)
        np.testing.assert_array_equal(h.run(x, "window", False), h.run(x, "window", True))
        for s in ("window", "window_atomic", "atomic"):
            y1, y2 = h.run(x, s, False), h.run(x, s, True)
            _check(m, x, y1, False, TOL["f64"])
            assert oracle.max_rel_err(m, x, y1, y2) <= 1e-12
    finally:
        h.close()


def _symmetrised(m, seed, integer=False):
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr))
    v = fe.hash_uniform(seed, np.minimum(rows, m.col), np.maximum(rows, m.col))
    if integer:
        v = np.round(v * 8.0)
    return fe.FEMatrix(m.n, m.row_ptr, m.col, v)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_symmetric_value_storage(cs, storage):
    # Section 2.2: au is not stored; the kernels scatter with al, and A^T x = A x
    for base in (fe.q1_hex(9, 1, 51), fe.q1_hex(14, 3, 52)):  # 4 and 16 lanes per row
        m = _symmetrised(base, 53)
        x = fe.source_vector(m.n, 54)
        if storage != "f64":
            x = x.astype(np.float32).astype(np.float64)
        plain = Handle(cs, m, storage)
        h = Handle(cs, m, storage, flags=cs.CSRC_FLAG_SYMMETRIC_VALUES, seed=5)
        mi = _symmetrised(base, 55, integer=True)
        xi = fe.integer_vector(m.n, 56)
        hi = Handle(cs, mi, storage, flags=cs.CSRC_FLAG_SYMMETRIC_VALUES, seed=6)
        try:
            for strategy in STRATS:
                for tr in (False, True):
                    _check(m, x, h.run(x, strategy, tr), tr, TOL[storage])
                    np.testing.assert_array_equal(hi.run(xi, strategy, tr), _ref(mi, xi, tr))
            plain.run(x)
            ip, ih = cs.csrc_get_info(plain.h), cs.csrc_get_info(h.h)
            vb = {"f64": 8, "f32": 4, "bf16": 2}[storage]
            assert ip["model_bytes"] - ih["model_bytes"] == vb * ip["pairs"]
        finally:
            plain.close()
            h.close()
            hi.close()


def test_symmetric_value_storage_other_paths(cs):
    # node blocks, several right-hand sides and the batched graph read al as the scatter operand too
    m = _symmetrised(fe.q1_hex(8, 3, 57), 58)
    c = oracle.from_matrix(m)
    flags = cs.CSRC_FLAG_SYMMETRIC_VALUES
    h = Handle(cs, m, flags=flags | cs.CSRC_FLAG_NODE_BLOCKS)
    try:
        x = fe.source_vector(m.n, 59)
        _check(m, x, h.run(x, "window_atomic", False), False, TOL["f64"])
        assert cs.csrc_get_info(h.h)["block"] == 3
    finally:
        h.close()
    h = Handle(cs, m, flags=flags)
    try:
        X = fe.source_vector(m.n, 60, nrhs=4)
        Xd = torch.as_tensor(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        cs.csrc_spmm_batched([h.h], [Xd], [Yd], 4, False, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert oracle.max_rel_err(m, X, Yd.cpu().numpy(), oracle.csrc_spmm(c, X)) <= TOL["f64"]
    finally:
        h.close()
    mats = [_symmetrised(fe.p1_grid(30 + 5 * i, 20, 61 + i), 62 + i) for i in range(3)]
    hs = [cs.csrc_create_from_csr(q.n, q.row_ptr, q.col, q.val, cs.CSRC_F32, flags) for q in mats]
    try:
        xs = [fe.source_vector(q.n, 70 + i).astype(np.float32).astype(np.float64) for i, q in enumerate(mats)]
        Xd = [torch.as_tensor(v, dtype=torch.float32).cuda() for v in xs]
        Yd = [torch.full_like(v, float("nan")) for v in Xd]
        cs.csrc_spmm_batched(hs, Xd, Yd, 1, False, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for q, v, y in zip(mats, xs, Yd):
            ref = oracle.csrc_spmv(oracle.from_matrix(q), v)
            assert oracle.max_rel_err(q, v, y.cpu().numpy().astype(np.float64), ref) <= TOL["f32"]
    finally:
        for hh in hs:
            cs.csrc_destroy(hh)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_index_compression(cs, storage):
    # 16-bit band-local window slots in place of 32-bit ones (the window strategy's plans)
    for base in (fe.q1_hex(9, 1, 81), fe.q1_hex(14, 3, 82)):
        x = fe.source_vector(base.n, 83)
        if storage != "f64":
            x = x.astype(np.float32).astype(np.float64)
        mi = fe.FEMatrix(base.n, base.row_ptr, base.col, fe.integer_values(base.row_ptr, base.col, 84))
        xi = fe.integer_vector(base.n, 85)
        plain = Handle(cs, base, storage)
        h = Handle(cs, base, storage, flags=cs.CSRC_FLAG_COMPRESS_INDICES, seed=7)
        hi = Handle(cs, mi, storage, flags=cs.CSRC_FLAG_COMPRESS_INDICES, seed=8)
        ms = _symmetrised(base, 86)
        hs = Handle(cs, ms, storage, flags=cs.CSRC_FLAG_COMPRESS_INDICES | cs.CSRC_FLAG_SYMMETRIC_VALUES)
        try:
            for nbands in (None, 9):
                for strategy in STRATS:
                    for tr in (False, True):
                        _check(base, x, h.run(x, strategy, tr, nbands=nbands), tr, TOL[storage])
                        np.testing.assert_array_equal(hi.run(xi, strategy, tr, nbands=nbands), _ref(mi, xi, tr))
                _check(ms, x, hs.run(x, "window", False, nbands=nbands), False, TOL[storage])
            plain.run(x)
            ip, ih = cs.csrc_get_info(plain.h), cs.csrc_get_info(h.h)
            assert ip["model_bytes"] - ih["model_bytes"] == 2 * ip["pairs"]
        finally:
            for hh in (plain, h, hi, hs):
                hh.close()


# --------------------------------------------------------------------------- failure detection
def test_bounded_wait_gives_up_and_the_context_stays_usable(cs):
    # a barrier nothing arrives at: the bounded wait gives up after ~1 ms, the kernel returns
    # normally and the host reads DEVICE_TIMEOUT from the status word
    import time

    t0 = time.perf_counter()
    assert cs.csrc_selftest_bounded_wait(2_000_000) == cs.CSRC_ERR_DEVICE_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    m = fe.q1_hex(6, 1, 131)
    x = fe.source_vector(m.n, 132)
    h = Handle(cs, m)
    try:
        _check(m, x, h.run(x), False, TOL["f64"])
    finally:
        h.close()


# --------------------------------------------------------------------------- interface behaviour
def test_host_pointers_are_staged(cs):
    m = fe.p1_grid(50, 40, 9)
    x = fe.source_vector(m.n, 10)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        y = np.full(m.n, np.nan)
        cs.csrc_spmv(h, x, y, cs.CSRC_STRAT_WINDOW, None)
        torch.cuda.synchronize()
        _check(m, x, y, False, TOL["f64"])
        xp = torch.from_numpy(x).pin_memory()
        yp = torch.empty_like(xp).pin_memory()
        cs.csrc_spmv_t(h, xp, yp, cs.CSRC_STRAT_AUTO, None)
        torch.cuda.synchronize()
        _check(m, x, yp.numpy(), True, TOL["f64"])
    finally:
        cs.csrc_destroy(h)


def test_interface_errors(cs):
    m = fe.p1_grid(10, 10, 1)
    h = cs.csrc_create_from_csr(m.n, m.row_ptr, m.col, m.val, cs.CSRC_F64)
    try:
        xd = torch.zeros(m.n, dtype=torch.float64, device="cuda")
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv(h, xd, xd, cs.CSRC_STRAT_WINDOW)
        assert e.value.status == cs.CSRC_ERR_ALIAS
        with pytest.raises(cs.CsrcError) as e:
            cs.csrc_spmv(h, xd, torch.zeros_like(xd), cs.CSRC_STRAT_COLOR)
        assert e.value.status == cs.CSRC_ERR_NOT_COLORED
    finally:
        cs.csrc_destroy(h)


def test_double_float_range_is_reported(cs):
    m = fe.p1_grid(20, 20, 2)
    x = fe.source_vector(m.n, 3)
    x[17] = 1e300
    h = Handle(cs, m, flags=cs.CSRC_FLAG_DF32_ARITH)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        cs.csrc_spmv(h.h, xd, yd, cs.CSRC_STRAT_WINDOW_ATOMIC)
        torch.cuda.synchronize()
        assert cs.csrc_get_last_device_error(h.h) == cs.CSRC_ERR_RANGE
        assert cs.csrc_get_last_device_error(h.h) == cs.CSRC_OK  # cleared by the read
        # the window strategy computes in FP64 whatever the flag
        _check(m, x, h.run(x, "window"), False, TOL["f64"])
    finally:
        h.close()
    # FP64 arithmetic (the default) handles the full double range, tiny entries included
    x2 = x.copy()
    x2[5:40] *= 1e-20
    x2[60:90] *= 1e20
    h = Handle(cs, m)
    try:
        for s in ("window", "window_atomic", "atomic"):
            for xx in (x, x2):
                _check(m, xx, h.run(xx, s), False, TOL["f64"])
        torch.cuda.synchronize()
        assert cs.csrc_get_last_device_error(h.h) == cs.CSRC_OK  # no false range error
    finally:
        h.close()
    # matrix values outside the double-float range switch a double-float handle to FP64 arithmetic
    m2 = fe.FEMatrix(m.n, m.row_ptr, m.col, m.val * 1e-30)
    h = Handle(cs, m2, flags=cs.CSRC_FLAG_DF32_ARITH)
    try:
        assert cs.csrc_get_info(h.h)["arith"] == 1
        x2 = fe.source_vector(m.n, 4)
        _check(m2, x2, h.run(x2, "window_atomic"), False, TOL["f64"])
    finally:
        h.close()


def test_degenerate_matrices(cs):
    # diagonal only, a single row, and rows without lower entries
    for n in (1, 5, 64, 65):
        rp = np.arange(n + 1, dtype=np.int64)
        col = np.arange(n, dtype=np.int32)
        val = np.arange(1, n + 1, dtype=np.float64)
        m = fe.FEMatrix(n, rp, col, val)
        x = fe.source_vector(n, n)
        xi = fe.integer_vector(n, n)
        h = Handle(cs, m, seed=1)
        try:
            for s in STRATS:
                np.testing.assert_array_equal(h.run(xi, s), val * xi)
                _check(m, x, h.run(x, s), False, TOL["f64"])
        finally:
            h.close()
    # empty matrix
    h = cs.csrc_create_from_csr(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    cs.csrc_spmv(h, torch.zeros(1, dtype=torch.float64, device="cuda"),
                 torch.zeros(1, dtype=torch.float64, device="cuda"))
    cs.csrc_destroy(h)


def test_coo_and_padding(cs):
    m = fe.p1_grid(12, 9, 4)
    rows = np.repeat(np.arange(m.n), np.diff(m.row_ptr)).astype(np.int32)
    # COO in shuffled order with one entry split into two duplicates
    perm = np.random.default_rng(0).permutation(m.nnz)
    r, c, v = rows[perm], m.col[perm], m.val[perm].copy()
    r = np.concatenate([r, r[:1]])
    c = np.concatenate([c, c[:1]])
    v = np.concatenate([v, [0.0]])
    h = cs.csrc_create_from_coo(m.n, len(r), r, c, v, cs.CSRC_F64)
    try:
        x = fe.source_vector(m.n, 5)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        cs.csrc_spmv(h, xd, yd, cs.CSRC_STRAT_WINDOW)
        _check(m, x, yd.cpu().numpy(), False, TOL["f64"])
    finally:
        cs.csrc_destroy(h)
    # drop the upper triangle: padding adds explicit zero mirrors
    keep = m.col <= rows
    rp = np.zeros(m.n + 1, np.int64)
    np.cumsum(np.bincount(rows[keep], minlength=m.n), out=rp[1:])
    lower = fe.FEMatrix(m.n, rp, m.col[keep], m.val[keep])
    with pytest.raises(cs.CsrcError) as e:
        cs.csrc_create_from_csr(lower.n, lower.row_ptr, lower.col, lower.val, cs.CSRC_F64)
    assert e.value.status == cs.CSRC_ERR_NOT_STRUCT_SYMMETRIC
    h = cs.csrc_create_from_csr(lower.n, lower.row_ptr, lower.col, lower.val, cs.CSRC_F64, cs.CSRC_FLAG_PAD_PATTERN)
    try:
        x = fe.source_vector(m.n, 6)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        cs.csrc_spmv(h, xd, yd, cs.CSRC_STRAT_WINDOW)
        yref = oracle.csr_spmv(lower.n, lower.row_ptr, lower.col, lower.val, x)
        assert oracle.max_rel_err(lower, x, yd.cpu().numpy(), yref) <= 1e-12
    finally:
        cs.csrc_destroy(h)


# --------------------------------------------------------------------------- autotuner
def test_autotune_picks_a_strategy_and_stays_correct(cs):
    m = fe.q1_hex(16, 3, 44)
    x = fe.source_vector(m.n, 45)
    h = Handle(cs, m, seed=9)  # coloured, so the colour strategy is a candidate too
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty_like(xd)
        cs.csrc_autotune(h.h, xd, yd, torch.cuda.current_stream())
        info = cs.csrc_get_info(h.h)
        assert info["tuned_strategy"] in (cs.CSRC_STRAT_WINDOW, cs.CSRC_STRAT_COLOR, cs.CSRC_STRAT_ATOMIC,
                                          cs.CSRC_STRAT_WINDOW_ATOMIC)
        for tr in (False, True):
            _check(m, x, h.run(x, "auto", tr), tr, TOL["f64"])
    finally:
        h.close()


# --------------------------------------------------------------------------- node blocks
@pytest.mark.parametrize("ndof", [2, 3])
def test_node_block_kernel_matches_plain_rows_and_oracle(cs, ndof):
    # with CSRC_FLAG_NODE_BLOCKS, matrices with ndof unknowns per node run node-block
    # units; they, the plain-row kernel and the oracle must agree
    m = fe.q1_hex(10, ndof, 51)
    im = fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 52))
    xi = fe.integer_vector(m.n, 53)
    x = fe.source_vector(m.n, 54)
    for storage in ("f64", "f32", "bf16"):
        hb = Handle(cs, im, storage, flags=cs.CSRC_FLAG_NODE_BLOCKS)
        hp = Handle(cs, im, storage)
        try:
            for tr in (False, True):
                yb = hb.run(xi, "window_atomic", tr)
                np.testing.assert_array_equal(yb, _ref(im, xi, tr))
                np.testing.assert_array_equal(hp.run(xi, "window_atomic", tr), yb)
                np.testing.assert_array_equal(hp.run(xi, "window", tr), yb)
            assert cs.csrc_get_info(hb.h)["block"] == ndof
            assert cs.csrc_get_info(hp.h)["block"] == 1
        finally:
            hb.close()
            hp.close()
    h = Handle(cs, m, flags=cs.CSRC_FLAG_NODE_BLOCKS)
    try:
        for nb in (1, 5, 152):
            for tr in (False, True):
                _check(m, x, h.run(x, "window_atomic", tr, nbands=nb), tr, TOL["f64"])
        # the atomic strategy runs plain rows on a second plan
        _check(m, x, h.run(x, "atomic"), False, TOL["f64"])
    finally:
        h.close()


def test_scalar_matrix_has_no_node_blocks(cs):
    m = fe.q1_hex(8, 1, 3)
    h = Handle(cs, m)
    try:
        h.run(fe.source_vector(m.n, 4))
        assert cs.csrc_get_info(h.h)["block"] == 1
    finally:
        h.close()


# --------------------------------------------------------------------------- stride-bounded colouring
@pytest.mark.parametrize("stride", [0, 1, 7, 64, 1000])
def test_stride_colouring_matches_oracle(cs, stride):
    # the library's host colouring (ascending rows, class gaps <= stride) equals the oracle's
    # bit for bit, is valid, and the colour product on its classes matches the oracle
    for m in (fe.p1_grid(40, 25, 3), fe.q1_hex(8, 3, 4), fe.tet_mesh(4000, 6, method="kuhn")):
        c = oracle.from_matrix(m)
        h = Handle(cs, m)
        try:
            colors = np.zeros(m.n, np.int32)
            k = cs.csrc_color_stride(h.h, stride, colors)
            k_ref, colors_ref = oracle.greedy_color_stride(c, stride)
            assert k == k_ref
            np.testing.assert_array_equal(colors, colors_ref)
            assert oracle.check_coloring(c, colors, k) == 0
            if stride > 0:
                assert oracle.max_class_gap(colors, k) <= stride
            h.ncolors = k
            x = fe.source_vector(m.n, 7)
            for tr in (False, True):
                _check(m, x, h.run(x, "color", tr), tr, TOL["f64"])
        finally:
            h.close()


def test_colour_product_many_classes(cs):
    # stride 1 on a P1 grid gives hundreds of classes: hundreds of grid barriers in one launch;
    # integer values make the result exact
    m = fe.p1_grid(30, 30, 11)
    mi = fe.FEMatrix(m.n, m.row_ptr, m.col, fe.integer_values(m.row_ptr, m.col, 12))
    xi = fe.integer_vector(m.n, 13)
    for storage in ("f64", "f32", "bf16"):
        h = Handle(cs, mi, storage)
        try:
            h.ncolors = cs.csrc_color_stride(h.h, 1)
            assert h.ncolors > 100
            for tr in (False, True):
                np.testing.assert_array_equal(h.run(xi, "color", tr), _ref(mi, xi, tr))
        finally:
            h.close()
