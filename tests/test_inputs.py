"""The seeded input generators (no method arithmetic): structured patterns built two ways agree,
and the configuration sizes are the ones the workloads are quoted on."""
import numpy as np
import pytest

import fe_inputs as fe


@pytest.mark.parametrize("nx,ny", [(2, 2), (7, 5), (13, 9)])
def test_p1_direct_pattern_equals_edge_pattern(nx, ny):
    a = fe.pattern_from_edges(nx * ny, *fe.p1_triangle_grid_edges(nx, ny))
    b = fe.p1_triangle_grid_pattern(nx, ny)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("dims", [(2, 2, 2), (4, 5, 6), (7, 3, 5)])
def test_kuhn_direct_pattern_equals_edge_pattern(dims):
    a = fe.pattern_from_edges(dims[0] * dims[1] * dims[2], *fe.kuhn_tet_grid_edges(*dims))
    b = fe.kuhn_tet_grid_pattern(*dims)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_kuhn_interior_nodes_have_14_neighbours():
    rp, _ = fe.kuhn_tet_grid_pattern(5, 5, 5)
    centre = (2 * 5 + 2) * 5 + 2
    assert rp[centre + 1] - rp[centre] == 15  # 14 neighbours and the diagonal


def test_batch_sizes_are_log_uniform_in_range():
    ms = fe.batch_meshes(16, 3, nmin=2000, nmax=400_000)
    ns = np.array([m.n for m in ms])
    assert ns.min() >= 1000 and ns.max() <= 500_000
    assert {m.meta["kind"] for m in ms} <= {"p1", "kuhn"}


def test_overlap_subdomain_layout():
    # one subdomain of an overlapping decomposition: own unknowns first, then the overlap in
    # increasing global order; columns stay sorted and the square block is the leading block
    g = fe.q1_hex(6, 3, 41)
    for n_sub in (1, g.n // 3, g.n // 2, g.n):
        a = fe.overlap_subdomain(g, n_sub)
        assert a.n == n_sub and a.m >= a.n
        assert a.row_ptr[0] == 0 and a.row_ptr[-1] == a.nnz == int(g.row_ptr[n_sub])
        for i in range(a.n):
            c = a.col[a.row_ptr[i]:a.row_ptr[i + 1]]
            assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < a.m
            gc = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
            np.testing.assert_array_equal(c[c < a.n], gc[gc < a.n])
        ext = a.meta["overlap"]
        assert len(ext) == a.m - a.n and np.all(np.diff(ext) > 0) and (len(ext) == 0 or ext.min() >= n_sub)
        # every overlap column is reached by some row
        assert np.all(np.bincount(a.col, minlength=a.m)[a.n:] > 0)
    assert fe.overlap_subdomain(g, g.n).m == g.n

