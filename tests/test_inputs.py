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
