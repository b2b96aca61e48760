"""Seeded synthetic finite-element matrices and vectors.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark. It generates *inputs only*: symmetric sparsity patterns of FE meshes,
random coefficients and source vectors. It contains none of the CSRC method's
arithmetic (no format conversion, no products, no partitioning, no colouring).

Every matrix is returned as a full CSR (both triangles plus the diagonal,
column indices sorted ascending within each row, 0-based), which is the input
format the library's ``csrc_create_from_csr`` and the oracle both accept.
"""
from .generators import (  # noqa: F401
    FEMatrix,
    RectMatrix,
    overlap_subdomain,
    splitmix64,
    hash_uniform,
    pattern_from_edges,
    p1_triangle_grid_edges,
    kuhn_tet_grid_edges,
    p1_triangle_grid_pattern,
    kuhn_tet_grid_pattern,
    q1_hex27_pattern,
    delaunay_edges,
    permute_pattern,
    rcm_permutation,
    expand_dofs,
    random_fe_values,
    integer_values,
    laplacian_values,
    convection_values,
    source_vector,
    integer_vector,
    p1_grid,
    q1_hex,
    tet_mesh,
    batch_meshes,
    random_symmetric_pattern,
    CONFIGS,
)
