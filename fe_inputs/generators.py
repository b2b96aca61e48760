"""Synthetic FE matrices standing in for the paper's test set (Section 4, Table 1).

The paper measures on University of Florida matrices and on the authors' own FE
matrices, none of which are available here. These generators produce matrices
with the same structure: symmetric non-zero patterns of 2D triangle meshes,
3D hexahedral 27-point stencils (scalar and 3-DOF vector), 3D tetrahedral
meshes and batches of mixed meshes. They use RCM or natural orderings, and
their values are non-symmetric U[-1,1) with a dominant diagonal.

Coefficients come from a counter-based generator (SplitMix64 applied to a key
built from the seed and the ordered pair (i, j)). So a_ij and a_ji are
independent, and the values do not depend on generation order or chunking.
Orderings and source vectors use numpy's seeded ``default_rng``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class FEMatrix:
    """A structurally symmetric matrix in full CSR form (0-based, sorted columns)."""

    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def pairs(self) -> int:
        """Number of stored off-diagonal pairs h = (nnz - n)/2 for a full diagonal."""
        return (self.nnz - self.n) // 2


# ----------------------------------------------------------------------------- hashing
@dataclass
class RectMatrix:
    """An n-by-m matrix (m >= n) in CSR form (0-based, sorted columns) whose leading
    n-by-n block has a symmetric pattern: one subdomain of an overlapping decomposition."""

    n: int
    m: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz], values in [0, m)
    val: np.ndarray  # float64[nnz]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def splitmix64(z) -> np.ndarray:
    """SplitMix64 output function applied to counter ``z`` (Steele, Lea & Flood, 2014).

    Computes mix(z + 0x9E3779B97F4A7C15) with the published multipliers; uint64
    arithmetic wraps modulo 2^64.
    """
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _pair_bits(seed: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    key = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
    s = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    return splitmix64(key ^ s)


def hash_uniform(seed: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """U[-1, 1) value attached to the ordered pair (i, j); 53 random bits."""
    h = _pair_bits(seed, i, j)
    u = (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


# ----------------------------------------------------------------------------- patterns
def pattern_from_edges(n: int, ei: np.ndarray, ej: np.ndarray):
    """Full symmetric CSR pattern (with diagonal) from undirected edges i != j."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    diag = np.arange(n, dtype=np.int64)
    rows = np.concatenate([ei, ej, diag])
    cols = np.concatenate([ej, ei, diag])
    key = np.unique(rows * n + cols)
    rows = key // n
    cols = (key - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols


def p1_triangle_grid_edges(nx: int, ny: int):
    """Edges of a structured P1 triangle mesh on nx*ny nodes, node id = iy*nx + ix.

    Each grid square is split by its diagonal (ix,iy)-(ix+1,iy+1).
    """
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ix = ix.ravel()
    iy = iy.ravel()
    nid = iy * nx + ix
    e = []
    m = ix + 1 < nx
    e.append((nid[m], nid[m] + 1))
    m = iy + 1 < ny
    e.append((nid[m], nid[m] + nx))
    m = (ix + 1 < nx) & (iy + 1 < ny)
    e.append((nid[m], nid[m] + nx + 1))
    ei = np.concatenate([a for a, _ in e])
    ej = np.concatenate([b for _, b in e])
    return ei, ej


def kuhn_tet_grid_edges(nx: int, ny: int, nz: int):
    """Edges of the Kuhn (Freudenthal) tetrahedralisation of an nx*ny*nz node grid.

    Every cube is cut into six tetrahedra sharing its main diagonal; interior
    nodes have exactly 14 neighbours. Node id = (iz*ny + iy)*nx + ix.
    """
    ids = np.arange(nx * ny * nz, dtype=np.int64)
    ix = ids % nx
    iy = (ids // nx) % ny
    iz = ids // (nx * ny)
    dirs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    ei, ej = [], []
    for dx, dy, dz in dirs:
        m = (ix + dx < nx) & (iy + dy < ny) & (iz + dz < nz)
        ei.append(ids[m])
        ej.append(ids[m] + dx + dy * nx + dz * nx * ny)
    return np.concatenate(ei), np.concatenate(ej)


def q1_hex27_pattern(nx: int, ny: int, nz: int):
    """Full CSR pattern of the Q1 hexahedral (27-point) stencil, natural node order."""
    n = nx * ny * nz
    ids = np.arange(n, dtype=np.int64)
    ix = ids % nx
    iy = (ids // nx) % ny
    iz = ids // (nx * ny)
    cols = np.empty((n, 27), dtype=np.int64)
    q = 0
    for dz in (-1, 0, 1):  # lexicographic (dz, dy, dx) gives ascending column ids
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                ok = (
                    (ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny)
                    & (iz + dz >= 0) & (iz + dz < nz)
                )
                cols[:, q] = np.where(ok, ids + dx + dy * nx + dz * nx * ny, -1)
                q += 1
    mask = cols >= 0
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols[mask].astype(np.int32)
    return row_ptr, col


def _stencil_pattern(dims, offsets):
    """Full CSR pattern of a structured grid stencil: node id = (iz*ny + iy)*nx + ix,
    neighbours at the given (dx, dy, dz) offsets (the centre included), columns ascending."""
    nx, ny, nz = dims
    n = nx * ny * nz
    ids = np.arange(n, dtype=np.int64)
    ix = ids % nx
    iy = (ids // nx) % ny
    iz = ids // (nx * ny)
    offs = sorted(offsets, key=lambda o: o[0] + o[1] * nx + o[2] * nx * ny)  # ascending column id
    cols = np.empty((n, len(offs)), dtype=np.int64)
    for q, (dx, dy, dz) in enumerate(offs):
        ok = ((ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny) & (iz + dz >= 0) & (iz + dz < nz))
        cols[:, q] = np.where(ok, ids + dx + dy * nx + dz * nx * ny, -1)
    mask = cols >= 0
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=row_ptr[1:])
    return row_ptr, cols[mask].astype(np.int32)


def p1_triangle_grid_pattern(nx: int, ny: int):
    """The pattern of p1_triangle_grid_edges (plus the diagonal), built directly in CSR form."""
    d = [(1, 0, 0), (0, 1, 0), (1, 1, 0)]
    offs = [(0, 0, 0)] + d + [(-a, -b, -c) for a, b, c in d]
    return _stencil_pattern((nx, ny, 1), offs)


def kuhn_tet_grid_pattern(nx: int, ny: int, nz: int):
    """The pattern of kuhn_tet_grid_edges (plus the diagonal), built directly in CSR form."""
    d = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
    offs = [(0, 0, 0)] + d + [(-a, -b, -c) for a, b, c in d]
    return _stencil_pattern((nx, ny, nz), offs)


def delaunay_edges(npts: int, seed: int):
    """Edges of the Delaunay tetrahedralisation of npts uniform points in the unit cube."""
    from scipy.spatial import Delaunay

    pts = np.random.default_rng(seed).random((npts, 3))
    simp = Delaunay(pts).simplices.astype(np.int64)
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    a = np.concatenate([simp[:, p] for p, _ in pairs])
    b = np.concatenate([simp[:, q] for _, q in pairs])
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = np.unique(lo * npts + hi)
    return key // npts, key % npts


def permute_pattern(row_ptr: np.ndarray, col: np.ndarray, perm: np.ndarray):
    """Symmetric permutation B = A[perm][:, perm] (perm[k] = old index at new position k)."""
    import scipy.sparse as sp

    n = len(row_ptr) - 1
    a = sp.csr_matrix((np.ones(len(col), dtype=np.int8), col, row_ptr), shape=(n, n))
    b = a[perm][:, perm].tocsr()
    b.sort_indices()
    return b.indptr.astype(np.int64), b.indices.astype(np.int32)


def rcm_permutation(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Reverse Cuthill-McKee order of a symmetric pattern (scipy's implementation)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    n = len(row_ptr) - 1
    a = sp.csr_matrix((np.ones(len(col), dtype=np.int8), col, row_ptr), shape=(n, n))
    return np.asarray(reverse_cuthill_mckee(a, symmetric_mode=True), dtype=np.int64)


def expand_dofs(row_ptr: np.ndarray, col: np.ndarray, d: int, chunk_nodes: int = 1 << 16):
    """Pattern of d DOFs per node with dense d*d node blocks, DOF id = d*node + a."""
    if d == 1:
        return row_ptr.astype(np.int64), col.astype(np.int32)
    nn = len(row_ptr) - 1
    m = np.diff(row_ptr)
    dof_len = np.repeat(m * d, d)
    out_ptr = np.zeros(nn * d + 1, dtype=np.int64)
    np.cumsum(dof_len, out=out_ptr[1:])
    out_col = np.empty(int(out_ptr[-1]), dtype=np.int32)
    ar = np.arange(d, dtype=np.int64)
    for s in range(0, nn, chunk_nodes):
        e = min(nn, s + chunk_nodes)
        blk = (col[row_ptr[s]:row_ptr[e]].astype(np.int64)[:, None] * d + ar).reshape(-1)
        lens = m[s:e] * d  # per node row, its column block length
        starts = np.zeros(e - s, dtype=np.int64)
        np.cumsum(lens[:-1], out=starts[1:])
        # each node row's block is repeated d times (once per DOF row)
        rep_len = np.repeat(lens, d)
        rep_start = np.repeat(starts, d)
        base = np.zeros(len(rep_len), dtype=np.int64)
        np.cumsum(rep_len[:-1], out=base[1:])
        total = int(rep_len.sum())
        idx = np.arange(total, dtype=np.int64) - np.repeat(base - rep_start, rep_len)
        out_col[out_ptr[s * d]:out_ptr[e * d]] = blk[idx]
    return out_ptr, out_col


def random_symmetric_pattern(n: int, density: float, seed: int, empty_rows: bool = True):
    """Random symmetric pattern for small tests; some rows may have no off-diagonals."""
    rng = np.random.default_rng(seed)
    if n <= 1:
        return pattern_from_edges(max(n, 0), np.zeros(0, np.int64), np.zeros(0, np.int64))
    m = max(0, int(density * n * (n - 1) / 2))
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n, size=m)
    keep = i != j
    i, j = i[keep], j[keep]
    if not empty_rows:
        ring_i = np.arange(1, n)
        i = np.concatenate([i, ring_i])
        j = np.concatenate([j, ring_i - 1])
    return pattern_from_edges(n, i, j)


def overlap_subdomain(g: "FEMatrix", n_sub: int, name: str = "") -> RectMatrix:
    """Rows 0..n_sub-1 of a global FE matrix as one subdomain of an overlapping
    decomposition: the subdomain's own unknowns keep their numbers 0..n_sub-1 and every
    other unknown its rows reach (the overlap) is numbered n_sub, n_sub+1, ... in
    increasing global order, so columns stay sorted within each row."""
    n_sub = int(min(max(n_sub, 0), g.n))
    rp = np.ascontiguousarray(g.row_ptr[:n_sub + 1], dtype=np.int64)
    col = g.col[:int(rp[-1])].astype(np.int64)
    val = np.array(g.val[:int(rp[-1])], dtype=np.float64)
    ext = np.unique(col[col >= n_sub])
    newcol = np.where(col < n_sub, col, n_sub + np.searchsorted(ext, col))
    return RectMatrix(n_sub, n_sub + len(ext), rp, newcol.astype(np.int32), val, name=name or f"{g.name}_sub{n_sub}",
                      meta={"global_n": g.n, "overlap": ext.astype(np.int64)})


# ----------------------------------------------------------------------------- values
def _rows_of(row_ptr: np.ndarray, s: int, e: int) -> np.ndarray:
    return np.repeat(np.arange(s, e, dtype=np.int64), np.diff(row_ptr[s:e + 1]))


def random_fe_values(row_ptr: np.ndarray, col: np.ndarray, seed: int, chunk_rows: int = 1 << 18):
    """Off-diagonals U[-1,1) independent per ordered pair; a_ii = 1 + sum_{j!=i} |a_ij|."""
    n = len(row_ptr) - 1
    val = np.empty(len(col), dtype=np.float64)
    for s in range(0, n, chunk_rows):
        e = min(n, s + chunk_rows)
        lo, hi = row_ptr[s], row_ptr[e]
        rows = _rows_of(row_ptr, s, e)
        c = col[lo:hi].astype(np.int64)
        v = hash_uniform(seed, rows, c)
        isdiag = rows == c
        v[isdiag] = 0.0
        rowsum = np.bincount(rows - s, weights=np.abs(v), minlength=e - s)
        v[isdiag] = 1.0 + rowsum[rows[isdiag] - s]
        val[lo:hi] = v
    return val


def integer_values(row_ptr: np.ndarray, col: np.ndarray, seed: int, lo: int = -8, hi: int = 8):
    """Integer coefficients in [lo, hi] (diagonal included), exact in FP64, FP32 and BF16."""
    n = len(row_ptr) - 1
    rows = _rows_of(row_ptr, 0, n)
    h = _pair_bits(seed, rows, col.astype(np.int64))
    span = np.uint64(hi - lo + 1)
    return (h % span).astype(np.int64).astype(np.float64) + lo


def laplacian_values(row_ptr: np.ndarray, col: np.ndarray):
    """Graph Laplacian of the pattern: off-diagonals -1, diagonal = number of neighbours."""
    n = len(row_ptr) - 1
    rows = _rows_of(row_ptr, 0, n)
    val = -np.ones(len(col), dtype=np.float64)
    isdiag = rows == col
    deg = np.bincount(rows[~isdiag], minlength=n).astype(np.float64)
    val[isdiag] = deg[rows[isdiag]]
    return val


def convection_values(row_ptr: np.ndarray, col: np.ndarray, coord: np.ndarray, beta: float):
    """Non-symmetric convection-diffusion stencil with zero row sums.

    a_ij = -(1 + beta*(c_j - c_i)) for j != i and a_ii = sum_{j != i} (1 + beta*(c_j - c_i)),
    where c is a per-node coordinate.
    """
    n = len(row_ptr) - 1
    rows = _rows_of(row_ptr, 0, n)
    dx = coord[col] - coord[rows]
    val = -(1.0 + beta * dx)
    isdiag = rows == col
    val[isdiag] = 0.0
    diag = -np.bincount(rows, weights=val, minlength=n)
    val[isdiag] = diag[rows[isdiag]]
    return val


def source_vector(n: int, seed: int, nrhs: int | None = None, dtype=np.float64) -> np.ndarray:
    """x ~ U[-1,1) (n, or n*nrhs row-major when nrhs is given)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs is None else (n, nrhs)
    return rng.uniform(-1.0, 1.0, size=shape).astype(dtype)


def integer_vector(n: int, seed: int, lo: int = -8, hi: int = 8, nrhs: int | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs is None else (n, nrhs)
    return rng.integers(lo, hi + 1, size=shape).astype(np.float64)


# ----------------------------------------------------------------------------- configurations
def p1_grid(nx: int = 100, ny: int = 100, seed: int = 1001) -> FEMatrix:
    """P1 triangles on an nx*ny node grid, natural order (100x100: n=10,000, nnz=69,202)."""
    ei, ej = p1_triangle_grid_edges(nx, ny)
    n = nx * ny
    rp, c = pattern_from_edges(n, ei, ej)
    return FEMatrix(n, rp, c, random_fe_values(rp, c, seed), f"p1_{nx}x{ny}",
                    {"nx": nx, "ny": ny, "order": "natural"})


def q1_hex(nn: int = 96, ndof: int = 1, seed: int = 1002, order: str = "rcm") -> FEMatrix:
    """Q1 hexahedral 27-point pattern on nn^3 nodes with ndof DOFs per node.

    order='rcm': random symmetric node permutation (default_rng(seed)), then RCM on
    the node graph; DOFs stay interleaved (row = ndof*node + a). order='natural'
    keeps node id = (iz*nn + iy)*nn + ix.
    """
    rp, c = q1_hex27_pattern(nn, nn, nn)
    meta = {"nn": nn, "ndof": ndof, "order": order}
    if order == "rcm":
        rng = np.random.default_rng(seed)
        p1 = rng.permutation(nn ** 3)
        rp, c = permute_pattern(rp, c, p1)
        r = rcm_permutation(rp, c)
        rp, c = permute_pattern(rp, c, r)
        meta["node_perm"] = p1[r]
    elif order != "natural":
        raise ValueError(order)
    rp, c = expand_dofs(rp, c, ndof)
    n = len(rp) - 1
    name = f"q1{'v' if ndof > 1 else 's'}_{nn}"
    return FEMatrix(n, rp, c, random_fe_values(rp, c, seed), name, meta)


def tet_mesh(npts: int = 2_000_000, seed: int = 1003, order: str = "rcm", method: str = "delaunay") -> FEMatrix:
    """P1 tetrahedral pattern: Delaunay of npts uniform points (or a Kuhn lattice).

    method='kuhn' uses the Kuhn tetrahedralisation of a cube lattice with
    ceil(npts^(1/3)) nodes per side (14 neighbours per interior node).
    """
    if method == "delaunay":
        ei, ej = delaunay_edges(npts, seed)
        n = npts
    elif method == "kuhn":
        side = int(math.ceil(npts ** (1.0 / 3.0) - 1e-9))
        ei, ej = kuhn_tet_grid_edges(side, side, side)
        n = side ** 3
    else:
        raise ValueError(method)
    rp, c = pattern_from_edges(n, ei, ej)
    if order == "rcm":
        rng = np.random.default_rng(seed)
        p1 = rng.permutation(n)
        rp, c = permute_pattern(rp, c, p1)
        rp, c = permute_pattern(rp, c, rcm_permutation(rp, c))
    elif order == "random":
        rp, c = permute_pattern(rp, c, np.random.default_rng(seed).permutation(n))
    return FEMatrix(n, rp, c, random_fe_values(rp, c, seed), f"tet_{method}_{n}",
                    {"order": order, "method": method})


def batch_meshes(count: int = 256, seed: int = 1005, nmin: int = 2000, nmax: int = 400_000) -> list[FEMatrix]:
    """Uneven batch: n log-uniform in [nmin, nmax]; 2D P1 triangle or 3D Kuhn-tet grid (p=1/2 each)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        target = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
        if rng.random() < 0.5:
            side = max(2, int(round(math.sqrt(target))))
            rp, c = p1_triangle_grid_pattern(side, side)
            n = side * side
            kind = "p1"
        else:
            side = max(2, int(round(target ** (1.0 / 3.0))))
            rp, c = kuhn_tet_grid_pattern(side, side, side)
            n = side ** 3
            kind = "kuhn"
        val = random_fe_values(rp, c, seed * 100003 + b)
        out.append(FEMatrix(n, rp, c, val, f"batch{b}_{kind}_{n}", {"kind": kind, "side": side}))
    return out


# Configuration registry: name -> (builder, x seed). Sizes are the full workloads.
CONFIGS = {
    "p1_100x100": (lambda: p1_grid(100, 100, 1001), 2001),
    "q1s_96": (lambda: q1_hex(96, 1, 1002), 2002),
    "q1v_96": (lambda: q1_hex(96, 3, 1002), 2002),
    # the same structure on 64^3 nodes (n = 786,432, nnz = 62.4M): a smaller case of q1v_96's
    # kernels for profiler captures (still several times larger than L2)
    "q1v_64": (lambda: q1_hex(64, 3, 1002), 2002),
    "tet_delaunay_2m": (lambda: tet_mesh(2_000_000, 1003), 2003),
    "q1s_96_multi": (lambda: q1_hex(96, 1, 1002), 2004),
    "batch_256": (lambda: batch_meshes(256, 1005), 2005),
}
