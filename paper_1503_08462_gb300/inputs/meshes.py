"""Seeded synthetic P1 finite-element eigenproblems A u = lambda M u.

These generators produce the inputs that both the CUDA solve path and the CPU
oracle consume.  They hold none of the eigensolver's arithmetic: they only
build meshes and assemble the linear finite-element stiffness matrix A and
mass matrix M (Sec. 4.1 of the paper discretises -Laplace u = lambda u and
-div(K grad u) = lambda u with linear finite elements; Examples 1-3).

Meshes are structured grids whose interior nodes are jittered by a seeded
uniform displacement; every square cell is split into two triangles along a
seeded random diagonal (2D) or into the six Kuhn tetrahedra (3D).  Homogeneous
Dirichlet nodes are eliminated, so M is SPD.  A and M are returned in CSR with
int32 indices and one shared sparsity pattern (the pattern is structural: an
entry exists when the two nodes share an element, even if the stiffness value
happens to be zero).

Random draws, in this order from ``numpy.random.default_rng(seed)``:
  1. the 16 checkerboard coefficients 10**U(-3, 3) (checkerboard problems only),
  2. the node jitter U(-j*h, j*h), one value per node and axis for ALL grid
     nodes in node order (boundary nodes then get zero displacement),
  3. the cell diagonals, one Bernoulli(1/2) integer per cell in cell order (2D).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Problem:
    """A generalized eigenproblem A u = lambda M u in shared-pattern CSR form."""

    name: str
    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col_idx: np.ndarray  # int32 [nnz], sorted within each row
    a_vals: np.ndarray  # float64 [nnz] stiffness
    m_vals: np.ndarray  # float64 [nnz] mass
    coords: np.ndarray  # float64 [n, dim] node coordinates (interior nodes)
    h: float

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def scipy(self):
        """Return (A, M) as scipy.sparse CSR matrices (test convenience)."""
        import scipy.sparse as sp

        shape = (self.n, self.n)
        a = sp.csr_matrix((self.a_vals, self.col_idx, self.row_ptr), shape=shape)
        m = sp.csr_matrix((self.m_vals, self.col_idx, self.row_ptr), shape=shape)
        return a, m


# --------------------------------------------------------------------------
# element matrices


def _p1_element(coords: np.ndarray):
    """Stiffness gradients and measure for a batch of simplices.

    coords: [E, d+1, d] vertex coordinates.  Returns (grads [E, d+1, d],
    measure [E], signed_det [E]) for the P1 barycentric basis functions.
    """
    e, nv, d = coords.shape
    jac = coords[:, 1:, :] - coords[:, :1, :]  # [E, d, d], rows = edge vectors
    det = np.linalg.det(jac)
    inv = np.linalg.inv(jac)  # columns give gradients of barycentrics 1..d
    g = np.empty((e, nv, d))
    g[:, 1:, :] = np.transpose(inv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    fact = 2.0 if d == 2 else 6.0
    return g, np.abs(det) / fact, det


def _assemble_stencil(n_nodes, elems, coords_all, kappa, offsets_lin, d, coords_ref):
    """Accumulate P1 element matrices into a per-node stencil array.

    elems: [E, d+1] global node ids; kappa: [E] coefficient per element.
    offsets_lin: sorted array of allowed linear node-id offsets.
    coords_ref: unjittered node coordinates; every element must keep the
    orientation (sign of its Jacobian determinant) it has on the unjittered grid.
    Returns (a_st, m_st, touched) each [n_nodes, S].
    """
    s = offsets_lin.shape[0]
    pos = {int(o): k for k, o in enumerate(offsets_lin)}
    lut_min = int(offsets_lin.min())
    lut = -np.ones(int(offsets_lin.max()) - lut_min + 1, dtype=np.int64)
    for o, k in pos.items():
        lut[o - lut_min] = k
    a_st = np.zeros(n_nodes * s)
    m_st = np.zeros(n_nodes * s)
    touched = np.zeros(n_nodes * s, dtype=np.int64)
    nv = d + 1
    chunk = 1 << 20
    for c0 in range(0, elems.shape[0], chunk):
        el = elems[c0:c0 + chunk]
        g, meas, det = _p1_element(coords_all[el])
        _, _, det_ref = _p1_element(coords_ref[el])
        if np.any(meas <= 0) or np.any(np.sign(det) != np.sign(det_ref)):
            raise ValueError("degenerate or inverted element after jitter")
        kap = kappa[c0:c0 + chunk]
        kloc = np.einsum("eid,ejd->eij", g, g) * (kap * meas)[:, None, None]
        mfac = meas / (12.0 if d == 2 else 20.0)
        for i in range(nv):
            for j in range(nv):
                rows = el[:, i]
                off = el[:, j] - rows
                slot = lut[off - lut_min]
                if np.any(slot < 0):
                    raise ValueError("element edge outside the stencil")
                flat = rows * s + slot
                a_st += np.bincount(flat, weights=kloc[:, i, j], minlength=n_nodes * s)
                mv = mfac * (2.0 if i == j else 1.0)
                m_st += np.bincount(flat, weights=mv, minlength=n_nodes * s)
                touched += np.bincount(flat, minlength=n_nodes * s)
    return a_st.reshape(n_nodes, s), m_st.reshape(n_nodes, s), touched.reshape(n_nodes, s)


def _stencil_to_csr(a_st, m_st, touched, offsets_lin, interior):
    """Eliminate Dirichlet nodes and convert the stencil arrays to CSR."""
    n_nodes, s = a_st.shape
    new_id = -np.ones(n_nodes, dtype=np.int64)
    new_id[interior] = np.arange(int(interior.sum()))
    rows_old = np.nonzero(interior)[0]
    nbr = rows_old[:, None] + offsets_lin[None, :]
    valid = (nbr >= 0) & (nbr < n_nodes)
    nbr_c = np.where(valid, nbr, 0)
    keep = valid & (touched[rows_old] > 0) & interior[nbr_c]
    cols = new_id[nbr_c]
    counts = keep.sum(axis=1)
    row_ptr = np.zeros(rows_old.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    # offsets_lin is sorted ascending and new_id is monotone, so columns are sorted
    col_idx = cols[keep].astype(np.int32)
    a_vals = a_st[rows_old][keep]
    m_vals = m_st[rows_old][keep]
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 range")
    return row_ptr.astype(np.int32), col_idx, a_vals, m_vals, new_id


# --------------------------------------------------------------------------
# 2D


def _grid2d(nx, ny, x0, y0, h, jitter, rng, boundary):
    """Jittered and reference coordinates of an (nx+1) x (ny+1) grid; boundary fixed."""
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    xy = np.stack([x0 + ii.ravel() * h, y0 + jj.ravel() * h], axis=1).astype(np.float64)
    disp = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    disp[boundary] = 0.0
    return xy + disp, xy


def _triangles(nx, ny, cell_keep, rng):
    """Two triangles per kept cell, split along a seeded random diagonal."""
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()
    diag = rng.integers(0, 2, size=ci.shape[0])
    w = nx + 1
    n00 = cj * w + ci
    n10 = n00 + 1
    n01 = n00 + w
    n11 = n01 + 1
    keep = cell_keep.ravel()
    n00, n10, n01, n11, diag = n00[keep], n10[keep], n01[keep], n11[keep], diag[keep]
    # diag 0: split along n00-n11; diag 1: split along n10-n01
    t1 = np.where(diag[:, None] == 0, np.stack([n00, n10, n11], 1), np.stack([n00, n10, n01], 1))
    t2 = np.where(diag[:, None] == 0, np.stack([n00, n11, n01], 1), np.stack([n10, n11, n01], 1))
    cells = np.nonzero(keep)[0]
    return np.concatenate([t1, t2]), np.concatenate([cells, cells])


def _offsets2d(w):
    return np.array(sorted(dj * w + di for dj in (-1, 0, 1) for di in (-1, 0, 1)), dtype=np.int64)


def square_2d(m: int = 32, jitter: float = 0.2, seed: int = 1, checker=None) -> Problem:
    """Unit square (0,1)^2, m cells per side, N = (m-1)^2 interior nodes.

    checker: None, or the number of checkerboard blocks per side (4 for the
    discontinuous-coefficient problem -div(kappa grad u) = lambda u of Sec. 4,
    Examples 3-4, with kappa = 10**U(-3, 3) drawn per block).
    """
    rng = np.random.default_rng(seed)
    kappa_blocks = None
    if checker:
        kappa_blocks = 10.0 ** rng.uniform(-3.0, 3.0, size=checker * checker)
    h = 1.0 / m
    w = m + 1
    ii, jj = np.meshgrid(np.arange(w), np.arange(w), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    boundary = (ii == 0) | (ii == m) | (jj == 0) | (jj == m)
    xy, xy_ref = _grid2d(m, m, 0.0, 0.0, h, jitter, rng, boundary)
    tris, cell_of = _triangles(m, m, np.ones((m, m), dtype=bool), rng)
    kappa = np.ones(tris.shape[0])
    if checker:
        if m % checker:
            raise ValueError("m must be a multiple of the checkerboard size")
        bs = m // checker
        cell_i = cell_of % m
        cell_j = cell_of // m
        kappa = kappa_blocks[(cell_j // bs) * checker + (cell_i // bs)]
    interior = ~boundary
    offs = _offsets2d(w)
    a_st, m_st, touched = _assemble_stencil(w * w, tris, xy, kappa, offs, 2, xy_ref)
    rp, ci, av, mv, _ = _stencil_to_csr(a_st, m_st, touched, offs, interior)
    name = f"square2d_m{m}" + (f"_checker{checker}" if checker else "")
    return Problem(name, int(interior.sum()), rp, ci, av, mv, xy[interior], h)


def lshape_2d(m_half: int = 512, jitter: float = 0.2, seed: int = 2) -> Problem:
    """L-shape (-1,1)^2 minus [0,1) x (-1,0], h = 1/m_half (Sec. 4, Example 2)."""
    rng = np.random.default_rng(seed)
    m = 2 * m_half
    h = 1.0 / m_half
    w = m + 1
    ii, jj = np.meshgrid(np.arange(w), np.arange(w), indexing="xy")
    ii = ii.ravel()
    jj = jj.ravel()
    # removed quadrant: x >= 0 and y <= 0  <=>  i >= m_half and j <= m_half
    outside_or_on = (ii >= m_half) & (jj <= m_half)
    boundary = (ii == 0) | (ii == m) | (jj == 0) | (jj == m) | outside_or_on
    xy, xy_ref = _grid2d(m, m, -1.0, -1.0, h, jitter, rng, boundary)
    ci_, cj_ = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
    cell_keep = ~((ci_ >= m_half) & (cj_ < m_half))
    tris, _ = _triangles(m, m, cell_keep, rng)
    interior = ~boundary
    offs = _offsets2d(w)
    a_st, m_st, touched = _assemble_stencil(w * w, tris, xy, np.ones(tris.shape[0]), offs, 2, xy_ref)
    rp, ci, av, mv, _ = _stencil_to_csr(a_st, m_st, touched, offs, interior)
    return Problem(f"lshape2d_m{m_half}", int(interior.sum()), rp, ci, av, mv, xy[interior], h)


# --------------------------------------------------------------------------
# 3D

_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def cube_3d(m: int = 128, jitter: float = 0.15, seed: int = 4) -> Problem:
    """Unit cube, m cells per side, six Kuhn tetrahedra per cell, N = (m-1)^3."""
    rng = np.random.default_rng(seed)
    h = 1.0 / m
    w = m + 1
    kk, jj, ii = np.meshgrid(np.arange(w), np.arange(w), np.arange(w), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    boundary = (ii == 0) | (ii == m) | (jj == 0) | (jj == m) | (kk == 0) | (kk == m)
    xyz_ref = np.stack([ii * h, jj * h, kk * h], axis=1).astype(np.float64)
    disp = rng.uniform(-jitter * h, jitter * h, size=xyz_ref.shape)
    disp[boundary] = 0.0
    xyz = xyz_ref + disp
    ck, cj, ci = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    base = ((ck.ravel() * w) + cj.ravel()) * w + ci.ravel()
    strides = np.array([1, w, w * w], dtype=np.int64)
    tets = []
    for perm in _KUHN_PERMS:
        o1 = strides[perm[0]]
        o2 = o1 + strides[perm[1]]
        o3 = o2 + strides[perm[2]]
        tets.append(np.stack([base, base + o1, base + o2, base + o3], axis=1))
    tets = np.concatenate(tets)
    offs = _kuhn_edge_offsets(strides)
    interior = ~boundary
    a_st, m_st, touched = _assemble_stencil(w ** 3, tets, xyz, np.ones(tets.shape[0]), offs, 3, xyz_ref)
    rp, ci, av, mv, _ = _stencil_to_csr(a_st, m_st, touched, offs, interior)
    return Problem(f"cube3d_m{m}", int(interior.sum()), rp, ci, av, mv, xyz[interior], h)


def _kuhn_edge_offsets(strides):
    """Linear node-id offsets of all vertex pairs within one Kuhn tetrahedron (15)."""
    out = set()
    for perm in _KUHN_PERMS:
        o1 = strides[perm[0]]
        o2 = o1 + strides[perm[1]]
        o3 = o2 + strides[perm[2]]
        verts = [0, int(o1), int(o2), int(o3)]
        out.update(a - b for a in verts for b in verts)
    return np.array(sorted(out), dtype=np.int64)
