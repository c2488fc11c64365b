"""Input generators: FE assembly, AMG setup and the hierarchy blob (CPU only)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_1503_08462_gb300.inputs import hierarchy, meshes
from oracle import amg_oracle as O

from helpers import problem_and_blob


def test_problem_sizes():
    assert meshes.square_2d(32).n == 31 ** 2 == 961
    assert meshes.lshape_2d(8).n == 15 ** 2 - 8 ** 2
    assert meshes.cube_3d(6).n == 5 ** 3
    # the L-shape at h = 1/512 has (1023^2 - 512^2) interior nodes
    assert 1023 ** 2 - 512 ** 2 == 784_385


@pytest.mark.parametrize("make", [lambda: meshes.square_2d(16), lambda: meshes.lshape_2d(8),
                                  lambda: meshes.square_2d(16, checker=4, seed=3), lambda: meshes.cube_3d(6)])
def test_fe_matrices_spd_and_shared_pattern(make):
    p = make()
    A, M = p.scipy()
    assert abs(A - A.T).max() < 1e-12 * abs(A).max()
    assert abs(M - M.T).max() < 1e-14 * abs(M).max()
    assert np.all(np.diff(p.row_ptr) > 0)
    for i in range(p.n):  # sorted, unique columns with the diagonal present
        cols = p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
    assert np.linalg.eigvalsh(A.toarray()).min() > 0
    assert np.linalg.eigvalsh(M.toarray()).min() > 0
    assert np.all(p.m_vals > 0)


def test_mass_matrix_integrates_one():
    # 1^T M 1 over all nodes (boundary included) is the domain area; with the
    # Dirichlet rows removed it is smaller but tends to the area as h -> 0.
    p = meshes.square_2d(64)
    _, M = p.scipy()
    total = M.sum()
    assert 0.9 < total < 1.0


def test_unit_square_eigenvalues_converge_at_h2():
    """Dense FE eigenvalues approach pi^2 (2, 5, 5, 8) at rate O(h^2)."""
    exact = np.pi ** 2 * np.array([2.0, 5.0, 5.0, 8.0])
    errs = []
    hs = []
    for m in (8, 16, 32):
        p = meshes.square_2d(m, seed=1)
        A, M = p.scipy()
        lam = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 3])
        errs.append(np.abs(lam - exact) / exact)
        hs.append(1.0 / m)
    errs = np.array(errs)
    assert np.all(errs[-1] < 0.02)
    slope = np.polyfit(np.log(hs), np.log(errs.mean(axis=1)), 1)[0]
    assert 1.7 < slope < 2.4, slope


def test_unit_cube_eigenvalues_converge_with_multiplicities():
    """Unit cube: pi^2 (3, 6, 6, 6, 9, 9, 9); the FE error falls like h^2."""
    exact = np.pi ** 2 * np.array([3.0, 6, 6, 6, 9, 9, 9])
    errs = []
    for m in (6, 12):
        p = meshes.cube_3d(m, seed=4)
        A, M = p.scipy()
        lam = sla.eigh(A.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 6])
        # group structure: the gap between groups dwarfs the splitting inside
        assert lam[1] - lam[0] > 5 * np.ptp(lam[1:4]) and lam[4] - lam[3] > 3 * np.ptp(lam[4:7])
        errs.append(np.abs(lam - exact) / exact)
    ratio = errs[0].mean() / errs[1].mean()
    assert 2.8 < ratio < 6.0, ratio


@pytest.mark.parametrize("kind,size,cap", [("square", 32, 50), ("checker", 32, 40), ("lshape", 16, 60),
                                           ("cube", 8, 40)])
def test_hierarchy_galerkin_and_interpolation(kind, size, cap):
    p, blob, h = problem_and_blob(kind, size, cap)
    assert h.sizes[-1] <= cap and all(a > b for a, b in zip(h.sizes, h.sizes[1:]))
    for l, P in enumerate(h.prolong):
        lv, lc = h.levels[l], h.levels[l + 1]
        Pm = sp.csr_matrix((P.vals, P.col_idx, P.row_ptr), shape=(lv.n, lc.n))
        for vals_f, vals_c in ((lv.a_vals, lc.a_vals), (lv.m_vals, lc.m_vals)):
            Af = sp.csr_matrix((vals_f, lv.col_idx, lv.row_ptr), shape=(lv.n, lv.n))
            Ac = sp.csr_matrix((vals_c, lc.col_idx, lc.row_ptr), shape=(lc.n, lc.n))
            diff = abs(Pm.T @ Af @ Pm - Ac).max()
            assert diff <= 1e-13 * abs(Ac).max()
        # C points are injected: their rows hold a single 1; every coarse column
        # has exactly one such row
        ones_rows = np.nonzero((np.diff(P.row_ptr) == 1))[0]
        inj = [P.col_idx[P.row_ptr[i]] for i in ones_rows if P.vals[P.row_ptr[i]] == 1.0]
        assert len(set(inj)) == lc.n
        # rows whose A row sums to zero interpolate constants exactly (Sec. 2.2)
        Af = sp.csr_matrix((lv.a_vals, lv.col_idx, lv.row_ptr), shape=(lv.n, lv.n))
        rowsum = np.asarray(Af.sum(axis=1)).ravel()
        zero = np.abs(rowsum) < 1e-12 * np.abs(Af).max()
        pc = Pm @ np.ones(lc.n)
        assert np.allclose(pc[zero], 1.0, atol=1e-12)


def test_blob_roundtrip_and_corruption():
    p, blob, h = problem_and_blob("square", 32, 50)
    oh = O.read_blob(blob)
    assert oh.sizes == h.sizes
    A, M = p.scipy()
    assert abs(oh.A[0] - A).max() == 0 and abs(oh.M[0] - M).max() == 0
    bad = bytearray(blob)
    bad[200] ^= 0x40
    with pytest.raises(ValueError):
        O.read_blob(bytes(bad))
    with pytest.raises(ValueError):
        O.read_blob(blob[:-16])
    with pytest.raises(ValueError):
        O.read_blob(b"XXXXXXXX" + blob[8:])


def test_single_level_hierarchy():
    p = meshes.square_2d(8)
    h = hierarchy.build_for_problem(p, coarse_cap=1000)
    assert h.sizes == [p.n] and h.prolong == []
