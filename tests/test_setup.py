"""The device AMG setup (amgeig_setup_blob) against the package's host setup (Sec. 2): same levels, C/F
splittings and sparsity patterns, interpolation weights and Galerkin coarse matrices equal up to the
rounding of sums taken in another order, and solves on either hierarchy agreeing."""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1503_08462_gb300 import amgeig as ae
from paper_1503_08462_gb300.inputs import hierarchy, meshes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


CASES = [("square", dict(m=32, seed=1), 50), ("lshape", dict(m_half=24, seed=2), 60),
         ("checker", dict(m=48, checker=4, seed=3), 60), ("cube", dict(m=12, seed=4), 40),
         # dense Galerkin rows on the coarse 3D levels: products with rows beyond the shared staging
         ("cube", dict(m=40, seed=4), 60)]


def _problem(kind, kw):
    if kind == "square":
        return meshes.square_2d(**kw)
    if kind == "checker":
        return meshes.square_2d(**kw)
    if kind == "lshape":
        return meshes.lshape_2d(**kw)
    return meshes.cube_3d(**kw)


@pytest.mark.parametrize("kind,kw,cap", CASES)
def test_device_setup_equals_host_setup(kind, kw, cap):
    p = _problem(kind, kw)
    blob_h, hh = hierarchy.problem_blob(p, coarse_cap=cap)
    blob_d, secs, split_s = ae.amgeig_setup_blob(p.row_ptr, p.col_idx, p.a_vals, p.m_vals, coarse_cap=cap)
    assert secs > 0 and 0 <= split_s <= secs
    oh, od = O.read_blob(blob_h), O.read_blob(blob_d)  # both parse, checksums included
    assert oh.sizes == od.sizes
    for l in range(len(oh.sizes)):
        # identical patterns: the same splitting and the same symbolic products
        assert np.array_equal(oh.A[l].indptr, od.A[l].indptr) and np.array_equal(oh.A[l].indices, od.A[l].indices)
        for X, Y in ((oh.A[l], od.A[l]), (oh.M[l], od.M[l])):
            scale = np.abs(X.data).max()
            assert np.abs(X.data - Y.data).max() <= 1e-13 * scale, (l, np.abs(X.data - Y.data).max() / scale)
    for l in range(len(oh.P)):
        assert np.array_equal(oh.P[l].indptr, od.P[l].indptr) and np.array_equal(oh.P[l].indices, od.P[l].indices)
        assert np.abs(oh.P[l].data - od.P[l].data).max() <= 1e-15
        # Galerkin identity on the device hierarchy itself
        for X, Xc in ((od.A[l], od.A[l + 1]), (od.M[l], od.M[l + 1])):
            G = (od.R[l] @ X @ od.P[l]).toarray() if Xc.shape[0] <= 2000 else None
            if G is not None:
                assert np.abs(G - Xc.toarray()).max() <= 1e-13 * np.abs(G).max()


def test_solve_on_the_device_built_hierarchy():
    p = _problem("lshape", dict(m_half=24, seed=2))
    blob_h, _ = hierarchy.problem_blob(p, coarse_cap=60)
    blob_d, _, _ = ae.amgeig_setup_blob(p.row_ptr, p.col_idx, p.a_vals, p.m_vals, coarse_cap=60)
    opt = ae.options(q_extra=3, max_corrections=80, precision=ae.AMGEIG_MIXED_FP32, v_cycles=2)
    with ae.Hierarchy(blob_h) as hh, ae.Hierarchy(blob_d) as hd:
        lh, _, ih, ch = hh.solve(6, tol=1e-9, opt=opt)
        ld, _, idd, cd = hd.solve(6, tol=1e-9, opt=opt)
    assert ch == cd == ae.AMGEIG_OK
    assert np.max(np.abs(lh - ld) / lh) <= 1e-10


def test_setup_argument_errors():
    p = _problem("square", dict(m=8, seed=1))
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_setup_blob(p.row_ptr, p.col_idx, p.a_vals, p.m_vals, theta=1.5)
    assert e.value.code == ae.AMGEIG_EINVAL
    bad = p.col_idx.copy()
    bad[3] = p.n + 7
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_setup_blob(p.row_ptr, bad, p.a_vals, p.m_vals)
    assert e.value.code == ae.AMGEIG_EINVAL
