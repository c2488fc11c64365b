"""Full-size checks on the timed workload.

L-shape h = 1/512 (N = 784,385), q = 20 with 8 buffer vectors, mixed path, two V-cycles
per correction, 64 coarse modes, relative residual 1e-4: the configuration and the launch
shapes that bench.py times.  The oracle cannot run the whole solve at this size in
seconds, so the checks are (a) properties that hold at any size, recomputed on the CPU
from their definitions (residuals, M-orthonormality, ordering, signs, agreement with the
float64 path, Ritz upper bounds), and (b) single building blocks at full size against the
oracle: the defect on sampled rows (including the ragged tail) and one V-cycle.
"""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1503_08462_gb300 import amgeig as ae
from paper_1503_08462_gb300.inputs import hierarchy, meshes

pytestmark = pytest.mark.gpu

Q, Q_EXTRA, TOL = 20, 8, 1e-4


@pytest.fixture(scope="module")
def workload():
    import __graft_entry__

    __graft_entry__.build()
    p = meshes.lshape_2d(m_half=512, seed=2)
    blob, _ = hierarchy.problem_blob(p, coarse_cap=400)
    oh = O.read_blob(blob)
    h = ae.Hierarchy(blob)
    yield oh, h
    h.close()


def test_full_size_solve_properties(workload):
    oh, h = workload
    opt = ae.options(q_extra=Q_EXTRA, max_corrections=60, precision=ae.AMGEIG_MIXED_FP32, coarse_modes=64,
                     v_cycles=2)
    lam, U, info, code = h.solve(Q, tol=TOL, opt=opt)
    assert code == ae.AMGEIG_OK and info.converged == 1 and info.dense_fallbacks == 0
    assert U.shape == (oh.A[0].shape[0], Q)
    assert np.all(O.relres(oh, lam, U) <= TOL * 1.0001)
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(Q)).max() < 1e-10
    assert np.all(np.diff(lam) >= 0)
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(Q)] > 0)
    # the float64 path with the paper's full coarse space, converged tightly
    lam64, _, _, code64 = h.solve(Q, tol=1e-8, opt=ae.options(q_extra=Q_EXTRA, max_corrections=150), vectors=False)
    assert code64 == ae.AMGEIG_OK
    assert np.max(np.abs(lam - lam64) / lam64) <= 1e-8
    # Ritz values bound the discrete eigenvalues from above: the less converged values
    # cannot lie below the tightly converged ones beyond rounding (the float-float
    # Rayleigh-Ritz resolves values to ~1e-11 relative)
    assert np.all(lam >= lam64 * (1.0 - 1e-10)), np.min((lam - lam64) / lam64)


@pytest.mark.parametrize("prec", [ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32])
def test_full_size_defect_sampled_rows(workload, prec):
    oh, h = workload
    A, M = oh.A[0], oh.M[0]
    n = A.shape[0]
    rng = np.random.default_rng(11)
    U = rng.standard_normal((n, Q + Q_EXTRA))
    lam = rng.uniform(9.0, 400.0, Q + Q_EXTRA)
    R, rr = ae.amgeig_apply_defect(h.handle, 0, U, lam, ae.options(precision=prec))
    rows = np.unique(np.concatenate([rng.integers(0, n, 4000), np.arange(256), np.arange(n - 257, n)]))
    As, Ms = A[rows], M[rows]
    ref = (Ms @ U) * lam[None, :] - As @ U
    scale = abs(As) @ abs(U) + (abs(Ms) @ abs(U)) * lam[None, :]
    if prec == ae.AMGEIG_FP64:
        assert np.all(np.abs(R[rows] - ref) <= 1e-14 * scale)
    else:
        assert np.all(np.abs(R[rows] - ref) <= 2.0 ** -23 * np.abs(ref) + 2.0 ** -42 * scale)
    np.testing.assert_allclose(rr, O.relres(oh, lam, U), rtol=1e-6 if prec != ae.AMGEIG_FP64 else 1e-10)


@pytest.mark.parametrize("prec,rtol", [(ae.AMGEIG_FP64, 1e-11), (ae.AMGEIG_MIXED_FP32, 2e-5)])
def test_full_size_vcycle(workload, prec, rtol):
    oh, h = workload
    n = oh.A[0].shape[0]
    b = np.random.default_rng(12).standard_normal((n, Q + Q_EXTRA))
    x = ae.amgeig_apply_vcycle(h.handle, 0, b, ae.options(precision=prec))
    xo = O.vcycle(oh, 0, b, np.zeros_like(b))
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < rtol
