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

from helpers import m_subspace_angle

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
    """One V-cycle from level 0 in the launch shapes the timed solve uses (28 columns: 4 lanes per
    row and 2 float4 groups per lane on the finest level, 8 lanes per row below 155,648 rows),
    element by element against the oracle: every entry within rtol of its column's largest entry
    (float32: a few units of 2^-24 per level, accumulated over 9 levels)."""
    oh, h = workload
    n = oh.A[0].shape[0]
    b = np.random.default_rng(12).standard_normal((n, Q + Q_EXTRA))
    x = ae.amgeig_apply_vcycle(h.handle, 0, b, ae.options(precision=prec))
    xo = O.vcycle(oh, 0, b, np.zeros_like(b))
    err = np.abs(x - xo).max(axis=0) / np.abs(xo).max(axis=0)
    assert np.all(err <= rtol), err.max()


def test_full_size_bench_settings_one_correction_matches_oracle(workload):
    """The timed solve's settings (mixed path, two V-cycles per correction, 64 coarse modes, 8 buffer
    vectors) against the oracle run with the same settings for exactly one finest-level correction
    (after the nested phase on every level).  The float32 V-cycle perturbs each correction by
    delta <= 2e-5 of its column (the V-cycle test above); that moves the corrected subspace by an
    angle of order delta and each Ritz value, stationary at eigenvectors, by about 2 delta times the
    pair's relative residual (below 1e-2 after the nested phase): the bounds are 1e-4 on the
    subspace angle and 1e-6 relative on the eigenvalues.  The float64 path meets the float64 parity
    bounds (1e-10, 1e-8)."""
    oh, h = workload
    kw = dict(q_extra=Q_EXTRA, fixed_corrections=1, coarse_modes=64, v_cycles=2)
    lam_o, U_o, info_o = O.solve(oh, Q, tol=0.0, opts=O.Options(**kw))
    for prec, ltol, atol in ((ae.AMGEIG_FP64, 1e-10, 1e-8), (ae.AMGEIG_MIXED_FP32, 1e-6, 1e-4)):
        lam, U, info, _ = h.solve(Q, tol=0.0, opt=ae.options(precision=prec, **kw))
        assert info.corrections == 1
        rel = np.max(np.abs(lam - lam_o) / lam_o)
        ang = m_subspace_angle(U, U_o, oh.M[0])
        assert rel <= ltol and ang <= atol, (prec, rel, ang, info_o.relres.max())
