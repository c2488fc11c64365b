"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the dense
generalized eigensolution (the plain definition of the fixed point), closed-form
continuum eigenvalues, linear-algebra identities of the V-cycle and of the
Rayleigh-Ritz step (Sec. 3: the pencil is the Galerkin projection on
V_n + span(V)), and invariants of the output.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl

from oracle import amg_oracle as O
from paper_1503_08462_gb300.inputs import hierarchy, meshes

from helpers import dense_pairs, eig_rel_tol, lam_max, m_subspace_angle, problem_and_blob


def _oh(kind="square", size=32, cap=50, seed=1):
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    return p, O.read_blob(blob)


# ---------------------------------------------------------------- V-cycle


def _vcycle_matrix(oh, l=0):
    n = oh.sizes[l]
    return np.stack([O.vcycle(oh, l, e, np.zeros(n)) for e in np.eye(n)], axis=1)


def test_vcycle_is_symmetric_and_contracting():
    """V(1,1) with the same symmetric smoother before and after and R = P^T is
    a symmetric operator B, and the error propagation I - BA contracts in the
    A-norm.  A transposed transfer, a missing sweep or a sign error breaks one
    of these."""
    p, oh = _oh("square", 16, 20)
    B = _vcycle_matrix(oh)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    A = oh.A[0].toarray()
    L = np.linalg.cholesky(A)
    E = np.eye(A.shape[0]) - B @ A
    rho = np.linalg.norm(L.T @ E @ np.linalg.inv(L.T), 2)  # A-norm of I - BA
    assert rho < 0.7, rho


def test_vcycle_two_level_dense():
    """A two-level cycle equals the dense formula S (I - P A_c^-1 P^T A) S' ..."""
    p = meshes.square_2d(8)
    h = hierarchy.build_for_problem(p, coarse_cap=25, max_levels=2)
    oh = O.read_blob(hierarchy.to_blob(h))
    assert oh.n_levels == 2
    A = oh.A[0].toarray()
    P = oh.P[0].toarray()
    D = np.diag(np.abs(A).sum(axis=1))
    Ac_inv = np.linalg.inv(P.T @ A @ P)
    rng = np.random.default_rng(7)
    b = rng.standard_normal(A.shape[0])
    x0 = rng.standard_normal(A.shape[0])
    x1 = x0 + np.linalg.solve(D, b - A @ x0)
    x2 = x1 + P @ Ac_inv @ P.T @ (b - A @ x1)
    x3 = x2 + np.linalg.solve(D, b - A @ x2)
    got = O.amg(oh, 0, b, x0, 1)
    assert np.allclose(got, x3, rtol=1e-12, atol=1e-12 * np.abs(x3).max())


def test_amg_iteration_solves_linear_system():
    p, oh = _oh("lshape", 16, 60)
    A = oh.A[0]
    rng = np.random.default_rng(3)
    b = rng.standard_normal((A.shape[0], 2))
    x = np.zeros_like(b)
    xs = np.column_stack([spl.spsolve(A.tocsc(), b[:, j]) for j in range(2)])
    x = O.amg(oh, 0, b, x, 60)
    assert np.abs(x - xs).max() <= 1e-10 * np.abs(xs).max()


def test_l1_jacobi_reduces_energy_error():
    """The l1 diagonal dominates A (2D - A is SPD), so each sweep is an A-norm contraction."""
    p, oh = _oh("checker", 16, 30, seed=3)
    A = oh.A[0]
    rng = np.random.default_rng(1)
    e = rng.standard_normal(A.shape[0])
    for _ in range(5):
        e_new = O.jacobi_l1(oh, 0, np.zeros_like(e), e)
        assert e_new @ (A @ e_new) < e @ (A @ e)
        e = e_new


# ---------------------------------------------------------------- Rayleigh-Ritz


def _chain_dense(oh, k):
    """I_n^k as a dense matrix (product of the prolongations)."""
    Pc = np.eye(oh.sizes[-1])
    for l in range(oh.n_levels - 2, k - 1, -1):
        Pc = oh.P[l] @ Pc
    return np.asarray(Pc)


@pytest.mark.parametrize("k", [0, 1])
def test_pencil_is_galerkin_projection(k):
    """(A_{n,k}, M_{n,k}) equals B^T (A_k, M_k) B with B = [I_n^k, V]."""
    p, oh = _oh("square", 16, 20)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((oh.sizes[k], 3))
    Ahat, Mhat = O.augmented_pencil(oh, k, V)
    Bm = np.hstack([_chain_dense(oh, k), V])
    for hat, mat in ((Ahat, oh.A[k]), (Mhat, oh.M[k])):
        ref = Bm.T @ (mat @ Bm)
        assert np.abs(hat - ref).max() <= 1e-12 * np.abs(ref).max()


def test_exact_eigenpairs_are_a_fixed_point():
    p, oh = _oh("square", 32, 50)
    lam, U = dense_pairs(p, 6)
    mu, U1 = O.correction(oh, 0, lam, U)
    assert np.allclose(mu, lam, rtol=1e-11)
    assert m_subspace_angle(U1[:, :4], U[:, :4], oh.M[0]) < 1e-8


def test_rayleigh_ritz_is_basis_invariant():
    """Replacing V by V Q (Q invertible) leaves the Ritz pairs unchanged."""
    p, oh = _oh("square", 16, 20)
    rng = np.random.default_rng(11)
    V = rng.standard_normal((oh.sizes[0], 4))
    Q = rng.standard_normal((4, 4)) + 4 * np.eye(4)
    res = []
    for W in (V, V @ Q):
        Ahat, Mhat = O.augmented_pencil(oh, 0, W)
        mu, X = O.smallest_pairs(Ahat, Mhat, 4)
        dn = oh.sizes[-1]
        res.append((mu, O.prolong_from_coarsest(oh, 0, X[:dn]) + W @ X[dn:]))
    assert np.allclose(res[0][0], res[1][0], rtol=1e-12)
    assert m_subspace_angle(res[0][1], res[1][1], oh.M[0]) < 1e-10


# ---------------------------------------------------------------- full solver


# tol: the relative-residual floor of FP64 grows with the coefficient contrast
# (rounding in A u is ~1e-16 ||A|| ||u||); the 10^(+-3) checkerboard sits near 1e-10.
@pytest.mark.parametrize("kind,size,cap,seed,q,qe,tol", [("square", 32, 50, 1, 4, 2, 1e-10),
                                                       ("lshape", 16, 60, 2, 6, 2, 1e-10),
                                                       ("checker", 32, 60, 3, 5, 2, 2e-9),
                                                       ("cube", 8, 40, 4, 4, 2, 1e-10)])
def test_converged_solve_matches_dense_definition(kind, size, cap, seed, q, qe, tol):
    """Pin 1: the converged iteration reproduces the q smallest dense eigenpairs."""
    p, oh = _oh(kind, size, cap, seed)
    lam, U, info = O.solve(oh, q, tol=tol, opts=O.Options(q_extra=qe, max_corrections=100))
    assert info.converged, info.relres
    lam_ex, U_ex = dense_pairs(p, q)
    assert np.all(np.abs(lam - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    # compare invariant subspaces (clusters handled by comparing spans)
    assert m_subspace_angle(U, U_ex, oh.M[0]) < 1e-8
    # invariants: U^T M U = I, residual, sign convention
    G = U.T @ (oh.M[0] @ U)
    assert np.abs(G - np.eye(q)).max() < 1e-11
    assert np.all(info.relres <= tol)
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(q)] > 0)


def test_ritz_values_are_upper_bounds_and_converge():
    """Every Ritz value bounds the exact eigenvalue from above (Courant-Fischer)
    and the total error e_l falls geometrically (Sec. 4.1 ratio)."""
    p, oh = _oh("square", 32, 50)
    q = 4
    lam_ex, _ = dense_pairs(p, q)
    _, _, info = O.solve(oh, q, tol=0.0, opts=O.Options(q_extra=2, fixed_corrections=8))
    errs = []
    for est in info.history:
        assert np.all(est >= lam_ex * (1 - 1e-12))
        errs.append(np.sum(est - lam_ex))
    ratio = (errs[-1] / errs[0]) ** (1.0 / (len(errs) - 1))
    assert ratio < 0.35, ratio


def test_single_level_hierarchy_is_dense_solve():
    p = meshes.square_2d(8)
    oh = O.read_blob(hierarchy.to_blob(hierarchy.build_for_problem(p, coarse_cap=1000)))
    lam, U, info = O.solve(oh, 3)
    lam_ex, U_ex = dense_pairs(p, 3)
    assert np.allclose(lam, lam_ex, rtol=1e-13)
    assert info.corrections == 0 and info.n1 == 0


def test_initial_level_above_the_coarsest():
    """Algorithm 3.2 step 1 with n1 < n: when q + q_extra exceeds the coarsest dimension the oracle
    starts on the coarsest level that holds that many pairs, and its initial pairs there are the dense
    eigenpairs of (A_n1, M_n1); with n1 = 0 the solve is the finest level's dense eigensolution (no
    correction runs); and the converged solve from an intermediate n1 equals the finest level's dense
    eigenpairs (the fixed point)."""
    p, oh = _oh("square", 32, 20, 1)  # coarsest level below 20 rows
    dn = oh.sizes[-1]
    q, qe = dn + 2, 3
    qt = q + qe
    n1 = O.initial_level(oh, qt)
    assert n1 < oh.n_levels - 1 and oh.sizes[n1] >= qt and oh.sizes[n1 + 1] < qt
    # initial pairs on level n1: exact for the level's own pencil (one Rayleigh quotient per pair)
    lam1, U1 = O.smallest_pairs(oh.A[n1].toarray(), oh.M[n1].toarray(), qt)
    A1, M1 = oh.A[n1], oh.M[n1]
    assert np.abs(U1.T @ (M1 @ U1) - np.eye(qt)).max() < 1e-12
    assert np.abs(A1 @ U1 - (M1 @ U1) * lam1).max() < 1e-10 * lam1.max()
    # n1 = 0 is the dense finest-level solve
    lam0, U0, info0 = O.solve(oh, 4, opts=O.Options(n1=0))
    lam_ex, U_ex = dense_pairs(p, 4)
    assert info0.n1 == 0 and info0.corrections == 0
    assert np.allclose(lam0, lam_ex, rtol=1e-12)
    # the default n1 for q + q_extra > d_n, converged: the dense eigenpairs
    lam, U, info = O.solve(oh, q, tol=1e-10, opts=O.Options(q_extra=qe, max_corrections=150))
    assert info.n1 == n1 and info.converged
    lam_ex, U_ex = dense_pairs(p, q)
    assert np.all(np.abs(lam - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(q)).max() < 1e-11
    # an explicit n1 that cannot hold q + q_extra pairs is refused
    with pytest.raises(ValueError):
        O.solve(oh, q, opts=O.Options(q_extra=qe, n1=oh.n_levels - 1))


def test_closed_form_unit_square():
    """The converged solver approaches pi^2 (2, 5, 5, 8) at O(h^2) (Example 1)."""
    exact = np.pi ** 2 * np.array([2.0, 5.0, 5.0, 8.0])
    errs = []
    for m in (8, 16, 32):
        p = meshes.square_2d(m, seed=1)
        oh = O.read_blob(hierarchy.to_blob(hierarchy.build_for_problem(p, coarse_cap=20)))
        lam, _, info = O.solve(oh, 4, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=60))
        assert info.converged
        errs.append(np.mean(np.abs(lam - exact) / exact))
    slope = np.polyfit(np.log([1 / 8, 1 / 16, 1 / 32]), np.log(errs), 1)[0]
    assert 1.7 < slope < 2.4, slope


def test_coarse_modes_option():
    """The library's coarse_modes option: m = d_n is the paper's pencil exactly, and a
    truncated coarse space still converges to the dense eigenpairs."""
    p, oh = _oh("lshape", 16, 60, 2)
    dn = oh.sizes[-1]
    full = O.solve(oh, 6, tol=0.0, opts=O.Options(q_extra=2, fixed_corrections=3))
    same = O.solve(oh, 6, tol=0.0, opts=O.Options(q_extra=2, fixed_corrections=3, coarse_modes=dn))
    assert np.allclose(full[0], same[0], rtol=1e-13)
    lam, U, info = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100, coarse_modes=16))
    assert info.converged
    lam_ex, U_ex = dense_pairs(p, 6)
    assert np.all(np.abs(lam - lam_ex) <= 1e-10 * lam_ex)
    assert m_subspace_angle(U, U_ex, oh.M[0]) < 1e-8


# ---------------------------------------------------------------- multicolour Gauss-Seidel


def test_greedy_colours_are_a_proper_colouring():
    """No two adjacent rows share a colour, and first-fit never needs more than
    max-degree + 1 colours."""
    for kind, size in (("square", 16), ("lshape", 8), ("cube", 6)):
        p, oh = _oh(kind, size, 20)
        A = oh.A[0]
        col = O.greedy_colours(A)
        rows, cols = A.nonzero()
        off = rows != cols
        assert np.all(col[rows[off]] != col[cols[off]])
        deg = np.diff(A.indptr) - 1
        assert col.max() + 1 <= deg.max() + 1


def test_multicolour_gs_is_gauss_seidel_in_colour_order():
    """A multicolour sweep is the textbook sequential Gauss-Seidel sweep over the rows
    taken colour by colour (row order inside a colour), written here as a plain loop;
    the descending sweep is the same over the reversed colour order."""
    p, oh = _oh("lshape", 8, 20, seed=2)
    A = oh.A[0].toarray()
    n = A.shape[0]
    col = O.greedy_colours(oh.A[0])
    rng = np.random.default_rng(3)
    b, x0 = rng.standard_normal(n), rng.standard_normal(n)
    for descending in (False, True):
        cs = sorted(set(col.tolist()), reverse=descending)
        order = [i for c in cs for i in range(n) if col[i] == c]
        x = x0.copy()
        for i in order:
            x[i] = (b[i] - A[i] @ x + A[i, i] * x[i]) / A[i, i]
        np.testing.assert_allclose(O.gauss_seidel(oh, 0, b, x0, descending), x, rtol=1e-12, atol=1e-12)


def test_gs_reduces_energy_error_and_vcycle_is_symmetric():
    """Gauss-Seidel is an A-norm contraction for SPD A; with ascending colours before and
    descending after the coarse correction the V-cycle operator is symmetric and its
    error propagation contracts (faster than with l1-Jacobi)."""
    p, oh = _oh("checker", 16, 30, seed=3)
    A = oh.A[0]
    e = np.random.default_rng(1).standard_normal(A.shape[0])
    for _ in range(5):
        e_new = O.gauss_seidel(oh, 0, np.zeros_like(e), e)
        assert e_new @ (A @ e_new) < e @ (A @ e)
        e = e_new
    p, oh = _oh("square", 16, 20)
    n = oh.sizes[0]
    B = np.stack([O.vcycle(oh, 0, ei, np.zeros(n), smoother="gs") for ei in np.eye(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    Ad = oh.A[0].toarray()
    L = np.linalg.cholesky(Ad)
    rho = np.linalg.norm(L.T @ (np.eye(n) - B @ Ad) @ np.linalg.inv(L.T), 2)
    Bj = _vcycle_matrix(oh)
    rho_j = np.linalg.norm(L.T @ (np.eye(n) - Bj @ Ad) @ np.linalg.inv(L.T), 2)
    assert rho < rho_j < 0.7, (rho, rho_j)


def test_gs_solve_matches_dense_definition():
    """Pin 1 with the Gauss-Seidel smoother: the same fixed point, reached in fewer corrections."""
    p, oh = _oh("lshape", 16, 60, 2)
    lam_ex, _ = dense_pairs(p, 6)
    lam, U, info = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100, smoother="gs"))
    assert info.converged
    assert np.all(np.abs(lam - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    _, _, info_j = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100))
    assert info.corrections < info_j.corrections


# ---------------------------------------------------------------- shifted inner solve


def test_shifted_two_level_dense():
    """The shifted solve's two-level cycle equals the dense formula for B = A - sigma M:
    l1-Jacobi with D = diag(sum_j |b_ij|), the exact coarse correction with P^T B P, and
    the same sweep after it.  A wrong sign of the shift, the unshifted diagonal or an
    unshifted coarse matrix breaks the equality."""
    p = meshes.square_2d(8)
    h = hierarchy.build_for_problem(p, coarse_cap=25, max_levels=2)
    oh = O.read_blob(hierarchy.to_blob(h))
    assert oh.n_levels == 2
    lam1 = sla.eigh(oh.A[0].toarray(), oh.M[0].toarray(), eigvals_only=True)[0]
    sigma = 0.7 * lam1
    B = oh.A[0].toarray() - sigma * oh.M[0].toarray()
    P = oh.P[0].toarray()
    D = np.diag(np.abs(B).sum(axis=1))
    Bc_inv = np.linalg.inv(P.T @ B @ P)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(B.shape[0])
    x0 = rng.standard_normal(B.shape[0])
    x1 = x0 + np.linalg.solve(D, b - B @ x0)
    x2 = x1 + P @ Bc_inv @ P.T @ (b - B @ x1)
    x3 = x2 + np.linalg.solve(D, b - B @ x2)
    got = O.amg(O.shifted(oh, sigma), 0, b, x0, 1)
    assert np.allclose(got, x3, rtol=1e-11, atol=1e-11 * np.abs(x3).max())


def test_shifted_vcycle_is_symmetric_and_contracting():
    """For sigma below the lowest eigenvalue, B = A - sigma M is SPD on every level and the
    shifted V-cycle is a symmetric operator whose error propagation contracts in the
    B-norm; a shift at or above the coarsest level's lowest eigenvalue is refused."""
    p, oh = _oh("square", 16, 20)
    lam1 = sla.eigh(oh.A[0].toarray(), oh.M[0].toarray(), eigvals_only=True)[0]
    hs = O.shifted(oh, 0.9 * lam1)
    n = oh.sizes[0]
    C = np.stack([O.vcycle(hs, 0, e, np.zeros(n)) for e in np.eye(n)], axis=1)
    assert np.abs(C - C.T).max() <= 1e-12 * np.abs(C).max()
    B = hs.A[0].toarray()
    L = np.linalg.cholesky(B)
    rho = np.linalg.norm(L.T @ (np.eye(n) - C @ B) @ np.linalg.inv(L.T), 2)
    assert rho < 1.0, rho
    lam1_coarse = sla.eigh(oh.An, oh.Mn, eigvals_only=True)[0]
    with pytest.raises(ValueError):
        O.shifted(oh, 1.01 * lam1_coarse)


def test_shifted_solve_matches_dense_definition():
    """Pin 1 with the shifted inner solve: exact eigenpairs stay a fixed point of the
    shifted correction and the converged iteration reproduces the dense eigenpairs;
    shifted inverse iteration needs no more corrections than the unshifted one."""
    p, oh = _oh("lshape", 16, 60, 2)
    lam_ex, U_ex = dense_pairs(p, 6)
    sigma = 0.8 * lam_ex[0]
    mu, U1 = O.correction(oh, 0, lam_ex, U_ex, O.Options(shift=sigma))
    assert np.allclose(mu, lam_ex, rtol=1e-11)
    assert m_subspace_angle(U1[:, :4], U_ex[:, :4], oh.M[0]) < 1e-8
    opts = O.Options(q_extra=2, max_corrections=100, shift=sigma)
    lam, U, info = O.solve(oh, 6, tol=1e-10, opts=opts)
    assert info.converged
    assert np.all(np.abs(lam - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    assert m_subspace_angle(U, U_ex, oh.M[0]) < 1e-8
    _, _, info0 = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100))
    assert info.corrections <= info0.corrections


# ---------------------------------------------------------------- Krylov-augmented correction space


def test_krylov_block_is_m_orthonormal_and_ritz_values_fall():
    """The depth-2 block [T U, T^2 U] comes out M-orthonormal, and since its span holds
    the paper's span(T U), the depth-2 Ritz values of one correction lie at or below
    the depth-1 ones (Courant-Fischer) and at or above the exact eigenvalues."""
    p, oh = _oh("lshape", 16, 60, 2)
    lam_ex, U_ex = dense_pairs(p, 8)
    rng = np.random.default_rng(4)
    U = U_ex + 1e-2 * rng.standard_normal(U_ex.shape)
    lam = np.array([(u @ (oh.A[0] @ u)) / (u @ (oh.M[0] @ u)) for u in U.T])
    K = O.krylov_block(oh, 0, lam, U, O.Options(krylov=2))
    assert K.shape[1] == 16
    assert np.abs(K.T @ (oh.M[0] @ K) - np.eye(K.shape[1])).max() < 1e-12
    mu1, _ = O.correction(oh, 0, lam, U, O.Options())
    mu2, _ = O.correction(oh, 0, lam, U, O.Options(krylov=2))
    assert np.all(mu2 <= mu1 * (1 + 1e-12))
    assert np.all(mu2 >= lam_ex * (1 - 1e-12))
    assert np.sum(mu2 - lam_ex) < 0.5 * np.sum(mu1 - lam_ex)


def test_krylov_solve_matches_dense_definition():
    """Pin 1 with the Krylov-augmented space: the same fixed point, in fewer corrections."""
    p, oh = _oh("lshape", 16, 60, 2)
    lam_ex, U_ex = dense_pairs(p, 6)
    lam, U, info = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100, krylov=2))
    assert info.converged
    assert np.all(np.abs(lam - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    assert m_subspace_angle(U, U_ex, oh.M[0]) < 1e-8
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(6)).max() < 1e-11
    _, _, info1 = O.solve(oh, 6, tol=1e-10, opts=O.Options(q_extra=2, max_corrections=100))
    assert info.corrections < info1.corrections
    # with the truncated coarse space of the library option the pencil border is the whole
    # depth-2 block; the fixed point is the same
    lam_t, U_t, info_t = O.solve(oh, 6, tol=1e-10,
                                 opts=O.Options(q_extra=2, max_corrections=100, krylov=2, coarse_modes=16))
    assert info_t.converged
    assert np.all(np.abs(lam_t - lam_ex) <= eig_rel_tol(lam_ex, lam_max(p)) * lam_ex)
    assert m_subspace_angle(U_t, U_ex, oh.M[0]) < 1e-8


# ---------------------------------------------------------------- output conventions


def test_relres_and_sign_convention():
    """relres is zero on exact eigenpairs, invariant to scaling a column and grows with a
    perturbation; sign_normalise makes each column's largest-magnitude entry positive,
    the lowest index winning a tie (reading of the paper's unsigned eigenvectors)."""
    p, oh = _oh("square", 16, 20)
    lam, U = dense_pairs(p, 3)
    assert np.all(O.relres(oh, lam, U) < 1e-12)
    np.testing.assert_allclose(O.relres(oh, lam, -3.0 * U), O.relres(oh, lam, U), atol=1e-15)
    assert np.all(O.relres(oh, lam * (1 + 1e-6), U) > 1e-7)
    X = np.array([[1.0, -2.0, 0.0], [-2.0, 2.0, 0.0], [0.5, 1.0, 0.0]])
    Y = O.sign_normalise(X)
    np.testing.assert_array_equal(Y[:, 0], [-1.0, 2.0, -0.5])  # largest |.| at row 1, was negative
    np.testing.assert_array_equal(Y[:, 1], [2.0, -2.0, -1.0])  # tie between rows 0 and 1: row 0 decides
    np.testing.assert_array_equal(Y[:, 2], [0.0, 0.0, 0.0])
