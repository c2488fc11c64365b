"""Shared test utilities: problem fixtures and subspace comparisons."""
import functools

import numpy as np
import scipy.linalg as sla

from paper_1503_08462_gb300.inputs import hierarchy, meshes


@functools.lru_cache(maxsize=None)
def problem_and_blob(kind: str, size: int, cap: int, seed: int = 1):
    if kind == "square":
        p = meshes.square_2d(size, seed=seed)
    elif kind == "checker":
        p = meshes.square_2d(size, checker=4, seed=seed)
    elif kind == "lshape":
        p = meshes.lshape_2d(size, seed=seed)
    elif kind == "cube":
        p = meshes.cube_3d(size, seed=seed)
    else:
        raise ValueError(kind)
    blob, h = hierarchy.problem_blob(p, coarse_cap=cap)
    return p, blob, h


def m_subspace_angle(U, W, M):
    """Largest principal angle between span(U) and span(W) in the M inner product."""
    Lu = sla.cholesky(U.T @ (M @ U), lower=True)
    Lw = sla.cholesky(W.T @ (M @ W), lower=True)
    Qu = sla.solve_triangular(Lu, U.T, lower=True).T
    Qw = sla.solve_triangular(Lw, W.T, lower=True).T
    # sine of the largest angle: M-norm of the part of span(W) outside span(U)
    D = Qw - Qu @ (Qu.T @ (M @ Qw))
    g = D.T @ (M @ D)
    smax = float(np.sqrt(max(0.0, np.linalg.eigvalsh(0.5 * (g + g.T)).max())))
    return float(np.arcsin(min(1.0, smax)))


def dense_pairs(p, q):
    A, M = p.scipy()
    return sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, q - 1])


U64 = np.finfo(np.float64).eps / 2  # unit roundoff of float64


def lam_max(p):
    A, M = p.scipy()
    n = p.n
    return float(sla.eigh(A.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[n - 1, n - 1])[0])


def eig_rel_tol(lam, lmax, base=1e-10, c=2.0):
    """Relative eigenvalue tolerance: `base`, widened to the FP64 floor c*u*lambda_max/lambda_j.

    A backward-stable FP64 solve perturbs eigenvalues by about u * lambda_max
    (absolute); for a pencil with a wide spectrum (coefficient jumps) that
    exceeds base * lambda_j for the smallest eigenvalues."""
    return np.maximum(base, c * U64 * lmax / np.abs(lam))
