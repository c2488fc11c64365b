"""Plain FP64 CPU oracle of the AMG multilevel-correction eigensolver's solve phase.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this module.  It shares no
code with the CUDA path: it parses the hierarchy blob itself and uses NumPy /
SciPy library primitives (sparse matrix products, dense Cholesky, LAPACK's
symmetric-definite eigensolver) as single steps.

It computes, in float64 and in the paper's order:

* ``amg``            AMG(k, b, x0, m): m V-cycles for A_k x = b from the initial
                     guess x0 (Algorithm 3.1, Eqs. Linear_Equation and
                     inexact_inverse_iter; one V-cycle by default, Sec. 4.1).
                     Each V-cycle smooths with point l1-Jacobi (one sweep before
                     and one after the coarse correction; the paper uses
                     Gauss-Seidel, this solver fixes l1-Jacobi), restricts with
                     I_k^{k+1} = (I_{k+1}^k)^T, solves the coarsest level exactly
                     with a Cholesky factor of A_n and prolongates with
                     I_{k+1}^k (Sec. 2.3).
* ``correction``     AMGCorrection(n, k, {lambda_j, u_j}) (Algorithm 3.1): the
                     inexact inverse iteration of step 1, the augmented pencil
                     (A_{n,k}, M_{n,k}) on V_n + span(V) of step 2, its q smallest
                     eigenpairs normalised x^T M_{n,k} x = 1 and the recombination
                     u_j = I_n^k x_j(1:d_n) + V x_j(d_n+1:d_n+q).
* ``solve``          the AMG Eigenvalue Solver (Algorithm 3.2): the eigenproblem
                     on level n1 (the coarsest level with at least q+q_extra
                     dofs, n1 = n by default, Sec. 4.1), then for k = n1-1..1
                     the prolongation u_k = I_{k+1}^k u_{k+1} and p_k corrections
                     (p_k = 1 on intermediate levels; on the finest level until the
                     residual test passes or max_corrections, p_1 <= 20, Sec. 4.1).

Levels are 0-based here: level 0 is the paper's finest level 1, level n-1 its
coarsest level n.

Readings of the paper taken here (they are listed with the rest of the design):
* the right-hand side of the AMG call is lambda_j M_k u_j (Eq. Linear_Equation;
  the shorthand AMG(k, lambda u, u, m) drops M);
* I_k^n is the restriction chain R_{n-1}...R_k and I_n^k the prolongation chain;
* the coarsest-level solve inside a V-cycle is exact (Cholesky of A_n);
* the stopping test is the relative residual
  max_j ||A u_j - lambda_j M u_j||_2 / (|lambda_j| ||M u_j||_2) <= tol, because the
  paper's total error e_l needs reference eigenvalues;
* "select the desired eigenpairs" means the q + q_extra smallest Ritz values;
* each output vector is signed so that its largest-magnitude entry (lowest
  index on ties) is positive;
* with ``Options.smoother = "gs"`` the V-cycle smooths with Gauss-Seidel as the
  paper does (Sec. 4.1), made parallel by a multicolour ordering: rows are
  coloured first-fit in row order (the smallest colour no earlier neighbour
  holds) and one sweep visits the colours in ascending order before the coarse
  correction and in descending order after it, so the V-cycle stays symmetric;
* with ``Options.shift = sigma`` the linear solve of step 1 is shifted, one of
  the strategies the remark after Algorithm 3.1 allows: m AMG iterations for
  (A_k - sigma M_k) u~ = (lambda_j - sigma) M_k u_j from u_j, on the hierarchy
  of A_l - sigma M_l (Galerkin-consistent, since both A and M are Galerkin
  products), with its l1-Jacobi diagonals and an exact coarsest solve; sigma
  must lie below the lowest eigenvalue of (A_n, M_n) so that every level's
  operator is positive definite.  sigma = 0 is the paper's unshifted solve;
* with ``Options.krylov = s`` the correction space is V_n plus a block Krylov
  space of step 1's inexact inverse iteration T (the remark after Algorithm 3.1
  names "V_n + Krylov spaces"): V_1 = T U, V_i = T V_{i-1}, all with the Ritz
  values lambda of the current step, and the pencil is taken on
  V_n + span(V_1, ..., V_s) after the block is M-orthonormalised (directions
  whose M-norm falls below 1e-10 of the largest are dropped).  s = 1 is the
  paper's V_n + span(V).
"""
from __future__ import annotations

import dataclasses
import struct
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

MAGIC = b"AMGEIGH1"


# --------------------------------------------------------------------------
# hierarchy


@dataclasses.dataclass
class OracleHierarchy:
    A: List[sp.csr_matrix]
    M: List[sp.csr_matrix]
    P: List[sp.csr_matrix]  # P[l] = I_{l+1}^l, N_l x N_{l+1}
    R: List[sp.csr_matrix]  # R[l] = P[l]^T
    dinv: List[np.ndarray]  # 1 / sum_j |a_ij|  (l1-Jacobi), levels 0..n-2
    An: np.ndarray  # dense coarsest A
    Mn: np.ndarray  # dense coarsest M
    An_chol: tuple  # scipy cho_factor of An
    colour_cache: dict = dataclasses.field(default_factory=dict)  # level -> Gauss-Seidel colours
    shift_cache: dict = dataclasses.field(default_factory=dict)  # sigma -> shifted hierarchy

    @property
    def n_levels(self) -> int:
        return len(self.A)

    @property
    def sizes(self) -> List[int]:
        return [a.shape[0] for a in self.A]


def read_blob(blob: bytes) -> OracleHierarchy:
    """Parse and validate a hierarchy blob (layout documented by its writer)."""
    if len(blob) < 24 or len(blob) % 8 or blob[:8] != MAGIC:
        raise ValueError("not a hierarchy blob")
    words = np.frombuffer(blob[:-8], dtype="<u8")
    (stored,) = struct.unpack("<Q", blob[-8:])
    if int(words.sum(dtype=np.uint64)) != stored:
        raise ValueError("hierarchy blob checksum mismatch")
    version, n = struct.unpack_from("<II", blob, 8)
    if version != 1 or n < 1:
        raise ValueError("unsupported hierarchy blob")
    off = 16
    rows = struct.unpack_from(f"<{n}Q", blob, off)
    off += 8 * n
    nnz = struct.unpack_from(f"<{n}Q", blob, off)
    off += 8 * n
    nnzp = struct.unpack_from(f"<{n - 1}Q", blob, off) if n > 1 else ()
    off += 8 * (n - 1)
    off += (-off) % 8

    def take(count, dt):
        nonlocal off
        itemsize = np.dtype(dt).itemsize
        end = off + count * itemsize
        if end > len(blob) - 8:
            raise ValueError("truncated hierarchy blob")
        arr = np.frombuffer(blob, dtype=dt, count=count, offset=off)
        off = end + ((-end) % 8)
        return arr

    A, M, P = [], [], []
    for l in range(n):
        rp = take(rows[l] + 1, "<i4")
        ci = take(nnz[l], "<i4")
        av = take(nnz[l], "<f8")
        mv = take(nnz[l], "<f8")
        shape = (rows[l], rows[l])
        A.append(sp.csr_matrix((av, ci, rp), shape=shape))
        M.append(sp.csr_matrix((mv, ci, rp), shape=shape))
    for l in range(n - 1):
        rp = take(rows[l] + 1, "<i4")
        ci = take(nnzp[l], "<i4")
        pv = take(nnzp[l], "<f8")
        P.append(sp.csr_matrix((pv, ci, rp), shape=(rows[l], rows[l + 1])))
    if off != len(blob) - 8:
        raise ValueError("trailing bytes in hierarchy blob")
    R = [p.T.tocsr() for p in P]
    dinv = [1.0 / np.asarray(abs(a).sum(axis=1)).ravel() for a in A[:-1]]
    An = A[-1].toarray()
    Mn = M[-1].toarray()
    return OracleHierarchy(A, M, P, R, dinv, An, Mn, sla.cho_factor(An, lower=True))


# --------------------------------------------------------------------------
# AMG linear solver (Algorithm 3.1 step 1)


def shifted(h: OracleHierarchy, sigma: float) -> OracleHierarchy:
    """The hierarchy of the shifted operators A_l - sigma M_l (same pattern, same
    transfers) with their l1-Jacobi diagonals and the Cholesky factor of the
    shifted coarsest matrix.  Raises ValueError when that matrix is not positive
    definite (sigma at or above the lowest eigenvalue of (A_n, M_n))."""
    if sigma in h.shift_cache:
        return h.shift_cache[sigma]
    B = [sp.csr_matrix((a.data - sigma * m.data, a.indices, a.indptr), shape=a.shape) for a, m in zip(h.A, h.M)]
    dinv = [1.0 / np.asarray(abs(b).sum(axis=1)).ravel() for b in B[:-1]]
    Bn = B[-1].toarray()
    try:
        chol = sla.cho_factor(Bn, lower=True)
    except np.linalg.LinAlgError as e:
        raise ValueError("shift not below the lowest coarse eigenvalue") from e
    # same sparsity pattern: the Gauss-Seidel colouring is shared
    hs = OracleHierarchy(B, h.M, h.P, h.R, dinv, Bn, h.Mn, chol, colour_cache=h.colour_cache)
    h.shift_cache[sigma] = hs
    return hs


def jacobi_l1(h: OracleHierarchy, l: int, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """One point l1-Jacobi sweep x <- x + D^-1 (b - A_l x), D = diag(sum_j |a_ij|)."""
    d = h.dinv[l] if x.ndim == 1 else h.dinv[l][:, None]
    return x + d * (b - h.A[l] @ x)


def greedy_colours(A: sp.csr_matrix) -> np.ndarray:
    """First-fit colouring in row order: row i takes the smallest colour that no
    neighbour j < i (a_ij != 0) holds.  Rows of one colour are never adjacent."""
    n = A.shape[0]
    colour = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        taken = set()
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j < i:
                taken.add(int(colour[j]))
        c = 0
        while c in taken:
            c += 1
        colour[i] = c
    return colour


def colours(h: OracleHierarchy, l: int) -> np.ndarray:
    """The colouring of level l, computed once per hierarchy."""
    if l not in h.colour_cache:
        h.colour_cache[l] = greedy_colours(h.A[l])
    return h.colour_cache[l]


def gauss_seidel(h: OracleHierarchy, l: int, b: np.ndarray, x: np.ndarray, descending: bool = False) -> np.ndarray:
    """One multicolour Gauss-Seidel sweep x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii,
    the colours in ascending (or descending) order; rows of one colour at once."""
    A = h.A[l]
    col = colours(h, l)
    diag = A.diagonal()
    x = x.copy()
    order = range(int(col.max()) + 1)
    for c in (reversed(order) if descending else order):
        rows = np.nonzero(col == c)[0]
        d = diag[rows] if x.ndim == 1 else diag[rows][:, None]
        x[rows] = x[rows] + (b[rows] - A[rows] @ x) / d
    return x


def vcycle(h: OracleHierarchy, l: int, b: np.ndarray, x: np.ndarray, pre: int = 1, post: int = 1,
           smoother: str = "jacobi") -> np.ndarray:
    """One V-cycle for A_l x = b from the initial guess x."""
    if l == h.n_levels - 1:
        return sla.cho_solve(h.An_chol, b)
    for _ in range(pre):
        x = gauss_seidel(h, l, b, x) if smoother == "gs" else jacobi_l1(h, l, b, x)
    r = b - h.A[l] @ x
    bc = h.R[l] @ r
    xc = vcycle(h, l + 1, bc, np.zeros_like(bc), pre, post, smoother)
    x = x + h.P[l] @ xc
    for _ in range(post):
        x = gauss_seidel(h, l, b, x, descending=True) if smoother == "gs" else jacobi_l1(h, l, b, x)
    return x


def amg(h: OracleHierarchy, k: int, b: np.ndarray, x0: np.ndarray, m: int = 1, pre: int = 1, post: int = 1,
        smoother: str = "jacobi"):
    """AMG(k, b, x0, m): m V-cycles on level k from the initial guess x0."""
    x = x0
    for _ in range(m):
        x = vcycle(h, k, b, x, pre, post, smoother)
    return x


# --------------------------------------------------------------------------
# transfers between level k and the coarsest level


def restrict_to_coarsest(h: OracleHierarchy, k: int, X: np.ndarray) -> np.ndarray:
    """I_k^n X = R_{n-1} ... R_k X (0-based: R[n-2] ... R[k])."""
    for l in range(k, h.n_levels - 1):
        X = h.R[l] @ X
    return X


def prolong_from_coarsest(h: OracleHierarchy, k: int, Xc: np.ndarray) -> np.ndarray:
    """I_n^k Xc = P_k ... P_{n-1} Xc (0-based: P[k] ... P[n-2])."""
    for l in range(h.n_levels - 2, k - 1, -1):
        Xc = h.P[l] @ Xc
    return Xc


# --------------------------------------------------------------------------
# correction step (Algorithm 3.1)


@dataclasses.dataclass
class Options:
    smoother: str = "jacobi"  # "jacobi" (point l1-Jacobi) or "gs" (multicolour Gauss-Seidel)
    max_corrections: int = 20
    v_cycles: int = 1
    pre_sweeps: int = 1
    post_sweeps: int = 1
    q_extra: int = 0
    fixed_corrections: int = 0  # > 0: run exactly this many finest-level corrections
    # > 0: the pencil's coarse part is spanned by the `coarse_modes` lowest
    # eigenvectors of (A_n, M_n) instead of all of V_n (an option of the GPU
    # library, not of the paper; 0 = the paper's pencil)
    coarse_modes: int = 0
    # sigma of the shifted linear solve in step 1 (0 = the paper's unshifted solve)
    shift: float = 0.0
    # depth s of the block Krylov correction space V_n + span(T U, ..., T^s U) (1 = the paper's)
    krylov: int = 1
    # initial level of Algorithm 3.2 step 1 (0-based); -1: the coarsest level with at least
    # q + q_extra rows (n1 = n whenever the coarsest level is large enough, Sec. 4.1)
    n1: int = -1


def augmented_pencil(h: OracleHierarchy, k: int, V: np.ndarray):
    """(A_{n,k}, M_{n,k}) of Algorithm 3.1 step 2 on V_n + span(V)."""
    AV = h.A[k] @ V
    MV = h.M[k] @ V
    CA = restrict_to_coarsest(h, k, AV)
    CM = restrict_to_coarsest(h, k, MV)
    Ahat = np.block([[h.An, CA], [CA.T, V.T @ AV]])
    Mhat = np.block([[h.Mn, CM], [CM.T, V.T @ MV]])
    return Ahat, Mhat


def smallest_pairs(Ahat: np.ndarray, Mhat: np.ndarray, count: int):
    """The `count` smallest eigenpairs of A x = mu M x with x^T M x = 1 (LAPACK)."""
    mu, X = sla.eigh(Ahat, Mhat, subset_by_index=[0, count - 1])
    return mu, X


def coarse_modes_basis(h: OracleHierarchy, m: int) -> np.ndarray:
    """The m lowest M_n-orthonormal eigenvectors of (A_n, M_n)."""
    _, Z = sla.eigh(h.An, h.Mn, subset_by_index=[0, m - 1])
    return Z


def inverse_iteration_step(h: OracleHierarchy, k: int, lam: np.ndarray, U: np.ndarray, opts: Options = Options()):
    """Step 1 of Algorithm 3.1, T U: m AMG iterations for A_k u~ = lambda_j M_k u_j from
    u_j (or the shifted system when opts.shift != 0)."""
    if opts.shift != 0.0:
        # (A_k - sigma M_k) u~ = (lambda_j - sigma) M_k u_j, on the shifted hierarchy
        hs = shifted(h, opts.shift)
        b = h.M[k] @ U * (lam - opts.shift)[None, :]
        return amg(hs, k, b, U, opts.v_cycles, opts.pre_sweeps, opts.post_sweeps, opts.smoother)
    b = h.M[k] @ U * lam[None, :]  # lambda_j M_k u_j
    return amg(h, k, b, U, opts.v_cycles, opts.pre_sweeps, opts.post_sweeps, opts.smoother)


def krylov_block(h: OracleHierarchy, k: int, lam: np.ndarray, U: np.ndarray, opts: Options = Options()):
    """[T U, T^2 U, ..., T^s U] M-orthonormalised (s = opts.krylov >= 2): eigenvectors
    of the block's M-Gram matrix scaled by 1/sqrt(eigenvalue), directions with an
    eigenvalue below 1e-20 of the largest (M-norm below 1e-10) dropped; done twice,
    since the consecutive blocks are nearly parallel and one pass leaves an error of
    the Gram matrix's condition number times the rounding unit."""
    blocks = [inverse_iteration_step(h, k, lam, U, opts)]
    for _ in range(opts.krylov - 1):
        blocks.append(inverse_iteration_step(h, k, lam, blocks[-1], opts))
    K = np.hstack(blocks)
    for _ in range(2):
        g, Q = np.linalg.eigh(K.T @ (h.M[k] @ K))
        keep = g > 1e-20 * g.max()
        K = K @ (Q[:, keep] / np.sqrt(g[keep])[None, :])
    return K


def correction(h: OracleHierarchy, k: int, lam: np.ndarray, U: np.ndarray, opts: Options = Options()):
    """One AMGCorrection(n, k, {lambda_j, u_j}) step; returns (lambda, U)."""
    qt = U.shape[1]
    V = inverse_iteration_step(h, k, lam, U, opts) if opts.krylov <= 1 else krylov_block(h, k, lam, U, opts)
    Ahat, Mhat = augmented_pencil(h, k, V)
    dn = h.sizes[-1]
    if 0 < opts.coarse_modes < dn:
        # restrict the coarse block to span(Z_m): the pencil of B = [I_n^k Z_m, V]
        m = opts.coarse_modes
        w = V.shape[1]
        T = np.zeros((m + w, dn + w))
        T[:m, :dn] = coarse_modes_basis(h, m).T
        T[m:, dn:] = np.eye(w)
        mu, X = smallest_pairs(T @ Ahat @ T.T, T @ Mhat @ T.T, qt)
        X = T.T @ X
    else:
        mu, X = smallest_pairs(Ahat, Mhat, qt)
    U_new = prolong_from_coarsest(h, k, X[:dn]) + V @ X[dn:]
    return mu, U_new


# --------------------------------------------------------------------------
# solver (Algorithm 3.2)


def relres(h: OracleHierarchy, lam: np.ndarray, U: np.ndarray, k: int = 0) -> np.ndarray:
    """||A u_j - lambda_j M u_j||_2 / (|lambda_j| ||M u_j||_2) per column."""
    AU = h.A[k] @ U
    MU = h.M[k] @ U
    return np.linalg.norm(AU - MU * lam[None, :], axis=0) / (np.abs(lam) * np.linalg.norm(MU, axis=0))


def initial_level(h: OracleHierarchy, qt: int) -> int:
    """n1: the coarsest level with at least qt dofs (Algorithm 3.2 step 1 allows any
    n1 <= n; the paper takes n1 = n, Sec. 4.1, which needs d_n >= qt)."""
    for l in range(h.n_levels - 1, -1, -1):
        if h.sizes[l] >= qt:
            return l
    raise ValueError("q + q_extra exceeds the finest dimension")


def sign_normalise(U: np.ndarray) -> np.ndarray:
    idx = np.argmax(np.abs(U), axis=0)
    s = np.sign(U[idx, np.arange(U.shape[1])])
    s[s == 0] = 1.0
    return U * s[None, :]


@dataclasses.dataclass
class Info:
    corrections: int  # finest-level corrections performed
    converged: bool
    relres: np.ndarray  # final relative residuals (q columns)
    history: list  # eigenvalue estimates after each finest-level correction
    n1: int


def solve(h: OracleHierarchy, q: int, tol: float = 1e-10, opts: Options = Options()):
    """Algorithm 3.2.  Returns (lambda[q] ascending, U[N_0, q], Info)."""
    qt = q + opts.q_extra
    n1 = initial_level(h, qt) if opts.n1 < 0 else opts.n1
    if not 0 <= n1 < h.n_levels or h.sizes[n1] < qt:
        raise ValueError("n1 must be a level with at least q + q_extra rows")
    An1 = h.A[n1].toarray()
    Mn1 = h.M[n1].toarray()
    lam, U = smallest_pairs(An1, Mn1, qt)
    for k in range(n1 - 1, 0, -1):
        U = h.P[k] @ U
        lam, U = correction(h, k, lam, U, opts)
    history = []
    done = 0
    converged = False
    if n1 > 0:
        U = h.P[0] @ U
        while True:
            rr = relres(h, lam, U)[:q]
            if opts.fixed_corrections > 0:
                if done == opts.fixed_corrections:
                    converged = bool(np.max(rr) <= tol)
                    break
            else:
                if np.max(rr) <= tol:
                    converged = True
                    break
                if done == opts.max_corrections:
                    break
            lam, U = correction(h, 0, lam, U, opts)
            done += 1
            history.append(lam[:q].copy())
    rr = relres(h, lam, U)[:q]
    if n1 == 0:
        converged = bool(np.max(rr) <= tol)
    return lam[:q].copy(), sign_normalise(U[:, :q]), Info(done, converged, rr, history, n1)
