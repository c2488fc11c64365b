"""GPU path vs the CPU oracle, through the C ABI (needs a GB300 and libamgeig.so)."""
import numpy as np
import pytest

from oracle import amg_oracle as O
from paper_1503_08462_gb300 import amgeig as ae

from helpers import dense_pairs, eig_rel_tol, lam_max, m_subspace_angle, problem_and_blob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


# ------------------------------------------------------------------ dense eigensolver


def _rand_sym(n, spectrum, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * spectrum) @ Q.T


@pytest.mark.parametrize("n,nwant,kind", [(1, 1, "plain"), (2, 2, "plain"), (7, 3, "plain"), (50, 10, "plain"),
                                          (131, 22, "plain"), (131, 22, "cluster"), (260, 60, "graded"),
                                          (64, 64, "plain"), (184, 72, "graded"), (300, 80, "group"),
                                          (257, 41, "group"), (1900, 20, "plain")])
def test_sym_eigh_matches_lapack(n, nwant, kind):
    """Against LAPACK.  "group": the 80 wanted eigenvalues lie within 1e-4 ||H|| of each other, one
    clean-up group too wide for shared memory (its vectors and factors use the global workspace), and 41 of
    them: an odd width, one player idle in every Jacobi round;
    (184, 72): the pencil size of the checkerboard workload; n = 1900: the back-transformation stages
    fewer reflectors per barrier than at small n."""
    rng = np.random.default_rng(n + nwant)
    if kind == "plain":
        spec = np.sort(rng.uniform(0.5, 100.0, n))
    elif kind == "cluster":
        spec = np.sort(np.concatenate([[3.0, 3.0 + 1e-9, 3.0 + 2e-9, 7.0, 7.0], rng.uniform(1.0, 50.0, n - 5)]))
    elif kind == "group":
        spec = np.sort(np.concatenate([rng.uniform(1.0, 1.5, nwant), rng.uniform(10.0, 1e4, n - nwant)]))
    else:
        spec = np.sort(10.0 ** rng.uniform(-2, 4, n))
    H = _rand_sym(n, spec, n)
    H = 0.5 * (H + H.T)
    w, V = ae.amgeig_sym_eigh(H, nwant)
    ref = np.linalg.eigvalsh(H)[:nwant]
    scale = np.abs(ref).max() if kind not in ("graded", "group") else np.abs(spec).max()
    assert np.all(np.abs(w - ref) <= 1e-12 * scale), np.abs(w - ref).max() / scale
    assert np.abs(V.T @ V - np.eye(nwant)).max() < 1e-12
    R = H @ V - V * w
    assert np.abs(R).max() <= 1e-11 * scale


# ------------------------------------------------------------------ V-cycle


@pytest.mark.parametrize("kind,size,cap,width", [("square", 32, 50, 4), ("lshape", 16, 60, 7), ("checker", 32, 40, 33)])
def test_vcycle_matches_oracle(kind, size, cap, width):
    p, blob, _ = problem_and_blob(kind, size, cap, 1 if kind != "checker" else 3)
    oh = O.read_blob(blob)
    rng = np.random.default_rng(width)
    with ae.Hierarchy(blob) as h:
        for level in range(oh.n_levels):
            b = rng.standard_normal((oh.sizes[level], width))
            ref = O.vcycle(oh, level, b, np.zeros_like(b))
            x64 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=ae.AMGEIG_FP64))
            assert np.abs(x64 - ref).max() <= 1e-11 * np.abs(ref).max()
            x32 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=ae.AMGEIG_MIXED_FP32))
            assert np.abs(x32 - ref).max() <= 2e-5 * np.abs(ref).max()
            if level < oh.n_levels - 1:
                x22 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(pre_sweeps=2, post_sweeps=3))
                ref22 = O.vcycle(oh, level, b, np.zeros_like(b), pre=2, post=3)
                assert np.abs(x22 - ref22).max() <= 1e-11 * np.abs(ref22).max()


@pytest.mark.parametrize("kind,size,cap,width", [("square", 32, 50, 4), ("lshape", 16, 60, 7), ("checker", 32, 40, 33)])
def test_gs_vcycle_matches_oracle(kind, size, cap, width):
    """The multicolour Gauss-Seidel V-cycle (colours ascending before the coarse correction,
    descending after) equals the oracle's on every level, float64 and float32."""
    p, blob, _ = problem_and_blob(kind, size, cap, 1 if kind != "checker" else 3)
    oh = O.read_blob(blob)
    rng = np.random.default_rng(width + 1)
    gs = ae.AMGEIG_SMOOTHER_GAUSS_SEIDEL
    with ae.Hierarchy(blob) as h:
        for level in range(oh.n_levels):
            b = rng.standard_normal((oh.sizes[level], width))
            ref = O.vcycle(oh, level, b, np.zeros_like(b), smoother="gs")
            x64 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=ae.AMGEIG_FP64, smoother=gs))
            assert np.abs(x64 - ref).max() <= 1e-11 * np.abs(ref).max()
            x32 = ae.amgeig_apply_vcycle(h.handle, level, b,
                                         ae.options(precision=ae.AMGEIG_MIXED_FP32, smoother=gs))
            assert np.abs(x32 - ref).max() <= 2e-5 * np.abs(ref).max()
            if level < oh.n_levels - 1:
                x23 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(pre_sweeps=2, post_sweeps=3, smoother=gs))
                ref23 = O.vcycle(oh, level, b, np.zeros_like(b), pre=2, post=3, smoother="gs")
                assert np.abs(x23 - ref23).max() <= 1e-11 * np.abs(ref23).max()


@pytest.mark.parametrize("kind,size,cap,seed,q,qe", [("lshape", 16, 60, 2, 6, 2), ("checker", 32, 60, 3, 5, 2)])
def test_gs_iteration_parity_and_convergence(kind, size, cap, seed, q, qe):
    """Gauss-Seidel smoothing: two corrections equal the oracle's; the converged mixed
    solve reaches the dense eigenvalues in fewer corrections than with l1-Jacobi."""
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    oh = O.read_blob(blob)
    gs = ae.AMGEIG_SMOOTHER_GAUSS_SEIDEL
    lam_o, U_o, _ = O.solve(oh, q, tol=0.0, opts=O.Options(q_extra=qe, fixed_corrections=2, smoother="gs"))
    lam_ex, _ = dense_pairs(p, q)
    lmax = lam_max(p)
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(q, tol=0.0, opt=ae.options(q_extra=qe, fixed_corrections=2, smoother=gs))
        tol = eig_rel_tol(lam_o, lmax)
        assert np.all(np.abs(lam - lam_o) <= tol * lam_o), np.max(np.abs(lam - lam_o) / lam_o)
        assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8
        ptol = max(2e-9, 4 * 2.0 ** -48 * lmax / lam_ex[0])
        mixed = dict(q_extra=qe, max_corrections=150, precision=ae.AMGEIG_MIXED_FP32)
        lam_g, _, info_g, code = h.solve(q, tol=ptol, opt=ae.options(smoother=gs, **mixed))
        assert code == ae.AMGEIG_OK
        prtol = np.maximum(eig_rel_tol(lam_ex, lmax), 4 * 2.0 ** -48 * lmax / lam_ex)
        assert np.all(np.abs(lam_g - lam_ex) <= prtol * lam_ex)
        _, _, info_j, _ = h.solve(q, tol=ptol, opt=ae.options(**mixed))
        assert info_g.corrections <= info_j.corrections


def _bf16(values):
    """float64 -> float32 -> bfloat16 (round to nearest even), back to float64."""
    u = np.asarray(values, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_vcycle_matches_oracle_with_rounded_operators():
    """AMGEIG_MIXED_BF16 stores the V-cycle's operators A_l, R_l, P_l in bfloat16: its
    float32 V-cycle equals the oracle's V-cycle run on a hierarchy whose operators hold
    the same rounded values (the l1 diagonals and the coarsest solve stay exact)."""
    import copy

    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    oh = O.read_blob(blob)
    ob = copy.copy(oh)
    last = oh.n_levels - 1
    ob.A = [a if l == last else a.copy() for l, a in enumerate(oh.A)]
    ob.P = [m.copy() for m in oh.P]
    for l in range(last):
        ob.A[l].data = _bf16(oh.A[l].data)
        ob.P[l].data = _bf16(oh.P[l].data)
    ob.R = [m.T.tocsr() for m in ob.P]
    ob.colour_cache = {}
    rng = np.random.default_rng(9)
    with ae.Hierarchy(blob) as h:
        for level in range(last):
            b = rng.standard_normal((oh.sizes[level], 8))
            ref = O.vcycle(ob, level, b, np.zeros_like(b))
            x = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=ae.AMGEIG_MIXED_BF16))
            assert np.abs(x - ref).max() <= 2e-5 * np.abs(ref).max()
            # and it is a different operator from the float32 one
            x32 = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=ae.AMGEIG_MIXED_FP32))
            assert np.abs(x - x32).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("kind,size,cap,seed,q,qe", [("lshape", 16, 60, 2, 6, 2), ("square", 32, 50, 1, 4, 2)])
def test_bf16_converged_solve(kind, size, cap, seed, q, qe):
    """The bfloat16 operators only change the correction direction: the defect uses the
    exact A, so the converged eigenpairs are the dense ones."""
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    oh = O.read_blob(blob)
    lam_ex, U_ex = dense_pairs(p, q)
    lmax = lam_max(p)
    ptol = max(1e-9, 4 * 2.0 ** -48 * lmax / lam_ex[0])
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(q, tol=ptol, opt=ae.options(q_extra=qe, max_corrections=150,
                                                                 precision=ae.AMGEIG_MIXED_BF16))
    assert code == ae.AMGEIG_OK
    prtol = np.maximum(eig_rel_tol(lam_ex, lmax), 4 * 2.0 ** -48 * lmax / lam_ex)
    assert np.all(np.abs(lam - lam_ex) <= prtol * lam_ex)
    assert m_subspace_angle(U, U_ex, oh.M[0]) < max(1e-8, 10 * ptol)
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(q)).max() < 1e-10


# ------------------------------------------------------------------ solver


CASES = [("square", 32, 50, 1, 4, 2), ("lshape", 16, 60, 2, 6, 2), ("checker", 32, 60, 3, 5, 2),
         ("cube", 8, 40, 4, 4, 2), ("square", 48, 120, 5, 20, 4)]


@pytest.mark.parametrize("kind,size,cap,seed,q,qe", CASES)
@pytest.mark.parametrize("L", [1, 2, 3])
def test_iteration_level_parity(kind, size, cap, seed, q, qe, L):
    """After exactly L finest-level corrections the GPU FP64 path equals the oracle."""
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    oh = O.read_blob(blob)
    lam_o, U_o, info_o = O.solve(oh, q, tol=0.0, opts=O.Options(q_extra=qe, fixed_corrections=L))
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(q, tol=0.0, opt=ae.options(q_extra=qe, fixed_corrections=L))
    assert info.corrections == L
    tol = eig_rel_tol(lam_o, lam_max(p))
    assert np.all(np.abs(lam - lam_o) <= tol * lam_o), np.max(np.abs(lam - lam_o) / lam_o)
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8
    assert np.allclose(info.max_relres, info_o.relres.max(), rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("kind,size,cap,seed,q,qe", CASES)
def test_converged_solve(kind, size, cap, seed, q, qe):
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    oh = O.read_blob(blob)
    # relative-residual floor: ~1e-10 for the coefficient jump; the q = 20 case converges
    # its last pair more slowly (tighter tolerances need many more corrections)
    tol = 2e-9 if kind == "checker" else (1e-9 if q >= 20 else 1e-10)
    lam_ex, U_ex = dense_pairs(p, q)
    rtol = eig_rel_tol(lam_ex, lam_max(p))
    lmax = lam_max(p)
    with ae.Hierarchy(blob) as h:
        for prec in (ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32):
            # the mixed path keeps its iterates in float-float (unit roundoff 2^-48):
            # its residual floor is ~2^-48 lambda_max / lambda instead of 2^-53 times that
            ptol = tol if prec == ae.AMGEIG_FP64 else max(tol, 4 * 2.0 ** -48 * lmax / lam_ex[0])
            prtol = rtol if prec == ae.AMGEIG_FP64 else np.maximum(rtol, 4 * 2.0 ** -48 * lmax / lam_ex)
            lam, U, info, code = h.solve(q, tol=ptol, opt=ae.options(q_extra=qe, max_corrections=150, precision=prec))
            assert code == ae.AMGEIG_OK and info.converged == 1
            assert np.all(np.abs(lam - lam_ex) <= prtol * lam_ex), np.max(np.abs(lam - lam_ex) / lam_ex)
            assert m_subspace_angle(U, U_ex, oh.M[0]) < max(1e-8, 10 * ptol)
            G = U.T @ (oh.M[0] @ U)
            assert np.abs(G - np.eye(q)).max() < 1e-10
            idx = np.argmax(np.abs(U), axis=0)
            assert np.all(U[idx, np.arange(q)] > 0)
            assert np.all(O.relres(oh, lam, U) <= ptol * 1.0001 + 1e-13)


def test_mixed_matches_fp64_iterates():
    """The float32 V-cycle changes the iterates by at most float32-level relative amounts."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    with ae.Hierarchy(blob) as h:
        l64, _, _, _ = h.solve(6, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=4))
        l32, _, _, _ = h.solve(6, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=4,
                                                          precision=ae.AMGEIG_MIXED_FP32))
    assert np.max(np.abs(l32 - l64) / l64) < 1e-6


def test_deterministic_repeat():
    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    with ae.Hierarchy(blob) as h:
        a = h.solve(4, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=3))
        b = h.solve(4, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=3))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_device_output_and_nonconvergence():
    import torch

    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    with ae.Hierarchy(blob) as h:
        vals = np.empty(4)
        vecs = torch.empty((p.n, 4), dtype=torch.float64, device="cuda:0")
        info = ae.amgeig_info()
        code = ae.amgeig_solve(h.handle, 4, 1e-14, ae.options(max_corrections=2), vals, vecs, True, info)
        assert code == ae.AMGEIG_ENOCONV and info.converged == 0 and info.corrections == 2
        lam_h, U_h, _, _ = h.solve(4, tol=1e-14, opt=ae.options(max_corrections=2))
        assert np.array_equal(vals, lam_h) and np.array_equal(vecs.cpu().numpy(), U_h)


def test_errors_are_reported():
    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    bad = bytearray(blob)
    bad[300] ^= 1
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_load_hierarchy(bytes(bad))
    assert e.value.code == ae.AMGEIG_ECORRUPT
    with ae.Hierarchy(blob) as h:
        with pytest.raises(ae.AmgEigError) as e:
            h.solve(h.sizes[0] + 1)
        assert e.value.code == ae.AMGEIG_EINVAL
        with pytest.raises(ae.AmgEigError) as e:
            h.solve(120, opt=ae.options(q_extra=9))  # q + q_extra above 128
        assert e.value.code == ae.AMGEIG_EINVAL
        with pytest.raises(ae.AmgEigError):
            h.solve(2, opt=ae.options(v_cycles=0))


def test_submit_poll_matches_direct():
    import time

    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    with ae.Hierarchy(blob) as h:
        # batch = 0: each request runs its own solve (a shared solve gives equal results within tolerance, not bits)
        direct = [h.solve(q, tol=1e-9, opt=ae.options(q_extra=2, max_corrections=60)) for q in (3, 6)]
        ids = [ae.amgeig_submit(h.handle, q, 1e-9, ae.options(q_extra=2, max_corrections=60, batch=0))
               for q in (3, 6)]
        for rid, q, d in zip(ids, (3, 6), direct):
            vals = np.empty(q)
            vecs = np.empty((p.n, q))
            t0 = time.time()
            while True:
                done, code = ae.amgeig_poll(rid, vals, vecs)
                if done:
                    break
                assert time.time() - t0 < 120
                time.sleep(0.01)
            assert code == ae.AMGEIG_OK
            assert np.array_equal(vals, d[0]) and np.array_equal(vecs, d[1])
        with pytest.raises(ae.AmgEigError):
            ae.amgeig_poll(ids[0])


def test_blob_alignment_and_validation():
    """The loader reads the blob in place: an unaligned blob (copied once) gives the
    same bits as an aligned one, and an out-of-range column index behind a valid
    checksum is rejected."""
    import ctypes
    import struct

    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    # autotune = 0: the two handles compared bit for bit use the rule's launch shapes
    opt = ae.options(q_extra=2, max_corrections=30, precision=ae.AMGEIG_MIXED_FP32, autotune=0)
    with ae.Hierarchy(blob) as h:
        ref = h.solve(3, tol=1e-9, opt=opt)
    raw = ctypes.create_string_buffer(len(blob) + 8)
    addr = ctypes.addressof(raw)
    base = addr + 1 if (addr + 1) % 8 != 0 else addr + 2  # not 8-byte aligned
    ctypes.memmove(base, blob, len(blob))
    hnd = ctypes.c_void_p()
    ae._check(ae.lib().amgeig_load_hierarchy(ctypes.c_void_p(base), len(blob), 0, ctypes.byref(hnd)), "load")
    try:
        vals = np.empty(3)
        vecs = np.empty((p.n, 3))
        ae.amgeig_solve(hnd, 3, 1e-9, opt, vals, vecs, False)
        assert np.array_equal(vals, ref[0]) and np.array_equal(vecs, ref[1])
    finally:
        ae.amgeig_free_hierarchy(hnd)
    # level 0's first column index out of range, checksum rewritten
    n_lev = struct.unpack_from("<I", blob, 12)[0]
    off = 16 + 8 * (3 * n_lev - 1)
    off += (8 - off % 8) % 8
    rows0 = struct.unpack_from("<Q", blob, 16)[0]
    ci0 = off + 4 * (rows0 + 1)
    ci0 += (8 - ci0 % 8) % 8
    bad = bytearray(blob)
    struct.pack_into("<i", bad, ci0, int(rows0) + 5)
    words = np.frombuffer(bytes(bad[:-8]), dtype="<u8")
    struct.pack_into("<Q", bad, len(bad) - 8, int(words.sum(dtype=np.uint64)))
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_load_hierarchy(bytes(bad))
    assert e.value.code == ae.AMGEIG_ECORRUPT and "CSR" in str(e.value)


def test_request_mix_matches_alone():
    """Requests on three hierarchies, submitted together so that they run at the same
    time on the library's workers, give the same bits as each solve run alone."""
    import time

    cases = [problem_and_blob("square", 32, 50, 1), problem_and_blob("lshape", 16, 60, 2),
             problem_and_blob("checker", 32, 60, 3)]
    hs = [ae.Hierarchy(blob) for _, blob, _ in cases]
    try:
        plan = [(i % 3, q, prec) for i, (q, prec) in
                enumerate([(2, ae.AMGEIG_FP64), (5, ae.AMGEIG_MIXED_FP32), (3, ae.AMGEIG_MIXED_FP32),
                           (4, ae.AMGEIG_FP64), (6, ae.AMGEIG_MIXED_FP32), (2, ae.AMGEIG_MIXED_FP32),
                           (7, ae.AMGEIG_FP64), (3, ae.AMGEIG_FP64), (5, ae.AMGEIG_MIXED_FP32)])]

        def opt(prec):
            # batch = 0: each request keeps its own solve, so its bits can be compared
            return ae.options(q_extra=2, max_corrections=40, precision=prec, v_cycles=2, batch=0)

        alone = [hs[k].solve(q, tol=1e-8, opt=opt(prec)) for k, q, prec in plan]
        ids = [ae.amgeig_submit(hs[k].handle, q, 1e-8, opt(prec)) for k, q, prec in plan]
        pending = dict(zip(ids, range(len(plan))))
        t0 = time.time()
        while pending:
            for rid in list(pending):
                j = pending[rid]
                k, q, _ = plan[j]
                vals = np.empty(q)
                vecs = np.empty((cases[k][0].n, q))
                done, code = ae.amgeig_poll(rid, vals, vecs)
                if not done:
                    continue
                del pending[rid]
                assert code == alone[j][3]
                assert np.array_equal(vals, alone[j][0]), (j, vals, alone[j][0])
                assert np.array_equal(vecs, alone[j][1]), j
            assert time.time() - t0 < 300
            time.sleep(0.005)
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("level", [0, 1])
def test_defect_matches_oracle(level):
    """r_j = lambda_j M u_j - A u_j and the relative residuals (Eq. Linear_Equation),
    float64 kernel and float-float kernel, against the oracle's sparse products; near
    eigenvectors too, where lambda M u and A u cancel to ~1e-6 of their size."""
    p, blob, _ = problem_and_blob("lshape", 24, 60, 2)
    oh = O.read_blob(blob)
    A, M = oh.A[level], oh.M[level]
    n = A.shape[0]
    rng = np.random.default_rng(5)
    import scipy.linalg as sla

    lam_d, V_d = sla.eigh(A.toarray(), M.toarray(), subset_by_index=[0, 5])
    cases = [(rng.standard_normal((n, 7)), rng.uniform(5.0, 200.0, 7)),
             (V_d + 1e-6 * rng.standard_normal(V_d.shape), lam_d)]
    with ae.Hierarchy(blob) as h:
        for U, lam in cases:
            ref = M @ U * lam[None, :] - A @ U
            scale = (abs(A) @ abs(U)) + (abs(M) @ abs(U)) * abs(lam)[None, :]
            rr_ref = np.linalg.norm(ref, axis=0) / (np.abs(lam) * np.linalg.norm(M @ U, axis=0))
            R64, rr64 = ae.amgeig_apply_defect(h.handle, level, U, lam, ae.options(precision=ae.AMGEIG_FP64))
            assert np.all(np.abs(R64 - ref) <= 1e-14 * scale + 1e-300)
            np.testing.assert_allclose(rr64, rr_ref, rtol=1e-10)
            R32, rr32 = ae.amgeig_apply_defect(h.handle, level, U, lam,
                                              ae.options(precision=ae.AMGEIG_MIXED_FP32))
            # float-float products (~2^-46 of the operand scale), then float32 rounding
            assert np.all(np.abs(R32 - ref) <= 2.0 ** -23 * np.abs(ref) + 2.0 ** -42 * scale)
            np.testing.assert_allclose(rr32, rr_ref, rtol=1e-6)


def test_multiple_vcycles_match_oracle():
    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    oh = O.read_blob(blob)
    lam_o, U_o, _ = O.solve(oh, 4, tol=0.0, opts=O.Options(q_extra=1, fixed_corrections=2, v_cycles=2,
                                                           pre_sweeps=2, post_sweeps=1))
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(4, tol=0.0, opt=ae.options(q_extra=1, fixed_corrections=2, v_cycles=2,
                                                             pre_sweeps=2, post_sweeps=1))
    assert np.max(np.abs(lam - lam_o) / lam_o) < 1e-10
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8


def test_wide_block_all_coarse_modes_matches_oracle():
    """q + q_extra = 90 with the full coarse space (255 modes): the pencil goes through
    the dense solver and the coarse reconstruction runs in column chunks."""
    p, blob, _ = problem_and_blob("square", 64, 400, 1)
    oh = O.read_blob(blob)
    lam_o, U_o, _ = O.solve(oh, 80, tol=0.0, opts=O.Options(q_extra=10, fixed_corrections=2))
    with ae.Hierarchy(blob) as h:
        assert h.sizes[-1] >= 200
        lam, U, info, _ = h.solve(80, tol=0.0, opt=ae.options(q_extra=10, fixed_corrections=2))
    assert info.dense_fallbacks > 0
    tol = eig_rel_tol(lam_o, lam_max(p))
    assert np.all(np.abs(lam - lam_o) / lam_o < tol)
    M = oh.M[0]
    assert np.max(np.abs(U.T @ (M @ U) - np.eye(80))) < 1e-10


def test_coarse_modes_on_demand():
    """The coarse eigenbasis is computed on the first solve with only the modes it needs
    and again, whole, when a later solve needs more: every solve gives the bits of the
    same solve on a fresh hierarchy."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    few = ae.options(q_extra=2, fixed_corrections=2, coarse_modes=16)
    full = ae.options(q_extra=2, fixed_corrections=2)
    with ae.Hierarchy(blob) as h:
        a_few = h.solve(6, tol=0.0, opt=few)
        a_full = h.solve(6, tol=0.0, opt=full)
        a_few2 = h.solve(6, tol=0.0, opt=few)
    with ae.Hierarchy(blob) as h:
        b_full = h.solve(6, tol=0.0, opt=full)
        b_few = h.solve(6, tol=0.0, opt=few)
    with ae.Hierarchy(blob) as h:
        c_few = h.solve(6, tol=0.0, opt=few)
    assert np.array_equal(a_full[0], b_full[0]) and np.array_equal(a_full[1], b_full[1])
    assert np.array_equal(a_few[0], c_few[0]) and np.array_equal(a_few[1], c_few[1])
    # a few-mode solve after the full basis exists uses its leading columns: same fixed point
    assert np.array_equal(a_few2[0], b_few[0])
    assert np.max(np.abs(a_few2[0] - a_few[0]) / a_few[0]) < 1e-10


def test_coarse_modes_during_load():
    """amgeig_load_hierarchy_modes computes the coarse modes on a side stream during the
    load: a solve on such a hierarchy gives the bits of the same solve on a hierarchy that
    computes them on demand (same mode count), for a truncated and for the full pencil, and
    a solve that needs more modes than were loaded computes them itself."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    few = ae.options(q_extra=2, fixed_corrections=2, coarse_modes=16)
    full = ae.options(q_extra=2, fixed_corrections=2)
    with ae.Hierarchy(blob) as h:
        ref_few = h.solve(6, tol=0.0, opt=few)
    with ae.Hierarchy(blob) as h:
        ref_full = h.solve(6, tol=0.0, opt=full)
    with ae.Hierarchy(blob, modes=16) as h:
        got_few = h.solve(6, tol=0.0, opt=few)
        # more modes than were loaded: the whole basis is computed on this solve
        got_full_after = h.solve(6, tol=0.0, opt=full)
    for modes in (0, 10 ** 6):  # all modes; a count above d_n is clamped to all
        with ae.Hierarchy(blob, modes=modes) as h:
            got_full = h.solve(6, tol=0.0, opt=full)
        assert np.array_equal(got_full[0], ref_full[0]) and np.array_equal(got_full[1], ref_full[1])
    assert np.array_equal(got_few[0], ref_few[0]) and np.array_equal(got_few[1], ref_few[1])
    assert np.array_equal(got_full_after[0], ref_full[0]) and np.array_equal(got_full_after[1], ref_full[1])
    with pytest.raises(ae.AmgEigError):
        ae.amgeig_load_hierarchy_modes(blob, 0, -1)


@pytest.mark.parametrize("L", [1, 3])
def test_coarse_modes_parity(L):
    """The truncated coarse space (coarse_modes option) matches the oracle's same option."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    oh = O.read_blob(blob)
    lam_o, U_o, _ = O.solve(oh, 6, tol=0.0, opts=O.Options(q_extra=2, fixed_corrections=L, coarse_modes=16))
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(6, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=L, coarse_modes=16))
    assert np.max(np.abs(lam - lam_o) / lam_o) < 1e-10
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8


# ------------------------------------------------------------------ initial level n1 < n


@pytest.mark.parametrize("L", [1, 2])
def test_initial_level_above_coarsest_matches_oracle(L):
    """q + q_extra above the coarsest dimension: both sides start on the coarsest level that holds the
    pairs (Algorithm 3.2 step 1 with n1 < n) and agree after L finest-level corrections."""
    p, blob, _ = problem_and_blob("square", 32, 20, 1)
    oh = O.read_blob(blob)
    q, qe = oh.sizes[-1] + 2, 3
    lam_o, U_o, info_o = O.solve(oh, q, tol=0.0, opts=O.Options(q_extra=qe, fixed_corrections=L))
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(q, tol=0.0, opt=ae.options(q_extra=qe, fixed_corrections=L))
    assert info.n1 == info_o.n1 < len(oh.sizes) - 1
    tol = eig_rel_tol(lam_o, lam_max(p))
    assert np.all(np.abs(lam - lam_o) <= tol * lam_o), np.max(np.abs(lam - lam_o) / lam_o)
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8


def test_initial_level_finest_and_converged_mixed():
    """n1 = 0 is the finest level's dense eigensolution; the mixed path from the default n1 < n
    converges to the dense eigenpairs."""
    p, blob, _ = problem_and_blob("square", 32, 20, 1)
    oh = O.read_blob(blob)
    lam_ex, U_ex = dense_pairs(p, 24)
    with ae.Hierarchy(blob) as h:
        lam0, U0, info0, _ = h.solve(4, tol=1e-8, opt=ae.options(n1=0))
        assert info0.n1 == 0 and info0.corrections == 0
        assert np.all(np.abs(lam0 - lam_ex[:4]) <= 1e-11 * lam_ex[:4])
        assert m_subspace_angle(U0, U_ex[:, :4], oh.M[0]) < 1e-8
        q = oh.sizes[-1] + 2
        lam, U, info, code = h.solve(q, tol=1e-9, opt=ae.options(q_extra=3, max_corrections=150,
                                                                 precision=ae.AMGEIG_MIXED_FP32))
        assert code == ae.AMGEIG_OK and info.n1 < len(oh.sizes) - 1
        assert np.all(np.abs(lam - lam_ex[:q]) <= 1e-10 * lam_ex[:q]), np.max(np.abs(lam - lam_ex[:q]) / lam_ex[:q])
        with pytest.raises(ae.AmgEigError) as e:
            h.solve(q, opt=ae.options(q_extra=3, n1=len(oh.sizes) - 1))
        assert e.value.code == ae.AMGEIG_EINVAL


# ------------------------------------------------------------------ mixed path against the oracle


@pytest.mark.parametrize("L", [1, 2])
def test_mixed_iteration_parity_multilane(L):
    """The mixed path (float32 V-cycle, float-float Rayleigh-Ritz, float64 Rayleigh quotients at the end)
    against the oracle's iterates after L finest-level corrections, on an L-shape with 247,681 rows:
    the finest level takes the multi-lane layout of the timed workload (4 lanes per row, 2 float4 groups
    per lane), the levels below 155,648 rows 8 lanes per row.  Tolerances as for the full-size check
    of the timed settings: the float32 V-cycle moves each correction by <= 2e-5 of its column, hence
    the subspace by an angle of order 1e-5 and the Ritz values by about twice that times the relative
    residual."""
    p, blob, _ = problem_and_blob("lshape", 288, 400, 2)
    oh = O.read_blob(blob)
    assert oh.sizes[0] >= 200_000
    q, qe = 12, 4
    kw = dict(q_extra=qe, fixed_corrections=L, v_cycles=2)
    lam_o, U_o, info_o = O.solve(oh, q, tol=0.0, opts=O.Options(**kw))
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(q, tol=0.0, opt=ae.options(precision=ae.AMGEIG_MIXED_FP32, **kw))
    rel = np.max(np.abs(lam - lam_o) / lam_o)
    ang = m_subspace_angle(U, U_o, oh.M[0])
    assert rel <= 1e-6 and ang <= 1e-4, (rel, ang, info_o.relres.max())
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(q)).max() < 1e-10


@pytest.mark.parametrize("prec", [ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32])
def test_graph_replay_gives_the_same_bits(prec):
    """The nested phase and the finest-level corrections replayed from captured CUDA graphs give the bits of
    direct launches, on the first (capturing) solve and on later (replaying) ones, and count the same
    kernels; the buffer roles alternate between corrections, so both capture states are exercised."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    base = dict(q_extra=2, max_corrections=40, precision=prec, v_cycles=2)
    with ae.Hierarchy(blob) as h:
        h.solve(5, tol=1e-9, opt=ae.options(graphs=0, **base))  # one-time work (coarse modes, tuning) first
        k0 = ae.amgeig_kernel_launches()
        direct = h.solve(5, tol=1e-9, opt=ae.options(graphs=0, **base))
        k1 = ae.amgeig_kernel_launches()
        runs = [h.solve(5, tol=1e-9, opt=ae.options(graphs=1, **base)) for _ in range(3)]
        k2 = ae.amgeig_kernel_launches()
    assert direct[2].corrections >= 3
    for lam, U, info, code in runs:
        assert code == direct[3] and info.corrections == direct[2].corrections
        assert np.array_equal(lam, direct[0]) and np.array_equal(U, direct[1])
    assert k2 - k1 == 3 * (k1 - k0)


def test_autotuned_launch_shapes():
    """The tuner picks each level's lane layout for the float32 smoothing and transfer kernels by timing.
    Solves on tuned shapes converge to the solve on the fixed rule's shapes (a layout with another stream
    count rounds the V-cycle differently: agreement to 1e-10 at relative residual 1e-9), a hierarchy's
    later solves repeat its bits, and the report lists every level below the coarsest, three kernels
    each, with a valid layout."""
    p, blob, _ = problem_and_blob("lshape", 48, 60, 2)
    oh = O.read_blob(blob)
    base = dict(q_extra=4, max_corrections=40, precision=ae.AMGEIG_MIXED_FP32, v_cycles=2)
    with ae.Hierarchy(blob) as h1:
        rule = h1.solve(8, tol=1e-9, opt=ae.options(autotune=0, **base))
        assert ae.amgeig_tuning_report(h1.handle) == []
    with ae.Hierarchy(blob) as h2:
        tuned = h2.solve(8, tol=1e-9, opt=ae.options(autotune=1, **base))
        again = h2.solve(8, tol=1e-9, opt=ae.options(autotune=1, **base))
        rep = ae.amgeig_tuning_report(h2.handle)
        nlev = len(h2.sizes)
    assert rule[3] == tuned[3] == ae.AMGEIG_OK
    assert np.max(np.abs(rule[0] - tuned[0]) / rule[0]) <= 1e-10
    assert m_subspace_angle(rule[1], tuned[1], oh.M[0]) <= 1e-7
    assert np.array_equal(tuned[0], again[0]) and np.array_equal(tuned[1], again[1])
    assert len(rep) == 3 * (nlev - 1)
    for e in rep:
        assert e["G"] in (1, 2, 4, 8, 16, 32) and 1 <= e["cpt"] <= 3 and e["S"] in (1, 2, 4)
        assert (e["G"] // e["S"]) * e["cpt"] >= e["w4"]
        assert 0 < e["us"] <= e["rule_us"] * 1.5


def test_batched_requests_match_alone_within_tolerance():
    """Requests queued together on one hierarchy share a solve (the widest q and buffer, the tightest
    tolerance); each receives its own leading pairs.  Against the same request solved alone: eigenvalues
    within 1e-8 relative (the metric's bound; both are converged to relative residual 1e-9, so they
    differ by about the square of that), the eigenvector subspaces within a principal angle of 1e-6
    (about ten times the residual over the relative gap after the wanted pairs), each request's
    residual at its own tolerance."""
    import time

    p, blob, _ = problem_and_blob("lshape", 24, 60, 2)
    oh = O.read_blob(blob)
    qs = [2, 6, 4, 9, 3, 6, 1, 8]
    tol = 1e-9

    def opt(batch):
        return ae.options(q_extra=3, max_corrections=80, precision=ae.AMGEIG_MIXED_FP32, v_cycles=2, batch=batch)

    with ae.Hierarchy(blob) as h:
        alone = [h.solve(q, tol=tol, opt=opt(0)) for q in qs]
        # hold the hierarchy busy with a first request so that the others queue up and join one solve
        ids = [ae.amgeig_submit(h.handle, q, tol, opt(1)) for q in qs]
        res = {}
        t0 = time.time()
        while len(res) < len(ids):
            for rid, q in zip(ids, qs):
                if rid in res:
                    continue
                vals, vecs, info = np.empty(q), np.empty((p.n, q)), ae.amgeig_info()
                done, code = ae.amgeig_poll(rid, vals, vecs, info)
                if done:
                    res[rid] = (code, vals, vecs, info)
            assert time.time() - t0 < 120
            time.sleep(0.002)
    shared = 0
    for rid, q, (lam_a, U_a, info_a, code_a) in zip(ids, qs, alone):
        code, lam, U, info = res[rid]
        assert code == ae.AMGEIG_OK and code_a == ae.AMGEIG_OK
        assert np.all(np.abs(lam - lam_a) <= 1e-8 * lam_a), np.max(np.abs(lam - lam_a) / lam_a)
        assert m_subspace_angle(U, U_a, oh.M[0]) <= 1e-6
        assert np.all(O.relres(oh, lam, U) <= tol * 1.0001)
        assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(q)).max() < 1e-10
        shared += int(not np.array_equal(U, U_a))
    assert shared >= 1  # at least one request was answered by a shared solve


def _exact_rayleigh(A, M, u):
    """u^T A u / u^T M u of the float64 vector u and float64 matrices, in exact rational arithmetic."""
    from fractions import Fraction

    uf = [Fraction(float(x)) for x in u]

    def quad(S):
        tot = Fraction(0)
        for i in range(S.shape[0]):
            row = Fraction(0)
            for p in range(S.indptr[i], S.indptr[i + 1]):
                row += Fraction(float(S.data[p])) * uf[S.indices[p]]
            tot += uf[i] * row
        return tot

    return float(quad(A) / quad(M))


@pytest.mark.parametrize("prec", [ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32])
def test_compensated_refinement_gives_exact_rayleigh_quotients(prec):
    """refine = 2: each returned eigenvalue is the Rayleigh quotient of the returned float64 vector to a few
    units of float64 rounding (checked against exact rational arithmetic), on the coefficient-jump problem
    where plain float64 sums lose digits to cancellation; the values are ascending and the residual
    reported is the returned pairs'."""
    p, blob, _ = problem_and_blob("checker", 32, 60, 3)
    oh = O.read_blob(blob)
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(5, tol=1e-8, opt=ae.options(q_extra=2, max_corrections=150, precision=prec,
                                                                 refine=2))
    assert code == ae.AMGEIG_OK and np.all(np.diff(lam) >= 0)
    exact = np.array([_exact_rayleigh(oh.A[0], oh.M[0], U[:, j]) for j in range(5)])
    assert np.all(np.abs(lam - exact) <= 8 * 2.0 ** -53 * exact), np.max(np.abs(lam - exact) / exact)
    rr = O.relres(oh, lam, U)
    assert np.allclose(info.max_relres, rr.max(), rtol=1e-6)


# ------------------------------------------------------------------ shifted inner solve


def _safe_shift(oh, frac=0.5):
    """A shift below the coarsest pencil's lowest eigenvalue (so every level's A - sigma M stays SPD)."""
    import scipy.linalg as sla

    lo = sla.eigh(oh.An, oh.Mn, eigvals_only=True, subset_by_index=[0, 0])[0]
    return frac * float(lo)


@pytest.mark.parametrize("prec,rtol", [(ae.AMGEIG_FP64, 1e-11), (ae.AMGEIG_MIXED_FP32, 2e-5)])
def test_shifted_vcycle_matches_oracle(prec, rtol):
    """One V-cycle on the hierarchy of A_l - sigma M_l (shifted values, their l1 diagonals, the shifted exact
    coarsest solve) against the oracle's shifted V-cycle, every level, element by element."""
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    oh = O.read_blob(blob)
    sigma = _safe_shift(oh)
    hs = O.shifted(oh, sigma)
    with ae.Hierarchy(blob) as h:
        for level in range(len(oh.sizes)):
            n = oh.sizes[level]
            b = np.random.default_rng(level).standard_normal((n, 6))
            x = ae.amgeig_apply_vcycle(h.handle, level, b, ae.options(precision=prec, shift=sigma))
            xo = O.vcycle(hs, level, b, np.zeros_like(b))
            err = np.abs(x - xo).max(axis=0) / np.abs(xo).max(axis=0)
            assert np.all(err <= rtol), (level, err.max())


@pytest.mark.parametrize("L", [1, 2])
def test_shifted_iteration_parity(L):
    """L finest-level corrections with the shifted inner solve: the GPU float64 path against the oracle's."""
    p, blob, _ = problem_and_blob("square", 32, 50, 1)
    oh = O.read_blob(blob)
    sigma = _safe_shift(oh, 0.9)
    lam_o, U_o, _ = O.solve(oh, 4, tol=0.0, opts=O.Options(q_extra=2, fixed_corrections=L, shift=sigma))
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(4, tol=0.0, opt=ae.options(q_extra=2, fixed_corrections=L, shift=sigma))
    assert np.all(np.abs(lam - lam_o) <= eig_rel_tol(lam_o, lam_max(p)) * lam_o)
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8


def test_shifted_mixed_solve_converges_and_refuses_a_large_shift():
    p, blob, _ = problem_and_blob("lshape", 16, 60, 2)
    oh = O.read_blob(blob)
    lam_ex, U_ex = dense_pairs(p, 6)
    sigma = _safe_shift(oh, 0.9)
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(6, tol=1e-9, opt=ae.options(q_extra=2, max_corrections=100, v_cycles=2,
                                                                 precision=ae.AMGEIG_MIXED_FP32, shift=sigma))
        assert code == ae.AMGEIG_OK
        assert np.all(np.abs(lam - lam_ex) <= 1e-10 * lam_ex)
        assert m_subspace_angle(U, U_ex, oh.M[0]) < 1e-7
        with pytest.raises(ae.AmgEigError) as e:
            h.solve(6, tol=1e-9, opt=ae.options(q_extra=2, shift=2.0 * _safe_shift(oh, 1.0)))
        assert e.value.code == ae.AMGEIG_EINVAL
        # after a refused shift the hierarchy still solves (unshifted and shifted)
        lam2, _, _, code2 = h.solve(6, tol=1e-9, opt=ae.options(q_extra=2, max_corrections=100))
        assert code2 == ae.AMGEIG_OK and np.all(np.abs(lam2 - lam_ex) <= 1e-10 * lam_ex)


# ------------------------------------------------------------------ Krylov-augmented correction space


@pytest.mark.parametrize("kind,size,cap,seed,q,qe", [("lshape", 16, 60, 2, 6, 2), ("square", 32, 50, 1, 4, 2)])
@pytest.mark.parametrize("L,m", [(1, 1), (2, 1), (3, 1), (2, 2)])
def test_krylov_iteration_parity(kind, size, cap, seed, q, qe, L, m):
    """Depth-2 Krylov space (V_n + span(TU, T^2 U)) on the GPU float64 path against the oracle's, after L
    finest-level corrections with m V-cycles per inverse-iteration step: the GPU takes the pencil on
    [TU | T^2 U - TU], the oracle on the M-orthonormalised [TU, T^2 U]; Rayleigh-Ritz depends only on the
    span, so the bounds are the float64 parity bounds."""
    p, blob, _ = problem_and_blob(kind, size, cap, seed)
    oh = O.read_blob(blob)
    lam_o, U_o, _ = O.solve(oh, q, tol=0.0, opts=O.Options(q_extra=qe, fixed_corrections=L, krylov=2, v_cycles=m))
    with ae.Hierarchy(blob) as h:
        lam, U, info, _ = h.solve(q, tol=0.0, opt=ae.options(q_extra=qe, fixed_corrections=L, krylov=2, v_cycles=m))
    rel = np.max(np.abs(lam - lam_o) / lam_o)
    assert np.all(np.abs(lam - lam_o) <= eig_rel_tol(lam_o, lam_max(p)) * lam_o), rel
    assert m_subspace_angle(U, U_o, oh.M[0]) < 1e-8


@pytest.mark.parametrize("prec", [ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32])
def test_krylov_converged_solve_and_fewer_corrections(prec):
    """The Krylov space converges to the dense eigenpairs in fewer corrections than the paper's space."""
    p, blob, _ = problem_and_blob("lshape", 24, 60, 2)
    oh = O.read_blob(blob)
    lam_ex, U_ex = dense_pairs(p, 6)
    with ae.Hierarchy(blob) as h:
        base = dict(q_extra=2, max_corrections=100, precision=prec)
        l1, _, i1, c1 = h.solve(6, tol=1e-9, opt=ae.options(krylov=1, **base))
        l2, U2, i2, c2 = h.solve(6, tol=1e-9, opt=ae.options(krylov=2, **base))
    assert c1 == c2 == ae.AMGEIG_OK
    assert i2.corrections < i1.corrections, (i2.corrections, i1.corrections)
    assert np.all(np.abs(l2 - lam_ex) <= 1e-10 * lam_ex)
    assert m_subspace_angle(U2, U_ex, oh.M[0]) < 1e-7
    assert np.abs(U2.T @ (oh.M[0] @ U2) - np.eye(6)).max() < 1e-10


def test_checkerboard_mixed_eigenvalues_at_the_metric_bound():
    """The C3 family (10^(+-3) checkerboard coefficient, dense low spectrum): the mixed path with compensated
    Rayleigh quotients gives each of its eigenvalues within 1e-8 (the metric's bound) of the dense generalized
    eigenvalue.  LAPACK's own eigenvalues carry ~u lambda_max / lambda_j of rounding on this pencil (~1e-8
    for the smallest), so the reference is the exact Rayleigh quotient of LAPACK's eigenvector, which is the
    eigenvalue to second order in that vector's error."""
    p, blob, _ = problem_and_blob("checker", 24, 40, 3)
    oh = O.read_blob(blob)
    q = 8
    lam_ex, U_ex = dense_pairs(p, q)
    ref = np.array([_exact_rayleigh(oh.A[0], oh.M[0], U_ex[:, j]) for j in range(q)])
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(q, tol=1e-8, opt=ae.options(q_extra=6, max_corrections=200, v_cycles=2,
                                                                 precision=ae.AMGEIG_MIXED_FP32, refine=2))
    assert code == ae.AMGEIG_OK
    rel = np.abs(lam - ref) / ref
    assert np.all(rel <= 1e-8), rel.max()


@pytest.mark.parametrize("q,qe", [(60, 12), (59, 12)])
def test_mixed_wide_border_parity(q, qe):
    """Mixed path with a border of 72 (even: the Gram's tile list split over two blocks per row chunk with
    bulk-copied slabs, the recombination streaming Y through shared memory) or 71 columns (odd: the
    register-staged fallbacks) against the oracle's iterates after 2 finest corrections; every pencil takes
    the dense path.  Tolerances as for the multi-lane check (the float32 V-cycle moves each correction by
    <= 2e-5 of its column); the subspace is compared on its leading columns up to a gap of at least 1e-3."""
    p, blob, _ = problem_and_blob("square", 64, 400, 5)
    oh = O.read_blob(blob)
    kw = dict(q_extra=qe, fixed_corrections=2, v_cycles=2)
    lam_o, U_o, info_o = O.solve(oh, q, tol=0.0, opts=O.Options(**kw))
    with ae.Hierarchy(blob) as h:
        lam, U, info, code = h.solve(q, tol=0.0, opt=ae.options(precision=ae.AMGEIG_MIXED_FP32, **kw))
    assert info.corrections == 2
    rel = np.max(np.abs(lam - lam_o) / lam_o)
    gaps = np.diff(lam_o) / lam_o[1:]
    k = int(np.nonzero(gaps > 1e-3)[0].max()) + 1  # columns 0..k-1 end at a gap
    assert k >= q // 2
    ang = m_subspace_angle(U[:, :k], U_o[:, :k], oh.M[0])
    assert rel <= 1e-6 and ang <= 1e-4, (rel, ang, k, info_o.relres.max())
    assert np.abs(U.T @ (oh.M[0] @ U) - np.eye(q)).max() < 1e-10


def test_reload_into_kept_blocks_gives_the_same_bits():
    """Device blocks released with a hierarchy are kept and handed to the next load: a hierarchy loaded into
    blocks that still hold another hierarchy's data (here the same problem's, then a different one's) solves to
    the same bits as on its first load, for both precisions."""
    _, blob, _ = problem_and_blob("lshape", 24, 60, 2)
    _, other, _ = problem_and_blob("square", 40, 60, 3)
    opts = [ae.options(q_extra=2, max_corrections=40, precision=prec, v_cycles=2)
            for prec in (ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32)]

    def run(b):
        with ae.Hierarchy(b) as h:
            return [h.solve(5, tol=1e-9, opt=o) for o in opts]

    first = run(blob)
    run(other)
    for again in (run(blob), run(blob)):
        for (l0, u0, i0, c0), (l1, u1, i1, c1) in zip(first, again):
            assert c0 == c1 and i0.corrections == i1.corrections
            assert np.array_equal(l0, l1) and np.array_equal(u0, u1)
