"""Failure paths of the GPU library, made on the host: non-positive-definite mass matrices, a
corrupt blob behind a valid layout, and admission refusal / eviction under the request service's
memory cap.  Nothing here faults or hangs the GPU: every failure is an input the library checks."""
import time

import numpy as np
import pytest

from paper_1503_08462_gb300 import amgeig as ae
from paper_1503_08462_gb300.inputs import hierarchy

from helpers import problem_and_blob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _copy(h):
    return hierarchy.Hierarchy([hierarchy.Level(lv.row_ptr.copy(), lv.col_idx.copy(), lv.a_vals.copy(),
                                                lv.m_vals.copy()) for lv in h.levels],
                               [hierarchy.Transfer(p.row_ptr.copy(), p.col_idx.copy(), p.vals.copy(), p.n_cols)
                                for p in h.prolong])


def _diag_positions(lv):
    pos = []
    for i in range(lv.n):
        for p in range(lv.row_ptr[i], lv.row_ptr[i + 1]):
            if lv.col_idx[p] == i:
                pos.append(p)
    return np.array(pos)


def test_non_spd_coarsest_mass_is_refused_at_load():
    """M_n with a negative diagonal entry: the loader's Cholesky of M_n reports ENOTSPD."""
    _, _, h = problem_and_blob("square", 32, 50, 1)
    bad = _copy(h)
    lv = bad.levels[-1]
    lv.m_vals[_diag_positions(lv)[3]] *= -1.0
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_load_hierarchy(hierarchy.to_blob(bad))
    assert e.value.code == ae.AMGEIG_ENOTSPD


@pytest.mark.parametrize("prec", [ae.AMGEIG_FP64, ae.AMGEIG_MIXED_FP32])
def test_negative_fine_mass_gives_enotspd_from_the_pencil(prec):
    """A negative definite finest-level M (the coarse levels untouched, so the load succeeds): the
    Gram block V^T M V of the first finest-level correction has no Cholesky factor, and the solve
    returns ENOTSPD instead of iterating on."""
    _, _, h = problem_and_blob("square", 32, 50, 1)
    bad = _copy(h)
    bad.levels[0].m_vals *= -1.0
    with ae.Hierarchy(hierarchy.to_blob(bad)) as hh:
        with pytest.raises(ae.AmgEigError) as e:
            hh.solve(4, tol=1e-9, opt=ae.options(q_extra=2, precision=prec))
        assert e.value.code == ae.AMGEIG_ENOTSPD


def test_checksum_mismatch_is_corrupt():
    _, blob, _ = problem_and_blob("square", 32, 50, 1)
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x10  # a value bit: layout intact, checksum wrong
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_load_hierarchy(bytes(bad))
    assert e.value.code == ae.AMGEIG_ECORRUPT and "checksum" in str(e.value)


def _poll_all(ids, sizes, timeout=300):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for rid, (n, q) in zip(ids, sizes):
            if rid in out:
                continue
            vals = np.empty(q)
            vecs = np.empty((n, q))
            done, code = ae.amgeig_poll(rid, vals, vecs)
            if done:
                out[rid] = (code, vals, vecs)
        assert time.time() - t0 < timeout
        time.sleep(0.005)
    return [out[r] for r in ids]


def test_service_memory_cap_refuses_and_evicts():
    """Under the service's memory cap a request whose workspace alone exceeds the cap is refused with
    ENOMEM; requests alternating between two hierarchies (two handles of one problem, so that their
    workspaces are alike) whose workspaces do not fit together each release the other's idle workspace
    and give the same bits as a solve run alone."""
    cases = [problem_and_blob("lshape", 16, 60, 2), problem_and_blob("lshape", 16, 60, 2)]
    hs = [ae.Hierarchy(blob) for _, blob, _ in cases]
    # autotune = 0: each handle would tune its own launch shapes, which may add a row's terms in another
    # order; with the rule's shapes every handle of the blob gives the same bits
    opt = ae.options(q_extra=2, max_corrections=40, precision=ae.AMGEIG_MIXED_FP32, autotune=0)
    try:
        alone = [h.solve(4, tol=1e-8, opt=opt) for h in hs]
        # a fresh pair of handles, so that no workspace is resident yet
        for h in hs:
            h.close()
        hs = [ae.Hierarchy(blob) for _, blob, _ in cases]
        ae.amgeig_service_set_memory_limit(1)  # nothing fits
        rid = ae.amgeig_submit(hs[0].handle, 4, 1e-8, opt)
        [(code, _, _)] = _poll_all([rid], [(cases[0][0].n, 4)])
        assert code == ae.AMGEIG_ENOMEM
        # one workspace at a time: measure one, cap just above the larger of the two
        ae.amgeig_service_set_memory_limit(0)
        sizes = []
        for k in (0, 1):
            rid = ae.amgeig_submit(hs[k].handle, 4, 1e-8, opt)
            [(code, _, _)] = _poll_all([rid], [(cases[k][0].n, 4)])
            assert code == ae.AMGEIG_OK
            sizes.append(ae.amgeig_service_memory()[0])
        one = max(sizes[0], sizes[1] - sizes[0])
        assert sizes[1] > 1.2 * one  # the two workspaces do not fit together under the cap below
        # fresh handles again (closing a handle releases its workspace), then the cap
        for h in hs:
            h.close()
        hs = [ae.Hierarchy(blob) for _, blob, _ in cases]
        ae.amgeig_service_set_memory_limit(int(one * 1.2))
        _, ev0 = ae.amgeig_service_memory()
        plan = [0, 1, 0, 1]
        ids = [ae.amgeig_submit(hs[k].handle, 4, 1e-8, opt) for k in plan]
        res = _poll_all(ids, [(cases[k][0].n, 4) for k in plan])
        for k, (code, vals, vecs) in zip(plan, res):
            assert code == ae.AMGEIG_OK
            assert np.array_equal(vals, alone[k][0]) and np.array_equal(vecs, alone[k][1])
        resident, ev1 = ae.amgeig_service_memory()
        assert ev1 - ev0 >= 1 and resident <= int(one * 1.2)
    finally:
        ae.amgeig_service_set_memory_limit(0)
        for h in hs:
            h.close()
