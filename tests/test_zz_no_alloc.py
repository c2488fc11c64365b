"""The allocation-free eigensolver entry point (amgeig_sym_eigh_noalloc).

It serves callers that cannot allocate device memory when they need the
eigensolver; its scratch is a fixed file-scope device array shared by all
calls.  This file is collected last so that a run stopping at the first
failure has already run every other test.  The test calls the entry point
through the C ABI twice in a row on device buffers and checks each result
against the allocating entry point amgeig_sym_eigh within the tolerance the
eigensolver tests use.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _rand_sym(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    spec = np.sort(rng.uniform(0.5, 100.0, n))
    H = (Q * spec) @ Q.T
    return 0.5 * (H + H.T)


def test_noalloc_matches_allocating_entry_point_twice():
    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    for call, (n, nwant, seed) in enumerate([(96, 24, 1), (128, 40, 2)]):
        H = _rand_sym(n, seed)
        ref_vals, ref_vecs = ae.amgeig_sym_eigh(H, nwant)
        Hd = torch.tensor(H, dtype=torch.float64, device=dev)
        vals = torch.empty(nwant, dtype=torch.float64, device=dev)
        vecs = torch.empty((n, nwant), dtype=torch.float64, device=dev)
        ae.amgeig_sym_eigh_noalloc(Hd, vals, vecs)
        torch.cuda.synchronize()
        w = vals.cpu().numpy()
        V = vecs.cpu().numpy()
        scale = np.abs(ref_vals).max()
        assert np.all(np.abs(w - ref_vals) <= 1e-12 * scale), (call, np.abs(w - ref_vals).max())
        assert np.abs(V.T @ V - np.eye(nwant)).max() < 1e-12
        # same eigenvectors up to sign (the spectra here have no repeated values)
        assert np.abs(np.abs(np.sum(V * ref_vecs, axis=0)) - 1.0).max() < 1e-10
        assert np.abs(H @ V - V * w).max() <= 1e-11 * scale


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    H = torch.eye(129, dtype=torch.float64, device=dev)
    vals = torch.empty(4, dtype=torch.float64, device=dev)
    vecs = torch.empty((129, 4), dtype=torch.float64, device=dev)
    with pytest.raises(ae.AmgEigError) as e:
        ae.amgeig_sym_eigh_noalloc(H, vals, vecs)
    assert e.value.code == ae.AMGEIG_EINVAL
