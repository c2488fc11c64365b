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
    # (128, 64) is the largest size the fixed scratch array takes (~452 KiB of 512 KiB)
    for call, (n, nwant, seed) in enumerate([(96, 24, 1), (128, 40, 2), (128, 64, 3)]):
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
        # orthonormality as good as the allocating entry point's on the same matrix (with 64 of 128 pairs
        # of a random spectrum some gaps are small, and both land near 5e-12)
        orth_ref = np.abs(ref_vecs.T @ ref_vecs - np.eye(nwant)).max()
        assert np.abs(V.T @ V - np.eye(nwant)).max() <= max(1e-12, 2.0 * orth_ref)
        # same eigenvectors up to sign (the spectra here have no repeated values)
        assert np.abs(np.abs(np.sum(V * ref_vecs, axis=0)) - 1.0).max() < 1e-10
        assert np.abs(H @ V - V * w).max() <= 1e-11 * scale


def test_noalloc_clean_up_group_matches_lapack():
    """41 wanted eigenvalues within 1e-4 ||H|| of each other: one clean-up group of odd width inside the
    one-block solver (its Rayleigh-Ritz step, with a dummy player in every Jacobi round)."""
    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    n, nwant = 120, 41
    rng = np.random.default_rng(11)
    spec = np.sort(np.concatenate([rng.uniform(1.0, 1.5, nwant), rng.uniform(10.0, 1e4, n - nwant)]))
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    H = (Q * spec) @ Q.T
    H = 0.5 * (H + H.T)
    Hd = torch.tensor(H, dtype=torch.float64, device=dev)
    vals = torch.empty(nwant, dtype=torch.float64, device=dev)
    vecs = torch.empty((n, nwant), dtype=torch.float64, device=dev)
    ae.amgeig_sym_eigh_noalloc(Hd, vals, vecs)
    torch.cuda.synchronize()
    w = vals.cpu().numpy()
    V = vecs.cpu().numpy()
    ref = np.linalg.eigvalsh(H)[:nwant]
    scale = np.abs(spec).max()
    assert np.all(np.abs(w - ref) <= 1e-12 * scale), np.abs(w - ref).max() / scale
    assert np.abs(V.T @ V - np.eye(nwant)).max() < 1e-12
    assert np.abs(H @ V - V * w).max() <= 1e-11 * scale


def test_noalloc_on_a_side_stream():
    """The call only enqueues on the given stream; its results are read after that stream synchronises."""
    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    n, nwant = 80, 16
    H = _rand_sym(n, 7)
    ref_vals, _ = ae.amgeig_sym_eigh(H, nwant)
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(side):
        Hd = torch.tensor(H, dtype=torch.float64, device=dev)
        vals = torch.empty(nwant, dtype=torch.float64, device=dev)
        vecs = torch.empty((n, nwant), dtype=torch.float64, device=dev)
        ae.amgeig_sym_eigh_noalloc(Hd, vals, vecs, stream=torch.cuda.current_stream().cuda_stream)
    side.synchronize()
    w = vals.cpu().numpy()
    assert np.all(np.abs(w - ref_vals) <= 1e-12 * np.abs(ref_vals).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import ctypes

    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    for n, nwant in ((129, 4), (128, 65)):
        H = torch.eye(n, dtype=torch.float64, device=dev)
        vals = torch.empty(nwant, dtype=torch.float64, device=dev)
        vecs = torch.empty((n, nwant), dtype=torch.float64, device=dev)
        with pytest.raises(ae.AmgEigError) as e:
            ae.amgeig_sym_eigh_noalloc(H, vals, vecs)
        assert e.value.code == ae.AMGEIG_EINVAL
        # the library's own message, not the text of an earlier call
        assert "scratch" in ae.lib().amgeig_last_error().decode()
    # through the C ABI directly as well (no binding-side checks in the way)
    L = ae.lib()
    code = L.amgeig_sym_eigh_noalloc(128, 65, ctypes.c_void_p(H.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                     ctypes.c_void_p(vecs.data_ptr()), None)
    assert code == ae.AMGEIG_EINVAL


def test_noalloc_binding_rejects_mis_shaped_or_host_buffers():
    """A mis-shaped output or a host tensor never reaches the library (it would be written out of bounds or
    handed to a kernel as a host pointer)."""
    import torch

    from paper_1503_08462_gb300 import amgeig as ae

    dev = torch.device("cuda:0")
    H = torch.eye(32, dtype=torch.float64, device=dev)
    vals = torch.empty(8, dtype=torch.float64, device=dev)
    launches = ae.amgeig_kernel_launches()
    bad = [
        (H, vals, torch.empty((32, 4), dtype=torch.float64, device=dev)),  # evecs too narrow
        (H[:, :16].contiguous(), vals, torch.empty((32, 8), dtype=torch.float64, device=dev)),  # H not square
        (H.cpu(), vals, torch.empty((32, 8), dtype=torch.float64, device=dev)),  # H on the host
        (H, vals, torch.empty((32, 8), dtype=torch.float64)),  # evecs on the host
    ]
    for args in bad:
        with pytest.raises(ae.AmgEigError) as e:
            ae.amgeig_sym_eigh_noalloc(*args)
        assert e.value.code == ae.AMGEIG_EINVAL
    assert ae.amgeig_kernel_launches() == launches
