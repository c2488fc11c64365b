"""The C-ABI library builds, loads and exports every symbol its header declares (CPU only)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols():
    names = set()
    for hdr in (ROOT / "include").glob("*.h"):
        text = hdr.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|const char\*|uint64_t)\s+(amgeig_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("amgeig_load_hierarchy", "amgeig_free_hierarchy", "amgeig_solve", "amgeig_submit",
                     "amgeig_poll", "amgeig_strerror"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1503_08462_gb300 import _build

    path = _build.build_cuda_lib()
    lib = ctypes.CDLL(str(path))  # loads without a GPU
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1503_08462_gb300 import amgeig

    assert set(amgeig.EXPORTED) == declared_symbols()


def test_host_only_calls_without_gpu():
    from paper_1503_08462_gb300 import amgeig

    o = amgeig.amgeig_default_options()
    assert (o.max_corrections, o.v_cycles, o.pre_sweeps, o.post_sweeps) == (20, 1, 1, 1)
    assert amgeig.strerror(amgeig.AMGEIG_ENOCONV).startswith("not converged")


def test_argument_errors_need_no_gpu():
    """Argument checks return their error codes before any CUDA call: a negative
    mode count and NULL pointers are EINVAL with a message, on any machine."""
    import ctypes

    from paper_1503_08462_gb300 import amgeig

    with pytest.raises(amgeig.AmgEigError) as e:
        amgeig.amgeig_load_hierarchy_modes(b"AMGEIGH1" + bytes(16), 0, -1)
    assert e.value.code == amgeig.AMGEIG_EINVAL and "modes" in str(e.value)
    L = amgeig.lib()
    h = ctypes.c_void_p()
    assert L.amgeig_load_hierarchy(None, 0, 0, ctypes.byref(h)) == amgeig.AMGEIG_EINVAL
    assert L.amgeig_load_hierarchy_modes(None, 0, 0, 4, ctypes.byref(h)) == amgeig.AMGEIG_EINVAL
    assert b"NULL" in L.amgeig_last_error()


def test_malformed_blobs_are_refused_by_the_loader_without_a_gpu():
    """The loader checks the blob's layout on the host before it touches a device: a truncated blob, a
    wrong magic, a bad version and trailing bytes are ECORRUPT on any machine (the checksum and every
    level's CSR are checked by the GPU loader, in the GPU tests)."""
    import ctypes

    from paper_1503_08462_gb300 import amgeig
    from paper_1503_08462_gb300.inputs import hierarchy, meshes

    blob, _ = hierarchy.problem_blob(meshes.square_2d(8, seed=1), coarse_cap=10)
    L = amgeig.lib()
    h = ctypes.c_void_p()

    def load(b):
        buf = ctypes.create_string_buffer(b, len(b))
        return L.amgeig_load_hierarchy(buf, len(b), 0, ctypes.byref(h))

    cut = len(blob) // 2 // 8 * 8
    assert load(blob[:cut]) == amgeig.AMGEIG_ECORRUPT
    assert b"truncated" in L.amgeig_last_error()
    assert load(b"AMGEIGH0" + blob[8:]) == amgeig.AMGEIG_ECORRUPT
    bad_version = blob[:8] + (7).to_bytes(4, "little") + blob[12:]
    assert load(bad_version) == amgeig.AMGEIG_ECORRUPT
    assert load(blob[:-8] + bytes(8) + blob[-8:]) == amgeig.AMGEIG_ECORRUPT
    assert load(blob[:-3]) == amgeig.AMGEIG_ECORRUPT  # not a whole number of words
