"""Thin ctypes binding of the C ABI in include/amgeig.h (argument marshalling only).

Every function here forwards to ``libamgeig.so``; no step of the solve runs in
Python.  Arrays may be NumPy arrays (host) or torch tensors (host or CUDA); they
must be C-contiguous float64.  If the library has not been built the import of
any entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import _build

AMGEIG_OK = 0
AMGEIG_EINVAL = -1
AMGEIG_ECORRUPT = -2
AMGEIG_ENOMEM = -3
AMGEIG_ENOTSPD = -4
AMGEIG_ENOCONV = -5
AMGEIG_ENAN = -6
AMGEIG_ECUDA = -7
AMGEIG_ENOTFOUND = -8

AMGEIG_FP64 = 0
AMGEIG_MIXED_FP32 = 1
AMGEIG_MIXED_BF16 = 2
AMGEIG_SMOOTHER_L1_JACOBI = 0
AMGEIG_SMOOTHER_GAUSS_SEIDEL = 1


class AmgEigError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (code {code})")
        self.code = code


class amgeig_options(ctypes.Structure):
    _fields_ = [("max_corrections", ctypes.c_int), ("v_cycles", ctypes.c_int), ("pre_sweeps", ctypes.c_int),
                ("post_sweeps", ctypes.c_int), ("q_extra", ctypes.c_int), ("precision", ctypes.c_int),
                ("fixed_corrections", ctypes.c_int), ("coarse_modes", ctypes.c_int), ("smoother", ctypes.c_int),
                ("n1", ctypes.c_int), ("refine", ctypes.c_int), ("graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("batch", ctypes.c_int), ("shift", ctypes.c_double),
                ("krylov", ctypes.c_int)]


class amgeig_prof_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class amgeig_info(ctypes.Structure):
    _fields_ = [("corrections", ctypes.c_int), ("converged", ctypes.c_int), ("n1", ctypes.c_int),
                ("status", ctypes.c_int), ("max_relres", ctypes.c_double), ("dense_fallbacks", ctypes.c_int)]


_lib = None
EXPORTED = ["amgeig_default_options", "amgeig_load_hierarchy", "amgeig_load_hierarchy_modes", "amgeig_free_hierarchy", "amgeig_hierarchy_info",
            "amgeig_solve", "amgeig_submit", "amgeig_poll", "amgeig_strerror", "amgeig_last_error",
            "amgeig_sym_eigh", "amgeig_apply_vcycle", "amgeig_apply_defect", "amgeig_profile_enable",
            "amgeig_profile_read", "amgeig_kernel_launches", "amgeig_sym_eigh_noalloc",
            "amgeig_service_set_memory_limit", "amgeig_service_memory", "amgeig_tuning_report",
            "amgeig_setup_blob", "amgeig_free_blob"]


def library_path() -> str:
    return str(_build.CUDA_LIB)


def lib():
    """Load libamgeig.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libamgeig.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.amgeig_default_options.argtypes = [ctypes.POINTER(amgeig_options)]
        L.amgeig_default_options.restype = None
        L.amgeig_load_hierarchy.argtypes = [vp, ctypes.c_size_t, i32, ctypes.POINTER(vp)]
        L.amgeig_load_hierarchy_modes.argtypes = [vp, ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)]
        L.amgeig_free_hierarchy.argtypes = [vp]
        L.amgeig_hierarchy_info.argtypes = [vp, ctypes.POINTER(i32), vp, i32]
        L.amgeig_solve.argtypes = [vp, i32, dbl, ctypes.POINTER(amgeig_options), vp, vp, i32,
                                   ctypes.POINTER(amgeig_info), vp]
        L.amgeig_submit.argtypes = [vp, i32, dbl, ctypes.POINTER(amgeig_options), ctypes.POINTER(ctypes.c_uint64)]
        L.amgeig_poll.argtypes = [ctypes.c_uint64, ctypes.POINTER(i32), vp, vp, ctypes.POINTER(amgeig_info)]
        L.amgeig_strerror.argtypes = [i32]
        L.amgeig_strerror.restype = ctypes.c_char_p
        L.amgeig_last_error.argtypes = []
        L.amgeig_last_error.restype = ctypes.c_char_p
        L.amgeig_sym_eigh.argtypes = [i32, i32, i32, vp, vp, vp]
        L.amgeig_apply_vcycle.argtypes = [vp, i32, i32, ctypes.POINTER(amgeig_options), vp, vp]
        L.amgeig_apply_defect.argtypes = [vp, i32, i32, ctypes.POINTER(amgeig_options), vp, vp, vp, vp]
        L.amgeig_profile_enable.argtypes = [i32]
        L.amgeig_profile_read.argtypes = [ctypes.POINTER(amgeig_prof_entry), i32, ctypes.POINTER(i32)]
        L.amgeig_sym_eigh_noalloc.argtypes = [i32, i32, vp, vp, vp, vp]
        L.amgeig_sym_eigh_noalloc.restype = i32
        L.amgeig_service_set_memory_limit.argtypes = [ctypes.c_uint64]
        L.amgeig_tuning_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        L.amgeig_setup_blob.argtypes = [ctypes.c_int64, vp, vp, vp, vp, dbl, ctypes.c_int64, i32, i32,
                                        ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_size_t), vp]
        L.amgeig_setup_blob.restype = i32
        L.amgeig_free_blob.argtypes = [vp]
        L.amgeig_free_blob.restype = None
        L.amgeig_service_memory.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
        L.amgeig_kernel_launches.argtypes = []
        L.amgeig_kernel_launches.restype = ctypes.c_uint64
        for name in ("amgeig_load_hierarchy", "amgeig_load_hierarchy_modes", "amgeig_free_hierarchy", "amgeig_hierarchy_info", "amgeig_solve",
                     "amgeig_submit", "amgeig_poll", "amgeig_sym_eigh", "amgeig_apply_vcycle",
                     "amgeig_apply_defect", "amgeig_profile_enable", "amgeig_profile_read",
                     "amgeig_service_set_memory_limit", "amgeig_service_memory", "amgeig_tuning_report"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(code: int, where: str, allow=(AMGEIG_OK,)) -> int:
    if code not in allow:
        L = lib()
        raise AmgEigError(code, where, f"{L.amgeig_strerror(code).decode()}: {L.amgeig_last_error().decode()}")
    return code


def _ptr(a) -> Optional[int]:
    """Data pointer of a C-contiguous float64 NumPy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous float64 array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def amgeig_default_options() -> amgeig_options:
    o = amgeig_options()
    lib().amgeig_default_options(ctypes.byref(o))
    return o


def amgeig_load_hierarchy(blob: bytes, device: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().amgeig_load_hierarchy(buf, len(blob), device, ctypes.byref(h)), "amgeig_load_hierarchy")
    return h


def amgeig_load_hierarchy_modes(blob: bytes, device: int = 0, modes: int = 0) -> ctypes.c_void_p:
    """Load and compute the `modes` lowest coarse eigenpairs during the load (0: all)."""
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(lib().amgeig_load_hierarchy_modes(buf, len(blob), device, modes, ctypes.byref(h)),
           "amgeig_load_hierarchy_modes")
    return h


def amgeig_free_hierarchy(h) -> None:
    _check(lib().amgeig_free_hierarchy(h), "amgeig_free_hierarchy")


def amgeig_hierarchy_info(h):
    n = ctypes.c_int()
    sizes = (ctypes.c_int64 * 64)()
    _check(lib().amgeig_hierarchy_info(h, ctypes.byref(n), sizes, 64), "amgeig_hierarchy_info")
    return [int(sizes[i]) for i in range(n.value)]


def amgeig_solve(h, q: int, tol: float, opt: Optional[amgeig_options], eigvals, eigvecs, eigvecs_on_device: bool,
                 info: Optional[amgeig_info] = None, stream: Optional[int] = None) -> int:
    """Forward to amgeig_solve; returns AMGEIG_OK or AMGEIG_ENOCONV, raises otherwise."""
    code = lib().amgeig_solve(h, q, tol, ctypes.byref(opt) if opt is not None else None, _ptr(eigvals),
                              _ptr(eigvecs), 1 if eigvecs_on_device else 0,
                              ctypes.byref(info) if info is not None else None, stream)
    return _check(code, "amgeig_solve", allow=(AMGEIG_OK, AMGEIG_ENOCONV))


def amgeig_submit(h, q: int, tol: float, opt: Optional[amgeig_options] = None) -> int:
    rid = ctypes.c_uint64()
    _check(lib().amgeig_submit(h, q, tol, ctypes.byref(opt) if opt is not None else None, ctypes.byref(rid)),
           "amgeig_submit")
    return rid.value


def amgeig_poll(request_id: int, eigvals=None, eigvecs=None, info: Optional[amgeig_info] = None) -> Tuple[bool, int]:
    done = ctypes.c_int()
    code = lib().amgeig_poll(request_id, ctypes.byref(done), _ptr(eigvals), _ptr(eigvecs),
                             ctypes.byref(info) if info is not None else None)
    if done.value == 0:
        _check(code, "amgeig_poll")
        return False, code
    return True, code


def amgeig_service_set_memory_limit(nbytes: int) -> None:
    _check(lib().amgeig_service_set_memory_limit(nbytes), "amgeig_service_set_memory_limit")


def amgeig_tuning_report(h) -> list:
    """The launch-shape tuner's choices on hierarchy h (parsed JSON)."""
    import json

    buf = ctypes.create_string_buffer(1 << 20)
    _check(lib().amgeig_tuning_report(h, buf, len(buf)), "amgeig_tuning_report")
    return json.loads(buf.value.decode())


def amgeig_setup_blob(row_ptr, col_idx, a_vals, m_vals, theta: float = 0.25, coarse_cap: int = 50,
                      max_levels: int = 25, device: int = 0):
    """The hierarchy blob of (A, M) built by the device setup; returns (blob bytes, total s, C/F split s)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    av = np.ascontiguousarray(a_vals, dtype=np.float64)
    mv = np.ascontiguousarray(m_vals, dtype=np.float64)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    secs = np.zeros(2)
    L = lib()
    _check(L.amgeig_setup_blob(rp.shape[0] - 1, rp.ctypes.data, ci.ctypes.data, av.ctypes.data, mv.ctypes.data,
                               theta, coarse_cap, max_levels, device, ctypes.byref(out), ctypes.byref(nbytes),
                               secs.ctypes.data), "amgeig_setup_blob")
    try:
        # numpy view of the library's buffer, copied once (ctypes.string_at cannot take 2 GB and more)
        view = np.ctypeslib.as_array((ctypes.c_uint8 * nbytes.value).from_address(out.value))
        blob = view.tobytes()
    finally:
        L.amgeig_free_blob(out)
    return blob, float(secs[0]), float(secs[1])


def amgeig_service_memory() -> Tuple[int, int]:
    """(bytes held by the service's resident workspaces, workspaces released so far to admit others)."""
    rb = ctypes.c_uint64()
    ev = ctypes.c_uint64()
    _check(lib().amgeig_service_memory(ctypes.byref(rb), ctypes.byref(ev)), "amgeig_service_memory")
    return int(rb.value), int(ev.value)


def amgeig_sym_eigh(H: np.ndarray, nwant: int, device: int = 0):
    H = np.ascontiguousarray(H, dtype=np.float64)
    n = H.shape[0]
    evals = np.empty(nwant)
    evecs = np.empty((n, nwant))
    _check(lib().amgeig_sym_eigh(device, n, nwant, _ptr(H), _ptr(evals), _ptr(evecs)), "amgeig_sym_eigh")
    return evals, evecs


def amgeig_sym_eigh_noalloc(H, evals, evecs, stream: Optional[int] = None) -> None:
    """Device-pointer form without allocation: H (n x n), evals (nwant), evecs (n x nwant) CUDA float64 tensors
    on the current CUDA device.  Shapes and devices are checked here, before any pointer reaches the library:
    a mis-shaped output would be written out of bounds on the device."""
    import torch

    tensors = (H, evals, evecs)
    if not all(isinstance(t, torch.Tensor) for t in tensors):
        raise AmgEigError(AMGEIG_EINVAL, "amgeig_sym_eigh_noalloc", "H, evals and evecs must be torch tensors")
    if H.dim() != 2 or H.shape[0] != H.shape[1] or evals.dim() != 1 or evecs.dim() != 2:
        raise AmgEigError(AMGEIG_EINVAL, "amgeig_sym_eigh_noalloc", "H must be n x n, evals 1-D, evecs 2-D")
    n = H.shape[0]
    nwant = evals.shape[0]
    if tuple(evecs.shape) != (n, nwant):
        raise AmgEigError(AMGEIG_EINVAL, "amgeig_sym_eigh_noalloc",
                          f"evecs has shape {tuple(evecs.shape)}, expected ({n}, {nwant})")
    cur = torch.cuda.current_device()
    if not all(t.is_cuda and t.device.index == cur for t in tensors):
        raise AmgEigError(AMGEIG_EINVAL, "amgeig_sym_eigh_noalloc",
                          f"H, evals and evecs must be CUDA tensors on the current device cuda:{cur}")
    _check(lib().amgeig_sym_eigh_noalloc(n, nwant, _ptr(H), _ptr(evals), _ptr(evecs), stream),
           "amgeig_sym_eigh_noalloc")


def amgeig_apply_defect(h, level: int, U: np.ndarray, lam: np.ndarray, opt: Optional[amgeig_options] = None):
    """(R, relres): r_j = lam_j M u_j - A u_j on `level` and the relative residuals."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    R = np.empty_like(U)
    rr = np.empty(U.shape[1])
    _check(lib().amgeig_apply_defect(h, level, U.shape[1], ctypes.byref(opt) if opt is not None else None, _ptr(U),
                                     _ptr(lam), _ptr(R), _ptr(rr)), "amgeig_apply_defect")
    return R, rr


def amgeig_apply_vcycle(h, level: int, b: np.ndarray, opt: Optional[amgeig_options] = None) -> np.ndarray:
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    _check(lib().amgeig_apply_vcycle(h, level, b.shape[1], ctypes.byref(opt) if opt is not None else None, _ptr(b),
                                     _ptr(x)), "amgeig_apply_vcycle")
    return x


def amgeig_profile_enable(enable: bool) -> None:
    _check(lib().amgeig_profile_enable(1 if enable else 0), "amgeig_profile_enable")


def amgeig_profile_read():
    """Per kernel class totals: {name: dict(launches, kernels, total_ms, bytes, flops)}."""
    buf = (amgeig_prof_entry * 512)()
    n = ctypes.c_int()
    _check(lib().amgeig_profile_read(buf, 512, ctypes.byref(n)), "amgeig_profile_read")
    return {buf[i].name.decode(): dict(launches=buf[i].launches, kernels=buf[i].kernels, total_ms=buf[i].total_ms,
                                       bytes=buf[i].bytes, flops=buf[i].flops) for i in range(n.value)}


def amgeig_kernel_launches() -> int:
    return int(lib().amgeig_kernel_launches())


def strerror(code: int) -> str:
    return lib().amgeig_strerror(code).decode()


# ---------------------------------------------------------------- convenience


def options(**kw) -> amgeig_options:
    o = amgeig_default_options()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


class Hierarchy:
    """Owns a loaded hierarchy handle (amgeig_load_hierarchy / amgeig_free_hierarchy).

    modes: None computes the coarse eigenbasis on the first solve; an int computes that
    many lowest coarse modes during the load (amgeig_load_hierarchy_modes, 0: all)."""

    def __init__(self, blob: bytes, device: int = 0, modes: Optional[int] = None):
        if modes is None:
            self.handle = amgeig_load_hierarchy(blob, device)
        else:
            self.handle = amgeig_load_hierarchy_modes(blob, device, modes)
        self.sizes = amgeig_hierarchy_info(self.handle)

    def solve(self, q: int, tol: float = 1e-10, opt: Optional[amgeig_options] = None, vectors: bool = True):
        """Return (eigvals[q], eigvecs[N0, q] or None, info, status) through amgeig_solve (host buffers)."""
        vals = np.empty(q)
        vecs = np.empty((self.sizes[0], q)) if vectors else None
        info = amgeig_info()
        code = amgeig_solve(self.handle, q, tol, opt, vals, vecs, False, info)
        return vals, vecs, info, code

    def close(self):
        if self.handle is not None:
            amgeig_free_hierarchy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
