"""AMG hierarchy construction (host) and the serialized hierarchy blob.

The setup of Sec. 2 (strength with theta, Ruge-Stueben splitting, direct
interpolation, Galerkin A_{k+1} = P^T A_k P and M_{k+1} = P^T M_k P) runs once in
the native host library ``libamgsetup.so``; its output is written as a blob
that both the CUDA solve path and the CPU oracle read with their own parsers.

Blob layout (little-endian, version 1):
  magic      8 bytes  b"AMGEIGH1"
  version    u32      1
  n_levels   u32      n (level 0 is the finest, level n-1 the coarsest)
  rows       u64[n]   N_l
  nnz        u64[n]   nnz of A_l (= nnz of M_l, one shared pattern)
  nnz_p      u64[n-1] nnz of P_l (N_l x N_{l+1})
  then, each array starting on an 8-byte boundary (zero padding between):
    for l in 0..n-1:  row_ptr int32[N_l+1], col int32[nnz_l], A f64[nnz_l], M f64[nnz_l]
    for l in 0..n-2:  row_ptr int32[N_l+1], col int32[nnz_p_l], P f64[nnz_p_l]
  checksum   u64      sum of all preceding 8-byte little-endian words, mod 2^64
"""
from __future__ import annotations

import ctypes
import dataclasses
import struct
from typing import List, Tuple

import numpy as np

from .. import _build

MAGIC = b"AMGEIGH1"
VERSION = 1

_lib = None


def _setup_lib():
    global _lib
    if _lib is None:
        path = _build.build_setup_lib()
        lib = ctypes.CDLL(str(path))
        i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.amgsetup_build.argtypes = [i64, vp, vp, vp, vp, ctypes.c_double, i64, i32, ctypes.POINTER(vp)]
        lib.amgsetup_build.restype = ctypes.c_int
        lib.amgsetup_num_levels.argtypes = [vp]
        lib.amgsetup_num_levels.restype = i32
        lib.amgsetup_level_sizes.argtypes = [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.amgsetup_get_level.argtypes = [vp, i32, vp, vp, vp, vp]
        lib.amgsetup_get_prolongation.argtypes = [vp, i32, vp, vp, vp]
        lib.amgsetup_free.argtypes = [vp]
        lib.amgsetup_free.restype = None
        _lib = lib
    return _lib


@dataclasses.dataclass
class Level:
    row_ptr: np.ndarray
    col_idx: np.ndarray
    a_vals: np.ndarray
    m_vals: np.ndarray

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)


@dataclasses.dataclass
class Transfer:
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray
    n_cols: int


@dataclasses.dataclass
class Hierarchy:
    levels: List[Level]
    prolong: List[Transfer]

    @property
    def sizes(self) -> List[int]:
        return [lv.n for lv in self.levels]

    def operator_complexity(self) -> float:
        return sum(lv.col_idx.shape[0] for lv in self.levels) / self.levels[0].col_idx.shape[0]

    def grid_complexity(self) -> float:
        return sum(self.sizes) / self.sizes[0]


def build_hierarchy(row_ptr, col_idx, a_vals, m_vals, theta: float = 0.25, coarse_cap: int = 50,
                    max_levels: int = 25) -> Hierarchy:
    """Run the AMG setup on (A, M) given in shared-pattern CSR."""
    lib = _setup_lib()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    av = np.ascontiguousarray(a_vals, dtype=np.float64)
    mv = np.ascontiguousarray(m_vals, dtype=np.float64)
    n = rp.shape[0] - 1
    h = ctypes.c_void_p()
    rc = lib.amgsetup_build(n, rp.ctypes.data, ci.ctypes.data, av.ctypes.data, mv.ctypes.data, theta,
                            coarse_cap, max_levels, ctypes.byref(h))
    if rc != 0:
        raise ValueError(f"amgsetup_build failed ({rc})")
    try:
        nl = lib.amgsetup_num_levels(h)
        levels, prolong = [], []
        sizes = []
        for l in range(nl):
            rows, nnz, nnzp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            lib.amgsetup_level_sizes(h, l, ctypes.byref(rows), ctypes.byref(nnz), ctypes.byref(nnzp))
            sizes.append((rows.value, nnz.value, nnzp.value))
        for l, (rows, nnz, _) in enumerate(sizes):
            lrp = np.empty(rows + 1, np.int32)
            lci = np.empty(nnz, np.int32)
            la = np.empty(nnz, np.float64)
            lm = np.empty(nnz, np.float64)
            lib.amgsetup_get_level(h, l, lrp.ctypes.data, lci.ctypes.data, la.ctypes.data, lm.ctypes.data)
            levels.append(Level(lrp, lci, la, lm))
        for l in range(nl - 1):
            rows, _, nnzp = sizes[l]
            prp = np.empty(rows + 1, np.int32)
            pci = np.empty(nnzp, np.int32)
            pv = np.empty(nnzp, np.float64)
            lib.amgsetup_get_prolongation(h, l, prp.ctypes.data, pci.ctypes.data, pv.ctypes.data)
            prolong.append(Transfer(prp, pci, pv, sizes[l + 1][0]))
    finally:
        lib.amgsetup_free(h)
    return Hierarchy(levels, prolong)


def build_for_problem(problem, theta: float = 0.25, coarse_cap: int = 50, max_levels: int = 25) -> Hierarchy:
    return build_hierarchy(problem.row_ptr, problem.col_idx, problem.a_vals, problem.m_vals, theta,
                           coarse_cap, max_levels)


def _pad8(b: bytearray) -> None:
    b.extend(b"\0" * ((-len(b)) % 8))


def to_blob(h: Hierarchy) -> bytes:
    """Serialize a hierarchy in the layout given in the module docstring."""
    n = len(h.levels)
    out = bytearray()
    out += MAGIC
    out += struct.pack("<II", VERSION, n)
    out += struct.pack(f"<{n}Q", *[lv.n for lv in h.levels])
    out += struct.pack(f"<{n}Q", *[lv.col_idx.shape[0] for lv in h.levels])
    if n > 1:
        out += struct.pack(f"<{n - 1}Q", *[p.col_idx.shape[0] for p in h.prolong])
    _pad8(out)
    for lv in h.levels:
        for arr, dt in ((lv.row_ptr, "<i4"), (lv.col_idx, "<i4"), (lv.a_vals, "<f8"), (lv.m_vals, "<f8")):
            out += np.ascontiguousarray(arr, dtype=dt).tobytes()
            _pad8(out)
    for p in h.prolong:
        for arr, dt in ((p.row_ptr, "<i4"), (p.col_idx, "<i4"), (p.vals, "<f8")):
            out += np.ascontiguousarray(arr, dtype=dt).tobytes()
            _pad8(out)
    words = np.frombuffer(bytes(out), dtype="<u8")
    checksum = int(words.sum(dtype=np.uint64))
    out += struct.pack("<Q", checksum)
    return bytes(out)


def problem_blob(problem, coarse_cap: int, theta: float = 0.25, max_levels: int = 25) -> Tuple[bytes, Hierarchy]:
    h = build_for_problem(problem, theta=theta, coarse_cap=coarse_cap, max_levels=max_levels)
    return to_blob(h), h
