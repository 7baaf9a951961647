"""ORACLE - test infrastructure only.

Plain CPU statement (C, single thread per calorimeter-fill) of the muon g-2
DAQ per-fill processing of Sec. 3 / Table 2: pedestals, crystal sum, threshold,
pre/post windows, merge, island save, Q decimation and fill-by-fill sum.  See
daq_oracle.c for the definition it follows, step by step.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "daq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ISLAND_DTYPE = np.dtype([("fill", "<i4"), ("calo", "<i4"), ("start", "<i4"), ("len", "<i4"),
                         ("pool_row", "<i8")])


class OracleParams(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_int32), ("pre", ctypes.c_int32), ("post", ctypes.c_int32),
                ("ped_samples", ctypes.c_int32), ("n_decim", ctypes.c_int32), ("decim", ctypes.c_int32 * 2)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.oracle_pedestal.argtypes = [vp, i64, i32]
    lib.oracle_pedestal.restype = i32
    lib.oracle_calofill.argtypes = [vp, i32, i64, i64, ctypes.POINTER(OracleParams), i32, i32, vp, vp,
                                    vp, vp, i64, i64, vp, i64, vp, vp, vp]
    lib.oracle_calofill.restype = i64
    lib.oracle_process_fills.argtypes = [vp, i32, i32, i32, i64, vp, ctypes.POINTER(OracleParams), vp,
                                         i64, vp, i64, vp, vp, vp, i32]
    lib.oracle_process_fills.restype = ctypes.c_int
    if hasattr(lib, "oracle_pack"):
        lib.oracle_pack.argtypes = [vp, i64, i32, vp, i64]
        lib.oracle_pack.restype = i64
        lib.oracle_unpack.argtypes = [vp, i64, vp, i64, i32]
        lib.oracle_unpack.restype = ctypes.c_int
    if hasattr(lib, "oracle_crystal_sum"):
        lib.oracle_crystal_sum.argtypes = [vp, i32, i32, i32, i64, vp, i32, vp]
        lib.oracle_crystal_sum.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _params(p: dict) -> OracleParams:
    decim = tuple(p.get("decim", ()))
    d = (list(decim) + [0, 0])[:2]
    return OracleParams(int(p["threshold"]), int(p["pre"]), int(p["post"]), int(p.get("ped_samples", 100)),
                        len(decim), (ctypes.c_int32 * 2)(*d))


def _ptr(a):
    return None if a is None else a.ctypes.data


def q_bins(n_samples: int, decim) -> list:
    """Bins per calorimeter for each decimation factor (ceil(n_samples / D))."""
    return [(n_samples + d - 1) // d for d in decim]


class Oracle:
    """The oracle bound to one compiled copy of daq_oracle.c (tests also bind
    deliberately broken copies to show that the pins catch them)."""

    def __init__(self, lib_path: str | None = None):
        self._lib = _bind(lib_path) if lib_path else _load()

    def pedestal(self, row: np.ndarray, length: int | None = None, ped_samples: int = 100) -> int:
        row = np.ascontiguousarray(row, dtype=np.int16)
        length = row.size if length is None else length
        return int(self._lib.oracle_pedestal(row.ctypes.data, length, ped_samples))

    def calofill(self, s: np.ndarray, params: dict, length: int | None = None, fill: int = 0,
                 calo: int = 0) -> dict:
        """Every intermediate of one calorimeter-fill.  s is [n_xtal][pitch] int16."""
        s = np.ascontiguousarray(s, dtype=np.int16)
        n_xtal, pitch = s.shape
        length = pitch if length is None else int(length)
        lib = self._lib
        op = _params(params)
        ped = np.zeros(n_xtal, np.int32)
        S = np.zeros(max(length, 1), np.int64)
        M = np.zeros(max(length, 1), np.uint8)
        isl = np.zeros(length // 2 + 1, ISLAND_DTYPE)
        pool = np.zeros((max(length, 1), n_xtal), np.int16)
        rows = ctypes.c_int64(0)
        nb = q_bins(length, params.get("decim", ()))
        bins = [np.zeros(max(n, 1), np.int64) for n in nb] + [None, None]
        n_isl = lib.oracle_calofill(s.ctypes.data, n_xtal, pitch, length, ctypes.byref(op), fill, calo,
                                    ped.ctypes.data, S.ctypes.data, M.ctypes.data, isl.ctypes.data, isl.size, 0,
                                    pool.ctypes.data, length, ctypes.byref(rows), _ptr(bins[0]), _ptr(bins[1]))
        return dict(pedestal=ped, S=S[:length], mark=M[:length].astype(bool), islands=isl[:n_isl],
                    pool=pool[:rows.value], bins=[b[:n] for b, n in zip(bins, nb)])

    def process_fills(self, samples: np.ndarray, params: dict, fill_len=None, n_threads: int = 1,
                      isl_cap: int | None = None, row_cap: int | None = None,
                      q: np.ndarray | None = None) -> dict:
        """The whole batch samples[F][C][X][pitch].  Q accumulates into `q` if given
        (flat int64: n_calo x ceil(pitch/D0) bins, then n_calo x ceil(pitch/D1))."""
        samples = np.ascontiguousarray(samples, dtype=np.int16)
        F, C, X, N = samples.shape
        decim = tuple(params.get("decim", ()))
        nb = q_bins(N, decim)
        if q is None:
            q = np.zeros(max(1, sum(C * n for n in nb)), np.int64)
        lens = None if fill_len is None else np.ascontiguousarray(fill_len, dtype=np.int32)
        max_rows = int(F * C * N) if lens is None else int(C * np.clip(lens, 0, N).sum())
        isl_cap = max_rows // 2 + F * C + 1 if isl_cap is None else isl_cap
        row_cap = max_rows if row_cap is None else row_cap
        isl = np.zeros(max(isl_cap, 1), ISLAND_DTYPE)
        pool = np.zeros((max(row_cap, 1), X), np.int16)
        ped = np.zeros((F, C, X), np.int32)
        counts = np.zeros(2, np.int64)
        op = _params(params)
        rc = self._lib.oracle_process_fills(samples.ctypes.data, F, C, X, N, _ptr(lens), ctypes.byref(op),
                                            isl.ctypes.data, isl_cap, pool.ctypes.data, row_cap,
                                            ped.ctypes.data, q.ctypes.data, counts.ctypes.data, int(n_threads))
        if rc != 0:
            raise ValueError("oracle rejected the arguments")
        n_isl, n_rows = int(counts[0]), int(counts[1])
        return dict(islands=isl[:min(n_isl, isl_cap)], pool=pool[:min(n_rows, row_cap)], pedestal=ped, q=q,
                    n_islands=n_isl, n_rows=n_rows)


    def crystal_sum(self, samples: np.ndarray, fill_len=None, ped_samples: int = 100,
                    q: np.ndarray | None = None) -> np.ndarray:
        """Per-crystal full-resolution fill sum of samples[F][C][X][pitch]:
        q[c][x][t] (int64) += s - pedestal over every fill, t < the fill's length."""
        samples = np.ascontiguousarray(samples, dtype=np.int16)
        F, C, X, N = samples.shape
        if q is None:
            q = np.zeros((C, X, N), np.int64)
        assert q.dtype == np.int64 and q.flags.c_contiguous and q.shape == (C, X, N)
        lens = None if fill_len is None else np.ascontiguousarray(fill_len, dtype=np.int32)
        rc = self._lib.oracle_crystal_sum(samples.ctypes.data, F, C, X, N, _ptr(lens), int(ped_samples),
                                          q.ctypes.data)
        if rc != 0:
            raise ValueError("oracle rejected the arguments")
        return q


    def pack(self, pool: np.ndarray) -> np.ndarray:
        """Packed stream (uint8) of pool rows [rows][n_xtal] int16."""
        pool = np.ascontiguousarray(pool, dtype=np.int16)
        rows, X = pool.shape
        n = int(self._lib.oracle_pack(pool.ctypes.data, rows, X, None, 0))
        if n < 0:
            raise ValueError("oracle rejected the arguments")
        out = np.zeros(n, np.uint8)
        self._lib.oracle_pack(pool.ctypes.data, rows, X, out.ctypes.data, n)
        return out

    def unpack(self, stream: np.ndarray, rows: int, n_xtal: int) -> np.ndarray:
        stream = np.ascontiguousarray(stream, dtype=np.uint8)
        out = np.zeros((rows, n_xtal), np.int16)
        if self._lib.oracle_unpack(stream.ctypes.data, stream.size, out.ctypes.data, rows, n_xtal) != 0:
            raise ValueError("malformed packed stream")
        return out


_default = None


def _oracle() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def pedestal(*a, **k) -> int:
    return _oracle().pedestal(*a, **k)


def calofill(*a, **k) -> dict:
    return _oracle().calofill(*a, **k)


def process_fills(*a, **k) -> dict:
    return _oracle().process_fills(*a, **k)


def crystal_sum(*a, **k) -> np.ndarray:
    return _oracle().crystal_sum(*a, **k)


def pack(*a, **k) -> np.ndarray:
    return _oracle().pack(*a, **k)


def unpack(*a, **k) -> np.ndarray:
    return _oracle().unpack(*a, **k)
