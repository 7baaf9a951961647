"""Seeded synthetic muon g-2 calorimeter waveforms (input generator).

This module feeds both the oracle and the CUDA path.  It holds none of the
method's arithmetic: it writes int16 samples shaped like the fills of Sec. 3
(24 calorimeters x 9x6 crystals, 800 MSPS 12-bit samples, 700 us fills) and
nothing else.  The C source (synth.c) documents the model; `workloads.py`
holds the concrete workload recipes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class SynthConfig(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_fills", ctypes.c_int32), ("n_calo", ctypes.c_int32),
        ("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32),
        ("n_samples", ctypes.c_int64),
        ("noise_sigma", ctypes.c_double),
        ("ped_lo", ctypes.c_int32), ("ped_hi", ctypes.c_int32),
        ("pulses_per_fill", ctypes.c_double),
        ("nominal_samples", ctypes.c_double),
        ("amp_lo", ctypes.c_double), ("amp_hi", ctypes.c_double),
        ("rise_ns", ctypes.c_double), ("decay_ns", ctypes.c_double), ("sample_ns", ctypes.c_double),
        ("tau_us", ctypes.c_double), ("osc_period_us", ctypes.c_double), ("osc_amp", ctypes.c_double),
        ("profile_sigma", ctypes.c_double),
        ("quiet_samples", ctypes.c_int32),
        ("beyond_value", ctypes.c_int32),
        ("tail_samples", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


PULSE_DTYPE = np.dtype([("arrival", "<f8"), ("amplitude", "<f8"), ("centre", "<i4"), ("reserved", "<i4")])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.synth_generate.argtypes = [P(SynthConfig), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int]
            lib.synth_generate.restype = ctypes.c_int
            lib.synth_generate_fills.argtypes = [P(SynthConfig), ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.synth_generate_fills.restype = ctypes.c_int
            lib.synth_fill_plan.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_fill_plan.restype = ctypes.c_int
            lib.synth_pulses.argtypes = [P(SynthConfig), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_int64]
            lib.synth_pulses.restype = ctypes.c_int64
            lib.synth_true_pedestal.argtypes = [P(SynthConfig), ctypes.c_int32, ctypes.c_int32]
            lib.synth_true_pedestal.restype = ctypes.c_int32
            for name in ("synth_exp", "synth_log", "synth_cos", "synth_phi"):
                getattr(lib, name).argtypes = [ctypes.c_double]
                getattr(lib, name).restype = ctypes.c_double
            lib.synth_noise_hist.argtypes = [ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_int]
            lib.synth_noise_hist.restype = ctypes.c_int
            _lib = lib
    return _lib


def make_config(**kw) -> SynthConfig:
    """Defaults reproduce one nominal muon fill of one calorimeter."""
    d = dict(seed=1611_04959, n_fills=1, n_calo=1, n_rows=6, n_cols=9, n_samples=560_000,
             noise_sigma=3.0, ped_lo=1700, ped_hi=1900, pulses_per_fill=1500.0, nominal_samples=560_000.0,
             amp_lo=50.0, amp_hi=2000.0, rise_ns=2.0, decay_ns=5.0, sample_ns=1.25, tau_us=64.4,
             osc_period_us=4.365, osc_amp=0.4, profile_sigma=1.0, quiet_samples=108, beyond_value=4095,
             tail_samples=64, reserved=0)
    d.update(kw)
    return SynthConfig(**d)


def generate(cfg: SynthConfig, fill_len=None, rate=None, out=None, n_threads: int = 0, fills=None) -> np.ndarray:
    """Return (or fill) samples[n_fills][n_calo][n_rows*n_cols][n_samples] int16.

    `fills` = (f0, n) generates only fills f0 .. f0 + n - 1 (their bytes equal
    those of a whole-batch call; fill_len / rate stay indexed by the absolute
    fill).  `out` may be any C-contiguous int16 buffer of that size (e.g. a
    pinned host tensor's numpy view)."""
    lib = _load()
    f0, nf = (0, cfg.n_fills) if fills is None else (int(fills[0]), int(fills[1]))
    shape = (nf, cfg.n_calo, cfg.n_rows * cfg.n_cols, cfg.n_samples)
    if out is None:
        out = np.empty(shape, dtype=np.int16)
    assert out.dtype == np.int16 and out.flags.c_contiguous and out.size == int(np.prod(shape))
    fl = None if fill_len is None else np.ascontiguousarray(fill_len, dtype=np.int32)
    rt = None if rate is None else np.ascontiguousarray(rate, dtype=np.float64)
    rc = lib.synth_generate_fills(ctypes.byref(cfg), f0, nf, None if fl is None else fl.ctypes.data,
                                  None if rt is None else rt.ctypes.data, out.ctypes.data, int(n_threads))
    if rc != 0:
        raise ValueError("synth_generate_fills rejected the configuration")
    return out


def fill_plan(seed: int, n_fills: int, len_lo: int, len_hi: int, rate_lo: float, rate_hi: float):
    """Uneven batch: per-fill lengths (uniform integers) and rate factors (log-uniform)."""
    lib = _load()
    ln = np.empty(n_fills, dtype=np.int32)
    rt = np.empty(n_fills, dtype=np.float64)
    if lib.synth_fill_plan(seed, n_fills, len_lo, len_hi, rate_lo, rate_hi, ln.ctypes.data, rt.ctypes.data):
        raise ValueError("bad fill plan")
    return ln, rt


def pulses(cfg: SynthConfig, fill: int, calo: int, length: int | None = None, rate: float = 1.0) -> np.ndarray:
    """Truth pulse list of one calorimeter-fill (arrival in samples, amplitude, centre crystal)."""
    lib = _load()
    length = cfg.n_samples if length is None else length
    n = lib.synth_pulses(ctypes.byref(cfg), fill, calo, length, rate, None, 0)
    out = np.zeros(n, dtype=PULSE_DTYPE)
    if n:
        lib.synth_pulses(ctypes.byref(cfg), fill, calo, length, rate, out.ctypes.data, n)
    return out


def true_pedestal(cfg: SynthConfig, calo: int, xtal: int) -> int:
    return int(_load().synth_true_pedestal(ctypes.byref(cfg), calo, xtal))


def noise_hist(sigma: float, seed: int, n: int, k_max: int) -> np.ndarray:
    h = np.zeros(2 * k_max + 1, dtype=np.int64)
    _load().synth_noise_hist(sigma, seed, n, h.ctypes.data, k_max)
    return h


def elementary(name: str, x: float) -> float:
    return float(getattr(_load(), "synth_" + name)(x))
