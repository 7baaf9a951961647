"""Island-finding efficiency across thresholds (arXiv:1611.04959, Sec. 3, Fig. 2).

Fig. 2 plots, for several thresholds, the islands identified in each dataset
against the dataset's truth islands: above the noise the two agree (slope 1).
Here a dataset is one calorimeter-fill.  The identified islands are those the
CUDA path finds in the data; the truth islands are built from the list of
pulses that were injected into it:

  - a pulse of summed amplitude A arriving at sample a adds A * shape(dt) to
    the pedestal-subtracted crystal sum at sample n, dt = (n - a) * sample_ns,
    with shape rising linearly from 0 to 1 over rise_ns and then decaying as
    exp(-(dt - rise_ns) / decay_ns) (the workload's pulse definition);
  - on its own it crosses a threshold T at the samples where A * shape > T: a
    single run of samples around its peak, empty when A <= T;
  - each crossing run [n0, n1] is widened to [n0 - pre, n1 + post] and the
    widened runs of a dataset are merged where they overlap or touch, clipped
    to the fill, exactly as the method merges its windows.

These truth islands ignore what the data add to a pulse: noise, rounding of
each crystal's share, and the sum of overlapping pulses.  They are the truth
of the pulse list, independent of the path under test.
"""
from __future__ import annotations

import math

import numpy as np

from . import process_fills


def crossing_runs(arrival, amplitude, threshold: float, length: int, rise_ns: float = 2.0, decay_ns: float = 5.0,
                  sample_ns: float = 1.25) -> np.ndarray:
    """[first, last] sample (int64 [n][2]) at which each pulse alone exceeds the
    threshold, for the pulses that do and whose run reaches [0, length)."""
    a = np.asarray(arrival, np.float64)
    amp = np.asarray(amplitude, np.float64)
    keep = amp > threshold
    a, amp = a[keep], amp[keep]
    if a.size == 0:
        return np.zeros((0, 2), np.int64)
    r = threshold / amp if threshold > 0 else np.zeros_like(amp)
    # shape > r for dt in (r * rise, rise + decay * ln(1 / r)) (the whole tail when r <= 0)
    lo_ns = np.maximum(r, 0.0) * rise_ns
    with np.errstate(divide="ignore"):
        hi_ns = np.where(r > 0, rise_ns + decay_ns * np.log(1.0 / np.where(r > 0, r, 1.0)), np.inf)
    first = np.floor(a + lo_ns / sample_ns).astype(np.int64) + 1  # first sample strictly inside
    last_f = a + hi_ns / sample_ns
    last = np.where(np.isfinite(last_f), np.ceil(np.where(np.isfinite(last_f), last_f, 0.0)).astype(np.int64) - 1,
                    length - 1)
    first = np.maximum(first, np.ceil(a).astype(np.int64))  # the pulse adds nothing before its arrival
    first, last = np.maximum(first, 0), np.minimum(last, length - 1)
    ok = first <= last
    return np.stack([first[ok], last[ok]], axis=1)


def merge_windows(runs: np.ndarray, pre: int, post: int, length: int) -> np.ndarray:
    """Widen each run [n0, n1] to [n0 - pre, n1 + post], clip to [0, length) and
    merge runs that overlap or touch.  Returns int64 [k][2] (first, last)."""
    if len(runs) == 0 or length <= 0:
        return np.zeros((0, 2), np.int64)
    w = np.stack([np.maximum(runs[:, 0] - pre, 0), np.minimum(runs[:, 1] + post, length - 1)], axis=1)
    w = w[np.argsort(w[:, 0], kind="stable")]
    out = [list(w[0])]
    for s, e in w[1:]:
        if s <= out[-1][1] + 1:
            out[-1][1] = max(out[-1][1], e)
        else:
            out.append([s, e])
    return np.asarray(out, np.int64)


def truth_islands(pulses, threshold: float, pre: int, post: int, length: int, **shape) -> np.ndarray:
    """Truth islands (first, last) of one calorimeter-fill from its pulse list
    (fields 'arrival' and 'amplitude')."""
    runs = crossing_runs(pulses["arrival"], pulses["amplitude"], threshold, length, **shape)
    return merge_windows(runs, pre, post, length)


def threshold_scan(samples, truth_pulses, params: dict, thresholds, fill_len=None) -> dict:
    """Identified islands (the CUDA path on `samples`, a CUDA int16 tensor
    [F][C][X][N]) against truth islands (from truth_pulses[f][c], each a pulse
    list) for every threshold.  Per threshold: both counts per dataset, the
    least-squares slope of identified on truth through the origin, the ratio of
    totals and the correlation over datasets."""
    F, C = int(samples.shape[0]), int(samples.shape[1])
    N = int(samples.shape[3])
    lens = [N] * F if fill_len is None else [int(v) for v in fill_len]
    rows = {}
    for T in thresholds:
        res = process_fills(samples, **dict(params, threshold=int(T)),
                            fill_len=None if fill_len is None else np.asarray(lens, np.int32))
        isl = res["outputs"].islands_host(res["n_islands"])
        ident = np.bincount(isl["fill"].astype(np.int64) * C + isl["calo"], minlength=F * C)
        truth = np.array([len(truth_islands(truth_pulses[f][c], T, params["pre"], params["post"], lens[f]))
                          for f in range(F) for c in range(C)], np.int64)
        t, i = truth.astype(np.float64), ident.astype(np.float64)
        slope = float((t * i).sum() / max(1e-9, (t * t).sum()))
        corr = float(np.corrcoef(t, i)[0, 1]) if t.std() > 0 and i.std() > 0 else None
        rows[str(T)] = {"slope": round(slope, 4), "ratio_of_totals": round(float(i.sum() / max(1.0, t.sum())), 4),
                        "corr": None if corr is None or math.isnan(corr) else round(corr, 4),
                        "truth": truth.tolist(), "identified": ident.tolist()}
    return {"thresholds": rows}
