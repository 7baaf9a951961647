"""Pins that tie the oracle to the paper's definitions and to mathematics
rather than to itself.  Each pin takes an `Oracle` (the real one, or a copy
with a planted mistake) and raises AssertionError when it disagrees.

Sources of truth used here:
  * hand-derived fixtures in tests/golden (closed-form results of tiny inputs)
  * an independent set-union restatement (marks = union of windows, islands =
    runs of consecutive marks, rounding by exact fractions)
  * special cases with closed-form answers (single crossing, merge boundary,
    strict threshold, clipping, constant channels)
  * invariants on generated fills and exact injected-pulse recovery
    (the slope-1 statement of Fig. 2 made exact in noise-free data)
"""
from __future__ import annotations

import glob
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- set-union restatement
def brute(s: np.ndarray, params: dict, length: int | None = None) -> dict:
    """Independent restatement on tiny inputs (pure Python, sets and fractions)."""
    X, N = s.shape
    L = N if length is None else length
    n = min(params["ped_samples"], L)
    ped = []
    for x in range(X):
        if n <= 0:
            ped.append(0)
        else:
            mean = Fraction(sum(int(v) for v in s[x, :n]), n)
            ped.append(math.floor(mean + Fraction(1, 2)))          # half up
    S = [sum(int(s[x, t]) for x in range(X)) - sum(ped) for t in range(L)]
    crossings = [t for t in range(L) if S[t] > params["threshold"]]
    marked = set()
    for u in crossings:
        marked |= set(range(max(0, u - params["pre"]), min(L, u + params["post"] + 1)))
    times = sorted(marked)
    islands, row = [], 0
    for _, grp in itertools.groupby(enumerate(times), key=lambda it: it[1] - it[0]):
        g = [t for _, t in grp]
        islands.append((g[0], len(g), row))
        row += len(g)
    bins = []
    for D in params.get("decim", ()):
        bins.append([sum(S[k:k + D]) for k in range(0, L, D)])
    pool = np.array([[int(s[x, t]) for x in range(X)] for t in times], dtype=np.int16).reshape(len(times), X)
    return dict(pedestal=ped, S=S, islands=islands, pool=pool, bins=bins, times=times)


def _islands(res) -> list:
    return [(int(i["start"]), int(i["len"]), int(i["pool_row"])) for i in res["islands"]]


# ---------------------------------------------------------------- pins
def pin_golden(orc):
    files = sorted(glob.glob(os.path.join(GOLDEN, "*.json")))
    assert files, "golden fixtures missing"
    for fn in files:
        g = json.load(open(fn))
        if g.get("kind", "islands") != "islands":
            continue
        s = np.array(g["samples"], dtype=np.int16)
        r = orc.calofill(s, g["params"], length=g["length"])
        e = g["expect"]
        name = os.path.basename(fn)
        assert r["pedestal"].tolist() == e["pedestal"], name
        assert r["S"].tolist() == e["S"], name
        assert [list(t) for t in _islands(r)] == e["islands"], name
        assert np.array_equal(r["pool"], s[:, e["pool_times"]].T), name
        assert [b.tolist() for b in r["bins"]] == e["bins"], name


def _flat(value: int, X: int, N: int) -> np.ndarray:
    return np.full((X, N), value, dtype=np.int16)


def pin_single_crossing(orc):
    """One crossing at u marks exactly [u - pre, u + post], clipped to the fill."""
    N, pre, post = 48, 3, 5
    p = dict(threshold=10, pre=pre, post=post, ped_samples=4, decim=(8,))
    for u in (6, 20, 47, 45, 4):
        s = _flat(100, 2, N)
        s[1, u] += 11                      # S[u] = 11 > 10; ped window [0,4) untouched for u >= 4
        r = orc.calofill(s, p)
        lo, hi = max(0, u - pre), min(N - 1, u + post)
        assert _islands(r) == [(lo, hi - lo + 1, 0)], (u, _islands(r))
        assert np.array_equal(r["pool"], s[:, lo:hi + 1].T)


def pin_merge_boundary(orc):
    """Crossings u1 < u2 merge iff u2 - u1 <= pre + post + 1 (windows touch)."""
    N, pre, post = 64, 2, 4
    p = dict(threshold=0, pre=pre, post=post, ped_samples=2, decim=())
    u1 = 10
    for gap in range(1, pre + post + 4):
        s = _flat(7, 1, N)
        s[0, u1] = 8
        s[0, u1 + gap] = 8
        r = orc.calofill(s, p)
        isl = _islands(r)
        if gap <= pre + post + 1:
            assert isl == [(u1 - pre, gap + pre + post + 1, 0)], (gap, isl)
        else:
            w = pre + post + 1
            assert isl == [(u1 - pre, w, 0), (u1 + gap - pre, w, w)], (gap, isl)


def pin_threshold_strict_and_extremes(orc):
    N = 40
    p = dict(threshold=5, pre=1, post=1, ped_samples=4, decim=(4,))
    s = _flat(3, 1, N)
    s[0, 10] = 8                           # S = 5 == T: not a crossing
    assert _islands(orc.calofill(s, p)) == []
    s[0, 10] = 9                           # S = 6 > T
    assert _islands(orc.calofill(s, p)) == [(9, 3, 0)]
    # all below: no islands, empty pool
    r = orc.calofill(_flat(3, 3, N), p)
    assert _islands(r) == [] and r["pool"].shape == (0, 3)
    # everything above after the pedestal window: one island covering all of the fill
    s = _flat(50, 2, N)
    s[:, :4] = 0
    r = orc.calofill(s, dict(p, pre=4))
    assert _islands(r) == [(0, N, 0)], _islands(r)


def pin_pedestal_rounding(orc):
    cases = [([1, 2], 2, 2), ([-1, -2], 2, -1), ([1, 1, 2], 3, 1), ([2, 2, 1], 3, 2), ([7] * 100, 100, 7),
             ([-3, -2], 2, -2), ([1, 2, 3, 4], 4, 3), ([0, 0, 0, 1], 4, 0), ([0, 0, 1, 1], 4, 1)]
    for row, n, want in cases:
        assert orc.pedestal(np.array(row, np.int16), ped_samples=n) == want, (row, want)
    # the window is the first ped_samples samples only, and is cut to the fill length
    row = np.array([4, 4, 4, 100, 100], np.int16)
    assert orc.pedestal(row, ped_samples=3) == 4
    assert orc.pedestal(row, length=2, ped_samples=100) == 4
    assert orc.pedestal(row, length=0, ped_samples=100) == 0
    # constant channel: pedestal equals the constant
    for v in (-32768, -5, 0, 1800, 4095, 32767):
        assert orc.pedestal(np.full(100, v, np.int16)) == v


def pin_decimation(orc):
    rng = np.random.default_rng(3)
    s = rng.integers(-20, 20, size=(2, 37)).astype(np.int16)
    p = dict(threshold=10 ** 6, pre=0, post=0, ped_samples=5, decim=(8, 3))
    r = orc.calofill(s, p)
    S = r["S"]
    for D, b in zip((8, 3), r["bins"]):
        assert len(b) == math.ceil(37 / D)
        assert int(b.sum()) == int(S.sum())
        assert b.tolist() == [int(S[k:k + D].sum()) for k in range(0, 37, D)]


def pin_against_brute(orc, n_cases: int = 150, seed: int = 11):
    rng = np.random.default_rng(seed)
    for case in range(n_cases):
        X = int(rng.integers(1, 4))
        N = int(rng.integers(1, 65))
        L = int(rng.integers(0, N + 1))
        params = dict(threshold=int(rng.integers(-30, 60)), pre=int(rng.integers(0, 6)),
                      post=int(rng.integers(0, 9)), ped_samples=int(rng.integers(1, 12)),
                      decim=tuple(int(d) for d in rng.integers(1, 9, size=int(rng.integers(0, 3)))))
        s = rng.integers(-40, 80, size=(X, N)).astype(np.int16)
        want = brute(s, params, L)
        got = orc.calofill(s, params, length=L)
        ctx = (case, X, N, L, params)
        assert got["pedestal"].tolist() == want["pedestal"], ctx
        assert got["S"].tolist() == want["S"], ctx
        assert _islands(got) == want["islands"], ctx
        assert np.array_equal(got["pool"], want["pool"]), ctx
        assert [b.tolist() for b in got["bins"]] == want["bins"], ctx


def pin_fill_sum_accumulates(orc):
    """Table 2 fill-by-fill sum: Q accumulates B_D over fills and calorimeters keep
    their own rows; every fill's island list follows in (fill, calo, start) order."""
    rng = np.random.default_rng(5)
    F, C, X, N = 3, 2, 3, 50
    s = rng.integers(0, 30, size=(F, C, X, N)).astype(np.int16)
    params = dict(threshold=20, pre=1, post=2, ped_samples=6, decim=(4, 7))
    lens = np.array([50, 33, 0], np.int32)
    res = orc.process_fills(s, params, fill_len=lens)
    nb = [math.ceil(N / 4), math.ceil(N / 7)]
    q = [np.zeros((C, nb[0]), np.int64), np.zeros((C, nb[1]), np.int64)]
    want_isl, row = [], 0
    for f in range(F):
        for c in range(C):
            b = brute(s[f, c], params, int(lens[f]))
            for d in range(2):
                q[d][c, :len(b["bins"][d])] += np.asarray(b["bins"][d], dtype=np.int64)
            for st, ln, _ in b["islands"]:
                want_isl.append((f, c, st, ln, row))
                row += ln
    got_isl = [(int(i["fill"]), int(i["calo"]), int(i["start"]), int(i["len"]), int(i["pool_row"]))
               for i in res["islands"]]
    assert len({(f, c) for f, c, *_ in want_isl}) >= 3, "fixture must put islands in several calo-fills"
    assert got_isl == want_isl
    assert res["n_rows"] == row
    assert np.array_equal(res["q"], np.concatenate([q[0].ravel(), q[1].ravel()]))


def pin_crystal_sum_golden(orc):
    """Per-crystal full-resolution fill sum on the hand-derived fixture."""
    n = 0
    for fn in sorted(glob.glob(os.path.join(GOLDEN, "*.json"))):
        g = json.load(open(fn))
        if g.get("kind") != "crystal_sum":
            continue
        q = orc.crystal_sum(np.array(g["samples"], np.int16), fill_len=g["fill_len"], ped_samples=g["ped_samples"])
        assert q.tolist() == g["expected_q"], os.path.basename(fn)
        n += 1
    assert n >= 1, "crystal-sum fixture missing"


def pin_crystal_sum_matches_decimated_q(orc):
    """Summed over crystals and over the samples of a bin, the per-crystal fill
    sum is the decimated fill sum Q_D (the oracle's separate Q-method path)."""
    rng = np.random.default_rng(8)
    F, C, X, N = 3, 3, 4, 61
    s = rng.integers(-40, 400, size=(F, C, X, N)).astype(np.int16)
    lens = np.array([61, 29, 4], np.int32)
    params = dict(threshold=10_000, pre=1, post=1, ped_samples=5, decim=(4, 7))
    qx = orc.crystal_sum(s, fill_len=lens, ped_samples=5)
    qd = orc.process_fills(s, params, fill_len=lens)["q"]
    off = 0
    for D in (4, 7):
        nb = math.ceil(N / D)
        want = qd[off: off + C * nb].reshape(C, nb)
        off += C * nb
        per_t = qx.sum(axis=1)                      # [C][N]
        got = np.stack([per_t[:, k * D: k * D + D].sum(axis=1) for k in range(nb)], axis=1)
        assert np.array_equal(got, want), D


def pin_pack_golden(orc):
    """The packed stream of a hand-derived 3-row pool, word by word."""
    n = 0
    for fn in sorted(glob.glob(os.path.join(GOLDEN, "*.json"))):
        g = json.load(open(fn))
        if g.get("kind") != "pack":
            continue
        pool = np.array(g["pool"], np.int16)
        st = orc.pack(pool)
        assert st.size % 4 == 0 and st.view("<u4").tolist() == g["expected_words"], os.path.basename(fn)
        assert np.array_equal(orc.unpack(st, *pool.shape), pool)
        n += 1
    assert n >= 1, "pack fixture missing"


def pin_pack_round_trip_and_size(orc):
    """Lossless for any int16 rows (extremes give 17-bit differences), and the
    size is the header, the offsets and one head word plus w planes per crystal
    and block."""
    rng = np.random.default_rng(21)
    cases = [rng.integers(-32768, 32768, size=(77, 3)), np.tile([[-32768], [32767]], (20, 5)),
             np.full((64, 54), 1800), rng.integers(1790, 1811, size=(200, 54)), np.zeros((0, 4))]
    for pool in cases:
        pool = np.asarray(pool).astype(np.int16)
        rows, X = pool.shape
        st = orc.pack(pool)
        assert np.array_equal(orc.unpack(st, rows, X), pool)
        nb = -(-rows // 32)
        words = 0
        for b in range(nb):
            blk = np.concatenate([pool[32 * b: 32 * b + 32], np.repeat(pool[-1:], max(0, 32 * b + 32 - rows), 0)])
            d = np.diff(blk.astype(np.int64), axis=0)
            z = np.where(d >= 0, 2 * d, -2 * d - 1)
            words += sum(1 + int(m).bit_length() for m in z.max(axis=0))
        assert st.size == 16 + 8 * (nb + 1) + 4 * words


PINS = [pin_golden, pin_single_crossing, pin_merge_boundary, pin_threshold_strict_and_extremes,
        pin_pedestal_rounding, pin_decimation, pin_against_brute, pin_fill_sum_accumulates,
        pin_crystal_sum_golden, pin_crystal_sum_matches_decimated_q, pin_pack_golden, pin_pack_round_trip_and_size]


# ---------------------------------------------------------------- invariants on any output
def check_invariants(s_cf: np.ndarray, params: dict, length: int, r: dict):
    """Structural facts every correct result of one calorimeter-fill satisfies."""
    S, M = r["S"], r["mark"]
    isl = _islands(r)
    pre, post, T = params["pre"], params["post"], params["threshold"]
    prev_end = -2
    rows = 0
    for st, ln, pr in isl:
        assert ln >= 1 and st >= 0 and st + ln <= length
        assert st > prev_end + 1, "islands overlap, touch or are out of order"
        assert pr == rows
        prev_end = st + ln - 1
        rows += ln
    assert rows == len(r["pool"]) == int(M.sum())
    covered = np.zeros(length, bool)
    for st, ln, _ in isl:
        covered[st:st + ln] = True
    assert np.array_equal(covered, M)
    cross = np.flatnonzero(S > T)
    # every crossing lies in an island together with its whole clipped window
    for u in cross:
        assert covered[max(0, u - pre):min(length, u + post + 1)].all()
    # minimality: every marked sample is inside some crossing's window
    if length:
        near = np.zeros(length + 1, np.int64)
        for u in cross:
            near[max(0, u - pre)] += 1
            near[min(length, u + post + 1)] -= 1
        assert np.array_equal(np.cumsum(near)[:length] > 0, M)
    # pool rows are the raw samples at the marked times
    assert np.array_equal(r["pool"], s_cf[:, :length][:, M].T)
    for D, b in zip(params.get("decim", ()), r["bins"]):
        assert int(b.sum()) == int(S.sum())
        assert len(b) == (length + D - 1) // D
