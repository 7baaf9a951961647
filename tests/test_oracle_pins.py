"""The oracle against what the paper and mathematics fix (CPU only)."""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.PINS, ids=lambda f: f.__name__)
def test_pin(pin, oracle_mod):
    pin(oracle_mod.Oracle())


def test_invariants_on_generated_fill(oracle_mod, synth_mod):
    """Invariants on a generated calorimeter-fill with literal noise (sigma 3 per crystal)."""
    from synth import workloads as W
    w = W.scaled(W.PLAIN_1CALO, n_samples=60_000)
    s = synth_mod.generate(w.config())[0, 0]
    for params in (w.params(), dict(w.params(), threshold=15, post=64, decim=(8, 32)),
                   dict(w.params(), threshold=60, pre=0, post=0, decim=(7,))):
        r = oracle_mod.calofill(s, params)
        P.check_invariants(s, params, s.shape[1], r)


def test_invariants_on_ragged_fill(oracle_mod, synth_mod):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_1CALO, n_samples=30_008)
    cfg = w.config()
    s = synth_mod.generate(cfg, fill_len=[21_111])[0, 0]
    assert (s[:, 21_111:] == cfg.beyond_value).all()
    r = oracle_mod.calofill(s, w.params(), length=21_111)
    P.check_invariants(s, w.params(), 21_111, r)


def test_injected_pulses_recovered_noise_free(oracle_mod, synth_mod):
    """Noise-free fills with a constant pedestal: every isolated pulse gives
    exactly one island, which holds its peak; nothing else crosses (Fig. 2's
    identified-vs-truth slope of 1, made exact)."""
    from synth import workloads as W
    params = dict(threshold=30, pre=8, post=24, ped_samples=100, decim=(32,))
    n = 120_000
    for seed, rate in ((7, 60.0), (8, 25.0)):
        w = W.scaled(W.PLAIN_1CALO, n_samples=n, noise_sigma=0.0, ped_lo=1800, ped_hi=1800,
                     pulses_per_fill=rate, seed=seed)
        cfg = w.config()
        s = synth_mod.generate(cfg)[0, 0]
        truth = synth_mod.pulses(cfg, 0, 0)
        r = oracle_mod.calofill(s, params)
        assert r["pedestal"].tolist() == [1800] * 54
        isl = [(int(i["start"]), int(i["len"])) for i in r["islands"]]
        arr = np.sort(truth["arrival"])
        assert len(arr) > 10
        support = np.zeros(n, bool)
        for a in arr:
            support[int(math.ceil(a)):int(math.ceil(a)) + cfg.tail_samples] = True
        for st, ln in isl:                       # every island comes from a pulse
            assert support[st:st + ln].any()
        gaps = np.diff(arr)
        iso = [a for i, a in enumerate(arr)
               if (i == 0 or gaps[i - 1] > 300) and (i == len(arr) - 1 or gaps[i] > 300)]
        assert len(iso) > 5
        for a in iso:
            lo, hi = int(a) - 150, int(a) + 150
            hit = [(st, ln) for st, ln in isl if st < hi and st + ln > lo]
            assert len(hit) == 1, (a, hit)
            k0 = int(math.ceil(a))
            peak = k0 + int(np.argmax(r["S"][k0:k0 + 10]))
            assert r["S"][peak] > params["threshold"]
            assert hit[0][0] <= peak < hit[0][0] + hit[0][1]
        if len(iso) == len(arr):
            assert len(isl) == len(arr)          # identified == truth
        assert len(iso) <= len(isl) <= len(arr)


def test_noise_only_crossing_fraction_closed_form(oracle_mod, synth_mod):
    """Noise only: P(S > T) follows the normal tail of the rounded-noise sum,
    shifted by the pedestal rounding offset the oracle itself reports."""
    from synth import workloads as W
    n = 200_000
    w = W.scaled(W.PLAIN_1CALO, n_samples=n, pulses_per_fill=0.0)
    cfg = w.config()
    s = synth_mod.generate(cfg)[0, 0]
    T = 30
    r = oracle_mod.calofill(s, dict(w.params(), threshold=T))
    offset = sum(synth_mod.true_pedestal(cfg, 0, x) for x in range(54)) - int(r["pedestal"].sum())
    # variance of one rounded N(0, 3^2) value, from the exact class probabilities
    sig = 3.0
    ks = np.arange(-40, 41)
    cdf = lambda z: 0.5 * math.erfc(-z / math.sqrt(2.0))
    pk = np.array([cdf((k + 0.5) / sig) - cdf((k - 0.5) / sig) for k in ks])
    var1 = float((pk * ks * ks).sum())
    sd = math.sqrt(54 * var1)
    # S > T  <=>  noise_sum + offset >= T + 1; continuity-corrected normal tail
    p_want = 0.5 * math.erfc((T + 0.5 - offset) / (sd * math.sqrt(2.0)))
    p_got = float((r["S"] > T).mean())
    tol = 5 * math.sqrt(p_want * (1 - p_want) / n) + 0.004
    assert abs(p_got - p_want) < tol, (p_got, p_want, offset)
    # the mean of S is the pedestal offset (noise has zero mean)
    assert abs(float(r["S"].mean()) - offset) < 5 * sd / math.sqrt(n)


def test_multithread_equals_single_thread(oracle_mod, synth_mod):
    from synth import workloads as W
    w = W.scaled(W.BATCH_UNEVEN, n_fills=3, n_calo=2, n_samples=40_000)
    lens = np.array([40_000, 17_333, 1], np.int32)
    s = synth_mod.generate(w.config(), fill_len=lens)
    a = oracle_mod.process_fills(s, w.params(), fill_len=lens, n_threads=1)
    b = oracle_mod.process_fills(s, w.params(), fill_len=lens, n_threads=4)
    assert np.array_equal(a["islands"], b["islands"])
    assert np.array_equal(a["pool"], b["pool"])
    assert np.array_equal(a["q"], b["q"]) and np.array_equal(a["pedestal"], b["pedestal"])


def test_capacity_truncation_counts_required_sizes(oracle_mod):
    rng = np.random.default_rng(1)
    s = rng.integers(0, 50, size=(1, 2, 2, 200)).astype(np.int16)
    params = dict(threshold=25, pre=1, post=1, ped_samples=4, decim=(4,))
    full = oracle_mod.process_fills(s, params)
    assert full["n_islands"] > 3
    part = oracle_mod.process_fills(s, params, isl_cap=2, row_cap=5)
    assert part["n_islands"] == full["n_islands"] and part["n_rows"] == full["n_rows"]
    assert np.array_equal(part["islands"], full["islands"][:2])
    assert np.array_equal(part["pool"], full["pool"][:5])
    assert np.array_equal(part["q"], full["q"])


# --------------------------------------------------------------------------- planted mistakes
MUTANTS = {
    "threshold_not_strict": ("S[t] > (int64_t)p->threshold", "S[t] >= (int64_t)p->threshold"),
    "pre_post_swapped": ("int64_t u_lo = t - p->post, u_hi = t + p->pre;",
                         "int64_t u_lo = t - p->pre, u_hi = t + p->post;"),
    "window_short_by_one": ("int64_t u_lo = t - p->post, u_hi = t + p->pre;",
                            "int64_t u_lo = t - p->post, u_hi = t + p->pre - 1;"),
    "pedestal_truncated": ("return (int32_t)floor_div(sum + n / 2, n);", "return (int32_t)(sum / n);"),
    "pedestal_not_subtracted": ("S[t] = acc - ped_total;", "S[t] = acc;"),
    "pedestal_added": ("S[t] = acc - ped_total;", "S[t] = acc + ped_total;"),
    "pool_crystals_reversed": ("pool[rows * n_xtal + x] = s[(int64_t)x * pitch + t];",
                               "pool[rows * n_xtal + x] = s[(int64_t)(n_xtal - 1 - x) * pitch + t];"),
    "bin_drops_last_sample": ("t < k * D + D && t < len; ++t) b += S[t];",
                              "t < k * D + D - 1 && t < len; ++t) b += S[t];"),
    "fill_sum_overwrites": ("for (int64_t k = 0; k < kmax; ++k) dst[k] += src[k];",
                            "for (int64_t k = 0; k < kmax; ++k) dst[k] = src[k];"),
    "island_run_cut": ("while (e + 1 < len && M[e + 1]) ++e;",
                       "while (e + 1 < len && M[e + 1] && e - t < 20) ++e;"),
    "crystal_dropped": ("for (int32_t x = 0; x < n_xtal; ++x) acc += s[(int64_t)x * pitch + t];",
                        "for (int32_t x = 1; x < n_xtal; ++x) acc += s[(int64_t)x * pitch + t];"),
    "pool_row_offset_lost": ("isl[tot_isl].pool_row += tot_rows;", "isl[tot_isl].pool_row += 0;"),
    "xtal_sum_pedestal_dropped": ("qrow[t] += (int64_t)row[t] - ped;", "qrow[t] += (int64_t)row[t];"),
    "xtal_sum_ignores_fill_len": ("for (int64_t t = 0; t < len; ++t) qrow[t]", "for (int64_t t = 0; t < pitch; ++t) qrow[t]"),
    "xtal_sum_rows_transposed": ("int64_t *qrow = q + ((int64_t)c * n_xtal + x) * pitch;",
                                 "int64_t *qrow = q + ((int64_t)x * n_calo + c) * pitch;"),
    "pack_zigzag_off_by_one": ("2u * (uint32_t)(-(int64_t)d) - 1u", "2u * (uint32_t)(-(int64_t)d)"),
    "pack_pads_with_zero": ("if (r >= rows) r = rows - 1;", "if (r >= rows) { v[i] = 0; continue; }"),
    "pack_width_short": ("const int w = bit_length(zmax);", "const int w = zmax ? bit_length(zmax) - 1 : 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, oracle_mod, tmp_path):
    """A copy of the oracle with one plausible mistake must fail some pin."""
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "daq_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", str(so), str(c)],
                   check=True)
    orc = oracle_mod.Oracle(str(so))
    failed = []
    for pin in P.PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {name} passed every pin"
