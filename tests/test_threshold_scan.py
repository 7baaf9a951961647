"""Island-finding efficiency across thresholds (arXiv:1611.04959, Sec. 3,
Fig. 2): identified islands against truth islands built from the generator's
injected pulse list (paper_1611_04959_gb300.fig2).

The truth construction is pinned on the CPU: its crossing runs against a brute
force over the pulse shape, its merging against hand-worked windows, and the
whole truth against the oracle's islands in noise-free fills.  On the GPU the
CUDA path's islands in noise-free fills equal the oracle's, and in noisy fills
the identified islands follow the truth with slope 1 above the noise."""
import numpy as np
import pytest


def _fig2():
    from paper_1611_04959_gb300 import fig2
    return fig2


def test_crossing_run_of_one_pulse_by_hand():
    # A = 100 at sample 1000, T = 30: shape > 0.3 for dt in (0.6, 2 + 5 ln(10/3)) ns = (0.6, 8.02) ns,
    # i.e. samples 1001 (dt 1.25 ns: 62.5 ADC) to 1006 (dt 7.5 ns: 33.3 ADC); 1007 gives 25.9 ADC
    runs = _fig2().crossing_runs([1000.0], [100.0], 30.0, 560_000)
    assert runs.tolist() == [[1001, 1006]]
    assert _fig2().crossing_runs([1000.0], [30.0], 30.0, 560_000).shape == (0, 2)   # peak equal to T: no crossing


def test_crossing_runs_match_a_brute_force_over_the_shape():
    rng = np.random.default_rng(7)
    a = rng.uniform(200, 5000, 300)
    amp = np.exp(rng.uniform(np.log(20), np.log(2000), 300))
    for T in (15.0, 30.0, 100.0, 300.0):
        runs = _fig2().crossing_runs(a, amp, T, 6000)
        want = []
        for ai, Ai in zip(a, amp):
            n = np.arange(int(ai) - 2, int(ai) + 200)
            dt = (n - ai) * 1.25
            shape = np.where(dt < 0, 0.0, np.where(dt < 2.0, dt / 2.0, np.exp(-(dt - 2.0) / 5.0)))
            above = n[Ai * shape > T]
            if above.size:
                assert above[-1] - above[0] + 1 == above.size      # one run per pulse
                want.append([above[0], above[-1]])
        assert runs.tolist() == want, T


def test_windows_merge_when_they_overlap_or_touch():
    m = _fig2().merge_windows
    r = lambda *p: np.array(p, np.int64)
    assert m(r([100, 105], [135, 140]), 8, 24, 10_000).tolist() == [[92, 164]]   # [92,129] + [127,164] overlap
    assert m(r([100, 105], [138, 140]), 8, 24, 10_000).tolist() == [[92, 164]]   # [92,129] + [130,164] touch
    assert m(r([100, 105], [139, 140]), 8, 24, 10_000).tolist() == [[92, 129], [131, 164]]
    assert m(r([3, 4], [9990, 9995]), 8, 24, 10_000).tolist() == [[0, 28], [9982, 9999]]   # clipped to the fill


@pytest.mark.parametrize("T", [30, 300])
def test_truth_islands_agree_with_the_oracle_in_noise_free_fills(oracle_mod, synth_mod, T):
    """Without noise, the oracle's islands are those of the summed pulses; the
    pulse-list truth differs only where rounding each crystal's share moves an
    edge by a sample or a neighbouring pulse's tail joins two islands.  The
    counts agree within 2%, and nearly every island of either list overlaps one
    of the other."""
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=1, n_calo=2, n_samples=200_000, noise_sigma=0.0)
    s = synth_mod.generate(w.config())
    params = dict(w.params(), threshold=T)
    ref = oracle_mod.process_fills(s, params, n_threads=2)
    fig2 = _fig2()
    for c in range(2):
        truth = fig2.truth_islands(synth_mod.pulses(w.config(), 0, c, 200_000), T, params["pre"], params["post"],
                                   200_000)
        isl = ref["islands"][ref["islands"]["calo"] == c]
        got = np.stack([isl["start"].astype(np.int64), (isl["start"] + isl["len"] - 1).astype(np.int64)], axis=1)
        want = np.asarray(truth, np.int64)
        assert len(want) > 50
        assert abs(len(got) - len(want)) <= 0.02 * len(want), (c, len(got), len(want))

        def covered(x, y):  # islands of x that overlap an island of y
            j = np.clip(np.searchsorted(y[:, 0], x[:, 1], side="right") - 1, 0, len(y) - 1)
            return int(((y[j, 0] <= x[:, 1]) & (y[j, 1] >= x[:, 0])).sum())
        assert covered(want, got) >= 0.99 * len(want), (c, covered(want, got), len(want))
        assert covered(got, want) >= 0.99 * len(got), (c, covered(got, want), len(got))


@pytest.fixture(scope="module")
def genv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    import paper_1611_04959_gb300 as daq
    return dict(torch=torch, oracle=oracle, synth=synth, daq=daq)


@pytest.mark.gpu
@pytest.mark.parametrize("T", [15, 30, 300])
def test_cuda_islands_equal_the_oracle_in_noise_free_fills(genv, T):
    torch, oracle, synth, daq = genv["torch"], genv["oracle"], genv["synth"], genv["daq"]
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=2, n_calo=2, noise_sigma=0.0)
    s = synth.generate(w.config())
    params = dict(w.params(), threshold=T)
    ref = oracle.process_fills(s, params, n_threads=8)
    res = daq.process_fills(torch.from_numpy(s).cuda(), **params)
    assert res["n_islands"] == ref["n_islands"] and res["n_rows"] == ref["n_rows"]
    assert np.array_equal(res["outputs"].islands_host(res["n_islands"]), ref["islands"])


@pytest.mark.gpu
def test_threshold_scan_slope_one_above_the_noise(genv):
    """Identified islands in noisy sparse-regime fills (pulse rate x
    log-uniform[0.2, 5] per fill) against the pulse-list truth."""
    torch, synth = genv["torch"], genv["synth"]
    from paper_1611_04959_gb300 import fig2
    from synth import workloads as W
    F, C = 6, 2
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=F, n_calo=C)
    N = w.n_samples
    _, rates = synth.fill_plan(w.synth["seed"] + 29, F, N, N, 0.2, 5.0)
    x = torch.from_numpy(synth.generate(w.config(), rate=rates)).cuda()
    truth = [[synth.pulses(w.config(), f, c, N, float(rates[f])) for c in range(C)] for f in range(F)]
    r = fig2.threshold_scan(x, truth, w.params(), (5, 15, 30, 300))["thresholds"]
    for T in ("15", "30", "300"):
        assert abs(r[T]["slope"] - 1.0) < 0.03, (T, r[T]["slope"], r[T]["ratio_of_totals"])
        assert r[T]["corr"] > 0.99, (T, r[T]["corr"])
    assert r["5"]["ratio_of_totals"] > 2.0                       # inside the noise: noise islands dominate
    assert sum(r["300"]["truth"]) < sum(r["30"]["truth"])        # fewer pulses clear a higher threshold
