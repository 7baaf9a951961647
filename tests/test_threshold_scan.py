"""Island-finding efficiency across thresholds (Fig. 2's check), run through
the CUDA path: identified islands in noisy calorimeter-fills against the
truth islands of their noise-free twins.  Above the noise the two agree on
every dataset (slope 1); at thresholds inside the noise, noise crossings add
islands."""
import numpy as np
import pytest


def test_noise_free_twin_has_the_same_pulses():
    import synth
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=2, n_calo=1, n_samples=40_000)
    w0 = W.scaled(W.SPARSE_FULL_FILL, n_fills=2, n_calo=1, n_samples=40_000, noise_sigma=0.0)
    for f in range(2):
        a = synth.pulses(w.config(), f, 0, 40_000, 2.0)
        b = synth.pulses(w0.config(), f, 0, 40_000, 2.0)
        assert len(a) > 0 and np.array_equal(a, b)
    x0 = synth.generate(w0.config())
    # no noise: a channel before the first pulse sits exactly at its pedestal
    first = int(np.ceil(synth.pulses(w0.config(), 0, 0, 40_000)["arrival"].min()))
    for xt in range(54):
        assert (x0[0, 0, xt, :first] == synth.true_pedestal(w0.config(), 0, xt)).all()


@pytest.mark.gpu
def test_threshold_scan_slope_one_above_the_noise():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import bench
    import synth
    import paper_1611_04959_gb300 as daq
    from synth import workloads as W
    r = bench.threshold_scan(torch, torch.device("cuda"), daq, synth, W, n_fills=6, n_calo=2,
                             thresholds=(5, 15, 30, 300))["thresholds"]
    for T in ("15", "30", "300"):
        assert abs(r[T]["slope"] - 1.0) < 0.03, (T, r[T])
        assert r[T]["corr"] > 0.99
    assert r["5"]["ratio_of_totals"] > 2.0           # inside the noise: noise islands dominate
    assert sum(r["300"]["truth"]) < sum(r["30"]["truth"])   # fewer pulses clear a higher threshold
