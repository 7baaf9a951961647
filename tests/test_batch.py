"""Batch plans: tuned configuration + CUDA graph replay of a fixed batch.

CPU tests check argument validation (no device work).  GPU tests check that a
graph replay gives, bit for bit, the oracle's islands, pool rows and
pedestals, that Q accumulates once per replay and is untouched by plan
creation, and that the tuner's cache and explicit configurations behave."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def daq():
    from paper_1611_04959_gb300 import build
    build.build()
    import paper_1611_04959_gb300 as d
    return d


@pytest.mark.parametrize("bad", ["null_plan", "n_xtal", "flags", "decim", "pre"])
def test_plan_create_rejects_bad_arguments_before_device_work(daq, bad):
    p = daq.make_params(decim=(0,) if bad == "decim" else (32,), pre=-1 if bad == "pre" else 8)
    isl = daq.DaqIslands(None, 0, None, 0, None, None)
    h = ctypes.c_void_p()
    L = daq.lib()
    rc = L.daq_batch_plan_create(None, 2, 0 if bad == "n_xtal" else 54, 1000, 1, ctypes.byref(p), ctypes.byref(isl),
                                 None, 8 if bad == "flags" else 0, None if bad == "null_plan" else ctypes.byref(h))
    assert rc == daq.DAQ_EINVAL
    assert h.value is None


def test_null_plan_calls(daq):
    assert daq.daq_batch_launch(None, None) == daq.DAQ_EINVAL
    assert daq.daq_batch_plan_destroy(None) == daq.DAQ_EINVAL
    daq.daq_tune_cache_clear()


# ------------------------------------------------------------------------------------------ GPU
@pytest.fixture(scope="module")
def genv(daq):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    return dict(torch=torch, oracle=oracle, synth=synth, daq=daq)


def _batch(genv, n_fills=5, n_calo=2, n_samples=48_000, seed_shift=0):
    from synth import workloads as W
    w = W.scaled(W.BATCH_UNEVEN, n_fills=n_fills, n_calo=n_calo, n_samples=n_samples)
    rng = np.random.default_rng(77 + seed_shift)
    fl = rng.integers(n_samples // 7, n_samples + 1, size=n_fills).astype(np.int32)
    fl[0] = n_samples
    rate = np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=n_fills))
    s = genv["synth"].generate(w.config(), fill_len=fl, rate=rate)
    return w, s, fl


def _outputs(genv, s, fl):
    torch, daq = genv["torch"], genv["daq"]
    F, C, X, N = s.shape
    rows = C * int(fl.sum())
    return daq.Outputs(torch, "cuda", F, C, X, rows // 2 + F * C + 1, rows)


def _check(genv, out, ref):
    counts = out.counts.cpu().numpy()
    assert genv["daq"].daq_status_from_counts(counts) == genv["daq"].DAQ_OK, counts
    assert int(counts[0]) == ref["n_islands"] and int(counts[1]) == ref["n_rows"]
    assert np.array_equal(out.islands_host(ref["n_islands"]), ref["islands"])
    assert np.array_equal(out.pool[: ref["n_rows"]].cpu().numpy(), ref["pool"])
    assert np.array_equal(out.pedestal.cpu().numpy(), ref["pedestal"])


@pytest.mark.gpu
def test_graph_replay_matches_oracle_and_accumulates_q(genv):
    torch, daq, oracle = genv["torch"], genv["daq"], genv["oracle"]
    w, s, fl = _batch(genv)
    params = w.params()
    ref = oracle.process_fills(s, params, fill_len=fl, n_threads=8)
    F, C, X, N = s.shape
    x = torch.from_numpy(s).cuda()
    fl_d = torch.as_tensor(fl, device="cuda")
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    out = _outputs(genv, s, fl)
    daq.daq_tune_cache_clear()
    plan = daq.BatchPlan(x, q, out, fill_len=fl_d, tune=True, force=True, **params)
    torch.cuda.synchronize()
    assert int(q.abs().sum().item()) == 0          # creation leaves Q alone
    t = plan.tuning()
    assert t["n_tried"] >= 5 and not t["from_cache"] and t["ms"] > 0
    assert (t["tile"], t["grid"]) in {(0, 0), (448, 0), (224, 0), (128, 0), (448, -4), (224, -4), (448, -1),
                                      (960, -1), (448, -2), (448, -3)} or t["grid"] > 0
    assert t["flags"] in (0, daq.DAQ_SPARSE) and (t["flags"] == 0 or (t["tile"], t["grid"]) == (0, 0))
    stream = torch.cuda.Stream()
    for k in range(3):
        out.counts.zero_()
        out.pool.fill_(-1)
        with torch.cuda.stream(stream):
            plan.launch(stream)
        stream.synchronize()
        _check(genv, out, ref)
        assert np.array_equal(q.cpu().numpy(), (k + 1) * ref["q"])
    plan.close()


@pytest.mark.gpu
def test_tuning_cache_and_explicit_configuration(genv):
    torch, daq, oracle = genv["torch"], genv["daq"], genv["oracle"]
    w, s, fl = _batch(genv, n_fills=3, n_calo=3, n_samples=24_000, seed_shift=1)
    params = w.params()
    ref = oracle.process_fills(s, params, fill_len=fl, n_threads=8)
    F, C, X, N = s.shape
    x = torch.from_numpy(s).cuda()
    fl_d = torch.as_tensor(fl, device="cuda")
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    out = _outputs(genv, s, fl)
    a = daq.BatchPlan(x, q, out, fill_len=fl_d, tune=True, force=True, **params)
    b = daq.BatchPlan(x, q, out, fill_len=fl_d, tune=True, **params)
    ta, tb = a.tuning(), b.tuning()
    assert tb["from_cache"] and tb["n_tried"] == 0
    assert (ta["tile"], ta["grid"], ta["flags"]) == (tb["tile"], tb["grid"], tb["flags"])
    a.close()
    for tile, grid, flags in [(224, -1, 0), (128, 3, 0), (448, -3, 0), (0, 0, daq.DAQ_SPARSE), (224, 5, daq.DAQ_SPARSE)]:
        c = daq.BatchPlan(x, q, out, fill_len=fl_d, tune=False, tile=tile, grid=grid, flags=flags, **params)
        tc = c.tuning()
        assert (tc["tile"], tc["grid"], tc["flags"]) == (tile, grid, flags) and tc["n_tried"] == 0
        q.zero_()
        c.launch()
        torch.cuda.synchronize()
        _check(genv, out, ref)
        assert np.array_equal(q.cpu().numpy(), ref["q"])
        c.close()
    b.close()


@pytest.mark.gpu
def test_replay_follows_new_fill_lengths(genv):
    torch, daq, oracle = genv["torch"], genv["daq"], genv["oracle"]
    w, s, fl = _batch(genv, n_fills=4, n_calo=2, n_samples=30_000, seed_shift=2)
    params = w.params()
    F, C, X, N = s.shape
    x = torch.from_numpy(s).cuda()
    full = np.full(F, N, np.int32)
    fl_d = torch.as_tensor(full, device="cuda")
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    out = _outputs(genv, s, full)
    plan = daq.BatchPlan(x, q, out, fill_len=fl_d, tune=False, **params)
    for lens in (full, fl):
        fl_d.copy_(torch.as_tensor(lens))
        q.zero_()
        plan.launch()
        torch.cuda.synchronize()
        ref = oracle.process_fills(s, params, fill_len=lens, n_threads=8)
        _check(genv, out, ref)
        assert np.array_equal(q.cpu().numpy(), ref["q"])
    plan.close()
