"""Serving runtime (daq_server_*): admission within a memory budget, fills
overlapping on several streams, resident Q, latency / deadtime accounting.

CPU tests: the structs match the C compiler's layout, invalid configurations
are rejected before any device work, and the latency / deadtime summary is
checked on hand-made records.  GPU tests: each fill's islands, pool rows and
pedestals are the same alone and in a mix of concurrent fills (and equal the
oracle's); the resident Q equals the sum of the fills' histograms; no more
fills run at once than the budget's slots; host-submitted fills match
device-submitted ones; replayed arrival times are honoured."""
import ctypes
import subprocess

import numpy as np
import pytest


@pytest.fixture(scope="module")
def daq():
    from paper_1611_04959_gb300 import build
    build.build()
    import paper_1611_04959_gb300 as d
    return d


def test_struct_sizes_match_the_c_compiler(daq, tmp_path):
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "sizes.c"
    names = ["daq_params", "daq_islands", "daq_island", "daq_host_io", "daq_tune_result", "daq_server_config",
             "daq_fill_record", "daq_fill_result", "daq_server_stats", "daq_serving_summary"]
    body = "".join(f'printf("%zu\\n", sizeof({n}));' for n in names)
    src.write_text(f'#include <stdio.h>\n#include "daq.h"\nint main(void){{{body}return 0;}}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    mine = [ctypes.sizeof(daq.DaqParams), ctypes.sizeof(daq.DaqIslands), daq.ISLAND_DTYPE.itemsize,
            ctypes.sizeof(daq.DaqHostIO), ctypes.sizeof(daq.DaqTuneResult), ctypes.sizeof(daq.DaqServerConfig),
            ctypes.sizeof(daq.DaqFillRecord), ctypes.sizeof(daq.DaqFillResult), ctypes.sizeof(daq.DaqServerStats),
            ctypes.sizeof(daq.DaqServingSummary)]
    assert got == mine, dict(zip(names, zip(got, mine)))


def _cfg(daq, **kw):
    c = daq.DaqServerConfig()
    c.n_calo, c.n_xtal, c.n_samples = kw.pop("n_calo", 2), kw.pop("n_xtal", 54), kw.pop("n_samples", 10_000)
    c.params = daq.make_params(**kw.pop("params", {}))
    c.mem_budget_bytes = kw.pop("budget", 1 << 30)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(n_calo=0), dict(n_xtal=0), dict(n_samples=0), dict(budget=0),
                                 dict(budget=1000), dict(n_streams=17), dict(max_slots=-1), dict(flags=8),
                                 dict(params=dict(pre=-1)), dict(hdr_cap=-5)])
def test_invalid_server_configuration_rejected_before_device_work(daq, bad):
    rc, h = daq.daq_server_create(_cfg(daq, **bad))
    assert rc == daq.DAQ_EINVAL and h is None


def test_server_calls_reject_null_handles(daq):
    L = daq.lib()
    t = ctypes.c_int64()
    assert L.daq_server_submit(None, None, 0, -1, -1.0, ctypes.byref(t)) == daq.DAQ_EINVAL
    assert L.daq_server_release(None, 1) == daq.DAQ_EINVAL
    assert L.daq_server_drain(None, 0.0) == daq.DAQ_EINVAL
    assert L.daq_server_destroy(None) == daq.DAQ_EINVAL
    assert L.daq_server_qhist(None) is None


def _rec(daq, arrival, done, nbytes=1000):
    r = daq.DaqFillRecord()
    r.t_arrival, r.t_done, r.raw_bytes, r.t_start, r.t_admit = arrival, done, nbytes, arrival, arrival
    return r


def test_serving_summary_latency_and_deadtime(daq):
    # arrivals every 100 us; fill k takes 50, 150, 50, 300, 50 us after arrival
    arr = [0.0, 100.0, 200.0, 300.0, 400.0]
    lat = [50.0, 150.0, 50.0, 300.0, 50.0]
    recs = [_rec(daq, a, a + l) for a, l in zip(arr, lat)]
    s = daq.daq_serving_summarize(recs[::-1])            # order of records does not matter
    assert s.n == 5
    assert s.latency_p50_us == pytest.approx(np.percentile(lat, 50))
    assert s.latency_p99_us == pytest.approx(np.percentile(lat, 99))
    assert s.latency_max_us == 300.0
    # fills with a successor: 0 (done 50 < 100), 1 (250 > 200), 2 (250 < 300), 3 (600 > 400)
    assert s.deadtime == pytest.approx(2 / 4)
    assert s.span_us == pytest.approx(600.0)
    assert s.gbs == pytest.approx(5 * 1000 / 600.0 / 1e3)
    one = daq.daq_serving_summarize(recs[:1])
    assert one.deadtime == 0.0 and one.latency_p99_us == 50.0
    assert daq.daq_serving_summarize([]).n == 0


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


def _fills(genv, n, n_calo=3, n_samples=40_000):
    from synth import workloads as W
    w = W.scaled(W.SERVING, n_fills=n, n_calo=n_calo, n_samples=n_samples)
    rng = np.random.default_rng(9)
    fl = rng.integers(n_samples // 3, n_samples + 1, size=n).astype(np.int32)
    fl[0] = n_samples
    rate = np.exp(rng.uniform(np.log(0.3), np.log(4.0), size=n))
    s = genv["synth"].generate(w.config(), fill_len=fl, rate=rate)
    return w, s, fl


def _server(genv, w, C, N, budget, **kw):
    return genv["daq"].DaqServer(C, 54, N, budget, **w.params(), **kw)


@pytest.mark.gpu
def test_each_fill_is_the_same_alone_and_in_the_mix(genv):
    torch, daq, oracle = genv["torch"], genv["daq"], genv["oracle"]
    n = 10
    w, s, fl = _fills(genv, n)
    F, C, X, N = s.shape
    dev = [torch.from_numpy(s[f]).cuda() for f in range(n)]
    # alone: one slot, one stream, one fill at a time
    alone = []
    srv = _server(genv, w, C, N, 1 << 40, max_slots=1, n_streams=1)
    for f in range(n):
        t = srv.submit(dev[f], int(fl[f]))
        r = srv.wait(t)
        assert r["status"] == daq.DAQ_OK
        alone.append(srv.fetch(t))
        srv.release(t)
    q_alone = srv.q.cpu().numpy().copy()
    srv.close()
    # mix: every fill submitted at once onto 6 slots and 4 streams
    srv = _server(genv, w, C, N, 1 << 40, max_slots=6, n_streams=4)
    tickets = [srv.submit(dev[f], int(fl[f])) for f in range(n)]
    got = []
    for t in tickets:
        r = srv.wait(t)
        assert r["status"] == daq.DAQ_OK
        got.append(srv.fetch(t))
        srv.release(t)
    st = srv.stats()
    assert st["max_running"] > 1           # the mix really overlapped
    q_mix = srv.q.cpu().numpy().copy()
    srv.close()
    q_ref = 0
    for f in range(n):
        ref = oracle.process_fills(s[f:f + 1], w.params(), fill_len=fl[f:f + 1], n_threads=8)
        for k, (a, b) in enumerate([(alone[f], got[f])]):
            for part_a, part_b in zip(a, b):
                assert np.array_equal(part_a, part_b), f
        isl = alone[f][0].copy()
        isl["fill"] = 0
        assert np.array_equal(isl, ref["islands"]), f
        assert np.array_equal(alone[f][1], ref["pool"]), f
        assert np.array_equal(alone[f][2], ref["pedestal"][0]), f
        q_ref = q_ref + ref["q"]
    assert np.array_equal(q_alone, q_ref) and np.array_equal(q_mix, q_ref)


@pytest.mark.gpu
def test_sparse_fills_served_with_the_sparse_flag(genv):
    """Processing flags reach the served fills: sparse fills served with
    DAQ_SPARSE, several at once, each match the oracle."""
    torch, daq, oracle = genv["torch"], genv["daq"], genv["oracle"]
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_fills=4, n_calo=2)
    s = genv["synth"].generate(w.config())
    F, C, X, N = s.shape
    dev = [torch.from_numpy(s[f]).cuda() for f in range(F)]
    srv = _server(genv, w, C, N, 1 << 40, max_slots=4, n_streams=4, flags=daq.DAQ_SPARSE)
    tickets = [srv.submit(dev[f]) for f in range(F)]
    q_ref = 0
    for f, t in enumerate(tickets):
        r = srv.wait(t)
        assert r["status"] == daq.DAQ_OK
        isl, pool, ped = srv.fetch(t)[:3]
        srv.release(t)
        ref = oracle.process_fills(s[f:f + 1], w.params(), n_threads=8)
        isl = isl.copy()
        isl["fill"] = 0
        assert np.array_equal(isl, ref["islands"]) and np.array_equal(pool, ref["pool"]), f
        assert np.array_equal(ped, ref["pedestal"][0]), f
        q_ref = q_ref + ref["q"]
    assert np.array_equal(srv.q.cpu().numpy(), q_ref)
    srv.close()


@pytest.mark.gpu
def test_admission_respects_the_memory_budget(genv):
    torch, daq = genv["torch"], genv["daq"]
    w, s, fl = _fills(genv, 8)
    F, C, X, N = s.shape
    dev = [torch.from_numpy(s[f]).cuda() for f in range(8)]
    probe = _server(genv, w, C, N, 1 << 40, max_slots=1)
    slot = probe.stats()["slot_bytes"]
    probe.close()
    srv = _server(genv, w, C, N, 2 * slot + slot // 2, n_streams=4, auto_release=True)
    st = srv.stats()
    assert st["n_slots"] == 2 and st["mem_bytes"] <= 2 * slot + slot // 2
    tickets = [srv.submit(dev[f], int(fl[f])) for f in range(8)]
    srv.drain(120.0)
    st = srv.stats()
    assert st["completed"] == 8 and st["failed"] == 0 and 1 <= st["max_running"] <= 2
    recs = srv.records()
    assert sorted(r.ticket for r in recs) == tickets
    assert all(r.slot in (0, 1) for r in recs)
    srv.close()


@pytest.mark.gpu
def test_host_submitted_fills_match_device_submitted(genv):
    torch, daq = genv["torch"], genv["daq"]
    w, s, fl = _fills(genv, 3, n_calo=2, n_samples=24_000)
    F, C, X, N = s.shape
    srv = _server(genv, w, C, N, 1 << 40, max_slots=3, host_input=True)
    host = [torch.from_numpy(s[f]).pin_memory() for f in range(3)]
    dev = [torch.from_numpy(s[f]).cuda() for f in range(3)]
    th = [srv.submit(host[f], int(fl[f])) for f in range(3)]
    res_h = []
    for t in th:
        srv.wait(t)
        res_h.append(srv.fetch(t))
        srv.release(t)
    for f in range(3):
        t = srv.submit(dev[f], int(fl[f]))
        srv.wait(t)
        for a, b in zip(res_h[f], srv.fetch(t)):
            assert np.array_equal(a, b)
        srv.release(t)
    srv.close()


@pytest.mark.gpu
def test_replayed_arrivals_are_honoured(genv):
    torch, daq = genv["torch"], genv["daq"]
    w, s, fl = _fills(genv, 4, n_calo=2, n_samples=24_000)
    F, C, X, N = s.shape
    dev = [torch.from_numpy(s[f]).cuda() for f in range(4)]
    srv = _server(genv, w, C, N, 1 << 40, max_slots=4, auto_release=True)
    t0 = srv.now_us() + 20_000.0
    arrivals = [t0 + 5_000.0 * k for k in range(4)]
    for f in range(4):
        srv.submit(dev[f], int(fl[f]), arrival_us=arrivals[f])
    srv.drain(60.0)
    recs = sorted(srv.records(), key=lambda r: r.ticket)
    for r, a in zip(recs, arrivals):
        assert r.t_arrival == a
        assert r.t_admit >= a                      # held until its arrival time
        assert a - 50.0 <= r.t_start <= r.t_done   # started after arrival (clock anchoring slack)
    summ = daq.daq_serving_summarize(recs)
    assert summ.deadtime == 0.0                    # 5 ms spacing, small fills
    srv.close()
