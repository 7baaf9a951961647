"""Stress workload at full size: 48 fills x 24 calorimeters x 54 crystals x
560,000 samples (69.67 GB on the device), 10x pulse rate, T = 15, post = 64,
decimations 8 and 32, in the launch configuration the benchmark times (one
call, default form).

The 48 fills cycle over 4 distinct generated fills (fill f holds fill f % 4 of
the stress generator), so that the oracle can give the exact expected output
of every fill: each distinct fill's records (fill index and pool offset
shifted), its pool rows and its Q bins times the number of times it occurs.
Every record, every pool row (compared on the device) and every Q bin is
checked."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_FILLS, N_DISTINCT = 48, 4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 160e9:
        pytest.skip("needs ~160 GB of free device memory")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    import paper_1611_04959_gb300 as daq
    return dict(torch=torch, oracle=oracle, synth=synth, daq=daq)


def test_stress_batch_full_size(env):
    import os
    torch, oracle, synth, daq = env["torch"], env["oracle"], env["synth"], env["daq"]
    from synth import workloads as W
    w = W.STRESS
    params = w.params()
    C, X, N = w.n_calo, 54, w.n_samples
    threads = os.cpu_count() or 1
    distinct = synth.generate(w.config(), fills=(0, N_DISTINCT), n_threads=threads)
    refs = [oracle.process_fills(distinct[d:d + 1], params, n_threads=threads) for d in range(N_DISTINCT)]

    x = torch.empty((N_FILLS, C, X, N), dtype=torch.int16, device="cuda")
    for d in range(N_DISTINCT):
        x[d].copy_(torch.from_numpy(distinct[d]))
    for f in range(N_DISTINCT, N_FILLS):
        x[f].copy_(x[f % N_DISTINCT])
    mult = N_FILLS // N_DISTINCT
    n_isl = sum(r["n_islands"] for r in refs) * mult
    n_rows = sum(r["n_rows"] for r in refs) * mult
    assert n_rows > 0.99 * N_FILLS * C * N                      # heavy merging: nearly every sample marked
    out = daq.Outputs(torch, "cuda", N_FILLS, C, X, n_isl + 16, n_rows + 16)
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    res = daq.process_fills(x, q=q, outputs=out, **params)
    assert res["status"] == daq.DAQ_OK
    assert res["n_islands"] == n_isl and res["n_rows"] == n_rows

    # Q: each distinct fill's bins, mult times
    q_ref = sum(r["q"] for r in refs) * mult
    assert np.array_equal(q.cpu().numpy(), q_ref)

    # records of every fill
    got = out.islands_host(n_isl)
    parts, rows_before = [], 0
    row_start = []
    for f in range(N_FILLS):
        r = refs[f % N_DISTINCT]
        e = r["islands"].copy()
        e["fill"] = f
        e["pool_row"] += rows_before
        parts.append(e)
        row_start.append(rows_before)
        rows_before += r["n_rows"]
    assert np.array_equal(got, np.concatenate(parts))

    # pool rows of every fill, compared on the device
    del x
    exp = [torch.from_numpy(refs[d]["pool"]).cuda() for d in range(N_DISTINCT)]
    for f in range(N_FILLS):
        d = f % N_DISTINCT
        seg = out.pool[row_start[f]: row_start[f] + refs[d]["n_rows"]]
        assert torch.equal(seg, exp[d]), f
    ped = out.pedestal.cpu().numpy()
    for f in range(N_FILLS):
        assert np.array_equal(ped[f], refs[f % N_DISTINCT]["pedestal"][0]), f
