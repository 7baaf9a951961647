"""The scratch-free entry point (daq_process_fills_static) against the regular one.

Some callers cannot allocate device memory (a fixed budget set at start-up, a
host framework that owns all allocations, a real-time loop that must not
allocate); daq_process_fills_static serves them from a scratch area built into
the library.  This file runs last so that a failure here leaves every other
test already run; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import synth
    import paper_1611_04959_gb300 as daq
    return torch, synth, daq


def _outputs(torch, daq, F, C, X, rows):
    return daq.Outputs(torch, torch.device("cuda"), F, C, X, rows // 2 + F * C + 1, rows)


def test_static_scratch_matches_regular_call_twice(env):
    torch, synth, daq = env
    from synth import workloads as W
    w = W.scaled(W.STRESS, n_fills=2, n_calo=3, n_samples=60_000)
    s = torch.from_numpy(synth.generate(w.config())).cuda()
    F, C, X, N = s.shape
    params = w.params()
    # regular entry point, caller-provided workspace
    ref = daq.process_fills(s, **params)
    ref_out, ref_q = ref["outputs"], ref["q"].cpu().numpy()
    n_isl, n_rows = ref["n_islands"], ref["n_rows"]
    for call in range(2):   # the shared area keeps the previous call's contents
        out = _outputs(torch, daq, F, C, X, F * C * N)
        q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
        p = daq.make_params(**params, flags=daq.DAQ_SYNC, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = daq.daq_process_fills_static(s.data_ptr(), C, X, N, F, p, out.struct(), q.data_ptr())
        assert rc == daq.DAQ_OK, (call, rc, daq.strerror(rc))
        if call == 1:  # the first call may place the area (lazy module loading); the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        counts = out.counts.cpu().numpy()
        assert int(counts[0]) == n_isl and int(counts[1]) == n_rows, call
        assert np.array_equal(out.islands_host(n_isl), ref_out.islands_host(n_isl)), call
        assert np.array_equal(out.pool[:n_rows].cpu().numpy(), ref_out.pool[:n_rows].cpu().numpy()), call
        assert np.array_equal(out.pedestal.cpu().numpy(), ref_out.pedestal.cpu().numpy()), call
        assert np.array_equal(q.cpu().numpy(), ref_q), call


def test_static_scratch_rejects_oversized_calls(env):
    torch, synth, daq = env
    p = daq.make_params()
    need = daq.daq_workspace_size(24, 54, 560_000, 4, p)
    assert need > daq.DAQ_STATIC_SCRATCH_BYTES
    assert daq.daq_workspace_size(24, 54, 560_000, 1, p) <= daq.DAQ_STATIC_SCRATCH_BYTES
    out = _outputs(torch, daq, 1, 1, 54, 16)
    # refused before any device work, so the sample pointer is never used
    rc = daq.daq_process_fills_static(out.pool.data_ptr(), 24, 54, 560_000, 4, p, out.struct(), None)
    assert rc == daq.DAQ_ESCRATCH
    assert "scratch" in daq.strerror(rc)
