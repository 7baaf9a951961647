"""End-to-end host form (daq_process_fills_host) and calorimeter-group calls.

The host form pipelines chunks of calorimeter-fills over copy and compute
streams; whatever the chunking, the host buffers must hold exactly the
oracle's records, pool rows, pedestals and counts, and Q must accumulate the
oracle's bins.  Calorimeter-group calls (calo_base / q_calos) must write the
true calorimeter indices and Q rows."""
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
    import oracle
    import synth
    import paper_1611_04959_gb300 as daq
    return dict(torch=torch, oracle=oracle, synth=synth, daq=daq)


def split_streams(buf: np.ndarray, total: int) -> list:
    """The back-to-back packed streams of the host form: (stream bytes, rows, n_xtal)."""
    out, at = [], 0
    while at < total:
        head = buf[at: at + 16]
        X = int(head[4:8].view("<u4")[0])
        rows = int(head[8:16].view("<u8")[0])
        nb = -(-rows // 32)
        payload = int(buf[at + 16 + 8 * nb: at + 24 + 8 * nb].view("<u8")[0])
        size = 16 + 8 * (nb + 1) + payload
        out.append((buf[at: at + size], rows, X))
        at += size
    assert at == total
    return out


def run_host(env, s, params, fill_len=None, dev_rows=None, dev_hdr=None, host_rows=None, q=None, pack=False,
             locked_out=True):
    """locked_out: page-locked record and pool buffers (the device writes them);
    else pageable ones (copy engines after host waits)."""
    torch, daq = env["torch"], env["daq"]
    F, C, X, N = s.shape
    host = torch.from_numpy(s).pin_memory()
    sdev = torch.empty_like(host, device="cuda")
    rows = F * C * N + 8 * 64
    out = daq.Outputs(torch, "cuda", F, C, X, dev_hdr if dev_hdr is not None else F * C * ((N + 1) // 2),
                      dev_rows if dev_rows is not None else rows)
    hrows = host_rows if host_rows is not None else F * C * N
    n_rec = max(1, F * C * N // 2 + F * C)
    if locked_out:
        hdr_t = torch.zeros(n_rec * daq.ISLAND_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
        hdr_h = hdr_t.numpy().view(daq.ISLAND_DTYPE)
        pool_t = torch.zeros((max(1, hrows), X), dtype=torch.int16).pin_memory()
    else:
        hdr_t, hdr_h = None, np.zeros(n_rec, daq.ISLAND_DTYPE)
        pool_t = torch.from_numpy(np.zeros((max(1, hrows), X), np.int16))
    ped_h = np.zeros((F, C, X), np.int32)
    counts_h = np.zeros(4, np.int64)
    if q is None:
        q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    fl = None if fill_len is None else torch.as_tensor(np.asarray(fill_len, np.int32), device="cuda")
    stream = torch.cuda.Stream()
    p = daq.make_params(**params, fill_len=fl, stream=stream)
    ws = torch.empty(daq.daq_workspace_size(C, X, N, F, p), dtype=torch.uint8, device="cuda")
    p.workspace, p.workspace_bytes = ws.data_ptr(), ws.numel()
    io = daq.DaqHostIO(host.data_ptr(), sdev.data_ptr(), hdr_h.ctypes.data, len(hdr_h), pool_t.data_ptr(), hrows,
                       ped_h.ctypes.data, counts_h.ctypes.data)
    if pack:
        p.flags |= daq.DAQ_PACK_POOL
        cap = daq.daq_pack_bound(F * C * N, X) + 64 * 8192
        pdev = torch.empty(cap, dtype=torch.uint8, device="cuda")
        phost = np.zeros(cap, np.uint8)
        pbytes = np.zeros(1, np.int64)
        io.packed_dev, io.packed_dev_cap = pdev.data_ptr(), cap
        io.packed_host, io.packed_host_cap, io.packed_bytes_host = phost.ctypes.data, cap, pbytes.ctypes.data
    rc = daq.daq_process_fills_host(C, X, N, F, p, out.struct(), q.data_ptr(), io)
    if pack:
        pool = [env["oracle"].unpack(st, rows, xx) for st, rows, xx in split_streams(phost, int(pbytes[0]))]
        pool = np.concatenate(pool) if pool else np.zeros((0, X), np.int16)
        return rc, counts_h, hdr_h.copy(), pool, ped_h, q
    return rc, counts_h, hdr_h.copy(), pool_t.numpy().copy(), ped_h, q


def check(res, ref):
    rc, counts, hdr, pool, ped, q = res
    assert rc == 0, (rc, counts)
    n, r = ref["n_islands"], ref["n_rows"]
    assert int(counts[0]) == n and int(counts[1]) == r and int(counts[2]) == 0
    assert np.array_equal(hdr[:n], ref["islands"])
    assert np.array_equal(pool[:r], ref["pool"])
    assert np.array_equal(ped, ref["pedestal"])
    assert np.array_equal(q.cpu().numpy(), ref["q"])


@pytest.mark.parametrize("locked_out", [True, False])
@pytest.mark.parametrize("F,C,N", [(1, 24, 20_000), (1, 5, 33_000), (3, 2, 16_000), (16, 3, 8_000), (1, 1, 50_000),
                                   (2, 3, 20_001)])
def test_pipelined_host_form_matches_oracle(env, F, C, N, locked_out):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_fills=F, n_calo=C, n_samples=N)
    s = env["synth"].generate(w.config())
    ref = env["oracle"].process_fills(s, w.params(), n_threads=8)
    check(run_host(env, s, w.params(), locked_out=locked_out), ref)


@pytest.mark.parametrize("pack", [False, True])
def test_host_form_passes_the_sparse_flag_through(env, pack):
    """DAQ_SPARSE reaches every chunk's processing: a sparse fill through the
    host form, plain and packed, matches the oracle."""
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_calo=3)
    s = env["synth"].generate(w.config())
    ref = env["oracle"].process_fills(s, w.params(), n_threads=8)
    assert 0 < ref["n_rows"] < 0.2 * s.shape[1] * s.shape[3]
    check(run_host(env, s, dict(w.params(), flags=env["daq"].DAQ_SPARSE), pack=pack), ref)


def test_host_form_with_fill_lengths_and_two_decimations(env):
    from synth import workloads as W
    w = W.scaled(W.STRESS, n_fills=4, n_calo=3, n_samples=24_000)
    fl = np.array([24_000, 7_001, 0, 19_999], np.int32)
    s = env["synth"].generate(w.config(), fill_len=fl)
    ref = env["oracle"].process_fills(s, w.params(), fill_len=fl, n_threads=8)
    check(run_host(env, s, w.params(), fill_len=fl), ref)


@pytest.mark.parametrize("locked_out", [True, False])
def test_host_form_single_chunk_when_device_capacity_is_small(env, locked_out):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=6, n_samples=20_000)
    s = env["synth"].generate(w.config())
    ref = env["oracle"].process_fills(s, w.params(), n_threads=8)
    rows = ref["n_rows"] + 1000                     # enough for the result, not for every chunk's worst case
    check(run_host(env, s, w.params(), dev_rows=rows, dev_hdr=ref["n_islands"] + 10, locked_out=locked_out), ref)


@pytest.mark.parametrize("locked_out", [True, False])
def test_host_form_reports_short_host_capacity(env, locked_out):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=4, n_samples=20_000)
    s = env["synth"].generate(w.config())
    ref = env["oracle"].process_fills(s, w.params(), n_threads=8)
    rc, counts, hdr, pool, ped, q = run_host(env, s, w.params(), host_rows=ref["n_rows"] // 2, locked_out=locked_out)
    assert rc == env["daq"].DAQ_ECAPACITY
    assert int(counts[1]) == ref["n_rows"] and int(counts[0]) == ref["n_islands"]
    assert np.array_equal(pool[: ref["n_rows"] // 2], ref["pool"][: ref["n_rows"] // 2])


def test_calorimeter_groups_write_true_indices_and_q_rows(env):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.scaled(W.STRESS, n_calo=7, n_fills=1, n_samples=16_000)
    s = env["synth"].generate(w.config())
    params = w.params()
    ref = oracle.process_fills(s, params, n_threads=8)
    F, C, X, N = s.shape
    x = torch.from_numpy(s).cuda()
    q = torch.zeros(daq.q_size(C, N, params["decim"]), dtype=torch.int64, device="cuda")
    isl, pools = [], []
    for c0, nc in [(0, 3), (3, 1), (4, 3)]:
        res = daq.process_fills(x[:, c0:c0 + nc].contiguous(), q=q, calo_base=c0, q_calos=C, **params)
        assert res["status"] == daq.DAQ_OK
        isl.append(res["outputs"].islands_host(res["n_islands"]))
        pools.append(res["outputs"].pool[: res["n_rows"]].cpu().numpy())
    rows = 0
    for part in isl:
        part["pool_row"] += rows
        rows += int(part["len"].sum())
    assert np.array_equal(np.concatenate(isl), ref["islands"])
    assert np.array_equal(np.concatenate(pools), ref["pool"])
    assert np.array_equal(q.cpu().numpy(), ref["q"])


@pytest.mark.parametrize("F,C,N", [(1, 24, 20_000), (3, 2, 16_000), (1, 1, 50_000)])
def test_packed_host_form_matches_oracle(env, F, C, N):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_fills=F, n_calo=C, n_samples=N)
    s = env["synth"].generate(w.config())
    ref = env["oracle"].process_fills(s, w.params(), n_threads=8)
    check(run_host(env, s, w.params(), pack=True), ref)
