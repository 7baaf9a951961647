"""GPU lossless packing of pool rows (daq_pack_pool / daq_unpack_pool) against
the oracle's encoder and decoder: the streams must be byte-identical, and
decoding must give the pool back exactly, for ragged sizes (partial last
block, block counts on and around the scan's chunk boundary), every crystal
count up to 64, extreme sample values, the benchmark fill's own pool, short
output capacity and damaged streams."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def daq():
    from paper_1611_04959_gb300 import build
    build.build()
    import paper_1611_04959_gb300 as d
    return d


def test_bounds_and_argument_checks(daq):
    assert daq.daq_pack_bound(0, 54) == 24
    assert daq.daq_pack_bound(33, 2) == 16 + 8 * 3 + 2 * 2 * 4 * 18
    assert daq.daq_pack_bound(10, 65) == -1 and daq.daq_pack_bound(-1, 5) == -1
    assert daq.daq_pack_workspace_size(1000, 54) > 0
    assert daq.daq_pack_pool(0, 0, 65, 0, 0, 8, 0, 0, None) == daq.DAQ_EUNSUPPORTED     # n_xtal > 64
    assert daq.daq_pack_pool(0, 10, 4, 0, 0, None, 0, 0, None) == daq.DAQ_EINVAL      # no out_bytes
    assert daq.daq_pack_pool(2, 10, 4, 16, 1000, 8, 16, 4096, None) == daq.DAQ_EINVAL  # pool not 16-byte aligned
    assert daq.daq_unpack_pool(None, 100, 10, 4, 0, 0, None) == daq.DAQ_EINVAL


@pytest.fixture(scope="module")
def env(daq):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    return dict(torch=torch, oracle=oracle, daq=daq)


CASES = [(0, 3), (1, 1), (31, 2), (32, 54), (33, 54), (1000, 5), (4097, 3), (32 * 1024, 2), (32 * 1024 + 5, 7),
         (32 * 2048, 1), (777, 64), (500, 63)]


@pytest.mark.gpu
@pytest.mark.parametrize("rows,X", CASES)
def test_stream_matches_oracle_and_round_trips(env, rows, X):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    rng = np.random.default_rng(rows * 131 + X)
    if rows % 3 == 0:
        pool = rng.integers(-32768, 32768, size=(rows, X))
    else:
        pool = 1800 + np.cumsum(rng.integers(-6, 7, size=(rows, X)), axis=0)
    pool = np.asarray(pool).astype(np.int16)
    want = oracle.pack(pool)
    dev = torch.from_numpy(pool).cuda() if rows else torch.zeros((1, X), dtype=torch.int16, device="cuda")
    got, n = daq.pack_pool(dev, rows)
    assert n == want.size
    assert np.array_equal(got.cpu().numpy(), want)
    back = daq.unpack_pool(got, rows, X)
    assert np.array_equal(back.cpu().numpy(), pool)
    back2 = daq.unpack_pool(torch.from_numpy(want).cuda(), rows, X)       # the oracle's stream decodes too
    assert np.array_equal(back2.cpu().numpy(), pool)


@pytest.mark.gpu
def test_crystal_counts_in_any_order(env):
    """The packing kernels size their shared memory by the crystal count: calls
    with a large, a small and again the large count, in one process, all run
    and match the oracle (a smaller call must not lower the kernels' limit)."""
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    for k, (rows, X) in enumerate([(4000, 64), (300, 1), (70, 2), (4000, 64), (1000, 54), (33, 3), (1000, 54)]):
        rng = np.random.default_rng(900 + k)
        pool = (1800 + np.cumsum(rng.integers(-9, 10, size=(rows, X)), axis=0)).astype(np.int16)
        got, n = daq.pack_pool(torch.from_numpy(pool).cuda(), rows)
        assert np.array_equal(got.cpu().numpy(), oracle.pack(pool)), (rows, X)


@pytest.mark.gpu
@pytest.mark.parametrize("rows,X", [(777, 54), (4096 + 13, 7), (2000, 64), (1500, 9)])
def test_every_width_class_and_mix(env, rows, X):
    """Columns whose row-to-row steps span every width class: <= 7 bits (four
    columns per transpose), 8-15 (pairs), 16-17 (alone), in every mix along a
    row, so each group size meets each fallback."""
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    rng = np.random.default_rng(rows * 7 + X)
    scale = 2 ** (np.arange(X) * 5 % 17)                     # step sizes 1 .. 65536 across the columns
    steps = rng.integers(-1, 2, size=(rows, X)) * rng.integers(0, scale + 1, size=(rows, X))
    pool = (np.cumsum(steps, axis=0) % 65536 - 32768).astype(np.int16)
    want = oracle.pack(pool)
    got, n = daq.pack_pool(torch.from_numpy(pool).cuda(), rows)
    assert n == want.size and np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(daq.unpack_pool(got, rows, X).cpu().numpy(), pool)
    assert np.array_equal(daq.unpack_pool(torch.from_numpy(want).cuda(), rows, X).cpu().numpy(), pool)


@pytest.mark.gpu
def test_full_fill_pool(env):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    import synth
    from synth import workloads as W
    w = W.PLAIN_FULL_FILL
    s = synth.generate(w.config())
    res = daq.process_fills(torch.from_numpy(s).cuda(), **w.params())
    rows = res["n_rows"]
    pool = res["outputs"].pool[:rows]
    got, n = daq.pack_pool(pool, rows)
    host_pool = pool.cpu().numpy()
    want = oracle.pack(host_pool)
    assert n == want.size and np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(daq.unpack_pool(got, rows, 54).cpu().numpy(), host_pool)
    assert host_pool.nbytes / n > 2.0          # noise-dominated rows: a few bits per sample


@pytest.mark.gpu
def test_short_capacity_and_damaged_streams(env):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    rng = np.random.default_rng(4)
    pool = (1800 + np.cumsum(rng.integers(-4, 5, size=(300, 6)), axis=0)).astype(np.int16)
    want = oracle.pack(pool)
    dev = torch.from_numpy(pool).cuda()
    cap = want.size // 2
    out = torch.full((want.size + 64,), 0xAB, dtype=torch.uint8, device="cuda")
    ws = torch.empty(daq.daq_pack_workspace_size(300, 6), dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = daq.daq_pack_pool(dev.data_ptr(), 300, 6, out.data_ptr(), cap, nbytes.data_ptr(), ws.data_ptr(), ws.numel(),
                           None)
    assert rc == daq.DAQ_OK
    torch.cuda.synchronize()
    assert int(nbytes.item()) == want.size                   # the size needed
    o = out.cpu().numpy()
    assert np.array_equal(o[:cap], want[:cap]) and (o[cap:] == 0xAB).all()
    with pytest.raises(daq.DaqError):                         # cut short
        daq.unpack_pool(torch.from_numpy(want[: want.size - 8]).cuda(), 300, 6)
    with pytest.raises(daq.DaqError):                         # header does not match
        daq.unpack_pool(torch.from_numpy(want).cuda(), 299, 6)
