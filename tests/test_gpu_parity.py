"""CUDA path vs oracle, bit-exact (every output is an integer).

Each case runs libdaq through the C ABI on seeded synthetic input and compares
island records, pool rows, pedestals, counts and int64 Q histograms element by
element with the oracle on the same input."""
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


def compare(env, s, params, fill_len=None, n_threads=8, **kw):
    torch, oracle, daq = env["torch"], env["oracle"], env["daq"]
    ref = oracle.process_fills(s, params, fill_len=fill_len, n_threads=n_threads)
    fl = None if fill_len is None else torch.as_tensor(np.asarray(fill_len, np.int32), device="cuda")
    res = daq.process_fills(torch.from_numpy(s).cuda(), fill_len=fl, **params, **kw)
    out = res["outputs"]
    ctx = dict(shape=s.shape, params=params, kw=kw)
    assert res["status"] == daq.DAQ_OK, (res["status"], res["counts"], ctx)
    assert res["n_islands"] == ref["n_islands"], ctx
    assert res["n_rows"] == ref["n_rows"], ctx
    got_isl = out.islands_host(res["n_islands"])
    assert np.array_equal(got_isl, ref["islands"]), ctx
    assert np.array_equal(out.pool[: res["n_rows"]].cpu().numpy(), ref["pool"]), ctx
    assert np.array_equal(out.pedestal.cpu().numpy(), ref["pedestal"]), ctx
    if params.get("decim"):
        assert np.array_equal(res["q"].cpu().numpy(), ref["q"]), ctx
    return res, ref


def test_plain_one_calorimeter_full_fill(env):
    from synth import workloads as W
    w = W.PLAIN_1CALO
    s = env["synth"].generate(w.config())
    res, ref = compare(env, s, w.params())
    assert ref["n_islands"] > 100


@pytest.mark.parametrize("tile", [128, 224, 384, 448, 960])
@pytest.mark.parametrize("grid", [0, -1, -2, -3, -4, -5, -6, 1, 5])
def test_tile_and_grid_invariance(env, tile, grid):
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=3, n_samples=40_000)
    s = env["synth"].generate(w.config())
    compare(env, s, w.params(), tile=tile, grid=grid)


def _random_case(rng):
    X = int(rng.choice([1, 2, 3, 5, 8, 17, 31, 32, 33, 54, 63, 64]))
    N = int(rng.integers(1, 6000))
    if rng.random() < 0.5:
        N = (N + 7) // 8 * 8
    F, C = int(rng.integers(1, 4)), int(rng.integers(1, 4))
    pre, post = int(rng.integers(0, 40)), int(rng.integers(0, 70))
    if rng.random() < 0.2:
        pre, post = int(rng.integers(0, 250)), int(rng.integers(0, 250))
    nd = int(rng.integers(0, 3))
    decim = tuple(int(rng.choice([1, 3, 8, 16, 32, 7, 64, 100])) for _ in range(nd))
    amp = int(rng.integers(1, 200))
    s = rng.integers(-amp, amp + 1, size=(F, C, X, N)).astype(np.int16)
    if rng.random() < 0.3:                                  # extreme int16 values
        s[rng.random(s.shape) < 0.01] = rng.choice([-32768, 32767])
    spread = amp * np.sqrt(X)
    T = int(rng.normal(0.3, 0.6) * spread)
    params = dict(threshold=T, pre=pre, post=post, ped_samples=int(rng.integers(1, 150)), decim=decim)
    fill_len = None
    if rng.random() < 0.5:
        fill_len = rng.integers(0, N + 1, size=F).astype(np.int32)
        fill_len[rng.random(F) < 0.2] = N
    tile = int(rng.choice([0, 128, 224, 384, 448]))
    return s, params, fill_len, tile


@pytest.mark.parametrize("seed", range(40))
def test_random_shapes(env, seed):
    rng = np.random.default_rng(1000 + seed)
    s, params, fill_len, tile = _random_case(rng)
    hl = (params["post"] + 8) // 8 * 8
    hr = (params["pre"] + 8) // 8 * 8
    if tile and tile + hl + hr > 1024:
        tile = 0
    grid = int(rng.choice([0, 0, -1, -2, -3, -4, -4, 2, -5, -5, -6, -6, -6]))
    flags = 32 if grid >= 0 and seed % 2 else 0  # DAQ_SPARSE on half the two-pass cases
    compare(env, s, params, fill_len=fill_len, tile=tile, grid=grid, flags=flags)


@pytest.mark.parametrize("grid", [1, 3, 0])
@pytest.mark.parametrize("sparse", [True, False])
def test_compact_passes_over_tiles_without_marks(env, grid, sparse):
    """A sparse fill with stretches of flat samples (no crossing, no marks).
    With DAQ_SPARSE the compact pass takes only tiles that hold a marked
    sample, reading 32 records of a CTA's sequence at a time.  With grid = 1 one
    CTA takes all 5,000 tiles and passes the flat stretch (tiles ~764 to
    ~4,387) over many such reads; grid = 3 gives shorter sequences."""
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_calo=4)
    s = env["synth"].generate(w.config())
    # each crystal's integer pedestal over the first 100 samples: a sample at
    # that value adds nothing to the pedestal-subtracted sum
    P = ((s[:, :, :, :100].astype(np.int64).sum(-1) + 50) // 100).astype(np.int16)
    s[0, 0, :, 448_000:] = P[0, 0][:, None]
    s[0, 1, :, :] = P[0, 1][:, None]
    s[0, 2, :, :] = P[0, 2][:, None]
    s[0, 3, :, 100:280_000] = P[0, 3][:, None]
    res, ref = compare(env, s, w.params(), grid=grid, flags=env["daq"].DAQ_SPARSE if sparse else 0)
    isl = ref["islands"]
    assert len(isl) > 100
    assert not np.any((isl["calo"] == 1) | (isl["calo"] == 2))


def test_uneven_batch_of_fills(env):
    from synth import workloads as W
    w = W.scaled(W.BATCH_UNEVEN, n_calo=2)
    fl, rate = w.plan()
    s = env["synth"].generate(w.config(), fill_len=fl, rate=rate)
    compare(env, s, w.params(), fill_len=fl)


@pytest.mark.parametrize("tile,grid,flags", [(0, 0, 0), (384, 0, 0), (448, 0, 0), (0, -6, 0), (0, 0, 32)])
def test_stress_parameters(env, tile, grid, flags):
    """post = 64: the default plan keeps 448-sample tiles with the halo-free
    count pass (the scan completes each tile's marks); 384 is the halo'd plan;
    flags 32 (DAQ_SPARSE) passes the halo-free records to the sparse compact
    loop."""
    from synth import workloads as W
    w = W.scaled(W.STRESS, n_fills=2, n_calo=3)
    s = env["synth"].generate(w.config())
    res, ref = compare(env, s, w.params(), tile=tile, grid=grid, flags=flags)
    assert ref["n_rows"] > 0.95 * s.shape[0] * s.shape[1] * s.shape[3]   # heavy merging


def test_degenerate_inputs(env):
    params = dict(threshold=0, pre=2, post=3, ped_samples=4, decim=(8,))
    rng = np.random.default_rng(5)
    # all below threshold, all above, zero-length fills, single-sample fills
    z = np.zeros((2, 2, 5, 1000), np.int16)
    compare(env, z, params)
    up = z.copy()
    up[:, :, :, 4:] = 9
    compare(env, up, params)
    compare(env, rng.integers(-5, 6, size=(3, 2, 4, 640)).astype(np.int16), params, fill_len=[0, 1, 0])
    compare(env, rng.integers(-5, 6, size=(1, 1, 54, 8)).astype(np.int16), params)


def test_empty_batch(env):
    torch, daq = env["torch"], env["daq"]
    for shape in [(0, 24, 54, 1000), (2, 0, 54, 1000), (1, 2, 54, 0)]:
        s = torch.zeros(shape, dtype=torch.int16, device="cuda")
        res = daq.process_fills(s, hdr_cap=4, pool_cap=4)
        assert res["status"] == daq.DAQ_OK
        assert res["n_islands"] == 0 and res["n_rows"] == 0


@pytest.mark.parametrize("grid", [0, -4, -5, -6])
def test_capacity_overflow_reports_sizes_and_keeps_prefix(env, grid):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=2, n_samples=30_000)
    s = env["synth"].generate(w.config())
    ref = oracle.process_fills(s, w.params())
    hc, pc = ref["n_islands"] // 3, ref["n_rows"] // 2
    q0 = torch.zeros(daq.q_size(2, 30_000, (32,)), dtype=torch.int64, device="cuda")
    res = daq.process_fills(torch.from_numpy(s).cuda(), hdr_cap=hc, pool_cap=pc, q=q0, grid=grid, **w.params())
    assert res["status"] == daq.DAQ_ECAPACITY
    assert res["n_islands"] == ref["n_islands"] and res["n_rows"] == ref["n_rows"]
    assert res["counts"][2] & (daq.DAQ_DEV_HDR_OVERFLOW | daq.DAQ_DEV_POOL_OVERFLOW)
    out = res["outputs"]
    assert np.array_equal(out.islands_host(hc), ref["islands"][:hc])
    assert np.array_equal(out.pool[:pc].cpu().numpy(), ref["pool"][:pc])
    assert np.array_equal(q0.cpu().numpy(), ref["q"])          # Q is accumulated exactly once


@pytest.mark.parametrize("grid", [0, -4, -5, -6])
def test_q_accumulates_across_calls_and_skip_flags(env, grid):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.scaled(W.STRESS, n_fills=1, n_calo=2, n_samples=50_000)
    s = env["synth"].generate(w.config())
    ref = oracle.process_fills(s, w.params())
    ds = torch.from_numpy(s).cuda()
    q = torch.zeros(daq.q_size(2, 50_000, (8, 32)), dtype=torch.int64, device="cuda")
    daq.process_fills(ds, q=q, grid=grid, **w.params())
    daq.process_fills(ds, q=q, flags=daq.DAQ_SKIP_ISLANDS, grid=grid, **w.params())
    r3 = daq.process_fills(ds, q=q, flags=daq.DAQ_SKIP_Q, grid=grid, **w.params())
    assert np.array_equal(q.cpu().numpy(), 2 * ref["q"])
    assert r3["n_islands"] == ref["n_islands"]


def test_fill_length_out_of_range_is_flagged(env):
    torch, daq = env["torch"], env["daq"]
    s = torch.zeros((2, 1, 3, 800), dtype=torch.int16, device="cuda")
    fl = torch.tensor([900, -3], dtype=torch.int32, device="cuda")
    with pytest.raises(daq.DaqError) as e:
        daq.process_fills(s, fill_len=fl, hdr_cap=10, pool_cap=10)
    assert e.value.status == daq.DAQ_EINVAL


@pytest.mark.parametrize("grid,flags", [(0, 0), (0, 32), (-4, 0), (-5, 0), (-6, 0)])
def test_full_fill_24_calorimeters(env, grid, flags):
    """The benchmark workload itself (1.45 GB), full parity: two-pass (also with
    DAQ_SPARSE = 32), single-launch, streaming and single-read forms."""
    from synth import workloads as W
    w = W.PLAIN_FULL_FILL
    s = env["synth"].generate(w.config())
    compare(env, s, w.params(), n_threads=16, grid=grid, flags=flags)


@pytest.mark.parametrize("grid,flags", [(0, 0), (0, 32), (-6, 0)])
def test_sparse_regime(env, grid, flags):
    """Per-crystal noise 3/sqrt(54): islands cover ~8% of the fill (flags 32:
    DAQ_SPARSE, the compact pass that passes over tiles without marks)."""
    from synth import workloads as W
    w = W.scaled(W.SPARSE_FULL_FILL, n_calo=3)
    s = env["synth"].generate(w.config())
    res, ref = compare(env, s, w.params(), grid=grid, flags=flags)
    assert 0.02 < ref["n_rows"] / (3 * s.shape[3]) < 0.2


def test_debug_checks_change_nothing_on_the_full_fill(env):
    """DAQ_DEBUG_CHECKS: the benchmark fill gives the same records, rows,
    pedestals and Q with the checks on as with them off, and no check fails."""
    torch, daq = env["torch"], env["daq"]
    from synth import workloads as W
    w = W.PLAIN_FULL_FILL
    s = torch.from_numpy(env["synth"].generate(w.config(), n_threads=16)).cuda()
    plain = daq.process_fills(s, **w.params())
    checked = daq.process_fills(s, flags=daq.DAQ_DEBUG_CHECKS, **w.params())
    assert plain["status"] == checked["status"] == daq.DAQ_OK
    assert checked["counts"][2] == 0
    assert plain["n_islands"] == checked["n_islands"] and plain["n_rows"] == checked["n_rows"]
    n, r = plain["n_rows"], plain["n_islands"]
    assert torch.equal(plain["outputs"].hdr[: 3 * r], checked["outputs"].hdr[: 3 * r])
    assert torch.equal(plain["outputs"].pool[:n], checked["outputs"].pool[:n])
    assert torch.equal(plain["outputs"].pedestal, checked["outputs"].pedestal)
    assert torch.equal(plain["q"], checked["q"])


@pytest.mark.parametrize("seed", range(0, 40, 3))
def test_random_shapes_with_debug_checks(env, seed):
    """The random cases again with every index checked before its store:
    bit-exact against the oracle and no check fails."""
    rng = np.random.default_rng(1000 + seed)
    s, params, fill_len, tile = _random_case(rng)
    grid = int(rng.choice([0, -1, -4, -5, -6]))
    res, _ = compare(env, s, params, fill_len=fill_len, tile=tile, grid=grid, flags=env["daq"].DAQ_DEBUG_CHECKS)
    assert res["counts"][2] == 0


@pytest.mark.parametrize("grid", [0, -1, -2, -3, -4, -5, -6])
def test_short_wait_limit_gives_up_cleanly(env, grid):
    """A 1 us limit on the waits for other CTAs' published state: the call ends
    (every CTA stops and its copies land), returns DAQ_OK or DAQ_ETIMEOUT, and
    the next call with the default limit is bit-exact against the oracle."""
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=4, n_samples=120_000)
    s = env["synth"].generate(w.config())
    ds = torch.from_numpy(s).cuda()
    statuses = []
    for _ in range(3):
        r = daq.process_fills(ds, grid=grid, wait_limit_ns=1000, allow=(daq.DAQ_ETIMEOUT,), **w.params())
        torch.cuda.synchronize()
        assert r["status"] in (daq.DAQ_OK, daq.DAQ_ETIMEOUT), r["status"]
        assert r["status"] == daq.DAQ_OK or r["counts"][2] & daq.DAQ_DEV_TIMEOUT
        statuses.append(r["status"])
    compare(env, s, w.params(), grid=grid)


def test_wait_limit_runs_out_and_the_next_call_is_exact(env):
    """The plain single-pass form launches one CTA per tile, and a tile's
    look-back reads the states its predecessors publish as they finish: on a
    fill of some 5,000 tiles many find one not yet published and must wait.
    With a 1 ns limit (the clock is read on every poll) such a wait runs out at
    its first poll.  The call returns DAQ_ETIMEOUT (flag set, no hang: every CTA
    returned), and the next call is bit-exact."""
    torch, daq = env["torch"], env["daq"]
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_calo=4)
    s = env["synth"].generate(w.config())
    ds = torch.from_numpy(s).cuda()
    r = daq.process_fills(ds, grid=-1, wait_limit_ns=1, allow=(daq.DAQ_ETIMEOUT,), **w.params())
    torch.cuda.synchronize()
    assert r["status"] == daq.DAQ_ETIMEOUT and r["counts"][2] & daq.DAQ_DEV_TIMEOUT
    compare(env, s, w.params(), grid=-1)
    compare(env, s, w.params(), grid=0)
