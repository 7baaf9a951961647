"""Per-crystal full-resolution fill sum (daq_crystal_sum) vs the oracle,
element by element (int64, exact): random shapes with ragged pitches, uneven
fill lengths and several fills per call; accumulation across calls; and the
benchmark's full fill (24 x 54 x 560,000) on sampled crystal rows."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def daq():
    from paper_1611_04959_gb300 import build
    build.build()
    import paper_1611_04959_gb300 as d
    return d


def test_workspace_and_argument_checks_without_device_work(daq):
    assert daq.daq_crystal_sum_workspace_size(24, 54, 1) >= 24 * 54 * 4
    p = daq.make_params(ped_samples=0)
    assert daq.daq_crystal_sum(0, 1, 1, 8, 1, p, None) == daq.DAQ_EINVAL      # ped_samples < 1
    p = daq.make_params()
    assert daq.daq_crystal_sum(0, 1, 1, 8, 1, p, None) == daq.DAQ_EINVAL      # no workspace
    with pytest.raises(daq.DaqError):
        daq.daq_crystal_sum_workspace_size(1, 0, 1)


@pytest.fixture(scope="module")
def env(daq):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import synth
    return dict(torch=torch, oracle=oracle, synth=synth, daq=daq)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(12))
def test_random_shapes_match_oracle(env, seed):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    rng = np.random.default_rng(500 + seed)
    F, C = int(rng.integers(1, 4)), int(rng.integers(1, 4))
    X = int(rng.choice([1, 3, 54, 64]))
    N = int(rng.integers(1, 3000))
    if seed % 2:
        N = (N + 7) // 8 * 8
    s = rng.integers(-3000, 4096, size=(F, C, X, N)).astype(np.int16)
    lens = None
    if seed % 3:
        lens = rng.integers(0, N + 1, size=F).astype(np.int32)
    ped = int(rng.integers(1, 150))
    want = oracle.crystal_sum(s, fill_len=lens, ped_samples=ped)
    got = daq.crystal_sum(torch.from_numpy(s).cuda(), ped_samples=ped, fill_len=lens)
    assert np.array_equal(got.cpu().numpy(), want), (F, C, X, N, ped)


@pytest.mark.gpu
def test_accumulates_across_calls_and_flags_bad_length(env):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.scaled(W.PLAIN_FULL_FILL, n_fills=3, n_calo=2, n_samples=24_000)
    s = env["synth"].generate(w.config())
    x = torch.from_numpy(s).cuda()
    q = daq.crystal_sum(x[:2].contiguous())
    q = daq.crystal_sum(x[2:].contiguous(), q=q)
    assert np.array_equal(q.cpu().numpy(), oracle.crystal_sum(s))
    with pytest.raises(daq.DaqError) as e:
        daq.crystal_sum(x, fill_len=[24_000, 24_001, 5])
    assert e.value.status == daq.DAQ_EINVAL


@pytest.mark.gpu
def test_full_fill_sampled_rows(env):
    torch, daq, oracle = env["torch"], env["daq"], env["oracle"]
    from synth import workloads as W
    w = W.PLAIN_FULL_FILL
    s = env["synth"].generate(w.config())
    q = daq.crystal_sum(torch.from_numpy(s).cuda())
    rng = np.random.default_rng(3)
    for c, x in zip(rng.integers(0, 24, 12), rng.integers(0, 54, 12)):
        want = oracle.crystal_sum(np.ascontiguousarray(s[:, c:c + 1, x:x + 1, :]))[0, 0]
        assert np.array_equal(q[c, x].cpu().numpy(), want), (c, x)
    # invariant at full size: per calorimeter, the crystal sum over all samples equals sum(S)
    tot = q.sum(dim=(1, 2)).cpu().numpy()
    ref = oracle.process_fills(s, dict(w.params(), threshold=10 ** 9, decim=(560_000,)), n_threads=16)["q"]
    assert np.array_equal(tot, ref)
