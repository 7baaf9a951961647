"""The C ABI library loads and exports every declared symbol; host-only calls
and argument validation work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def daq():
    from paper_1611_04959_gb300 import build
    build.build()
    import paper_1611_04959_gb300 as d
    return d


def declared_functions() -> list:
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(daq_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(daq):
    names = declared_functions()
    assert "daq_process_fills" in names and "daq_workspace_size" in names
    lib = ctypes.CDLL(daq.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header(daq):
    # daq_params: 8 int32, pointer, uint32 + 3 int32, 2 pointers, size_t, 2 pointers, 2 int32, uint64
    assert ctypes.sizeof(daq.DaqParams) == 32 + 8 + 16 + 8 + 8 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(daq.DaqIslands) == 6 * 8
    assert daq.ISLAND_DTYPE.itemsize == 24


def test_binding_layout_matches_the_c_compiler(daq, tmp_path):
    """The ctypes mirrors of daq_params, daq_islands and daq_tune_result have
    the sizes and field offsets a C compiler gives the header's structs."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "daq.h"\n'
        'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(daq_params), offsetof(daq_params, wait_limit_ns),'
        ' offsetof(daq_params, lag_tiles), offsetof(daq_params, stream), sizeof(daq_islands),'
        ' sizeof(daq_tune_result), offsetof(daq_tune_result, flags)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    P = daq.DaqParams
    assert got == [ctypes.sizeof(P), P.wait_limit_ns.offset, P.lag_tiles.offset, P.stream.offset,
                   ctypes.sizeof(daq.DaqIslands), ctypes.sizeof(daq.DaqTuneResult), daq.DaqTuneResult.flags.offset]


def test_debug_checks_flag_and_status(daq):
    """DAQ_DEBUG_CHECKS is its own flag bit; a failed device index check
    (DAQ_DEV_BAD_INDEX) maps to DAQ_EINDEX, after timeouts and bad fill
    lengths and before capacity shortfalls."""
    flags = [daq.DAQ_SKIP_Q, daq.DAQ_SKIP_ISLANDS, daq.DAQ_SYNC, daq.DAQ_PACK_POOL, daq.DAQ_DEBUG_CHECKS, daq.DAQ_SPARSE]
    assert len(set(flags)) == len(flags) and all(f & (f - 1) == 0 for f in flags)
    bits = [daq.DAQ_DEV_HDR_OVERFLOW, daq.DAQ_DEV_POOL_OVERFLOW, daq.DAQ_DEV_TIMEOUT, daq.DAQ_DEV_BAD_FILL_LEN,
            daq.DAQ_DEV_BAD_INDEX]
    assert len(set(bits)) == len(bits) and all(b & (b - 1) == 0 for b in bits)
    assert daq.daq_status_from_counts([0, 0, daq.DAQ_DEV_BAD_INDEX, 0]) == daq.DAQ_EINDEX
    assert daq.daq_status_from_counts([0, 0, daq.DAQ_DEV_BAD_INDEX | daq.DAQ_DEV_POOL_OVERFLOW, 0]) == daq.DAQ_EINDEX
    assert daq.daq_status_from_counts([0, 0, daq.DAQ_DEV_BAD_INDEX | daq.DAQ_DEV_TIMEOUT, 0]) == daq.DAQ_ETIMEOUT
    assert "index" in daq.strerror(daq.DAQ_EINDEX)
    assert daq.make_params(flags=daq.DAQ_DEBUG_CHECKS).flags == daq.DAQ_DEBUG_CHECKS
    assert daq.make_params(wait_limit_ns=1000).wait_limit_ns == 1000
    assert daq.lib().daq_version() >= 102


def test_host_calls(daq):
    p = daq.daq_params_default()
    assert (p.threshold, p.pre, p.post, p.ped_samples, p.n_decim, p.decim[0]) == (30, 8, 24, 100, 1, 32)
    assert daq.daq_q_bins(560_000, 32) == 17_500 and daq.daq_q_bins(560_001, 32) == 17_501
    ws = daq.daq_workspace_size(24, 54, 560_000, 1, p)
    tiles = 24 * -(-560_000 // 448)
    assert ws >= 16 * tiles        # one 16-byte scan status per tile
    assert daq.strerror(daq.DAQ_ECAPACITY).startswith("island records")
    assert daq.lib().daq_version() >= 100
    assert daq.daq_status_from_counts([5, 5, 0, 1]) == daq.DAQ_OK
    assert daq.daq_status_from_counts([5, 5, daq.DAQ_DEV_POOL_OVERFLOW, 1]) == daq.DAQ_ECAPACITY
    assert daq.daq_status_from_counts([5, 5, daq.DAQ_DEV_TIMEOUT, 1]) == daq.DAQ_ETIMEOUT


@pytest.mark.parametrize("pre,post,grid,tile,expect", [
    (8, 24, 0, 0, 448),      # nominal windows: 448-sample tiles, two count CTAs per SM
    (8, 64, 0, 0, 448),      # the count pass loads no halo, so wide windows keep 448
    (250, 250, 0, 0, 448),   # windows wider than a 128-sample tile
    (8, 64, 0, 448, 448),    # an explicit tile is kept while its plan fits
    (8, 64, 0, 384, 384),
    (8, 64, -4, 0, 448),     # other forms: 448 unless it does not fit
    (8, 64, -4, 384, 224),   # 384 is a two-pass width only
    (8, 24, 0, 384, 384),
])
def test_tile_choice(daq, pre, post, grid, tile, expect):
    """The plan's tile width, read back through the tile count of a full fill."""
    p = daq.make_params(threshold=15, pre=pre, post=post, decim=(8, 32), grid=grid, tile=tile)
    assert daq.daq_trace_tiles(24, 54, 560_000, 1, p) == 24 * -(-560_000 // expect)


@pytest.mark.parametrize("bad", [
    dict(pre=-1), dict(post=-2), dict(ped_samples=0), dict(decim=(0,)), dict(pre=300, post=300),
    dict(tile=100), dict(grid=-7), dict(lag_tiles=-1), dict(calo_base=-1), dict(q_calos=-1), dict(calo_base=1, q_calos=1),
])
def test_bad_parameters_rejected_before_any_device_work(daq, bad):
    kw = dict(threshold=30, pre=8, post=24, ped_samples=100, decim=(32,))
    kw.update(bad)
    p = daq.make_params(**kw)
    with pytest.raises(daq.DaqError) as e:
        daq.daq_workspace_size(1, 54, 1000, 1, p)
    assert e.value.status == daq.DAQ_EINVAL


def _has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="passes fake device addresses; host-only check")
def test_bad_shapes_rejected(daq):
    p = daq.make_params()
    isl = daq.DaqIslands(0, 0, 0, 0, 0, 0)
    assert daq.daq_process_fills(0, 1, 54, 1000, 1, p, isl, None) == daq.DAQ_EINVAL   # counts NULL
    assert daq.daq_process_fills(0, 1, 65, 1000, 1, p, isl, None) == daq.DAQ_EUNSUPPORTED
    assert daq.daq_process_fills(0, 1, 0, 1000, 1, p, isl, None) == daq.DAQ_EINVAL
    assert daq.daq_process_fills(0, -1, 54, 1000, 1, p, isl, None) == daq.DAQ_EINVAL
    isl = daq.DaqIslands(0, 0, 0, 0, 0, 64)
    assert daq.daq_process_fills(0, 1, 54, 1000, 1, p, isl, None) == daq.DAQ_EINVAL   # samples NULL
    # misaligned pool / short workspace
    isl = daq.DaqIslands(4096, 10, 4098, 10, 0, 64)
    assert daq.daq_process_fills(4096, 1, 54, 1000, 1, p, isl, 8192) == daq.DAQ_EINVAL
    isl = daq.DaqIslands(4096, 10, 4096, 10, 0, 64)
    p.workspace, p.workspace_bytes = 4096, 16
    assert daq.daq_process_fills(4096, 1, 54, 1000, 1, p, isl, 8192) == daq.DAQ_EINVAL


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    import paper_1611_04959_gb300 as d
    monkeypatch.setattr(d, "_lib", None)
    monkeypatch.setattr(d, "LIB_PATH", str(tmp_path / "libdaq.so"))
    with pytest.raises(RuntimeError, match="not built"):
        d.lib()
