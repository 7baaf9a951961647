"""Per-tile stage timeline of the tile kernels (profiling aid).

    python -m paper_1611_04959_gb300.trace [--calos 24] [--grid 0] [--tile 448]

runs one traced call on a generated fill (after warm-up) and prints, for each
stage of the tile pipeline, the median / 90th-percentile time since the
previous stage, plus how many tiles were in each stage at once.  Stamps are
%globaltimer nanoseconds written by the kernels (daq_params.trace).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import DAQ_TRACE_WORDS, TRACE_STAGES

STAGE_PAIRS = [("slot_free", "ticket"), ("ticket", "load_issued"), ("load_issued", "load_landed"), ("load_landed", "sums_done"),
               ("sums_done", "marks_done"), ("marks_done", "lookback_start"), ("lookback_start", "prefix_known"),
               ("marks_done", "rows_staged"), ("prefix_known", "writer_start"), ("rows_staged", "writer_start"),
               ("writer_start", "copy_start"), ("copy_start", "copy_done"), ("copy_done", "rows_written"),
               ("writer_start", "rows_written"), ("ticket", "rows_written")]


def summarize(tr: np.ndarray) -> dict:
    """tr: [tiles][16] uint64 stamps of one call."""
    idx = {n: i for i, n in enumerate(TRACE_STAGES)}
    valid = tr[:, idx["ticket"]] > 0
    tr = tr[valid].astype(np.int64)
    t0 = tr[:, idx["ticket"]].min()
    out = {"tiles": int(len(tr)), "span_us": float((tr[:, idx["rows_written"]].max() - t0) / 1e3)}
    stages = {}
    for a, b in STAGE_PAIRS:
        if not (tr[:, idx[a]] > 0).any() or not (tr[:, idx[b]] > 0).any():
            continue
        both = (tr[:, idx[a]] > 0) & (tr[:, idx[b]] > 0)  # tiles a pass skips carry none of its stamps
        if not both.any():
            continue
        d = (tr[both, idx[b]] - tr[both, idx[a]]) / 1e3
        stages[f"{a}->{b}"] = {"p50_us": round(float(np.median(d)), 3), "p90_us": round(float(np.percentile(d, 90)), 3),
                               "max_us": round(float(d.max()), 3)}
    out["stages"] = stages
    lb = tr[:, idx["lookback_rounds_waits"]]
    if lb.any():
        out["lookback_rounds_p50"] = float(np.median(lb // 100000))
        out["lookback_wait_polls_p50"] = float(np.median(lb % 100000))
        out["lookback_wait_polls_p90"] = float(np.percentile(lb % 100000, 90))
    # tiles in flight (ticket .. rows_written) sampled on a time grid
    done = tr[:, idx["rows_written"]] > 0
    starts, ends = tr[done, idx["ticket"]] - t0, tr[done, idx["rows_written"]] - t0
    grid = np.linspace(0, ends.max(), 200)
    inflight = [(int(((starts <= g) & (ends > g)).sum())) for g in grid[20:180]]
    out["tiles_in_flight_p50"] = float(np.median(inflight))
    n_sm = len(np.unique(tr[:, idx["sm"]]))
    out["sms"] = n_sm
    return out


def main():
    import torch

    import synth
    import paper_1611_04959_gb300 as daq
    from synth import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--calos", type=int, default=24)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--flags", type=int, default=0, help="daq_params.flags (1 = skip Q, 2 = skip islands)")
    ap.add_argument("--lag", type=int, default=0, help="daq_params.lag_tiles (single-launch form, grid -4)")
    ap.add_argument("--out", default=None, help="save the raw trace (.npy)")
    ap.add_argument("--stress", type=int, default=0,
                    help="trace this many fills of the stress workload (10x rate, T=15, post=64, D=8 and 32) instead")
    args = ap.parse_args()
    if args.stress:
        w = W.scaled(W.STRESS, n_fills=args.stress, n_calo=args.calos)
    else:
        w = W.scaled(W.PLAIN_FULL_FILL, n_calo=args.calos)
    s = torch.from_numpy(synth.generate(w.config())).cuda()
    F, C, X, N = s.shape
    p = daq.make_params(**w.params(), tile=args.tile, grid=args.grid, lag_tiles=args.lag)
    n_tiles = daq.daq_trace_tiles(C, X, N, F, p)
    trace = torch.zeros((n_tiles, DAQ_TRACE_WORDS), dtype=torch.int64, device="cuda")
    res = daq.process_fills(s, tile=args.tile, grid=args.grid, flags=args.flags, lag_tiles=args.lag,
                            **w.params())   # warm-up
    outs, ws = res["outputs"], res["workspace"]
    for _ in range(3):
        daq.process_fills(s, tile=args.tile, grid=args.grid, outputs=outs, workspace=ws, flags=args.flags,
                          lag_tiles=args.lag, **w.params())
    p = daq.make_params(**w.params(), tile=args.tile, grid=args.grid, flags=args.flags, lag_tiles=args.lag,
                        stream=torch.cuda.current_stream())
    p.workspace, p.workspace_bytes = ws.data_ptr(), ws.numel()
    p.trace = trace.data_ptr()
    p.flags |= daq.DAQ_SYNC
    q = torch.zeros(daq.q_size(C, N, w.params()["decim"]), dtype=torch.int64, device="cuda")
    rc = daq.daq_process_fills(s.data_ptr(), C, X, N, F, p, outs.struct(), q.data_ptr())
    assert rc == daq.DAQ_OK, rc
    tr = trace.cpu().numpy().astype(np.uint64)
    if args.out:
        np.save(args.out, tr)
    summary = summarize(tr)
    summary.update(grid=args.grid, tile=args.tile, calos=args.calos, flags=args.flags)
    print(json.dumps(summary, indent=1))


if __name__ == "__main__":
    main()
