"""The per-tile trace summary (host logic, no GPU): stage times come only from
tiles that carry both stamps of a stage, so tiles a pass skips (the compact
pass under DAQ_SPARSE writes no stamp for a tile without marks) do not distort
the medians or the tiles-in-flight count."""
import numpy as np

from paper_1611_04959_gb300 import DAQ_TRACE_WORDS, TRACE_STAGES
from paper_1611_04959_gb300.trace import summarize


def _trace(n, skipped=()):
    idx = {s: i for i, s in enumerate(TRACE_STAGES)}
    tr = np.zeros((n, DAQ_TRACE_WORDS), np.uint64)
    for t in range(n):
        base = 1_000_000 + 1000 * t
        tr[t, idx["ticket"]] = base
        tr[t, idx["load_issued"]] = base + 100
        tr[t, idx["load_landed"]] = base + 2100
        tr[t, idx["sums_done"]] = base + 3100
        tr[t, idx["marks_done"]] = base + 4100
        if t not in skipped:  # the compact pass's stamps
            tr[t, idx["writer_start"]] = base + 9100
            tr[t, idx["rows_written"]] = base + 12100
        tr[t, idx["sm"]] = t % 7
    return tr


def test_skipped_tiles_leave_the_stage_times_alone():
    full = summarize(_trace(40))
    part = summarize(_trace(40, skipped=set(range(0, 40, 3))))
    for key in ("ticket->load_issued", "load_issued->load_landed", "marks_done->rows_staged"):
        if key in full["stages"]:
            assert part["stages"][key] == full["stages"][key]
    assert full["stages"]["writer_start->rows_written"]["p50_us"] == 3.0
    assert part["stages"]["writer_start->rows_written"]["p50_us"] == 3.0       # not pulled to 0 or negative
    assert part["stages"]["ticket->rows_written"]["p50_us"] == 12.1
    assert full["tiles"] == part["tiles"] == 40 and part["sms"] == 7
    assert part["tiles_in_flight_p50"] <= full["tiles_in_flight_p50"]


def test_a_stage_no_tile_reached_is_left_out():
    s = summarize(_trace(10))
    assert "lookback_start->prefix_known" not in s["stages"]   # single-pass stamps absent in a two-pass trace
