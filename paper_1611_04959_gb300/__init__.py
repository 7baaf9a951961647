"""GB300 (sm_103a) muon g-2 waveform DAQ hot path: Python binding of libdaq.

The binding marshals arguments into the C ABI of include/daq.h (ctypes) and
uses PyTorch only for device memory and streams.  Every step of the path runs
in the CUDA kernels of libdaq.so; there is no CPU fallback, and importing the
binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

# status codes and flags (include/daq.h)
DAQ_OK, DAQ_EINVAL, DAQ_ECAPACITY, DAQ_ECUDA, DAQ_ETIMEOUT, DAQ_EUNSUPPORTED, DAQ_ESCRATCH, DAQ_EINDEX = \
    0, -1, -2, -3, -4, -5, -6, -7
DAQ_STATIC_SCRATCH_BYTES = 8 << 20
DAQ_SKIP_Q, DAQ_SKIP_ISLANDS, DAQ_SYNC, DAQ_PACK_POOL, DAQ_DEBUG_CHECKS, DAQ_SPARSE = 1, 2, 4, 8, 16, 32
DAQ_DEV_HDR_OVERFLOW, DAQ_DEV_POOL_OVERFLOW, DAQ_DEV_TIMEOUT, DAQ_DEV_BAD_FILL_LEN, DAQ_DEV_BAD_INDEX = 1, 2, 4, 8, 16

ISLAND_DTYPE = np.dtype([("fill", "<i4"), ("calo", "<i4"), ("start", "<i4"), ("len", "<i4"),
                         ("pool_row", "<i8")])


class DaqParams(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_int32), ("pre", ctypes.c_int32), ("post", ctypes.c_int32),
                ("ped_samples", ctypes.c_int32), ("n_decim", ctypes.c_int32), ("decim", ctypes.c_int32 * 2),
                ("fill_base", ctypes.c_int32), ("fill_len", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("tile", ctypes.c_int32), ("grid", ctypes.c_int32), ("calo_base", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("events", ctypes.c_void_p), ("trace", ctypes.c_void_p),
                ("q_calos", ctypes.c_int32), ("lag_tiles", ctypes.c_int32), ("wait_limit_ns", ctypes.c_uint64)]


class DaqIslands(ctypes.Structure):
    _fields_ = [("hdr", ctypes.c_void_p), ("hdr_cap", ctypes.c_int64), ("pool", ctypes.c_void_p),
                ("pool_row_cap", ctypes.c_int64), ("pedestal", ctypes.c_void_p), ("counts", ctypes.c_void_p)]


class DaqHostIO(ctypes.Structure):
    _fields_ = [("samples_host", ctypes.c_void_p), ("samples_dev", ctypes.c_void_p), ("hdr_host", ctypes.c_void_p),
                ("hdr_host_cap", ctypes.c_int64), ("pool_host", ctypes.c_void_p), ("pool_host_cap", ctypes.c_int64),
                ("pedestal_host", ctypes.c_void_p), ("counts_host", ctypes.c_void_p),
                ("packed_dev", ctypes.c_void_p), ("packed_dev_cap", ctypes.c_int64), ("packed_host", ctypes.c_void_p),
                ("packed_host_cap", ctypes.c_int64), ("packed_bytes_host", ctypes.c_void_p)]


class DaqTuneResult(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("grid", ctypes.c_int32), ("n_tried", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("ms", ctypes.c_float), ("ms_default", ctypes.c_float),
                ("flags", ctypes.c_uint32)]


DAQ_TUNE, DAQ_TUNE_FORCE = 1, 2
DAQ_SERVER_HOST_INPUT, DAQ_SERVER_AUTO_RELEASE = 1, 2
DAQ_FILL_QUEUED, DAQ_FILL_RUNNING, DAQ_FILL_DONE, DAQ_FILL_RELEASED = 0, 1, 2, 3


class DaqServerConfig(ctypes.Structure):
    _fields_ = [("n_calo", ctypes.c_int32), ("n_xtal", ctypes.c_int32), ("n_samples", ctypes.c_int64),
                ("params", DaqParams), ("mem_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("hdr_cap", ctypes.c_int64), ("pool_row_cap", ctypes.c_int64),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32), ("qhist", ctypes.c_void_p)]


class DaqFillRecord(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("n_islands", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("raw_bytes", ctypes.c_int64), ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("status", ctypes.c_int32),
                ("slot", ctypes.c_int32)]


class DaqFillResult(ctypes.Structure):
    _fields_ = [("rec", DaqFillRecord), ("state", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hdr", ctypes.c_void_p), ("pool", ctypes.c_void_p), ("pedestal", ctypes.c_void_p)]


class DaqServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("released", ctypes.c_int64), ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("running", ctypes.c_int64), ("max_running", ctypes.c_int64), ("n_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("slot_bytes", ctypes.c_size_t), ("mem_bytes", ctypes.c_size_t)]


class DaqServingSummary(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("latency_p50_us", ctypes.c_double), ("latency_p99_us", ctypes.c_double),
                ("latency_max_us", ctypes.c_double), ("deadtime", ctypes.c_double), ("gbs", ctypes.c_double),
                ("span_us", ctypes.c_double)]


class DaqError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = f"{what}: {strerror(status)} ({status})" if what else f"{strerror(status)} ({status})"
        if status == DAQ_ECUDA:
            msg += " [" + lib().daq_last_cuda_error().decode() + "]"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libdaq.so.  Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdaq.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            L.daq_params_default.argtypes = [ctypes.POINTER(DaqParams)]
            L.daq_params_default.restype = None
            L.daq_workspace_size.argtypes = [i32, i32, i64, i32, ctypes.POINTER(DaqParams),
                                             ctypes.POINTER(ctypes.c_size_t)]
            L.daq_workspace_size.restype = i32
            L.daq_q_bins.argtypes = [i64, ctypes.c_int32]
            L.daq_q_bins.restype = i64
            L.daq_process_fills.argtypes = [vp, i32, i32, i64, i32, ctypes.POINTER(DaqParams),
                                            ctypes.POINTER(DaqIslands), vp]
            L.daq_process_fills.restype = i32
            L.daq_process_fills_static.argtypes = [vp, i32, i32, i64, i32, ctypes.POINTER(DaqParams),
                                                   ctypes.POINTER(DaqIslands), vp]
            L.daq_process_fills_static.restype = i32
            L.daq_process_fills_host.argtypes = [i32, i32, i64, i32, ctypes.POINTER(DaqParams),
                                                 ctypes.POINTER(DaqIslands), vp, ctypes.POINTER(DaqHostIO)]
            L.daq_process_fills_host.restype = i32
            L.daq_trace_tiles.argtypes = [i32, i32, i64, i32, ctypes.POINTER(DaqParams)]
            L.daq_trace_tiles.restype = i64
            L.daq_status_from_counts.argtypes = [vp]
            L.daq_status_from_counts.restype = i32
            L.daq_strerror.argtypes = [i32]
            L.daq_strerror.restype = ctypes.c_char_p
            L.daq_last_cuda_error.argtypes = []
            L.daq_last_cuda_error.restype = ctypes.c_char_p
            L.daq_version.argtypes = []
            L.daq_version.restype = i32
            L.daq_batch_plan_create.argtypes = [vp, i32, i32, i64, i32, ctypes.POINTER(DaqParams),
                                                ctypes.POINTER(DaqIslands), vp, ctypes.c_uint32,
                                                ctypes.POINTER(vp)]
            L.daq_batch_plan_create.restype = i32
            L.daq_batch_launch.argtypes = [vp, vp]
            L.daq_batch_launch.restype = i32
            L.daq_batch_plan_tuning.argtypes = [vp, ctypes.POINTER(DaqTuneResult)]
            L.daq_batch_plan_tuning.restype = i32
            L.daq_batch_plan_destroy.argtypes = [vp]
            L.daq_batch_plan_destroy.restype = i32
            L.daq_tune_cache_clear.argtypes = []
            L.daq_tune_cache_clear.restype = None
            L.daq_crystal_sum_workspace_size.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
            L.daq_crystal_sum_workspace_size.restype = i32
            L.daq_crystal_sum.argtypes = [vp, i32, i32, i64, i32, ctypes.POINTER(DaqParams), vp]
            L.daq_crystal_sum.restype = i32
            L.daq_pack_bound.argtypes = [i64, i32]
            L.daq_pack_bound.restype = i64
            L.daq_pack_workspace_size.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_size_t)]
            L.daq_pack_workspace_size.restype = i32
            L.daq_pack_pool.argtypes = [vp, i64, i32, vp, i64, vp, vp, ctypes.c_size_t, vp]
            L.daq_pack_pool.restype = i32
            L.daq_unpack_pool.argtypes = [vp, i64, i64, i32, vp, vp, vp]
            L.daq_unpack_pool.restype = i32
            L.daq_server_create.argtypes = [ctypes.POINTER(DaqServerConfig), ctypes.POINTER(vp)]
            L.daq_server_create.restype = i32
            L.daq_server_submit.argtypes = [vp, vp, i32, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(i64)]
            L.daq_server_submit.restype = i32
            L.daq_server_poll.argtypes = [vp, i64, ctypes.POINTER(DaqFillResult)]
            L.daq_server_poll.restype = i32
            L.daq_server_wait.argtypes = [vp, i64, ctypes.c_double, ctypes.POINTER(DaqFillResult)]
            L.daq_server_wait.restype = i32
            L.daq_server_fetch.argtypes = [vp, i64, vp, i64, vp, i64, vp]
            L.daq_server_fetch.restype = i32
            L.daq_server_release.argtypes = [vp, i64]
            L.daq_server_release.restype = i32
            L.daq_server_drain.argtypes = [vp, ctypes.c_double]
            L.daq_server_drain.restype = i32
            L.daq_server_get_stats.argtypes = [vp, ctypes.POINTER(DaqServerStats)]
            L.daq_server_get_stats.restype = i32
            L.daq_server_records.argtypes = [vp, ctypes.POINTER(DaqFillRecord), i64, ctypes.POINTER(i64), i32]
            L.daq_server_records.restype = i32
            L.daq_server_qhist.argtypes = [vp]
            L.daq_server_qhist.restype = vp
            L.daq_server_now_us.argtypes = [vp]
            L.daq_server_now_us.restype = ctypes.c_double
            L.daq_server_destroy.argtypes = [vp]
            L.daq_server_destroy.restype = i32
            L.daq_serving_summarize.argtypes = [ctypes.POINTER(DaqFillRecord), i64, ctypes.POINTER(DaqServingSummary)]
            L.daq_serving_summarize.restype = i32
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().daq_strerror(int(status)).decode()


# ------------------------------------------------------------------- same names as the C ABI
def daq_params_default() -> DaqParams:
    p = DaqParams()
    lib().daq_params_default(ctypes.byref(p))
    return p


def daq_workspace_size(n_calo: int, n_xtal: int, n_samples: int, n_fills: int, params: DaqParams) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().daq_workspace_size(n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params), ctypes.byref(out))
    if rc:
        raise DaqError(rc, "daq_workspace_size")
    return int(out.value)


def daq_trace_tiles(n_calo: int, n_xtal: int, n_samples: int, n_fills: int, params: DaqParams) -> int:
    return int(lib().daq_trace_tiles(n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params)))


DAQ_TRACE_WORDS = 16
TRACE_STAGES = ["ticket", "load_issued", "load_landed", "sums_done", "marks_done", "lookback_start",
                "prefix_known", "rows_staged", "writer_start", "rows_written", "sm", "tile_width",
                "copy_start", "copy_done", "lookback_rounds_waits", "slot_free"]


def daq_q_bins(n_samples: int, decim: int) -> int:
    return int(lib().daq_q_bins(n_samples, decim))


def daq_process_fills(samples_ptr: int, n_calo: int, n_xtal: int, n_samples: int, n_fills: int,
                      params: DaqParams, islands: DaqIslands, qhist_ptr: int | None) -> int:
    return int(lib().daq_process_fills(samples_ptr, n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params),
                                       ctypes.byref(islands), qhist_ptr))


def daq_process_fills_static(samples_ptr: int, n_calo: int, n_xtal: int, n_samples: int, n_fills: int,
                             params: DaqParams, islands: DaqIslands, qhist_ptr: int | None) -> int:
    """daq_process_fills with the library's built-in scratch area (allocates nothing)."""
    return int(lib().daq_process_fills_static(samples_ptr, n_calo, n_xtal, n_samples, n_fills,
                                              ctypes.byref(params), ctypes.byref(islands), qhist_ptr))


def daq_process_fills_host(n_calo: int, n_xtal: int, n_samples: int, n_fills: int, params: DaqParams,
                           islands_dev: DaqIslands, qhist_ptr: int | None, io: DaqHostIO) -> int:
    return int(lib().daq_process_fills_host(n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params),
                                            ctypes.byref(islands_dev), qhist_ptr, ctypes.byref(io)))


def daq_batch_plan_create(samples_ptr: int, n_calo: int, n_xtal: int, n_samples: int, n_fills: int,
                          params: DaqParams, islands: DaqIslands, qhist_ptr: int | None, plan_flags: int):
    """Returns (status, plan handle or None)."""
    h = ctypes.c_void_p()
    rc = lib().daq_batch_plan_create(samples_ptr, n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params),
                                     ctypes.byref(islands), qhist_ptr, int(plan_flags), ctypes.byref(h))
    return int(rc), h.value


def daq_batch_launch(plan, stream_ptr: int | None) -> int:
    return int(lib().daq_batch_launch(plan, stream_ptr))


def daq_batch_plan_tuning(plan) -> DaqTuneResult:
    r = DaqTuneResult()
    rc = lib().daq_batch_plan_tuning(plan, ctypes.byref(r))
    if rc:
        raise DaqError(rc, "daq_batch_plan_tuning")
    return r


def daq_batch_plan_destroy(plan) -> int:
    return int(lib().daq_batch_plan_destroy(plan))


def daq_tune_cache_clear() -> None:
    lib().daq_tune_cache_clear()


def daq_crystal_sum_workspace_size(n_calo: int, n_xtal: int, n_fills: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().daq_crystal_sum_workspace_size(n_calo, n_xtal, n_fills, ctypes.byref(out))
    if rc:
        raise DaqError(rc, "daq_crystal_sum_workspace_size")
    return int(out.value)


def daq_crystal_sum(samples_ptr: int, n_calo: int, n_xtal: int, n_samples: int, n_fills: int, params: DaqParams,
                    q_ptr: int | None) -> int:
    return int(lib().daq_crystal_sum(samples_ptr, n_calo, n_xtal, n_samples, n_fills, ctypes.byref(params), q_ptr))


def crystal_sum(samples, q=None, ped_samples: int = 100, fill_len=None, stream=None, sync: bool = True,
                workspace=None):
    """Per-crystal full-resolution fill sum of a CUDA int16 tensor [F][C][X][N]
    into q (int64 [C][X][N], allocated zeroed if not given).  Returns q."""
    import torch
    if not samples.is_cuda or samples.dtype != torch.int16 or samples.dim() != 4 or not samples.is_contiguous():
        raise ValueError("samples must be a contiguous CUDA int16 tensor [fills][calo][xtal][samples]")
    F, C, X, N = (int(v) for v in samples.shape)
    dev = samples.device
    if q is None:
        q = torch.zeros((C, X, N), dtype=torch.int64, device=dev)
    if fill_len is not None and not torch.is_tensor(fill_len):
        fill_len = torch.as_tensor(np.asarray(fill_len, np.int32), device=dev)
    stream = torch.cuda.current_stream(dev) if stream is None else stream
    p = make_params(ped_samples=ped_samples, fill_len=fill_len, stream=stream, flags=DAQ_SYNC if sync else 0)
    need = daq_crystal_sum_workspace_size(C, X, F)
    if workspace is None or workspace.numel() * workspace.element_size() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    p.workspace, p.workspace_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    rc = daq_crystal_sum(samples.data_ptr(), C, X, N, F, p, q.data_ptr())
    if rc != DAQ_OK:
        raise DaqError(rc, "daq_crystal_sum")
    return q


def daq_pack_bound(rows: int, n_xtal: int) -> int:
    return int(lib().daq_pack_bound(rows, n_xtal))


def daq_pack_workspace_size(rows: int, n_xtal: int) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().daq_pack_workspace_size(rows, n_xtal, ctypes.byref(out))
    if rc:
        raise DaqError(rc, "daq_pack_workspace_size")
    return int(out.value)


def daq_pack_pool(pool_ptr, rows, n_xtal, out_ptr, out_cap, out_bytes_ptr, ws_ptr, ws_bytes, stream_ptr) -> int:
    return int(lib().daq_pack_pool(pool_ptr, rows, n_xtal, out_ptr, out_cap, out_bytes_ptr, ws_ptr, ws_bytes,
                                   stream_ptr))


def daq_unpack_pool(in_ptr, in_bytes, rows, n_xtal, out_ptr, err_ptr, stream_ptr) -> int:
    return int(lib().daq_unpack_pool(in_ptr, in_bytes, rows, n_xtal, out_ptr, err_ptr, stream_ptr))


def pack_pool(pool, rows: int | None = None, stream=None, out=None, workspace=None):
    """Pack the first `rows` rows of a CUDA int16 pool [rows][X].  Returns
    (stream uint8 tensor view of its exact size, size)."""
    import torch
    rows = pool.shape[0] if rows is None else int(rows)
    X = int(pool.shape[1])
    dev = pool.device
    cap = daq_pack_bound(rows, X)
    if out is None or out.numel() < cap:
        out = torch.empty(cap, dtype=torch.uint8, device=dev)
    need = daq_pack_workspace_size(rows, X)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    nbytes = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev) if stream is None else stream
    rc = daq_pack_pool(pool.data_ptr(), rows, X, out.data_ptr(), out.numel(), nbytes.data_ptr(), workspace.data_ptr(),
                       workspace.numel(), stream.cuda_stream)
    if rc != DAQ_OK:
        raise DaqError(rc, "daq_pack_pool")
    n = int(nbytes.item())
    return out[:n], n


def unpack_pool(packed, rows: int, n_xtal: int, stream=None):
    """Decode a packed stream (CUDA uint8 tensor) into a new int16 [rows][n_xtal] tensor."""
    import torch
    dev = packed.device
    out = torch.empty((max(1, rows), n_xtal), dtype=torch.int16, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev) if stream is None else stream
    rc = daq_unpack_pool(packed.data_ptr(), packed.numel(), rows, n_xtal, out.data_ptr(), err.data_ptr(),
                         stream.cuda_stream)
    if rc != DAQ_OK:
        raise DaqError(rc, "daq_unpack_pool")
    if int(err.item()) != 0:
        raise DaqError(DAQ_EINVAL, f"daq_unpack_pool: malformed stream (code {int(err.item())})")
    return out[:rows]


def daq_status_from_counts(counts_host) -> int:
    c = np.ascontiguousarray(counts_host, dtype=np.int64)
    return int(lib().daq_status_from_counts(c.ctypes.data))


# ------------------------------------------------------------------- torch marshalling helpers
def make_params(threshold=30, pre=8, post=24, ped_samples=100, decim=(32,), fill_base=0, fill_len=None,
                flags=0, tile=0, grid=0, stream=None, workspace=None, calo_base=0, q_calos=0,
                lag_tiles=0, wait_limit_ns=0) -> DaqParams:
    p = daq_params_default()
    p.threshold, p.pre, p.post, p.ped_samples = int(threshold), int(pre), int(post), int(ped_samples)
    decim = tuple(decim)
    p.n_decim = len(decim)
    for i, d in enumerate(decim):
        p.decim[i] = int(d)
    p.fill_base = int(fill_base)
    p.fill_len = None if fill_len is None else int(fill_len.data_ptr())
    p.flags = int(flags)
    p.tile, p.grid = int(tile), int(grid)
    p.calo_base, p.q_calos, p.lag_tiles = int(calo_base), int(q_calos), int(lag_tiles)
    p.wait_limit_ns = int(wait_limit_ns)
    p.stream = None if stream is None else int(stream.cuda_stream)
    if workspace is not None:
        p.workspace = int(workspace.data_ptr())
        p.workspace_bytes = int(workspace.numel() * workspace.element_size())
    return p


def q_size(n_calo: int, n_samples: int, decim) -> int:
    return sum(n_calo * daq_q_bins(n_samples, d) for d in decim)


class Outputs:
    """Caller-owned device buffers of one call (torch tensors)."""

    def __init__(self, torch, device, n_fills, n_calo, n_xtal, hdr_cap, pool_cap, pedestal=True):
        self.hdr = torch.empty(max(1, hdr_cap) * 3, dtype=torch.int64, device=device)
        self.hdr_cap = int(hdr_cap)
        self.pool = torch.empty((max(1, pool_cap), n_xtal), dtype=torch.int16, device=device)
        self.pool_cap = int(pool_cap)
        self.pedestal = (torch.empty((n_fills, n_calo, n_xtal), dtype=torch.int32, device=device)
                         if pedestal else None)
        self.counts = torch.zeros(4, dtype=torch.int64, device=device)

    def struct(self) -> DaqIslands:
        return DaqIslands(self.hdr.data_ptr(), self.hdr_cap, self.pool.data_ptr(), self.pool_cap,
                          None if self.pedestal is None else self.pedestal.data_ptr(), self.counts.data_ptr())

    def islands_host(self, n: int) -> np.ndarray:
        n = min(int(n), self.hdr_cap)
        raw = self.hdr[: n * 3].cpu().numpy()
        return raw.view(ISLAND_DTYPE)[:n].copy()


def process_fills(samples, threshold=30, pre=8, post=24, ped_samples=100, decim=(32,), fill_len=None,
                  fill_base=0, q=None, outputs: Outputs | None = None, hdr_cap=None, pool_cap=None,
                  workspace=None, flags=0, tile=0, grid=0, stream=None, sync=True, calo_base=0, q_calos=0,
                  lag_tiles=0, wait_limit_ns=0, allow=()) -> dict:
    """Run the path on a CUDA int16 tensor samples[F][C][X][N].

    Allocates (with torch) whatever output the caller did not pass; returns a
    dict with the tensors, the host counts (when sync) and the status.  Raises
    DaqError for any status but DAQ_OK, DAQ_ECAPACITY and those in `allow`."""
    import torch
    if not samples.is_cuda or samples.dtype != torch.int16 or samples.dim() != 4 or not samples.is_contiguous():
        raise ValueError("samples must be a contiguous CUDA int16 tensor [fills][calo][xtal][samples]")
    F, C, X, N = (int(v) for v in samples.shape)
    dev = samples.device
    decim = tuple(decim)
    if fill_len is not None and not torch.is_tensor(fill_len):
        fill_len = torch.as_tensor(np.asarray(fill_len, np.int32), device=dev)
    if outputs is None:
        rows = F * C * N if fill_len is None else C * int(fill_len.clamp(0, N).sum().item())
        hdr_cap = rows // 2 + F * C + 1 if hdr_cap is None else hdr_cap
        pool_cap = rows if pool_cap is None else pool_cap
        outputs = Outputs(torch, dev, F, C, X, hdr_cap, pool_cap)
    if q is None and decim:
        q = torch.zeros(q_size(q_calos or C, N, decim), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev) if stream is None else stream
    p = make_params(threshold, pre, post, ped_samples, decim, fill_base, fill_len, flags, tile, grid, stream,
                    calo_base=calo_base, q_calos=q_calos, lag_tiles=lag_tiles, wait_limit_ns=wait_limit_ns)
    ws_bytes = daq_workspace_size(C, X, N, F, p)
    if workspace is None or workspace.numel() * workspace.element_size() < ws_bytes:
        workspace = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    p.workspace, p.workspace_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if sync:
        p.flags |= DAQ_SYNC
    rc = daq_process_fills(samples.data_ptr(), C, X, N, F, p, outputs.struct(),
                           None if q is None else q.data_ptr())
    res = dict(outputs=outputs, q=q, workspace=workspace, status=rc)
    if rc not in (DAQ_OK, DAQ_ECAPACITY) and rc not in allow:
        raise DaqError(rc, "daq_process_fills")
    if sync:
        counts = outputs.counts.cpu().numpy()
        res.update(counts=counts, n_islands=int(counts[0]), n_rows=int(counts[1]))
    return res


class BatchPlan:
    """A tuned, graph-captured batch (daq_batch_plan_create / daq_batch_launch).

    Keeps references to every tensor the graph reads or writes."""

    def __init__(self, samples, q, outputs: Outputs, threshold=30, pre=8, post=24, ped_samples=100, decim=(32,),
                 fill_len=None, fill_base=0, flags=0, tile=0, grid=0, tune=True, force=False, workspace=None):
        import torch
        if not samples.is_cuda or samples.dtype != torch.int16 or samples.dim() != 4 or not samples.is_contiguous():
            raise ValueError("samples must be a contiguous CUDA int16 tensor [fills][calo][xtal][samples]")
        F, C, X, N = (int(v) for v in samples.shape)
        self.shape = (F, C, X, N)
        self._keep = (samples, q, outputs, fill_len, workspace)
        self.outputs = outputs
        self.q = q
        p = make_params(threshold, pre, post, ped_samples, decim, fill_base, fill_len, flags, tile, grid, None,
                        workspace)
        pf = (DAQ_TUNE if tune else 0) | (DAQ_TUNE_FORCE if force else 0)
        rc, h = daq_batch_plan_create(samples.data_ptr(), C, X, N, F, p, outputs.struct(),
                                      None if q is None else q.data_ptr(), pf)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_batch_plan_create")
        self._h = h

    def launch(self, stream=None) -> None:
        rc = daq_batch_launch(self._h, None if stream is None else int(stream.cuda_stream))
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_batch_launch")

    def tuning(self) -> dict:
        r = daq_batch_plan_tuning(self._h)
        return dict(tile=r.tile, grid=r.grid, n_tried=r.n_tried, from_cache=bool(r.from_cache), ms=r.ms,
                    ms_default=r.ms_default, flags=r.flags)

    def close(self) -> None:
        if getattr(self, "_h", None):
            daq_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------- serving (same names as the C ABI)
def daq_server_create(cfg: DaqServerConfig):
    """Returns (status, server handle or None)."""
    h = ctypes.c_void_p()
    rc = lib().daq_server_create(ctypes.byref(cfg), ctypes.byref(h))
    return int(rc), h.value


def daq_server_submit(server, samples_ptr: int, on_host: bool, fill_len: int, arrival_us: float):
    t = ctypes.c_int64(0)
    rc = lib().daq_server_submit(server, samples_ptr, int(bool(on_host)), int(fill_len), float(arrival_us),
                                 ctypes.byref(t))
    return int(rc), int(t.value)


def daq_server_poll(server, ticket: int):
    r = DaqFillResult()
    rc = lib().daq_server_poll(server, int(ticket), ctypes.byref(r))
    return int(rc), r


def daq_server_wait(server, ticket: int, timeout_s: float):
    r = DaqFillResult()
    rc = lib().daq_server_wait(server, int(ticket), float(timeout_s), ctypes.byref(r))
    return int(rc), r


def daq_server_release(server, ticket: int) -> int:
    return int(lib().daq_server_release(server, int(ticket)))


def daq_server_drain(server, timeout_s: float) -> int:
    return int(lib().daq_server_drain(server, float(timeout_s)))


def daq_server_get_stats(server) -> DaqServerStats:
    st = DaqServerStats()
    rc = lib().daq_server_get_stats(server, ctypes.byref(st))
    if rc:
        raise DaqError(rc, "daq_server_get_stats")
    return st


def daq_server_records(server, clear: bool = False) -> list:
    n = ctypes.c_int64(0)
    lib().daq_server_records(server, None, 0, ctypes.byref(n), 0)
    buf = (DaqFillRecord * max(1, n.value))()
    m = ctypes.c_int64(0)
    rc = lib().daq_server_records(server, buf, n.value, ctypes.byref(m), int(bool(clear)))
    if rc:
        raise DaqError(rc, "daq_server_records")
    return [buf[i] for i in range(min(n.value, m.value))]


def daq_server_destroy(server) -> int:
    return int(lib().daq_server_destroy(server))


def daq_serving_summarize(records) -> DaqServingSummary:
    n = len(records)
    arr = (DaqFillRecord * max(1, n))(*records)
    out = DaqServingSummary()
    rc = lib().daq_serving_summarize(arr, n, ctypes.byref(out))
    if rc:
        raise DaqError(rc, "daq_serving_summarize")
    return out


def record_dict(r: DaqFillRecord) -> dict:
    return {k: getattr(r, k) for k, _ in DaqFillRecord._fields_}


class DaqServer:
    """Request loop over fills of one shape (daq_server_*), Q resident in a
    caller-visible torch tensor."""

    def __init__(self, n_calo: int, n_xtal: int, n_samples: int, budget_bytes: int, threshold=30, pre=8, post=24,
                 ped_samples=100, decim=(32,), tile=0, grid=0, max_slots=0, n_streams=0, hdr_cap=0, pool_cap=0,
                 host_input=False, auto_release=False, device=None, q=None, flags=0):
        import torch
        self.torch = torch
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        self.shape = (int(n_calo), int(n_xtal), int(n_samples))
        self.q = q if q is not None else torch.zeros(max(1, q_size(n_calo, n_samples, decim)), dtype=torch.int64,
                                                     device=dev)
        cfg = DaqServerConfig()
        cfg.n_calo, cfg.n_xtal, cfg.n_samples = self.shape
        cfg.params = make_params(threshold, pre, post, ped_samples, decim, 0, None, flags, tile, grid)
        cfg.mem_budget_bytes = int(budget_bytes)
        cfg.max_slots, cfg.n_streams = int(max_slots), int(n_streams)
        cfg.hdr_cap, cfg.pool_row_cap = int(hdr_cap), int(pool_cap)
        cfg.flags = (DAQ_SERVER_HOST_INPUT if host_input else 0) | (DAQ_SERVER_AUTO_RELEASE if auto_release else 0)
        cfg.qhist = self.q.data_ptr() if decim else None
        with torch.cuda.device(dev):
            rc, h = daq_server_create(cfg)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_create")
        self._h = h
        self._inputs = {}   # ticket -> tensor kept alive until the fill is done

    def now_us(self) -> float:
        return float(lib().daq_server_now_us(self._h))

    def submit(self, samples, fill_len: int = -1, arrival_us: float = -1.0) -> int:
        """samples: CUDA (or, with host_input, CPU) int16 tensor [C][X][N] (or [1][C][X][N])."""
        on_host = not samples.is_cuda
        rc, t = daq_server_submit(self._h, samples.data_ptr(), on_host, fill_len, arrival_us)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_submit")
        self._inputs[t] = samples
        return t

    def wait(self, ticket: int, timeout_s: float = 60.0) -> dict:
        rc, r = daq_server_wait(self._h, ticket, timeout_s)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_wait")
        self._inputs.pop(ticket, None)
        return dict(record_dict(r.rec), state=r.state)

    def poll(self, ticket: int) -> dict:
        rc, r = daq_server_poll(self._h, ticket)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_poll")
        return dict(record_dict(r.rec), state=r.state)

    def fetch(self, ticket: int):
        """(islands ISLAND_DTYPE[n], pool int16[rows][X], pedestal int32[C][X]) of a done fill."""
        r = self.poll(ticket)
        C, X, _ = self.shape
        hdr = np.empty(max(1, r["n_islands"]), ISLAND_DTYPE)
        pool = np.empty((max(1, r["n_rows"]), X), np.int16)
        ped = np.empty((C, X), np.int32)
        rc = lib().daq_server_fetch(self._h, int(ticket), hdr.ctypes.data, r["n_islands"], pool.ctypes.data,
                                    r["n_rows"], ped.ctypes.data)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_fetch")
        return hdr[: r["n_islands"]], pool[: r["n_rows"]], ped

    def release(self, ticket: int) -> None:
        rc = daq_server_release(self._h, ticket)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_release")

    def drain(self, timeout_s: float = 120.0) -> None:
        rc = daq_server_drain(self._h, timeout_s)
        if rc != DAQ_OK:
            raise DaqError(rc, "daq_server_drain")
        self._inputs.clear()

    def stats(self) -> dict:
        st = daq_server_get_stats(self._h)
        return {k: getattr(st, k) for k, _ in DaqServerStats._fields_}

    def records(self, clear: bool = False) -> list:
        return daq_server_records(self._h, clear)

    def close(self) -> None:
        if getattr(self, "_h", None):
            daq_server_destroy(self._h)
            self._h = None
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
