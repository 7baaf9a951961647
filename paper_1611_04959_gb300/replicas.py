"""Multi-GPU form: independent replicas, one process per GPU.

Every calorimeter-fill is processed independently (the experiment gives each
calorimeter its own GPU, Sec. 3), so ranks share no data: each takes its own
share of the fills and keeps its own Q rows.  The only cross-rank step is the
timing: a barrier before and after the timed region and the maximum of the
ranks' elapsed times, from which the whole-job throughput is the units all
ranks processed over that maximum (weak scaling: fixed work per rank).
"""
from __future__ import annotations


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous block of units [lo, hi) of `rank` among `world` ranks; the
    blocks cover 0 .. n_units - 1 once, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_units, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def aggregate(bytes_local: float, ms_local: float, device=None) -> tuple:
    """Whole-job (bytes, max elapsed ms, GB/s) over the process group, or the
    local values when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return bytes_local, ms_local, bytes_local / (ms_local * 1e-3) / 1e9
    t = torch.tensor([float(bytes_local), float(ms_local)], dtype=torch.float64, device=device)
    b = t[:1].clone()
    m = t[1:].clone()
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    tot, mx = float(b.item()), float(m.item())
    return tot, mx, tot / (mx * 1e-3) / 1e9


def barrier(device=None) -> None:
    """Barrier over the process group (no-op without one)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        import torch
        t = torch.zeros(1, device=device)
        dist.all_reduce(t)
