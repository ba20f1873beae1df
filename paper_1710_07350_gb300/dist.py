"""Combining per-rank bench results when every rank tracks its own bunch.

The ranks share no data-path collective (particles are independent, so the
ranks are replicas of the workload); only the timing summary is combined:
the job time is the slowest rank's, the work is the sum over ranks.
"""


def combine(total_ms, passes, device=None):
    """(max over ranks of total_ms, sum over ranks of passes)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms), float(passes)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    p = torch.tensor([float(passes)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())
