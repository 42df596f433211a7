"""Row sharding of one log-likelihood evaluation across ranks: the paper's
within-chain multi-GPU split (Sec. 2.3.2).  The N rows are partitioned
uniformly; rank g evaluates rows [b_g, e_g) against all N sources
(``hawkes_loglik_grad`` with a row window, where every row costs the same),
and one all-reduce of 7 doubles gives the whole sum.  Chains, by contrast,
are independent and need no collective.
"""
import numpy as np


def row_bounds(n, world):
    """Uniform contiguous row windows [b_g, e_g) for g = 0 .. world-1."""
    edges = np.linspace(0, n, world + 1).round().astype(np.int64)
    return [(int(edges[g]), int(edges[g + 1])) for g in range(world)]


def sharded_loglik_grad(evaluate, n, rank, world, group=None, device=None):
    """evaluate(row_begin, row_end) -> (loglik, grad[6]) on this rank's
    window; returns the all-reduced (loglik, grad) of all ranks.  The reduce
    runs on ``device`` (a CUDA device for NCCL, None: host tensors, gloo)."""
    import torch
    import torch.distributed as dist

    a, b = row_bounds(n, world)[rank]
    if b > a:
        ll, g = evaluate(a, b)
    else:
        ll, g = 0.0, np.zeros(6)
    t = torch.tensor([ll, *np.asarray(g, dtype=np.float64)], dtype=torch.float64, device=device)
    dist.all_reduce(t, group=group)
    t = t.cpu().numpy()
    return float(t[0]), t[1:]
