"""Splitting one log-likelihood evaluation across ranks (Sec. 2.3.2: the
paper splits the rows of one evaluation over GPUs and gathers the per-row
results).

Two splits are provided:

* ``sharded_loglik_grad_symmetric`` keeps the sweep's symmetric shortcut.
  Rank g sweeps the row tiles [b_g, b_{g+1}) of the symmetric work list,
  with boundaries chosen by ``hawkes_shard_bounds`` so that every rank holds
  about 1/G of the N(N-1)/2 pairs (boundaries near N sqrt(g / G)).  A
  background term formed in rank g's rows is also added to the earlier row
  it pairs with, which may belong to another rank, so the ranks add their
  six moment vectors (one all-reduce of 6 N doubles) and each finalises the
  whole sum from the total.
* ``sharded_loglik_grad`` is the paper's literal split: uniform row windows,
  each row against all N sources without the symmetric shortcut, and one
  all-reduce of 7 doubles.  It does about 1.5 times the arithmetic of the
  symmetric sweep (every ordered pair's background term, no column sums).

Chains, by contrast, are independent and need no collective.
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


def symmetric_row_bounds(n, tile_rows, world):
    """Row boundaries [world + 1] of the symmetric split (whole row tiles,
    about equal pair counts); computed by the library on the host."""
    from .hawkes import hawkes_shard_bounds
    return hawkes_shard_bounds(n, tile_rows, world)


def sharded_loglik_grad_symmetric(hk, d_params, rank, world, flags=0, group=None):
    """One evaluation split over ``world`` ranks with the symmetric sweep.
    hk: this rank's ``Hawkes`` context holding all N events (the same events
    and locations on every rank); d_params: device pointer to its
    hawkes_params.  Returns (loglik, grad[6]), the same on every rank.  The
    all-reduce runs on the context's device (NCCL for a CUDA process group,
    gloo otherwise)."""
    import torch
    import torch.distributed as dist

    n = hk.n
    m = torch.empty(6 * n, dtype=torch.float64, device="cuda")
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    hk.shard_moments(d_params, rank, world, m.data_ptr(), flags)
    torch.cuda.current_stream().synchronize()
    if world > 1:
        dist.all_reduce(m, group=group)
    hk.finalize_moments(d_params, m.data_ptr(), out.data_ptr(), flags)
    o = out.cpu().numpy()
    return float(o[0]), o[1:]
