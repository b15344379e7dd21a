"""Host logic of the multi-process path: point shards and the one exchange.

Point i of a run depends only on (seed, i), so ranks take contiguous,
disjoint point ranges and need no communication while they compute.  The
only exchange is the combination of the per-rank Monte Carlo sums into the
job's cross section, and of the per-rank histograms into the job's
distributions (the summation step of the paper's program, Sec. 3.1, spread
over processes).  Each gathers the ranks' sums and combines them in rank
order with error-free transformations, so every rank gets the same bits
whatever the process timing.
"""
from __future__ import annotations

import numpy as np

from . import heget as H


def shard(N: int, world: int, rank: int) -> tuple[int, int]:
    """(first point, point count) of `rank` among `world` ranks: contiguous
    ranges, the first N % world ranks take one extra point."""
    if world < 1 or not 0 <= rank < world or N < 0:
        raise ValueError("bad shard request")
    q, r = divmod(N, world)
    return rank * q + min(rank, r), q + (1 if rank < r else 0)


def combine(results, sampler_kind: int) -> H.heget_xsec_result:
    """Merge per-shard results (in the given order) as if one call had
    processed all their points: heget_xsec_combine (the sums combined with
    TwoSum and rounded once, counts added, sigma and its error recomputed
    with the formulas of heget_xsec)."""
    return H.heget_xsec_combine(list(results), sampler_kind)


def allreduce_result(res: H.heget_xsec_result, sampler_kind: int, group=None) -> H.heget_xsec_result:
    """The job's result on every rank: all-gather of each rank's sums and
    counts (8 values) over `group` (any torch.distributed backend), combined
    in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([res.sum_w, res.sum_w2], dtype=torch.float64, device=device)
    cnt = torch.tensor([res.n_pass, res.n_total, res.n_tries, res.n_escalated], dtype=torch.int64, device=device)
    fs = [torch.empty_like(mine) for _ in range(world)]
    cs = [torch.empty_like(cnt) for _ in range(world)]
    dist.all_gather(fs, mine, group=group)
    dist.all_gather(cs, cnt, group=group)
    parts = []
    for f, c in zip(fs, cs):
        r = H.heget_xsec_result()
        r.sum_w, r.sum_w2 = float(f[0]), float(f[1])
        r.n_pass, r.n_total, r.n_tries, r.n_escalated = (int(x) for x in c.tolist())
        parts.append(r)
    return combine(parts, sampler_kind)


def combine_hists(parts) -> np.ndarray:
    """Histograms of disjoint point shards (heget_hist outputs: for every bin
    of every spec, sum w and sum w^2), in the given order: heget_hist_combine
    (each entry combined with TwoSum across the shards and rounded once).
    ValueError for arrays of different layouts."""
    arrs = [np.asarray(p, dtype=np.float64).ravel() for p in parts]
    if not arrs or any(a.shape != arrs[0].shape for a in arrs):
        raise ValueError("histograms of different layouts (or none)")
    return H.heget_hist_combine(arrs)


def allreduce_hist(hist, group=None) -> np.ndarray:
    """The job's histograms on every rank: all-gather of each rank's
    heget_hist output over `group`, combined in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.as_tensor(np.asarray(hist, dtype=np.float64).ravel(), device=device)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return combine_hists([p.cpu().numpy() for p in parts])
