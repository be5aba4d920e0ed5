"""Multi-path ensembles sharded over ranks, one context per GPU (Alg. 2 with the branch list
split between processes).  Between measurements the ranks' branches evolve independently;
TopKByWeight needs one exchange per measurement: an all-gather of every rank's path
probabilities, after which every rank computes the same ensemble-wide selection and keeps its
own share.  The ensemble's list order is the rank-major concatenation of the ranks' lists:
children stay on their parent's rank in the paper's order (m = 0 before m = 1, parents in list
order), so that concatenation is the order one context holding every branch would have.
Marshalling and one collective only: the selection is the library's dcs_topk_select_global,
the compaction its dcs_branch_keep, everything else the library's own multi-path calls."""
from __future__ import annotations

from typing import List, Optional, Tuple

import numpy as np
import torch

from .sim import topk_select_global


def select_across_ranks(p_local, M: int, p_min: float = 0.0, group=None,
                        device="cpu") -> Tuple[np.ndarray, int]:
    """The keep mask of this rank's branches (its list order) under the top-M and pruning
    rules applied to the whole ensemble, and the number of branches kept on all ranks.
    p_local holds this rank's path probabilities in list order; `device` is where the
    collective's buffers live (CPU for gloo, this rank's GPU for NCCL)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    p = torch.as_tensor(np.ascontiguousarray(p_local, dtype=np.float64), device=device)
    n = torch.tensor([p.numel()], dtype=torch.int64, device=device)
    counts_t = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts_t, n, group=group)
    counts = [int(c.item()) for c in counts_t]
    buf = torch.zeros(max(max(counts), 1), dtype=torch.float64, device=device)
    buf[: p.numel()] = p
    got = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(got, buf, group=group)
    p_all = np.concatenate([g[:c].cpu().numpy() for g, c in zip(got, counts)])
    keep = topk_select_global(p_all, M, p_min)
    off = sum(counts[:rank])
    return keep[off: off + counts[rank]], int(keep.sum())


def topk_across_ranks(sim, M: int, p_min: float = 0.0, group=None,
                      device: Optional[str] = None) -> Tuple[int, int]:
    """TopKByWeight over a sharded ensemble: this rank's Simulator keeps its share of the M
    branches with the largest p over all ranks (then the p_min rule).  Every rank calls it
    after the same measurement.  Returns (branches kept here, branches kept on all ranks)."""
    res = sim.results()
    p = res["p"][: res["n_active"]]
    keep, total = select_across_ranks(p, M, p_min, group, device or "cpu")
    sim.branch_keep(keep)
    return int(keep.sum()), total


def _is_measurement(op) -> bool:
    return type(op).__name__ in ("Measure", "Reset")


def run_multi_path_sharded(sim, ops, M: int, p_min: float = 0.0, group=None,
                           device: Optional[str] = None) -> List[Tuple[int, int]]:
    """Alg. 2 on an ensemble split between ranks.  Every rank calls it with the same ops and
    its own multi-path Simulator.  The ops run in calls that end at each measurement (each a
    dcs_run_circuit without pruning: every rank splits and compresses the branches it holds).
    Until the list has at least one branch per rank every rank holds all of it (the same
    computation on each) and applies the top-M and p_min rules itself; the first time it has,
    rank r keeps the r-th of `world` contiguous shares of the list.  From then on children stay
    on their parent's rank, and after each measurement the ensemble-wide rules are applied
    through one all-gather (topk_across_ranks).  A reset's conditional X is applied in the call
    that holds the reset, before the selection (which does not depend on it).  Returns, per
    measurement after the split into shares, (branches kept here, branches kept in total)."""
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    sim.init_state(1, multipath=True)
    ops = ops.ops if hasattr(ops, "ops") else list(ops)
    shared = world > 1
    history: List[Tuple[int, int]] = []
    seg = []
    for op in ops:
        seg.append(op)
        if not _is_measurement(op):
            continue
        sim.run_circuit(seg)
        seg = []
        if not shared:
            history.append(topk_across_ranks(sim, M, p_min, group, device))
            continue
        # the whole list is on every rank: select here, then split into shares if it is long
        # enough
        res = sim.results()
        keep = topk_select_global(res["p"][: res["n_active"]], M, p_min)
        idx = np.flatnonzero(keep)
        if idx.size >= world:
            lo, hi = rank * idx.size // world, (rank + 1) * idx.size // world
            keep = np.zeros_like(keep)
            keep[idx[lo:hi]] = 1
            shared = False
        sim.branch_keep(keep)
    if seg:
        sim.run_circuit(seg)
    return history
