"""Multi-path ensembles sharded over ranks, one context per GPU (Alg. 2 with the branch list
split between processes).  Between measurements the ranks' branches evolve independently;
TopKByWeight needs one exchange per measurement: an all-gather of every rank's path
probabilities (with each branch's place in the ensemble's list order), after which every rank
computes the same ensemble-wide selection and keeps its own share.

Two ways to keep the list order across ranks: ``select_across_ranks`` / ``topk_across_ranks``
take it to be the rank-major concatenation of the ranks' lists (true while children stay on
their parent's rank, since a split keeps the paper's order: m = 0 before m = 1, parents in
list order); ``run_multi_path_sharded`` gives every branch an order key instead, so branches
can also move between ranks to even out their shares.  The selection is the library's
dcs_topk_select_global, the compaction its dcs_branch_keep, a move dcs_export_mps and
dcs_branch_append; everything else is the library's own multi-path calls."""
from __future__ import annotations

from typing import List, Optional, Tuple

import numpy as np
import torch

from . import _native as N
from .sim import topk_select_global


def _gather(values: np.ndarray, dtype, group, device) -> List[np.ndarray]:
    """Every rank's 1-D array (lengths may differ), in rank order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([values.size], dtype=torch.int64, device=device)
    counts_t = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts_t, n, group=group)
    counts = [int(c.item()) for c in counts_t]
    buf = torch.zeros(max(max(counts), 1), dtype=dtype, device=device)
    buf[: values.size] = torch.as_tensor(values, dtype=dtype, device=device)
    got = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(got, buf, group=group)
    return [g[:c].cpu().numpy() for g, c in zip(got, counts)]


def select_across_ranks(p_local, M: int, p_min: float = 0.0, group=None,
                        device="cpu") -> Tuple[np.ndarray, int]:
    """The keep mask of this rank's branches (its list order) under the top-M and pruning
    rules applied to the whole ensemble, and the number of branches kept on all ranks, for an
    ensemble whose list order is the rank-major concatenation of the ranks' lists.  p_local
    holds this rank's path probabilities in list order; `device` is where the collective's
    buffers live (CPU for gloo, this rank's GPU for NCCL)."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    parts = _gather(np.ascontiguousarray(p_local, dtype=np.float64), torch.float64, group, device)
    keep = topk_select_global(np.concatenate(parts), M, p_min)
    off = sum(len(x) for x in parts[:rank])
    return keep[off: off + len(parts[rank])], int(keep.sum())


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


def _child_keys(bits: np.ndarray, p_child: np.ndarray, cbit: int, parent_keys: np.ndarray,
                p_parent: np.ndarray, eps: float = 1e-12) -> np.ndarray:
    """Order keys of the children a split left in the list (child key = 2 parent key + m,
    which keeps the ensemble's list order).  A parent's children are consecutive, m = 0 before
    m = 1, and a parent has two children exactly when both outcomes have p_m > eps (the
    split's rule), i.e. when its m = 0 child carries less than p_parent (1 - eps); its m = 1
    child then follows, the two summing to p_parent.  So a parent whose only child is m = 0
    followed by one whose only child is m = 1 (deterministic re-measurements, as in resets)
    is told apart from one parent with both."""
    n = len(bits)
    keys = np.zeros(n, dtype=np.int64)
    i = j = 0
    while i < n:
        m = int(bits[i][cbit])
        keys[i] = 2 * parent_keys[j] + m
        two = (m == 0 and i + 1 < n and int(bits[i + 1][cbit]) == 1
               and p_child[i] < p_parent[j] * (1.0 - eps)
               and abs(p_child[i] + p_child[i + 1] - p_parent[j]) <= 1e-10 * p_parent[j])
        if two:
            keys[i + 1] = 2 * parent_keys[j] + 1
            i += 2
        else:
            i += 1
        j += 1
    assert j == len(parent_keys), "children do not match their parents"
    return keys


def _balance_moves(counts: List[int]) -> List[Tuple[int, int, int]]:
    """(source rank, destination rank, branches) moves that even out the ranks' counts,
    the same on every rank."""
    world, K = len(counts), sum(counts)
    target = [K // world + (r < K % world) for r in range(world)]
    surplus = [[r, counts[r] - target[r]] for r in range(world) if counts[r] > target[r]]
    deficit = [[r, target[r] - counts[r]] for r in range(world) if counts[r] < target[r]]
    moves, i, j = [], 0, 0
    while i < len(surplus) and j < len(deficit):
        m = min(surplus[i][1], deficit[j][1])
        moves.append((surplus[i][0], deficit[j][0], m))
        surplus[i][1] -= m
        deficit[j][1] -= m
        i += surplus[i][1] == 0
        j += deficit[j][1] == 0
    return moves


# one moved branch: p, F (float64); order key, flags, MPS byte count (int64); the register
# (N.CWORDS uint64 words); then the MPS in the dcs_export_mps format
_CWORDS = N.CWORDS
_HEAD = 2 * 8 + 3 * 8 + _CWORDS * 8


def _send_branch(sim, pos: int, res: dict, key: int, dst: int, group, device):
    import torch.distributed as dist
    raw = sim.export_mps_bytes(pos)
    cw = np.zeros(_CWORDS, dtype=np.uint64)
    src = np.asarray(res["cwords"][pos], dtype=np.uint64).ravel()
    cw[: src.size] = src
    head = (np.array([res["p"][pos], res["F"][pos]], dtype=np.float64).tobytes()
            + np.array([key, int(res["flags"][pos]), len(raw)], dtype=np.int64).tobytes()
            + cw.tobytes())
    msg = np.frombuffer(head + raw, dtype=np.uint8)
    dist.send(torch.tensor([msg.size], dtype=torch.int64, device=device), dst, group=group)
    dist.send(torch.as_tensor(msg.copy(), device=device), dst, group=group)


def _recv_branch(sim, src: int, group, device) -> int:
    import torch.distributed as dist
    n = torch.zeros(1, dtype=torch.int64, device=device)
    dist.recv(n, src, group=group)
    msg = torch.zeros(int(n.item()), dtype=torch.uint8, device=device)
    dist.recv(msg, src, group=group)
    b = msg.cpu().numpy().tobytes()
    p, F = np.frombuffer(b, dtype=np.float64, count=2)
    key, flags, nraw = np.frombuffer(b, dtype=np.int64, count=3, offset=16)
    cw = np.frombuffer(b, dtype=np.uint64, count=_CWORDS, offset=40)
    raw = b[_HEAD: _HEAD + int(nraw)]
    sim.branch_append(raw, float(p), float(F), cw, int(flags))
    return int(key)


def run_multi_path_sharded(sim, ops, M: int, p_min: float = 0.0, group=None,
                           device: Optional[str] = None,
                           balance: bool = True) -> Tuple[np.ndarray, List[Tuple[int, int]]]:
    """Alg. 2 on an ensemble split between ranks.  Every rank calls it with the same ops and
    its own multi-path Simulator.  The ops run in calls that end at each measurement (each a
    dcs_run_circuit without pruning: every rank splits and compresses the branches it holds).
    Until the list has at least one branch per rank every rank holds all of it (the same
    computation on each) and applies the top-M and p_min rules itself; the first time it has,
    rank r keeps the r-th of `world` contiguous shares of the list.  Each branch carries an
    order key, its place in the ensemble's list order (children: 2 key + m); after each
    measurement one all-gather of every rank's (p, key) gives every rank the whole list in
    that order, the same selection (dcs_topk_select_global) and the keys renumbered densely.
    With `balance`, branches then move (export, point-to-point send, dcs_branch_append) from
    ranks above an even share to ranks below it.  A reset's conditional X is applied in the
    call that holds the reset, before the selection (which does not depend on it).  Returns
    the order keys of this rank's final list (the ensemble's order is ascending key) and, per
    measurement after the split into shares, (branches held here, branches in total)."""
    import torch.distributed as dist
    device = device or "cpu"
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    sim.init_state(1, multipath=True)
    ops = ops.ops if hasattr(ops, "ops") else list(ops)
    shared = world > 1
    keys = np.zeros(1, dtype=np.int64)
    history: List[Tuple[int, int]] = []
    seg = []
    for op in ops:
        seg.append(op)
        if not _is_measurement(op):
            continue
        p_parent = None if shared else sim.results()["p"]
        sim.run_circuit(seg)
        seg = []
        res = sim.results()
        n = res["n_active"]
        if shared:
            # the whole list is on every rank: select here, then split into shares if it is
            # long enough
            keep = topk_select_global(res["p"][:n], M, p_min)
            idx = np.flatnonzero(keep)
            keys = np.arange(idx.size, dtype=np.int64)
            if idx.size >= world:
                lo, hi = rank * idx.size // world, (rank + 1) * idx.size // world
                keep = np.zeros_like(keep)
                keep[idx[lo:hi]] = 1
                keys = keys[lo:hi]
                shared = False
            sim.branch_keep(keep)
            continue
        ckeys = _child_keys(res["bits"][:n], res["p"][:n], op.cbit, keys, p_parent)
        all_p = _gather(res["p"][:n], torch.float64, group, device)
        all_k = _gather(ckeys, torch.int64, group, device)
        owner = np.concatenate([np.full(len(k), r) for r, k in enumerate(all_k)])
        p_cat, k_cat = np.concatenate(all_p), np.concatenate(all_k)
        order = np.argsort(k_cat, kind="stable")
        keep_sorted = topk_select_global(p_cat[order], M, p_min)
        dense = np.cumsum(keep_sorted) - 1
        keep_cat = np.zeros(k_cat.size, dtype=np.uint8)
        new_cat = np.zeros(k_cat.size, dtype=np.int64)
        keep_cat[order] = keep_sorted
        new_cat[order] = dense
        off = sum(len(k) for k in all_k[:rank])
        keep = keep_cat[off: off + n]
        keys = new_cat[off: off + n][keep.astype(bool)]
        sim.branch_keep(keep)
        counts = [int(keep_cat[owner == r].sum()) for r in range(world)]
        if balance:
            moves = _balance_moves(counts)
            if moves:
                res = sim.results()
                nloc = res["n_active"]
                sent = 0
                recv_keys = []
                for src, dst, m in moves:
                    if rank == src:
                        for t in range(m):
                            pos = nloc - sent - m + t
                            _send_branch(sim, pos, res, int(keys[pos]), dst, group, device)
                        sent += m
                    elif rank == dst:
                        recv_keys += [_recv_branch(sim, src, group, device) for _ in range(m)]
                if sent:
                    sim.branch_keep([1] * (nloc - sent) + [0] * sent)
                    keys = keys[: nloc - sent]
                if recv_keys:
                    keys = np.concatenate([keys, np.array(recv_keys, dtype=np.int64)])
                for src, dst, m in moves:
                    counts[src] -= m
                    counts[dst] += m
        history.append((counts[rank], sum(counts)))
    if seg:
        sim.run_circuit(seg)
    return keys, history
