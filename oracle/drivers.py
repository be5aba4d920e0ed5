"""Alg. 1 (single-path) and Alg. 2 (multi-path) on the FP64 MPS (oracle side; test
infrastructure only).

Single path (Alg. 1, Sec. "Single-path simulation"): start from |0...0>, c = 0, p = 1,
F = 1; compress each non-empty chunk (F *= f); at a measurement compute (p_0, p_1) at the
orthogonality centre, draw u = Philox(seed, shot, ordinal), take m = 0 iff u < p_0, collapse,
p *= p_m, c_j := m.

Multi path (Alg. 2, Sec. "Multi-path simulation"): every branch compresses its chunk; at a
measurement every branch spawns the children m in {0, 1} with p_m > P_EPS (m = 0 first,
parents in list order) with p_{gamma m} = p_gamma p_m, F copied; then, if more than M
branches are active, the M with the largest p are kept (ties: ``topk_select``), and with
adaptive pruning (p_min > 0) branches below p_min are dropped (``prune_select``).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from circuits import Circuit, Measure
from .layers import (blocks_mpo, chunk_blocks, chunk_circuit, chunk_sublayer_blocks,
                     compose_mpo)
from .mps import MPS, collapse, compress, measure_probs, product_zero
from .philox import uniform
from .statevector import FLAG_WINDOW, P_EPS, prune_select


@dataclass
class Params:
    chi_max: int = 8
    tol: float = 1e-10
    sweeps: int = 2
    k: int = 0  # maximum ops per chunk (0: no limit)
    layers: int = 1  # sub-layers per chunk (1: the one-layer rule)


@dataclass
class ShotResult:
    p: float
    F: float
    c: np.ndarray
    mps: MPS
    outcomes: List[int]
    p0s: List[float]
    flagged: List[int]
    fids: List[float]


def _chunk_operator(n, chunk, c, layers):
    """The chunk's blocks and MPO for register c: one layer of disjoint blocks, or with
    several sub-layers the list of their blocks and the composed MPO."""
    if layers <= 1:
        blocks, empty = chunk_blocks(n, chunk, c)
        return blocks, blocks_mpo(n, blocks), empty
    sub, empty = chunk_sublayer_blocks(n, chunk, c)
    if len(sub) == 1:
        return sub[0], blocks_mpo(n, sub[0]), empty
    return sub, compose_mpo([blocks_mpo(n, b) for b in sub]), empty


class SinglePathRun:
    """One run of Alg. 1 carried across calls: ``run(ops)`` continues it with the next ops.
    Calls that each end where a chunk closes (at a measurement, or at the end of the circuit)
    make the same chunks, draws and compressions as one pass over the concatenated ops."""

    def __init__(self, n: int, n_cbits: int, prm: Params, seed: int, shot: int):
        self.n, self.n_cbits, self.prm, self.seed, self.shot = n, n_cbits, prm, seed, shot
        self.mps = product_zero(n)
        self.c = np.zeros(n_cbits, dtype=np.int64)
        self.p, self.F = 1.0, 1.0
        self.outcomes, self.p0s, self.flagged, self.fids = [], [], [], []
        self.ordinal = 0
        self.sweeps_run = 0

    def run(self, ops, stop_after_flag: bool = False) -> None:
        n, steps = chunk_circuit(Circuit(self.n, self.n_cbits, list(ops)), self.prm.k,
                                 self.prm.layers)
        for st in steps:
            if isinstance(st, Measure):
                r0, r1 = measure_probs(self.mps, st.qubit)
                p0 = r0 / (r0 + r1)
                u = uniform(self.seed, self.shot, self.ordinal)
                m = 0 if u < p0 else 1
                if abs(u - p0) < FLAG_WINDOW:
                    self.flagged.append(self.ordinal)
                pm = p0 if m == 0 else 1.0 - p0
                if pm <= P_EPS:
                    raise FloatingPointError("collapse onto an outcome of zero probability")
                collapse(self.mps, st.qubit, m, r0 if m == 0 else r1)
                self.p *= pm
                self.c[st.cbit] = m
                self.outcomes.append(m)
                self.p0s.append(p0)
                self.ordinal += 1
                if self.flagged and stop_after_flag:
                    return
            else:
                blocks, W, empty = _chunk_operator(n, st, self.c, self.prm.layers)
                if empty:
                    continue
                self.mps, info = compress(self.mps, blocks, W, self.prm.chi_max, self.prm.tol,
                                          self.prm.sweeps)
                self.F *= info.f
                self.fids.append(info.f)
                self.sweeps_run += len(info.fidelities_per_sweep)

    def result(self) -> ShotResult:
        return ShotResult(self.p, self.F, self.c, self.mps, self.outcomes, self.p0s,
                          self.flagged, self.fids)


def run_single_path(circ: Circuit, prm: Params, seed: int, shot: int,
                    stop_after_flag: bool = False) -> ShotResult:
    r = SinglePathRun(circ.n_qubits, circ.n_cbits, prm, seed, shot)
    r.run(circ.ops, stop_after_flag)
    return r.result()


@dataclass
class MPBranch:
    p: float
    F: float
    c: np.ndarray
    mps: MPS
    path: List[int] = field(default_factory=list)


def run_multi_path(circ: Circuit, prm: Params, M: Optional[int] = None,
                   max_steps: Optional[int] = None, p_min: float = 0.0) -> List[MPBranch]:
    n, steps = chunk_circuit(circ, prm.k, prm.layers)
    Lst = [MPBranch(1.0, 1.0, np.zeros(circ.n_cbits, dtype=np.int64), product_zero(n))]
    for si, st in enumerate(steps):
        if max_steps is not None and si >= max_steps:
            break
        if isinstance(st, Measure):
            nxt = []
            for b in Lst:
                r0, r1 = measure_probs(b.mps, st.qubit)
                tot = r0 + r1
                for m, rm in ((0, r0), (1, r1)):
                    pm = rm / tot
                    if pm > P_EPS:
                        child = b.mps.copy()
                        collapse(child, st.qubit, m, rm)
                        c = b.c.copy()
                        c[st.cbit] = m
                        nxt.append(MPBranch(b.p * pm, b.F, c, child, b.path + [m]))
            Lst = nxt
            if (M is not None and len(Lst) > M) or p_min > 0.0:
                keep = prune_select([b.p for b in Lst], M, p_min)
                Lst = [Lst[i] for i in keep]
        else:
            for b in Lst:
                blocks, W, empty = _chunk_operator(n, st, b.c, prm.layers)
                if empty:
                    continue
                b.mps, info = compress(b.mps, blocks, W, prm.chi_max, prm.tol, prm.sweeps)
                b.F *= info.f
    return Lst


def multipath_fidelity(branches: List[MPBranch]) -> float:
    """Ensemble fidelity: branch fidelities weighted by branch probabilities
    (Sec. "Random dynamic circuits": normalised by the branch probabilities)."""
    ps = np.array([b.p for b in branches])
    fs = np.array([b.F for b in branches])
    return float((ps * fs).sum() / ps.sum())
