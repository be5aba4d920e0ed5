"""O1: dense FP64 state-vector simulation of dynamic circuits (n <= ~20 qubits).

Test infrastructure only (see the package header).  It follows the definitions directly:

* pure state: a normalised vector in C^(2^n), stored as an order-n tensor with one axis
  per qubit (Def. "Pure quantum state");
* unitary operation: U on k qubits embedded with identities (Def. "Unitary operation");
* mid-circuit measurement: p_m = <psi|P_m|psi>, psi_m = P_m psi / sqrt(p_m)
  (Def. "Mid-circuit measurement");
* classically controlled operation: U applied iff phi(c) holds (Def. "Classically
  controlled operation");
* the branch state {(p_gamma, c_gamma, psi_gamma)} with sum p_gamma = 1
  (Def. "State of a dynamic circuit"), evolved by the single-path strategy (Alg. 1:
  one sampled path) or the multi-path strategy (Alg. 2: every outcome with p_m != 0,
  top-M truncation after each measurement).

Gates are applied one by one (no chunking, no compression): this is the exact semantics
the MPS method approximates.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from circuits import X, Circuit, Cond, Gate, Measure, Reset
from .philox import uniform

# a measurement outcome with conditional probability <= P_EPS is treated as impossible
P_EPS = 1e-12
# a draw u with |u - p0| < FLAG_WINDOW is reported as flagged
FLAG_WINDOW = 1e-6


def lower_resets(circ: Circuit) -> Circuit:
    """Reset -> measurement into its bit, then X conditioned on that bit == 1
    (Sec. "Reset operations")."""
    ops = []
    for o in circ.ops:
        if isinstance(o, Reset):
            ops.append(Measure(o.qubit, o.cbit))
            ops.append(Gate((o.qubit,), X, cond=Cond((o.cbit,), "xor", 1), name="resetX"))
        else:
            ops.append(o)
    return Circuit(circ.n_qubits, circ.n_cbits, ops, circ.name, dict(circ.meta))


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_gate(psi: np.ndarray, qubits, mat: np.ndarray) -> np.ndarray:
    """psi' = (U on ``qubits``) psi, by contracting U's input legs with those axes."""
    k = len(qubits)
    u = np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * k))
    out = np.tensordot(u, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    # tensordot puts U's output legs first; move them back to their qubit axes
    return np.moveaxis(out, list(range(k)), list(qubits))


def probabilities(psi: np.ndarray, q: int):
    """(p_0, p_1) = (<psi|P_0|psi>, <psi|P_1|psi>) for qubit q."""
    sl0 = np.take(psi, 0, axis=q)
    sl1 = np.take(psi, 1, axis=q)
    return float(np.vdot(sl0, sl0).real), float(np.vdot(sl1, sl1).real)


def project(psi: np.ndarray, q: int, m: int, p_m: float) -> np.ndarray:
    """P_m psi / sqrt(p_m) on qubit q."""
    out = psi.copy()
    idx = [slice(None)] * psi.ndim
    idx[q] = 1 - m
    out[tuple(idx)] = 0.0
    return out / np.sqrt(p_m)


def cond_holds(cond: Optional[Cond], c: np.ndarray) -> bool:
    """phi(c) of a classically controlled operation (Sec. "Classically controlled
    operations": phi is a Boolean function of the register): XOR, AND or OR of the listed
    bits compared with ``value``, or a truth table (``op == "table"``: bit i of ``value``,
    i the listed bits read in ascending order as a binary number, smallest bit first)."""
    if cond is None:
        return True
    vals = [int(c[b]) for b in cond.bits]
    if cond.op == "xor":
        v = 0
        for x in vals:
            v ^= x
    elif cond.op == "and":
        v = int(all(vals))
    elif cond.op == "or":
        v = int(any(vals))
    elif cond.op == "table":
        idx = 0
        for k, b in enumerate(sorted(cond.bits)):
            idx += int(c[b]) << k
        return (int(cond.value) >> idx) & 1 == 1
    else:
        raise ValueError(cond.op)
    return v == int(cond.value)


@dataclass
class Branch:
    p: float
    c: np.ndarray
    psi: np.ndarray
    path: List[int] = field(default_factory=list)


@dataclass
class SinglePathResult:
    p: float
    c: np.ndarray
    psi: np.ndarray
    outcomes: List[int]
    p0s: List[float]
    flagged: List[int]


def run_single_path(circ: Circuit, seed: int, shot: int, forced=None) -> SinglePathResult:
    """Alg. 1 on the exact state vector: sample each measurement from u = Philox(seed, shot,
    ordinal), m = 0 iff u < p_0; p_gamma *= p_m; c_j := m.  ``forced`` (a list) replaces the
    sampled outcomes in order (used to follow a given path)."""
    circ = lower_resets(circ)
    n = circ.n_qubits
    psi = zero_state(n)
    c = np.zeros(circ.n_cbits, dtype=np.int64)
    p = 1.0
    outcomes, p0s, flagged = [], [], []
    ordinal = 0
    for op in circ.ops:
        if isinstance(op, Gate):
            if cond_holds(op.cond, c):
                psi = apply_gate(psi, op.qubits, op.matrix)
        elif isinstance(op, Measure):
            r0, r1 = probabilities(psi, op.qubit)
            p0 = r0 / (r0 + r1)
            u = uniform(seed, shot, ordinal)
            m = 0 if u < p0 else 1
            if forced is not None:
                m = int(forced[ordinal])
            if abs(u - p0) < FLAG_WINDOW:
                flagged.append(ordinal)
            pm = p0 if m == 0 else 1.0 - p0
            if pm <= P_EPS:
                raise FloatingPointError("outcome with zero probability")
            psi = project(psi, op.qubit, m, r0 if m == 0 else r1)
            p *= pm
            c[op.cbit] = m
            outcomes.append(m)
            p0s.append(p0)
            ordinal += 1
        else:
            raise TypeError(op)
    return SinglePathResult(p, c, psi, outcomes, p0s, flagged)


def topk_select(ps: List[float], M: int, tau: float = 1e-5) -> List[int]:
    """Indices (in list order) of the M retained branches (Alg. 2: keep the M largest p).

    Reading of ties: p values are compared through the integer key
    round(p / (tau * max p)); equal keys are ties, broken by list order (earlier wins)."""
    if len(ps) <= M:
        return list(range(len(ps)))
    pmax = max(ps)
    keys = [int(np.floor(p / (tau * pmax) + 0.5)) for p in ps]
    order = sorted(range(len(ps)), key=lambda i: (-keys[i], i))
    return sorted(order[:M])


def prune_select(ps: List[float], M: Optional[int], p_min: float = 0.0,
                 tau: float = 1e-5) -> List[int]:
    """Indices (in list order) of the branches kept after a measurement: the top-M rule of
    Alg. 2 (``topk_select``; all when M is None), then adaptive pruning (the paper names
    pruning beyond top-M as future work; reading: a branch whose path probability is below
    the absolute threshold p_min is dropped, except the first branch of the key order, so
    the list never empties)."""
    keep = list(range(len(ps))) if (M is None or len(ps) <= M) else topk_select(ps, M, tau)
    if p_min <= 0.0 or not keep:
        return keep
    pmax = max(ps)
    keys = {i: int(np.floor(ps[i] / (tau * pmax) + 0.5)) for i in keep}
    first = min(keep, key=lambda i: (-keys[i], i))
    return [i for i in keep if ps[i] >= p_min or i == first]


def run_multi_path(circ: Circuit, M: Optional[int] = None, p_min: float = 0.0) -> List[Branch]:
    """Alg. 2 on the exact state vector: every outcome with p_m > P_EPS spawns a child
    (m = 0 child before m = 1, parents in list order); after each measurement the kept
    branches are chosen by ``prune_select`` (top-M, then the probability threshold)."""
    circ = lower_resets(circ)
    L = [Branch(1.0, np.zeros(circ.n_cbits, dtype=np.int64), zero_state(circ.n_qubits))]
    for op in circ.ops:
        if isinstance(op, Gate):
            for b in L:
                if cond_holds(op.cond, b.c):
                    b.psi = apply_gate(b.psi, op.qubits, op.matrix)
        elif isinstance(op, Measure):
            nxt = []
            for b in L:
                r0, r1 = probabilities(b.psi, op.qubit)
                tot = r0 + r1
                for m, rm in ((0, r0), (1, r1)):
                    pm = rm / tot
                    if pm > P_EPS:
                        c = b.c.copy()
                        c[op.cbit] = m
                        nxt.append(Branch(b.p * pm, c, project(b.psi, op.qubit, m, rm),
                                          b.path + [m]))
            L = nxt
            if (M is not None and len(L) > M) or p_min > 0.0:
                keep = prune_select([b.p for b in L], M, p_min)
                L = [L[i] for i in keep]
        else:
            raise TypeError(op)
    return L


def tvd(p: dict, q: dict) -> float:
    """Total variation distance 1/2 sum |p - q| (Sec. "Quantum teleportation protocol")."""
    keys = set(p) | set(q)
    return 0.5 * sum(abs(p.get(k, 0.0) - q.get(k, 0.0)) for k in keys)
