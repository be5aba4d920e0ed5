"""Chunk construction and the chunk MPO (oracle side; test infrastructure only).

Chunks (Sec. "Handling unitary chunks in dynamic circuits"): operations are scanned in
order; unitary gates, conditional or not, are appended to the current chunk; a mid-circuit
measurement closes the chunk (it is compressed first if non-empty).

Reading used here (one gate layer per compression step): the chunk also closes *before* a
two-qubit gate one of whose qubits already carries a two-qubit gate of the chunk, and
before the (k+1)-th operation when a maximum size k > 0 is given.  Single-qubit gates never
close a chunk.  A conditional gate counts for these rules whether or not its condition
holds, so chunk boundaries are the same on every path; the condition itself is evaluated
on the branch's classical register when the chunk's operator is built (Alg. 1, Alg. 2:
conditions are evaluated at chunk construction, and the register cannot change inside a
chunk because measurements close it).  With these rules a chunk is one layer of disjoint
nearest-neighbour blocks, so its MPO has bond dimension <= 4.
"""
from __future__ import annotations

from typing import List, Tuple, Union

import numpy as np

from circuits import Circuit, Gate, Measure
from .statevector import cond_holds, lower_resets

Step = Union[List[Gate], Measure]


def chunk_circuit(circ: Circuit, k: int = 0, layers: int = 1) -> Tuple[int, List[Step]]:
    """Split the (reset-lowered) circuit into unitary chunks (lists of Gates) and
    measurements, in order.  Returns (n_qubits, steps).

    A chunk holds up to ``layers`` sub-layers: a two-qubit gate touching a qubit that already
    carries a two-qubit gate of the current sub-layer opens a new sub-layer, or closes the
    chunk when it has ``layers`` of them (``layers`` = 1: the one-layer rule).  Measurements
    and the k-operation limit close it as well."""
    circ = lower_resets(circ)
    n = circ.n_qubits
    steps: List[Step] = []
    cur: List[Gate] = []
    busy = set()  # qubits carrying a two-qubit gate of the current sub-layer
    nsub = 1

    def close():
        nonlocal cur, busy, nsub
        if cur:
            steps.append(cur)
        cur, busy, nsub = [], set(), 1

    for op in circ.ops:
        if isinstance(op, Measure):
            close()
            steps.append(op)
            continue
        if not isinstance(op, Gate):
            raise TypeError(op)
        if len(op.qubits) == 2:
            a, b = op.qubits
            if abs(a - b) != 1:
                raise ValueError("only nearest-neighbour two-qubit gates are supported")
            if a in busy or b in busy:
                if nsub < layers:
                    nsub += 1
                    busy = set()
                else:
                    close()
        elif len(op.qubits) != 1:
            raise ValueError("gates act on one or two qubits")
        if k > 0 and len(cur) >= k:
            close()
        cur.append(op)
        if len(op.qubits) == 2:
            busy.update(op.qubits)
    close()
    return n, steps


def sublayers(chunk: List[Gate]) -> List[List[Gate]]:
    """A chunk's gates cut into sub-layers by the one-layer rule (a two-qubit gate touching a
    qubit that carries a two-qubit gate of the current sub-layer starts the next one);
    single-qubit gates stay with the sub-layer they follow."""
    out: List[List[Gate]] = [[]]
    busy = set()
    for g in chunk:
        if len(g.qubits) == 2 and (set(g.qubits) & busy):
            out.append([])
            busy = set()
        out[-1].append(g)
        if len(g.qubits) == 2:
            busy.update(g.qubits)
    return out


def _pair_matrix(g: Gate, q: int) -> np.ndarray:
    """The 4x4 matrix of gate g acting on the pair (q, q+1), basis |s_q s_{q+1}>."""
    m = np.asarray(g.matrix, dtype=np.complex128)
    if len(g.qubits) == 1:
        return np.kron(m, np.eye(2)) if g.qubits[0] == q else np.kron(np.eye(2), m)
    a, b = g.qubits
    if a == q:
        return m
    # gate given on (q+1, q): reorder both the output and the input legs
    return m.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)


def chunk_blocks(n: int, chunk: List[Gate], c: np.ndarray):
    """The chunk as disjoint blocks for a branch with classical register c.

    Returns (blocks, empty): blocks is a list of (q, matrix) with a 4x4 matrix for a
    two-qubit block on (q, q+1) and a 2x2 matrix for a site without one.  Each block is the
    ordered product of the branch's applied gates on its qubits (a skipped conditional gate
    contributes the identity).  ``empty`` is True when every gate is skipped on this branch:
    then no compression step is made (Alg. 1 / Alg. 2 only compress non-empty chunks)."""
    applied = [g for g in chunk if cond_holds(g.cond, c)]
    left_of_pair = {min(g.qubits) for g in chunk if len(g.qubits) == 2}
    in_pair = left_of_pair | {q + 1 for q in left_of_pair}
    blocks = []
    for q in sorted(left_of_pair):
        G = np.eye(4, dtype=np.complex128)
        for g in applied:
            if set(g.qubits) <= {q, q + 1}:
                G = _pair_matrix(g, q) @ G
        blocks.append((q, G))
    for q in range(n):
        if q in in_pair:
            continue
        gs = [g for g in applied if g.qubits == (q,)]
        if not gs:
            continue
        U1 = np.eye(2, dtype=np.complex128)
        for g in gs:
            U1 = np.asarray(g.matrix, dtype=np.complex128) @ U1
        blocks.append((q, U1))
    return blocks, len(applied) == 0


def blocks_mpo(n: int, blocks):
    """MPO of a layer of disjoint blocks: W[j] of shape [D_l, 2(out), 2(in), D_r].

    A two-qubit block G on (q, q+1) is split by the SVD of G reshaped as
    (s_q' s_q) x (s_{q+1}' s_{q+1}) (operator-Schmidt decomposition):
    W_q[0, s', s, d] = U[(s's), d] sqrt(sigma_d), W_{q+1}[d, s', s, 0] =
    sqrt(sigma_d) Vh[d, (s's)], d over the non-zero sigma.  Other sites carry their 2x2
    block or the identity."""
    W = [np.eye(2, dtype=np.complex128).reshape(1, 2, 2, 1) for _ in range(n)]
    for q, G in blocks:
        if G.shape == (2, 2):
            W[q] = G.reshape(1, 2, 2, 1)
            continue
        M = G.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
        U, s, Vh = np.linalg.svd(M)
        r = max(1, int(np.sum(s > 1e-14 * s[0])))
        sq = np.sqrt(s[:r])
        W[q] = (U[:, :r] * sq[None, :]).reshape(1, 2, 2, r)
        W[q + 1] = (sq[:, None] * Vh[:r, :]).reshape(r, 2, 2, 1)
    return W


def chunk_unitary_dense(n: int, W) -> np.ndarray:
    """Contract an MPO into its dense 2^n x 2^n matrix (tests only; small n)."""
    T = W[0]  # [1, o, i, D]
    for j in range(1, n):
        T = np.einsum("aoiD,DpjE->aopijE", T.reshape(1, 2 ** j, 2 ** j, -1), W[j])
        T = T.reshape(1, 2 ** (j + 1), 2 ** (j + 1), -1)
    return T.reshape(2 ** n, 2 ** n)


def chunk_sublayer_blocks(n: int, chunk: List[Gate], c: np.ndarray):
    """The blocks of each sub-layer of a chunk for register c (``chunk_blocks`` per
    sub-layer), and whether every gate of the chunk is skipped."""
    subs = sublayers(chunk)
    blocks = [chunk_blocks(n, sub, c)[0] for sub in subs]
    applied = [g for g in chunk if cond_holds(g.cond, c)]
    return blocks, len(applied) == 0


def compose_mpo(Ws):
    """MPO of sub-layers applied in order (Ws[0] first): per site
    W[(d_1 .. d_L), s, t, (e_1 .. e_L)] = sum over the inner physical indices of
    W_L[d_L, s, u, e_L] ... W_1[d_1, v, t, e_1]; bond dimensions multiply."""
    out = Ws[0]
    for W2 in Ws[1:]:
        nxt = []
        for a, b in zip(out, W2):
            # a: [Da, s', t, Ea] applied first; b: [Db, s, s', Eb]
            # bonds grouped (a's, b's) on both sides of the site
            c = np.einsum("dsue,auvf->adsvfe", b, a)
            Da, Db, Ea, Eb = a.shape[0], b.shape[0], a.shape[3], b.shape[3]
            nxt.append(c.reshape(Da * Db, 2, 2, Ea * Eb))
        out = nxt
    return out
