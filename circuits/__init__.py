"""Seeded synthetic dynamic circuits shared by the CUDA path, the oracle and the tests.

This module only *generates inputs*: operation records and the random unitaries drawn
from a circuit seed.  It holds none of the simulation method's arithmetic (no chunking,
no MPO construction, no contraction, no measurement rule), so both independent sides
(the CPU oracle and the GPU library) can consume the same circuits.

Circuit model (paper, Sec. "Quantum states, quantum operations and dynamic circuits",
Defs. of unitary operation, mid-circuit measurement, classically controlled operation and
dynamic circuit D=(Q,C,O)):

* ``Gate``    -- a 1- or 2-qubit unitary, optionally classically controlled by a ``Cond``.
* ``Measure`` -- a computational-basis measurement of one qubit whose outcome overwrites
  one classical bit.
* ``Reset``   -- forces a qubit to |0> (Sec. "Reset operations"); each simulator lowers it
  itself.

Index conventions: qubit q is tensor axis q of the state (axis 0 = qubit 0 = MPS site 0).
A 2-qubit gate on ``qubits=(a, b)`` has a 4x4 matrix over the basis |s_a s_b> with s_a the
more significant bit, i.e. ``matrix.reshape(2,2,2,2)[out_a, out_b, in_a, in_b]``.

Workloads (synthetic, shaped like the paper's benchmarks, Sec. "Evaluation"):

* ``teleport``      -- 3-qubit teleportation, input Rz(phi)Ry(theta)|0> (Sec. "Quantum
  teleportation protocol"), optional final measurement of Bob's qubit.
* ``ghz_dynamic``   -- constant-depth dynamic GHZ preparation with parity feed-forward and
  ancilla resets (Sec. "Dynamic procedure for GHZ state preparation").
* ``brickwork``     -- random dynamic brickwork: Haar SU(4) layers, random mid-circuit
  measurements and outcome-conditioned Haar single-qubit gates (stand-in for the paper's
  random dynamic circuits of Sec. "Random dynamic circuits", whose generator and circuits
  are not available).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple, Union

import numpy as np

__all__ = [
    "Cond", "Gate", "Measure", "Reset", "Circuit",
    "H", "X", "Z", "CNOT", "ry", "rz", "haar_unitary", "haar_su4",
    "state_prep", "teleport", "ghz_dynamic", "brickwork",
]

# ----------------------------------------------------------------------------- records


@dataclass(frozen=True)
class Cond:
    """Boolean condition phi(c) over classical bits (Def. classically controlled operation).

    ``op == "xor"``: phi = (XOR of the listed bits) == value   (single bit, prefix parity)
    ``op == "and"``: phi = (AND of the listed bits) == value
    ``op == "or"``: phi = (OR of the listed bits) == value
    ``op == "table"``: any Boolean function of at most 5 bits, given by its truth table: the
    listed bits, taken in ascending bit order, form the index i = sum_k c[b_k] 2^k (b_0 the
    smallest), and phi = bit i of ``value`` (a non-negative integer below 2^32).
    """

    bits: Tuple[int, ...]
    op: str = "xor"
    value: int = 1


@dataclass(frozen=True)
class Gate:
    qubits: Tuple[int, ...]
    matrix: np.ndarray = field(compare=False)
    cond: Optional[Cond] = None
    name: str = ""


@dataclass(frozen=True)
class Measure:
    qubit: int
    cbit: int


@dataclass(frozen=True)
class Reset:
    qubit: int
    cbit: int


Op = Union[Gate, Measure, Reset]


@dataclass
class Circuit:
    n_qubits: int
    n_cbits: int
    ops: List[Op]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_measurements(self) -> int:
        return sum(isinstance(o, (Measure, Reset)) for o in self.ops)


# ----------------------------------------------------------------------------- gates

H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
# control = first listed qubit (most significant), target = second
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)


def ry(theta: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(phi: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * phi), 0], [0, np.exp(0.5j * phi)]], dtype=np.complex128)


def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random U(d): QR of a complex Ginibre matrix with the phases of diag(R) fixed
    (Mezzadri, Notices AMS 54 (2007))."""
    zr = rng.standard_normal((d, d))
    zi = rng.standard_normal((d, d))
    z = (zr + 1j * zi) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def haar_su4(rng: np.random.Generator) -> np.ndarray:
    """Haar SU(4): Haar U(4) divided by a fourth root of its determinant."""
    u = haar_unitary(rng, 4)
    det = np.linalg.det(u)
    return u / det ** 0.25


def state_prep(alpha: complex, beta: complex) -> np.ndarray:
    """A unitary whose first column is the normalised (alpha, beta)."""
    nrm = np.sqrt(abs(alpha) ** 2 + abs(beta) ** 2)
    a, b = alpha / nrm, beta / nrm
    return np.array([[a, -np.conj(b)], [b, np.conj(a)]], dtype=np.complex128)


# ----------------------------------------------------------------------------- workloads


def teleport(seed: int = 1, bob_measure: bool = False,
             amplitudes: Optional[Tuple[complex, complex]] = None) -> Circuit:
    """3-qubit teleportation (Sec. "Quantum teleportation protocol").

    q0 carries the input, either ``amplitudes`` (normalised) or Rz(phi)Ry(theta)|0> with
    theta ~ U[0, pi), phi ~ U[0, 2 pi) drawn from ``seed``.  Bell pair on (q1, q2) by H,
    CNOT; Alice applies CNOT(q0 -> q1), H(q0); measures q0 -> c0, q1 -> c1; Bob applies X
    if c1 and Z if c0.  With ``bob_measure`` q2 is finally measured into c2.
    """
    if amplitudes is not None:
        prep = state_prep(*amplitudes)
        theta = phi = None
    else:
        rng = np.random.default_rng(seed)
        theta = float(rng.uniform(0.0, np.pi))
        phi = float(rng.uniform(0.0, 2.0 * np.pi))
        prep = rz(phi) @ ry(theta)
    ops: List[Op] = [
        Gate((0,), prep, name="prep"),
        Gate((1,), H, name="H"),
        Gate((1, 2), CNOT, name="CNOT"),
        Gate((0, 1), CNOT, name="CNOT"),
        Gate((0,), H, name="H"),
        Measure(0, 0),
        Measure(1, 1),
        Gate((2,), X, cond=Cond((1,), "xor", 1), name="cX"),
        Gate((2,), Z, cond=Cond((0,), "xor", 1), name="cZ"),
    ]
    n_cbits = 2
    if bob_measure:
        ops.append(Measure(2, 2))
        n_cbits = 3
    return Circuit(3, n_cbits, ops, name="teleport",
                   meta={"theta": theta, "phi": phi, "input": prep[:, 0].copy()})


def ghz_dynamic(n: int) -> Circuit:
    """Constant-depth dynamic GHZ preparation (Sec. "Dynamic procedure for GHZ state
    preparation", after Baeumer et al.).

    Data qubits on even sites, ancillas on odd sites.  Sublayers: H on data; CNOT from each
    data qubit 2i to ancilla 2i+1; CNOT from data 2i+2 to ancilla 2i+1; measure the
    ancillas in ascending order (ancilla 2i+1 -> cbit i); X on data 2k iff the XOR of the
    outcomes of ancillas 1, 3, ..., 2k-1 is 1; reset every ancilla, lowered as in Sec.
    "Reset operations" and applied as one parallel layer: the reset measurement of ancilla
    i goes to cbit n_anc + i, then X on it conditioned on that bit.

    For odd n this is the paper's layout with r = (n-1)/2 random outcomes.  For even n the
    last site n-1 is an ancilla with a single data neighbour; it receives no CNOT, so its
    measurement is deterministically 0 and r = n/2 - 1 random outcomes remain.
    """
    assert n >= 3
    data = list(range(0, n, 2))
    anc = list(range(1, n, 2))
    ops: List[Op] = []
    for d in data:
        ops.append(Gate((d,), H, name="H"))
    for a in anc:
        if a + 1 < n:  # an ancilla with two data neighbours
            ops.append(Gate((a - 1, a), CNOT, name="CNOT"))
    for a in anc:
        if a + 1 < n:
            ops.append(Gate((a + 1, a), CNOT, name="CNOT"))
    n_anc = len(anc)
    for i, a in enumerate(anc):
        ops.append(Measure(a, i))
    for k in range(1, len(data)):
        bits = tuple(range(0, k))  # ancillas 1,3,...,2k-1 carry cbits 0..k-1
        ops.append(Gate((data[k],), X, cond=Cond(bits, "xor", 1), name="cX"))
    # ancilla resets as one parallel layer, already lowered: all reset measurements, then
    # the X corrections conditioned on each ancilla's own reset bit
    for i, a in enumerate(anc):
        ops.append(Measure(a, n_anc + i))
    for i, a in enumerate(anc):
        ops.append(Gate((a,), X, cond=Cond((n_anc + i,), "xor", 1), name="resetX"))
    r = sum(1 for a in anc if a + 1 < n)
    return Circuit(n, 2 * n_anc, ops, name=f"ghz{n}", meta={"r": r, "data": data, "anc": anc})


def brickwork(n: int, depth: int, p_meas: float, seed: int) -> Circuit:
    """Random dynamic brickwork (stand-in for the paper's random dynamic circuits).

    Layer l applies Haar SU(4) gates on the pairs (j, j+1) with j = l (mod 2).  After the
    layer each qubit is selected for measurement with probability ``p_meas`` (selection
    drawn from ``seed``: the circuit is static, identical for all shots); selected qubits
    are measured in ascending order, each into a fresh classical bit; then for each
    measured q < n-1 a Haar U(2) on q+1 is applied iff that bit is 1.
    """
    rng = np.random.default_rng(seed)
    ops: List[Op] = []
    cbit = 0
    for layer in range(depth):
        for j in range(layer % 2, n - 1, 2):
            ops.append(Gate((j, j + 1), haar_su4(rng), name="U4"))
        sel = rng.random(n) < p_meas
        measured = [q for q in range(n) if sel[q]]
        bits = {}
        for q in measured:
            ops.append(Measure(q, cbit))
            bits[q] = cbit
            cbit += 1
        for q in measured:
            u = haar_unitary(rng, 2)
            if q + 1 < n:
                ops.append(Gate((q + 1,), u, cond=Cond((bits[q],), "xor", 1), name="cU"))
    return Circuit(n, max(cbit, 1), ops, name=f"brick{n}x{depth}",
                   meta={"depth": depth, "p": p_meas, "seed": seed})


def split_layers(circ: Circuit) -> List[List[Op]]:
    """The circuit cut into segments of one chunk and the measurements that follow it: a cut
    before the first non-measurement after a measurement, and before a two-qubit gate that
    touches a qubit already carrying a two-qubit gate of the segment.  For ``brickwork``
    segment l holds the conditional gates of layer l-1, the two-qubit gates of layer l and
    the measurements of layer l.  Concatenated, the segments give the circuit back."""
    out: List[List[Op]] = []
    cur: List[Op] = []
    busy: set = set()
    prev_meas = False
    for op in circ.ops:
        meas = isinstance(op, (Measure, Reset))
        two = isinstance(op, Gate) and len(op.qubits) == 2
        if cur and ((prev_meas and not meas) or (two and busy & set(op.qubits))):
            out.append(cur)
            cur, busy = [], set()
        cur.append(op)
        if two:
            busy |= set(op.qubits)
        prev_meas = meas
    if cur:
        out.append(cur)
    return out
