"""O2: FP64 matrix product states and the variational compression step (oracle side;
test infrastructure only).

MPS (Sec. "Representing pure quantum states with tensor networks", paragraph "Matrix
Product States"): sites T[0..n-1], T[j] of shape [chi_j, 2, chi_{j+1}], chi_0 = chi_n = 1,
psi[s_0..s_{n-1}] = T[0][:, s_0, :] ... T[n-1][:, s_{n-1}, :].  The object also records
its orthogonality centre c: sites left of c are left-orthonormal, sites right of c are
right-orthonormal.

Compression step (Sec. "Simulating unitary quantum circuits with DMRG", Defs. "Unitary
chunk" and "Compression step"): given the ket A (normalised) and the chunk's MPO W, fit a
bra B of bond dimension <= chi_max maximising |<B|W A>|^2 by optimising one tensor at a
time with the others fixed: the environment F of a site is the overlap network with that
bra tensor removed, the optimum is F / sqrt(<F|F>), and the partial fidelity is
f = |<B|W A>|^2.

The paper states only the one-site update.  Readings used for what it leaves open:

1. Initial guess (this is where bond dimensions grow).  The chunk is a single layer of
   disjoint blocks; the initial bra is A with every block applied gate-by-gate in
   canonical form, two-qubit blocks followed by a truncated SVD of the two-site tensor
   (keep the smallest rank k <= chi_max whose discarded weight sum_{i>=k} s_i^2 is
   <= tol * sum_i s_i^2).  Without truncation this guess is the exact W|A>.  The two-qubit
   blocks are taken in order of q starting from the end of the layer nearest to the
   orthogonality centre (ascending when |c - q_min| <= |c - (q_max + 1)|), the centre
   moved to the nearer site of each block, and the singular values put on the site facing
   the next block (B_q = U, B_{q+1} = S Vh ascending; B_q = U S, B_{q+1} = Vh descending),
   so the centre crosses the layer once.
2. If no block discarded more than the tolerance (sum_{i>=k} s_i^2 <= tol * sum_i s_i^2
   for every block), the guess is W|A> up to that tolerance and is itself the optimum the
   sweeps converge to (f = 1 up to rounding): the sweeps are skipped, f is the product of
   the kept weight fractions and the centre stays where the guess left it.
3. Otherwise s one-site sweeps against the exact target W|A> (W the chunk's MPO), starting
   at the end of the chain nearest the centre the guess left (left to right when
   c <= n-1-c), then alternating; each site takes F / ||F|| re-orthonormalised by QR (LQ when
   moving right to left), the triangular factor being dropped because the next site's
   update is recomputed from the environments.  One direction is one sweep; the centre ends
   at the end the last sweep runs to.  Bond dimensions do not change in the sweeps.
4. f is ||F||^2 at the last update of the last sweep: B is normalised with every other
   site orthonormal, W unitary and A normalised, so ||F|| = |<B|W A>|.

Pins (tests/test_oracle_mps.py): the exact regime equals the dense state; every truncation
of the guess is the Eckart-Young projection at its bond with the kept weight fraction; f is
|<B|W A>|^2 recomputed densely, <= 1 and non-decreasing over sweeps; with one truncated bond
the sweeps reach the optimal truncation; converged sweeps are a stationary point (the
brute-force local optimum equals every site).  The state after a fixed small number of
sweeps in the truncated regime has no value fixed by the paper: parity unpinned beyond
these invariants.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

EINSUM = dict(optimize=True)


@dataclass
class MPS:
    T: List[np.ndarray]
    centre: int = 0

    @property
    def n(self) -> int:
        return len(self.T)

    def bonds(self) -> List[int]:
        return [1] + [t.shape[2] for t in self.T[:-1]] + [1]

    def copy(self) -> "MPS":
        return MPS([t.copy() for t in self.T], self.centre)


def product_zero(n: int) -> MPS:
    """|0...0> (Alg. 1 / Alg. 2 initial state): all bonds 1."""
    T = []
    for _ in range(n):
        t = np.zeros((1, 2, 1), dtype=np.complex128)
        t[0, 0, 0] = 1.0
        T.append(t)
    return MPS(T, 0)


def to_dense(mps: MPS) -> np.ndarray:
    """Contract the chain into the order-n amplitude tensor (tests only)."""
    v = mps.T[0]
    for t in mps.T[1:]:
        v = np.tensordot(v, t, axes=([v.ndim - 1], [0]))
    return v.reshape((2,) * mps.n)


# ----------------------------------------------------------------------------- gauge moves


def qr_hop_right(mps: MPS, j: int) -> None:
    """Move the centre from j to j+1: T_j = Q R, T_j := Q, T_{j+1} := R T_{j+1}."""
    t = mps.T[j]
    al, _, ar = t.shape
    Q, R = np.linalg.qr(t.reshape(al * 2, ar))
    mps.T[j] = Q.reshape(al, 2, Q.shape[1])
    mps.T[j + 1] = np.einsum("ka,asb->ksb", R, mps.T[j + 1])
    mps.centre = j + 1


def lq_hop_left(mps: MPS, j: int) -> None:
    """Move the centre from j to j-1: T_j = L Q (as al x (2 ar)), T_j := Q,
    T_{j-1} := T_{j-1} L."""
    t = mps.T[j]
    al, _, ar = t.shape
    Qh, Rh = np.linalg.qr(t.reshape(al, 2 * ar).conj().T)
    mps.T[j] = Qh.conj().T.reshape(Qh.shape[1], 2, ar)
    mps.T[j - 1] = np.einsum("asb,bk->ask", mps.T[j - 1], Rh.conj().T)
    mps.centre = j - 1


def move_centre(mps: MPS, target: int) -> None:
    while mps.centre < target:
        qr_hop_right(mps, mps.centre)
    while mps.centre > target:
        lq_hop_left(mps, mps.centre)


# ----------------------------------------------------------------------------- measurement


def measure_probs(mps: MPS, q: int):
    """p_m = <psi|P_m^{Q_q}|psi> (Sec. "Mid-circuit measurements"), evaluated at the
    orthogonality centre moved to q.  Returns the raw slice weights (r_0, r_1); their sum
    is the squared norm (1 up to rounding)."""
    move_centre(mps, q)
    t = mps.T[q]
    r0 = float(np.vdot(t[:, 0, :], t[:, 0, :]).real)
    r1 = float(np.vdot(t[:, 1, :], t[:, 1, :]).real)
    return r0, r1


def collapse(mps: MPS, q: int, m: int, r_m: float) -> None:
    """P_m on the physical leg of the centre tensor q, rescaled by 1/sqrt(r_m) so the
    state has norm 1 (Sec. "Mid-circuit measurements": only the local tensor changes)."""
    assert mps.centre == q
    t = mps.T[q].copy()
    t[:, 1 - m, :] = 0.0
    mps.T[q] = t / np.sqrt(r_m)


# ----------------------------------------------------------------------------- compression


# The three sums below are evaluated one pair of tensors at a time, in the order written
# (the usual order of MPS environment updates).  A single four-tensor einsum is the same sum,
# but numpy caps its intermediates at the largest operand and, once the MPO bond reaches 16,
# falls back to one loop nest over every index (hours instead of milliseconds).


def env_left(L, B, W, A):
    """L_{j+1}[c,e,x] = sum L_j[b,d,a] conj(B_j[b,s,c]) W_j[d,s,t,e] A_j[a,t,x]."""
    t = np.einsum("bda,atx->bdtx", L, A, **EINSUM)
    t = np.einsum("bdtx,dste->bsex", t, W, **EINSUM)
    return np.einsum("bsex,bsc->cex", t, B.conj(), **EINSUM)


def env_right(R, B, W, A):
    """R_j[b,d,a] = sum R_{j+1}[c,e,x] conj(B_j[b,s,c]) W_j[d,s,t,e] A_j[a,t,x]."""
    t = np.einsum("cex,atx->ceat", R, A, **EINSUM)
    t = np.einsum("ceat,dste->csda", t, W, **EINSUM)
    return np.einsum("csda,bsc->bda", t, B.conj(), **EINSUM)


def site_env(L, W, A, R):
    """F_j[b,s,c] = sum L_j[b,d,a] W_j[d,s,t,e] A_j[a,t,x] R_{j+1}[c,e,x]."""
    t = np.einsum("bda,atx->bdtx", L, A, **EINSUM)
    t = np.einsum("bdtx,dste->bsex", t, W, **EINSUM)
    return np.einsum("bsex,cex->bsc", t, R, **EINSUM)


def trunc_rank(s: np.ndarray, cap: int, tol: float) -> int:
    """Smallest k >= 1 with sum_{i>=k} s_i^2 <= tol * sum_i s_i^2, then min(k, cap)."""
    w = s.astype(np.float64) ** 2
    total = float(w.sum())
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]])  # tail[k] = sum_{i>=k}
    k = 1
    while k < len(s) and tail[k] > tol * total:
        k += 1
    return max(1, min(k, cap, len(s)))


@dataclass
class CompressInfo:
    f: float
    fidelities_per_sweep: List[float]
    guess_weights: List[float]


def initial_guess(A: MPS, blocks, chi_max: int, tol: float):
    """Initial bra: the chunk applied block by block to a copy of A in canonical form (the
    usual gate-by-gate update), blocks ordered as in reading 1 of the module header.  A
    two-qubit block G on (q, q+1): move the centre to the nearer of q, q+1,
    Theta[a,s,u,b] = sum G[s,u,t,v] A_q[a,t,x] A_{q+1}[x,v,b], truncated SVD of Theta as
    (2 chi_q) x (2 chi_{q+2}) with rank ``trunc_rank(s, chi_max, tol)``; S / ||S|| goes to
    q+1 (ascending order, centre q+1) or to q (descending, centre q).  A single-qubit block
    U on q: B_q[a,s,b] = sum_t U[s,t] A_q[a,t,b].  Returns (B, kept weight fractions,
    exact), exact meaning no block discarded more than tol of its weight."""
    B = A.copy()
    kept = []
    exact = True
    two = sorted((q, G) for q, G in blocks if G.shape == (4, 4))
    for q, G in blocks:
        if G.shape == (2, 2):
            B.T[q] = np.einsum("st,atb->asb", G, B.T[q])
    if two:
        c = B.centre
        ascending = abs(c - two[0][0]) <= abs(c - (two[-1][0] + 1))
        if not ascending:
            two = two[::-1]
    for q, G in two:
        move_centre(B, q if B.centre <= q else q + 1)
        th = np.einsum("asx,xtb->astb", B.T[q], B.T[q + 1])
        th = np.einsum("uvst,astb->auvb", G.reshape(2, 2, 2, 2), th)
        al, br = th.shape[0], th.shape[3]
        U, s, Vh = np.linalg.svd(th.reshape(al * 2, 2 * br), full_matrices=False)
        k = trunc_rank(s, chi_max, tol)
        w = float(np.sum(s[:k] ** 2))
        tot = float(np.sum(s ** 2))
        kept.append(w / tot)
        if tot - w > tol * tot:
            exact = False
        sk = s[:k] / np.sqrt(w)
        if ascending:
            B.T[q] = U[:, :k].reshape(al, 2, k)
            B.T[q + 1] = (sk[:, None] * Vh[:k]).reshape(k, 2, br)
            B.centre = q + 1
        else:
            B.T[q] = (U[:, :k] * sk[None, :]).reshape(al, 2, k)
            B.T[q + 1] = Vh[:k].reshape(k, 2, br)
            B.centre = q
    return B, kept, exact


def initial_guess_layers(A: MPS, sub_blocks, chi_max: int, tol: float):
    """The initial guess of a chunk of several sub-layers (each a list of disjoint blocks):
    ``initial_guess`` applied sub-layer after sub-layer, each starting from the state and
    centre the previous one left; the kept weight fractions of all truncations, and whether
    none discarded more than tol."""
    B, kept, exact = A, [], True
    for blocks in sub_blocks:
        B, k, e = initial_guess(B, blocks, chi_max, tol)
        kept += k
        exact = exact and e
    return B, kept, exact


def compress(A: MPS, blocks, W, chi_max: int, tol: float, sweeps: int, skip_exact: bool = True):
    """CompressionStep (Sec. "Simulating unitary quantum circuits with DMRG") with the
    readings in the module header.  ``blocks`` is the chunk as [(q, 4x4 or 2x2 matrix)], or
    for a chunk of several sub-layers a list of such lists (the guess takes them in order),
    W its MPO.  A is not modified.  Returns (B, info), B normalised; after the sweeps its
    centre is at the end the last sweep ran to; an exact guess (reading 2) is returned as it
    is unless ``skip_exact`` is False, which runs the sweeps on it all the same."""
    assert sweeps >= 1
    n = A.n
    if blocks and isinstance(blocks[0], list):  # a chunk of several sub-layers
        B0, kept, exact = initial_guess_layers(A, blocks, chi_max, tol)
    else:
        B0, kept, exact = initial_guess(A, blocks, chi_max, tol)
    if exact and skip_exact:
        f = float(np.prod(kept)) if kept else 1.0
        return B0, CompressInfo(f, [], kept)
    first = 0 if B0.centre <= n - 1 - B0.centre else 1  # 0: left to right first
    move_centre(B0, 0 if first == 0 else n - 1)
    B = B0.T
    one = np.ones((1, 1, 1), dtype=np.complex128)
    L: List = [None] * (n + 1)
    R: List = [None] * (n + 1)
    L[0] = one
    R[n] = one
    if first == 0:
        for j in range(n - 1, 0, -1):
            R[j] = env_right(R[j + 1], B[j], W[j], A.T[j])
    else:
        for j in range(0, n - 1):
            L[j + 1] = env_left(L[j], B[j], W[j], A.T[j])
    fids = []
    centre = B0.centre
    for sw in range(sweeps):
        if (sw + first) % 2 == 0:  # left to right
            for j in range(0, n - 1):
                F = site_env(L[j], W[j], A.T[j], R[j + 1])
                bl, br = F.shape[0], F.shape[2]
                Q, _ = np.linalg.qr(F.reshape(bl * 2, br))
                B[j] = Q.reshape(bl, 2, Q.shape[1])
                L[j + 1] = env_left(L[j], B[j], W[j], A.T[j])
            F = site_env(L[n - 1], W[n - 1], A.T[n - 1], R[n])
            nrm2 = float(np.vdot(F, F).real)
            B[n - 1] = F / np.sqrt(nrm2)
            centre = n - 1
        else:  # right to left
            for j in range(n - 1, 0, -1):
                F = site_env(L[j], W[j], A.T[j], R[j + 1])
                bl, br = F.shape[0], F.shape[2]
                Qh, _ = np.linalg.qr(F.reshape(bl, 2 * br).conj().T)
                B[j] = Qh.conj().T.reshape(Qh.shape[1], 2, br)
                R[j] = env_right(R[j + 1], B[j], W[j], A.T[j])
            F = site_env(L[0], W[0], A.T[0], R[1])
            nrm2 = float(np.vdot(F, F).real)
            B[0] = F / np.sqrt(nrm2)
            centre = 0
        fids.append(nrm2)
    return MPS(B, centre), CompressInfo(fids[-1], fids, kept)


# ----------------------------------------------------------------------------- exact mode


def apply_mpo_exact(A: MPS, W, svd_tol: float = 1e-14) -> MPS:
    """Exact W|A>: site-wise product with bonds chi*D, then an SVD sweep that drops only
    singular values below svd_tol * s_max (exact up to rounding).  Centre ends at 0."""
    n = A.n
    T = []
    for j in range(n):
        a, w = A.T[j], W[j]
        t = np.einsum("dste,atx->adsxe", w, a, **EINSUM)
        T.append(t.reshape(a.shape[0] * w.shape[0], 2, a.shape[2] * w.shape[3]))
    out = MPS(T, n - 1)
    out.centre = n - 1  # not canonical yet: sweep QR left to right, then SVD back
    for j in range(n - 1):
        t = out.T[j]
        al, _, ar = t.shape
        Q, R = np.linalg.qr(t.reshape(al * 2, ar))
        out.T[j] = Q.reshape(al, 2, Q.shape[1])
        out.T[j + 1] = np.einsum("ka,asb->ksb", R, out.T[j + 1])
    for j in range(n - 1, 0, -1):
        t = out.T[j]
        al, _, ar = t.shape
        U, s, Vh = np.linalg.svd(t.reshape(al, 2 * ar), full_matrices=False)
        k = max(1, int(np.sum(s > svd_tol * s[0])))
        out.T[j] = Vh[:k].reshape(k, 2, ar)
        out.T[j - 1] = np.einsum("asb,bk->ask", out.T[j - 1], U[:, :k] * s[None, :k])
    out.centre = 0
    return out
