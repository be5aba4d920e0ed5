"""Pins of the MPS oracle (O2): gauge moves, measurement, the chunk MPO and the
compression step against the state-vector oracle, dense brute force, Eckart-Young and the
invariants the method fixes (f <= 1, f non-decreasing over sweeps, exactness when chi is
large enough)."""
import itertools

import numpy as np
import pytest

import circuits as C
from conftest import read_golden_rows
from oracle import drivers as D, layers as LY, mps as M, statevector as SV


def random_mps(rng, n, chi):
    bonds = [1] + [min(chi, 2 ** min(b, n - b)) for b in range(1, n)] + [1]
    T = [rng.standard_normal((bonds[j], 2, bonds[j + 1]))
         + 1j * rng.standard_normal((bonds[j], 2, bonds[j + 1])) for j in range(n)]
    m = M.MPS(T, n - 1)
    # canonicalise (centre 0) and normalise
    for j in range(n - 1, 0, -1):
        M.lq_hop_left(m, j)
    m.T[0] /= np.linalg.norm(m.T[0])
    return m


def dense(m):
    return M.to_dense(m).reshape(-1)


def test_product_zero():
    v = dense(M.product_zero(4))
    assert v[0] == 1 and np.count_nonzero(v) == 1


@pytest.mark.parametrize("n,chi", [(4, 4), (6, 3)])
def test_gauge_moves_preserve_state_and_orthonormality(n, chi):
    rng = np.random.default_rng(n * 10 + chi)
    m = random_mps(rng, n, chi)
    v0 = dense(m)
    for tgt in [n - 1, 2, 0, n - 2]:
        M.move_centre(m, tgt)
        np.testing.assert_allclose(dense(m), v0, atol=1e-12)
        for j in range(tgt):  # left-orthonormal
            t = m.T[j]
            g = np.einsum("asb,asc->bc", t.conj(), t)
            np.testing.assert_allclose(g, np.eye(g.shape[0]), atol=1e-12)
        for j in range(tgt + 1, n):  # right-orthonormal
            t = m.T[j]
            g = np.einsum("asb,csb->ac", t, t.conj())
            np.testing.assert_allclose(g, np.eye(g.shape[0]), atol=1e-12)


def test_measure_and_collapse_match_statevector():
    rng = np.random.default_rng(5)
    n = 5
    m = random_mps(rng, n, 4)
    psi = M.to_dense(m)
    for q in [3, 0, 4, 2]:
        r0, r1 = M.measure_probs(m, q)
        s0, s1 = SV.probabilities(psi, q)
        assert abs(r0 - s0) < 1e-12 and abs(r1 - s1) < 1e-12
    M.measure_probs(m, 2)
    r0, r1 = M.measure_probs(m, 2)
    M.collapse(m, 2, 1, r1)
    want = SV.project(psi, 2, 1, SV.probabilities(psi, 2)[1])
    np.testing.assert_allclose(M.to_dense(m), want, atol=1e-12)


def test_collapse_normalises_an_unnormalised_state():
    # the rescale uses the raw slice weight r_m, so the post-measurement state has norm 1
    # whatever the norm before (a state whose norm rounding moved); the conditional
    # probability r_m / (r_0 + r_1) is unchanged by the scale
    rng = np.random.default_rng(11)
    m = random_mps(rng, 6, 4)
    psi = M.to_dense(m).reshape(-1)
    m.T[m.centre] = m.T[m.centre] * 1.7
    r0, r1 = M.measure_probs(m, 3)
    assert abs((r0 + r1) - 1.7 ** 2) < 1e-12
    p0 = SV.probabilities(psi.reshape([2] * 6), 3)[0]
    assert abs(r0 / (r0 + r1) - p0) < 1e-12
    M.collapse(m, 3, 0, r0)
    out = M.to_dense(m).reshape(-1)
    assert abs(np.vdot(out, out).real - 1.0) < 1e-12
    want = SV.project(psi.reshape([2] * 6), 3, 0, p0).reshape(-1)
    assert abs(abs(np.vdot(want, out)) - 1.0) < 1e-12


def test_blocks_mpo_matches_dense_layer():
    rng = np.random.default_rng(3)
    n = 5
    chunk = [C.Gate((1,), C.haar_unitary(rng, 2)),
             C.Gate((1, 2), C.haar_su4(rng)),
             C.Gate((4, 3), C.CNOT),
             C.Gate((0,), C.H),
             C.Gate((2,), C.X, cond=C.Cond((0,), "xor", 1)),
             C.Gate((3,), C.Z, cond=C.Cond((0,), "xor", 0))]
    for c0 in (0, 1):
        c = np.array([c0])
        blocks, empty = LY.chunk_blocks(n, chunk, c)
        assert not empty
        W = LY.blocks_mpo(n, blocks)
        got = LY.chunk_unitary_dense(n, W)
        # brute force: apply the applied gates in order to every basis vector
        want = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
        for col in range(2 ** n):
            e = np.zeros(2 ** n, dtype=np.complex128)
            e[col] = 1
            v = e.reshape((2,) * n)
            for g in chunk:
                if SV.cond_holds(g.cond, c):
                    v = SV.apply_gate(v, g.qubits, g.matrix)
            want[:, col] = v.reshape(-1)
        np.testing.assert_allclose(got, want, atol=1e-12)
        # CNOT has operator-Schmidt rank 2
        assert W[3].shape[3] == 2


def test_chunking_rules():
    circ = C.ghz_dynamic(7)
    n, steps = LY.chunk_circuit(circ)
    kinds = ["M" if isinstance(s, C.Measure) else len(s) for s in steps]
    # H+CNOT layer, second CNOT layer, 3 measurements, feed-forward X layer,
    # 3 reset measurements, reset X layer
    assert kinds == [7, 3, "M", "M", "M", 3, "M", "M", "M", 3]
    circ = C.Circuit(3, 0, [C.Gate((0, 1), C.CNOT), C.Gate((1, 2), C.CNOT)])
    assert len(LY.chunk_circuit(circ)[1]) == 2
    assert len(LY.chunk_circuit(circ, k=1)[1]) == 2
    circ = C.Circuit(4, 0, [C.Gate((0, 1), C.CNOT), C.Gate((2, 3), C.CNOT), C.Gate((0,), C.H)])
    assert len(LY.chunk_circuit(circ)[1]) == 1
    assert len(LY.chunk_circuit(circ, k=2)[1]) == 2


def _layer_blocks(rng, n, parity):
    return [(q, C.haar_su4(rng)) for q in range(parity, n - 1, 2)]


@pytest.mark.parametrize("n", [4, 7])
def test_compress_exact_regime_equals_statevector(n):
    rng = np.random.default_rng(n)
    A = random_mps(rng, n, 2)
    blocks = _layer_blocks(rng, n, 1) + [(0, C.haar_unitary(rng, 2))]
    W = LY.blocks_mpo(n, blocks)
    want = LY.chunk_unitary_dense(n, W) @ dense(A)
    # the guess is exact: returned as it is (the sweeps are skipped)
    B, info = M.compress(A.copy(), blocks, W, 64, 0.0, 2)
    assert info.fidelities_per_sweep == []
    assert abs(info.f - 1.0) < 1e-12
    assert abs(abs(np.vdot(dense(B), want)) - 1.0) < 1e-12
    # ... and sweeping it all the same returns the same state: the shortcut loses nothing.
    # The sweeps start at the end nearest the guess's centre and alternate.
    first = 0 if B.centre <= n - 1 - B.centre else 1
    for s in (1, 2, 3):
        B2, info = M.compress(A.copy(), blocks, W, 64, 0.0, s, skip_exact=False)
        assert abs(info.f - 1.0) < 1e-12
        assert abs(abs(np.vdot(dense(B2), dense(B))) - 1.0) < 1e-12
        assert B2.centre == (n - 1 if (s - 1 + first) % 2 == 0 else 0)


@pytest.mark.parametrize("centre", [0, 3, 8])
def test_guess_block_order_starts_nearest_the_centre(centre):
    # n = 9, blocks on (1,2), (3,4), (5,6): from the left end the guess runs ascending and
    # leaves the centre at q_max + 1 = 6; from the right end descending, centre q_min = 1.
    rng = np.random.default_rng(5)
    n = 9
    A = random_mps(rng, n, 2)
    M.move_centre(A, centre)
    blocks = [(q, C.haar_su4(rng)) for q in (1, 3, 5)]
    W = LY.blocks_mpo(n, blocks)
    want = LY.chunk_unitary_dense(n, W) @ dense(A)
    B, kept, exact = M.initial_guess(A, blocks, 64, 0.0)
    assert exact and all(abs(x - 1.0) < 1e-12 for x in kept)
    assert B.centre == (6 if centre <= 4 else 1)
    assert abs(abs(np.vdot(dense(B), want)) - 1.0) < 1e-12
    # canonical form around the centre: left sites left-orthonormal, right sites right-
    for j, t in enumerate(B.T):
        al, _, ar = t.shape
        if j < B.centre:
            m = t.reshape(al * 2, ar)
            np.testing.assert_allclose(m.conj().T @ m, np.eye(ar), atol=1e-12)
        elif j > B.centre:
            m = t.reshape(al, 2 * ar)
            np.testing.assert_allclose(m @ m.conj().T, np.eye(al), atol=1e-12)


@pytest.mark.parametrize("seed,centre", [(1, 0), (2, 0), (3, 0), (4, 7), (5, 7)])
def test_compress_truncated_fidelity_definition_and_monotone(seed, centre):
    # centre 0: the guess runs left to right and the sweeps start right to left; centre 7:
    # the other way round
    rng = np.random.default_rng(seed)
    n = 8
    A = random_mps(rng, n, 3)  # bonds <= chi_max, as every compression leaves them
    M.move_centre(A, centre)
    blocks = _layer_blocks(rng, n, seed % 2)
    W = LY.blocks_mpo(n, blocks)
    target = LY.chunk_unitary_dense(n, W) @ dense(A)
    fs = []
    for s in range(1, 7):
        B, info = M.compress(A.copy(), blocks, W, 3, 0.0, s)
        # f is |<B|W A>|^2, recomputed densely; B normalised
        assert abs(np.linalg.norm(dense(B)) - 1.0) < 1e-12
        assert abs(abs(np.vdot(dense(B), target)) ** 2 - info.f) < 1e-12
        assert info.f <= 1.0 + 1e-12
        assert all(b <= 3 for b in B.bonds())
        fs.append(info.f)
        # the per-sweep record is non-decreasing too
        assert all(y >= x - 1e-12 for x, y in zip(info.fidelities_per_sweep,
                                                   info.fidelities_per_sweep[1:]))
    assert all(y >= x - 1e-12 for x, y in zip(fs, fs[1:]))
    assert fs[-1] < 1.0 - 1e-6  # truncation really happened


def test_compress_two_sites_is_eckart_young():
    rng = np.random.default_rng(11)
    A = random_mps(rng, 2, 2)
    G = C.haar_su4(rng)
    blocks = [(0, G)]
    W = LY.blocks_mpo(2, blocks)
    target = (G @ dense(A)).reshape(2, 2)
    s = np.linalg.svd(target, compute_uv=False)
    B, info = M.compress(A.copy(), blocks, W, 1, 0.0, 2)
    assert abs(info.f - s[0] ** 2) < 1e-12


def test_compress_converges_to_optimal_middle_truncation():
    # n = 4, chi_max = 2: only the middle bond (exact rank 4) needs truncating, so the global
    # optimum is the rank-2 SVD truncation of the exact state at that bond.
    rng = np.random.default_rng(4)
    n = 4
    A = random_mps(rng, n, 2)
    blocks = [(1, C.haar_su4(rng))]
    W = LY.blocks_mpo(n, blocks)
    target = LY.chunk_unitary_dense(n, W) @ dense(A)
    s = np.linalg.svd(target.reshape(4, 4), compute_uv=False)
    B, info = M.compress(A.copy(), blocks, W, 2, 0.0, 12)
    assert abs(info.f - (s[0] ** 2 + s[1] ** 2)) < 1e-9


def test_truncation_rank_rule():
    s = np.array([0.8, 0.5, 0.3, 1e-6, 1e-9])
    assert M.trunc_rank(s, 10, 0.0) == 5
    assert M.trunc_rank(s, 10, 1e-10) == 3    # 1e-12 + 1e-18 discarded relative to ~0.98
    assert M.trunc_rank(s, 2, 1e-10) == 2
    assert M.trunc_rank(np.array([1.0, 0.0]), 4, 1e-12) == 1


def test_apply_mpo_exact_matches_dense():
    rng = np.random.default_rng(8)
    n = 6
    A = random_mps(rng, n, 4)
    blocks = _layer_blocks(rng, n, 0)
    W = LY.blocks_mpo(n, blocks)
    B = M.apply_mpo_exact(A, W)
    np.testing.assert_allclose(dense(B), LY.chunk_unitary_dense(n, W) @ dense(A), atol=1e-12)


# ----------------------------------------------------------------------------- drivers


@pytest.mark.parametrize("circ", [C.teleport(2), C.ghz_dynamic(9), C.ghz_dynamic(10),
                                  C.brickwork(8, 6, 0.2, 5)], ids=lambda c: c.name)
def test_single_path_mps_equals_statevector(circ):
    prm = D.Params(chi_max=64, tol=1e-12, sweeps=2)
    for shot in range(3):
        r = D.run_single_path(circ, prm, 17, shot)
        s = SV.run_single_path(circ, 17, shot)
        assert r.outcomes == s.outcomes
        assert abs(r.p - s.p) < 1e-12
        assert abs(r.F - 1.0) < 1e-10
        assert abs(abs(np.vdot(M.to_dense(r.mps), s.psi)) ** 2 - 1.0) < 1e-10


@pytest.mark.parametrize("row", read_golden_rows("ghz_paper.txt")[:3])
def test_multi_path_mps_ghz(row):
    n, r, npaths = (int(x) for x in row)
    circ = C.ghz_dynamic(n)
    prm = D.Params(chi_max=4, tol=1e-10, sweeps=2)  # the paper's chi = 4 for GHZ
    br = D.run_multi_path(circ, prm)
    assert len(br) == npaths
    for b in br:
        assert abs(b.p - 2.0 ** -r) < 1e-12
        assert abs(b.F - 1.0) < 1e-10
    assert abs(D.multipath_fidelity(br) - 1.0) < 1e-10


def test_multi_path_mps_equals_statevector_with_topm():
    circ = C.brickwork(6, 5, 0.3, 2)
    prm = D.Params(chi_max=64, tol=1e-12, sweeps=2)
    for Mcap in (None, 4):
        a = D.run_multi_path(circ, prm, M=Mcap)
        b = SV.run_multi_path(circ, M=Mcap)
        assert [x.path for x in a] == [y.path for y in b]
        for x, y in zip(a, b):
            assert abs(x.p - y.p) < 1e-12
            assert abs(abs(np.vdot(M.to_dense(x.mps), y.psi)) ** 2 - 1) < 1e-10


def test_teleport_chi2_paper_setting():
    # the paper's teleport setting chi = 2, s = 2 reproduces the circuit semantics
    circ = C.teleport(3)
    br = D.run_multi_path(circ, D.Params(chi_max=2, tol=1e-10, sweeps=2))
    assert len(br) == 4
    inp = circ.meta["input"]
    for b in br:
        assert abs(b.p - 0.25) < 1e-12
        psi = M.to_dense(b.mps)
        bob = psi[b.path[0], b.path[1], :]
        assert abs(abs(np.vdot(bob, inp)) ** 2 - 1.0) < 1e-12


# ----------------------------------------------------------------------------- truncated guess
# Pins of the initial guess in the truncated regime (reading 1 of the oracle's compression
# step: blocks applied in canonical form, each followed by a truncated SVD).  In canonical
# form with the centre on the block, the SVD of the two-site tensor is the Schmidt
# decomposition of the whole state at the block's middle bond, so each truncation must equal
# the Eckart-Young best rank-k approximation of the dense state at that cut, renormalised,
# and its kept weight fraction is sum_{i<k} s_i^2 / sum_i s_i^2 of the dense singular values.


def _dense_gate2(psi, q, G):
    """(G on qubits q, q+1) psi for psi of shape (2,)*n, G over |s_q s_{q+1}>."""
    out = np.tensordot(G.reshape(2, 2, 2, 2), psi, axes=([2, 3], [q, q + 1]))
    return np.moveaxis(out, [0, 1], [q, q + 1])


def _eckart_young(psi, cut, k):
    """Best rank-k approximation of psi across (first `cut` qubits | rest), normalised, and
    the kept weight fraction."""
    Mx = psi.reshape(2 ** cut, -1)
    U, s, Vh = np.linalg.svd(Mx, full_matrices=False)
    assert s[k - 1] > s[k] * (1 + 1e-6), "degenerate cut: the truncation is not unique"
    Mk = (U[:, :k] * s[:k]) @ Vh[:k]
    w, tot = float(np.sum(s[:k] ** 2)), float(np.sum(s ** 2))
    return (Mk / np.sqrt(w)).reshape(psi.shape), w / tot


def _assert_canonical(m):
    for j in range(m.centre):
        t = m.T[j]
        g = np.einsum("asb,asc->bc", t.conj(), t)
        np.testing.assert_allclose(g, np.eye(g.shape[0]), atol=1e-12)
    for j in range(m.centre + 1, m.n):
        t = m.T[j]
        g = np.einsum("asb,csb->ac", t, t.conj())
        np.testing.assert_allclose(g, np.eye(g.shape[0]), atol=1e-12)


@pytest.mark.parametrize("n,q,chi", [(3, 0, 1), (3, 1, 1), (4, 1, 2), (4, 0, 1), (4, 2, 1)])
@pytest.mark.parametrize("start", ["left", "right"])
def test_guess_single_truncated_block_is_eckart_young(n, q, chi, start):
    rng = np.random.default_rng(100 * n + 10 * q + chi)
    A = random_mps(rng, n, 4)
    M.move_centre(A, 0 if start == "left" else n - 1)
    G = C.haar_su4(rng)
    B, kept, exact = M.initial_guess(A, [(q, G)], chi, 1e-10)
    want, frac = _eckart_young(_dense_gate2(M.to_dense(A), q, G), q + 1, chi)
    assert not exact
    np.testing.assert_allclose(M.to_dense(B), want, atol=1e-12)
    assert abs(kept[0] - frac) < 1e-12 and frac < 1 - 1e-6
    assert B.bonds()[q + 1] == chi
    # ascending (centre left of the block) leaves the centre on q+1, descending on q
    assert B.centre == (q + 1 if start == "left" else q)
    _assert_canonical(B)
    assert abs(np.linalg.norm(M.to_dense(B)) - 1) < 1e-12


@pytest.mark.parametrize("start", ["left", "right"])
def test_guess_two_truncated_blocks_sequential_eckart_young(start):
    # blocks on (1, 2) and (3, 4) of 6 qubits, both cut to chi = 2: the guess truncates the
    # block nearest the centre first; each truncation is the dense Eckart-Young projection
    # of the state the previous one left, and the kept weights are those fractions
    n, chi = 6, 2
    rng = np.random.default_rng(61)
    A = random_mps(rng, n, 8)
    M.move_centre(A, 0 if start == "left" else n - 1)
    G1, G3 = C.haar_su4(rng), C.haar_su4(rng)
    B, kept, exact = M.initial_guess(A, [(1, G1), (3, G3)], chi, 1e-10)
    psi = _dense_gate2(_dense_gate2(M.to_dense(A), 1, G1), 3, G3)
    order = [1, 3] if start == "left" else [3, 1]
    fracs = []
    for q in order:
        psi, fr = _eckart_young(psi, q + 1, chi)
        fracs.append(fr)
    assert not exact
    np.testing.assert_allclose(M.to_dense(B), psi, atol=1e-11)
    np.testing.assert_allclose(kept, fracs, atol=1e-12)
    assert abs(np.prod(kept) - np.prod(fracs)) < 1e-12 and np.prod(fracs) < 1 - 1e-4
    assert B.centre == (4 if start == "left" else 1)
    _assert_canonical(B)
    # the two orders give different states here, so the test fixes the order
    other = _dense_gate2(_dense_gate2(M.to_dense(A), 1, G1), 3, G3)
    for q in order[::-1]:
        other, _ = _eckart_young(other, q + 1, chi)
    assert np.linalg.norm(other - psi) > 1e-6


def test_single_path_run_in_segments_equals_one_pass():
    # the oracle's step-wise Alg. 1 (used for bounded CPU timings) makes the same draws and
    # compressions as one pass when each call ends at a measurement run
    circ = C.brickwork(10, 8, 0.2, 4)
    prm = D.Params(chi_max=8, tol=1e-10, sweeps=2)
    one = D.run_single_path(circ, prm, 2, 5)
    r = D.SinglePathRun(circ.n_qubits, circ.n_cbits, prm, 2, 5)
    for seg in C.split_layers(circ):
        r.run(seg)
    two = r.result()
    assert two.outcomes == one.outcomes and two.fids == one.fids and two.p == one.p
    np.testing.assert_allclose(M.to_dense(two.mps), M.to_dense(one.mps), atol=1e-12)


# ----------------------------------------------------------------------------- multi-layer
# Chunks of several layers (Sec. "Handling unitary chunks in dynamic circuits": a chunk
# holds up to k operations), with the composed MPO (bond dimensions multiply) and the guess
# taken sub-layer by sub-layer.


def _dense_of_gates(n, gates, c):
    want = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    for col in range(2 ** n):
        e = np.zeros(2 ** n, dtype=np.complex128)
        e[col] = 1
        v = e.reshape((2,) * n)
        for g in gates:
            if SV.cond_holds(g.cond, c):
                v = SV.apply_gate(v, g.qubits, g.matrix)
        want[:, col] = v.reshape(-1)
    return want


@pytest.mark.parametrize("layers", [2, 3, 4])
def test_composed_mpo_matches_dense_chunk(layers):
    rng = np.random.default_rng(40 + layers)
    n = 5
    circ = C.brickwork(n, layers, 0.0, 17)
    chunk = [op for op in circ.ops]
    chunk.insert(2, C.Gate((3,), C.haar_unitary(rng, 2)))
    chunk.append(C.Gate((0,), C.X, cond=C.Cond((0,), "xor", 1)))
    for c0 in (0, 1):
        c = np.array([c0])
        sub, empty = LY.chunk_sublayer_blocks(n, chunk, c)
        assert not empty and len(sub) == layers
        W = LY.compose_mpo([LY.blocks_mpo(n, b) for b in sub])
        np.testing.assert_allclose(LY.chunk_unitary_dense(n, W), _dense_of_gates(n, chunk, c),
                                   atol=1e-12)
        # brickwork layers alternate bonds: two layers give D = 4, three and four give 16 on
        # the bonds the first and third layer both cross
        assert max(w.shape[3] for w in W) == (4 if layers == 2 else 16)


@pytest.mark.parametrize("layers", [2, 3])
def test_composed_mpo_of_stacked_layers_matches_dense(layers):
    # every sub-layer on the same pairs: bond dimensions 4^layers, the product still the
    # dense chunk (sub-layers applied in order)
    n = 4
    lay = C.split_layers(C.brickwork(n, 2 * layers, 0.0, 23))
    chunk = [g for i in range(layers) for g in lay[2 * i]]
    c = np.zeros(1, dtype=np.int64)
    sub, empty = LY.chunk_sublayer_blocks(n, chunk, c)
    assert len(sub) == layers
    W = LY.compose_mpo([LY.blocks_mpo(n, b) for b in sub])
    assert max(w.shape[3] for w in W) == 4 ** layers
    np.testing.assert_allclose(LY.chunk_unitary_dense(n, W), _dense_of_gates(n, chunk, c),
                               atol=1e-12)
    # the reversed order is a different operator: the composition order is pinned
    Wr = LY.compose_mpo([LY.blocks_mpo(n, b) for b in sub[::-1]])
    assert np.abs(LY.chunk_unitary_dense(n, Wr) - _dense_of_gates(n, chunk, c)).max() > 1e-3


def test_multi_layer_chunking_rules():
    circ = C.brickwork(6, 6, 0.0, 2)
    assert len(LY.chunk_circuit(circ)[1]) == 6
    assert len(LY.chunk_circuit(circ, layers=2)[1]) == 3
    assert len(LY.chunk_circuit(circ, layers=3)[1]) == 2
    assert len(LY.chunk_circuit(circ, layers=4)[1]) == 2
    n, steps = LY.chunk_circuit(circ, layers=3)
    assert [len(LY.sublayers(s)) for s in steps] == [3, 3]
    # a measurement still closes a chunk
    circ2 = C.brickwork(6, 6, 0.5, 2)
    n, steps = LY.chunk_circuit(circ2, layers=4)
    for st in steps:
        if isinstance(st, list):
            assert len(LY.sublayers(st)) <= 4


@pytest.mark.parametrize("layers", [2, 3, 4])
def test_multi_layer_exact_regime_equals_statevector(layers):
    # chi large enough for every cut: the multi-layer compression is exact, the outcomes are
    # those of the state-vector oracle and the final state equals its state
    circ = C.brickwork(8, 7, 0.15, 21)
    for shot in (0, 3):
        ref = SV.run_single_path(circ, 1, shot)
        got = D.run_single_path(circ, D.Params(chi_max=16, layers=layers), 1, shot)
        assert got.outcomes == ref.outcomes
        v = M.to_dense(got.mps).reshape(-1)
        assert abs(abs(np.vdot(v, ref.psi.reshape(-1))) ** 2 - 1) < 1e-10
        assert abs(got.F - 1) < 1e-10


def test_multi_layer_truncated_fidelity_is_monotone():
    rng = np.random.default_rng(9)
    n = 8
    A = random_mps(rng, n, 8)
    circ = C.brickwork(n, 3, 0.0, 5)
    chunk = list(circ.ops)
    sub, _ = LY.chunk_sublayer_blocks(n, chunk, np.zeros(1, dtype=np.int64))
    W = LY.compose_mpo([LY.blocks_mpo(n, b) for b in sub])
    target = LY.chunk_unitary_dense(n, W) @ M.to_dense(A).reshape(-1)
    prev = 0.0
    for s in (1, 2, 3, 4):
        B, info = M.compress(A.copy(), sub, W, 4, 1e-10, s, skip_exact=False)
        v = M.to_dense(B).reshape(-1)
        f_true = abs(np.vdot(v, target)) ** 2
        assert abs(info.f - f_true) < 1e-10 and info.f <= 1 + 1e-12
        assert info.f >= prev - 1e-12
        prev = info.f
    assert prev < 1 - 1e-3


def _brute_site_env(B, psi, j):
    """The optimal local tensor at site j, from dense vectors only: <B with site j left
    out | psi> (B centred at j, so its left and right parts are isometries)."""
    n = B.n
    left = np.ones((1, 1), dtype=np.complex128)
    for k in range(j):
        t = B.T[k]
        left = np.einsum("xa,asb->xsb", left, t).reshape(-1, t.shape[2])
    right = np.ones((1, 1), dtype=np.complex128)
    for k in range(n - 1, j, -1):
        t = B.T[k]
        right = np.einsum("asb,by->asy", t, right).reshape(t.shape[0], -1)
    P = psi.reshape(left.shape[0], 2, right.shape[1])
    return np.einsum("xb,xsy,cy->bsc", left.conj(), P, right.conj())


@pytest.mark.parametrize("seed,layers", [(1, 1), (2, 1), (3, 2)])
def test_converged_sweeps_are_stationary(seed, layers):
    # Sec. "Simulating unitary quantum circuits with DMRG": each one-site update replaces the
    # site by F/||F||, the optimum for the rest of the bra held fixed.  Once the sweeps have
    # converged in the truncated regime the bra is a fixed point: at every site the optimal
    # local tensor, computed here by brute force from the dense target state (none of the
    # oracle's environment sums), is the site itself up to a phase and its norm^2 is f.
    rng = np.random.default_rng(seed)
    n = 8
    A = random_mps(rng, n, 3)
    if layers == 1:
        chunk = _layer_blocks(rng, n, seed % 2)
        W = LY.blocks_mpo(n, chunk)
    else:
        ops = list(C.brickwork(n, layers, 0.0, 30 + seed).ops)
        chunk, _ = LY.chunk_sublayer_blocks(n, ops, np.zeros(1, dtype=np.int64))
        W = LY.compose_mpo([LY.blocks_mpo(n, b) for b in chunk])
    psi = LY.chunk_unitary_dense(n, W) @ dense(A)
    B, info = M.compress(A.copy(), chunk, W, 3, 0.0, 60, skip_exact=False)
    assert info.f < 1 - 1e-4  # truncated
    for j in range(n):
        Bc = B.copy()
        M.move_centre(Bc, j)
        F = _brute_site_env(Bc, psi, j)
        nf = np.vdot(F, F).real
        assert abs(nf - info.f) < 1e-10
        assert 1 - abs(np.vdot(F / np.sqrt(nf), Bc.T[j])) < 1e-10
