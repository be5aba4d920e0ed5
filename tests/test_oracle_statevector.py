"""Pins of the state-vector oracle (O1) and the Philox generator against values the paper
prints, closed forms, published known answers and brute force."""
import itertools

import numpy as np
import pytest

import circuits as C
from conftest import read_golden_kv, read_golden_rows
from oracle import philox, statevector as SV


# ----------------------------------------------------------------------------- Philox


def test_philox_known_answers():
    rows = read_golden_rows("philox_kat.txt")
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        ctr, key, out = vals[0:4], vals[4:6], vals[6:10]
        assert list(philox.philox4x32_10(ctr, key)) == out


def test_uniform_range_and_mean():
    us = np.array([philox.uniform(7, s, o) for s in range(200) for o in range(10)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert abs(us.mean() - 0.5) < 0.02
    # different (shot, ordinal) give different draws
    assert len(set(us.tolist())) == len(us)


# ----------------------------------------------------------------------------- gates


def _kron_operator(n, qubits, mat):
    """Brute force: the full 2^n x 2^n operator of ``mat`` on ``qubits`` by enumerating
    basis states (independent of tensordot/moveaxis)."""
    k = len(qubits)
    dim = 2 ** n
    op = np.zeros((dim, dim), dtype=np.complex128)
    for col in range(dim):
        bits = [(col >> (n - 1 - q)) & 1 for q in range(n)]
        sub_in = 0
        for q in qubits:
            sub_in = 2 * sub_in + bits[q]
        for sub_out in range(2 ** k):
            ob = list(bits)
            for i, q in enumerate(qubits):
                ob[q] = (sub_out >> (k - 1 - i)) & 1
            row = 0
            for b in ob:
                row = 2 * row + b
            op[row, col] += mat[sub_out, sub_in]
    return op


@pytest.mark.parametrize("n", [2, 3, 5])
def test_apply_gate_matches_brute_force(n):
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(2 ** n) + 1j * rng.standard_normal(2 ** n)
    psi /= np.linalg.norm(psi)
    for qubits in itertools.permutations(range(n), 2):
        if len(qubits) == 2 and n > 3 and abs(qubits[0] - qubits[1]) > 2:
            continue
        U = C.haar_unitary(rng, 4)
        ref = _kron_operator(n, qubits, U) @ psi
        got = SV.apply_gate(psi.reshape((2,) * n), qubits, U).reshape(-1)
        np.testing.assert_allclose(got, ref, atol=1e-13)
    for q in range(n):
        U = C.haar_unitary(rng, 2)
        ref = _kron_operator(n, (q,), U) @ psi
        got = SV.apply_gate(psi.reshape((2,) * n), (q,), U).reshape(-1)
        np.testing.assert_allclose(got, ref, atol=1e-13)


def test_bell_state_closed_form():
    psi = SV.zero_state(2)
    psi = SV.apply_gate(psi, (0,), C.H)
    psi = SV.apply_gate(psi, (0, 1), C.CNOT)
    np.testing.assert_allclose(psi.reshape(-1), np.array([1, 0, 0, 1]) / np.sqrt(2), atol=1e-15)
    r0, r1 = SV.probabilities(psi, 1)
    assert abs(r0 - 0.5) < 1e-15 and abs(r1 - 0.5) < 1e-15
    post = SV.project(psi, 1, 1, r1)
    np.testing.assert_allclose(post.reshape(-1), [0, 0, 0, 1], atol=1e-15)


def test_conditions():
    c = np.array([1, 0, 1, 1])
    assert SV.cond_holds(C.Cond((0,), "xor", 1), c)
    assert not SV.cond_holds(C.Cond((1,), "xor", 1), c)
    assert SV.cond_holds(C.Cond((0, 2), "xor", 0), c)          # 1 ^ 1 = 0
    assert SV.cond_holds(C.Cond((0, 2, 3), "and", 1), c)
    assert not SV.cond_holds(C.Cond((0, 1), "and", 1), c)
    assert SV.cond_holds(None, c)


# ----------------------------------------------------------------------------- teleport


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_teleport_four_paths_and_state(seed):
    g = read_golden_kv("teleport_paper.txt")
    circ = C.teleport(seed)
    branches = SV.run_multi_path(circ)
    assert sorted(tuple(b.path) for b in branches) == [(0, 0), (0, 1), (1, 0), (1, 1)]
    inp = circ.meta["input"]
    for b in branches:
        assert abs(b.p - g["path_prob"]) < 1e-12
        # Bob's qubit (q2) carries the input; Alice's qubits hold the outcomes
        bob = b.psi[b.path[0], b.path[1], :]
        assert abs(abs(np.vdot(bob, inp)) ** 2 - 1.0) < 1e-12


def test_teleport_bob_measurement_paper_values():
    g = read_golden_kv("teleport_paper.txt")
    amps = (complex(g["input_re0"], g["input_im0"]), complex(g["input_re1"], g["input_im1"]))
    circ = C.teleport(amplitudes=amps, bob_measure=True)
    branches = SV.run_multi_path(circ)
    assert len(branches) == 8
    tol = g["printed_abs_tol"]
    for b in branches:
        want = g["path_p_bob0"] if b.path[2] == 0 else g["path_p_bob1"]
        assert abs(b.p - want) < tol
    p_bob0 = sum(b.p for b in branches if b.path[2] == 0)
    assert abs(p_bob0 - g["bob_p0"]) < tol
    assert abs(sum(b.p for b in branches) - 1.0) < 1e-12


# ----------------------------------------------------------------------------- GHZ


def _ghz_ok(psi, n):
    data = list(range(0, n, 2))
    want = np.zeros((2,) * n, dtype=np.complex128)
    idx0 = [0] * n
    idx1 = [0] * n
    for d in data:
        idx1[d] = 1
    want[tuple(idx0)] = want[tuple(idx1)] = 1 / np.sqrt(2)
    return abs(abs(np.vdot(want, psi)) ** 2 - 1.0) < 1e-12


@pytest.mark.parametrize("row", read_golden_rows("ghz_paper.txt")[:4])
def test_ghz_paths_equiprobable_and_state(row):
    n, r, npaths = (int(x) for x in row)
    circ = C.ghz_dynamic(n)
    assert circ.meta["r"] == r
    branches = SV.run_multi_path(circ)
    assert len(branches) == npaths
    for b in branches:
        assert abs(b.p - 2.0 ** -r) < 1e-13
        assert _ghz_ok(b.psi, n)


def test_ghz_even_layout_idle_ancilla():
    circ = C.ghz_dynamic(10)  # last ancilla idle: deterministic 0, r = 4
    branches = SV.run_multi_path(circ)
    assert len(branches) == 16
    for b in branches:
        assert b.c[4] == 0 and _ghz_ok(b.psi, 10)


@pytest.mark.parametrize("M", [1, 3, 8, 16, 64])
def test_ghz_topm_tvd_is_discarded_mass(M):
    n = 9
    r = 4
    circ = C.ghz_dynamic(n)
    kept = SV.run_multi_path(circ, M=M)
    ideal = {k: 2.0 ** -r for k in itertools.product((0, 1), repeat=r)}
    # the simulated distribution is the retained branches' p normalised by their sum
    z = sum(b.p for b in kept)
    sim = {}
    for b in kept:
        key = tuple(b.path[:r])
        sim[key] = sim.get(key, 0.0) + b.p / z
    d = SV.tvd(ideal, sim)
    discarded = 1.0 - sum(b.p for b in kept)
    assert abs(d - discarded) < 1e-12
    if M >= 2 ** r:
        assert d < 1e-12
    else:
        assert len(kept) == M and d > 0


def test_topk_selection_ties_and_order():
    ps = [0.1, 0.3, 0.3, 0.05, 0.25]
    assert SV.topk_select(ps, 3) == [1, 2, 4]
    assert SV.topk_select(ps, 1) == [1]            # tie 0.3/0.3: earlier wins
    assert SV.topk_select([0.5, 0.5 * (1 + 1e-9), 0.2], 1) == [0]  # within tolerance: tie
    assert SV.topk_select([0.5, 0.5 * (1 + 1e-3), 0.2], 1) == [1]  # beyond: larger wins


# ----------------------------------------------------------------------------- invariants


@pytest.mark.parametrize("seed", [1, 2])
def test_branch_probabilities_sum_to_one(seed):
    circ = C.brickwork(6, 5, 0.3, seed)
    branches = SV.run_multi_path(circ)
    assert abs(sum(b.p for b in branches) - 1.0) < 1e-12
    for b in branches:
        assert abs(np.linalg.norm(b.psi) - 1.0) < 1e-12


def test_single_path_matches_multi_path_branch():
    circ = C.brickwork(6, 4, 0.3, 3)
    branches = {tuple(b.path): b for b in SV.run_multi_path(circ)}
    for shot in range(5):
        r = SV.run_single_path(circ, 11, shot)
        b = branches[tuple(r.outcomes)]
        assert abs(r.p - b.p) < 1e-12
        assert abs(abs(np.vdot(r.psi, b.psi)) - 1) < 1e-12


def test_single_path_sampling_converges():
    circ = C.teleport(5)
    counts = {}
    N = 2000
    for shot in range(N):
        r = SV.run_single_path(circ, 3, shot)
        counts[tuple(r.outcomes)] = counts.get(tuple(r.outcomes), 0) + 1
    emp = {k: v / N for k, v in counts.items()}
    ideal = {k: 0.25 for k in itertools.product((0, 1), repeat=2)}
    # chi-square with 3 degrees of freedom at the 99.9% level is 16.27
    chi2 = sum((counts.get(k, 0) - N * 0.25) ** 2 / (N * 0.25) for k in ideal)
    assert chi2 < 16.27
    assert SV.tvd(ideal, emp) < 0.05


def test_topk_non_degenerate_values_near_the_tie_scale():
    # keys round(p / (1e-5 p_max)): values more than a key unit apart are ordered by size
    # whatever their list order; values inside one unit share a key and keep list order.
    # 1e-5 is the probability tolerance of the accuracy contract, so two p values the
    # contract cannot tell apart are never ordered by their rounding.
    pmax = 0.2
    ps = [pmax * (1 - 6e-5), pmax, pmax * (1 - 3e-5), 0.1]
    assert SV.topk_select(ps, 1) == [1]
    assert SV.topk_select(ps, 2) == [1, 2]
    assert SV.topk_select(ps, 3) == [0, 1, 2]
    assert SV.topk_select([pmax * (1 - 3e-5), pmax * (1 - 6e-5), pmax], 2) == [0, 2]
    base = pmax * (1 - 10e-5)  # key 99990, a whole unit below its neighbours
    assert SV.topk_select([base, base * (1 + 2e-7), pmax], 2) == [0, 2]
    assert SV.topk_select([base * (1 + 2e-7), base, pmax], 2) == [0, 2]
    assert SV.topk_select([base, base * (1 + 2.5e-5), pmax], 2) == [1, 2]


def test_general_boolean_conditions_by_enumeration():
    # Sec. "Classically controlled operations": phi is a Boolean function of the register.
    # Truth tables of three bits (index = c_b0 + 2 c_b1 + 4 c_b2 over the bits in ascending
    # order) against the functions written out, on every register value
    import itertools
    cases = {0b11101000: lambda a, b, c: int(a + b + c >= 2),   # majority
             0b11111110: lambda a, b, c: int(a or b or c),
             0b10010110: lambda a, b, c: a ^ b ^ c,
             0b10000000: lambda a, b, c: int(a and b and c),
             0b00100100: lambda a, b, c: int((a == 0 and b == 1 and c == 0) or
                                             (a == 1 and b == 0 and c == 1))}
    for table, fn in cases.items():
        for bits in itertools.product([0, 1], repeat=3):
            creg = np.array([0, bits[0], 0, bits[1], bits[2]], dtype=np.int64)
            # listed in any order; the index reads them in ascending bit order (1, 3, 4)
            cond = C.Cond((4, 1, 3), "table", table)
            assert SV.cond_holds(cond, creg) == bool(fn(*bits))
            assert SV.cond_holds(C.Cond((1, 3, 4), "or", 1), creg) == any(bits)
            assert SV.cond_holds(C.Cond((1, 3, 4), "or", 0), creg) == (not any(bits))


def test_adaptive_pruning_selection_and_ensemble():
    # prune_select: the top-M rule, then branches below p_min dropped except the first of
    # the key order; by brute force on a list
    ps = [0.30, 0.01, 0.20, 0.004, 0.20, 0.09]
    assert SV.prune_select(ps, None, 0.05) == [0, 2, 4, 5]
    assert SV.prune_select(ps, 3, 0.05) == [0, 2, 4]
    assert SV.prune_select(ps, None, 0.5) == [0]          # never empty: the first stays
    assert SV.prune_select(ps, None, 0.0) == list(range(6))
    # the pruned ensemble is the full one with every branch below p_min removed at each
    # measurement: each survivor has the same p and register as in the unpruned run, and
    # each unpruned leaf whose prefixes all stayed above p_min survives
    circ = C.brickwork(6, 5, 0.4, 8)
    full = SV.run_multi_path(circ)
    pruned = SV.run_multi_path(circ, p_min=0.02)
    byp = {tuple(b.path): b.p for b in full}
    assert 0 < len(pruned) < len(full)
    for b in pruned:
        assert abs(byp[tuple(b.path)] - b.p) < 1e-12
        assert b.p >= 0.02 or len(pruned) == 1
    # a leaf survives iff every prefix probability of its path is >= p_min; recompute the
    # prefix probabilities from the full run's branch list at each measurement depth
    def prefix_p(path):
        return sum(bb.p for bb in full if tuple(bb.path[:len(path)]) == tuple(path))
    for b in full:
        ok = all(prefix_p(b.path[:d]) >= 0.02 for d in range(1, len(b.path) + 1))
        assert ok == (tuple(b.path) in {tuple(x.path) for x in pruned})
