"""Parity of the CUDA path (through the libdcs C ABI) with the FP64 oracle.

Bars (tolerances of the accuracy contract): measurement outcomes bit-exact except draws
the oracle flags (|u - p_0| < 1e-6); probabilities within 1e-5 absolute; state fidelity
|<psi_gpu|psi_oracle>|^2 >= 1 - 1e-6 (gauge-invariant: MPS tensors are compared only
through the state they represent); the estimated fidelity F within ``f_tol``."""
import numpy as np
import pytest

import circuits as C
from oracle import drivers as D, mps as OM, statevector as SV

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P_TOL = 1e-5
STATE_TOL = 1e-6
# The estimated fidelity F = prod f has no tolerance in the accuracy contract.  Each f is
# the end of an FP32 chain of n site updates, so its rounding error grows like n u
# (u = 2^-24); the bound allows 8 u per site update plus 1e-5.
U32 = 2.0 ** -24


def f_tol(n_sites, n_compressions):
    return 1e-5 + 8 * U32 * n_sites * max(1, n_compressions)


def _sim(n, chi, slots, ncb, tol=1e-10, sweeps=2, seed=1, path=0, prec=0):
    from paper_2609_26516_b300 import Simulator
    return Simulator(n, chi, slots, max(ncb, 1), tol=tol, sweeps=sweeps, seed=seed,
                     kernel_path=path, precision=prec)


def _overlap(A, B):
    """<A|B> of two MPS by transfer matrices (host FP64, any n)."""
    E = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        # E'[u, v] = sum_{x, s, y} conj(a[x, s, u]) E[x, y] b[y, s, v], as two products
        t = np.tensordot(E, np.asarray(b, dtype=np.complex128), axes=(1, 0))
        E = np.tensordot(np.conj(np.asarray(a, dtype=np.complex128)), t, axes=([0, 1], [0, 1]))
    return E[0, 0]


def _state_fid(sim, pos, ref_mps):
    _, _, T = sim.export_mps(pos)
    ab = _overlap(T, ref_mps.T)
    aa = _overlap(T, T).real
    bb = _overlap(ref_mps.T, ref_mps.T).real
    return abs(ab) ** 2 / (aa * bb)


def _single_path_parity(circ, chi, shots, check_shots, seed=1, tol=1e-10, sweeps=2,
                        state_check=True, path=0, prec=0, bond_slack=0):
    sim = _sim(circ.n_qubits, chi, shots, circ.n_cbits, tol, sweeps, seed, path, prec)
    sim.init_state(shots)
    sim.run_circuit(circ)
    res = sim.results()
    assert res["n_active"] == shots
    prm = D.Params(chi_max=chi, tol=tol, sweeps=sweeps)
    compared = 0
    for s in check_shots:
        ref = D.run_single_path(circ, prm, seed, s)
        if ref.flagged:
            continue
        compared += 1
        assert res["bits"][s].tolist() == [int(x) for x in ref.c], f"shot {s}"
        if state_check:
            bonds, _, _ = sim.export_mps(s)
            if bond_slack == 0:
                assert list(bonds) == ref.mps.bonds(), f"shot {s}: bond dimensions differ"
            else:  # ranks decided at the tolerance edge may differ by a few (FP32 vs FP64)
                assert max(abs(int(x) - y) for x, y in zip(bonds, ref.mps.bonds())) <= bond_slack
            assert _state_fid(sim, s, ref.mps) >= 1 - STATE_TOL
        assert abs(res["p"][s] - ref.p) < P_TOL
        assert abs(res["F"][s] - ref.F) < f_tol(circ.n_qubits, len(ref.fids))
    assert compared >= len(check_shots) // 2
    return sim, res


def test_teleport_single_path_1000_shots():
    circ = C.teleport(1)
    sim, res = _single_path_parity(circ, 4, 1000, list(range(0, 1000, 37)))
    # the four paths at 1/4 each: 1000 shots land within 5 sigma
    paths = res["bits"][:, 0] * 2 + res["bits"][:, 1]
    counts = np.bincount(paths, minlength=4)
    assert np.all(np.abs(counts - 250) < 5 * np.sqrt(1000 * 0.25 * 0.75))
    assert np.all(np.abs(res["p"] - 0.25) < P_TOL)


@pytest.mark.parametrize("n", [9, 20])
def test_ghz_single_path_small(n):
    circ = C.ghz_dynamic(n)
    _single_path_parity(circ, 8, 64, list(range(0, 64, 9)))


def test_ghz64_full_config_sampled_shots():
    circ = C.ghz_dynamic(64)
    shots = 10000
    sim = _sim(64, 8, shots, circ.n_cbits)
    sim.init_state(shots)
    sim.run_circuit(circ)
    res = sim.results()
    prm = D.Params(chi_max=8)
    r = circ.meta["r"]
    assert np.all(np.abs(res["p"] - 2.0 ** -r) < P_TOL * 2.0 ** -r)
    assert np.all(np.abs(res["F"] - 1.0) < f_tol(64, 4))
    for s in (0, 4999, 9999):
        ref = D.run_single_path(circ, prm, 1, s)
        assert res["bits"][s].tolist() == [int(x) for x in ref.c]
        assert _state_fid(sim, s, ref.mps) >= 1 - STATE_TOL


def test_odd_slot_counts_every_shot():
    # odd slot counts on the one-warp (4-wide tile) path: every shot against the oracle
    _single_path_parity(C.ghz_dynamic(12), 8, 37, list(range(37)))
    _single_path_parity(C.teleport(5), 4, 33, list(range(33)))


def test_shot_offset_reproduces_the_same_shots():
    # the sampler is keyed by the global shot index shot0 + slot, so a batch started at
    # shot0 = 20 gives shots 20.. of a batch started at 0 (how shots are split over ranks)
    circ = C.ghz_dynamic(12)
    a = _sim(12, 8, 64, circ.n_cbits)
    a.init_state(64)
    a.run_circuit(circ)
    ra = a.results()
    b = _sim(12, 8, 24, circ.n_cbits)
    b.init_state(24, shot0=20)
    b.run_circuit(circ)
    rb = b.results()
    assert rb["n_active"] == 24
    np.testing.assert_array_equal(rb["bits"], ra["bits"][20:44])
    np.testing.assert_allclose(rb["p"], ra["p"][20:44], rtol=0, atol=1e-12)
    np.testing.assert_allclose(rb["F"], ra["F"][20:44], rtol=0, atol=1e-12)
    prm = D.Params(chi_max=8)
    for i in (0, 7, 23):
        ref = D.run_single_path(circ, prm, 1, 20 + i)
        if not ref.flagged:
            assert rb["bits"][i].tolist() == [int(x) for x in ref.c]


# tol = 0 is not a parity case: FP32 rounding leaves singular values ~1e-7 where FP64 has
# exact zeros, so the two sides would keep different (noise) bond directions.
@pytest.mark.parametrize("chi,tol", [(8, 1e-10), (5, 1e-10), (32, 1e-12)])
def test_brickwork_single_path(chi, tol):
    circ = C.brickwork(10, 8, 0.2, 3)
    _single_path_parity(circ, chi, 16, list(range(16)), tol=tol)


def test_brickwork_three_sweeps_and_ragged():
    circ = C.brickwork(7, 6, 0.25, 11)
    _single_path_parity(circ, 3, 8, list(range(8)), sweeps=3)


def test_multi_path_ghz_topm():
    circ = C.ghz_dynamic(9)
    for M in (4, 16):
        sim = _sim(9, 8, 2 * M, circ.n_cbits)
        sim.init_state(1, multipath=True)
        sim.run_circuit(circ, max_branches=M)
        res = sim.results()
        ref = D.run_multi_path(circ, D.Params(chi_max=8), M=M)
        assert res["n_active"] == len(ref)
        for i, b in enumerate(ref):
            assert res["bits"][i].tolist() == [int(x) for x in b.c]
            assert abs(res["p"][i] - b.p) < P_TOL
            assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL


def test_multi_path_brickwork_uneven():
    circ = C.brickwork(8, 6, 0.2, 5)
    M = 8
    sim = _sim(8, 8, 2 * M, circ.n_cbits)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    ref = D.run_multi_path(circ, D.Params(chi_max=8), M=M)
    assert res["n_active"] == len(ref)
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c]
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
        assert abs(res["p"][i] - b.p) < P_TOL
        assert abs(res["F"][i] - b.F) < f_tol(8, 6)


def test_teleport_multi_path_pool_exhaustion():
    circ = C.teleport(2)
    from paper_2609_26516_b300 import DCSError
    sim = _sim(3, 4, 2, circ.n_cbits)  # four paths do not fit in two slots
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ)
    with pytest.raises(DCSError):
        sim.results()


def test_measure_prob_and_forced_collapse():
    circ = C.brickwork(6, 4, 0.0, 2)
    sim = _sim(6, 8, 4, 2)
    sim.init_state(4)
    sim.run_circuit(circ)
    p0 = sim.measure_prob(3).cpu().numpy()
    ref = D.run_single_path(circ, D.Params(chi_max=8), 1, 0)
    r0, r1 = OM.measure_probs(ref.mps, 3)
    assert np.all(np.abs(p0 - r0 / (r0 + r1)) < P_TOL)
    sim.collapse(3, 0, [0, 1, 0, 1])
    res = sim.results()
    assert res["bits"][:, 0].tolist() == [0, 1, 0, 1]
    for s, m in enumerate([0, 1, 0, 1]):
        mm = ref.mps.copy()
        OM.measure_probs(mm, 3)
        OM.collapse(mm, 3, m, r0 if m == 0 else r1)
        assert abs(res["p"][s] - (r0 if m == 0 else r1) / (r0 + r1)) < P_TOL
        assert _state_fid(sim, s, mm) >= 1 - STATE_TOL


def test_empty_chunk_leaves_slot_unchanged():
    # X on q0 conditioned on c0 == 1; no slot has c0 set, so nothing is compressed
    g = [C.Gate((0,), C.X, cond=C.Cond((0,), "xor", 1))]
    sim = _sim(4, 4, 3, 1)
    sim.init_state(3)
    fid = torch.zeros(3, dtype=torch.float64, device="cuda")
    sim.apply_layer(g, fid)
    assert torch.all(fid == 1.0)
    res = sim.results()
    assert np.all(res["F"] == 1.0)
    _, _, T = sim.export_mps(0)
    assert abs(T[0][0, 0, 0] - 1) < 1e-7


def test_export_import_round_trip():
    circ = C.brickwork(6, 5, 0.0, 4)
    sim = _sim(6, 8, 2, 1)
    sim.init_state(2)
    sim.run_circuit(circ)
    b, c, T = sim.export_mps(0)
    sim.import_mps(1, T, c)
    b2, c2, T2 = sim.export_mps(1)
    assert list(b) == list(b2) and c == c2
    for x, y in zip(T, T2):
        assert np.array_equal(x, y)


def test_single_qubit_chain_and_launch_count():
    # n = 1: a lone qubit, Hadamard then a measurement
    circ = C.Circuit(1, 1, [C.Gate((0,), C.H), C.Measure(0, 0)])
    sim = _sim(1, 4, 256, 1)
    sim.init_state(256)
    before = sim.launches
    sim.run_circuit(circ)
    res = sim.results()
    assert sim.launches - before == 2
    assert np.all(np.abs(res["p"] - 0.5) < P_TOL)
    for s in range(0, 256, 17):
        ref = SV.run_single_path(circ, 1, s)
        assert res["bits"][s, 0] == ref.outcomes[0]


# ----------------------------------------------------------------------------- global tiles
# kernel_path=2 forces the large-bond kernels (tiles in a per-slot global work area, tiled
# GEMM contractions) so they are checked on cases the oracle finishes in seconds.


@pytest.mark.parametrize("chi,sweeps", [(8, 2), (16, 3)])
def test_global_tiles_brickwork(chi, sweeps):
    circ = C.brickwork(10, 8, 0.2, 3)
    _single_path_parity(circ, chi, 8, list(range(8)), sweeps=sweeps, path=2)


def test_global_tiles_ghz_and_teleport():
    _single_path_parity(C.ghz_dynamic(20), 8, 16, list(range(0, 16, 5)), path=2)
    _single_path_parity(C.teleport(4), 4, 64, list(range(0, 64, 13)), path=2)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp32", "tf32x3", "bf16x3"])
def test_global_tiles_ragged_chi_above_shared_limit(prec):
    # chi_max = 40 is above the shared-memory tiles and not a multiple of the GEMM tile
    circ = C.brickwork(14, 16, 0.02, 9)  # the middle bonds reach 40 and are truncated
    _single_path_parity(circ, 40, 3, [0, 1, 2], prec=prec)


def test_global_tiles_tensor_cores_at_chi_96():
    # bonds up to 96: the environment and site products are large enough for the tensor
    # cores (M, N >= 64) on the TF32x3 path
    circ = C.brickwork(16, 14, 0.0, 21)
    _single_path_parity(circ, 96, 2, [0, 1], prec=1)


@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp32", "tf32x3", "bf16x3"])
def test_global_tiles_blocked_qr_at_chi_128(prec):
    # middle bonds saturate at 128 and are truncated: the sweeps' QRs of 256 x 128 and
    # 128 x 128 matrices take the blocked (panel + GEMM) form
    circ = C.brickwork(16, 14, 0.0, 21)
    _single_path_parity(circ, 128, 2, [0, 1], prec=prec)


def test_global_tiles_multi_path():
    circ = C.brickwork(8, 6, 0.2, 5)
    M = 8
    sim = _sim(8, 8, 2 * M, circ.n_cbits, path=2)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    ref = D.run_multi_path(circ, D.Params(chi_max=8), M=M)
    assert res["n_active"] == len(ref)
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c]
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
        assert abs(res["p"][i] - b.p) < P_TOL


# ---- the large-bond workload shapes at reduced depth (the oracle computes them exactly)

def test_brickwork_n40_chi256_exact_layers():
    # n = 40 random dynamic brickwork with chi_max = 256 (the large-bond slot capacity), the
    # first 10 layers: bonds stay below chi_max, so every step is exact on both sides
    circ = C.brickwork(40, 10, 0.1, 3)
    _single_path_parity(circ, 256, 2, [0, 1])


def test_brickwork_n64_chi1024_first_8_layers():
    # n = 64, chi_max = 1024 (the largest capacity), measurement rate 0.02: the first 8
    # layers, checked against the oracle shot by shot; middle bonds reach about 160.  At
    # these sizes a singular value can sit at the 1e-10 truncation edge, where the FP32 and
    # FP64 rank decisions differ by one; the state itself must still agree to 1e-6.
    circ = C.brickwork(64, 8, 0.02, 5)
    sim, _ = _single_path_parity(circ, 1024, 1, [0], bond_slack=2)
    bonds, _, _ = sim.export_mps(0)
    assert max(bonds) >= 128


def test_multi_path_brickwork_large_bonds():
    # multi-path ensemble on the large-bond kernels (chi_max = 48 > the shared-memory
    # tiles): n = 12, top-M with M = 16
    circ = C.brickwork(12, 10, 0.08, 7)
    M = 16
    sim = _sim(12, 48, 2 * M, circ.n_cbits)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    ref = D.run_multi_path(circ, D.Params(chi_max=48), M=M)
    assert res["n_active"] == len(ref) > 1
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c]
        assert abs(res["p"][i] - b.p) < P_TOL
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL


# ---- edge cases: the largest chain, a single qubit, the smallest bond cap

def test_ghz_max_qubits_128():
    # n = 128 (the library's maximum), 64 data qubits and 63 random outcomes per shot
    circ = C.ghz_dynamic(128)
    shots = 256
    sim = _sim(128, 8, shots, circ.n_cbits)
    sim.init_state(shots)
    sim.run_circuit(circ)
    res = sim.results()
    r = circ.meta["r"]
    assert np.all(np.abs(res["p"] - 2.0 ** -r) < P_TOL * 2.0 ** -r)
    prm = D.Params(chi_max=8)
    for s in (0, 255):
        ref = D.run_single_path(circ, prm, 1, s)
        assert res["bits"][s].tolist() == [int(x) for x in ref.c]
        assert _state_fid(sim, s, ref.mps) >= 1 - STATE_TOL


def test_single_qubit_dynamic_circuit():
    # n = 1: H, measure, X conditioned on the outcome, measure again (always 0)
    circ = C.Circuit(1, 2, [C.Gate((0,), C.H), C.Measure(0, 0),
                            C.Gate((0,), C.X, cond=C.Cond((0,), "xor", 1)), C.Measure(0, 1)])
    _, res = _single_path_parity(circ, 1, 64, list(range(64)))
    assert np.all(res["bits"][:, 1] == 0)
    assert 10 < int(res["bits"][:, 0].sum()) < 54


def test_bond_cap_one():
    # chi_max = 1: every entangling layer is truncated to a product state
    circ = C.brickwork(6, 4, 0.3, 2)
    _, res = _single_path_parity(circ, 1, 8, list(range(8)))
    assert np.all(res["F"] < 1.0)


# ---- general Boolean conditions and the final measurement of Bob's qubit

def test_general_boolean_conditions():
    # X on q3 iff majority(c0, c1, c2) (a truth-table condition), X on q4 iff c0 OR c2;
    # then q3 and q4 are measured: their bits must equal those functions on every shot
    ops = [C.Gate((q,), C.H) for q in range(3)]
    ops += [C.Measure(q, q) for q in range(3)]
    ops += [C.Gate((3,), C.X, cond=C.Cond((0, 1, 2), "table", 0b11101000)),
            C.Gate((4,), C.X, cond=C.Cond((0, 2), "or", 1)),
            C.Gate((2, 3), C.CNOT), C.Gate((2, 3), C.CNOT)]  # identity pair: a two-qubit block
    ops += [C.Measure(3, 3), C.Measure(4, 4)]
    circ = C.Circuit(5, 5, ops)
    _, res = _single_path_parity(circ, 4, 256, list(range(0, 256, 17)))
    b = res["bits"].astype(int)
    maj = (b[:, 0] + b[:, 1] + b[:, 2] >= 2).astype(int)
    assert np.array_equal(b[:, 3], maj)
    assert np.array_equal(b[:, 4], b[:, 0] | b[:, 2])
    assert 0 < maj.sum() < 256


def test_teleport_bob_measurement_eight_paths():
    # multi-path teleportation with Bob's final measurement (Sec. "Quantum teleportation
    # protocol"): eight paths, p = 0.25 Pr(m_Bob), Pr(0) ~ 0.37 for the printed input state
    from conftest import read_golden_kv
    g = read_golden_kv("teleport_paper.txt")
    amps = (complex(g["input_re0"], g["input_im0"]), complex(g["input_re1"], g["input_im1"]))
    circ = C.teleport(amplitudes=amps, bob_measure=True)
    sim = _sim(3, 4, 16, circ.n_cbits)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ)
    res = sim.results()
    ref = SV.run_multi_path(circ)
    assert res["n_active"] == len(ref) == 8
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.path]
        assert abs(res["p"][i] - b.p) < P_TOL
        want = g["path_p_bob0"] if b.path[2] == 0 else g["path_p_bob1"]
        assert abs(res["p"][i] - want) < g["printed_abs_tol"]
    p0 = sum(res["p"][i] for i in range(8) if res["bits"][i][2] == 0)
    assert abs(p0 - g["bob_p0"]) < g["printed_abs_tol"]


def test_multi_path_adaptive_pruning():
    # branches whose path probability falls below p_min are dropped after each measurement
    # (beyond top-M); branch by branch against the oracle's ensemble with the same rule
    circ = C.brickwork(10, 8, 0.25, 8)
    p_min = 2e-3
    ref = D.run_multi_path(circ, D.Params(chi_max=16), M=32, p_min=p_min)
    full = D.run_multi_path(circ, D.Params(chi_max=16), M=32)
    sim = _sim(10, 16, 64, circ.n_cbits)
    sim.set_pruning(p_min)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=32)
    res = sim.results()
    assert res["n_active"] == len(ref) < len(full)
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c]
        assert abs(res["p"][i] - b.p) < P_TOL
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
    assert np.all(res["p"] >= p_min) or res["n_active"] == 1


def test_final_register_sampling_distribution():
    # every qubit measured at the end of a random circuit: per-shot outcomes bit-exact with
    # the oracle, and the empirical distribution of 8192 shots close to the exact one
    n = 6
    base = C.brickwork(n, 6, 0.0, 12)
    circ = C.Circuit(n, n, base.ops + [C.Measure(q, q) for q in range(n)])
    shots = 8192
    _, res = _single_path_parity(circ, 8, shots, list(range(0, shots, 1024)))
    psi = SV.run_single_path(base, 1, 0).psi.reshape(-1)
    exact = np.abs(psi) ** 2
    idx = (res["bits"].astype(np.int64) * (1 << np.arange(n - 1, -1, -1))).sum(axis=1)
    emp = np.bincount(idx, minlength=2 ** n) / shots
    assert 0.5 * np.abs(emp - exact).sum() < 0.06
