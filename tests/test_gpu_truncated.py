"""Parity with the FP64 oracle in the truncated regime, at the large-bond workloads' bond
sizes (chi_max = 256 single-path, chi_max = 64 and 128 multi-path with M = 64 and pruning).

Per-step parity: the oracle's state after a saturated layer is imported into the GPU (rounded
to complex64) and both run the same compression step (Sec. "Simulating unitary quantum
circuits with DMRG") on it; the results must agree to the accuracy contract (state fidelity
>= 1 - 1e-6, partial fidelity within ``f_tol``).  This isolates one step from the
amplification of rounding differences over many truncated layers.  End-to-end parity runs
whole circuits shot by shot (single-path, Alg. 1) and branch by branch (multi-path, Alg. 2)."""
import functools

import numpy as np
import pytest

import circuits as C
from oracle import drivers as D, layers as LY, mps as OM
from test_gpu_parity import P_TOL, STATE_TOL, _overlap, _sim, _single_path_parity, _state_fid, f_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2]
PREC_IDS = ["fp32", "tf32x3", "bf16x3"]


def _fid_T(A, B):
    return abs(_overlap(A, B)) ** 2 / (_overlap(A, A).real * _overlap(B, B).real)


@functools.lru_cache(maxsize=None)
def _ref_prefix(n, layers, seed, chi):
    """The oracle's own state after the first `layers` layers (the common input of a step)."""
    circ = C.brickwork(n, layers, 0.0, seed)
    return D.run_single_path(circ, D.Params(chi_max=chi, tol=1e-10, sweeps=2), 1, 0).mps


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("layer", [20, 21])
def test_step_parity_chi256_saturated(prec, layer):
    # n = 20 random brickwork without measurements: the middle bonds sit at chi_max = 256 from
    # about layer 14 on, so the guess truncates (cap 256 of up to 512) and both sweeps run.
    # The input is the oracle's state after `layer` layers, imported into the GPU (rounded
    # to complex64); both then compress layer `layer`.
    n, chi, tol, sweeps, seed = 20, 256, 1e-10, 2, 11
    A = _ref_prefix(n, layer, seed, chi)
    assert max(A.bonds()) == chi
    chunk = C.split_layers(C.brickwork(n, layer + 1, 0.0, seed))[layer]
    blocks, empty = LY.chunk_blocks(n, chunk, np.zeros(1, dtype=np.int64))
    assert not empty
    B, info = OM.compress(A, blocks, LY.blocks_mpo(n, blocks), chi, tol, sweeps)
    assert info.fidelities_per_sweep, "the step must run its sweeps (truncated guess)"
    sim = _sim(n, chi, 1, 1, tol, sweeps, 1, 0, prec)
    sim.init_state(1)
    sim.import_mps(0, A.T, A.centre)
    fid = torch.zeros(1, dtype=torch.float64, device="cuda")
    sim.apply_layer(chunk, fid)
    b2, c2, T2 = sim.export_mps(0)
    assert list(b2) == B.bonds()
    assert int(c2) == B.centre
    assert _fid_T(T2, B.T) >= 1 - STATE_TOL
    assert abs(fid.item() - info.f) < f_tol(n, 1)
    assert info.f < 1 - 1e-3  # a real truncation, not a rounding-level one


@functools.lru_cache(maxsize=None)
def _ref_single(n, depth, p, seed, chi, shot):
    circ = C.brickwork(n, depth, p, seed)
    return D.run_single_path(circ, D.Params(chi_max=chi, tol=1e-10, sweeps=2), 1, shot)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_single_path_chi256_truncated_end_to_end(prec):
    # n = 20, 24 layers, measurement rate 0.02: about ten layers past saturation at 256;
    # outcomes, p, state and F shot by shot
    n, depth, p, seed, chi = 20, 24, 0.02, 3, 256
    circ = C.brickwork(n, depth, p, seed)
    refs = [_ref_single(n, depth, p, seed, chi, s) for s in (0, 1)]
    assert all(r.F < 0.995 for r in refs)  # truncated well beyond the tolerance
    _single_path_parity(circ, chi, 2, [0, 1], prec=prec, bond_slack=2)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_multi_path_m64_truncated_pruned(prec):
    # multi-path ensemble with M = 64, bonds truncated at chi_max = 64 in the middle, p values
    # non-degenerate so top-M really cuts (Alg. 2)
    n, depth, p, seed, chi, M = 16, 16, 0.03, 3, 64, 64
    circ = C.brickwork(n, depth, p, seed)
    ref = _ref_multi(n, depth, p, seed, chi, M)
    sim = _sim(n, chi, 2 * M, circ.n_cbits, prec=prec)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    assert res["n_active"] == len(ref) == M
    ps = np.array([b.p for b in ref])
    assert len(np.unique(np.round(ps / (1e-5 * ps.max())))) == M  # no tied keys
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c], f"branch {i}"
        assert abs(res["p"][i] - b.p) < P_TOL
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
    # truncated at the cap (every branch loses fidelity), pruned to M of many more paths
    # (the retained mass is far below 1)
    assert max(max(b.mps.bonds()) for b in ref) == chi
    assert max(b.F for b in ref) < 1 - 1e-4
    assert sum(b.p for b in ref) < 0.5
    for i, b in enumerate(ref):
        assert abs(res["F"][i] - b.F) < f_tol(n, depth)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_multi_path_m64_chi128_truncated(prec):
    # the multi-path ensemble at a larger bond: n = 18, every one of the M = 64 retained
    # branches truncated at chi_max = 128 (each loses fidelity), 64 distinct keys, top-M cut
    # through many more paths (Alg. 2; the one-site updates of Sec. "Simulating unitary
    # quantum circuits with DMRG" on every branch)
    n, depth, p, seed, chi, M = 18, 16, 0.03, 3, 128, 64
    circ = C.brickwork(n, depth, p, seed)
    ref = _ref_multi(n, depth, p, seed, chi, M)
    sim = _sim(n, chi, 2 * M, circ.n_cbits, prec=prec)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    assert res["n_active"] == len(ref) == M
    ps = np.array([b.p for b in ref])
    assert len(np.unique(np.round(ps / (1e-5 * ps.max())))) == M
    assert min(max(b.mps.bonds()) for b in ref) == chi
    assert max(b.F for b in ref) < 1 - 1e-6
    assert sum(b.p for b in ref) < 0.5
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c], f"branch {i}"
        assert abs(res["p"][i] - b.p) < P_TOL
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
        assert abs(res["F"][i] - b.F) < f_tol(n, depth)


@functools.lru_cache(maxsize=None)
def _ref_multi(n, depth, p, seed, chi, M):
    circ = C.brickwork(n, depth, p, seed)
    return D.run_multi_path(circ, D.Params(chi_max=chi, tol=1e-10, sweeps=2), M=M)
