"""Chunks of several gate layers (chunk_layers = 2, 3, 4) against the FP64 oracle.

A chunk of L layers is compressed in one step (Sec. "Simulating unitary quantum circuits
with DMRG", CompressionStep) against the composed MPO of its layers (bond <= 4^L); the
initial guess applies the layers one after another with a truncated SVD per block.  The
oracle builds the same chunks (chunk_circuit with ``layers``), composes the layer MPOs and
takes the guess layer by layer.  Checked: per-step parity at a saturated bond (sweeps with
MPO bonds of 4 to 256, FP32 and both tensor-core precisions), whole dynamic circuits
shot by shot (single path) and branch by branch (multi path)."""
import functools

import numpy as np
import pytest

import circuits as C
from oracle import drivers as D, layers as LY, mps as OM
from test_gpu_parity import P_TOL, STATE_TOL, _overlap, _state_fid, f_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2]
PREC_IDS = ["fp32", "tf32x3", "bf16x3"]


def _sim(n, chi, slots, ncb, layers, prec=0, seed=1, tol=1e-10, sweeps=2):
    from paper_2609_26516_b300 import Simulator
    return Simulator(n, chi, slots, max(ncb, 1), tol=tol, sweeps=sweeps, seed=seed,
                     precision=prec, chunk_layers=layers)


def _fid_T(A, B):
    return abs(_overlap(A, B)) ** 2 / (_overlap(A, A).real * _overlap(B, B).real)


@functools.lru_cache(maxsize=None)
def _ref_prefix(n, depth, seed, chi):
    circ = C.brickwork(n, depth, 0.0, seed)
    return D.run_single_path(circ, D.Params(chi_max=chi, tol=1e-10, sweeps=2), 1, 0).mps


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("layers,stacked", [(2, False), (3, False), (4, False), (2, True),
                                            (3, True), (4, True)],
                         ids=["2-brick", "3-brick", "4-brick", "2-stacked", "3-stacked",
                              "4-stacked"])
def test_step_parity_saturated(prec, layers, stacked):
    # n = 14 brickwork: after 12 layers the middle bonds sit at chi_max = 64; the next
    # layers form one chunk whose guess truncates, so both sweeps run.  Consecutive
    # brickwork layers alternate their pairs (composed MPO bond 4^ceil(layers/2));
    # "stacked" takes every other layer instead, so each pair carries a gate in every
    # sub-layer and the MPO bond is 4^layers (16, 64, 256).  Contractions of 64 x 64 and more
    # take the tensor cores on the TF32X3 / BF16X3 paths.
    n, chi, depth, seed = 14, 64, 12, 21
    A = _ref_prefix(n, depth, seed, chi)
    assert max(A.bonds()) == chi
    step = 2 if stacked else 1
    lay = C.split_layers(C.brickwork(n, depth + step * layers, 0.0, seed))
    chunk = [g for i in range(layers) for g in lay[depth + step * i]]
    sub, empty = LY.chunk_sublayer_blocks(n, chunk, np.zeros(1, dtype=np.int64))
    assert not empty and len(sub) == layers
    W = LY.compose_mpo([LY.blocks_mpo(n, b) for b in sub])
    assert max(w.shape[0] for w in W) == (4 ** layers if stacked else 4 ** ((layers + 1) // 2))
    B, info = OM.compress(A, sub, W, chi, 1e-10, 2)
    assert info.fidelities_per_sweep, "the step must run its sweeps (truncated guess)"
    sim = _sim(n, chi, 1, 1, layers, prec)
    sim.init_state(1)
    sim.import_mps(0, A.T, A.centre)
    fid = torch.zeros(1, dtype=torch.float64, device="cuda")
    sim.apply_layer(chunk, fid)
    b2, c2, T2 = sim.export_mps(0)
    assert list(b2) == B.bonds()
    assert int(c2) == B.centre
    assert _fid_T(T2, B.T) >= 1 - STATE_TOL
    assert abs(fid.item() - info.f) < f_tol(n, 1)
    assert info.f < 1 - 1e-3


@pytest.mark.parametrize("layers", [2, 3, 4])
def test_apply_layer_rejects_more_sublayers_than_configured(layers):
    from paper_2609_26516_b300 import DCSError
    n = 6
    circ = C.brickwork(n, layers + 1, 0.0, 4)
    chunk = [g for layer in C.split_layers(circ) for g in layer]
    sim = _sim(n, 8, 1, 1, layers)
    sim.init_state(1)
    with pytest.raises(DCSError):
        sim.apply_layer(chunk)


@pytest.mark.parametrize("layers,chi", [(2, 8), (3, 8), (4, 8), (2, 32), (3, 32), (4, 32)])
def test_single_path_dynamic_brickwork(layers, chi):
    # n = 10 random dynamic brickwork with sparse measurements, so that chunks hold up to
    # `layers` layers between them: chi 32 holds the state exactly (guess exact, sweeps
    # skipped), chi 8 truncates; outcomes, p, state and F shot by shot
    n, depth, p, seed = 10, 9, 0.05, 3
    circ = C.brickwork(n, depth, p, seed)
    _, steps = LY.chunk_circuit(circ, 0, layers)
    assert max(len(LY.sublayers(st)) for st in steps if isinstance(st, list)) == layers
    shots = 4
    sim = _sim(n, chi, shots, circ.n_cbits, layers)
    sim.init_state(shots)
    sim.run_circuit(circ)
    res = sim.results()
    prm = D.Params(chi_max=chi, tol=1e-10, sweeps=2, layers=layers)
    compared = 0
    for s in range(shots):
        ref = D.run_single_path(circ, prm, 1, s)
        if ref.flagged:
            continue
        compared += 1
        assert res["bits"][s].tolist() == [int(x) for x in ref.c], f"shot {s}"
        bonds, _, _ = sim.export_mps(s)
        assert list(bonds) == ref.mps.bonds(), f"shot {s}"
        assert _state_fid(sim, s, ref.mps) >= 1 - STATE_TOL
        assert abs(res["p"][s] - ref.p) < P_TOL
        assert abs(res["F"][s] - ref.F) < f_tol(n, len(ref.fids))
    assert compared >= shots // 2


@pytest.mark.parametrize("layers", [2, 3, 4])
def test_multi_path_dynamic_brickwork(layers):
    # four measurements (16 paths) between chunks of up to `layers` layers, top-8 kept,
    # chi 16 truncating; branch by branch
    n, depth, p, seed, chi, M = 10, 9, 0.05, 6, 16, 8
    circ = C.brickwork(n, depth, p, seed)
    _, steps = LY.chunk_circuit(circ, 0, layers)
    assert max(len(LY.sublayers(st)) for st in steps if isinstance(st, list)) == layers
    ref = D.run_multi_path(circ, D.Params(chi_max=chi, layers=layers), M=M)
    sim = _sim(n, chi, 2 * M, circ.n_cbits, layers)
    sim.init_state(1, multipath=True)
    sim.run_circuit(circ, max_branches=M)
    res = sim.results()
    assert res["n_active"] == len(ref)
    for i, b in enumerate(ref):
        assert res["bits"][i].tolist() == [int(x) for x in b.c]
        assert _state_fid(sim, i, b.mps) >= 1 - STATE_TOL
        assert abs(res["p"][i] - b.p) < P_TOL
        assert abs(res["F"][i] - b.F) < f_tol(n, depth)


def test_layers_agree_on_an_exact_state():
    # chi 64 holds n = 12 exactly: one to four layers per chunk give the same state
    # (the exact state vector's), so the chunking changes the cost, not the result
    n, depth, seed = 12, 7, 2
    circ = C.brickwork(n, depth, 0.0, seed)
    T = []
    for layers in (1, 2, 3, 4):
        sim = _sim(n, 64, 1, 1, layers)
        sim.init_state(1)
        sim.run_circuit(circ)
        T.append(sim.export_mps(0)[2])
    for t in T[1:]:
        assert _fid_T(t, T[0]) >= 1 - STATE_TOL
