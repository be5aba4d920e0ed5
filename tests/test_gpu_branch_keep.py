"""Branch compaction by an explicit selection (dcs_branch_keep) and TopKByWeight over an
ensemble split between contexts (Alg. 2 with the branch list sharded over ranks).  Two
contexts on one GPU stand in for two ranks: each holds one part of the list and runs on its
own (no kernel waits on another context); the selection applied to them is the one every
rank computes after the all-gather of p (dcs_topk_select_global).  The result must be what a
single context holding the whole list keeps with dcs_branch_topk, branch by branch."""
import numpy as np
import pytest

import circuits as C
from test_gpu_parity import _sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# 7 measurements, 128 branches at the end without pruning, distinct path probabilities
N, DEPTH, P, SEED, CHI, SLOTS = 10, 8, 0.1, 3, 16, 256


def _circuit():
    return C.brickwork(N, DEPTH, P, SEED)


def _split_after_measurements(ops, at_least):
    """Index just past the first run of measurements that brings their count to at_least."""
    seen = 0
    for i, op in enumerate(ops):
        if type(op).__name__ == "Measure":
            seen += 1
        elif seen >= at_least:
            return i
    raise AssertionError("circuit has too few measurements")


def _same_branches(a_sims, b):
    """The concatenated lists of a_sims equal b's list: p, F, register, every site tensor."""
    ra = [s.results() for s in a_sims]
    rb = b.results()
    assert sum(r["n_active"] for r in ra) == rb["n_active"]
    for key in ("p", "F", "bits"):
        got = np.concatenate([r[key] for r in ra])
        np.testing.assert_array_equal(got, rb[key])
    pos = 0
    for s, r in zip(a_sims, ra):
        for i in range(r["n_active"]):
            ba, ca, Ta = s.export_mps(i)
            bb, cb, Tb = b.export_mps(pos)
            assert ba.tolist() == bb.tolist() and ca == cb
            for x, y in zip(Ta, Tb):
                np.testing.assert_array_equal(x, y)
            pos += 1


def _multipath(circ):
    sim = _sim(N, CHI, SLOTS, circ.n_cbits)
    sim.init_state(1, multipath=True)
    return sim


def test_branch_keep_with_the_global_selection_equals_topk():
    from paper_2609_26516_b300 import topk_select_global
    circ = _circuit()
    a, b = _multipath(circ), _multipath(circ)
    a.run_circuit(circ)
    b.run_circuit(circ)
    K = a.results()["n_active"]
    M = 40
    assert K == 128
    a.branch_topk(M)
    keep = topk_select_global(b.results()["p"], M)
    assert keep.sum() == M
    b.branch_keep(keep)
    _same_branches([b], a)


def test_sharded_ensemble_keeps_what_one_context_keeps():
    from paper_2609_26516_b300 import topk_select_global
    circ = _circuit()
    cut = _split_after_measurements(circ.ops, 2)
    pre, post = circ.ops[:cut], circ.ops[cut:]
    one, r0, r1 = _multipath(circ), _multipath(circ), _multipath(circ)
    for s in (one, r0, r1):
        s.run_circuit(pre)
    K0 = one.results()["n_active"]
    assert K0 >= 3
    h = K0 // 2
    r0.branch_keep([1] * h + [0] * (K0 - h))   # rank 0: the first h branches of the list
    r1.branch_keep([0] * h + [1] * (K0 - h))   # rank 1: the rest
    _same_branches([r0, r1], one)
    for s in (one, r0, r1):
        s.run_circuit(post, meas_idx0=sum(type(o).__name__ == "Measure" for o in pre))
    M = 40
    one.branch_topk(M)
    p0, p1 = r0.results()["p"], r1.results()["p"]
    keep = topk_select_global(np.concatenate([p0, p1]), M)
    r0.branch_keep(keep[: len(p0)])
    r1.branch_keep(keep[len(p0):])
    assert r0.results()["n_active"] > 0 and r1.results()["n_active"] > 0
    _same_branches([r0, r1], one)


def test_branch_keep_length_mismatch_is_reported():
    from paper_2609_26516_b300 import DCSError
    circ = _circuit()
    s = _multipath(circ)
    s.run_circuit(circ.ops[: _split_after_measurements(circ.ops, 2)])
    K = s.results()["n_active"]
    s.branch_keep([1] * (K + 1))
    with pytest.raises(DCSError) as e:
        s.results()
    assert e.value.status == 1  # DCS_ERR_INVALID
    s.init_state(1, multipath=True)  # a fresh state clears the status
    assert s.results()["n_active"] == 1
