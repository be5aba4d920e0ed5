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


def _reference_by_measurement(circ, M):
    """One context holding the whole list, the ops run in the same calls as the sharded run
    (each ending at a measurement), pruned to M at every measurement (dcs_run_circuit)."""
    sim = _multipath(circ)
    seg = []
    for op in circ.ops:
        seg.append(op)
        if type(op).__name__ == "Measure":
            sim.run_circuit(seg, max_branches=M)
            seg = []
    if seg:
        sim.run_circuit(seg, max_branches=M)
    return sim


def _rank_main(rank, world, port, M, out):
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path[:0] = [root, os.path.join(root, "tests")]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import circuits as Cc
        from paper_2609_26516_b300.ranks import run_multi_path_sharded
        from test_gpu_parity import _sim as mk
        circ = Cc.brickwork(N, DEPTH, P, SEED)
        sim = mk(N, CHI, SLOTS, circ.n_cbits)
        hist = run_multi_path_sharded(sim, circ, M)
        r = sim.results()
        states = [sim.export_mps(i) for i in range(r["n_active"])]
        out.put((rank, r["p"], r["F"], r["bits"], states, hist))
    finally:
        dist.destroy_process_group()


def test_two_processes_sharded_run_equals_one_context():
    # Alg. 2 end to end with the list split between two ranks (two processes, gloo for the
    # one all-gather per measurement; their kernels never wait on each other), against one
    # context holding the whole list: the same branches, bit for bit, in the same order
    import multiprocessing as mp
    import socket
    M = 40
    circ = _circuit()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, M, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=600) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = _reference_by_measurement(circ, M)
    rr = ref.results()
    assert rr["n_active"] == M
    assert sum(len(g[1]) for g in got) == M
    # the list was split between the ranks early on, and both held branches after cuts
    assert len(got[0][5]) == len(got[1][5]) >= 4
    assert all(t0 == t1 for (_, t0), (_, t1) in zip(got[0][5], got[1][5]))
    assert any(k > 0 for k, _ in got[1][5]) and any(k > 0 for k, _ in got[0][5])
    np.testing.assert_array_equal(np.concatenate([g[1] for g in got]), rr["p"])
    np.testing.assert_array_equal(np.concatenate([g[2] for g in got]), rr["F"])
    np.testing.assert_array_equal(np.concatenate([g[3] for g in got]), rr["bits"])
    states = [s for g in got for s in g[4]]
    for i, (bonds, centre, T) in enumerate(states):
        b2, c2, T2 = ref.export_mps(i)
        assert bonds.tolist() == b2.tolist() and centre == c2
        for x, y in zip(T, T2):
            np.testing.assert_array_equal(x, y)
