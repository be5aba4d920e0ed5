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


def _fid(Ta, Tb):
    """|<a|b>|^2 / (<a|a><b|b>) of two MPS given by their site tensors."""
    def ov(X, Y):
        E = np.ones((1, 1), dtype=np.complex128)
        for x, y in zip(X, Y):
            E = np.einsum("ab,asc,bsd->cd", E, np.conj(x.astype(np.complex128)),
                          y.astype(np.complex128))
        return E[0, 0]
    return abs(ov(Ta, Tb)) ** 2 / (ov(Ta, Ta).real * ov(Tb, Tb).real)


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
        keys, hist = run_multi_path_sharded(sim, circ, M)
        r = sim.results()
        states = [sim.export_mps(i) for i in range(r["n_active"])]
        out.put((rank, keys, r["p"], r["F"], r["bits"], states, hist))
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
    # every branch with its order key; the ensemble's order is ascending key
    rows = sorted(((int(k), g[2][i], g[3][i], g[4][i], g[5][i]) for g in got
                   for i, k in enumerate(g[1])), key=lambda r: r[0])
    assert [r[0] for r in rows] == list(range(M))
    np.testing.assert_array_equal(np.array([r[1] for r in rows]), rr["p"])
    np.testing.assert_array_equal(np.array([r[2] for r in rows]), rr["F"])
    np.testing.assert_array_equal(np.array([r[3] for r in rows]), rr["bits"])
    for i, r in enumerate(rows):
        bonds, centre, T = r[4]
        b2, c2, T2 = ref.export_mps(i)
        assert bonds.tolist() == b2.tolist() and centre == c2
        for x, y in zip(T, T2):
            np.testing.assert_array_equal(x, y)
    # the list was split between the ranks early on and the shares stayed even
    h0, h1 = got[0][6], got[1][6]
    assert len(h0) == len(h1) >= 4
    for (a, t0), (b, t1) in zip(h0, h1):
        assert t0 == t1 == a + b and abs(a - b) <= 1


def test_branch_append_moves_a_branch_between_contexts():
    # export + dcs_branch_append: the moved branches are the same branches, and they evolve
    # the same afterwards; a full pool refuses the append
    from paper_2609_26516_b300 import DCSError
    circ = _circuit()
    cut = _split_after_measurements(circ.ops, 3)
    a, b = _multipath(circ), _multipath(circ)
    a.run_circuit(circ.ops[:cut])
    b.branch_keep([0])  # an empty list
    ra = a.results()
    for i in range(ra["n_active"]):
        b.branch_append(a.export_mps_bytes(i), ra["p"][i], ra["F"][i], ra["cwords"][i],
                        ra["flags"][i])
    _same_branches([b], a)
    # evolved further, the moved branches stay the same branches; the receiving context sized
    # its tiles from the bonds it was given, not from the circuit's bond bound, so its kernels
    # may round differently: compared to the accuracy contract
    a.run_circuit(circ.ops[cut:])
    b.run_circuit(circ.ops[cut:])
    ra, rb = a.results(), b.results()
    assert ra["n_active"] == rb["n_active"]
    np.testing.assert_array_equal(ra["bits"], rb["bits"])
    np.testing.assert_allclose(rb["p"], ra["p"], rtol=0, atol=1e-7)
    np.testing.assert_allclose(rb["F"], ra["F"], rtol=0, atol=1e-5)
    for i in range(ra["n_active"]):
        Ta, Tb = a.export_mps(i)[2], b.export_mps(i)[2]
        assert _fid(Ta, Tb) >= 1 - 1e-6
    small = _sim(N, CHI, 2, circ.n_cbits)
    small.init_state(1, multipath=True)
    raw = a.export_mps_bytes(0)
    small.branch_append(raw, 0.5, 1.0, np.zeros(8, dtype=np.uint64))
    with pytest.raises(DCSError) as e:
        small.branch_append(raw, 0.5, 1.0, np.zeros(8, dtype=np.uint64))
    assert e.value.status == 2  # DCS_ERR_OOM
