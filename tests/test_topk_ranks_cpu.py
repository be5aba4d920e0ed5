"""TopKByWeight (Alg. 2) and adaptive pruning over an ensemble split between ranks: the
library's host-only selection (dcs_topk_select_global) against the oracle's rule on the whole
list, and the two-rank exchange (one all-gather of p per measurement, gloo on the CPU) that
feeds it.  No GPU is needed: the selection touches no device."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.statevector import prune_select  # noqa: E402

pytest.importorskip("torch")
LIB = os.path.join(ROOT, "paper_2609_26516_b300", "libdcs.so")
pytestmark = pytest.mark.skipif(not os.path.exists(LIB), reason="libdcs.so not built")


def _cases():
    rng = np.random.default_rng(7)
    out = []
    # distinct values over several decades
    out.append((list(rng.lognormal(-4.0, 2.0, 97)), 16, 0.0))
    # every value tied (dynamic GHZ: all paths at 2^-r): list order decides
    out.append(([2.0 ** -6] * 64, 20, 0.0))
    # values closer than the key unit (1e-5 p_max) and values just across it
    base = 0.01
    vals = [base, base * (1 - 3e-6), base * (1 - 2e-5), base * (1 - 0.4e-5), base * 0.5,
            base * 0.5 * (1 + 1e-7), base * 0.25]
    out.append((vals * 5, 9, 0.0))
    # fewer branches than M: all kept
    out.append((list(rng.random(7)), 16, 0.0))
    # top-M, then the probability threshold (the first of the key order always stays)
    out.append((list(rng.lognormal(-5.0, 1.5, 80)), 40, 5e-3))
    out.append(([1e-4, 2e-4, 5e-5], 2, 0.5))
    # zero probabilities and an exact zero maximum
    out.append(([0.0, 0.3, 0.0, 0.3, 0.1], 2, 0.0))
    out.append(([0.0, 0.0, 0.0], 2, 0.0))
    return out


@pytest.mark.parametrize("case", range(len(_cases())))
def test_global_selection_is_the_oracles_rule(case):
    from paper_2609_26516_b300 import topk_select_global
    ps, M, p_min = _cases()[case]
    keep = topk_select_global(ps, M, p_min)
    if max(ps) > 0.0:
        want = prune_select(list(ps), M, p_min)
    else:  # no scale to compare with: every key is 0, list order decides
        want = list(range(min(M, len(ps))))
    assert np.flatnonzero(keep).tolist() == want


def test_global_selection_refuses_invalid_input():
    from paper_2609_26516_b300 import DCSError, topk_select_global
    for ps, M, p_min in [([0.1, -0.1], 1, 0.0), ([0.1, float("nan")], 1, 0.0),
                         ([0.1, float("inf")], 1, 0.0), ([0.1], 0, 0.0), ([0.1], 1, 1.0),
                         ([0.1], 1, -0.1)]:
        with pytest.raises(DCSError):
            topk_select_global(ps, M, p_min)
    assert topk_select_global([], 3).size == 0


def _rank(rank, world, port, slices, M, p_min, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    from paper_2609_26516_b300.ranks import select_across_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        keep, total = select_across_ranks(slices[rank], M, p_min)
        out.put((rank, keep.tolist(), total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("split", [(40, 57), (0, 97), (96, 1)])
def test_two_ranks_keep_what_one_list_keeps(split):
    # the ensemble's list order is rank 0's branches, then rank 1's; a rank may hold none
    rng = np.random.default_rng(11)
    ps = list(rng.lognormal(-4.0, 2.0, sum(split)))
    slices = [ps[: split[0]], ps[split[0]:]]
    M, p_min = 24, 1e-4
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, slices, M, p_min, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    keep = got[0][1] + got[1][1]
    assert np.flatnonzero(keep).tolist() == prune_select(ps, M, p_min)
    assert got[0][2] == got[1][2] == sum(keep)


class _OracleSim:
    """CPU stand-in for a multi-path Simulator, for the host logic of the sharded run: the
    oracle's state-vector branches behind the library's call semantics (dcs_run_circuit
    splits every branch at a measurement without pruning, children m = 0 before m = 1;
    dcs_get_results lists p in list order; dcs_branch_keep compacts the list)."""

    def __init__(self, n_qubits, n_cbits):
        self.n, self.ncb = n_qubits, n_cbits

    def init_state(self, n_active, multipath=False):
        from oracle import statevector as SV
        self.L = [SV.Branch(1.0, np.zeros(self.ncb, dtype=np.int64), SV.zero_state(self.n))]

    def run_circuit(self, ops, meas_idx0=0, max_branches=0):
        from circuits import Gate, Measure, Reset, X
        from oracle import statevector as SV
        assert max_branches == 0
        for op in ops:
            if isinstance(op, Gate):
                for b in self.L:
                    if SV.cond_holds(op.cond, b.c):
                        b.psi = SV.apply_gate(b.psi, op.qubits, op.matrix)
            elif isinstance(op, (Measure, Reset)):
                nxt = []
                for b in self.L:
                    r0, r1 = SV.probabilities(b.psi, op.qubit)
                    for m, rm in ((0, r0), (1, r1)):
                        pm = rm / (r0 + r1)
                        if pm > SV.P_EPS:
                            c = b.c.copy()
                            c[op.cbit] = m
                            nxt.append(SV.Branch(b.p * pm, c, SV.project(b.psi, op.qubit, m, rm),
                                                 b.path + [m]))
                self.L = nxt
                if isinstance(op, Reset):  # measure into the bit, then X if it reads 1
                    for b in self.L:
                        if b.c[op.cbit] == 1:
                            b.psi = SV.apply_gate(b.psi, (op.qubit,), X)
            else:
                raise TypeError(op)

    def results(self):
        n = len(self.L)
        return {"n_active": n, "p": np.array([b.p for b in self.L]),
                "F": np.ones(n), "flags": np.zeros(n, dtype=np.uint8),
                "cwords": np.zeros((n, 8), dtype=np.uint64),
                "bits": np.array([b.c for b in self.L]).reshape(n, self.ncb)}

    def branch_keep(self, keep):
        keep = list(keep)
        assert len(keep) == len(self.L)
        self.L = [b for b, k in zip(self.L, keep) if k]

    def export_mps_bytes(self, pos):
        import pickle
        return pickle.dumps(self.L[pos])

    def branch_append(self, raw, p, F, cwords, flags=0):
        import pickle
        b = pickle.loads(raw)
        assert b.p == p and F == 1.0
        self.L.append(b)


def _sharded_circuit(which):
    import circuits as C
    # brickwork: every measurement splits every branch; dynamic GHZ: the resets re-measure
    # collapsed ancillas, so parents with only an m = 0 or only an m = 1 child alternate
    return C.brickwork(8, 6, 0.15, 2) if which == "brick" else C.ghz_dynamic(9)


def _sharded_rank(rank, world, port, M, p_min, balance, which, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import circuits as C
    from paper_2609_26516_b300.ranks import run_multi_path_sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        circ = _sharded_circuit(which)
        sim = _OracleSim(circ.n_qubits, circ.n_cbits)
        keys, hist = run_multi_path_sharded(sim, circ, M, p_min, balance=balance)
        assert len(keys) == len(sim.L)
        out.put((rank, [(int(k), b.p, b.c.tolist(), b.path) for k, b in zip(keys, sim.L)], hist))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,M,p_min,balance,which",
                         [(2, 6, 0.0, False, "brick"), (3, 10, 2e-3, False, "brick"),
                          (2, 6, 0.0, True, "brick"), (3, 10, 2e-3, True, "brick"),
                          (2, 64, 0.0, True, "ghz"), (3, 5, 0.0, True, "ghz")])
def test_sharded_run_keeps_the_oracles_ensemble(world, M, p_min, balance, which):
    # the driver's host logic (replicas, contiguous shares, order keys, one exchange per
    # measurement, moves that even out the shares) on world gloo ranks against Alg. 2 on one
    # list (the oracle's run_multi_path)
    import circuits as C
    from oracle import statevector as SV
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_sharded_rank,
                         args=(r, world, port, M, p_min, balance, which, out))
             for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=300) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ref = SV.run_multi_path(_sharded_circuit(which), M, p_min)
    mine = sorted((b for g in got for b in g[1]), key=lambda b: b[0])
    assert [b[0] for b in mine] == list(range(len(ref)))  # dense keys: the list order
    assert [b[3] for b in mine] == [b.path for b in ref]
    assert [b[2] for b in mine] == [b.c.tolist() for b in ref]
    assert [b[1] for b in mine] == [b.p for b in ref]
    # the list was split into shares and the cuts were ensemble-wide
    assert len(got[0][2]) > 0 and all(g[2][-1][1] == len(ref) for g in got)
    assert sum(1 for g in got if any(k for k, _ in g[2])) >= 2
    if balance:  # shares even after every measurement
        for step in zip(*[g[2] for g in got]):
            held = [k for k, _ in step]
            assert max(held) - min(held) <= 1


def test_balance_moves():
    from paper_2609_26516_b300.ranks import _balance_moves
    assert _balance_moves([5, 0, 1]) == [(0, 1, 2), (0, 2, 1)]
    assert _balance_moves([0, 7]) == [(1, 0, 4)]
    assert _balance_moves([3, 3]) == []
    for counts in ([9, 0, 0, 0], [1, 2, 30, 4], [0, 0, 5]):
        after = list(counts)
        for s_, d_, m in _balance_moves(counts):
            after[s_] -= m
            after[d_] += m
        assert sum(after) == sum(counts) and max(after) - min(after) <= 1


class _FailingSim(_OracleSim):
    """A stand-in whose host raises at its `fail_at`-th call (a rank that fails between
    measurements)."""

    def __init__(self, n_qubits, n_cbits, fail_at):
        super().__init__(n_qubits, n_cbits)
        self.calls, self.fail_at = 0, fail_at

    def run_circuit(self, ops, meas_idx0=0, max_branches=0):
        self.calls += 1
        if self.calls == self.fail_at:
            raise RuntimeError("injected rank failure")
        super().run_circuit(ops, meas_idx0, max_branches)


def _failing_rank(rank, world, port, out):
    import datetime
    import time
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import circuits as C
    from paper_2609_26516_b300.ranks import run_multi_path_sharded
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=20))
    circ = C.brickwork(8, 6, 0.15, 2)
    sim = _FailingSim(circ.n_qubits, circ.n_cbits, fail_at=4 if rank == 1 else 0)
    t0 = time.time()
    try:
        run_multi_path_sharded(sim, circ, 6)
        out.put((rank, "finished", time.time() - t0))
    except Exception as e:  # noqa: BLE001 - the failure is the result
        out.put((rank, type(e).__name__ + ": " + str(e)[:80], time.time() - t0))
    # a failed rank leaves without joining further collectives; its exit closes its links


def test_a_failed_rank_ends_the_others_next_exchange():
    # failure detection on the host: rank 1 raises between measurements (after the list was
    # split into shares); rank 0 must not hang, its next all-gather fails within the process
    # group's timeout
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_failing_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=120) for _ in procs), key=lambda g: g[0])
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert "injected rank failure" in got[1][1]
    assert got[0][1] != "finished" and got[0][2] < 60


def test_child_keys_tell_single_child_parents_apart():
    # parents A (only m = 0), B (only m = 1), C (both): children in list order 0, 1, 0, 1
    from paper_2609_26516_b300.ranks import _child_keys
    p_parent = np.array([0.5, 0.3, 0.2])
    p_child = np.array([0.5 * (1 - 1e-14), 0.3, 0.2 * 0.4, 0.2 * 0.6])
    bits = np.array([[0], [1], [0], [1]])
    got = _child_keys(bits, p_child, 0, np.array([0, 1, 2]), p_parent)
    assert got.tolist() == [0, 3, 4, 5]
    # the same bits from two parents with both children each
    got = _child_keys(bits, np.array([0.2, 0.3, 0.1, 0.4]), 0, np.array([7, 9]),
                      np.array([0.5, 0.5]))
    assert got.tolist() == [14, 15, 18, 19]
