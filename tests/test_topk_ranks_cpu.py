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
