"""Hybrid single-path start (dcs_fork_shots): a circuit's measurement-free prefix run once on
one shot and copied into every shot gives, bit for bit, the shots that running the prefix on
every shot gives (Alg. 1; the paper's GHZ runtime comparison notes that multi-path evaluates
the common prefix once while repeated single-path runs repeat it).  The single-path results
themselves are checked against the oracle by the other parity tests."""
import numpy as np
import pytest

import circuits as C
from test_gpu_parity import _sim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHOT0 = 5


def _first_measurement(ops):
    return next(i for i, o in enumerate(ops) if type(o).__name__ in ("Measure", "Reset"))


def _same_shots(a, b, shots):
    ra, rb = a.results(), b.results()
    assert ra["n_active"] == rb["n_active"] == shots
    for key in ("p", "F", "bits", "flags"):
        np.testing.assert_array_equal(ra[key], rb[key])
    for i in range(shots):
        ba, ca, Ta = a.export_mps(i)
        bb, cb, Tb = b.export_mps(i)
        assert ba.tolist() == bb.tolist() and ca == cb
        for x, y in zip(Ta, Tb):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("case", ["brick-chi32-truncated-prefix", "brick-chi64-global-tiles",
                                  "ghz9"])
def test_forked_prefix_equals_every_shot_running_it(case):
    if case == "brick-chi32-truncated-prefix":
        circ, chi, shots = C.brickwork(12, 10, 0.02, 1), 32, 48   # 7 layers before the first measurement
    elif case == "brick-chi64-global-tiles":
        circ, chi, shots = C.brickwork(14, 10, 0.03, 6), 64, 16
    else:
        circ, chi, shots = C.ghz_dynamic(9), 4, 64
    cut = _first_measurement(circ.ops)
    assert cut > 0
    n = circ.n_qubits
    every = _sim(n, chi, shots, circ.n_cbits)
    every.init_state(shots, shot0=SHOT0)
    every.run_circuit(circ.ops[:cut])
    every.run_circuit(circ.ops[cut:])
    once = _sim(n, chi, shots, circ.n_cbits)
    once.init_state(1, shot0=SHOT0)
    once.run_circuit(circ.ops[:cut])
    once.fork_shots(shots)
    once.run_circuit(circ.ops[cut:])
    _same_shots(every, once, shots)
    # the shots really differ after the prefix: sampled outcomes are not all equal
    assert len({tuple(b) for b in once.results()["bits"].tolist()}) > 1


def test_fork_needs_one_shot():
    from paper_2609_26516_b300 import DCSError
    circ = C.ghz_dynamic(9)
    s = _sim(circ.n_qubits, 4, 8, circ.n_cbits)
    s.init_state(4)
    s.fork_shots(8)            # the list holds 4 shots: refused on the device
    with pytest.raises(DCSError) as e:
        s.results()
    assert e.value.status == 1  # DCS_ERR_INVALID
    s.init_state(1)
    s.fork_shots(8)
    assert s.results()["n_active"] == 8
    m = _sim(circ.n_qubits, 4, 8, circ.n_cbits)
    m.init_state(1, multipath=True)
    with pytest.raises(DCSError):
        m.fork_shots(8)        # multi-path context: refused on the host
