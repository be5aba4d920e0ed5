"""Where the compression and measurement kernels spend their cycles, from the per-phase
counters of a library built with them:

    DCS_NVCC_FLAGS=-DDCS_PHASE_TIMERS DCS_LIB_PATH=/tmp/libdcs_phases.so \\
        python paper_2609_26516_b300/build.py --force
    DCS_LIB_PATH=/tmp/libdcs_phases.so python -m paper_2609_26516_b300.phases ghz64
    DCS_LIB_PATH=/tmp/libdcs_phases.so python -m paper_2609_26516_b300.phases brick \\
        --n 20 --depth 12 --chi 256 --shots 148

At each phase boundary the first thread of every slot adds the clock64() difference since
the previous boundary (after a barrier over the slot's threads) to a device counter.  The
sums are cycles spent per slot, not wall time, and the barriers the counters add slow the
kernels down: read the shares, and time the plain build for durations.
"""
from __future__ import annotations

import argparse
import ctypes

# counter slots of the kernels (k_compress_big: 0-9, k_compress: 10-15, k_measure: 16-17;
# 20/21 and 22/23: Jacobi sweeps and SVD count of the large and small paths)
LARGE = ["copy+1q", "guess hops", "guess gemm+mix", "guess svd", "guess write",
         "centre to end", "env cache", "sweep gemm", "sweep qr", "sweep env+write"]
SMALL = ["set-up+copies", "centre hops", "block product+mix", "block svd", "rank+write",
         "copy-back/sweeps"]
MEAS = ["measure hops", "measure rest"]


def _counters(sim):
    try:
        fn = sim.lib.dcs_debug_phase_cycles
    except AttributeError:
        raise RuntimeError("this libdcs has no phase counters: build it with "
                           "DCS_NVCC_FLAGS=-DDCS_PHASE_TIMERS") from None
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int]
    buf = (ctypes.c_ulonglong * 24)()

    def read(reset=True):
        if fn(buf, 1 if reset else 0) != 0:
            raise RuntimeError("dcs_debug_phase_cycles failed")
        return list(buf)

    return read


def _timed(sim, fn):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(sim.stream)
    fn()
    b.record(sim.stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _shares(v, names, base):
    tot = sum(v[base:base + len(names)]) or 1
    return " ".join(f"{nm}={100.0 * v[base + i] / tot:4.1f}%" for i, nm in enumerate(names))


def ghz64(shots: int) -> None:
    """Dynamic GHZ n=64, chi_max=8: each run of gates or of measurements separately."""
    import circuits as C
    from .sim import Simulator
    n = 64
    circ = C.ghz_dynamic(n)
    groups, cur = [], []
    for o in circ.ops:
        meas = isinstance(o, (C.Measure, C.Reset))
        if cur and meas != isinstance(cur[0], (C.Measure, C.Reset)):
            groups.append(cur)
            cur = []
        cur.append(o)
    groups.append(cur)
    sim = Simulator(n, 8, shots, circ.n_cbits, tol=1e-10, sweeps=2, seed=1)
    read = _counters(sim)
    sim.init_state(shots)
    read()
    n_meas = 0
    for g in groups:
        ms = _timed(sim, lambda: sim.run_circuit(g, meas_idx0=n_meas))
        v = read()
        n_meas += sum(isinstance(o, (C.Measure, C.Reset)) for o in g)
        kind = "measure" if isinstance(g[0], (C.Measure, C.Reset)) else "gates"
        cyc = sum(v[10:18]) / shots / 1e3
        if sum(v[10:16]):
            parts = _shares(v, SMALL, 10)
        elif sum(v[16:18]):
            parts = _shares(v, MEAS, 16)
        else:  # the register-resident measurement runs of bonds <= 4 have no counters
            parts = "no counters on this path"
        print(f"{kind:8s} {len(g):3d} ops {ms:8.3f} ms  {cyc:8.1f} k cycles/shot | {parts}",
              flush=True)


def brick(n: int, depth: int, chi: int, shots: int, precision: int) -> None:
    """Random brickwork without measurements: one line per gate layer."""
    import circuits as C
    from .sim import Simulator
    circ = C.brickwork(n, depth, 0.0, 3)
    layers, cur = [], []
    for o in circ.ops:
        if cur and o.qubits[0] % 2 != cur[0].qubits[0] % 2:
            layers.append(cur)
            cur = []
        cur.append(o)
    layers.append(cur)
    sim = Simulator(n, chi, shots, 1, tol=1e-10, sweeps=2, seed=1, precision=precision)
    read = _counters(sim)
    sim.init_state(shots)
    read()
    for i, lay in enumerate(layers):
        ms = _timed(sim, lambda: sim.apply_layer(lay))
        v = read()
        bonds, _, _ = sim.export_mps(0)
        big = sum(v[0:10]) > 0
        parts = _shares(v, LARGE, 0) if big else _shares(v, SMALL, 10)
        sw = v[20] / max(1, v[21]) if big else v[22] / max(1, v[23])
        print(f"layer {i:2d} {ms:9.1f} ms  max bond {int(max(bonds)):4d}  svd sweeps {sw:4.1f} "
              f"| {parts}", flush=True)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("workload", choices=["ghz64", "brick"])
    ap.add_argument("--shots", type=int, default=10000)
    ap.add_argument("--n", type=int, default=20)
    ap.add_argument("--depth", type=int, default=12)
    ap.add_argument("--chi", type=int, default=256)
    ap.add_argument("--precision", type=int, default=0, help="0 FP32, 1 TF32x3")
    a = ap.parse_args(argv)
    if a.workload == "ghz64":
        ghz64(a.shots)
    else:
        brick(a.n, a.depth, a.chi, a.shots if a.shots != 10000 else 148, a.precision)


if __name__ == "__main__":
    main()
