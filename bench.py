"""Benchmark of the dynamic-circuit MPS simulator on one B300 (or N, weak scaling).

Workload: random dynamic brickwork (the stand-in for the paper's random dynamic circuits,
Sec. "Random dynamic circuits"), n = 40 qubits, depth 40, measurement rate p = 0.1 with an
outcome-conditioned Haar U(2) on the right neighbour, chi_max = 256, truncation tolerance
1e-10, s = 2 one-site sweeps per compression step, single-path, 512 shots per GPU in one
batch, seeded synthetic circuit (generator seed 3, sampler seed 1).

One step is one segment of the circuit over the whole batch: the compression of one chunk
(the previous layer's conditional gates and one layer of Haar SU(4) gates: initial guess,
environment cache, two sweeps, on every shot) and that layer's mid-circuit measurements
(MeasureProb, sampling, collapse, register writes).  Segments 0-13, in which the bonds grow
to chi_max, prepare the state untimed; the warm-up and timed steps are the segments that
follow, in circuit order (when the circuit runs out it is restarted, untimed).

Metric: one-site compression sweeps per second over all shots (the line's value, mixed
precision: TF32x3 tensor-core contractions with an FP32 last sweep), the plain FP32 path
timed on the same segments beside it (and the BF16x3 mode), shots/s, and the error of each
against the FP64 oracle on one sampled compression step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dcs|reference]

The reference arm (--impl reference) is the CPU FP64 oracle on the same workload, one
segment of one shot per step, on the host cores.  Under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_QUBITS = 40
DEPTH = 40
P_MEAS = 0.1
CHI_MAX = 256
TOL = 1e-10
SWEEPS = 2
SHOTS = 512
CIRCUIT_SEED = 3
SEED = 1
PREFIX = 14          # segments that grow the bonds to chi_max (untimed preparation)
SAMPLE_SEGMENT = 16  # the compression step compared with the oracle
PREC_FP32, PREC_TF32X3, PREC_BF16X3 = 0, 1, 2
WORKLOAD = (f"random dynamic brickwork n={N_QUBITS}, depth {DEPTH}, p={P_MEAS}, "
            f"chi_max={CHI_MAX}, tol={TOL:g}, s={SWEEPS}, single-path, {SHOTS} shots/GPU "
            "batched; step = one circuit segment (one compression + its measurements)")
METRIC = ("compression sweeps/s & shots/s, batched mixed vs plain FP32, at fidelity>=1-1e-6 "
          "(random dynamic brickwork n=40, chi_max=256)")
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rate


def shard_shot0(rank: int, shots_per_rank: int) -> int:
    """First global shot index of a rank.  Ranks take consecutive disjoint ranges, and the
    outcome sampler is keyed by the global shot index, so the results of a shot do not depend
    on which rank runs it."""
    return rank * shots_per_rank


def job_rate(t_step: float, world: int, units_per_rank: float, dist=None, device="cpu"):
    """Step time as the maximum over ranks, and the whole job's units/s at that time."""
    if dist is not None:
        import torch
        t = torch.tensor([t_step], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    return t_step, world * units_per_rank / t_step


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the timed region.

    NVML is polled every 5 ms from a thread (the timed region of a step is milliseconds long),
    the GPU found by its UUID; nvidia-smi at 50 ms is the fallback.  Read-only queries."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, cuda_index: int):
        self.cuda_index = cuda_index
        self.samples = []  # (sm_mhz, max_mhz, reason bits)
        self.stop_flag = threading.Event()
        self.t = None
        self.proc = None
        self.ready = threading.Event()

    def _uuid(self):
        try:
            import torch
            return "GPU-" + str(torch.cuda.get_device_properties(self.cuda_index).uuid)
        except Exception:
            return None

    def _nvml_open(self, uuid):
        """libnvidia-ml through ctypes (read-only queries); returns (lib, handle) or None."""
        import ctypes
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return None
        if nv.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if uuid and nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0:
            return nv, h
        cnt = ctypes.c_uint(0)
        nv.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
        idx = 0 if cnt.value == 1 else self.cuda_index
        if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) == 0:
            return nv, h
        return None

    def _nvml_loop(self, nv, h):
        import ctypes
        try:
            reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            smax = ctypes.c_uint(0)
            nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(smax))  # NVML_CLOCK_SM = 1
            clk = ctypes.c_uint(0)
            rs = ctypes.c_ulonglong(0)
            while not self.stop_flag.is_set():
                ok = nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
                ok = ok and reasons_fn(h, ctypes.byref(rs)) == 0
                if ok:
                    self.samples.append((float(clk.value), float(smax.value), int(rs.value)))
                    self.ready.set()
                time.sleep(0.005)
        finally:
            self.ready.set()

    def start(self):
        uuid = self._uuid()
        opened = self._nvml_open(uuid)
        if opened is not None:
            self.t = threading.Thread(target=self._nvml_loop, args=opened, daemon=True)
            self.t.start()
            self.ready.wait(2.0)
            if self.samples:
                return
            self.stop_flag.set()
            self.t.join(timeout=2)
            self.stop_flag.clear()
            self.t = None
        fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", uuid or str(self.cuda_index), f"--query-gpu={fields}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._smi_read, daemon=True)
            self.t.start()
            self.ready.wait(3.0)
        except OSError:
            self.proc = None

    def _smi_read(self):
        bits = (0x8, 0x40, 0x20, 0x4)
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            try:
                r = sum(b for b, v in zip(bits, parts[2:6]) if v.lower().startswith("active"))
                self.samples.append((float(parts[0]), float(parts[1]), r))
                self.ready.set()
            except (ValueError, IndexError):
                continue

    def stop(self):
        self.stop_flag.set()
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=5)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for _, _, r in self.samples:
            for bit, nm in self.REASONS.items():
                if r & bit:
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(x[0] for x in self.samples),
                "sm_max_mhz": max(x[1] for x in self.samples),
                "reasons": sorted(reasons), "samples": len(self.samples),
                "source": "nvml 5 ms" if self.proc is None else "nvidia-smi 50 ms"}


# ----------------------------------------------------------------------------- workload


def workload():
    """The circuit and its segments (one chunk and the measurements after it, each)."""
    import circuits as C
    circ = C.brickwork(N_QUBITS, DEPTH, P_MEAS, CIRCUIT_SEED)
    return circ, C.split_layers(circ)


def split_segment(ops):
    """(gates, measurements) of a segment: the chunk comes first, the measurements after."""
    from circuits import Measure, Reset
    k = next((i for i, o in enumerate(ops) if isinstance(o, (Measure, Reset))), len(ops))
    return ops[:k], ops[k:]


def mpo_bonds(gates, n):
    """MPO bond dimension per bond of a chunk: 4 across each two-qubit gate (Haar SU(4) has
    full operator-Schmidt rank), 1 elsewhere."""
    D = np.ones(n + 1, dtype=np.float64)
    for g in gates:
        if len(g.qubits) == 2:
            D[min(g.qubits) + 1] = 4.0
    return D


def contraction_flops(alpha, beta, D, sweeps):
    """Algorithmic real flops of one compression step per slot (rows of alpha / beta: ket and
    bra bond dimensions): each one-site update costs 8 (2 b_l D_l a_l a_r + 4 b_l b_r D_r a_r +
    4 b_l a_r D_l D_r) (T1 = L A, the MPO mix, F = T2 R and the environment update; a complex
    multiply-add is 8 flops), each environment of the cache 8 (2 b_l D_l a_l a_r + 2 b_l b_r
    D_r a_r + 4 b_l a_r D_l D_r); the guess and the QR factorisations are not counted."""
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)
    al, ar, bl, br = a[:, :-1], a[:, 1:], b[:, :-1], b[:, 1:]
    Dl, Dr = D[:-1][None, :], D[1:][None, :]
    t1 = 2 * bl * Dl * al * ar
    mix = 4 * bl * ar * Dl * Dr
    site = 8 * (t1 + 4 * bl * br * Dr * ar + mix)
    env = 8 * (t1 + 2 * bl * br * Dr * ar + mix)
    return sweeps * site.sum(axis=1) + env[:, :-1].sum(axis=1)


class SegmentRunner:
    """A batch of shots driven through the circuit one segment at a time."""

    def __init__(self, sim, segs, shots, shot0):
        from paper_2609_26516_b300.sim import encode_ops
        self.sim, self.segs, self.shots, self.shot0 = sim, segs, shots, shot0
        self.enc = []
        self.meas0 = []
        count = 0
        from circuits import Measure, Reset
        for ops in segs:
            g, m = split_segment(ops)
            self.enc.append((encode_ops(g) if g else None, len(g), encode_ops(m) if m else None,
                             len(m)))
            self.meas0.append(count)
            count += sum(isinstance(o, (Measure, Reset)) for o in ops)
        self.pos = None

    def restart(self):
        self.sim.init_state(self.shots, shot0=self.shot0)
        for k in range(PREFIX):
            self.run(k)
        self.pos = PREFIX

    def next_segment(self):
        """Index of the next segment to run, restarting the circuit (untimed) at its end."""
        if self.pos is None or self.pos >= len(self.segs):
            self.restart()
        k = self.pos
        self.pos += 1
        return k

    def run(self, k, mid=None):
        """Segment k: the chunk's compression, then the measurement run (mid: an event
        recorded between the two)."""
        ge, gn, me, mn = self.enc[k]
        if ge is not None:
            self.sim.run_encoded(ge, gn, self.meas0[k])
        if mid is not None:
            mid.record(self.sim.stream)
        if me is not None:
            self.sim.run_encoded(me, mn, self.meas0[k])


def time_arm(precision, segs, shots, shot0, warmup, steps, local, flush, clocks=None,
             barrier=lambda: None):
    """Device-timed steps of one precision arm: per step the compression launch and the whole
    segment (CUDA events on the library's stream, L2 flushed between steps), the one-site
    sweeps run, the algorithmic contraction flops and the library's launches."""
    import torch
    from paper_2609_26516_b300 import Simulator
    circ_cbits = max(1, sum(1 for ops in segs for o in ops if hasattr(o, "cbit")))
    sim = Simulator(N_QUBITS, CHI_MAX, shots, circ_cbits, tol=TOL, sweeps=SWEEPS, seed=SEED,
                    precision=precision, device=f"cuda:{local}")
    run = SegmentRunner(sim, segs, shots, shot0)
    for _ in range(warmup):
        run.run(run.next_segment())
    torch.cuda.synchronize()
    stream = sim.stream
    recs = []
    if clocks is not None:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    for _ in range(steps):
        k = run.next_segment()
        alpha = sim.bonds()
        c0 = sim.counters()[1]
        l0 = sim.launches
        flush.fill_(1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        with torch.cuda.stream(stream):
            e0.record(stream)
            run.run(k, mid=e1)
            e2.record(stream)
        torch.cuda.synchronize()
        launches = sim.launches - l0
        beta = sim.bonds()
        sw = sim.counters()[1] - c0
        g, _ = split_segment(segs[k])
        fl = contraction_flops(alpha, beta, mpo_bonds(g, N_QUBITS), SWEEPS)
        frac = sw / (SWEEPS * len(fl))  # share of the shots whose step ran its sweeps
        recs.append({"segment": k, "ms": e0.elapsed_time(e2), "compress_ms": e0.elapsed_time(e1),
                     "sweeps": int(sw), "flops": float(fl.sum() * frac),
                     "launches": int(launches)})
    barrier()
    clk = clocks.stop() if clocks is not None else None
    return sim, run, recs, clk


def oracle_sample():
    """The oracle's own shot-0 state before SAMPLE_SEGMENT (the common input of the sampled
    step) and its compression of that segment's chunk, probabilities of the segment's first
    measured qubit after it."""
    import circuits as C
    from oracle import drivers as D, layers as LY, mps as OM
    circ, segs = workload()
    prm = D.Params(chi_max=CHI_MAX, tol=TOL, sweeps=SWEEPS)
    r = D.SinglePathRun(circ.n_qubits, circ.n_cbits, prm, SEED, 0)
    for k in range(SAMPLE_SEGMENT):
        r.run(segs[k])
    A = r.mps.copy()
    gates, meas = split_segment(segs[SAMPLE_SEGMENT])
    blocks, _ = LY.chunk_blocks(N_QUBITS, gates, r.c)
    B, info = OM.compress(A, blocks, LY.blocks_mpo(N_QUBITS, blocks), CHI_MAX, TOL, SWEEPS)
    q = meas[0].qubit if meas else 0
    r0, r1 = OM.measure_probs(B.copy(), q)
    return {"A": A, "c": r.c.copy(), "gates": gates, "B": B, "f": info.f, "q": q,
            "p0": r0 / (r0 + r1), "run": r}


def _overlap(A, B):
    E = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        # E'[u, v] = sum_{x, s, y} conj(a[x, s, u]) E[x, y] b[y, s, v], as two products
        t = np.tensordot(E, np.asarray(b, dtype=np.complex128), axes=(1, 0))
        E = np.tensordot(np.conj(np.asarray(a, dtype=np.complex128)), t, axes=([0, 1], [0, 1]))
    return E[0, 0]


def sample_error(precision, ref, local):
    """Error of one precision arm against the FP64 oracle on the sampled step: the oracle's
    state is imported into a one-shot context (rounded to complex64), both compress the same
    chunk, and the results are compared: state infidelity 1 - |<psi_gpu|psi_oracle>|^2,
    |f_gpu - f_oracle| and |p0_gpu - p0_oracle| of the next measured qubit."""
    import torch
    from paper_2609_26516_b300 import Simulator
    ncb = max(1, len(ref["c"]))
    sim = Simulator(N_QUBITS, CHI_MAX, 1, ncb, tol=TOL, sweeps=SWEEPS, seed=SEED,
                    precision=precision, device=f"cuda:{local}")
    sim.init_state(1)
    sim.import_mps(0, ref["A"].T, ref["A"].centre)
    # the chunk's conditions read the oracle's register, which the imported context does
    # not hold: they are evaluated on the host and the chunk handed over holds the gates
    # that apply, unconditioned
    from oracle.statevector import cond_holds
    gates = [type(g)(g.qubits, g.matrix) for g in ref["gates"] if cond_holds(g.cond, ref["c"])]
    fid = torch.zeros(1, dtype=torch.float64, device=f"cuda:{local}")
    sim.apply_layer(gates, fid)
    p0 = sim.measure_prob(ref["q"])
    torch.cuda.synchronize()
    _, _, T = sim.export_mps(0)
    B = ref["B"].T
    ab = _overlap(T, B)
    inf = 1.0 - abs(ab) ** 2 / (_overlap(T, T).real * _overlap(B, B).real)
    out = {"state_infidelity": float(max(inf, 0.0)), "f_abs_err": abs(fid.item() - ref["f"]),
           "p0_abs_err": abs(float(p0[0].item()) - ref["p0"]), "f_oracle": ref["f"],
           "step": f"segment {SAMPLE_SEGMENT}, shot 0, oracle's own input state"}
    out["meets_contract"] = bool(out["state_infidelity"] <= 1e-6 and out["p0_abs_err"] <= 1e-5)
    del sim
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- CPU oracle


def _blas_threads():
    """Threads of the BLAS the oracle's NumPy calls (threadpoolctl), else the host cores
    (OpenBLAS and MKL start one thread per core by default)."""
    try:
        from threadpoolctl import threadpool_info
        return max((int(x.get("num_threads", 1)) for x in threadpool_info()), default=1)
    except Exception:  # pragma: no cover
        return host_cores()


def oracle_steps(run, segs, first, n_steps, seconds=None):
    """The oracle (FP64 NumPy MPS, unchanged) continuing one shot's run segment by segment:
    per segment its wall time and the one-site sweeps it ran."""
    out = []
    t_all = time.perf_counter()
    for k in range(first, first + n_steps):
        if seconds is not None and out and time.perf_counter() - t_all > seconds:
            break
        s0 = run.sweeps_run
        t0 = time.perf_counter()
        run.run(segs[k % len(segs)])
        out.append((time.perf_counter() - t0, run.sweeps_run - s0))
    return out


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def run_reference(args):
    """The oracle on the same workload: shot 0 prepared through the first segments (untimed),
    then one segment per step, BLAS on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import drivers as D
    circ, segs = workload()
    prm = D.Params(chi_max=CHI_MAX, tol=TOL, sweeps=SWEEPS)
    run = D.SinglePathRun(circ.n_qubits, circ.n_cbits, prm, SEED, 0)
    for k in range(PREFIX):
        run.run(segs[k])
    warm = oracle_steps(run, segs, PREFIX, args.warmup)
    del warm
    rec = oracle_steps(run, segs, PREFIX + args.warmup, args.steps)
    t = sum(x[0] for x in rec)
    sw = sum(x[1] for x in rec)
    value = sw / t
    cores = _blas_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "the oracle on shot 0, one segment per step "
                   f"(segments {PREFIX + args.warmup}..{PREFIX + args.warmup + args.steps - 1}, "
                   f"after {PREFIX} untimed segments and {args.warmup} warm-up segments)"},
        "shots_per_s": value / (SWEEPS * DEPTH),
        "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sw} one-site sweeps over {args.steps} segments of shot 0, "
                                   f"FP64 NumPy, BLAS on {cores} threads"},
        "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- extras


def measure_ghz(shots=10000, steps=10):
    """Dynamic GHZ preparation, n = 64 (32 data + 32 ancilla qubits), chi_max = 8, 10^4 shots
    per batch: shots/s (the small-bond kernels)."""
    import torch
    import circuits as C
    from paper_2609_26516_b300 import Simulator
    from paper_2609_26516_b300.sim import encode_ops
    circ = C.ghz_dynamic(64)
    ops, n_ops = encode_ops(circ.ops), len(circ.ops)
    sim = Simulator(64, 8, shots, circ.n_cbits, tol=TOL, sweeps=SWEEPS, seed=SEED)

    def one():
        sim.init_state(shots)
        sim.run_encoded(ops, n_ops)

    for _ in range(3):
        one()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(sim.stream)
    for _ in range(steps):
        one()
    e.record(sim.stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / steps
    res = sim.results()
    out = {"workload": f"dynamic GHZ n=64, chi_max=8, {shots} shots per batch",
           "shots_per_s": shots / (ms / 1000.0), "ms_per_batch": ms,
           "max_rel_p_err": float(np.max(np.abs(res["p"] / 2.0 ** -circ.meta["r"] - 1)))}
    del sim
    torch.cuda.empty_cache()
    return out


def _run_segments(sim, segs, count, multipath_m=0):
    """Runs the first `count` segments of a circuit on a context, timing each with CUDA
    events on the library's stream; returns per-segment ms and the sweeps run."""
    import torch
    from circuits import Measure, Reset
    ms, m0 = [], 0
    for ops in segs[:count]:
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.run_circuit(ops, meas_idx0=m0, max_branches=multipath_m)
        e.record(sim.stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
        m0 += sum(isinstance(o, (Measure, Reset)) for o in ops)
    return ms, sim.counters()[1]


def measure_multipath(layers=16, M=64, chi=512, n=32):
    """The multi-path ensemble workload (n = 32, depth 30, p = 0.05, top-M with M = 64 of a
    128-slot pool, chi_max = 512): its first `layers` segments, BF16x3 and plain FP32."""
    import torch
    import circuits as C
    from paper_2609_26516_b300 import Simulator
    circ = C.brickwork(n, 30, 0.05, CIRCUIT_SEED)
    segs = C.split_layers(circ)
    out = {"workload": f"multi-path brickwork n={n}, depth 30 (first {layers} segments), p=0.05, "
                       f"M={M}, chi_max={chi}, s=2"}
    for prec, name in ((2, "bf16x3"), (0, "fp32")):
        sim = Simulator(n, chi, 2 * M, circ.n_cbits, tol=TOL, sweeps=SWEEPS, seed=SEED,
                        precision=prec)
        sim.init_state(1, multipath=True)
        ms, sw = _run_segments(sim, segs, layers, M)
        res = sim.results()
        bonds = sim.bonds()
        out[name] = {"ms_total": sum(ms), "segment_ms": [round(x, 1) for x in ms],
                     "sweeps": int(sw), "sweeps_per_s": sw / (sum(ms) / 1000.0),
                     "branches": int(res["n_active"]), "retained_p": float(res["p"].sum()),
                     "max_bond": int(bonds.max()), "min_branch_max_bond": int(bonds.max(axis=1).min()),
                     "arena_gb": sim.arena_bytes / 1e9}
        del sim
        torch.cuda.empty_cache()
    out["mixed_over_fp32"] = out["fp32"]["ms_total"] / out["bf16x3"]["ms_total"]
    return out


def measure_large_chi(layers=8, shots=64, chi=1024, n=64):
    """The large-chi workload (n = 64, depth 64, p = 0.02, chi_max = 1024, s = 3, 64 shots):
    its first `layers` segments (bonds up to 2^8), TF32x3, and the arena it takes."""
    import torch
    import circuits as C
    from paper_2609_26516_b300 import Simulator
    circ = C.brickwork(n, 64, 0.02, 5)
    segs = C.split_layers(circ)
    sim = Simulator(n, chi, shots, circ.n_cbits, tol=TOL, sweeps=3, seed=SEED, precision=1)
    sim.init_state(shots)
    ms, sw = _run_segments(sim, segs, layers)
    bonds = sim.bonds()
    out = {"workload": f"large-chi brickwork n={n}, depth 64 (first {layers} segments), p=0.02, "
                       f"chi_max={chi}, s=3, {shots} shots, TF32x3",
           "arena_gb": sim.arena_bytes / 1e9, "ms_total": sum(ms),
           "segment_ms": [round(x, 1) for x in ms], "sweeps": int(sw),
           "max_bond": int(bonds.max()), "F_mean": float(sim.results()["F"].mean())}
    del sim
    torch.cuda.empty_cache()
    return out


def measure_cgemm(chi, batch):
    """The contraction primitive alone at the site-contraction shape of chi_max: M = 2 chi,
    N = chi, K = 4 chi complex (F = T2 R^T with an MPO bond of 4), one problem per CTA,
    CUDA cores vs tensor cores."""
    import ctypes
    import torch
    from paper_2609_26516_b300 import _native as N_
    lib = N_.load()
    M, Nn, K = 2 * chi, chi, 4 * chi
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((batch, M, K), dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn((batch, Nn, K), dtype=torch.complex64, device="cuda", generator=g)
    Cm = torch.zeros((batch, M, Nn), dtype=torch.complex64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    out = {"workload": f"complex GEMM M={M} N={Nn} K={K} batch={batch} (B transposed)",
           "flops_per_call": 8.0 * M * Nn * K * batch}
    for mode, name in ((1, "tensor_tf32x3"), (2, "tensor_bf16x3"), (0, "simt_fp32")):
        times = []
        for i in range(5):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(st)
            rc = lib.dcs_cgemm(mode, batch, M, Nn, K, ctypes.c_void_p(A.data_ptr()), K, 1, M * K, 0,
                               ctypes.c_void_p(B.data_ptr()), 1, K, Nn * K, 0,
                               ctypes.c_void_p(Cm.data_ptr()), Nn, 1, M * Nn,
                               ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(st.cuda_stream))
            e.record(st)
            torch.cuda.synchronize()
            assert rc == 0 and int(err.item()) == 0
            if i >= 2:
                times.append(a.elapsed_time(e))
        ms = statistics.median(times)
        out[name] = {"ms": ms, "tflops": out["flops_per_call"] / (ms / 1000.0) / 1e12}
    del A, B, Cm
    torch.cuda.empty_cache()
    return out


def run_profile_case(args):
    """The first segments of the workload with a small shot count: the last compression
    launch is a saturated one of the workload's shape, for a profiler to capture."""
    import torch
    from paper_2609_26516_b300 import Simulator
    circ, segs = workload()
    sim = Simulator(N_QUBITS, CHI_MAX, args.shots, circ.n_cbits, tol=TOL, sweeps=SWEEPS,
                    seed=SEED, precision=args.precision)
    sim.init_state(args.shots)
    run = SegmentRunner(sim, segs, args.shots, 0)
    for k in range(args.profile_segments):
        run.run(k)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"{args.profile_segments} segments", "shots": args.shots,
                      "precision": args.precision, "max_bond": int(sim.bonds().max()),
                      "launches": sim.launches}), flush=True)


# ----------------------------------------------------------------------------- main


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dcs", choices=["dcs", "reference"])
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--fp32-steps", type=int, default=3,
                    help="timed steps of the plain FP32 arm (the same segments as the first "
                         "steps of the mixed arm)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--profile-segments", type=int, default=0,
                    help="run only the first K segments of the workload with --shots shots at "
                         "--precision (a small case for a profiler) and exit")
    ap.add_argument("--precision", type=int, default=PREC_TF32X3)
    ap.add_argument("--cgemm", type=int, nargs=2, metavar=("CHI", "BATCH"), default=None,
                    help="only the contraction primitive at the site shape of CHI, BATCH "
                         "problems (a small case for a profiler)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_segments > 0:
        run_profile_case(args)
        return
    if args.cgemm is not None:
        print(json.dumps(measure_cgemm(*args.cgemm)), flush=True)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    from paper_2609_26516_b300.sim import encode_ops

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    circ, segs = workload()
    shot0 = shard_shot0(rank, args.shots)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > L2 (126 MB)

    # ---- mixed-precision arm: the line's value
    t_prep = time.perf_counter()
    clocks = ClockSampler(local)
    sim, run, recs, clk = time_arm(PREC_TF32X3, segs, args.shots, shot0, args.warmup,
                                   args.steps, local, flush, clocks, barrier)
    ms = [r["ms"] for r in recs]
    t_step, value = job_rate(sum(ms) / len(ms) / 1000.0, world,
                             sum(r["sweeps"] for r in recs) / len(recs), dist, f"cuda:{local}")
    launches = sum(r["launches"] for r in recs)
    comp_ms = sum(r["compress_ms"] for r in recs) / len(recs)
    flops = sum(r["flops"] for r in recs) / len(recs)
    achieved = flops / (comp_ms / 1000.0) / 1e12
    peaks, peak_kind = measured_peaks()
    peak_tf32 = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])) * TF32_PER_BF16

    # ---- end to end through the C ABI: each step encodes the segment on the host, uploads
    # its tables from the pinned stage and reads the results back
    e2e_t, e2e_sw = [], []
    up0 = sim.bytes_uploaded
    n_e2e = min(args.steps, 3)
    for _ in range(n_e2e):
        k = run.next_segment()
        c0 = sim.counters()[1]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g, m = split_segment(segs[k])
        if g:
            sim.run_encoded(encode_ops(g), len(g), run.meas0[k])
        if m:
            sim.run_encoded(encode_ops(m), len(m), run.meas0[k])
        res = sim.results()
        e2e_t.append(time.perf_counter() - t0)
        e2e_sw.append(sim.counters()[1] - c0)
    h2d = (sim.bytes_uploaded - up0) // n_e2e
    d2h = 8 + args.shots * (4 + 8 + 8 + 8 * 8 + 4)
    _, e2e_value = job_rate(sum(e2e_t) / n_e2e, world, sum(e2e_sw) / n_e2e, dist, f"cuda:{local}")
    F_mean = float(np.mean(res["F"]))
    del sim, run
    torch.cuda.empty_cache()

    # ---- plain FP32 arm on the same segments
    n32 = min(args.fp32_steps, args.steps)
    sim32, run32, recs32, _ = time_arm(PREC_FP32, segs, args.shots, shot0, args.warmup, n32,
                                       local, flush, None, barrier)
    del sim32, run32
    torch.cuda.empty_cache()
    ms32 = [r["ms"] for r in recs32]
    _, value32 = job_rate(sum(ms32) / len(ms32) / 1000.0, world,
                          sum(r["sweeps"] for r in recs32) / len(recs32), dist, f"cuda:{local}")
    same = [r["ms"] for r in recs[: len(recs32)]]
    speedup = (sum(ms32) / len(ms32)) / (sum(same) / len(same))
    # ---- BF16x3 arm on the same segments
    sim16, run16, recs16, _ = time_arm(PREC_BF16X3, segs, args.shots, shot0, args.warmup, n32,
                                       local, flush, None, barrier)
    del sim16, run16
    torch.cuda.empty_cache()
    ms16 = [r["ms"] for r in recs16]
    _, value16 = job_rate(sum(ms16) / len(ms16) / 1000.0, world,
                          sum(r["sweeps"] for r in recs16) / len(recs16), dist, f"cuda:{local}")
    wall = time.perf_counter() - t_prep

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---- error against the FP64 oracle on one sampled step, each arm; the oracle's timing
    # on the same workload continues that run (rank 0, one GPU only)
    err = {}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ref = oracle_sample()
        err = {"tf32x3": sample_error(PREC_TF32X3, ref, local),
               "bf16x3": sample_error(PREC_BF16X3, ref, local),
               "fp32": sample_error(PREC_FP32, ref, local)}
        cores = _blas_threads()
        rec = oracle_steps(ref["run"], segs, SAMPLE_SEGMENT, 4, seconds=20.0)
        t_o = sum(x[0] for x in rec)
        sw_o = sum(x[1] for x in rec)
        cpu = {"value": sw_o / t_o, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
               "sample": f"shot 0, segments {SAMPLE_SEGMENT}..{SAMPLE_SEGMENT + len(rec) - 1} "
                         f"({sw_o} one-site sweeps, {t_o:.1f} s), FP64 NumPy, BLAS on {cores} "
                         "threads"}
    mean_sweeps = sum(r["sweeps"] for r in recs) / len(recs)
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shots_per_gpu": args.shots,
                   "segments_timed": [r["segment"] for r in recs],
                   "precision": "TF32x3 tensor-core contractions, FP32 last sweep",
                   "l2": "flushed between timed steps (256 MB write outside the events)",
                   "parallelism": f"shots sharded over {world} GPU(s), no collective"},
        "shots_per_s": value / (SWEEPS * DEPTH),
        "shots_per_s_note": "sweeps/s over the 2 sweeps x 40 layers of a shot: the rate of a "
                            "whole circuit if every layer cost a saturated one",
        "sweeps_per_step": mean_sweeps,
        "fp32": {"value": value32, "unit": "sweeps/s", "steps": len(recs32),
                 "ms_per_step": sum(ms32) / len(ms32),
                 "segments_timed": [r["segment"] for r in recs32]},
        "bf16x3": {"value": value16, "unit": "sweeps/s", "steps": len(recs16),
                   "ms_per_step": sum(ms16) / len(ms16),
                   "segments_timed": [r["segment"] for r in recs16],
                   "over_fp32": (sum(ms32) / len(ms32)) / (sum(ms16) / len(ms16))},
        "mixed_over_fp32": speedup,
        "error_vs_oracle": err,
        "F_mean_after_e2e": F_mean,
        "roofline": {"bound": "tensor", "kernel": "k_compress_big<512,TC> (one compression, "
                     "all shots)", "achieved": achieved, "peak": peak_tf32, "unit": "TFLOP/s",
                     "frac": achieved / peak_tf32, "traffic": None,
                     "flops_per_launch": flops, "launch_ms": comp_ms,
                     "peak_source": f"bf16_tflops_sustained of MEASURED_PEAKS.json ({peak_kind}) "
                                    "x nominal TF32/BF16 ratio 1.1/2.25",
                     "flops_source": "algorithmic contraction flops from the bond dimensions "
                                     "before and after each step (guess SVD and QR excluded)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "sweeps/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": n_e2e},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / len(recs),
        "clocks": clk,
        "bench_wall_s": wall,
    }
    if world == 1 and not args.no_extras:
        line["ghz64"] = measure_ghz()
        line["contraction"] = measure_cgemm(256, 148)
        line["contraction_chi512"] = measure_cgemm(512, 148)
        line["multipath"] = measure_multipath()
        line["large_chi"] = measure_large_chi()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
