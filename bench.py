"""Benchmark of the dynamic-circuit MPS simulator on one B300 (or N, weak scaling).

Workload (default): dynamic GHZ preparation on n = 64 qubits (32 data on even sites, 32
ancillas on odd sites), chi_max = 8, 2 one-site sweeps per compression step, truncation
tolerance 1e-10, single-path, 10,000 shots per GPU in one batch.  One step is one pass of
the whole hot path over the batch: InitializeState, then the circuit (4 compression steps,
64 mid-circuit measurements with sampling, collapse and register writes, conditional X
layers).  Metric: shots/s (whole job); sweeps/s reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dcs|reference]

The reference arm (--impl reference) is the CPU FP64 oracle run on a bounded sample of the
same workload on the host cores.  Under torchrun only rank 0 runs it.
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

N_QUBITS = 64
CHI_MAX = 8
SWEEPS = 2
TOL = 1e-10
SHOTS = 10000
SEED = 1
WORKLOAD = "dynamic GHZ n=64 (32 data + 32 ancilla), chi_max=8, s=2, tol=1e-10, single-path, 10000 shots/GPU"
METRIC = "shots/s (single-path dynamic GHZ n=64, chi_max=8)"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def sweeps_per_shot(bits: np.ndarray) -> np.ndarray:
    """Compression sweeps each shot ran: 2 unconditional chunks, plus the data feed-forward
    chunk unless no prefix parity is 1, plus the reset chunk unless every ancilla read 0
    (a chunk whose gates are all skipped is not compressed); s sweeps each."""
    n_anc = N_QUBITS // 2
    meas = bits[:, :n_anc - 1]  # ancilla outcomes that enter the prefix parities
    ff = np.any(np.cumsum(meas, axis=1) % 2 == 1, axis=1)
    rst = np.any(bits[:, n_anc:2 * n_anc] == 1, axis=1)
    return SWEEPS * (2 + ff.astype(np.int64) + rst.astype(np.int64))


def algorithmic_flops_per_shot() -> float:
    """Algorithmic real flops of the compression sweeps of one GHZ shot (contractions only):
    per one-site update 8 (2 b_l D_l a_l a_r + 4 b_l b_r D_r a_r + 4 b_l a_r D_l D_r) with the
    bond dimensions this circuit has (all internal bonds 2 after the first layer; the CNOT
    MPO bond is 2, the single-qubit layers 1)."""
    n = N_QUBITS
    total = 0.0
    # chunk 1 (H + CNOT pairs (2i, 2i+1)): bonds after guess 2 on odd bonds, 1 on even bonds
    # chunk 2 (CNOT pairs (2i+1, 2i+2)): all internal bonds 2 except the idle last ancilla
    # chunks 3, 4 (conditional X): bonds 2, D = 1
    def upd(bl, br, al, ar, dl, dr):
        return 8.0 * (2 * bl * dl * al * ar + 4 * bl * br * dr * ar + 4 * bl * ar * dl * dr)

    def chunk(bonds_b, bonds_a, D):
        f = 0.0
        for j in range(n):
            f += upd(bonds_b[j], bonds_b[j + 1], bonds_a[j], bonds_a[j + 1], D[j], D[j + 1])
        return f

    one = [1] * (n + 1)
    b1 = [1] + [2 if (b % 2 == 1) else 1 for b in range(1, n)] + [1]
    b2 = [1] + [2] * (n - 2) + [1, 1]
    D1 = [1] + [2 if b % 2 == 1 else 1 for b in range(1, n)] + [1]
    D2 = [1] + [2 if (b % 2 == 0 and b < n - 1) else 1 for b in range(1, n)] + [1]
    total += SWEEPS * chunk(b1, one, D1)
    total += SWEEPS * chunk(b2, b1, D2)
    total += 2 * SWEEPS * chunk(b2, b2, one)
    return total


def cpu_oracle_sample(seconds: float = 15.0, max_shots: int = 200):
    """The oracle (FP64 NumPy MPS, unchanged) on a bounded sample of the workload."""
    import circuits as C
    from oracle import drivers as D
    try:
        from threadpoolctl import threadpool_limits
        lim = threadpool_limits(1)
    except Exception:  # pragma: no cover
        lim = None
    circ = C.ghz_dynamic(N_QUBITS)
    prm = D.Params(chi_max=CHI_MAX, tol=TOL, sweeps=SWEEPS)
    t0 = time.perf_counter()
    shots = 0
    while shots < max_shots and (time.perf_counter() - t0) < seconds:
        D.run_single_path(circ, prm, SEED, shots)
        shots += 1
    dt = time.perf_counter() - t0
    if lim is not None:
        lim.unregister() if hasattr(lim, "unregister") else None
    return shots, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    shots_per_step = []
    times = []
    for i in range(args.warmup + args.steps):
        n, dt = cpu_oracle_sample(seconds=6.0, max_shots=40)
        if i >= args.warmup:
            shots_per_step.append(n)
            times.append(dt)
    total_shots, total_t = sum(shots_per_step), sum(times)
    value = total_shots / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "shots/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "oracle shots 0.. of the same circuit, "
                   "about 6 s of CPU per step"},
        "cpu_baseline": {"value": value, "unit": "shots/s", "cores": 1, "kind": "oracle",
                         "sample": f"{total_shots} shots over {args.steps} steps"},
        "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dcs", choices=["dcs", "reference"])
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    import circuits as C
    from paper_2609_26516_b300 import Simulator
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

    circ = C.ghz_dynamic(N_QUBITS)
    ops = encode_ops(circ.ops)
    n_ops = len(circ.ops)
    sim = Simulator(N_QUBITS, CHI_MAX, args.shots, circ.n_cbits, tol=TOL, sweeps=SWEEPS,
                    seed=SEED, device=f"cuda:{local}")
    stream = sim.stream
    shot0 = rank * args.shots
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > L2 (126 MB)

    def step():
        sim.init_state(args.shots, shot0=shot0)
        sim.run_encoded(ops, n_ops)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, L2 flushed between steps (outside the events)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    l0 = sim.launches
    durs = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            durs.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    launches = (sim.launches - l0) // args.steps
    ms = [a.elapsed_time(b) for a, b in durs]
    clk = clocks.stop()
    t_step = sum(ms) / len(ms) / 1000.0
    if dist is not None:
        t = torch.tensor([t_step], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    res = sim.results()
    sps = sweeps_per_shot(res["bits"])
    value = world * args.shots / t_step
    sweeps_s = world * float(sps.sum()) / t_step

    # ---- dominant kernel: the compression kernel timed alone on the same stream
    from paper_2609_26516_b300.sim import encode_ops as enc
    layer_ops = [o for o in circ.ops[: N_QUBITS // 2 + (N_QUBITS // 2 - 1)]]  # H + CNOT layer
    k_ms = []
    gl = enc(layer_ops)
    for i in range(6):
        sim.init_state(args.shots, shot0=shot0)
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.lib.dcs_apply_layer(sim.ctx, gl, len(layer_ops), None)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            k_ms.append(a.elapsed_time(b))
    comp_ms = statistics.median(k_ms)
    # algorithmic flops of that launch: chunk 1 with bra bonds (1,2,1,2,...) and s sweeps
    peaks, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak_tflops = sm_count * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    n = N_QUBITS
    one = [1] * (n + 1)
    b1 = [1] + [2 if (b % 2 == 1) else 1 for b in range(1, n)] + [1]
    D1 = [1] + [2 if b % 2 == 1 else 1 for b in range(1, n)] + [1]
    f_launch = 0.0
    for j in range(n):
        bl, br, al, ar, dl, dr = b1[j], b1[j + 1], one[j], one[j + 1], D1[j], D1[j + 1]
        f_launch += 8.0 * (2 * bl * dl * al * ar + 4 * bl * br * dr * ar + 4 * bl * ar * dl * dr)
    f_launch *= SWEEPS * args.shots
    achieved = f_launch / (comp_ms / 1000.0) / 1e12

    # ---- end to end through the C ABI with host buffers (tables up, results down)
    e2e_t = []
    up0 = sim.bytes_uploaded
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_state(args.shots, shot0=shot0)
        arr = encode_ops(circ.ops)
        sim.run_encoded(arr, n_ops)
        sim.results()
        e2e_t.append(time.perf_counter() - t0)
    h2d = (sim.bytes_uploaded - up0) // 3
    d2h = 8 + args.shots * (4 + 8 + 8 + 8 * 8 + 4)
    e2e_value = world * args.shots / statistics.median(e2e_t)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ns, dt = cpu_oracle_sample(seconds=15.0)
        cpu = {"value": ns / dt, "unit": "shots/s", "cores": 1, "kind": "oracle",
               "sample": f"{ns} shots of the same circuit (shots 0..{ns - 1}), FP64 NumPy, "
                         f"{dt:.1f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1000.0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "shots_per_gpu": args.shots,
                   "l2": "flushed between timed steps (256 MB write outside the events)",
                   "parallelism": f"shots sharded over {world} GPU(s), no collective"},
        "sweeps_per_s": sweeps_s,
        "roofline": {"bound": "alu", "kernel": "k_compress<8,32> (H+CNOT chunk, all shots)",
                     "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak_tflops, "traffic": None,
                     "peak_source": f"FP32 SIMT: {sm_count} SMs x 128 lanes x 2 x "
                                    f"{peaks.get('sm_max_mhz', 2032.0)} MHz ({peak_kind} clock)",
                     "launch_ms": comp_ms},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "shots/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
