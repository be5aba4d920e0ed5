"""The benchmark's reference arm (the oracle on the host cores) runs without a GPU and prints
the line the result format asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "sweeps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "sweeps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _bench_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, v = bench.job_rate(0.010 * (rank + 1), world, 100, dist, "cpu")
        out.put((rank, t, v, bench.shard_shot0(rank, 100)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_is_max_and_shots_are_disjoint():
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, v, lo in got:
        assert t == 0.020  # the slower rank's step time on every rank
        assert abs(v - 2 * 100 / 0.020) < 1e-9
        assert lo == 100 * rank
    ranges = [set(range(lo, lo + 100)) for _, _, _, lo in got]
    assert not (ranges[0] & ranges[1]) and (ranges[0] | ranges[1]) == set(range(200))


def test_contraction_flops_count():
    # every bond chi, MPO bonds 4 on odd bonds: per site 8 (2 chi^3 D_l + 4 chi^3 D_r +
    # 4 chi^2 D_l D_r) per sweep, the environment cache 8 (2 chi^3 D_l + 2 chi^3 D_r + 4 chi^2
    # D_l D_r) per site but the last
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    n, chi = 6, 16
    a = np.full((2, n + 1), chi)
    a[:, 0] = a[:, n] = 1
    D = np.array([1.0 if b % 2 == 0 else 4.0 for b in range(n + 1)])
    got = bench.contraction_flops(a, a, D, 2)
    want = 0.0
    for j in range(n):
        bl, br, Dl, Dr = a[0, j], a[0, j + 1], D[j], D[j + 1]
        site = 8 * (2 * bl * Dl * bl * br + 4 * bl * br * Dr * br + 4 * bl * br * Dl * Dr)
        env = 8 * (2 * bl * Dl * bl * br + 2 * bl * br * Dr * br + 4 * bl * br * Dl * Dr)
        want += 2 * site + (env if j < n - 1 else 0)
    assert np.allclose(got, want)


def test_workload_segments_are_chunk_then_measurements():
    sys.path.insert(0, ROOT)
    import circuits as C
    import bench
    circ, segs = bench.workload()
    assert sum(segs, []) == circ.ops and len(segs) == bench.DEPTH + 1
    for ops in segs:
        g, m = bench.split_segment(ops)
        assert all(isinstance(o, C.Gate) for o in g) and all(isinstance(o, C.Measure) for o in m)
