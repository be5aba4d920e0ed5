"""The library's host-side chunk tables (build_layer in csrc/dcs_tables.h), run on the CPU
through a small C++ driver (tests/host_tables_harness.cpp): the operator-Schmidt split of
each two-qubit gate into the MPO factors of its block (Sec. "Simulating unitary quantum
circuits with DMRG": the chunk as an MPO), the blocks composed on the host, the per-site
description of the chunk, the conditional gates kept per block for the device to apply
(Sec. "Classically controlled operations"), and the errors of invalid chunks.  Checked
against NumPy and against the oracle's block construction."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import circuits as C
from oracle import layers as LY
from paper_2609_26516_b300.sim import encode_ops

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2609_26516_b300", "csrc")
F32 = 2e-6  # the tables hold complex64 values computed in FP64


def _cond(v):
    return {"op": v[0], "value": v[1], "mask": [int(x) for x in v[2:]]}


def _c16(t):
    f = np.array([float(x) for x in t])
    return f[0::2] + 1j * f[1::2]


def _parse(out):
    lines = out.splitlines()
    if lines and lines[0].startswith("ERR"):
        return {"err": lines[0][4:]}
    res = {"sites": [], "blocks": [], "g1": [], "conds": []}
    for ln in lines:
        t = ln.split()
        if t[0] == "LAYER":
            res["layer"] = dict(zip(["n_blocks", "blk_off", "uncond", "cond_off", "n_conds"],
                                    map(int, t[1:])))
        elif t[0] == "SITE":
            kind, blk, g_off, g_n = map(int, t[2:])
            res["sites"].append({"kind": kind, "blk": blk, "g_off": g_off, "g_n": g_n})
        elif t[0] == "BLOCK":
            v = [int(x) for x in t[1:]]
            res["blocks"].append({
                "q": v[0], "D": v[1], "composed": v[2],
                "pre": [(v[3], v[4]), (v[7], v[8])], "post": [(v[5], v[6]), (v[9], v[10])],
                "cond": _cond(v[11:])})
        elif t[0] in ("G", "WL", "WR", "GC"):
            res["blocks"][-1][t[0]] = _c16(t[1:])
        elif t[0] == "G1":
            res["g1"].append((_c16(t[1:9]).reshape(2, 2), _cond([int(x) for x in t[9:]])))
        elif t[0] == "COND":
            res["conds"].append(_cond([int(x) for x in t[1:]]))
    return res


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    d = tmp_path_factory.mktemp("tables")
    exe = str(d / "harness")
    cxx = shutil.which("g++") or shutil.which("c++")
    assert cxx, "a C++ compiler is needed to build the table driver"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", cuda_inc, "-I", CSRC,
                        os.path.join(HERE, "host_tables_harness.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(n, ops):
        p = d / "ops.bin"
        p.write_bytes(bytes(encode_ops(ops)) if ops else b"")
        out = subprocess.run([exe, str(n), str(p)], capture_output=True, text=True, timeout=60)
        assert out.returncode == 0, out.stderr
        return _parse(out.stdout)

    def plan(n, ops, chunk_k=0, idx0=0, layers=1):
        p = d / "circ.bin"
        p.write_bytes(bytes(encode_ops(ops)) if ops else b"")
        out = subprocess.run([exe, "plan", str(n), str(chunk_k), str(idx0), str(p), str(layers)],
                             capture_output=True, text=True, timeout=60)
        assert out.returncode == 0, out.stderr
        steps = []
        for ln in out.stdout.splitlines():
            t = ln.split()
            if t[0] == "ERR":
                return {"err": ln[4:]}
            if t[0] == "STEP":
                steps.append({"kind": int(t[1]), "n": int(t[3]), "items": []})
            elif t[0] == "CHUNK":  # one line per sub-layer
                v = [int(x) for x in t[1:]]
                steps[-1]["items"].append({"n_blocks": v[0], "uncond": v[1], "n_conds": v[2],
                                           "kinds": v[3:]})
            elif t[0] == "MEAS":
                steps[-1]["items"].append(tuple(int(x) for x in t[1:]))
        return steps

    run.plan = plan
    return run


SWAP = np.eye(4, dtype=np.complex128)[[0, 2, 1, 3]]


def _reshuffle(G):
    """M[(o0 i0), (o1 i1)] = G[(o0 o1), (i0 i1)]: the matrix whose SVD is the
    operator-Schmidt decomposition of G."""
    return G.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)


def _on_pair(m, qubits, q):
    """Matrix of a two-qubit gate over |s_q s_{q+1}> (a gate listed as (q+1, q) swaps legs)."""
    m = np.asarray(m, dtype=np.complex128)
    return m if qubits[0] == q else m.reshape(2, 2, 2, 2).transpose(1, 0, 3, 2).reshape(4, 4)


def test_operator_schmidt_split_reconstructs_each_gate(tables):
    rng = np.random.default_rng(2)
    gates = [(C.CNOT, (0, 1), 2), (C.CNOT, (3, 2), 2), (C.haar_su4(rng), (4, 5), 4),
             (np.kron(C.H, C.rz(0.3)), (6, 7), 1), (SWAP, (9, 8), 4)]
    t = tables(10, [C.Gate(qs, m) for m, qs, _ in gates])
    lay = t["layer"]
    assert (lay["n_blocks"], lay["uncond"], lay["n_conds"]) == (5, 1, 0)
    assert [b["q"] for b in t["blocks"]] == [8, 6, 4, 2, 0]  # decreasing q
    by_q = {b["q"]: b for b in t["blocks"]}
    for m, qs, rank in gates:
        q = min(qs)
        b = by_q[q]
        G = _on_pair(m, qs, q)
        np.testing.assert_allclose(b["G"].reshape(4, 4), G, atol=F32)
        assert b["D"] == rank
        WL = b["WL"].reshape(4, 4)[:, :rank]
        WR = b["WR"].reshape(4, 4)[:rank, :]
        np.testing.assert_allclose(WL @ WR, _reshuffle(G), atol=4 * F32)
        # U sqrt(sigma) and sqrt(sigma) V^H: both factors carry the singular values' roots
        s = np.linalg.svd(_reshuffle(G), compute_uv=False)[:rank]
        np.testing.assert_allclose(np.linalg.norm(WL, axis=0) ** 2, s, atol=4 * F32)
        np.testing.assert_allclose(np.linalg.norm(WR, axis=1) ** 2, s, atol=4 * F32)
        # the oracle's MPO of the same block is the same two-site operator
        W = LY.blocks_mpo(10, [(q, G)])
        two = np.einsum("aoiD,DpjE->opij", W[q], W[q + 1]).reshape(4, 4)
        np.testing.assert_allclose(two, G, atol=1e-12)
    kinds = [s["kind"] for s in t["sites"]]
    assert kinds == [2, 3] * 5


def _gate1_product(entries):
    """U of a list of (2x2, cond) applied in order (later gates on the left)."""
    U = np.eye(2, dtype=np.complex128)
    for u, _ in entries:
        U = u @ U
    return U


def test_composed_blocks_match_the_oracle_blocks(tables):
    rng = np.random.default_rng(4)

    def U():
        return C.haar_unitary(rng, 2)

    ops = [C.Gate((1,), U()), C.Gate((2,), U()), C.Gate((2,), U()),
           C.Gate((1, 2), C.haar_su4(rng)), C.Gate((1,), U()), C.Gate((2,), U()),
           C.Gate((4,), U()), C.Gate((4,), U()), C.Gate((6, 5), C.CNOT), C.Gate((6,), U())]
    n = 8
    t = tables(n, ops)
    ref, empty = LY.chunk_blocks(n, ops, np.zeros(16, dtype=np.int64))
    assert not empty
    ref = dict(ref)
    assert [s["kind"] for s in t["sites"]] == [0, 2, 3, 0, 1, 2, 3, 0]
    assert sorted(b["q"] for b in t["blocks"]) == [1, 5]
    for b in t["blocks"]:
        assert b["composed"] == 1
        np.testing.assert_allclose(b["GC"].reshape(4, 4), ref[b["q"]], atol=4 * F32)
    b1 = next(b for b in t["blocks"] if b["q"] == 1)
    assert [b1["pre"][0][1], b1["pre"][1][1], b1["post"][0][1], b1["post"][1][1]] == [1, 2, 1, 1]
    s4 = t["sites"][4]
    assert s4["g_n"] == 2
    U4 = _gate1_product(t["g1"][s4["g_off"]:s4["g_off"] + s4["g_n"]])
    np.testing.assert_allclose(U4, ref[4], atol=4 * F32)


def _holds(cond, c):
    """phi(c) from a table's condition: XOR (parity) or AND of the mask bits, == value."""
    if cond["op"] == 0:
        return True
    bits = [w * 64 + b for w, m in enumerate(cond["mask"]) for b in range(64) if (m >> b) & 1]
    vals = [int(c[b]) for b in bits]
    v = sum(vals) % 2 if cond["op"] == 1 else int(all(vals))
    return v == cond["value"]


def _block_from_tables(t, b, c):
    """A block as the device builds it for register c from the tables:
    (Post_q x Post_q+1) (G2 if its condition holds, else I) (Pre_q x Pre_q+1)."""
    def side(part, s):
        off, cnt = b[part][s]
        return _gate1_product([e for e in t["g1"][off:off + cnt] if _holds(e[1], c)])

    G = b["G"].reshape(4, 4) if _holds(b["cond"], c) else np.eye(4)
    return np.kron(side("post", 0), side("post", 1)) @ G @ np.kron(side("pre", 0), side("pre", 1))


def test_conditional_gates_are_kept_for_the_device(tables):
    rng = np.random.default_rng(9)
    a, b, u, v = (C.haar_unitary(rng, 2) for _ in range(4))
    ops = [C.Gate((2,), a, cond=C.Cond((0, 3), "xor", 1)), C.Gate((2, 3), C.haar_su4(rng)),
           C.Gate((3,), b, cond=C.Cond((1, 70), "and", 1)),
           C.Gate((0,), u, cond=C.Cond((5,), "xor", 0)), C.Gate((0,), v),
           C.Gate((5, 4), C.CNOT, cond=C.Cond((2,), "xor", 1))]
    n = 6
    t = tables(n, ops)
    lay = t["layer"]
    assert (lay["n_blocks"], lay["uncond"], lay["n_conds"]) == (2, 1, 4)
    assert [s["kind"] for s in t["sites"]] == [1, 0, 2, 3, 2, 3]
    assert all(b["composed"] == 0 for b in t["blocks"])
    regs = []
    for bits in [(), (0,), (3,), (0, 3), (1,), (1, 70), (2,), (5,), (0, 1, 2, 5, 70)]:
        c = np.zeros(80, dtype=np.int64)
        c[list(bits)] = 1
        regs.append(c)
    for c in regs:
        ref = dict(LY.chunk_blocks(n, ops, c)[0])
        for blk in t["blocks"]:
            np.testing.assert_allclose(_block_from_tables(t, blk, c), ref[blk["q"]], atol=4 * F32)
        s0 = t["sites"][0]
        U0 = _gate1_product([e for e in t["g1"][s0["g_off"]:s0["g_off"] + s0["g_n"]]
                             if _holds(e[1], c)])
        np.testing.assert_allclose(U0, ref[0], atol=4 * F32)


def test_invalid_chunks_are_refused(tables):
    two = tables(4, [C.Gate((0, 1), C.CNOT), C.Gate((2, 1), C.CNOT)])
    assert "two two-qubit gates" in two["err"]
    far = tables(4, [C.Gate((0, 2), C.CNOT)])
    assert "neighbouring" in far["err"]


def test_every_brickwork_chunk_matches_the_oracle(tables):
    circ = C.brickwork(9, 6, 0.3, 7)
    n, steps = LY.chunk_circuit(circ)
    rng = np.random.default_rng(1)
    regs = [np.zeros(circ.n_cbits + 1, dtype=np.int64)]
    regs += [rng.integers(0, 2, circ.n_cbits + 1) for _ in range(3)]
    seen = 0
    for st in steps:
        if not isinstance(st, list):
            continue
        seen += 1
        t = tables(n, st)
        for c in regs:
            ref = dict(LY.chunk_blocks(n, st, c)[0])
            assert sorted(b["q"] for b in t["blocks"]) == sorted(q for q, G in ref.items()
                                                                 if G.shape == (4, 4))
            for blk in t["blocks"]:
                got = blk["GC"].reshape(4, 4) if blk["composed"] else _block_from_tables(t, blk, c)
                np.testing.assert_allclose(got, ref[blk["q"]], atol=4 * F32)
            for q, G in ref.items():
                if G.shape == (2, 2):
                    s = t["sites"][q]
                    assert s["kind"] == 1
                    U = _gate1_product([e for e in t["g1"][s["g_off"]:s["g_off"] + s["g_n"]]
                                        if _holds(e[1], c)])
                    np.testing.assert_allclose(U, G, atol=4 * F32)
    assert seen >= 6


def _oracle_chunk_summary(n, chunk):
    kinds = [0] * n
    for g in chunk:
        if len(g.qubits) == 2:
            q = min(g.qubits)
            kinds[q], kinds[q + 1] = 2, 3
    for g in chunk:
        if len(g.qubits) == 1 and kinds[g.qubits[0]] == 0:
            kinds[g.qubits[0]] = 1
    return {"n_blocks": sum(len(g.qubits) == 2 for g in chunk),
            "uncond": int(any(g.cond is None for g in chunk)),
            "n_conds": sum(g.cond is not None for g in chunk), "kinds": kinds}


@pytest.mark.parametrize("layers", [1, 2, 3, 4])
@pytest.mark.parametrize("chunk_k", [0, 3, 11])
@pytest.mark.parametrize("name", ["teleport", "ghz", "brickwork"])
def test_circuit_plan_matches_the_oracle_chunking(tables, name, chunk_k, layers):
    circ = {"teleport": C.teleport(2), "ghz": C.ghz_dynamic(20),
            "brickwork": C.brickwork(9, 6, 0.3, 7)}[name]
    idx0 = 5
    steps = tables.plan(circ.n_qubits, circ.ops, chunk_k, idx0, layers)
    n, ref = LY.chunk_circuit(circ, chunk_k, layers)
    want, runs, ord_ = [], 0, idx0
    for i, st in enumerate(ref):
        if isinstance(st, list):
            # one launch per chunk, its sub-layers in order
            want.append([_oracle_chunk_summary(n, sub) for sub in LY.sublayers(st)])
        else:
            want.append((st.qubit, st.cbit, ord_))
            ord_ += 1
            runs += int(i == 0 or isinstance(ref[i - 1], list))
    got = []
    for s in steps:
        if s["kind"] == 0:
            got.append(s["items"])
        else:
            got += s["items"]
    assert got == want
    # one launch per chunk and one per maximal run of consecutive measurements
    assert sum(s["kind"] == 1 for s in steps) == runs
    assert all(s["n"] == len(s["items"]) for s in steps)
    assert all(1 <= s["n"] <= max(layers, 1) for s in steps if s["kind"] == 0)


@pytest.mark.parametrize("layers", [1, 2, 3, 4])
def test_unitary_brickwork_chunks_hold_the_layer_count(tables, layers):
    # without measurements, depth 7 gives ceil(7 / layers) chunks of `layers` sub-layers
    # (the last one shorter), each sub-layer one brickwork layer
    circ = C.brickwork(9, 7, 0.0, 3)
    steps = tables.plan(circ.n_qubits, circ.ops, 0, 0, layers)
    assert all(s["kind"] == 0 for s in steps)
    sizes = [s["n"] for s in steps]
    assert sizes == [layers] * (7 // layers) + ([7 % layers] if 7 % layers else [])
    blocks = [it["n_blocks"] for s in steps for it in s["items"]]
    assert blocks == [4] * 7  # n = 9: pairs from 0 and from 1 both give four blocks
