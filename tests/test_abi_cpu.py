"""The C ABI without a GPU: the library builds and loads, exports every function declared in
include/dcs.h, its struct layouts match the Python binding, and the host-only argument
checks answer as documented."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dcs.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2609_26516_b300 import build
    build.build()
    from paper_2609_26516_b300 import _native as N
    return N.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dcs_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["dcs_create", "dcs_destroy", "dcs_init_state", "dcs_apply_layer",
                 "dcs_measure_prob", "dcs_measure_sample", "dcs_collapse", "dcs_branch_split",
                 "dcs_branch_topk", "dcs_get_results", "dcs_export_mps", "dcs_import_mps",
                 "dcs_run_circuit", "dcs_arena_bytes", "dcs_last_error"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2609_26516_b300 import _native as N
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in N.SIGNATURES, f"binding lacks {name}"


def test_struct_layout_matches_binding(tmp_path):
    from paper_2609_26516_b300 import _native as N
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "dcs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(dcs_op), offsetof(dcs_op, m),
         offsetof(dcs_op, cond), sizeof(dcs_cond), sizeof(dcs_config),
         offsetof(dcs_config, tol), offsetof(dcs_config, seed));
  return 0;
}
'''
    c = tmp_path / "layout.c"
    c.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [ctypes.sizeof(N.dcs_op), N.dcs_op.m.offset, N.dcs_op.cond.offset,
            ctypes.sizeof(N.dcs_cond), ctypes.sizeof(N.dcs_config), N.dcs_config.tol.offset,
            N.dcs_config.seed.offset]
    assert got == want


def _cfg(N, **kw):
    base = dict(n_qubits=64, chi_max=8, tol=1e-10, sweeps=2, chunk_k=0, precision=0, n_cbits=64,
                n_slots=10000, seed=1)
    base.update(kw)
    return N.dcs_config(**base)


def _slot_elems(n, C):
    cap = [min(C, 2 ** min(b, n - b)) for b in range(n + 1)]
    return sum(2 * 2 * cap[j] * cap[j + 1] for j in range(n)) + sum(4 * c * c for c in cap)


@pytest.mark.parametrize("n,chi,slots,limit_gb", [(40, 256, 512, 80), (64, 1024, 64, 230),
                                                    (32, 512, 128, 140)])
def test_arena_fits_the_large_bond_workloads(lib, n, chi, slots, limit_gb):
    # bond-sized sites and a single environment cache: the large-bond workloads fit the
    # B300's HBM (n = 64, chi_max = 1024, 64 slots needed 432 GB with fixed-stride sites)
    from paper_2609_26516_b300 import _native as N
    nb = lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=n, chi_max=chi, n_slots=slots)))
    assert slots * _slot_elems(n, chi) * 8 < nb < limit_gb * 1e9


def test_arena_bytes_and_argument_checks(lib):
    from paper_2609_26516_b300 import _native as N
    cfg = _cfg(N)
    nb = lib.dcs_arena_bytes(ctypes.byref(cfg))
    # two MPS buffers + one environment cache dominate, sized by the bond capacities
    # cap_b = min(C, 2^min(b, n - b)) (C = 8 here): site j holds cap_j 2 cap_{j+1} complex64,
    # bond b's environment cap_b 4 cap_b
    assert nb > 10000 * _slot_elems(64, 8) * 8
    assert nb < 1.25 * 10000 * _slot_elems(64, 8) * 8
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=0))) == 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, chi_max=2048))) == 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, chi_max=64, kernel_path=1))) == 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_cbits=513))) == 0
    # the largest chain the library takes, and one qubit more
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=N.MAX_QUBITS))) > 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=N.MAX_QUBITS + 1))) == 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=1))) > 0
    ctx = ctypes.c_void_p()
    assert lib.dcs_create(ctypes.byref(ctx), ctypes.byref(_cfg(N, sweeps=0)), None, 0, None) == N.ERR_INVALID
    assert lib.dcs_create(ctypes.byref(ctx), ctypes.byref(_cfg(N, chi_max=2048)), None, 0, None) == N.ERR_UNSUPPORTED
    assert lib.dcs_create(ctypes.byref(ctx), ctypes.byref(cfg), None, 0, None) == N.ERR_OOM
    assert lib.dcs_last_error(None) == b"null context"


def test_chunk_layers_configuration(lib):
    # chunks of several layers run on the global work area only, up to four layers; their
    # environment caches hold the composed MPO bond 4^layers
    from paper_2609_26516_b300 import _native as N
    n, chi, S = 24, 64, 4
    one = lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=n, chi_max=chi, n_slots=S)))
    assert one > 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=n, chi_max=chi, n_slots=S,
                                                 chunk_layers=1))) == one
    sizes = [one]
    for layers in (2, 3, 4):
        nb = lib.dcs_arena_bytes(ctypes.byref(_cfg(N, n_qubits=n, chi_max=chi, n_slots=S,
                                                   chunk_layers=layers)))
        cap = [min(chi, 2 ** min(b, n - b)) for b in range(n + 1)]
        env = S * sum(4 ** layers * c * c for c in cap) * 8
        assert nb > env
        sizes.append(nb)
    assert sizes[0] < sizes[1] < sizes[2] < sizes[3]
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, chunk_layers=N.MAX_CHUNK_LAYERS + 1))) == 0
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, chunk_layers=-1))) == 0
    # the shared-memory tiles hold one layer's MPO only
    assert lib.dcs_arena_bytes(ctypes.byref(_cfg(N, chi_max=8, kernel_path=N.PATH_SHARED,
                                                 chunk_layers=2))) == 0
    ctx = ctypes.c_void_p()
    assert lib.dcs_create(ctypes.byref(ctx), ctypes.byref(_cfg(N, kernel_path=N.PATH_SHARED,
                                                               chunk_layers=2)),
                          None, 0, None) == N.ERR_UNSUPPORTED
    assert lib.dcs_create(ctypes.byref(ctx), ctypes.byref(_cfg(N, chunk_layers=5)), None, 0,
                          None) == N.ERR_INVALID


def test_encode_ops_round_trip():
    import numpy as np
    import circuits as C
    from paper_2609_26516_b300.sim import encode_ops
    from paper_2609_26516_b300 import _native as N
    circ = C.teleport(1)
    arr = encode_ops(circ.ops)
    g = circ.ops[2]  # CNOT(1, 2)
    d = arr[2]
    assert d.kind == N.OP_GATE2 and (d.q0, d.q1) == (1, 2)
    m = np.array(d.m[:32]).reshape(16, 2)
    np.testing.assert_array_equal(m[:, 0] + 1j * m[:, 1], g.matrix.reshape(-1))
    cx = arr[7]
    assert cx.cond.op == N.COND_XOR and cx.cond.mask[0] == 0b10 and cx.cond.value == 1
    assert arr[5].kind == N.OP_MEASURE and arr[5].cbit == 0


def _encode_fieldwise(ops):
    """dcs_op records set one ctypes field at a time (the plain form of the binding's encoder)."""
    import numpy as np
    import circuits as C
    from paper_2609_26516_b300 import _native as N
    arr = (N.dcs_op * max(1, len(ops)))()
    for i, o in enumerate(ops):
        d = arr[i]
        if isinstance(o, C.Gate):
            m = np.asarray(o.matrix, dtype=np.complex128).reshape(-1)
            d.kind = N.OP_GATE1 if len(o.qubits) == 1 else N.OP_GATE2
            d.q0 = o.qubits[0]
            d.q1 = o.qubits[1] if len(o.qubits) == 2 else -1
            for k, z in enumerate(m):
                d.m[2 * k] = float(z.real)
                d.m[2 * k + 1] = float(z.imag)
            if o.cond is not None:
                d.cond.op = {"xor": N.COND_XOR, "and": N.COND_AND}[o.cond.op]
                d.cond.value = int(o.cond.value)
                for b in o.cond.bits:
                    d.cond.mask[b >> 6] |= 1 << (b & 63)
        else:
            d.kind = N.OP_MEASURE if isinstance(o, C.Measure) else N.OP_RESET
            d.q0, d.q1, d.cbit = o.qubit, -1, o.cbit
    return arr


def test_encode_ops_matches_fieldwise_encoding():
    import numpy as np
    import circuits as C
    from paper_2609_26516_b300.sim import encode_ops
    rng = np.random.default_rng(7)
    u2 = C.haar_unitary(rng, 2)
    extra = [C.Gate((3,), u2, cond=C.Cond((0, 65, 127, 300), "and", 0)),
             C.Gate((0, 1), C.haar_su4(rng), cond=C.Cond((64,), "xor", 1)),
             C.Reset(5, 511), C.Measure(2, 63)]
    for ops in (C.teleport(3).ops, C.ghz_dynamic(64).ops, C.brickwork(12, 6, 0.3, 5).ops,
                extra, []):
        fast, ref = encode_ops(ops), _encode_fieldwise(ops)
        assert len(fast) == len(ref)
        assert bytes(fast) == bytes(ref)


def test_bits_of_matches_plain_unpacking():
    import numpy as np
    from paper_2609_26516_b300.sim import bits_of
    rng = np.random.default_rng(3)
    cw = rng.integers(0, 2**63, size=(37, 8), dtype=np.int64).astype(np.uint64)
    cw[:, 1] |= np.uint64(1) << np.uint64(63)
    for n_bits in (1, 63, 64, 65, 200, 512):
        got = bits_of(cw, n_bits)
        want = np.array([[(int(cw[i, b >> 6]) >> (b & 63)) & 1 for b in range(n_bits)]
                         for i in range(cw.shape[0])], dtype=np.uint8)
        assert got.dtype == np.uint8 and got.shape == (37, n_bits)
        np.testing.assert_array_equal(got, want)


def test_noalloc_argument_checks_need_no_device(lib):
    # sizes beyond the fixed scratch and invalid arguments are refused before any CUDA call
    from paper_2609_26516_b300 import _native as N
    arr = (N.dcs_op * 1)()
    d = ctypes.c_void_p(1)  # never dereferenced: every call below returns first

    def call(n=8, chi=8, sweeps=2, n_gates=0, centre=0, gates=arr):
        return lib.dcs_compress_noalloc(n, chi, 1e-10, sweeps, gates, n_gates, None, d, d,
                                        centre, d, d, None, d, None)

    assert call(n=65) == N.ERR_OOM
    assert call(chi=16) == N.ERR_OOM
    assert call(n_gates=257) == N.ERR_OOM
    assert call(sweeps=0) == N.ERR_INVALID
    assert call(centre=8) == N.ERR_INVALID
    assert call(n_gates=1) == N.ERR_INVALID  # record of kind 0: not a gate
    g = (N.dcs_op * 1)()
    g[0].kind, g[0].q0, g[0].q1 = N.OP_GATE1, 0, -1
    g[0].m[0] = g[0].m[6] = 1.0
    g[0].cond.op = 7  # neither NONE, XOR nor AND
    assert call(n_gates=1, gates=g) == N.ERR_INVALID


def test_list_calls_refuse_a_null_context(lib):
    # the sharded-ensemble and shot-fork calls answer before any device access
    from paper_2609_26516_b300 import _native as N
    keep = (ctypes.c_uint8 * 2)(1, 0)
    assert lib.dcs_branch_keep(None, keep, 2) == N.ERR_INVALID
    assert lib.dcs_fork_shots(None, 4) == N.ERR_INVALID
    buf = (ctypes.c_uint8 * 64)()
    cw = (ctypes.c_uint64 * N.CWORDS)()
    assert lib.dcs_branch_append(None, buf, 64, 0.5, 1.0, cw, 0) == N.ERR_INVALID
