"""dcs_compress_noalloc against dcs_apply_layer.

The allocation-free call serves callers that cannot allocate device memory (a framework
that owns the GPU through its own pool, or a section where cudaMalloc is not allowed).  Here
the test allocates the input and output buffers itself, as such a caller would hand them
over, and checks two calls in a row against the context path: the first compresses a state
prepared by the context path, the second compresses the first call's output.

This file is collected last so a run that stops at its first failure has run every other
test already; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import circuits as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATE_TOL = 1e-6
F_TOL = 1e-6


def _overlap(A, B):
    E = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(A, B):
        # E'[u, v] = sum_{x, s, y} conj(a[x, s, u]) E[x, y] b[y, s, v], as two products
        t = np.tensordot(E, np.asarray(b, dtype=np.complex128), axes=(1, 0))
        E = np.tensordot(np.conj(np.asarray(a, dtype=np.complex128)), t, axes=([0, 1], [0, 1]))
    return E[0, 0]


def _fid(A, B):
    return abs(_overlap(A, B)) ** 2 / (_overlap(A, A).real * _overlap(B, B).real)


def test_noalloc_matches_context_path_two_calls():
    from paper_2609_26516_b300 import Simulator, _native as N
    from paper_2609_26516_b300.sim import encode_ops

    n, chi, tol, sweeps = 10, 8, 1e-10, 2
    circ = C.brickwork(n, 6, 0.3, 7)
    ops = circ.ops
    # the prefix prepares a state (with measurements and a classical register); the last two
    # runs of gates between measurement groups are the two calls
    runs, run = [], []
    for k, o in enumerate(ops):
        if isinstance(o, C.Measure):
            if run:
                runs.append(run)
            run = []
        else:
            run.append(k)
    if run:
        runs.append(run)
    layer_a, layer_b = runs[-2], runs[-1]

    def chunk_of(idx):
        # a run holds the previous layer's conditional gates and the next two-qubit layer:
        # one chunk (no qubit carries two two-qubit gates)
        return [ops[k] for k in idx]

    sim = Simulator(n, chi, 1, circ.n_cbits, tol=tol, sweeps=sweeps, seed=3)
    sim.init_state(1)
    sim.run_circuit(ops[: layer_a[0]])
    bits = sim.results()["cwords"][0]
    creg = (ctypes.c_uint64 * N.CWORDS)(*[int(x) for x in bits])
    bonds, centre, T = sim.export_mps(0)

    Cc = 4 if chi <= 4 else 8
    stride = 2 * Cc * Cc

    def to_dev(Ts):
        buf = np.zeros(n * stride, dtype=np.complex64)
        for j, t in enumerate(Ts):
            buf[j * stride: j * stride + t.size] = t.reshape(-1)
        return torch.from_numpy(buf).cuda()

    def from_dev(buf, bnd):
        h = buf.cpu().numpy()
        return [h[j * stride: j * stride + bnd[j] * 2 * bnd[j + 1]].reshape(bnd[j], 2, bnd[j + 1])
                for j in range(n)]

    ket = to_dev(T)
    ket_bonds = torch.tensor(np.asarray(bonds, dtype=np.int32), device="cuda")
    ket_centre = int(centre)
    lib = N.load()
    stream = torch.cuda.current_stream()
    for call, idx in enumerate((layer_a, layer_b)):
        gates = chunk_of(idx)
        arr = encode_ops(gates)
        # reference: the context path on the same state
        fid_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        sim.apply_layer(gates, fid_ref)
        rb, rc, RT = sim.export_mps(0)
        # the allocation-free call (all buffers owned by the caller)
        bra = torch.zeros(n * stride, dtype=torch.complex64, device="cuda")
        bra_bonds = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
        bra_centre = torch.zeros(1, dtype=torch.int32, device="cuda")
        f = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = lib.dcs_compress_noalloc(
            n, chi, tol, sweeps, arr, len(gates), ctypes.cast(creg, ctypes.c_void_p),
            ctypes.c_void_p(ket.data_ptr()), ctypes.c_void_p(ket_bonds.data_ptr()), ket_centre,
            ctypes.c_void_p(bra.data_ptr()), ctypes.c_void_p(bra_bonds.data_ptr()),
            ctypes.c_void_p(bra_centre.data_ptr()), ctypes.c_void_p(f.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
        assert st == N.OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        nb = bra_bonds.cpu().numpy()
        assert list(nb) == list(rb), f"call {call}: bonds differ"
        assert int(bra_centre.item()) == int(rc)
        BT = from_dev(bra, nb)
        assert abs(f.item() - fid_ref.item()) < F_TOL
        assert _fid(BT, RT) >= 1 - STATE_TOL
        # the next call starts from this call's output
        ket, ket_bonds, ket_centre = bra, bra_bonds, int(bra_centre.item())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2609_26516_b300 import _native as N

    lib = N.load()
    arr = (N.dcs_op * 1)()
    dummy = ctypes.c_void_p(1)
    assert lib.dcs_compress_noalloc(65, 8, 1e-10, 2, arr, 0, None, dummy, dummy, 0, dummy,
                                    dummy, None, dummy, None) == N.ERR_OOM
    assert lib.dcs_compress_noalloc(8, 16, 1e-10, 2, arr, 0, None, dummy, dummy, 0, dummy,
                                    dummy, None, dummy, None) == N.ERR_OOM
    assert lib.dcs_compress_noalloc(8, 8, 1e-10, 0, arr, 0, None, dummy, dummy, 0, dummy,
                                    dummy, None, dummy, None) == N.ERR_INVALID


def test_noalloc_reports_malformed_ket_bonds():
    # a ket bond above the site capacity (Cc = 8 for chi_max = 8) is caught on the device
    # before any tensor is indexed: bra_bonds[0] = 0, bra_centre = -1, f = NaN
    from paper_2609_26516_b300 import _native as N
    from paper_2609_26516_b300.sim import encode_ops

    n, chi, Cc = 6, 8, 8
    stride = 2 * Cc * Cc
    lib = N.load()
    gates = [C.Gate((1, 2), C.haar_su4(np.random.default_rng(2)))]
    arr = encode_ops(gates)
    ket = torch.zeros(n * stride, dtype=torch.complex64, device="cuda")
    bra = torch.zeros_like(ket)
    for bad in ([1, 2, 4, Cc + 1, 4, 2, 1], [2, 2, 4, 4, 4, 2, 1], [1, 2, 0, 4, 4, 2, 1]):
        ket_bonds = torch.tensor(bad, dtype=torch.int32, device="cuda")
        bra_bonds = torch.full((n + 1,), 5, dtype=torch.int32, device="cuda")
        bra_centre = torch.zeros(1, dtype=torch.int32, device="cuda")
        f = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = lib.dcs_compress_noalloc(
            n, chi, 1e-10, 2, arr, len(gates), None, ctypes.c_void_p(ket.data_ptr()),
            ctypes.c_void_p(ket_bonds.data_ptr()), 0, ctypes.c_void_p(bra.data_ptr()),
            ctypes.c_void_p(bra_bonds.data_ptr()), ctypes.c_void_p(bra_centre.data_ptr()),
            ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == N.OK
        torch.cuda.synchronize()
        assert int(bra_bonds[0].item()) == 0 and int(bra_centre.item()) == -1
        assert np.isnan(f.item())
