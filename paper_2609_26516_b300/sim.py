"""Python binding of libdcs: the same calls as the C ABI (include/dcs.h), with PyTorch
providing the device arena and the stream.  Argument marshalling only: every step of the
simulation runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
from typing import Iterable, List, Optional, Sequence

import numpy as np
import torch

from . import _native as N


def topk_select_global(p, M: int, p_min: float = 0.0) -> np.ndarray:
    """dcs_topk_select_global (host-only): the keep mask (uint8 per entry) of TopKByWeight and
    adaptive pruning over p, every rank's branch probabilities in rank order."""
    lib = N.load()
    pa = np.ascontiguousarray(p, dtype=np.float64)
    keep = np.zeros(pa.size, dtype=np.uint8)
    st = lib.dcs_topk_select_global(pa.ctypes.data_as(ctypes.c_void_p), int(pa.size), int(M),
                                    float(p_min), keep.ctypes.data_as(ctypes.c_void_p))
    if st != N.OK:
        raise DCSError(st, "dcs_topk_select_global: invalid arguments")
    return keep


class DCSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libdcs {N.STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _op_dtype() -> np.dtype:
    """NumPy view of one dcs_op record, field offsets taken from the ctypes declaration."""
    co = N.dcs_op.cond.offset
    return np.dtype({
        "names": ["kind", "q0", "q1", "cbit", "m", "mask", "cop", "cval"],
        "formats": [np.int32, np.int32, np.int32, np.int32, (np.float64, 32),
                    (np.uint64, N.CWORDS), np.int32, np.int32],
        "offsets": [N.dcs_op.kind.offset, N.dcs_op.q0.offset, N.dcs_op.q1.offset,
                    N.dcs_op.cbit.offset, N.dcs_op.m.offset, co + N.dcs_cond.mask.offset,
                    co + N.dcs_cond.op.offset, co + N.dcs_cond.value.offset],
        "itemsize": ctypes.sizeof(N.dcs_op)})


_OP_DTYPE = _op_dtype()
_COND_OPS = {"xor": N.COND_XOR, "and": N.COND_AND, "or": N.COND_OR, "table": N.COND_TABLE}


def encode_ops(ops: Sequence) -> ctypes.Array:
    """circuits.Gate / Measure / Reset records -> dcs_op array (filled column by column
    through a NumPy view of the same bytes; the ctypes array keeps that buffer alive)."""
    from circuits import Gate, Measure, Reset  # input records only

    n = len(ops)
    rec = np.zeros(max(1, n), dtype=_OP_DTYPE)
    kind = np.zeros(n, dtype=np.int32)
    q0 = np.zeros(n, dtype=np.int32)
    q1 = np.full(n, -1, dtype=np.int32)
    cbit = np.zeros(n, dtype=np.int32)
    g1, m1, g2, m2, conds = [], [], [], [], []
    for i, o in enumerate(ops):
        if isinstance(o, Gate):
            if len(o.qubits) == 1:
                kind[i] = N.OP_GATE1
                q0[i] = o.qubits[0]
                g1.append(i)
                m1.append(o.matrix)
            else:
                kind[i] = N.OP_GATE2
                q0[i], q1[i] = o.qubits
                g2.append(i)
                m2.append(o.matrix)
            if o.cond is not None:
                conds.append((i, o.cond))
        elif isinstance(o, (Measure, Reset)):
            kind[i] = N.OP_MEASURE if isinstance(o, Measure) else N.OP_RESET
            q0[i] = o.qubit
            cbit[i] = o.cbit
        else:
            raise TypeError(o)
    if n:
        rec["kind"][:n], rec["q0"][:n], rec["q1"][:n], rec["cbit"][:n] = kind, q0, q1, cbit
    m = rec["m"]
    if g1:
        m[g1, :8] = np.asarray(m1, dtype=np.complex128).reshape(len(g1), 4).view(np.float64)
    if g2:
        m[g2, :32] = np.asarray(m2, dtype=np.complex128).reshape(len(g2), 16).view(np.float64)
    if conds:
        words = np.zeros((len(conds), N.CWORDS), dtype=np.uint64)
        for r, (_, cd) in enumerate(conds):
            w = [0] * N.CWORDS
            for b in cd.bits:
                w[b >> 6] |= 1 << (b & 63)
            words[r] = w
        rows = [i for i, _ in conds]
        rec["mask"][rows] = words
        rec["cop"][rows] = [_COND_OPS[cd.op] for _, cd in conds]
        # a truth table is a 32-bit word stored in the int32 field
        rec["cval"][rows] = [int(np.uint32(int(cd.value)).view(np.int32)) for _, cd in conds]
    return (N.dcs_op * rec.shape[0]).from_buffer(rec)


def bits_of(cwords: np.ndarray, n_bits: int) -> np.ndarray:
    """Unpack [n, CWORDS] uint64 registers into [n, n_bits] uint8 (bit b of the register is
    bit b & 63 of word b >> 6)."""
    cw = np.ascontiguousarray(np.asarray(cwords, dtype=np.uint64).astype("<u8", copy=False))
    raw = cw.view(np.uint8).reshape(cw.shape[0], -1)[:, : (n_bits + 7) // 8]
    bits = np.unpackbits(raw, axis=1, bitorder="little")
    return np.ascontiguousarray(bits[:, :n_bits])


class Simulator:
    """One libdcs context: n_slots shots (single-path) or a branch pool (multi-path)."""

    def __init__(self, n_qubits: int, chi_max: int, n_slots: int, n_cbits: int,
                 tol: float = 1e-10, sweeps: int = 2, seed: int = 0, chunk_k: int = 0,
                 device: str = "cuda:0", stream: Optional[torch.cuda.Stream] = None,
                 kernel_path: int = 0, precision: int = 0, chunk_layers: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("libdcs needs a CUDA device; there is no CPU path")
        self.lib = N.load()
        self.cfg = N.dcs_config(n_qubits=n_qubits, chi_max=chi_max, tol=tol, sweeps=sweeps,
                                chunk_k=chunk_k, chunk_layers=chunk_layers,
                                precision=precision, kernel_path=kernel_path,
                                n_cbits=n_cbits,
                                n_slots=n_slots, seed=seed)
        self.device = torch.device(device)
        nbytes = self.lib.dcs_arena_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise DCSError(N.ERR_INVALID if chi_max <= N.MAX_CHI else N.ERR_UNSUPPORTED,
                           "configuration rejected")
        self.arena_bytes = nbytes
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        self._base = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = ctypes.c_void_p()
        st = self.lib.dcs_create(ctypes.byref(self.ctx), ctypes.byref(self.cfg),
                                 ctypes.c_void_p(self._base), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if st != N.OK:
            raise DCSError(st, "dcs_create failed")
        self.n_qubits, self.n_slots, self.n_cbits = n_qubits, n_slots, n_cbits

    # ------------------------------------------------------------------ plumbing
    def _check(self, st: int):
        if st != N.OK:
            raise DCSError(st, self.lib.dcs_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.dcs_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(self.lib.dcs_kernel_launches(self.ctx))

    @property
    def bytes_uploaded(self) -> int:
        return int(self.lib.dcs_bytes_uploaded(self.ctx))

    def counters(self):
        """(compression steps run, one-site sweeps run) since the last init_state."""
        a, b = ctypes.c_uint64(0), ctypes.c_uint64(0)
        self._check(self.lib.dcs_get_counters(self.ctx, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    # ------------------------------------------------------------------ calls
    def init_state(self, n_active: int, multipath: bool = False, shot0: int = 0):
        self._check(self.lib.dcs_init_state(self.ctx, n_active, int(multipath), shot0))

    def fork_shots(self, n_active: int):
        """dcs_fork_shots: copy the one shot's state (its measurement-free prefix run once)
        into n_active shots, each with its own sampler counter."""
        self._check(self.lib.dcs_fork_shots(self.ctx, n_active))

    def run_circuit(self, circ_or_ops, meas_idx0: int = 0, max_branches: int = 0):
        ops = circ_or_ops.ops if hasattr(circ_or_ops, "ops") else circ_or_ops
        arr = encode_ops(ops)
        self._check(self.lib.dcs_run_circuit(self.ctx, arr, len(ops), meas_idx0, max_branches))

    def run_encoded(self, arr, n_ops: int, meas_idx0: int = 0, max_branches: int = 0):
        self._check(self.lib.dcs_run_circuit(self.ctx, arr, n_ops, meas_idx0, max_branches))

    def apply_layer(self, gates: Sequence, fid_out: Optional[torch.Tensor] = None):
        arr = encode_ops(gates)
        ptr = ctypes.c_void_p(fid_out.data_ptr()) if fid_out is not None else None
        self._check(self.lib.dcs_apply_layer(self.ctx, arr, len(gates), ptr))

    def measure_prob(self, qubit: int) -> torch.Tensor:
        out = torch.full((self.n_slots,), float("nan"), dtype=torch.float64, device=self.device)
        self._check(self.lib.dcs_measure_prob(self.ctx, qubit, ctypes.c_void_p(out.data_ptr())))
        return out

    def measure_sample(self, qubit: int, cbit: int, meas_idx: int):
        self._check(self.lib.dcs_measure_sample(self.ctx, qubit, cbit, meas_idx))

    def collapse(self, qubit: int, cbit: int, outcomes: Iterable[int]):
        o = np.zeros(self.n_slots, dtype=np.uint8)
        vals = np.asarray(list(outcomes), dtype=np.uint8)
        o[: len(vals)] = vals
        buf = (ctypes.c_uint8 * self.n_slots).from_buffer_copy(o.tobytes())
        self._check(self.lib.dcs_collapse(self.ctx, qubit, cbit, buf))

    def branch_split(self, qubit: int, cbit: int, eps: float = 1e-12):
        self._check(self.lib.dcs_branch_split(self.ctx, qubit, cbit, eps))

    def set_pruning(self, p_min: float):
        self._check(self.lib.dcs_set_pruning(self.ctx, p_min))

    def branch_topk(self, M: int):
        self._check(self.lib.dcs_branch_topk(self.ctx, M))

    def branch_keep(self, keep):
        """dcs_branch_keep: keep entry i of the active list iff keep[i] is true."""
        k = np.ascontiguousarray(np.asarray(keep) != 0, dtype=np.uint8)
        self._check(self.lib.dcs_branch_keep(self.ctx, k.ctypes.data_as(ctypes.c_void_p),
                                             int(k.size)))

    def results(self) -> dict:
        S = self.n_slots
        p = np.zeros(S, dtype=np.float64)
        F = np.zeros(S, dtype=np.float64)
        cw = np.zeros((S, N.CWORDS), dtype=np.uint64)
        fl = np.zeros(S, dtype=np.uint8)
        cnt = ctypes.c_int(0)
        self._check(self.lib.dcs_get_results(
            self.ctx, p.ctypes.data_as(ctypes.c_void_p), F.ctypes.data_as(ctypes.c_void_p),
            cw.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt),
            fl.ctypes.data_as(ctypes.c_void_p)))
        n = cnt.value
        return {"n_active": n, "p": p[:n], "F": F[:n], "cwords": cw[:n], "flags": fl[:n],
                "bits": bits_of(cw[:n], self.n_cbits)}

    def bonds(self) -> np.ndarray:
        """[n_active, n_qubits + 1] bond dimensions of the active slots, in list order."""
        out = np.zeros((self.n_slots, self.n_qubits + 1), dtype=np.int32)
        cnt = ctypes.c_int(0)
        self._check(self.lib.dcs_get_bonds(self.ctx, out.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(cnt)))
        return out[: cnt.value]

    def export_mps_bytes(self, pos: int) -> bytes:
        """dcs_export_mps of active slot ``pos`` as the raw bytes of its format."""
        size = ctypes.c_size_t(0)
        self._check(self.lib.dcs_export_mps(self.ctx, pos, None, ctypes.byref(size)))
        buf = (ctypes.c_uint8 * size.value)()
        self._check(self.lib.dcs_export_mps(self.ctx, pos, buf, ctypes.byref(size)))
        return bytes(buf)

    def branch_append(self, raw: bytes, p: float, F: float, cwords, flags: int = 0):
        """dcs_branch_append: one branch (MPS bytes of export_mps_bytes, p, F, register words,
        flags) at the end of the active list."""
        cw = np.zeros(N.CWORDS, dtype=np.uint64)
        src = np.asarray(cwords, dtype=np.uint64).ravel()
        cw[: src.size] = src
        buf = (ctypes.c_uint8 * len(raw)).from_buffer_copy(raw)
        self._check(self.lib.dcs_branch_append(self.ctx, buf, len(raw), float(p), float(F),
                                               cw.ctypes.data_as(ctypes.c_void_p),
                                               int(flags) & 0xFF))

    def export_mps(self, pos: int):
        """(bonds, centre, [tensors [chi_l, 2, chi_r] complex64]) of active slot ``pos``."""
        size = ctypes.c_size_t(0)
        self._check(self.lib.dcs_export_mps(self.ctx, pos, None, ctypes.byref(size)))
        buf = (ctypes.c_uint8 * size.value)()
        self._check(self.lib.dcs_export_mps(self.ctx, pos, buf, ctypes.byref(size)))
        raw = bytes(buf)
        n = int(np.frombuffer(raw, dtype=np.int32, count=1)[0])
        bonds = np.frombuffer(raw, dtype=np.int32, count=n + 1, offset=4).copy()
        centre = int(np.frombuffer(raw, dtype=np.int32, count=1, offset=4 * (n + 2))[0])
        off = 4 * (n + 3)
        T: List[np.ndarray] = []
        for j in range(n):
            cnt = int(bonds[j]) * 2 * int(bonds[j + 1])
            t = np.frombuffer(raw, dtype=np.complex64, count=cnt, offset=off).copy()
            T.append(t.reshape(int(bonds[j]), 2, int(bonds[j + 1])))
            off += cnt * 8
        return bonds, centre, T

    def import_mps(self, pos: int, tensors: Sequence[np.ndarray], centre: int):
        n = len(tensors)
        bonds = [1] + [int(t.shape[2]) for t in tensors[:-1]] + [1]
        parts = [np.array([n], dtype=np.int32).tobytes(), np.array(bonds, dtype=np.int32).tobytes(),
                 np.array([centre], dtype=np.int32).tobytes()]
        parts += [np.ascontiguousarray(t, dtype=np.complex64).tobytes() for t in tensors]
        raw = b"".join(parts)
        buf = (ctypes.c_uint8 * len(raw)).from_buffer_copy(raw)
        self._check(self.lib.dcs_import_mps(self.ctx, pos, buf, len(raw)))


def mps_to_dense(tensors: Sequence[np.ndarray]) -> np.ndarray:
    """Contract exported MPS tensors into the 2^n amplitude vector (small n, host FP64)."""
    v = np.asarray(tensors[0], dtype=np.complex128)
    for t in tensors[1:]:
        v = np.tensordot(v, np.asarray(t, dtype=np.complex128), axes=([v.ndim - 1], [0]))
    return v.reshape(-1)
