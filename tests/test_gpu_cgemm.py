"""dcs_cgemm (the contraction primitive of the large-bond kernels) against PyTorch complex128
matmul: FP32 SIMT, tcgen05 tensor-core 3xTF32 and BF16x3 modes, ragged sizes, strided and
conjugated operands.  Bars: relative Frobenius error <= 1e-5 (SIMT, 3xTF32 up to K = 500)
and <= 3e-5 for BF16x3, whose split x = hi + lo keeps x to 2^-18 relative and drops a
lo lo term of at most 2^-18 |a||b| per product (three such terms: <= 1.2e-5 per product).
The tensor modes also round once per MMA into the FP32 accumulator in tensor memory, an
error that grows with K (measured: 3xTF32 1.4e-6 at K = 64, 1.5e-5 at K = 1024, 5.9e-5 at
K = 4096; SIMT 2e-7, 8e-7, 1.6e-6): the long-K test bounds it."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(mode, batch, M, N, K, transA=False, transB=False, conjA=False, conjB=False, seed=0):
    from paper_2609_26516_b300 import _native as N_
    lib = N_.load()
    g = torch.Generator(device="cpu").manual_seed(seed)
    # stored A is M x K (row-major) or K x M when transA; likewise B
    a_shape = (batch, K, M) if transA else (batch, M, K)
    b_shape = (batch, N, K) if transB else (batch, K, N)
    A = torch.complex(torch.randn(a_shape, generator=g), torch.randn(a_shape, generator=g)).to(torch.complex64).cuda()
    B = torch.complex(torch.randn(b_shape, generator=g), torch.randn(b_shape, generator=g)).to(torch.complex64).cuda()
    C = torch.zeros((batch, M, N), dtype=torch.complex64, device="cuda")
    sam, sak = (1, M) if transA else (K, 1)
    sbk, sbn = (1, K) if transB else (N, 1)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.dcs_cgemm(mode, batch, M, N, K,
                       ctypes.c_void_p(A.data_ptr()), sam, sak, A[0].numel(), int(conjA),
                       ctypes.c_void_p(B.data_ptr()), sbk, sbn, B[0].numel(), int(conjB),
                       ctypes.c_void_p(C.data_ptr()), N, 1, M * N,
                       ctypes.c_void_p(err.data_ptr()),
                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a = A.to(torch.complex128)
    b = B.to(torch.complex128)
    if transA:
        a = a.transpose(1, 2)
    if transB:
        b = b.transpose(1, 2)
    if conjA:
        a = a.conj()
    if conjB:
        b = b.conj()
    ref = a @ b
    rel = (C.to(torch.complex128) - ref).norm() / ref.norm()
    return float(rel)


BAR = {0: 1e-5, 1: 1e-5, 2: 3e-5}
MODES = [0, 1, 2]
IDS = ["simt", "tensor", "tensor_bf16x3"]


@pytest.mark.parametrize("mode", MODES, ids=IDS)
@pytest.mark.parametrize("shape", [(1, 128, 128, 8), (2, 128, 128, 64), (3, 200, 130, 37),
                                   (1, 64, 300, 500), (1, 7, 5, 3)])
def test_cgemm_plain(mode, shape):
    assert _run(mode, *shape) <= BAR[mode]


@pytest.mark.parametrize("mode", MODES, ids=IDS)
def test_cgemm_long_k(mode):
    # the site-contraction shape of chi 256 (K = 1024) and a four times longer product: the
    # tensor modes' accumulation error grows about linearly with K, the SIMT mode's slowly
    bars = {0: 8e-6, 1: 1.2e-4, 2: 1.2e-4}
    e1 = _run(mode, 1, 512, 256, 1024, transB=True, seed=5)
    e4 = _run(mode, 1, 256, 256, 4096, seed=5)
    assert e1 <= bars[mode] / 4 and e4 <= bars[mode]


@pytest.mark.parametrize("mode", MODES, ids=IDS)
def test_cgemm_strided_and_conjugated(mode):
    assert _run(mode, 2, 150, 90, 70, transA=True, conjA=True) <= BAR[mode]
    assert _run(mode, 2, 150, 90, 70, transB=True, conjB=True) <= BAR[mode]
    assert _run(mode, 1, 260, 140, 96, transA=True, transB=True, conjA=True, conjB=True) <= BAR[mode]

