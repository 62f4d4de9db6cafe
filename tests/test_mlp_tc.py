"""Tensor-core dense layer of the warm-start network (tcgen05, BF16 operands,
FP32 accumulation) against a plain PyTorch FP32 reference of the same op,
computed from the same BF16-rounded inputs."""
import ctypes as C

import numpy as np
import pytest

from paper_1803_07772_gb300 import hcran

pytestmark = pytest.mark.gpu

EPI_BIAS_RELU, EPI_BIAS_F32, EPI_RELU_MASK, EPI_F32 = 0, 1, 2, 3


def _dense(A, W, b, H, epi):
    import torch
    lib = hcran.load()
    T, Q = A.shape
    P = W.shape[0]
    f32 = epi in (EPI_BIAS_F32, EPI_F32)
    out = torch.empty((T, P), dtype=torch.float32 if f32 else torch.bfloat16, device=A.device)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    rc = lib.hcran_mlp_dense(ptr(A), ptr(W), ptr(b), ptr(H), T, Q, P, epi, ptr(out), None)
    assert rc == 0
    failed = C.c_int32(-1)
    assert lib.hcran_mlp_tc_status(C.byref(failed)) == 0
    assert failed.value == 0
    return out


@pytest.mark.parametrize("T,Q,P", [(1, 16, 16), (300, 256, 256), (1000, 16, 256), (777, 256, 16),
                                   (128 * 152 + 5, 256, 256)])
@pytest.mark.parametrize("epi", [EPI_BIAS_RELU, EPI_BIAS_F32, EPI_RELU_MASK, EPI_F32])
def test_dense_layer_matches_fp32_reference(T, Q, P, epi):
    import torch
    g = torch.Generator().manual_seed(1000 * T + 10 * Q + P + epi)
    A = (torch.randn(T, Q, generator=g) * 0.5).to(torch.bfloat16)
    W = (torch.randn(P, Q, generator=g) / Q ** 0.5).to(torch.bfloat16)
    b = torch.randn(P, generator=g) * 0.1
    H = torch.randn(T, P, generator=g).to(torch.bfloat16)
    ref = A.float() @ W.float().T
    if epi in (EPI_BIAS_RELU, EPI_BIAS_F32):
        ref = ref + b
    if epi == EPI_BIAS_RELU:
        ref = torch.relu(ref)
    if epi == EPI_RELU_MASK:
        ref = ref * (H.float() > 0)
    dev = "cuda:0"
    out = _dense(A.to(dev), W.to(dev), b.to(dev), H.to(dev) if epi == EPI_RELU_MASK else None, epi).cpu().float()
    if epi in (EPI_BIAS_F32, EPI_F32):
        # FP32 accumulation in another order: relative ~1e-6 of the row scale
        tol = 1e-5 * (A.float().abs() @ W.float().abs().T) + 1e-6
    else:
        # then one rounding to BF16 (8 significant bits)
        tol = 2.0 ** -8 * ref.abs() + 1e-5 * (A.float().abs() @ W.float().abs().T) + 1e-6
    err = (out - ref).abs()
    assert torch.all(err <= tol), float((err / (tol + 1e-30)).max())
