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


def _bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _rounded_weights(theta):
    """The kernels multiply with BF16 copies of the weights and add FP32 biases."""
    from oracle import mlp_oracle as mo
    return mo.pack([(_bf16(W), b) for W, b in mo.unpack(theta)])


def _batch(T, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((T, 16), np.float32)
    x[:, :4] = rng.normal(0, 1, (T, 4))
    target = np.zeros((T, 16), np.float32)
    target[:, :3] = rng.normal(0, 1, (T, 3))
    mask = np.zeros((T, 16), np.float32)
    mask[:, :3] = (rng.random((T, 3)) < 0.8)
    return x, target, mask


def test_network_forward_and_gradients_match_fp64_oracle():
    """Forward and backward of the whole network on the tensor cores against
    the FP64 oracle with the same BF16 inputs and BF16-rounded weights.  The
    kernels round each hidden activation and each back-propagated dZ to BF16
    (8 significant bits), which bounds the agreement at a few percent."""
    import torch
    from oracle import mlp_oracle as mo
    from paper_1803_07772_gb300.mlp import MLP
    T = 1000
    net = MLP(seed=11, max_rows=T)
    theta = net.params().astype(np.float64)
    x, target, mask = _batch(T, 5)
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    out = torch.empty((T, 16), dtype=torch.float32, device="cuda")
    net.forward(xd, out)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(out, torch.from_numpy(target).cuda(), torch.from_numpy(mask).cuda(), loss)
    net.backward(xd)
    g_gpu = net.grads().astype(np.float64)
    assert not net.tc_failed()
    th = _rounded_weights(theta)
    xo = _bf16(x)
    o_orc, _ = mo.forward(th, xo)
    l_orc, g_orc = mo.loss_and_grad(th, xo, target.astype(np.float64), mask.astype(np.float64))
    o_gpu = out.cpu().numpy().astype(np.float64)
    scale = np.sqrt(np.mean(o_orc[:, :3] ** 2))
    print("forward max err / rms", np.max(np.abs(o_gpu[:, :3] - o_orc[:, :3])) / scale)
    assert np.max(np.abs(o_gpu[:, :3] - o_orc[:, :3])) <= 0.03 * scale
    assert abs(float(loss.item()) - l_orc) <= 0.02 * l_orc
    gl_gpu, gl_orc = mo.unpack(g_gpu), mo.unpack(g_orc)
    for i in range(4):
        for a, b, name in ((gl_gpu[i][0], gl_orc[i][0], "W%d" % (i + 1)), (gl_gpu[i][1], gl_orc[i][1], "b%d" % (i + 1))):
            a, b = a.ravel(), b.ravel()
            nb = np.linalg.norm(b)
            if nb == 0:
                assert np.linalg.norm(a) == 0
                continue
            rel = np.linalg.norm(a - b) / nb
            cos = float(a @ b / (np.linalg.norm(a) * nb))
            print(name, "rel", rel, "cos", cos)
            assert rel <= 0.05 and cos >= 0.998, (name, rel, cos)


def test_training_reduces_the_loss():
    """Adam on a fixed regression target (a random teacher network) for 150
    steps: the tensor-core training loop must drive the loss down."""
    import torch
    from oracle import mlp_oracle as mo
    from paper_1803_07772_gb300.mlp import MLP
    T = 2048
    teacher = MLP(seed=99, max_rows=T)
    th_t = teacher.params().astype(np.float64)
    teacher.close()
    x, _, mask = _batch(T, 7)
    tgt, _ = mo.forward(th_t, _bf16(x))
    target = np.zeros((T, 16), np.float32)
    target[:, :3] = tgt[:, :3] * 10.0
    mask[:, :3] = 1.0
    net = MLP(seed=3, max_rows=T)
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    td, md = torch.from_numpy(target).cuda(), torch.from_numpy(mask).cuda()
    out = torch.empty((T, 16), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for step in range(150):
        net.forward(xd, out)
        net.loss_grad(out, td, md, loss)
        net.backward(xd)
        net.adam(1e-3)
        if step % 30 == 0 or step == 149:
            hist.append(float(loss.item()))
    print("loss", hist)
    assert not net.tc_failed()
    assert hist[-1] < 0.3 * hist[0]
