"""FP64 CPU oracle of the warm-start network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: used by the tests to check the tensor-core
forward and backward of the network, never by the product path; it shares
no code with the CUDA kernels.

The network is the one the warm start uses: dims (16, 256, 256, 256, 16),
weights stored [out][in],

    H1 = relu(W1 x + b1), H2 = relu(W2 H1 + b2), H3 = relu(W3 H2 + b3),
    out = W4 H3 + b4,

and the training loss is the masked squared error of the first ``nout``
outputs averaged over the rows,

    L = (1/T) sum_t sum_{j < nout} mask[t, j] (out[t, j] - target[t, j])^2.

The backward is the chain rule written out layer by layer (dZ = dH * [Z > 0],
dW = dZ^T H_prev, db = column sums of dZ, dH_prev = dZ W).  Parameters travel
as one packed array [W1 b1 W2 b2 W3 b3 W4 b4], the layout of the C ABI.
"""
import numpy as np

DIMS = (16, 256, 256, 256, 16)


def unpack(theta):
    """Packed parameters -> list of (W [out][in], b [out]) in FP64."""
    theta = np.asarray(theta, dtype=np.float64)
    layers, o = [], 0
    for i in range(4):
        q, p = DIMS[i], DIMS[i + 1]
        W = theta[o:o + p * q].reshape(p, q)
        o += p * q
        b = theta[o:o + p]
        o += p
        layers.append((W, b))
    assert o == theta.size
    return layers


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def forward(theta, x):
    """out [T][16] and the pre-activations / activations of every layer."""
    layers = unpack(theta)
    h = np.asarray(x, dtype=np.float64)
    cache = [h]
    for i, (W, b) in enumerate(layers):
        z = h @ W.T + b
        if i < 3:
            h = np.maximum(z, 0.0)
            cache.append(h)
        else:
            h = z
    return h, cache


def loss_and_grad(theta, x, target, mask, nout=3):
    """Masked mean squared error and its gradient w.r.t. the packed parameters."""
    out, cache = forward(theta, x)
    T = out.shape[0]
    diff = np.zeros_like(out)
    diff[:, :nout] = (out[:, :nout] - target[:, :nout]) * mask[:, :nout]
    loss = float(np.sum(diff[:, :nout] * (out[:, :nout] - target[:, :nout])) / T)
    dz = 2.0 * diff / T                      # dL/dout
    layers = unpack(theta)
    grads = [None] * 4
    for i in range(3, -1, -1):
        W, _ = layers[i]
        h_prev = cache[i]
        grads[i] = (dz.T @ h_prev, dz.sum(axis=0))
        if i > 0:
            dh = dz @ W
            dz = dh * (h_prev > 0.0)
    return loss, pack(grads)
