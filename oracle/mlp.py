"""Learned colour estimator: the plain FP64 reference of the network.

TEST INFRASTRUCTURE ONLY (see the package header).

The network maps the features of one overlap pair (three channel histograms
of side i then side j, each scaled by 256 / count) to M - I and the three
balance slopes (the labels ``oracle.pairs`` computes). Layers are dense,
y = x W^T + b with W stored [out][in], ReLU after every layer except the last.
The loss is the mean squared error over the normalised targets
t_n = (t - mu) / sd. Training uses Adam with bias correction.

The GPU keeps weights, activations and gradient signals in bfloat16 and
accumulates in float32. With ``bf16=True`` this module rounds at exactly the
same points (the input, the weights, every hidden activation, the output
gradient and every back-propagated gradient signal) and does everything else
in float64, so that the only difference left is the accumulation precision.
With ``bf16=False`` it is the exact float64 network, which the finite
difference pin checks.

Parameter layout (flat float32/float64 vector): layer by layer, W [out][in]
row-major then b [out]. The network used by the library pads its last layer
from 12 to 16 outputs; ``sizes`` gives the padded widths and ``n_out`` the
outputs the loss sees.
"""
from __future__ import annotations

import numpy as np

SIZES = (1536, 512, 512, 256, 16)
N_OUT = 12


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through float32, as a
    float64 array. bfloat16 keeps the top 16 bits of a float32."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, sizes=SIZES):
    """Split a flat parameter vector into [(W, b), ...] float64 arrays."""
    p = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = p[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = p[o:o + n_out]
        o += n_out
        out.append((W, b))
    assert o == p.size, "parameter count does not match the layer sizes"
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in layers])


def forward(params, X, sizes=SIZES, bf16=True):
    """Network output (batch, sizes[-1]) in normalised units, and the list of
    layer inputs (needed by the backward pass)."""
    layers = unpack(params, sizes)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    h = r(X)
    inputs = []
    for li, (W, b) in enumerate(layers):
        inputs.append(h)
        z = h @ r(W).T + b
        if li < len(layers) - 1:
            h = r(np.maximum(z, 0.0))
        else:
            h = z
    return h, inputs


def loss_and_grads(params, X, T, mu, sd, sizes=SIZES, n_out=N_OUT, bf16=True):
    """Mean squared error over batch x n_out normalised targets and its
    gradient with respect to every parameter (flat, same layout)."""
    layers = unpack(params, sizes)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Y, inputs = forward(params, X, sizes, bf16)
    batch = Y.shape[0]
    Tn = (np.asarray(T, dtype=np.float64) - np.asarray(mu)[:n_out]) / np.asarray(sd)[:n_out]
    D = Y[:, :n_out] - Tn
    loss = float(np.sum(D * D) / (batch * n_out))
    dz = np.zeros_like(Y)
    dz[:, :n_out] = 2.0 * D / (batch * n_out)
    dz = r(dz)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        x_in = inputs[li]
        grads[li] = (dz.T @ x_in, dz.sum(axis=0))
        if li > 0:
            dx = dz @ r(W)
            dz = r(np.where(inputs[li] > 0.0, dx, 0.0))
    return loss, pack(grads)


def adam_step(params, grads, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update with bias correction (step counts from 1). Returns the
    new (params, m, v)."""
    g = np.asarray(grads, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return np.asarray(params, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def residual(A, B, M_hat) -> float:
    """The fallback test of the learned estimator, float64: how much M_hat
    raises the least-squares error of Eq. 2 over the plain fit M* = A^-1 B,
    relative to the energy of the fitted colours,
    r = ||X (M_hat - M*)||^2 / ||X M*||^2 = tr(D^T A D) / tr(M*^T A M*),
    D = M_hat - M*, A = X^T X, B = X^T Y (the cross term vanishes at M*)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Ms = np.linalg.solve(A, B)
    D = np.asarray(M_hat, dtype=np.float64) - Ms
    den = float(np.trace(Ms.T @ A @ Ms))
    if den <= 0.0:
        return np.inf
    return float(np.trace(D.T @ A @ D) / den)
