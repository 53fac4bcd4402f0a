"""Pins of the learned estimator's oracle (oracle.mlp, oracle.pairs) against
things other than itself: a hand-computed network, central finite
differences of the float64 loss, torch's bfloat16 conversion and Adam, and
closed forms of the pair labels."""
import numpy as np
import pytest
import torch

from oracle import mlp as om
from oracle import pairs as opairs


def test_round_bf16_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e4, 1000), rng.uniform(-1e-30, 1e-30, 100),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 255.0, 256.5]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    got = om.round_bf16(x32)
    assert np.array_equal(got, ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert om.round_bf16(np.float32(1.0 + 2 ** -8)) == 1.0
    assert om.round_bf16(np.float32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6


def test_forward_hand_computed():
    # 2 -> 2 -> 1: h = relu(x W1^T + b1), y = h W2^T + b2
    W1 = np.array([[1.0, -1.0], [2.0, 0.5]])
    b1 = np.array([0.5, -10.0])
    W2 = np.array([[3.0, -2.0]])
    b2 = np.array([0.25])
    params = om.pack([(W1, b1), (W2, b2)])
    X = np.array([[3.0, 1.0], [1.0, 4.0]])
    # sample 0: z1 = (3-1+0.5, 6+0.5-10) = (2.5, -3.5) -> h = (2.5, 0) -> y = 7.5 + 0.25
    # sample 1: z1 = (1-4+0.5, 2+2-10) = (-2.5, -6) -> h = (0, 0) -> y = 0.25
    Y, _ = om.forward(params, X, sizes=(2, 2, 1), bf16=False)
    assert np.allclose(Y[:, 0], [7.75, 0.25], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    sizes = (7, 6, 5, 4, 6)
    n_out = 4                        # the last two outputs are padding, as in the library's layout
    n_params = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    params = rng.normal(0, 0.7, n_params)
    X = rng.normal(0, 1, (5, sizes[0]))
    T = rng.normal(0, 1, (5, n_out))
    mu = rng.normal(0, 0.3, n_out)
    sd = rng.uniform(0.5, 2.0, n_out)
    loss, g = om.loss_and_grads(params, X, T, mu, sd, sizes=sizes, n_out=n_out, bf16=False)
    h = 1e-6
    fd = np.zeros_like(params)
    for k in range(n_params):
        e = np.zeros_like(params)
        e[k] = h
        lp, _ = om.loss_and_grads(params + e, X, T, mu, sd, sizes=sizes, n_out=n_out, bf16=False)
        lm, _ = om.loss_and_grads(params - e, X, T, mu, sd, sizes=sizes, n_out=n_out, bf16=False)
        fd[k] = (lp - lm) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    # the loss itself: mean squared error on the normalised targets
    Y, _ = om.forward(params, X, sizes=sizes, bf16=False)
    assert np.isclose(loss, np.mean((Y[:, :n_out] - (T - mu) / sd) ** 2), rtol=1e-14)
    # padding outputs get no gradient
    W_last = g[-(sizes[-2] * sizes[-1] + sizes[-1]):-sizes[-1]].reshape(sizes[-1], sizes[-2])
    assert np.all(W_last[n_out:] == 0.0)


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    p0 = rng.normal(0, 1, 50)
    grads = [rng.normal(0, 1, 50) for _ in range(4)]
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step, g in enumerate(grads, 1):
        opt.zero_grad()
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = om.adam_step(p, g, m, v, step, 1e-2)
    assert np.allclose(p, tp.detach().numpy(), rtol=0, atol=1e-12)


def test_residual_closed_forms():
    A = np.array([[4.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 2.0]])
    M = np.array([[1.1, 0.0, 0.1], [0.0, 0.9, 0.0], [0.2, 0.0, 1.0]])
    B = A @ M
    assert abs(om.residual(A, B, M)) < 1e-28
    # A = 2 I, M* = I, M_hat = 1.01 I: tr(D^T A D) / tr(M*^T A M*) = 3 * 2e-4 / 6
    A = np.diag([2.0, 2.0, 2.0])
    B = A @ np.eye(3)
    assert np.isclose(om.residual(A, B, np.eye(3) * 1.01), 1e-4, rtol=1e-10)


def test_residual_is_the_excess_least_squares_error():
    """Against the literal Eq. 2 objective on a stacked system: the extra
    error of M_hat over the least-squares M*, relative to ||X M*||^2."""
    rng = np.random.default_rng(8)
    X = rng.uniform(0, 255, (500, 3))
    Y = X @ np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, 0.02, 1.1]]) + rng.normal(0, 3, (500, 3))
    Ms = np.linalg.lstsq(X, Y, rcond=None)[0]
    M_hat = Ms + rng.normal(0, 0.01, (3, 3))
    f = lambda M: np.sum((X @ M - Y) ** 2)
    want = (f(M_hat) - f(Ms)) / np.sum((X @ Ms) ** 2)
    assert np.isclose(om.residual(X.T @ X, X.T @ Y, M_hat), want, rtol=1e-8)


def _patch(rng, n=900):
    return rng.integers(20, 236, size=(n, 3)).astype(np.uint8)


def test_pair_label_self_transfer_is_identity():
    rng = np.random.default_rng(5)
    p = _patch(rng)
    feat, targ, M, flag = opairs.label(p, p)
    assert flag == 0
    assert np.allclose(M, np.eye(3), atol=1e-12)
    assert np.allclose(targ[:9], 0.0, atol=1e-12)
    # both halves of the features are the same histograms
    assert np.array_equal(feat[:768], feat[768:])
    # each channel's scaled histogram sums to 256 (up to bfloat16 rounding of the bins)
    for c in range(6):
        assert abs(feat[256 * c:256 * (c + 1)].sum() - 256.0) < 256.0 * 2 ** -7


def test_pair_label_known_gain_and_flat_patch():
    rng = np.random.default_rng(6)
    p = rng.integers(0, 120, size=(2000, 3)).astype(np.uint8)
    q = (2 * p.astype(np.int64)).astype(np.uint8)   # exact gain 2: the spec LUT is v -> 2v
    _, targ, M, flag = opairs.label(p, q)
    assert flag == 0
    assert np.allclose(M, 2 * np.eye(3), atol=1e-12)
    assert np.allclose(targ[:9], np.eye(3).reshape(-1), atol=1e-12)
    flat = np.full((400, 3), 77, dtype=np.uint8)
    _, targ, M, flag = opairs.label(flat, flat)
    assert flag == 1 and np.array_equal(M, np.eye(3))
    # flat pooled histogram: m1 == m2, zero span
    assert np.array_equal(targ[9:], np.zeros(3))


def test_pair_label_balance_span_uniform():
    # every level 0..255 once per side: pooled CDF(v) = 2 (v + 1), N = 512;
    # m1 = smallest v with CDF >= 0.05 N = 25.6 -> 2 (v + 1) = 26 -> v = 12;
    # m2 = smallest v with CDF >= 0.95 N = 486.4 -> 2 (v + 1) = 488 -> v = 243
    lv = np.arange(256, dtype=np.uint8)
    p = np.stack([lv, lv, lv], 1)
    _, targ, _, _ = opairs.label(p, p, lam=0.05)
    assert np.allclose(targ[9:], (243 - 12) / 255.0, rtol=1e-15)
