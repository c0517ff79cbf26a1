"""Pins of the learned-proposal oracle against things other than itself: scipy's 2-D
correlation, the GELU identities, finite differences of the loss through the whole network,
Adam's closed-form first step, torch's BF16 conversion and published splitmix64 outputs."""
import math

import numpy as np
import pytest
import torch
from scipy.signal import correlate2d

from oracle import proposal_oracle as P


def test_conv3x3_is_a_sum_of_scipy_correlations():
    rng = np.random.default_rng(1)
    H, W, ci, co = 7, 9, 3, 4
    x = rng.standard_normal((H, W, ci))
    w = rng.standard_normal((co, 9, ci))
    b = rng.standard_normal(co)
    out = P.conv3x3(x, w, b)
    for o in range(co):
        ref = b[o] + sum(correlate2d(x[:, :, i], w[o, :, i].reshape(3, 3), mode="same", boundary="fill")
                         for i in range(ci))
        np.testing.assert_allclose(out[:, :, o], ref, rtol=1e-12, atol=1e-12)


def test_conv3x3_single_tap_is_a_shift():
    """A weight with one nonzero tap (dy, dx) moves the image by (-dy, -dx): out[y, x] = in[y+dy, x+dx]."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 6, 1))
    for t, (dy, dx) in enumerate(P.TAPS):
        w = np.zeros((1, 9, 1))
        w[0, t, 0] = 1.0
        out = P.conv3x3(x, w)[:, :, 0]
        for y in range(5):
            for xx in range(6):
                yy, xs = y + dy, xx + dx
                want = x[yy, xs, 0] if 0 <= yy < 5 and 0 <= xs < 6 else 0.0
                assert out[y, xx] == want


def test_data_and_weight_gradients_are_the_adjoint_of_the_convolution():
    """<conv(x), g> = <x, data_grad(g)> and = <w, weight_grad(g, x)> (both bilinear forms)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 5, 3))
    w = rng.standard_normal((4, 9, 3))
    g = rng.standard_normal((6, 5, 4))
    lhs = np.sum(P.conv3x3(x, w) * g)
    assert abs(lhs - np.sum(x * P.conv3x3_data_grad(g, w))) < 1e-10 * abs(lhs) + 1e-10
    dW, db = P.conv3x3_weight_grad(g, x)
    assert abs(lhs - np.sum(w * dW)) < 1e-10 * abs(lhs) + 1e-10
    np.testing.assert_allclose(db, g.reshape(-1, 4).sum(0), rtol=1e-12)


def test_gelu_identities_and_derivative():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(P.gelu(x) - P.gelu(-x), x, atol=1e-12)      # Phi(x) + Phi(-x) = 1
    assert P.gelu(np.array([0.0]))[0] == 0.0
    np.testing.assert_allclose(P.gelu(np.array([1.0])), [0.8413447460685429], rtol=1e-12)  # Phi(1)
    h = 1e-6
    fd = (P.gelu(x + h) - P.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(P.gelu_grad(x), fd, atol=1e-8)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 5000),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -1 - 2 ** -8, 0.0, -0.0], dtype=np.float32)])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(P.bf16(x), want)


def test_splitmix64_published_outputs():
    """The first outputs of splitmix64 from state 1234567, as printed with its reference code."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [P.splitmix64(1234567, i) for i in range(5)] == want


def test_init_is_uniform_within_the_bound():
    L = 2
    p = P.init(L, seed=7)
    assert p.dtype == np.float32 and p.size == P.param_count(L)
    for i, (ci, co, wo, bo) in enumerate(P.layout(L)):
        bound = math.sqrt(6.0 / (9 * ci + 9 * co)) * (0.1 if i == P.LAYERS - 1 else 1.0)
        w = p[wo:bo]
        assert np.all(np.abs(w) <= bound * (1 + 1e-6))
        assert abs(w.mean()) < 0.1 * bound and abs(w.std() - bound / math.sqrt(3)) < 0.1 * bound
        assert np.all(p[bo:bo + co] == 0)
    assert not np.array_equal(P.init(L, seed=8), p)


def test_parameter_layout():
    L = 4
    lay = P.layout(L)
    assert [(a, b) for a, b, _, _ in lay] == [(8, 64), (64, 64), (64, 64), (64, 64), (64, 64), (64, 4)]
    assert P.param_count(L) == sum(co * 9 * ci + co for ci, co, _, _ in lay)


def _tiny(seed=5, L=2, H=5, W=6):
    rng = np.random.default_rng(seed)
    params = P.init(L, seed=11).astype(np.float64)
    params += 0.05 * rng.standard_normal(params.size)     # nonzero biases, a less symmetric net
    V = rng.standard_normal((L, H, W))
    G = rng.standard_normal((L, H, W))
    T = 0.3 * rng.standard_normal((L, H, W))
    return params, L, V, G, T


def test_network_gradient_matches_finite_differences():
    """The chain rule through all six layers (quantisation off) against central differences of
    the loss, on a sample of weights and every bias of every layer."""
    params, L, V, G, T = _tiny()
    sv, sg, sd = 0.7, 1.3, 0.5
    loss, grad = P.loss_and_grad(params, L, V, G, T, sv, sg, sd, quantize=False)
    rng = np.random.default_rng(6)
    idx = []
    for ci, co, wo, bo in P.layout(L):
        idx += list(rng.choice(np.arange(wo, bo), 6, replace=False)) + list(range(bo, bo + co))[:3]
    h = 1e-6
    for k in idx:
        e = np.zeros_like(params)
        e[k] = h
        lp, _ = P.loss_and_grad(params + e, L, V, G, T, sv, sg, sd, quantize=False)
        lm, _ = P.loss_and_grad(params - e, L, V, G, T, sv, sg, sd, quantize=False)
        fd = (lp - lm) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, grad[k], fd)


def test_loss_is_the_mean_squared_error_of_the_proposal():
    params, L, V, G, T = _tiny(seed=8)
    sv, sg, sd = 0.7, 1.3, 0.5
    prop = P.proposal(params, L, V, G, sv, sg, sd, quantize=False)
    loss, _ = P.loss_and_grad(params, L, V, G, T, sv, sg, sd, quantize=False)
    T32 = T.astype(np.float32).astype(np.float64)
    assert abs(loss - np.mean((prop - T32) ** 2) / sd ** 2) < 1e-12 * loss


def test_adam_first_steps_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2 at every step, so each
    step moves every parameter by lr g / (|g| + 1e-8)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in (1, 2, 3):
        p, m, v = P.adam(p, m, v, g, t, 0.01)
        np.testing.assert_allclose(p, -t * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_quantised_forward_rounds_every_hidden_activation():
    params, L, V, G, T = _tiny(seed=9)
    pres, ins = P.forward(params, L, V, G, 1.0, 1.0)
    for a in ins:
        np.testing.assert_array_equal(a, P.bf16(a))
    pres_f, _ = P.forward(params, L, V, G, 1.0, 1.0, quantize=False)
    rel = np.linalg.norm(pres[-1] - pres_f[-1]) / np.linalg.norm(pres_f[-1])
    assert 1e-5 < rel < 3e-2      # BF16 storage moves the output, but only by a few BF16 ulps
