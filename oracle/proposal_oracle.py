"""FP64 CPU oracle of the learned-proposal network (a convolutional update proposer for the
slice potentials; the paper itself has no learned component).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module: only the tests,
the smoke check and the benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
library.

What it computes, written from the definitions:
  * conv3x3: out[y, x, o] = b[o] + sum_{dy, dx in -1..1} sum_i w[o, t, i] in[y + dy, x + dx, i],
    t = 3 (dy + 1) + (dx + 1), zero outside the image.
  * GELU(x) = x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)); GELU'(x) = Phi(x) + x phi(x).
  * The network: six conv3x3 layers 2L -> 64 -> 64 -> 64 -> 64 -> 64 -> L, GELU after the first
    five.  Input channels [s_V V_1..L, s_G G_1..L] (image planes [L][H][W]); proposal s_D out.
  * Storage precision is part of the method: the input, the weights and the hidden activations
    are BF16 (round to nearest, ties to even, of the FP32 value), the pre-activations are kept
    exactly (FP64 here); in the backward pass the gradient of every pre-activation is BF16 too.
  * Loss: mean over the L H W values of (proposal - target)^2 / s_D^2.  Gradients by the chain
    rule: the data gradient as the scatter-transpose of the convolution, the weight gradient as
    the correlation of the gradient with the shifted input.
  * Adam (Kingma and Ba 2015): m <- 0.9 m + 0.1 g, v <- 0.999 v + 0.001 g^2,
    p <- p - lr (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8).
  * Initialisation: weights uniform in +-sqrt(6 / (9 c_in + 9 c_out)) (last layer x 0.1) from
    the splitmix64 generator (Steele, Lea and Flood 2014) at state seed + (index + 1) *
    0x9E3779B97F4A7C15, mapped to [-1, 1) by its top 53 bits; biases 0.

Parity status: pinned by `tests/test_oracle_proposal_pins.py` (scipy's 2-D correlation, the GELU
identities and finite differences, finite differences of the loss through the whole network,
Adam's closed-form first step, torch's BF16 conversion, published splitmix64 outputs).

`jitter` (tests only): (generator, rel) adds noise of rel x the RMS value of the array to every
pre-activation and every pre-rounding gradient before BF16 rounding, to measure how far a
different FP32 accumulation order moves the BF16 roundings.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

LAYERS = 6
HIDDEN = 64
GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def channels(L: int) -> list[int]:
    return [2 * L, HIDDEN, HIDDEN, HIDDEN, HIDDEN, HIDDEN, L]


def layout(L: int) -> list[tuple[int, int, int, int]]:
    """(c_in, c_out, weight offset, bias offset) of every layer in the parameter array."""
    ch = channels(L)
    out, off = [], 0
    for i in range(LAYERS):
        ci, co = ch[i], ch[i + 1]
        out.append((ci, co, off, off + co * 9 * ci))
        off += co * 9 * ci + co
    return out


def param_count(L: int) -> int:
    ci, co, _, b = layout(L)[-1]
    return b + co


# ---------------------------------------------------------------------------------------------
# number formats and generators
# ---------------------------------------------------------------------------------------------
def bf16(x) -> np.ndarray:
    """Round to BF16 (nearest, ties to even) from FP32; returned as float64 values."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def splitmix64(seed: int, index: int) -> int:
    z = (seed + GOLDEN * (index + 1)) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def uniform_pm1(seed: int, index: int) -> float:
    return float(np.float32((splitmix64(seed, index) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0))


def init(L: int, seed: int) -> np.ndarray:
    """The deterministic initial parameters (FP32)."""
    p = np.zeros(param_count(L), dtype=np.float32)
    for i, (ci, co, wo, bo) in enumerate(layout(L)):
        bound = np.float32(math.sqrt(6.0 / (9.0 * ci + 9.0 * co)))
        if i == LAYERS - 1:
            bound = np.float32(bound * np.float32(0.1))
        for k in range(co * 9 * ci):
            p[wo + k] = np.float32(bound * np.float32(uniform_pm1(seed, wo + k)))
    return p


def unpack(params: np.ndarray, L: int):
    """[(w [c_out][9][c_in], b [c_out])] of every layer, as float64."""
    out = []
    for ci, co, wo, bo in layout(L):
        w = np.asarray(params[wo:bo], dtype=np.float64).reshape(co, 9, ci)
        b = np.asarray(params[bo:bo + co], dtype=np.float64)
        out.append((w, b))
    return out


# ---------------------------------------------------------------------------------------------
# layers
# ---------------------------------------------------------------------------------------------
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shifted(img: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """s[y, x] = img[y + dy, x + dx], zero outside (img [H][W][C])."""
    H, W = img.shape[:2]
    s = np.zeros_like(img)
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    s[yd, xd] = img[ys, xs]
    return s


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """x [H][W][c_in], w [c_out][9][c_in] -> [H][W][c_out] (FP64)."""
    H, W, _ = x.shape
    out = np.zeros((H, W, w.shape[0]))
    for t, (dy, dx) in enumerate(TAPS):
        out += shifted(x, dy, dx) @ w[:, t, :].T
    if b is not None:
        out += b
    return out


def conv3x3_data_grad(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Gradient with respect to the input of conv3x3 from g = dLoss/dout [H][W][c_out]:
    every output pixel (y, x) sends w[o, t, i] g[y, x, o] back to input pixel (y + dy, x + dx)."""
    dx_ = np.zeros((g.shape[0], g.shape[1], w.shape[2]))
    for t, (dy, dx) in enumerate(TAPS):
        contrib = g @ w[:, t, :]                    # [H][W][c_in] at the output pixel
        dx_ += shifted(contrib, -dy, -dx)           # moved to the input pixel it came from
    return dx_


def conv3x3_weight_grad(g: np.ndarray, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(dW [c_out][9][c_in], db [c_out]) of conv3x3 from g = dLoss/dout."""
    co, ci = g.shape[2], x.shape[2]
    dW = np.zeros((co, 9, ci))
    G = g.reshape(-1, co)
    for t, (dy, dx) in enumerate(TAPS):
        dW[:, t, :] = G.T @ shifted(x, dy, dx).reshape(-1, ci)
    return dW, G.sum(axis=0)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


# ---------------------------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------------------------
def _q(a, quantize: bool):
    return bf16(a) if quantize else np.asarray(a, dtype=np.float64)


def _jit(a, jitter):
    if jitter is None:
        return a
    rng, rel = jitter
    return a + rel * np.sqrt(np.mean(a * a)) * rng.standard_normal(a.shape)


def net_input(V: np.ndarray, G: np.ndarray, sv: float, sg: float, quantize: bool = True) -> np.ndarray:
    """[H][W][2L] from V, G [L][H][W]: channels s_V V then s_G G (each rounded to FP32 first)."""
    x = np.concatenate([np.float32(sv) * V.astype(np.float32), np.float32(sg) * G.astype(np.float32)], axis=0)
    return _q(np.moveaxis(x, 0, -1), quantize)


def forward(params, L, V, G, sv, sg, quantize=True, jitter=None):
    """(pre-activations of the six layers, inputs of the six layers)."""
    layers = unpack(params, L)
    a = net_input(V, G, sv, sg, quantize)
    pres, ins = [], []
    for i, (w, b) in enumerate(layers):
        ins.append(a)
        pre = _jit(conv3x3(a, _q(w, quantize), b), jitter)
        pres.append(pre)
        if i < LAYERS - 1:
            a = _q(gelu(pre), quantize)
    return pres, ins


def proposal(params, L, V, G, sv, sg, sd, quantize=True, jitter=None) -> np.ndarray:
    """s_D x network output, planes [L][H][W]."""
    pres, _ = forward(params, L, V, G, sv, sg, quantize, jitter)
    return sd * np.moveaxis(pres[-1], -1, 0)


def loss_and_grad(params, L, V, G, target, sv, sg, sd, quantize=True, jitter=None, abs_sums=False):
    """(loss, gradient of the loss with respect to the parameters in their FP32 layout); with
    abs_sums also the sums of the magnitudes of the terms of every weight- and bias-gradient
    entry (sum_p |g| |x| and sum_p |g|), the scale of the FP32 accumulation error of each."""
    layers = unpack(params, L)
    pres, ins = forward(params, L, V, G, sv, sg, quantize, jitter)
    t = np.moveaxis(np.asarray(target, dtype=np.float32).astype(np.float64), 0, -1) / sd
    n = t.size
    d = pres[-1] - t
    loss = float(np.sum(d * d) / n)
    g = _q(_jit(2.0 / n * d, jitter), quantize)
    grad = np.zeros(param_count(L))
    mags = np.zeros(param_count(L))
    for i in range(LAYERS - 1, -1, -1):
        ci, co, wo, bo = layout(L)[i]
        dW, db = conv3x3_weight_grad(g, ins[i])
        grad[wo:bo] = dW.ravel()
        grad[bo:bo + co] = db
        if abs_sums:
            aW, ab = conv3x3_weight_grad(np.abs(g), np.abs(ins[i]))
            mags[wo:bo] = aW.ravel()
            mags[bo:bo + co] = ab
        if i > 0:
            gx = conv3x3_data_grad(g, _q(layers[i][0], quantize))
            g = _q(_jit(gx * gelu_grad(pres[i - 1]), jitter), quantize)
    return (loss, grad, mags) if abs_sums else (loss, grad)


def adam(params, m, v, grad, step: int, lr: float):
    """One Adam step in FP64; returns (params, m, v)."""
    m = 0.9 * m + 0.1 * grad
    v = 0.999 * v + 0.001 * grad * grad
    mh = m / (1.0 - 0.9 ** step)
    vh = v / (1.0 - 0.999 ** step)
    return params - lr * mh / (np.sqrt(vh) + 1e-8), m, v
