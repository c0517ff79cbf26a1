"""The learned-proposal workflow over the C ABI (include/msp.h, include/msp_learn.h).

A six-layer convolutional network proposes an update of all slice potentials from the current
potentials V and their gradient dL/dV.  It is trained on trajectories of the plain method
(Algorithm 1, msp_reconstruct): from a state V_k of a trajectory the target is the change that
trajectory still makes, V_K - V_k (or, with a horizon h, the change of the next h sweeps).  In use every proposal is judged by the true multislice loss
(Sec. 3.2): msp_learned_propose keeps it only if the loss drops, and otherwise this driver takes
one sweep of the plain method instead.

Everything numeric runs in the library's kernels; this module only sequences the calls and reads
one acceptance flag per iteration.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import msp


@dataclass
class Corpus:
    """Training samples (device tensors [n][L][Ny][Nx], FP32): potentials, gradients, targets."""
    V: list = field(default_factory=list)
    G: list = field(default_factory=list)
    T: list = field(default_factory=list)

    def __len__(self):
        return len(self.V)


def plain_trajectory(g, probe, V0, pos, I_meas, sweeps: int, ws=None, stream=None):
    """States V_0 .. V_sweeps of the plain method (one msp_reconstruct sweep at a time, fixed
    probe) and the loss at each."""
    pl = msp.plan(1)   # one sweep, no probe steps: the probe stays as it is
    V = V0.clone()
    states, losses = [V.clone()], []
    for _ in range(sweeps):
        h = msp.reconstruct(g, pl, probe, V, pos, I_meas, ws=ws, stream=stream)
        losses.append(h[0])
        states.append(V.clone())
    losses.append(h[-1])
    return states, torch.stack(losses).cpu().numpy()


def add_trajectory(corpus: Corpus, g, probe, pos, I_meas, states, every: int = 1, horizon=None, ws=None,
                   stream=None):
    """Samples (V_k, dL/dV at V_k, V_j - V_k) for k = 0, every, 2 every, ... < K, with j = K (the
    trajectory's end) or, given a horizon h, j = min(k + h, K)."""
    K = len(states) - 1
    for k in range(0, K, every):
        j = K if horizon is None else min(k + horizon, K)
        _, G, _ = msp.loss_grad(g, probe, states[k], pos, I_meas, want_dprobe=False, ws=ws, stream=stream)
        corpus.V.append(states[k])
        corpus.G.append(G)
        corpus.T.append(states[j] - states[k])


def input_scales(corpus: Corpus) -> tuple[float, float, float]:
    """(s_V, s_G, s_D): the reciprocal RMS of the potentials and of the gradients, and the RMS of
    the targets, over the corpus."""
    rms = lambda xs: float(torch.sqrt(torch.stack([(x.double() ** 2).mean() for x in xs]).mean()))
    return 1.0 / max(rms(corpus.V), 1e-30), 1.0 / max(rms(corpus.G), 1e-30), max(rms(corpus.T), 1e-30)


def train(shape, corpus: Corpus, steps: int, lr: float = 1e-3, seed: int = 0, params=None, stream=None):
    """Adam on the corpus, one sample per step in a seeded order.  Returns (params, losses)."""
    dev = corpus.V[0].device
    if params is None:
        params = msp.net_init(shape, seed, device=dev, stream=stream)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    ws = msp.net_make_workspace(shape, dev)
    order = np.random.default_rng(seed).integers(0, len(corpus), size=steps)
    loss = torch.empty(steps, dtype=torch.float64, device=dev)
    for k, i in enumerate(order):
        msp.net_train_step(shape, params, m, v, k + 1, lr, corpus.V[i], corpus.G[i], corpus.T[i], loss=loss[k],
                           ws=ws, stream=stream)
    msp.check_workspace(ws, stream)
    return params, loss.cpu().numpy()


def reconstruct_learned(g, shape, params, probe, V, pos, I_meas, iterations: int, target_loss=None, ws=None,
                        learn_ws=None, stream=None):
    """The acceptance loop: each iteration tries one proposal (msp_learned_propose) and takes one
    plain sweep when it is rejected.  V is updated in place.  Stops early once the loss is at or
    below `target_loss`.  Returns a list of (loss before, accepted, loss after) per iteration."""
    dev = V.device
    ws = msp.make_workspace(g, dev) if ws is None else ws
    learn_ws = msp.learned_make_workspace(g, shape, dev) if learn_ws is None else learn_ws
    pl = msp.plan(1)
    accepted = torch.zeros((), dtype=torch.int32, device=dev)
    loss = torch.empty(2, dtype=torch.float64, device=dev)
    hist = []
    for _ in range(iterations):
        msp.learned_propose(g, shape, params, probe, V, pos, I_meas, accepted=accepted, loss=loss, ws=ws,
                            learn_ws=learn_ws, stream=stream)
        a = int(accepted.item())
        l0, l1 = loss.tolist()
        if a:
            after = l1
        else:
            h = msp.reconstruct(g, pl, probe, V, pos, I_meas, ws=ws, stream=stream)   # no probe steps
            after = float(h[-1].item())
        hist.append((l0, a, after))
        if target_loss is not None and after <= target_loss:
            break
    msp.check_workspace(ws, stream)
    msp.check_workspace(learn_ws, stream)
    return hist
