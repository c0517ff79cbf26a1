"""Host logic of the learned-proposal driver (paper_2205_03902_gb300/learned.py) against a
stand-in for the library: which calls it makes and in what order, what it keeps, when it stops.
No GPU and no kernel runs here; the stand-in records the calls and plays back scripted losses."""
import numpy as np
import pytest
import torch

from paper_2205_03902_gb300 import learned


class FakeMsp:
    """Scripted acceptance flags and losses; every call is logged."""

    def __init__(self, accepts=(), losses=(), sweep_losses=()):
        self.log = []
        self.accepts = list(accepts)
        self.losses = list(losses)            # (loss before, loss after proposal) per propose call
        self.sweep_losses = list(sweep_losses)

    # workspaces and plans
    def make_workspace(self, g, dev):
        return "ws"

    def learned_make_workspace(self, g, s, dev):
        return "lws"

    def plan(self, sweeps, probe_steps=0):
        return ("plan", sweeps, probe_steps)

    def check_workspace(self, ws, stream=None):
        self.log.append(("check", ws))

    # the calls the driver sequences
    def learned_propose(self, g, s, params, probe, V, pos, I, accepted=None, loss=None, ws=None, learn_ws=None,
                        stream=None):
        a = self.accepts.pop(0)
        l0, l1 = self.losses.pop(0)
        accepted.fill_(a)
        loss[0], loss[1] = l0, l1
        if a:
            V.add_(1.0)
        self.log.append(("propose", a))

    def reconstruct(self, g, plan, probe, V, pos, I, ws=None, stream=None):
        self.log.append(("sweep", plan))
        V.sub_(0.5)
        return torch.tensor([0.0, self.sweep_losses.pop(0)], dtype=torch.float64)

    def loss_grad(self, g, probe, V, pos, I, want_dprobe=True, ws=None, stream=None):
        self.log.append(("loss_grad", float(V.mean())))
        return torch.zeros(1, dtype=torch.float64), 2.0 * V, None


@pytest.fixture
def fake(monkeypatch):
    def install(**kw):
        f = FakeMsp(**kw)
        monkeypatch.setattr(learned, "msp", f)
        return f
    return install


def test_rejected_proposals_fall_back_to_one_plain_sweep(fake):
    f = fake(accepts=[1, 0, 1], losses=[(10.0, 8.0), (8.0, 9.0), (7.0, 6.0)], sweep_losses=[7.0])
    V = torch.zeros(2, 4, 4)
    hist = learned.reconstruct_learned("g", "s", "p", "probe", V, "pos", "I", iterations=3)
    assert [e for e in f.log if e[0] != "check"] == [("propose", 1), ("propose", 0), ("sweep", ("plan", 1, 0)),
                                                      ("propose", 1)]
    assert hist == [(10.0, 1, 8.0), (8.0, 0, 7.0), (7.0, 1, 6.0)]
    assert torch.all(V == 1.0 - 0.5 + 1.0)          # two accepted proposals, one sweep
    assert ("check", "ws") in f.log and ("check", "lws") in f.log


def test_the_loop_stops_at_the_target_loss(fake):
    f = fake(accepts=[0, 1, 1], losses=[(10.0, 11.0), (9.0, 5.0), (5.0, 4.0)], sweep_losses=[9.0])
    V = torch.zeros(1, 2, 2)
    hist = learned.reconstruct_learned("g", "s", "p", "probe", V, "pos", "I", iterations=10, target_loss=5.0)
    assert len(hist) == 2 and hist[-1][2] == 5.0
    assert sum(1 for e in f.log if e[0] == "propose") == 2


def test_add_trajectory_targets_and_horizon(fake):
    fake()
    states = [torch.full((1, 2, 2), float(k)) for k in range(5)]      # V_0 .. V_4
    c = learned.Corpus()
    learned.add_trajectory(c, "g", "probe", "pos", "I", states, every=2)
    assert len(c) == 2                                                 # k = 0, 2
    assert [float(t.mean()) for t in c.T] == [4.0, 2.0]               # V_K - V_k
    assert [float(g.mean()) for g in c.G] == [0.0, 4.0]               # the library's gradient at V_k
    c2 = learned.Corpus()
    learned.add_trajectory(c2, "g", "probe", "pos", "I", states, every=1, horizon=3)
    assert [float(t.mean()) for t in c2.T] == [3.0, 3.0, 2.0, 1.0]    # V_min(k+3, 4) - V_k


def test_input_scales_are_the_corpus_rms():
    c = learned.Corpus()
    rng = np.random.default_rng(0)
    for _ in range(3):
        c.V.append(torch.from_numpy(rng.normal(0, 2.0, (2, 8, 8))))
        c.G.append(torch.from_numpy(rng.normal(0, 0.1, (2, 8, 8))))
        c.T.append(torch.from_numpy(rng.normal(0, 5.0, (2, 8, 8))))
    sv, sg, sd = learned.input_scales(c)
    rms = lambda xs: float(np.sqrt(np.mean([np.mean(x.numpy() ** 2) for x in xs])))
    assert sv == pytest.approx(1 / rms(c.V)) and sg == pytest.approx(1 / rms(c.G)) and sd == pytest.approx(rms(c.T))
