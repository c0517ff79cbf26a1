"""The acceptance rule of the learned proposal (msp_learned_propose) and the workflow around it
(paper_2205_03902_gb300.learned): a proposal is kept only if the true multislice loss drops,
otherwise the potentials are left as they were and the driver takes a plain sweep."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    return m


SMALL = dataclasses.replace(synth.C5, name="c5_small_L2_obj256_W64_S64", n_slices=2, obj=256, win=64, scan=(8, 8),
                            step_px=16)


def problem(msp, seed):
    cfg = synth.c5_specimen(seed, base=SMALL)
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd)
    dev = torch.device("cuda")
    probe = torch.from_numpy(synth.probe(cfg).astype(np.complex64)).to(dev)
    V_true = torch.from_numpy(synth.potential_slices(cfg).astype(np.float32)).to(dev)
    d_pos = torch.from_numpy(pos).to(dev)
    ws = msp.make_workspace(g, dev)
    I = msp.forward(g, probe, V_true, d_pos, ws=ws).cpu().numpy().astype(np.float64)
    I = torch.from_numpy(synth.poisson_counts(I, cfg.dose, cfg.seed).astype(np.float32)).to(dev)
    return cfg, gd, g, probe, d_pos, I, ws, V_true


def test_propose_rejects_a_proposal_that_raises_the_loss(msp):
    """From the true potentials (the loss is at its noise floor) a huge proposal raises the loss:
    rejected, V untouched, loss[0] the library's loss at V."""
    cfg, gd, g, probe, pos, I, ws, V_true = problem(msp, 1)
    L, N = cfg.n_slices, cfg.obj
    s = msp.net_shape(L, N, N, scale_v=1.0, scale_g=1.0, scale_d=1e3)     # huge proposals
    params = msp.net_init(s, 2)
    V = V_true.clone()
    acc, loss = msp.learned_propose(g, s, params, probe, V, pos, I, ws=ws)
    assert acc.item() == 0
    assert torch.equal(V, V_true)
    l0, l1 = loss.tolist()
    assert l1 > l0
    ref, _, _ = msp.loss_grad(g, probe, V, pos, I, want_dV=False, want_dprobe=False, ws=ws)
    assert l0 == ref.item()
    # the loss the rule compares is the multislice loss: at V = 0 against the oracle
    Z = torch.zeros_like(V)
    acc, loss = msp.learned_propose(g, s, params, probe, Z, pos, I, ws=ws)
    lo = O.loss_grad(gd, probe.cpu().numpy().astype(np.complex128), pos.cpu().numpy(),
                     I.cpu().numpy().astype(np.float64), V=np.zeros((L, N, N)), want_probe=False)["loss"]
    assert abs(loss[0].item() - lo) / lo < 1e-5


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_propose_keeps_exactly_the_candidate_or_nothing(msp, seed):
    cfg, gd, g, probe, pos, I, ws, _ = problem(msp, seed)
    L, N = cfg.n_slices, cfg.obj
    s = msp.net_shape(L, N, N, scale_v=1.0, scale_g=1e-3, scale_d=10.0 ** (-seed))
    params = msp.net_init(s, seed)
    V0 = 0.01 * torch.rand((L, N, N), generator=torch.Generator().manual_seed(seed)).cuda()
    V = V0.clone()
    acc, loss = msp.learned_propose(g, s, params, probe, V, pos, I, ws=ws)
    msp.check_workspace(ws)
    _, G, _ = msp.loss_grad(g, probe, V0, pos, I, want_dprobe=False, ws=ws)
    cand = V0 + msp.net_forward(s, params, V0, G)
    l_cand, _, _ = msp.loss_grad(g, probe, cand, pos, I, want_dV=False, want_dprobe=False, ws=ws)
    l0, l1 = loss.tolist()
    assert l1 == l_cand.item()
    if acc.item():
        assert l1 < l0 and torch.equal(V, cand)
    else:
        assert not (l1 < l0) and torch.equal(V, V0)


def test_trained_proposals_and_the_acceptance_loop(msp):
    from paper_2205_03902_gb300 import learned
    corpus = learned.Corpus()
    for seed in (10, 11):
        cfg, gd, g, probe, pos, I, ws, _ = problem(msp, seed)
        V0 = torch.zeros((cfg.n_slices, cfg.obj, cfg.obj), dtype=torch.float32, device="cuda")
        states, losses = learned.plain_trajectory(g, probe, V0, pos, I, sweeps=8, ws=ws)
        assert losses[-1] < losses[0]
        learned.add_trajectory(corpus, g, probe, pos, I, states, ws=ws)
    assert len(corpus) == 16
    sv, sg, sd = learned.input_scales(corpus)
    s = msp.net_shape(cfg.n_slices, cfg.obj, cfg.obj, sv, sg, sd)
    def corpus_loss(params):
        return np.mean([msp.net_loss_grad(s, params, corpus.V[i], corpus.G[i], corpus.T[i])[0].item()
                        for i in range(len(corpus))])

    p0 = msp.net_init(s, 1)
    before = corpus_loss(p0)
    params, tl = learned.train(s, corpus, steps=200, lr=1e-3, seed=1, params=p0.clone())
    assert np.all(np.isfinite(tl))
    assert corpus_loss(params) < before
    cfg, gd, g, probe, pos, I, ws, _ = problem(msp, 20)
    V = torch.zeros((cfg.n_slices, cfg.obj, cfg.obj), dtype=torch.float32, device="cuda")
    hist = learned.reconstruct_learned(g, s, params, probe, V, pos, I, iterations=6, ws=ws)
    for l0, a, after in hist:
        if a:
            assert after < l0
    assert hist[-1][2] < hist[0][0]
