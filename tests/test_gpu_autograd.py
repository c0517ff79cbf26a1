"""Differentiation form: the loss as a torch.autograd.Function over the fused forward /
adjoint kernel, checked by central finite differences of the same library's loss and
against the oracle's adjoint (Sec. 3.2 gradient composed through the slices)."""
import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def msp():
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    m.lib()
    return m


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def problem(msp):
    """A small strong-misfit state (well conditioned): W = 64, 4 x 4 sub-scan, 3 slices."""
    cfg = synth.Workload("ad_L3_obj80_W64_S16", 3, 80, 0.2, 2.0, 30, 64, (4, 4), 4, 25.0, 50.0, None, seed=5)
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    Vt = synth.potential_slices(cfg)
    probe = synth.probe(cfg).astype(np.complex64).astype(np.complex128)
    I = f32(O.forward(gd, probe, pos, V=Vt))
    V0 = f32(Vt + 300.0 * np.random.default_rng(3).standard_normal(Vt.shape))
    g = msp.geometry(**gd)
    t = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x).astype(dt)).to(DEV)
    return cfg, gd, g, pos, probe, I, V0, t(pos, np.int32), t(probe, np.complex64), t(I, np.float32), t(V0, np.float32)


def test_autograd_matches_the_oracle_adjoint(msp):
    cfg, gd, g, pos, probe, I, V0, dpos, dprobe_in, dI, dV0 = problem(msp)
    V = dV0.clone().requires_grad_(True)
    p = dprobe_in.clone().requires_grad_(True)
    loss = msp.multislice_loss(g, V, p, dpos, dI)
    (3.0 * loss).backward()
    ref = O.loss_grad(gd, probe, pos, I, V=V0)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= 1e-5
    rel = lambda a, b: np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())
    assert rel(V.grad.cpu().numpy(), 3.0 * ref["dV"]) <= 1e-5
    assert rel(p.grad.cpu().numpy(), 3.0 * 2.0 * ref["dprobe"]) <= 1e-5


def test_autograd_matches_central_finite_differences(msp):
    """(L(V + h d) - L(V - h d)) / 2h = <dL/dV, d>, and likewise for the probe with
    Re <grad, d> (PyTorch's complex gradient), h = 1e-4 relative to the argument's scale.
    The difference of two FP32 losses resolves the slope to ~1e-3, so this check is for
    wrong gradients (sign, factor, conjugation) at 1e-2; precision is checked against the
    oracle above."""
    cfg, gd, g, pos, probe, I, V0, dpos, dprobe_in, dI, dV0 = problem(msp)
    V = dV0.clone().requires_grad_(True)
    p = dprobe_in.clone().requires_grad_(True)
    msp.multislice_loss(g, V, p, dpos, dI).backward()
    rng = np.random.default_rng(11)
    for _ in range(3):
        d = torch.from_numpy(rng.standard_normal(V0.shape).astype(np.float32)).to(DEV)
        h = 1e-4 * float(dV0.abs().max())
        with torch.no_grad():
            lp = msp.multislice_loss(g, dV0 + h * d, dprobe_in, dpos, dI).item()
            lm = msp.multislice_loss(g, dV0 - h * d, dprobe_in, dpos, dI).item()
        fd = (lp - lm) / (2 * h)
        an = float((V.grad.double() * d.double()).sum())
        assert fd == pytest.approx(an, rel=1e-2)
        # relative perturbation p o r: the amplitude loss curves sharply where |p| is small
        r = rng.standard_normal(probe.shape) + 1j * rng.standard_normal(probe.shape)
        dp = torch.from_numpy((probe * r).astype(np.complex64)).to(DEV)
        hp = 1e-4
        with torch.no_grad():
            lp = msp.multislice_loss(g, dV0, dprobe_in + hp * dp, dpos, dI).item()
            lm = msp.multislice_loss(g, dV0, dprobe_in - hp * dp, dpos, dI).item()
        fd = (lp - lm) / (2 * hp)
        an = float((p.grad.conj() * dp).real.double().sum())
        assert fd == pytest.approx(an, rel=1e-2)
