"""GPU parity: libmsp (FP32, sm_103a) against the FP64 oracle on identical seeded inputs.

Bar: relative L2 error <= 1e-5 on intensities, loss, potential and probe
gradients and on the state after a step (the FP32 target of the benchmark
specification).  Cases span several CTA waves with a ragged tail, the full
benchmark workload (sampled outputs), and the degenerate cases of the method.
"""
import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def msp():
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    m.lib()
    return m


DEV = torch.device("cuda", 0)


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x).astype(dtype)).to(DEV)


class Case:
    """A seeded problem: geometry, probe, positions, measured intensities, current V."""

    def __init__(self, cfg, sub=None, noisy=True, probe_guess=True, v_scale=0.5, seed=0, pos=None):
        self.cfg = cfg
        self.pos = synth.scan_positions(cfg, sub=sub) if pos is None else np.asarray(pos, dtype=np.int32)
        self.gd = synth.geometry(cfg, n_pos=len(self.pos))
        self.V_true = synth.potential_slices(cfg)
        p_true = synth.probe(cfg)
        I = O.forward(self.gd, p_true, self.pos, V=self.V_true) if len(self.pos) else np.zeros((0, cfg.win, cfg.win))
        # every input is rounded to the library's FP32 once, so both sides see identical values
        self.I = f32(synth.poisson_counts(I, cfg.dose, cfg.seed) if noisy else I)
        probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A) if (probe_guess and cfg.defocus_guess_A) else p_true
        self.probe = probe.astype(np.complex64).astype(np.complex128)
        rng = np.random.default_rng(seed + 5)
        self.V = f32(v_scale * self.V_true + 0.5 * rng.standard_normal(self.V_true.shape))

    def dev(self, msp):
        g = msp.geometry(**self.gd)
        return g, to_dev(self.probe, np.complex64), to_dev(self.V, np.float32), to_dev(self.pos, np.int32), \
            to_dev(self.I, np.float32)


@pytest.fixture(scope="module")
def c1():
    return Case(synth.C1, noisy=False)


@pytest.fixture(scope="module")
def c2_ragged():
    # 13 x 13 = 169 positions: more than one CTA per SM on a 152-SM part, with a ragged tail
    return Case(synth.C2, sub=(13, 13))


# --------------------------------------------------------------------------- forward

@pytest.mark.parametrize("which", ["c1", "c2_ragged"])
def test_forward_intensities(msp, which, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, _ = c.dev(msp)
    I = msp.forward(g, p, V, pos).cpu().numpy()
    ref = O.forward(c.gd, c.probe, c.pos, V=c.V)
    assert rel(I, ref) <= TOL
    # per-pattern check as well: no single pattern may be off
    for s in range(0, len(c.pos), max(1, len(c.pos) // 16)):
        assert rel(I[s], ref[s]) <= TOL


# --------------------------------------------------------------------------- loss and gradients

@pytest.mark.parametrize("which", ["c1", "c2_ragged"])
def test_loss_and_gradients(msp, which, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= TOL
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL
    # per-slice as well
    for l in range(c.gd["n_slices"]):
        assert rel(dV.cpu().numpy()[l], ref["dV"][l]) <= TOL


def test_gradients_are_bit_reproducible(msp, c2_ragged):
    g, p, V, pos, I = c2_ragged.dev(msp)
    ws = msp.make_workspace(g)
    a = [t.clone() for t in msp.loss_grad(g, p, V, pos, I, ws=ws)]
    b = msp.loss_grad(g, p, V, pos, I, ws=ws)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_optional_outputs(msp, c1):
    g, p, V, pos, I = c1.dev(msp)
    loss_a, dV_a, dp_a = msp.loss_grad(g, p, V, pos, I)
    loss_b, dV_b, dp_b = msp.loss_grad(g, p, V, pos, I, want_dV=False, want_dprobe=False)
    assert dV_b is None and dp_b is None
    assert loss_a.item() == loss_b.item()
    _, dV_c, _ = msp.loss_grad(g, p, V, pos, I, want_dprobe=False)
    assert torch.equal(dV_a, dV_c)


# --------------------------------------------------------------------------- steps

@pytest.mark.parametrize("which,layer", [("c1", 0), ("c1", 1), ("c2_ragged", 0), ("c2_ragged", 2)])
def test_layer_step(msp, which, layer, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    loss, mu = msp.layer_step(g, p, V, pos, I, layer)
    Vn, loss_ref, mu_ref = O.layer_step(c.gd, c.probe, c.pos, c.I, layer, V=c.V)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    assert abs(mu.item() - mu_ref) / mu_ref <= TOL
    Vg = V.cpu().numpy()
    assert rel(Vg[layer] - c.V[layer], Vn[layer] - c.V[layer]) <= TOL   # the update itself
    assert rel(Vg, Vn) <= TOL
    others = [m for m in range(c.gd["n_slices"]) if m != layer]
    assert np.array_equal(Vg[others], c.V[others].astype(np.float32))


def test_layer_step_fixed_step(msp, c1):
    g, p, V, pos, I = c1.dev(msp)
    _, mu = msp.layer_step(g, p, V, pos, I, 1, step=1234.5)
    assert mu.item() == 1234.5
    Vn, _, _ = O.layer_step(c1.gd, c1.probe, c1.pos, c1.I, 1, V=c1.V, step=1234.5)
    assert rel(V.cpu().numpy()[1] - c1.V[1], Vn[1] - c1.V[1]) <= TOL


@pytest.mark.parametrize("normalize", [False, True])
def test_probe_step(msp, c2_ragged, normalize):
    c = c2_ragged
    g, p, V, pos, I = c.dev(msp)
    loss, mu = msp.probe_step(g, p, V, pos, I, normalize=normalize)
    pn, loss_ref, mu_ref = O.probe_step(c.gd, c.probe, c.pos, c.I, V=c.V, normalize=normalize)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    assert mu.item() == pytest.approx(mu_ref, rel=1e-15)
    assert rel(p.cpu().numpy(), pn) <= TOL
    assert rel(p.cpu().numpy() - c.probe, pn - c.probe) <= TOL


def test_layerwise_trajectory(msp):
    """Algorithm 1, three sweeps from V = 0 with the known probe on noiseless data."""
    c = Case(synth.C1, sub=(4, 4), noisy=False, v_scale=0.0)
    c.V = np.zeros_like(c.V_true)
    g, p, V, pos, I = c.dev(msp)
    Vref, hist = O.layerwise_estimation(c.gd, c.probe, c.pos, c.I, c.V, sweeps=3)
    losses = []
    ws = msp.make_workspace(g)
    for _ in range(3):
        for layer in range(c.gd["n_slices"]):
            lb, _ = msp.layer_step(g, p, V, pos, I, layer, ws=ws)
            losses.append(lb.item())
    assert rel(V.cpu().numpy(), Vref) <= 1e-4
    np.testing.assert_allclose(losses, hist, rtol=1e-4)
    assert losses[-1] < losses[0]


# --------------------------------------------------------------------------- edge and degenerate cases

def test_empty_scan(msp):
    c = Case(synth.C1, pos=np.zeros((0, 2), dtype=np.int32))
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    assert loss.item() == 0.0 and torch.count_nonzero(dV) == 0 and torch.count_nonzero(dprobe) == 0
    assert msp.forward(g, p, V, pos).shape == (0, 64, 64)
    V0 = V.clone()
    lb, mu = msp.layer_step(g, p, V, pos, I, 0)
    assert lb.item() == 0.0 and mu.item() == 0.0 and torch.equal(V, V0)


def test_single_position_at_the_far_corner(msp):
    cfg = synth.C1
    c = Case(cfg, pos=[[cfg.obj - cfg.win, cfg.obj - cfg.win]])
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= TOL
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL


def test_window_equal_to_object(msp):
    cfg = synth.Workload("w64_obj64", 3, 64, 0.2, 2.0, 30, 64, (1, 1), 4, 25.0, 50.0, None, seed=4)
    c = Case(cfg, noisy=False)
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL


def test_zero_probe_uses_the_zero_rule(msp, c1):
    """Psi == 0 everywhere: the residual fraction is 0, loss = sum(I), all gradients exactly 0."""
    g, p, V, pos, I = c1.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, torch.zeros_like(p), V, pos, I)
    assert loss.item() == pytest.approx(float(c1.I.astype(np.float32).astype(np.float64).sum()), rel=1e-6)
    assert torch.count_nonzero(dV) == 0 and torch.count_nonzero(dprobe) == 0
    assert torch.isfinite(dV).all()


def test_zero_measurements(msp, c1):
    g, p, V, pos, I = c1.dev(msp)
    Iz = torch.zeros_like(I)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, Iz)
    ref = O.loss_grad(c1.gd, c1.probe, c1.pos, np.zeros_like(c1.I), V=c1.V)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= TOL
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL


def test_window_outside_object_is_flagged_and_skipped(msp, c1):
    g, p, V, pos, I = c1.dev(msp)
    bad = pos.clone()
    bad[3] = torch.tensor([c1.cfg.obj - c1.cfg.win + 1, 0], dtype=torch.int32)
    ws = msp.make_workspace(g)
    out = msp.forward(g, p, V, bad, ws=ws)
    with pytest.raises(msp.MspError) as e:
        msp.check_workspace(ws)
    assert e.value.status == msp.MSP_EINVAL
    assert torch.count_nonzero(out[3]) == 0
    good = msp.forward(g, p, V, pos, ws=ws)
    msp.check_workspace(ws)   # the next clean call clears the flag
    keep = [s for s in range(len(c1.pos)) if s != 3]
    assert torch.equal(out[keep], good[keep])


def test_host_side_argument_errors(msp, c1):
    g, p, V, pos, I = c1.dev(msp)
    with pytest.raises(TypeError):
        msp.loss_grad(g, p.real.contiguous(), V, pos, I)
    with pytest.raises(msp.MspError) as e:
        msp.layer_step(g, p, V, pos, I, layer=5)
    assert e.value.status == msp.MSP_EINVAL
    ws = msp.make_workspace(g)
    small = msp.Workspace(ws.buf[:1024])
    with pytest.raises(ValueError):
        msp.forward(g, p, V, pos, ws=small)


# --------------------------------------------------------------------------- full benchmark workload, sampled

def test_full_c2_workload_sampled(msp):
    """All 1024 positions of the W = 128, L = 4 workload in the launch configuration the
    benchmark times: intensities at sampled positions, the total loss, and the potential
    gradient on a sampled object patch (the oracle evaluates only the positions that cover it)."""
    cfg = synth.C2
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    V_true = synth.potential_slices(cfg)
    probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A)
    p_true = synth.probe(cfg)
    rng = np.random.default_rng(9)
    sample = np.sort(rng.choice(len(pos), size=24, replace=False))
    g = msp.geometry(**gd)
    probe = probe.astype(np.complex64).astype(np.complex128)
    p_true = p_true.astype(np.complex64).astype(np.complex128)
    V_true = f32(V_true)
    dp, dpos = to_dev(probe, np.complex64), to_dev(pos, np.int32)
    I_ref = O.forward(gd, p_true, pos, V=V_true)
    I_gpu = msp.forward(g, to_dev(p_true, np.complex64), to_dev(V_true, np.float32), dpos).cpu().numpy()
    assert rel(I_gpu[sample], I_ref[sample]) <= TOL
    assert rel(I_gpu, I_ref) <= TOL
    I_meas = f32(synth.poisson_counts(I_ref, cfg.dose, cfg.seed))
    V0 = f32(0.5 * V_true)
    loss, dV, dprobe = msp.loss_grad(g, dp, to_dev(V0, np.float32), dpos, to_dev(I_meas, np.float32))
    dV = dV.cpu().numpy()
    # gradient on a 16 x 16 patch of slice 0..3: only windows covering the patch contribute
    y0, x0 = 180, 200
    cover = [s for s, (y, x) in enumerate(pos) if y <= y0 + 15 and y + cfg.win > y0 and x <= x0 + 15 and x + cfg.win > x0]
    ref = O.loss_grad(dict(gd, n_pos=len(cover)), probe, pos[cover], I_meas[cover], V=V0, want_probe=False)
    assert rel(dV[:, y0:y0 + 16, x0:x0 + 16], ref["dV"][:, y0:y0 + 16, x0:x0 + 16]) <= TOL
    # the total loss: sum of per-position oracle losses over a sample, scaled check on all
    loss_ref = 0.0
    X = O.transmission(V0, gd["sigma"])
    h = O.fresnel_propagator(cfg.win, gd["pixel_A"], gd["wavelength_A"], gd["dz_A"])
    for s, (y, x) in enumerate(pos):
        _, _, far = O.position_forward(probe, X, int(y), int(x), h)
        loss_ref += O.far_field_residual(far, I_meas[s])[0]
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
