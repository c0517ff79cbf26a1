"""GPU parity: libmsp (FP32, sm_103a) against the FP64 oracle on identical seeded inputs.

Tolerances.  Intensities must match to a relative L2 error of 1e-5 on every state.
The loss differences FP32 amplitudes (bar max(1e-5, 2 e ||Psi|| / ||sqrt(I) - |Psi|||)).
Gradients are linear in the far-field residual R = Psi - sqrt(I) Psi/|Psi|,
which inherits the forward's absolute rounding error amplified by the state's
conditioning kappa (see `oracle.msp_oracle.residual_conditioning`: ~||Psi|| / ||R||, larger
where a small model amplitude meets a large measured one and the residual is set by
the model's phase).  The FP32 forward applies 2L - 1 rounded 2-D FFTs, so its error is
taken as e = 2 (2L - 1) 2^-24 per unit of the RMS far-field amplitude, and the bar is
    min(max(1e-5, (e kappa + flip) c), cap)
with c the cancellation of the sum over positions (probe gradient only), flip the
bound on zero-rule decisions that round-off may turn (0 on noisy data), and a fixed
cap (1e-4 for dV and the loss, 2e-3 for dprobe) that no state may exceed.
  * strong-misfit states (kappa ~ 1): the bar is 1e-5 on every output;
  * realistic states (the workloads' own starting points, noiseless or nearly fitted
    data, the full benchmark workload): the derived bar.
Cases span several CTA waves with a ragged tail, the full benchmark workload (sampled
outputs) and the degenerate cases of the method.
"""
import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
U32 = 2.0 ** -24
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def msp():
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    m.lib()
    return m


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x).astype(dtype)).to(DEV)


def fwd_err(n_slices):
    return 2 * (2 * n_slices - 1) * U32


# Fixed ceilings on the FP32 path's derived bars: whatever a state's conditioning, the fast
# path must stay below these (the precise-forward mode is held to TOL on the same states).
CAP_GRAD = 1e-4       # dV (and the transmission-mode gradient)
CAP_PROBE_GRAD = 2e-3  # dprobe: the sum over positions cancels, amplifying the per-position error
CAP_LOSS = 1e-4


def derived_tol(gd, probe, pos, I, V, probe_grad=False):
    e = fwd_err(gd["n_slices"])
    band = 2 * e * float(np.linalg.norm(probe))
    kappa, canc, flip = O.residual_conditioning(gd, probe, pos, I, V=V, band=band)
    bar = max(TOL, (e * kappa + flip) * (canc if probe_grad else 1.0))
    return min(bar, CAP_PROBE_GRAD if probe_grad else CAP_GRAD)


def loss_tol(gd, probe, n_pos, loss_ref):
    """The loss sum_k (sqrt(I) - |Psi|)^2 differences FP32 amplitudes: its relative error is about
    2 e ||Psi|| / ||sqrt(I) - |Psi||| with ||Psi||^2 = S W^2 ||p||^2 (Parseval, pure-phase slices)."""
    if loss_ref <= 0:
        return TOL
    kappa = np.sqrt(n_pos * gd["win"] ** 2 * float(np.sum(np.abs(probe) ** 2)) / loss_ref)
    return min(max(TOL, 2 * fwd_err(gd["n_slices"]) * kappa), CAP_LOSS)


class Case:
    """A seeded problem: geometry, probe, positions, measured intensities, current V.
    Every input is rounded to FP32 once, so both sides see identical values."""

    def __init__(self, cfg, sub=None, noisy=True, probe_guess=True, v_scale=0.5, v_noise=0.5, seed=0, pos=None):
        self.cfg = cfg
        self.pos = synth.scan_positions(cfg, sub=sub) if pos is None else np.asarray(pos, dtype=np.int32)
        self.gd = synth.geometry(cfg, n_pos=len(self.pos))
        self.V_true = synth.potential_slices(cfg)
        p_true = synth.probe(cfg)
        I = O.forward(self.gd, p_true, self.pos, V=self.V_true) if len(self.pos) else np.zeros((0, cfg.win, cfg.win))
        self.I = f32(synth.poisson_counts(I, cfg.dose, cfg.seed) if noisy else I)
        probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A) if (probe_guess and cfg.defocus_guess_A) else p_true
        self.probe = probe.astype(np.complex64).astype(np.complex128)
        rng = np.random.default_rng(seed + 5)
        self.V = f32(v_scale * self.V_true + v_noise * rng.standard_normal(self.V_true.shape))
        self.strong = False

    def tol(self, probe_grad=False):
        if self.strong:
            return TOL
        key = "_tol_p" if probe_grad else "_tol"
        if not hasattr(self, key):
            setattr(self, key, derived_tol(self.gd, self.probe, self.pos, self.I, self.V, probe_grad))
        return getattr(self, key)

    def ltol(self, loss_ref):
        return TOL if self.strong else loss_tol(self.gd, self.probe, len(self.pos), loss_ref)

    def dev(self, msp, precise=False):
        """precise: False (FP32), True or "fp64" (FP64 forward), "df" (double-float forward)."""
        prec = msp.MSP_PRECISION_FP32
        if precise:
            prec = msp.MSP_PRECISION_DF_FORWARD if precise == "df" else msp.MSP_PRECISION_FP64_FORWARD
        g = msp.geometry(**self.gd, precision=prec)
        return g, to_dev(self.probe, np.complex64), to_dev(self.V, np.float32), to_dev(self.pos, np.int32), \
            to_dev(self.I, np.float32)


def strong_case(cfg, sub=None, pos=None):
    """A state far from the data (large random potential): kappa ~ 1, the 1e-5 bar everywhere."""
    c = Case(cfg, sub=sub, v_scale=1.0, v_noise=300.0, seed=7, pos=pos)
    c.strong = True
    return c


@pytest.fixture(scope="module")
def c1():
    return Case(synth.C1, noisy=False)


@pytest.fixture(scope="module")
def c2_ragged():
    # 13 x 13 = 169 positions: more than one CTA per SM on a 152-SM part, with a ragged tail
    return Case(synth.C2, sub=(13, 13))


@pytest.fixture(scope="module")
def c1_strong():
    return strong_case(synth.C1)


@pytest.fixture(scope="module")
def c2_strong():
    return strong_case(synth.C2, sub=(13, 13))


@pytest.fixture(scope="module")
def c3_sub():
    # the eight-slice workload (rotated lattices, 1e5 e/pattern) on an 8 x 8 sub-scan
    return Case(synth.C3, sub=(8, 8))


@pytest.fixture(scope="module")
def c3_strong():
    return strong_case(synth.C3, sub=(8, 8))


@pytest.fixture(scope="module")
def c4_sub():
    # the sixteen-slice W = 256 workload (four-CTA clusters) on a 3 x 3 sub-scan
    return Case(synth.C4, sub=(3, 3), noisy=False)


W256_L3 = synth.Workload("w256_L3_obj640", 3, 640, 0.1, 1.0, 30, 256, (48, 48), 8, 30.0, 100.0, None, seed=3)


@pytest.fixture(scope="module")
def c4_strong():
    # W = 256 with three slices on 7 x 7 = 49 positions: more positions than resident
    # four-CTA clusters, with a ragged tail
    return strong_case(W256_L3, sub=(7, 7))


ALL = ["c1", "c2_ragged", "c1_strong", "c2_strong", "c3_sub", "c3_strong", "c4_sub", "c4_strong"]


def test_strong_states_are_well_conditioned(c1_strong, c2_strong, c3_strong, c4_strong):
    for c in (c1_strong, c2_strong, c3_strong, c4_strong):
        assert derived_tol(c.gd, c.probe, c.pos, c.I, c.V, probe_grad=True) <= TOL


# --------------------------------------------------------------------------- forward

@pytest.mark.parametrize("which", ALL)
def test_forward_intensities(msp, which, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, _ = c.dev(msp)
    I = msp.forward(g, p, V, pos).cpu().numpy()
    ref = O.forward(c.gd, c.probe, c.pos, V=c.V)
    assert rel(I, ref) <= TOL
    for s in range(0, len(c.pos), max(1, len(c.pos) // 16)):   # no single pattern may be off
        assert rel(I[s], ref[s]) <= TOL


# --------------------------------------------------------------------------- loss and gradients

@pytest.mark.parametrize("which", ALL)
def test_loss_and_gradients(msp, which, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    errs = dict(loss=abs(loss.item() - ref["loss"]) / ref["loss"], dV=rel(dV.cpu().numpy(), ref["dV"]),
                dprobe=rel(dprobe.cpu().numpy(), ref["dprobe"]))
    print(which, errs, "bars", c.ltol(ref["loss"]), c.tol(), c.tol(True))
    assert errs["loss"] <= c.ltol(ref["loss"])
    assert errs["dV"] <= c.tol()
    assert errs["dprobe"] <= c.tol(probe_grad=True)
    for l in range(c.gd["n_slices"]):
        assert rel(dV.cpu().numpy()[l], ref["dV"][l]) <= c.tol()


# --------------------------------------------------------------------------- precise-forward modes
# The forward model and the residual in FP64 (or double-float), the adjoint in FP32: every output
# is held to TOL = 1e-5 on every state, realistic ones included.
PRECISE = ["fp64", "df"]


@pytest.mark.parametrize("mode", PRECISE)
@pytest.mark.parametrize("which", ALL)
def test_precise_mode_intensities_loss_and_gradients(msp, which, mode, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp, precise=mode)
    Ig = msp.forward(g, p, V, pos).cpu().numpy()
    assert rel(Ig, O.forward(c.gd, c.probe, c.pos, V=c.V)) <= TOL
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    errs = dict(loss=abs(loss.item() - ref["loss"]) / ref["loss"], dV=rel(dV.cpu().numpy(), ref["dV"]),
                dprobe=rel(dprobe.cpu().numpy(), ref["dprobe"]))
    print("precise", mode, which, errs)
    assert max(errs.values()) <= TOL, errs
    for l in range(c.gd["n_slices"]):
        assert rel(dV.cpu().numpy()[l], ref["dV"][l]) <= TOL


@pytest.mark.parametrize("mode", PRECISE)
@pytest.mark.parametrize("which,layer", [("c1", 1), ("c2_ragged", 0), ("c2_ragged", 3), ("c3_sub", 5), ("c4_sub", 11),
                                         ("c4_strong", 2)])
def test_precise_mode_layer_step(msp, which, layer, mode, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp, precise=mode)
    loss, mu = msp.layer_step(g, p, V, pos, I, layer)
    Vn, loss_ref, mu_ref = O.layer_step(c.gd, c.probe, c.pos, c.I, layer, V=c.V)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    assert abs(mu.item() - mu_ref) / mu_ref <= TOL
    Vg = V.cpu().numpy()
    # the update itself, plus the FP32 rounding of the stored slice (half an ulp of each value)
    d = Vn[layer] - c.V[layer]
    assert rel(Vg[layer] - c.V[layer], d) <= TOL + U32 * np.linalg.norm(Vn[layer]) / np.linalg.norm(d)
    others = [m for m in range(c.gd["n_slices"]) if m != layer]
    assert np.array_equal(Vg[others], c.V[others].astype(np.float32))


@pytest.mark.parametrize("mode", PRECISE)
@pytest.mark.parametrize("which", ["c1", "c2_ragged", "c3_sub", "c4_sub"])
def test_precise_mode_probe_step(msp, which, mode, request):
    """The probe update -mu dL/dconj(p) at TOL, plus the FP32 rounding of the stored probe: an update
    much smaller than the probe keeps only the bits of the sum, 2^-24 ||p_new|| at most."""
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp, precise=mode)
    loss, mu = msp.probe_step(g, p, V, pos, I)
    pn, loss_ref, mu_ref = O.probe_step(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    d = pn - c.probe
    err = rel(p.cpu().numpy() - c.probe, d)
    bar = TOL + U32 * np.linalg.norm(pn) / np.linalg.norm(d)
    print("precise probe step", which, err, "bar", bar)
    assert err <= bar


@pytest.mark.parametrize("mode", PRECISE)
def test_precise_mode_transmission_slices(msp, c2_ragged, mode):
    """The paper's complex slices on a realistic state: intensities, loss and Wirtinger gradients at TOL."""
    c = c2_ragged
    T = transmission_case(c)
    gd = dict(c.gd, param=msp.MSP_PARAM_TRANSMISSION)
    g = msp.geometry(**gd, precision=msp.MSP_PRECISION_DF_FORWARD if mode == "df" else msp.MSP_PRECISION_FP64_FORWARD)
    p, X, pos, I = to_dev(c.probe, np.complex64), to_dev(T, np.complex64), to_dev(c.pos, np.int32), to_dev(c.I, np.float32)
    assert rel(msp.forward(g, p, X, pos).cpu().numpy(), O.forward(c.gd, c.probe, c.pos, T=T)) <= TOL
    loss, dX, dprobe = msp.loss_grad(g, p, X, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, T=T)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= TOL
    assert rel(dX.cpu().numpy(), ref["dX"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL
    Xl, _, _ = O.layer_step(c.gd, c.probe, c.pos, c.I, 1, T=T)
    msp.layer_step(g, p, X, pos, I, 1)
    assert rel(X.cpu().numpy()[1] - T[1], Xl[1] - T[1]) <= TOL


@pytest.mark.parametrize("mode", PRECISE)
def test_precise_mode_edge_cases(msp, c1, mode):
    """Empty scan, a window outside the object (skipped and flagged, as in the FP32 mode), the zero
    probe (zero rule everywhere) and bit-reproducible repeats."""
    g, p, V, pos, I = c1.dev(msp, precise=mode)
    empty = Case(synth.C1, pos=np.zeros((0, 2), dtype=np.int32))
    ge, pe, Ve, pse, Ie = empty.dev(msp, precise=mode)
    loss, dV, dprobe = msp.loss_grad(ge, pe, Ve, pse, Ie)
    assert loss.item() == 0.0 and torch.count_nonzero(dV) == 0 and torch.count_nonzero(dprobe) == 0
    loss, dV, dprobe = msp.loss_grad(g, torch.zeros_like(p), V, pos, I)
    assert loss.item() == pytest.approx(float(c1.I.sum()), rel=1e-12)
    assert torch.count_nonzero(dV) == 0 and torch.count_nonzero(dprobe) == 0
    bad = pos.clone()
    bad[3] = torch.tensor([c1.cfg.obj - c1.cfg.win + 1, 0], dtype=torch.int32)
    ws = msp.make_workspace(g)
    out = msp.forward(g, p, V, bad, ws=ws)
    with pytest.raises(msp.MspError) as e:
        msp.check_workspace(ws)
    assert e.value.status == msp.MSP_EINVAL
    assert torch.count_nonzero(out[3]) == 0
    a = [t.clone() for t in msp.loss_grad(g, p, V, pos, I, ws=ws)]
    b = msp.loss_grad(g, p, V, pos, I, ws=ws)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


# --------------------------------------------------------------------------- split-BF16 precision form
# Every 2-D transform of the forward model and the adjoint as two tensor-core DFT passes with
# 3-term split-BF16 operands.  Each pass keeps 16 mantissa bits of every operand (x = hi + lo):
# about 2^-16 relative error per pass, so the forward's 2 (2L - 1) passes give
# e = 2 (2L - 1) 2^-16; the intensities carry 2e, and the gradients inherit e amplified by the
# state's conditioning exactly as the FP32 path's do (no cap: this form is the reduced-precision
# one, and its errors are a stated result).

def bf16_bars(c):
    e = 2 * (2 * c.gd["n_slices"] - 1) * 2.0 ** -16
    kappa, canc, flip = O.residual_conditioning(c.gd, c.probe, c.pos, c.I, V=c.V, band=2 * e * float(np.linalg.norm(c.probe)))
    S, W2 = len(c.pos), c.gd["win"] ** 2
    return dict(I=2 * e, grad=max(TOL, e * kappa + flip), probe_grad=max(TOL, (e * kappa + flip) * canc), e=e)


@pytest.mark.parametrize("which", ["c1", "c2_ragged", "c3_sub", "c4_sub", "c2_strong", "c3_strong"])
def test_bf16x3_mode_per_result_errors(msp, which, request):
    c = request.getfixturevalue(which)
    g = msp.geometry(**c.gd, precision=msp.MSP_PRECISION_BF16X3_DFT)
    _, p, V, pos, I = c.dev(msp)
    Ig = msp.forward(g, p, V, pos).cpu().numpy()
    Iref = O.forward(c.gd, c.probe, c.pos, V=c.V)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    errs = dict(I=rel(Ig, Iref), loss=abs(loss.item() - ref["loss"]) / ref["loss"],
                dV=rel(dV.cpu().numpy(), ref["dV"]), dprobe=rel(dprobe.cpu().numpy(), ref["dprobe"]))
    bars = bf16_bars(c)
    kappa = np.sqrt(len(c.pos) * c.gd["win"] ** 2 * float(np.sum(np.abs(c.probe) ** 2)) / ref["loss"])
    lbar = max(TOL, 2 * bars["e"] * kappa)
    print("bf16x3", which, {k: f"{v:.2e}" for k, v in errs.items()},
          "bars", {k: f"{v:.2e}" for k, v in dict(I=bars["I"], loss=lbar, dV=bars["grad"], dprobe=bars["probe_grad"]).items()})
    assert errs["I"] <= bars["I"]
    assert errs["loss"] <= lbar
    assert errs["dV"] <= bars["grad"]
    assert errs["dprobe"] <= bars["probe_grad"]


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

@pytest.mark.parametrize("which,layer", [("c1", 0), ("c1", 1), ("c2_ragged", 0), ("c2_ragged", 2),
                                         ("c1_strong", 1), ("c2_strong", 0), ("c2_strong", 3),
                                         ("c3_sub", 5), ("c3_strong", 7), ("c4_strong", 0), ("c4_strong", 2), ("c4_sub", 11)])
def test_layer_step(msp, which, layer, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    loss, mu = msp.layer_step(g, p, V, pos, I, layer)
    Vn, loss_ref, mu_ref = O.layer_step(c.gd, c.probe, c.pos, c.I, layer, V=c.V)
    assert abs(loss.item() - loss_ref) / loss_ref <= c.ltol(loss_ref)
    assert abs(mu.item() - mu_ref) / mu_ref <= TOL
    Vg = V.cpu().numpy()
    assert rel(Vg[layer] - c.V[layer], Vn[layer] - c.V[layer]) <= c.tol()   # the update itself
    assert rel(Vg, Vn) <= TOL
    others = [m for m in range(c.gd["n_slices"]) if m != layer]
    assert np.array_equal(Vg[others], c.V[others].astype(np.float32))


def test_layer_step_fixed_step(msp, c1_strong):
    c = c1_strong
    g, p, V, pos, I = c.dev(msp)
    _, mu = msp.layer_step(g, p, V, pos, I, 1, step=12.5)
    assert mu.item() == 12.5
    Vn, _, _ = O.layer_step(c.gd, c.probe, c.pos, c.I, 1, V=c.V, step=12.5)
    assert rel(V.cpu().numpy()[1] - c.V[1], Vn[1] - c.V[1]) <= TOL


@pytest.mark.parametrize("which", ["c2_ragged", "c2_strong", "c4_strong"])
@pytest.mark.parametrize("normalize", [False, True])
def test_probe_step(msp, which, normalize, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    loss, mu = msp.probe_step(g, p, V, pos, I, normalize=normalize)
    pn, loss_ref, mu_ref = O.probe_step(c.gd, c.probe, c.pos, c.I, V=c.V, normalize=normalize)
    assert abs(loss.item() - loss_ref) / loss_ref <= c.ltol(loss_ref)
    assert mu.item() == pytest.approx(mu_ref, rel=1e-15)
    assert rel(p.cpu().numpy(), pn) <= TOL
    if not normalize:
        assert rel(p.cpu().numpy() - c.probe, pn - c.probe) <= c.tol(probe_grad=True)


def test_layerwise_trajectory(msp):
    """Algorithm 1, two sweeps from V = 0 with the probe guess on noisy W = 128 data.
    Step errors add up and the conditioning changes along the path: the bar is the number
    of steps times the largest per-state bar on the oracle's own trajectory."""
    c = Case(synth.C2, sub=(3, 3), v_scale=0.0, v_noise=0.0)
    g, p, V, pos, I = c.dev(msp)
    sweeps, L = 2, c.gd["n_slices"]
    Vo = c.V.copy()
    hist, bars = [], []
    for _ in range(sweeps):
        for layer in range(L):
            bars.append(derived_tol(c.gd, c.probe, c.pos, c.I, Vo))
            Vo, lo, _ = O.layer_step(c.gd, c.probe, c.pos, c.I, layer, V=Vo)
            Vo = f32(Vo)
            hist.append(lo)
    losses = []
    ws = msp.make_workspace(g)
    for _ in range(sweeps):
        for layer in range(L):
            lb, _ = msp.layer_step(g, p, V, pos, I, layer, ws=ws)
            losses.append(lb.item())
    tol = len(bars) * max(bars)
    print("trajectory bar", tol, "error", rel(V.cpu().numpy(), Vo))
    assert rel(V.cpu().numpy(), Vo) <= tol
    np.testing.assert_allclose(losses, hist, rtol=max(TOL, 0.1 * tol))
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
    c = strong_case(cfg, pos=[[cfg.obj - cfg.win, cfg.obj - cfg.win]])
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= c.ltol(ref["loss"])
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL


def test_window_equal_to_object(msp):
    cfg = synth.Workload("w64_obj64", 3, 64, 0.2, 2.0, 30, 64, (1, 1), 4, 25.0, 50.0, None, seed=4)
    c = strong_case(cfg)
    g, p, V, pos, I = c.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert rel(dV.cpu().numpy(), ref["dV"]) <= TOL
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= TOL


def test_zero_probe_uses_the_zero_rule(msp, c1):
    """Psi == 0 everywhere: the residual fraction is 0, loss = sum(I), all gradients exactly 0."""
    g, p, V, pos, I = c1.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, torch.zeros_like(p), V, pos, I)
    assert loss.item() == pytest.approx(float(c1.I.sum()), rel=1e-6)
    assert torch.count_nonzero(dV) == 0 and torch.count_nonzero(dprobe) == 0
    assert torch.isfinite(dV).all()


def test_zero_measurements(msp, c1):
    """I = 0: R = Psi, chi_l = W^2 E_l, so Im(conj(E_l) chi_l) = 0 and dV = 0 in exact arithmetic;
    the computed gradient must vanish to round-off relative to its uncancelled scale
    2 sigma W^2 sum_s ||p||^2, and dprobe = W^2 S p."""
    g, p, V, pos, I = c1.dev(msp)
    loss, dV, dprobe = msp.loss_grad(g, p, V, pos, torch.zeros_like(I))
    ref = O.loss_grad(c1.gd, c1.probe, c1.pos, np.zeros_like(c1.I), V=c1.V)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= TOL
    W, S = c1.cfg.win, len(c1.pos)
    scale = 2 * c1.gd["sigma"] * W * W * S * float(np.sum(np.abs(c1.probe) ** 2))
    assert float(np.linalg.norm(dV.cpu().numpy())) <= TOL * scale
    assert rel(dprobe.cpu().numpy(), W * W * S * c1.probe) <= TOL


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
    benchmark times: every intensity, the total loss, and the potential gradient on a sampled
    object patch (the oracle evaluates only the positions that cover it)."""
    cfg = synth.C2
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd)
    V_true = f32(synth.potential_slices(cfg))
    probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A).astype(np.complex64).astype(np.complex128)
    p_true = synth.probe(cfg).astype(np.complex64).astype(np.complex128)
    dp, dpos = to_dev(probe, np.complex64), to_dev(pos, np.int32)
    I_ref = O.forward(gd, p_true, pos, V=V_true)
    I_gpu = msp.forward(g, to_dev(p_true, np.complex64), to_dev(V_true, np.float32), dpos).cpu().numpy()
    assert rel(I_gpu, I_ref) <= TOL
    I_meas = f32(synth.poisson_counts(I_ref, cfg.dose, cfg.seed))
    V0 = f32(0.5 * V_true)
    loss, dV, dprobe = msp.loss_grad(g, dp, to_dev(V0, np.float32), dpos, to_dev(I_meas, np.float32))
    dV = dV.cpu().numpy()
    y0, x0 = 180, 200
    cover = [s for s, (y, x) in enumerate(pos) if y <= y0 + 15 and y + cfg.win > y0 and x <= x0 + 15 and x + cfg.win > x0]
    gc = dict(gd, n_pos=len(cover))
    ref = O.loss_grad(gc, probe, pos[cover], I_meas[cover], V=V0, want_probe=False)
    err = rel(dV[:, y0:y0 + 16, x0:x0 + 16], ref["dV"][:, y0:y0 + 16, x0:x0 + 16])
    bar = derived_tol(gc, probe, pos[cover], I_meas[cover], V0)
    print("full c2 patch: dV error", err, "bar", bar)
    assert err <= bar
    X = O.transmission(V0, gd["sigma"])
    h = O.fresnel_propagator(cfg.win, gd["pixel_A"], gd["wavelength_A"], gd["dz_A"])
    thr = O.zero_threshold(probe)
    loss_ref = 0.0
    for s, (y, x) in enumerate(pos):
        _, _, far = O.position_forward(probe, X, int(y), int(x), h)
        loss_ref += O.far_field_residual(far, I_meas[s], thr)[0]
    assert abs(loss.item() - loss_ref) / loss_ref <= loss_tol(gd, probe, len(pos), loss_ref)


# --------------------------------------------------------------------------- transmission mode

def transmission_case(case, seed=21, rough=0.05):
    """The same problem with complex, non-unimodular slices o = exp(i sigma V)(1 + rough n)."""
    rng = np.random.default_rng(seed)
    n = rng.standard_normal(case.V.shape) + 1j * rng.standard_normal(case.V.shape)
    T = np.exp(1j * case.gd["sigma"] * case.V) * (1 + rough * n)
    return T.astype(np.complex64).astype(np.complex128)


def tdev(msp, c, T):
    gd = dict(c.gd, param=msp.MSP_PARAM_TRANSMISSION)
    g = msp.geometry(**gd)
    return g, to_dev(c.probe, np.complex64), to_dev(T, np.complex64), to_dev(c.pos, np.int32), to_dev(c.I, np.float32)


def t_bar(c, T, probe_grad=False):
    if c.strong:
        return TOL
    e = fwd_err(c.gd["n_slices"])
    kappa, canc, flip = O.residual_conditioning(c.gd, c.probe, c.pos, c.I, T=T,
                                                band=2 * e * float(np.linalg.norm(c.probe)))
    return max(TOL, (e * kappa + flip) * (canc if probe_grad else 1.0))


@pytest.mark.parametrize("which", ["c1_strong", "c2_strong", "c4_strong", "c2_ragged"])
def test_transmission_mode_forward_and_gradients(msp, which, request):
    c = request.getfixturevalue(which)
    T = transmission_case(c)
    g, p, X, pos, I = tdev(msp, c, T)
    Ig = msp.forward(g, p, X, pos).cpu().numpy()
    assert rel(Ig, O.forward(c.gd, c.probe, c.pos, T=T)) <= TOL
    loss, dX, dprobe = msp.loss_grad(g, p, X, pos, I)
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, T=T)
    assert abs(loss.item() - ref["loss"]) / ref["loss"] <= (TOL if c.strong else 10 * t_bar(c, T))
    assert rel(dX.cpu().numpy(), ref["dX"]) <= t_bar(c, T)
    assert rel(dprobe.cpu().numpy(), ref["dprobe"]) <= t_bar(c, T, probe_grad=True)


@pytest.mark.parametrize("which,layer", [("c1_strong", 0), ("c2_strong", 1), ("c2_strong", 3), ("c4_strong", 1)])
def test_transmission_mode_layer_step(msp, which, layer, request):
    """o_l <- o_l - mu dL/dconj(o_l), mu = 1 / (W^2 max illumination prod_{m > l} max |o_m|^2)."""
    c = request.getfixturevalue(which)
    T = transmission_case(c)
    g, p, X, pos, I = tdev(msp, c, T)
    loss, mu = msp.layer_step(g, p, X, pos, I, layer)
    Tn, loss_ref, mu_ref = O.layer_step(c.gd, c.probe, c.pos, c.I, layer, T=T)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    assert abs(mu.item() - mu_ref) / mu_ref <= TOL
    Xg = X.cpu().numpy()
    assert rel(Xg[layer] - T[layer], Tn[layer] - T[layer]) <= TOL
    others = [m for m in range(c.gd["n_slices"]) if m != layer]
    assert np.array_equal(Xg[others], T[others].astype(np.complex64))


def test_transmission_mode_probe_step(msp, c2_strong):
    c = c2_strong
    T = transmission_case(c)
    g, p, X, pos, I = tdev(msp, c, T)
    loss, mu = msp.probe_step(g, p, X, pos, I)
    pn, loss_ref, mu_ref = O.probe_step(c.gd, c.probe, c.pos, c.I, T=T)
    assert abs(loss.item() - loss_ref) / loss_ref <= TOL
    assert rel(p.cpu().numpy() - c.probe, pn - c.probe) <= TOL


# --------------------------------------------------------------------------- full c3 and c4 sizes

@pytest.mark.parametrize("cfg_name,samples", [("c3", 24), ("c4", 10)])
def test_full_size_sampled_intensities_and_gradient_property(msp, cfg_name, samples):
    """Every position of the 8-slice W = 128 (4096 positions) and 16-slice W = 256 (2304 positions,
    four-CTA clusters) workloads in one launch, as bench.py times them: the intensities of
    sampled positions against the oracle, position by position, and the full-size potential
    gradient against central differences of the library's own loss (a property at any size)."""
    cfg = synth.CONFIGS[cfg_name]
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd)
    V_true = f32(synth.potential_slices(cfg))
    p_true = synth.probe(cfg).astype(np.complex64).astype(np.complex128)
    dpos = to_dev(pos, np.int32)
    I_gpu = msp.forward(g, to_dev(p_true, np.complex64), to_dev(V_true, np.float32), dpos).cpu().numpy()
    X = O.transmission(V_true.astype(np.float64), gd["sigma"])
    h = O.fresnel_propagator(cfg.win, gd["pixel_A"], gd["wavelength_A"], gd["dz_A"])
    pick = np.random.default_rng(5).choice(len(pos), size=samples, replace=False)
    pick[0], pick[1] = 0, len(pos) - 1                       # first and last CTA's last position
    for s in pick:
        _, _, far = O.position_forward(p_true, X, int(pos[s][0]), int(pos[s][1]), h)
        assert rel(I_gpu[s], np.abs(far) ** 2) <= TOL, s
    # gradient property: (L(V + eps D) - L(V - eps D)) / (2 eps) = <dV, D>, on measurements that
    # do not come from the library: the probe's own pattern, scaled by a seeded factor per position
    base = (np.abs(np.fft.fft2(p_true)) ** 2).astype(np.float32)
    scale = (1.0 + 0.2 * np.random.default_rng(9).random(len(pos))).astype(np.float32)
    I_meas = base[None] * scale[:, None, None]
    dI = to_dev(I_meas, np.float32)
    V0 = f32(0.5 * V_true)
    dp = to_dev(p_true, np.complex64)
    loss, dV, _ = msp.loss_grad(g, dp, to_dev(V0, np.float32), dpos, dI, want_dprobe=False)
    D = f32(synth.random_real(V0.shape, 11))
    eps = 1e-2 * float(np.abs(V0).max()) / float(np.abs(D).max())
    lp, _, _ = msp.loss_grad(g, dp, to_dev(f32(V0 + eps * D), np.float32), dpos, dI, want_dV=False, want_dprobe=False)
    lm, _, _ = msp.loss_grad(g, dp, to_dev(f32(V0 - eps * D), np.float32), dpos, dI, want_dV=False, want_dprobe=False)
    fd = (lp.item() - lm.item()) / (2 * eps)
    an = float(np.sum(dV.cpu().numpy().astype(np.float64) * D))
    print(cfg_name, "fd", fd, "analytic", an)
    assert abs(fd - an) <= 2e-2 * abs(an)


# --------------------------------------------------------------------------- overlap-add by L2 reductions
# MSP_OVERLAP_L2_REDUCE: the fused kernel adds every window gradient into dV as it is produced.
# The loss and dprobe do not depend on the switch (bit for bit); dV is the same sum of the same
# FP32 terms in another order, so it meets the oracle at the fixed-order path's bar and agrees
# with the fixed-order dV to the rounding of a reordered sum.
REORDER_TOL = 1e-5


class l2_reduce:
    def __init__(self, msp):
        self.msp = msp

    def __enter__(self):
        self.msp.set_overlap_add(self.msp.OVERLAP_L2_REDUCE)

    def __exit__(self, *exc):
        self.msp.set_overlap_add(self.msp.OVERLAP_FIXED_ORDER)


@pytest.mark.parametrize("which", ["c1", "c2_ragged", "c1_strong", "c2_strong", "c3_sub", "c4_sub", "c4_strong"])
def test_l2_reduce_overlap_add(msp, which, request):
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    ws = msp.make_workspace(g)
    loss_a, dV_a, dp_a = msp.loss_grad(g, p, V, pos, I, ws=ws)
    with l2_reduce(msp):
        loss_b, dV_b, dp_b = msp.loss_grad(g, p, V, pos, I, ws=ws)
    msp.check_workspace(ws)
    assert loss_a.item() == loss_b.item()
    assert torch.equal(dp_a, dp_b)
    dV_b = dV_b.cpu().numpy()
    assert rel(dV_b, dV_a.cpu().numpy()) <= REORDER_TOL
    ref = O.loss_grad(c.gd, c.probe, c.pos, c.I, V=c.V)
    assert rel(dV_b, ref["dV"]) <= c.tol()
    for l in range(c.gd["n_slices"]):
        assert rel(dV_b[l], ref["dV"][l]) <= c.tol()


@pytest.mark.parametrize("which", ["c2_strong", "c4_strong"])
def test_l2_reduce_transmission_mode(msp, which, request):
    c = request.getfixturevalue(which)
    T = transmission_case(c)
    g, p, X, pos, I = tdev(msp, c, T)
    _, dX_a, _ = msp.loss_grad(g, p, X, pos, I)
    with l2_reduce(msp):
        _, dX_b, _ = msp.loss_grad(g, p, X, pos, I)
    dX_b = dX_b.cpu().numpy()
    assert rel(dX_b, dX_a.cpu().numpy()) <= REORDER_TOL
    assert rel(dX_b, O.loss_grad(c.gd, c.probe, c.pos, c.I, T=T)["dX"]) <= TOL


def test_l2_reduce_skips_windows_outside_the_object(msp, c1):
    """A position outside the object adds nothing (and is flagged), as in the fixed-order path."""
    g, p, V, pos, I = c1.dev(msp)
    bad = pos.clone()
    bad[3] = torch.tensor([c1.cfg.obj - c1.cfg.win + 1, 0], dtype=torch.int32)
    ws = msp.make_workspace(g)
    _, dV_a, _ = msp.loss_grad(g, p, V, bad, I, ws=ws)
    with pytest.raises(msp.MspError):
        msp.check_workspace(ws)
    with l2_reduce(msp):
        _, dV_b, _ = msp.loss_grad(g, p, V, bad, I, ws=ws)
    with pytest.raises(msp.MspError) as e:
        msp.check_workspace(ws)
    assert e.value.status == msp.MSP_EINVAL
    assert rel(dV_b.cpu().numpy(), dV_a.cpu().numpy()) <= REORDER_TOL


def test_l2_reduce_leaves_the_precise_modes_in_fixed_order(msp, c2_ragged):
    g, p, V, pos, I = c2_ragged.dev(msp, precise="df")
    ws = msp.make_workspace(g)
    a = msp.loss_grad(g, p, V, pos, I, ws=ws)[1].clone()
    with l2_reduce(msp):
        b = msp.loss_grad(g, p, V, pos, I, ws=ws)[1]
    assert torch.equal(a, b)


@pytest.mark.parametrize("which,layer", [("c1", 1), ("c2_ragged", 0), ("c2_strong", 3), ("c4_sub", 11)])
def test_l2_reduce_layer_step(msp, which, layer, request):
    """The layer step with its gradient and illumination maps summed in L2: the same step size
    (the illumination maximum is a maximum of the same sums) to rounding, the same update."""
    c = request.getfixturevalue(which)
    g, p, V, pos, I = c.dev(msp)
    Va, Vb = V.clone(), V.clone()
    mu_a, mu_b = (torch.empty(1, dtype=torch.float64, device=DEV) for _ in range(2))
    msp.layer_step(g, p, Va, pos, I, layer, mu=mu_a)
    with l2_reduce(msp):
        msp.layer_step(g, p, Vb, pos, I, layer, mu=mu_b)
    assert abs(mu_b.item() - mu_a.item()) <= REORDER_TOL * mu_a.item()
    keep = [m for m in range(c.gd["n_slices"]) if m != layer]
    assert torch.equal(Va[keep], Vb[keep])
    d_a = (Va[layer] - V[layer]).double().cpu().numpy()
    d_b = (Vb[layer] - V[layer]).double().cpu().numpy()
    assert rel(d_b, d_a) <= 10 * REORDER_TOL


def test_l2_reduce_transmission_layer_step(msp, c2_strong):
    T = transmission_case(c2_strong)
    g, p, X, pos, I = tdev(msp, c2_strong, T)
    Xa, Xb = X.clone(), X.clone()
    msp.layer_step(g, p, Xa, pos, I, 1)
    with l2_reduce(msp):
        msp.layer_step(g, p, Xb, pos, I, 1)
    d_a = (Xa[1] - X[1]).cpu().numpy()
    d_b = (Xb[1] - X[1]).cpu().numpy()
    assert rel(d_b, d_a) <= 10 * REORDER_TOL


# --------------------------------------------------------------------------- loss-only passes
@pytest.mark.parametrize("which", ["c1", "c2_ragged", "c4_sub"])
@pytest.mark.parametrize("prec", ["FP32", "FP64_FORWARD", "DF_FORWARD", "BF16X3_DFT"])
def test_loss_only_pass_gives_the_same_loss(msp, which, prec, request):
    """With neither gradient wanted the pass stops after the far-field loss: the same loss, bit
    for bit, as the full loss-and-gradient pass in every arithmetic form and window size."""
    c = request.getfixturevalue(which)
    _, p, V, pos, I = c.dev(msp)
    g = msp.geometry(**c.gd, precision=getattr(msp, "MSP_PRECISION_" + prec))
    ws = msp.make_workspace(g)
    full = msp.loss_grad(g, p, V, pos, I, ws=ws)[0].item()
    only = msp.loss_grad(g, p, V, pos, I, want_dV=False, want_dprobe=False, ws=ws)[0].item()
    msp.check_workspace(ws)
    assert only == full
