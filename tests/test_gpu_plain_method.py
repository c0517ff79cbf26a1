"""GPU parity of the plain method (msp_reconstruct): Algorithm 1 (Sec. 3.3) with optional probe
steps (Sec. 3.5), run by the library on the device, against the oracle's plain_method on the same
seeded inputs.

The library stores the slices and the probe in FP32 between steps, so the oracle's path is
rounded the same way after every step (its arithmetic stays FP64); what remains is the
gradient error of each step.  A trajectory adds those up: after N steps the potentials may
differ from the oracle's by at most
    b * sum_k ||V_{k+1} - V_k|| + N 2^-24 max_k ||V_k||
(relative to the final ||V||), b being the largest per-step gradient bar on the oracle's path:
TOL in the precise-forward mode, the FP32 bar of test_gpu_parity (without its cap, evaluated at
every state of the path) in the FP32 mode; the second term covers FP32 rounding decisions that
the two sides take differently.  That sum assumes the iteration does not amplify a deviation;
the reconstruction problem has nearly flat directions (the slice ambiguities of Sec. 5), along
which gradient descent carries a deviation on, so the bar is multiplied by the amplification
measured on the oracle itself: the divergence of its path with and without FP32 storage of the
state, over the size those roundings would have unamplified.  The loss before step k depends on
the accumulated deviation of V_k: its bar is the loss bar of the state plus b times the steps
taken so far."""
import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
U32 = 2.0 ** -24
TOL = 1e-5


@pytest.fixture(scope="module")
def msp():
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    m.lib()
    return m


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x).astype(dtype)).to(DEV)


def grad_bar(gd, probe, pos, I, V):
    """The per-state FP32 gradient bar of test_gpu_parity (uncapped: here it is a bound, and the
    trajectory bar takes the largest one met)."""
    e = 2 * (2 * gd["n_slices"] - 1) * U32
    kappa, canc, flip = O.residual_conditioning(gd, probe, pos, I, V=V, band=2 * e * float(np.linalg.norm(probe)))
    return max(TOL, e * kappa + flip), max(TOL, (e * kappa + flip) * canc)


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def oracle_path(gd, probe, pos, I, V0, sweeps, probe_steps=0, bars=True, round32=True):
    """The oracle's plain method step by step, its slices and probe rounded to FP32 after every
    step as the library stores them (unless round32 is False), keeping what the trajectory bar
    needs: the path length, the largest ||V||, the per-step FP32 bars (gradient, probe gradient)
    and each state's FP32 loss bar."""
    r32 = f32 if round32 else (lambda x: np.asarray(x, dtype=np.float64))
    rc = c64 if round32 else (lambda x: np.asarray(x, dtype=np.complex128))
    V, p = r32(V0), rc(probe)
    hist, path, vmax, b, bp, lbar = [], 0.0, float(np.linalg.norm(V)), 0.0, 0.0, []
    L = gd["n_slices"]
    e = 2 * (2 * L - 1) * U32
    S, W2 = len(pos), gd["win"] ** 2

    def loss_bar(loss, p):   # the FP32 loss bar of test_gpu_parity (uncapped)
        return max(TOL, 2 * e * np.sqrt(S * W2 * float(np.sum(np.abs(p) ** 2)) / loss)) if loss > 0 else TOL

    for _ in range(sweeps):
        for layer in range(L):
            if bars:
                bv, bpv = grad_bar(gd, p, pos, I, V)
                b, bp = max(b, bv), max(bp, bpv)
            Vn, loss, _ = O.layer_step(gd, p, pos, I, layer, V=V)
            Vn = r32(Vn)
            path += float(np.linalg.norm(Vn - V))
            V = Vn
            vmax = max(vmax, float(np.linalg.norm(V)))
            hist.append(loss)
            lbar.append(loss_bar(loss, p))
        for _ in range(probe_steps):
            p, loss, _ = O.probe_step(gd, p, pos, I, V=V)
            p = rc(p)
            hist.append(loss)
            lbar.append(loss_bar(loss, p))
    hist.append(O.loss_grad(gd, p, pos, I, V=V, want_probe=False)["loss"])
    lbar.append(loss_bar(hist[-1], p))
    return dict(V=V, p=p, hist=hist, path=path, vmax=vmax, b=b, bp=bp, lbar=np.asarray(lbar))


def amplification(o, unrounded, n):
    """How strongly the path amplifies step-level perturbations: the divergence between the oracle
    path with and without FP32 rounding of the stored state, over what n independent roundings
    of half an ulp would give without amplification (U32 sqrt(n) max||V||)."""
    d = rel(unrounded["V"], o["V"])
    return max(1.0, d / (U32 * np.sqrt(n) * o["vmax"] / float(np.linalg.norm(o["V"])))), d


def check_path(tag, h, o, V, b, n, loss_bars, amp=1.0, p=None, bp=None):
    Vr, hist = o["V"], np.asarray(o["hist"])
    v_bar = amp * (b * o["path"] + n * U32 * o["vmax"]) / float(np.linalg.norm(Vr))
    v_err = rel(V, Vr)
    h_err = np.abs(h - hist) / hist
    h_bar = loss_bars + b * np.minimum(np.arange(len(hist)), n)
    msg = (f"{tag}: V error {v_err:.3e} (bar {v_bar:.3e}, amplification {amp:.1f}), loss-history error max "
           f"{h_err.max():.3e} (first {h_err[0]:.2e}, last {h_err[-1]:.2e}), final loss {h[-1]:.6e} vs "
           f"{hist[-1]:.6e}, per-step bar {b:.2e}")
    pr = o["p"]
    if p is not None:
        msg += f", probe error {rel(p, pr):.3e} (bar {bp * n:.3e})"
    print(msg)
    assert v_err <= v_bar, msg
    assert np.all(h_err <= h_bar), msg
    if p is not None:
        assert rel(p, pr) <= bp * n, msg


PRECISIONS = ["fp32", "precise", "df"]


@pytest.mark.parametrize("mode", PRECISIONS)
def test_c1_fifty_sweeps_from_zero_with_known_probe(msp, mode):
    """The oracle-size workload as specified: 2 slices, 8 x 8 scan, noiseless, known probe,
    50 layer-wise iterations from V = 0; trajectory and final loss against the oracle."""
    cfg = synth.C1
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    V_true = synth.potential_slices(cfg)
    probe = c64(synth.probe(cfg))
    I = f32(O.forward(gd, probe, pos, V=V_true))
    V0 = np.zeros_like(V_true)
    sweeps = 50
    n = sweeps * cfg.n_slices
    o = oracle_path(gd, probe, pos, I, V0, sweeps, bars=mode == "fp32")
    assert o["hist"][-1] < 0.05 * o["hist"][0]          # the method converges on noiseless data
    amp, d = amplification(o, oracle_path(gd, probe, pos, I, V0, sweeps, bars=False, round32=False), n)
    print(f"c1 50 sweeps: oracle paths with and without FP32 storage differ by {d:.3e}")
    prec = {"fp32": msp.MSP_PRECISION_FP32, "precise": msp.MSP_PRECISION_FP64_FORWARD,
            "df": msp.MSP_PRECISION_DF_FORWARD}[mode]
    g = msp.geometry(**gd, precision=prec)
    V = to_dev(V0, np.float32)
    h = msp.reconstruct(g, msp.plan(sweeps), to_dev(probe, np.complex64), V, to_dev(pos, np.int32),
                        to_dev(I, np.float32)).cpu().numpy()
    assert len(h) == len(o["hist"]) == n + 1
    if mode != "fp32":
        check_path(f"c1 50 sweeps {mode}", h, o, V.cpu().numpy(), TOL, n, TOL, amp)
    else:
        check_path("c1 50 sweeps fp32", h, o, V.cpu().numpy(), o["b"], n, o["lbar"], amp)


@pytest.mark.parametrize("mode", PRECISIONS)
def test_c2_sub_scan_with_probe_estimation(msp, mode):
    """The W = 128, L = 4 workload's plain method with probe estimation on a 4 x 4 sub-scan:
    from V = 0 and the probe guess with a 20 angstrom defocus error, three sweeps of the four
    slice steps followed by one probe step each."""
    cfg = synth.C2
    pos = synth.scan_positions(cfg, sub=(4, 4))
    gd = synth.geometry(cfg, n_pos=len(pos))
    V_true = synth.potential_slices(cfg)
    I = f32(synth.poisson_counts(O.forward(gd, synth.probe(cfg), pos, V=V_true), cfg.dose, cfg.seed))
    probe = c64(synth.probe(cfg, defocus_A=cfg.defocus_guess_A))
    V0 = np.zeros_like(V_true)
    sweeps = 3
    n = sweeps * (cfg.n_slices + 1)
    o = oracle_path(gd, probe, pos, I, V0, sweeps, probe_steps=1, bars=mode == "fp32")
    amp, d = amplification(o, oracle_path(gd, probe, pos, I, V0, sweeps, probe_steps=1, bars=False, round32=False), n)
    prec = {"fp32": msp.MSP_PRECISION_FP32, "precise": msp.MSP_PRECISION_FP64_FORWARD,
            "df": msp.MSP_PRECISION_DF_FORWARD}[mode]
    g = msp.geometry(**gd, precision=prec)
    V = to_dev(V0, np.float32)
    p = to_dev(probe, np.complex64)
    h = msp.reconstruct(g, msp.plan(sweeps, probe_steps=1), p, V, to_dev(pos, np.int32),
                        to_dev(I, np.float32)).cpu().numpy()
    assert len(h) == len(o["hist"]) == n + 1
    if mode != "fp32":
        check_path(f"c2 4x4 probe estimation {mode}", h, o, V.cpu().numpy(), TOL, n, TOL, amp,
                   p=p.cpu().numpy(), bp=TOL)
    else:
        check_path("c2 4x4 probe estimation fp32", h, o, V.cpu().numpy(), o["b"], n, o["lbar"], amp,
                   p=p.cpu().numpy(), bp=o["bp"])
    assert h[-1] < h[0]


def test_reconstruct_equals_chained_steps(msp):
    """msp_reconstruct issues exactly the steps a caller would: bit-identical to chaining
    msp_layer_step and msp_probe_step on the same workspace."""
    cfg = synth.C1
    pos = synth.scan_positions(cfg, sub=(4, 4))
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd)
    V_true = synth.potential_slices(cfg)
    probe = synth.probe(cfg)
    I = to_dev(O.forward(gd, probe, pos, V=V_true), np.float32)
    dpos = to_dev(pos, np.int32)
    ws = msp.make_workspace(g)
    Va, pa = torch.zeros((cfg.n_slices, cfg.obj, cfg.obj), device=DEV), to_dev(probe * 1.05, np.complex64)
    Vb, pb = Va.clone(), pa.clone()
    h = msp.reconstruct(g, msp.plan(2, probe_steps=1), pa, Va, dpos, I, ws=ws)
    losses = []
    for _ in range(2):
        for layer in range(cfg.n_slices):
            losses.append(msp.layer_step(g, pb, Vb, dpos, I, layer, ws=ws)[0].clone())
        losses.append(msp.probe_step(g, pb, Vb, dpos, I, ws=ws)[0].clone())
    losses.append(msp.loss_grad(g, pb, Vb, dpos, I, want_dV=False, want_dprobe=False, ws=ws)[0])
    assert torch.equal(Va, Vb) and torch.equal(pa, pb)
    assert torch.equal(h, torch.cat(losses))
