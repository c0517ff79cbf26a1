"""GPU parity of the plain method (msp_reconstruct): Algorithm 1 (Sec. 3.3) with optional probe
steps (Sec. 3.5), run by the library on the device, against the oracle's plain_method on the same
seeded inputs.

Tolerances.  Every step of the FP32 path carries the gradient error bounded in test_gpu_parity
(relative, per state) plus the FP32 rounding of the stored slices, and a trajectory adds them
up: after N steps the potentials may differ from the oracle's by at most
    b * sum_k ||V_{k+1} - V_k|| + N 2^-24 max_k ||V_k||
with b the largest per-state gradient bar met on the oracle's path (sampled at its start,
middle and end).  The loss history is compared entry by entry at b N (each entry's state
carries the accumulated deviation)."""
import numpy as np
import pytest
import torch

import __graft_entry__
from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
U32 = 2.0 ** -24


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
    """The per-state FP32 gradient bar of test_gpu_parity (uncapped here: it is a bound, and the
    trajectory bar below takes the largest one met)."""
    e = 2 * (2 * gd["n_slices"] - 1) * U32
    kappa, _, flip = O.residual_conditioning(gd, probe, pos, I, V=V, band=2 * e * float(np.linalg.norm(probe)))
    return max(1e-5, e * kappa + flip)


def oracle_path(gd, probe, pos, I, V0, sweeps, probe_steps=0):
    """The oracle's plain method step by step, keeping what the trajectory bar needs."""
    V, p = np.array(V0, dtype=np.float64), np.asarray(probe, dtype=np.complex128).copy()
    hist, path, vmax, states = [], 0.0, float(np.linalg.norm(V)), []
    L = gd["n_slices"]
    for t in range(sweeps):
        for layer in range(L):
            if t in (0, sweeps // 2, sweeps - 1) and layer == 0:
                states.append((V.copy(), p.copy()))
            Vn, loss, _ = O.layer_step(gd, p, pos, I, layer, V=V)
            path += float(np.linalg.norm(Vn - V))
            V = Vn
            vmax = max(vmax, float(np.linalg.norm(V)))
            hist.append(loss)
        for _ in range(probe_steps):
            p, loss, _ = O.probe_step(gd, p, pos, I, V=V)
            hist.append(loss)
    hist.append(O.loss_grad(gd, p, pos, I, V=V, want_probe=False)["loss"])
    return V, p, hist, path, vmax, states


def test_c1_fifty_sweeps_from_zero_with_known_probe(msp):
    """The oracle-size workload as specified: 2 slices, 8 x 8 scan, noiseless, known probe,
    50 layer-wise iterations from V = 0; trajectory and final loss against the oracle."""
    cfg = synth.C1
    pos = synth.scan_positions(cfg)
    gd = synth.geometry(cfg, n_pos=len(pos))
    V_true = synth.potential_slices(cfg)
    probe = synth.probe(cfg).astype(np.complex64).astype(np.complex128)
    I = f32(O.forward(gd, probe, pos, V=V_true))
    V0 = np.zeros_like(V_true)
    sweeps = 50
    Vr, _, hist, path, vmax, states = oracle_path(gd, probe, pos, I, V0, sweeps)
    assert hist[-1] < 0.05 * hist[0]          # the method converges on noiseless data
    g = msp.geometry(**gd)
    V = to_dev(V0, np.float32)
    h = msp.reconstruct(g, msp.plan(sweeps), to_dev(probe, np.complex64), V, to_dev(pos, np.int32),
                        to_dev(I, np.float32)).cpu().numpy()
    assert len(h) == len(hist) == sweeps * cfg.n_slices + 1
    b = max(grad_bar(gd, probe, pos, I, Vs) for Vs, _ in states)
    n = sweeps * cfg.n_slices
    v_bar = (b * path + n * U32 * vmax) / float(np.linalg.norm(Vr))
    v_err = rel(V.cpu().numpy(), Vr)
    h_err = float(np.max(np.abs(h - np.asarray(hist)) / np.asarray(hist)))
    print(f"c1 50 sweeps: V error {v_err:.3e} (bar {v_bar:.3e}), loss-history error {h_err:.3e} "
          f"(bar {b * n:.3e}), final loss {h[-1]:.6e} vs {hist[-1]:.6e}, per-step bar {b:.2e}")
    assert v_err <= v_bar
    assert h_err <= b * n


def test_c2_sub_scan_with_probe_estimation(msp):
    """The W = 128, L = 4 workload's plain method with probe estimation on a 4 x 4 sub-scan:
    from V = 0 and the probe guess with a 20 angstrom defocus error, three sweeps of the four
    slice steps followed by one probe step each."""
    cfg = synth.C2
    pos = synth.scan_positions(cfg, sub=(4, 4))
    gd = synth.geometry(cfg, n_pos=len(pos))
    V_true = synth.potential_slices(cfg)
    I = f32(synth.poisson_counts(O.forward(gd, synth.probe(cfg), pos, V=V_true), cfg.dose, cfg.seed))
    probe = synth.probe(cfg, defocus_A=cfg.defocus_guess_A).astype(np.complex64).astype(np.complex128)
    V0 = np.zeros_like(V_true)
    sweeps = 3
    Vr, pr, hist, path, vmax, states = oracle_path(gd, probe, pos, I, V0, sweeps, probe_steps=1)
    g = msp.geometry(**gd)
    V = to_dev(V0, np.float32)
    p = to_dev(probe, np.complex64)
    h = msp.reconstruct(g, msp.plan(sweeps, probe_steps=1), p, V, to_dev(pos, np.int32),
                        to_dev(I, np.float32)).cpu().numpy()
    assert len(h) == len(hist) == sweeps * (cfg.n_slices + 1) + 1
    b = max(grad_bar(gd, ps, pos, I, Vs) for Vs, ps in states)
    n = sweeps * (cfg.n_slices + 1)
    v_bar = (b * path + n * U32 * vmax) / float(np.linalg.norm(Vr))
    v_err = rel(V.cpu().numpy(), Vr)
    p_err = rel(p.cpu().numpy(), pr)
    h_err = float(np.max(np.abs(h - np.asarray(hist)) / np.asarray(hist)))
    print(f"c2 4x4 probe estimation: V error {v_err:.3e} (bar {v_bar:.3e}), probe error {p_err:.3e}, "
          f"loss-history error {h_err:.3e} (bar {b * n:.3e}), per-step bar {b:.2e}")
    assert v_err <= v_bar
    assert p_err <= b * n
    assert h_err <= b * n
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
