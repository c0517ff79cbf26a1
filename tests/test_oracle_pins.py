"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, the paper's dense N^2 x N^2 matrix formulation
(Sec. 2.2 / 3.3) built explicitly on tiny grids, Parseval, finite differences
and brute-force spectral norms.  A dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import msp_oracle as O
from workloads import physics, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_geom(win=8, obj=12, L=3, n_pos=None):
    return dict(n_slices=L, obj_ny=obj, obj_nx=obj, win=win, n_pos=n_pos,
                wavelength_A=0.07, sigma=0.9, dz_A=20.0, pixel_A=0.5)


def rng(seed):
    return np.random.default_rng(seed)


def cplx(shape, seed):
    r = rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def vdot(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


# --------------------------------------------------------------------------- physics constants

def test_wavelength_and_sigma_match_paper_values():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    for row in g["wavelength_pm"]:
        lam_pm = physics.wavelength_A(row["kv"] * 1e3) * 100.0
        assert abs(lam_pm - row["value"]) <= row["abs_tol"], (row, lam_pm)
    ratio = physics.interaction_constant(80e3) / physics.interaction_constant(200e3)
    r = g["sigma_ratio_80_over_200"]
    assert abs(ratio - r["value"]) <= r["abs_tol"]


def test_interaction_constant_nonrelativistic_limit():
    # For eU << mc^2, sigma -> 2 pi m e lambda / h^2 = pi / (lambda U) (rad/(V m) -> per angstrom)
    U = 10.0
    lam = physics.wavelength_A(U)
    assert physics.interaction_constant(U) == pytest.approx(math.pi / (lam * U), rel=1e-4)


# --------------------------------------------------------------------------- Fourier operator

@pytest.mark.parametrize("shape", [(8, 8), (6, 10)])
def test_dft2_is_the_unnormalised_dft(shape):
    a = cplx(shape, 1)
    ny, nx = shape
    ky = np.arange(ny)[:, None, None, None]
    kx = np.arange(nx)[None, :, None, None]
    ny_ = np.arange(ny)[None, None, :, None]
    nx_ = np.arange(nx)[None, None, None, :]
    kern = np.exp(-2j * np.pi * (ky * ny_ / ny + kx * nx_ / nx))
    naive = np.einsum("abyx,yx->ab", kern, a)
    np.testing.assert_allclose(O.dft2(a), naive, atol=1e-11)
    # F^H is the conjugate transpose of that matrix
    b = cplx(shape, 2)
    assert abs(vdot(O.dft2(a), b) - vdot(a, O.dft2_adjoint(b))) < 1e-10


# --------------------------------------------------------------------------- propagator

def test_propagator_acts_on_plane_waves_by_the_fresnel_phase():
    """A plane wave exp(2 pi i (ky y + kx x) / W) is an eigenvector of G with eigenvalue
    exp(-i pi dz lambda q^2), q = k / (W * pixel) on the cyclic grid (Eq. fresnel_element)."""
    g = tiny_geom()
    w, px, lam, dz = g["win"], g["pixel_A"], g["wavelength_A"], g["dz_A"]
    h = O.fresnel_propagator(w, px, lam, dz)
    yy, xx = np.mgrid[0:w, 0:w]
    for ky, kx in [(0, 0), (1, 0), (0, 3), (5, 2), (4, 4), (7, 6)]:
        wave = np.exp(2j * np.pi * (ky * yy + kx * xx) / w)
        qy = (ky if ky < w // 2 else ky - w) / (w * px)
        qx = (kx if kx < w // 2 else kx - w) / (w * px)
        expect = np.exp(-1j * np.pi * dz * lam * (qy * qy + qx * qx)) * wave
        np.testing.assert_allclose(O.propagate(wave, h), expect, atol=1e-12)


def test_propagator_unitary_semigroup_identity():
    g = tiny_geom()
    w = g["win"]
    h1 = O.fresnel_propagator(w, g["pixel_A"], g["wavelength_A"], 7.0)
    h2 = O.fresnel_propagator(w, g["pixel_A"], g["wavelength_A"], 13.0)
    h12 = O.fresnel_propagator(w, g["pixel_A"], g["wavelength_A"], 20.0)
    h0 = O.fresnel_propagator(w, g["pixel_A"], g["wavelength_A"], 0.0)
    x = cplx((w, w), 3)
    y = cplx((w, w), 4)
    np.testing.assert_allclose(np.abs(h1), 1.0, atol=1e-15)
    assert np.linalg.norm(O.propagate(x, h1)) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    np.testing.assert_allclose(O.propagate(O.propagate(x, h1), h2), O.propagate(x, h12), atol=1e-12)
    np.testing.assert_allclose(O.propagate(x, h0), x, atol=1e-13)
    # adjoint identity <G x, y> = <x, G^H y>, and G^H G = I
    assert abs(vdot(O.propagate(x, h1), y) - vdot(x, O.propagate_adjoint(y, h1))) < 1e-12
    np.testing.assert_allclose(O.propagate_adjoint(O.propagate(x, h1), h1), x, atol=1e-12)


@pytest.mark.parametrize("wrap", [False, True])
def test_window_and_scatter_are_adjoint(wrap):
    a = cplx((3, 12, 12), 5)
    b = cplx((3, 8, 8), 6)
    y, x = (4, 3) if not wrap else (9, 7)
    lhs = vdot(O.window(a, y, x, 8, wrap), b)
    acc = np.zeros_like(a)
    O.window_add(acc, y, x, b, wrap)
    assert abs(lhs - vdot(a, acc)) < 1e-12


# --------------------------------------------------------------------------- forward model

def probe_and_positions(g, seed=0, n=5):
    r = rng(seed)
    w, obj = g["win"], g["obj_ny"]
    probe = cplx((w, w), seed + 100) * 0.3
    pos = np.stack([r.integers(0, obj - w + 1, n), r.integers(0, obj - w + 1, n)], 1).astype(np.int32)
    return probe, pos


def test_zero_potential_gives_the_probe_diffraction_pattern():
    g = tiny_geom()
    probe, pos = probe_and_positions(g)
    V = np.zeros((g["n_slices"], 12, 12))
    I = O.forward(g, probe, pos, V=V)
    expect = np.abs(np.fft.fft2(probe)) ** 2
    for s in range(len(pos)):
        np.testing.assert_allclose(I[s], expect, rtol=1e-12, atol=1e-12)


def test_parseval_for_pure_phase_slices():
    g = tiny_geom()
    probe, pos = probe_and_positions(g, 1)
    V = rng(7).standard_normal((g["n_slices"], 12, 12))
    I = O.forward(g, probe, pos, V=V)
    for s in range(len(pos)):
        assert I[s].sum() == pytest.approx(g["win"] ** 2 * np.sum(np.abs(probe) ** 2), rel=1e-12)


def test_constant_potential_is_a_global_phase():
    g = tiny_geom()
    probe, pos = probe_and_positions(g, 2)
    V = rng(8).standard_normal((g["n_slices"], 12, 12))
    I0 = O.forward(g, probe, pos, V=V)
    I1 = O.forward(g, probe, pos, V=V + np.array([0.3, -1.1, 2.0])[:, None, None])
    np.testing.assert_allclose(I1, I0, rtol=1e-11, atol=1e-11)


def test_phase_ramp_shifts_the_pattern():
    """A slice-1 phase ramp exp(2 pi i k0.r / W), other slices empty: I(k) = |F p|^2 (k - k0)."""
    g = tiny_geom(L=2)
    w = g["win"]
    probe, pos = probe_and_positions(g, 3)
    k0 = (2, 5)
    yy, xx = np.mgrid[0:12, 0:12]
    V = np.zeros((2, 12, 12))
    V[0] = 2 * np.pi * (k0[0] * yy + k0[1] * xx) / (w * g["sigma"])
    I = O.forward(g, probe, pos, V=V)
    base = np.abs(np.fft.fft2(probe)) ** 2
    expect = np.roll(base, k0, axis=(0, 1))
    for s in range(len(pos)):
        np.testing.assert_allclose(I[s], expect, rtol=1e-10, atol=1e-10)


def test_windowed_equals_circulant_when_window_is_the_object():
    """The paper shifts the probe cyclically over an N x N object; the window model with a
    wrapped window of side N gives the same intensities (the shift only moves the wave)."""
    n = 8
    g = tiny_geom(win=n, obj=n)
    probe = cplx((n, n), 9)
    T = cplx((3, n, n), 10)
    shifts = np.array([[0, 0], [3, 5], [7, 1], [2, 6]], dtype=np.int32)
    Iw = O.forward(g, probe, shifts, T=T, wrap=True)
    Ic = O.forward_circulant(g, probe, shifts, T=T)
    np.testing.assert_allclose(Iw, Ic, rtol=1e-11, atol=1e-11)


def dense_operators(g, n, T):
    """The paper's matrices (Sec. 2.2) on an n x n grid, row-major vec."""
    f1 = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    F = np.kron(f1, f1)
    Finv = np.conj(F).T / n ** 2
    h = O.fresnel_propagator(n, g["pixel_A"], g["wavelength_A"], g["dz_A"])
    G = Finv @ np.diag(h.ravel()) @ F
    Om = [np.diag(T[m].ravel()) for m in range(T.shape[0])]
    return F, G, Om


def shifted_probe_matrix(probe, shifts):
    return np.stack([np.roll(probe, (int(a), int(b)), axis=(0, 1)).ravel() for a, b in shifts], axis=1)


def test_forward_matches_the_dense_matrix_formulation():
    """I = |F_2D A_M P|^2 with A_M = O_M prod G_m O_m (Eq. exit_wave_mslices, Eq. measurement FAP)."""
    n, M = 8, 3
    g = tiny_geom(win=n, obj=n, L=M)
    probe = cplx((n, n), 11)
    T = cplx((M, n, n), 12)
    shifts = np.array([[0, 0], [1, 2], [5, 3], [6, 7], [4, 4]])
    F, G, Om = dense_operators(g, n, T)
    A = Om[0]
    for m in range(1, M):
        A = Om[m] @ G @ A
    P = shifted_probe_matrix(probe, shifts)
    I_dense = np.abs(F @ A @ P) ** 2                      # [n^2][S]
    I_or = O.forward_circulant(g, probe, shifts, T=T)      # [S][n][n]
    np.testing.assert_allclose(I_or.reshape(len(shifts), -1).T, I_dense, rtol=1e-10, atol=1e-10)


def layer_matrix(g, n, T, probe, shifts, layer):
    """Q_l of Eq. (Single_Layer_Matrix): stacked F R_l diag(S_l p^s), with
    R_l = prod_{m>l} O_m G and S_l = prod_{m<l} G O_m (Eq. Layerwise_Prefix_Suffix)."""
    M = T.shape[0]
    F, G, Om = dense_operators(g, n, T)
    R = np.eye(n * n, dtype=complex)
    for m in range(layer + 1, M):
        R = Om[m] @ G @ R
    Sl = np.eye(n * n, dtype=complex)
    for m in range(0, layer):
        Sl = G @ Om[m] @ Sl
    P = shifted_probe_matrix(probe, shifts)
    return np.vstack([F @ R @ np.diag(Sl @ P[:, s]) for s in range(P.shape[1])])


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_layer_gradient_and_step_size_match_the_dense_phase_retrieval(layer):
    """The matrix-free layer gradient equals Q_l^H (Q_l o_l - Q_l o_l / |Q_l o_l| o sqrt(y)) (Sec. 3.2),
    and ||Q_l||^2 = N^2 max sum_s |S_l p^s|^2 when the later slices are unimodular."""
    n, M = 8, 3
    g = tiny_geom(win=n, obj=n, L=M)
    probe = cplx((n, n), 13)
    T = cplx((M, n, n), 14)
    for m in range(layer + 1, M):       # later slices unimodular -> R_l unitary up to F
        T[m] = T[m] / np.abs(T[m])
    shifts = np.array([[0, 0], [2, 3], [5, 1], [7, 6]], dtype=np.int32)
    y_meas = np.abs(cplx((len(shifts), n, n), 15)) ** 2
    Q = layer_matrix(g, n, T, probe, shifts, layer)
    z = T[layer].ravel()
    u = Q @ z
    ph = np.where(np.abs(u) > 0, u / np.where(np.abs(u) > 0, np.abs(u), 1), 0)
    yv = y_meas.reshape(len(shifts), -1).ravel()
    grad_dense = np.conj(Q).T @ (u - ph * np.sqrt(yv))
    loss_dense = np.sum((np.sqrt(yv) - np.abs(u)) ** 2)
    loss, dXl, illum, _ = O.layer_quantities(g, probe, shifts, y_meas, layer, T=T, wrap=True)
    assert loss == pytest.approx(loss_dense, rel=1e-11)
    np.testing.assert_allclose(dXl.ravel(), grad_dense, rtol=1e-9, atol=1e-9)
    norm2 = np.linalg.norm(Q, 2) ** 2
    assert n * n * illum.max() == pytest.approx(norm2, rel=1e-9)


def test_probe_step_size_is_the_spectral_norm():
    """For unimodular slices ||Q_p||^2 = S N^2 (the probe-problem matrix stacks F A_s, Sec. 3.5)."""
    n, M = 8, 3
    g = tiny_geom(win=n, obj=n, L=M)
    T = np.exp(1j * rng(16).standard_normal((M, n, n)))
    shifts = np.array([[0, 0], [2, 3], [5, 1], [7, 6], [3, 3]])
    F, G, Om = dense_operators(g, n, T)
    A = Om[0]
    for m in range(1, M):
        A = Om[m] @ G @ A
    # windowed form: position s sees the object rolled by -s; the probe enters unshifted
    blocks = []
    for a, b in shifts:
        Ts = np.roll(T, (-a, -b), axis=(1, 2))
        _, _, Oms = dense_operators(g, n, Ts)
        As = Oms[0]
        for m in range(1, M):
            As = Oms[m] @ G @ As
        blocks.append(F @ As)
    Qp = np.vstack(blocks)
    assert np.linalg.norm(Qp, 2) ** 2 == pytest.approx(len(shifts) * n * n, rel=1e-10)


# --------------------------------------------------------------------------- adjoint / gradients

def test_backward_is_the_adjoint_of_the_linearised_forward():
    """Psi^s is linear in each slice, so J(d) = Psi^s(slice l := d); the backward recursion
    applied to an arbitrary far-field vector r must give J^H r: <J d, r> = <d, J^H r>."""
    g = tiny_geom()
    probe, pos = probe_and_positions(g, 4, n=4)
    w = g["win"]
    h = O.fresnel_propagator(w, g["pixel_A"], g["wavelength_A"], g["dz_A"])
    T = cplx((3, 12, 12), 17)
    for layer in range(3):
        d = cplx((12, 12), 18 + layer)
        lhs = 0.0
        rhs = 0.0
        for s, (y, x) in enumerate(pos):
            r = cplx((w, w), 40 + s)
            Td = T.copy()
            Td[layer] = d
            _, _, jd = O.position_forward(probe, Td, int(y), int(x), h)
            lhs += vdot(jd, r)
            inc, _, _ = O.position_forward(probe, T, int(y), int(x), h)
            grads, _ = O.position_backward(T, int(y), int(x), h, inc, O.dft2_adjoint(r), layer)
            back = np.zeros((12, 12), dtype=complex)
            O.window_add(back, int(y), int(x), grads[layer])
            rhs += vdot(d, back)
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def make_problem(seed=0, L=3, win=8, obj=14, n=6):
    g = tiny_geom(win=win, obj=obj, L=L)
    r = rng(seed)
    probe = cplx((win, win), seed + 200) * 0.4
    pos = np.stack([r.integers(0, obj - win + 1, n), r.integers(0, obj - win + 1, n)], 1).astype(np.int32)
    V_true = r.standard_normal((L, obj, obj))
    I = O.forward(g, probe, pos, V=V_true)
    V = V_true + 0.3 * r.standard_normal((L, obj, obj))
    return g, probe, pos, I, V


def test_potential_gradient_matches_finite_differences():
    g, probe, pos, I, V = make_problem(1)
    res = O.loss_grad(g, probe, pos, I, V=V)
    r = rng(50)
    for trial in range(3):
        d = r.standard_normal(V.shape)
        hstep = 1e-5
        lp = O.loss_grad(g, probe, pos, I, V=V + hstep * d)["loss"]
        lm = O.loss_grad(g, probe, pos, I, V=V - hstep * d)["loss"]
        fd = (lp - lm) / (2 * hstep)
        an = float(np.sum(res["dV"] * d))
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-9)
    # single pixels, inside and on the edge of the scanned area
    for (l, yy, xx) in [(0, 5, 5), (2, 0, 0), (1, 13, 7)]:
        e = np.zeros_like(V)
        e[l, yy, xx] = 1.0
        lp = O.loss_grad(g, probe, pos, I, V=V + 1e-5 * e)["loss"]
        lm = O.loss_grad(g, probe, pos, I, V=V - 1e-5 * e)["loss"]
        assert (lp - lm) / 2e-5 == pytest.approx(res["dV"][l, yy, xx], rel=1e-5, abs=1e-8)


def test_wirtinger_gradients_match_finite_differences():
    """dL = 2 Re <grad, delta> for the conjugate (Wirtinger) gradients of the probe and of
    complex transmission slices (Sec. 3.2)."""
    g, probe, pos, I, V = make_problem(2)
    T = np.exp(1j * g["sigma"] * V) * (1 + 0.1 * rng(3).standard_normal(V.shape))
    res = O.loss_grad(g, probe, pos, I, T=T)
    hstep = 1e-6
    for seed in range(2):
        dT = cplx(T.shape, 60 + seed)
        lp = O.loss_grad(g, probe, pos, I, T=T + hstep * dT)["loss"]
        lm = O.loss_grad(g, probe, pos, I, T=T - hstep * dT)["loss"]
        assert (lp - lm) / (2 * hstep) == pytest.approx(2 * np.real(vdot(res["dX"], dT)), rel=1e-6)
        dp = cplx(probe.shape, 70 + seed)
        lp = O.loss_grad(g, probe + hstep * dp, pos, I, T=T)["loss"]
        lm = O.loss_grad(g, probe - hstep * dp, pos, I, T=T)["loss"]
        assert (lp - lm) / (2 * hstep) == pytest.approx(2 * np.real(vdot(res["dprobe"], dp)), rel=1e-6)


def test_zero_rule_and_zero_probe():
    """With Psi == 0 everywhere the fraction Qz/|Qz| is 0 (Sec. 3.2): the residual vanishes,
    the loss is sum(I) and every gradient is exactly zero."""
    g, probe, pos, I, V = make_problem(3)
    res = O.loss_grad(g, np.zeros_like(probe), pos, I, V=V)
    assert res["loss"] == pytest.approx(float(I.sum()), rel=1e-14)
    assert np.all(res["dV"] == 0) and np.all(res["dprobe"] == 0)
    assert np.all(np.isfinite(res["dV"]))


def test_layer_step_descends_with_the_spectral_step_in_transmission_mode():
    """mu = ||Q_l||^-2 guarantees a non-increasing loss (Sec. 3.2, the convergence guarantee)."""
    g, probe, pos, I, V = make_problem(4)
    T = np.exp(1j * g["sigma"] * V)
    for layer in [0, 1, 2]:
        losses = []
        Tc = T.copy()
        for _ in range(4):
            Tc, loss, mu = O.layer_step(g, probe, pos, I, layer, T=Tc)
            losses.append(loss)
        assert all(b <= a * (1 + 1e-12) for a, b in zip(losses, losses[1:])), losses
        assert losses[-1] < losses[0]


def test_probe_step_descends_and_normalises():
    g, probe, pos, I, V = make_problem(5)
    p = probe * np.exp(0.3j) * 1.2 + 0.05 * cplx(probe.shape, 80)
    losses = []
    for _ in range(4):
        p, loss, mu = O.probe_step(g, p, pos, I, V=V)
        losses.append(loss)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(losses, losses[1:]))
    assert mu == pytest.approx(1.0 / (len(pos) * g["win"] ** 2))
    pn, _, _ = O.probe_step(g, p, pos, I, V=V, normalize=True)
    target = I.reshape(len(pos), -1).sum(1).mean()
    assert g["win"] ** 2 * np.sum(np.abs(pn) ** 2) == pytest.approx(target, rel=1e-12)


def test_layerwise_estimation_lowers_the_loss_on_a_small_workload():
    """Algorithm 1 from V = 0 with the known probe on noiseless data (a reduced c1 shape)."""
    cfg = synth.C1
    g = synth.geometry(cfg)
    pos = synth.scan_positions(cfg, sub=(3, 3))
    V_true = synth.potential_slices(cfg)
    p = synth.probe(cfg)
    I = O.forward(g, p, pos, V=V_true)
    V, hist = O.layerwise_estimation(g, p, pos, I, np.zeros_like(V_true), sweeps=3)
    final = O.loss_grad(g, p, pos, I, V=V, want_probe=False)["loss"]
    assert final < 0.5 * hist[0]
    err0 = O.relative_measurement_error(hist[0], I)
    err1 = O.relative_measurement_error(final, I)
    assert err1 < err0


def test_layerwise_estimation_is_gauss_seidel_over_ascending_slices():
    """Algorithm 1 (Sec. 3.3): within a sweep the slices are taken in ascending order and the
    prefix S_l of slice l is formed from the slices already updated in this sweep.  Two sweeps
    must equal six explicitly chained single-slice steps; a Jacobi sweep (every slice stepped
    from the sweep's starting slices) and a descending sweep give different potentials, so
    either mistake fails here."""
    g, probe, pos, I, V0 = make_problem(21, L=3)
    V_alg, hist = O.layerwise_estimation(g, probe, pos, I, V0, sweeps=2)
    Vc, losses = np.array(V0, copy=True), []
    for _ in range(2):
        for layer in range(3):
            Vc, loss, _ = O.layer_step(g, probe, pos, I, layer, V=Vc)
            losses.append(loss)
    assert np.array_equal(V_alg, Vc)
    assert hist == losses
    # Jacobi order
    Vj = np.array(V0, copy=True)
    for _ in range(2):
        nxt = Vj.copy()
        for layer in range(3):
            nxt[layer] = O.layer_step(g, probe, pos, I, layer, V=Vj)[0][layer]
        Vj = nxt
    # descending order
    Vd = np.array(V0, copy=True)
    for _ in range(2):
        for layer in (2, 1, 0):
            Vd, _, _ = O.layer_step(g, probe, pos, I, layer, V=Vd)
    for other in (Vj, Vd):
        assert np.linalg.norm(other - V_alg) > 1e-3 * np.linalg.norm(V_alg - V0)


def test_plain_method_orders_slice_sweeps_and_probe_steps():
    """The plain method runs, per sweep, Algorithm 1's ascending Gauss-Seidel slice steps and then the
    probe steps of Sec. 3.5 with the slices just estimated; its history is the loss before each step
    and the loss after the last.  Without probe steps it is Algorithm 1 itself.  Swapping the probe
    steps before the slice steps, or leaving the history's final loss out, fails here."""
    g, probe, pos, I, V0 = make_problem(23, L=2)
    p0 = probe * np.exp(0.2j) * 1.1
    V, p, hist = O.plain_method(g, p0, pos, I, V0, sweeps=2, probe_steps=1)
    Vc, pc, ref = np.array(V0, copy=True), p0.copy(), []
    for _ in range(2):
        for layer in range(2):
            Vc, loss, _ = O.layer_step(g, pc, pos, I, layer, V=Vc)
            ref.append(loss)
        pc, loss, _ = O.probe_step(g, pc, pos, I, V=Vc)
        ref.append(loss)
    ref.append(O.loss_grad(g, pc, pos, I, V=Vc, want_probe=False)["loss"])
    assert np.array_equal(V, Vc) and np.array_equal(p, pc)
    assert hist == ref
    # probe steps first in each sweep give a different trajectory
    Vs, ps = np.array(V0, copy=True), p0.copy()
    for _ in range(2):
        ps, _, _ = O.probe_step(g, ps, pos, I, V=Vs)
        for layer in range(2):
            Vs, _, _ = O.layer_step(g, ps, pos, I, layer, V=Vs)
    assert np.linalg.norm(ps - p) > 1e-6 * np.linalg.norm(p)
    # no probe steps: Algorithm 1
    V1, p1, h1 = O.plain_method(g, p0, pos, I, V0, sweeps=2)
    Va, ha = O.layerwise_estimation(g, p0, pos, I, V0, sweeps=2)
    assert np.array_equal(V1, Va) and np.array_equal(p1, p0) and h1[:-1] == ha
    assert h1[-1] == O.loss_grad(g, p0, pos, I, V=Va, want_probe=False)["loss"] < ha[0]


def test_relative_reconstruction_error_closed_form():
    """Eq. (error_metric_object): the mean over slices of ||O_m - O^_m||_F / ||O_m||_F.  An estimate
    that scales slice m by a_m has error |a_m - 1| on that slice; with a = (1.1, 0.7, 1 + 0.2i) the
    metric is exactly (0.1 + 0.3 + 0.2) / 3 = 0.2.  Normalising by the estimate, summing instead of
    averaging, or averaging squares instead of norms gives 0.239, 0.6 or 0.216."""
    X = cplx((3, 9, 7), 33)
    a = np.array([1.1, 0.7, 1 + 0.2j])
    est = a[:, None, None] * X
    assert O.relative_reconstruction_error(X, est) == pytest.approx(0.2, rel=1e-12)
    assert O.relative_reconstruction_error(X, X) == 0.0
    # the error of each slice is relative to that slice: rescaling one true slice and its
    # estimate together leaves the metric unchanged
    X2, est2 = X.copy(), est.copy()
    X2[1] *= 1e3
    est2[1] *= 1e3
    assert O.relative_reconstruction_error(X2, est2) == pytest.approx(0.2, rel=1e-12)


@pytest.mark.parametrize("layer", [0, 2])
def test_potential_step_is_the_tangent_projection_of_the_transmission_step(layer):
    """Potential mode moves V so that exp(i sigma V) follows the transmission-mode amplitude-flow
    step projected onto the unit circle: dV = Im(dT conj(T)) / sigma, which fixes mu_V = mu / (2 sigma^2)."""
    g, probe, pos, I, V = make_problem(6)
    T = np.exp(1j * g["sigma"] * V)
    Vn, _, _ = O.layer_step(g, probe, pos, I, layer, V=V)
    Tn, _, _ = O.layer_step(g, probe, pos, I, layer, T=T)
    tangent = np.imag((Tn[layer] - T[layer]) * np.conj(T[layer])) / g["sigma"]
    np.testing.assert_allclose(Vn[layer] - V[layer], tangent, rtol=1e-9, atol=1e-14)
    others = [m for m in range(V.shape[0]) if m != layer]
    assert np.array_equal(Vn[others], V[others])


def test_zero_rule_gives_the_exact_arithmetic_residual_at_identity_initialisation():
    """With identity slices (V = 0, the paper's initialisation) and an aperture-limited probe,
    Psi = h^(L-1) F(p) vanishes outside the aperture in exact arithmetic, and so does the
    exact residual.  The rule's residual there is Psi itself (round-off, ~1e-15) and
    Psi (1 - sqrt(I)/|Psi|) inside; the literal '== 0' test applied to round-off values gives
    residuals of size sqrt(I) outside, with phases set by round-off."""
    cfg = synth.C1
    gd = synth.geometry(cfg, n_pos=1)
    p = synth.probe(cfg)
    X = np.ones((cfg.n_slices, cfg.obj, cfg.obj), dtype=complex)
    h = O.fresnel_propagator(cfg.win, gd["pixel_A"], gd["wavelength_A"], gd["dz_A"])
    _, _, far = O.position_forward(p, X, 10, 12, h)
    q = np.fft.fftfreq(cfg.win, d=cfg.pixel_A)
    inside = (q[:, None] ** 2 + q[None, :] ** 2) <= (cfg.aperture_mrad * 1e-3 / gd["wavelength_A"]) ** 2
    I = np.abs(far) ** 2 * 1.1 + 0.5          # dark-field counts everywhere
    _, r = O.far_field_residual(far, I, O.zero_threshold(p))
    assert np.abs(r[~inside]).max() <= 1e-12
    np.testing.assert_allclose(r[inside], far[inside] * (1 - np.sqrt(I[inside]) / np.abs(far[inside])), rtol=1e-12)
    _, r_literal = O.far_field_residual(far, I, 0.0)
    assert np.abs(r_literal[~inside]).max() > 0.5
    # the threshold sits far below every in-aperture amplitude
    assert O.zero_threshold(p) < 1e-3 * np.abs(far[inside]).min()


def test_residual_conditioning_closed_forms():
    """With I = 0 the residual is Psi itself and every m_k = 1, so kappa = ||p|| sqrt(S W^2) / ||Psi||
    = 1 for pure-phase slices (Parseval); scaling all intensities does not change the
    cancellation of a single position (1 exactly)."""
    g, probe, pos, I, V = make_problem(7)
    kappa, canc, flip = O.residual_conditioning(g, probe, pos, np.zeros_like(I), V=V)
    assert kappa == pytest.approx(1.0, rel=1e-12)
    assert flip == 0.0
    _, canc1, _ = O.residual_conditioning(g, probe, pos[:1], I[:1], V=V)
    assert canc1 == pytest.approx(1.0, rel=1e-12)
