"""Pins for the oracle's Algorithm 2 (Sparse Matrix Decomposition, Sec. 3.4).

Each test checks the oracle against something other than itself: numpy's FFT,
the FFT-based circulant forward model, singular values computed by LAPACK,
finite differences, closed forms of special cases (one slice, an exact
factorisation) and the descent property that the paper's step sizes guarantee.
"""
import numpy as np
import pytest

from oracle import msp_oracle as O


def geom(M=3, dz=20.0):
    return dict(n_slices=M, obj_ny=0, obj_nx=0, win=0, n_pos=0,
                wavelength_A=0.07, sigma=0.9, dz_A=dz, pixel_A=0.5)


def cplx(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def full_raster(n):
    return np.array([(y, x) for y in range(n) for x in range(n)])


def phase_slices(M, n, seed, amp=0.6):
    r = np.random.default_rng(seed)
    return [np.exp(1j * amp * r.standard_normal(n * n)) for _ in range(M)]


def test_dft_matrix_is_numpy_fft2():
    n = 6
    x = cplx((n, n), 1)
    np.testing.assert_allclose(O.dft_matrix_2d(n) @ x.ravel(), np.fft.fft2(x).ravel(), atol=1e-11)


def test_propagator_matrix_is_fft_convolution_and_unitary():
    n = 6
    g = geom()
    G = O.propagator_matrix(g, n)
    x = cplx((n, n), 2)
    h = O.fresnel_propagator(n, g["pixel_A"], g["wavelength_A"], g["dz_A"])
    np.testing.assert_allclose(G @ x.ravel(), np.fft.ifft2(h * np.fft.fft2(x)).ravel(), atol=1e-12)
    np.testing.assert_allclose(np.conj(G).T @ G, np.eye(n * n), atol=1e-12)
    np.testing.assert_allclose(O.propagator_matrix(geom(dz=0.0), n), np.eye(n * n), atol=1e-12)


def test_transfer_matrix_times_probes_is_the_fft_multislice():
    """|F A_M P|^2 equals the FFT-based circulant forward model column by column."""
    n, M = 8, 3
    g = geom(M)
    o = [cplx(n * n, 10 + m) for m in range(M)]
    probe = cplx((n, n), 3)
    shifts = np.array([[0, 0], [2, 5], [7, 1], [3, 3]])
    A = O.transfer_matrix(O.propagator_matrix(g, n), o)
    I = np.abs(O.dft_matrix_2d(n) @ A @ O.probe_matrix(probe, shifts)) ** 2
    T = np.stack([x.reshape(n, n) for x in o])
    Ic = O.forward_circulant(dict(g, obj_ny=n, obj_nx=n, win=n), probe, shifts, T=T)
    np.testing.assert_allclose(O.measurement_matrix(Ic), I, rtol=1e-10, atol=1e-10)


def test_shift_operator_norm_is_the_spectral_norm_on_the_full_raster_and_bounds_subsets():
    n = 6
    probe = cplx((n, n), 4)
    P = O.probe_matrix(probe, full_raster(n))
    assert O.shift_operator_norm(probe) == pytest.approx(np.linalg.norm(P, 2), rel=1e-12)
    sub = O.probe_matrix(probe, full_raster(n)[::5])
    assert np.linalg.norm(sub, 2) <= O.shift_operator_norm(probe) * (1 + 1e-12)
    F = O.dft_matrix_2d(n)
    assert np.linalg.norm(F, 2) ** 2 == pytest.approx(n * n, rel=1e-12)
    assert O.matrix_step_size(probe) == pytest.approx(1.0 / (np.linalg.norm(F, 2) ** 2 * np.linalg.norm(P, 2) ** 2), rel=1e-12)


def test_matrix_objective_is_half_the_windowed_loss():
    """1/2 sum (sqrt(I) - |FAP|)^2 equals half the per-position loss of the FFT-based path
    when A is a transfer matrix and the window wraps (Sec. 3.2 vs Sec. 3.4)."""
    n, M = 8, 2
    g = geom(M)
    o = [cplx(n * n, 20 + m) for m in range(M)]
    probe = cplx((n, n), 5)
    shifts = np.array([[0, 0], [1, 6], [4, 2]])
    I = np.abs(cplx((len(shifts), n, n), 6)) ** 2
    A = O.transfer_matrix(O.propagator_matrix(g, n), o)
    obj, _ = O.matrix_objective_residual(A, O.dft_matrix_2d(n), O.probe_matrix(probe, shifts), O.measurement_matrix(I))
    T = np.stack([x.reshape(n, n) for x in o])
    out = O.loss_grad(dict(g, obj_ny=n, obj_nx=n, win=n), probe, shifts, I, T=T, wrap=True, want_probe=False)
    assert obj == pytest.approx(0.5 * out["loss"], rel=1e-12)


def test_matrix_gradient_matches_finite_differences():
    """The step direction F^H R P^H is the real gradient of the objective of Eq. (Opt_Prob_Matrix)."""
    n, S = 4, 5
    r = np.random.default_rng(7)
    A = cplx((n * n, n * n), 8)
    P = O.probe_matrix(cplx((n, n), 9), r.integers(0, n, (S, 2)))
    I = np.abs(cplx((n * n, S), 10)) ** 2
    F = O.dft_matrix_2d(n)
    _, R = O.matrix_objective_residual(A, F, P, I)
    grad = np.conj(F).T @ R @ np.conj(P).T
    for seed in range(3):
        d = cplx(A.shape, 100 + seed)
        eps = 1e-6
        fp, _ = O.matrix_objective_residual(A + eps * d, F, P, I)
        fm, _ = O.matrix_objective_residual(A - eps * d, F, P, I)
        assert (fp - fm) / (2 * eps) == pytest.approx(np.real(np.vdot(grad, d)), rel=1e-6)


@pytest.mark.parametrize("raster", ["full", "subset"])
def test_matrix_steps_never_increase_the_objective(raster):
    """mu = 1/(N^2 ||P||^2) is the inverse Lipschitz constant of the majoriser, so the
    amplitude-flow objective is non-increasing (Sec. 3.2, 3.4)."""
    n, M = 6, 2
    g = geom(M)
    G = O.propagator_matrix(g, n)
    probe = cplx((n, n), 11)
    shifts = full_raster(n) if raster == "full" else full_raster(n)[::3]
    P = O.probe_matrix(probe, shifts)
    F = O.dft_matrix_2d(n)
    A_true = O.transfer_matrix(G, phase_slices(M, n, 12))
    I = np.abs(F @ A_true @ P) ** 2
    A = O.transfer_matrix(G, phase_slices(M, n, 13, amp=0.3))
    mu = O.matrix_step_size(probe)
    prev = np.inf
    for _ in range(12):
        A, obj = O.matrix_step(A, F, P, I, mu)
        assert obj <= prev * (1 + 1e-12)
        prev = obj
    _, last = O.matrix_step(A, F, P, I, mu)
    assert last < 0.5 * O.matrix_step(O.transfer_matrix(G, phase_slices(M, n, 13, amp=0.3)), F, P, I, mu)[1]


def test_matrix_step_keeps_an_exact_solution():
    n = 6
    G = O.propagator_matrix(geom(2), n)
    A = O.transfer_matrix(G, phase_slices(2, n, 14))
    probe = cplx((n, n), 15)
    P = O.probe_matrix(probe, full_raster(n)[::2])
    F = O.dft_matrix_2d(n)
    I = np.abs(F @ A @ P) ** 2
    A1, obj = O.matrix_step(A, F, P, I, O.matrix_step_size(probe))
    assert obj < 1e-20
    np.testing.assert_allclose(A1, A, atol=1e-12)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_prefix_and_suffix_rebuild_the_transfer_matrix(layer):
    n, M = 4, 3
    G = O.propagator_matrix(geom(M), n)
    o = [cplx(n * n, 30 + m) for m in range(M)]
    R, S = O.prefix_suffix(G, o, layer)
    np.testing.assert_allclose(R @ np.diag(o[layer]) @ S, O.transfer_matrix(G, o), atol=1e-11)


def decomposition_objective(Ahat, G, o, lam, layer, d):
    R, S = O.prefix_suffix(G, o, layer)
    return 0.5 * np.sum(np.abs(Ahat - lam * (R * d[None, :]) @ S) ** 2)


@pytest.mark.parametrize("layer", [0, 1, 2])
def test_decomposition_gradient_step_size_and_descent(layer):
    """The gradient of Eq. (Prox_Min) matches finite differences; c bounds
    (lam ||R_l|| ||S_l||)^2 by LAPACK's spectral norms; the step before the projection descends."""
    n, M, lam = 4, 3, 1.7
    G = O.propagator_matrix(geom(M), n)
    o = [cplx(n * n, 40 + m) for m in range(M)]
    Ahat = cplx((n * n, n * n), 44)
    g = O.decomposition_gradient(Ahat, G, o, lam, layer)
    for seed in range(3):
        d = cplx(n * n, 50 + seed)
        eps = 1e-6
        fp = decomposition_objective(Ahat, G, o, lam, layer, o[layer] + eps * d)
        fm = decomposition_objective(Ahat, G, o, lam, layer, o[layer] - eps * d)
        assert (fp - fm) / (2 * eps) == pytest.approx(np.real(np.vdot(g, d)), rel=1e-6)
    R, S = O.prefix_suffix(G, o, layer)
    mu = O.decomposition_step_size(o, lam, layer)
    assert 1.0 / mu >= (lam * np.linalg.norm(R, 2) * np.linalg.norm(S, 2)) ** 2 * (1 - 1e-12)
    f0 = decomposition_objective(Ahat, G, o, lam, layer, o[layer])
    assert decomposition_objective(Ahat, G, o, lam, layer, o[layer] - mu * g) <= f0


def test_exact_factorisation_is_a_fixed_point():
    n, M, lam = 4, 3, 2.5
    G = O.propagator_matrix(geom(M), n)
    o = [O.project_diagonal_unit(cplx(n * n, 60 + m)) for m in range(M)]
    Ahat = lam * O.transfer_matrix(G, o)
    new, lam1, A1, obj = O.decomposition_update(Ahat, G, o, lam)
    assert obj < 1e-24
    for a, b in zip(new, o):
        np.testing.assert_allclose(a, b, atol=1e-12)
    assert lam1 == pytest.approx(lam, rel=1e-12)
    np.testing.assert_allclose(A1, Ahat, atol=1e-12)


def test_one_slice_decomposition_is_the_diagonal_of_ahat():
    """M = 1: R = S = I and mu = 1/lambda^2, so the update is diag(Ahat)/||diag(Ahat)||,
    lambda becomes ||diag(Ahat)|| and A^{t+1} is the diagonal part of Ahat."""
    n = 5
    G = O.propagator_matrix(geom(1), n)
    Ahat = cplx((n * n, n * n), 70)
    new, lam1, A1, _ = O.decomposition_update(Ahat, G, [cplx(n * n, 71)], 1.0)
    dg = np.diag(Ahat)
    np.testing.assert_allclose(new[0], dg / np.linalg.norm(dg), atol=1e-13)
    assert lam1 == pytest.approx(np.linalg.norm(dg), rel=1e-12)
    np.testing.assert_allclose(A1, np.diag(dg), atol=1e-12)


def test_lambda_is_the_real_least_squares_scale():
    At = cplx((9, 9), 80)
    assert O.update_lambda(3.0 * At, At) == pytest.approx(3.0, rel=1e-13)
    assert O.update_lambda((3.0 + 2.0j) * At, At) == pytest.approx(3.0, rel=1e-13)
    Ahat = cplx((9, 9), 81)
    lam = O.update_lambda(Ahat, At)
    f = lambda t: np.sum(np.abs(Ahat - t * At) ** 2)
    assert f(lam) <= min(f(lam + 1e-3), f(lam - 1e-3))


def test_final_slices_carry_lambda():
    n, M = 4, 3
    G = O.propagator_matrix(geom(M), n)
    o = [cplx(n * n, 90 + m) for m in range(M)]
    for lam in (2.0, -0.5):
        np.testing.assert_allclose(O.transfer_matrix(G, O.final_slices(o, lam)),
                                   lam * O.transfer_matrix(G, o), atol=1e-10)


def test_algorithm_two_reduces_the_matrix_objective_on_noise_free_data():
    n, M = 6, 2
    g = geom(M, dz=40.0)
    G = O.propagator_matrix(g, n)
    truth = phase_slices(M, n, 95, amp=0.4)
    r = np.random.default_rng(96)
    probe = np.exp(1j * r.uniform(0, 2 * np.pi, (n, n))) * (1 + 0.3 * r.standard_normal((n, n)))
    shifts = full_raster(n)
    A = O.transfer_matrix(G, truth)
    I = (np.abs(O.dft_matrix_2d(n) @ A @ O.probe_matrix(probe, shifts)) ** 2).T.reshape(len(shifts), n, n)
    slices, lam, hm, hd = O.sparse_decomposition(g, probe, shifts, I, iterations=6, matrix_steps=3)
    assert len(hm) == 18 and len(hd) == 6
    assert hm[-1] < 0.2 * hm[0]
    assert all(np.isfinite(hm)) and all(np.isfinite(hd))
