"""FP64 CPU oracle for inverse multislice ptychography (arXiv 2205.03902).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
It shares no code with the CUDA library; the two meet only through the seeded
inputs of `workloads.synth`.

Plain, slow and literal: one scan position at a time, one slice at a time,
numpy's FFT as the Fourier operator, float64 / complex128 throughout.

Conventions (readings of the paper where it is silent):
  * F is the unnormalised 2-D DFT with kernel exp(-2 pi i k n / N); the paper
    uses ||F_2D||^2 = N^2 (Sec. 3.4, the learning rate of the matrix step), so
    F^-1 = F^H / N^2 and the propagator G_m = F^-1 diag(h) F is unitary.
  * Window model: position s crops the W x W window whose top-left corner is
    pos[s] = (y, x) from every slice; the probe is fixed.  The paper's own model
    shifts the probe cyclically over an N x N object (Sec. 2.1); `forward_circulant`
    implements that form and the tests show the two agree when W equals the
    object side and the window wraps around.
  * Spatial frequencies q_k = k / (W * pixel) for k < W/2, else (k - W) / (W * pixel).
  * The loss is the amplitude-flow objective without a factor 1/2 (Sec. 3.2).
  * Potential mode: X_m = exp(i sigma V_m) with a real projected potential V_m.
    Transmission mode: X_m is a free complex array (the paper's o_m).
  * Zero rule (Sec. 3.2 sets Qz/|Qz| to 0 where Qz = 0): a far-field value counts as
    zero when |Psi_k| <= ZERO_RULE_TAU * ||p||_2.  By Parseval ||p||_2 is the RMS
    far-field amplitude of every pattern of pure-phase slices, so this resolves
    "Psi_k = 0" at 1e-5 of the RMS amplitude, far above round-off.  At the paper's
    identity initialisation the exit wave is band-limited by the probe aperture and
    Psi vanishes outside it in exact arithmetic; the rule gives that exact-arithmetic
    residual instead of one whose phase is set by round-off.

Parity status: every function here is pinned by `tests/test_oracle_pins.py`
(closed forms, the paper's dense-matrix formulation, Parseval, finite
differences, brute-force spectral norms); no function is unpinned.
"""
from __future__ import annotations

import numpy as np

ZERO_RULE_TAU = 1e-5


# ----------------------------------------------------------------------------
# Operators of Sec. 2.1 / 2.2
# ----------------------------------------------------------------------------

def spatial_frequencies(n: int, pixel_A: float) -> np.ndarray:
    """Discrete reciprocal grid q_k of an n-point axis (cyclic index order, Sec. 1.4)."""
    k = np.arange(n)
    k = np.where(k < n // 2, k, k - n)
    return k / (n * pixel_A)


def fresnel_propagator(win: int, pixel_A: float, wavelength_A: float, dz_A: float) -> np.ndarray:
    """Fresnel propagator H_m, Eq. (fresnel_element) with zero tilt:
    h_{y,x} = exp(-i pi dz lambda (q_y^2 + q_x^2))."""
    q = spatial_frequencies(win, pixel_A)
    q2 = q[:, None] ** 2 + q[None, :] ** 2
    return np.exp(-1j * np.pi * dz_A * wavelength_A * q2)


def dft2(a: np.ndarray) -> np.ndarray:
    """F: unnormalised 2-D DFT (the paper's Fourier operator)."""
    return np.fft.fft2(a)


def dft2_adjoint(a: np.ndarray) -> np.ndarray:
    """F^H = N^2 F^-1."""
    return np.fft.ifft2(a) * (a.shape[-1] * a.shape[-2])


def propagate(e: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Fresnel transform V_z(E) = F^-1(F(E) o H)  (Sec. 2.1)."""
    return np.fft.ifft2(np.fft.fft2(e) * h)


def propagate_adjoint(c: np.ndarray, h: np.ndarray) -> np.ndarray:
    """G^H = F^H diag(conj h) F^-H = F^-1 diag(conj h) F (G is unitary, Sec. 2.2)."""
    return np.fft.ifft2(np.fft.fft2(c) * np.conj(h))


def transmission(V: np.ndarray, sigma: float) -> np.ndarray:
    """Phase grating X_m = exp(i sigma V_m) of a slice with projected potential V_m."""
    return np.exp(1j * sigma * V)


def window(a: np.ndarray, y: int, x: int, w: int, wrap: bool = False) -> np.ndarray:
    """Crop a[y:y+w, x:x+w] (cyclically if `wrap`)."""
    if wrap:
        ny, nx = a.shape[-2:]
        iy = (y + np.arange(w)) % ny
        ix = (x + np.arange(w)) % nx
        return a[..., iy[:, None], ix[None, :]]
    return a[..., y:y + w, x:x + w]


def window_add(dst: np.ndarray, y: int, x: int, val: np.ndarray, wrap: bool = False) -> None:
    """Adjoint of `window`: add `val` back into the window of `dst`."""
    w = val.shape[-1]
    if wrap:
        ny, nx = dst.shape[-2:]
        iy = (y + np.arange(w)) % ny
        ix = (x + np.arange(w)) % nx
        np.add.at(dst, (Ellipsis, iy[:, None], ix[None, :]), val)
    else:
        dst[..., y:y + w, x:x + w] += val


# ----------------------------------------------------------------------------
# Forward model, Sec. 2.1: E_1 = P o X_1, E_m = V_z(E_{m-1}) o X_m, I = |F(E_M)|^2
# ----------------------------------------------------------------------------

def slices_of(geom: dict, V=None, T=None) -> np.ndarray:
    """Complex slices X_m: exp(i sigma V) in potential mode, or T itself."""
    if T is not None:
        return np.asarray(T, dtype=np.complex128)
    return transmission(np.asarray(V, dtype=np.float64), geom["sigma"])


def position_forward(probe, X, y, x, h, wrap=False):
    """Multislice recursion for one scan position.

    Returns the wave incident on every slice, the exit wave of every slice and the
    far-field wave Psi = F(E_M).  No propagation follows the last slice.
    """
    L, w = X.shape[0], probe.shape[0]
    psi = np.asarray(probe, dtype=np.complex128)
    incident, exits = [], []
    for l in range(L):
        t = window(X[l], y, x, w, wrap)
        incident.append(psi)
        e = psi * t
        exits.append(e)
        if l < L - 1:
            psi = propagate(e, h)
    return incident, exits, dft2(exits[-1])


def forward(geom: dict, probe, pos, V=None, T=None, wrap=False) -> np.ndarray:
    """Far-field intensities I^s = |F(E^s_M)|^2, float64 [S][W][W] (Eq. intensity measurements)."""
    X = slices_of(geom, V, T)
    h = fresnel_propagator(geom["win"], geom["pixel_A"], geom["wavelength_A"], geom["dz_A"])
    out = np.zeros((len(pos), geom["win"], geom["win"]))
    for s, (y, x) in enumerate(np.asarray(pos)):
        _, _, psi_far = position_forward(probe, X, int(y), int(x), h, wrap)
        out[s] = np.abs(psi_far) ** 2
    return out


def forward_circulant(geom: dict, probe, shifts, V=None, T=None) -> np.ndarray:
    """The paper's own full-field form: the probe is shifted cyclically,
    p^s_{y,x} = p_{y - y_s, x - x_s}, over an N x N object (Sec. 2.1)."""
    X = slices_of(geom, V, T)
    n = X.shape[-1]
    h = fresnel_propagator(n, geom["pixel_A"], geom["wavelength_A"], geom["dz_A"])
    out = np.zeros((len(shifts), n, n))
    for s, (ys, xs) in enumerate(np.asarray(shifts)):
        ps = np.roll(np.asarray(probe, dtype=np.complex128), (int(ys), int(xs)), axis=(0, 1))
        _, _, psi_far = position_forward(ps, X, 0, 0, h)
        out[s] = np.abs(psi_far) ** 2
    return out


# ----------------------------------------------------------------------------
# Amplitude flow, Sec. 3.2: A(z) = || sqrt(y) - |Qz| ||^2,
# grad = Q^H (Qz - Qz/|Qz| o sqrt(y)) with the fraction set to 0 where Qz = 0.
# ----------------------------------------------------------------------------

def zero_threshold(probe) -> float:
    """Amplitude at or below which a far-field value counts as zero (see the zero rule)."""
    return ZERO_RULE_TAU * float(np.linalg.norm(np.asarray(probe).ravel()))


def far_field_residual(psi_far, i_meas, thr=0.0):
    """Loss term and the residual R = Psi - sqrt(I) Psi/|Psi|, the fraction taken as 0
    where |Psi| <= thr (Sec. 3.2; thr = 0 is the literal rule)."""
    amp = np.abs(psi_far)
    root = np.sqrt(np.asarray(i_meas, dtype=np.float64))
    loss = float(np.sum((root - amp) ** 2))
    nz = amp > thr
    phase = np.zeros_like(psi_far)
    phase[nz] = psi_far[nz] / amp[nz]
    return loss, psi_far - root * phase


def position_backward(X, y, x, h, incident, chi, lowest=0, wrap=False):
    """Back-propagate chi = dL/d conj(E_M) through the slices (Sec. 3.3, R_l and S_l).

    Yields, for l = L-1 .. lowest, the window gradient dL/d conj(X_l) = conj(psi_in,l) o chi_l
    and, when lowest == 0, returns the probe gradient conj(X_1) o chi_1 as well.
    Recursion: chi_{l-1} = G^H (conj(X_l) o chi_l).
    """
    L, w = X.shape[0], chi.shape[0]
    grads = {}
    dprobe = None
    for l in range(L - 1, lowest - 1, -1):
        t = window(X[l], y, x, w, wrap)
        grads[l] = np.conj(incident[l]) * chi
        chi_in = np.conj(t) * chi
        if l > 0:
            chi = propagate_adjoint(chi_in, h)
        else:
            dprobe = chi_in
    return grads, dprobe


def loss_grad(geom: dict, probe, pos, i_meas, V=None, T=None, wrap=False, want_probe=True):
    """Loss, object gradient and probe gradient over all positions.

    Returns (loss, dX, dprobe) where dX = dL/d conj(X) (Wirtinger, complex [L][Ny][Nx]),
    and in potential mode additionally dV = dL/dV = 2 sigma Im(conj(X) o dX) (real).
    """
    X = slices_of(geom, V, T)
    w = geom["win"]
    h = fresnel_propagator(w, geom["pixel_A"], geom["wavelength_A"], geom["dz_A"])
    dX = np.zeros_like(X)
    dprobe = np.zeros((w, w), dtype=np.complex128)
    loss = 0.0
    thr = zero_threshold(probe)
    for s, (y, x) in enumerate(np.asarray(pos)):
        y, x = int(y), int(x)
        incident, _, psi_far = position_forward(probe, X, y, x, h, wrap)
        ls, r = far_field_residual(psi_far, i_meas[s], thr)
        loss += ls
        chi = dft2_adjoint(r)
        grads, dp = position_backward(X, y, x, h, incident, chi, 0, wrap)
        for l, g in grads.items():
            window_add(dX[l], y, x, g, wrap)
        dprobe += dp
    out = dict(loss=loss, dX=dX, dprobe=dprobe)
    if T is None:
        out["dV"] = 2.0 * geom["sigma"] * np.imag(np.conj(X) * dX)
    return out


def layer_quantities(geom: dict, probe, pos, i_meas, layer: int, V=None, T=None, wrap=False):
    """Everything one gradient step on slice `layer` needs (Sec. 3.3, Eq. Single_Layer):
    the loss, dL/d conj(o_l) and the illumination map sum_s |S_l p^s|^2 scattered
    into the object frame (the diagonal of Q_l^H Q_l / N^2 when R_l is unitary)."""
    X = slices_of(geom, V, T)
    w = geom["win"]
    h = fresnel_propagator(w, geom["pixel_A"], geom["wavelength_A"], geom["dz_A"])
    dXl = np.zeros(X.shape[1:], dtype=np.complex128)
    illum = np.zeros(X.shape[1:])
    loss = 0.0
    thr = zero_threshold(probe)
    for s, (y, x) in enumerate(np.asarray(pos)):
        y, x = int(y), int(x)
        incident, _, psi_far = position_forward(probe, X, y, x, h, wrap)
        ls, r = far_field_residual(psi_far, i_meas[s], thr)
        loss += ls
        grads, _ = position_backward(X, y, x, h, incident, dft2_adjoint(r), layer, wrap)
        window_add(dXl, y, x, grads[layer], wrap)
        window_add(illum, y, x, np.abs(incident[layer]) ** 2, wrap)
    return loss, dXl, illum, X


def layer_step(geom: dict, probe, pos, i_meas, layer: int, V=None, T=None, step=None, wrap=False):
    """One gradient step of Algorithm 1 on slice `layer` (Eq. Opt_Prob_Amplitude_Flow_Step).

    Step size mu = ||Q_l||^-2 with ||Q_l||^2 = N^2 max_pixel sum_s |S_l p^s|^2, exact when the
    later slices are unimodular (R_l unitary).  In transmission mode a non-unimodular later
    slice enlarges the bound by prod_{m>l} max|o_m|^2.  In potential mode the tangent step
    on exp(i sigma V) gives mu_V = mu / (2 sigma^2).
    Returns (new V or T, loss before the step, mu used).
    """
    loss, dXl, illum, X = layer_quantities(geom, probe, pos, i_meas, layer, V, T, wrap)
    w2 = geom["win"] ** 2
    norm2 = w2 * float(np.max(illum))
    if T is not None:
        for m in range(layer + 1, X.shape[0]):
            norm2 *= float(np.max(np.abs(X[m]))) ** 2
    mu_t = 1.0 / norm2 if norm2 > 0 else 0.0
    if T is not None:
        mu = mu_t if step is None or step <= 0 else step
        Tn = np.array(X, copy=True)
        Tn[layer] = Tn[layer] - mu * dXl
        return Tn, loss, mu
    sig = geom["sigma"]
    mu = mu_t / (2.0 * sig * sig) if step is None or step <= 0 else step
    dVl = 2.0 * sig * np.imag(np.conj(X[layer]) * dXl)
    Vn = np.array(V, dtype=np.float64, copy=True)
    Vn[layer] = Vn[layer] - mu * dVl
    return Vn, loss, mu


def probe_step(geom: dict, probe, pos, i_meas, V=None, T=None, step=None, normalize=False, wrap=False):
    """One amplitude-flow step on the probe (Sec. 3.5, Eq. Opt_Est_Probe), generalised from the
    centre position to all S positions: p <- p - mu sum_s conj(X_1[win_s]) o chi_1^s.

    For unimodular slices ||Q_p||^2 = S N^2, so mu = 1 / (S N^2).  With `normalize`, the probe is
    rescaled afterwards so that N^2 ||p||^2 equals the mean measured pattern sum (Parseval).
    Returns (new probe, loss before the step, mu used).
    """
    r = loss_grad(geom, probe, pos, i_meas, V, T, wrap)
    s_count = len(pos)
    w2 = geom["win"] ** 2
    mu = (1.0 / (s_count * w2) if s_count else 0.0) if step is None or step <= 0 else step
    p = np.asarray(probe, dtype=np.complex128) - mu * r["dprobe"]
    if normalize and s_count:
        target = float(np.mean(np.sum(np.asarray(i_meas, dtype=np.float64).reshape(s_count, -1), axis=1)))
        cur = w2 * float(np.sum(np.abs(p) ** 2))
        if cur > 0:
            p = p * np.sqrt(target / cur)
    return p, r["loss"], mu


def layerwise_estimation(geom: dict, probe, pos, i_meas, V0, sweeps: int, steps_per_layer: int = 1):
    """Algorithm 1 (Layer-wise Estimation) in potential mode: for each sweep, for each slice in
    ascending order (Gauss-Seidel: earlier slices already updated), K gradient steps."""
    V = np.array(V0, dtype=np.float64, copy=True)
    history = []
    for _ in range(sweeps):
        for layer in range(V.shape[0]):
            for _ in range(steps_per_layer):
                V, loss, _ = layer_step(geom, probe, pos, i_meas, layer, V=V)
                history.append(loss)
    return V, history


def plain_method(geom: dict, probe, pos, i_meas, V0, sweeps: int, steps_per_layer: int = 1, probe_steps: int = 0,
                 normalize=False, layer_mu=None, probe_mu=None):
    """Algorithm 1 (Sec. 3.3) with probe estimation (Sec. 3.5), potential mode.  Each sweep takes
    every slice in ascending order for `steps_per_layer` gradient steps (Gauss-Seidel), then the
    probe for `probe_steps` amplitude-flow steps with the slices just estimated.  The paper
    estimates the probe after the object; alternating the two per sweep is what a probe guess
    with a defocus error needs, and steps_per_layer = 0 leaves probe steps only.
    Returns (V, probe, history): history holds the loss before every step, in the order the steps
    run, and last the loss after the final step."""
    V = np.array(V0, dtype=np.float64, copy=True)
    p = np.asarray(probe, dtype=np.complex128).copy()
    history = []
    for _ in range(sweeps):
        for layer in range(V.shape[0]):
            for _ in range(steps_per_layer):
                V, loss, _ = layer_step(geom, p, pos, i_meas, layer, V=V, step=layer_mu)
                history.append(loss)
        for _ in range(probe_steps):
            p, loss, _ = probe_step(geom, p, pos, i_meas, V=V, step=probe_mu, normalize=normalize)
            history.append(loss)
    history.append(loss_grad(geom, p, pos, i_meas, V=V, want_probe=False)["loss"])
    return V, p, history


def residual_conditioning(geom: dict, probe, pos, i_meas, V=None, T=None, band=0.0):
    """How strongly a state amplifies rounding in the forward model into its gradients.

    A forward whose far field carries an absolute error e ||p|| per value (||p|| being the
    RMS far-field amplitude) changes R = Psi - sqrt(I) Psi/|Psi| by about e ||p|| m_k at
    value k, with m_k = max(1, sqrt(I_k) / |Psi_k|) above the zero-rule threshold (the phase
    of a small Psi_k is scaled by sqrt(I_k)) and m_k = 1 below it.  Returns
    (kappa, cancellation, flip):
      kappa = ||p|| sqrt(sum_k m_k^2) / ||R||, so the relative gradient error is ~ e kappa
        (it reduces to ||Psi|| / ||R|| where every |Psi_k| >= sqrt(I_k));
      cancellation = sum_s ||g_s|| / ||sum_s g_s|| of the per-position probe gradients g_s;
      flip = sqrt(sum I_k over far-field values within `band` (absolute amplitude) of the
        threshold) / ||R||: the largest relative change of R if a computation uncertain by
        `band` decided those values the other way.
    """
    X = slices_of(geom, V, T)
    w = geom["win"]
    h = fresnel_propagator(w, geom["pixel_A"], geom["wavelength_A"], geom["dz_A"])
    thr = zero_threshold(probe)
    pnorm = float(np.linalg.norm(np.asarray(probe).ravel()))
    nR = m2 = terms = flip2 = 0.0
    acc = np.zeros((w, w), dtype=np.complex128)
    for s, (y, x) in enumerate(np.asarray(pos)):
        incident, _, psi_far = position_forward(probe, X, int(y), int(x), h)
        _, r = far_field_residual(psi_far, i_meas[s], thr)
        amp = np.abs(psi_far)
        root = np.sqrt(np.asarray(i_meas[s], dtype=np.float64))
        above = amp > thr
        m = np.ones_like(amp)
        m[above] = np.maximum(1.0, root[above] / amp[above])
        m2 += float(np.sum(m * m))
        nR += float(np.sum(np.abs(r) ** 2))
        flip2 += float(np.sum((root ** 2)[np.abs(amp - thr) <= band]))
        _, g = position_backward(X, int(y), int(x), h, incident, dft2_adjoint(r), 0)
        terms += float(np.linalg.norm(g))
        acc += g
    kappa = pnorm * float(np.sqrt(m2 / nR)) if nR > 0 else float("inf")
    flip = float(np.sqrt(flip2 / nR)) if nR > 0 else 0.0
    return kappa, terms / max(float(np.linalg.norm(acc)), 1e-300), flip


# ----------------------------------------------------------------------------
# Algorithm 2 (Sparse Matrix Decomposition, Sec. 3.4) on the paper's circulant model:
# an N x N object, the probe shifted cyclically, dense N^2 x N^2 matrices, row-major vec.
# ----------------------------------------------------------------------------

def dft_matrix_2d(n: int) -> np.ndarray:
    """F_2D = F_1 (x) F_1, the unnormalised 2-D DFT of a row-major vectorised n x n array (Sec. 2.2)."""
    f1 = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    return np.kron(f1, f1)


def propagator_matrix(geom: dict, n: int) -> np.ndarray:
    """G = F^-1 diag(vec H) F (Sec. 2.2)."""
    F = dft_matrix_2d(n)
    h = fresnel_propagator(n, geom["pixel_A"], geom["wavelength_A"], geom["dz_A"]).ravel()
    return (np.conj(F).T / n ** 2) @ (h[:, None] * F)


def probe_matrix(probe, shifts) -> np.ndarray:
    """P = (p^1, ..., p^S), p^s = vec of the probe shifted cyclically by shift s (Sec. 2.1)."""
    return np.stack([np.roll(np.asarray(probe, dtype=np.complex128), (int(a), int(b)), axis=(0, 1)).ravel()
                     for a, b in np.asarray(shifts)], axis=1)


def measurement_matrix(i_meas) -> np.ndarray:
    """I = (i^1, ..., i^S) with i^s = vec I^s."""
    i_meas = np.asarray(i_meas, dtype=np.float64)
    return i_meas.reshape(i_meas.shape[0], -1).T


def transfer_matrix(G, o) -> np.ndarray:
    """A_M = O_M prod_m G O_m (Eq. exit_wave_mslices) from the slice diagonals o [M][N^2]."""
    A = np.diag(o[0])
    for m in range(1, len(o)):
        A = o[m][:, None] * (G @ A)
    return A


def shift_operator_norm(probe) -> float:
    """||P||_2 taken as max_k |(F p)_k|.  P x is the cyclic convolution of p with the shifts'
    impulses weighted by x, so ||P||_2 <= ||C(p)||_2 = max |F p|, with equality when the shifts
    are all N^2 cyclic shifts (the paper's full raster scan, Table 1)."""
    return float(np.max(np.abs(np.fft.fft2(np.asarray(probe, dtype=np.complex128)))))


def matrix_objective_residual(A, F, P, I):
    """U = F A P, the objective 1/2 sum (sqrt(I) - |U|)^2 of Eq. (Opt_Prob_Matrix) and
    R = (|U| - sqrt(I)) o U/|U| = U - sqrt(I) U/|U|, the fraction taken as 0 where
    |U| <= 1e-5 times the RMS measured amplitude sqrt(mean I)."""
    U = F @ (A @ P)
    amp = np.abs(U)
    root = np.sqrt(I)
    objective = 0.5 * float(np.sum((root - amp) ** 2))
    thr = ZERO_RULE_TAU * float(np.sqrt(np.mean(I)))
    ph = np.zeros_like(U)
    nz = amp > thr
    ph[nz] = U[nz] / amp[nz]
    return objective, U - root * ph


def matrix_step(A, F, P, I, mu):
    """One gradient step of Eq. (Opt_Prob_Matrix):
    A <- A - mu F^H ((|FAP| - sqrt(I)) o FAP/|FAP|) P^H.  Returns (new A, objective before)."""
    objective, R = matrix_objective_residual(A, F, P, I)
    return A - mu * (np.conj(F).T @ R @ np.conj(P).T), objective


def matrix_step_size(probe) -> float:
    """mu = 1 / (||F_2D||^2 ||P||^2) = 1 / (N^2 ||P||^2) (Sec. 3.4)."""
    n2 = np.asarray(probe).size
    return 1.0 / (n2 * shift_operator_norm(probe) ** 2)


def prefix_suffix(G, o, layer):
    """R_l = prod_{m > l} O_m G and S_l = prod_{m < l} G O_m (Eq. Layerwise_Prefix_Suffix), dense."""
    n = G.shape[0]
    R = np.eye(n, dtype=complex)
    for m in range(layer + 1, len(o)):
        R = o[m][:, None] * (G @ R)
    S = np.eye(n, dtype=complex)
    for m in range(0, layer):
        S = G @ (o[m][:, None] * S)
    return R, S


def decomposition_gradient(Ahat, G, o, lam, layer):
    """diag of lam R_l^H (lam R_l O_l S_l - Ahat) S_l^H, the gradient of
    1/2 ||Ahat - lam R_l O_l S_l||_F^2 with respect to conj(diag O_l) (Eq. Prox_Min)."""
    R, S = prefix_suffix(G, o, layer)
    M = lam * ((R * o[layer][None, :]) @ S) - Ahat
    return lam * np.sum((np.conj(R).T @ M) * np.conj(S), axis=1)


def decomposition_step_size(o, lam, layer) -> float:
    """mu = 1/c with c = (lam prod_{m != l} max|o_m|)^2 >= (lam ||R_l|| ||S_l||)^2, since every
    G_m is unitary and ||O_m||_2 = max |o_m|."""
    bound = abs(lam) * float(np.prod([np.max(np.abs(o[m])) for m in range(len(o)) if m != layer]))
    return 1.0 / bound ** 2 if bound > 0 else 0.0


def project_diagonal_unit(x) -> np.ndarray:
    """The projection P of Eq. (Prox_Min): keep the diagonal, scale it to unit Frobenius norm."""
    nrm = float(np.linalg.norm(x))
    return x / nrm if nrm > 0 else x


def decomposition_sweep(Ahat, G, o, lam):
    """One pass of the layer loop of Algorithm 2: every slice takes the proximal step of
    Eq. (Prox_Min) with the prefix, suffix and lambda of iteration t (all slices at O^t).
    Returns (new slices, objective 1/2 ||Ahat - lam A(O^t)||_F^2)."""
    objective = 0.5 * float(np.sum(np.abs(Ahat - lam * transfer_matrix(G, o)) ** 2))
    new = []
    for layer in range(len(o)):
        g = decomposition_gradient(Ahat, G, o, lam, layer)
        new.append(project_diagonal_unit(o[layer] - decomposition_step_size(o, lam, layer) * g))
    return new, objective


def update_lambda(Ahat, Atilde) -> float:
    """lambda = Re Tr(Ahat^H Atilde) / Tr(Atilde^H Atilde) (Eq. Update Lambda), the real
    least-squares scale of Atilde."""
    den = float(np.real(np.vdot(Atilde.ravel(), Atilde.ravel())))
    return float(np.real(np.vdot(Ahat.ravel(), Atilde.ravel()))) / den if den > 0 else 0.0


def decomposition_update(Ahat, G, o, lam):
    """Layer sweep, lambda update and A^{t+1} = lambda^{t+1} A(O^{t+1}) (Algorithm 2, one iteration
    after the matrix estimate).  Returns (new slices, new lambda, new A, objective before)."""
    new, objective = decomposition_sweep(Ahat, G, o, lam)
    At = transfer_matrix(G, new)
    lam_new = update_lambda(Ahat, At)
    return new, lam_new, lam_new * At, objective


def final_slices(o, lam):
    """The returned slices lambda^(1/M) O_m (principal complex root, so their product carries lambda)."""
    root = complex(lam) ** (1.0 / len(o))
    return [root * x for x in o]


def sparse_decomposition(geom: dict, probe, shifts, i_meas, iterations: int, matrix_steps: int = 1, o0=None):
    """Algorithm 2 from slices o0 (default: all ones) and lambda^0 = 1: per iteration, `matrix_steps`
    gradient steps on Eq. (Opt_Prob_Matrix), then the decomposition update.  Returns
    (slices lambda^(1/M) O_m, lambda, matrix-objective history, decomposition-objective history)."""
    n = np.asarray(probe).shape[0]
    M = geom["n_slices"]
    F = dft_matrix_2d(n)
    G = propagator_matrix(geom, n)
    P = probe_matrix(probe, shifts)
    I = measurement_matrix(i_meas)
    mu = matrix_step_size(probe)
    o = [np.ones(n * n, dtype=complex) for _ in range(M)] if o0 is None else [np.asarray(x, dtype=complex).ravel() for x in o0]
    lam = 1.0
    A = lam * transfer_matrix(G, o)
    hist_m, hist_d = [], []
    for _ in range(iterations):
        for _ in range(matrix_steps):
            A, obj = matrix_step(A, F, P, I, mu)
            hist_m.append(obj)
        o, lam, A, obj = decomposition_update(A, G, o, lam)
        hist_d.append(obj)
    return final_slices(o, lam), lam, hist_m, hist_d


# ----------------------------------------------------------------------------
# Error metrics, Sec. 5.1
# ----------------------------------------------------------------------------

def relative_measurement_error(loss: float, i_meas) -> float:
    """|| sqrt(I) - |F A P| ||_F / || sqrt(I) ||_F (Eq. error_metric_intensity) from the loss."""
    tot = float(np.sum(np.asarray(i_meas, dtype=np.float64)))
    return float(np.sqrt(loss / tot)) if tot > 0 else 0.0


def relative_reconstruction_error(X_true, X_est) -> float:
    """(1/M) sum_m ||O_m - O^_m||_F / ||O_m||_F (Eq. error_metric_object)."""
    X_true = np.asarray(X_true)
    return float(np.mean([np.linalg.norm(X_true[m] - X_est[m]) / np.linalg.norm(X_true[m])
                          for m in range(X_true.shape[0])]))
