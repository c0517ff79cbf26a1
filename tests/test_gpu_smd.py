"""Parity of the CUDA Sparse Matrix Decomposition path (Algorithm 2, Sec. 3.4) with the oracle.

Every entry point of include/msp_smd.h is compared with the FP64 oracle on the same
seeded inputs, rounded once to the library's precision (complex64 / float32) and fed
to both sides.

Tolerances (relative L2).  The library sums in FP32: a contraction of length K
rounds like a random walk, sqrt(K) 2^-24 of the result.  The matrix step's two
contractions run on the tensor cores with every operand split into a pair of tf32
values and FP32 accumulation over groups of 128 K (then round-to-nearest FP32 sums):
their error is at most max(sqrt(K), 32) 2^-24 (32 2^-24 = 1.9e-6, the measured level
at any K).  So one matrix step carries e = (max(N, 32) + max(sqrt(S), 32) + 4 sqrt(N))
2^-24 (A P over N^2 terms, C P^H over S terms, four DFT passes of at most N terms: the
kernels factor the N-point DFT, N1 + N2 + 1 terms per output), and a
multislice impulse pass through M slices e = 8 (M - 1) sqrt(N) 2^-24 (four passes per
propagator, forward and adjoint).  The
residual R = U - sqrt(I) U/|U| and the decomposition residual lambda A(o) - Ahat
amplify that error by kappa = ||U|| / ||R|| (resp. ||lambda A(o)|| / ||M||), so the bar
is max(1e-5, 2 e (1 + kappa)); scalars that are sums of positive terms take
max(1e-5, 2 e kappa).
"""
import math

import numpy as np
import pytest
import torch

from oracle import msp_oracle as O
from workloads import synth

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -24


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def bar(e, kappa=1.0):
    return max(1e-5, 2.0 * e * (1.0 + kappa))


def e_matrix(n, S):
    return (max(n, 32) + max(math.sqrt(S), 32) + 4 * math.sqrt(n)) * EPS


def e_chain(n, M):
    return max(1, 8 * (M - 1)) * math.sqrt(n) * EPS


@pytest.fixture(scope="module")
def msp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp as m
    return m


def c64(x):
    return np.asarray(x).astype(np.complex64)


def f32(x):
    return np.asarray(x).astype(np.float32)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


class Case:
    """Seeded Algorithm 2 inputs: geometry, probe, shifts, truth slices and noise-free I."""

    def __init__(self, n, M, S=None, seed=0, dz=20.0, count=None, truth_amp=0.5, lattice=False):
        cfg = synth.SMD_GAAS
        self.n, self.M = n, M
        self.geom = dict(synth.smd_geometry(cfg), n=n, n_slices=M, dz_A=dz, obj_ny=n, obj_nx=n, win=n)
        self.shifts = synth.cyclic_shifts(n, count=count, seed=seed) if count else synth.cyclic_shifts(n)
        self.geom["n_pos"] = len(self.shifts)
        pc = synth.Workload("p", M, n, cfg.pixel_A, dz, cfg.kv, n, (1, 1), 1, cfg.aperture_mrad, 0.0, None)
        self.probe = c64(synth.probe(pc))
        if lattice and n == cfg.obj and M == cfg.n_slices:
            V = synth.potential_slices(cfg)
            self.truth = c64(np.exp(1j * self.geom["sigma"] * V))
        else:
            self.truth = c64(synth.random_phase_slices(M, n, seed + 100, truth_amp))
        self.I = f32(O.forward_circulant(self.geom, self.probe.astype(np.complex128), self.shifts,
                                         T=self.truth.astype(np.complex128)))
        self.Imat = O.measurement_matrix(self.I.astype(np.float64))
        self.F = O.dft_matrix_2d(n)
        self.P = O.probe_matrix(self.probe, self.shifts)
        self._G = None

    @property
    def G(self):
        if self._G is None:
            self._G = O.propagator_matrix(self.geom, self.n)
        return self._G

    def sg(self, msp):
        return msp.smd_geometry(**self.geom)


def slices_list(o):
    return [x.ravel().astype(np.complex128) for x in np.asarray(o)]


# ----------------------------------------------------------------------------- transfer

@pytest.mark.parametrize("n,M", [(16, 1), (16, 3), (24, 2), (40, 3), (48, 5)])
def test_transfer_matrix(msp, n, M):
    case = Case(n, M, seed=n + M, count=4)
    o = c64(synth.random_complex((M, n, n), 7 + n))
    lam = 1.75
    A = msp.smd_transfer(case.sg(msp), dev(o), lam).cpu().numpy()
    ref = lam * O.transfer_matrix(case.G, slices_list(o))
    assert rel(A.T, ref) <= bar(e_chain(n, M))


def test_transfer_matrix_sampled_columns_at_the_largest_grid(msp):
    """N = 64 (a 4096 x 4096 matrix): sampled columns against the oracle's FFT multislice of
    a unit impulse (column j of A is the exit wave of an impulse at pixel j)."""
    n, M = 64, 3
    case = Case(n, M, seed=9, count=4)
    o = c64(synth.random_complex((M, n, n), 77))
    A = msp.smd_transfer(case.sg(msp), dev(o), 1.0).cpu().numpy()
    h = O.fresnel_propagator(n, case.geom["pixel_A"], case.geom["wavelength_A"], case.geom["dz_A"])
    X = o.astype(np.complex128)
    for j in (0, 1, 63, 64, 2047, 4095):
        delta = np.zeros((n, n), complex)
        delta.flat[j] = 1.0
        _, exits, _ = O.position_forward(delta, X, 0, 0, h)
        assert rel(A[j], exits[-1].ravel()) <= bar(e_chain(n, M)), j


# ----------------------------------------------------------------------------- matrix step

def matrix_step_check(msp, case, A0, step=0.0):
    g = case.sg(msp)
    A = dev(A0)
    obj, mu = msp.smd_matrix_step(g, A, dev(case.probe), dev(case.shifts), dev(case.I), step=step)
    torch.cuda.synchronize()
    A1 = A.cpu().numpy()
    mu_ref = step if step > 0 else O.matrix_step_size(case.probe.astype(np.complex128))
    A_ref, obj_ref = O.matrix_step(A0.T.astype(np.complex128), case.F, case.P, case.Imat, mu_ref)
    _, R = O.matrix_objective_residual(A0.T.astype(np.complex128), case.F, case.P, case.Imat)
    U = case.F @ (A0.T.astype(np.complex128) @ case.P)
    kappa = np.linalg.norm(U) / max(np.linalg.norm(R), 1e-300)
    e = e_matrix(case.n, len(case.shifts))
    assert mu.item() == pytest.approx(mu_ref, rel=1e-6)
    dA = A1.T.astype(np.complex128) - A0.T
    assert rel(dA, A_ref - A0.T) <= bar(e, kappa), (rel(dA, A_ref - A0.T), bar(e, kappa))
    assert obj.item() == pytest.approx(obj_ref, rel=max(1e-5, 2 * e * kappa))
    return A1


@pytest.mark.parametrize("n,M,count", [(16, 2, None), (24, 3, 37), (32, 2, 200), (48, 2, 64)])
def test_matrix_step_from_identity_slices(msp, n, M, count):
    """The first matrix step of Algorithm 2 (A^0 from all-one slices), full raster and
    random shift subsets (ragged GEMM tiles, split contractions)."""
    case = Case(n, M, seed=3 * n + M, count=count)
    A0 = c64(O.transfer_matrix(case.G, [np.ones(n * n, complex)] * M).T)
    matrix_step_check(msp, case, A0)


def test_matrix_step_at_the_largest_grid(msp):
    """N = 64 with a generic dense A (4096 x 4096) and 96 shifts."""
    n = 64
    case = Case(n, 2, seed=13, count=96)
    A0 = c64(synth.random_complex((n * n, n * n), 12) / n)
    matrix_step_check(msp, case, A0)


def test_matrix_step_fixed_step_and_generic_matrix(msp):
    n = 16
    case = Case(n, 2, seed=5, count=100)
    A0 = c64(synth.random_complex((n * n, n * n), 9) / n)
    matrix_step_check(msp, case, A0, step=3.0e-4)


def test_matrix_step_table1_size(msp):
    """The paper's setting: N = 40, all 1600 cyclic shifts, three lattice slices."""
    case = Case(40, 3, seed=1, lattice=True)
    A0 = c64(O.transfer_matrix(case.G, [np.ones(1600, complex)] * 3).T)
    A1 = matrix_step_check(msp, case, A0)
    # monotone: a second step from the GPU's own iterate does not raise the objective
    g = case.sg(msp)
    A = dev(A1)
    obj2, _ = msp.smd_matrix_step(g, A, dev(case.probe), dev(case.shifts), dev(case.I))
    obj1 = O.matrix_objective_residual(A0.T.astype(np.complex128), case.F, case.P, case.Imat)[0]
    assert obj2.item() <= obj1 * (1 + 1e-6)


def test_matrix_step_keeps_an_exact_solution(msp):
    n = 24
    case = Case(n, 2, seed=11, count=150)
    A0 = c64(O.transfer_matrix(case.G, slices_list(case.truth)).T)
    A = dev(A0)
    obj, _ = msp.smd_matrix_step(case.sg(msp), A, dev(case.probe), dev(case.shifts), dev(case.I))
    Ar = A.cpu().numpy()
    assert rel(Ar, A0) <= 1e-5
    sumI = float(np.sum(case.I.astype(np.float64)))
    assert obj.item() <= 1e-8 * sumI


# ----------------------------------------------------------------------------- decomposition

def decompose_check(msp, case, Ahat, o, lam):
    g = case.sg(msp)
    A = dev(Ahat)
    ot = dev(o)
    lt = torch.tensor([lam], dtype=torch.float64, device="cuda")
    obj = msp.smd_decompose(g, A, ot, lt)
    torch.cuda.synchronize()
    new_ref, lam_ref, A_ref, obj_ref = O.decomposition_update(Ahat.T.astype(np.complex128), case.G, slices_list(o), lam)
    M_res = Ahat.T.astype(np.complex128) - lam * O.transfer_matrix(case.G, slices_list(o))
    kappa = abs(lam) * np.linalg.norm(O.transfer_matrix(case.G, slices_list(o))) / max(np.linalg.norm(M_res), 1e-300)
    e = e_chain(case.n, case.M)
    got = ot.cpu().numpy()
    for m in range(case.M):
        assert rel(got[m].ravel(), new_ref[m]) <= bar(e, kappa), (m, rel(got[m].ravel(), new_ref[m]))
    assert lt.item() == pytest.approx(lam_ref, rel=bar(e, kappa))
    assert rel(A.cpu().numpy().T, A_ref) <= bar(e, kappa)
    assert obj.item() == pytest.approx(obj_ref, rel=max(1e-5, 2 * e * kappa))


@pytest.mark.parametrize("n,M", [(16, 1), (16, 3), (24, 2), (32, 4), (24, 5)])
def test_decomposition_from_a_matrix_estimate(msp, n, M):
    """Ahat = the transfer matrix of the truth slices plus a perturbation; slices start at
    all ones (the first decomposition of Algorithm 2, lambda = 1)."""
    case = Case(n, M, seed=7 * n + M, count=min(64, n * n))
    At = O.transfer_matrix(case.G, slices_list(case.truth))
    Ahat = c64((At + 0.05 * synth.random_complex(At.shape, 3) / n).T)
    o = c64(np.ones((M, n, n)))
    decompose_check(msp, case, Ahat, o, 1.0)


def test_decomposition_from_unit_slices_and_negative_lambda(msp):
    n, M = 24, 3
    case = Case(n, M, seed=21, count=50)
    o = c64(np.stack([O.project_diagonal_unit(x) for x in slices_list(synth.random_complex((M, n, n), 4))]).reshape(M, n, n))
    Ahat = c64(synth.random_complex((n * n, n * n), 5) / n)
    decompose_check(msp, case, Ahat, o, -0.8)


def test_decomposition_table1_size(msp):
    case = Case(40, 3, seed=2, lattice=True)
    At = O.transfer_matrix(case.G, slices_list(case.truth))
    Ahat = c64((At + 0.02 * synth.random_complex(At.shape, 6) / 40).T)
    decompose_check(msp, case, Ahat, c64(np.ones((3, 40, 40))), 1.0)


def test_one_slice_decomposition_at_the_largest_grid(msp):
    """N = 64, M = 1: R = S = I, so the slice becomes diag(Ahat)/||diag(Ahat)||, lambda
    ||diag(Ahat)|| and A the diagonal part of Ahat (the closed form of the one-slice case)."""
    n = 64
    case = Case(n, 1, seed=17, count=4)
    Ahat = c64(synth.random_complex((n * n, n * n), 14) / n)
    A, ot = dev(Ahat), dev(c64(np.ones((1, n, n))))
    lt = torch.tensor([1.0], dtype=torch.float64, device="cuda")
    msp.smd_decompose(case.sg(msp), A, ot, lt)
    d = np.diag(Ahat).astype(np.complex128)       # Ahat[j][j]: row j is column j
    assert rel(ot.cpu().numpy().ravel(), d / np.linalg.norm(d)) <= 1e-5
    assert lt.item() == pytest.approx(np.linalg.norm(d), rel=1e-5)
    Ag = A.cpu().numpy()
    assert rel(np.diag(Ag), d) <= 1e-5
    off = Ag - np.diag(np.diag(Ag))
    assert np.abs(off).max() <= 1e-6 * np.abs(d).max()


def test_exact_factorisation_is_kept(msp):
    n, M, lam = 16, 3, 2.5
    case = Case(n, M, seed=31, count=20)
    o = c64(np.stack([O.project_diagonal_unit(x) for x in slices_list(case.truth)]).reshape(M, n, n))
    Ahat = c64(lam * O.transfer_matrix(case.G, slices_list(o)).T)
    g = case.sg(msp)
    A, ot = dev(Ahat), dev(o)
    lt = torch.tensor([lam], dtype=torch.float64, device="cuda")
    obj = msp.smd_decompose(g, A, ot, lt)
    assert rel(ot.cpu().numpy(), o) <= 1e-5
    assert lt.item() == pytest.approx(lam, rel=1e-5)
    assert obj.item() <= 1e-9 * float(np.sum(np.abs(Ahat.astype(np.complex128)) ** 2))


# ----------------------------------------------------------------------------- final slices, trajectory

def test_final_slices(msp):
    n, M = 16, 3
    case = Case(n, M, seed=41, count=10)
    o = c64(synth.random_complex((M, n, n), 8))
    for lam in (3.0, -0.4):
        out = msp.smd_final_slices(case.sg(msp), dev(o), torch.tensor([lam], dtype=torch.float64, device="cuda"))
        ref = O.final_slices(slices_list(o), lam)
        assert rel(out.cpu().numpy().reshape(M, -1), np.stack(ref)) <= 1e-6


def test_algorithm_two_trajectory(msp):
    """Two iterations of Algorithm 2 (two matrix steps each) against the oracle's own run."""
    n, M = 16, 2
    case = Case(n, M, seed=51, dz=40.0)
    g = case.sg(msp)
    slices, lam, hm, hd = msp.sparse_decomposition(g, dev(case.probe), dev(case.shifts), dev(case.I),
                                                   iterations=2, matrix_steps=2)
    torch.cuda.synchronize()
    s_ref, lam_ref, hm_ref, hd_ref = O.sparse_decomposition(case.geom, case.probe.astype(np.complex128), case.shifts,
                                                            case.I.astype(np.float64), iterations=2, matrix_steps=2)
    np.testing.assert_allclose(hm.cpu().numpy(), hm_ref, rtol=1e-4)
    np.testing.assert_allclose(hd.cpu().numpy(), hd_ref, rtol=1e-4)
    assert lam.item() == pytest.approx(lam_ref, rel=1e-4)
    assert rel(slices.cpu().numpy().reshape(M, -1), np.stack(s_ref)) <= 1e-4
    assert hm_ref[-1] < hm_ref[0]


def test_null_and_misaligned_arguments_are_rejected_on_the_host(msp):
    import ctypes
    g = msp.smd_geometry(16, 2, 10, 0.025, 20.0, 0.28)
    ws = msp.smd_make_workspace(g)
    lib = msp.lib()
    A = torch.zeros((256, 256), dtype=torch.complex64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s = lib.msp_smd_matrix_step(ctypes.byref(g), None, None, None, None, 0.0, None, None, ws.ptr(), ws.nbytes, st)
    assert s == msp.MSP_EINVAL and b"A is NULL" in lib.msp_last_error_message()
    s = lib.msp_smd_transfer(ctypes.byref(g), ctypes.c_void_p(A.data_ptr() + 8), 1.0, ctypes.c_void_p(A.data_ptr()),
                             ws.ptr(), ws.nbytes, st)
    assert s == msp.MSP_EINVAL and b"aligned" in lib.msp_last_error_message()
    s = lib.msp_smd_decompose(ctypes.byref(g), ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(A.data_ptr()), None,
                              None, ws.ptr(), ws.nbytes, st)
    assert s == msp.MSP_EINVAL
    s = lib.msp_smd_transfer(ctypes.byref(g), ctypes.c_void_p(A.data_ptr()), 1.0, ctypes.c_void_p(A.data_ptr()),
                             ws.ptr(), 16, st)
    assert s == msp.MSP_EINVAL and b"workspace too small" in lib.msp_last_error_message()
