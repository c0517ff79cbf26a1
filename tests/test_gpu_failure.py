"""Failure detection of the tensor-core kernels, without a GPU fault.

Their mbarrier waits are bounded.  With the bound cut to one poll (msp_set_wait_limit),
the producers' first wait for the tensor core runs out: the kernel raises the workspace
flag, stops, waits for the MMAs it issued and frees its tensor memory.  The host reads
MSP_ETIMEOUT from msp_check_workspace, and the same process then runs correct calls again.
"""
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


def smd_inputs(msp, n=40, M=3):
    g = msp.smd_geometry(n=n, n_slices=M, n_pos=n * n, wavelength_A=0.02508, dz_A=20.0, pixel_A=0.2827)
    probe = torch.from_numpy(synth.random_complex((n, n), 1).astype(np.complex64)).cuda()
    shifts = torch.from_numpy(synth.cyclic_shifts(n)).cuda()
    I = torch.from_numpy((np.abs(synth.random_complex((n * n, n, n), 2)) ** 2).astype(np.float32)).cuda()
    A = torch.from_numpy((synth.random_complex((n * n, n * n), 3) / n).astype(np.complex64)).cuda()
    return g, probe, shifts, I, A


def test_a_wait_that_runs_out_is_reported_and_the_device_stays_usable(msp):
    g, probe, shifts, I, A0 = smd_inputs(msp)
    ws = msp.smd_make_workspace(g)
    timed_out = False
    try:
        msp.set_wait_limit(1)
        for _ in range(3):
            A = A0.clone()
            msp.smd_matrix_step(g, A, probe, shifts, I, ws=ws)
            try:
                msp.check_workspace(ws)
            except msp.MspError as e:
                assert e.status == msp.MSP_ETIMEOUT
                timed_out = True
                break
    finally:
        msp.set_wait_limit(0)
    assert timed_out
    # the context is intact: a normal call succeeds and is correct
    A = A0.clone()
    obj, mu = msp.smd_matrix_step(g, A, probe, shifts, I, ws=ws)
    msp.check_workspace(ws)
    n2 = g.n * g.n
    F = O.dft_matrix_2d(g.n)
    P = O.probe_matrix(probe.cpu().numpy().astype(np.complex128), shifts.cpu().numpy())
    Im = O.measurement_matrix(I.cpu().numpy().astype(np.float64))
    A_ref, _ = O.matrix_step(A0.cpu().numpy().T.astype(np.complex128), F, P, Im, mu.item())
    dA = A.cpu().numpy().T.astype(np.complex128) - A0.cpu().numpy().T
    d_ref = A_ref - A0.cpu().numpy().T
    assert np.linalg.norm(dA - d_ref) / np.linalg.norm(d_ref) < 1e-4
    x = torch.from_numpy(synth.random_complex((4, 64, 64), 5).astype(np.complex64)).cuda()
    y = msp.dft2_tc(x).cpu().numpy()
    ref = np.stack([O.dft2(v) for v in x.cpu().numpy().astype(np.complex128)])
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5


def test_split_bf16_dft_wait_that_runs_out_is_reported(msp):
    """The split-BF16 DFT passes wait for their own MMAs with the same bound: cut to one poll, a
    pass gives up, the call's workspace flag reads MSP_ETIMEOUT, and the same process then runs the
    mode correctly (its forward intensities against the oracle at the mode's bar)."""
    cfg = synth.C1
    pos = synth.scan_positions(cfg, sub=(2, 2))
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd, precision=msp.MSP_PRECISION_BF16X3_DFT)
    probe = synth.probe(cfg).astype(np.complex64)
    V = synth.potential_slices(cfg).astype(np.float32)
    dp, dV, dpos = (torch.from_numpy(probe).cuda(), torch.from_numpy(V).cuda(), torch.from_numpy(pos).cuda())
    ws = msp.make_workspace(g)
    timed_out = False
    try:
        msp.set_wait_limit(1)
        for _ in range(3):
            msp.forward(g, dp, dV, dpos, ws=ws)
            try:
                msp.check_workspace(ws)
            except msp.MspError as e:
                assert e.status == msp.MSP_ETIMEOUT
                timed_out = True
                break
    finally:
        msp.set_wait_limit(0)
    assert timed_out
    I = msp.forward(g, dp, dV, dpos, ws=ws).cpu().numpy()
    msp.check_workspace(ws)
    ref = O.forward(gd, probe.astype(np.complex128), pos, V=V.astype(np.float64))
    bar = 2 * 2 * (2 * cfg.n_slices - 1) * 2.0 ** -16
    assert np.linalg.norm(I - ref) / np.linalg.norm(ref) <= bar
