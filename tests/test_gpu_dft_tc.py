"""Parity of the batched tensor-core 2-D DFT (include/msp_dft.h) with the oracle's DFT.

The oracle's Fourier operator is the unnormalised 2-D DFT (numpy's fft2, pinned in
tests/test_oracle_pins.py).  Tolerance: each of the two passes is a contraction of length W
on the tensor cores with tf32-split operands, whose error is at most 32 2^-24 (the measured
level, see tests/test_gpu_smd.py), plus the rounding of the DFT matrix to FP32; the bar is
max(1e-5, 4 * 32 * 2^-24) = 1e-5 relative L2.
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


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("W,S", [(32, 5), (64, 37), (128, 19), (256, 3)])
@pytest.mark.parametrize("inverse", [False, True])
def test_batched_dft_matches_the_oracle(msp, W, S, inverse):
    x = synth.random_complex((S, W, W), W + S).astype(np.complex64)
    y = msp.dft2_tc(torch.from_numpy(x).cuda(), inverse=inverse).cpu().numpy()
    xd = x.astype(np.complex128)
    ref = np.stack([O.dft2_adjoint(v) if inverse else O.dft2(v) for v in xd])
    assert rel(y, ref) <= 1e-5


def test_in_place_and_workspace_reuse(msp):
    W, S = 64, 8
    x = synth.random_complex((S, W, W), 3).astype(np.complex64)
    t = torch.from_numpy(x).cuda()
    msp.dft2_tc(t, out=t)
    assert rel(t.cpu().numpy(), np.stack([O.dft2(v) for v in x.astype(np.complex128)])) <= 1e-5


def test_unsupported_sizes_are_rejected(msp):
    assert msp.lib().msp_dft2_tc_workspace_bytes(48, 4) == 0
    assert msp.lib().msp_dft2_tc_workspace_bytes(128, 0) == 0
    with pytest.raises(msp.MspError):
        msp.dft2_tc(torch.zeros((2, 48, 48), dtype=torch.complex64, device="cuda"))
