"""msp_forward_noalloc: the forward model for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a host application that owns all device memory
through its own pool, or a loop that must not allocate once running), so they cannot
provide the workspace msp_forward takes.  The no-allocation entry point keeps its scratch
in a fixed file-scope device array instead.  These checks call it through the C ABI and
compare it with msp_forward on the same inputs, two calls in a row with different
potentials (the shared scratch must not carry state from one call to the next).
"""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
from workloads import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("cfg,sub", [(synth.C2, (13, 13)), (synth.C1, None)])
def test_noalloc_forward_matches_msp_forward_on_two_calls(cfg, sub):
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp
    lib = msp.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pos = synth.scan_positions(cfg, sub=sub)
    gd = synth.geometry(cfg, n_pos=len(pos))
    g = msp.geometry(**gd)
    probe = torch.from_numpy(synth.probe(cfg).astype(np.complex64)).to(dev)
    V_true = synth.potential_slices(cfg)
    dpos = torch.from_numpy(pos).to(dev)
    werr = torch.full((1,), 7, dtype=torch.int32, device=dev)
    for scale in (1.0, 0.3):                      # two calls in a row, different inputs
        V = torch.from_numpy((scale * V_true).astype(np.float32)).to(dev)
        ref = msp.forward(g, probe, V, dpos)      # the existing entry point, with a workspace
        out = torch.full_like(ref, float("nan"))
        st = lib.msp_forward_noalloc(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(dpos), _ptr(out), _ptr(werr),
                                     stream)
        assert st == msp.MSP_OK, lib.msp_last_error_message()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= TOL
        assert werr.item() == 0


def test_noalloc_forward_w256_cluster_path_on_two_calls():
    """W = 256 runs each position on a four-CTA cluster; its forward mode must not touch the
    exit-wave stash or the loss buffers, which the no-allocation entry point does not have.
    Two slices of 320 x 320 (204,800 cells, inside the fixed scratch) on a 3 x 3 scan."""
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp
    lib = msp.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cfg = synth.C4
    obj, L = 320, 2
    pos = np.array([(y, x) for y in (0, 32, 64) for x in (0, 32, 64)], dtype=np.int32)
    gd = dict(synth.geometry(cfg, n_pos=len(pos)), n_slices=L, obj_ny=obj, obj_nx=obj)
    g = msp.geometry(**gd)
    probe = torch.from_numpy(synth.probe(cfg).astype(np.complex64)).to(dev)
    V_true = synth.potential_slices(cfg)[:L, :obj, :obj]
    dpos = torch.from_numpy(pos).to(dev)
    werr = torch.full((1,), 7, dtype=torch.int32, device=dev)
    for scale in (1.0, 0.3):
        V = torch.from_numpy(np.ascontiguousarray(scale * V_true).astype(np.float32)).to(dev)
        ref = msp.forward(g, probe, V, dpos)
        out = torch.full_like(ref, float("nan"))
        st = lib.msp_forward_noalloc(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(dpos), _ptr(out), _ptr(werr),
                                     stream)
        assert st == msp.MSP_OK, lib.msp_last_error_message()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) <= TOL
        assert werr.item() == 0


def test_noalloc_forward_limits_and_window_flag():
    __graft_entry__.build()
    from paper_2205_03902_gb300 import msp
    lib = msp.lib()
    dev = torch.device("cuda", 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cfg = synth.C1
    pos = synth.scan_positions(cfg, sub=(2, 2))
    gd = synth.geometry(cfg, n_pos=len(pos))
    probe = torch.from_numpy(synth.probe(cfg).astype(np.complex64)).to(dev)
    V = torch.from_numpy(synth.potential_slices(cfg).astype(np.float32)).to(dev)
    # beyond the fixed scratch: 16 slices of 640 x 640 cells
    big = msp.geometry(**dict(gd, n_slices=16, obj_ny=640, obj_nx=640))
    st = lib.msp_forward_noalloc(ctypes.byref(big), _ptr(probe), _ptr(V), None, None, None, stream)
    assert st == msp.MSP_EUNSUPPORTED
    assert b"16 MiB" in lib.msp_last_error_message()
    # a window outside the object is skipped (zero pattern) and reported
    bad = pos.copy()
    bad[1] = (cfg.obj - cfg.win + 3, 0)
    dpos = torch.from_numpy(bad).to(dev)
    g = msp.geometry(**gd)
    out = torch.full((len(pos), cfg.win, cfg.win), float("nan"), device=dev)
    werr = torch.zeros(1, dtype=torch.int32, device=dev)
    st = lib.msp_forward_noalloc(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(dpos), _ptr(out), _ptr(werr), stream)
    assert st == msp.MSP_OK
    torch.cuda.synchronize()
    assert werr.item() == 1
    assert torch.count_nonzero(out[1]) == 0
    ref = msp.forward(g, probe, V, torch.from_numpy(pos).to(dev))
    assert _rel(out[[0, 2, 3]], ref[[0, 2, 3]]) <= TOL
