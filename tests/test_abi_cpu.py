"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol `include/msp.h` declares, and rejects bad arguments on the host
before anything is launched."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2205_03902_gb300 import msp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return msp.lib()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(msp_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["msp_forward", "msp_loss_grad", "msp_layer_step", "msp_probe_step", "msp_workspace_bytes",
                 "msp_smd_transfer", "msp_smd_matrix_step", "msp_smd_decompose", "msp_smd_final_slices",
                 "msp_smd_workspace_bytes"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def geom(**kw):
    base = dict(n_slices=4, obj_ny=384, obj_nx=384, win=128, n_pos=16, wavelength_A=0.06979,
                sigma=1.5433e-3, dz_A=2.0, pixel_A=0.15)
    base.update(kw)
    return msp.geometry(**base)


@pytest.mark.parametrize("kw,status", [
    ({}, msp.MSP_OK),
    (dict(win=64, obj_ny=96, obj_nx=96), msp.MSP_OK),
    (dict(win=96), msp.MSP_EUNSUPPORTED),
    (dict(win=256, obj_ny=640, obj_nx=640), msp.MSP_OK),
    (dict(win=512, obj_ny=640, obj_nx=640), msp.MSP_EUNSUPPORTED),
    (dict(param=msp.MSP_PARAM_TRANSMISSION), msp.MSP_OK),
    (dict(param=7), msp.MSP_EINVAL),
    (dict(n_slices=0), msp.MSP_EINVAL),
    (dict(obj_ny=100), msp.MSP_EINVAL),
    (dict(n_pos=-1), msp.MSP_EINVAL),
    (dict(wavelength_A=0.0), msp.MSP_EINVAL),
    (dict(pixel_A=-1.0), msp.MSP_EINVAL),
    (dict(dz_A=float("nan")), msp.MSP_EINVAL),
    (dict(sigma=float("inf")), msp.MSP_EINVAL),
])
def test_geometry_validation(lib, kw, status):
    assert msp.validate_geometry(geom(**kw)) == status


def test_null_geometry_and_status_strings(lib):
    assert lib.msp_validate_geometry(None) == msp.MSP_EINVAL
    assert b"NULL" in lib.msp_last_error_message()
    for s, name in enumerate(["MSP_OK", "MSP_EINVAL", "MSP_ENOMEM", "MSP_ECUDA", "MSP_EUNSUPPORTED", "MSP_ETIMEOUT",
                              "MSP_EDEVICE"]):
        assert msp.status_string(s) == name
    assert msp.status_string(99) == "MSP_UNKNOWN"


def test_compute_calls_reject_bad_geometry_before_touching_the_device(lib):
    g = geom(win=32)
    st = lib.msp_forward(ctypes.byref(g), None, None, None, None, None, 0, None)
    assert st == msp.MSP_EUNSUPPORTED
    g = geom(n_slices=0)
    st = lib.msp_loss_grad(ctypes.byref(g), None, None, None, None, None, None, None, None, 0, None)
    assert st == msp.MSP_EINVAL
    assert lib.msp_workspace_bytes(ctypes.byref(g)) == 0


def smd_geom(**kw):
    base = dict(n=40, n_slices=3, n_pos=1600, wavelength_A=0.02508, dz_A=20.0, pixel_A=0.2827)
    base.update(kw)
    return msp.smd_geometry(**base)


@pytest.mark.parametrize("kw,status", [
    ({}, msp.MSP_OK),
    (dict(n=16, n_pos=1), msp.MSP_OK),
    (dict(n=64, n_slices=3), msp.MSP_OK),
    (dict(n=64, n_slices=4), msp.MSP_EUNSUPPORTED),
    (dict(n=48, n_slices=5), msp.MSP_OK),
    (dict(n=48, n_slices=6), msp.MSP_EUNSUPPORTED),
    (dict(n=36), msp.MSP_EUNSUPPORTED),
    (dict(n=128), msp.MSP_EUNSUPPORTED),
    (dict(n_slices=0), msp.MSP_EINVAL),
    (dict(n_pos=0), msp.MSP_EINVAL),
    (dict(wavelength_A=-1.0), msp.MSP_EINVAL),
    (dict(pixel_A=float("nan")), msp.MSP_EINVAL),
    (dict(dz_A=-2.0), msp.MSP_EINVAL),
    (dict(dz_A=0.0), msp.MSP_OK),
])
def test_smd_geometry_validation(lib, kw, status):
    assert msp.smd_validate_geometry(smd_geom(**kw)) == status


def test_smd_calls_reject_bad_geometry_before_touching_the_device(lib):
    g = smd_geom(n=36)
    assert lib.msp_smd_transfer(ctypes.byref(g), None, 1.0, None, None, 0, None) == msp.MSP_EUNSUPPORTED
    g = smd_geom(n_slices=0)
    assert lib.msp_smd_decompose(ctypes.byref(g), None, None, None, None, None, 0, None) == msp.MSP_EINVAL
    assert lib.msp_smd_final_slices(ctypes.byref(g), None, None, None, None) == msp.MSP_EINVAL
    assert lib.msp_smd_workspace_bytes(ctypes.byref(g)) == 0
    assert lib.msp_smd_validate_geometry(None) == msp.MSP_EINVAL


@pytest.mark.parametrize("W,S,ok", [(32, 1, True), (64, 37, True), (128, 4096, True), (256, 3, True),
                                    (48, 4, False), (512, 1, False), (128, 0, False), (128, 70000, False)])
def test_dft_workspace_sizes_and_host_validation(lib, W, S, ok):
    n = lib.msp_dft2_tc_workspace_bytes(W, S)
    if ok:
        # error word, the DFT matrix and the intermediate batch, each 256-byte aligned
        assert n >= W * W * 8 + S * W * W * 8
    else:
        assert n == 0
        assert lib.msp_dft2_tc(W, S, 0, None, None, None, 0, None) == msp.MSP_EUNSUPPORTED


def test_reconstruct_history_length_and_plan_validation(lib):
    g = geom()
    pl = msp.plan(50, steps_per_layer=1, probe_steps=1)
    assert lib.msp_reconstruct_history_length(ctypes.byref(g), ctypes.byref(pl)) == 50 * (4 + 1) + 1
    pl = msp.plan(3, steps_per_layer=2)
    assert lib.msp_reconstruct_history_length(ctypes.byref(g), ctypes.byref(pl)) == 3 * 8 + 1
    pl = msp.plan(0)
    assert lib.msp_reconstruct_history_length(ctypes.byref(g), ctypes.byref(pl)) == 1
    for bad in (msp.plan(-1), msp.plan(2, steps_per_layer=-1), msp.plan(2, probe_steps=-3),
                msp.plan(2, layer_step=float("nan"))):
        assert lib.msp_reconstruct_history_length(ctypes.byref(g), ctypes.byref(bad)) == 0
        st = lib.msp_reconstruct(ctypes.byref(g), ctypes.byref(bad), None, None, None, None, None, None, 0, None)
        assert st == msp.MSP_EINVAL
    assert lib.msp_reconstruct_history_length(ctypes.byref(g), None) == 0
    assert lib.msp_reconstruct(ctypes.byref(g), None, None, None, None, None, None, None, 0, None) == msp.MSP_EINVAL
    assert b"plan" in lib.msp_last_error_message()


def test_wait_limit_hook_needs_no_device(lib):
    assert lib.msp_set_wait_limit(5) == msp.MSP_OK
    assert lib.msp_set_wait_limit(0) == msp.MSP_OK


def test_overlap_add_switch(lib):
    assert lib.msp_set_overlap_add(msp.OVERLAP_L2_REDUCE) == msp.MSP_OK
    assert lib.msp_set_overlap_add(msp.OVERLAP_FIXED_ORDER) == msp.MSP_OK
    for bad in (-1, 2, 1 << 30):
        assert lib.msp_set_overlap_add(bad) == msp.MSP_EINVAL
    assert b"overlap" in lib.msp_last_error_message()


# ---- learned proposal (include/msp_learn.h) ----------------------------------------------------
@pytest.mark.parametrize("kw,status", [
    ({}, msp.MSP_OK),
    (dict(n_slices=8, height=1, width=128), msp.MSP_OK),
    (dict(n_slices=0), msp.MSP_EUNSUPPORTED),
    (dict(n_slices=9), msp.MSP_EUNSUPPORTED),
    (dict(width=200), msp.MSP_EUNSUPPORTED),
    (dict(width=0), msp.MSP_EUNSUPPORTED),
    (dict(height=0), msp.MSP_EUNSUPPORTED),
    (dict(height=70000), msp.MSP_EUNSUPPORTED),
    (dict(scale_v=0.0), msp.MSP_EINVAL),
    (dict(scale_d=float("nan")), msp.MSP_EINVAL),
])
def test_net_shape_validation(lib, kw, status):
    base = dict(n_slices=4, height=384, width=384, scale_v=1.0, scale_g=1.0, scale_d=1.0)
    base.update(kw)
    assert msp.net_validate(msp.net_shape(**base)) == status


def test_net_parameter_count_matches_the_layer_list(lib):
    from oracle import proposal_oracle as P
    for L in (1, 2, 4, 8):
        assert msp.net_param_count(msp.net_shape(L, 128, 128)) == P.param_count(L)
    assert lib.msp_net_param_count(None) == 0
    assert lib.msp_net_workspace_bytes(ctypes.byref(msp.net_shape(4, 128, 100))) == 0
    assert lib.msp_net_workspace_bytes(ctypes.byref(msp.net_shape(4, 384, 384))) > 0


def test_net_calls_reject_bad_arguments_before_any_launch(lib):
    s = msp.net_shape(4, 128, 128)
    n = lib.msp_net_workspace_bytes(ctypes.byref(s))
    assert lib.msp_net_forward(ctypes.byref(s), None, None, None, None, None, n, None) != msp.MSP_OK
    bad = msp.net_shape(4, 128, 120)
    assert lib.msp_net_forward(ctypes.byref(bad), None, None, None, None, None, 0, None) == msp.MSP_EUNSUPPORTED
    assert lib.msp_net_train_step(ctypes.byref(bad), None, None, None, 1, 1e-3, None, None, None, None, None, 0,
                                  None) == msp.MSP_EUNSUPPORTED
    for args in [(4, 128, 16, 64), (4, 130, 16, 64), (4, 128, 32, 64), (0, 128, 16, 16), (4, 128, 64, 8)]:
        want = 0 if args[1] % 128 or args[2] not in (16, 64) or args[3] not in (16, 64) or args[0] < 1 else 1
        got = lib.msp_conv3x3_test_workspace_bytes(*args)
        assert (got > 0) == bool(want), args
    assert lib.msp_conv3x3_test(4, 130, 16, 64, None, None, None, None, None, 0, None) == msp.MSP_EUNSUPPORTED
