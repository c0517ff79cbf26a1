"""Python binding of libmsp (ctypes).  Argument marshalling only.

Every entry point takes CUDA tensors, checks their dtype / shape / device,
hands raw device pointers and the current stream to the C ABI declared in
`include/msp.h`, and raises `MspError` on a non-zero status.  All arithmetic
runs in the library's kernels; there is no fallback of any kind: without the
built `lib/libmsp.so` every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmsp.so")

MSP_OK, MSP_EINVAL, MSP_ENOMEM, MSP_ECUDA, MSP_EUNSUPPORTED, MSP_ETIMEOUT, MSP_EDEVICE = range(7)
MSP_PARAM_POTENTIAL, MSP_PARAM_TRANSMISSION = 0, 1
MSP_PRECISION_FP32, MSP_PRECISION_FP64_FORWARD, MSP_PRECISION_BF16X3_DFT, MSP_PRECISION_DF_FORWARD = 0, 1, 2, 3


class MspError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class Geometry(ctypes.Structure):
    """msp_geometry (include/msp.h): the statement of the problem, Sec. 2.1."""
    _fields_ = [
        ("n_slices", ctypes.c_int32),
        ("obj_ny", ctypes.c_int32),
        ("obj_nx", ctypes.c_int32),
        ("win", ctypes.c_int32),
        ("n_pos", ctypes.c_int32),
        ("param", ctypes.c_int32),
        ("wavelength_A", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("dz_A", ctypes.c_double),
        ("pixel_A", ctypes.c_double),
        ("precision", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def geometry(n_slices, obj_ny, obj_nx, win, n_pos, wavelength_A, sigma, dz_A, pixel_A,
             param=MSP_PARAM_POTENTIAL, precision=MSP_PRECISION_FP32, **_ignored) -> Geometry:
    return Geometry(int(n_slices), int(obj_ny), int(obj_nx), int(win), int(n_pos), int(param),
                    float(wavelength_A), float(sigma), float(dz_A), float(pixel_A), int(precision))


class SmdGeometry(ctypes.Structure):
    """msp_smd_geometry (include/msp_smd.h): Algorithm 2 on the N x N full-field model (Sec. 3.4)."""
    _fields_ = [
        ("n", ctypes.c_int32),
        ("n_slices", ctypes.c_int32),
        ("n_pos", ctypes.c_int32),
        ("wavelength_A", ctypes.c_double),
        ("dz_A", ctypes.c_double),
        ("pixel_A", ctypes.c_double),
    ]


class Plan(ctypes.Structure):
    """msp_plan (include/msp.h): Algorithm 1 (Sec. 3.3) with optional probe steps (Sec. 3.5)."""
    _fields_ = [
        ("sweeps", ctypes.c_int32),
        ("steps_per_layer", ctypes.c_int32),
        ("probe_steps", ctypes.c_int32),
        ("normalize_probe", ctypes.c_int32),
        ("layer_step", ctypes.c_double),
        ("probe_step", ctypes.c_double),
    ]


def plan(sweeps, steps_per_layer=1, probe_steps=0, normalize_probe=False, layer_step=0.0, probe_step=0.0) -> Plan:
    return Plan(int(sweeps), int(steps_per_layer), int(probe_steps), 1 if normalize_probe else 0,
                float(layer_step), float(probe_step))


def smd_geometry(n, n_slices, n_pos, wavelength_A, dz_A, pixel_A, **_ignored) -> SmdGeometry:
    return SmdGeometry(int(n), int(n_slices), int(n_pos), float(wavelength_A), float(dz_A), float(pixel_A))


class NetShape(ctypes.Structure):
    """msp_net_shape of include/msp_learn.h."""
    _fields_ = [
        ("n_slices", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("scale_v", ctypes.c_double),
        ("scale_g", ctypes.c_double),
        ("scale_d", ctypes.c_double),
    ]


def net_shape(n_slices, height, width, scale_v=1.0, scale_g=1.0, scale_d=1.0) -> NetShape:
    return NetShape(int(n_slices), int(height), int(width), float(scale_v), float(scale_g), float(scale_d))


_lib = None
_P = ctypes.c_void_p
_G = ctypes.POINTER(Geometry)
_GS = ctypes.POINTER(SmdGeometry)
_SIGS = {
    "msp_validate_geometry": ([_G], ctypes.c_int),
    "msp_workspace_bytes": ([_G], ctypes.c_size_t),
    "msp_forward": ([_G, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_loss_grad": ([_G, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_layer_step": ([_G, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double, _P, _P, _P, ctypes.c_size_t, _P],
                       ctypes.c_int),
    "msp_probe_step": ([_G, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P],
                       ctypes.c_int),
    "msp_reconstruct_history_length": ([_G, ctypes.POINTER(Plan)], ctypes.c_size_t),
    "msp_reconstruct": ([_G, ctypes.POINTER(Plan), _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_check_workspace": ([_P, _P], ctypes.c_int),
    "msp_forward_noalloc": ([_G, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "msp_profile_enable": ([ctypes.c_int32], ctypes.c_int),
    "msp_set_wait_limit": ([ctypes.c_int32], ctypes.c_int),
    "msp_set_overlap_add": ([ctypes.c_int32], ctypes.c_int),
    "msp_profile_read": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int32], ctypes.c_int),
    "msp_smd_validate_geometry": ([_GS], ctypes.c_int),
    "msp_smd_workspace_bytes": ([_GS], ctypes.c_size_t),
    "msp_smd_transfer": ([_GS, _P, ctypes.c_double, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_smd_matrix_step": ([_GS, _P, _P, _P, _P, ctypes.c_double, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_smd_decompose": ([_GS, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_smd_final_slices": ([_GS, _P, _P, _P, _P], ctypes.c_int),
    "msp_dft2_tc_workspace_bytes": ([ctypes.c_int32, ctypes.c_int32], ctypes.c_size_t),
    "msp_dft2_tc": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_net_validate": ([ctypes.POINTER(NetShape)], ctypes.c_int),
    "msp_net_param_count": ([ctypes.POINTER(NetShape)], ctypes.c_size_t),
    "msp_net_workspace_bytes": ([ctypes.POINTER(NetShape)], ctypes.c_size_t),
    "msp_net_init": ([ctypes.POINTER(NetShape), _P, ctypes.c_uint64, _P], ctypes.c_int),
    "msp_net_forward": ([ctypes.POINTER(NetShape), _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_net_loss_grad": ([ctypes.POINTER(NetShape), _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_net_train_step": ([ctypes.POINTER(NetShape), _P, _P, _P, ctypes.c_int32, ctypes.c_double, _P, _P, _P, _P, _P,
                            ctypes.c_size_t, _P], ctypes.c_int),
    "msp_learned_workspace_bytes": ([_G, ctypes.POINTER(NetShape)], ctypes.c_size_t),
    "msp_learned_propose": ([_G, ctypes.POINTER(NetShape), _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P,
                             ctypes.c_size_t, _P], ctypes.c_int),
    "msp_conv3x3_test": ([ctypes.c_int32] * 4 + [_P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_conv3x3_wgrad_test": ([ctypes.c_int32] * 4 + [_P, _P, _P, _P, _P, ctypes.c_size_t, _P], ctypes.c_int),
    "msp_conv3x3_test_workspace_bytes": ([ctypes.c_int32] * 4, ctypes.c_size_t),
    "msp_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "msp_last_error_message": ([], ctypes.c_char_p),
}


def lib() -> ctypes.CDLL:
    """The loaded libmsp; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmsp is not built ({LIB_PATH} missing): run paper_2205_03902_gb300/build.py")
        dll = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(dll, name)
            fn.argtypes = args
            fn.restype = res
        _lib = dll
    return _lib


def _check(status: int, where: str) -> None:
    if status != MSP_OK:
        l = lib()
        detail = l.msp_last_error_message().decode() or l.msp_status_string(status).decode()
        raise MspError(status, where, detail)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, name, dtype, shape, device):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.device != device:
        raise ValueError(f"{name} must live on {device}, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def workspace_bytes(g: Geometry) -> int:
    n = lib().msp_workspace_bytes(ctypes.byref(g))
    if n == 0:
        _check(lib().msp_validate_geometry(ctypes.byref(g)), "msp_workspace_bytes")
        raise MspError(MSP_ECUDA, "msp_workspace_bytes", "no CUDA device")
    return int(n)


@dataclass
class Workspace:
    """Caller-owned scratch for one call at a time (allocated through torch)."""
    buf: torch.Tensor

    @property
    def nbytes(self) -> int:
        return self.buf.numel()

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())


def make_workspace(g: Geometry, device=None) -> Workspace:
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = workspace_bytes(g)
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return Workspace(buf[off:off + n])


def _ws(g, ws, device):
    if ws is None:
        return make_workspace(g, device)
    if ws.nbytes < workspace_bytes(g):
        raise ValueError("workspace too small for this geometry")
    return ws


def _arrays(g: Geometry, probe, V, pos, I=None, I_name="I_meas"):
    device = V.device
    W, L, Ny, Nx, S = g.win, g.n_slices, g.obj_ny, g.obj_nx, g.n_pos
    _need(probe, "probe", torch.complex64, (W, W), device)
    cplx = g.param == MSP_PARAM_TRANSMISSION   # complex slices o_m instead of potentials
    _need(V, "V", torch.complex64 if cplx else torch.float32, (L, Ny, Nx), device)
    _need(pos, "pos", torch.int32, (S, 2), device)
    if I is not None:
        _need(I, I_name, torch.float32, (S, W, W), device)
    return device


def forward(g: Geometry, probe, V, pos, out=None, ws=None, stream=None):
    """Far-field intensities [S][W][W] (msp_forward)."""
    device = _arrays(g, probe, V, pos)
    if out is None:
        out = torch.empty((g.n_pos, g.win, g.win), dtype=torch.float32, device=device)
    _arrays(g, probe, V, pos, out, "out")
    ws = _ws(g, ws, device)
    _check(lib().msp_forward(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(pos), _ptr(out), ws.ptr(), ws.nbytes,
                             _stream(stream)), "msp_forward")
    return out


def forward_noalloc(g: Geometry, probe, V, pos, out, window_error=None, stream=None):
    """msp_forward without a workspace: for callers that cannot allocate device memory.
    `out` (and the optional int32 `window_error`) must be supplied by the caller."""
    _arrays(g, probe, V, pos)
    _arrays(g, probe, V, pos, out, "out")
    _check(lib().msp_forward_noalloc(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(pos), _ptr(out),
                                     _ptr(window_error), _stream(stream)), "msp_forward_noalloc")
    return out


def loss_grad(g: Geometry, probe, V, pos, I_meas, want_dV=True, want_dprobe=True, ws=None, stream=None,
              loss=None, dV=None, dprobe=None):
    """(loss [1] float64, dV [L][Ny][Nx] or None, dprobe [W][W] complex64 or None) (msp_loss_grad)."""
    device = _arrays(g, probe, V, pos, I_meas)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=device)
    if want_dV and dV is None:
        dV = torch.empty_like(V)
    if want_dprobe and dprobe is None:
        dprobe = torch.empty_like(probe)
    ws = _ws(g, ws, device)
    _check(lib().msp_loss_grad(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(pos), _ptr(I_meas), _ptr(loss),
                               _ptr(dV if want_dV else None), _ptr(dprobe if want_dprobe else None), ws.ptr(),
                               ws.nbytes, _stream(stream)), "msp_loss_grad")
    return loss, (dV if want_dV else None), (dprobe if want_dprobe else None)


def layer_step(g: Geometry, probe, V, pos, I_meas, layer: int, step: float = 0.0, ws=None, stream=None,
               loss_before=None, mu=None):
    """One Algorithm-1 gradient step on slice `layer`, V updated in place; returns (loss_before, mu)."""
    device = _arrays(g, probe, V, pos, I_meas)
    if loss_before is None:
        loss_before = torch.empty(1, dtype=torch.float64, device=device)
    if mu is None:
        mu = torch.empty(1, dtype=torch.float64, device=device)
    ws = _ws(g, ws, device)
    _check(lib().msp_layer_step(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(pos), _ptr(I_meas), int(layer),
                                float(step), _ptr(loss_before), _ptr(mu), ws.ptr(), ws.nbytes, _stream(stream)),
           "msp_layer_step")
    return loss_before, mu


def probe_step(g: Geometry, probe, V, pos, I_meas, step: float = 0.0, normalize: bool = False, ws=None,
               stream=None, loss_before=None, mu=None):
    """One amplitude-flow step on the probe, updated in place; returns (loss_before, mu)."""
    device = _arrays(g, probe, V, pos, I_meas)
    if loss_before is None:
        loss_before = torch.empty(1, dtype=torch.float64, device=device)
    if mu is None:
        mu = torch.empty(1, dtype=torch.float64, device=device)
    ws = _ws(g, ws, device)
    _check(lib().msp_probe_step(ctypes.byref(g), _ptr(probe), _ptr(V), _ptr(pos), _ptr(I_meas), float(step),
                                1 if normalize else 0, _ptr(loss_before), _ptr(mu), ws.ptr(), ws.nbytes,
                                _stream(stream)), "msp_probe_step")
    return loss_before, mu


def reconstruct(g: Geometry, pl: Plan, probe, V, pos, I_meas, ws=None, stream=None, history=None):
    """The plain method (msp_reconstruct): `pl.sweeps` iterations of Algorithm 1 with optional probe
    steps; probe and V are updated in place.  Returns the loss history (float64, on the device):
    the loss before every step in order, then the loss after the last step."""
    device = _arrays(g, probe, V, pos, I_meas)
    n = int(lib().msp_reconstruct_history_length(ctypes.byref(g), ctypes.byref(pl)))
    if n == 0:
        _check(lib().msp_validate_geometry(ctypes.byref(g)), "msp_reconstruct")
        raise MspError(MSP_EINVAL, "msp_reconstruct", "invalid plan")
    if history is None:
        history = torch.empty(n, dtype=torch.float64, device=device)
    elif history.numel() < n or history.dtype != torch.float64 or history.device != device:
        raise ValueError(f"history must be a float64 tensor of at least {n} entries on {device}")
    ws = _ws(g, ws, device)
    _check(lib().msp_reconstruct(ctypes.byref(g), ctypes.byref(pl), _ptr(probe), _ptr(V), _ptr(pos), _ptr(I_meas),
                                 _ptr(history), ws.ptr(), ws.nbytes, _stream(stream)), "msp_reconstruct")
    return history[:n]


def check_workspace(ws: Workspace, stream=None) -> None:
    """Raises MspError(MSP_EINVAL) if the last call on `ws` skipped a window outside the object."""
    _check(lib().msp_check_workspace(ws.ptr(), _stream(stream)), "msp_check_workspace")


def set_wait_limit(polls: int = 0) -> None:
    """Poll bound of the tensor-core kernels' waits (0: the default, < 0: no poll at all); a test hook
    for failure detection."""
    _check(lib().msp_set_wait_limit(int(polls)), "msp_set_wait_limit")


OVERLAP_FIXED_ORDER, OVERLAP_L2_REDUCE = 0, 1


def set_overlap_add(mode: int = OVERLAP_FIXED_ORDER) -> None:
    """How loss_grad and layer_step (so also reconstruct) sum the per-position windows into the
    object-frame maps: OVERLAP_FIXED_ORDER (a gather in scan order, bit-reproducible; the
    default) or OVERLAP_L2_REDUCE (reductions in L2 from the fused kernel, no gather;
    reproducible to rounding).  FP32 mode only; process-wide."""
    _check(lib().msp_set_overlap_add(int(mode)), "msp_set_overlap_add")


def profile_enable(on: bool = True) -> None:
    """Bracket every fused-kernel launch with CUDA events on its stream."""
    _check(lib().msp_profile_enable(1 if on else 0), "msp_profile_enable")


def profile_read(reset: bool = True) -> dict:
    """{'fused_ms', 'fused_launches', 'all_launches'} since the last reset (waits for the events)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    total = ctypes.c_int64(0)
    _check(lib().msp_profile_read(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(total), 1 if reset else 0),
           "msp_profile_read")
    return {"fused_ms": ms.value, "fused_launches": n.value, "all_launches": total.value}


def validate_geometry(g: Geometry) -> int:
    return int(lib().msp_validate_geometry(ctypes.byref(g)))


def status_string(status: int) -> str:
    return lib().msp_status_string(int(status)).decode()


# ---------------------------------------------------------------------------
# Algorithm 2, Sparse Matrix Decomposition (include/msp_smd.h)
# ---------------------------------------------------------------------------

def smd_validate_geometry(g: SmdGeometry) -> int:
    return int(lib().msp_smd_validate_geometry(ctypes.byref(g)))


def smd_make_workspace(g: SmdGeometry, device=None) -> Workspace:
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = int(lib().msp_smd_workspace_bytes(ctypes.byref(g)))
    if n == 0:
        _check(lib().msp_smd_validate_geometry(ctypes.byref(g)), "msp_smd_workspace_bytes")
        raise MspError(MSP_ECUDA, "msp_smd_workspace_bytes", "no CUDA device")
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return Workspace(buf[off:off + n])


def _smd_ws(g, ws, device):
    return smd_make_workspace(g, device) if ws is None else ws


def _smd_slices(g: SmdGeometry, o, name="o"):
    _need(o, name, torch.complex64, (g.n_slices, g.n, g.n), o.device)


def _smd_matrix(g: SmdGeometry, A, device):
    n2 = g.n * g.n
    _need(A, "A", torch.complex64, (n2, n2), device)   # A[j] is column j of the N^2 x N^2 matrix


def smd_transfer(g: SmdGeometry, o, lam: float = 1.0, A=None, ws=None, stream=None):
    """lambda * O_M prod G O_m as an [N^2][N^2] complex64 tensor whose row j is column j of the
    matrix (the exit wave of an impulse at pixel j) (msp_smd_transfer)."""
    _smd_slices(g, o)
    n2 = g.n * g.n
    if A is None:
        A = torch.empty((n2, n2), dtype=torch.complex64, device=o.device)
    _smd_matrix(g, A, o.device)
    ws = _smd_ws(g, ws, o.device)
    _check(lib().msp_smd_transfer(ctypes.byref(g), _ptr(o), float(lam), _ptr(A), ws.ptr(), ws.nbytes,
                                  _stream(stream)), "msp_smd_transfer")
    return A


def smd_matrix_step(g: SmdGeometry, A, probe, shifts, I, step: float = 0.0, ws=None, stream=None,
                    objective=None, mu=None):
    """One gradient step of Eq. (Opt_Prob_Matrix) on A in place; returns (objective_before, mu)."""
    device = A.device
    _smd_matrix(g, A, device)
    _need(probe, "probe", torch.complex64, (g.n, g.n), device)
    _need(shifts, "shifts", torch.int32, (g.n_pos, 2), device)
    _need(I, "I", torch.float32, (g.n_pos, g.n, g.n), device)
    if objective is None:
        objective = torch.empty(1, dtype=torch.float64, device=device)
    if mu is None:
        mu = torch.empty(1, dtype=torch.float64, device=device)
    ws = _smd_ws(g, ws, device)
    _check(lib().msp_smd_matrix_step(ctypes.byref(g), _ptr(A), _ptr(probe), _ptr(shifts), _ptr(I), float(step),
                                     _ptr(objective), _ptr(mu), ws.ptr(), ws.nbytes, _stream(stream)),
           "msp_smd_matrix_step")
    return objective, mu


def smd_decompose(g: SmdGeometry, A, o, lam, ws=None, stream=None, objective=None):
    """Proximal slice updates, lambda update and A = lambda A(o) (Algorithm 2); A, o and the
    float64 [1] tensor lam are updated in place; returns the decomposition objective before."""
    device = A.device
    _smd_matrix(g, A, device)
    _smd_slices(g, o)
    _need(lam, "lam", torch.float64, (1,), device)
    if objective is None:
        objective = torch.empty(1, dtype=torch.float64, device=device)
    ws = _smd_ws(g, ws, device)
    _check(lib().msp_smd_decompose(ctypes.byref(g), _ptr(A), _ptr(o), _ptr(lam), _ptr(objective), ws.ptr(),
                                   ws.nbytes, _stream(stream)), "msp_smd_decompose")
    return objective


def smd_final_slices(g: SmdGeometry, o, lam, out=None, stream=None):
    """lambda^(1/M) o_m (msp_smd_final_slices)."""
    _smd_slices(g, o)
    _need(lam, "lam", torch.float64, (1,), o.device)
    if out is None:
        out = torch.empty_like(o)
    _check(lib().msp_smd_final_slices(ctypes.byref(g), _ptr(o), _ptr(lam), _ptr(out), _stream(stream)),
           "msp_smd_final_slices")
    return out


def sparse_decomposition(g: SmdGeometry, probe, shifts, I, iterations: int, matrix_steps: int = 1, o0=None,
                         ws=None, stream=None):
    """Algorithm 2 from slices o0 (default all ones) and lambda = 1.  Returns
    (slices lambda^(1/M) o_m, lambda [1] float64, matrix objectives [iterations*matrix_steps],
    decomposition objectives [iterations]) -- all on the device."""
    device = probe.device
    o = torch.ones((g.n_slices, g.n, g.n), dtype=torch.complex64, device=device) if o0 is None else o0.clone()
    lam = torch.ones(1, dtype=torch.float64, device=device)
    ws = _smd_ws(g, ws, device)
    A = smd_transfer(g, o, 1.0, ws=ws, stream=stream)
    hm = torch.empty(iterations * matrix_steps, dtype=torch.float64, device=device)
    hd = torch.empty(iterations, dtype=torch.float64, device=device)
    for t in range(iterations):
        for k in range(matrix_steps):
            smd_matrix_step(g, A, probe, shifts, I, ws=ws, stream=stream, objective=hm[t * matrix_steps + k:][:1])
        smd_decompose(g, A, o, lam, ws=ws, stream=stream, objective=hd[t:][:1])
    return smd_final_slices(g, o, lam, stream=stream), lam, hm, hd


# ---------------------------------------------------------------------------
# Batched 2-D DFT on the tensor cores (include/msp_dft.h)
# ---------------------------------------------------------------------------

def dft2_tc(x, inverse: bool = False, out=None, ws=None, stream=None):
    """F x_s F for a batch x [S][W][W] complex64 (inverse: the conjugate kernel, unnormalised),
    as two tensor-core contractions (msp_dft2_tc)."""
    if not isinstance(x, torch.Tensor) or x.dim() != 3 or x.shape[1] != x.shape[2]:
        raise ValueError("x must be a [S][W][W] tensor")
    S, W = int(x.shape[0]), int(x.shape[1])
    _need(x, "x", torch.complex64, (S, W, W), x.device)
    if out is None:
        out = torch.empty_like(x)
    _need(out, "out", torch.complex64, (S, W, W), x.device)
    n = int(lib().msp_dft2_tc_workspace_bytes(W, S))
    if n == 0:
        raise MspError(MSP_EUNSUPPORTED, "msp_dft2_tc", f"W = {W}, S = {S} not supported")
    if ws is None or ws.nbytes < n:
        buf = torch.empty(n + 256, dtype=torch.uint8, device=x.device)
        off = (-buf.data_ptr()) % 256
        ws = Workspace(buf[off:off + n])
    _check(lib().msp_dft2_tc(W, S, 1 if inverse else 0, _ptr(x), _ptr(out), ws.ptr(), ws.nbytes, _stream(stream)),
           "msp_dft2_tc")
    return out


class MultisliceLoss(torch.autograd.Function):
    """The amplitude-flow loss of the multislice model as a differentiable function of the
    slice potentials V (real) and the probe (complex), computed by msp_loss_grad in one fused
    forward + adjoint pass: the gradients are produced together with the loss and returned
    by `backward` (scaled by the incoming gradient of the loss).

    PyTorch's gradient of a real function of a complex tensor is the conjugate Wirtinger
    derivative times two; the library returns dL/dconj(P), so the probe gradient is 2 dprobe.
    """

    @staticmethod
    def forward(ctx, V, probe, geom, pos, I_meas, ws):
        loss, dV, dprobe = loss_grad(geom, probe.detach(), V.detach(), pos, I_meas,
                                     want_dV=V.requires_grad, want_dprobe=probe.requires_grad, ws=ws)
        ctx.save_for_backward(*(t for t in (dV, dprobe) if t is not None))
        ctx.has = (dV is not None, dprobe is not None)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_loss):
        saved = list(ctx.saved_tensors)
        dV = saved.pop(0) if ctx.has[0] else None
        dprobe = saved.pop(0) if ctx.has[1] else None
        gV = None if dV is None else dV * grad_loss.to(dV.dtype)
        gp = None if dprobe is None else dprobe * (2.0 * grad_loss.to(torch.float32))
        return gV, gp, None, None, None, None


def multislice_loss(geom: Geometry, V, probe, pos, I_meas, ws=None):
    """Differentiable loss L(V, probe) (float64 scalar tensor); see MultisliceLoss."""
    return MultisliceLoss.apply(V, probe, geom, pos, I_meas, _ws(geom, ws, V.device))


# ---------------------------------------------------------------------------------------------
# learned proposal (include/msp_learn.h)
# ---------------------------------------------------------------------------------------------
def net_validate(s: NetShape) -> int:
    return lib().msp_net_validate(ctypes.byref(s))


def net_param_count(s: NetShape) -> int:
    n = lib().msp_net_param_count(ctypes.byref(s))
    if n == 0:
        _check(net_validate(s), "msp_net_param_count")
    return int(n)


def _aligned_buffer(n: int, device) -> Workspace:
    buf = torch.empty(n + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return Workspace(buf[off:off + n])


def net_make_workspace(s: NetShape, device=None) -> Workspace:
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = lib().msp_net_workspace_bytes(ctypes.byref(s))
    if n == 0:
        _check(net_validate(s), "msp_net_workspace_bytes")
    return _aligned_buffer(int(n), device)


def _net_ws(s, ws, device):
    if ws is None:
        return net_make_workspace(s, device)
    if ws.nbytes < lib().msp_net_workspace_bytes(ctypes.byref(s)):
        raise ValueError("workspace too small for this network shape")
    return ws


def net_init(s: NetShape, seed: int, device=None, stream=None) -> torch.Tensor:
    """The network's initial FP32 parameters (msp_net_init)."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    params = torch.empty(net_param_count(s), dtype=torch.float32, device=device)
    _check(lib().msp_net_init(ctypes.byref(s), _ptr(params), ctypes.c_uint64(seed), _stream(stream)), "msp_net_init")
    return params


def _net_planes(s: NetShape, params, V, G, target=None):
    device = V.device
    _need(params, "params", torch.float32, (net_param_count(s),), device)
    shp = (s.n_slices, s.height, s.width)
    _need(V, "V", torch.float32, shp, device)
    _need(G, "G", torch.float32, shp, device)
    if target is not None:
        _need(target, "target", torch.float32, shp, device)
    return device


def net_forward(s: NetShape, params, V, G, out=None, ws=None, stream=None):
    """Proposal dV_prop [L][H][W] = s_D net(s_V V, s_G G) (msp_net_forward)."""
    device = _net_planes(s, params, V, G)
    if out is None:
        out = torch.empty_like(V)
    _need(out, "dV_prop", torch.float32, tuple(V.shape), device)
    ws = _net_ws(s, ws, device)
    _check(lib().msp_net_forward(ctypes.byref(s), _ptr(params), _ptr(V), _ptr(G), _ptr(out), ws.ptr(), ws.nbytes,
                                 _stream(stream)), "msp_net_forward")
    return out


def net_loss_grad(s: NetShape, params, V, G, target, ws=None, stream=None):
    """(loss (device float64 scalar), gradient (FP32, parameter layout)) (msp_net_loss_grad)."""
    device = _net_planes(s, params, V, G, target)
    ws = _net_ws(s, ws, device)
    grad = torch.empty_like(params)
    loss = torch.empty((), dtype=torch.float64, device=device)
    _check(lib().msp_net_loss_grad(ctypes.byref(s), _ptr(params), _ptr(V), _ptr(G), _ptr(target), _ptr(grad),
                                   _ptr(loss), ws.ptr(), ws.nbytes, _stream(stream)), "msp_net_loss_grad")
    return loss, grad


def net_train_step(s: NetShape, params, adam_m, adam_v, step: int, lr: float, V, G, target, loss=None, ws=None,
                   stream=None):
    """One Adam step in place on params / adam_m / adam_v (msp_net_train_step); returns the loss
    before the step (device float64 scalar)."""
    device = _net_planes(s, params, V, G, target)
    _need(adam_m, "adam_m", torch.float32, tuple(params.shape), device)
    _need(adam_v, "adam_v", torch.float32, tuple(params.shape), device)
    ws = _net_ws(s, ws, device)
    if loss is None:
        loss = torch.empty((), dtype=torch.float64, device=device)
    _check(lib().msp_net_train_step(ctypes.byref(s), _ptr(params), _ptr(adam_m), _ptr(adam_v), int(step), float(lr),
                                    _ptr(V), _ptr(G), _ptr(target), _ptr(loss), ws.ptr(), ws.nbytes,
                                    _stream(stream)), "msp_net_train_step")
    return loss


def learned_make_workspace(g: Geometry, s: NetShape, device=None) -> Workspace:
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = lib().msp_learned_workspace_bytes(ctypes.byref(g), ctypes.byref(s))
    if n == 0:
        _check(net_validate(s), "msp_learned_workspace_bytes")
        _check(validate_geometry(g), "msp_learned_workspace_bytes")
        raise MspError(MSP_EINVAL, "msp_learned_workspace_bytes", "network shape and geometry disagree")
    return _aligned_buffer(int(n), device)


def learned_propose(g: Geometry, s: NetShape, params, probe, V, pos, I_meas, accepted=None, loss=None, ws=None,
                    learn_ws=None, stream=None):
    """One proposal under the acceptance rule (msp_learned_propose): V becomes V + net(V, dL/dV)
    if that lowers the loss, in place.  Returns (accepted (device int32), loss (device float64
    [2]: before, at the candidate))."""
    device = _arrays(g, probe, V, pos, I_meas)
    _need(params, "params", torch.float32, (net_param_count(s),), device)
    ws = _ws(g, ws, device)
    if learn_ws is None:
        learn_ws = learned_make_workspace(g, s, device)
    if accepted is None:
        accepted = torch.zeros((), dtype=torch.int32, device=device)
    if loss is None:
        loss = torch.empty(2, dtype=torch.float64, device=device)
    _check(lib().msp_learned_propose(ctypes.byref(g), ctypes.byref(s), _ptr(params), _ptr(probe), _ptr(V), _ptr(pos),
                                     _ptr(I_meas), _ptr(accepted), _ptr(loss), ws.ptr(), ws.nbytes, learn_ws.ptr(),
                                     learn_ws.nbytes, _stream(stream)), "msp_learned_propose")
    return accepted, loss


def _conv_ws(H, W, cin, cout, device):
    n = lib().msp_conv3x3_test_workspace_bytes(H, W, cin, cout)
    if n == 0:
        raise MspError(MSP_EUNSUPPORTED, "msp_conv3x3_test", "c_in, c_out in {16, 64}, width a multiple of 128")
    return _aligned_buffer(int(n), device)


def conv3x3_test(x_bf16, w, bias=None, stream=None):
    """Pre-activation conv(x) + bias (FP32 [H][W][c_out]) of one BF16 NHWC image (msp_conv3x3_test)."""
    H, W, cin = x_bf16.shape
    cout = w.shape[0]
    device = x_bf16.device
    _need(x_bf16, "in", torch.bfloat16, (H, W, cin), device)
    _need(w, "w", torch.float32, (cout, 9, cin), device)
    if bias is not None:
        _need(bias, "bias", torch.float32, (cout,), device)
    out = torch.empty((H, W, cout), dtype=torch.float32, device=device)
    ws = _conv_ws(H, W, cin, cout, device)
    _check(lib().msp_conv3x3_test(H, W, cin, cout, _ptr(x_bf16), _ptr(w), _ptr(bias), _ptr(out), ws.ptr(), ws.nbytes,
                                  _stream(stream)), "msp_conv3x3_test")
    return out, ws


def conv3x3_wgrad_test(x_bf16, g_bf16, stream=None):
    """(dW [c_out][9][c_in], db [c_out]) of a 3 x 3 convolution (msp_conv3x3_wgrad_test)."""
    H, W, cin = x_bf16.shape
    cout = g_bf16.shape[2]
    device = x_bf16.device
    _need(x_bf16, "in", torch.bfloat16, (H, W, cin), device)
    _need(g_bf16, "grad_pre", torch.bfloat16, (H, W, cout), device)
    dW = torch.empty((cout, 9, cin), dtype=torch.float32, device=device)
    db = torch.empty((cout,), dtype=torch.float32, device=device)
    ws = _conv_ws(H, W, cin, cout, device)
    _check(lib().msp_conv3x3_wgrad_test(H, W, cin, cout, _ptr(x_bf16), _ptr(g_bf16), _ptr(dW), _ptr(db), ws.ptr(),
                                        ws.nbytes, _stream(stream)), "msp_conv3x3_wgrad_test")
    return dW, db, ws
