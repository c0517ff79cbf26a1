"""The normal-CDF fit of the proposal network's GELU (csrc/msp_learn.cu, phi_cdf): the table in
the kernel is the one csrc/gen_phi_fit.py fits, and in FP32 it stays within 1e-7 of Phi
(scipy's ndtr) over the whole line, both tails included."""
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_03902_gb300", "csrc")


def _gen():
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_phi_fit", os.path.join(CSRC, "gen_phi_fit.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_kernel_table_is_the_fit():
    src = open(os.path.join(CSRC, "msp_learn.cu")).read()
    body = src[src.index("float phi_cdf(float x)"):src.index("return x < 0.f ? t : 1.f - t;")]
    lits = [float(v) for v in re.findall(r"(-?\d\.\d+e[+-]\d+)f", body)]
    kernel = np.array(lits[::-1], dtype=np.float32)        # Horner runs from the top coefficient
    fit = _gen().fit()
    assert kernel.shape == fit.shape
    assert np.all(np.abs(kernel - fit) <= 1e-6 * np.abs(fit))


def test_fp32_phi_error():
    g = _gen()
    p = g.fit()
    x = np.linspace(-12, 12, 480001)
    err = np.abs(g.phi32(p, x) - scipy_special.ndtr(x))
    assert err.max() < 1.2e-7
    neg = (x < -1) & (x > -8)       # the lower tail keeps its relative accuracy
    ref = scipy_special.ndtr(x[neg])
    assert np.max(np.abs(g.phi32(p, x[neg]) - ref) / ref) < 2e-5
