"""Coefficients of the normal CDF used by the proposal network's GELU (csrc/msp_learn.cu).

Phi(x) = erfc(-x / sqrt 2) / 2.  With z = |x| / sqrt 2 and g(z) = -log(erfc(z)):
    Phi(x) = exp(-g(z)) / 2          for x < 0,
    Phi(x) = 1 - exp(-g(z)) / 2      for x >= 0,
so both tails keep their accuracy and no branch is needed.  g(z) / z is smooth on [0, 6]
(from 2 / sqrt(pi) at 0); it is fitted by least squares in the Chebyshev basis of
u = z / 3 - 1 and written as monomial coefficients in u for Horner evaluation in FP32.  Beyond
z = 6 (|x| > 8.49) z is clamped: Phi is then within 1e-17 of 0 or 1.

Run:  python gen_phi_fit.py    (prints the C++ table and the FP32 error against scipy)
"""
import numpy as np
from scipy.special import erfc, ndtr

ZMAX, DEG = 6.0, 11


def fit():
    z = np.linspace(1e-6, ZMAX, 300001)
    h = -np.log(erfc(z)) / z
    c = np.polynomial.chebyshev.chebfit(z / (ZMAX / 2) - 1, h, DEG)
    return np.polynomial.chebyshev.cheb2poly(c).astype(np.float32)


def phi32(p32, x):
    """Phi as the kernel evaluates it: FP32 Horner with fused multiply-adds, exact exp."""
    z = np.minimum(np.abs(x).astype(np.float32) * np.float32(0.70710678118654752), np.float32(ZMAX))
    u = (z.astype(np.float64) * np.float32(1 / (ZMAX / 2)) - 1).astype(np.float32)
    acc = np.full_like(u, p32[-1])
    for k in range(len(p32) - 2, -1, -1):
        acc = (acc.astype(np.float64) * u + p32[k]).astype(np.float32)
    g = (acc.astype(np.float64) * z).astype(np.float32)
    t = (0.5 * np.exp(-g.astype(np.float64))).astype(np.float32)
    return np.where(x < 0, t, np.float32(1) - t).astype(np.float64)


if __name__ == "__main__":
    p = fit()
    x = np.linspace(-10, 10, 800001)
    err = np.max(np.abs(phi32(p, x) - ndtr(x)))
    print(f"// max |Phi error| on [-10, 10] in FP32: {err:.2e}")
    print("constexpr float kPhiFit[%d] = {" % len(p))
    print(",\n".join("    %.9ef" % v for v in p) + "};")
