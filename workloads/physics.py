"""Electron-optical parameters for the synthetic workloads.

These are host-side helpers that turn an accelerating voltage into the two
physical constants the multislice model takes as inputs: the relativistic
electron wavelength (Sec. 5.3.2, the wavelength relation) and the interaction
constant that scales a projected potential into a phase shift (Sec. 5.3.2
says it grows by about 40% from 200 to 80 kV but prints no formula; the
textbook relativistic form is used).  Neither is part of the per-position
arithmetic; both are passed to the oracle and to the CUDA library as plain
numbers.
"""
import math

# CODATA 2018 exact / recommended values (SI)
PLANCK_H = 6.62607015e-34          # J s
LIGHT_C = 299792458.0              # m / s
CHARGE_E = 1.602176634e-19         # C
ELECTRON_M = 9.1093837015e-31      # kg
ELECTRON_REST_EV = ELECTRON_M * LIGHT_C ** 2 / CHARGE_E   # ~510998.95 eV


def wavelength_A(volts: float) -> float:
    """Relativistic electron wavelength in angstrom, lambda = hc / sqrt(e^2U^2 + 2eUmc^2)
    (Sec. 5.3.2, the wavelength relation)."""
    eU = CHARGE_E * volts
    mc2 = ELECTRON_M * LIGHT_C ** 2
    lam_m = PLANCK_H * LIGHT_C / math.sqrt(eU * eU + 2.0 * eU * mc2)
    return lam_m * 1e10


def interaction_constant(volts: float) -> float:
    """Relativistic interaction constant sigma in rad / (V * angstrom):
    sigma = 2 pi / (lambda U) * (mc^2 + eU) / (2 mc^2 + eU), lambda in angstrom.
    The transmission of a slice with projected potential V (V * angstrom) is
    exp(i sigma V) (Sec. 2.1, the phase grating X_m)."""
    lam = wavelength_A(volts)
    e0 = ELECTRON_REST_EV
    return 2.0 * math.pi / (lam * volts) * (e0 + volts) / (2.0 * e0 + volts)
