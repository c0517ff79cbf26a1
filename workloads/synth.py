"""Seeded synthetic inputs shaped like the paper's multislice workloads.

The paper reconstructs simulated GaAs / SrTiO3 / MoS2 crystals (Table 1) and an
experimental MoS2 4D-STEM scan (Sec. 4.2); neither dataset exists here.  These
generators stand in for them with seeded Gaussian-lattice projected potentials,
an aperture-limited defocused probe and a regular raster of integer scan
positions, so that the oracle and the CUDA library are driven by identical
inputs.

This module holds none of the method's arithmetic: it draws random numbers,
places Gaussian sites on a lattice, builds the probe as the inverse Fourier
transform of a circular aperture (Sec. 2.1 describes the probe that way) and
applies Poisson counting noise.  The forward model that turns a specimen into
intensities lives in the oracle (for tests) and in the CUDA library (for
benchmarks), never here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import physics


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_slices: int          # L (the paper's M)
    obj: int               # object side in pixels (square object)
    pixel_A: float         # real-space pixel size
    dz_A: float            # slice thickness = Fresnel distance
    kv: float              # accelerating voltage in kV
    win: int               # probe window = detector side W
    scan: tuple            # (ny, nx) raster points
    step_px: int           # raster step in pixels
    aperture_mrad: float   # probe semi-convergence angle
    defocus_A: float       # true probe defocus
    defocus_guess_A: float | None  # initial probe guess (None: probe known)
    lattice_A: float = 3.9
    species_vnm: tuple | None = None   # discrete site amplitudes (V nm); None: U(0.5, 2)
    vacancy: float = 0.0
    rotate: bool = False   # random lattice rotation per slice in [0, 90) deg
    dose: float | None = None  # electrons per pattern for Poisson noise; None: noiseless
    gauss_sigma_A: float = 0.3
    seed: int = 0

    @property
    def n_pos(self) -> int:
        return self.scan[0] * self.scan[1]

    @property
    def volts(self) -> float:
        return self.kv * 1e3


# The five configurations of the benchmark specification; sizes as stated there.
C1 = Workload("c1_L2_obj96_W64_S64", 2, 96, 0.2, 2.0, 30, 64, (8, 8), 4, 25.0, 50.0, None,
              lattice_A=3.9, species_vnm=None, seed=0)
C2 = Workload("c2_L4_obj384_W128_S1024", 4, 384, 0.15, 2.0, 30, 128, (32, 32), 8, 30.0, 100.0, 120.0,
              lattice_A=3.9, species_vnm=(1.0, 2.5), vacancy=0.3, dose=1e6, seed=1)
C3 = Workload("c3_L8_obj384_W128_S4096", 8, 384, 0.15, 2.0, 30, 128, (64, 64), 4, 30.0, 100.0, 120.0,
              lattice_A=3.9, species_vnm=(1.0, 2.5), vacancy=0.3, rotate=True, dose=1e5, seed=2)
C4 = Workload("c4_L16_obj640_W256_S2304", 16, 640, 0.1, 1.0, 30, 256, (48, 48), 8, 30.0, 100.0, None,
              lattice_A=3.9, species_vnm=None, seed=3)
# The learned-proposal workload: the c2 scan geometry with eight slices; every specimen of its
# corpus draws its own lattice constant (3-5 A), rotation, one to three species, vacancy fraction
# (0-40 %) and dose (1e5-1e7 electrons per pattern): `c5_specimen(seed)`.
C5 = Workload("c5_L8_obj384_W128_S1024", 8, 384, 0.15, 2.0, 30, 128, (32, 32), 8, 30.0, 100.0, None,
              lattice_A=3.9, species_vnm=(1.0, 2.5), vacancy=0.3, rotate=True, dose=1e6, seed=6)
CONFIGS = {"c1": C1, "c2": C2, "c3": C3, "c4": C4, "c5": C5}


def c5_specimen(seed: int, base: Workload = C5) -> Workload:
    """One seeded specimen of the learned-proposal corpus (see C5)."""
    rng = np.random.default_rng([seed, 55])
    n_species = int(rng.integers(1, 4))
    return dataclasses.replace(
        base, lattice_A=float(rng.uniform(3.0, 5.0)),
        species_vnm=tuple(float(a) for a in rng.uniform(0.5, 3.0, size=n_species)),
        vacancy=float(rng.uniform(0.0, 0.4)), rotate=True, dose=float(10.0 ** rng.uniform(5.0, 7.0)),
        seed=int(seed))

# Algorithm 2 on the paper's own setting (Table 1, GaAs): a 2 x 2 supercell of the
# 5.6533 A cubic cell on a 40 x 40 grid, every one of the 40 x 40 cyclic probe shifts,
# 200 kV, 32 mrad, three slices 2 nm apart (the distance at which the paper's sparse
# decomposition separates the slices, Sec. 5.3).  Atomic columns every a/2; a 2 nm slice
# holds several atoms per column, so each column is given 40-45 V nm (about 0.3 rad).
GAAS_CELL_A = 5.6533
SMD_GAAS = Workload("smd_gaas_N40_M3_S1600", 3, 40, 2 * GAAS_CELL_A / 40, 20.0, 200, 40, (40, 40), 1,
                    32.0, 0.0, None, lattice_A=GAAS_CELL_A / 2, species_vnm=(40.0, 45.0), seed=5)
SMD_CONFIGS = {"smd_gaas": SMD_GAAS}


def smd_geometry(cfg: Workload, n_pos: int | None = None) -> dict:
    """Scalar statement of the full-field problem of Algorithm 2 (N = object = probe = detector side)."""
    return dict(n=cfg.obj, n_slices=cfg.n_slices, n_pos=cfg.n_pos if n_pos is None else n_pos,
                wavelength_A=physics.wavelength_A(cfg.volts), sigma=physics.interaction_constant(cfg.volts),
                dz_A=cfg.dz_A, pixel_A=cfg.pixel_A, obj_ny=cfg.obj, obj_nx=cfg.obj, win=cfg.obj)


def cyclic_shifts(n: int, step: int = 1, count: int | None = None, seed: int | None = None) -> np.ndarray:
    """Probe shifts (ys, xs) of a cyclic raster with the given step (step 1: all n^2 shifts,
    the paper's full scan); `count` draws that many distinct shifts at random instead."""
    if count is not None:
        rng = np.random.default_rng([0 if seed is None else seed, 41])
        flat = rng.choice(n * n, size=count, replace=False)
        return np.stack([flat // n, flat % n], axis=1).astype(np.int32)
    g = np.arange(0, n, step)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    return np.stack([yy.ravel(), xx.ravel()], axis=1).astype(np.int32)


def random_phase_slices(M: int, n: int, seed: int, amp: float = 0.5) -> np.ndarray:
    """Unimodular slices exp(i amp g) with Gaussian g, complex128 [M][n][n]."""
    rng = np.random.default_rng([seed, 43])
    return np.exp(1j * amp * rng.standard_normal((M, n, n)))


def geometry(cfg: Workload, n_pos: int | None = None) -> dict:
    """Scalar problem statement shared by the oracle and the library."""
    return dict(
        n_slices=cfg.n_slices, obj_ny=cfg.obj, obj_nx=cfg.obj, win=cfg.win,
        n_pos=cfg.n_pos if n_pos is None else n_pos,
        wavelength_A=physics.wavelength_A(cfg.volts),
        sigma=physics.interaction_constant(cfg.volts),
        dz_A=cfg.dz_A, pixel_A=cfg.pixel_A,
    )


def scan_positions(cfg: Workload, sub: tuple | None = None) -> np.ndarray:
    """Window top-left corners (y, x) of a raster centred in the object.

    `sub=(ny, nx)` keeps the centred ny x nx block of the raster (a sub-scan).
    """
    ny, nx = cfg.scan
    span_y = (ny - 1) * cfg.step_px + cfg.win
    span_x = (nx - 1) * cfg.step_px + cfg.win
    pad_y = (cfg.obj - span_y) // 2
    pad_x = (cfg.obj - span_x) // 2
    assert pad_y >= 0 and pad_x >= 0, "raster does not fit the object"
    iy = np.arange(ny)
    ix = np.arange(nx)
    if sub is not None:
        oy = (ny - sub[0]) // 2
        ox = (nx - sub[1]) // 2
        iy = iy[oy:oy + sub[0]]
        ix = ix[ox:ox + sub[1]]
    yy, xx = np.meshgrid(pad_y + iy * cfg.step_px, pad_x + ix * cfg.step_px, indexing="ij")
    return np.stack([yy.ravel(), xx.ravel()], axis=1).astype(np.int32)


def potential_slices(cfg: Workload, seed: int | None = None) -> np.ndarray:
    """Projected potential of every slice in V*angstrom, float64 [L][N][N].

    Each slice is a sum of isotropic Gaussians a*exp(-r^2 / (2 s^2)) (s = 0.3 A,
    truncated at 5 s) on a square lattice with a random sub-lattice offset and,
    if requested, a random rotation; site amplitudes are drawn per site.
    """
    rng = np.random.default_rng([cfg.seed if seed is None else seed, 11])
    n, px = cfg.obj, cfg.pixel_A
    extent = n * px
    out = np.zeros((cfg.n_slices, n, n))
    s = cfg.gauss_sigma_A
    rad = int(math.ceil(5 * s / px))
    dy, dx = np.mgrid[-rad:rad + 1, -rad:rad + 1]
    for l in range(cfg.n_slices):
        off = rng.uniform(0.0, cfg.lattice_A, size=2)
        th = rng.uniform(0.0, 0.5 * math.pi) if cfg.rotate else 0.0
        c, sn = math.cos(th), math.sin(th)
        m = int(math.ceil(extent * 1.5 / cfg.lattice_A)) + 2
        ii, jj = np.mgrid[-m:m + 1, -m:m + 1]
        u = ii.ravel() * cfg.lattice_A
        v = jj.ravel() * cfg.lattice_A
        sy = c * u - sn * v + off[0]
        sx = sn * u + c * v + off[1]
        keep = (sy > -5 * s) & (sy < extent + 5 * s) & (sx > -5 * s) & (sx < extent + 5 * s)
        sy, sx = sy[keep], sx[keep]
        if cfg.species_vnm is None:
            amp = rng.uniform(0.5, 2.0, size=sy.size)
        else:
            amp = rng.choice(np.asarray(cfg.species_vnm), size=sy.size)
        if cfg.vacancy > 0:
            amp = amp * (rng.uniform(size=sy.size) >= cfg.vacancy)
        amp = amp * 10.0  # V*nm -> V*angstrom
        for y0, x0, a in zip(sy, sx, amp):
            if a == 0.0:
                continue
            cy, cx = int(round(y0 / px)), int(round(x0 / px))
            yy, xx = cy + dy, cx + dx
            r2 = (yy * px - y0) ** 2 + (xx * px - x0) ** 2
            val = a * np.exp(-r2 / (2 * s * s)) * (r2 <= (5 * s) ** 2)
            ok = (yy >= 0) & (yy < n) & (xx >= 0) & (xx < n)
            np.add.at(out[l], (yy[ok], xx[ok]), val[ok])
    return out


def probe(cfg: Workload, defocus_A: float | None = None, norm2: float | None = None) -> np.ndarray:
    """Aperture-limited probe with defocus, complex128 [W][W], centred at (W/2, W/2).

    p = IFT[ 1{|q| <= alpha/lambda} * exp(-i pi lambda df q^2) ], scaled so that
    sum |p|^2 = norm2 (default: dose / W^2, so a pattern of a pure-phase object
    carries `dose` counts; 1 for noiseless workloads).
    """
    w, px = cfg.win, cfg.pixel_A
    lam = physics.wavelength_A(cfg.volts)
    df = cfg.defocus_A if defocus_A is None else defocus_A
    q = np.fft.fftfreq(w, d=px)
    qy, qx = np.meshgrid(q, q, indexing="ij")
    q2 = qy ** 2 + qx ** 2
    qmax = cfg.aperture_mrad * 1e-3 / lam
    spec = (q2 <= qmax * qmax) * np.exp(-1j * math.pi * lam * df * q2)
    p = np.fft.fftshift(np.fft.ifft2(spec))
    if norm2 is None:
        norm2 = 1.0 if cfg.dose is None else cfg.dose / (w * w)
    p *= math.sqrt(norm2 / np.sum(np.abs(p) ** 2))
    return p


def poisson_counts(intensity: np.ndarray, dose: float | None, seed: int, index=None) -> np.ndarray:
    """Counting noise: each pattern is scaled to `dose` expected counts, then Poisson-sampled.

    Pattern k draws from its own stream, seeded by (seed, its scan index); `index` gives the
    scan indices of the patterns passed (default 0, 1, ...), so the noise of a sample of
    positions equals that of the same positions in the full scan."""
    if dose is None:
        return intensity.copy()
    index = np.arange(intensity.shape[0]) if index is None else np.asarray(index)
    tot = intensity.reshape(intensity.shape[0], -1).sum(axis=1)
    scale = np.where(tot > 0, dose / np.maximum(tot, 1e-300), 0.0)
    out = np.empty(intensity.shape, dtype=np.float64)
    for k in range(intensity.shape[0]):
        rng = np.random.default_rng([seed, 23, int(index[k])])
        out[k] = rng.poisson(intensity[k] * scale[k])
    return out


def random_complex(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 31])
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_real(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng([seed, 37])
    return scale * rng.standard_normal(shape)
