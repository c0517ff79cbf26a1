"""The seeded input recipe (workloads/synth.py) that both the oracle and the library are fed:
scan rasters inside the object, reproducible potentials and probes, the learned-proposal
specimens within their stated ranges, and counting noise that depends only on (seed, scan
index).  CPU only."""
import numpy as np
import pytest

from workloads import synth


@pytest.mark.parametrize("name", sorted(synth.CONFIGS))
def test_scan_raster_lies_in_the_object(name):
    cfg = synth.CONFIGS[name]
    pos = synth.scan_positions(cfg)
    assert pos.shape == (cfg.n_pos, 2) and pos.dtype == np.int32
    assert pos.min() >= 0 and pos.max() <= cfg.obj - cfg.win
    ys, xs = np.unique(pos[:, 0]), np.unique(pos[:, 1])
    assert len(ys) == cfg.scan[0] and len(xs) == cfg.scan[1]
    assert np.all(np.diff(ys) == cfg.step_px) and np.all(np.diff(xs) == cfg.step_px)
    sub = synth.scan_positions(cfg, sub=(3, 3))
    assert len(sub) == 9 and set(map(tuple, sub)) <= set(map(tuple, pos))
    g = synth.geometry(cfg)
    assert (g["n_slices"], g["obj_ny"], g["win"], g["n_pos"]) == (cfg.n_slices, cfg.obj, cfg.win, cfg.n_pos)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_potentials_and_probe_are_reproducible(name):
    cfg = synth.CONFIGS[name]
    a, b = synth.potential_slices(cfg), synth.potential_slices(cfg)
    assert a.shape == (cfg.n_slices, cfg.obj, cfg.obj) and np.all(np.isfinite(a))
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.potential_slices(cfg, seed=cfg.seed + 1))
    p = synth.probe(cfg)
    assert p.shape == (cfg.win, cfg.win) and np.array_equal(p, synth.probe(cfg))
    if cfg.defocus_guess_A is not None:
        assert not np.allclose(p, synth.probe(cfg, defocus_A=cfg.defocus_guess_A))


def test_learned_specimens_stay_in_their_ranges():
    seen = set()
    for seed in range(40):
        c = synth.c5_specimen(seed)
        assert c == synth.c5_specimen(seed)
        assert 3.0 <= c.lattice_A <= 5.0
        assert 1 <= len(c.species_vnm) <= 3 and all(0.5 <= a <= 3.0 for a in c.species_vnm)
        assert 0.0 <= c.vacancy <= 0.4 and 1e5 <= c.dose <= 1e7 and c.rotate
        assert (c.n_slices, c.obj, c.win, c.scan) == (synth.C5.n_slices, synth.C5.obj, synth.C5.win, synth.C5.scan)
        seen.add(round(c.lattice_A, 6))
    assert len(seen) == 40          # every seed draws its own specimen


def test_counting_noise_depends_on_seed_and_scan_index_only():
    rng = np.random.default_rng(3)
    I = rng.uniform(0.0, 1.0, size=(12, 8, 8))
    dose = 1e4
    full = synth.poisson_counts(I, dose, seed=7)
    assert np.all(full == np.round(full)) and np.all(full >= 0)
    # a sample of positions sees the same noise as those positions in the full scan
    idx = np.array([2, 5, 11])
    assert np.array_equal(synth.poisson_counts(I[idx], dose, seed=7, index=idx), full[idx])
    assert not np.array_equal(synth.poisson_counts(I, dose, seed=8), full)
    # each pattern is scaled to `dose` expected counts: totals within 5 sigma of it
    tot = full.reshape(12, -1).sum(axis=1)
    assert np.all(np.abs(tot - dose) < 5 * np.sqrt(dose))
    assert np.array_equal(synth.poisson_counts(I, None, seed=7), I)    # noiseless workloads
