"""The synthetic inputs follow their stated recipe (CPU): octave counts and
scales, Gaussians in octave 0, and the amplitude normalisation c_rho that gives
the Gaussian band a mean optical depth of tau_target per unit path."""
import math

import numpy as np
from scipy import stats

import oracle
import synth


def test_octave_counts_and_scales():
    assert synth.octave_counts(100_000, 4) == [1176, 4704, 18816, 75304]
    assert synth.octave_counts(1_000_000, 6)[0] == 732
    p = synth.octave_field(20_000, 4, seed=1)
    s = np.exp(p["log_scale"].astype(np.float64))
    for o, n in enumerate(p["octave_counts"]):
        sel = p["band"] == o
        assert sel.sum() == n
        assert s[sel].min() >= 0.02 * 2.0 ** -o * (1 - 1e-6)
        assert s[sel].max() <= 0.1 * 2.0 ** -o * (1 + 1e-6)
    g = p["band"] == 0
    assert np.all(p["omega"][g] == 0) and np.all(p["phase"][g] == 0)
    assert np.all(p["omega"][~g] > 0)


def test_gaussian_band_mass_matches_tau_target():
    """Rays along z over a square wide enough to hold every kernel whole: the
    mean line integral times the square's area is the band's total mass, which
    c_rho sets to tau_target per unit path (unit cube), less the mass outside
    the 3-sigma support (chi^2_3 tail)."""
    p = synth.octave_field(200_000, 1, seed=4)
    f = oracle.Field(p, omega_frame="local")
    rng = np.random.default_rng(1)
    n, lo, hi = 2048, -0.35, 1.35
    xy = rng.uniform(lo, hi, (n, 2))
    o = np.concatenate([xy, np.full((n, 1), -0.5)], 1).astype(np.float32)
    d = np.tile(np.array([0, 0, 1.0], np.float32), (n, 1))
    tr = np.tile(np.array([0.0, 3.0], np.float32), (n, 1))
    _, tau = f.transmittance(o, d, tr)
    area = (hi - lo) ** 2
    mass, se = tau.mean() * area, tau.std(ddof=1) / math.sqrt(n) * area
    expected = 4.0 * stats.chi2.cdf(9.0, 3)
    assert abs(mass - expected) < 4 * se + 0.01 * expected, (mass, se, expected)
