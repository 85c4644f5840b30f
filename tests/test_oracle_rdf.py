"""Pins of the oracle's radial distribution functions and structure factors
(Sec. II.C, Eq. 18): the histogram holds every pair within r_max once
(KD-tree count); an ideal gas gives g = 1 (one and two species) and S(q) = 1;
a step-function g(r) gives S(q) = 1 - 4 pi rho0 (sin qs - qs cos qs) / q^3."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import oracle as O


def _gas(n, L, n_species, seed):
    rng = np.random.default_rng(seed)
    return rng.random((n, 3)) * L, rng.integers(0, n_species, n)


def test_histogram_holds_every_pair_once():
    x, sp = _gas(3000, 4.0, 3, 1)
    c = O.rdf_counts(x, sp, 3, np.array([[4.0, 4.0, 4.0]]), [0, 3000], 1.2, 60)
    n_tree = len(cKDTree(x, boxsize=4.0).query_pairs(1.2))
    assert int(np.triu(c.sum(2)).sum()) == n_tree
    assert np.array_equal(c, c.transpose(1, 0, 2))


def test_ideal_gas_g_is_one():
    L, n = 5.0, 8000
    x, sp = _gas(n, L, 2, 2)
    c = O.rdf_counts(x, sp, 2, np.array([[L, L, L]]), [0, n], 1.2, 24)
    na = [int((sp == k).sum()) for k in range(2)]
    for a, b in ((0, 0), (0, 1), (1, 1)):
        r, g = O.rdf(c[a, b], na[a], na[b], a == b, L ** 3, 1.2)
        keep = r > 0.3
        expected = c[a, b][keep]
        rel = 3.0 / np.sqrt(np.maximum(expected, 1))       # 3 sigma, Poisson
        assert np.all(np.abs(g[keep] - 1.0) < rel), (a, b, g)


def test_structure_factor_of_a_step_function():
    rho0, s, r_max, n_bins = 30.0, 0.3, 1.2, 12000
    dr = r_max / n_bins
    r = (np.arange(n_bins) + 0.5) * dr
    g = (r >= s).astype(float)
    q = np.array([5.0, 12.0, 25.0, 40.0])
    S = O.structure_factor(r, g, rho0, q, dr)
    ref = 1.0 - 4.0 * math.pi * rho0 * (np.sin(q * s) - q * s * np.cos(q * s)) / q ** 3
    assert np.allclose(S, ref, atol=2e-3)


def test_structure_factor_of_an_ideal_gas_is_one():
    r = np.linspace(0.005, 1.195, 120)
    S = O.structure_factor(r, np.ones_like(r), 30.0, np.array([3.0, 10.0, 30.0]), 0.01)
    assert np.allclose(S, 1.0, atol=1e-12)
