"""Host-side statistics of the Section 4 experiments (no device needed):
the Gamma-law bin probabilities of Eq. (dist-analytic), the histogram error
of Eq. (error-dist) and its sampling floor, the drift slope and the reduced
time unit of Eq. (reduced-units)."""
import math

import numpy as np
import pytest

pytest.importorskip("scipy")

from paper_1707_04232_gb300 import experiments as X  # noqa: E402


def test_gamma_bins_sum_to_one_and_match_quadrature():
    C = 6.0
    p = X.gamma_bin_probabilities(C, 1.0, 1e-9, 200.0, 1000)
    assert abs(p.sum() - 1.0) < 1e-12
    # bin probabilities against Simpson quadrature of x^(C-1) e^-x / Gamma(C)
    lo, hi, nb, scale = 0.1, 20.0, 150, 0.8
    p = X.gamma_bin_probabilities(C, scale, lo, hi, nb)
    edges = np.linspace(lo, hi, nb + 1) * scale
    for b in (0, 17, 75, 149):
        x = np.linspace(edges[b], edges[b + 1], 201)
        f = x ** (C - 1) * np.exp(-x) / math.gamma(C)
        h = x[1] - x[0]
        simpson = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
        assert abs(p[b] - simpson) <= 1e-10 * max(simpson, 1e-300) + 1e-15


def test_distribution_error_is_zero_at_the_law_and_at_its_floor_when_sampled():
    C, lo, hi, nb = 6.0, 0.1, 20.0, 150
    p = X.gamma_bin_probabilities(C, 1.0, lo, hi, nb)
    n = 10 ** 7
    from scipy import special
    below, above = special.gammainc(C, lo), special.gammaincc(C, hi)
    exact = np.concatenate([p * n, [below * n, above * n]])  # every sample counted somewhere
    assert X.distribution_error(exact, C, 1.0, lo, hi)["error"] < 1e-12
    # independent Gamma samples histogrammed on the same grid: the error sits
    # at the multinomial floor (its expectation, up to a few per cent)
    rng = np.random.default_rng(3)
    errs = []
    for _ in range(20):
        x = rng.gamma(C, 1.0, size=200000)
        counts = np.histogram(x, bins=nb, range=(lo, hi))[0].astype(float)
        counts = np.concatenate([counts, [(x < lo).sum(), (x >= hi).sum()]])
        r = X.distribution_error(counts, C, 1.0, lo, hi)
        errs.append(r["error"] / r["floor_independent"])
    assert 0.85 < np.sqrt(np.mean(np.square(errs))) < 1.15
    # a biased law (wrong shape) sits far above the floor
    x = rng.gamma(C * 1.05, 1.0, size=200000)
    counts = np.concatenate([np.histogram(x, bins=nb, range=(lo, hi))[0], [0, 0]]).astype(float)
    r = X.distribution_error(counts, C, 1.0, lo, hi)
    assert r["error"] > 5 * r["floor_independent"]


def test_energy_drift_slope_recovers_a_line():
    rng = np.random.default_rng(1)
    t = np.linspace(0.0, 100.0, 401)
    E = 3.0 - 2.5e-3 * t + 1e-4 * rng.standard_normal(t.size)
    assert abs(X.energy_drift_slope(t, E) + 2.5e-3) < 1e-6


def test_reduced_time_unit():
    # m = 1, a = 1, kT = 1: t_K = 1 / sqrt(K)
    assert abs(X.reduced_time_unit(5.0) - 1 / math.sqrt(5.0)) < 1e-15
    # l_K = (m/rho)^(1/3), m_K = m, eps_K = K kB T
    assert abs(X.reduced_time_unit(20.0, m=8.0, rho=1.0, kT=0.5) - 2.0 * math.sqrt(8.0 / 10.0)) < 1e-14
