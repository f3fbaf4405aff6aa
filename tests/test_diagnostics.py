"""Diagnostics of read-back fields (spherical profiles, volume-weighted
distributions, front radius) and the black-body photon rate of the Test-3
input recipe, on cases with exact answers."""
import math

import numpy as np
import pytest

from paper_1101_4127_gb300 import diagnostics as D
from paper_1101_4127_gb300 import inputs


def test_radial_profile_of_a_ball_and_counts():
    n, R = 20, 6.0
    c = (10.0, 10.0, 10.0)
    r = D.cell_radii((n, n, n), c)
    ball = (r < R).astype(float)
    edges = np.arange(0.0, 12.0, 1.0)
    mean, count = D.radial_profile(ball, c, edges)
    assert count.sum() == int((r < edges[-1]).sum())
    assert np.all(mean[:6] == 1.0) and np.all(mean[6:] == 0.0)
    m2, _ = D.radial_profile(r, c, edges)           # the field r averages inside its shell
    assert np.all((m2 >= edges[:-1]) & (m2 < edges[1:]))


def test_volume_pdf_integrates_to_the_covered_volume():
    rng = np.random.default_rng(1)
    f = rng.uniform(0.0, 1.0, (8, 8, 8))
    edges = np.linspace(0.0, 0.5, 6)
    pdf = D.volume_pdf(f, edges)
    assert np.sum(pdf * np.diff(edges)) == pytest.approx(np.mean(f < 0.5))
    lp = D.volume_pdf(np.full((4, 4, 4), 1e-3), np.array([-4.0, -2.5, -1.0]), log=True)
    assert lp[0] == pytest.approx(1.0 / 1.5) and lp[1] == 0.0


def test_front_radius_of_a_sphere_and_an_octant():
    n = 48
    r = D.cell_radii((n, n, n), (24.0, 24.0, 24.0))
    assert D.front_radius(r < 15.0) == pytest.approx(15.0, rel=0.01, abs=0)
    ro = D.cell_radii((n, n, n), (0.0, 0.0, 0.0))
    assert D.front_radius(ro < 30.0, octant=True) == pytest.approx(30.0, rel=0.01, abs=0)


def test_blackbody_ionising_rate_matches_the_exact_series():
    """The photon integral of x^2/(e^x - 1) above x0 equals
    sum_k e^{-k x0} (x0^2/k + 2 x0/k^2 + 2/k^3) (expand 1/(e^x - 1))."""
    for T in (3e4, 6e4, 1e5):
        kT_eV = 8.617333262e-5 * T
        x0 = 13.6 / kT_eV
        series = sum(math.exp(-k * x0) * (x0 * x0 / k + 2 * x0 / k ** 2 + 2 / k ** 3)
                     for k in range(1, 400))
        want = 1e38 / (kT_eV * 1.602176634e-12) * series / (math.pi ** 4 / 15)
        assert inputs.blackbody_ionising_rate(1e38, T) == pytest.approx(want, rel=1e-10, abs=0)
