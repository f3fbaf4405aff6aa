"""The seeded synthetic inputs that stand in for the paper's datasets: the
lognormal density field (exact mean, log-scatter sigma, P(k) slope,
seeding), source placement and luminosities, black-body bins, and the
workload recipes against the paper's stated parameters."""
import math

import numpy as np
import pytest

from paper_1101_4127_gb300 import inputs


def test_lognormal_field_mean_scatter_and_seeding():
    n, sig, mean = 48, 1.5, 2e-4
    f = inputs.lognormal_field(n, sig, mean, seed=7)
    assert f.shape == (n, n, n) and f.dtype == np.float32 and np.all(f > 0)
    assert float(f.astype(np.float64).mean()) == pytest.approx(mean, rel=1e-6, abs=0)
    assert float(np.log(f.astype(np.float64)).std()) == pytest.approx(sig, rel=0.02, abs=0)
    assert np.array_equal(f, inputs.lognormal_field(n, sig, mean, seed=7))
    assert not np.array_equal(f, inputs.lognormal_field(n, sig, mean, seed=8))


def test_lognormal_field_power_spectrum_slope():
    """The Gaussian field under the exponential has P(k) ~ k^-2.5: fit the
    slope of the shell-averaged |g_k|^2 over the middle of the k range."""
    n = 64
    f = inputs.lognormal_field(n, 1.0, 1.0, seed=3).astype(np.float64)
    g = np.log(f)
    g -= g.mean()
    pk = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(n) ** 2] * 3, indexing="ij")))
    edges = np.geomspace(4.0 / n, 0.3, 12)
    kc, pc = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        m = (k >= a) & (k < b)
        kc.append(k[m].mean())
        pc.append(pk[m].mean())
    slope = np.polyfit(np.log(kc), np.log(pc), 1)[0]
    assert slope == pytest.approx(-2.5, abs=0.2)


def test_sources_sit_in_the_densest_cells_ties_to_the_lower_index():
    f = np.zeros((4, 4, 4), np.float32)
    f.reshape(-1)[[5, 9, 40]] = 3.0
    f.reshape(-1)[17] = 5.0
    idx = inputs.densest_cells(f, 3)
    assert list(idx) == [17, 5, 9]
    c = inputs.cell_centres(idx, 4, 4)
    assert np.allclose(c[0], [17 % 4 + 0.5, (17 // 4) % 4 + 0.5, 17 // 16 + 0.5])


def test_powerlaw_luminosities_follow_dn_dl_l_minus_2():
    L = inputs.powerlaw_luminosities(20000, 1e46, 1e50, seed=1)
    assert L.min() >= 1e46 and L.max() <= 1e50
    # CDF of dN/dL ~ L^-2 on [a, b]: (1/a - 1/L) / (1/a - 1/b)
    a, b = 1e46, 1e50
    Ls = np.sort(L)
    cdf = (1 / a - 1 / Ls) / (1 / a - 1 / b)
    emp = (np.arange(1, len(Ls) + 1) - 0.5) / len(Ls)
    assert np.max(np.abs(cdf - emp)) < 0.015                  # Kolmogorov-Smirnov distance


def test_blackbody_bins_are_consistent():
    E, f = inputs.blackbody_bins(1e5)
    edges = np.asarray(inputs.BB_EDGES_EV)
    assert len(E) == 8 and f.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all((E > edges[:-1]) & (E < edges[1:])) and np.all(np.diff(E) > 0)
    # the photon share of the first bin against a fine trapezoid integration
    x = np.linspace(13.6, 200.0, 400001)
    kT = inputs.K_B_EV * 1e5
    y = x * x / np.expm1(x / kT)
    tot = np.trapezoid(y, x) if hasattr(np, "trapezoid") else np.trapz(y, x)
    m = x <= edges[1]
    first = np.trapezoid(y[m], x[m]) if hasattr(np, "trapezoid") else np.trapz(y[m], x[m])
    assert f[0] == pytest.approx(first / tot, rel=1e-4, abs=0)


def test_workload_recipes_match_the_paper():
    w0 = inputs.stromgren_32()
    b = w0.boxes[0]
    assert (b.n, b.nH0, b.T0, b.x_HII0, b.isothermal, b.caseB) == (32, 1e-3, 1e4, 1.2e-3, 1, 1)
    assert b.src_ndot[0] == 5e48 and np.all(b.src_pos == 0)
    assert b.box_cm == pytest.approx(6.6 * inputs.KPC_CM)
    assert w0.packets_per_step == [100_000] and w0.n_steps == 20
    assert w0.dt_s == pytest.approx(0.5 * inputs.MYR_S)
    w5 = inputs.lognormal_512(n=32, n_src=100, packets=10_000)
    b5 = w5.boxes[0]
    assert b5.he_over_h == 0.08 and b5.n_src == 100 and len(b5.bin_eV) == 8
    assert float(b5.nH.astype(np.float64).mean()) == pytest.approx(2e-4, rel=1e-6, abs=0)
    wb = inputs.batch_64(scale=1e-3)
    assert len(wb.boxes) == 64
    assert {bx.n for bx in wb.boxes} <= {32, 48, 64, 96, 128}
    assert all(1 <= bx.n_src <= 100 for bx in wb.boxes)
    assert all(p % bx.n_src == 0 for p, bx in zip(wb.packets_per_step, wb.boxes))
    w1 = inputs.stromgren_rec(n=16)
    assert w1.boxes[0].f_rec == 0.1 and w1.boxes[0].caseB == 0
    assert w1.n_steps * w1.dt_s == pytest.approx(5e8 * 3.15576e7, rel=0.01, abs=0)
