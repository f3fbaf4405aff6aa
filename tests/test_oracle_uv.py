"""Pins of the uniform background (the grid option uv_rate / uv_heat_eV: a
reading of Sec. 2's background field as a photo-ionisation rate per atom
and a heat per photo-ionisation, the same in every cell and not attenuated).
CPU only.

  * photo-ionisation equilibrium of pure H under the background alone
    (recombination on, collisions off): the quadratic
    alpha n_H x^2 + Gamma x - Gamma = 0;
  * energy: with every cooling process off, 1.5 k d(n_tot T) equals the heat
    per photo-ionisation times the ionisations, for H and for He I -> He II;
  * He I under its background alone ends as He II, none as He III;
  * a grid of uniform density with a source of no photons: every cell takes
    the single-cell update;
  * a negative or non-finite rate is rejected."""
import math

import numpy as np
import pytest

import oracle

K_B = 1.380649e-16
EV = 1.602176634e-12


def test_background_alone_reaches_the_photoionisation_equilibrium():
    nH, T, G = 1e-3, 1e4, 3e-13
    a = oracle.rates(T, 1)[0]                 # case B alpha_HII (pinned against Osterbrock)
    st, _ = oracle.chem_cell(1e16, nH=nH, xHII=0.0, T=T, U_HI=G, isothermal=1,
                             cool_mask=oracle.C_RECOMB)
    x = (-G + math.sqrt(G * G + 4.0 * a * nH * G)) / (2.0 * a * nH)
    assert st["xHII"] == pytest.approx(x, rel=1e-9, abs=0)


@pytest.mark.parametrize("species", ["H", "HeI"])
def test_background_heat_is_energy_per_ionisation(species):
    nH, nHe, T0, e_eV = 1e-3, 1e-4, 5e3, 7.5
    kw = dict(nH=nH, nHe=nHe, xHII=0.2, xHeII=0.1, xHeIII=0.0, T=T0, isothermal=0, cool_mask=0)
    if species == "H":
        kw.update(U_HI=2e-13, Ue_HI=e_eV * EV)
    else:
        kw.update(xHII=1.0, U_HeI=2e-13, Ue_HeI=e_eV * EV)
    st, n = oracle.chem_cell(3e12, **kw)
    ntot0 = nH + nHe + nH * kw["xHII"] + nHe * kw["xHeII"]
    ntot1 = nH + nHe + nH * st["xHII"] + nHe * (st["xHeII"] + 2 * st["xHeIII"])
    if species == "H":
        ions = nH * (st["xHII"] - kw["xHII"])
    else:
        ions = nHe * (st["xHeII"] - kw["xHeII"])
    assert ions > 0 and n > 1
    assert 1.5 * K_B * (ntot1 * st["T"] - ntot0 * T0) == pytest.approx(e_eV * EV * ions, rel=1e-10, abs=0)


def test_helium_one_background_alone_ends_in_helium_two():
    st, _ = oracle.chem_cell(1e16, nH=1e-3, nHe=1e-4, xHII=1.0, xHeII=0.0, T=2e4, U_HeI=1e-12,
                             isothermal=1, cool_mask=0)
    assert st["xHeII"] == pytest.approx(1.0, rel=1e-12, abs=0) and st["xHeIII"] == 0.0


def test_uniform_grid_with_a_dark_source_takes_the_single_cell_update():
    g = oracle.OracleGrid(5, 4, 3, 1e21, n_H0=1e-3, he_over_h=0.08, x_HII0=0.1, x_HeII0=0.05,
                          T0=8e3, isothermal=0, uv_rate=(1e-13, 5e-14, 1e-15),
                          uv_heat_eV=(3.0, 5.0, 9.0), z_compton=-1.0)
    g.add_sources([[1.5, 1.5, 1.5]], [0.0], [20.0], [[1.0]])
    g.step(2e12, 3)
    nH = float(np.float32(1e-3))               # a uniform n_H0 is rounded to FP32
    st, _ = oracle.chem_cell(2e12, nH=nH, nHe=nH * 0.08, xHII=0.1, xHeII=0.05, T=8e3,
                             U_HI=1e-13, U_HeI=5e-14, U_HeII=1e-15, Ue_HI=3.0 * EV,
                             Ue_HeI=5.0 * EV, Ue_HeII=9.0 * EV)
    for f, k in ((oracle.F_XHII, "xHII"), (oracle.F_XHEII, "xHeII"), (oracle.F_XHEIII, "xHeIII"),
                 (oracle.F_T, "T")):
        v = g.read(f)
        assert np.all(v == v.ravel()[0]) and v.ravel()[0] == pytest.approx(st[k], rel=1e-12, abs=0), k


@pytest.mark.parametrize("bad", [(-1e-13, 0.0, 0.0), (float("nan"), 0.0, 0.0), (0.0, float("inf"), 0.0)])
def test_bad_background_is_rejected(bad):
    with pytest.raises(RuntimeError):
        oracle.OracleGrid(4, 4, 4, 1e21, uv_rate=bad)
