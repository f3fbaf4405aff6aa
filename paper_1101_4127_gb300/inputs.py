"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds the *inputs* of a radiative-transfer run: density fields,
source lists, source spectra discretised into frequency bins, initial states
and the run recipes of the five workloads.  It holds none of the transfer or
chemistry arithmetic; both the CUDA library and the CPU oracle consume what it
returns, so it is the only code the two sides share.

Workload shapes follow the paper's tests:
  * Test 0 setup (Sec. 4.1): uniform pure-H medium, n_H = 1e-3 cm^-3,
    T = 1e4 K, x_HII = 1.2e-3, a 5e48 photons/s source.
  * Test 2 (Sec. 4.2.2): the same medium with T evolving from 100 K and a
    1e5 K black-body source.
  * Test 4 (Sec. 4.2.4) and the 1000-source run (Sec. 5.2): many sources in a
    cosmological density field; the field is replaced by a seeded lognormal
    Gaussian-random-field stand-in because the paper's fields are not
    available.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# unit conversions (CODATA / IAU values)
KPC_CM = 3.0856775814913673e21
MPC_CM = 1e3 * KPC_CM
MYR_S = 3.15576e13          # Julian Myr
EV_ERG = 1.602176634e-12
K_B_EV = 8.617333262e-5     # Boltzmann constant in eV/K


# ---------------------------------------------------------------- fields
def lognormal_field(n: int, sigma_ln: float, mean: float, seed: int,
                    slope: float = -2.5) -> np.ndarray:
    """Seeded lognormal density field on an n^3 grid, float32, shape (n, n, n)
    indexed [z, y, x] so that x is the fastest-varying index in memory.

    A white Gaussian field is filtered in Fourier space to P(k) ~ k^slope,
    normalised to unit variance (g), exponentiated as mean*exp(sigma*g -
    sigma^2/2) and rescaled so that its arithmetic mean is exactly `mean`
    (in float64, before the float32 cast).
    """
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kx = np.fft.rfftfreq(n)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)          # sqrt(P(k)) with P ~ k^slope
    amp[0, 0, 0] = 0.0
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    rho *= mean / rho.mean()
    return rho.astype(np.float32)


def densest_cells(nH: np.ndarray, k: int) -> np.ndarray:
    """Linear indices of the k densest cells; ties go to the lower index."""
    flat = np.asarray(nH).reshape(-1)
    order = np.argsort(-flat.astype(np.float64), kind="stable")
    return order[:k].astype(np.int64)


def cell_centres(lin: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Grid-unit centre coordinates (x, y, z) of linear cell indices."""
    lin = np.asarray(lin, dtype=np.int64)
    x = lin % nx
    y = (lin // nx) % ny
    z = lin // (nx * ny)
    return np.stack([x + 0.5, y + 0.5, z + 0.5], axis=1).astype(np.float64)


def powerlaw_luminosities(n: int, lmin: float, lmax: float, seed: int) -> np.ndarray:
    """n photon rates drawn from dN/dL ~ L^-2 on [lmin, lmax] by inverse CDF:
    L = 1 / (1/lmin - u (1/lmin - 1/lmax)), u uniform in [0, 1)."""
    u = np.random.default_rng(seed).random(n)
    return 1.0 / (1.0 / lmin - u * (1.0 / lmin - 1.0 / lmax))


# ---------------------------------------------------------------- spectra
def _photon_number_bb(E_eV: np.ndarray, T_K: float) -> np.ndarray:
    """Black-body photon number spectrum dN/dE ~ E^2 / (exp(E/kT) - 1)."""
    x = E_eV / (K_B_EV * T_K)
    return E_eV * E_eV / np.expm1(x)


BB_EDGES_EV = (
    list(np.geomspace(13.6, 24.6, 3)[:-1])
    + list(np.geomspace(24.6, 54.4, 3)[:-1])
    + list(np.geomspace(54.4, 200.0, 5))
)


def blackbody_bins(T_K: float = 1e5, edges_eV=None, order: int = 64):
    """Discretise a black-body source into frequency bins.

    Edges default to 2 log bins on [13.6, 24.6), 2 on [24.6, 54.4) and 4 on
    [54.4, 200] eV, aligned with the H I, He I and He II thresholds.  Returns
    (E_j, frac_j): the photon-number-weighted mean energy of each bin and the
    bin's share of the photon number over the whole range, each integral done
    with fixed `order`-point Gauss-Legendre quadrature.
    """
    edges = np.asarray(BB_EDGES_EV if edges_eV is None else edges_eV, dtype=np.float64)
    xg, wg = np.polynomial.legendre.leggauss(order)
    E = np.empty(len(edges) - 1)
    N = np.empty(len(edges) - 1)
    for j in range(len(edges) - 1):
        a, b = edges[j], edges[j + 1]
        e = 0.5 * (b - a) * xg + 0.5 * (b + a)
        f = _photon_number_bb(e, T_K) * 0.5 * (b - a)
        N[j] = np.sum(wg * f)
        E[j] = np.sum(wg * f * e) / N[j]
    return E, N / N.sum()


# ---------------------------------------------------------------- workloads
@dataclass
class Box:
    """One grid with its medium, initial state and sources."""
    n: int                      # cells per side (cubic grid)
    box_cm: float
    nH: Optional[np.ndarray]    # float32 (n,n,n) [z,y,x] or None for uniform
    nH0: float
    he_over_h: float
    x_HII0: float
    x_HeII0: float
    x_HeIII0: float
    T0: float
    isothermal: int
    caseB: int
    z_compton: float
    seed: int
    src_pos: np.ndarray         # (n_src, 3) grid units
    src_ndot: np.ndarray        # (n_src,) photons / s
    bin_eV: np.ndarray          # (n_bins,)
    bin_frac: np.ndarray        # (n_src, n_bins)
    dims: Optional[tuple] = None  # (nx, ny, nz) for non-cubic grids; default (n, n, n)
    f_rec: float = 0.0            # > 0: diffuse recombination field with this threshold
    coupling: int = 0             # 1: photon-conserving transport -> chemistry coupling
    periodic: int = 0             # 1: periodic box, packets stop after the light-travel distance
    uv_rate: tuple = (0.0, 0.0, 0.0)     # uniform background photo-ionisations per atom (H I, He I, He II), s^-1
    uv_heat_eV: tuple = (0.0, 0.0, 0.0)  # heat left by each such photo-ionisation, eV

    @property
    def n_src(self) -> int:
        return int(self.src_ndot.shape[0])

    @property
    def shape_xyz(self):
        return tuple(self.dims) if self.dims is not None else (self.n, self.n, self.n)


@dataclass
class Workload:
    name: str
    boxes: List[Box]
    packets_per_step: List[int]     # per box, total over its sources
    n_steps: int
    dt_s: float
    precision: str                  # "fp64" | "mixed"
    notes: str = ""
    extra: dict = field(default_factory=dict)


def _bins_for(n_src: int, E: np.ndarray, f: np.ndarray):
    return np.asarray(E, np.float64), np.tile(np.asarray(f, np.float64), (n_src, 1))


SEED_BASE = 0x1101412701


def stromgren_32(n: int = 32) -> Workload:
    """Test-0-like isothermal pure-H Stroemgren sphere (Sec. 4.1), 32^3 cells,
    6.6 kpc box, corner source of 5e48 photons/s at 13.6 eV, 1e5 packets per
    step, 20 steps of 0.5 Myr, FP64."""
    E = np.array([13.6])
    bE, bf = _bins_for(1, E, np.array([1.0]))
    box = Box(n=n, box_cm=6.6 * KPC_CM, nH=None, nH0=1e-3, he_over_h=0.0,
              x_HII0=1.2e-3, x_HeII0=0.0, x_HeIII0=0.0, T0=1e4,
              isothermal=1, caseB=1, z_compton=-1.0, seed=SEED_BASE,
              src_pos=np.zeros((1, 3)), src_ndot=np.array([5e48]),
              bin_eV=bE, bin_frac=bf)
    return Workload("stromgren_32^3_H_1src_1bin", [box], [100_000], 20,
                    0.5 * MYR_S, "fp64")


def stromgren_rec(n: int = 128, packets: int = 1_000_000, steps: int = 20,
                  f_rec: float = 0.1) -> Workload:
    """Test-1-like Stroemgren sphere with the diffuse recombination field
    (Sec. 4.2.1): isothermal pure H, n_H = 1e-3, T = 1e4 K, x_HII0 = 1.2e-3,
    corner source of 5e48 photons/s at 13.6 eV in a 6.6 kpc box of n^3 cells;
    case A recombination, a cell re-emits once 10% of its atoms have
    recombined to the ground state; the paper's 5e8 yr in 20 steps of 25 Myr
    (an ionised cell's count passes the threshold within a step or two)."""
    E = np.array([13.6])
    bE, bf = _bins_for(1, E, np.array([1.0]))
    box = Box(n=n, box_cm=6.6 * KPC_CM, nH=None, nH0=1e-3, he_over_h=0.0,
              x_HII0=1.2e-3, x_HeII0=0.0, x_HeIII0=0.0, T0=1e4,
              isothermal=1, caseB=0, z_compton=-1.0, seed=SEED_BASE + 7,
              src_pos=np.zeros((1, 3)), src_ndot=np.array([5e48]),
              bin_eV=bE, bin_frac=bf, f_rec=f_rec)
    return Workload(f"stromgren_rec_{n}^3_H_1src_1bin_frec{f_rec:g}", [box], [packets], steps,
                    25.0 * MYR_S, "fp64")


def blackbody_ionising_rate(L_erg_s: float, T_K: float) -> float:
    """Photons per second above 13.6 eV of a black body of bolometric
    luminosity L: L / (k T) times the photon integral of x^2 / (e^x - 1)
    above x0 = 13.6 eV / kT (64-point Gauss-Legendre on [x0, x0 + 60]) over
    the energy integral pi^4 / 15."""
    kT_eV = 8.617333262e-5 * T_K
    x0 = 13.6 / kT_eV
    xg, wg = np.polynomial.legendre.leggauss(64)
    a, b = x0, x0 + 60.0
    x = 0.5 * (b - a) * xg + 0.5 * (b + a)
    num = 0.5 * (b - a) * np.sum(wg * x * x / np.expm1(x))
    return L_erg_s / (kT_eV * 1.602176634e-12) * num / (np.pi ** 4 / 15.0)


def cloudy_hhe(n: int = 64, packets: int = 6_666_667, steps: int = 30) -> Workload:
    """Test-3-like H II region in H+He (Sec. 4.2.3): uniform n = 1 cm^-3 of
    90% H and 10% He by number, T from 100 K, a 6e4 K black body of 1e38
    erg/s at the centre of a 128 pc box of n^3 cells, 8 bins; 6e5 yr in
    `steps` steps, the paper's 2e8 packets spread over them.  Readings: the
    source sits at the centre and x_HII0 = 1.2e-3 as in the other tests."""
    E, f = blackbody_bins(6e4)
    bE, bf = _bins_for(1, E, f)
    box = Box(n=n, box_cm=128.0 * 3.0857e18, nH=None, nH0=0.9, he_over_h=0.1 / 0.9,
              x_HII0=1.2e-3, x_HeII0=0.0, x_HeIII0=0.0, T0=100.0,
              isothermal=0, caseB=1, z_compton=-1.0, seed=SEED_BASE + 9,
              src_pos=np.array([[n / 2, n / 2, n / 2]]),
              src_ndot=np.array([blackbody_ionising_rate(1e38, 6e4)]),
              bin_eV=bE, bin_frac=bf)
    return Workload(f"cloudy_hhe_{n}^3_1src_8bin", [box], [packets], steps,
                    6e5 * 3.15576e7 / steps, "fp64")


def hhe_blackbody_128(n: int = 128, packets: int = 10_000_000, steps: int = 50) -> Workload:
    """Test-2-like H+He expansion (Sec. 4.2.2) in a 6.6 kpc box of 128^3 cells,
    He/H = 0.08, T evolving from 100 K, corner 1e5 K black-body source of
    5e48 photons/s in 8 bins, 1e7 packets per step, 50 steps of 0.2 Myr."""
    E, f = blackbody_bins(1e5)
    bE, bf = _bins_for(1, E, f)
    box = Box(n=n, box_cm=6.6 * KPC_CM, nH=None, nH0=1e-3, he_over_h=0.08,
              x_HII0=1.2e-3, x_HeII0=0.0, x_HeIII0=0.0, T0=100.0,
              isothermal=0, caseB=1, z_compton=-1.0, seed=SEED_BASE + 2,
              src_pos=np.zeros((1, 3)), src_ndot=np.array([5e48]),
              bin_eV=bE, bin_frac=bf)
    return Workload("hhe_bb_128^3_1src_8bin", [box], [packets], steps,
                    0.2 * MYR_S, "fp64")


def _lognormal_box(n, box_cm, sigma_ln, mean_nH, n_src, lmin, lmax, seed,
                   z_compton=9.0, thin=False) -> Box:
    nH = lognormal_field(n, sigma_ln, mean_nH, seed)
    lin = densest_cells(nH, n_src)
    pos = cell_centres(lin, n, n)
    ndot = powerlaw_luminosities(n_src, lmin, lmax, seed + 1)
    E, f = blackbody_bins(1e5)
    bE, bf = _bins_for(n_src, E, f)
    x0 = (1.0 - 1e-4) if thin else 1.2e-3
    return Box(n=n, box_cm=box_cm, nH=nH, nH0=mean_nH, he_over_h=0.08,
               x_HII0=x0, x_HeII0=1e-4 if thin else 0.0,
               x_HeIII0=(1.0 - 2e-4) if thin else 0.0,
               T0=1e4 if thin else 100.0, isothermal=0, caseB=1,
               z_compton=z_compton, seed=seed, src_pos=pos, src_ndot=ndot,
               bin_eV=bE, bin_frac=bf)


def lognormal_128(n: int = 128, n_src: int = 1000, packets: int = 200_000_000,
                  thin: bool = False) -> Workload:
    """Test-4-like many-source field (Sec. 4.2.4): 128^3 lognormal stand-in
    (sigma_ln = 1.0, mean n_H = 1e-3, He/H = 0.08), 1000 sources at the
    densest cells with L from dN/dL ~ L^-2 on [1e46, 1e50] photons/s, 8-bin
    1e5 K black body, 2e8 packets per step, 10 steps of 0.02 Myr, mixed."""
    box = _lognormal_box(n, 6.6 * KPC_CM, 1.0, 1e-3, n_src, 1e46, 1e50,
                         SEED_BASE + 3, thin=thin)
    return Workload(f"lognormal_{n}^3_{n_src}src_8bin" + ("_thin" if thin else ""),
                    [box], [packets], 10, 0.02 * MYR_S, "mixed")


def lognormal_512(n: int = 512, n_src: int = 10_000, packets: int = 1_000_000_000,
                  thin: bool = True) -> Workload:
    """The 1000-source-run-like large field (Sec. 5.2), scaled: 512^3
    lognormal stand-in (sigma_ln = 1.5, mean n_H = 2e-4, He/H = 0.08) in a
    100 Mpc/h comoving box at z = 9 (h = 0.7), 1e4 power-law sources, 8-bin
    black body, 1e9 packets per step, 10 steps of 0.1 Myr, mixed precision.
    `thin` starts from the paper's optically thin idealisation (Sec. 5.3):
    x_HI = x_HeI = x_HeII = 1e-4 in every cell."""
    box_cm = 100.0 / 0.7 * MPC_CM / (1.0 + 9.0)
    box = _lognormal_box(n, box_cm, 1.5, 2e-4, n_src, 1e46, 1e50,
                         SEED_BASE + 5, thin=thin)
    return Workload(f"lognormal_{n}^3_{n_src}src_8bin" + ("_thin" if thin else "_neutral"),
                    [box], [packets], 10, 0.1 * MYR_S, "mixed")


def batch_64(n_boxes: int = 64, seed: int = SEED_BASE + 4, scale: float = 1.0) -> Workload:
    """64 independent lognormal boxes with sizes from {32,48,64,96,128}^3,
    1-100 power-law sources each and log-uniform 1e5-1e7 packets per step
    (rounded to a multiple of the box's source count), mixed precision.
    `scale` multiplies every box's packet count (for small tests)."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([32, 48, 64, 96, 128], size=n_boxes)
    boxes, packets = [], []
    for b in range(n_boxes):
        n = int(sizes[b])
        n_src = int(rng.integers(1, 101))
        p = int(10 ** rng.uniform(5, 7) * scale)
        p = max(n_src, (p // n_src) * n_src)
        box_cm = 6.6 * KPC_CM * n / 128.0
        boxes.append(_lognormal_box(n, box_cm, 1.0, 1e-3, n_src, 1e46, 1e50,
                                    seed + 1000 * (b + 1)))
        packets.append(p)
    return Workload(f"batch_{n_boxes}_boxes_32-128^3", boxes, packets, 10,
                    0.02 * MYR_S, "mixed")


def thin_state(box: Box) -> Box:
    """The optically thin idealisation: every cell ionised so that the
    neutral H, neutral He and He II fractions are each 1e-4."""
    box.x_HII0 = 1.0 - 1e-4
    box.x_HeII0 = 1e-4
    box.x_HeIII0 = 1.0 - 2e-4
    box.T0 = 1e4
    return box
