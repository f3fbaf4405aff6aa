"""Helpers shared by the parity tests: run the same seeded workload through
the CUDA library and the CPU oracle."""
import numpy as np

import oracle
from paper_1101_4127_gb300 import inputs, native

DEP_FIELDS = [(native.F_DEP_HI, oracle.F_DEP_HI), (native.F_DEP_HEI, oracle.F_DEP_HEI),
              (native.F_DEP_HEII, oracle.F_DEP_HEII), (native.F_DEP_E, oracle.F_DEP_E)]
STATE_FIELDS = [(native.F_XHII, oracle.F_XHII), (native.F_XHEII, oracle.F_XHEII),
                (native.F_XHEIII, oracle.F_XHEIII), (native.F_T, oracle.F_T)]


def pair(box, precision=native.CRASH_FP64_PLAIN):
    return native.Grid(box, precision), oracle.OracleGrid.from_box(box)


def assert_deposits_equal(g, o, box=0):
    for fg, fo in DEP_FIELDS:
        a, b = g.read(fg, box), o.read(fo)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"deposit field {fg}: {len(bad)} cells differ, first {bad[:3].tolist()} "
                                 f"gpu={a[tuple(bad[0])]} oracle={b[tuple(bad[0])]}")
    bg, bo = g.read(native.F_BUDGET, box), o.read(oracle.F_BUDGET)
    assert np.array_equal(bg[:7], bo[:7]), (bg, bo)


def max_rel(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.maximum(np.abs(b), floor)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(den > 0, np.abs(a - b) / den, np.abs(a - b))
    return float(np.max(r))


def copy_state(src_oracle, dst_grid, box=0):
    for fg, fo in STATE_FIELDS:
        dst_grid.write(fg, src_oracle.read(fo), box)


def small_hhe_box(n=(16, 16, 16), n_src=3, seed=21, nbins=8, thin=False, T0=100.0):
    """Lognormal H+He box with a few sources (odd sizes allowed)."""
    rng = np.random.default_rng(seed)
    nx = n[0]
    nH = inputs.lognormal_field(nx, 1.0, 1e-3, seed)[: n[2], : n[1], : n[0]]
    E, f = inputs.blackbody_bins(1e5)
    if nbins == 1:
        E, f = np.array([20.0]), np.array([1.0])
    pos = np.stack([rng.uniform(0, n[0], n_src), rng.uniform(0, n[1], n_src),
                    rng.uniform(0, n[2], n_src)], axis=1)
    return inputs.Box(n=nx, box_cm=6.6 * inputs.KPC_CM * nx / 128, nH=np.ascontiguousarray(nH),
                      nH0=1e-3, he_over_h=0.08, x_HII0=(1 - 1e-4) if thin else 1.2e-3,
                      x_HeII0=1e-4 if thin else 0.0, x_HeIII0=(1 - 2e-4) if thin else 0.0,
                      T0=1e4 if thin else T0, isothermal=0, caseB=1, z_compton=9.0, seed=seed,
                      src_pos=pos, src_ndot=rng.uniform(1e47, 1e49, n_src), bin_eV=E,
                      bin_frac=np.tile(f, (n_src, 1)), dims=tuple(n))
