"""Measured accuracy of the mixed form (FP32 traversal and attenuation, int64
deposits, FP64 chemistry) against the FP64 oracle, per state field and for
the ionisation-front radius, on the workloads' own layouts:

  * Test 0 (32^3, one corner source, 20 steps of 0.5 Myr) in full;
  * the 128^3 H+He black-body workload (1e7 packets per step) and the 128^3
    lognormal 1000-source workload (2e8 packets per step), three coupled
    steps over a window of packet ids of every source (the contents are those
    of the full step);
  * the per-cell deposits of one step of those windows.

Each test asserts the mixed form's bounds (fields within 1e-4 relative above
a floor of 1e-6, front within 0.5 cell) and the measured statistics; with
CRASH_ACCURACY_OUT set, it also appends its table to that JSON-lines file."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1101_4127_gb300 import inputs, native
from _common import DEP_FIELDS, STATE_FIELDS

pytestmark = pytest.mark.gpu
MIXED = native.CRASH_MIXED
FIELD_TOL = 1e-4
FLOOR = 1e-6
NAMES = ["x_HII", "x_HeII", "x_HeIII", "T"]


def _report(name, table):
    path = os.environ.get("CRASH_ACCURACY_OUT")
    line = json.dumps({"workload": name, **table})
    print(line)
    if path:
        with open(path, "a") as f:
            f.write(line + "\n")


def _field_errors(g, o):
    """Per field: relative error against max(|oracle|, 1e-6) (max, median,
    99th percentile), the largest relative error over the cells where the
    oracle's value is at least 1e-4 and 1e-3, and the largest absolute error."""
    out = {}
    for (fg, fo), nm in zip(STATE_FIELDS, NAMES):
        a, b = g.read(fg).astype(np.float64).ravel(), o.read(fo).astype(np.float64).ravel()
        d = np.abs(a - b)
        r = d / np.maximum(np.abs(b), FLOOR)
        e = {"max_rel": float(r.max()), "median_rel": float(np.median(r)),
             "p99_rel": float(np.quantile(r, 0.99)), "max_abs": float(d.max())}
        for lim in (1e-4, 1e-3):
            big = np.abs(b) >= lim
            e[f"max_rel_where_ge_{lim:g}"] = float((d[big] / np.abs(b[big])).max()) if big.any() else 0.0
        out[nm] = e
    return out


def _front(x, x0, octant):
    return (3 * (8 if octant else 1) * (x - x0).sum() / (4 * math.pi)) ** (1 / 3)


def _deposit_stats(g, o):
    """Per-cell relative difference of the deposits where the oracle's
    deposit is at least 1e-3 of the largest (the cells that carry the
    step's absorption), and the share of the absorbed photons in the cells
    below that floor."""
    out = {}
    for (fg, fo), nm in zip(DEP_FIELDS, ["HI", "HeI", "HeII", "heat"]):
        a, b = g.read(fg).astype(np.float64).ravel(), o.read(fo).astype(np.float64).ravel()
        if b.max() <= 0:
            continue
        big = b >= 1e-3 * b.max()
        r = np.abs(a[big] - b[big]) / b[big]
        out[nm] = {"cells": int(big.sum()), "median_rel": float(np.median(r)),
                   "p99_rel": float(np.quantile(r, 0.99)), "max_rel": float(r.max()),
                   "share_below_floor": float(b[~big].sum() / b.sum()),
                   "sum_rel": float(abs(a.sum() - b.sum()) / b.sum())}
    return out


def test_mixed_accuracy_test0_full_run():
    w = inputs.stromgren_32()
    box = w.boxes[0]
    g = native.Grid(box, MIXED)
    o = oracle.OracleGrid.from_box(box)
    fronts = []
    for _ in range(w.n_steps):
        g.step(w.dt_s, w.packets_per_step[0])
        o.step(w.dt_s, w.packets_per_step[0])
        fronts.append(_front(g.read(native.F_XHII), box.x_HII0, True) -
                      _front(o.read(oracle.F_XHII), box.x_HII0, True))
    err = _field_errors(g, o)
    _report(w.name, {"steps": w.n_steps, "fields": {"x_HII": err["x_HII"]},
                     "front_offset_cells_max": float(np.max(np.abs(fronts))),
                     "front_offset_cells_last": float(fronts[-1])})
    assert err["x_HII"]["max_rel"] < FIELD_TOL
    assert np.max(np.abs(fronts)) < 0.5


@pytest.mark.parametrize("name", ["hhe_bb_128", "lognormal_128"])
def test_mixed_accuracy_128_windows(name):
    w = inputs.hhe_blackbody_128() if name == "hhe_bb_128" else inputs.lognormal_128()
    box = w.boxes[0]
    P = w.packets_per_step[0]
    K = 20000 // box.n_src                      # packet ids [0, K) of every source
    g = native.Grid(box, MIXED)
    o = oracle.OracleGrid.from_box(box)
    for s in (g, o):
        s.set_options(pkt_begin=0, pkt_end=K)
    dt = w.dt_s
    steps = 3
    dep = None
    for k in range(steps):
        if k == 0:                                # deposits of the first step, before chemistry
            for s in (g, o):
                s.set_options(chemistry=0, pkt_begin=0, pkt_end=K)
            g.step(dt, P)
            o.step(dt, P)
            dep = _deposit_stats(g, o)
            g.set_step_index(0)
            o.set_step_index(0)
            for s in (g, o):
                s.set_options(chemistry=1, pkt_begin=0, pkt_end=K)
        g.step(dt, P)
        o.step(dt, P)
    err = _field_errors(g, o)
    bg, bo = g.read(native.F_BUDGET), o.read(oracle.F_BUDGET)
    _report(name + "_window", {"steps": steps, "packet_ids": [0, K], "fields": err, "deposits": dep,
                               "absorbed_rel": float(abs(bg[1] - bo[1]) / bo[0]),
                               "crossings_rel": float(abs(bg[3] - bo[3]) / bo[3])})
    for nm in NAMES:
        assert err[nm]["max_rel_where_ge_0.0001"] < FIELD_TOL, (nm, err[nm])
        assert err[nm]["p99_rel"] < FIELD_TOL, (nm, err[nm])
    for nm, d in dep.items():
        assert d["sum_rel"] < 1e-4, (nm, d)
        assert d["median_rel"] < 1e-4, (nm, d)
        assert d["max_rel"] < 1e-4, (nm, d)        # every cell above the floor
