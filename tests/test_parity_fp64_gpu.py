"""FP64 form on the GPU against the CPU oracle, element by element, through
the C ABI.  Deposits (int64) must be bit-identical from an identical input
state; fields within 1e-9 relative after several coupled steps."""
import math

import numpy as np
import pytest

import oracle
from paper_1101_4127_gb300 import inputs, native
from _common import (DEP_FIELDS, STATE_FIELDS, assert_deposits_equal, copy_state, max_rel,
                     pair, small_hhe_box)

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-9


def test_stromgren_32_step1_deposits_bit_exact():
    w = inputs.stromgren_32()
    g, o = pair(w.boxes[0])
    g.set_options(chemistry=0)
    o.set_options(chemistry=0)
    g.step(w.dt_s, w.packets_per_step[0])
    o.step(w.dt_s, w.packets_per_step[0])
    assert_deposits_equal(g, o)
    b = g.read(native.F_BUDGET)
    assert b[0] == b[1] + b[2] and b[4] == 100000


def test_stromgren_32_all_steps_fields_and_per_step_deposits():
    """20 steps of 0.5 Myr: at every step the transport from the oracle's
    state is bit-exact, and the coupled fields stay within 1e-9."""
    w = inputs.stromgren_32()
    g, o = pair(w.boxes[0])
    gt = native.Grid(w.boxes[0])          # transport-only twin fed the oracle's state
    gt.set_options(chemistry=0)
    for k in range(w.n_steps):
        copy_state(o, gt)
        gt.set_step_index(k)
        gt.step(w.dt_s, w.packets_per_step[0])
        o.step(w.dt_s, w.packets_per_step[0])
        assert_deposits_equal(gt, o)
        g.step(w.dt_s, w.packets_per_step[0])
        bg = g.read(native.F_BUDGET)
        assert bg[0] == bg[1] + bg[2]
    for fg, fo in STATE_FIELDS:
        assert max_rel(g.read(fg), o.read(fo)) < FIELD_TOL, fg


@pytest.mark.parametrize("dims,n_src,P,nbins", [
    ((16, 16, 16), 3, 3 * 1000, 8),
    ((13, 7, 5), 2, 2 * 777, 8),        # ragged grid, packets not a multiple of 32
    ((9, 9, 9), 5, 5 * 33, 1),          # one bin above the He I threshold
    ((24, 17, 11), 7, 7 * 4099, 8),
])
def test_hhe_deposits_bit_exact_and_fields(dims, n_src, P, nbins):
    box = small_hhe_box(dims, n_src=n_src, seed=sum(dims) + n_src, nbins=nbins)
    g, o = pair(box)
    gt = native.Grid(box)
    gt.set_options(chemistry=0)
    dt = 0.01 * inputs.MYR_S
    for k in range(4):
        copy_state(o, gt)
        gt.set_step_index(k)
        gt.step(dt, P)
        o.step(dt, P)
        assert_deposits_equal(gt, o)
        g.step(dt, P)
    for fg, fo in STATE_FIELDS:
        assert max_rel(g.read(fg), o.read(fo), floor=1e-30) < FIELD_TOL, fg


def test_edge_sources_and_windows():
    """Sources on the lower faces and corners, a dark source, one packet per
    source, and a packet-id window: all bit-exact."""
    box = small_hhe_box((10, 10, 10), n_src=4, seed=3)
    box.src_pos = np.array([[0.0, 0.0, 0.0], [9.999999, 0.0, 5.0], [0.0, 9.5, 9.999], [5.5, 5.5, 5.5]])
    box.src_ndot = np.array([1e48, 3e48, 0.0, 2e47])
    g, o = pair(box)
    for (P, win) in [(4, (0, 0xFFFFFFFF)), (4 * 500, (0, 0xFFFFFFFF)), (4 * 500, (123, 321))]:
        g.set_options(chemistry=0, pkt_begin=win[0], pkt_end=win[1])
        o.set_options(chemistry=0, pkt_begin=win[0], pkt_end=win[1])
        g.step(0.02 * inputs.MYR_S, P)
        o.step(0.02 * inputs.MYR_S, P)
        assert_deposits_equal(g, o)


def test_batch_of_boxes_matches_independent_oracles():
    boxes = [small_hhe_box((12, 12, 12), n_src=2, seed=40),
             small_hhe_box((7, 5, 3), n_src=1, seed=41),
             small_hhe_box((16, 9, 4), n_src=3, seed=42)]
    P = [2 * 900, 1 * 55, 3 * 1201]
    g = native.Grid(boxes)
    os_ = [oracle.OracleGrid.from_box(b) for b in boxes]
    dt = 0.01 * inputs.MYR_S
    for k in range(2):
        g.step(dt, P)
        for i, o in enumerate(os_):
            o.step(dt, P[i])
    for i, o in enumerate(os_):
        for fg, fo in STATE_FIELDS:
            assert max_rel(g.read(fg, i), o.read(fo), floor=1e-30) < FIELD_TOL
        bg, bo = g.read(native.F_BUDGET, i), o.read(oracle.F_BUDGET)
        assert bg[0] == bg[1] + bg[2] and bg[4] == bo[4]


def test_batch_transport_bit_exact_per_box():
    boxes = [small_hhe_box((12, 12, 12), n_src=2, seed=50),
             small_hhe_box((8, 8, 8), n_src=4, seed=51)]
    P = [2 * 1500, 4 * 333]
    g = native.Grid(boxes)
    g.set_options(chemistry=0)
    g.step(0.01 * inputs.MYR_S, P)
    for i, b in enumerate(boxes):
        o = oracle.OracleGrid.from_box(b)
        o.set_options(chemistry=0)
        o.step(0.01 * inputs.MYR_S, P[i])
        assert_deposits_equal(g, o, box=i)


def test_hhe_128_full_size_sampled_window_bit_exact():
    """The 128^3 H+He black-body workload at its full packet count and launch
    configuration: a window of packet ids traced by both sides is
    bit-identical, and the full step closes its photon budget."""
    w = inputs.hhe_blackbody_128()
    box = w.boxes[0]
    P = w.packets_per_step[0]
    g = native.Grid(box)
    g.step(w.dt_s, P)                          # one full coupled step (state now evolved)
    b = g.read(native.F_BUDGET)
    assert b[0] == b[1] + b[2] and b[4] == P
    o = oracle.OracleGrid.from_box(box)
    copy_state_from_grid(g, o)
    for gi in (g,):
        gi.set_options(chemistry=0, pkt_begin=1000, pkt_end=1000 + 20000)
    o.set_options(chemistry=0, pkt_begin=1000, pkt_end=1000 + 20000)
    o.set_step_index(1)
    g.step(w.dt_s, P)
    o.step(w.dt_s, P)
    assert_deposits_equal(g, o)


def copy_state_from_grid(g, o):
    for fg, fo in STATE_FIELDS:
        o.write(fo, g.read(fg))


def test_resume_from_fields_and_step_index_is_bit_identical():
    box = small_hhe_box((12, 12, 12), n_src=2, seed=60)
    P = 2 * 1000
    dt = 0.01 * inputs.MYR_S
    g1 = native.Grid(box)
    for _ in range(3):
        g1.step(dt, P)
    g2 = native.Grid(box)
    for _ in range(2):
        g2.step(dt, P)
    g3 = native.Grid(box)            # resume from g2's checkpoint
    for fg, _ in STATE_FIELDS:
        g3.write(fg, g2.read(fg))
    g3.set_step_index(2)
    g3.step(dt, P)
    for fg, _ in STATE_FIELDS:
        assert np.array_equal(g1.read(fg), g3.read(fg))
    for fg, _ in DEP_FIELDS:
        assert np.array_equal(g1.read(fg), g3.read(fg))


def test_graph_replay_matches_plain_launches():
    box = small_hhe_box((12, 12, 12), n_src=2, seed=70)
    P = 2 * 1000
    dt = 0.01 * inputs.MYR_S
    a = native.Grid(box)
    b = native.Grid(box)
    b.set_options(use_graph=1)
    for _ in range(3):
        a.step(dt, P)
        b.step(dt, P)
    for fg, _ in STATE_FIELDS + DEP_FIELDS:
        assert np.array_equal(a.read(fg), b.read(fg))


def test_device_checkpoint_restore_repeats_step_bit_for_bit():
    box = small_hhe_box((12, 10, 8), n_src=2, seed=80)
    P = 2 * 1000
    dt = 0.01 * inputs.MYR_S
    for prec in (native.CRASH_FP64_PLAIN, native.CRASH_MIXED):
        g = native.Grid(box, prec)
        g.step(dt, P)
        g.checkpoint(native.CKPT_SAVE)
        g.step(dt, P)
        first = [g.read(f) for f, _ in STATE_FIELDS + DEP_FIELDS]
        g.checkpoint(native.CKPT_RESTORE)           # state and step index
        g.step(dt, P)
        again = [g.read(f) for f, _ in STATE_FIELDS + DEP_FIELDS]
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
        g.checkpoint(native.CKPT_RESTORE_STATE)     # state only: new directions
        g.step(dt, P)
        other = g.read(native.F_DEP_HI)
        assert not np.array_equal(other, first[4])
        b = g.read(native.F_BUDGET)
        assert b[0] == b[1] + b[2]
