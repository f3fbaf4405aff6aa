"""crash_autotune on a small mixed-form box: it returns the configuration it
keeps (crash_get_options reads the same values back, the launch style
included), it leaves no trace in the state, the diffuse field's counts or
the step index, and a step with the tuned options gives the same bits as a
step with the default ones (results do not depend on the launch shape)."""
import numpy as np
import pytest

from paper_1101_4127_gb300 import inputs, native
from _common import DEP_FIELDS, STATE_FIELDS, small_hhe_box

pytestmark = pytest.mark.gpu


def _fields(g):
    return [g.read(f) for f, _ in STATE_FIELDS + DEP_FIELDS] + [g.read(native.F_BUDGET)]


def test_autotune_keeps_its_choice_and_leaves_no_trace():
    box = small_hhe_box((40, 36, 33), n_src=4, seed=501, thin=True)
    P = 4 * 20000
    dt = 0.05 * inputs.MYR_S
    g = native.Grid(box, native.CRASH_MIXED)
    g.step(dt, P)                                   # a state that is not the initial one
    before = [g.read(f) for f, _ in STATE_FIELDS]
    tuned = g.autotune(dt, [P])
    after = [g.read(f) for f, _ in STATE_FIELDS]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    o = g.get_options()
    assert (o["block_size"], o["seg_per_iter"], o["resort_interval"], o["reg_cap"], o["tile"],
            o["sort_curve"]) == tuple(tuned)
    assert o["persistent"] in (0, 1) and o["chemistry"] == 1
    assert o["pkt_begin"] == 0 and o["pkt_end"] == 0xFFFFFFFF    # trial windows are not kept
    g.step(dt, P)
    ref = native.Grid(box, native.CRASH_MIXED)
    ref.step(dt, P)
    ref.step(dt, P)
    for a, b in zip(_fields(g), _fields(ref)):
        assert np.array_equal(a, b)
