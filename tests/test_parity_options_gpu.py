"""GPU parity of the options beyond the default step and of the exchange of
a split step, through the C ABI against the CPU oracle:

  * photon-conserving coupling: FP64 deposits bit-exact, fields within 1e-9
    over coupled steps; mixed form within 1e-4;
  * periodic boxes: FP64 deposits and budget bit-exact, fields within 1e-9;
    mixed form within its tolerance, the budget exact, launch shapes alike;
  * a step split by packet-id windows over several contexts (the stand-in
    for several processes), deposits summed on the host or on the device,
    then crash_chemistry: the same bits as one context tracing every packet;
  * the mixed wavefront crossing its chunk boundary with re-sort on: the same
    bits as one thread per packet."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1101_4127_gb300 import inputs, native
from _common import DEP_FIELDS, STATE_FIELDS, assert_deposits_equal, copy_state, max_rel, small_hhe_box
from test_mixed_accuracy_gpu import FIELD_TOL, NAMES, _field_errors

pytestmark = pytest.mark.gpu
FP64, MIXED = native.CRASH_FP64_PLAIN, native.CRASH_MIXED
C_LIGHT = 2.99792458e10


def _pair(box, precision):
    return native.Grid(box, precision), oracle.OracleGrid.from_box(box)


# ------------------------------------------------ photon-conserving coupling
def test_photon_conserving_coupling_fp64_against_oracle():
    """Every step from the oracle's state: the deposits bit for bit, the
    fields after the photon-conserving update within 1e-8 relative (above
    1e-2; 1e-10 absolute below).  Where a constant source has used up its
    species the fraction left is set by the last sub-steps (about h R y): on
    the CPU a 1e-15 change of the state moves it by up to 6e-10 relative, so
    the differences between the two machines' roundings (FMA contraction,
    reciprocals, libm) exceed the default coupling's 1e-9."""
    box = dataclasses.replace(small_hhe_box((14, 12, 10), n_src=3, seed=401), coupling=1)
    P = 3 * 3000
    dt = 0.5 * inputs.MYR_S
    g, o = _pair(box, FP64)
    for k in range(4):
        copy_state(o, g)
        g.step(dt, P)
        o.step(dt, P)
        assert_deposits_equal(g, o)
        for fg, fo in STATE_FIELDS:
            assert max_rel(g.read(fg), o.read(fo), floor=1e-2 if fg != native.F_T else 1e-300) < 1e-8, (k, fg)


def test_photon_conserving_coupling_mixed_against_oracle():
    """The mixed form under the photon-conserving coupling.  Its deposits
    differ from the oracle's by about 1e-7; where a constant source uses up
    its species the fraction left depends on the sub-steps (the constant
    source has no equilibrium there), and that 1e-7 moves the small He II
    fraction of such cells by up to about 6e-4 and their temperature by up to
    about 4e-4 relative.  Bounds: x_HII within 1e-4 relative (above 1e-4), T
    within 1e-3, He fractions within 1e-3 absolute, the summed He III within
    1e-5."""
    box = dataclasses.replace(small_hhe_box((16, 16, 16), n_src=4, seed=402), coupling=1)
    P = 4 * 5000
    dt = 0.2 * inputs.MYR_S
    g, o = _pair(box, MIXED)
    for _ in range(3):
        g.step(dt, P)
        o.step(dt, P)
    b = g.read(native.F_BUDGET)
    assert b[0] == b[1] + b[2]
    err = _field_errors(g, o)
    assert err["x_HII"]["max_rel_where_ge_0.0001"] < FIELD_TOL, err["x_HII"]
    assert err["T"]["max_rel"] < 1e-3 and err["T"]["p99_rel"] < FIELD_TOL, err["T"]
    for nm in ("x_HeII", "x_HeIII"):
        assert err[nm]["max_abs"] < 1e-3, (nm, err[nm])
    a, b = g.read(native.F_XHEIII).sum(), o.read(oracle.F_XHEIII).sum()
    assert abs(a - b) <= 1e-5 * b


# ------------------------------------------------------------ periodic box
def _periodic_box(n=(14, 12, 10), seed=411, path_cells=25.0, thin=True):
    box = dataclasses.replace(small_hhe_box(n, n_src=3, seed=seed, thin=thin), periodic=1)
    dl = box.box_cm / n[0]
    return box, path_cells * dl / C_LIGHT


def test_periodic_fp64_deposits_bit_exact_and_fields_close():
    box, dt = _periodic_box()
    P = 3 * 2000
    g, o = _pair(box, FP64)
    for _ in range(3):
        copy_state(o, g)
        g.step(dt, P)
        o.step(dt, P)
        assert_deposits_equal(g, o)
        b = g.read(native.F_BUDGET)
        assert b[0] == b[1] + b[2]
        for fg, fo in STATE_FIELDS:
            assert max_rel(g.read(fg), o.read(fo), floor=1e-300) < 1e-9, fg


def test_periodic_mixed_against_oracle_and_launch_shapes():
    box, dt = _periodic_box(seed=412)
    P = 3 * 4000
    ref = None
    for opts in (dict(wavefront=0), dict(wavefront=1), dict(wavefront=1, use_graph=1)):
        g = native.Grid(box, MIXED)
        g.set_options(chemistry=0, **opts)
        g.step(dt, P)
        got = [g.read(f) for f, _ in DEP_FIELDS] + [g.read(native.F_BUDGET)]
        if ref is None:
            ref = got
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), opts
    o = oracle.OracleGrid.from_box(box)
    o.set_options(chemistry=0)
    o.step(dt, P)
    bg, bo = ref[-1], o.read(oracle.F_BUDGET)
    assert bg[0] == bg[1] + bg[2]
    assert abs(bg[0] - bo[0]) <= 1e-8 * bo[0]
    assert abs(bg[1] - bo[1]) <= 1e-4 * bo[0]
    assert abs(bg[3] - bo[3]) <= 2e-3 * bo[3]
    a = ref[0].astype(np.float64)
    b = o.read(oracle.F_DEP_HI).astype(np.float64)
    assert abs(a.sum() - b.sum()) <= 1e-4 * b.sum()


def test_periodic_box_rejects_a_light_path_beyond_its_bound():
    box, _ = _periodic_box()
    g = native.Grid(box, FP64)
    with pytest.raises(native.CrashError) as ei:
        g.step(1e30, 3)
    assert ei.value.status == native.CRASH_ERR_ARG


# ------------------------------------------------------- split-step exchange
def _split_run(box, precision, P, dt, windows, device_sum=False):
    """Each window traced by its own context (chemistry off); deposits summed
    into the first context, which then runs the per-cell update."""
    Ns = P // box.n_src
    grids = []
    for lo, hi in windows:
        g = native.Grid(box, precision)
        g.set_options(chemistry=0, pkt_begin=lo, pkt_end=min(hi, Ns))
        g.step(dt, P)
        grids.append(g)
    if device_sum:
        torch = pytest.importorskip("torch")

        class _Dev:
            def __init__(self, ptr, n):
                self.__cuda_array_interface__ = {"shape": (n, 4), "typestr": "<i8",
                                                 "data": (ptr, False), "version": 2}
        for g in grids:
            g.sync()
        ts = [torch.as_tensor(_Dev(*g.deposits_device()), device="cuda") for g in grids]
        for t in ts[1:]:
            ts[0] += t                # the all-reduce of the exchange, in place
        torch.cuda.synchronize()
    else:
        total = sum(g.read_deposits() for g in grids)
        grids[0].write_deposits(total)
    grids[0].chemistry(dt)
    return grids[0]


@pytest.mark.parametrize("precision", [FP64, MIXED])
@pytest.mark.parametrize("device_sum", [False, True])
def test_split_step_with_exchange_equals_one_run(precision, device_sum):
    box = small_hhe_box((16, 12, 14), n_src=4, seed=421)
    P = 4 * 2500
    dt = 0.05 * inputs.MYR_S
    full = native.Grid(box, precision)
    full.step(dt, P)
    split = _split_run(box, precision, P, dt, [(0, 700), (700, 1900), (1900, 2500)], device_sum)
    for f, _ in STATE_FIELDS:
        assert np.array_equal(split.read(f), full.read(f)), f
    assert np.array_equal(split.read_deposits(), full.read_deposits())


def test_chemistry_call_needs_a_transport_only_step():
    box = small_hhe_box((8, 8, 8), n_src=1, seed=422)
    g = native.Grid(box, FP64)
    with pytest.raises(native.CrashError) as ei:
        g.chemistry(1e12)
    assert ei.value.status == native.CRASH_ERR_STATE
    g.set_options(chemistry=0)
    g.step(1e12, 100)
    with pytest.raises(native.CrashError) as ei:
        g.chemistry(2e12)                      # not the step's dt
    assert ei.value.status == native.CRASH_ERR_ARG
    g.chemistry(1e12)
    with pytest.raises(native.CrashError) as ei:
        g.chemistry(1e12)                      # once only
    assert ei.value.status == native.CRASH_ERR_STATE


# ------------------------------------------------------- wavefront chunks
def test_mixed_chunks_with_resort_equal_one_thread_per_packet():
    """Small wavefront chunks (several per step) with re-sort every pass and
    both key curves: the same bits as one thread per packet."""
    box = small_hhe_box((20, 18, 16), n_src=3, seed=431, thin=True)
    P = 3 * 9001
    dt = 0.01 * inputs.MYR_S

    def run(**opts):
        g = native.Grid(box, MIXED)
        g.set_options(**opts)
        for _ in range(2):
            g.step(dt, P)
        return [g.read(f) for f, _ in STATE_FIELDS + DEP_FIELDS] + [g.read(native.F_BUDGET)]

    ref = run(wavefront=0)
    for opts in (dict(chunk_packets=4096, resort_interval=1, seg_per_iter=8),
                 dict(chunk_packets=5000, resort_interval=2, seg_per_iter=16, sort_curve=1),
                 dict(chunk_packets=7777, resort_interval=1, seg_per_iter=32, tile=1)):
        got = run(wavefront=1, **opts)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), opts


# ------------------------------------------------------- uniform background
def _uv_box(seed):
    return dataclasses.replace(small_hhe_box((14, 12, 10), n_src=2, seed=seed),
                               uv_rate=(2e-13, 8e-14, 3e-15), uv_heat_eV=(4.0, 6.0, 12.0))


def test_uniform_background_fp64_against_oracle():
    """The background adds to the photo-ionisation rates and the heating of
    every cell: FP64 deposits bit-exact (the transport does not see it),
    fields within 1e-9 after each step from the oracle's state."""
    box = _uv_box(441)
    P = 2 * 3000
    dt = 0.1 * inputs.MYR_S
    g, o = _pair(box, FP64)
    for k in range(3):
        copy_state(o, g)
        g.step(dt, P)
        o.step(dt, P)
        assert_deposits_equal(g, o)
        for fg, fo in STATE_FIELDS:
            assert max_rel(g.read(fg), o.read(fo), floor=1e-300) < 1e-9, (k, fg)
    # the background did act: cells with no deposit were ionised
    ref = native.Grid(dataclasses.replace(box, uv_rate=(0.0, 0.0, 0.0), uv_heat_eV=(0.0, 0.0, 0.0)), FP64)
    for _ in range(3):
        ref.step(dt, P)
    assert g.read(native.F_XHII).min() > 10 * ref.read(native.F_XHII).min()


def test_uniform_background_mixed_against_oracle():
    box = _uv_box(442)
    P = 2 * 4000
    dt = 0.1 * inputs.MYR_S
    g, o = _pair(box, MIXED)
    for _ in range(3):
        g.step(dt, P)
        o.step(dt, P)
    err = _field_errors(g, o)
    for nm in NAMES:
        assert err[nm]["max_rel_where_ge_0.0001"] < FIELD_TOL, (nm, err[nm])
        assert err[nm]["p99_rel"] < FIELD_TOL, (nm, err[nm])


@pytest.mark.parametrize("precision", [FP64, MIXED])
def test_dark_sources_under_the_background_alone(precision):
    """Degenerate step: every source emits nothing (the photon quantum falls
    back to 2^0), so every deposit is zero and the budget holds no photons;
    the background alone updates the cells, as in the oracle."""
    box = dataclasses.replace(_uv_box(451), src_ndot=np.zeros(2))
    P = 2 * 512
    dt = 0.2 * inputs.MYR_S
    g, o = _pair(box, precision)
    for _ in range(2):
        g.step(dt, P)
        o.step(dt, P)
    for f, _ in DEP_FIELDS:
        assert not g.read(f).any(), f
    b = g.read(native.F_BUDGET)
    assert b[0] == b[1] == b[2] == 0 and b[4] == P
    tol = 1e-9 if precision == FP64 else FIELD_TOL
    for fg, fo in STATE_FIELDS:
        assert max_rel(g.read(fg), o.read(fo), floor=1e-6) < tol, fg
