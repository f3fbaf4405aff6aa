"""crash_transport_noalloc: the mixed-form transport of one grid for one step
without any device allocation, for callers that cannot call cudaMalloc (code
inside another framework's memory pool or under a fixed memory budget,
plug-ins that may only use the buffers they are handed).  Its scratch is a
static device array; the caller hands in the absorbers and the deposit
buffer.  Checked through the C ABI against crash_step of a context with the
same grid, sources and options (chemistry off, no re-sort): deposits and
budget must be identical, on two calls in a row.  This file is collected
last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_1101_4127_gb300 import inputs, native
from _common import small_hhe_box

pytestmark = pytest.mark.gpu

DEPS = [native.F_DEP_HI, native.F_DEP_HEI, native.F_DEP_HEII, native.F_DEP_E]


def _absorbers(box):
    """n_HI, n_HeI, n_HeII of the box's uniform initial state, formed in FP64
    and rounded to FP32 as the library's per-step freeze does."""
    nH = np.ascontiguousarray(box.nH, np.float32).reshape(-1).astype(np.float64)
    nHe = nH * box.he_over_h
    a = np.zeros((nH.size, 4), np.float32)
    a[:, 0] = (nH * (1.0 - box.x_HII0)).astype(np.float32)
    a[:, 1] = (nHe * ((1.0 - box.x_HeII0) - box.x_HeIII0)).astype(np.float32)
    a[:, 2] = (nHe * box.x_HeII0).astype(np.float32)
    return a


def test_noalloc_transport_matches_crash_step_two_calls():
    torch = pytest.importorskip("torch")
    box = small_hhe_box((24, 20, 16), n_src=5, seed=301)
    P = 5 * 40001                          # several 65536-packet queue chunks
    dt = 0.01 * inputs.MYR_S
    S = 16
    g = native.Grid(box, native.CRASH_MIXED)
    g.set_options(chemistry=0, wavefront=1, seg_per_iter=S, resort_interval=-1)
    L = native.lib()
    desc = native.make_desc(box, native.CRASH_MIXED)
    pos = np.ascontiguousarray(box.src_pos, np.float64)
    ndot = np.ascontiguousarray(box.src_ndot, np.float64)
    E = np.ascontiguousarray(box.bin_eV, np.float64)
    frac = np.ascontiguousarray(box.bin_frac, np.float64)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    dev = torch.device("cuda", 0)
    absorbers = torch.from_numpy(_absorbers(box)).to(dev)
    ncell = absorbers.shape[0]
    deposits = torch.zeros((ncell, 4), dtype=torch.int64, device=dev)
    for k in range(2):                     # two calls in a row, steps 0 and 1
        g.step(dt, P)
        ref = [g.read(f).reshape(-1) for f in DEPS]
        ref_budget = g.read(native.F_BUDGET)
        deposits.zero_()
        torch.cuda.synchronize()
        budget = np.zeros(8, np.int64)
        st = L.crash_transport_noalloc(C.byref(desc), len(ndot), dp(pos), dp(ndot), len(E), dp(E),
                                       dp(frac), dt, k, P, S, C.c_void_p(absorbers.data_ptr()),
                                       C.c_void_p(deposits.data_ptr()),
                                       budget.ctypes.data_as(C.POINTER(C.c_int64)), None)
        assert st == native.CRASH_OK, L.crash_noalloc_last_error().decode()
        got = deposits.cpu().numpy()
        for i in range(4):
            assert np.array_equal(got[:, i], ref[i]), (k, i)
        assert np.array_equal(budget[:7], ref_budget[:7]), (budget, ref_budget)
        assert budget[0] == budget[1] + budget[2]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """Host-side checks, before anything reaches the GPU: more sources or
    packets than the static scratch holds, and device buffers whose
    alignment the kernels' vector loads and 64-bit reductions need (nothing
    is launched, so the fake addresses are never dereferenced)."""
    L = native.lib()
    box = small_hhe_box((8, 8, 8), n_src=1, seed=302)
    desc = native.make_desc(box, native.CRASH_MIXED)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    budget = np.zeros(8, np.int64)

    def call(n, P, absorbers, deposits):
        pos = np.full((n, 3), 1.5)
        ndot = np.ones(n)
        E = np.array([20.0])
        frac = np.ones(n)
        return L.crash_transport_noalloc(C.byref(desc), n, dp(pos), dp(ndot), 1, dp(E), dp(frac), 1e12,
                                         0, P, 0, C.c_void_p(absorbers), C.c_void_p(deposits),
                                         budget.ctypes.data_as(C.POINTER(C.c_int64)), None)

    n = 1025                               # one more than CRASH_NOALLOC_MAX_SOURCES
    assert call(n, n, 256, 256) == native.CRASH_ERR_OVERFLOW
    assert b"CRASH_NOALLOC_MAX_SOURCES" in L.crash_noalloc_last_error()
    assert call(4, 4 * ((1 << 30) // 4 + 1), 256, 256) == native.CRASH_ERR_OVERFLOW
    assert b"CRASH_NOALLOC_MAX_PACKETS" in L.crash_noalloc_last_error()
    assert call(4, 64, 256 + 8, 256) == native.CRASH_ERR_ARG      # float4 loads need 16 B
    assert b"absorbers_dev" in L.crash_noalloc_last_error()
    assert call(4, 64, 256, 256 + 4) == native.CRASH_ERR_ARG      # 64-bit reductions need 8 B
    assert b"deposits_dev" in L.crash_noalloc_last_error()
