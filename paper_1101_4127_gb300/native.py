"""ctypes binding of libcrash.so, the C ABI declared in include/crash.h.

Argument marshalling only: every step of the radiative-transfer path runs in
the library's CUDA kernels.  The functions keep the C names
(crash_init_grid, crash_add_sources, crash_step, crash_read_fields, ...);
`Grid` is a small convenience wrapper over them.  There is no fallback: if
the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

CRASH_OK, CRASH_ERR_ARG, CRASH_ERR_OOM, CRASH_ERR_CUDA = 0, -1, -2, -3
CRASH_ERR_OVERFLOW, CRASH_ERR_TIMEOUT, CRASH_ERR_STATE = -4, -5, -6
CRASH_FP64_PLAIN, CRASH_MIXED = 0, 1
F_XHII, F_XHEII, F_XHEIII, F_T = 0, 1, 2, 3
F_DEP_HI, F_DEP_HEI, F_DEP_HEII, F_DEP_E = 4, 5, 6, 7
F_BUDGET, F_NH, F_TOTALS = 8, 9, 10
F_REC_HI, F_REC_HEI, F_REC_HEII = 11, 12, 13

EXPORTED = [
    "crash_default_opts", "crash_init_grid", "crash_init_batch", "crash_add_sources",
    "crash_add_sources_box", "crash_set_options", "crash_get_options", "crash_step", "crash_step_batch",
    "crash_read_fields", "crash_read_fields_box", "crash_write_fields", "crash_write_fields_box",
    "crash_set_step_index", "crash_sync", "crash_kernel_time", "crash_reset_kernel_time",
    "crash_stream", "crash_launch_count", "crash_autotune", "crash_free", "crash_last_error",
    "crash_transport_noalloc", "crash_noalloc_last_error", "crash_checkpoint",
    "crash_deposits_device", "crash_read_deposits", "crash_write_deposits", "crash_chemistry",
]
CKPT_SAVE, CKPT_RESTORE_STATE, CKPT_RESTORE = 0, 1, 2


class crash_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("box_cm", C.c_double),
                ("n_H", C.POINTER(C.c_float)), ("n_H0", C.c_double), ("he_over_h", C.c_double),
                ("x_HII", C.POINTER(C.c_double)), ("x_HeII", C.POINTER(C.c_double)),
                ("x_HeIII", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double)),
                ("x_HII0", C.c_double), ("x_HeII0", C.c_double), ("x_HeIII0", C.c_double),
                ("T0", C.c_double), ("isothermal", C.c_int), ("caseB", C.c_int),
                ("z_compton", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int),
                ("f_rec", C.c_double), ("coupling", C.c_int), ("periodic", C.c_int),
                ("uv_rate", C.c_double * 3), ("uv_heat_eV", C.c_double * 3)]


class crash_run_opts(C.Structure):
    _fields_ = [("chemistry", C.c_int), ("pkt_begin", C.c_uint32), ("pkt_end", C.c_uint32),
                ("chem_eps", C.c_double), ("chem_max_sub", C.c_int), ("cool_mask", C.c_int),
                ("block_size", C.c_int), ("seg_per_iter", C.c_int), ("resort_interval", C.c_int),
                ("wavefront", C.c_int), ("use_graph", C.c_int), ("timing", C.c_int),
                ("reg_cap", C.c_int), ("tile", C.c_int), ("pass_limit", C.c_int),
                ("sort_curve", C.c_int), ("chunk_packets", C.c_int), ("persistent", C.c_int)]


def library_path() -> str:
    return _build.SO


def lib(build_if_missing: bool = True):
    """Load libcrash.so (building it first if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.SO
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libcrash.so not built ({path})")
                path = _build.build()
            L = C.CDLL(path)
            P, dp = C.c_void_p, C.POINTER(C.c_double)
            L.crash_default_opts.argtypes = [C.POINTER(crash_run_opts)]
            L.crash_default_opts.restype = None
            L.crash_init_grid.argtypes = [C.POINTER(crash_grid_desc), C.POINTER(P)]
            L.crash_init_batch.argtypes = [C.c_int, C.POINTER(crash_grid_desc), C.POINTER(P)]
            L.crash_add_sources.argtypes = [P, C.c_int, dp, dp, C.c_int, dp, dp]
            L.crash_add_sources_box.argtypes = [P, C.c_int, C.c_int, dp, dp, C.c_int, dp, dp]
            L.crash_set_options.argtypes = [P, C.POINTER(crash_run_opts)]
            L.crash_get_options.argtypes = [P, C.POINTER(crash_run_opts)]
            L.crash_step.argtypes = [P, C.c_double, C.c_uint64]
            L.crash_step_batch.argtypes = [P, C.c_double, C.POINTER(C.c_uint64)]
            L.crash_read_fields.argtypes = [P, C.c_int, P]
            L.crash_read_fields_box.argtypes = [P, C.c_int, C.c_int, P]
            L.crash_write_fields.argtypes = [P, C.c_int, P]
            L.crash_write_fields_box.argtypes = [P, C.c_int, C.c_int, P]
            L.crash_set_step_index.argtypes = [P, C.c_uint64]
            L.crash_checkpoint.argtypes = [P, C.c_int]
            L.crash_sync.argtypes = [P]
            L.crash_kernel_time.argtypes = [P, dp, C.POINTER(C.c_int64)]
            L.crash_reset_kernel_time.argtypes = [P]
            L.crash_stream.argtypes = [P]
            L.crash_stream.restype = P
            L.crash_launch_count.argtypes = [P]
            L.crash_launch_count.restype = C.c_int64
            L.crash_autotune.argtypes = [P, C.c_double, C.POINTER(C.c_uint64), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.crash_transport_noalloc.argtypes = [
                C.POINTER(crash_grid_desc), C.c_int, dp, dp, C.c_int, dp, dp, C.c_double, C.c_uint64,
                C.c_uint64, C.c_int, P, P, C.POINTER(C.c_int64), P]
            L.crash_deposits_device.argtypes = [P, C.c_int, C.POINTER(P), C.POINTER(C.c_int64)]
            L.crash_read_deposits.argtypes = [P, C.c_int, P]
            L.crash_write_deposits.argtypes = [P, C.c_int, P]
            L.crash_chemistry.argtypes = [P, C.c_double]
            L.crash_noalloc_last_error.argtypes = []
            L.crash_noalloc_last_error.restype = C.c_char_p
            L.crash_free.argtypes = [P]
            L.crash_last_error.argtypes = [P]
            L.crash_last_error.restype = C.c_char_p
            for name in EXPORTED:
                if name not in ("crash_default_opts", "crash_stream", "crash_last_error",
                                "crash_launch_count", "crash_noalloc_last_error"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


class CrashError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"crash status {status}: {msg}")
        self.status = status


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def default_opts() -> crash_run_opts:
    o = crash_run_opts()
    lib().crash_default_opts(C.byref(o))
    return o


def make_desc(box, precision=CRASH_FP64_PLAIN, keep=None):
    """crash_grid_desc of an inputs.Box (arrays kept alive in `keep`)."""
    d = crash_grid_desc()
    d.nx, d.ny, d.nz = box.shape_xyz
    d.box_cm = box.box_cm
    if box.nH is not None:
        a = np.ascontiguousarray(box.nH, np.float32).reshape(-1)
        if keep is not None:
            keep.append(a)
        d.n_H = a.ctypes.data_as(C.POINTER(C.c_float))
    d.n_H0 = box.nH0
    d.he_over_h = box.he_over_h
    d.x_HII0, d.x_HeII0, d.x_HeIII0, d.T0 = box.x_HII0, box.x_HeII0, box.x_HeIII0, box.T0
    d.isothermal, d.caseB, d.z_compton, d.seed = box.isothermal, box.caseB, box.z_compton, box.seed
    d.precision = precision
    d.f_rec = getattr(box, "f_rec", 0.0)
    d.coupling = getattr(box, "coupling", 0)
    d.periodic = getattr(box, "periodic", 0)
    for k in range(3):
        d.uv_rate[k] = float(getattr(box, "uv_rate", (0.0, 0.0, 0.0))[k])
        d.uv_heat_eV[k] = float(getattr(box, "uv_heat_eV", (0.0, 0.0, 0.0))[k])
    return d


class Grid:
    """One context of the CUDA library holding one box or a batch of boxes."""

    def __init__(self, boxes, precision=CRASH_FP64_PLAIN):
        self.L = lib()
        if not isinstance(boxes, (list, tuple)):
            boxes = [boxes]
        self.boxes = list(boxes)
        keep = []
        descs = (crash_grid_desc * len(boxes))(*[make_desc(b, precision, keep) for b in boxes])
        ctx = C.c_void_p()
        st = self.L.crash_init_batch(len(boxes), descs, C.byref(ctx))
        if st != CRASH_OK:
            raise CrashError(st, self.L.crash_last_error(None).decode())
        self.ctx = ctx
        self._keep = []
        for i, b in enumerate(boxes):
            self.add_sources(b.src_pos, b.src_ndot, b.bin_eV, b.bin_frac, box=i)

    def _check(self, st):
        if st != CRASH_OK:
            raise CrashError(st, self.L.crash_last_error(self.ctx).decode())

    def add_sources(self, pos, ndot, bin_eV, bin_frac, box=0):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        ndot = np.ascontiguousarray(ndot, np.float64).reshape(-1)
        bin_eV = np.ascontiguousarray(bin_eV, np.float64).reshape(-1)
        bf = np.asarray(bin_frac, np.float64)
        if bf.ndim == 1:
            bf = np.tile(bf, (len(ndot), 1))
        bf = np.ascontiguousarray(bf)
        self._check(self.L.crash_add_sources_box(self.ctx, box, len(ndot), _dptr(pos), _dptr(ndot),
                                                 len(bin_eV), _dptr(bin_eV), _dptr(bf)))

    def set_options(self, **kw):
        o = default_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        self._check(self.L.crash_set_options(self.ctx, C.byref(o)))

    def get_options(self):
        """The context's current options as a dict (field name -> value)."""
        o = crash_run_opts()
        self._check(self.L.crash_get_options(self.ctx, C.byref(o)))
        return {k: getattr(o, k) for k, _ in crash_run_opts._fields_}

    def step(self, dt_s, packets):
        if isinstance(packets, (list, tuple, np.ndarray)):
            arr = (C.c_uint64 * len(packets))(*[int(p) for p in packets])
            self._check(self.L.crash_step_batch(self.ctx, float(dt_s), arr))
        else:
            self._check(self.L.crash_step(self.ctx, float(dt_s), int(packets)))

    def sync(self):
        self._check(self.L.crash_sync(self.ctx))

    def set_step_index(self, k):
        self._check(self.L.crash_set_step_index(self.ctx, int(k)))

    def checkpoint(self, op=CKPT_SAVE):
        self._check(self.L.crash_checkpoint(self.ctx, int(op)))

    def read(self, field, box=0):
        b = self.boxes[box]
        nx, ny, nz = b.shape_xyz
        n = nx * ny * nz
        if field in (F_BUDGET, F_TOTALS):
            out = np.zeros(8, np.int64)
        elif field in (F_DEP_HI, F_DEP_HEI, F_DEP_HEII, F_DEP_E):
            out = np.zeros(n, np.int64)
        else:
            out = np.zeros(n, np.float64)
        self._check(self.L.crash_read_fields_box(self.ctx, box, field, out.ctypes.data_as(C.c_void_p)))
        return out if field in (F_BUDGET, F_TOTALS) else out.reshape(nz, ny, nx)

    def write(self, field, arr, box=0):
        a = np.ascontiguousarray(arr, np.float64).reshape(-1)
        self._check(self.L.crash_write_fields_box(self.ctx, box, field, a.ctypes.data_as(C.c_void_p)))

    def deposits_device(self, box=0):
        """Device address and cell count of a box's deposits, uint64[cells][4]."""
        p, n = C.c_void_p(), C.c_int64()
        self._check(self.L.crash_deposits_device(self.ctx, box, C.byref(p), C.byref(n)))
        return p.value, n.value

    def read_deposits(self, box=0):
        """The box's deposits as int64[cells, 4] (H I, He I, He II, heat)."""
        nx, ny, nz = self.boxes[box].shape_xyz
        out = np.zeros((nx * ny * nz, 4), np.int64)
        self._check(self.L.crash_read_deposits(self.ctx, box, out.ctypes.data_as(C.c_void_p)))
        return out

    def write_deposits(self, dep, box=0):
        a = np.ascontiguousarray(dep, np.int64).reshape(-1, 4)
        self._check(self.L.crash_write_deposits(self.ctx, box, a.ctypes.data_as(C.c_void_p)))

    def chemistry(self, dt_s):
        """The per-cell update of the last (transport-only) step."""
        self._check(self.L.crash_chemistry(self.ctx, float(dt_s)))

    def kernel_time(self):
        ms = C.c_double(0)
        n = C.c_int64(0)
        self._check(self.L.crash_kernel_time(self.ctx, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def reset_kernel_time(self):
        self._check(self.L.crash_reset_kernel_time(self.ctx))

    def stream(self):
        return self.L.crash_stream(self.ctx)

    def launch_count(self):
        return self.L.crash_launch_count(self.ctx)

    def autotune(self, dt_s, packets):
        """Returns (block_size, seg_per_iter, resort_interval, reg_cap, tile,
        sort_curve) of the fastest trial, which the context keeps."""
        arr = (C.c_uint64 * len(packets))(*[int(p) for p in packets])
        out = [C.c_int() for _ in range(6)]
        self._check(self.L.crash_autotune(self.ctx, float(dt_s), arr, *[C.byref(v) for v in out]))
        return tuple(v.value for v in out)

    def close(self):
        if getattr(self, "ctx", None):
            self.L.crash_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
