"""CPU oracle of the radiative-transfer step: a plain sequential FP64 C
library (crash_oracle.c) and its ctypes binding.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg (bench.py cpu_baseline / --impl reference)
import this package.  The product (paper_1101_4127_gb300) never does.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crash_oracle.c")
_HDR = os.path.join(_HERE, "crash_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

F_XHII, F_XHEII, F_XHEIII, F_T = 0, 1, 2, 3
F_DEP_HI, F_DEP_HEI, F_DEP_HEII, F_DEP_E = 4, 5, 6, 7
F_BUDGET, F_NH = 8, 9
F_REC_HI, F_REC_HEI, F_REC_HEII = 11, 12, 13
C_COLL_EXC, C_COLL_ION, C_RECOMB, C_BREMS, C_COMPTON, C_DIELEC, C_ALL = 1, 2, 4, 8, 16, 32, 63


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("box_cm", C.c_double), ("n_H", C.POINTER(C.c_float)), ("n_H0", C.c_double),
                ("he_over_h", C.c_double),
                ("x_HII", C.POINTER(C.c_double)), ("x_HeII", C.POINTER(C.c_double)),
                ("x_HeIII", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double)),
                ("x_HII0", C.c_double), ("x_HeII0", C.c_double), ("x_HeIII0", C.c_double),
                ("T0", C.c_double), ("isothermal", C.c_int), ("caseB", C.c_int),
                ("z_compton", C.c_double), ("seed", C.c_uint64), ("f_rec", C.c_double),
                ("coupling", C.c_int), ("periodic", C.c_int),
                ("uv_rate", C.c_double * 3), ("uv_heat_eV", C.c_double * 3)]


class ChemCell(C.Structure):
    _fields_ = [("nH", C.c_double), ("nHe", C.c_double),
                ("xHII", C.c_double), ("xHeII", C.c_double), ("xHeIII", C.c_double),
                ("T", C.c_double), ("G_HI", C.c_double), ("G_HeI", C.c_double),
                ("G_HeII", C.c_double), ("heat_per_ion", C.c_double),
                ("S_HI", C.c_double), ("S_HeI", C.c_double), ("S_HeII", C.c_double),
                ("heat_rate", C.c_double),
                ("U_HI", C.c_double), ("U_HeI", C.c_double), ("U_HeII", C.c_double),
                ("Ue_HI", C.c_double), ("Ue_HeI", C.c_double), ("Ue_HeII", C.c_double),
                ("isothermal", C.c_int), ("caseB", C.c_int), ("T_cmb", C.c_double),
                ("eps", C.c_double), ("max_sub", C.c_int), ("cool_mask", C.c_int),
                ("count_rec", C.c_int), ("rec", C.c_double * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            dp, ip, u32p = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
            L.oracle_init_grid.restype = P
            L.oracle_init_grid.argtypes = [C.POINTER(GridDesc)]
            L.oracle_add_sources.argtypes = [P, C.c_int, dp, dp, C.c_int, dp, dp]
            L.oracle_set_options.argtypes = [P, C.c_int, C.c_uint32, C.c_uint32, C.c_double, C.c_int, C.c_int]
            L.oracle_step.argtypes = [P, C.c_double, C.c_uint64]
            L.oracle_read_fields.argtypes = [P, C.c_int, P]
            L.oracle_write_fields.argtypes = [P, C.c_int, P]
            L.oracle_set_step_index.argtypes = [P, C.c_uint64]
            L.oracle_set_chem_sample.argtypes = [P, C.c_uint32, C.c_double]
            L.oracle_write_deposits.argtypes = [P, P]
            L.oracle_chemistry.argtypes = [P, C.c_double]
            L.oracle_free.argtypes = [P]
            L.oracle_free.restype = None
            L.oracle_last_error.argtypes = [P]
            L.oracle_last_error.restype = C.c_char_p
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_philox4x32_10.restype = None
            L.or_exp_neg.argtypes = [C.c_double]
            L.or_exp_neg.restype = C.c_double
            L.or_direction.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp]
            L.or_cross_sections.argtypes = [C.c_int, dp, dp]
            L.or_cross_sections.restype = None
            L.or_trace_packet.argtypes = [P, dp, dp, ip, ip, ip, C.c_int, ip, dp, C.POINTER(C.c_int)]
            L.or_trace_packet.restype = C.c_int64
            L.or_freeze_absorbers.argtypes = [P]
            L.or_chem_cell.argtypes = [C.POINTER(ChemCell), C.c_double]
            L.or_rates.argtypes = [C.c_double, C.c_int, dp]
            L.or_rates.restype = None
            L.or_compton_coef.argtypes = [C.c_double]
            L.or_compton_coef.restype = C.c_double
            L.or_rec_start.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, C.c_int, dp, dp]
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------ building blocks
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().or_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), o.ctypes.data_as(u32p))
    return o


def exp_neg(tau: float) -> float:
    return lib().or_exp_neg(float(tau))


def direction(seed: int, step: int, src: int, pkt: int):
    d = np.zeros(3)
    k = lib().or_direction(seed, step, src, pkt, _dptr(d))
    return d, k


def cross_sections(E_eV):
    E = np.ascontiguousarray(E_eV, dtype=np.float64)
    s = np.zeros(3 * len(E))
    lib().or_cross_sections(len(E), _dptr(E), _dptr(s))
    return s.reshape(3, len(E))


def rates(T: float, caseB: int = 1):
    o = np.zeros(17)
    lib().or_rates(float(T), int(caseB), _dptr(o))
    return o


def compton_coef(T_cmb: float) -> float:
    return lib().or_compton_coef(float(T_cmb))


def chem_cell(dt: float, **kw):
    """Integrate one cell; keyword fields of ChemCell (defaults: isothermal 0,
    caseB 1, eps 0.1, max_sub 10000, all processes on, no recombination
    count).  Returns (state dict, sub-steps); with count_rec=1 the dict also
    holds 'rec', the recombinations to the ground state per cm^3 into H I,
    He I, He II."""
    c = ChemCell()
    defaults = dict(nH=1e-3, nHe=0.0, xHII=0.0, xHeII=0.0, xHeIII=0.0, T=1e4, G_HI=0.0,
                    G_HeI=0.0, G_HeII=0.0, heat_per_ion=0.0, S_HI=0.0, S_HeI=0.0, S_HeII=0.0,
                    heat_rate=0.0, U_HI=0.0, U_HeI=0.0, U_HeII=0.0, Ue_HI=0.0, Ue_HeI=0.0,
                    Ue_HeII=0.0, isothermal=0, caseB=1,
                    T_cmb=0.0, eps=0.1, max_sub=10000, cool_mask=C_ALL, count_rec=0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(c, k, v)
    n = lib().or_chem_cell(C.byref(c), float(dt))
    out = {k: getattr(c, k) for k in ("xHII", "xHeII", "xHeIII", "T")}
    out["rec"] = np.array(list(c.rec))
    return out, n


def rec_start(seed: int, step: int, cell: int, nx: int, ny: int):
    """Start point (grid units) and direction of a cell's re-emission packet."""
    pos, d = np.zeros(3), np.zeros(3)
    k = lib().or_rec_start(seed, step, cell, nx, ny, _dptr(pos), _dptr(d))
    return pos, d, k


# ------------------------------------------------------------ grid context
class OracleGrid:
    """One grid run by the oracle, with the same calls as the CUDA library:
    init_grid / add_sources / step / read_fields / write_fields."""

    def __init__(self, nx, ny, nz, box_cm, n_H=None, n_H0=1e-3, he_over_h=0.0,
                 x_HII=None, x_HeII=None, x_HeIII=None, T=None,
                 x_HII0=0.0, x_HeII0=0.0, x_HeIII0=0.0, T0=1e4,
                 isothermal=0, caseB=1, z_compton=-1.0, seed=0, f_rec=0.0, coupling=0,
                 periodic=0, uv_rate=(0.0, 0.0, 0.0), uv_heat_eV=(0.0, 0.0, 0.0)):
        self.L = lib()
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz
        d = GridDesc()
        d.nx, d.ny, d.nz, d.box_cm = nx, ny, nz, box_cm
        keep = []

        def fp(a, dt, ct):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt).reshape(-1)
            assert a.size == self.ncell
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(ct))

        d.n_H = fp(n_H, np.float32, C.c_float)
        d.n_H0 = n_H0
        d.he_over_h = he_over_h
        d.x_HII = fp(x_HII, np.float64, C.c_double)
        d.x_HeII = fp(x_HeII, np.float64, C.c_double)
        d.x_HeIII = fp(x_HeIII, np.float64, C.c_double)
        d.T = fp(T, np.float64, C.c_double)
        d.x_HII0, d.x_HeII0, d.x_HeIII0, d.T0 = x_HII0, x_HeII0, x_HeIII0, T0
        d.isothermal, d.caseB, d.z_compton, d.seed = isothermal, caseB, z_compton, seed
        d.f_rec = f_rec
        d.coupling, d.periodic = coupling, periodic
        for k in range(3):
            d.uv_rate[k] = float(uv_rate[k])
            d.uv_heat_eV[k] = float(uv_heat_eV[k])
        self.ctx = self.L.oracle_init_grid(C.byref(d))
        if not self.ctx:
            raise RuntimeError("oracle_init_grid failed")

    @classmethod
    def from_box(cls, box, precision_unused=None):
        nx, ny, nz = box.shape_xyz
        g = cls(nx, ny, nz, box.box_cm, n_H=box.nH, n_H0=box.nH0,
                he_over_h=box.he_over_h, x_HII0=box.x_HII0, x_HeII0=box.x_HeII0,
                x_HeIII0=box.x_HeIII0, T0=box.T0, isothermal=box.isothermal,
                caseB=box.caseB, z_compton=box.z_compton, seed=box.seed,
                f_rec=getattr(box, "f_rec", 0.0), coupling=getattr(box, "coupling", 0),
                periodic=getattr(box, "periodic", 0),
                uv_rate=getattr(box, "uv_rate", (0.0, 0.0, 0.0)),
                uv_heat_eV=getattr(box, "uv_heat_eV", (0.0, 0.0, 0.0)))
        g.add_sources(box.src_pos, box.src_ndot, box.bin_eV, box.bin_frac)
        return g

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError("oracle: " + self.L.oracle_last_error(self.ctx).decode())

    def add_sources(self, pos, ndot, bin_eV, bin_frac):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        ndot = np.ascontiguousarray(ndot, np.float64).reshape(-1)
        bin_eV = np.ascontiguousarray(bin_eV, np.float64).reshape(-1)
        bf = np.asarray(bin_frac, np.float64)
        if bf.ndim == 1:
            bf = np.tile(bf, (len(ndot), 1))
        bf = np.ascontiguousarray(bf)
        self._src_keep = (pos, ndot, bin_eV, bf)
        self._check(self.L.oracle_add_sources(self.ctx, len(ndot), _dptr(pos), _dptr(ndot),
                                              len(bin_eV), _dptr(bin_eV), _dptr(bf)))

    def set_options(self, chemistry=1, pkt_begin=0, pkt_end=0xFFFFFFFF, chem_eps=0.1,
                    chem_max_sub=10000, cool_mask=C_ALL):
        self._check(self.L.oracle_set_options(self.ctx, chemistry, pkt_begin, pkt_end,
                                              chem_eps, chem_max_sub, cool_mask))

    def step(self, dt_s, packets_per_step):
        self._check(self.L.oracle_step(self.ctx, float(dt_s), int(packets_per_step)))

    def set_step_index(self, k):
        self._check(self.L.oracle_set_step_index(self.ctx, int(k)))

    def read_deposits(self):
        """Deposits as int64[cells, 4] (H I, He I, He II, heat)."""
        return np.stack([self.read(f).reshape(-1) for f in (F_DEP_HI, F_DEP_HEI, F_DEP_HEII,
                                                             F_DEP_E)], axis=1)

    def write_deposits(self, dep):
        a = np.ascontiguousarray(dep, np.int64).reshape(-1, 4)
        assert a.shape[0] == self.ncell
        self._check(self.L.oracle_write_deposits(self.ctx, a.ctypes.data_as(C.c_void_p)))

    def chemistry(self, dt_s):
        """The per-cell update of the last step, which ran without chemistry."""
        self._check(self.L.oracle_chemistry(self.ctx, float(dt_s)))

    def set_chem_sample(self, stride, dep_scale=1.0):
        """Timing sample of the per-cell update (CPU baseline only)."""
        self._check(self.L.oracle_set_chem_sample(self.ctx, int(stride), float(dep_scale)))

    def read(self, field):
        if field == F_BUDGET:
            out = np.zeros(8, np.int64)
        elif field in (F_DEP_HI, F_DEP_HEI, F_DEP_HEII, F_DEP_E):
            out = np.zeros(self.ncell, np.int64)
        else:
            out = np.zeros(self.ncell, np.float64)
        self._check(self.L.oracle_read_fields(self.ctx, field, out.ctypes.data_as(C.c_void_p)))
        return out if field == F_BUDGET else out.reshape(self.shape)

    def write(self, field, arr):
        a = np.ascontiguousarray(arr, np.float64).reshape(-1)
        assert a.size == self.ncell
        self._check(self.L.oracle_write_fields(self.ctx, field, a.ctypes.data_as(C.c_void_p)))

    def freeze(self):
        self.L.or_freeze_absorbers(self.ctx)

    def trace(self, pos, d, content, log=0):
        """Trace one packet through the frozen absorbers (call freeze() first).
        Returns (crossings, remaining content, escaped, absorbed, log)."""
        pos = np.ascontiguousarray(pos, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        N = np.ascontiguousarray(content, np.int64).copy()
        esc = np.zeros(1, np.int64)
        ab = np.zeros(1, np.int64)
        ip = C.POINTER(C.c_int64)
        lc = np.zeros(max(log, 1), np.int64)
        ll = np.zeros(max(log, 1), np.float64)
        nl = C.c_int(0)
        cr = self.L.or_trace_packet(self.ctx, _dptr(pos), _dptr(d), N.ctypes.data_as(ip),
                                    esc.ctypes.data_as(ip), ab.ctypes.data_as(ip), log,
                                    lc.ctypes.data_as(ip), _dptr(ll), C.byref(nl))
        if cr < 0:
            self._check(-1)
        return cr, N, int(esc[0]), int(ab[0]), (lc[:nl.value], ll[:nl.value])

    def close(self):
        if getattr(self, "ctx", None):
            self.L.oracle_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
