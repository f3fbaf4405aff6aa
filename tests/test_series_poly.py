"""The mixed form's series for the absorbed fraction: the degree-5
polynomial in k_mixed.cu approximates (1 - e^-tau)/tau on [0, 0.5] within
1e-8 (its own error, FP32 coefficients) and, evaluated in FP32 by Horner's rule with fused
multiply-adds as the kernels do, within 6e-8.  Reference values from
numpy's expm1 in FP64.  CPU only."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1101_4127_gb300", "csrc", "k_mixed.cu")


def _coeffs():
    src = open(SRC).read()
    c = {int(k): float(v) for k, v in re.findall(r"#define CRASH_AOT_C(\d) (\S+?)f\b", src)}
    assert sorted(c) == list(range(6))
    return [c[k] for k in range(6)]


def _f(t):
    t = np.asarray(t, np.float64)
    out = np.ones_like(t)
    nz = t > 0
    out[nz] = -np.expm1(-t[nz]) / t[nz]
    return out


def test_polynomial_error_below_bound():
    c = np.array(_coeffs(), np.float64)
    t = np.linspace(0.0, 0.5, 100001)
    p = np.polyval(c[::-1], t)
    assert np.max(np.abs(p - _f(t)) / _f(t)) < 1e-8


def test_fp32_horner_error_below_bound():
    c = np.array(_coeffs(), np.float32)
    t = np.linspace(0.0, 0.5, 200001).astype(np.float32)
    p = np.full_like(t, c[5])
    for k in range(4, -1, -1):           # one rounding per step, as fmaf
        p = (p.astype(np.float64) * t.astype(np.float64) + np.float64(c[k])).astype(np.float32)
    ref = _f(t.astype(np.float64))
    assert np.max(np.abs(p.astype(np.float64) - ref) / ref) < 6e-8
    assert p[0] == 1.0
