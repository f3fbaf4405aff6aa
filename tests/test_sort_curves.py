"""The re-sort keys of the wavefront (Morton or Hilbert order of 8^3-cell
buckets): the kernels' curve_key3 compiled for the host.  Both curves number
the 2^(3b) buckets one to one; consecutive Hilbert keys are face neighbours
(the property that makes it a Hilbert curve), consecutive Morton keys are
not always."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("curve") / "curve_probe")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_1101_4127_gb300", "csrc"),
                           "-o", exe, os.path.join(HERE, "curve_probe.cu")])
    out = subprocess.check_output([exe], text=True)
    return {(int(h), int(b)): (int(p), int(j)) for h, b, p, j in (l.split() for l in out.split("\n") if l)}


def test_both_curves_number_every_bucket_once(probe):
    for (h, b), (bad, _) in probe.items():
        assert bad == 0, (h, b)


def test_consecutive_hilbert_keys_are_face_neighbours(probe):
    for b in range(1, 6):
        assert probe[(1, b)][1] == 0, b
        assert probe[(0, b)][1] > 0, b      # Morton jumps
