"""Diagnostics of the fields a run reads back (the paper's figures of
Sec. 4): spherically averaged profiles around a source, volume-weighted
distributions of a field, and the ionisation-front radius by volume.

These analyse host copies of the fields after `Grid.read`; they are not
part of the radiative-transfer step, which runs in the CUDA library.
Fields are arrays indexed [z, y, x] as `Grid.read` returns them; positions
are in grid units (cell i spans [i, i+1))."""
from __future__ import annotations

import math

import numpy as np


def cell_radii(shape, centre):
    """Distance (in cells) of every cell centre from `centre` (x, y, z)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    return np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)


def radial_profile(field, centre, edges):
    """Spherically averaged profile of `field` around `centre`: the mean over
    the cells whose centres fall in each shell [edges[k], edges[k+1]) (grid
    units).  Returns (mean per shell, cells per shell); empty shells give
    NaN."""
    f = np.asarray(field, dtype=np.float64)
    r = cell_radii(f.shape, centre).ravel()
    edges = np.asarray(edges, dtype=np.float64)
    k = np.digitize(r, edges) - 1
    ok = (k >= 0) & (k < len(edges) - 1)
    count = np.bincount(k[ok], minlength=len(edges) - 1).astype(np.int64)
    total = np.bincount(k[ok], weights=f.ravel()[ok], minlength=len(edges) - 1)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(count > 0, total / np.maximum(count, 1), np.nan)
    return mean, count


def volume_pdf(field, edges, log=False):
    """Volume-weighted distribution of `field` over the bins `edges` (of
    log10(field) when log=True): the fraction of the grid's volume in each
    bin, divided by the bin width, so that it integrates to the covered
    fraction of the volume (cells are equal cubes)."""
    v = np.asarray(field, dtype=np.float64).ravel()
    if log:
        v = np.log10(np.where(v > 0, v, np.nan))
    v = v[np.isfinite(v)]
    edges = np.asarray(edges, dtype=np.float64)
    h, _ = np.histogram(v, bins=edges)
    total = np.asarray(field).size
    return h / total / np.diff(edges)


def front_radius(x_ion, octant=False):
    """Radius of the ionised region by volume, r = (3 f V / (4 pi))^(1/3)
    with V = sum of the ionised fraction over the cells (in cells^3) and
    f = 8 when the source sits at a corner and sees one octant."""
    V = float(np.asarray(x_ion, dtype=np.float64).sum())
    return (3.0 * (8.0 if octant else 1.0) * V / (4.0 * math.pi)) ** (1.0 / 3.0)
