"""Host-side work split of a step over several processes or GPUs.

The step shards by packets: every packet is independent given the absorbers
frozen at the start of the step (Sec. 2), so processes holding replicas of
the grid may trace disjoint sets of packets and sum their int64 deposits
(the one exchange of the step, Sec. 2's "reduction" strategy) before the
per-cell update.  Two ways to split:

  * packet_windows: every process traces a window of packet ids of every
    source (the library's run options pkt_begin/pkt_end).  Packets of one
    source are statistically alike, so equal windows balance the work in
    expectation whatever the sources and the medium.
  * split_sources: whole sources per process, balanced by a per-source load
    estimate built on the optically thin work estimator of Eq. 2 (Sec. 3.1),
    rho_gamma(cell) = sum over sources of |r_s - r_cell|^-2.  Summed over the
    cells of the grid it gives each source's share of that estimate:
    L_s = sum_cell |r_s - r_cell|^-2, about the integral over directions of
    the distance from the source to the grid's boundary (the chords its
    packets cross when the medium is thin).  Sources near a face or a corner
    load less than central ones.

Nothing here touches the device; the library's C ABI does the transport.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np


def packet_windows(packets_per_source: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous windows [lo, hi) of packet ids, one per rank, covering
    [0, packets_per_source) with sizes that differ by at most one."""
    if world < 1 or packets_per_source < 0:
        raise ValueError("world >= 1 and packets_per_source >= 0")
    return [(r * packets_per_source // world, (r + 1) * packets_per_source // world)
            for r in range(world)]


def eq2_cell_sum(pos: np.ndarray, shape_xyz: Sequence[int], r_min: float = 0.5) -> np.ndarray:
    """Eq. 2 summed over the cells of the grid for every source:
    L_s = sum_c max(|r_s - r_c|, r_min)^-2, with r_c the cell centres (grid
    units).  r_min keeps a source's own cell finite.  Cost: n_src x cells."""
    nx, ny, nz = shape_xyz
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    c = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    out = np.empty(len(pos))
    for s, p in enumerate(np.asarray(pos, np.float64)):
        d2 = np.maximum(((c - p) ** 2).sum(axis=1), r_min * r_min)
        out[s] = (1.0 / d2).sum()
    return out


def _fibonacci_sphere(n: int) -> np.ndarray:
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = math.pi * (1.0 + math.sqrt(5.0)) * k
    r = np.sqrt(1.0 - z * z)
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def eq2_source_load(pos: np.ndarray, shape_xyz: Sequence[int], n_dirs: int = 2048) -> np.ndarray:
    """The same per-source load as eq2_cell_sum for grids too large to sum
    cell by cell: sum_c |r_s - r_c|^-2 ~ integral over directions of the
    distance to the boundary, evaluated on n_dirs quasi-uniform directions
    (a Fibonacci sphere).  Returns 4 pi times the mean exit distance (cells)."""
    P = np.asarray(pos, np.float64)
    n = np.asarray(shape_xyz, np.float64)
    D = _fibonacci_sphere(n_dirs)
    with np.errstate(divide="ignore", invalid="ignore"):
        t_hi = np.where(D[None, :, :] > 0, (n[None, None, :] - P[:, None, :]) / D[None, :, :], np.inf)
        t_lo = np.where(D[None, :, :] < 0, -P[:, None, :] / D[None, :, :], np.inf)
    t = np.minimum(t_hi, t_lo).min(axis=2)
    return 4.0 * math.pi * t.mean(axis=1)


def split_sources(load: Sequence[float], world: int) -> List[List[int]]:
    """Sources per rank by longest-processing-time-first: sources in
    decreasing load, each to the rank with the least load so far (ties to the
    lower rank).  Within 4/3 of the best possible largest rank load."""
    if world < 1:
        raise ValueError("world >= 1")
    order = sorted(range(len(load)), key=lambda s: (-float(load[s]), s))
    ranks: List[List[int]] = [[] for _ in range(world)]
    tot = [0.0] * world
    for s in order:
        r = min(range(world), key=lambda k: (tot[k], k))
        ranks[r].append(s)
        tot[r] += float(load[s])
    return [sorted(r) for r in ranks]


def imbalance(load: Sequence[float], parts: Sequence[Sequence[int]]) -> float:
    """Largest rank load over the mean rank load (1 = perfect balance)."""
    per = [sum(float(load[s]) for s in p) for p in parts]
    mean = sum(per) / len(per)
    return max(per) / mean if mean > 0 else 1.0
