"""Mesh quality measures -- the oracle of mesh_quality (test infrastructure,
used only by the tests and the checks of bench.py / smoke).

Plain numpy in float64 from a mesh's vertex coordinates and triangles, one
measure per definition of the experiments section:

- interior angles, the smallest of each triangle, and "slivers": triangles
  whose smallest angle is below 5 degrees (Sec. 4.2, Table "mesh quality");
- triangle areas, their minimum and their (population) variance (Sec. 4.4,
  Table "comparison", "Area Var.");
- the equilateral ratio by an edge-length test (Table "mesh quality");
- the aspect ratio AR = longest edge / shortest altitude, of which the
  median, 95th percentile and maximum are reported (Table "aspect-ratio
  statistics"); an equilateral triangle has AR = 2 / sqrt(3);
- the distribution of the smallest angles in 2-degree bins (Fig. "minimum
  angle histograms").

Readings where the paper gives no number: the edge-length test calls a
triangle equilateral when its longest and shortest squared edge lengths
differ by at most 1e-9 of the longest; percentiles are nearest-rank (the
k-th smallest value with k = ceil(p T)); the 30 histogram bins are
[0, 2), [2, 4), ..., [58, 60], the last one closed.
"""
from __future__ import annotations

import math

import numpy as np

SLIVER_DEG = 5.0
EQUILATERAL_RTOL = 1e-9
HIST_BINS = 30


def triangle_measures(xy: np.ndarray, tri: np.ndarray):
    """Per triangle: smallest interior angle (degrees), area, aspect ratio,
    equilateral flag."""
    p = np.asarray(xy, dtype=np.float64)[np.asarray(tri, dtype=np.int64)]
    a, b, c = p[:, 0], p[:, 1], p[:, 2]

    def angle(o, u, v):
        d1, d2 = u - o, v - o
        cross = np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])
        dot = d1[:, 0] * d2[:, 0] + d1[:, 1] * d2[:, 1]
        return np.degrees(np.arctan2(cross, dot))

    ang = np.minimum(np.minimum(angle(a, b, c), angle(b, c, a)), angle(c, a, b))
    ab, bc, ca = b - a, c - b, a - c
    l2 = np.stack([(ab * ab).sum(1), (bc * bc).sum(1), (ca * ca).sum(1)], axis=1)
    area = 0.5 * np.abs(ab[:, 0] * (c - a)[:, 1] - ab[:, 1] * (c - a)[:, 0])
    lmax, lmin = l2.max(1), l2.min(1)
    ar = lmax / (2.0 * area)  # longest edge / (2 area / longest edge)
    equi = (lmax - lmin) <= EQUILATERAL_RTOL * lmax
    return ang, area, ar, equi


def nearest_rank(sorted_vals: np.ndarray, q: float) -> float:
    k = max(1, math.ceil(q * len(sorted_vals)))
    return float(sorted_vals[k - 1])


def quality(xy: np.ndarray, tri: np.ndarray) -> dict:
    ang, area, ar, equi = triangle_measures(xy, tri)
    s = np.sort(ar)
    hist = np.zeros(HIST_BINS, dtype=np.int64)
    idx = np.minimum((ang / 2.0).astype(np.int64), HIST_BINS - 1)
    np.add.at(hist, idx, 1)
    return {
        "triangles": int(len(tri)),
        "min_angle_deg": float(ang.min()),
        "min_area": float(area.min()),
        "slivers": int((ang < SLIVER_DEG).sum()),
        "equilateral": int(equi.sum()),
        "area_mean": float(area.mean()),
        "area_var": float(area.var()),
        "ar_median": nearest_rank(s, 0.5),
        "ar_p95": nearest_rank(s, 0.95),
        "ar_max": float(s[-1]),
        "angle_hist": hist,
        "min_angles": ang,
    }
