"""Mesh invariants that hold for any correct output of the method, whoever
produced it: orientation, closure, Euler characteristic, exact area, per-label
area = pixel count, and boundary conformity (every label change happens
across a mesh edge lying on a pixel line, and those edges add up to the
boundary length of the bitmap)."""
from __future__ import annotations

import math

import numpy as np

OUTSIDE = 0xFFFF


def boundary_length(img: np.ndarray) -> int:
    """Number of unit pixel edges separating different labels (the image
    border against the outside included)."""
    p = np.pad(img.astype(np.int64), 1, constant_values=-1)
    horiz = (p[1:, 1:-1] != p[:-1, 1:-1]).sum()
    vert = (p[1:-1, 1:] != p[1:-1, :-1]).sum()
    return int(horiz + vert)


def signed_areas(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    a = xy[tri]
    return 0.5 * ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1])
                  - (a[:, 1, 1] - a[:, 0, 1]) * (a[:, 2, 0] - a[:, 0, 0]))


def check_mesh(img: np.ndarray, xy: np.ndarray, tri: np.ndarray, label: np.ndarray, h: float, n_cells: int):
    H, W = img.shape
    V, T = len(xy), len(tri)
    assert tri.min() >= 0 and tri.max() < V
    area = signed_areas(xy, tri)
    assert (area > 0).all(), "triangle not counter-clockwise"
    assert len(np.unique(tri)) == V, "unused vertex"
    # closure and Euler characteristic of a disk
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    es = np.sort(e, axis=1)
    key = es[:, 0].astype(np.int64) * V + es[:, 1]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    uniq, cnt = np.unique(ks, return_counts=True)
    assert cnt.max() <= 2, "edge in more than two triangles"
    assert V - len(uniq) + T == 1, "Euler characteristic"
    # each interior edge appears once in each direction
    dirs = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    dk = dirs[:, 0].astype(np.int64) * V + dirs[:, 1]
    assert len(np.unique(dk)) == len(dk), "directed edge repeated (orientation clash)"
    # exact total area: every base cell is tiled
    total = n_cells * math.sqrt(3) / 4 * h * h
    assert abs(area.sum() - total) <= 1e-9 * total + 1e-9
    # per-label area equals the pixel count
    labs, counts = np.unique(img, return_counts=True)
    for l, c in zip(labs, counts):
        got = area[label == l].sum()
        assert abs(got - c) <= 1e-9 * W * H + 1e-7, (int(l), got, int(c))
    out_area = area[label == OUTSIDE].sum()
    assert abs(out_area - (total - W * H)) <= 1e-9 * total + 1e-7
    # boundary conformity: label changes only across edges on pixel lines,
    # and those edges cover the whole boundary
    tidx = np.concatenate([np.arange(T)] * 3)[order]
    pair = np.nonzero(ks[1:] == ks[:-1])[0]
    t1, t2 = tidx[pair], tidx[pair + 1]
    chg = label[t1] != label[t2]
    ce = es[order][pair[chg]]
    p, q = xy[ce[:, 0]], xy[ce[:, 1]]
    onh = (np.abs(p[:, 1] - q[:, 1]) < 1e-9) & (np.abs(p[:, 1] - np.round(p[:, 1] - 0.5) - 0.5) < 1e-9)
    onv = (np.abs(p[:, 0] - q[:, 0]) < 1e-9) & (np.abs(p[:, 0] - np.round(p[:, 0] - 0.5) - 0.5) < 1e-9)
    assert (onh | onv).all(), "label change across an edge off the pixel lines"
    # boundary edges of the mesh that separate image from outside are on the
    # image border; they are part of the label-change set via OUTSIDE labels
    blen = np.abs(p - q).sum(axis=1).sum()
    # mesh-border edges (count 1) lie outside the image except where the
    # image border itself is the mesh border (never: cells meeting the closed
    # rectangle cover a neighbourhood of it)
    assert abs(blen - boundary_length(img)) < 1e-6 * max(1, boundary_length(img)), (blen, boundary_length(img))
    return dict(V=V, T=T, E=len(uniq), min_area=float(area.min()))
