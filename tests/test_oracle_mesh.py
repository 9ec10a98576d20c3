"""Whole-mesh pins of the CPU oracle (no GPU needed): closed forms, the mesh
invariants, brute force over every tiny bitmap, the paper's regime (Lemma
3.1 / Thm. 3.2) and properties of the Tier-G greedy rule."""
import itertools
import math

import numpy as np
import pytest

import oracle
from mesh_checks import check_mesh
from paper_2602_19474_gb300 import synth

R3 = math.sqrt(3.0)


def mesh_and_check(img, hn, hd=1):
    m = oracle.mesh_bitmap(img, hn, hd)
    check_mesh(img, m["xy"], m["tri"], m["label"], hn / hd, m["n_cells"])
    return m


def test_constant_image_is_the_lattice():
    img = np.full((7, 5), 3, np.uint8)
    m = mesh_and_check(img, 2)
    # four border segments, nothing else
    assert len(m["seg"]) == 4
    segs = sorted(map(tuple, m["seg"][:, :4].tolist()))
    assert segs == [(0, 0, 0, 5), (0, 0, 1, 7), (0, 7, 0, 5), (5, 0, 1, 7)]
    # only the border cuts cells; every untouched cell is one lattice triangle
    uncut = m["n_cells"] - m["n_cut_cells"]
    assert (m["code"] == 0).sum() == uncut
    lab = m["label"]
    assert set(np.unique(lab)) == {3, 0xFFFF}


def test_disk_closed_forms():
    img = synth.disk()
    assert img.sum() == 1257  # pixel centres with (x-32)^2+(y-32)^2 <= 400
    m = mesh_and_check(img, 2)
    # cut cells contain exactly the patches; Tier-T + Tier-G = cut cells
    assert m["n_tierG_cells"] < m["n_cut_cells"]
    # segments cover every boundary pixel edge exactly once
    from mesh_checks import boundary_length
    assert m["seg"][:, 3].sum() == boundary_length(img)
    # 8-fold symmetry of the digital disk: equal horizontal and vertical run length
    inner = m["seg"][(m["seg"][:, 4] != 0x10000) & (m["seg"][:, 5] != 0x10000)]
    assert inner[inner[:, 2] == 0, 3].sum() == inner[inner[:, 2] == 1, 3].sum()


def test_half_plane_segments():
    img = np.zeros((13, 20), np.uint8)
    img[:, :10] = 1
    m = mesh_and_check(img, 4)
    lens = sorted(m["seg"][:, 3].tolist())
    # interior run x = 9.5 (13), left and right borders (13 each), top and
    # bottom borders split at the junction (10 + 10 each)
    assert lens == [10, 10, 10, 10, 13, 13, 13]
    # segment orientation: lower label on the left
    for cx, cy, d, ln, l0, l1, rev in m["seg"].tolist():
        left = l1 if d == 0 else l0
        right = l0 if d == 0 else l1
        if rev:
            left, right = right, left
        assert left < right


def test_every_3x3_binary_bitmap():
    for bits in range(512):
        img = np.array([(bits >> k) & 1 for k in range(9)], np.uint8).reshape(3, 3)
        for hn, hd in ((2, 1), (4, 1), (2, 3)):
            mesh_and_check(img, hn, hd)


def test_random_4x4_multilabel():
    rng = np.random.default_rng(7)
    for _ in range(300):
        img = rng.integers(0, 3, (4, 4)).astype(np.uint8)
        for hn, hd in ((2, 1), (8, 1), (2, 3)):
            mesh_and_check(img, hn, hd)


def test_checkerboard_and_islands():
    # every corner a pinch or junction; single-pixel islands inside big cells
    cb = (np.indices((9, 11)).sum(axis=0) % 2).astype(np.uint8)
    for hn in (2, 8):
        mesh_and_check(cb, hn)
    isl = np.zeros((40, 40), np.uint8)
    isl[5::9, 7::11] = 1
    m = mesh_and_check(isl, 8)
    assert m["n_tierG_cells"] > 0


def test_u16_multilabel_voronoi_small():
    v = synth.voronoi_labels(size=96, nseeds=40, nlabels=6)
    mesh_and_check(v, 2)


def test_ellipses_and_noise_small():
    e = synth.ellipses(size=160, n=12, amin=5, amax=30)
    mesh_and_check(e, 4)
    for img in synth.noise_batch(n=3, lo=40, hi=90, first=3):
        mesh_and_check(img, 2)


@pytest.mark.parametrize("hn,hd", [(2, 3), (4, 7)])
def test_paper_regime_has_no_tier_g(hn, hd):
    """With h below one pixel (Sec. 3.2's length constraint holds for the
    pixel staircase) Lemma 3.1 holds: every cut cell is in the table, and its
    (m,n) class is one of Thm. 3.2's list."""
    img = synth.disk(size=48, cx=24, cy=24, r=15)
    m = mesh_and_check(img, hn, hd)
    assert m["n_tierG_cells"] == 0
    cut = m["cut"]
    key = (cut[:, 1] >> 6) & 63
    klass = (cut[:, 1] >> 12) & 15
    assert (key >= 1).all() and (key <= 15).all()
    # binary images have no junction: every cut cell is one of the paper's keys
    assert set(np.unique(key)) <= {1, 2, 3, 4, 5, 6}
    assert (klass >= 1).all()


def test_codes_are_consistent_with_counts():
    img = synth.voronoi_labels(size=80, nseeds=30, nlabels=5)
    m = mesh_and_check(img, 2)
    cut = m["cut"]
    # ntri = 2 * (chain vertices) + (boundary vertices) - 2 via the code's bitmask
    assert (cut[:, 2] >= 1).all()
    tierg = cut[:, 4] == 1
    assert (((cut[:, 1] >> 6) & 63)[tierg] == 63).all()
    assert (((cut[:, 1] >> 6) & 63)[~tierg] < 63).all()
    # chain-vertex bit set iff the cell holds a chain vertex
    assert (((cut[:, 1] & 1) == 1) == (cut[:, 3] > 0)).all()
    # triangle count per cell matches the emitted triangles
    assert cut[:, 2].sum() + (m["n_cells"] - len(cut)) == m["n_triangles"]


def _greedy_case(rng, npts):
    """random points in the triangle (0,0),(2S,0),(S, S*sqrt3) with a few
    non-crossing constraint edges taken from a first greedy pass"""
    S = 60
    tri = [[0, 0, 0, 0], [2 * S, 0, 0, 0], [S, 0, 0, S]]
    pts = list(tri)
    while len(pts) < npts:
        a, b = rng.uniform(0.05, 0.9, 2)
        if a + b >= 0.95:
            continue
        x = a * 2 * S + b * S
        y = b * S  # times sqrt3
        pts.append([int(round(x)), 0, 0, int(round(y))])
    pts = [list(p) for p in dict.fromkeys(map(tuple, pts))]
    return pts


def test_greedy_triangulates_and_is_maximal():
    rng = np.random.default_rng(3)
    for _ in range(40):
        pts = _greedy_case(rng, int(rng.integers(4, 14)))
        n = len(pts)
        cons = [[0, 1], [1, 2], [2, 0]]
        tri = oracle.greedy(pts, cons)
        P = np.array([[p[0] + p[1] * R3, p[2] + p[3] * R3] for p in pts], dtype=float)
        # hull = the triangle; boundary points are the three corners unless
        # another point landed on an edge (none do at these coordinates)
        assert len(tri) == 2 * (n - 3) + 3 - 2
        a = P[tri]
        ar = 0.5 * ((a[:, 1, 0] - a[:, 0, 0]) * (a[:, 2, 1] - a[:, 0, 1]) - (a[:, 1, 1] - a[:, 0, 1]) * (a[:, 2, 0] - a[:, 0, 0]))
        assert (ar > 0).all()
        assert abs(ar.sum() - 0.5 * 120 * 60 * R3) < 1e-6
        # constraints kept
        edges = {tuple(sorted(e)) for t in tri for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
        assert {(0, 1), (1, 2), (0, 2)} <= edges
        # greedy choice on a convex quad: the shorter diagonal
    quad = [[0, 0, 0, 0], [100, 0, 0, 0], [130, 0, 60, 0], [10, 0, 70, 0]]
    tri = oracle.greedy(quad, [[0, 1], [1, 2], [2, 3], [3, 0]])
    edges = {tuple(sorted(e)) for t in tri for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    d02 = math.hypot(130, 60)
    d13 = math.hypot(90, 70)
    assert ((1, 3) in edges) == (d13 < d02)


def test_greedy_keeps_chain_constraints():
    # a staircase chain through the triangle must survive as mesh edges
    S = 60
    pts = [[0, 0, 0, 0], [2 * S, 0, 0, 0], [S, 0, 0, S],
           [30, 0, 0, 5], [50, 0, 0, 5], [50, 0, 0, 20], [70, 0, 0, 20]]
    cons = [[0, 1], [1, 2], [2, 0], [3, 4], [4, 5], [5, 6]]
    tri = oracle.greedy(pts, cons)
    edges = {tuple(sorted(e)) for t in tri for e in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    assert {(3, 4), (4, 5), (5, 6)} <= edges
    assert len(tri) == 2 * 4 + 3 - 2


def test_patches_depend_only_on_their_neighbourhood():
    """Cor. "lookup-driven parallel retriangulation": every patch is a function
    of its cell's local configuration, so meshing any crop on the same lattice
    (grid origin moved by the crop offset) reproduces the full mesh's
    triangles away from the crop border, vertex order, label and code
    included."""
    from gpu_util import assert_window_matches_crop

    img = synth.voronoi_labels(size=700, nseeds=120, nlabels=9)
    for hn in (2, 4):
        m = oracle.mesh_bitmap(img, hn, 1)
        for x0, y0 in [(0, 0), (150, 260), (316, 316)]:
            assert assert_window_matches_crop(img, m, hn, 1, x0, y0, 384, 384) > 1000
