"""Pins of the Region III oracle (Alg. 2, the template retriangulation, run
on the preprocessed mesh T of Alg. 3; the pipelined-scheduling corollary
puts it after Regions I-II, one cell at a time).

- On the unmoved base mesh T0 the per-cell retriangulation must give the
  plain path's mesh: the oracle's exact Z[sqrt3] mesher, written
  independently, triangle for triangle with the same labels and codes.
- On preprocessed meshes: the invariants of any correct embedded mesh
  (orientation, closure, Euler characteristic, area, per-label area = pixel
  count, boundary conformity and length).
- Degenerate cells built by hand, each against the paper: a vertex on the
  segment (App. G (2,3) case (c1), Fig. "lookup_table"'s three-intersection
  atom), an overlap with an endpoint on the edge (Alg. 1's third and first
  branches), a glancing contact (App. G single-segment cases (a)/(d)).
- Planted mistakes in the oracle each fail one of these pins.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import preprocess as P
from paper_2602_19474_gb300 import synth

TRIPLET = (0.26, 0.125, 0.183)
# a label boundary meeting the right border 1 px below the image corner
BORDER_BAND = np.zeros((10, 33), np.uint8)
BORDER_BAND[9:, :] = 1
_ELL = synth.ellipses(256, 20, 2, 5.0, 40.0)


def _areas(P3):
    return 0.5 * ((P3[:, 1, 0] - P3[:, 0, 0]) * (P3[:, 2, 1] - P3[:, 0, 1])
                  - (P3[:, 1, 1] - P3[:, 0, 1]) * (P3[:, 2, 0] - P3[:, 0, 0]))


def check_embedded(img, T, R):
    """Invariants of a correct embedding of img's boundary into the mesh T."""
    H, W = img.shape
    xy, tri, lab = R["xy"], R["tri"], R["label"]
    ar = _areas(xy[tri])
    assert (ar > 0).all(), "triangle not counter-clockwise"
    used = np.zeros(len(xy), bool)
    used[tri.ravel()] = True
    assert used.all(), "unused vertex"
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]).astype(np.int64)
    assert len(np.unique(e, axis=0)) == len(e), "directed edge repeated"
    es = np.sort(e, axis=1)
    u, cnt = np.unique(es, axis=0, return_counts=True)
    assert cnt.max() <= 2, "edge in three triangles"
    assert len(xy) - len(u) + len(tri) == 1, "Euler characteristic"
    aT = _areas(T["xy"][T["tri"]]).sum()
    assert abs(ar.sum() - aT) <= 1e-9 * aT, "total area differs from T's"
    for l, c in zip(*np.unique(img, return_counts=True)):
        assert abs(ar[lab == l].sum() - c) <= 1e-9 * W * H + 1e-7, "area of label %d" % l
    # edges between triangles of different labels lie on pixel lines and add
    # up to the boundary length (outer edges of T carrying an image label lie
    # on the image border)
    tt = np.tile(np.arange(len(tri)), 3)
    order = np.lexsort((es[:, 1], es[:, 0]))
    es, tt = es[order], tt[order]
    pair = np.nonzero((es[1:] == es[:-1]).all(1))[0]
    diff = lab[tt[pair]] != lab[tt[pair + 1]]
    single = np.ones(len(es), bool)
    single[pair] = single[pair + 1] = False
    outer_img = np.nonzero(single)[0][lab[tt[single]] != 0xFFFF]
    ends = np.concatenate([es[pair[diff]], es[outer_img]])
    a, b = xy[ends[:, 0]], xy[ends[:, 1]]
    onh = (a[:, 1] == b[:, 1]) & ((a[:, 1] + 0.5) % 1 == 0)
    onv = (a[:, 0] == b[:, 0]) & ((a[:, 0] + 0.5) % 1 == 0)
    assert (onh | onv).all(), "label change off the pixel lines"
    pad = np.pad(img.astype(np.int64), 1, constant_values=1 << 20)
    blen = (pad[1:, 1:-1] != pad[:-1, 1:-1]).sum() + (pad[1:-1, 1:] != pad[1:-1, :-1]).sum()
    assert abs(np.abs(a - b).sum() - blen) <= 1e-6 * blen, "boundary length"


def _same_as_plain(img, hn, hd, plant=0):
    H, W = img.shape
    o = oracle.mesh_bitmap(img, hn, hd)
    xy0, cells = oracle.base_mesh(W, H, hn, hd)
    r = oracle.region3(img, xy0, cells, plant)
    assert r["tri"].shape == o["tri"].shape
    assert np.abs(r["xy"][r["tri"]] - o["xy"][o["tri"]]).max() <= 1e-9
    assert np.array_equal(r["label"], o["label"]) and np.array_equal(r["code"], o["code"])
    assert (r["n_cut_cells"], r["n_tierG_cells"], r["n_events"]) == (o["n_cut_cells"], o["n_tierG_cells"], len(o["ev"]))


def _cases():
    rng = np.random.default_rng(260219)
    out = [("disk64", synth.disk(64), 2, 1), ("voronoi_u16", synth.voronoi_labels(96, 24, 16).astype(np.uint16), 2, 1),
           ("ellipses256_h4", _ELL, 4, 1)]  # the last has nested chords (keys 5)
    for hn, hd in [(2, 1), (4, 1), (8, 1), (2, 3), (6, 5)]:
        for t in range(3):
            W, Hh = (int(x) for x in rng.integers(5, 36, 2))
            k = int(rng.integers(2, 5))
            img = rng.integers(0, k, (Hh, W)).astype(np.uint8)
            if t == 1:
                img = np.ascontiguousarray(np.kron(img[: Hh // 3 + 1, : W // 3 + 1], np.ones((3, 3), np.uint8))[:Hh, :W])
            out.append(("rand%d_%d_%d" % (t, hn, hd), img, hn, hd))
    return out


@pytest.mark.parametrize("name,img,hn,hd", _cases(), ids=[c[0] for c in _cases()])
def test_base_mesh_gives_the_plain_mesh(name, img, hn, hd):
    _same_as_plain(np.ascontiguousarray(img), hn, hd)


def test_every_3x3_bitmap_on_the_base_mesh():
    for b in range(512):
        img = np.array([(b >> k) & 1 for k in range(9)], np.uint8).reshape(3, 3)
        _same_as_plain(img, 2, 1)


@pytest.mark.parametrize("name,img,hn,hd", [
    ("disk64", synth.disk(64), 2, 1),
    ("voronoi", synth.voronoi_labels(96, 24, 16), 2, 1),
    ("noise_h4", synth.noise_bitmap(synth.rng_for(31), 36, 30, 1.5), 4, 1),
    ("noise_third", synth.noise_bitmap(synth.rng_for(32), 28, 24, 1.5), 2, 3),
    ("pixels_h2", (np.random.default_rng(5).random((20, 26)) < 0.5).astype(np.uint8), 2, 1),
    ("border_band", BORDER_BAND, 2, 1),
])
def test_preprocessed_mesh_invariants(name, img, hn, hd):
    img = np.ascontiguousarray(img)
    T = P.preprocess(img, hn, hd, *TRIPLET)
    R = oracle.region3(img, T["xy"], T["tri"])
    assert R["n_vertices_grid"] == len(T["xy"]) and R["n_cells"] == len(T["tri"])
    check_embedded(img, T, R)
    # every event lies on an edge between two cells, and a cut cell has
    # 2 n_i + n_b - 2 triangles
    assert len(R["tri"]) == len(T["tri"]) + 2 * R["n_inside"] + 2 * R["n_events"]
    # the degenerate incidences occur: snapped vertices sit on the boundary
    assert (T["status"] == 1).sum() > 0


def _quadrant(n=6, x0=2, y0=2):
    img = np.zeros((n, n), np.uint8)
    img[y0:, x0:] = 1
    return img


def test_vertex_on_segment_is_app_g_case_23_c1():
    """Corner A on a PSLG vertex, the boundary leaving A through the cell to
    Q on BC: App. G (2,3) case (c1), triangles ABQ and AQC; Alg. 1 counts the
    vertex on the segment twice (edges AB and CA) and the crossing on BC once,
    the three-intersection atom of Fig. "lookup_table"."""
    img = _quadrant()
    xy = np.array([[1.5, 1.5], [4.2, 1.1], [2.3, 4.1]])
    R = oracle.region3(img, xy, np.array([[0, 1, 2]]))
    qx = 4.2 + ((1.5 - 1.1) * (2.3 - 4.2)) / (4.1 - 1.1)  # from the lower-id end B
    assert R["n_events"] == 1 and R["n_inside"] == 0
    assert np.array_equal(R["xy"][3], [qx, 1.5])
    assert R["tri"].tolist() == [[0, 1, 3], [0, 3, 2]]
    assert R["label"].tolist() == [0, 1]
    mask, key, klass = R["code"] & 15, (R["code"] >> 6) & 63, R["code"] >> 12
    assert (mask == 2 | 4 | 8).all() and (key == 63).all() and (klass == 3).all()  # class (0,3)


def test_overlap_with_an_endpoint_on_the_edge():
    """Edge AB lies on the boundary line y = 1/2 + 1 for x <= 2.5; the boundary
    turns up at the pixel corner (2.5, 1.5), which lies on AB (an endpoint on
    the edge: one event), and leaves through CA.  The corner (1.5, 1.5) on AB,
    where the boundary runs straight along AB, is not an event (Alg. 1's
    overlap: embedded by AB itself).  One chord cutting corner A: App. G's
    single-segment case (b), turned so that the cut corner is A."""
    img = np.zeros((6, 6), np.uint8)
    img[2:, :3] = 1
    xy = np.array([[0.5, 1.5], [4.5, 1.5], [3.2, 4.0]])
    R = oracle.region3(img, xy, np.array([[0, 1, 2]]))
    qy = 1.5 + ((2.5 - 0.5) * (4.0 - 1.5)) / (3.2 - 0.5)  # from the lower-id end A
    assert R["n_events"] == 2 and R["n_inside"] == 0
    E, Q = 3, 4
    assert np.array_equal(R["xy"][E], [2.5, 1.5]) and np.array_equal(R["xy"][Q], [2.5, qy])
    A, B, C = 0, 1, 2
    assert R["tri"].tolist() == [[E, Q, A], [E, B, C], [Q, E, C]]
    assert R["label"].tolist() == [1, 0, 0]
    code = int(R["code"][0])
    assert (code & 15) == 2 | 8  # E on AB, Q on CA; the overlap is on AB too
    assert (code >> 6) & 63 == 1 and (code >> 4) & 3 == 1 and code >> 12 == 2  # key 1, sigma 1, class (0,2)


def test_glancing_contact_leaves_the_cell():
    """A cell touching the boundary only at a corner stays as it is (App. G
    single-segment cases (a) and (d))."""
    img = _quadrant()
    xy = np.array([[1.5, 1.5], [0.3, 0.4], [1.4, 0.3]])
    R = oracle.region3(img, xy, np.array([[0, 1, 2]]))
    assert R["tri"].tolist() == [[0, 1, 2]] and R["code"].tolist() == [0] and R["n_cut_cells"] == 0


def test_planted_mistakes_fail_the_pins():
    img = np.zeros((6, 6), np.uint8)
    img[2:, :3] = 1
    xy = np.array([[0.5, 1.5], [4.5, 1.5], [3.2, 4.0]])
    # 1: the straight-through corner on an overlapping edge becomes an event
    R = oracle.region3(img, xy, np.array([[0, 1, 2]]), plant=1)
    assert R["n_events"] == 3
    # 2: pieces oriented the wrong way: nested chords take the mirror key
    assert ((oracle.mesh_bitmap(_ELL, 4, 1)["code"] >> 6) & 63 == 5).any()
    with pytest.raises(AssertionError):
        _same_as_plain(_ELL, 4, 1, plant=2)
    # 3: the inside test takes the closed chord: vertices at pixel corners
    # (snapped, inserted) count as inside too
    im = synth.disk(64)
    T = P.preprocess(im, 2, 1, *TRIPLET)
    with pytest.raises((AssertionError, oracle.OracleError)):
        check_embedded(im, T, oracle.region3(im, T["xy"], T["tri"], plant=3))


def _corner_noise():
    # a 33 x 10 noise bitmap whose boundary meets the right border 1 px below
    # the top-right corner
    rng = np.random.default_rng(3)
    W, H = rng.integers(8, 40, 2)
    rng.integers(0, 3, (H // 3 + 1, W // 3 + 1))
    return (rng.random((H, W)) < 0.5).astype(np.uint8)


def test_the_preprocessed_mesh_must_cover_the_image(monkeypatch):
    """With the outer boundary snapping onto any border point, a vertex
    outside the image moves onto the right border 1 px below the corner and
    the corner is left uncovered: the per-label area pin fails."""
    img = _corner_noise()
    assert img.shape == (10, 33)
    T = P.preprocess(img, 2, 1, *TRIPLET)
    check_embedded(img, T, oracle.region3(img, T["xy"], T["tri"]))
    monkeypatch.setattr(P, "border_safe", lambda pid, W, H, reach: np.ones(len(pid), bool))
    T = P.preprocess(img, 2, 1, *TRIPLET)
    with pytest.raises(AssertionError):
        check_embedded(img, T, oracle.region3(img, T["xy"], T["tri"]))


# ---------------------------------------------------------------------------
# degenerate origins: the general path (base mesh, then Region III)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("hn,hd,stride", [(2, 1, 1), (4, 1, 1), (2, 3, 3)])
def test_every_4x4_bitmap_at_origin_minus_half(hn, hd, stride):
    """At origin (-1/2, -1/2) the lattice's row 0 lies on the image border and
    the vertices of every even row on vertical pixel lines: every cell the
    boundary meets is degenerate.  Every binary 4x4 bitmap (every third at
    h = 2/3) meshes to a correct embedding (the invariants of brute())."""
    n = oracle.brute_general(4, 4, hn, hd, -1, -1, 0, stride)
    assert n == (65536 + stride - 1) // stride


@pytest.mark.parametrize("ox,oy", [(-1, -1), (1, 0), (0, 3), (-1, 5)])
def test_degenerate_origins_on_label_images(ox, oy):
    rng = np.random.default_rng(100 + ox + 7 * oy)
    for hn, hd in [(2, 1), (4, 1), (2, 3)]:
        W, H = (int(x) for x in rng.integers(6, 24, 2))
        img = np.ascontiguousarray(rng.integers(0, 3, (H, W)).astype(np.uint8))
        R = oracle.mesh_general(img, hn, hd, ox, oy)
        check_embedded(img, dict(xy=R["base_xy"], tri=R["base_tri"]), R)
        # the degeneracy is there: lattice vertices exactly on pixel lines
        on_line = ((R["base_xy"] + 0.5) % 1.0 == 0.0).any(axis=1)
        assert on_line.any()
        # an event on an edge of the outer boundary (a lattice row on the
        # image border) adds one triangle, not two
        assert len(R["base_tri"]) + 2 * R["n_inside"] + R["n_events"] <= len(R["tri"])
        assert len(R["tri"]) <= len(R["base_tri"]) + 2 * R["n_inside"] + 2 * R["n_events"]


def test_general_path_at_an_integer_origin_is_the_plain_mesh():
    """At an integer origin the general path is the lattice path."""
    img = np.ascontiguousarray(synth.voronoi_labels(64, 12, 16))
    o = oracle.mesh_bitmap(img, 2, 1, 2, -4)
    g = oracle.mesh_general(img, 2, 1, 2, -4)
    assert np.abs(g["xy"][g["tri"]] - o["xy"][o["tri"]]).max() <= 1e-9
    assert np.array_equal(g["label"], o["label"]) and np.array_equal(g["code"], o["code"])


def _cell(img, xy):
    return oracle.region3(np.ascontiguousarray(img), np.array(xy, dtype=np.float64), np.array([[0, 1, 2]]))


def test_app_g_case_22_a1_star_from_the_inside_vertex():
    """App. G (2,2) case (a1): the inside vertex P2 with two boundary segments
    leaving it through two corners (each a vertex on the segment, counted twice
    by Alg. 1): the patch is the star from P2 over A, B, C, and the class is
    (2,2)."""
    img = _quadrant(8, 3, 2)  # boundary turns at (2.5, 1.5), runs +x and +y
    R = _cell(img, [[4.5, 1.5], [2.5, 3.5], [1.0, 0.0]])  # A, B on the two runs
    assert R["n_events"] == 0 and R["n_inside"] == 1 and np.array_equal(R["xy"][3], [2.5, 1.5])
    assert sorted(map(tuple, R["tri"].tolist())) == [(0, 1, 3), (0, 3, 2), (1, 2, 3)]  # A B P2, C A P2, B C P2
    code = int(R["code"][0])
    assert (code & 15) == 1 | 2 | 4 | 8 and code >> 12 == 6  # mask, class (2,2)


def test_app_g_case_12_a1_star_with_an_event():
    """App. G (1,2) case (a1): P2 inside, one segment leaving through Q on BC
    (one intersection), the other through corner C (two): the star from P2 over
    A, B, Q, C; class (1,2)."""
    img = _quadrant(8, 3, 2)
    R = _cell(img, [[1.0, 0.5], [4.0, 0.0], [2.5, 3.5]])  # C on the vertical run
    qx = 4.0 + ((1.5 - 0.0) * (2.5 - 4.0)) / (3.5 - 0.0)  # from the lower-id end B
    assert R["n_events"] == 1 and np.array_equal(R["xy"][3], [qx, 1.5]) and np.array_equal(R["xy"][4], [2.5, 1.5])
    A, B, C, Q, P = 0, 1, 2, 3, 4
    assert sorted(map(tuple, R["tri"].tolist())) == [(A, B, P), (A, P, C), (B, Q, P), (C, P, Q)]
    code = int(R["code"][0])
    assert (code & 15) == 1 | 4 | 8 and code >> 12 == 5  # class (1,2)


def test_app_g_case_13_vertex_to_an_endpoint_on_the_opposite_edge():
    """App. G's (1,3) case: a segment from corner B (a vertex on the segment)
    to the PSLG vertex P2 on edge CA (an endpoint on the edge), where a second
    segment only touches the cell: triangles A B P2 and P2 B C.  The class
    counts the pieces inside the cell (reading): the touching segment has none,
    so the cell reports (0,3) where the paper, counting every segment meeting
    the cell, names (1,3)."""
    img = np.zeros((6, 7), np.uint8)
    img[1:3, 3:] = 1  # left side x = 2.5 for y in [0.5, 2.5], turning at both ends
    R = _cell(img, [[4.0, 0.75], [2.5, 2.5], [1.0, 0.25]])  # CA passes through (2.5, 0.5)
    assert R["n_events"] == 1 and np.array_equal(R["xy"][3], [2.5, 0.5])
    A, B, C, P2 = 0, 1, 2, 3
    assert sorted(map(tuple, R["tri"].tolist())) == [(A, B, P2), (B, C, P2)]
    code = int(R["code"][0])
    assert (code & 15) == 2 | 4 | 8 and code >> 12 == 3  # class (0,3)


@pytest.mark.parametrize("seed", [1, 2])
def test_embedding_into_a_delaunay_mesh(seed):
    """Alg. 2 applies to any conforming mesh (Sec. 3.5): on a Delaunay mesh
    of random points, never preprocessed, the boundary is embedded with the
    same invariants (areas per label, label changes on pixel lines, boundary
    length)."""
    img = np.ascontiguousarray(synth.voronoi_labels(size=64, nseeds=7))
    xy, tri = synth.delaunay_mesh(64, 64, 900, seed)
    R = oracle.region3(img, xy, tri)
    check_embedded(img, {"xy": xy, "tri": tri}, R)
    assert R["n_cut_cells"] > 100 and R["n_events"] > 100
