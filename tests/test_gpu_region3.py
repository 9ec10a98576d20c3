"""Alg. 3 in full on the device: mesh_bitmap with SBMT_PREPROCESS (Regions
I-II, the barrier, Region III: Alg. 2 on the preprocessed mesh) and
mesh_retriangulate, against the oracle's preprocessing followed by its
Region III on the same image.  Every decision and coordinate is the same
sequence of double-precision operations on both sides, so the meshes agree
bit for bit: coordinates, triangles, labels and codes.  At full size
(voronoi8192) the oracle runs on windows cut from the image.  The minimal
angle and minimal area theorems' bounds are asserted on the Tier-T cells at
the paper's edge length (h = 2/3 px, the reference edge sqrt(0.45) px)."""
import math

import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from oracle import preprocess as P
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu

TRIPLET = (0.26, 0.125, 0.183)  # App. I's first admissible triplet


def gpu_full(img, hn, hd, a=TRIPLET[0], b=TRIPLET[1], c=TRIPLET[2], origin2x=0, origin2y=0):
    cx = ctx()
    m = sb.mesh_preprocessed(cx, img, hn, hd, a, b, c, origin2x, origin2y)
    v = sb.mesh_query(cx, m, -1)
    out = sb.view_numpy(v)
    out.update(n_cut=v.n_cut_cells, n_tierG=v.n_tierG_cells, n_events=v.n_events, n_inside=v.n_inside_vertices,
               n_base=v.n_lattice_vertices, n_cells=v.n_cells, n_tierG_triangles=v.n_tierG_triangles)
    sb.mesh_release(cx, m)
    return out


def oracle_full(img, hn, hd, origin2x=0, origin2y=0):
    T = P.preprocess(img, hn, hd, *TRIPLET, origin2x=origin2x, origin2y=origin2y)
    return T, oracle.region3(img, T["xy"], T["tri"])


def assert_same(g, o):
    assert g["xy"].shape == o["xy"].shape, (g["xy"].shape, o["xy"].shape)
    bad = np.nonzero((g["xy"] != o["xy"]).any(axis=1))[0]
    assert len(bad) == 0, "vertex %d: gpu %r oracle %r" % (bad[0], g["xy"][bad[0]], o["xy"][bad[0]])
    assert g["tri"].shape == o["tri"].shape, (g["tri"].shape, o["tri"].shape)
    bad = np.nonzero((g["tri"] != o["tri"]).any(axis=1))[0]
    assert len(bad) == 0, "triangle %d: gpu %s oracle %s" % (bad[0], g["tri"][bad[0]], o["tri"][bad[0]])
    assert np.array_equal(g["label"], o["label"])
    bad = np.nonzero(g["code"] != o["code"])[0]
    assert len(bad) == 0, "code of triangle %d: gpu %d oracle %d" % (bad[0], g["code"][bad[0]], o["code"][bad[0]])
    assert (g["n_cut"], g["n_tierG"], g["n_events"], g["n_inside"]) == (
        o["n_cut_cells"], o["n_tierG_cells"], o["n_events"], o["n_inside"])
    assert g["n_base"] == o["n_vertices_grid"] and g["n_cells"] == o["n_cells"]
    key = (o["code"] >> 6) & 63
    assert g["n_tierG_triangles"] == int((key == 63).sum())


CASES = [
    ("disk64", lambda: synth.disk(), 2, 1),
    ("voronoi96", lambda: synth.voronoi_labels(size=96, nseeds=12), 2, 1),
    ("noise_third", lambda: synth.noise_bitmap(synth.rng_for(17), 40, 32, 2.0), 2, 3),
    ("noise_u16_h4", lambda: (synth.noise_bitmap(synth.rng_for(5), 70, 50, 3.0).astype(np.uint16) * 300), 4, 1),
    ("voronoi_fine", lambda: synth.voronoi_labels(size=48, nseeds=9), 2, 5),
    ("voronoi_coarse", lambda: synth.voronoi_labels(size=120, nseeds=10), 8, 1),
    ("pixels_h2", lambda: (np.random.default_rng(5).random((20, 26)) < 0.5).astype(np.uint8), 2, 1),
]


@pytest.mark.parametrize("name,make,hn,hd", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(name, make, hn, hd):
    img = np.ascontiguousarray(make())
    g = gpu_full(img, hn, hd)
    T, o = oracle_full(img, hn, hd)
    assert_same(g, o)
    assert o["n_cut_cells"] > 0 and (T["status"] == 1).any()


def test_retriangulate_a_preprocessed_mesh():
    """mesh_retriangulate on mesh_preprocess's handle gives mesh_bitmap's
    SBMT_PREPROCESS mesh; the base mesh stays valid."""
    img = synth.voronoi_labels(size=96, nseeds=12)
    c = ctx()
    t = sb.mesh_preprocess(c, img, 2, 1, *TRIPLET)
    r = sb.mesh_retriangulate(c, img, t)
    a = sb.view_numpy(sb.mesh_query(c, r, -1))
    base = sb.view_numpy(sb.mesh_query(c, t, -1))
    b = gpu_full(img, 2, 1)
    for k in ("xy", "tri", "label", "code"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["xy"][: len(base["xy"])], base["xy"])
    sb.mesh_release(c, r)
    sb.mesh_release(c, t)


def _min_angle_deg(P3):
    a = np.linalg.norm(P3[:, 1] - P3[:, 2], axis=1)
    b = np.linalg.norm(P3[:, 2] - P3[:, 0], axis=1)
    c = np.linalg.norm(P3[:, 0] - P3[:, 1], axis=1)
    A = np.arccos(np.clip((b * b + c * c - a * a) / (2 * b * c), -1, 1))
    B = np.arccos(np.clip((a * a + c * c - b * b) / (2 * a * c), -1, 1))
    return np.degrees(np.minimum(np.minimum(A, B), math.pi - A - B))


@pytest.mark.parametrize("name,make", [
    ("disk64", lambda: synth.disk()),
    ("voronoi160", lambda: synth.voronoi_labels(size=160, nseeds=40)),
    ("noise", lambda: synth.noise_bitmap(synth.rng_for(3), 96, 80, 2.0)),
])
def test_bounds_on_tier_t_cells_at_the_papers_edge(name, make):
    """The minimal-angle and minimal-area theorems (Sec. 3.3.4): at the
    paper's edge length every Tier-T sub-triangle has its smallest angle above
    min(atan(b / (e + a - sqrt(a^2 - b^2))), atan(c / (e + a))) and its area
    above b c / 2 (thresholds in pixels)."""
    img = np.ascontiguousarray(make())
    g = gpu_full(img, 2, 3)
    h = 2 / 3
    A, B, C = P.thresholds_px(*TRIPLET, h=h)
    theta = math.degrees(min(math.atan(B / (h + A - math.sqrt(A * A - B * B))), math.atan(C / (h + A))))
    key = (g["code"] >> 6) & 63
    tt = (key >= 1) & (key <= 15)
    assert tt.sum() > 1000
    P3 = g["xy"][g["tri"][tt]]
    area = 0.5 * ((P3[:, 1, 0] - P3[:, 0, 0]) * (P3[:, 2, 1] - P3[:, 0, 1]) - (P3[:, 1, 1] - P3[:, 0, 1]) * (P3[:, 2, 0] - P3[:, 0, 0]))
    assert _min_angle_deg(P3).min() > theta
    assert area.min() > 0.5 * B * C


def test_a_cell_over_the_limits_is_reported():
    """A checkerboard at h = 8 puts about 28 boundary vertices into a cell,
    past the per-cell limit of 16: SBMT_ECAPACITY, and the context stays
    usable."""
    img = (np.indices((48, 48)).sum(axis=0) % 2).astype(np.uint8)
    c = ctx()
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_preprocessed(c, img, 8, 1)
    assert e.value.code == sb.SBMT_ECAPACITY
    g = gpu_full(synth.disk(), 2, 1)
    assert g["n_cut"] > 0


def test_full_size_windows():
    """voronoi8192 (8192^2 u16, h = 2) through mesh_bitmap with
    SBMT_PREPROCESS: the device mesh against the oracle on five 160 x 160
    windows (grid origin moved so that the lattice is the same); triangles
    with every vertex at least 2h + 2 px inside a window must agree."""
    import torch

    img = synth.voronoi_labels()
    c = ctx()
    m = sb.mesh_preprocessed(c, img, 2, 1)
    v = sb.mesh_query(c, m, -1)
    # every event lies on an edge between two cells, and a cut cell has
    # 2 n_i + n_b - 2 triangles
    assert v.n_triangles == v.n_cells + 2 * v.n_inside_vertices + 2 * v.n_events
    assert v.n_vertices == v.n_lattice_vertices + v.n_events + v.n_inside_vertices
    t = sb.view_tensors(v)
    S = img.shape[0]
    n = 0
    for x0, y0 in [(0, 0), (S - 160, 0), (0, S - 160), (S - 160, S - 160), (S // 2 - 80, S // 2 - 80)]:
        lo = torch.tensor([x0 - 1.0, y0 - 1.0], dtype=torch.float64, device="cuda")
        hi = torch.tensor([x0 + 161.0, y0 + 161.0], dtype=torch.float64, device="cuda")
        tr = t["tri"].long()
        sel_xy, sel_lab, sel_code = [], [], []
        for s0 in range(0, tr.shape[0], 1 << 25):
            p = t["xy"][tr[s0:s0 + (1 << 25)]]
            sel = ((p >= lo) & (p <= hi)).all(dim=2).all(dim=1)
            sel_xy.append(p[sel].cpu().numpy())
            sel_lab.append(t["label"][s0:s0 + (1 << 25)][sel].cpu().numpy().view(np.uint16))
            sel_code.append(t["code"][s0:s0 + (1 << 25)][sel].cpu().numpy().view(np.uint16))
        g_xy, g_lab, g_code = np.concatenate(sel_xy), np.concatenate(sel_lab), np.concatenate(sel_code)
        crop = np.ascontiguousarray(img[y0:y0 + 160, x0:x0 + 160])
        _, o = oracle_full(crop, 2, 1, origin2x=-2 * x0, origin2y=-2 * y0)
        oxy = o["xy"] + np.array([x0, y0], dtype=np.float64)
        mrg = 2 * 2 + 2
        wlo = np.array([x0 - 0.5 + mrg, y0 - 0.5 + mrg])
        whi = np.array([x0 + 160 - 0.5 - mrg, y0 + 160 - 0.5 - mrg])
        P3 = oxy[o["tri"]]
        osel = np.all((P3 >= wlo) & (P3 <= whi), axis=(1, 2))
        gsel = np.all((g_xy >= wlo) & (g_xy <= whi), axis=(1, 2))
        assert osel.sum() == gsel.sum() and osel.sum() > 0, (osel.sum(), gsel.sum())
        a = np.concatenate([g_xy[gsel].reshape(-1, 6), g_lab[gsel, None], g_code[gsel, None]], axis=1)
        b = np.concatenate([P3[osel].reshape(-1, 6), o["label"][osel, None], o["code"][osel, None]], axis=1)
        a = a[np.lexsort(a.T[::-1])]
        b = b[np.lexsort(b.T[::-1])]
        # the crop's coordinates differ from the image's by an exact integer
        # shift; the events' rounding by a unit of the last place
        assert np.abs(a[:, :6] - b[:, :6]).max() <= 1e-9
        assert np.array_equal(a[:, 6:], b[:, 6:])
        n += int(osel.sum())
    assert n > 20000
    del t
    sb.mesh_release(c, m)
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# degenerate origins: mesh_bitmap's general path against the oracle's
# ---------------------------------------------------------------------------
def gpu_general(img, hn, hd, ox, oy):
    cx = ctx()
    m = sb.mesh_bitmap(cx, img, hn, hd, ox, oy)
    v = sb.mesh_query(cx, m, -1)
    out = sb.view_numpy(v)
    out.update(n_cut=v.n_cut_cells, n_tierG=v.n_tierG_cells, n_events=v.n_events, n_inside=v.n_inside_vertices,
               n_base=v.n_lattice_vertices, n_cells=v.n_cells, n_tierG_triangles=v.n_tierG_triangles)
    sb.mesh_release(cx, m)
    return out


@pytest.mark.parametrize("ox,oy", [(-1, -1), (1, 0), (0, 3), (-1, 5)])
def test_degenerate_origins_match_the_oracle(ox, oy):
    rng = np.random.default_rng(200 + ox + 7 * oy)
    for hn, hd in [(2, 1), (4, 1), (2, 3)]:
        W, H = (int(x) for x in rng.integers(6, 40, 2))
        img = np.ascontiguousarray(rng.integers(0, 3, (H, W)).astype(np.uint8))
        assert_same(gpu_general(img, hn, hd, ox, oy), oracle.mesh_general(img, hn, hd, ox, oy))
    img = synth.voronoi_labels(size=96, nseeds=12)
    assert_same(gpu_general(img, 2, 1, ox, oy), oracle.mesh_general(img, 2, 1, ox, oy))


def test_every_3x3_bitmap_at_origin_minus_half():
    for b in range(512):
        img = np.array([(b >> k) & 1 for k in range(9)], np.uint8).reshape(3, 3)
        assert_same(gpu_general(img, 2, 1, -1, -1), oracle.mesh_general(img, 2, 1, -1, -1))


def test_4x4_bitmaps_at_origin_minus_half():
    """Every 16th binary 4x4 bitmap at origin (-1/2, -1/2), h = 2 and 2/3."""
    for hn, hd in [(2, 1), (2, 3)]:
        for b in range(0, 65536, 16):
            img = np.array([(b >> k) & 1 for k in range(16)], np.uint8).reshape(4, 4)
            assert_same(gpu_general(img, hn, hd, -1, -1), oracle.mesh_general(img, hn, hd, -1, -1))


def test_degenerate_origin_refused_where_not_meshed():
    img = synth.disk()
    c = ctx()
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_bitmap(c, img, 2, 1, -1, -1, format=sb.SBMT_COMPACT)
    assert e.value.code == sb.SBMT_EINVAL
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_preprocess(c, img, 2, 1, 0.26, 0.125, 0.183, -1, -1)
    assert e.value.code == sb.SBMT_EINVAL


def _imported(img, xy, tri):
    """mesh_retriangulate on the caller's own mesh (mesh_import)."""
    c = ctx()
    b = sb.mesh_import(c, xy, tri)
    r = sb.mesh_retriangulate(c, img, b)
    v = sb.mesh_query(c, r, -1)
    g = sb.view_numpy(v)
    g.update(n_cut=v.n_cut_cells, n_tierG=v.n_tierG_cells, n_events=v.n_events, n_inside=v.n_inside_vertices,
             n_base=v.n_lattice_vertices, n_cells=v.n_cells, n_tierG_triangles=v.n_tierG_triangles)
    base = sb.view_numpy(sb.mesh_query(c, b, -1))
    assert np.array_equal(base["xy"], np.asarray(xy, np.float64)) and np.array_equal(base["tri"], np.asarray(tri))
    sb.mesh_release(c, r)
    sb.mesh_release(c, b)
    return g


def _quadrant(n, x0, y0):
    img = np.zeros((n, n), np.uint8)
    img[y0:, x0:] = 1
    return img


def _wedge():
    img = np.zeros((6, 7), np.uint8)
    img[1:3, 3:] = 1
    return img


def _overlap():
    img = np.zeros((6, 6), np.uint8)
    img[2:, :3] = 1
    return img


# single cells of App. G's cases that only Alg. 1's degenerate incidences
# reach (vertex on a segment, overlap, endpoint on an edge), the oracle's
# pins of the same cells stating the expected patches
APP_G_CELLS = [
    ("22_a1", lambda: _quadrant(8, 3, 2), [[4.5, 1.5], [2.5, 3.5], [1.0, 0.0]]),
    ("12_a1", lambda: _quadrant(8, 3, 2), [[1.0, 0.5], [4.0, 0.0], [2.5, 3.5]]),
    ("13", _wedge, [[4.0, 0.75], [2.5, 2.5], [1.0, 0.25]]),
    ("23_c1", lambda: _quadrant(6, 2, 2), [[1.5, 1.5], [4.2, 1.1], [2.3, 4.1]]),
    ("overlap", _overlap, [[0.5, 1.5], [4.5, 1.5], [3.2, 4.0]]),
    ("glancing", lambda: _quadrant(6, 2, 2), [[1.5, 1.5], [0.3, 0.4], [1.4, 0.3]]),
]


@pytest.mark.parametrize("name,make,xy", APP_G_CELLS, ids=[c[0] for c in APP_G_CELLS])
def test_app_g_degenerate_cells_match_the_oracle(name, make, xy):
    img = np.ascontiguousarray(make())
    tri = np.array([[0, 1, 2]], np.int32)
    g = _imported(img, np.array(xy), tri)
    assert_same(g, oracle.region3(img, np.array(xy, np.float64), tri))


@pytest.mark.parametrize("seed", [1, 2])
def test_retriangulate_a_delaunay_mesh(seed):
    """Alg. 2 on a mesh that is no lattice and was never preprocessed: every
    cell classified and retriangulated as the oracle does, bit for bit."""
    img = np.ascontiguousarray(synth.voronoi_labels(size=64, nseeds=7))
    xy, tri = synth.delaunay_mesh(64, 64, 900, seed)
    g = _imported(img, xy, tri)
    o = oracle.region3(img, xy, tri)
    assert_same(g, o)
    assert o["n_cut_cells"] > 100 and o["n_events"] > 100


def _near_lines(W, H, seed):
    """A Delaunay mesh whose points sit on pixel lines and corners or just
    off them: offsets below the device filters' fixed-point resolution
    (2^-37), near it (1e-13, 3e-11) and well above (1e-7), on both sides,
    so that the exact paths of the pixel-line tests and of the crossing
    filter decide."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    base, _ = synth.delaunay_mesh(W, H, 500, seed)
    pts = base.copy()
    offs = np.array([0.0, 2.0 ** -37, -2.0 ** -37, 1e-13, -1e-13, 3e-11, -3e-11, 1e-7, -1e-7])
    inner = np.arange(4 + 4 * ((W - 1) // 2), len(pts))
    pick = rng.choice(inner, size=len(inner) // 2, replace=False)
    for k, i in enumerate(pick):
        ax = k % 3  # x on a line, y on a line, or both (a corner)
        if ax in (0, 2):
            pts[i, 0] = np.floor(pts[i, 0]) + 0.5 + offs[rng.integers(len(offs))]
        if ax in (1, 2):
            pts[i, 1] = np.floor(pts[i, 1]) + 0.5 + offs[rng.integers(len(offs))]
    pts = np.clip(pts, -0.5, [W - 0.5, H - 0.5])
    _, keep = np.unique(np.round(pts, 6), axis=0, return_index=True)
    pts = pts[np.sort(keep)]
    tri = Delaunay(pts).simplices.astype(np.int32)
    P = pts[tri]
    o = (P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) - (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0])
    tri[o < 0] = tri[o < 0][:, [0, 2, 1]]
    return pts, np.ascontiguousarray(tri[np.abs(o) > 1e-9])


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_retriangulate_points_on_and_near_pixel_lines(seed):
    img = np.ascontiguousarray(synth.voronoi_labels(size=48, nseeds=9))
    xy, tri = _near_lines(48, 48, seed)
    o = oracle.region3(img, xy, tri)
    g = _imported(img, xy, tri)
    assert_same(g, o)
    assert o["n_cut_cells"] > 50
