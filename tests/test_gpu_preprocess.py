"""mesh_preprocess (Alg. 3, Steps 1-3) on the device against the
preprocessing oracle on the same image: vertex status, snap targets and
coordinates bit for bit (every decision and every moved coordinate is the
same sequence of double-precision operations), the eliminations, and the
triangles and labels exactly.  At full size the oracle runs on windows cut
from the image, and the device mesh must agree with it away from the
windows' edges; the thresholds' admissible range is enforced."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from oracle import preprocess as P
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu

TRIPLET = (0.26, 0.125, 0.183)  # App. I's first admissible triplet


def gpu_pre(img, hn, hd, a=TRIPLET[0], b=TRIPLET[1], c=TRIPLET[2], origin2x=0, origin2y=0):
    cx = ctx()
    m = sb.mesh_preprocess(cx, img, hn, hd, a, b, c, origin2x, origin2y)
    v = sb.mesh_query(cx, m, -1)
    out = sb.view_numpy(v)
    out.update(sb.pre_info_numpy(sb.mesh_preprocess_info(cx, m)))
    out["n_triangles"], out["n_vertices"] = v.n_triangles, v.n_vertices
    sb.mesh_release(cx, m)
    return out


def assert_same_pre(g, o):
    V = o["n_lattice_vertices"]
    assert g["n_lattice_vertices"] == V
    assert np.array_equal(g["status"], o["status"].astype(np.uint8))
    assert np.array_equal(g["snap"], o["snap"].astype(np.int32))
    assert g["xy"].shape == o["xy"].shape, (g["xy"].shape, o["xy"].shape)
    bad = np.nonzero((g["xy"] != o["xy"]).any(axis=1))[0]
    assert len(bad) == 0, "vertex %d: gpu %r oracle %r (status %d)" % (
        bad[0], g["xy"][bad[0]], o["xy"][bad[0]], o["status"][bad[0]] if bad[0] < V else -1)
    assert np.array_equal(g["elim"], o["eliminations"].astype(np.int32))
    assert g["tri"].shape == o["tri"].shape, (g["tri"].shape, o["tri"].shape)
    bad = np.nonzero((g["tri"] != o["tri"]).any(axis=1))[0]
    assert len(bad) == 0, "triangle %d: gpu %s oracle %s" % (bad[0], g["tri"][bad[0]], o["tri"][bad[0]])
    bad = np.nonzero(g["label"] != o["label"])[0]
    assert len(bad) == 0, "label of triangle %d: gpu %d oracle %d" % (bad[0], g["label"][bad[0]], o["label"][bad[0]])
    assert not g["code"].any()
    assert g["n_snapped"] == int((o["status"] == 1).sum()) and g["n_repelled"] == int((o["status"] == 2).sum())
    assert g["n_split_cells"] == len(o["tri"]) - g["n_cells"]
    assert np.allclose(g["thresholds_px"], o["thresholds_px"], rtol=0, atol=0)


CASES = [
    ("disk", lambda: synth.disk(), 2, 1),
    ("voronoi96", lambda: synth.voronoi_labels(size=96, nseeds=12), 2, 1),
    ("noise_third", lambda: synth.noise_bitmap(synth.rng_for(17), 40, 32, 2.0), 2, 3),
    ("noise_u16_h4", lambda: (synth.noise_bitmap(synth.rng_for(5), 70, 50, 3.0).astype(np.uint16) * 300), 4, 1),
    ("voronoi_fine", lambda: synth.voronoi_labels(size=48, nseeds=9), 2, 5),
    ("voronoi_coarse", lambda: synth.voronoi_labels(size=120, nseeds=10), 8, 1),
]


@pytest.mark.parametrize("name,make,hn,hd", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(name, make, hn, hd):
    img = make()
    g = gpu_pre(img, hn, hd)
    o = P.preprocess(img, hn, hd, *TRIPLET)
    assert_same_pre(g, o)
    assert len(o["eliminations"]) > 0


def test_other_triplets_and_origin():
    img = synth.voronoi_labels(size=80, nseeds=10)
    for (a, b, c) in [(0.3, 0.14, 0.2), (0.2, 0.0, 0.05), (0.5, 0.24, 0.35)]:
        h = 2.0
        if not (a * h / np.sqrt(0.45) < h / 2):
            continue
        assert_same_pre(gpu_pre(img, 2, 1, a, b, c), P.preprocess(img, 2, 1, a, b, c))
    assert_same_pre(gpu_pre(img, 2, 1, origin2x=-6, origin2y=4), P.preprocess(img, 2, 1, *TRIPLET, -6, 4))


def test_small_and_degenerate_images():
    # one pixel, a constant image (only the four image corners are boundary
    # points), one-pixel strips, a checkerboard (a boundary point at every corner)
    cases = [np.ones((1, 1), np.uint8), np.full((9, 13), 3, np.uint8), np.arange(37, dtype=np.uint8)[None, :] % 3,
             (np.arange(23, dtype=np.uint8)[:, None] // 4) % 2, (np.indices((12, 12)).sum(0) % 2).astype(np.uint8)]
    for img in cases:
        for hn, hd in [(2, 1), (2, 3)]:
            assert_same_pre(gpu_pre(img, hn, hd), P.preprocess(img, hn, hd, *TRIPLET))


def test_extreme_grid_sizes():
    # h = 2/63 px (about 1.4e5 lattice vertices over a 12 x 10 image: the
    # finest grid), h = 64 px (snapping radius near 25 px: the general paths
    # of the neighbourhood screens), and h = 6/5
    for img, hn, hd in [(synth.noise_bitmap(synth.rng_for(13), 12, 10, 1.0), 2, 63),
                        (synth.voronoi_labels(size=300, nseeds=6), 64, 1),
                        (synth.voronoi_labels(size=70, nseeds=7), 6, 5)]:
        assert_same_pre(gpu_pre(img, hn, hd), P.preprocess(img, hn, hd, *TRIPLET))


def test_thresholds_outside_the_admissible_range_are_rejected():
    img = synth.disk()
    for a, b, c in [(0.24, 0.115, 0.17), (0.26, 0.13, 0.1), (0.4, 0.1, 0.1), (0.0, 0.0, 0.0)]:
        with pytest.raises(sb.SbmtError) as e:
            sb.mesh_preprocess(ctx(), img, 2, 1, a, b, c)
        assert e.value.code == sb.SBMT_EINVAL
    with pytest.raises(sb.SbmtError) as e:  # mesh_bitmap's full Alg. 3 checks them too
        sb.mesh_bitmap(ctx(), img, 2, 1, mode=sb.SBMT_PREPROCESS)
    assert e.value.code == sb.SBMT_EINVAL


def test_angle_and_area_bounds_on_the_preprocessed_mesh():
    # the minimal-angle and minimal-area theorems' bounds, with the
    # thresholds in pixels, hold on the preprocessed mesh of these inputs
    import math

    for img, hn, hd in [(synth.voronoi_labels(size=256, nseeds=40), 2, 1),
                        (synth.noise_bitmap(synth.rng_for(21), 128, 96, 2.0), 2, 3)]:
        c = ctx()
        m = sb.mesh_preprocess(c, img, hn, hd)
        q = sb.mesh_quality(c, m)
        info = sb.mesh_preprocess_info(c, m)
        sb.mesh_release(c, m)
        A, B, C, e = info.a_px, info.b_px, info.c_px, hn / hd
        theta = min(math.atan(B / (e + A - math.sqrt(A * A - B * B))), math.atan(C / (e + A)))
        assert q["min_angle_deg"] > math.degrees(theta), (q["min_angle_deg"], math.degrees(theta))
        assert q["min_area"] > 0.5 * B * C, (q["min_area"], 0.5 * B * C)


def test_stage_records_of_a_preprocessed_mesh():
    # no Tier-G cells (stage 4 is empty); the kept stages of meshing do not exist
    c = ctx()
    m = sb.mesh_preprocess(c, synth.disk(), 2, 1)
    assert len(sb.mesh_stage(c, m, 4)) == 0
    with pytest.raises(sb.SbmtError):
        sb.mesh_stage(c, m, 1)
    sb.mesh_release(c, m)


def test_quality_and_projection_accept_the_preprocessed_mesh():
    img = synth.voronoi_labels(size=96, nseeds=12)
    c = ctx()
    m = sb.mesh_preprocess(c, img, 2, 1)
    q = sb.mesh_quality(c, m)
    o = P.preprocess(img, 2, 1, *TRIPLET)
    assert q["triangles"] == len(o["tri"])
    p = o["xy"][o["tri"]]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert abs(q["min_area"] - area.min()) <= 1e-12 * max(1.0, area.min())
    sb.mesh_release(c, m)


def _window_check(crop, hn, hd, x0, y0, w, hh, g_tri_xy, g_lab):
    """Oracle on the crop [x0, x0+w) x [y0, y0+hh) with the grid origin moved
    so that the lattice is the same; triangles with every vertex at least
    2h + 2 px inside the crop must match the device's."""
    from scipy.spatial import cKDTree

    h = hn / hd
    o = P.preprocess(crop, hn, hd, *TRIPLET, origin2x=-2 * x0, origin2y=-2 * y0)
    oxy = o["xy"] + np.array([x0, y0], dtype=np.float64)
    mrg = 2 * h + 2
    lo = np.array([x0 - 0.5 + mrg, y0 - 0.5 + mrg])
    hi = np.array([x0 + w - 0.5 - mrg, y0 + hh - 0.5 - mrg])
    P3 = oxy[o["tri"]]
    osel = np.all((P3 >= lo) & (P3 <= hi), axis=(1, 2))
    gsel = np.all((g_tri_xy >= lo) & (g_tri_xy <= hi), axis=(1, 2))
    assert osel.sum() == gsel.sum() and osel.sum() > 0, (osel.sum(), gsel.sum())
    a = np.concatenate([g_tri_xy[gsel].reshape(-1, 6), g_lab[gsel, None].astype(np.float64)], axis=1)
    b = np.concatenate([P3[osel].reshape(-1, 6), o["label"][osel, None].astype(np.float64)], axis=1)
    a = a[np.lexsort(a.T[::-1])]
    b = b[np.lexsort(b.T[::-1])]
    # coordinates: the crop's lattice differs from the image's by the
    # origin shift, an exact integer in double; moved coordinates to 1e-9
    assert np.abs(a[:, :6] - b[:, :6]).max() <= 1e-9, np.abs(a[:, :6] - b[:, :6]).max()
    assert np.array_equal(a[:, 6], b[:, 6])
    return int(osel.sum())


def test_full_size_windows():
    """voronoi8192 (8192^2 u16, h = 2): the device mesh against the oracle on
    five 160 x 160 windows, and the closed-form counts."""
    import torch

    img = synth.voronoi_labels()
    c = ctx()
    m = sb.mesh_preprocess(c, img, 2, 1)
    v = sb.mesh_query(c, m, -1)
    info = sb.mesh_preprocess_info(c, m)
    assert v.n_triangles == v.n_cells + info.n_split_cells
    assert v.n_vertices == v.n_lattice_vertices + info.n_eliminated
    assert info.n_split_cells <= 2 * info.n_eliminated and info.n_eliminated > 1000
    t = sb.view_tensors(v)
    S = img.shape[0]
    n = 0
    for x0, y0 in [(0, 0), (S - 160, 0), (0, S - 160), (S - 160, S - 160), (S // 2 - 80, S // 2 - 80)]:
        lo = torch.tensor([x0 - 1.0, y0 - 1.0], dtype=torch.float64, device="cuda")
        hi = torch.tensor([x0 + 161.0, y0 + 161.0], dtype=torch.float64, device="cuda")
        tr = t["tri"].long()
        # triangles near the window, chunked
        sel_xy, sel_lab = [], []
        for s0 in range(0, tr.shape[0], 1 << 25):
            p = t["xy"][tr[s0:s0 + (1 << 25)]]
            sel = ((p >= lo) & (p <= hi)).all(dim=2).all(dim=1)
            sel_xy.append(p[sel].cpu().numpy())
            sel_lab.append(t["label"][s0:s0 + (1 << 25)][sel].cpu().numpy().view(np.uint16))
        n += _window_check(img[y0:y0 + 160, x0:x0 + 160], 2, 1, x0, y0, 160, 160,
                           np.concatenate(sel_xy), np.concatenate(sel_lab))
    assert n > 20000
    del t
    sb.mesh_release(c, m)
    torch.cuda.empty_cache()
