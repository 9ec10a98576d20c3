"""Pins of the preprocessing oracle (Alg. 3): the thresholds' scale and
admissible range, a single pixel worked by hand, a constant image whose
border distances have a closed form, and on label images: every snap to the
nearest boundary point (a k-d tree query), every repelled vertex at distance
c from the boundary (dense sampling of the boundary), every elimination
within b, and the re-fanned mesh's triangle count, orientation and area
(that of the moved base mesh)."""
import math

import numpy as np
import pytest

import oracle
from oracle import preprocess as P
from paper_2602_19474_gb300 import synth

TRIPLET = (0.26, 0.125, 0.183)  # App. I's first admissible triplet


def test_thresholds_scale_and_admissible_range():
    A, B, C = P.thresholds_px(*TRIPLET, h=2.0)
    s = 2.0 / math.sqrt(0.45)
    assert abs(A - 0.26 * s) < 1e-15 and abs(B - 0.125 * s) < 1e-15 and abs(C - 0.183 * s) < 1e-15
    with pytest.raises(P.NotAdmissible):  # c >= a / sqrt(2): the paper's (0.24, 0.115, 0.17)
        P.thresholds_px(0.24, 0.115, 0.17, h=2.0)
    with pytest.raises(P.NotAdmissible):  # b >= a / 2
        P.thresholds_px(0.26, 0.13, 0.1, h=2.0)
    with pytest.raises(P.NotAdmissible):  # a >= h / 2
        P.thresholds_px(0.4, 0.1, 0.1, h=2.0)


def test_single_pixel_by_hand():
    # one pixel [-1/2, 1/2]^2; lattice vertex v(0,0) at the origin is 1/sqrt(2)
    # from all four corners, inside the snapping radius 0.775: it snaps, the
    # tie going to corner (0, 0) at (-1/2, -1/2)
    img = np.ones((1, 1), np.uint8)
    r = P.preprocess(img, 2, 1, *TRIPLET)
    xy0, _ = oracle.base_mesh(1, 1, 2, 1)
    k = int(np.nonzero((xy0 == [0.0, 0.0]).all(1))[0][0])
    assert r["status"][k] == 1 and r["snap"][k] == 0
    assert tuple(r["xy"][k]) == (-0.5, -0.5)
    pid, ppos = P.boundary_points(img)
    assert list(pid) == [0, 1, 2, 3] and np.array_equal(ppos, [[-0.5, -0.5], [0.5, -0.5], [-0.5, 0.5], [0.5, 0.5]])


def test_constant_image_border_in_closed_form():
    H, W = 9, 13
    img = np.full((H, W), 3, np.uint8)
    A, B, C = P.thresholds_px(*TRIPLET, h=2.0)
    xy0, cells = oracle.base_mesh(W, H, 2, 1)
    r = P.preprocess(img, 2, 1, *TRIPLET)
    corners = np.array([[-0.5, -0.5], [W - 0.5, -0.5], [-0.5, H - 0.5], [W - 0.5, H - 0.5]])
    lo, hi = np.array([-0.5, -0.5]), np.array([W - 0.5, H - 0.5])
    # the only boundary points are the image corners, onto which the base
    # mesh's outer boundary snaps too
    for k, v in enumerate(xy0):
        dc = np.sqrt(((corners - v) ** 2).sum(1))
        if dc.min() < A:  # snaps to the nearest image corner
            assert r["status"][k] == 1 and np.array_equal(r["xy"][k], corners[np.argmin(dc)])
            continue
        inside = (v > lo).all() and (v < hi).all()
        if inside:  # nearest point of the border: the nearest side
            ds = np.array([v[0] - lo[0], hi[0] - v[0], v[1] - lo[1], hi[1] - v[1]])
            s = int(np.argmin(ds))
            q = v.copy()
            q[s // 2] = lo[s // 2] if s % 2 == 0 else hi[s // 2]
            d = ds[s]
        else:
            q = np.clip(v, lo, hi)
            d = float(np.sqrt(((v - q) ** 2).sum()))
        if d < C:
            assert r["status"][k] == 2
            assert np.allclose(r["xy"][k], q + C * (v - q) / d, rtol=0, atol=1e-12)
        else:
            assert r["status"][k] == 0 and np.array_equal(r["xy"][k], v)


# a label boundary meeting the right border 1 px below the image corner:
# vertices outside the image lie within a of that border point, too near the
# corner to snap onto it
BORDER_BAND = np.zeros((10, 33), np.uint8)
BORDER_BAND[9:, :] = 1


def test_outer_boundary_snaps_only_far_from_image_corners():
    """Step 1 on BORDER_BAND: two vertices outside the image lie within a of
    the border point 1 px below the image corner and do not snap; every other
    vertex within a of a boundary point snaps onto the nearest."""
    from scipy.spatial import cKDTree

    img, h = BORDER_BAND, 2.0
    H, W = img.shape
    A, B, C = P.thresholds_px(*TRIPLET, h=h)
    xy0, cells = oracle.base_mesh(W, H, 2, 1)
    r = P.preprocess(img, 2, 1, *TRIPLET)
    outer = np.bincount(cells.ravel(), minlength=len(xy0)) < 6
    pid, ppos = P.boundary_points(img)
    d, near = cKDTree(ppos).query(xy0)
    pcx, pcy = ppos[near, 0] + 0.5, ppos[near, 1] + 0.5
    onx, ony = (pcx == 0) | (pcx == W), (pcy == 0) | (pcy == H)
    side = np.where(onx, np.minimum(pcy, H - pcy), np.minimum(pcx, W - pcx))
    safe = (onx & ony) | ((onx | ony) & (side >= h + A))
    assert ((d < A) & outer & ~safe).sum() == 2
    assert np.array_equal(r["status"] == 1, (d < A) & (~outer | safe))


def _sampled_boundary(img, step=1e-3):
    _, seg = P.boundary_edges(img)
    t = np.arange(0.0, 1.0 + step / 2, step)
    pts = seg[:, None, 0, :] + t[None, :, None] * (seg[:, None, 1, :] - seg[:, None, 0, :])
    return pts.reshape(-1, 2)


@pytest.mark.parametrize("name,img,hn,hd", [
    ("disk", synth.disk(), 2, 1),
    ("voronoi", synth.voronoi_labels(size=96, nseeds=12), 2, 1),
    ("noise_third", synth.noise_bitmap(synth.rng_for(17), 40, 32, 2.0), 2, 3),
])
def test_steps_on_label_images(name, img, hn, hd):
    from scipy.spatial import cKDTree

    h = hn / hd
    A, B, C = P.thresholds_px(*TRIPLET, h=h)
    xy0, cells = oracle.base_mesh(img.shape[1], img.shape[0], hn, hd)
    r = P.preprocess(img, hn, hd, *TRIPLET)
    V = len(xy0)
    pid, ppos = P.boundary_points(img)
    # Step 1: a snap is to the nearest boundary point, closer than a; a
    # vertex of the base mesh's outer boundary (fewer than six cells around
    # it) snaps only onto an image corner or a border point at least h + a
    # from the ends of its side
    outer = np.bincount(cells.ravel(), minlength=V) < 6
    d, near = cKDTree(ppos).query(xy0)
    H, W = img.shape
    pcx, pcy = ppos[near, 0] + 0.5, ppos[near, 1] + 0.5
    onx, ony = (pcx == 0) | (pcx == W), (pcy == 0) | (pcy == H)
    side = np.where(onx, np.minimum(pcy, H - pcy), np.minimum(pcx, W - pcx))
    safe = (onx & ony) | ((onx | ony) & (side >= h + A))
    snapped = r["status"] == 1
    assert np.array_equal(snapped, (d < A) & (~outer | safe))
    assert np.allclose(np.sqrt(((r["xy"][:V][snapped] - xy0[snapped]) ** 2).sum(1)), d[snapped], rtol=0, atol=1e-12)
    # Step 2: a repelled vertex was closer than c to the boundary and ends at
    # distance c from it (dense samples of the boundary pixel edges)
    tree = cKDTree(_sampled_boundary(img))
    before, _ = tree.query(xy0)
    after, _ = tree.query(r["xy"][:V])
    rep = r["status"] == 2
    kept = r["status"] == 0
    assert (before[rep] < C + 1e-3).all() and (before[kept] >= C - 1e-3).all()
    assert np.abs(after[rep] - C).max() <= 2e-3
    # Step 3: every elimination point is within b of its edge (after Steps 1-2),
    # and is the inserted vertex of its rank, at the pixel corner
    for k, (p, u, w) in enumerate(r["eliminations"]):
        q = ppos[np.searchsorted(pid, p)]
        assert tuple(r["xy"][V + k]) == (p % (img.shape[1] + 1) - 0.5, p // (img.shape[1] + 1) - 0.5)
        a_, b_ = r["xy"][u], r["xy"][w]
        t = np.clip(np.dot(q - a_, b_ - a_) / np.dot(b_ - a_, b_ - a_), 0, 1)
        assert np.linalg.norm(q - (a_ + t * (b_ - a_))) < B
    # re-fanned mesh: one more triangle per cell beside an eliminated edge,
    # every triangle counter-clockwise
    edges = {}
    for c_ in cells:
        for k in range(3):
            e = (min(c_[k], c_[(k + 1) % 3]), max(c_[k], c_[(k + 1) % 3]))
            edges[e] = edges.get(e, 0) + 1
    extra = sum(edges[(min(u, w), max(u, w))] for _, u, w in r["eliminations"])
    assert len(r["tri"]) == len(cells) + extra
    assert len(r["xy"]) == V + len(r["eliminations"])
    p3 = r["xy"][r["tri"]]
    area = (p3[:, 1, 0] - p3[:, 0, 0]) * (p3[:, 2, 1] - p3[:, 0, 1]) - (p3[:, 1, 1] - p3[:, 0, 1]) * (p3[:, 2, 0] - p3[:, 0, 0])
    assert (area > 0).all()
    # re-fanning two triangles around a point of their common quadrilateral
    # keeps the area: T covers what the moved base mesh covers.  An edge on
    # the outer boundary has one triangle (u, w, x); its halves (u, p, x) and
    # (p, w, x) cover it less the triangle (u, w, p) (signed areas:
    # A(u,w,x) = A(u,p,x) + A(p,w,x) + A(u,w,p) for any p)
    q3 = r["xy"][:V][cells]
    area0 = (q3[:, 1, 0] - q3[:, 0, 0]) * (q3[:, 2, 1] - q3[:, 0, 1]) - (q3[:, 1, 1] - q3[:, 0, 1]) * (q3[:, 2, 0] - q3[:, 0, 0])
    ccw = {(int(c_[k]), int(c_[(k + 1) % 3])) for c_ in cells for k in range(3)}
    lost = 0.0
    for k, (p, u, w) in enumerate(r["eliminations"]):
        if edges[(min(u, w), max(u, w))] != 1:
            continue
        a_, b_ = (u, w) if (int(u), int(w)) in ccw else (w, u)
        pa, pb, pc = r["xy"][a_], r["xy"][b_], r["xy"][V + k]
        lost += (pb[0] - pa[0]) * (pc[1] - pa[1]) - (pb[1] - pa[1]) * (pc[0] - pa[0])
    assert abs(area.sum() - (area0.sum() - lost)) <= 1e-9 * area0.sum()


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Each planted mistake makes a committed pin fail when that pin runs
    under it."""
    # ties going to the larger id: the hand-worked pixel snaps elsewhere
    def nearest_larger(vals, ids):
        m = vals.min(axis=1, keepdims=True)
        cand = np.where(vals == m, ids[None, :], -1)
        return np.argmax(cand, axis=1)

    good = P._nearest
    monkeypatch.setattr(P, "_nearest", nearest_larger)
    with pytest.raises(AssertionError):
        test_single_pixel_by_hand()
    monkeypatch.setattr(P, "_nearest", good)
    # repelled vertices moved the wrong way: the closed-form border positions fail
    real = P.region_one

    def wrong_way(xy0_, img_, A, C, *rest, **kw):
        out, status, snap = real(xy0_, img_, A, C, *rest, **kw)
        rep = status == 2
        out[rep] = 2 * xy0_[rep] - out[rep]
        return out, status, snap

    monkeypatch.setattr(P, "region_one", wrong_way)
    with pytest.raises(AssertionError):
        test_constant_image_border_in_closed_form()
    monkeypatch.setattr(P, "region_one", real)
    # the outer boundary snapping anywhere (no border rule): the Step 1 pin
    # on a Voronoi image fails
    monkeypatch.setattr(P, "border_safe", lambda pid, W, H, reach: np.ones(len(pid), bool))
    with pytest.raises(AssertionError):
        test_outer_boundary_snaps_only_far_from_image_corners()
