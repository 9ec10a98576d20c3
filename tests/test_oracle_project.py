"""Pins of the field-projection oracle: a triangle whose pixel overlaps are
known in closed form, box clipping against its definition, a constant field,
the label image as the field (every triangle lies in one label region, so
its mean is its label), conservation of the field's integral, brute-force
quadrature on random triangles, and bilinear vertex values of a linear
field."""
import math

import numpy as np

import oracle
from oracle import project as P
from paper_2602_19474_gb300 import synth


def test_closed_form_triangle():
    # legs of 2 px from the corner (-0.5, -0.5): pixel (0,0) is covered, (1,0)
    # and (0,1) half covered, (1,1) touched at one point; |T| = 2
    f = np.array([[1.0, 10.0, 0.0], [100.0, 1000.0, 0.0], [0.0, 0.0, 0.0]], np.float32)
    xy = np.array([[-0.5, -0.5], [1.5, -0.5], [-0.5, 1.5]])
    v = P.project_triangles(xy, [[0, 1, 2]], f)[0]
    assert abs(v - (1.0 + 0.5 * 10.0 + 0.5 * 100.0) / 2.0) < 1e-12


def test_box_area():
    t = [(0.0, 0.0), (4.0, 0.0), (0.0, 4.0)]
    assert abs(P.tri_box_area(t, -1, 5, -1, 5) - 8.0) < 1e-12  # whole triangle
    assert abs(P.tri_box_area(t, 0.5, 1.5, 0.5, 1.5) - 1.0) < 1e-12  # whole box
    assert abs(P.tri_box_area(t, 3, 5, 0, 1) - 0.5) < 1e-12  # the tip (3,0)-(4,0)-(3,1)
    assert P.tri_box_area(t, 3, 5, 3, 5) == 0.0
    # a box cut by the hypotenuse x + y = 4: [1,3] x [1,3] keeps its lower half
    assert abs(P.tri_box_area(t, 1, 3, 1, 3) - 2.0) < 1e-12


def test_constant_field_and_outside():
    img = synth.disk()
    m = oracle.mesh_bitmap(img, 2, 1)
    f = np.full(img.shape, 3.25, np.float32)
    v = P.project_triangles(m["xy"], m["tri"], f)
    inside = m["label"] != 0xFFFF
    assert np.allclose(v[inside], 3.25, rtol=0, atol=1e-12)
    assert (v[~inside] == 0.0).all()


def test_label_field_gives_labels():
    # conformity: each triangle lies inside one label region
    for img, hn, hd in [(synth.disk(), 2, 1), (synth.voronoi_labels(size=160, nseeds=24), 4, 1),
                        (synth.voronoi_labels(size=120, nseeds=12), 2, 3)]:
        m = oracle.mesh_bitmap(img, hn, hd)
        v = P.project_triangles(m["xy"], m["tri"], img.astype(np.float32))
        inside = m["label"] != 0xFFFF
        err = np.abs(v[inside] - m["label"][inside].astype(np.float64))
        assert err.max() <= 1e-9 * max(1, img.max()), err.max()


def test_conservation():
    rng = np.random.default_rng(7)
    img = synth.voronoi_labels(size=128, nseeds=20)
    m = oracle.mesh_bitmap(img, 2, 1)
    f = rng.standard_normal(img.shape).astype(np.float32)
    v = P.project_triangles(m["xy"], m["tri"], f)
    p = m["xy"][m["tri"]]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    total = float(f.astype(np.float64).sum())
    assert abs((v * area).sum() - total) <= 1e-9 * np.abs(f).sum()
    # and per label region
    for lab in np.unique(img)[:5]:
        sel = m["label"] == lab
        assert abs((v[sel] * area[sel]).sum() - f[img == lab].astype(np.float64).sum()) <= 1e-9 * np.abs(f).sum()


def test_brute_force_quadrature():
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, (12, 12)).astype(np.float32)
    N = 700
    for _ in range(6):
        t = rng.uniform(0.0, 10.0, (3, 2))
        area = 0.5 * abs((t[1, 0] - t[0, 0]) * (t[2, 1] - t[0, 1]) - (t[1, 1] - t[0, 1]) * (t[2, 0] - t[0, 0]))
        if area < 2.0:
            continue
        lo, hi = t.min(0), t.max(0)
        xs = lo[0] + (np.arange(N) + 0.5) * (hi[0] - lo[0]) / N
        ys = lo[1] + (np.arange(N) + 0.5) * (hi[1] - lo[1]) / N
        X, Y = np.meshgrid(xs, ys)

        def side(a, b):
            return (b[0] - a[0]) * (Y - a[1]) - (b[1] - a[1]) * (X - a[0])

        s0, s1, s2 = side(t[0], t[1]), side(t[1], t[2]), side(t[2], t[0])
        inside = ((s0 >= 0) & (s1 >= 0) & (s2 >= 0)) | ((s0 <= 0) & (s1 <= 0) & (s2 <= 0))
        vals = f[np.floor(Y + 0.5).astype(int), np.floor(X + 0.5).astype(int)]
        quad = vals[inside].mean()
        v = P.project_triangles(t, [[0, 1, 2]], f)[0]
        # midpoint sampling misplaces at most the samples within a sample
        # spacing of the triangle's edges or of the pixel lines it crosses
        d = max(hi - lo) / N
        per = sum(np.hypot(*(t[(k + 1) % 3] - t[k])) for k in range(3))
        lines = (math.ceil(hi[0]) - math.floor(lo[0]) + math.ceil(hi[1]) - math.floor(lo[1])) * max(hi - lo)
        tol = 4 * d * (per + lines) / area * np.abs(f).max()
        assert abs(v - quad) <= tol, (v, quad, tol)


def test_vertex_values_linear_field():
    H, W = 40, 50
    y, x = np.mgrid[0:H, 0:W]
    f = (3.0 * x - 2.0 * y + 5.0).astype(np.float32)
    rng = np.random.default_rng(1)
    pts = np.concatenate([rng.uniform([0, 0], [W - 1, H - 1], (200, 2)), [[-3.0, 10.0], [W + 2.0, H + 5.0]]])
    v = P.vertex_values(pts, f)
    inner = v[:200]
    assert np.allclose(inner, 3 * pts[:200, 0] - 2 * pts[:200, 1] + 5, rtol=0, atol=1e-9)
    # clamped: (-3, 10) samples (0, 10); (W+2, H+5) samples (W-1, H-1)
    assert abs(v[200] - (0 - 20 + 5)) < 1e-12
    assert abs(v[201] - (3 * (W - 1) - 2 * (H - 1) + 5)) < 1e-12
