"""Pins of the quality-measure oracle against closed forms: the equilateral,
right isosceles and thin triangles, nearest-rank percentiles, and the
lattice of a constant image (uncut cells are equilateral with area
sqrt(3) h^2 / 4 and AR 2 / sqrt(3))."""
import math

import numpy as np

import oracle
from oracle import quality as Q

S3 = math.sqrt(3.0)


def q_of(points, tris):
    return Q.quality(np.asarray(points, float), np.asarray(tris))


def test_equilateral_triangle():
    r = q_of([(0, 0), (2, 0), (1, S3)], [(0, 1, 2)])
    assert abs(r["min_angle_deg"] - 60.0) < 1e-12
    assert abs(r["ar_max"] - 2 / S3) < 1e-12
    assert r["equilateral"] == 1 and r["slivers"] == 0
    assert abs(r["min_area"] - S3) < 1e-12
    assert r["angle_hist"][29] == 1 and r["angle_hist"].sum() == 1


def test_right_isosceles_and_thin_triangles():
    r = q_of([(0, 0), (1, 0), (0, 1), (10, 0), (20, 0), (15, 0.1)], [(0, 1, 2), (3, 4, 5)])
    # right isosceles: 45 degrees, AR = 2 (longest^2 / 2A = 2 / 1)
    ang, area, ar, equi = Q.triangle_measures(np.array([(0, 0), (1, 0), (0, 1)], float), np.array([(0, 1, 2)]))
    assert abs(ang[0] - 45.0) < 1e-12 and abs(ar[0] - 2.0) < 1e-12 and abs(area[0] - 0.5) < 1e-15
    assert not equi[0]
    # thin: smallest angle atan(0.1 / 5), AR = 100 / (2 * 0.5) = 100
    assert abs(r["min_angle_deg"] - math.degrees(math.atan(0.1 / 5))) < 1e-9
    assert abs(r["ar_max"] - 100.0) < 1e-9
    assert r["slivers"] == 1 and r["equilateral"] == 0
    assert r["angle_hist"][22] == 1 and r["angle_hist"][0] == 1


def test_nearest_rank():
    s = np.arange(1, 21, dtype=float)
    assert Q.nearest_rank(s, 0.5) == 10.0
    assert Q.nearest_rank(s, 0.95) == 19.0
    assert Q.nearest_rank(np.array([7.0]), 0.95) == 7.0


def test_constant_image_lattice():
    img = np.zeros((160, 160), np.uint8)
    h = 4.0
    m = oracle.mesh_bitmap(img, 4, 1)
    r = Q.quality(m["xy"], m["tri"])
    uncut = m["n_cells"] - m["n_cut_cells"]
    assert r["equilateral"] >= uncut > r["triangles"] // 2
    assert abs(r["ar_median"] - 2 / S3) < 1e-12
    ang, area, ar, equi = Q.triangle_measures(m["xy"], m["tri"])
    uncut_tris = m["code"] == 0
    assert uncut_tris.sum() == uncut and equi[uncut_tris].all()
    assert np.allclose(area[uncut_tris], S3 * h * h / 4, rtol=1e-12)
    assert np.allclose(ar[uncut_tris], 2 / S3, rtol=1e-12)
    # the in-image triangles tile the image rectangle exactly
    assert abs(area[m["label"] != 0xFFFF].sum() - 160 * 160) < 1e-6


def test_area_mean_and_population_variance_closed_form():
    # right triangles of areas 1, 2 and 6: mean 3, population variance
    # ((1-3)^2 + (2-3)^2 + (6-3)^2) / 3 = 14/3 (the sample variance would be 7)
    pts = [(0, 0), (2, 0), (0, 1), (10, 0), (12, 0), (10, 2), (20, 0), (23, 0), (20, 4)]
    r = q_of(pts, [(0, 1, 2), (3, 4, 5), (6, 7, 8)])
    assert abs(r["area_mean"] - 3.0) < 1e-15
    assert abs(r["area_var"] - 14.0 / 3.0) < 1e-14
    assert abs(r["min_area"] - 1.0) < 1e-15


def test_area_mean_over_every_triangle_of_a_mesh():
    # the patches tile their cells, so the areas of all T triangles (those
    # outside the image included) add up to n_cells equilateral cells of
    # area sqrt(3) h^2 / 4
    from paper_2602_19474_gb300 import synth

    img = synth.noise_batch(n=2, lo=60, hi=90, first=2)[1]
    for hn in (2, 4):
        m = oracle.mesh_bitmap(img, hn, 1)
        r = Q.quality(m["xy"], m["tri"])
        cell = S3 * hn * hn / 4.0
        assert abs(r["area_mean"] * r["triangles"] - m["n_cells"] * cell) < 1e-9 * m["n_cells"] * cell
        # variance from the closed-form second moment of the same areas
        _, area, _, _ = Q.triangle_measures(m["xy"], m["tri"])
        mean = m["n_cells"] * cell / len(area)
        assert abs(r["area_var"] - (np.sum(area * area) / len(area) - mean * mean)) < 1e-9 * cell * cell
