"""mesh_quality on the device against the quality oracle on the same mesh,
and the paper's regime (h < 1 px) on a star and a blob: no Tier-G cells,
the quality measures reported."""
import math

import numpy as np
import pytest

import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from oracle import quality as Q
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def gpu_quality(img, hn, hd):
    c = ctx()
    m = sb.mesh_bitmap(c, img, hn, hd)
    v = sb.mesh_query(c, m, -1)
    mesh = sb.view_numpy(v)
    q = sb.mesh_quality(c, m)
    sb.mesh_release(c, m)
    return mesh, q


def check_against_oracle(mesh, q):
    o = Q.quality(mesh["xy"], mesh["tri"])
    assert q["triangles"] == o["triangles"]
    assert abs(q["min_angle_deg"] - o["min_angle_deg"]) <= 1e-9
    assert math.isclose(q["min_area"], o["min_area"], rel_tol=1e-12)
    assert q["equilateral"] == o["equilateral"]
    assert math.isclose(q["area_mean"], o["area_mean"], rel_tol=1e-12)
    assert abs(q["area_var"] - o["area_var"]) <= 1e-9 * o["area_var"] + 1e-12 * o["area_mean"] ** 2
    assert math.isclose(q["ar_max"], o["ar_max"], rel_tol=1e-12)
    # percentiles are taken over AR rounded to single precision
    for k in ("ar_median", "ar_p95"):
        assert q[k] == float(np.float32(o[k])), (k, q[k], o[k])
    # counts by thresholds: equal up to angles within 1e-9 degrees of a
    # threshold or bin edge, where the two atan2 implementations may differ
    ang = o["min_angles"]
    near = lambda edge: int((np.abs(ang - edge) <= 1e-9).sum())
    assert abs(q["slivers"] - o["slivers"]) <= near(5.0)
    slack = sum(near(2.0 * k) for k in range(1, 30))
    assert np.abs(np.array(q["angle_hist"]) - o["angle_hist"]).sum() <= 2 * slack
    return o


@pytest.mark.parametrize("name,img,hn,hd", [
    ("disk", synth.disk(), 2, 1),
    ("noise", synth.noise_batch(n=3, lo=200, hi=400, first=1)[0], 2, 1),
    ("ellipses", synth.ellipses(size=400, n=30, amin=8, amax=70), 4, 1),
    ("voronoi", synth.voronoi_labels(size=512, nseeds=64), 2, 1),
])
def test_quality_matches_oracle(name, img, hn, hd):
    mesh, q = gpu_quality(img, hn, hd)
    check_against_oracle(mesh, q)


@pytest.mark.parametrize("name", ["star", "blob"])
def test_paper_regime_quality(name):
    img = synth.star() if name == "star" else synth.blob()
    c = ctx()
    m = sb.mesh_bitmap(c, img, 2, 3)
    v = sb.mesh_query(c, m, -1)
    assert v.n_tierG_cells == 0  # Lemma 3.1's regime: every cut cell takes the table
    mesh = sb.view_numpy(v)
    q = sb.mesh_quality(c, m)
    sb.mesh_release(c, m)
    check_against_oracle(mesh, q)
    # uncut cells are equilateral: the median AR is 2 / sqrt(3)
    assert abs(q["ar_median"] - float(np.float32(2 / math.sqrt(3)))) == 0.0
    assert q["equilateral"] > q["triangles"] // 2
