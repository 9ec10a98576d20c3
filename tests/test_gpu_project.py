"""mesh_project on the device against the projection oracle on the same mesh:
per-triangle means of a pixel field and bilinear vertex values, with a
tolerance derived from single-precision arithmetic in a frame at each
triangle's first vertex; at full size, conservation of the field's integral
and the label image projecting onto the labels."""
import numpy as np
import pytest

import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from oracle import project as P
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def smooth_field(H, W, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    f = np.sin(x / 17.0 + rng.uniform(0, 6)) * np.cos(y / 23.0) + 0.25 * rng.standard_normal((H, W))
    return f.astype(np.float32)


def project_on_gpu(c, m, v, field):
    import torch

    tv = torch.empty(v.n_triangles, dtype=torch.float32, device="cuda")
    vv = torch.empty(v.n_vertices, dtype=torch.float32, device="cuda")
    sb.mesh_project(c, m, torch.from_numpy(field).cuda(), tv, vv)
    sb.mesh_query(c, m, -1)
    return tv.cpu().numpy(), vv.cpu().numpy()


def triangle_tolerance(xy, tri, W, H, frange):
    """Rounding the frame coordinates (relative 2^-24 each) moves every
    pixel weight by a few eps * L (L + 1), L the longest edge; the mean moves
    by the weights' total error / |T| times the field's range.  Thin
    triangles (L (L + 1) > 64 |T|) are computed in double precision."""
    p = xy[tri]
    e = [p[:, (k + 1) % 3] - p[:, k] for k in range(3)]
    L = np.sqrt(np.max([(d * d).sum(1) for d in e], axis=0))
    area = 0.5 * np.abs(e[0][:, 0] * (-e[2][:, 1]) - e[0][:, 1] * (-e[2][:, 0]))
    q = np.minimum(L * (L + 1) / np.maximum(area, 1e-300), 64.0 * 1.01)
    c0 = np.clip(np.floor(p[:, :, 0].min(1) + 0.5), 0, W - 1)
    c1 = np.clip(np.floor(p[:, :, 0].max(1) + 0.5), 0, W - 1)
    r0 = np.clip(np.floor(p[:, :, 1].min(1) + 0.5), 0, H - 1)
    r1 = np.clip(np.floor(p[:, :, 1].max(1) + 0.5), 0, H - 1)
    npieces = (c1 - c0 + 1) * (r1 - r0 + 1)
    return 32 * EPS32 * q * npieces * frange


@pytest.mark.parametrize("name,img,hn,hd", [
    ("disk", synth.disk(), 2, 1),
    ("voronoi", synth.voronoi_labels(size=600, nseeds=60), 2, 1),
    ("noise_h8", synth.noise_batch(n=2, lo=300, hi=500, first=2)[1], 8, 1),
    ("star_third", synth.star(), 2, 3),
])
def test_project_matches_oracle(name, img, hn, hd):
    c = ctx()
    H, W = img.shape
    m = sb.mesh_bitmap(c, img, hn, hd)
    v = sb.mesh_query(c, m, -1)
    mesh = sb.view_numpy(v)
    f = smooth_field(H, W, seed=hn * 31 + H)
    tv, vv = project_on_gpu(c, m, v, f)
    sb.mesh_release(c, m)
    o_t = P.project_triangles(mesh["xy"], mesh["tri"], f)
    o_v = P.vertex_values(mesh["xy"], f)
    frange = float(f.max() - f.min())
    tol = triangle_tolerance(mesh["xy"], mesh["tri"], W, H, frange) + 4 * EPS32 * np.abs(o_t)
    err = np.abs(tv - o_t)
    bad = np.nonzero(err > tol)[0]
    assert len(bad) == 0, "triangle %d: gpu %r oracle %r tol %r" % (bad[0], tv[bad[0]], o_t[bad[0]], tol[bad[0]])
    assert (tv[mesh["label"] == 0xFFFF] == 0).all()
    # bilinear: three roundings of the weights, one of the sum
    assert np.abs(vv - o_v).max() <= 16 * EPS32 * np.abs(f).max()


def test_label_field_and_conservation_full_size():
    # 4096^2 Voronoi labels at h = 2: every triangle lies in one label
    # region, so projecting the label image gives each triangle its label,
    # and the field's integral is kept overall
    import torch

    c = ctx()
    img = synth.voronoi_labels(size=4096, nseeds=1024)
    m = sb.mesh_bitmap(c, img, 2, 1)
    v = sb.mesh_query(c, m, -1)
    t = sb.view_tensors(v)
    lab = t["label"].to(torch.int32) & 0xFFFF
    field = torch.from_numpy(img.astype(np.float32)).cuda()
    tv = torch.empty(v.n_triangles, dtype=torch.float32, device="cuda")
    sb.mesh_project(c, m, field, tv, None)
    sb.mesh_query(c, m, -1)
    inside = lab != 0xFFFF
    assert torch.equal(tv[~inside], torch.zeros_like(tv[~inside]))
    err = (tv[inside].double() - lab[inside].double()).abs()
    top = max(1, int(img.max()))
    assert err.max().item() <= 1e-3 * top, err.max().item()
    assert (err <= 1e-5 * top).double().mean().item() > 0.999
    # conservation of a random field: sum of mean * area = sum of the pixels
    rng = np.random.default_rng(5)
    f = rng.standard_normal(img.shape).astype(np.float32)
    sb.mesh_project(c, m, torch.from_numpy(f).cuda(), tv, None)
    sb.mesh_query(c, m, -1)
    xy, tri = t["xy"], t["tri"].long()
    p = xy[tri]
    area = 0.5 * ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                  - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])).abs()
    total = (tv.double() * area).sum().item()
    ref = float(f.astype(np.float64).sum())
    assert abs(total - ref) <= 1e-5 * float(np.abs(f).astype(np.float64).sum()), (total, ref)
    sb.mesh_release(c, m)


def test_host_field_and_errors():
    import torch

    c = ctx()
    img = synth.voronoi_labels(size=300, nseeds=30)
    m = sb.mesh_bitmap(c, img, 4, 1)
    v = sb.mesh_query(c, m, -1)
    f = smooth_field(*img.shape, seed=9)
    a = torch.empty(v.n_triangles, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    sb.mesh_project(c, m, f, a, None)  # host field
    sb.mesh_project(c, m, torch.from_numpy(f).cuda(), b, None)
    sb.mesh_query(c, m, -1)
    assert torch.equal(a, b)
    with pytest.raises(sb.SbmtError):
        sb.mesh_project(c, m, f[:-1], a, None)  # wrong size
    sb.mesh_release(c, m)
    k = sb.mesh_bitmap(c, img, 4, 1, format=sb.SBMT_COMPACT)
    with pytest.raises(sb.SbmtError):
        sb.mesh_project(c, k, f, a, None)
    sb.mesh_release(c, k)
