"""The boundary's limits: images up to 32768 px on a side, h_num up to 1024 and
h_den up to 63.  Strips of maximum width and height and both extreme grid
sizes are compared with the oracle in full; a 32768 x 32768 image (about 7e8
triangles) is checked by its closed-form counts and by oracle parity on
windows at its corners and centre, selected on the device so that the mesh
is never copied whole; sizes just past the limits are rejected."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import assert_same_mesh, ctx, gpu_mesh
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def run_both(img, hn, hd=1):
    g = gpu_mesh(img, hn, hd, stages=True)
    o = oracle.mesh_bitmap(img, hn, hd)
    assert_same_mesh(g, o, hn / hd, W=img.shape[1], stages=True)
    return g


def test_maximum_width_and_height_strips():
    run_both(synth.noise_bitmap(synth.rng_for(11), 32768, 40, 4.0), 2)
    run_both(synth.noise_bitmap(synth.rng_for(12), 36, 32768, 4.0).astype(np.uint16), 2)


def test_extreme_grid_sizes():
    # h = 1024 px: a few cells over the whole image; a small square inside one
    img = np.zeros((500, 700), np.uint8)
    img[200:203, 300:303] = 1
    run_both(img, 1024, 1)
    # h = 2/63 px: about 2.8e5 cells over a 12 x 10 image
    run_both(synth.noise_bitmap(synth.rng_for(13), 12, 10, 1.0), 2, 63)


def test_sizes_past_the_limits_are_rejected():
    c = ctx()
    with pytest.raises(sb.SbmtError):
        sb.mesh_bitmap(c, np.zeros((1, 32769), np.uint8), 2)
    with pytest.raises(sb.SbmtError):
        sb.mesh_bitmap(c, np.zeros((4, 4), np.uint8), 1026)
    with pytest.raises(sb.SbmtError):
        sb.mesh_bitmap(c, np.zeros((4, 4), np.uint8), 2, 65)


def test_misaligned_device_u16_image_is_rejected():
    """A device u16 image is read in place with 2-byte loads, so an odd pitch
    or an odd address is refused before any launch."""
    import ctypes

    import torch

    c = ctx()
    lib = sb.load()
    t = torch.zeros((8, 18), dtype=torch.int16, device="cuda")
    pr = sb._params(2)
    out = ctypes.c_uint64()
    for ptr, pitch in ((t.data_ptr(), 33), (t.data_ptr() + 1, 36)):
        im = sb.sbmt_image(16, 8, pitch, 2, ptr, 1)
        assert lib.mesh_bitmap(c, ctypes.byref(im), ctypes.byref(pr), ctypes.byref(out)) == sb.SBMT_EINVAL
    # the context stays usable
    m = sb.mesh_bitmap(c, t, 2)
    assert sb.mesh_query(c, m, -1).n_triangles > 0
    sb.mesh_release(c, m)


def _device_window_triangles(t, lo, hi, chunk=1 << 26):
    """Triangles of a device-resident mesh with every vertex inside the box
    [lo, hi]: their vertex coordinates (n, 3, 2), labels and codes on the host."""
    import torch

    xy, tri = t["xy"], t["tri"]
    lo_t = torch.tensor(lo, dtype=torch.float64, device="cuda")
    hi_t = torch.tensor(hi, dtype=torch.float64, device="cuda")
    P, L, C = [], [], []
    for s in range(0, tri.shape[0], chunk):
        tr = tri[s:s + chunk].long()
        p = xy[tr]  # (m, 3, 2)
        sel = ((p >= lo_t) & (p <= hi_t)).all(dim=2).all(dim=1)
        if sel.any():
            P.append(p[sel].cpu().numpy())
            L.append(t["label"][s:s + chunk][sel].cpu().numpy().view(np.uint16))
            C.append(t["code"][s:s + chunk][sel].cpu().numpy().view(np.uint16))
    if not P:
        return np.zeros((0, 3, 2)), np.zeros(0, np.uint16), np.zeros(0, np.uint16)
    return np.concatenate(P), np.concatenate(L), np.concatenate(C)


def _window_parity(tensors, crop_fn, hn, hd, x0, y0, w, hh):
    """Oracle parity on the interior of the crop [x0, x0+w) x [y0, y0+hh)."""
    from scipy.spatial import cKDTree

    h = hn / hd
    crop = crop_fn(x0, y0, w, hh)
    o = oracle.mesh_bitmap(crop, hn, hd, origin2x=-2 * x0, origin2y=-2 * y0)
    oxy = o["xy"] + np.array([x0, y0], dtype=np.float64)
    m = 2 * h + 2
    lo = [x0 - 0.5 + m, y0 - 0.5 + m]
    hi = [x0 + w - 0.5 - m, y0 + hh - 0.5 - m]
    gp, gl, gc = _device_window_triangles(tensors, lo, hi)
    P = oxy[o["tri"]]
    os_ = np.all((P >= lo) & (P <= hi), axis=(1, 2))
    assert len(gp) == os_.sum() and len(gp) > 0, (len(gp), os_.sum())
    d, idx = cKDTree(oxy).query(gp.reshape(-1, 2))
    assert d.max() <= 1e-6 * h, d.max()
    a = np.concatenate([idx.reshape(-1, 3), gl[:, None].astype(np.int64), gc[:, None].astype(np.int64)], axis=1)
    b = np.concatenate([o["tri"][os_].astype(np.int64), o["label"][os_, None].astype(np.int64),
                        o["code"][os_, None].astype(np.int64)], axis=1)
    a = a[np.lexsort(a.T[::-1])]
    b = b[np.lexsort(b.T[::-1])]
    assert np.array_equal(a, b), "window (%d, %d) differs from the oracle" % (x0, y0)
    return len(gp)


def test_maximum_image_32768_squared():
    import torch

    S = 32768
    # rectangles of 37 x 53 px, labels 0..6: boundary everywhere, with
    # junctions where four rectangles meet
    def labels(x0, y0, w, hh):
        y = np.arange(y0, y0 + hh)[:, None]
        x = np.arange(x0, x0 + w)[None, :]
        return (((x // 37) * 3 + (y // 53) * 5) % 7).astype(np.uint8)

    yy = torch.arange(S, device="cuda", dtype=torch.int32)[:, None]
    xx = torch.arange(S, device="cuda", dtype=torch.int32)[None, :]
    img = (((xx // 37) * 3 + (yy // 53) * 5) % 7).to(torch.uint8)
    c = ctx()
    m = sb.mesh_bitmap(c, img, 2, 1)
    v = sb.mesh_query(c, m, -1)
    del img
    assert v.status == 0
    assert v.n_triangles == v.n_cells + 2 * v.n_inside_vertices + 2 * v.n_events
    assert v.n_vertices == v.n_lattice_vertices + v.n_events + v.n_inside_vertices
    assert v.n_triangles > 6e8
    t = sb.view_tensors(v)
    n = 0
    for x0, y0 in [(0, 0), (S - 256, 0), (0, S - 256), (S - 256, S - 256), (S // 2 - 128, S // 2 - 128)]:
        n += _window_parity(t, labels, 2, 1, x0, y0, 256, 256)
    assert n > 50000
    del t
    sb.mesh_release(c, m)
    torch.cuda.empty_cache()
