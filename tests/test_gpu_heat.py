"""mesh_heat (App. H) on the device against the heat-diffusion oracle on the
same mesh: the solution after several backward-Euler steps and the peak per
step.  The device solves each step by conjugate gradients to a relative
residual of 1e-12 and sums in a different order, so the two agree to a
tolerance of 1e-8 of the pulse's amplitude rather than bit for bit.  At
full size the device's solution is checked against the oracle's operator:
the residual of the backward-Euler equation of its first step."""
import numpy as np
import pytest

import oracle
import paper_2602_19474_gb300 as sb
from gpu_util import ctx
from oracle import heat as H
from paper_2602_19474_gb300 import synth

pytestmark = pytest.mark.gpu


def run_gpu(m, L, alpha, dt, steps, x0, y0, sigma, amp=100.0, tol=1e-12):
    u, peaks, its = sb.mesh_heat(ctx(), m, L, alpha, dt, steps, x0, y0, sigma, amp, tol)
    return u.cpu().numpy(), np.array(peaks), its


CASES = [
    # image, h, label, alpha, dt, steps, pulse centre and width
    ("rectangle", lambda: np.pad(np.ones((40, 60), np.uint8), 10), 2, 1, 1, 500.0, 0.01, 5, (40.0, 30.0), 15.0),
    ("voronoi", lambda: synth.voronoi_labels(size=128, nseeds=12), 2, 1, None, 50.0, 0.05, 4, (64.0, 64.0), 20.0),
    ("voronoi_fine", lambda: synth.voronoi_labels(size=64, nseeds=6), 2, 3, None, 20.0, 0.05, 3, (30.0, 34.0), 10.0),
    ("disk", lambda: synth.disk(), 2, 1, 1, 100.0, 0.02, 6, (31.5, 31.5), 12.0),
]


@pytest.mark.parametrize("name,make,hn,hd,L,alpha,dt,steps,c,sigma", CASES, ids=[c[0] for c in CASES])
def test_parity_with_oracle(name, make, hn, hd, L, alpha, dt, steps, c, sigma):
    img = make()
    if L is None:
        L = int(np.bincount(img.ravel()).argmax())
    cx = ctx()
    m = sb.mesh_bitmap(cx, img, hn, hd)
    g = sb.view_numpy(sb.mesh_query(cx, m, -1))
    u, peaks, its = run_gpu(m, L, alpha, dt, steps, c[0], c[1], sigma)
    sb.mesh_release(cx, m)
    uo, po = H.heat(g["xy"], g["tri"], g["label"], L, alpha, dt, steps, c[0], c[1], sigma)
    assert np.abs(u - uo).max() <= 1e-8 * 100.0, np.abs(u - uo).max()
    assert np.allclose(peaks, po, rtol=0, atol=1e-8 * 100.0)
    assert all(0 < k < 10000 for k in its)
    _, free, _ = H.region(g["tri"], g["label"], L)
    assert (u[~free] == 0).all()


def test_on_the_preprocessed_mesh():
    img = synth.voronoi_labels(size=96, nseeds=10)
    L = int(np.bincount(img.ravel()).argmax())
    cx = ctx()
    m = sb.mesh_preprocess(cx, img, 2, 1)
    g = sb.view_numpy(sb.mesh_query(cx, m, -1))
    u, peaks, _ = run_gpu(m, L, 30.0, 0.05, 3, 48.0, 48.0, 15.0)
    sb.mesh_release(cx, m)
    uo, po = H.heat(g["xy"], g["tri"], g["label"], L, 30.0, 0.05, 3, 48.0, 48.0, 15.0)
    assert np.abs(u - uo).max() <= 1e-6, np.abs(u - uo).max()


def test_bad_parameters_and_no_convergence():
    cx = ctx()
    m = sb.mesh_bitmap(cx, synth.disk(), 2, 1)
    with pytest.raises(sb.SbmtError) as e:
        sb.mesh_heat(cx, m, 1, 100.0, -1.0, 2, 0.0, 0.0, 5.0)
    assert e.value.code == sb.SBMT_EINVAL
    with pytest.raises(sb.SbmtError) as e:  # one iteration cannot reach 1e-14
        sb.mesh_heat(cx, m, 1, 100.0, 0.05, 1, 31.5, 31.5, 12.0, tol=1e-14, max_iterations=1)
    assert e.value.code == sb.SBMT_ETIMEDOUT
    # a label with no triangles: nothing is free, u stays 0
    u, peaks, its = sb.mesh_heat(cx, m, 77, 100.0, 0.05, 2, 31.5, 31.5, 12.0)
    assert float(u.abs().max()) == 0.0 and peaks == [0.0, 0.0] and its == [0, 0]
    sb.mesh_release(cx, m)


def test_full_size_residual():
    """voronoi8192's mesh (8192^2 u16, h = 2), the most frequent label: the
    device's first step satisfies the oracle's backward-Euler equation to the
    solver's tolerance."""
    import scipy.sparse as sp

    img = synth.voronoi_labels()
    L = int(np.bincount(img.ravel()).argmax())
    cx = ctx()
    m = sb.mesh_bitmap(cx, img, 2, 1)
    # host copies of the mesh first: the views die with the mesh
    t = sb.view_tensors(sb.mesh_query(cx, m, -1))
    lab = t["label"].cpu().numpy().view(np.uint16)
    tri_all = t["tri"].cpu().numpy()
    xy = t["xy"].cpu().numpy()
    del t
    tri = tri_all[lab == L]
    alpha, dt, sigma = 500.0, 0.01, 127.0
    u, peaks, its = run_gpu(m, L, alpha, dt, 1, 4096.0, 4096.0, sigma, tol=1e-10)
    sb.mesh_release(cx, m)
    nv = len(xy)
    allsel, free, _ = H.region(tri_all, lab, L)
    K = H.stiffness(xy, tri, nv)
    M = H.lumped_mass(xy, tri, nv)
    u0 = np.where(free, H.pulse(xy, 4096.0, 4096.0, sigma, 100.0), 0.0)
    res = (sp.diags(M) @ u + alpha * dt * (K @ u) - M * u0)[free]
    rhs = (M * u0)[free]
    assert np.linalg.norm(res) <= 2e-10 * np.linalg.norm(rhs), np.linalg.norm(res) / np.linalg.norm(rhs)
    assert free.sum() > 100000 and 0 < peaks[0] <= 100.0


def test_runs_are_bit_identical():
    """The assembly and the solver's reductions sum in fixed orders (records
    placed by a scan, each vertex's mass and diagonal gathered in record
    order, rows sorted by column, block partials added in block order), so
    two runs give the same bits."""
    img = synth.voronoi_labels(size=700, nseeds=40)
    L = int(np.bincount(img.ravel()).argmax())
    cx = ctx()
    m = sb.mesh_bitmap(cx, img, 2, 1)
    a = run_gpu(m, L, 500.0, 0.01, 4, 350.0, 350.0, 60.0)
    b = run_gpu(m, L, 500.0, 0.01, 4, 350.0, 350.0, 60.0)
    sb.mesh_release(cx, m)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
