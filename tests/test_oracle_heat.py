"""Pins of the heat-diffusion oracle (App. H): the lumped mass of a label's
triangles sums to the label's pixel count (the mesh tiles each label region
exactly), the cotangent stiffness annihilates constants everywhere and
linear functions at free vertices (exactness of linear elements), the
lattice's equilateral triangles have cotangent 1/sqrt3, and on a rectangle
the first Dirichlet eigenmode decays by the backward-Euler factor of its
analytic eigenvalue pi^2 (1/Lx^2 + 1/Ly^2)."""
import math

import numpy as np
import pytest

import oracle
from oracle import heat as H
from paper_2602_19474_gb300 import synth


def rect_image():
    img = np.zeros((60, 80), np.uint8)
    img[10:50, 10:70] = 1  # a 60 x 40 px rectangle of label 1
    return img


@pytest.mark.parametrize("hn,hd", [(2, 1), (2, 3), (4, 1)])
def test_mass_is_the_label_area(hn, hd):
    for img in (rect_image(), synth.voronoi_labels(size=80, nseeds=8)):
        m = oracle.mesh_bitmap(img, hn, hd)
        for L in np.unique(img)[:3]:
            sel, _, _ = H.region(m["tri"], m["label"], L)
            M = H.lumped_mass(m["xy"], m["tri"][sel], len(m["xy"]))
            assert abs(M.sum() - (img == L).sum()) <= 1e-9 * (img == L).sum()


def test_stiffness_kernel():
    img = synth.voronoi_labels(size=80, nseeds=8)
    m = oracle.mesh_bitmap(img, 2, 1)
    xy = m["xy"]
    L = int(np.bincount(img.ravel()).argmax())
    sel, free, bnd = H.region(m["tri"], m["label"], L)
    K = H.stiffness(xy, m["tri"][sel], len(xy))
    assert abs(K - K.T).max() == 0.0
    assert np.abs(np.asarray(K.sum(axis=1))).max() <= 1e-12
    lin = 3.0 * xy[:, 0] - 2.0 * xy[:, 1] + 5.0
    assert np.abs((K @ lin)[free]).max() <= 1e-11
    # at boundary vertices the region's one-sided stencil does not vanish
    assert np.abs((K @ lin)[bnd]).max() > 1e-3


def test_equilateral_cotangents():
    m = oracle.mesh_bitmap(np.ones((20, 20), np.uint8), 2, 1)
    uncut = m["code"] == 0
    cot = H.cotangents(m["xy"], m["tri"][uncut])
    assert np.allclose(cot, 1.0 / math.sqrt(3.0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("hn,hd,tol", [(2, 1, 5e-3), (2, 3, 1e-3)])
def test_eigenmode_decay(hn, hd, tol):
    img = rect_image()
    m = oracle.mesh_bitmap(img, hn, hd)
    xy = m["xy"]
    Lx, Ly, xa, ya = 60.0, 40.0, 9.5, 9.5
    u0 = np.sin(math.pi * (xy[:, 0] - xa) / Lx) * np.sin(math.pi * (xy[:, 1] - ya) / Ly)
    alpha, dt, n = 500.0, 0.01, 20
    u, peaks = H.heat(xy, m["tri"], m["label"], 1, alpha, dt, n, 0.0, 0.0, 1.0, u0=u0)
    lam = math.pi ** 2 * (1.0 / Lx ** 2 + 1.0 / Ly ** 2)
    f = (1.0 / (1.0 + alpha * dt * lam)) ** n
    _, free, bnd = H.region(m["tri"], m["label"], 1)
    assert np.abs(u[free] - f * u0[free]).max() <= tol * f
    assert (u[bnd] == 0).all()
    assert all(b < a for a, b in zip(peaks, peaks[1:]))


def test_gaussian_pulse_peak():
    # a pulse much wider than the region's distance to the boundary is held
    # down by it; a narrow one far from the boundary keeps the free-space
    # decay of its peak, A sigma^2 / (sigma^2 + 2 alpha t), to within the
    # discretisation error
    img = np.zeros((200, 200), np.uint8)
    img[5:195, 5:195] = 1
    m = oracle.mesh_bitmap(img, 2, 1)
    sigma, alpha, dt, n = 12.0, 5.0, 0.1, 10
    u, peaks = H.heat(m["xy"], m["tri"], m["label"], 1, alpha, dt, n, 99.7, 100.3, sigma)
    t = n * dt
    free_space = 100.0 * sigma ** 2 / (sigma ** 2 + 2 * alpha * t)
    assert abs(peaks[-1] - free_space) <= 0.02 * free_space


def _wrong_corner_stiffness(xy, tri, nv):
    import scipy.sparse as sp

    tri = np.asarray(tri)
    cot = H.cotangents(xy, tri)
    rows, cols, vals = [], [], []
    for k in range(3):
        i, j = tri[:, (k + 1) % 3], tri[:, (k + 2) % 3]
        w = 0.5 * cot[:, (k + 1) % 3]  # planted: the angle at the wrong corner
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-w, -w, w, w]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nv, nv))


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """Each planted mistake makes a committed pin fail when that pin runs
    under it."""
    good_stiff, good_mass = H.stiffness, H.lumped_mass
    # the cotangent of the wrong corner: linear functions leave the kernel
    monkeypatch.setattr(H, "stiffness", _wrong_corner_stiffness)
    with pytest.raises(AssertionError):
        test_stiffness_kernel()
    # the stiffness with the wrong sign: the eigenmode grows instead of decaying
    monkeypatch.setattr(H, "stiffness", lambda a, b, c: -good_stiff(a, b, c))
    with pytest.raises(Exception):
        test_eigenmode_decay(2, 1, 5e-3)
    monkeypatch.setattr(H, "stiffness", good_stiff)
    # half instead of a third of each area: the label area is missed
    monkeypatch.setattr(H, "lumped_mass", lambda a, b, c: 1.5 * good_mass(a, b, c))
    with pytest.raises(AssertionError):
        test_mass_is_the_label_area(2, 1)


def test_energy_decreases():
    # backward Euler with a symmetric positive semi-definite K: the M-norm of
    # u cannot grow from one step to the next
    img = synth.voronoi_labels(size=96, nseeds=9)
    m = oracle.mesh_bitmap(img, 2, 3)
    L = int(np.bincount(img.ravel()).argmax())
    sel, free, _ = H.region(m["tri"], m["label"], L)
    M = H.lumped_mass(m["xy"], m["tri"][sel], len(m["xy"]))
    u = np.where(free, H.pulse(m["xy"], 40.0, 50.0, 15.0, 100.0), 0.0)
    e = [float(u @ (M * u))]
    for _ in range(4):
        u, _ = H.heat(m["xy"], m["tri"], m["label"], L, 20.0, 0.05, 1, 0.0, 0.0, 1.0, u0=u)
        e.append(float(u @ (M * u)))
    assert all(b < a for a, b in zip(e, e[1:])), e
