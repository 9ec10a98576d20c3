"""Transient heat diffusion on a region of the output mesh (App. H) -- the
oracle of mesh_heat (test infrastructure, used only by the tests and the
benchmark's checks).

App. H evolves du/dt = alpha Lap u on a region Omega of the mesh, u = 0 on
its boundary, from a centred Gaussian pulse u0 = A exp(-|x - x0|^2 / (2
sigma^2)), and reports the peak temperature over time.  The paper names no
discretisation; the readings here:

- Omega is the set of triangles carrying one label L.  Its boundary
  vertices -- vertices of an Omega triangle that also lie on a triangle of
  another label (or outside the image) -- are held at 0; the other vertices
  of Omega are free.  Vertices outside Omega have u = 0.
- Space: linear finite elements.  The stiffness matrix K is the cotangent
  Laplacian: a triangle with angle theta_k at vertex k adds -cot(theta_k) / 2
  to K_ij and K_ji for its edge ij and cot(theta_k) / 2 to K_ii and K_jj.
  The mass matrix is lumped: M_ii is a third of the area of the Omega
  triangles at i.
- Time: backward Euler with step dt, (M + alpha dt K) u_{n+1} = M u_n on the
  free vertices.

Plain numpy / scipy in double precision: the matrices assembled entry by
entry from their definition, each step solved directly.
"""
from __future__ import annotations

import numpy as np


def region(tri, label, L):
    """(in Omega mask per triangle, free-vertex mask, boundary-vertex mask)
    for the triangles of label L."""
    tri = np.asarray(tri)
    nv = int(tri.max()) + 1 if len(tri) else 0
    sel = np.asarray(label) == L
    inside = np.zeros(nv, bool)
    other = np.zeros(nv, bool)
    inside[tri[sel].ravel()] = True
    other[tri[~sel].ravel()] = True
    return sel, inside & ~other, inside & other


def cotangents(xy, tri):
    """cot of the angle at each corner of each triangle: (n, 3), column k at
    vertex tri[:, k]."""
    p = np.asarray(xy)[np.asarray(tri)]
    out = np.empty((len(p), 3))
    for k in range(3):
        a, b, c = p[:, k], p[:, (k + 1) % 3], p[:, (k + 2) % 3]
        u, v = b - a, c - a
        dot = u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1]
        cross = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
        out[:, k] = dot / cross
    return out


def areas(xy, tri):
    p = np.asarray(xy)[np.asarray(tri)]
    return 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))


def stiffness(xy, tri, nv):
    """The cotangent stiffness matrix (scipy CSR, nv x nv) of the triangles."""
    import scipy.sparse as sp

    tri = np.asarray(tri)
    cot = cotangents(xy, tri)
    rows, cols, vals = [], [], []
    for k in range(3):
        i, j = tri[:, (k + 1) % 3], tri[:, (k + 2) % 3]  # the edge opposite corner k
        w = 0.5 * cot[:, k]
        rows += [i, j, i, j]
        cols += [j, i, i, j]
        vals += [-w, -w, w, w]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nv, nv))


def lumped_mass(xy, tri, nv):
    m = np.zeros(nv)
    np.add.at(m, np.asarray(tri).ravel(), np.repeat(areas(xy, tri) / 3.0, 3))
    return m


def pulse(xy, x0, y0, sigma, amplitude):
    xy = np.asarray(xy)
    return amplitude * np.exp(-((xy[:, 0] - x0) ** 2 + (xy[:, 1] - y0) ** 2) / (2.0 * sigma * sigma))


def heat(xy, tri, label, L, alpha, dt, nsteps, x0, y0, sigma, amplitude=100.0, u0=None):
    """u after nsteps backward-Euler steps (one value per mesh vertex) and
    the peak of u after each step."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    xy = np.asarray(xy)
    nv = len(xy)
    sel, free, _ = region(tri, label, L)
    t = np.asarray(tri)[sel]
    K = stiffness(xy, t, nv)
    M = lumped_mass(xy, t, nv)
    idx = np.nonzero(free)[0]
    A = (K * (alpha * dt))[idx][:, idx] + sp.diags(M[idx])
    u = np.zeros(nv)
    u[idx] = (pulse(xy, x0, y0, sigma, amplitude) if u0 is None else np.asarray(u0))[idx]
    A = A.tocsc()
    peaks = []
    for _ in range(nsteps):
        u[idx] = spla.spsolve(A, M[idx] * u[idx])
        peaks.append(float(u.max()) if nv else 0.0)
    return u, peaks
