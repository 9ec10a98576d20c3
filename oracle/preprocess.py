"""Geometric preprocessing of the base mesh (Alg. 3, Steps 1-3) -- the oracle
of mesh_preprocess (test infrastructure, used only by the tests and the
benchmark's checks).

Alg. 3 takes the base mesh T0 (Sec. 3.3) and the boundary, and returns the
preprocessed mesh T that the template retriangulation (Alg. 2) then works
on.  Region I (Steps 1 and 2, which commute, Prop. "safe decoupling")
moves lattice vertices; Region II (Step 3) removes mesh edges that pass too
close to a boundary point and re-fans their two triangles around that point
(Fig. "b threshold split").  Plain numpy in double precision, each step as
its definition over all candidates.

Readings where the paper leaves a choice open:

- thresholds: a, b, c are given relative to the reference edge length
  sqrt(0.45) px of the experiments (Sec. 4, App. I), so in pixels they are
  a h / sqrt(0.45) etc.  They must satisfy the admissible range b < a/2,
  c < a/sqrt(2) (Eq. "admissible range") and a < h/2 (the remark on
  snapping collisions); otherwise the request is refused.
- boundary points are the PSLG vertices (pixel corners where boundary pixel
  edges meet other than straight through, the image corners included);
  boundary segments are the boundary pixel edges (the image border
  included), whose union is the PSLG's segments.
- Step 1: a lattice vertex v moves onto the boundary point nearest to it
  when that point is closer than a (squared distances compared); ties go to
  the smaller corner id y (W + 1) + x.
- Step 2: a vertex that did not snap and whose nearest boundary point q (the
  nearest point of any boundary pixel edge; ties to the smaller edge id) is
  closer than c moves along q -> v to distance c from q: for q inside a
  segment that is the segment's normal.
- Steps 1 and 2 both read the positions of T0.  A vertex of T0's outer
  boundary (an end of an edge with one cell beside it) snaps only onto an
  image corner or onto a point of the image border at least h + a from both
  ends of its side; Step 2 applies to it as to any vertex.  Otherwise the
  outer boundary could cut into the image: a neighbour O of v lies within h
  of v, and v within a of its target p, so only a target within h + a of an
  image corner lets an outer-boundary edge (p, O) cross the image's corner
  region (and a target off the border would pull the boundary inside).
- Step 3: a candidate is a boundary point p and an edge e of T (after
  Steps 1-2) closer to p than b, neither end of e lying at p.  It is applied
  when p is the smallest candidate point of e, e the smallest candidate
  edge of p (edge id = smaller vertex id * V + larger), and p the smallest
  candidate point over the edges of both triangles beside e: so no triangle
  loses two edges and no point is inserted twice; and when the re-fan keeps
  every half strictly counter-clockwise (p inside the quadrilateral: a point
  on the line of two of a cell's moved vertices, both snapped onto one
  pixel line, would leave a degenerate half).  An applied candidate
  inserts p as a vertex and splits each triangle (u, w, x) beside e = uw
  into (u, p, x) and (p, w, x).
- output: the lattice vertices (moved) in their ids, then the inserted
  points by corner id; the cells in id order, a split cell's two halves in
  that order; a triangle's label is that of the pixel holding its centroid
  (column floor(x + 1/2), OUTSIDE beyond the image); no pattern codes.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

OUTSIDE = 0xFFFF
REF_EDGE = math.sqrt(0.45)


class NotAdmissible(ValueError):
    pass


def thresholds_px(a: float, b: float, c: float, h: float):
    s = h / REF_EDGE
    A, B, C = a * s, b * s, c * s
    if not (B < A / 2 and C < A / math.sqrt(2) and A < h / 2 and A > 0 and B >= 0 and C >= 0):
        raise NotAdmissible("thresholds outside the admissible range")
    return A, B, C


def _padded(img):
    H, W = img.shape
    P = np.full((H + 2, W + 2), OUTSIDE, np.int64)
    P[1:-1, 1:-1] = img
    return P


def boundary_points(img):
    """PSLG vertices: (corner ids, positions) in corner-id order."""
    H, W = img.shape
    P = _padded(img)
    # corner (cx, cy): pixels a = (cx-1, cy-1), b = (cx, cy-1), c = (cx-1, cy), d = (cx, cy)
    a, b, c, d = P[:-1, :-1], P[:-1, 1:], P[1:, :-1], P[1:, 1:]
    E, Wm, N, S = b != d, a != c, c != d, a != b
    any_ = E | Wm | N | S
    straight = (E & Wm & ~N & ~S) | (N & S & ~E & ~Wm)
    vert = any_ & ~straight
    cy, cx = np.nonzero(vert)
    ids = cy * (W + 1) + cx
    order = np.argsort(ids)
    return ids[order], np.stack([cx[order] - 0.5, cy[order] - 0.5], axis=1).astype(np.float64)


def boundary_edges(img):
    """Boundary pixel edges: (edge ids, end points (n, 2, 2)) in id order;
    horizontal edge (m, k) between pixels (m, k-1) and (m, k) has id k W + m,
    vertical edge (m, k) between (m-1, k) and (m, k) has id
    (H + 1) W + k (W + 1) + m."""
    H, W = img.shape
    P = _padded(img)
    hk, hm = np.nonzero(P[:-1, 1:-1] != P[1:, 1:-1])  # k in 0..H, m in 0..W-1
    vk, vm = np.nonzero(P[1:-1, :-1] != P[1:-1, 1:])  # k in 0..H-1, m in 0..W
    hid = hk * W + hm
    vid = (H + 1) * W + vk * (W + 1) + vm
    hseg = np.stack([np.stack([hm - 0.5, hk - 0.5], 1), np.stack([hm + 0.5, hk - 0.5], 1)], 1)
    vseg = np.stack([np.stack([vm - 0.5, vk - 0.5], 1), np.stack([vm - 0.5, vk + 0.5], 1)], 1)
    ids = np.concatenate([hid, vid])
    segs = np.concatenate([hseg, vseg]).astype(np.float64)
    order = np.argsort(ids)
    return ids[order], segs[order]


def _nearest(vals, ids):
    """Index of the smallest value per row, ties to the smallest id."""
    m = vals.min(axis=1, keepdims=True)
    cand = np.where(vals == m, ids[None, :], np.iinfo(np.int64).max)
    return np.argmin(cand, axis=1)


def outer_vertices(cells, V):
    """The vertices on the outer boundary of the mesh: the ends of the edges
    that only one cell has."""
    e = np.concatenate([cells[:, [0, 1]], cells[:, [1, 2]], cells[:, [2, 0]]]).astype(np.int64)
    key = np.minimum(e[:, 0], e[:, 1]) * V + np.maximum(e[:, 0], e[:, 1])
    u, cnt = np.unique(key, return_counts=True)
    one = u[cnt == 1]
    out = np.zeros(V, bool)
    out[one // V] = True
    out[one % V] = True
    return out


def border_safe(pid, W, H, reach):
    """Per boundary point: an image corner, or a point of the image border
    at least `reach` from both ends of its side (corner id y (W+1) + x)."""
    cx, cy = pid % (W + 1), pid // (W + 1)
    onx, ony = (cx == 0) | (cx == W), (cy == 0) | (cy == H)
    corner = onx & ony
    dside = np.where(onx, np.minimum(cy, H - cy), np.minimum(cx, W - cx)).astype(np.float64)
    return corner | ((onx | ony) & (dside >= reach))


def region_one(xy0, img, A, C, fixed=None, reach=0.0, chunk=2048):
    """Steps 1 and 2 on the lattice positions xy0: new positions, status
    (0 kept, 1 snapped, 2 repelled) and the corner id snapped to (-1); a
    vertex marked in fixed snaps only onto a point border_safe(reach)."""
    pid, ppos = boundary_points(img)
    H, W = img.shape
    safe = border_safe(pid, W, H, reach)
    eid, eseg = boundary_edges(img)
    V = len(xy0)
    out = xy0.copy()
    status = np.zeros(V, np.int8)
    snap = np.full(V, -1, np.int64)
    for s in range(0, V, chunk):
        v = xy0[s:s + chunk]
        # Step 1
        if len(pid):
            dx = v[:, None, 0] - ppos[None, :, 0]
            dy = v[:, None, 1] - ppos[None, :, 1]
            d2 = dx * dx + dy * dy
            k = _nearest(d2, pid)
            best = d2[np.arange(len(v)), k]
            hit = best < A * A
            if fixed is not None:
                hit &= ~fixed[s:s + chunk] | safe[k]
            out[s:s + chunk][hit] = ppos[k[hit]]
            status[s:s + chunk][hit] = 1
            snap[s:s + chunk][hit] = pid[k[hit]]
        else:
            hit = np.zeros(len(v), bool)
        # Step 2 (vertices that did not snap)
        if len(eid):
            qx = np.clip(v[:, None, 0], eseg[None, :, 0, 0], eseg[None, :, 1, 0])
            qy = np.clip(v[:, None, 1], eseg[None, :, 0, 1], eseg[None, :, 1, 1])
            dx = v[:, None, 0] - qx
            dy = v[:, None, 1] - qy
            d2 = dx * dx + dy * dy
            k = _nearest(d2, eid)
            r = np.arange(len(v))
            best = d2[r, k]
            rep = (~hit) & (best < C * C)
            if rep.any():
                d = np.sqrt(best[rep])
                t = C / d
                out[s:s + chunk][rep, 0] = qx[r, k][rep] + t * dx[r, k][rep]
                out[s:s + chunk][rep, 1] = qy[r, k][rep] + t * dy[r, k][rep]
                status[s:s + chunk][rep] = 2
    return out, status, snap


def _seg_d2(p, u, w):
    """Squared distance from points p (n, 2) to segments u -> w (n, 2)."""
    ex, ey = w[:, 0] - u[:, 0], w[:, 1] - u[:, 1]
    px, py = p[:, 0] - u[:, 0], p[:, 1] - u[:, 1]
    den = ex * ex + ey * ey
    t = np.clip((px * ex + py * ey) / den, 0.0, 1.0)
    dx, dy = px - t * ex, py - t * ey
    return dx * dx + dy * dy


def preprocess(img, h_num, h_den, a, b, c, origin2x=0, origin2y=0):
    """Alg. 3 on a label image: the preprocessed mesh and the steps' records."""
    img = np.ascontiguousarray(img)
    H, W = img.shape
    h = h_num / h_den
    A, B, C = thresholds_px(a, b, c, h)
    xy0, cells = oracle.base_mesh(W, H, h_num, h_den, origin2x, origin2y)
    V = len(xy0)
    xy, status, snap = region_one(xy0, img, A, C, outer_vertices(cells, V), h + A)
    # Step 3: candidates over every (boundary point, edge of T)
    pid, ppos = boundary_points(img)
    e = np.concatenate([cells[:, [0, 1]], cells[:, [1, 2]], cells[:, [2, 0]]])
    ekey = np.minimum(e[:, 0], e[:, 1]).astype(np.int64) * V + np.maximum(e[:, 0], e[:, 1])
    ukey, inv = np.unique(ekey, return_inverse=True)
    eu, ew = ukey // V, ukey % V
    cand_p, cand_e = [], []
    for k in range(len(pid)):
        p = np.broadcast_to(ppos[k], (len(ukey), 2))
        d2 = _seg_d2(p, xy[eu], xy[ew])
        at = ((xy[eu] == ppos[k]).all(1)) | ((xy[ew] == ppos[k]).all(1))
        sel = np.nonzero((d2 < B * B) & ~at)[0]
        cand_p += [pid[k]] * len(sel)
        cand_e += list(sel)
    cand_p = np.array(cand_p, np.int64)
    cand_e = np.array(cand_e, np.int64)
    big = np.iinfo(np.int64).max
    emin = np.full(len(ukey), big, np.int64)
    np.minimum.at(emin, cand_e, cand_p)
    pmin = {}
    for pp, ee in zip(cand_p, cand_e):
        pmin[pp] = min(pmin.get(pp, big), ukey[ee])
    # the cells beside each edge
    ncell = len(cells)
    cell_of = np.tile(np.arange(ncell), 3)
    cmin = np.full(ncell, big, np.int64)
    edge_cells = {}
    for j, ee in enumerate(inv):
        edge_cells.setdefault(ee, []).append(cell_of[j])
    for pp, ee in zip(cand_p, cand_e):
        for cc in edge_cells[ee]:
            cmin[cc] = min(cmin[cc], pp)
    applied = []
    for pp, ee in zip(cand_p, cand_e):
        if emin[ee] == pp and pmin[pp] == ukey[ee] and all(cmin[cc] == pp for cc in edge_cells[ee]):
            applied.append((pp, ee))
    pos_of = dict(zip(pid.tolist(), map(tuple, ppos)))

    def orient(a_, b_, c_):
        return (b_[0] - a_[0]) * (c_[1] - a_[1]) - (b_[1] - a_[1]) * (c_[0] - a_[0])

    def refan_ok(pp, ee):
        # both halves (u, p, x) and (p, w, x) of every cell beside e stay
        # counter-clockwise: p inside the quadrilateral the re-fan covers
        q = pos_of[pp]
        for cc in edge_cells[ee]:
            t = [int(x_) for x_ in cells[cc]]
            for kk in range(3):
                u_, w_, x_ = t[kk], t[(kk + 1) % 3], t[(kk + 2) % 3]
                if {u_, w_} == {int(eu[ee]), int(ew[ee])}:
                    if not (orient(xy[u_], q, xy[x_]) > 0.0 and orient(q, xy[w_], xy[x_]) > 0.0):
                        return False
        return True

    applied = [(pp, ee) for pp, ee in applied if refan_ok(pp, ee)]
    applied.sort()
    new_id = {pp: V + r for r, (pp, _) in enumerate(applied)}
    split = {}  # cell -> (local edge k, new vertex id)
    for pp, ee in applied:
        for cc in edge_cells[ee]:
            t = cells[cc]
            for kk in range(3):
                if {int(t[kk]), int(t[(kk + 1) % 3])} == {int(eu[ee]), int(ew[ee])}:
                    split[cc] = (kk, new_id[pp])
    xy_all = np.concatenate([xy, np.array([pos_of[pp] for pp, _ in applied], np.float64).reshape(-1, 2)])
    tris = []
    for cc in range(ncell):
        t = [int(x) for x in cells[cc]]
        if cc in split:
            kk, q = split[cc]
            u, w, x = t[kk], t[(kk + 1) % 3], t[(kk + 2) % 3]
            tris += [(u, q, x), (q, w, x)]
        else:
            tris.append(tuple(t))
    tri = np.array(tris, np.int32).reshape(-1, 3)
    P = xy_all[tri]
    cx = ((P[:, 0, 0] + P[:, 1, 0]) + P[:, 2, 0]) / 3.0
    cy = ((P[:, 0, 1] + P[:, 1, 1]) + P[:, 2, 1]) / 3.0
    col = np.floor(cx + 0.5).astype(np.int64)
    row = np.floor(cy + 0.5).astype(np.int64)
    inside = (col >= 0) & (col < W) & (row >= 0) & (row < H)
    label = np.full(len(tri), OUTSIDE, np.uint16)
    label[inside] = img[row[inside], col[inside]]
    return dict(xy=xy_all, tri=tri, label=label, n_lattice_vertices=V, status=status, snap=snap,
                eliminations=np.array([(pp, int(eu[ee]), int(ew[ee])) for pp, ee in applied], np.int64).reshape(-1, 3),
                candidates=len(cand_p), thresholds_px=(A, B, C))
