// sbmt_walk.cuh -- the closed-form walk of a boundary segment over the
// base grid (Sec. 3.3's lattice), shared by the extraction kernel (which
// counts each segment's cells) and the traversal kernels (which walk them).
#pragma once
#include "sbmt_dev.cuh"

namespace sbmt {

// Closed-form walk of one segment.  The walk runs from the segment's lower
// end along +x / +y; pair k is the k-th cell it visits and crossing k the
// k-th grid edge it crosses (between pair k and pair k + 1).  Both are O(1)
// for any k, so a segment can be walked in independent chunks.
struct SegWalk {
  i64 X, Y, X0, X1, Y0, Y1, U;  // scaled end coordinates; U = (Y - oy) / 3 for horizontal runs
  i64 j, j1, c0;                // strip (first strip) and first cell index
  int dir, s0;                  // vertical: the first strip's slanted crossing lies above the start
  u32 ncross;
};

SBMT_DEV i64 strip_ab(const GridP& g, i64 X, i64 j) { return ifloordiv(X - g.ox - 3 * g.p * j, 6 * g.p); }

// slanted crossing of x = X inside strip j: its height, grid edge and the
// cell above it (the cell below is up(ab, j) = 2 ab)
SBMT_DEV void strip_slant(const GridP& g, i64 X, i64 j, Zq* ys, i64* ei, i64* ej, int* fam, i64* upper) {
  const i64 p = g.p, ab = strip_ab(g, X, j), xab = g.ox + 3 * p * (2 * ab + j);
  if (X - xab < 3 * p) {  // left of the apex: the 60-degree edge from v(ab, j)
    *ys = zq(g.oy, 3 * p * j + (X - xab));
    *ei = ab, *ej = j, *fam = 1, *upper = 2 * ab - 1;
  } else {  // right of it: the 120-degree edge from v(ab + 1, j)
    *ys = zq(g.oy, 3 * p * j + (xab + 6 * p - X));
    *ei = ab + 1, *ej = j, *fam = 2, *upper = 2 * ab + 1;
  }
}

SBMT_DEV SegWalk seg_setup(const GridP& g, const Seg& s) {
  SegWalk w;
  const i64 q = g.q, P6 = 6 * g.p, L = seg_len(s);
  w.dir = seg_dir(s);
  if (w.dir == 0) {
    w.Y = 6 * q * s.cy - 3 * q;
    w.X0 = 6 * q * s.cx - 3 * q, w.X1 = w.X0 + 6 * q * L;
    w.j = strip_of(g, zq(w.Y));
    // at height Y the 60-degree lines sit at ox + 6p i + U sqrt3 and the
    // 120-degree lines at ox + 6p (k + j) - U sqrt3; the cell index is the
    // number of lines of both families left of x
    w.U = (w.Y - g.oy) / 3;
    w.c0 = zfloordiv(zq(w.X0 - g.ox, -w.U), P6) + zfloordiv(zq(w.X0 - g.ox - P6 * w.j, w.U), P6);
    const i64 c1 = zfloordiv(zq(w.X1 - g.ox, -w.U), P6) + zfloordiv(zq(w.X1 - g.ox - P6 * w.j, w.U), P6);
    w.ncross = (u32)(c1 - w.c0);
    return w;
  }
  w.X = 6 * q * s.cx - 3 * q;
  w.Y0 = 6 * q * s.cy - 3 * q, w.Y1 = w.Y0 + 6 * q * L;
  w.j = strip_of(g, zq(w.Y0)), w.j1 = strip_of(g, zq(w.Y1));
  Zq ys;
  i64 ei, ej, up;
  int fam;
  strip_slant(g, w.X, w.j, &ys, &ei, &ej, &fam, &up);
  w.s0 = zcmp(ys, zq(w.Y0)) > 0 ? 1 : 0;
  strip_slant(g, w.X, w.j1, &ys, &ei, &ej, &fam, &up);
  const int e1 = zcmp(ys, zq(w.Y1)) < 0 ? 1 : 0;
  // virtual sequence S_j0, H_j0+1, S_j0+1, ..., S_j1; the first and last
  // slanted crossings count only when they lie inside (Y0, Y1)
  w.ncross = (u32)(2 * (w.j1 - w.j) + 1 - (1 - w.s0) - (1 - e1));
  return w;
}

// cells a segment visits: its crossings plus one
SBMT_DEV u32 seg_pairs(const GridP& g, const Seg& s) { return seg_setup(g, s).ncross + 1u; }

}  // namespace sbmt
