// sbmt_cell.cuh -- per-cell helpers shared by the classification and
// emission kernels: cell geometry from its id, counter-clockwise order of
// events along a cell edge, pixel-corner ids, centroid labels, block scans.
#pragma once
#include "sbmt_dev.cuh"

namespace sbmt {

struct CellGeo {
  i64 c, j;
  i64 ci[3], cj[3];
  u32 edge[3];
  int down;
};
SBMT_DEV CellGeo cell_geo(const GridP& g, u32 cid, int r) {
  CellGeo cg;
  cg.j = g.j0 + r;
  cg.c = g.clo[r] + ((i64)cid - g.cbase[r]);
  cell_corners(cg.c, cg.j, cg.ci, cg.cj);
  cell_edges(g, cg.c, cg.j, cg.edge);
  cg.down = (int)(cg.c & 1);
  return cg;
}
// strip row of cell id cid: a proportional estimate, corrected
SBMT_DEV int cell_row_near(const GridP& g, u32 cid) {
  int r = (int)((float)cid * ((float)g.nrows / i2f(g.ncells)));
  r = max(0, min(g.nrows - 1, r));
  while (r > 0 && g.cbase[r] > (i64)cid) --r;
  while (r + 1 < g.nrows && g.cbase[r + 1] <= (i64)cid) ++r;
  return r;
}
// from strip row r, the strip row of a cell id at or after that row's first cell
SBMT_DEV int advance_row(const GridP& g, int r, u32 cid) {
  while (r + 1 < g.nrows && g.cbase[r + 1] <= (i64)cid) ++r;
  return r;
}
SBMT_DEV int local_edge(const CellGeo& cg, u32 e) {
  return cg.edge[0] == e ? 0 : cg.edge[1] == e ? 1 : cg.edge[2] == e ? 2 : -1;
}
// a number increasing counter-clockwise along local edge k (corner k -> k+1):
// up cells run AB +x, BC +y, CA -y; down cells AB +y, BC -x, CA -y
SBMT_DEV Zq ccw_pos_xy(int down, int k, Zq x, Zq y) {
  if (k == 2) return zq(-y.a, -y.b);
  if (down == 0) return k == 0 ? x : y;
  return k == 0 ? y : zq(-x.a, -x.b);
}
SBMT_DEV Zq ccw_pos(int down, int k, const Event& e) { return ccw_pos_xy(down, k, zq(e.xa, e.xb), zq(e.ya, e.yb)); }
SBMT_DEV u32 corner_id(const GridP& g, const Seg& s, int upper) {
  i64 cx = s.cx, cy = s.cy;
  if (upper) {
    if (seg_dir(s) == 0) cx += seg_len(s);
    else cy += seg_len(s);
  }
  return (u32)(cy * (g.W + 1) + cx);
}
SBMT_DEV Pq corner_of_id(const GridP& g, u32 id) {
  return corner_pt(g, (i64)(id % (u32)(g.W + 1)), (i64)(id / (u32)(g.W + 1)));
}

// label of the pixel holding the point (sx / 3, sy / 3), sx and sy the sums of
// a triangle's three global coordinates: its centroid.  Pixel k spans
// [k - 1/2, k + 1/2) in pixel units, so the column is floor(x/S + 1/2).
template <typename T>
SBMT_DEV unsigned short centroid_label_sum(const GridP& g, const unsigned char* img, i64 pitch, const Zq& sx,
                                           const Zq& sy) {
  const i64 col = zfloordiv(Zq{2 * sx.a + 3 * g.S, 2 * sx.b}, 6 * g.S);
  const i64 row = zfloordiv(Zq{2 * sy.a + 3 * g.S, 2 * sy.b}, 6 * g.S);
  const int l = pix<T>(img, pitch, g.W, g.H, col, row);
  return l == OUTSIDE ? (unsigned short)0xFFFF : (unsigned short)l;
}
SBMT_DEV unsigned short label_at_sum(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Zq& sx,
                                     const Zq& sy) {
  return dtype == 1 ? centroid_label_sum<unsigned char>(g, img, pitch, sx, sy)
                    : centroid_label_sum<unsigned short>(g, img, pitch, sx, sy);
}
SBMT_DEV unsigned short label_of(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pq& a,
                                 const Pq& b, const Pq& c) {
  return label_at_sum(g, img, pitch, dtype, a.x + b.x + c.x, a.y + b.y + c.y);
}

// exclusive scan of one value per thread over a block of 256 threads
SBMT_DEV u32 block_exscan256(u32 v, u32* total, u32* sh /* 8 words */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  u32 x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    u32 s = lane < 8 ? sh[lane] : 0u;
    for (int o = 1; o < 8; o <<= 1) {
      const u32 y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < 8) sh[lane] = s;
  }
  __syncthreads();
  const u32 before = (w ? sh[w - 1] : 0u) + x - v;
  *total = sh[7];
  __syncthreads();
  return before;
}

}  // namespace sbmt
