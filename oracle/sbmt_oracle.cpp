/*
 * sbmt_oracle.cpp -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded CPU statement of what the Structured
 * Bitmap-to-Mesh Triangulation (SBMT) hot path computes: label bitmap ->
 * boundary PSLG -> equilateral base grid -> segment/edge events (Alg. 1) ->
 * frozen registry -> canonical key kappa(K) and single-valued lookup
 * (Sec. 3.3.3, Assumption "frozen registry", Alg. 2, App. G) -> conforming mesh.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * path; the two are written independently and compared output for output.
 *
 * Arithmetic is exact: every coordinate is an element a + b*sqrt(3) of
 * Z[sqrt(3)] scaled by S = 6*h_den (h = h_num/h_den), held in __int128, so no
 * geometric predicate has a tolerance (the paper's epsilon of Thm. "edge
 * conformity under finite precision" is taken as 0).
 *
 * Readings of the paper that this file takes:
 *  - pixels are unit squares centred at integer points (Sec. 3.3); outside the
 *    image the label is OUTSIDE, larger than every pixel label; every pixel
 *    edge between different labels is boundary, the image border included;
 *  - boundary segments are the maximal straight runs of boundary pixel edges
 *    between PSLG vertices (turns, junctions, pinches), each oriented with the
 *    lower label on its left (Sec. 3.1 "input boundary as prescribed prior");
 *  - the grid is v(i,j) = o + h*(i + j/2, (sqrt3/2) j) and the mesh holds every
 *    grid cell meeting the closed image rectangle (Sec. 3.3);
 *  - only the degeneracy-free parameter class is meshed: integer origin, h_num
 *    even, h_den odd.  Then no grid vertex lies on a pixel line, no grid edge
 *    is collinear with a pixel edge and no pixel corner lies on a grid edge, so
 *    every Alg. 1 event of the pipeline is a proper crossing.  Alg. 1 itself
 *    (all four branches) is implemented and exported for the paper's atoms;
 *  - Tier-T cells (inside the regime of Lemma 3.1) take the App. G templates;
 *    every other cut cell (Tier-G) takes the greedy triangulation of its local
 *    PSLG (shortest exact edge first, ties by local index), Steiner-free;
 *  - canonicalisation is over the three rotations (C3); mirror images are
 *    distinct keys (App. G "orientation handling"); the nested-chord pair is
 *    split by the direction of the chord nearest the cut corner;
 *  - a triangle's label is the label of the pixel holding its centroid.
 *
 * Region III of Alg. 3's schedule (oracle_region3, at the end of this file)
 * retriangulates an arbitrary counter-clockwise mesh, the preprocessed one,
 * cell by cell in double precision with the same two-tier rule; it handles
 * Alg. 1's degenerate incidences (vertex on the segment, overlap, endpoint
 * on the edge), which the moved vertices create.
 *
 * parity pinned: Alg. 1 by the single-segment atoms of Fig. "lookup_table";
 * intersection points by the printed coordinates of App. F; templates by the
 * printed triangle lists of App. G at the printed coordinates; the mesh by
 * closed forms and invariants (see tests/test_oracle_*.py).
 */
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <stdexcept>
#include <string>
#include <vector>

typedef __int128 i128;
typedef int64_t i64;

namespace {

/* ------------------------------------------------------------------------- */
/* exact numbers a + b*sqrt(3)                                                */
/* ------------------------------------------------------------------------- */
struct Z3 {
  i128 a, b;
};
Z3 z(i128 a, i128 b = 0) { return Z3{a, b}; }
Z3 operator+(Z3 x, Z3 y) { return Z3{x.a + y.a, x.b + y.b}; }
Z3 operator-(Z3 x, Z3 y) { return Z3{x.a - y.a, x.b - y.b}; }
Z3 operator*(Z3 x, Z3 y) { return Z3{x.a * y.a + 3 * x.b * y.b, x.a * y.b + x.b * y.a}; }
Z3 times(Z3 x, i128 k) { return Z3{x.a * k, x.b * k}; }

/* sign of a + b*sqrt(3); sqrt(3) is irrational so a^2 == 3 b^2 only at 0 */
int sgn(Z3 v) {
  int sa = (v.a > 0) - (v.a < 0), sb = (v.b > 0) - (v.b < 0);
  if (sa == 0) return sb;
  if (sb == 0 || sa == sb) return sa;
  i128 l = v.a * v.a, r = 3 * v.b * v.b;
  return l > r ? sa : sb;
}
int cmp(Z3 x, Z3 y) { return sgn(x - y); }
double to_double(Z3 v) { return (double)v.a + (double)v.b * 1.7320508075688772935; }

struct Pt {
  Z3 x, y;
};
int orient(const Pt& p, const Pt& q, const Pt& r) {
  return sgn((q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x));
}
Z3 dot(const Pt& o, const Pt& p, const Pt& q) {
  return (p.x - o.x) * (q.x - o.x) + (p.y - o.y) * (q.y - o.y);
}
/* w on the closed segment uv (u != v) */
bool on_closed_seg(const Pt& u, const Pt& v, const Pt& w) {
  return orient(u, v, w) == 0 && sgn(dot(u, v, w)) >= 0 && sgn(dot(v, u, w)) >= 0;
}
/* w strictly inside the open segment uv */
bool on_open_seg(const Pt& u, const Pt& v, const Pt& w) {
  return orient(u, v, w) == 0 && sgn(dot(u, v, w)) > 0 && sgn(dot(v, u, w)) > 0;
}

/* floor(n / d) for n in Z[sqrt3], integer d > 0, exact */
i64 floor_div(Z3 n, i64 d) {
  double approx = to_double(n) / (double)d;
  i64 k = (i64)std::floor(approx);
  while (sgn(n - z((i128)k * d)) < 0) --k;
  while (sgn(n - z((i128)(k + 1) * d)) >= 0) ++k;
  return k;
}

/* ------------------------------------------------------------------------- */
/* Alg. 1 (Sec. 3.3.1): classify segment L = PQ against triangle edge e = UV.  */
/* ------------------------------------------------------------------------- */
enum { EV_NONE = 0, EV_CROSS = 1, EV_VERTEX = 2, EV_OVERLAP = 3 };
struct Alg1 {
  int kind;
  bool u_on, v_on; /* which vertices of e lie on L (EV_VERTEX) */
};
/* The three branches in the paper's priority order:
 *  1. L crosses e at one point of e's relative interior ("interior or
 *     endpoint-on-edge")                                   -> one intersection;
 *  2. else a vertex of e lies on L                         -> two intersections,
 *     one for each edge incident to that vertex;
 *  3. else L overlaps e collinearly (positive length)      -> one intersection. */
Alg1 alg1(const Pt& U, const Pt& V, const Pt& P, const Pt& Q) {
  Alg1 r{EV_NONE, false, false};
  int o1 = orient(U, V, P), o2 = orient(U, V, Q);
  int o3 = orient(P, Q, U), o4 = orient(P, Q, V);
  bool colinear = (o1 == 0 && o2 == 0);
  if (!colinear) {
    bool meet = (o1 * o2 <= 0) && (o3 * o4 <= 0);
    if (meet && o3 != 0 && o4 != 0) {
      r.kind = EV_CROSS;
      return r;
    }
  }
  r.u_on = on_closed_seg(P, Q, U);
  r.v_on = on_closed_seg(P, Q, V);
  if (r.u_on || r.v_on) {
    r.kind = EV_VERTEX;
    return r;
  }
  if (colinear) {
    /* positive-length overlap with neither U nor V covered: L lies inside e */
    if (on_open_seg(U, V, P) || on_open_seg(U, V, Q)) r.kind = EV_OVERLAP;
  }
  return r;
}

/* intersection point of lines PQ and UV (not parallel), as a fraction
 * (nx, ny) / den with den a positive integer */
void line_meet(const Pt& P, const Pt& Q, const Pt& U, const Pt& V, Z3* nx, Z3* ny, i128* den) {
  /* P + s (Q - P), s = cross(U - P, V - U) / cross(Q - P, V - U) */
  Z3 dx = Q.x - P.x, dy = Q.y - P.y, ex = V.x - U.x, ey = V.y - U.y;
  Z3 num = (U.x - P.x) * ey - (U.y - P.y) * ex;
  Z3 dd = dx * ey - dy * ex;
  Z3 conj{dd.a, -dd.b};
  i128 d = (dd * conj).a; /* a^2 - 3 b^2, nonzero */
  Z3 s_num = num * conj;  /* s = s_num / d */
  if (d < 0) {
    d = -d;
    s_num = Z3{-s_num.a, -s_num.b};
  }
  *nx = times(P.x, d) + s_num * dx;
  *ny = times(P.y, d) + s_num * dy;
  *den = d;
}
Z3 exact_div(Z3 n, i128 d) {
  if (n.a % d != 0 || n.b % d != 0) throw std::runtime_error("inexact event point");
  return Z3{n.a / d, n.b / d};
}

/* ------------------------------------------------------------------------- */
/* input image and the boundary PSLG (Sec. 3.1, Sec. 3.2)                     */
/* ------------------------------------------------------------------------- */
const int32_t OUTSIDE = 0x10000; /* larger than any u8/u16 label */

struct Image {
  int W, H;
  i64 pitch;
  int dtype; /* 1 = u8, 2 = u16 */
  const uint8_t* data;
  int32_t at(i64 x, i64 y) const {
    if (x < 0 || y < 0 || x >= W || y >= H) return OUTSIDE;
    const uint8_t* row = data + y * pitch;
    if (dtype == 1) return row[x];
    uint16_t v;
    std::memcpy(&v, row + 2 * x, 2);
    return v;
  }
};

/* Pixel corner (cx, cy), 0 <= cx <= W, 0 <= cy <= H, sits at (cx-1/2, cy-1/2).
 * Its four incident unit pixel edges: E to (cx+1,cy), W to (cx-1,cy), N to
 * (cx,cy+1), S to (cx,cy-1); an edge is boundary when the two pixels it
 * separates have different labels. */
enum { CE_E = 1, CE_N = 2, CE_W = 4, CE_S = 8 };
int corner_mask(const Image& im, i64 cx, i64 cy) {
  int m = 0;
  if (im.at(cx, cy - 1) != im.at(cx, cy)) m |= CE_E;
  if (im.at(cx - 1, cy - 1) != im.at(cx - 1, cy)) m |= CE_W;
  if (im.at(cx - 1, cy) != im.at(cx, cy)) m |= CE_N;
  if (im.at(cx - 1, cy - 1) != im.at(cx, cy - 1)) m |= CE_S;
  return m;
}
/* A corner is a PSLG vertex unless it has no boundary edge or exactly two
 * collinear ones (a straight run passes through it). */
bool is_vertex(int m) { return m != 0 && m != (CE_E | CE_W) && m != (CE_N | CE_S); }

struct Segment {
  i64 cx, cy; /* start corner (lower coordinate end) */
  int dir;    /* 0: along +x, 1: along +y */
  i64 len;
  int32_t lab0, lab1; /* dir 0: below / above; dir 1: left / right */
  int rev;            /* 1 when the oriented direction (lower label on the left) is -x / -y */
};

std::vector<Segment> extract_segments(const Image& im) {
  std::vector<Segment> segs;
  const i64 W = im.W, H = im.H;
  std::vector<uint8_t> mask((size_t)(W + 1) * (H + 1));
  for (i64 cy = 0; cy <= H; ++cy)
    for (i64 cx = 0; cx <= W; ++cx) mask[cy * (W + 1) + cx] = (uint8_t)corner_mask(im, cx, cy);
  auto M = [&](i64 cx, i64 cy) { return (int)mask[cy * (W + 1) + cx]; };
  for (i64 cy = 0; cy <= H; ++cy)
    for (i64 cx = 0; cx <= W; ++cx) {
      int m = M(cx, cy);
      if (!is_vertex(m)) continue;
      if (m & CE_E) {
        i64 x = cx + 1;
        while (!is_vertex(M(x, cy))) ++x;
        Segment s{cx, cy, 0, x - cx, im.at(cx, cy - 1), im.at(cx, cy), 0};
        s.rev = (s.lab1 < s.lab0) ? 0 : 1; /* going +x the left side is above */
        segs.push_back(s);
      }
      if (m & CE_N) {
        i64 y = cy + 1;
        while (!is_vertex(M(cx, y))) ++y;
        Segment s{cx, cy, 1, y - cy, im.at(cx - 1, cy), im.at(cx, cy), 0};
        s.rev = (s.lab0 < s.lab1) ? 0 : 1; /* going +y the left side is -x */
        segs.push_back(s);
      }
    }
  return segs;
}

/* ------------------------------------------------------------------------- */
/* the equilateral base grid (Sec. 3.3)                                       */
/* ------------------------------------------------------------------------- */
struct Grid {
  i64 p, q, S, ox, oy; /* h = p/q; scaled origin */
  i64 W, H;
  i64 xl, xr, yl, yr; /* closed image rectangle, scaled */
  i64 j0, j1;         /* strip rows meeting it */
  std::vector<i64> clo, chi, cbase;
  i64 vj0, vj1;
  std::vector<i64> vlo, vhi, vbase;
  i64 ncells = 0, nverts = 0;

  Pt vtx(i64 i, i64 j) const { return Pt{z(ox + 3 * p * (2 * i + j)), z(oy, 3 * p * j)}; }
  Z3 ystrip(i64 j) const { return z(oy, 3 * p * j); }
  Pt pixcorner(i64 cx, i64 cy) const { return Pt{z(6 * q * cx - 3 * q), z(6 * q * cy - 3 * q)}; }

  /* lattice coordinates of the corners A, B, C of cell c = 2i+d in strip j */
  void corners(i64 c, i64 j, i64 ci[3], i64 cj[3]) const {
    i64 i = (c >= 0) ? c / 2 : -((-c + 1) / 2);
    int d = (int)(c - 2 * i);
    if (d == 0) { /* up: v(i,j), v(i+1,j), v(i,j+1) */
      ci[0] = i, cj[0] = j, ci[1] = i + 1, cj[1] = j, ci[2] = i, cj[2] = j + 1;
    } else { /* down: v(i+1,j), v(i+1,j+1), v(i,j+1) */
      ci[0] = i + 1, cj[0] = j, ci[1] = i + 1, cj[1] = j + 1, ci[2] = i, cj[2] = j + 1;
    }
  }
  std::array<Pt, 3> cell_pts(i64 c, i64 j) const {
    i64 ci[3], cj[3];
    corners(c, j, ci, cj);
    return {vtx(ci[0], cj[0]), vtx(ci[1], cj[1]), vtx(ci[2], cj[2])};
  }

  /* separating-axis test: closed triangle meets the closed rectangle */
  bool meets_rect(const std::array<Pt, 3>& t) const {
    Z3 mnx = t[0].x, mxx = t[0].x, mny = t[0].y, mxy = t[0].y;
    for (int k = 1; k < 3; ++k) {
      if (cmp(t[k].x, mnx) < 0) mnx = t[k].x;
      if (cmp(t[k].x, mxx) > 0) mxx = t[k].x;
      if (cmp(t[k].y, mny) < 0) mny = t[k].y;
      if (cmp(t[k].y, mxy) > 0) mxy = t[k].y;
    }
    if (cmp(mxx, z(xl)) < 0 || cmp(mnx, z(xr)) > 0) return false;
    if (cmp(mxy, z(yl)) < 0 || cmp(mny, z(yr)) > 0) return false;
    Pt rc[4] = {{z(xl), z(yl)}, {z(xr), z(yl)}, {z(xr), z(yr)}, {z(xl), z(yr)}};
    for (int k = 0; k < 3; ++k) {
      const Pt &a = t[k], &b = t[(k + 1) % 3];
      bool all_out = true; /* triangle is CCW: its interior is left of ab */
      for (auto& r : rc)
        if (orient(a, b, r) >= 0) all_out = false;
      if (all_out) return false;
    }
    return true;
  }

  bool has_cell(i64 c, i64 j) const {
    if (j < j0 || j > j1) return false;
    return c >= clo[j - j0] && c <= chi[j - j0];
  }
  i64 cell_id(i64 c, i64 j) const { return cbase[j - j0] + (c - clo[j - j0]); }
  i64 vid(i64 i, i64 j) const {
    if (j < vj0 || j > vj1 || i < vlo[j - vj0] || i > vhi[j - vj0]) throw std::runtime_error("vertex not in mesh");
    return vbase[j - vj0] + (i - vlo[j - vj0]);
  }
  /* grid-edge id: 3 * (id of the lower-id endpoint) + family, family 0 = +x,
   * 1 = 60 degrees, 2 = 120 degrees seen from that endpoint */
  i64 edge_id(i64 i1, i64 j1_, i64 i2, i64 j2) const {
    i64 a = vid(i1, j1_), b = vid(i2, j2);
    if (b < a) std::swap(i1, i2), std::swap(j1_, j2), std::swap(a, b);
    i64 di = i2 - i1, dj = j2 - j1_;
    int fam = (dj == 0 && di == 1) ? 0 : (dj == 1 && di == 0) ? 1 : (dj == 1 && di == -1) ? 2 : -1;
    if (fam < 0) throw std::runtime_error("not a grid edge");
    return 3 * a + fam;
  }
  /* strip row containing a point whose y is never on a grid line */
  i64 strip_of(Z3 y) const {
    double approx = (to_double(y) - (double)oy) / (3.0 * (double)p * 1.7320508075688772935);
    i64 j = (i64)std::floor(approx);
    while (cmp(ystrip(j), y) > 0) --j;
    while (cmp(ystrip(j + 1), y) <= 0) ++j;
    return j;
  }
  /* cell-index range in strip j whose cells could meet x in [xa, xb] */
  void cand_range(i64 j, double xa, double xb, i64* ca, i64* cb) const {
    double ia = ((xa - (double)ox) / (3.0 * (double)p) - (double)j) / 2.0;
    double ib = ((xb - (double)ox) / (3.0 * (double)p) - (double)j) / 2.0;
    *ca = 2 * ((i64)std::floor(ia) - 2);
    *cb = 2 * ((i64)std::ceil(ib) + 2) + 1;
  }
};

bool build_grid(Grid& g, i64 W, i64 H, i64 p, i64 q, i64 o2x, i64 o2y) {
  g.p = p, g.q = q, g.S = 6 * q, g.ox = 3 * q * o2x, g.oy = 3 * q * o2y, g.W = W, g.H = H;
  g.xl = -3 * q, g.xr = 6 * q * W - 3 * q, g.yl = -3 * q, g.yr = 6 * q * H - 3 * q;
  /* strip rows j with y_j <= yr and y_{j+1} >= yl */
  g.j0 = g.strip_of(z(g.yl));
  g.j1 = g.strip_of(z(g.yr));
  i64 nrows = g.j1 - g.j0 + 1;
  g.clo.assign(nrows, 0), g.chi.assign(nrows, -1), g.cbase.assign(nrows, 0);
  std::map<i64, std::pair<i64, i64>> vr; /* vertex row -> [lo, hi] */
  i64 base = 0;
  for (i64 j = g.j0; j <= g.j1; ++j) {
    i64 ca, cb;
    g.cand_range(j, (double)g.xl - 6.0 * p, (double)g.xr + 6.0 * p, &ca, &cb);
    i64 lo = 0, hi = -1;
    bool any = false;
    for (i64 c = ca; c <= cb; ++c) {
      if (g.meets_rect(g.cell_pts(c, j))) {
        if (!any) lo = c;
        if (any && c != hi + 1) throw std::runtime_error("cell row not contiguous");
        hi = c, any = true;
      }
    }
    if (!any) throw std::runtime_error("empty cell row");
    if (lo == ca || hi == cb) throw std::runtime_error("cell candidate range too small");
    g.clo[j - g.j0] = lo, g.chi[j - g.j0] = hi, g.cbase[j - g.j0] = base;
    base += hi - lo + 1;
    for (i64 c = lo; c <= hi; ++c) {
      i64 ci[3], cj[3];
      g.corners(c, j, ci, cj);
      for (int k = 0; k < 3; ++k) {
        auto it = vr.find(cj[k]);
        if (it == vr.end()) vr[cj[k]] = {ci[k], ci[k]};
        else it->second.first = std::min(it->second.first, ci[k]), it->second.second = std::max(it->second.second, ci[k]);
      }
    }
  }
  g.ncells = base;
  g.vj0 = vr.begin()->first, g.vj1 = vr.rbegin()->first;
  i64 nv = g.vj1 - g.vj0 + 1;
  g.vlo.assign(nv, 0), g.vhi.assign(nv, -1), g.vbase.assign(nv, 0);
  base = 0;
  for (i64 j = g.vj0; j <= g.vj1; ++j) {
    auto& r = vr.at(j);
    g.vlo[j - g.vj0] = r.first, g.vhi[j - g.vj0] = r.second, g.vbase[j - g.vj0] = base;
    base += r.second - r.first + 1;
  }
  g.nverts = base;
  /* every vertex in a row range must be a corner of some cell (no isolated vertex) */
  std::vector<std::vector<uint8_t>> used(nv);
  for (i64 j = g.vj0; j <= g.vj1; ++j) used[j - g.vj0].assign(g.vhi[j - g.vj0] - g.vlo[j - g.vj0] + 1, 0);
  for (i64 j = g.j0; j <= g.j1; ++j)
    for (i64 c = g.clo[j - g.j0]; c <= g.chi[j - g.j0]; ++c) {
      i64 ci[3], cj[3];
      g.corners(c, j, ci, cj);
      for (int k = 0; k < 3; ++k) used[cj[k] - g.vj0][ci[k] - g.vlo[cj[k] - g.vj0]] = 1;
    }
  for (auto& row : used)
    for (auto u : row)
      if (!u) throw std::runtime_error("vertex row not contiguous");
  return true;
}

/* ------------------------------------------------------------------------- */
/* finite lookup table (App. G) in the canonical frame                        */
/* ------------------------------------------------------------------------- */
/* Template labels: canonical corners A', B', C'; E0..E3 are the events read
 * counter-clockwise from A' (edge A'B', then B'C', then C'A'); P is the chain
 * vertex inside the cell. */
enum { LA = 0, LB = 1, LC = 2, E0 = 3, E1 = 4, E2 = 5, E3 = 6, LP = 7 };
typedef std::array<int, 3> Tri;

/* Canonical code of a Tier-T cell under rotation r:
 *   star<<10 | n(r)<<7 | n(r+1)<<4 | n(r+2)<<1 | dir
 * n(k) = number of events on actual edge k (0 AB, 1 BC, 2 CA); star = one chain
 * vertex inside; dir = direction bit of the nearer of two nested chords.  The
 * canonical rotation sigma minimises the code (ties: smallest sigma). */
int tcode(int star, int n0, int n1, int n2, int dir) { return (star << 10) | (n0 << 7) | (n1 << 4) | (n2 << 1) | dir; }

struct TplEntry {
  int key;
  std::vector<Tri> tri;
};
const std::map<int, TplEntry>& lut() {
  static std::map<int, TplEntry> m;
  if (!m.empty()) return m;
  /* single segment, case (b): chord with Q1 on BC and Q2 on CA cuts corner C */
  m[tcode(0, 0, 1, 1, 0)] = {1, {{E1, E0, LC}, {E1, LA, LB}, {E0, E1, LB}}};
  /* (1,1) case (a): P inside, Q1 on CA, Q2 on BC (E0 = Q2, E1 = Q1) */
  m[tcode(1, 0, 1, 1, 0)] = {2, {{E1, LP, LC}, {LP, E0, LC}, {E1, LA, LP}, {LA, LB, LP}, {E0, LP, LB}}};
  /* (1,1) case (c): P inside, Q1 and Q2 on CA, Q1 nearer C (E0 = Q1, E1 = Q2) */
  m[tcode(1, 0, 0, 2, 0)] = {3, {{E0, LP, LC}, {LP, E0, E1}, {E1, LA, LP}, {LB, LC, LP}, {LA, LB, LP}}};
  /* (2,2) case (b1): Q1 on AB, Q3 on BC, Q4 and Q2 on CA (E0=Q1, E1=Q3, E2=Q4, E3=Q2) */
  m[tcode(0, 1, 1, 2, 0)] = {4, {{E0, E3, LA}, {E0, E2, E3}, {E0, E1, E2}, {E0, LB, E1}, {E2, E1, LC}}};
  /* (2,2) case (d3): nested chords at C, nearer chord runs BC -> CA
   * (App. G attribution: Q1, Q2 on CA with Q1 nearer C; Q3, Q4 on BC with Q3
   * nearer C; E0 = Q4, E1 = Q3, E2 = Q1, E3 = Q2) */
  m[tcode(0, 0, 2, 2, 1)] = {5, {{LA, LB, E3}, {E3, LB, E0}, {E2, E3, E0}, {E2, E0, E1}, {E2, E1, LC}}};
  /* (2,2) case (a4): the mirror image, drawn at corner A, rotated here so the
   * cut corner is C' (paper A -> C', B -> A', C -> B'); E0 = Q2, E1 = Q1,
   * E2 = Q3, E3 = Q4 */
  m[tcode(0, 0, 2, 2, 0)] = {6, {{E2, E1, LC}, {E3, E1, E2}, {E1, E3, E0}, {E0, E3, LA}, {E0, LA, LB}}};
  /* keys the paper does not list: one chain vertex P of degree 3 or 4 inside
   * the cell, every segment incident to P -> star from P over the boundary
   * cycle read counter-clockwise from A' */
  const int star_counts[9][3] = {{0, 0, 3}, {0, 1, 2}, {0, 2, 1}, {1, 1, 1}, {0, 0, 4},
                                 {0, 1, 3}, {0, 2, 2}, {0, 3, 1}, {1, 1, 2}};
  for (int s = 0; s < 9; ++s) {
    const int* n = star_counts[s];
    std::vector<int> cyc;
    int e = E0;
    for (int k = 0; k < 3; ++k) {
      cyc.push_back(k); /* corner A', B', C' */
      for (int t = 0; t < n[k]; ++t) cyc.push_back(e++);
    }
    std::vector<Tri> tri;
    for (size_t t = 0; t < cyc.size(); ++t) tri.push_back({cyc[t], cyc[(t + 1) % cyc.size()], LP});
    m[tcode(1, n[0], n[1], n[2], 0)] = {7 + s, tri};
  }
  return m;
}

/* (m,n) class index in Thm. 3.2's list, 1-based; 0 = not applicable */
int class_index(int m, int n) {
  if (m > n) std::swap(m, n);
  const int lst[8][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 1}, {1, 2}, {2, 2}, {1, 3}, {2, 3}};
  for (int k = 0; k < 8; ++k)
    if (lst[k][0] == m && lst[k][1] == n) return k + 1;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* per-cell key and Tier-T patch (Sec. 3.3.2, Sec. 3.3.3, Alg. 2)             */
/* ------------------------------------------------------------------------- */
/* Local numbering of a cell: 0,1,2 = corners A,B,C; then the events in CCW
 * order from A (those on AB, then BC, then CA); then the chain vertices
 * strictly inside (by pixel-corner id).  A chain edge is the piece of one
 * boundary segment inside the cell, stored oriented along the segment. */
struct LocalResult {
  int tierG = 0, key = 0, sigma = 0, klass = 0, mask = 0;
  std::vector<Tri> tri; /* Tier-T only, local indices */
};

LocalResult classify_local(const int nev[3], int nchain, const std::vector<std::pair<int, int>>& ce) {
  LocalResult r;
  const int ne = nev[0] + nev[1] + nev[2];
  auto edge_of = [&](int v) -> int {
    if (v < 3) return -1;
    int k = v - 3;
    for (int e = 0; e < 3; ++e) {
      if (k < nev[e]) return e;
      k -= nev[e];
    }
    return -2; /* chain vertex */
  };
  /* Alg. 1 bitmask (AB=2, BC=4, CA=8) per segment; bit 0 marks a chain vertex
   * strictly inside the cell (the paper leaves bit value 1 unused) */
  r.mask = nchain > 0 ? 1 : 0;
  std::vector<int> counts;
  for (auto& e : ce) {
    int mb = 0;
    for (int w : {e.first, e.second}) {
      int k = edge_of(w);
      if (k >= 0) mb |= 2 << k;
    }
    r.mask |= mb;
    counts.push_back(__builtin_popcount(mb));
  }
  if (ce.size() == 1) r.klass = class_index(0, counts[0]);
  else if (ce.size() == 2) r.klass = class_index(counts[0], counts[1]);

  /* regime of Lemma 3.1: no chain vertex and one or two chords, or a single
   * chain vertex P with every segment in the cell incident to P */
  int star = 0, dir = 0;
  bool tierT = false;
  if (nchain == 0) {
    for (auto& e : ce)
      if (edge_of(e.first) < 0 || edge_of(e.second) < 0) throw std::runtime_error("chord end not an event");
    tierT = (ce.size() == 1 || ce.size() == 2);
    if (ce.size() == 2) {
      /* corner cut off by a chord: the corner shared by the chord's two edges */
      auto cut = [&](const std::pair<int, int>& e) {
        int a = edge_of(e.first), b = edge_of(e.second);
        if (a == b) throw std::runtime_error("chord with both ends on one edge");
        return (b == (a + 1) % 3) ? b : a; /* edges k and k+1 share corner k+1 */
      };
      int x0 = cut(ce[0]), x1 = cut(ce[1]);
      if (x0 == x1) { /* nested chords at corner X */
        int X = x0, ein = (X + 2) % 3, eout = X;
        /* on the edge ending at X the event nearer X comes later in CCW order */
        int near = -1, best = -1;
        for (int c = 0; c < 2; ++c)
          for (int w : {ce[c].first, ce[c].second})
            if (edge_of(w) == ein && w > best) best = w, near = c;
        dir = (edge_of(ce[near].first) == ein && edge_of(ce[near].second) == eout) ? 1 : 0;
      }
    }
  } else if (nchain == 1) {
    const int P = 3 + ne;
    tierT = !ce.empty();
    for (auto& e : ce)
      if (e.first != P && e.second != P) tierT = false;
    star = 1;
  }
  if (!tierT) {
    r.tierG = 1;
    r.key = 63;
    return r;
  }
  int best = -1, sigma = 0;
  for (int rr = 0; rr < 3; ++rr) {
    int code = tcode(star, nev[rr], nev[(rr + 1) % 3], nev[(rr + 2) % 3], dir);
    if (best < 0 || code < best) best = code, sigma = rr;
  }
  auto it = lut().find(best);
  if (it == lut().end()) throw std::runtime_error("Tier-T key missing from the table");
  r.key = it->second.key;
  r.sigma = sigma;
  /* instantiate: pi maps canonical labels to local vertices, pre-composed with sigma */
  int map[8];
  for (int k = 0; k < 3; ++k) map[k] = (sigma + k) % 3;
  std::vector<int> evs; /* events CCW from corner sigma */
  for (int k = 0; k < 3; ++k) {
    int e = (sigma + k) % 3, first = 3;
    for (int t = 0; t < e; ++t) first += nev[t];
    for (int t = 0; t < nev[e]; ++t) evs.push_back(first + t);
  }
  for (int k = 0; k < 4; ++k) map[E0 + k] = k < (int)evs.size() ? evs[k] : -1;
  map[LP] = nchain == 1 ? 3 + ne : -1;
  for (auto& t : it->second.tri) {
    Tri o{map[t[0]], map[t[1]], map[t[2]]};
    if (o[0] < 0 || o[1] < 0 || o[2] < 0) throw std::runtime_error("template label unmapped");
    r.tri.push_back(o);
  }
  return r;
}

/* ------------------------------------------------------------------------- */
/* Tier-G: greedy triangulation of the cell's local PSLG                      */
/* ------------------------------------------------------------------------- */
/* All local vertices lie in the convex cell.  Start from the constraint edges
 * (boundary sub-edges of the cell and chain edges), then take every other
 * vertex pair in order of exact squared length (ties: smaller local index
 * pair) and keep it when its open segment holds no vertex and crosses no kept
 * edge.  A maximal plane straight-line graph on a point set triangulates its
 * convex hull, so the result triangulates the cell, embeds every chain edge
 * and adds no Steiner point. */
std::vector<Tri> greedy_triangulate(const std::vector<Pt>& v, const std::vector<std::pair<int, int>>& constraints) {
  const int n = (int)v.size();
  std::vector<std::vector<uint8_t>> adj(n, std::vector<uint8_t>(n, 0));
  std::vector<std::pair<int, int>> edges;
  for (auto& e : constraints) {
    int a = std::min(e.first, e.second), b = std::max(e.first, e.second);
    if (!adj[a][b]) adj[a][b] = adj[b][a] = 1, edges.push_back({a, b});
  }
  struct Cand {
    Z3 len2;
    int u, w;
  };
  std::vector<Cand> cand;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (!adj[a][b]) {
        Z3 dx = v[b].x - v[a].x, dy = v[b].y - v[a].y;
        cand.push_back({dx * dx + dy * dy, a, b});
      }
  std::sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) {
    int c = cmp(x.len2, y.len2);
    if (c != 0) return c < 0;
    if (x.u != y.u) return x.u < y.u;
    return x.w < y.w;
  });
  for (auto& c : cand) {
    bool ok = true;
    for (int k = 0; k < n && ok; ++k)
      if (k != c.u && k != c.w && on_open_seg(v[c.u], v[c.w], v[k])) ok = false;
    for (size_t t = 0; t < edges.size() && ok; ++t) {
      int a = edges[t].first, b = edges[t].second;
      if (a == c.u || a == c.w || b == c.u || b == c.w) continue;
      int o1 = orient(v[c.u], v[c.w], v[a]), o2 = orient(v[c.u], v[c.w], v[b]);
      int o3 = orient(v[a], v[b], v[c.u]), o4 = orient(v[a], v[b], v[c.w]);
      if (o1 * o2 < 0 && o3 * o4 < 0) ok = false;
    }
    if (ok) adj[c.u][c.w] = adj[c.w][c.u] = 1, edges.push_back({c.u, c.w});
  }
  /* faces: 3-cycles holding no vertex in their interior, rotated so the
   * smallest local index leads, counter-clockwise, listed in sorted order */
  std::vector<Tri> tri;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      if (!adj[a][b]) continue;
      for (int c = b + 1; c < n; ++c) {
        if (!adj[a][c] || !adj[b][c]) continue;
        int o = orient(v[a], v[b], v[c]);
        if (o == 0) continue;
        bool empty = true;
        for (int k = 0; k < n && empty; ++k) {
          if (k == a || k == b || k == c) continue;
          int s1 = orient(v[a], v[b], v[k]), s2 = orient(v[b], v[c], v[k]), s3 = orient(v[c], v[a], v[k]);
          if (s1 == o && s2 == o && s3 == o) empty = false;
        }
        if (empty) tri.push_back(o > 0 ? Tri{a, b, c} : Tri{a, c, b});
      }
    }
  std::sort(tri.begin(), tri.end());
  return tri;
}

/* ------------------------------------------------------------------------- */
/* the whole mesh                                                             */
/* ------------------------------------------------------------------------- */
struct Event {
  i64 edge;
  i64 seg;
  Pt pt;
  Z3 t; /* position along the edge from its lower endpoint */
};

struct Mesh {
  std::vector<double> xy;
  std::vector<int32_t> tri;
  std::vector<uint16_t> label, code;
  std::vector<Segment> segs;
  std::vector<Event> events; /* registry order */
  i64 nverts_grid = 0, ncells = 0;
  std::vector<i64> cut_cell, cut_code, cut_ntri, cut_nchain, cut_tierG;
  i64 n_tierG = 0;
};

/* label of the pixel holding the centroid of (a, b, c); OUTSIDE off-image */
int32_t centroid_label(const Grid& g, const Image& im, const Pt& a, const Pt& b, const Pt& c) {
  /* pixel column = floor(x/S + 1/2) with x = (xa+xb+xc)/3 */
  Z3 sx = a.x + b.x + c.x, sy = a.y + b.y + c.y;
  i64 col = floor_div(times(sx, 2) + z(3 * g.S), 6 * g.S);
  i64 row = floor_div(times(sy, 2) + z(3 * g.S), 6 * g.S);
  return im.at(col, row);
}

uint16_t out_label(int32_t l) { return l == OUTSIDE ? (uint16_t)0xFFFF : (uint16_t)l; }

uint16_t make_code(const LocalResult& r) {
  return (uint16_t)((r.mask & 15) | ((r.sigma & 3) << 4) | ((r.key & 63) << 6) | ((r.klass & 15) << 12));
}

void mesh_image(const Image& im, i64 p, i64 q, i64 o2x, i64 o2y, Mesh& M) {
  Grid g;
  build_grid(g, im.W, im.H, p, q, o2x, o2y);
  M.segs = extract_segments(im);

  /* events and cell incidences: Alg. 1 for every segment against the edges of
   * the cells near it */
  std::map<std::pair<i64, i64>, Event> ev; /* (edge id, segment) */
  std::map<i64, std::set<i64>> cell_segs;  /* cell id -> segments meeting it */
  std::map<i64, std::vector<std::pair<i64, i64>>> cell_chain; /* cell id -> (corner id, segment) */
  const i64 S = g.S;
  for (size_t s = 0; s < M.segs.size(); ++s) {
    const Segment& sg = M.segs[s];
    Pt P = g.pixcorner(sg.cx, sg.cy);
    Pt Q = sg.dir == 0 ? g.pixcorner(sg.cx + sg.len, sg.cy) : g.pixcorner(sg.cx, sg.cy + sg.len);
    i64 ja = g.strip_of(P.y), jb = g.strip_of(Q.y);
    for (i64 j = ja; j <= jb; ++j) {
      i64 ca, cb;
      g.cand_range(j, to_double(P.x) - 6.0 * p, to_double(Q.x) + 6.0 * p, &ca, &cb);
      for (i64 c = ca; c <= cb; ++c) {
        if (!g.has_cell(c, j)) continue;
        i64 ci[3], cj[3];
        g.corners(c, j, ci, cj);
        auto T = g.cell_pts(c, j);
        i64 cid = g.cell_id(c, j);
        for (int k = 0; k < 3; ++k) {
          int k2 = (k + 1) % 3;
          Alg1 a = alg1(T[k], T[k2], P, Q);
          if (a.kind == EV_NONE) continue;
          if (a.kind != EV_CROSS) throw std::runtime_error("degenerate event in the degeneracy-free class");
          i64 eid = g.edge_id(ci[k], cj[k], ci[k2], cj[k2]);
          cell_segs[cid].insert((i64)s);
          if (ev.count({eid, (i64)s})) continue;
          Z3 nx, ny;
          i128 den;
          line_meet(P, Q, T[k], T[k2], &nx, &ny, &den);
          Pt X{exact_div(nx, den), exact_div(ny, den)};
          /* lower endpoint of the edge: horizontal edges run +x, the others +y */
          Z3 t = (cj[k] == cj[k2]) ? X.x : X.y;
          ev[{eid, (i64)s}] = Event{eid, (i64)s, X, t};
        }
        for (int end = 0; end < 2; ++end) {
          const Pt& E = end == 0 ? P : Q;
          int o0 = orient(T[0], T[1], E), o1 = orient(T[1], T[2], E), o2 = orient(T[2], T[0], E);
          if (o0 > 0 && o1 > 0 && o2 > 0) {
            i64 ecx = sg.cx + (end == 1 && sg.dir == 0 ? sg.len : 0);
            i64 ecy = sg.cy + (end == 1 && sg.dir == 1 ? sg.len : 0);
            cell_segs[cid].insert((i64)s);
            cell_chain[cid].push_back({ecy * (g.W + 1) + ecx, (i64)s});
          } else if (o0 * o1 * o2 == 0 && o0 >= 0 && o1 >= 0 && o2 >= 0) {
            throw std::runtime_error("segment end on a grid edge in the degeneracy-free class");
          }
        }
      }
    }
  }

  /* frozen registry: events ordered by edge id, then position along the edge */
  std::vector<Event> evs;
  for (auto& kv : ev) evs.push_back(kv.second);
  std::sort(evs.begin(), evs.end(), [](const Event& a, const Event& b) {
    if (a.edge != b.edge) return a.edge < b.edge;
    return cmp(a.t, b.t) < 0;
  });
  std::map<std::pair<i64, i64>, i64> ev_gid; /* (edge, seg) -> vertex id */
  std::map<i64, std::vector<i64>> edge_events; /* edge -> registry indices */
  const i64 NVg = g.nverts;
  for (size_t k = 0; k < evs.size(); ++k) {
    ev_gid[{evs[k].edge, evs[k].seg}] = NVg + (i64)k;
    edge_events[evs[k].edge].push_back((i64)k);
  }
  const i64 NE = (i64)evs.size();

  /* chain vertices: by cell id, then pixel-corner id */
  std::map<i64, std::vector<i64>> cell_corners; /* cell -> sorted unique corner ids */
  i64 NC = 0;
  for (auto& kv : cell_chain) {
    std::vector<i64> cs;
    for (auto& pr : kv.second) cs.push_back(pr.first);
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    cell_corners[kv.first] = cs;
    NC += (i64)cs.size();
  }
  std::map<i64, i64> chain_base;
  {
    i64 b = NVg + NE;
    for (auto& kv : cell_corners) chain_base[kv.first] = b, b += (i64)kv.second.size();
  }

  /* coordinates */
  const i64 NV = NVg + NE + NC;
  M.xy.assign(2 * NV, 0.0);
  auto put_xy = [&](i64 id, const Pt& pt) {
    M.xy[2 * id] = to_double(pt.x) / (double)S;
    M.xy[2 * id + 1] = to_double(pt.y) / (double)S;
  };
  for (i64 j = g.vj0; j <= g.vj1; ++j)
    for (i64 i = g.vlo[j - g.vj0]; i <= g.vhi[j - g.vj0]; ++i) put_xy(g.vid(i, j), g.vtx(i, j));
  for (size_t k = 0; k < evs.size(); ++k) put_xy(NVg + (i64)k, evs[k].pt);
  for (auto& kv : cell_corners)
    for (size_t t = 0; t < kv.second.size(); ++t) {
      i64 cid = kv.second[t];
      put_xy(chain_base[kv.first] + (i64)t, g.pixcorner(cid % (g.W + 1), cid / (g.W + 1)));
    }

  /* cells in id order: untouched cells keep their base triangle, cut cells
   * are replaced by the patch of their key (Alg. 2) */
  M.nverts_grid = NVg;
  M.ncells = g.ncells;
  M.tri.reserve(3 * (size_t)g.ncells + 64);
  for (i64 j = g.j0; j <= g.j1; ++j) {
    for (i64 c = g.clo[j - g.j0]; c <= g.chi[j - g.j0]; ++c) {
      i64 cid = g.cell_id(c, j);
      i64 ci[3], cj[3];
      g.corners(c, j, ci, cj);
      auto T = g.cell_pts(c, j);
      i64 gid[3] = {g.vid(ci[0], cj[0]), g.vid(ci[1], cj[1]), g.vid(ci[2], cj[2])};
      auto cs = cell_segs.find(cid);
      if (cs == cell_segs.end()) {
        M.tri.insert(M.tri.end(), {(int32_t)gid[0], (int32_t)gid[1], (int32_t)gid[2]});
        M.label.push_back(out_label(centroid_label(g, im, T[0], T[1], T[2])));
        M.code.push_back(0);
        continue;
      }
      /* local PSLG of the cut cell */
      std::vector<Pt> lv(T.begin(), T.end());
      std::vector<i64> lg(gid, gid + 3);
      int nev[3];
      std::map<i64, int> seg_event_local[3];
      for (int k = 0; k < 3; ++k) {
        int k2 = (k + 1) % 3;
        i64 eid = g.edge_id(ci[k], cj[k], ci[k2], cj[k2]);
        std::vector<i64> idx;
        auto it = edge_events.find(eid);
        if (it != edge_events.end()) idx = it->second;
        /* registry order runs from the lower-id endpoint; the cell reads CCW
         * from corner k to corner k+1 */
        if (gid[k] > gid[k2]) std::reverse(idx.begin(), idx.end());
        nev[k] = (int)idx.size();
        for (i64 r : idx) {
          seg_event_local[k][evs[r].seg] = (int)lv.size();
          lv.push_back(evs[r].pt);
          lg.push_back(NVg + r);
        }
      }
      std::map<i64, int> corner_local;
      auto cc = cell_corners.find(cid);
      int nchain = 0;
      if (cc != cell_corners.end()) {
        nchain = (int)cc->second.size();
        for (size_t t = 0; t < cc->second.size(); ++t) {
          i64 corner = cc->second[t];
          corner_local[corner] = (int)lv.size();
          lv.push_back(g.pixcorner(corner % (g.W + 1), corner / (g.W + 1)));
          lg.push_back(chain_base[cid] + (i64)t);
        }
      }
      std::vector<std::pair<int, int>> ce;
      for (i64 s : cs->second) {
        const Segment& sg = M.segs[s];
        std::vector<int> ends;
        for (int k = 0; k < 3; ++k) {
          auto f = seg_event_local[k].find(s);
          if (f != seg_event_local[k].end()) ends.push_back(f->second);
        }
        i64 c0 = sg.cy * (g.W + 1) + sg.cx;
        i64 c1 = sg.dir == 0 ? c0 + sg.len : c0 + sg.len * (g.W + 1);
        for (i64 corner : {c0, c1}) {
          auto f = corner_local.find(corner);
          if (f != corner_local.end()) ends.push_back(f->second);
        }
        if (ends.size() != 2) throw std::runtime_error("segment piece without two ends");
        /* orient along the segment: forward is +x / +y unless rev */
        const Pt &a = lv[ends[0]], &b = lv[ends[1]];
        int ord = sg.dir == 0 ? cmp(a.x, b.x) : cmp(a.y, b.y);
        bool a_first = sg.rev ? (ord > 0) : (ord < 0);
        ce.push_back(a_first ? std::make_pair(ends[0], ends[1]) : std::make_pair(ends[1], ends[0]));
      }
      LocalResult lr = classify_local(nev, nchain, ce);
      std::vector<Tri> tris;
      if (lr.tierG) {
        std::vector<std::pair<int, int>> cons = ce;
        /* boundary sub-edges: consecutive vertices of the CCW cycle of the cell */
        std::vector<int> cyc;
        int e = 3;
        for (int k = 0; k < 3; ++k) {
          cyc.push_back(k);
          for (int t = 0; t < nev[k]; ++t) cyc.push_back(e++);
        }
        for (size_t t = 0; t < cyc.size(); ++t) cons.push_back({cyc[t], cyc[(t + 1) % cyc.size()]});
        tris = greedy_triangulate(lv, cons);
        M.n_tierG++;
      } else {
        tris = lr.tri;
      }
      int nb = 3 + nev[0] + nev[1] + nev[2];
      if ((int)tris.size() != 2 * nchain + nb - 2) throw std::runtime_error("patch triangle count");
      uint16_t code = make_code(lr);
      for (auto& t : tris) {
        if (orient(lv[t[0]], lv[t[1]], lv[t[2]]) <= 0) throw std::runtime_error("patch triangle not CCW");
        M.tri.insert(M.tri.end(), {(int32_t)lg[t[0]], (int32_t)lg[t[1]], (int32_t)lg[t[2]]});
        M.label.push_back(out_label(centroid_label(g, im, lv[t[0]], lv[t[1]], lv[t[2]])));
        M.code.push_back(code);
      }
      M.cut_cell.push_back(cid);
      M.cut_code.push_back(code);
      M.cut_ntri.push_back((i64)tris.size());
      M.cut_nchain.push_back(nchain);
      M.cut_tierG.push_back(lr.tierG);
    }
  }
  M.events = evs;
}

/* ------------------------------------------------------------------------- */
char g_err[512];
template <class T>
T* dup(const std::vector<T>& v) {
  T* p = (T*)std::malloc(sizeof(T) * (v.size() ? v.size() : 1));
  if (!v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

}  // namespace

/* ------------------------------------------------------------------------- */
/* C interface (ctypes)                                                       */
/* ------------------------------------------------------------------------- */
extern "C" {

typedef struct {
  int64_t n_vertices, n_triangles, n_cells, n_cut_cells, n_tierG_cells, n_vertices_grid;
  double* xy;
  int32_t* tri;
  uint16_t* label;
  uint16_t* code;
  int64_t n_segments;
  int32_t* seg; /* 7 per segment: cx, cy, dir, len, lab0, lab1, rev */
  int64_t n_events;
  int64_t* ev; /* 3 per event in registry order: edge id, segment index, vertex id */
  int64_t* cut; /* 5 per cut cell in id order: cell id, code, ntri, nchain, tierG */
} oracle_mesh;

const char* oracle_last_error(void) { return g_err; }

/* 0 on success, -1 bad arguments (incl. parameters outside the
 * degeneracy-free class), -2 internal consistency failure */
int oracle_mesh_bitmap(const void* data, int32_t width, int32_t height, int64_t pitch_bytes, int32_t dtype,
                       int32_t h_num, int32_t h_den, int32_t origin2x, int32_t origin2y, oracle_mesh* out) {
  g_err[0] = 0;
  if (!data || !out || width < 1 || height < 1 || width > 32768 || height > 32768 || (dtype != 1 && dtype != 2) ||
      pitch_bytes < (int64_t)width * dtype || h_num < 1 || h_den < 1 || h_num > 4096 || h_den > 64 ||
      (h_num % 2) != 0 || (h_den % 2) != 1 || (origin2x % 2) != 0 || (origin2y % 2) != 0) {
    std::snprintf(g_err, sizeof g_err, "invalid arguments");
    return -1;
  }
  try {
    Image im{width, height, pitch_bytes, dtype, (const uint8_t*)data};
    Mesh M;
    mesh_image(im, h_num, h_den, origin2x, origin2y, M);
    std::memset(out, 0, sizeof *out);
    out->n_vertices = (int64_t)M.xy.size() / 2;
    out->n_triangles = (int64_t)M.label.size();
    out->n_cells = M.ncells;
    out->n_cut_cells = (int64_t)M.cut_cell.size();
    out->n_tierG_cells = M.n_tierG;
    out->n_vertices_grid = M.nverts_grid;
    out->xy = dup(M.xy);
    out->tri = dup(M.tri);
    out->label = dup(M.label);
    out->code = dup(M.code);
    out->n_segments = (int64_t)M.segs.size();
    std::vector<int32_t> sg;
    for (auto& s : M.segs)
      sg.insert(sg.end(), {(int32_t)s.cx, (int32_t)s.cy, s.dir, (int32_t)s.len, s.lab0, s.lab1, s.rev});
    out->seg = dup(sg);
    out->n_events = (int64_t)M.events.size();
    std::vector<int64_t> e;
    for (size_t k = 0; k < M.events.size(); ++k)
      e.insert(e.end(), {M.events[k].edge, M.events[k].seg, M.nverts_grid + (int64_t)k});
    out->ev = dup(e);
    std::vector<int64_t> cu;
    for (size_t k = 0; k < M.cut_cell.size(); ++k)
      cu.insert(cu.end(), {M.cut_cell[k], M.cut_code[k], M.cut_ntri[k], M.cut_nchain[k], M.cut_tierG[k]});
    out->cut = dup(cu);
    return 0;
  } catch (const std::exception& ex) {
    std::snprintf(g_err, sizeof g_err, "%s", ex.what());
    return -2;
  }
}

void oracle_mesh_free(oracle_mesh* m) {
  if (!m) return;
  std::free(m->xy), std::free(m->tri), std::free(m->label), std::free(m->code);
  std::free(m->seg), std::free(m->ev), std::free(m->cut);
  std::memset(m, 0, sizeof *m);
}

/* Alg. 1 on one triangle ABC (CCW) and one segment PQ given by integer
 * coordinates (x + xs*sqrt3, y + ys*sqrt3), 4 numbers per point.  Writes the
 * event kind for edges AB, BC, CA (0 none, 1 crossing, 2 vertex on L,
 * 3 overlap) and returns the bitmask AB=2, BC=4, CA=8 (a vertex on L sets both
 * incident edges, an overlap its own edge). */
int oracle_alg1(const int64_t* tri12, const int64_t* seg8, int32_t* kinds3) {
  Pt T[3], P[2];
  for (int k = 0; k < 3; ++k) T[k] = Pt{z(tri12[4 * k], tri12[4 * k + 1]), z(tri12[4 * k + 2], tri12[4 * k + 3])};
  for (int k = 0; k < 2; ++k) P[k] = Pt{z(seg8[4 * k], seg8[4 * k + 1]), z(seg8[4 * k + 2], seg8[4 * k + 3])};
  int mask = 0;
  for (int k = 0; k < 3; ++k) {
    int k2 = (k + 1) % 3;
    Alg1 a = alg1(T[k], T[k2], P[0], P[1]);
    kinds3[k] = a.kind;
    if (a.kind == EV_CROSS || a.kind == EV_OVERLAP) mask |= 2 << k;
    /* vertex k is shared by edges k-1 and k; vertex k2 by edges k and k2 */
    if (a.kind == EV_VERTEX) {
      if (a.u_on) mask |= (2 << k) | (2 << ((k + 2) % 3));
      if (a.v_on) mask |= (2 << k) | (2 << k2);
    }
  }
  return mask;
}

/* crossing point of segment PQ with segment UV (coordinates as in
 * oracle_alg1), as doubles in the same units; returns 0 if lines are parallel */
int oracle_line_meet(const int64_t* pq8, const int64_t* uv8, double* xy2) {
  Pt a{z(pq8[0], pq8[1]), z(pq8[2], pq8[3])}, b{z(pq8[4], pq8[5]), z(pq8[6], pq8[7])};
  Pt u{z(uv8[0], uv8[1]), z(uv8[2], uv8[3])}, v{z(uv8[4], uv8[5]), z(uv8[6], uv8[7])};
  Z3 dd = (b.x - a.x) * (v.y - u.y) - (b.y - a.y) * (v.x - u.x);
  if (sgn(dd) == 0) return 0;
  Z3 nx, ny;
  i128 den;
  line_meet(a, b, u, v, &nx, &ny, &den);
  xy2[0] = to_double(nx) / (double)den;
  xy2[1] = to_double(ny) / (double)den;
  return 1;
}

/* Key and Tier-T patch of one cell from its combinatorial description:
 * nev[3] events on AB, BC, CA (local indices 3.. in CCW order from A), nchain
 * chain vertices after them, n_ce chain edges as oriented local index pairs.
 * Writes key, sigma, class, mask, tierG into info5 and up to cap triangles
 * (local indices) into tri; returns the triangle count (0 for Tier-G),
 * -1 on a malformed description. */
int oracle_local_patch(const int32_t* nev3, int32_t nchain, const int32_t* ce, int32_t n_ce, int32_t* info5,
                       int32_t* tri, int32_t cap) {
  try {
    int nev[3] = {nev3[0], nev3[1], nev3[2]};
    std::vector<std::pair<int, int>> e;
    for (int k = 0; k < n_ce; ++k) e.push_back({ce[2 * k], ce[2 * k + 1]});
    LocalResult r = classify_local(nev, nchain, e);
    info5[0] = r.key, info5[1] = r.sigma, info5[2] = r.klass, info5[3] = r.mask, info5[4] = r.tierG;
    if ((int)r.tri.size() > cap) return -1;
    for (size_t t = 0; t < r.tri.size(); ++t)
      for (int k = 0; k < 3; ++k) tri[3 * t + k] = r.tri[t][k];
    return (int)r.tri.size();
  } catch (const std::exception& ex) {
    std::snprintf(g_err, sizeof g_err, "%s", ex.what());
    return -1;
  }
}

/* The lookup table: for key id k (1..15) writes its canonical code and its
 * template (labels 0..2 = A',B',C', 3..6 = E0..E3, 7 = P); returns the number
 * of triangles, 0 if the key does not exist. */
int oracle_template(int32_t key, int32_t* code, int32_t* tri, int32_t cap) {
  for (auto& kv : lut())
    if (kv.second.key == key) {
      *code = kv.first;
      int n = (int)kv.second.tri.size();
      if (n > cap) return -1;
      for (int t = 0; t < n; ++t)
        for (int k = 0; k < 3; ++k) tri[3 * t + k] = kv.second.tri[t][k];
      return n;
    }
  return 0;
}

/* Greedy Tier-G triangulation of explicit points (integer coordinates as in
 * oracle_alg1) with constraint edges; returns the triangle count or -1. */
int oracle_greedy(const int64_t* pts4, int32_t n, const int32_t* cons, int32_t ncons, int32_t* tri, int32_t cap) {
  std::vector<Pt> v;
  for (int k = 0; k < n; ++k) v.push_back(Pt{z(pts4[4 * k], pts4[4 * k + 1]), z(pts4[4 * k + 2], pts4[4 * k + 3])});
  std::vector<std::pair<int, int>> c;
  for (int k = 0; k < ncons; ++k) c.push_back({cons[2 * k], cons[2 * k + 1]});
  auto t = greedy_triangulate(v, c);
  if ((int)t.size() > cap) return -1;
  for (size_t q = 0; q < t.size(); ++q)
    for (int k = 0; k < 3; ++k) tri[3 * q + k] = t[q][k];
  return (int)t.size();
}

/* The base mesh T0 of Sec. 3.3 (the lattice cells meeting the closed image
 * rectangle, no boundary embedded), the input of the preprocessing of
 * Alg. 3: lattice vertex coordinates (2 doubles each, vertex-id order) and
 * the cells' corners A, B, C (3 vertex ids each, cell-id order).  Any
 * integer origin2x, origin2y: an odd one puts the origin on a pixel line
 * (the degenerate origins).  Free the two arrays with oracle_free. */
int oracle_base_mesh(int32_t width, int32_t height, int32_t h_num, int32_t h_den, int32_t origin2x, int32_t origin2y,
                     int64_t* nverts, int64_t* ncells, double** xy, int32_t** tri) {
  g_err[0] = 0;
  if (!nverts || !ncells || !xy || !tri || width < 1 || height < 1 || h_num < 1 || h_den < 1 || (h_num % 2) != 0 ||
      (h_den % 2) != 1) {
    std::snprintf(g_err, sizeof g_err, "invalid arguments");
    return -1;
  }
  try {
    Grid g;
    build_grid(g, width, height, h_num, h_den, origin2x, origin2y);
    std::vector<double> v;
    for (i64 j = g.vj0; j <= g.vj1; ++j)
      for (i64 i = g.vlo[j - g.vj0]; i <= g.vhi[j - g.vj0]; ++i) {
        const Pt q = g.vtx(i, j);
        v.push_back(to_double(q.x) / (double)g.S), v.push_back(to_double(q.y) / (double)g.S);
      }
    std::vector<int32_t> t;
    for (i64 j = g.j0; j <= g.j1; ++j)
      for (i64 c = g.clo[j - g.j0]; c <= g.chi[j - g.j0]; ++c) {
        i64 ci[3], cj[3];
        g.corners(c, j, ci, cj);
        for (int k = 0; k < 3; ++k) t.push_back((int32_t)g.vid(ci[k], cj[k]));
      }
    *nverts = g.nverts, *ncells = g.ncells;
    *xy = dup(v), *tri = dup(t);
    return 0;
  } catch (const std::exception& ex) {
    std::snprintf(g_err, sizeof g_err, "%s", ex.what());
    return -2;
  }
}

void oracle_free(void* p) { free(p); }

/* ------------------------------------------------------------------------
 * Mesh invariants of any correct output (test infrastructure): every
 * triangle counter-clockwise, every vertex used, each undirected edge in at
 * most two triangles and each directed edge in at most one (closure and
 * consistent orientation), Euler characteristic V - E + T = 1 (a disk),
 * total area = n_cells * sqrt(3)/4 h^2 (every base cell tiled), the area of
 * each pixel label = its pixel count and the outside area = the rest, and
 * boundary conformity: every edge between triangles of different labels
 * lies on a pixel line, and those edges add up to the bitmap's boundary
 * length.  Returns 0, or the number of the failed check (message in
 * g_err).
 * ------------------------------------------------------------------------ */
static int check_invariants(const uint8_t* img, int W, int H, double h, const Mesh& M) {
  const i64 V = (i64)M.xy.size() / 2, T = (i64)M.label.size();
  auto X = [&](i64 v) { return M.xy[2 * v]; };
  auto Y = [&](i64 v) { return M.xy[2 * v + 1]; };
  std::vector<char> used(V, 0);
  double total = 0.0;
  double lab_area[2] = {0.0, 0.0}, out_area = 0.0;
  for (i64 t = 0; t < T; ++t) {
    const int32_t a = M.tri[3 * t], b = M.tri[3 * t + 1], c = M.tri[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) return std::snprintf(g_err, sizeof g_err, "vertex id"), 1;
    used[a] = used[b] = used[c] = 1;
    const double ar = 0.5 * ((X(b) - X(a)) * (Y(c) - Y(a)) - (Y(b) - Y(a)) * (X(c) - X(a)));
    if (!(ar > 0)) return std::snprintf(g_err, sizeof g_err, "triangle %lld not counter-clockwise", (long long)t), 2;
    total += ar;
    const uint16_t l = M.label[t];
    if (l == 0xFFFF) out_area += ar;
    else if (l < 2) lab_area[l] += ar;
    else return std::snprintf(g_err, sizeof g_err, "label %d", (int)l), 3;
  }
  for (i64 v = 0; v < V; ++v)
    if (!used[v]) return std::snprintf(g_err, sizeof g_err, "unused vertex %lld", (long long)v), 4;
  // edges: (min, max, triangle, directed) sorted
  std::vector<std::array<i64, 4>> e;
  e.reserve(3 * T);
  for (i64 t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const i64 u = M.tri[3 * t + k], w = M.tri[3 * t + (k + 1) % 3];
      e.push_back({std::min(u, w), std::max(u, w), t, u < w ? 1 : 0});
    }
  std::sort(e.begin(), e.end());
  i64 E = 0;
  double blen = 0.0;
  for (size_t k = 0; k < e.size();) {
    size_t m = k + 1;
    while (m < e.size() && e[m][0] == e[k][0] && e[m][1] == e[k][1]) ++m;
    if (m - k > 2) return std::snprintf(g_err, sizeof g_err, "edge in three triangles"), 5;
    if (m - k == 1 && M.label[e[k][2]] != 0xFFFF) {
      // an outer edge of the mesh with an image label inside: it must lie
      // on the image border (a lattice row on the border line)
      const i64 u = e[k][0], w = e[k][1];
      const bool onh = Y(u) == Y(w) && (Y(u) == -0.5 || Y(u) == H - 0.5);
      const bool onv = X(u) == X(w) && (X(u) == -0.5 || X(u) == W - 0.5);
      if (!onh && !onv) return std::snprintf(g_err, sizeof g_err, "an image label on the mesh's outer boundary"), 13;
      blen += std::fabs(X(u) - X(w)) + std::fabs(Y(u) - Y(w));
    }
    if (m - k == 2) {
      if (e[k][3] == e[k + 1][3]) return std::snprintf(g_err, sizeof g_err, "directed edge repeated"), 6;
      if (M.label[e[k][2]] != M.label[e[k + 1][2]]) {
        const i64 u = e[k][0], w = e[k][1];
        const bool onh = std::fabs(Y(u) - Y(w)) < 1e-9 && std::fabs(Y(u) - std::round(Y(u) - 0.5) - 0.5) < 1e-9;
        const bool onv = std::fabs(X(u) - X(w)) < 1e-9 && std::fabs(X(u) - std::round(X(u) - 0.5) - 0.5) < 1e-9;
        if (!onh && !onv) return std::snprintf(g_err, sizeof g_err, "label change off the pixel lines"), 7;
        blen += std::fabs(X(u) - X(w)) + std::fabs(Y(u) - Y(w));
      }
    }
    ++E;
    k = m;
  }
  if (V - E + T != 1) return std::snprintf(g_err, sizeof g_err, "Euler characteristic %lld", (long long)(V - E + T)), 8;
  const double want = (double)M.ncells * std::sqrt(3.0) / 4.0 * h * h;
  if (std::fabs(total - want) > 1e-9 * want + 1e-9) return std::snprintf(g_err, sizeof g_err, "total area"), 9;
  int cnt[2] = {0, 0}, bl = 0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int l = img[y * W + x];
      cnt[l]++;
      bl += (x == 0) + (y == 0) + (x == W - 1) + (y == H - 1);
      if (x + 1 < W && img[y * W + x + 1] != l) ++bl;
      if (y + 1 < H && img[(y + 1) * W + x] != l) ++bl;
    }
  for (int l = 0; l < 2; ++l)
    if (std::fabs(lab_area[l] - cnt[l]) > 1e-9 * W * H + 1e-7)
      return std::snprintf(g_err, sizeof g_err, "area of label %d", l), 10;
  if (std::fabs(out_area - (want - W * H)) > 1e-9 * want + 1e-7)
    return std::snprintf(g_err, sizeof g_err, "outside area"), 11;
  if (std::fabs(blen - bl) > 1e-6 * std::max(1, bl))
    return std::snprintf(g_err, sizeof g_err, "boundary length %g of %d", blen, bl), 12;
  return 0;
}

/* The invariants above for a given mesh of a binary bitmap (W x H bytes,
 * row-major): 0, or the number of the failed check (message in
 * oracle_last_error). */
int oracle_check_mesh(const uint8_t* img, int32_t W, int32_t H, int32_t h_num, int32_t h_den, int64_t ncells,
                      int64_t V, const double* xy, int64_t T, const int32_t* tri, const uint16_t* label) {
  g_err[0] = 0;
  Mesh M;
  M.xy.assign(xy, xy + 2 * V);
  M.tri.assign(tri, tri + 3 * T);
  M.label.assign(label, label + T);
  M.ncells = ncells;
  return check_invariants(img, W, H, (double)h_num / h_den, M);
}

/* Every binary bitmap of W x H <= 25 pixels (bit k of the bitmap's number =
 * pixel k in row-major order) from `first`, every `stride`-th, meshed at
 * h = h_num / h_den and checked against the invariants; returns the number
 * checked, or -(1 + the first failing bitmap's number) with the message in
 * oracle_last_error. */
int64_t oracle_brute(int32_t W, int32_t H, int32_t h_num, int32_t h_den, int64_t first, int64_t stride) {
  if (W < 1 || H < 1 || W * H > 25 || stride < 1 || first < 0) return -1;
  std::vector<uint8_t> img(W * H);
  const int64_t n = (int64_t)1 << (W * H);
  int64_t done = 0;
  for (int64_t b = first; b < n; b += stride) {
    for (int k = 0; k < W * H; ++k) img[k] = (uint8_t)((b >> k) & 1);
    try {
      Image im{W, H, (int64_t)W, 1, img.data()};
      Mesh M;
      mesh_image(im, h_num, h_den, 0, 0, M);
      if (check_invariants(img.data(), W, H, (double)h_num / h_den, M)) {
        const std::string what = g_err;
        std::snprintf(g_err, sizeof g_err, "bitmap %lld: %.400s", (long long)b, what.c_str());
        return -(1 + b);
      }
    } catch (const std::exception& ex) {
      std::snprintf(g_err, sizeof g_err, "bitmap %lld: %s", (long long)b, ex.what());
      return -(1 + b);
    }
    ++done;
  }
  return done;
}

}  // extern "C"

/* ========================================================================= */
/* Region III of the pipelined schedule (Alg. 3 with the corollary on        */
/* pipelined parallel scheduling): Alg. 2, the template retriangulation, on  */
/* an arbitrary counter-clockwise triangle mesh T (the preprocessed mesh),   */
/* each cell on its own from its local intersection class.                   */
/*                                                                           */
/* T's vertices are doubles (Steps 1-2 move them off the lattice), so every  */
/* quantity here is a double computed by one fixed formula, each operation   */
/* rounded once (the library is built without floating-point contraction).   */
/* Degenerate incidences are exact: a pixel line is k - 1/2, and a vertex   */
/* snapped to a pixel corner sits on it exactly.                             */
/*                                                                           */
/* Readings:                                                                 */
/*  - an event of a mesh edge e is a point of the open edge where the        */
/*    boundary meets it: a crossing of a boundary pixel edge, or a pixel     */
/*    corner on e with a boundary pixel edge not collinear with e (a run of  */
/*    boundary along e itself is embedded by e: Alg. 1's overlap); an end    */
/*    of e on the boundary (a vertex on the segment) is not an event of e;   */
/*  - an edge's events are computed from its lower-id end P to its other    */
/*    end Q: on the horizontal pixel line y0 the crossing is                 */
/*    x = P.x + ((y0 - P.y) (Q.x - P.x)) / (Q.y - P.y), on the vertical line  */
/*    x0 likewise; the two cells beside the edge see the same points;        */
/*  - the boundary vertices inside a cell are the PSLG vertices strictly     */
/*    inside its chord on their horizontal pixel line;                       */
/*  - the boundary pieces in a cell are the boundary runs of each pixel line */
/*    strictly between the cell's lowest and highest corner (resp. leftmost  */
/*    and rightmost), cut at the cell's nodes on that line;                  */
/*  - a cell is cut when it has an event or an inside vertex; Tier-T when,   */
/*    as on the lattice, no piece ends at a corner of the cell and every     */
/*    event ends exactly one piece, with no inside vertex and one or two     */
/*    chords, or one inside vertex every piece ends at; then the App. G      */
/*    template of its key; every other cut cell takes the greedy rule with   */
/*    double-precision predicates;                                           */
/*  - Alg. 1's mask: an event sets its edge, a corner on a piece sets both   */
/*    edges at that corner (vertex on the segment), an edge lying on a       */
/*    boundary run sets its own bit (overlap), bit 0 an inside vertex; the   */
/*    (m, n) class from the first two pieces' popcounts;                     */
/*  - numbering: T's vertices, then the events by owning cell (the smaller   */
/*    of the two cells beside the edge), local edge and position from the    */
/*    lower-id end, then the inside vertices by cell and pixel-corner id;    */
/*    triangles by cell, then the patch order; a triangle's label is that of */
/*    the pixel holding ((x1 + x2) + x3) / 3.                                */
/* ========================================================================= */
namespace {

/* planted mistakes for the tests (0 = none): 1 = a pixel corner on an edge
 * is an event even when its only boundary edges run along the edge; 2 =
 * boundary pieces oriented the wrong way; 3 = the inside test takes the
 * closed chord */
int g_r3_plant = 0;

struct R3Ev {
  double x, y, s;
  int kind;  /* 0 on horizontal line k, 1 on vertical line m, 2 at pixel corner (m, k) */
  i64 m, k;
};

struct R3Pt {
  double x, y;
};

bool r3_hb(const Image& im, i64 m, i64 k) { return im.at(m, k - 1) != im.at(m, k); }
bool r3_vb(const Image& im, i64 m, i64 k) { return im.at(m - 1, k) != im.at(m, k); }

/* position t on a pixel line: the pixel edge j holding it (edge j spans
 * [j - 1/2, j + 1/2]), or the corner c with t = c - 1/2 (returns true) */
bool r3_at_corner(double t, i64* idx) {
  const double fl = std::floor(t), fr = t - fl;
  if (fr == 0.5) {
    *idx = (i64)fl + 1;
    return true;
  }
  *idx = fr < 0.5 ? (i64)fl : (i64)fl + 1;
  return false;
}

double r3_hx(const R3Pt& P, const R3Pt& Q, double y0) { return P.x + ((y0 - P.y) * (Q.x - P.x)) / (Q.y - P.y); }
double r3_vy(const R3Pt& P, const R3Pt& Q, double x0) { return P.y + ((x0 - P.x) * (Q.y - P.y)) / (Q.x - P.x); }

/* the boundary pixel edges at corner (cx, cy) not collinear with an edge
 * that is horizontal (hz) or vertical (vt) */
bool r3_corner_event(const Image& im, i64 cx, i64 cy, bool hz, bool vt) {
  int m = corner_mask(im, cx, cy);
  if (g_r3_plant == 1) return m != 0;
  if (hz) m &= ~(CE_E | CE_W);
  if (vt) m &= ~(CE_N | CE_S);
  return m != 0;
}

/* events of the edge from P (its lower-id end) to Q, in order from P */
std::vector<R3Ev> r3_edge_events(const Image& im, const R3Pt& P, const R3Pt& Q) {
  std::vector<R3Ev> ev;
  const double dx = Q.x - P.x, dy = Q.y - P.y;
  const bool hz = dy == 0.0, vt = dx == 0.0;
  const double ylo = std::min(P.y, Q.y), yhi = std::max(P.y, Q.y);
  const double xlo = std::min(P.x, Q.x), xhi = std::max(P.x, Q.x);
  const i64 k0 = std::max<i64>(0, (i64)std::floor(ylo + 0.5)), k1 = std::min<i64>(im.H, (i64)std::ceil(yhi + 0.5));
  for (i64 k = k0; k <= k1; ++k) {
    const double y0 = (double)k - 0.5;
    if (!(ylo < y0 && y0 < yhi)) continue;
    const double x = r3_hx(P, Q, y0);
    i64 j;
    if (r3_at_corner(x, &j)) {
      if (r3_corner_event(im, j, k, hz, vt)) ev.push_back({x, y0, 0.0, 2, j, k});
    } else if (r3_hb(im, j, k)) {
      ev.push_back({x, y0, 0.0, 0, j, k});
    }
  }
  const i64 m0 = std::max<i64>(0, (i64)std::floor(xlo + 0.5)), m1 = std::min<i64>(im.W, (i64)std::ceil(xhi + 0.5));
  for (i64 m = m0; m <= m1; ++m) {
    const double x0 = (double)m - 0.5;
    if (!(xlo < x0 && x0 < xhi)) continue;
    const double y = r3_vy(P, Q, x0);
    i64 j;
    if (r3_at_corner(y, &j)) {
      bool dup = false;
      for (auto& e : ev)
        if (e.kind == 2 && e.m == m && e.k == j) dup = true;
      if (!dup && r3_corner_event(im, m, j, hz, vt)) ev.push_back({x0, y, 0.0, 2, m, j});
    } else if (r3_vb(im, m, j)) {
      ev.push_back({x0, y, 0.0, 1, m, j});
    }
  }
  const bool alongx = std::fabs(dx) >= std::fabs(dy);
  for (auto& e : ev) e.s = alongx ? (e.x - P.x) / dx : (e.y - P.y) / dy;
  std::sort(ev.begin(), ev.end(), [](const R3Ev& a, const R3Ev& b) {
    if (a.s != b.s) return a.s < b.s;
    if (a.kind != b.kind) return a.kind < b.kind;
    if (a.k != b.k) return a.k < b.k;
    return a.m < b.m;
  });
  return ev;
}

double r3_orient(const R3Pt& p, const R3Pt& q, const R3Pt& r) {
  return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);
}

/* greedy rule of the Tier-G cells with double predicates; on_edge[v] is the
 * set of cell edges v lies on (pairs on one cell edge are never
 * candidates: they are the cell's own boundary) */
std::vector<Tri> r3_greedy(const std::vector<R3Pt>& v, const std::vector<int>& on_edge,
                           const std::vector<std::pair<int, int>>& constraints) {
  const int n = (int)v.size();
  std::vector<std::vector<uint8_t>> adj(n, std::vector<uint8_t>(n, 0));
  std::vector<std::pair<int, int>> edges;
  for (auto& e : constraints) {
    const int a = std::min(e.first, e.second), b = std::max(e.first, e.second);
    if (!adj[a][b]) adj[a][b] = adj[b][a] = 1, edges.push_back({a, b});
  }
  /* candidates in order of squared length rounded to single precision,
   * ties by local index pair: lengths that are equal in exact arithmetic
   * (symmetric configurations) but differ by a few units of the double's
   * last place stay tied */
  struct Cand {
    float key;
    double len2;
    int u, w;
  };
  std::vector<Cand> cand;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      if (!adj[a][b] && (on_edge[a] & on_edge[b]) == 0) {
        const double dx = v[b].x - v[a].x, dy = v[b].y - v[a].y;
        const double l2 = dx * dx + dy * dy;
        cand.push_back({(float)l2, l2, a, b});
      }
  std::sort(cand.begin(), cand.end(), [](const Cand& x, const Cand& y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.u != y.u) return x.u < y.u;
    return x.w < y.w;
  });
  auto sgn = [](double o) { return o > 0.0 ? 1 : (o < 0.0 ? -1 : 0); };
  for (auto& c : cand) {
    bool ok = true;
    const double ex = v[c.w].x - v[c.u].x, ey = v[c.w].y - v[c.u].y;
    for (int k = 0; k < n && ok; ++k) {
      if (k == c.u || k == c.w || r3_orient(v[c.u], v[c.w], v[k]) != 0.0) continue;
      const double t = (v[k].x - v[c.u].x) * ex + (v[k].y - v[c.u].y) * ey;
      if (t > 0.0 && t < c.len2) ok = false;
    }
    for (size_t t = 0; t < edges.size() && ok; ++t) {
      const int a = edges[t].first, b = edges[t].second;
      if (a == c.u || a == c.w || b == c.u || b == c.w) continue;
      const int o1 = sgn(r3_orient(v[c.u], v[c.w], v[a])), o2 = sgn(r3_orient(v[c.u], v[c.w], v[b]));
      const int o3 = sgn(r3_orient(v[a], v[b], v[c.u])), o4 = sgn(r3_orient(v[a], v[b], v[c.w]));
      if (o1 * o2 < 0 && o3 * o4 < 0) ok = false;
    }
    if (ok) adj[c.u][c.w] = adj[c.w][c.u] = 1, edges.push_back({c.u, c.w});
  }
  std::vector<Tri> tri;
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      if (!adj[a][b]) continue;
      for (int c = b + 1; c < n; ++c) {
        if (!adj[a][c] || !adj[b][c]) continue;
        const int o = sgn(r3_orient(v[a], v[b], v[c]));
        if (o == 0) continue;
        bool empty = true;
        for (int k = 0; k < n && empty; ++k) {
          if (k == a || k == b || k == c) continue;
          if (sgn(r3_orient(v[a], v[b], v[k])) == o && sgn(r3_orient(v[b], v[c], v[k])) == o &&
              sgn(r3_orient(v[c], v[a], v[k])) == o)
            empty = false;
        }
        if (empty) tri.push_back(o > 0 ? Tri{a, b, c} : Tri{a, c, b});
      }
    }
  std::sort(tri.begin(), tri.end());
  return tri;
}

struct R3Mesh {
  std::vector<double> xy;
  std::vector<int32_t> tri;
  std::vector<uint16_t> label, code;
  i64 n_cut = 0, n_tierG = 0, n_events = 0, n_inside = 0;
};

/* the cell's two chord ends on a pixel line: horizontal (vert = false,
 * coordinate c0 = the line's y) or vertical; each end is (position along the
 * line, source) with source = corner 0..2 or 3 + edge */
int r3_chord(const R3Pt* K, const int* id, bool vert, double c0, double* pos, int* src) {
  int n = 0;
  for (int c = 0; c < 3; ++c)
    if ((vert ? K[c].x : K[c].y) == c0) {
      if (n == 2) return 3;
      pos[n] = vert ? K[c].y : K[c].x, src[n++] = c;
    }
  for (int j = 0; j < 3; ++j) {
    const int a = j, b = (j + 1) % 3;
    const R3Pt& P = id[a] < id[b] ? K[a] : K[b];
    const R3Pt& Q = id[a] < id[b] ? K[b] : K[a];
    const double pa = vert ? P.x : P.y, pb = vert ? Q.x : Q.y;
    if (!((pa < c0 && c0 < pb) || (pb < c0 && c0 < pa))) continue;
    if (n == 2) return 3;
    pos[n] = vert ? r3_vy(P, Q, c0) : r3_hx(P, Q, c0), src[n++] = 3 + j;
  }
  if (n == 2 && pos[1] < pos[0]) std::swap(pos[0], pos[1]), std::swap(src[0], src[1]);
  return n;
}

void r3_mesh(const Image& im, const std::vector<R3Pt>& X, const std::vector<int32_t>& T, R3Mesh& R) {
  const i64 nv = (i64)X.size(), nt = (i64)T.size() / 3;
  /* edge owners: the smaller cell beside each edge */
  std::map<std::pair<i64, i64>, std::vector<std::pair<i64, int>>> uses;
  for (i64 c = 0; c < nt; ++c)
    for (int j = 0; j < 3; ++j) {
      const i64 u = T[3 * c + j], w = T[3 * c + (j + 1) % 3];
      if (u < 0 || w < 0 || u >= nv || w >= nv || u == w) throw std::runtime_error("bad triangle");
      uses[{std::min(u, w), std::max(u, w)}].push_back({c, j});
    }
  for (auto& kv : uses)
    if (kv.second.size() > 2) throw std::runtime_error("edge in more than two cells");
  struct CellInfo {
    std::vector<R3Ev> ev[3]; /* in CCW order along the cell's edge j */
    std::vector<std::pair<i64, i64>> inside; /* (corner id, cx | cy << 32) sorted */
    std::vector<i64> evid[3];
  };
  std::vector<CellInfo> info(nt);
  /* events per cell edge, and global ids by owner, edge, position */
  i64 next = nv;
  std::vector<double> evxy;
  for (i64 c = 0; c < nt; ++c) {
    R3Pt K[3];
    int id[3];
    for (int q = 0; q < 3; ++q) id[q] = T[3 * c + q], K[q] = X[id[q]];
    if (!(r3_orient(K[0], K[1], K[2]) > 0.0)) throw std::runtime_error("cell not counter-clockwise");
    for (int j = 0; j < 3; ++j) {
      const int a = j, b = (j + 1) % 3;
      const bool fwd = id[a] < id[b];
      auto ev = r3_edge_events(im, fwd ? K[a] : K[b], fwd ? K[b] : K[a]);
      const auto& us = uses[{std::min(id[a], id[b]), std::max(id[a], id[b])}];
      i64 owner = c;
      for (auto& u : us) owner = std::min(owner, u.first);
      std::vector<i64> ids(ev.size(), -1);
      if (owner == c) {
        for (size_t t = 0; t < ev.size(); ++t) ids[t] = next++, evxy.push_back(ev[t].x), evxy.push_back(ev[t].y);
      }
      if (!fwd) std::reverse(ev.begin(), ev.end()), std::reverse(ids.begin(), ids.end());
      info[c].ev[j] = ev;
      info[c].evid[j] = ids;
    }
  }
  /* the non-owners take the owner's ids */
  for (i64 c = 0; c < nt; ++c)
    for (int j = 0; j < 3; ++j) {
      if (info[c].ev[j].empty() || info[c].evid[j][0] >= 0) continue;
      const i64 u = T[3 * c + j], w = T[3 * c + (j + 1) % 3];
      for (auto& us : uses[{std::min(u, w), std::max(u, w)}]) {
        if (us.first == c) continue;
        auto ids = info[us.first].evid[us.second];
        if (ids.size() != info[c].ev[j].size()) throw std::runtime_error("the cells beside an edge disagree");
        std::reverse(ids.begin(), ids.end());
        info[c].evid[j] = ids;
      }
    }
  R.n_events = next - nv;
  /* inside vertices */
  for (i64 c = 0; c < nt; ++c) {
    R3Pt K[3];
    int id[3];
    for (int q = 0; q < 3; ++q) id[q] = T[3 * c + q], K[q] = X[id[q]];
    const double ylo = std::min({K[0].y, K[1].y, K[2].y}), yhi = std::max({K[0].y, K[1].y, K[2].y});
    const double xlo = std::min({K[0].x, K[1].x, K[2].x}), xhi = std::max({K[0].x, K[1].x, K[2].x});
    const i64 cy0 = std::max<i64>(0, (i64)std::floor(ylo + 0.5)), cy1 = std::min<i64>(im.H, (i64)std::ceil(yhi + 0.5));
    const i64 cx0 = std::max<i64>(0, (i64)std::floor(xlo + 0.5)), cx1 = std::min<i64>(im.W, (i64)std::ceil(xhi + 0.5));
    for (i64 cy = cy0; cy <= cy1; ++cy) {
      const double y0 = (double)cy - 0.5;
      if (!(ylo < y0 && y0 < yhi)) continue;
      double pos[2];
      int src[2];
      if (r3_chord(K, id, false, y0, pos, src) != 2) throw std::runtime_error("chord");
      for (i64 cx = cx0; cx <= cx1; ++cx) {
        const double x0 = (double)cx - 0.5;
        if (g_r3_plant == 3 ? !(pos[0] <= x0 && x0 <= pos[1]) : !(pos[0] < x0 && x0 < pos[1])) continue;
        if (!is_vertex(corner_mask(im, cx, cy))) continue;
        info[c].inside.push_back({cy * (im.W + 1) + cx, cx | (cy << 32)});
      }
    }
    std::sort(info[c].inside.begin(), info[c].inside.end());
  }
  R.xy.reserve(2 * (nv + R.n_events));
  for (auto& p : X) R.xy.push_back(p.x), R.xy.push_back(p.y);
  R.xy.insert(R.xy.end(), evxy.begin(), evxy.end());
  i64 nin = 0;
  for (i64 c = 0; c < nt; ++c)
    for (auto& q : info[c].inside) {
      const i64 cx = q.second & 0xFFFFFFFF, cy = q.second >> 32;
      R.xy.push_back((double)cx - 0.5), R.xy.push_back((double)cy - 0.5);
      ++nin;
    }
  R.n_inside = nin;
  /* the cells' patches */
  i64 inbase = nv + R.n_events;
  auto label_of = [&](const R3Pt& a, const R3Pt& b, const R3Pt& d) {
    const double cx = ((a.x + b.x) + d.x) / 3.0, cy = ((a.y + b.y) + d.y) / 3.0;
    return out_label(im.at((i64)std::floor(cx + 0.5), (i64)std::floor(cy + 0.5)));
  };
  for (i64 c = 0; c < nt; ++c) {
    R3Pt K[3];
    int id[3];
    for (int q = 0; q < 3; ++q) id[q] = T[3 * c + q], K[q] = X[id[q]];
    const CellInfo& ci = info[c];
    const int nev[3] = {(int)ci.ev[0].size(), (int)ci.ev[1].size(), (int)ci.ev[2].size()};
    const int ne = nev[0] + nev[1] + nev[2], ni = (int)ci.inside.size();
    if (ne == 0 && ni == 0) {
      for (int q = 0; q < 3; ++q) R.tri.push_back(id[q]);
      R.label.push_back(label_of(K[0], K[1], K[2]));
      R.code.push_back(0);
      continue;
    }
    ++R.n_cut;
    /* local nodes */
    std::vector<R3Pt> v;
    std::vector<i64> gid;
    std::vector<int> on_edge;
    for (int q = 0; q < 3; ++q) v.push_back(K[q]), gid.push_back(id[q]), on_edge.push_back((1 << q) | (1 << ((q + 2) % 3)));
    for (int j = 0; j < 3; ++j)
      for (size_t t = 0; t < ci.ev[j].size(); ++t)
        v.push_back({ci.ev[j][t].x, ci.ev[j][t].y}), gid.push_back(ci.evid[j][t]), on_edge.push_back(1 << j);
    for (size_t t = 0; t < ci.inside.size(); ++t) {
      const i64 cx = ci.inside[t].second & 0xFFFFFFFF, cy = ci.inside[t].second >> 32;
      v.push_back({(double)cx - 0.5, (double)cy - 0.5}), gid.push_back(inbase + (i64)t), on_edge.push_back(0);
    }
    inbase += ni;
    auto ev_local = [&](int j, bool vert, i64 line) -> int {
      int base = 3;
      for (int t = 0; t < j; ++t) base += nev[t];
      for (int t = 0; t < nev[j]; ++t) {
        const R3Ev& e = ci.ev[j][t];
        if (e.kind == 2 ? (vert ? e.m == line : e.k == line) : (e.kind == (vert ? 1 : 0) && (vert ? e.m : e.k) == line))
          return base + t;
      }
      return -1;
    };
    /* pieces, oriented with the lower label on the left */
    std::vector<std::pair<int, int>> pieces;
    const double ylo = std::min({K[0].y, K[1].y, K[2].y}), yhi = std::max({K[0].y, K[1].y, K[2].y});
    const double xlo = std::min({K[0].x, K[1].x, K[2].x}), xhi = std::max({K[0].x, K[1].x, K[2].x});
    for (int vert = 0; vert < 2; ++vert) {
      const double lo = vert ? xlo : ylo, hi = vert ? xhi : yhi;
      const i64 L0 = std::max<i64>(0, (i64)std::floor(lo + 0.5));
      const i64 L1 = std::min<i64>(vert ? im.W : im.H, (i64)std::ceil(hi + 0.5));
      for (i64 line = L0; line <= L1; ++line) {
        const double c0 = (double)line - 0.5;
        if (!(lo < c0 && c0 < hi)) continue;
        double pos[2];
        int src[2];
        if (r3_chord(K, id, vert, c0, pos, src) != 2) throw std::runtime_error("chord");
        std::vector<std::pair<double, int>> nodes;
        auto end_node = [&](int e) {
          if (src[e] < 3) return src[e];
          return ev_local(src[e] - 3, vert, line);
        };
        const int n0 = end_node(0), n1 = end_node(1);
        if (n0 >= 0) nodes.push_back({pos[0], n0});
        for (int t = 0; t < ni; ++t) {
          const i64 cx = ci.inside[t].second & 0xFFFFFFFF, cy = ci.inside[t].second >> 32;
          if ((vert ? cx : cy) == line) nodes.push_back({vert ? (double)cy - 0.5 : (double)cx - 0.5, 3 + ne + t});
        }
        if (n1 >= 0) nodes.push_back({pos[1], n1});
        std::sort(nodes.begin() + (n0 >= 0 ? 1 : 0), nodes.end() - (n1 >= 0 ? 1 : 0));
        for (size_t t = 0; t + 1 < nodes.size(); ++t) {
          const double mid = (nodes[t].first + nodes[t + 1].first) * 0.5;
          i64 j;
          r3_at_corner(mid, &j); /* at a corner: the pixel edge starting there */
          bool bnd;
          int32_t l0, l1;
          if (!vert) {
            bnd = r3_hb(im, j, line), l0 = im.at(j, line - 1), l1 = im.at(j, line);
            /* going +x the left side is above: lower label above runs +x */
            if (bnd) pieces.push_back(l1 < l0 ? std::make_pair(nodes[t].second, nodes[t + 1].second)
                                              : std::make_pair(nodes[t + 1].second, nodes[t].second));
          } else {
            bnd = r3_vb(im, line, j), l0 = im.at(line - 1, j), l1 = im.at(line, j);
            /* going +y the left side is -x */
            if (bnd) pieces.push_back(l0 < l1 ? std::make_pair(nodes[t].second, nodes[t + 1].second)
                                              : std::make_pair(nodes[t + 1].second, nodes[t].second));
          }
        }
      }
    }
    if (g_r3_plant == 2)
      for (auto& p : pieces) std::swap(p.first, p.second);
    /* Alg. 1 mask and the (m, n) class */
    auto node_bits = [&](int w) {
      if (w < 3) return (2 << w) | (2 << ((w + 2) % 3));
      if (w < 3 + ne) {
        int k = w - 3;
        for (int j = 0; j < 3; ++j) {
          if (k < nev[j]) return 2 << j;
          k -= nev[j];
        }
      }
      return 0;
    };
    int mask = ni > 0 ? 1 : 0;
    std::vector<int> pc;
    for (auto& p : pieces) {
      const int b = node_bits(p.first) | node_bits(p.second);
      mask |= b;
      pc.push_back(__builtin_popcount(b));
    }
    for (int j = 0; j < 3; ++j) {
      const R3Pt &a = K[j], &b = K[(j + 1) % 3];
      for (int vert = 0; vert < 2; ++vert) {
        const double ca = vert ? a.x : a.y, cb = vert ? b.x : b.y;
        i64 line;
        if (ca != cb || !r3_at_corner(ca, &line)) continue; /* not on a pixel line */
        const double ta = vert ? a.y : a.x, tb = vert ? b.y : b.x;
        const double t0 = std::min(ta, tb), t1 = std::max(ta, tb);
        for (i64 q = (i64)std::floor(t0 + 0.5) - 1; q <= (i64)std::ceil(t1 + 0.5) + 1; ++q) {
          if (!((double)q + 0.5 > t0 && (double)q - 0.5 < t1)) continue;
          if (vert ? r3_vb(im, line, q) : r3_hb(im, q, line)) mask |= 2 << j;
        }
      }
    }
    int klass = 0;
    if (pieces.size() == 1) klass = class_index(0, pc[0]);
    else if (pieces.size() == 2) klass = class_index(pc[0], pc[1]);
    /* Tier-T or Tier-G */
    bool tierT = ni <= 1;
    std::vector<int> deg(v.size(), 0);
    for (auto& p : pieces) {
      if (p.first < 3 || p.second < 3) tierT = false;
      deg[p.first]++, deg[p.second]++;
    }
    for (int w = 3; w < 3 + ne; ++w)
      if (deg[w] != 1) tierT = false;
    if (ni == 0 && !(pieces.size() == 1 || pieces.size() == 2)) tierT = false;
    if (ni == 1)
      for (auto& p : pieces)
        if (p.first != 3 + ne && p.second != 3 + ne) tierT = false;
    LocalResult r;
    if (tierT) {
      r = classify_local(nev, ni, pieces);
      if (r.tierG) throw std::runtime_error("Tier-T cell outside the table");
    } else {
      std::vector<std::pair<int, int>> cons = pieces;
      std::vector<int> cyc;
      for (int j = 0; j < 3; ++j) {
        cyc.push_back(j);
        int base = 3;
        for (int t = 0; t < j; ++t) base += nev[t];
        for (int t = 0; t < nev[j]; ++t) cyc.push_back(base + t);
      }
      for (size_t t = 0; t < cyc.size(); ++t) cons.push_back({cyc[t], cyc[(t + 1) % cyc.size()]});
      r.tri = r3_greedy(v, on_edge, cons);
      r.tierG = 1, r.key = 63, r.sigma = 0;
      ++R.n_tierG;
      if ((int)r.tri.size() != 2 * ni + (3 + ne) - 2) throw std::runtime_error("greedy triangle count");
    }
    r.mask = mask, r.klass = klass;
    const uint16_t code = make_code(r);
    for (auto& t : r.tri) {
      for (int q = 0; q < 3; ++q) R.tri.push_back((int32_t)gid[t[q]]);
      R.label.push_back(label_of(v[t[0]], v[t[1]], v[t[2]]));
      R.code.push_back(code);
    }
  }
}

/* the base mesh T0 as arrays: lattice vertices in id order, cells' corners */
void base_mesh_arrays(i64 W, i64 H, i64 p, i64 q, i64 o2x, i64 o2y, std::vector<R3Pt>& X, std::vector<int32_t>& T,
                      i64* ncells) {
  Grid g;
  build_grid(g, W, H, p, q, o2x, o2y);
  X.clear(), T.clear();
  for (i64 j = g.vj0; j <= g.vj1; ++j)
    for (i64 i = g.vlo[j - g.vj0]; i <= g.vhi[j - g.vj0]; ++i) {
      const Pt v = g.vtx(i, j);
      X.push_back({to_double(v.x) / (double)g.S, to_double(v.y) / (double)g.S});
    }
  for (i64 j = g.j0; j <= g.j1; ++j)
    for (i64 c = g.clo[j - g.j0]; c <= g.chi[j - g.j0]; ++c) {
      i64 ci[3], cj[3];
      g.corners(c, j, ci, cj);
      for (int k = 0; k < 3; ++k) T.push_back((int32_t)g.vid(ci[k], cj[k]));
    }
  *ncells = g.ncells;
}

}  // namespace

extern "C" {

/* Every binary W x H <= 25 bitmap (bit k = pixel k, row-major; from first,
 * every stride-th) meshed by the general path -- the base mesh at origin
 * (o2x/2, o2y/2), any integer o2x, o2y, then Region III -- and checked
 * against the invariants of any correct output.  Returns the number checked,
 * or -(1 + the first failing bitmap) with the message in oracle_last_error. */
int64_t oracle_brute_general(int32_t W, int32_t H, int32_t h_num, int32_t h_den, int32_t o2x, int32_t o2y,
                             int64_t first, int64_t stride) {
  g_err[0] = 0;
  if (W < 1 || H < 1 || W * H > 25 || stride < 1 || first < 0) return -1;
  std::vector<uint8_t> img(W * H);
  const int64_t n = (int64_t)1 << (W * H);
  int64_t done = 0;
  std::vector<R3Pt> X;
  std::vector<int32_t> T;
  for (int64_t b = first; b < n; b += stride) {
    for (int k = 0; k < W * H; ++k) img[k] = (uint8_t)((b >> k) & 1);
    try {
      Image im{W, H, (int64_t)W, 1, img.data()};
      i64 ncells = 0;
      base_mesh_arrays(W, H, h_num, h_den, o2x, o2y, X, T, &ncells);
      R3Mesh R;
      r3_mesh(im, X, T, R);
      Mesh M;
      M.xy = R.xy, M.tri = R.tri, M.label = R.label, M.ncells = ncells;
      if (check_invariants(img.data(), W, H, (double)h_num / h_den, M)) {
        const std::string what = g_err;
        std::snprintf(g_err, sizeof g_err, "bitmap %lld: %.400s", (long long)b, what.c_str());
        return -(1 + b);
      }
    } catch (const std::exception& ex) {
      std::snprintf(g_err, sizeof g_err, "bitmap %lld: %s", (long long)b, ex.what());
      return -(1 + b);
    }
    ++done;
  }
  return done;
}

/* Region III: Alg. 2 on the counter-clockwise triangle mesh T (nv vertices
 * as 2 doubles, nt cells as 3 vertex ids) against the boundary of the image;
 * the result in out (n_cells = nt, n_vertices_grid = nv, n_events; seg, ev
 * and cut empty).  plant != 0 plants a mistake (tests only).  0, -1 bad
 * arguments, -2 a consistency failure. */
int oracle_region3(const void* data, int32_t width, int32_t height, int64_t pitch_bytes, int32_t dtype,
                   const double* xy, int64_t nv, const int32_t* tri, int64_t nt, int32_t plant, oracle_mesh* out) {
  g_err[0] = 0;
  g_r3_plant = plant;
  if (!data || !out || !xy || !tri || width < 1 || height < 1 || (dtype != 1 && dtype != 2) ||
      pitch_bytes < (int64_t)width * dtype || nv < 3 || nt < 1) {
    std::snprintf(g_err, sizeof g_err, "invalid arguments");
    return -1;
  }
  try {
    Image im{width, height, pitch_bytes, dtype, (const uint8_t*)data};
    std::vector<R3Pt> X((size_t)nv);
    for (i64 v = 0; v < nv; ++v) X[v] = {xy[2 * v], xy[2 * v + 1]};
    std::vector<int32_t> T(tri, tri + 3 * nt);
    R3Mesh R;
    r3_mesh(im, X, T, R);
    std::memset(out, 0, sizeof *out);
    out->n_vertices = (int64_t)R.xy.size() / 2;
    out->n_triangles = (int64_t)R.label.size();
    out->n_cells = nt;
    out->n_cut_cells = R.n_cut;
    out->n_tierG_cells = R.n_tierG;
    out->n_vertices_grid = nv;
    out->xy = dup(R.xy);
    out->tri = dup(R.tri);
    out->label = dup(R.label);
    out->code = dup(R.code);
    out->n_events = R.n_events;
    out->seg = dup(std::vector<int32_t>());
    out->ev = dup(std::vector<int64_t>());
    out->cut = dup(std::vector<int64_t>());
    return 0;
  } catch (const std::exception& ex) {
    std::snprintf(g_err, sizeof g_err, "%s", ex.what());
    return -2;
  }
}

}  // extern "C"
