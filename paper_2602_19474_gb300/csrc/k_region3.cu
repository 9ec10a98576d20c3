// k_region3.cu -- Region III of Alg. 3's schedule (the corollary on
// pipelined parallel scheduling: Regions I and II, a barrier, then Region
// III): Alg. 2, the template retriangulation, run on the preprocessed mesh T,
// one cell at a time from its local intersection class (the corollary on
// lookup-driven parallel retriangulation: patches out of place, then one
// deterministic stitching by scan offsets).
//
// T's vertices are doubles (Steps 1-2 move them off the lattice), so every
// quantity is a double computed by one fixed formula, each operation rounded
// once (explicit round-to-nearest intrinsics: no contraction into FMAs).
// Degenerate incidences are exact: a pixel line is k - 1/2, and a vertex
// snapped onto a pixel corner sits on it exactly.
//
//  - An event of a mesh edge e is a point of the open edge where the
//    boundary meets it: the crossing of a boundary pixel edge, or a pixel
//    corner on e with a boundary pixel edge not collinear with e (Alg. 1's
//    endpoint on the edge; a run of boundary along e is embedded by e
//    itself: Alg. 1's overlap).  An end of e on the boundary (Alg. 1's
//    vertex on the segment) is not an event of e.  An edge's events are
//    computed from its lower-id end P: on the horizontal pixel line y0 the
//    crossing is x = P.x + ((y0 - P.y)(Q.x - P.x)) / (Q.y - P.y), on a
//    vertical line likewise; the two cells beside the edge see the same
//    points.
//  - The boundary vertices inside a cell are the PSLG vertices strictly
//    inside its chord on their horizontal pixel line.
//  - The boundary pieces of a cell are the boundary runs of each pixel line
//    strictly between the cell's extreme corners, cut at the cell's nodes on
//    the line.
//  - Tier-T (the table's regime, as on the lattice): no piece ends at a
//    corner of the cell and every event ends one piece; no inside vertex
//    and one or two chords, or one inside vertex every piece ends at.  The
//    patch is the App. G template of the cell's key.  Every other cut cell
//    (Tier-G) takes the greedy rule: vertex pairs in order of squared length
//    rounded to single precision (ties by local index pair), kept when the
//    open segment holds no vertex and crosses no kept edge.
//
// Kernels: k_r3_deg / k_r3_fill (cells around each vertex); k_r3_screen
// (every cell: a cell whose pixel box carries one label is uncut and takes
// that label, with no double-precision work; the others are listed);
// k_r3_count (the listed cells: triangles, events on the edges each owns --
// the smaller of the two cells beside an edge -- and inside vertices); three
// scans; k_r3_emit_uncut; k_r3_emit (the listed cells: Tier-T patches, the
// greedy rule for Tier-G cells of at most 12 nodes, larger ones queued);
// k_r3_tierg (one warp per queued cell).
#include "sbmt_cell.cuh"
#include "sbmt_keys.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

constexpr int R3_MAXE = 16;  // events on one edge
constexpr int R3_MAXI = 16;  // boundary vertices inside one cell
constexpr int R3_MAXN = 48;  // nodes of one cell: 3 corners, events, inside vertices
constexpr int R3_MAXP = 48;  // boundary pieces of one cell
constexpr int R3_OUTSIDE = 0x10000;

SBMT_DEV double dad(double a, double b) { return __dadd_rn(a, b); }
SBMT_DEV double dsb(double a, double b) { return __dsub_rn(a, b); }
SBMT_DEV double dml(double a, double b) { return __dmul_rn(a, b); }
SBMT_DEV double ddv(double a, double b) { return __ddiv_rn(a, b); }

SBMT_DEV int r3_px(const R3Args& a, i64 x, i64 y) {
  if (x < 0 || y < 0 || x >= a.W || y >= a.H) return R3_OUTSIDE;
  const unsigned char* row = a.img + y * a.pitch;
  return a.dtype == 1 ? (int)row[x] : (int)reinterpret_cast<const unsigned short*>(row)[x];
}
// horizontal pixel edge (m, k): from corner (m, k) to (m + 1, k), between
// pixels (m, k - 1) and (m, k); vertical edge (m, k): from corner (m, k) to
// (m, k + 1), between pixels (m - 1, k) and (m, k)
SBMT_DEV bool r3_hb(const R3Args& a, i64 m, i64 k) { return r3_px(a, m, k - 1) != r3_px(a, m, k); }
SBMT_DEV bool r3_vb(const R3Args& a, i64 m, i64 k) { return r3_px(a, m - 1, k) != r3_px(a, m, k); }
enum { R3E = 1, R3N = 2, R3W = 4, R3S = 8 };
SBMT_DEV int r3_cmask(const R3Args& a, i64 cx, i64 cy) {
  return (r3_hb(a, cx, cy) ? R3E : 0) | (r3_vb(a, cx, cy) ? R3N : 0) | (r3_hb(a, cx - 1, cy) ? R3W : 0) |
         (r3_vb(a, cx, cy - 1) ? R3S : 0);
}
SBMT_DEV bool r3_is_vertex(int m) { return m != 0 && m != (R3E | R3W) && m != (R3N | R3S); }

// position t on a pixel line: the pixel edge j holding it (edge j spans
// [j - 1/2, j + 1/2]), or the corner c with t = c - 1/2 (returns true)
SBMT_DEV bool r3_at_corner(double t, i64* idx) {
  const double fl = floor(t), fr = dsb(t, fl);
  if (fr == 0.5) {
    *idx = (i64)fl + 1;
    return true;
  }
  *idx = fr < 0.5 ? (i64)fl : (i64)fl + 1;
  return false;
}
SBMT_DEV double r3_hx(double2 P, double2 Q, double y0) {
  return dad(P.x, ddv(dml(dsb(y0, P.y), dsb(Q.x, P.x)), dsb(Q.y, P.y)));
}
SBMT_DEV double r3_vy(double2 P, double2 Q, double x0) {
  return dad(P.y, ddv(dml(dsb(x0, P.x), dsb(Q.y, P.y)), dsb(Q.x, P.x)));
}
SBMT_DEV double r3_orient(double2 p, double2 q, double2 r) {
  return dsb(dml(dsb(q.x, p.x), dsb(r.y, p.y)), dml(dsb(q.y, p.y), dsb(r.x, p.x)));
}
SBMT_DEV int r3_sgn(double o) { return o > 0.0 ? 1 : (o < 0.0 ? -1 : 0); }
SBMT_DEV i64 r3_lo(double v) { return (i64)floor(dad(v, 0.5)); }
SBMT_DEV i64 r3_hi(double v) { return (i64)ceil(dad(v, 0.5)); }

struct R3Ev {
  double x, y, s;
  int kind;  // 0 on horizontal line k, 1 on vertical line m, 2 at pixel corner (m, k)
  int m, k;
};

// the boundary pixel edges at corner (cx, cy) not collinear with an edge
// that is horizontal (hz) or vertical (vt)
SBMT_DEV bool r3_corner_event(const R3Args& a, i64 cx, i64 cy, bool hz, bool vt) {
  int m = r3_cmask(a, cx, cy);
  if (hz) m &= ~(R3E | R3W);
  if (vt) m &= ~(R3N | R3S);
  return m != 0;
}

// ---------------------------------------------------------------------------
// single-precision filters for the positions on pixel lines.  The double
// formulas above are the definition (the oracle's arithmetic); a float
// computation decides where a proven bound allows, the double formula
// where it does not, so that every decision is the double formula's.
// ---------------------------------------------------------------------------
// This GPU converts from double to float, from 64-bit integers to double
// and from float to 64-bit integers at about the rate of its FP64
// arithmetic (a few per clock per SM, against about a hundred for float
// arithmetic and for integer to float conversions), so the filters take
// doubles apart with integer instructions.
//
// v (|v| <= 2^24) as a 64-bit fixed-point number with 36 fraction bits:
// floor(v 2^36), exactly, and whether v 2^36 was not an integer (*inexact)
SBMT_DEV i64 r3_fix36(double v, bool* inexact) {
  const u64 b = (u64)__double_as_longlong(v);
  const bool neg = (b >> 63) != 0;
  const int e = (int)((b >> 52) & 0x7FF);
  const u64 frac = b & 0xFFFFFFFFFFFFFull;
  i64 f;
  bool lost;
  if (e == 0) {
    lost = frac != 0;  // zero, or a denormal (below one unit)
    f = (neg && lost) ? 1 : 0;
  } else {
    const i64 m = (i64)(frac | (1ull << 52));
    const int sh = e - 1039;  // v = m 2^(e - 1075), so v 2^36 = m 2^(e - 1039); sh <= 8 up to 2^24
    if (sh >= 0) {
      f = m << sh, lost = false;
    } else if (sh > -63) {
      lost = (m & ((1ll << -sh) - 1)) != 0;
      f = (m >> -sh) + ((neg && lost) ? 1 : 0);  // magnitude rounded towards the floor
    } else {
      f = neg ? 1 : 0, lost = true;
    }
  }
  *inexact = lost;
  return neg ? -f : f;
}
// the float of an integer |n| < 2^22, exactly: n in the mantissa of 1.5 2^23 + n
SBMT_DEV float r3_i2f(int n) { return __fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f); }
// the nearest integer to a float |z| < 2^22, and the floor
SBMT_DEV int r3_fint(float z) { return __float_as_int(__fadd_rn(z, 12582912.0f)) - 0x4B400000; }
SBMT_DEV int r3_ffloor(float z) {
  const int n = r3_fint(z);
  return r3_i2f(n) > z ? n - 1 : n;
}
// A coordinate v as an integer i = floor(v) and f: the remainder v - i (in
// [0, 1), exact in double) truncated to a multiple of 2^-23, so that
// v - i - 2^-23 - 2^-36 < f <= v - i.
struct R3Split {
  i64 i, fx;
  float f;
  bool inexact;
};
SBMT_DEV R3Split r3_split(double v) {
  R3Split s;
  s.fx = r3_fix36(v, &s.inexact);
  s.i = s.fx >> 36;
  const int n23 = (int)((s.fx & ((1ll << 36) - 1)) >> 13);
  s.f = __fmul_rn(__fsub_rn(__int_as_float(0x4B000000 | n23), 8388608.0f), 1.1920928955078125e-7f);  // n23 2^-23
  return s;
}
// v against the pixel line k - 1/2, exactly, from fx = floor(v 2^36):
// below iff fx < (k - 1/2) 2^36; above iff fx is greater, or equal with
// bits dropped
SBMT_DEV i64 r3_line36(i64 k) { return (k << 36) - (1ll << 35); }
SBMT_DEV bool r3_lt(const R3Split& v, i64 k) { return v.fx < r3_line36(k); }
SBMT_DEV bool r3_gt(const R3Split& v, i64 k) {
  const i64 t = r3_line36(k);
  return v.fx > t || (v.fx == t && v.inexact);
}
// the float of a coordinate difference from the fixed-point values (within
// 2^-35 + 2^-24 |d| of the double difference's real value; integer to
// float conversions run at the float rate)
SBMT_DEV float r3_fdiff(const R3Split& q, const R3Split& p) {
  return __fmul_rn((float)(q.fx - p.fx), 1.4551915228366852e-11f);
}

// The crossing of the edge from P (its lower-id end) with the line at
// coordinate c0 = k - 1/2 across it, as w = (position along the line) - B,
// B the integer part of P's coordinate along the line.  With A = c0 - P (in
// the crossing direction: k - 1/2 - Pi - Pr, the integer part exact) and
// s = the edge's slope in float, w = Pr + A s.  The remainders are within
// 2^-22 of their values, the differences within 2^-35 + 2^-23 |d|, the
// slope within 5 2^-24 |s| relatively, so the float w is within
// 2^-24 (8 + 8|s| + 7 D + |w|) of the real w of the double inputs (D: the
// edge's larger extent; |A| is below the extent across the line, |A s|
// below the extent along it), and the double formula within
// 2^-53 (|position| + 3 D) of that real value; T (below) is above their
// sum at every coordinate up to 2^24.
SBMT_DEV float r3_cross_tol(float D, float s, float w) {
  return 6.0e-7f * (D + fabsf(s) + 2.0f * fabsf(w) + 3.0f) + 1.5e-8f;
}
// the double formula's crossing with the line c0 (vert: x = c0, giving y):
// its pixel edge or corner index in *j, *corner set
__device__ __noinline__ void r3_cross_exact(double2 P, double2 Q, double c0, bool vert, i64* j, bool* corner) {
  *corner = r3_at_corner(vert ? r3_vy(P, Q, c0) : r3_hx(P, Q, c0), j);
}

// the number of events of the edge from P (its lower-id end) to Q, or -1
// past R3_MAXE, through the filters (the count pass's form: positions are
// not needed there); ev receives the events' kinds and pixel indices, for
// the corner found on both line families to count once
SBMT_DEV int r3_edge_count(const R3Args& a, double2 P, double2 Q, R3Ev* ev) {
  int n = 0;
  const bool hz = P.y == Q.y, vt = P.x == Q.x;
  const R3Split px = r3_split(P.x), py = r3_split(P.y), qx = r3_split(Q.x), qy = r3_split(Q.y);
  const float dxf = r3_fdiff(qx, px), dyf = r3_fdiff(qy, py);
  const float D = fmaxf(fabsf(dxf), fabsf(dyf));
  if (!hz) {
    // horizontal lines y = k - 1/2 strictly between P.y and Q.y
    const float sl = __fdiv_rn(dxf, dyf);
    const i64 k0 = max((i64)0, min(py.i, qy.i) - 1), k1 = min((i64)a.H, max(py.i, qy.i) + 3);
    for (i64 k = k0; k <= k1; ++k) {
      if (!((r3_lt(py, k) && r3_gt(qy, k)) || (r3_lt(qy, k) && r3_gt(py, k)))) continue;
      const float hp = r3_i2f((int)(k - py.i)) - 0.5f;
      const float w = __fadd_rn(px.f, __fmul_rn(__fsub_rn(hp, py.f), sl));
      const float z = __fadd_rn(w, 0.5f);
      const int zi = r3_ffloor(z);
      const float fr = __fsub_rn(z, r3_i2f(zi)), T = r3_cross_tol(D, sl, w);
      i64 j;
      bool corner = false;
      if (fr > T && fr < 1.0f - T) j = px.i + zi;
      else r3_cross_exact(P, Q, (double)k - 0.5, false, &j, &corner);
      if (corner ? r3_corner_event(a, j, k, hz, vt) : r3_hb(a, j, k)) {
        if (n == R3_MAXE) return -1;
        ev[n].kind = corner ? 2 : 0, ev[n].m = (int)j, ev[n].k = (int)k;
        ++n;
      }
    }
  }
  if (!vt) {
    // vertical lines x = m - 1/2 strictly between P.x and Q.x
    const float sl = __fdiv_rn(dyf, dxf);
    const i64 m0 = max((i64)0, min(px.i, qx.i) - 1), m1 = min((i64)a.W, max(px.i, qx.i) + 3);
    for (i64 m = m0; m <= m1; ++m) {
      if (!((r3_lt(px, m) && r3_gt(qx, m)) || (r3_lt(qx, m) && r3_gt(px, m)))) continue;
      const float hp = r3_i2f((int)(m - px.i)) - 0.5f;
      const float w = __fadd_rn(py.f, __fmul_rn(__fsub_rn(hp, px.f), sl));
      const float z = __fadd_rn(w, 0.5f);
      const int zi = r3_ffloor(z);
      const float fr = __fsub_rn(z, r3_i2f(zi)), T = r3_cross_tol(D, sl, w);
      i64 j;
      bool corner = false;
      if (fr > T && fr < 1.0f - T) j = py.i + zi;
      else r3_cross_exact(P, Q, (double)m - 0.5, true, &j, &corner);
      if (corner) {
        bool dup = false;
        for (int t = 0; t < n; ++t)
          if (ev[t].kind == 2 && ev[t].m == (int)m && ev[t].k == (int)j) dup = true;
        if (dup || !r3_corner_event(a, m, j, hz, vt)) continue;
      } else if (!r3_vb(a, m, j)) {
        continue;
      }
      if (n == R3_MAXE) return -1;
      ev[n].kind = corner ? 2 : 1, ev[n].m = (int)m, ev[n].k = (int)j;
      ++n;
    }
  }
  return n;
}

// the cell's two chord ends on a pixel line (vert: the vertical line x = c0,
// else the horizontal y = c0): (position along the line, source = corner 0..2
// or 3 + edge); the number of ends found (2 for a proper cell)
SBMT_DEV int r3_chord(const double2* K, const int* id, bool vert, double c0, double* pos, int* src) {
  int n = 0;
  for (int c = 0; c < 3; ++c)
    if ((vert ? K[c].x : K[c].y) == c0) {
      if (n == 2) return 3;
      pos[n] = vert ? K[c].y : K[c].x, src[n++] = c;
    }
  for (int j = 0; j < 3; ++j) {
    const int u = j, w = j == 2 ? 0 : j + 1;
    const double2 P = id[u] < id[w] ? K[u] : K[w], Q = id[u] < id[w] ? K[w] : K[u];
    const double pa = vert ? P.x : P.y, pb = vert ? Q.x : Q.y;
    if (!((pa < c0 && c0 < pb) || (pb < c0 && c0 < pa))) continue;
    if (n == 2) return 3;
    pos[n] = vert ? r3_vy(P, Q, c0) : r3_hx(P, Q, c0), src[n++] = 3 + j;
  }
  if (n == 2 && pos[1] < pos[0]) {
    const double t = pos[0];
    pos[0] = pos[1], pos[1] = t;
    const int s = src[0];
    src[0] = src[1], src[1] = s;
  }
  return n;
}

struct R3Cell {
  double2 K[3];
  int id[3];
  double ylo, yhi, xlo, xhi;
};
// the corners alone (the bounding box left unset)
SBMT_DEV R3Cell r3_load_k(const R3Args& a, u32 c) {
  R3Cell C;
  const int* t = a.ttri + 3 * (u64)c;
  for (int q = 0; q < 3; ++q) C.id[q] = t[q], C.K[q] = reinterpret_cast<const double2*>(a.txy)[C.id[q]];
  return C;
}
SBMT_DEV R3Cell r3_load(const R3Args& a, u32 c) {
  R3Cell C;
  const int* t = a.ttri + 3 * (u64)c;
  for (int q = 0; q < 3; ++q) C.id[q] = t[q], C.K[q] = reinterpret_cast<const double2*>(a.txy)[C.id[q]];
  C.ylo = fmin(fmin(C.K[0].y, C.K[1].y), C.K[2].y), C.yhi = fmax(fmax(C.K[0].y, C.K[1].y), C.K[2].y);
  C.xlo = fmin(fmin(C.K[0].x, C.K[1].x), C.K[2].x), C.xhi = fmax(fmax(C.K[0].x, C.K[1].x), C.K[2].x);
  return C;
}

// one label over the pixels touching the cell's bounding box: no boundary
// pixel edge meets the cell, and every pixel the cell covers has that label
// (returned, OUTSIDE as 0xFFFF), or -1.  The box is the double-precision one
// grown by 1e-6 px, or any box holding it: a larger box finds a cell of one
// label at most where the exact one does, and a cell it misses becomes a
// candidate with no event and no inside vertex, emitted as it is with the
// label of the pixel holding its centroid, a pixel of the exact box -- the
// same output.  Here the box comes from the corners' fixed-point values
// (within 2^-36 of the doubles), its ends moved outwards by 2^-36 and
// 2e-6 px, all in integer arithmetic.
SBMT_DEV int r3_uniform(const R3Args& a, const i64* X, const i64* Y) {
  constexpr i64 HALF = 1ll << 35, GROW = 137439 + 1;  // 1/2 and 2e-6 (rounded up) plus 2^-36, in 2^-36 units
  const i64 xlo = min(min(X[0], X[1]), X[2]), xhi = max(max(X[0], X[1]), X[2]);
  const i64 ylo = min(min(Y[0], Y[1]), Y[2]), yhi = max(max(Y[0], Y[1]), Y[2]);
  // ceil(lo - 1/2 - grow) and floor(hi + 1/2 + grow) in pixels
  const i64 x0 = -((-(xlo - HALF - GROW)) >> 36), x1 = (xhi + HALF + GROW) >> 36;
  const i64 y0 = -((-(ylo - HALF - GROW)) >> 36), y1 = (yhi + HALF + GROW) >> 36;
  const int l0 = r3_px(a, x0, y0);
  // every pixel beyond the image reads OUTSIDE, like those of the one-pixel
  // margin kept: the scan stops there without changing its answer
  for (i64 y = max(y0, (i64)-1), ye = min(y1, (i64)a.H); y <= ye; ++y)
    for (i64 x = max(x0, (i64)-1), xe = min(x1, (i64)a.W); x <= xe; ++x)
      if (r3_px(a, x, y) != l0) return -1;
  return l0 == R3_OUTSIDE ? 0xFFFF : l0;
}

// counter-clockwise (a positive orientation of the doubles), with a
// single-precision filter: the coordinate differences from the fixed-point
// values are within 2^-35 + 2^-24 |d| of the doubles' (D: the largest), so
// the float orientation is within 2^-33 D + 7 2^-24 D^2 of the exact one,
// and the double formula within 2^-50 D^2 of it; beyond twice that the
// float sign decides, else the double formula
SBMT_DEV bool r3_ccw(const double2* K, const i64* X, const i64* Y) {
  constexpr float S36 = 1.4551915228366852e-11f;  // 2^-36
  const float ax = __fmul_rn((float)(X[1] - X[0]), S36), ay = __fmul_rn((float)(Y[1] - Y[0]), S36);
  const float bx = __fmul_rn((float)(X[2] - X[0]), S36), by = __fmul_rn((float)(Y[2] - Y[0]), S36);
  const float o = __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
  const float D = fmaxf(fmaxf(fabsf(ax), fabsf(ay)), fmaxf(fabsf(bx), fabsf(by))) + 5.9604645e-8f;
  const float T = 4.7e-10f * D + 1.4e-6f * D * D;
  if (o > T) return true;
  if (o < -T) return false;
  return r3_orient(K[0], K[1], K[2]) > 0.0;
}

// the boundary vertices strictly inside the cell, as corner ids y (W+1) + x
// in id order; the count, -1 past R3_MAXI, -2 for a row the cell meets in
// other than two points.  Rows strictly inside the cell's y-range; on each,
// the chord's two ends (a corner on the row, or an edge crossing it, as in
// r3_chord): a corner compared with the pixel corners exactly through its
// fixed-point value, a crossing as a float interval around the double
// formula's position (the crossing filter's bound), the double formula
// taken only where the interval holds the pixel corner compared with.
struct R3End {
  i64 b;     // integer base of the position
  float w, T;
  int src;   // corner 0..2, or 3 + edge
};
// the sign of (an edge end's position) - (cx - 1/2), from the double formula
__device__ __noinline__ int r3_end_cmp_exact(const R3Cell& C, int src, i64 cx, double c0) {
  const int j = src - 3, u = j, v = j == 2 ? 0 : j + 1;
  const bool fwd = C.id[u] < C.id[v];
  const double p = r3_hx(fwd ? C.K[u] : C.K[v], fwd ? C.K[v] : C.K[u], c0);
  const double x0 = dsb((double)cx, 0.5);
  return p < x0 ? -1 : (p > x0 ? 1 : 0);
}
// the end's position below x0 = cx - 1/2: a corner's exactly from its
// fixed-point value, a crossing's from the float interval or the double
// formula
SBMT_DEV bool r3_end_below(const R3Cell& C, const R3Split* sx, const R3End& e, i64 cx, double c0) {
  if (e.src < 3) return r3_lt(sx[e.src], cx);
  const float h = r3_i2f((int)(cx - e.b)) - 0.5f;
  if (__fsub_rn(h, e.w) > e.T) return true;
  if (__fsub_rn(e.w, h) > e.T) return false;
  return r3_end_cmp_exact(C, e.src, cx, c0) < 0;
}
SBMT_DEV bool r3_end_above(const R3Cell& C, const R3Split* sx, const R3End& e, i64 cx, double c0) {
  if (e.src < 3) return r3_gt(sx[e.src], cx);
  const float h = r3_i2f((int)(cx - e.b)) - 0.5f;
  if (__fsub_rn(e.w, h) > e.T) return true;
  if (__fsub_rn(h, e.w) > e.T) return false;
  return r3_end_cmp_exact(C, e.src, cx, c0) > 0;
}
SBMT_DEV int r3_inside(const R3Args& a, const R3Cell& C, u32* out) {
  R3Split sx[3], sy[3];
  for (int q = 0; q < 3; ++q) sx[q] = r3_split(C.K[q].x), sy[q] = r3_split(C.K[q].y);
  float sl[3], D[3];
  for (int j = 0; j < 3; ++j) {
    const int u = j, v = j == 2 ? 0 : j + 1;
    const int P = C.id[u] < C.id[v] ? u : v, Q = P == u ? v : u;
    const float dxf = r3_fdiff(sx[Q], sx[P]), dyf = r3_fdiff(sy[Q], sy[P]);
    sl[j] = __fdiv_rn(dxf, dyf), D[j] = fmaxf(fabsf(dxf), fabsf(dyf));
  }
  const i64 cy0 = max((i64)0, min(min(sy[0].i, sy[1].i), sy[2].i) - 1);
  const i64 cy1 = min((i64)a.H, max(max(sy[0].i, sy[1].i), sy[2].i) + 3);
  const i64 cx0 = max((i64)0, min(min(sx[0].i, sx[1].i), sx[2].i) - 1);
  const i64 cx1 = min((i64)a.W, max(max(sx[0].i, sx[1].i), sx[2].i) + 3);
  int n = 0;
  for (i64 cy = cy0; cy <= cy1; ++cy) {
    bool below = false, above = false, lt[3], gt[3];
    for (int q = 0; q < 3; ++q) {
      lt[q] = r3_lt(sy[q], cy), gt[q] = r3_gt(sy[q], cy);
      below |= lt[q], above |= gt[q];
    }
    if (!(below && above)) continue;
    const double c0 = (double)cy - 0.5;
    R3End e[2];
    int ne = 0;
    for (int q = 0; q < 3; ++q)
      if (!lt[q] && !gt[q]) {  // the corner lies on the row
        if (ne == 2) return -2;
        e[ne++] = R3End{sx[q].i, sx[q].f, 0.0f, q};  // compared exactly
      }
    for (int j = 0; j < 3; ++j) {
      const int u = j, v = j == 2 ? 0 : j + 1;
      if (!((lt[u] && gt[v]) || (lt[v] && gt[u]))) continue;
      if (ne == 2) return -2;
      const int P = C.id[u] < C.id[v] ? u : v;
      const float hP = r3_i2f((int)(cy - sy[P].i)) - 0.5f;
      const float w = __fadd_rn(sx[P].f, __fmul_rn(__fsub_rn(hP, sy[P].f), sl[j]));
      e[ne++] = R3End{sx[P].i, w, r3_cross_tol(D[j], sl[j], w), 3 + j};
    }
    if (ne != 2) return -2;
    for (i64 cx = cx0; cx <= cx1; ++cx) {
      const bool inside = (r3_end_below(C, sx, e[0], cx, c0) && r3_end_above(C, sx, e[1], cx, c0)) ||
                          (r3_end_below(C, sx, e[1], cx, c0) && r3_end_above(C, sx, e[0], cx, c0));
      if (!inside) continue;
      if (!r3_is_vertex(r3_cmask(a, cx, cy))) continue;
      if (n == R3_MAXI) return -1;
      if (out) out[n] = (u32)(cy * (a.W + 1) + cx);
      ++n;
    }
  }
  return n;
}

// events of the edge from P (its lower-id end) to Q, in order from P, with
// their coordinates, all in the double formulas (the emission's form: every
// event's position is needed there); the count, or -1 past R3_MAXE
SBMT_DEV int r3_edge_events_d(const R3Args& a, double2 P, double2 Q, R3Ev* ev) {
  int n = 0;
  const double dx = dsb(Q.x, P.x), dy = dsb(Q.y, P.y);
  const bool hz = dy == 0.0, vt = dx == 0.0;
  const double ylo = fmin(P.y, Q.y), yhi = fmax(P.y, Q.y), xlo = fmin(P.x, Q.x), xhi = fmax(P.x, Q.x);
  const i64 k0 = max((i64)0, r3_lo(ylo)), k1 = min((i64)a.H, r3_hi(yhi));
  for (i64 k = k0; k <= k1; ++k) {
    const double y0 = (double)k - 0.5;
    if (!(ylo < y0 && y0 < yhi)) continue;
    const double x = r3_hx(P, Q, y0);
    i64 j;
    const bool corner = r3_at_corner(x, &j);
    if (corner ? r3_corner_event(a, j, k, hz, vt) : r3_hb(a, j, k)) {
      if (n == R3_MAXE) return -1;
      ev[n++] = R3Ev{x, y0, 0.0, corner ? 2 : 0, (int)j, (int)k};
    }
  }
  const i64 m0 = max((i64)0, r3_lo(xlo)), m1 = min((i64)a.W, r3_hi(xhi));
  for (i64 m = m0; m <= m1; ++m) {
    const double x0 = (double)m - 0.5;
    if (!(xlo < x0 && x0 < xhi)) continue;
    const double y = r3_vy(P, Q, x0);
    i64 j;
    const bool corner = r3_at_corner(y, &j);
    if (corner) {
      bool dup = false;
      for (int t = 0; t < n; ++t)
        if (ev[t].kind == 2 && ev[t].m == (int)m && ev[t].k == (int)j) dup = true;
      if (dup || !r3_corner_event(a, m, j, hz, vt)) continue;
    } else if (!r3_vb(a, m, j)) {
      continue;
    }
    if (n == R3_MAXE) return -1;
    ev[n++] = R3Ev{x0, y, 0.0, corner ? 2 : 1, (int)m, (int)j};
  }
  const bool alongx = fabs(dx) >= fabs(dy);
  for (int t = 0; t < n; ++t) ev[t].s = alongx ? ddv(dsb(ev[t].x, P.x), dx) : ddv(dsb(ev[t].y, P.y), dy);
  // insertion sort by (s, kind, k, m)
  for (int t = 1; t < n; ++t) {
    const R3Ev e = ev[t];
    int u = t - 1;
    while (u >= 0) {
      const R3Ev& f = ev[u];
      const bool gt = f.s != e.s ? f.s > e.s : f.kind != e.kind ? f.kind > e.kind : f.k != e.k ? f.k > e.k : f.m > e.m;
      if (!gt) break;
      ev[u + 1] = f;
      --u;
    }
    ev[u + 1] = e;
  }
  return n;
}

// the boundary vertices strictly inside the cell, as corner ids y (W+1) + x
// in id order, in the double formulas (the emission's form); the count, or
// -1 past R3_MAXI (ids written when out != null)
SBMT_DEV int r3_inside_d(const R3Args& a, const R3Cell& C, u32* out) {
  int n = 0;
  const i64 cy0 = max((i64)0, r3_lo(C.ylo)), cy1 = min((i64)a.H, r3_hi(C.yhi));
  const i64 cx0 = max((i64)0, r3_lo(C.xlo)), cx1 = min((i64)a.W, r3_hi(C.xhi));
  for (i64 cy = cy0; cy <= cy1; ++cy) {
    const double y0 = (double)cy - 0.5;
    if (!(C.ylo < y0 && y0 < C.yhi)) continue;
    double pos[2];
    int src[2];
    if (r3_chord(C.K, C.id, false, y0, pos, src) != 2) return -2;
    for (i64 cx = cx0; cx <= cx1; ++cx) {
      const double x0 = (double)cx - 0.5;
      if (!(pos[0] < x0 && x0 < pos[1])) continue;
      if (!r3_is_vertex(r3_cmask(a, cx, cy))) continue;
      if (n == R3_MAXI) return -1;
      if (out) out[n] = (u32)(cy * (a.W + 1) + cx);
      ++n;
    }
  }
  return n;
}

// the other cell beside the cell's edge j (-1 on the mesh's outer boundary;
// -2 when more than one other cell has the edge)
SBMT_DEV int r3_neighbour(const R3Args& a, u32 c, const R3Cell& C, int j) {
  const int u = C.id[j], w = C.id[j == 2 ? 0 : j + 1];
  int found = -1;
  for (u32 e = a.vptr[u]; e < a.vptr[u + 1]; ++e) {
    const u32 c2 = a.inc[e];
    if (c2 == c) continue;
    const int* t = a.ttri + 3 * (u64)c2;
    if (t[0] == w || t[1] == w || t[2] == w) {
      if (found >= 0) return -2;
      found = (int)c2;
    }
  }
  return found;
}

// the local edge of cell c2 running between vertices u and w
SBMT_DEV int r3_edge_in(const R3Args& a, u32 c2, int u, int w) {
  const int* t = a.ttri + 3 * (u64)c2;
  for (int j = 0; j < 3; ++j) {
    const int p = t[j], q = t[j == 2 ? 0 : j + 1];
    if ((p == u && q == w) || (p == w && q == u)) return j;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// cells around each vertex (CSR): counts, then the lists
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_r3_deg(R3Args a) {
  for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < a.nt; c += (u64)gridDim.x * blockDim.x)
    for (int q = 0; q < 3; ++q) {
      const int v = a.ttri[3 * c + q];
      if (v < 0 || (u64)v >= a.nv) {
        atomicOr(a.err, R3_GEOMETRY);
        continue;
      }
      atomicAdd(a.deg + v, 1u);
    }
}
__global__ void __launch_bounds__(256) k_r3_fill(R3Args a) {
  for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < a.nt; c += (u64)gridDim.x * blockDim.x)
    for (int q = 0; q < 3; ++q) {
      const int v = a.ttri[3 * c + q];
      if (v < 0 || (u64)v >= a.nv) continue;
      const u32 slot = atomicSub(a.deg + v, 1u) - 1u;
      a.inc[a.vptr[v] + slot] = (u32)c;
    }
}

// ---------------------------------------------------------------------------
// screen: every cell; a cell whose pixel box carries one label is uncut (its
// label is the box's); the others go to the candidate list
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_r3_screen(R3Args a) {
  const int lane = threadIdx.x & 31;
  for (u64 c0 = (u64)blockIdx.x * blockDim.x; c0 < a.nt; c0 += (u64)gridDim.x * blockDim.x) {
    const u64 c = c0 + threadIdx.x;
    bool cand = false;
    if (c < a.nt) {
      const int* t = a.ttri + 3 * c;
      double2 K[3];
      i64 X[3], Y[3];
      for (int q = 0; q < 3; ++q) {
        K[q] = reinterpret_cast<const double2*>(a.txy)[t[q]];
        bool ix, iy;
        X[q] = r3_fix36(K[q].x, &ix), Y[q] = r3_fix36(K[q].y, &iy);
      }
      int l = -1;
      if (!r3_ccw(K, X, Y)) atomicOr(a.err, R3_GEOMETRY);
      else l = r3_uniform(a, X, Y);
      cand = l < 0;
      a.ntri[c] = 1, a.nown[c] = 0, a.nin[c] = 0, a.own3[c] = 0;
      a.ulab[c] = (unsigned short)(cand ? 0 : l);
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
    // a warp's 32 cells fill one word of the candidate bit-plane
    const u64 w0 = c0 + (threadIdx.x & ~31u);
    if (lane == 0 && w0 < a.nt) a.cmark[w0 >> 5] = m;
    if (m) {
      u32 base = 0;
      if (lane == 0) base = atomicAdd(a.ncand, (u32)__popc(m));
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (cand) a.cand[base + __popc(m & ((1u << lane) - 1u))] = (u32)c;
    }
  }
}

// the candidates: events on the edges, inside vertices, the cells beside
// the edges that carry events
__global__ void __launch_bounds__(128) k_r3_count(R3Args a) {
  R3Ev ev[R3_MAXE];
  const u32 n = *a.ncand;
  for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const u32 c = a.cand[q];
    const R3Cell C = r3_load_k(a, c);
    int ne = 0, cnt[3];
    bool bad = false;
    for (int j = 0; j < 3; ++j) {
      const int u = j, w = j == 2 ? 0 : j + 1;
      const bool fwd = C.id[u] < C.id[w];
      cnt[j] = r3_edge_count(a, fwd ? C.K[u] : C.K[w], fwd ? C.K[w] : C.K[u], ev);
      if (cnt[j] < 0) bad = true;
      else ne += cnt[j];
    }
    const int ni = bad ? 0 : r3_inside(a, C, nullptr);
    if (bad || ni == -1 || 3 + ne + ni > R3_MAXN) {
      atomicOr(a.err, R3_CAPACITY);
    } else if (ni < 0) {
      atomicOr(a.err, R3_GEOMETRY);
    } else if (ne + ni > 0) {
      // the cut cells' list for the emission, one atomic per group of lanes
      const unsigned act = __activemask();
      const int lane = threadIdx.x & 31, lead = __ffs(act) - 1;
      u32 base = 0;
      if (lane == lead) base = atomicAdd(a.ncut, (u32)__popc(act));
      base = __shfl_sync(act, base, lead);
      a.cutl[base + __popc(act & ((1u << lane) - 1u))] = c;
      u32 nown = 0, own3 = 0;
      for (int j = 0; j < 3; ++j) {
        if (cnt[j] == 0) continue;
        const int nb = r3_neighbour(a, c, C, j);
        if (nb == -2) atomicOr(a.err, R3_GEOMETRY);
        if (nb < 0 || (u32)nb > c) nown += (u32)cnt[j], own3 |= (u32)cnt[j] << (8 * j);
      }
      a.ntri[c] = (u32)(2 * ni + 3 + ne - 2), a.nin[c] = (u32)ni, a.nown[c] = nown, a.own3[c] = own3;
    }
  }
}

// ---------------------------------------------------------------------------
// the local boundary graph of a cut cell
// ---------------------------------------------------------------------------
struct R3Local {
  int nev[3], ne, ni, n, np;
  double2 v[R3_MAXN];
  u32 gid[R3_MAXN];
  unsigned char on_edge[R3_MAXN];
  unsigned char pa[R3_MAXP], pb[R3_MAXP];
  int mask, klass;
};

// the global id of an event base: the first event id of cell c's edge j
SBMT_DEV u32 r3_edge_base(const R3Args& a, u32 c, int j) {
  const u32 o = a.own3[c];
  u32 b = a.nv + a.eoff[c];
  for (int t = 0; t < j; ++t) b += (o >> (8 * t)) & 255u;
  return b;
}

// builds L for cut cell c; writes the coordinates of the events of the edges
// c owns and of its inside vertices when write is set; 0, or an R3_ error
template <typename EvBuf>
SBMT_DEV u32 r3_build(const R3Args& a, u32 c, const R3Cell& C, R3Local& L, EvBuf& ev, bool write) {
  L.ne = 0;
  L.n = 3;
  for (int q = 0; q < 3; ++q) {
    L.v[q] = C.K[q], L.gid[q] = (u32)C.id[q];
    L.on_edge[q] = (unsigned char)((1 << q) | (1 << (q == 0 ? 2 : q - 1)));
  }
  // events per edge, in counter-clockwise order along the cell's edge j
  for (int j = 0; j < 3; ++j) {
    const int u = j, w = j == 2 ? 0 : j + 1;
    const bool fwd = C.id[u] < C.id[w];
    R3Ev* e = ev[j];
    const int n = r3_edge_events_d(a, fwd ? C.K[u] : C.K[w], fwd ? C.K[w] : C.K[u], e);
    if (n < 0 || L.n + n > R3_MAXN) return R3_CAPACITY;
    L.nev[j] = n;
    if (n == 0) continue;
    const int nb = r3_neighbour(a, c, C, j);
    if (nb == -2) return R3_GEOMETRY;
    u32 base;
    if (nb < 0 || (u32)nb > c) {
      base = r3_edge_base(a, c, j);
      if (write)
        for (int t = 0; t < n; ++t) reinterpret_cast<double2*>(a.xy)[base + t] = make_double2(e[t].x, e[t].y);
    } else {
      const int j2 = r3_edge_in(a, (u32)nb, C.id[u], C.id[w]);
      if (j2 < 0) return R3_GEOMETRY;
      base = r3_edge_base(a, (u32)nb, j2);
    }
    if (!fwd)  // counter-clockwise along j runs from the higher-id end
      for (int t = 0; t < n / 2; ++t) {
        const R3Ev x = e[t];
        e[t] = e[n - 1 - t], e[n - 1 - t] = x;
      }
    for (int t = 0; t < n; ++t) {
      L.v[L.n] = make_double2(e[t].x, e[t].y);
      L.gid[L.n] = base + (fwd ? (u32)t : (u32)(n - 1 - t));
      L.on_edge[L.n] = (unsigned char)(1 << j);
      ++L.n;
    }
    L.ne += n;
  }
  // inside vertices
  u32 ins[R3_MAXI];
  const int ni = r3_inside_d(a, C, ins);
  if (ni == -1 || L.n + ni > R3_MAXN) return R3_CAPACITY;
  if (ni < 0) return R3_GEOMETRY;
  L.ni = ni;
  const u32 ibase = a.nv + a.ne_total + a.ioff[c];
  for (int t = 0; t < ni; ++t) {
    const u32 cid = ins[t];
    const double2 p = make_double2((double)(cid % (u32)(a.W + 1)) - 0.5, (double)(cid / (u32)(a.W + 1)) - 0.5);
    L.v[L.n] = p, L.gid[L.n] = ibase + (u32)t, L.on_edge[L.n] = 0;
    if (write) reinterpret_cast<double2*>(a.xy)[ibase + t] = p;
    ++L.n;
  }
  // pieces: horizontal lines by y, then vertical lines by x, each along the
  // line; oriented with the lower label on the left
  L.np = 0;
  for (int vert = 0; vert < 2; ++vert) {
    const double lo = vert ? C.xlo : C.ylo, hi = vert ? C.xhi : C.yhi;
    const i64 L0 = max((i64)0, r3_lo(lo)), L1 = min((i64)(vert ? a.W : a.H), r3_hi(hi));
    for (i64 line = L0; line <= L1; ++line) {
      const double c0 = (double)line - 0.5;
      if (!(lo < c0 && c0 < hi)) continue;
      double pos[2];
      int src[2];
      if (r3_chord(C.K, C.id, vert, c0, pos, src) != 2) return R3_GEOMETRY;
      // nodes on the line: the chord ends that are nodes, the inside vertices
      int nd[R3_MAXI + 2];
      double np_[R3_MAXI + 2];
      int nn = 0;
      for (int end = 0; end < 2; ++end) {
        int node = -1;
        if (src[end] < 3) {
          node = src[end];
        } else {
          const int j = src[end] - 3;
          int b = 3;
          for (int t = 0; t < j; ++t) b += L.nev[t];
          for (int t = 0; t < L.nev[j]; ++t) {
            const R3Ev& e = ev[j][t];
            const bool hit = e.kind == 2 ? (vert ? e.m == line : e.k == line)
                                         : (e.kind == (vert ? 1 : 0) && (vert ? e.m : e.k) == line);
            if (hit) {
              node = b + t;
              break;
            }
          }
        }
        if (end == 1) {
          for (int t = 0; t < ni; ++t) {
            const u32 cid = ins[t];
            const i64 cx = cid % (u32)(a.W + 1), cy = cid / (u32)(a.W + 1);
            if ((vert ? cx : cy) == line)
              nd[nn] = 3 + L.ne + t, np_[nn++] = vert ? (double)cy - 0.5 : (double)cx - 0.5;
          }
        }
        if (node >= 0) nd[nn] = node, np_[nn++] = pos[end];
      }
      for (int t = 0; t + 1 < nn; ++t) {
        const double mid = dml(dad(np_[t], np_[t + 1]), 0.5);
        i64 j;
        r3_at_corner(mid, &j);  // at a corner: the pixel edge starting there
        int l0, l1;
        bool fwd;
        if (!vert) {
          if (!r3_hb(a, j, line)) continue;
          l0 = r3_px(a, j, line - 1), l1 = r3_px(a, j, line);
          fwd = l1 < l0;  // going +x the left side is above
        } else {
          if (!r3_vb(a, line, j)) continue;
          l0 = r3_px(a, line - 1, j), l1 = r3_px(a, line, j);
          fwd = l0 < l1;  // going +y the left side is -x
        }
        if (L.np == R3_MAXP) return R3_CAPACITY;
        L.pa[L.np] = (unsigned char)(fwd ? nd[t] : nd[t + 1]);
        L.pb[L.np] = (unsigned char)(fwd ? nd[t + 1] : nd[t]);
        ++L.np;
      }
    }
  }
  // Alg. 1 mask (a corner on a piece sets both its edges, an event its
  // edge, an edge on a boundary run its own bit, bit 0 an inside vertex) and
  // the (m, n) class of the first two pieces
  auto bits = [&](int w) -> int {
    if (w < 3) return (2 << w) | (2 << (w == 0 ? 2 : w - 1));
    if (w < 3 + L.ne) {
      int k = w - 3;
      for (int j = 0; j < 3; ++j) {
        if (k < L.nev[j]) return 2 << j;
        k -= L.nev[j];
      }
    }
    return 0;
  };
  int mask = L.ni > 0 ? 1 : 0, pc0 = 0, pc1 = 0;
  for (int t = 0; t < L.np; ++t) {
    const int b = bits(L.pa[t]) | bits(L.pb[t]);
    mask |= b;
    if (t == 0) pc0 = __popc(b);
    if (t == 1) pc1 = __popc(b);
  }
  for (int j = 0; j < 3; ++j) {
    const double2 p = C.K[j], q = C.K[j == 2 ? 0 : j + 1];
    for (int vert = 0; vert < 2; ++vert) {
      const double ca = vert ? p.x : p.y, cb = vert ? q.x : q.y;
      i64 line;
      if (ca != cb || !r3_at_corner(ca, &line)) continue;
      const double ta = vert ? p.y : p.x, tb = vert ? q.y : q.x;
      const double t0 = fmin(ta, tb), t1 = fmax(ta, tb);
      for (i64 g = r3_lo(t0) - 1; g <= r3_hi(t1) + 1; ++g) {
        if (!((double)g + 0.5 > t0 && (double)g - 0.5 < t1)) continue;
        if (vert ? r3_vb(a, line, g) : r3_hb(a, g, line)) mask |= 2 << j;
      }
    }
  }
  L.mask = mask;
  L.klass = L.np == 1 ? thm32_class(0, pc0) : L.np == 2 ? thm32_class(pc0, pc1) : 0;
  return 0;
}

// the label of the pixel holding ((x1 + x2) + x3) / 3
SBMT_DEV unsigned short r3_label(const R3Args& a, double2 p, double2 q, double2 r) {
  const double cx = ddv(dad(dad(p.x, q.x), r.x), 3.0), cy = ddv(dad(dad(p.y, q.y), r.y), 3.0);
  const int l = r3_px(a, (i64)floor(dad(cx, 0.5)), (i64)floor(dad(cy, 0.5)));
  return l == R3_OUTSIDE ? (unsigned short)0xFFFF : (unsigned short)l;
}

// Tier-T: the key and rotation of the cell in the table's regime, or key 0
SBMT_DEV int r3_tier_t(const R3Local& L, int* sigma_out) {
  if (L.ni > 1) return 0;
  int deg[R3_MAXN];
  for (int w = 0; w < L.n; ++w) deg[w] = 0;
  for (int t = 0; t < L.np; ++t) {
    if (L.pa[t] < 3 || L.pb[t] < 3) return 0;
    deg[L.pa[t]]++, deg[L.pb[t]]++;
  }
  for (int w = 3; w < 3 + L.ne; ++w)
    if (deg[w] != 1) return 0;
  const int P = 3 + L.ne;
  if (L.ni == 0 && !(L.np == 1 || L.np == 2)) return 0;
  if (L.ni == 1)
    for (int t = 0; t < L.np; ++t)
      if (L.pa[t] != P && L.pb[t] != P) return 0;
  auto edge_of = [&](int w) -> int {
    int k = w - 3;
    for (int j = 0; j < 3; ++j) {
      if (k < L.nev[j]) return j;
      k -= L.nev[j];
    }
    return -1;
  };
  int dir = 0;
  if (L.ni == 0 && L.np == 2) {
    int X[2];
    for (int c = 0; c < 2; ++c) {
      const int ea = edge_of(L.pa[c]), eb = edge_of(L.pb[c]);
      if (ea == eb) return -1;  // a chord with both ends on one edge
      X[c] = eb == (ea + 1) % 3 ? eb : ea;
    }
    if (X[0] == X[1]) {  // nested chords at corner X
      const int ein = (X[0] + 2) % 3, eout = X[0];
      int near = -1, best = -1;
      for (int c = 0; c < 2; ++c)
        for (int end = 0; end < 2; ++end) {
          const int w = end ? L.pb[c] : L.pa[c];
          if (edge_of(w) == ein && w > best) best = w, near = c;
        }
      dir = (edge_of(L.pa[near]) == ein && edge_of(L.pb[near]) == eout) ? 1 : 0;
    }
  }
  const int st = L.ni == 1 ? 1 : 0, n0 = L.nev[0], n1 = L.nev[1], n2 = L.nev[2];
  const int cr0 = (st << 10) | (n0 << 7) | (n1 << 4) | (n2 << 1) | dir;
  const int cr1 = (st << 10) | (n1 << 7) | (n2 << 4) | (n0 << 1) | dir;
  const int cr2 = (st << 10) | (n2 << 7) | (n0 << 4) | (n1 << 1) | dir;
  int best = cr0, sigma = 0;
  if (cr1 < best) best = cr1, sigma = 1;
  if (cr2 < best) best = cr2, sigma = 2;
  for (int k = 0; k < NKEYS; ++k)
    if (g_keys.code[k] == best) {
      *sigma_out = sigma;
      return k + 1;
    }
  return -1;
}

// ---------------------------------------------------------------------------
// the greedy rule for a small cell (n <= R3_SMALL nodes) in one thread:
// candidate pairs by (squared length rounded to single precision, u, w),
// each kept when its open segment holds no node and it crosses no kept edge;
// the faces (3-cycles with no node inside, smallest index first,
// counter-clockwise) in sorted order.  Returns the face count, -1 past the
// limits.
// ---------------------------------------------------------------------------
constexpr int R3_SMALL = 12;

// Orientation signs with a single-precision filter.  The nodes' coordinates
// relative to the first corner, rounded once to float, are within
// 2^-24 M (1 + 2^-23) of the exact differences (M: the largest of them);
// a float orientation of three such points is then within 48 2^-24 M^2 of
// the exact orientation of the doubles, and the double-precision formula
// within 32 2^-53 M^2 of it.  Outside 80 2^-24 M^2 the float sign is the
// sign the double formula gives; inside it the double formula decides.
struct R3Filt {
  float2 l[R3_SMALL];
  float T;
};
SBMT_DEV void r3_filt_init(const R3Local& L, R3Filt& F) {
  float M = 0.0f;
  for (int k = 0; k < L.n; ++k) {
    F.l[k] = make_float2(__double2float_rn(dsb(L.v[k].x, L.v[0].x)), __double2float_rn(dsb(L.v[k].y, L.v[0].y)));
    M = fmaxf(M, fmaxf(fabsf(F.l[k].x), fabsf(F.l[k].y)));
  }
  F.T = 80.0f * 5.9604645e-8f * M * M * 1.0001f;  // 80 2^-24 M^2, rounded up
}
__device__ __noinline__ int r3_osgn_exact(const R3Local& L, int p, int q, int r) {
  return r3_sgn(r3_orient(L.v[p], L.v[q], L.v[r]));
}
SBMT_DEV int r3_osgn(const R3Local& L, const R3Filt& F, int p, int q, int r) {
  const float2 a = F.l[p], b = F.l[q], c = F.l[r];
  const float o = __fsub_rn(__fmul_rn(__fsub_rn(b.x, a.x), __fsub_rn(c.y, a.y)),
                            __fmul_rn(__fsub_rn(b.y, a.y), __fsub_rn(c.x, a.x)));
  if (o > F.T) return 1;
  if (o < -F.T) return -1;
  return r3_osgn_exact(L, p, q, r);  // within the filter's bound: the double formula
}

SBMT_DEV int r3_greedy_small(const R3Local& L, int* face) {
  const int n = L.n;
  R3Filt F;
  r3_filt_init(L, F);
  unsigned short adj[R3_SMALL];
  unsigned char ea[3 * R3_SMALL], eb[3 * R3_SMALL];
  int ne = 0;
  for (int w = 0; w < n; ++w) adj[w] = 0;
  auto add = [&](int p, int q) {
    if ((adj[p] >> q) & 1) return;
    adj[p] |= (unsigned short)(1 << q), adj[q] |= (unsigned short)(1 << p);
    if (ne < 3 * R3_SMALL) ea[ne] = (unsigned char)p, eb[ne] = (unsigned char)q;
    ++ne;
  };
  for (int t = 0; t < L.np; ++t) add(L.pa[t], L.pb[t]);
  {
    int prev = 0, b = 3;
    for (int j = 0; j < 3; ++j) {
      if (j) add(prev, j), prev = j;
      for (int t = 0; t < L.nev[j]; ++t) add(prev, b + t), prev = b + t;
      b += L.nev[j];
    }
    add(prev, 0);
  }
  // candidates, insertion-sorted by (key, u, w)
  float key[R3_SMALL * (R3_SMALL - 1) / 2];
  unsigned char pr[R3_SMALL * (R3_SMALL - 1) / 2];
  int nc = 0;
  for (int u = 0; u < n; ++u)
    for (int w = u + 1; w < n; ++w) {
      if (((adj[u] >> w) & 1) || (L.on_edge[u] & L.on_edge[w])) continue;
      const double dx = dsb(L.v[w].x, L.v[u].x), dy = dsb(L.v[w].y, L.v[u].y);
      const float k = __double2float_rn(dad(dml(dx, dx), dml(dy, dy)));
      const unsigned char code = (unsigned char)(u << 4 | w);
      int t = nc++;
      while (t > 0 && (key[t - 1] > k || (key[t - 1] == k && pr[t - 1] > code))) key[t] = key[t - 1], pr[t] = pr[t - 1], --t;
      key[t] = k, pr[t] = code;
    }
  for (int r = 0; r < nc; ++r) {
    const int u = pr[r] >> 4, w = pr[r] & 15;
    const double2 pu = L.v[u], pw = L.v[w];
    const double ex = dsb(pw.x, pu.x), ey = dsb(pw.y, pu.y), len2 = dad(dml(ex, ex), dml(ey, ey));
    bool bad = false;
    for (int k = 0; k < n && !bad; ++k) {
      if (k == u || k == w || r3_osgn(L, F, u, w, k) != 0) continue;
      const double t = dad(dml(dsb(L.v[k].x, pu.x), ex), dml(dsb(L.v[k].y, pu.y), ey));
      if (t > 0.0 && t < len2) bad = true;
    }
    for (int t = 0; t < ne && t < 3 * R3_SMALL && !bad; ++t) {
      const int p = ea[t], q = eb[t];
      if (p == u || p == w || q == u || q == w) continue;
      const int o1 = r3_osgn(L, F, u, w, p), o2 = r3_osgn(L, F, u, w, q);
      if (o1 * o2 >= 0) continue;
      const int o3 = r3_osgn(L, F, p, q, u), o4 = r3_osgn(L, F, p, q, w);
      if (o3 * o4 < 0) bad = true;
    }
    if (!bad) add(u, w);
  }
  if (ne > 3 * R3_SMALL) return -1;
  int nf = 0;
  for (int p = 0; p < n; ++p)
    for (int q = p + 1; q < n; ++q) {
      if (!((adj[p] >> q) & 1)) continue;
      for (int r = q + 1; r < n; ++r) {
        if (!((adj[p] >> r) & 1) || !((adj[q] >> r) & 1)) continue;
        const int o = r3_osgn(L, F, p, q, r);
        if (o == 0) continue;
        bool empty = true;
        for (int k = 0; k < n && empty; ++k) {
          if (k == p || k == q || k == r) continue;
          if (r3_osgn(L, F, p, q, k) == o && r3_osgn(L, F, q, r, k) == o && r3_osgn(L, F, r, p, k) == o)
            empty = false;
        }
        if (!empty) continue;
        if (nf == 2 * R3_SMALL) return -1;
        const int f = o > 0 ? (p << 12 | q << 6 | r) : (p << 12 | r << 6 | q);
        int t = nf++;
        while (t > 0 && face[t - 1] > f) face[t] = face[t - 1], --t;
        face[t] = f;
      }
    }
  return nf;
}

// ---------------------------------------------------------------------------
// the cells left as they are: uncut cells of one label, labelled by their
// pixel box, and candidates the boundary only touches (at a corner or along
// an edge), labelled by the pixel holding the centroid
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_r3_emit_uncut(R3Args a) {
  for (u64 c = (u64)blockIdx.x * blockDim.x + threadIdx.x; c < a.nt; c += (u64)gridDim.x * blockDim.x) {
    const u32 t0 = a.toff[c];
    if (a.toff[c + 1] - t0 != 1) continue;
    const int* t = a.ttri + 3 * c;
    const int3 tv = make_int3(t[0], t[1], t[2]);
    unsigned short lab;
    if ((a.cmark[c >> 5] >> (c & 31)) & 1u) {
      const double2* K = reinterpret_cast<const double2*>(a.txy);
      lab = r3_label(a, K[tv.x], K[tv.y], K[tv.z]);
    } else {
      lab = a.ulab[c];
    }
    reinterpret_cast<int3*>(a.tri)[t0] = tv;
    a.label[t0] = lab;
    a.code[t0] = 0;
  }
}

// ---------------------------------------------------------------------------
// the cut cells (k_r3_count's list): Tier-T cells take their template;
// Tier-G cells are queued (those over R3_SMALL nodes
// flagged) for the greedy kernels, so that this kernel's warps stay on the
// short template path and the greedy runs in warps of Tier-G cells only
// ---------------------------------------------------------------------------
constexpr u32 R3_BIG = 0x80000000u;  // a queued cell over R3_SMALL nodes (cell ids stay below 2^31)

struct R3EvBuf {
  R3Ev e[3][R3_MAXE];
  SBMT_DEV R3Ev* operator[](int j) { return e[j]; }
};

__global__ void __launch_bounds__(128) k_r3_emit(R3Args a) {
  R3EvBuf ev;
  R3Local L;
  const u32 n = *a.ncut;
  for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const u32 c = a.cutl[q];
    const R3Cell C = r3_load(a, c);
    const u32 t0 = a.toff[c];
    int3* tri = reinterpret_cast<int3*>(a.tri);
    const u32 e = r3_build(a, c, C, L, ev, true);
    if (e) {
      atomicOr(a.err, e);
      continue;
    }
    const int nt = 2 * L.ni + 3 + L.ne - 2;
    if ((u32)nt != a.toff[c + 1] - t0) {
      atomicOr(a.err, R3_COUNT);
      continue;
    }
    int sigma = 0;
    const int key = r3_tier_t(L, &sigma);
    if (key < 0) {
      atomicOr(a.err, R3_GEOMETRY);
      continue;
    }
    if (key == 0) {
      // one queue slot per lane, one atomic per group of lanes here
      const unsigned act = __activemask();
      const int lane = threadIdx.x & 31, lead = __ffs(act) - 1;
      u32 base = 0;
      if (lane == lead) base = atomicAdd(a.ng, (u32)__popc(act));
      base = __shfl_sync(act, base, lead);
      a.glist[base + __popc(act & ((1u << lane) - 1u))] = c | (L.n > R3_SMALL ? R3_BIG : 0u);
      continue;
    }
    const unsigned long long w = g_keys.tris[(key - 1) * 3 + sigma];
    const unsigned short code =
        (unsigned short)((L.mask & 15) | (sigma << 4) | (key << 6) | (L.klass << 12));
    for (int k = 0; k < nt; ++k) {
      int q3[3];
      for (int u = 0; u < 3; ++u) {
        const int l = tri_label(w, k, u);
        q3[u] = l == 7 ? 3 + L.ne : l;
      }
      tri[t0 + k] = make_int3((int)L.gid[q3[0]], (int)L.gid[q3[1]], (int)L.gid[q3[2]]);
      a.label[t0 + k] = r3_label(a, L.v[q3[0]], L.v[q3[1]], L.v[q3[2]]);
      a.code[t0 + k] = code;
    }
  }
}

// ---------------------------------------------------------------------------
// Tier-G cells of at most R3_SMALL nodes: one thread per queued cell, the
// local graph rebuilt (the event and inside-vertex coordinates are written
// by k_r3_emit), the greedy rule, the faces written in sorted order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_r3_gsmall(R3Args a) {
  R3EvBuf ev;
  R3Local L;
  const u32 n = *a.ng;
  for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const u32 c = a.glist[q];
    if (c & R3_BIG) continue;
    const R3Cell C = r3_load(a, c);
    const u32 e = r3_build(a, c, C, L, ev, false);
    if (e) {
      atomicOr(a.err, e);
      continue;
    }
    const u32 t0 = a.toff[c];
    int face[2 * R3_SMALL];
    const int nf = r3_greedy_small(L, face);
    if (nf != (int)(a.toff[c + 1] - t0)) {
      atomicOr(a.err, nf < 0 ? R3_CAPACITY : R3_COUNT);
      continue;
    }
    const unsigned short code = (unsigned short)((L.mask & 15) | (63 << 6) | (L.klass << 12));
    atomicAdd(a.ngtri, (u32)nf);
    atomicAdd(a.ngsmall, 1u);
    int3* tri = reinterpret_cast<int3*>(a.tri);
    for (int i = 0; i < nf; ++i) {
      const int f = face[i], p = f >> 12, r2 = (f >> 6) & 63, s2 = f & 63;
      tri[t0 + i] = make_int3((int)L.gid[p], (int)L.gid[r2], (int)L.gid[s2]);
      a.label[t0 + i] = r3_label(a, L.v[p], L.v[r2], L.v[s2]);
      a.code[t0 + i] = code;
    }
  }
}

// ---------------------------------------------------------------------------
// Tier-G: one warp per cell.  Lane 0 builds the cell's boundary graph in
// shared memory; the warp ranks the candidate pairs, runs the greedy pass
// (each candidate tested by the lanes against the nodes and the kept
// edges), lists the faces and writes them in sorted order.
// ---------------------------------------------------------------------------
constexpr int R3G_WARPS = 2;
constexpr int R3G_MAXC = R3_MAXN * (R3_MAXN - 1) / 2;
constexpr int R3G_MAXE = 3 * R3_MAXN;  // kept edges of a triangulation of n points
constexpr int R3G_MAXF = 2 * R3_MAXN;

struct R3GShared {
  R3Local L;
  R3Ev ev[3][R3_MAXE];
  float key[R3G_MAXC];
  unsigned short cand[R3G_MAXC], sorted[R3G_MAXC];
  unsigned long long adj[R3_MAXN];
  unsigned char ea[R3G_MAXE], eb[R3G_MAXE];
  int face[R3G_MAXF];
  int ncand, nedge, nface;
  u32 err;
};
struct R3SharedEv {
  R3Ev (*e)[R3_MAXE];
  SBMT_DEV R3Ev* operator[](int j) { return e[j]; }
};

__global__ void __launch_bounds__(32 * R3G_WARPS) k_r3_tierg(R3Args a) {
  __shared__ R3GShared sh[R3G_WARPS];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R3GShared& S = sh[wid];
  const u32 ng = *a.ng;
  for (u32 g = blockIdx.x * R3G_WARPS + wid; g < ng; g += gridDim.x * R3G_WARPS) {
    const u32 c = a.glist[g] & ~R3_BIG;
    if (!(a.glist[g] & R3_BIG)) continue;  // k_r3_gsmall's (the whole warp reads one entry)
    if (lane == 0) {
      const R3Cell C = r3_load(a, c);
      R3SharedEv ev{S.ev};
      S.err = r3_build(a, c, C, S.L, ev, false);
    }
    __syncwarp();
    if (S.err) {
      if (lane == 0) atomicOr(a.err, S.err);
      __syncwarp();
      continue;
    }
    const R3Local& L = S.L;
    const int n = L.n;
    // constraints: the cell's boundary cycle and the pieces
    if (lane == 0) {
      for (int w = 0; w < n; ++w) S.adj[w] = 0;
      S.nedge = 0;
      auto add = [&](int p, int q) {
        if ((S.adj[p] >> q) & 1ull) return;
        S.adj[p] |= 1ull << q, S.adj[q] |= 1ull << p;
        const int lo = p < q ? p : q, hi = p < q ? q : p;
        S.ea[S.nedge] = (unsigned char)lo, S.eb[S.nedge] = (unsigned char)hi;
        ++S.nedge;
      };
      for (int t = 0; t < L.np; ++t) add(L.pa[t], L.pb[t]);
      int cyc[R3_MAXN], nc = 0, b = 3;
      for (int j = 0; j < 3; ++j) {
        cyc[nc++] = j;
        for (int t = 0; t < L.nev[j]; ++t) cyc[nc++] = b + t;
        b += L.nev[j];
      }
      for (int t = 0; t < nc; ++t) add(cyc[t], cyc[t + 1 == nc ? 0 : t + 1]);
      S.ncand = 0;
    }
    __syncwarp();
    // candidate pairs, keyed by squared length rounded to single precision
    for (int p0 = 0; p0 < n * n; p0 += 32) {
      const int p = p0 + lane, u = p / n, w = p % n;
      bool ok = p < n * n && u < w && !((S.adj[u] >> w) & 1ull) && (L.on_edge[u] & L.on_edge[w]) == 0;
      const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
      int base = 0;
      if (lane == 0) base = S.ncand, S.ncand += __popc(m);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      if (ok) {
        const int slot = base + __popc(m & ((1u << lane) - 1u));
        const double dx = dsb(L.v[w].x, L.v[u].x), dy = dsb(L.v[w].y, L.v[u].y);
        S.key[slot] = __double2float_rn(dad(dml(dx, dx), dml(dy, dy)));
        S.cand[slot] = (unsigned short)(u * R3_MAXN + w);
      }
      __syncwarp();
    }
    const int ncand = S.ncand;
    // rank each candidate among all by (key, u, w)
    for (int i = lane; i < ncand; i += 32) {
      const float ki = S.key[i];
      const unsigned short ci = S.cand[i];
      int r = 0;
      for (int k = 0; k < ncand; ++k) {
        const float kk = S.key[k];
        r += (kk < ki || (kk == ki && S.cand[k] < ci)) ? 1 : 0;
      }
      S.sorted[r] = ci;
    }
    __syncwarp();
    // greedy pass
    for (int r = 0; r < ncand; ++r) {
      const int u = S.sorted[r] / R3_MAXN, w = S.sorted[r] % R3_MAXN;
      const double2 pu = L.v[u], pw = L.v[w];
      const double ex = dsb(pw.x, pu.x), ey = dsb(pw.y, pu.y), len2 = dad(dml(ex, ex), dml(ey, ey));
      bool bad = false;
      for (int k = lane; k < n; k += 32) {
        if (k == u || k == w || r3_orient(pu, pw, L.v[k]) != 0.0) continue;
        const double t = dad(dml(dsb(L.v[k].x, pu.x), ex), dml(dsb(L.v[k].y, pu.y), ey));
        if (t > 0.0 && t < len2) bad = true;
      }
      const int ne = min(S.nedge, R3G_MAXE);
      for (int t = lane; t < ne && !bad; t += 32) {
        const int p = S.ea[t], q = S.eb[t];
        if (p == u || p == w || q == u || q == w) continue;
        const int o1 = r3_sgn(r3_orient(pu, pw, L.v[p])), o2 = r3_sgn(r3_orient(pu, pw, L.v[q]));
        const int o3 = r3_sgn(r3_orient(L.v[p], L.v[q], pu)), o4 = r3_sgn(r3_orient(L.v[p], L.v[q], pw));
        if (o1 * o2 < 0 && o3 * o4 < 0) bad = true;
      }
      if (__any_sync(0xFFFFFFFFu, bad)) continue;
      if (lane == 0) {
        if (S.nedge < R3G_MAXE) {
          S.adj[u] |= 1ull << w, S.adj[w] |= 1ull << u;
          S.ea[S.nedge] = (unsigned char)u, S.eb[S.nedge] = (unsigned char)w;
        }
        ++S.nedge;
      }
      __syncwarp();
    }
    if (S.nedge > R3G_MAXE) {
      if (lane == 0) atomicOr(a.err, R3_CAPACITY);
      __syncwarp();
      continue;
    }
    // faces: 3-cycles with no node inside, smallest index first, CCW
    if (lane == 0) S.nface = 0;
    __syncwarp();
    for (int p = lane; p < n; p += 32) {
      unsigned long long mb = S.adj[p] & ~((2ull << p) - 1ull);
      while (mb) {
        const int q = __ffsll((long long)mb) - 1;
        mb &= mb - 1;
        unsigned long long mc = S.adj[p] & S.adj[q] & ~((2ull << q) - 1ull);
        while (mc) {
          const int r = __ffsll((long long)mc) - 1;
          mc &= mc - 1;
          const int o = r3_sgn(r3_orient(L.v[p], L.v[q], L.v[r]));
          if (o == 0) continue;
          bool empty = true;
          for (int k = 0; k < n && empty; ++k) {
            if (k == p || k == q || k == r) continue;
            if (r3_sgn(r3_orient(L.v[p], L.v[q], L.v[k])) == o && r3_sgn(r3_orient(L.v[q], L.v[r], L.v[k])) == o &&
                r3_sgn(r3_orient(L.v[r], L.v[p], L.v[k])) == o)
              empty = false;
          }
          if (!empty) continue;
          const int f = o > 0 ? (p << 12 | q << 6 | r) : (p << 12 | r << 6 | q);
          const int slot = atomicAdd(&S.nface, 1);
          if (slot < R3G_MAXF) S.face[slot] = f;
        }
      }
    }
    __syncwarp();
    const int nf = S.nface;
    const u32 t0 = a.toff[c];
    if (nf != (int)(a.toff[c + 1] - t0)) {
      if (lane == 0) atomicOr(a.err, R3_COUNT);
      __syncwarp();
      continue;
    }
    const unsigned short code = (unsigned short)((L.mask & 15) | (63 << 6) | (L.klass << 12));
    if (lane == 0) atomicAdd(a.ngtri, (u32)nf);
    int3* tri = reinterpret_cast<int3*>(a.tri);
    for (int i = lane; i < nf; i += 32) {
      const int f = S.face[i];
      int r = 0;
      for (int k = 0; k < nf; ++k) r += S.face[k] < f ? 1 : 0;
      const int p = f >> 12, q = (f >> 6) & 63, s = f & 63;
      tri[t0 + r] = make_int3((int)L.gid[p], (int)L.gid[q], (int)L.gid[s]);
      a.label[t0 + r] = r3_label(a, L.v[p], L.v[q], L.v[s]);
      a.code[t0 + r] = code;
    }
    __syncwarp();
  }
}

}  // namespace

int launch_r3_adjacency(const R3Args& a, u32* scr, cudaStream_t st) {
  const unsigned gc = (unsigned)std::min<u64>((a.nt + 255) / 256, 152 * 16);
  k_r3_deg<<<std::max(gc, 1u), 256, 0, st>>>(a);
  launch_scan(a.deg, 1, a.vptr, (u32)a.nv, scr, st);
  k_r3_fill<<<std::max(gc, 1u), 256, 0, st>>>(a);
  return 4;
}

int launch_r3_count(const R3Args& a, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<u64>((a.nt + 255) / 256, 152 * 16);
  k_r3_screen<<<std::max(g, 1u), 256, 0, st>>>(a);
  k_r3_count<<<152 * 16, 128, 0, st>>>(a);
  return 2;
}

int launch_r3_emit(const R3Args& a, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<u64>((a.nt + 255) / 256, 152 * 16);
  k_r3_emit_uncut<<<std::max(g, 1u), 256, 0, st>>>(a);
  k_r3_emit<<<152 * 16, 128, 0, st>>>(a);
  k_r3_gsmall<<<152 * 16, 128, 0, st>>>(a);
  k_r3_tierg<<<152 * 8, 32 * R3G_WARPS, 0, st>>>(a);
  return 4;
}

}  // namespace sbmt
