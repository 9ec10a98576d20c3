// sbmt_dev.cuh -- device-side definitions shared by the SBMT kernels.
//
// Geometry is exact.  With h = p/q and S = 6q, every point the method
// touches (grid vertices, pixel corners, boundary/grid-edge crossings) has
// coordinates (a + b*sqrt3)/S with integers a, b (Sec. 3.3 grid
// v(i,j) = o + h(i + j/2, (sqrt3/2) j); pixel corners at half-integers).  The
// kernels keep such numbers as Zq{a, b} in 64-bit integers and decide every
// predicate by an exact sign test; no tolerance is ever used.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define SBMT_DEV __device__ __forceinline__
#define SBMT_HD __host__ __device__ __forceinline__

namespace sbmt {

typedef long long i64;
typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u32 NONE = 0xFFFFFFFFu;
constexpr int OUTSIDE = 0x10000;  // label outside the image: above every pixel label
constexpr int CB_LOG = 10;        // base cells per cell bucket (2^10)
constexpr int EB_LOG = 11;        // grid-edge ids per event bucket (2^11)
constexpr int TIERG_TN = 9;      // Tier-G cells up to this many local vertices may run one thread each
constexpr int TIERG_WN = 16;     // Tier-G cells up to this many local vertices fit the warp path's small state
constexpr u32 OVER_CAP = 1024;   // ids of cells over the Tier-G vertex limit kept per mesh
constexpr u32 RANK_SMALL = 256;  // event buckets up to this size are ranked by one small block each

// device error bits (reported through mesh_query)
enum : u32 {
  ERR_TRAVERSAL = 1u,  // a segment left the cell set / inconsistent walk
  ERR_CAPACITY = 2u,   // a Tier-G cell exceeded the per-cell vertex limit (ids listed, OVER_CAP at most)
  ERR_COUNT = 4u,      // a patch did not have the expected triangle count
  ERR_SEGBUF = 8u,     // segment buffer too small (retried by the host)
  ERR_TIMEOUT = 16u,   // a bounded device wait ran out (reported as SBMT_ETIMEDOUT)
};

// ---------------------------------------------------------------------------
// exact numbers a + b*sqrt(3)
// ---------------------------------------------------------------------------
struct Zq {
  i64 a, b;
};
SBMT_HD Zq zq(i64 a, i64 b = 0) { return Zq{a, b}; }
SBMT_HD Zq operator+(Zq x, Zq y) { return Zq{x.a + y.a, x.b + y.b}; }
SBMT_HD Zq operator-(Zq x, Zq y) { return Zq{x.a - y.a, x.b - y.b}; }
SBMT_HD Zq operator*(Zq x, Zq y) { return Zq{x.a * y.a + 3 * x.b * y.b, x.a * y.b + x.b * y.a}; }
// sign of a + b sqrt3: when a and b disagree in sign compare a^2 with 3 b^2.
// The components of a cell-local determinant can reach ~1e15 (points on
// rational pixel lines against lattice rows at y ~ 3pj sqrt3), so large
// squares are taken in 128 bits; below 1.7e9 they fit in 64.
SBMT_HD int zsign(Zq v) {
  if (v.b == 0) return (v.a > 0) - (v.a < 0);
  if (v.a == 0) return (v.b > 0) - (v.b < 0);
  if ((v.a > 0) == (v.b > 0)) return v.a > 0 ? 1 : -1;
  const i64 aa = v.a < 0 ? -v.a : v.a, bb = v.b < 0 ? -v.b : v.b;
  bool a_wins;
  if (aa < 1700000000ll && bb < 1700000000ll) {
    a_wins = aa * aa > 3 * (bb * bb);
  } else {
    const __int128 l = (__int128)aa * aa, r = 3 * ((__int128)bb * bb);
    a_wins = l > r;
  }
  return a_wins ? (v.a > 0 ? 1 : -1) : (v.b > 0 ? 1 : -1);
}
SBMT_HD int zcmp(Zq x, Zq y) { return zsign(x - y); }
SBMT_HD double zdouble(Zq v) { return (double)v.a + (double)v.b * 1.7320508075688772935; }

// Conversions between 64-bit integers and float on the 32-bit path: this
// part runs 64-bit conversions at its double-precision rate, a small
// fraction of the single-precision one.  A value within 32 bits converts in
// one instruction; a larger one as two halves joined by an FMA (one more
// rounding).  floor_i64 takes the 32-bit path below 2e9.
SBMT_HD float i2f(i64 v) {
#ifdef __CUDA_ARCH__
  const int lo = (int)v;
  if ((i64)lo == v) return (float)lo;
  return fmaf((float)(int)(v >> 32), 4294967296.0f, (float)(unsigned)v);
#else
  return (float)v;
#endif
}
SBMT_HD i64 floor_i64(float x) {
#ifdef __CUDA_ARCH__
  if (fabsf(x) < 2.0e9f) return (i64)(int)floorf(x);
#endif
  return (i64)floorf(x);
}

// floor(a / d) for d > 0: a float estimate corrected exactly (|a / d| < 2^30)
SBMT_HD i64 ifloordiv(i64 a, i64 d) {
  i64 k = floor_i64(i2f(a) / i2f(d));
  while (k * d > a) --k;
  while ((k + 1) * d <= a) ++k;
  return k;
}

// floor(v / d) for d > 0, exact.  A single-precision estimate x of
// (a + b sqrt3) / d is off by at most 2.4e-7 (|a| + 2|b|) / d (rounding of
// the two conversions, the constant, the product, the sum and the quotient,
// each 2^-24 relative), and by at most 3.0e-7 (|a| + 2|b|) / d when a or b
// needs more than 32 bits (one more rounding in its conversion, i2f); when
// x is farther than 4e-7 (|a| + 2|b|) / d from an integer its floor is the
// answer, else the exact sign of v - k d decides.
SBMT_HD i64 zfloordiv(Zq v, i64 d) {
  const float fd = i2f(d);
  const float x = (i2f(v.a) + i2f(v.b) * 1.7320508f) / fd;
  i64 k = floor_i64(x);
  const float fr = x - i2f(k);
  const float tol = 4e-7f * (i2f(v.a < 0 ? -v.a : v.a) + 2.0f * i2f(v.b < 0 ? -v.b : v.b)) / fd + 1e-6f;
  if (fr > tol && fr < 1.0f - tol) return k;
  while (zsign(v - zq(k * d)) < 0) --k;
  while (zsign(v - zq((k + 1) * d)) >= 0) ++k;
  return k;
}

// 2-D point with exact coordinates (K-local points fit in 32 bits)
struct Pq {
  Zq x, y;
};
SBMT_HD int orient3(const Pq& p, const Pq& q, const Pq& r) {
  return zsign((q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x));
}

// ---------------------------------------------------------------------------
// records
// ---------------------------------------------------------------------------
// boundary segment: a maximal straight run of boundary pixel edges between
// two PSLG vertices, starting at its lower corner (cx, cy)
struct Seg {
  int cx, cy;
  u32 ldr;  // length | dir << 30 (0 = +x, 1 = +y) | rev << 31 (oriented -x / -y)
  u32 lab;  // label below/left | label above/right << 16 (0xFFFF = outside)
};
SBMT_HD int seg_len(const Seg& s) { return (int)(s.ldr & 0x3FFFFFFFu); }
SBMT_HD int seg_dir(const Seg& s) { return (int)((s.ldr >> 30) & 1u); }
SBMT_HD int seg_rev(const Seg& s) { return (int)(s.ldr >> 31); }

// a segment's visit of one base cell; ev_in / ev_out are the events where the
// walk (from the lower end, along +x / +y) enters / leaves the cell, NONE
// when the walk starts / ends inside it
struct Pair {
  u32 cell, seg, ev_in, ev_out;
};

// a crossing of a boundary segment with a grid edge; xa..yb are the exact
// global scaled coordinates, gid the vertex id once the registry is frozen
struct Event {
  u32 edge, seg, gid, pad;
  int xa, xb, ya, yb;
};

// one cut cell.  tri_off / chain_base: the cell's first output triangle and
// first inside vertex, stored for Tier-G cells at emission; between
// classification and emission a Tier-T record keeps in tri_off the pixel
// corner of its inside vertex P (NONE without one).
struct CutRec {
  u32 cell, pair_lo, npairs, code;  // code: bits 0-15 pattern code, bit 16 outside-regime
  u32 ntri, nchain, tri_off, chain_base;
};

// where emission writes: the compact format keeps the uncut cells as one
// label and one code per base cell, lists the cut cells' patches, and stores
// coordinates only for the vertices after the lattice (ids from xy0 up)
struct CompactOut {
  int on;                     // 0: explicit format (the other fields unused)
  u32 xy0;                    // id of the first vertex stored in xy
  unsigned short* cell_label;
  unsigned short* cell_code;
  u32* patch_cell;            // per cut cell (in cell order): its id
  u32* patch_off;             // per cut cell: its first patch triangle; then the total
  const u32* cut_scan;        // exclusive scan of the cut cells per bucket
};

// a Tier-T patch between classification and emission: the vertex ids of the
// cell's events in counter-clockwise order from A, and the label of each
// patch triangle
struct __align__(16) TStage {
  u32 ev[4];
  unsigned short lab[8];
};

// ---------------------------------------------------------------------------
// grid (Sec. 3.3): strip rows j, cells c = 2i (up) / 2i+1 (down) per row
// ---------------------------------------------------------------------------
struct GridP {
  int W, H;
  i64 p, q, S, ox, oy;  // h = p/q, S = 6q, origin scaled by S
  int j0, nrows;        // strip rows meeting the image rectangle
  int vj0, nvrows;      // lattice vertex rows used
  const i64* clo;       // per strip row: first cell index c
  const i64* chi;       // per strip row: last cell index c
  const i64* cbase;     // per strip row: id of its first cell
  const i64* vlo;       // per vertex row: first i
  const i64* vhi;
  const i64* vbase;     // per vertex row: id of its first vertex
  const int* lrow;      // per strip row: pixel row of up-cell / down-cell centroids
  i64 ncells, nverts;
};

SBMT_DEV u32 vid(const GridP& g, i64 i, i64 j) {
  int r = (int)(j - g.vj0);
  return (u32)(g.vbase[r] + (i - g.vlo[r]));
}
SBMT_DEV bool cell_in(const GridP& g, i64 c, i64 j) {
  if (j < g.j0 || j >= g.j0 + g.nrows) return false;
  int r = (int)(j - g.j0);
  return c >= g.clo[r] && c <= g.chi[r];
}
SBMT_DEV u32 cell_id(const GridP& g, i64 c, i64 j) {
  int r = (int)(j - g.j0);
  return (u32)(g.cbase[r] + (c - g.clo[r]));
}
// lattice indices of corners A, B, C of cell c in strip j; A is the corner
// with least (y, x), then counter-clockwise
SBMT_DEV void cell_corners(i64 c, i64 j, i64* ci, i64* cj) {
  i64 i = c >> 1;  // floor(c / 2)
  if ((c & 1) == 0) {
    ci[0] = i, cj[0] = j, ci[1] = i + 1, cj[1] = j, ci[2] = i, cj[2] = j + 1;
  } else {
    ci[0] = i + 1, cj[0] = j, ci[1] = i + 1, cj[1] = j + 1, ci[2] = i, cj[2] = j + 1;
  }
}
// grid-edge ids of the cell's edges AB, BC, CA: 3 * (lower endpoint id) + family
// (0 horizontal, 1 sixty degrees, 2 one hundred twenty degrees)
SBMT_DEV void cell_edges(const GridP& g, i64 c, i64 j, u32* e) {
  i64 i = c >> 1;
  if ((c & 1) == 0) {
    e[0] = 3u * vid(g, i, j) + 0u;
    e[1] = 3u * vid(g, i + 1, j) + 2u;
    e[2] = 3u * vid(g, i, j) + 1u;
  } else {
    e[0] = 3u * vid(g, i + 1, j) + 1u;
    e[1] = 3u * vid(g, i, j + 1) + 0u;
    e[2] = 3u * vid(g, i + 1, j) + 2u;
  }
}
// scaled coordinates of lattice vertex v(i, j)
SBMT_DEV Pq lattice_pt(const GridP& g, i64 i, i64 j) {
  return Pq{zq(g.ox + 3 * g.p * (2 * i + j)), zq(g.oy, 3 * g.p * j)};
}
SBMT_DEV Pq corner_pt(const GridP& g, i64 cx, i64 cy) {
  return Pq{zq(6 * g.q * cx - 3 * g.q), zq(6 * g.q * cy - 3 * g.q)};
}
// strip row holding a point of height y (never on a grid line)
SBMT_HD i64 strip_of(const GridP& g, Zq y) {
  // y_j = oy + 3 p j sqrt3
  i64 j = floor_i64((i2f(y.a - g.oy) + i2f(y.b) * 1.7320508f) / (3.0f * (float)g.p * 1.7320508f));
  while (zcmp(zq(g.oy, 3 * g.p * j), y) > 0) --j;
  while (zcmp(zq(g.oy, 3 * g.p * (j + 1)), y) <= 0) ++j;
  return j;
}

// image access with the OUTSIDE label beyond the border
template <typename T>
SBMT_DEV int pix(const unsigned char* img, i64 pitch, int W, int H, i64 x, i64 y) {
  if (x < 0 || y < 0 || x >= W || y >= H) return OUTSIDE;
  return (int)((const T*)(img + y * pitch))[x];
}

}  // namespace sbmt
