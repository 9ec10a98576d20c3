// k_project.cu -- projection of a scalar pixel field onto a finished mesh.
//
// Sec. 3.3 projects the bitmap's scalar fields onto every triangle; Sec. 3.6
// and App. C price that interpolation stage at constant work per triangle.
// Two outputs, each a pass over the mesh:
//
//  * per triangle T: the mean of the piecewise-constant pixel field over T,
//    (1/|T|) sum_p f_p |T n p|, pixel (x, y) the unit square centred at
//    (x, y).  One thread per triangle.  The overlap of T with pixel (c, r)
//    is A_r(x_{c+1}) - A_r(x_c), where A_r(t) is the area of T inside row
//    band r and left of the line x = t.  By Green's theorem with the form
//    (x - t) dy, which vanishes on both the band's horizontal lines and on
//    x = t, A_r(t) is a sum over T's three edges of the integral of
//    (x - t) dy along the part of the edge inside the band and left of t: a
//    closed form per edge, with no polygon clipping.  The arithmetic is
//    single precision in a frame at T's first vertex (float-float for the
//    few thin triangles, see COND_F32), and the mean is the weighted
//    sum divided by the sum of the weights (a convex combination).  A
//    triangle outside the image (its centroid outside the image rectangle)
//    gets 0.
//  * per vertex: the bilinear interpolation of the field between pixel
//    centres, the point clamped to [0, W-1] x [0, H-1].
//
// This part runs FP64 at a small fraction of its FP32 rate, so neither kernel
// has a double-precision instruction: every coordinate is split, with integer
// operations on its bits, into an integer and a fraction, and the frame
// offsets are formed from those, in float, or in float-float (hi + lo) for
// the thin triangles.
#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

// float-float numbers (hi + lo, about 48 significant bits) for the thin
// triangles, from error-free sums and FMA products (Dekker, Knuth)
struct DF {
  float hi, lo;
  SBMT_DEV DF(float h = 0.f, float l = 0.f) : hi(h), lo(l) {}
  SBMT_DEV explicit operator float() const { return hi + lo; }
};
SBMT_DEV DF quick_two_sum(float a, float b) {
  const float s = a + b;
  return DF(s, b - (s - a));
}
SBMT_DEV DF two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return DF(s, (a - (s - bb)) + (b - bb));
}
SBMT_DEV DF operator+(DF x, DF y) {
  DF s = two_sum(x.hi, y.hi);
  const DF t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
SBMT_DEV DF operator-(DF x) { return DF(-x.hi, -x.lo); }
SBMT_DEV DF operator-(DF x, DF y) { return x + (-y); }
SBMT_DEV DF operator*(DF x, DF y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return quick_two_sum(p, e);
}
SBMT_DEV DF operator/(DF x, DF y) {
  const float q1 = x.hi / y.hi;
  const DF r = x - y * DF(q1);
  const float q2 = r.hi / y.hi;
  const DF r2 = r - y * DF(q2);
  return quick_two_sum(q1, q2) + DF(r2.hi / y.hi);
}
SBMT_DEV bool operator<(DF x, DF y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
SBMT_DEV bool operator>(DF x, DF y) { return y < x; }
SBMT_DEV bool operator<=(DF x, DF y) { return !(y < x); }
SBMT_DEV bool operator==(DF x, DF y) { return x.hi == y.hi && x.lo == y.lo; }
SBMT_DEV DF fabs(DF x) { return x.hi < 0.f ? -x : x; }
// the float versions, so that one overload set serves both number types
SBMT_DEV float fabs(float x) { return fabsf(x); }
SBMT_DEV float fmin(float x, float y) { return fminf(x, y); }
SBMT_DEV float fmax(float x, float y) { return fmaxf(x, y); }
SBMT_DEV DF fmin(DF x, DF y) { return y < x ? y : x; }
SBMT_DEV DF fmax(DF x, DF y) { return x < y ? y : x; }
SBMT_DEV float quot(float a, float b) { return __fdividef(a, b); }
SBMT_DEV DF quot(DF a, DF b) { return a / b; }

// the part of edge p -> q with lo <= y <= hi, end points and whether it is
// there (a horizontal edge inside the band is kept whole: it bounds the
// band's polygon but adds nothing to the integrals)
template <typename R>
struct Sub {
  R px, py, qx, qy;
  bool in;
};
template <typename R>
SBMT_DEV Sub<R> band_part(R px, R py, R qx, R qy, R dy, R inv, R lo, R hi) {
  if (dy == R(0)) return Sub<R>{px, py, qx, qy, lo <= py && py <= hi};
  const R s0 = (lo - py) * inv, s1 = (hi - py) * inv;
  const R u0 = fmax(R(0), fmin(s0, s1)), u1 = fmin(R(1), fmax(s0, s1));
  if (u1 <= u0) return Sub<R>{px, py, px, py, false};
  const R dx = qx - px;
  return Sub<R>{px + u0 * dx, py + u0 * dy, px + u1 * dx, py + u1 * dy, true};
}

// One edge's part inside a row band, set up for the integral of
// min(x - t, 0) dy along it as a function of the column line x = t: with
// xmin <= xmax its ends' x, the whole part lies left of t when t >= xmax,
// giving (cx - t) dy with cx its mid x; otherwise only the part left of t
// counts, a triangle of height xmin - t (when negative) over a length
// (t - xmin) / (xmax - xmin) of the part: -(min(xmin - t, 0))^2 k with
// k = dy / (2 (xmax - xmin)).  A horizontal or absent part has dy = 0.
template <typename R>
struct Row {
  R xmin, xmax, cx, dy, k;
  SBMT_DEV R left(R t) const {
    const R n = fmin(xmin - t, R(0));
    return t < xmax ? -(n * n * k) : (cx - t) * dy;
  }
};
template <typename R>
SBMT_DEV Row<R> row_edge(const Sub<R>& e) {
  Row<R> g;
  g.xmin = fmin(e.px, e.qx), g.xmax = fmax(e.px, e.qx);
  g.cx = R(0.5f) * (e.px + e.qx);
  g.dy = e.in ? e.qy - e.py : R(0);
  g.k = quot(g.dy, R(2) * fmax(g.xmax - g.xmin, R(1e-30f)));
  return g;
}

// the weighted sum over the pixels (c0..c1) x (r0..r1), divided by the sum
// of the weights.  Coordinates are in the frame at the first vertex: the
// other two vertices (bx, by), (qx, qy), the left edge of pixel column c0 at
// X0 and the lower edge of pixel row r0 at Y0.  In each row band the area
// left of a column line is 0 before the band's polygon and the polygon's
// whole area after it; only the lines crossing the polygon are integrated.
template <typename R>
SBMT_DEV float tri_mean(R bx, R by, R qx, R qy, R X0, R Y0, int c0, int c1, int r0, int r1, const float* f,
                        i64 fpitch) {
  // the edges' rises and their reciprocals, once per triangle
  const R d0 = by, d1 = qy - by, d2 = -qy;
  const R i0 = d0 == R(0) ? R(0) : quot(R(1), d0), i1 = d1 == R(0) ? R(0) : quot(R(1), d1);
  const R i2 = d2 == R(0) ? R(0) : quot(R(1), d2);
  R s(0), tot(0);
  for (int r = r0; r <= r1; ++r) {
    const R lo = Y0 + R((float)(r - r0)), hi = lo + R(1);
    const Sub<R> e0 = band_part<R>(R(0), R(0), bx, by, d0, i0, lo, hi);
    const Sub<R> e1 = band_part<R>(bx, by, qx, qy, d1, i1, lo, hi);
    const Sub<R> e2 = band_part<R>(qx, qy, R(0), R(0), d2, i2, lo, hi);
    if (!(e0.in || e1.in || e2.in)) continue;
    R xlo(3e38f), xhi(-3e38f);
    if (e0.in) xlo = fmin(xlo, fmin(e0.px, e0.qx)), xhi = fmax(xhi, fmax(e0.px, e0.qx));
    if (e1.in) xlo = fmin(xlo, fmin(e1.px, e1.qx)), xhi = fmax(xhi, fmax(e1.px, e1.qx));
    if (e2.in) xlo = fmin(xlo, fmin(e2.px, e2.qx)), xhi = fmax(xhi, fmax(e2.px, e2.qx));
    const Row<R> g0 = row_edge(e0), g1 = row_edge(e1), g2 = row_edge(e2);
    // the polygon's area: the integral of x dy over its edges on the triangle
    const R whole = g0.cx * g0.dy + g1.cx * g1.dy + g2.cx * g2.dy;
    const float* row = reinterpret_cast<const float*>((const char*)f + r * fpitch);
    R prev(0);
    for (int cc = c0; cc <= c1; ++cc) {
      const R t = X0 + R((float)(cc + 1 - c0));
      R next;
      if (!(t < xhi)) {
        next = whole;
      } else if (t <= xlo) {
        next = R(0);
      } else {
        next = g0.left(t) + g1.left(t) + g2.left(t);
      }
      const R piece = next - prev;
      prev = next;
      s = s + piece * R(__ldg(row + cc));
      tot = tot + piece;
    }
  }
  return (float)tot != 0.f ? (float)(s / tot) : 0.f;
}

// x = X + d with X = trunc(x) and |d| < 1: the fraction's leading 48 bits
// (truncated) as hi + lo floats, from the bits of the double alone (no FP64
// instruction); |x| < 2^31, values below 2^-60 give 0
struct Split {
  int X;
  float d, e;  // d: the fraction to 24 bits; d + e: to 48 bits
};
SBMT_DEV Split split(double x) {
  const long long bits = __double_as_longlong(x);
  const unsigned long long ab = (unsigned long long)bits & 0x7FFFFFFFFFFFFFFFull;
  const int be = (int)(ab >> 52);
  if (be < 1023 - 60) return Split{0, 0.f, 0.f};
  const unsigned long long m = (ab & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;  // x = m 2^-sh
  const int sh = 1075 - be;
  const unsigned long long ip = sh < 64 ? m >> sh : 0ull;
  const unsigned long long fb = sh < 64 ? m & ((1ull << sh) - 1ull) : m;
  float d = 0.f, e = 0.f;
  if (fb) {
    const int lz = __clzll(fb);
    const unsigned long long top = (fb << lz) >> 16;  // 48 bits, the leading one at bit 47
    const int E = 63 - lz - sh;                        // the fraction is in [2^E, 2^(E+1))
    if (E >= -126) d = __int_as_float(((E + 127) << 23) | (int)((top >> 24) & 0x7FFFFFull));
    if (E - 47 >= -126) e = (float)(int)(top & 0xFFFFFFull) * __int_as_float((E - 47 + 127) << 23);
  }
  return bits < 0 ? Split{-(int)ip, -d, -e} : Split{(int)ip, d, e};
}

// a vertex split once by the vertex pass, read by the triangle pass (16 B)
struct SplitV {
  int X, Y;
  float dx, dy;
};

// pixel index floor(x + 1/2) of a split coordinate
SBMT_DEV int pixel_of(Split s) { return s.X + (int)floorf(s.d + 0.5f); }

// frame offsets u - a of split coordinates, in float and in float-float
SBMT_DEV float off_f(Split u, Split a) { return (float)(u.X - a.X) + (u.d - a.d); }
SBMT_DEV DF off_df(Split u, Split a) { return DF((float)(u.X - a.X)) + ((DF(u.d) + DF(u.e)) - (DF(a.d) + DF(a.e))); }

// Single precision loses about eps * L (L + 1) / |T| of the weights (L the
// longest edge): a triangle with L (L + 1) > (COND_F32 / 2) |T| and more
// than one pixel is queued and done in float-float at the end of its block,
// so that the few thin ones do not hold whole warps on the long path.  A
// block takes PT_ITER x 256 consecutive triangles, so its queue never
// overflows.
constexpr float COND_F32 = 128.f;
constexpr int PT_ITER = 8;
constexpr int QCAP = PT_ITER * 256;

__global__ void __launch_bounds__(256, 4) k_project_tri(const double* xy, const int* tri, const SplitV* sv, u64 T,
                                                        const float* f, i64 fpitch, int W, int H, float* out) {
  __shared__ u32 s_q[QCAP];
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (int it = 0; it < PT_ITER; ++it) {
    const u64 t = ((u64)blockIdx.x * PT_ITER + it) * blockDim.x + threadIdx.x;
    if (t >= T) break;
    const int4 va = __ldg(reinterpret_cast<const int4*>(sv) + tri[3 * t]);
    const int4 vb = __ldg(reinterpret_cast<const int4*>(sv) + tri[3 * t + 1]);
    const int4 vc = __ldg(reinterpret_cast<const int4*>(sv) + tri[3 * t + 2]);
    const Split ax{va.x, __int_as_float(va.z), 0.f}, ay{va.y, __int_as_float(va.w), 0.f};
    const Split bx{vb.x, __int_as_float(vb.z), 0.f}, by{vb.y, __int_as_float(vb.w), 0.f};
    const Split cx{vc.x, __int_as_float(vc.z), 0.f}, cy{vc.y, __int_as_float(vc.w), 0.f};
    // centroid inside the image rectangle: 3 x_c in (-3/2, 3W - 3/2), the
    // integer parts summed exactly, the fractions in float
    const int IX = ax.X + bx.X + cx.X, IY = ay.X + by.X + cy.X;
    const float FX = ax.d + bx.d + cx.d, FY = ay.d + by.d + cy.d;
    if (!(FX > (float)(-IX) - 1.5f && FX < (float)(3 * W - IX) - 1.5f && FY > (float)(-IY) - 1.5f &&
          FY < (float)(3 * H - IY) - 1.5f)) {
      out[t] = 0.f;
      continue;
    }
    const int pa = pixel_of(ax), pb = pixel_of(bx), pc = pixel_of(cx);
    const int qa = pixel_of(ay), qb = pixel_of(by), qc = pixel_of(cy);
    const int c0 = max(0, min(min(pa, pb), pc)), c1 = min(W - 1, max(max(pa, pb), pc));
    const int r0 = max(0, min(min(qa, qb), qc)), r1 = min(H - 1, max(max(qa, qb), qc));
    if (c0 == c1 && r0 == r1) {  // inside one pixel
      out[t] = __ldg(reinterpret_cast<const float*>((const char*)f + r0 * fpitch) + c0);
      continue;
    }
    const float ux = off_f(bx, ax), uy = off_f(by, ay), vx = off_f(cx, ax), vy = off_f(cy, ay);
    const float wx = vx - ux, wy = vy - uy;
    const float L = sqrtf(fmaxf(fmaxf(ux * ux + uy * uy, vx * vx + vy * vy), wx * wx + wy * wy));
    const float area2 = fabsf(ux * vy - uy * vx);
    if (L * (L + 1.f) * 2.f > COND_F32 * area2) {
      s_q[atomicAdd(&s_n, 1)] = (u32)t;  // T < 2^32 (checked by the launcher)
      continue;
    }
    const float X0 = (float)(c0 - ax.X) - 0.5f - ax.d, Y0 = (float)(r0 - ay.X) - 0.5f - ay.d;
    out[t] = tri_mean<float>(ux, uy, vx, vy, X0, Y0, c0, c1, r0, r1, f, fpitch);
  }
  __syncthreads();
  const int nq = s_n;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const u64 t = s_q[k];
    const double2 a = reinterpret_cast<const double2*>(xy)[tri[3 * t]];
    const double2 b = reinterpret_cast<const double2*>(xy)[tri[3 * t + 1]];
    const double2 c = reinterpret_cast<const double2*>(xy)[tri[3 * t + 2]];
    const Split ax = split(a.x), ay = split(a.y), bx = split(b.x), by = split(b.y), cx = split(c.x), cy = split(c.y);
    const int c0 = max(0, min(min(pixel_of(ax), pixel_of(bx)), pixel_of(cx)));
    const int c1 = min(W - 1, max(max(pixel_of(ax), pixel_of(bx)), pixel_of(cx)));
    const int r0 = max(0, min(min(pixel_of(ay), pixel_of(by)), pixel_of(cy)));
    const int r1 = min(H - 1, max(max(pixel_of(ay), pixel_of(by)), pixel_of(cy)));
    const DF X0 = DF((float)(c0 - ax.X)) - DF(0.5f) - (DF(ax.d) + DF(ax.e));
    const DF Y0 = DF((float)(r0 - ay.X)) - DF(0.5f) - (DF(ay.d) + DF(ay.e));
    out[t] = tri_mean<DF>(off_df(bx, ax), off_df(by, ay), off_df(cx, ax), off_df(cy, ay), X0, Y0, c0, c1, r0, r1, f,
                          fpitch);
  }
}

// the vertex pass: every vertex split once into sv (when given) and its
// bilinear value into out (when given)
__global__ void __launch_bounds__(256) k_project_vert(const double* xy, u64 V, const float* f, i64 fpitch, int W,
                                                      int H, float* out, SplitV* sv) {
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < V; k += (u64)gridDim.x * blockDim.x) {
    const double2 p = reinterpret_cast<const double2*>(xy)[k];
    // clamp x = X + d to [0, W - 1] with d in [0, 1): i0 = X, u = d
    Split sx = split(p.x), sy = split(p.y);
    if (sv) sv[k] = SplitV{sx.X, sy.X, sx.d, sy.d};
    if (!out) continue;
    if (sx.d < 0.f) sx.X -= 1, sx.d += 1.f;
    if (sy.d < 0.f) sy.X -= 1, sy.d += 1.f;
    if (sx.X < 0) sx.X = 0, sx.d = 0.f;
    if (sy.X < 0) sy.X = 0, sy.d = 0.f;
    if (sx.X >= W - 1) sx.X = W - 1, sx.d = 0.f;
    if (sy.X >= H - 1) sy.X = H - 1, sy.d = 0.f;
    const int i0 = sx.X, j0 = sy.X;
    const int i1 = min(i0 + 1, W - 1), j1 = min(j0 + 1, H - 1);
    const float u = sx.d, w = sy.d;
    const float* row0 = reinterpret_cast<const float*>((const char*)f + j0 * fpitch);
    const float* row1 = reinterpret_cast<const float*>((const char*)f + j1 * fpitch);
    const float f00 = __ldg(row0 + i0), f10 = __ldg(row0 + i1), f01 = __ldg(row1 + i0), f11 = __ldg(row1 + i1);
    out[k] = (1.f - w) * ((1.f - u) * f00 + u * f10) + w * ((1.f - u) * f01 + u * f11);
  }
}

}  // namespace

size_t project_scratch_bytes(u64 V) { return sizeof(SplitV) * (size_t)V; }

int launch_project(const double* xy, const int* tri, u64 T, u64 V, const float* f, i64 fpitch, int W, int H,
                   float* tri_value, float* vertex_value, void* scratch, cudaStream_t st) {
  if (T >= (1ull << 32)) return -1;
  int n = 0;
  SplitV* sv = tri_value && T ? (SplitV*)scratch : nullptr;
  if ((vertex_value || sv) && V) {
    const u64 blocks = std::min<u64>((V + 255) / 256, 152ull * 16);
    k_project_vert<<<(unsigned)blocks, 256, 0, st>>>(xy, V, f, fpitch, W, H, vertex_value, sv);
    ++n;
  }
  if (sv) {
    const u64 blocks = (T + QCAP - 1) / QCAP;
    k_project_tri<<<(unsigned)blocks, 256, 0, st>>>(xy, tri, sv, T, f, fpitch, W, H, tri_value);
    ++n;
  }
  return n;
}

}  // namespace sbmt
