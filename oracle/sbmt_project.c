/* Projection of a scalar pixel field onto a triangle mesh -- the oracle of
 * mesh_project (test infrastructure: only the tests, the smoke check and the
 * benchmark's CPU baseline use it).
 *
 * Sec. 3.3 projects the bitmap's scalar fields onto every triangle of the
 * mesh; the complexity analysis (Sec. 3.6 and App. C) prices that
 * interpolation stage at constant work per triangle.  Two projections are
 * written out here, each as its plain definition, in double precision:
 *
 *  - per triangle T, the mean of the piecewise-constant pixel field over T:
 *      value(T) = (1 / |T|) * sum over image pixels p of f_p * |T n p|,
 *    where pixel (x, y) is the unit square centred at (x, y) (Sec. 3.3).
 *    |T n p| is found by clipping T against the square's four half-planes
 *    (Sutherland-Hodgman) and taking the shoelace area of what is left.  A
 *    triangle outside the image meets no pixel and gets 0.
 *  - per vertex, the bilinear interpolation of the field between the four
 *    nearest pixel centres, the sample point clamped to [0, W-1] x [0, H-1]
 *    (the vertex values of a linear, barycentric interpolant).
 */
#include <math.h>
#include <stdint.h>

/* keep the part of polygon in[0..n) on one side of the line x = bound
 * (axis 0) or y = bound (axis 1): below it when below != 0, else above */
static int clip_half(const double* in, int n, double* out, int axis, double bound, int below) {
  int m = 0;
  for (int k = 0; k < n; ++k) {
    const double* p = in + 2 * k;
    const double* q = in + 2 * ((k + 1) % n);
    const double dp = below ? bound - p[axis] : p[axis] - bound;
    const double dq = below ? bound - q[axis] : q[axis] - bound;
    if (dp >= 0) {
      out[2 * m] = p[0], out[2 * m + 1] = p[1], ++m;
    }
    if ((dp >= 0) != (dq >= 0)) {
      const double t = dp / (dp - dq);
      out[2 * m] = p[0] + t * (q[0] - p[0]);
      out[2 * m + 1] = p[1] + t * (q[1] - p[1]);
      ++m;
    }
  }
  return m;
}

static double shoelace(const double* p, int n) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    const double* a = p + 2 * k;
    const double* b = p + 2 * ((k + 1) % n);
    s += a[0] * b[1] - a[1] * b[0];
  }
  return 0.5 * fabs(s);
}

/* |T n [x0, x1] x [y0, y1]| */
double sbmt_oracle_tri_box_area(const double* t, double x0, double x1, double y0, double y1) {
  double a[32], b[32];
  int n = 3;
  for (int k = 0; k < 6; ++k) a[k] = t[k];
  n = clip_half(a, n, b, 0, x0, 0);
  n = clip_half(b, n, a, 0, x1, 1);
  n = clip_half(a, n, b, 1, y0, 0);
  n = clip_half(b, n, a, 1, y1, 1);
  return n >= 3 ? shoelace(a, n) : 0.0;
}

void sbmt_oracle_project_triangles(const double* xy, const int32_t* tri, int64_t T, const float* f, int W, int H,
                                   double* out) {
  for (int64_t t = 0; t < T; ++t) {
    double v[6];
    for (int k = 0; k < 3; ++k) v[2 * k] = xy[2 * tri[3 * t + k]], v[2 * k + 1] = xy[2 * tri[3 * t + k] + 1];
    double xmin = v[0], xmax = v[0], ymin = v[1], ymax = v[1];
    for (int k = 1; k < 3; ++k) {
      xmin = fmin(xmin, v[2 * k]), xmax = fmax(xmax, v[2 * k]);
      ymin = fmin(ymin, v[2 * k + 1]), ymax = fmax(ymax, v[2 * k + 1]);
    }
    /* every pixel whose square meets the bounding box */
    long c0 = (long)floor(xmin + 0.5), c1 = (long)floor(xmax + 0.5);
    long r0 = (long)floor(ymin + 0.5), r1 = (long)floor(ymax + 0.5);
    if (c0 < 0) c0 = 0;
    if (r0 < 0) r0 = 0;
    if (c1 > W - 1) c1 = W - 1;
    if (r1 > H - 1) r1 = H - 1;
    /* areas are translation invariant: clip in a frame at the first vertex,
       so that rounding scales with the triangle's size, not its position */
    const double ox = v[0], oy = v[1];
    for (int k = 0; k < 3; ++k) v[2 * k] -= ox, v[2 * k + 1] -= oy;
    double s = 0.0;
    for (long r = r0; r <= r1; ++r)
      for (long c = c0; c <= c1; ++c)
        s += (double)f[r * (long)W + c] *
             sbmt_oracle_tri_box_area(v, (c - 0.5) - ox, (c + 0.5) - ox, (r - 0.5) - oy, (r + 0.5) - oy);
    const double area = shoelace(v, 3);
    out[t] = area > 0.0 ? s / area : 0.0;
  }
}

void sbmt_oracle_vertex_values(const double* xy, int64_t V, const float* f, int W, int H, double* out) {
  for (int64_t k = 0; k < V; ++k) {
    double x = xy[2 * k], y = xy[2 * k + 1];
    x = x < 0.0 ? 0.0 : (x > W - 1 ? W - 1 : x);
    y = y < 0.0 ? 0.0 : (y > H - 1 ? H - 1 : y);
    long i0 = (long)floor(x), j0 = (long)floor(y);
    long i1 = i0 + 1 < W ? i0 + 1 : W - 1, j1 = j0 + 1 < H ? j0 + 1 : H - 1;
    const double u = x - i0, w = y - j0;
    const double f00 = f[j0 * (long)W + i0], f10 = f[j0 * (long)W + i1];
    const double f01 = f[j1 * (long)W + i0], f11 = f[j1 * (long)W + i1];
    out[k] = (1 - w) * ((1 - u) * f00 + u * f10) + w * ((1 - u) * f01 + u * f11);
  }
}
