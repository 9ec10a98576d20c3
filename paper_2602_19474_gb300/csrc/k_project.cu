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
//    single precision in a frame at T's first vertex (double precision for
//    the few thin triangles, see COND_F32), and the mean is the weighted
//    sum divided by the sum of the weights (a convex combination).  A
//    triangle outside the image (its centroid outside the image rectangle)
//    gets 0.
//  * per vertex: the bilinear interpolation of the field between pixel
//    centres, the point clamped to [0, W-1] x [0, H-1].
#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

// integral of min(x - t, 0) dy along the segment p -> q, in the form
// dy * I with I the mean of min(., 0) over the segment's linear x - t
template <typename R>
SBMT_DEV R left_integral(R px, R py, R qx, R qy, R t) {
  const R a = px - t, b = qx - t, dy = qy - py;
  if (a <= R(0) && b <= R(0)) return R(0.5) * (a + b) * dy;
  if (a > R(0) && b > R(0)) return R(0);
  const R neg = a <= R(0) ? a : b;  // the end left of t; |b - a| >= |neg| > 0
  return -(neg * neg) / (R(2) * fabs(b - a)) * dy;
}

// the part of edge p -> q with lo <= y <= hi, as end points (equal when empty)
template <typename R>
struct Sub {
  R px, py, qx, qy;
};
template <typename R>
SBMT_DEV Sub<R> band_part(R px, R py, R qx, R qy, R lo, R hi) {
  const R dy = qy - py;
  Sub<R> s{px, py, px, py};
  if (dy == R(0)) return s;  // horizontal: no dy, no contribution
  const R inv = R(1) / dy;
  const R s0 = (lo - py) * inv, s1 = (hi - py) * inv;
  const R u0 = fmax(R(0), fmin(s0, s1)), u1 = fmin(R(1), fmax(s0, s1));
  if (u1 <= u0) return s;
  const R dx = qx - px;
  s.px = px + u0 * dx, s.py = py + u0 * dy;
  s.qx = px + u1 * dx, s.qy = py + u1 * dy;
  return s;
}

// the weighted sum over the pixels (c0..c1) x (r0..r1), divided by the sum
// of the weights, in the frame at vertex a
template <typename R>
SBMT_DEV float tri_mean(double2 a, double2 b, double2 c, int c0, int c1, int r0, int r1, const float* f,
                        i64 fpitch) {
  const R bx = (R)(b.x - a.x), by = (R)(b.y - a.y), qx = (R)(c.x - a.x), qy = (R)(c.y - a.y);
  const R X0 = (R)((c0 - 0.5) - a.x);
  R s = 0, tot = 0;
  for (int r = r0; r <= r1; ++r) {
    const R lo = (R)((r - 0.5) - a.y), hi = (R)((r + 0.5) - a.y);
    const Sub<R> e0 = band_part<R>(0, 0, bx, by, lo, hi);
    const Sub<R> e1 = band_part<R>(bx, by, qx, qy, lo, hi);
    const Sub<R> e2 = band_part<R>(qx, qy, 0, 0, lo, hi);
    auto A = [&](R x) {
      return left_integral<R>(e0.px, e0.py, e0.qx, e0.qy, x) + left_integral<R>(e1.px, e1.py, e1.qx, e1.qy, x) +
             left_integral<R>(e2.px, e2.py, e2.qx, e2.qy, x);
    };
    const float* row = reinterpret_cast<const float*>((const char*)f + r * fpitch);
    R prev = A(X0);
    for (int cc = c0; cc <= c1; ++cc) {
      const R next = A(X0 + (R)(cc + 1 - c0));
      const R piece = next - prev;
      prev = next;
      s += piece * (R)__ldg(row + cc);
      tot += piece;
    }
  }
  return tot != R(0) ? (float)(s / tot) : 0.f;
}

// Single precision loses about eps * L (L + 1) / |T| of the weights (L the
// longest edge): a triangle with L (L + 1) > (COND_F32 / 2) |T| and more
// than one pixel is queued and done in double precision at the end of its
// block, so that the few thin ones do not hold whole warps on the FP64 pipe.
constexpr float COND_F32 = 128.f;
constexpr int QCAP = 1024;

SBMT_DEV void pixel_range(double2 a, double2 b, double2 c, int W, int H, int& c0, int& c1, int& r0, int& r1) {
  c0 = max(0, (int)floor(fmin(fmin(a.x, b.x), c.x) + 0.5));
  c1 = min(W - 1, (int)floor(fmax(fmax(a.x, b.x), c.x) + 0.5));
  r0 = max(0, (int)floor(fmin(fmin(a.y, b.y), c.y) + 0.5));
  r1 = min(H - 1, (int)floor(fmax(fmax(a.y, b.y), c.y) + 0.5));
}

__global__ void __launch_bounds__(256) k_project_tri(const double* xy, const int* tri, u64 T, const float* f,
                                                     i64 fpitch, int W, int H, float* out) {
  __shared__ u32 s_q[QCAP];
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x) {
    const double2 a = reinterpret_cast<const double2*>(xy)[tri[3 * t]];
    const double2 b = reinterpret_cast<const double2*>(xy)[tri[3 * t + 1]];
    const double2 c = reinterpret_cast<const double2*>(xy)[tri[3 * t + 2]];
    const double cx = a.x + b.x + c.x, cy = a.y + b.y + c.y;
    if (cx <= -1.5 || cy <= -1.5 || cx >= 3.0 * W - 1.5 || cy >= 3.0 * H - 1.5) {
      out[t] = 0.f;  // outside the image rectangle
      continue;
    }
    int c0, c1, r0, r1;
    pixel_range(a, b, c, W, H, c0, c1, r0, r1);
    if (c0 == c1 && r0 == r1) {  // inside one pixel
      out[t] = __ldg(reinterpret_cast<const float*>((const char*)f + r0 * fpitch) + c0);
      continue;
    }
    const float ux = (float)(b.x - a.x), uy = (float)(b.y - a.y), vx = (float)(c.x - a.x), vy = (float)(c.y - a.y);
    const float wx = vx - ux, wy = vy - uy;
    const float L = sqrtf(fmaxf(fmaxf(ux * ux + uy * uy, vx * vx + vy * vy), wx * wx + wy * wy));
    const float area2 = fabsf(ux * vy - uy * vx);
    if (L * (L + 1.f) * 2.f > COND_F32 * area2) {
      const int slot = atomicAdd(&s_n, 1);
      if (slot < QCAP) {
        s_q[slot] = (u32)t;  // T < 2^32 (checked by the launcher)
        continue;
      }
      out[t] = tri_mean<double>(a, b, c, c0, c1, r0, r1, f, fpitch);
      continue;
    }
    out[t] = tri_mean<float>(a, b, c, c0, c1, r0, r1, f, fpitch);
  }
  __syncthreads();
  const int nq = min(s_n, QCAP);
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    const u64 t = s_q[k];
    const double2 a = reinterpret_cast<const double2*>(xy)[tri[3 * t]];
    const double2 b = reinterpret_cast<const double2*>(xy)[tri[3 * t + 1]];
    const double2 c = reinterpret_cast<const double2*>(xy)[tri[3 * t + 2]];
    int c0, c1, r0, r1;
    pixel_range(a, b, c, W, H, c0, c1, r0, r1);
    out[t] = tri_mean<double>(a, b, c, c0, c1, r0, r1, f, fpitch);
  }
}

__global__ void __launch_bounds__(256) k_project_vert(const double* xy, u64 V, const float* f, i64 fpitch, int W,
                                                      int H, float* out) {
  for (u64 k = (u64)blockIdx.x * blockDim.x + threadIdx.x; k < V; k += (u64)gridDim.x * blockDim.x) {
    const double2 p = reinterpret_cast<const double2*>(xy)[k];
    const double x = fmin(fmax(p.x, 0.0), (double)(W - 1)), y = fmin(fmax(p.y, 0.0), (double)(H - 1));
    const int i0 = (int)floor(x), j0 = (int)floor(y);
    const int i1 = min(i0 + 1, W - 1), j1 = min(j0 + 1, H - 1);
    const float u = (float)(x - i0), w = (float)(y - j0);
    const float* row0 = reinterpret_cast<const float*>((const char*)f + j0 * fpitch);
    const float* row1 = reinterpret_cast<const float*>((const char*)f + j1 * fpitch);
    const float f00 = __ldg(row0 + i0), f10 = __ldg(row0 + i1), f01 = __ldg(row1 + i0), f11 = __ldg(row1 + i1);
    out[k] = (1.f - w) * ((1.f - u) * f00 + u * f10) + w * ((1.f - u) * f01 + u * f11);
  }
}

}  // namespace

int launch_project(const double* xy, const int* tri, u64 T, u64 V, const float* f, i64 fpitch, int W, int H,
                   float* tri_value, float* vertex_value, cudaStream_t st) {
  if (T >= (1ull << 32)) return -1;
  int n = 0;
  if (tri_value && T) {
    const u64 blocks = std::min<u64>((T + 255) / 256, 152ull * 16);
    k_project_tri<<<(unsigned)blocks, 256, 0, st>>>(xy, tri, T, f, fpitch, W, H, tri_value);
    ++n;
  }
  if (vertex_value && V) {
    const u64 blocks = std::min<u64>((V + 255) / 256, 152ull * 16);
    k_project_vert<<<(unsigned)blocks, 256, 0, st>>>(xy, V, f, fpitch, W, H, vertex_value);
    ++n;
  }
  return n;
}

}  // namespace sbmt
