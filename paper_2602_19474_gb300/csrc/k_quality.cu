// k_quality.cu -- the mesh quality measures of the experiments section
// (Sec. 4): smallest interior angles and slivers (< 5 degrees), areas and
// their variance, the equilateral ratio by an edge-length test, the aspect
// ratio AR = longest edge / shortest altitude (median, 95th percentile,
// maximum) and the 2-degree histogram of the smallest angles.
//
// One pass over the triangles computes every per-triangle measure in double
// precision from the output coordinates, reduces minima, maxima, counts and
// the histogram per block, writes each block's area sums, and stores AR as
// a float per triangle.  Percentiles are nearest-rank (the k-th smallest
// value) and exact on those floats: a radix select over the float's bits in
// three levels (bits 31-20, 19-10, 9-0), each a histogram pass for both
// ranks at once, the host choosing the bin that holds each rank in between.
#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

constexpr int QHIST = 30;  // 2-degree bins of the smallest angle

// positive doubles order as their bit patterns
SBMT_DEV void atomic_min_pos(unsigned long long* a, double v) { atomicMin(a, (unsigned long long)__double_as_longlong(v)); }
SBMT_DEV void atomic_max_pos(unsigned long long* a, double v) { atomicMax(a, (unsigned long long)__double_as_longlong(v)); }

SBMT_DEV double angle_at(double ox, double oy, double ux, double uy, double vx, double vy) {
  const double d1x = ux - ox, d1y = uy - oy, d2x = vx - ox, d2y = vy - oy;
  return atan2(fabs(d1x * d2y - d1y * d2x), d1x * d2x + d1y * d2y);
}

// mm: [0] min angle, [1] min area, [2] max AR (double bits); cnt: [0]
// slivers, [1] equilateral; part: per block (sum of areas, of squares)
__global__ void __launch_bounds__(256) k_quality(const double* xy, const int* tri, u64 T, float* ar_out,
                                                 unsigned long long* mm, unsigned long long* cnt, double* part,
                                                 u32* hist) {
  __shared__ u32 s_hist[QHIST];
  __shared__ double s_red[2][8];
  __shared__ unsigned long long s_cnt[2];
  if (threadIdx.x < QHIST) s_hist[threadIdx.x] = 0;
  if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  double amin = 1e300, armax = 0.0, angmin = 1e300, sa = 0.0, sa2 = 0.0;
  u32 slv = 0, equ = 0;
  const double rad2deg = 57.295779513082320876798;
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x) {
    const int ia = tri[3 * t], ib = tri[3 * t + 1], ic = tri[3 * t + 2];
    const double2 a = reinterpret_cast<const double2*>(xy)[ia];
    const double2 b = reinterpret_cast<const double2*>(xy)[ib];
    const double2 c = reinterpret_cast<const double2*>(xy)[ic];
    const double ang = fmin(fmin(angle_at(a.x, a.y, b.x, b.y, c.x, c.y), angle_at(b.x, b.y, c.x, c.y, a.x, a.y)),
                            angle_at(c.x, c.y, a.x, a.y, b.x, b.y)) *
                       rad2deg;
    const double abx = b.x - a.x, aby = b.y - a.y, bcx = c.x - b.x, bcy = c.y - b.y, cax = a.x - c.x,
                 cay = a.y - c.y;
    const double l0 = abx * abx + aby * aby, l1 = bcx * bcx + bcy * bcy, l2 = cax * cax + cay * cay;
    const double area = 0.5 * fabs(abx * (c.y - a.y) - aby * (c.x - a.x));
    const double lmax = fmax(fmax(l0, l1), l2), lmin = fmin(fmin(l0, l1), l2);
    const double ar = lmax / (2.0 * area);
    ar_out[t] = (float)ar;
    angmin = fmin(angmin, ang), amin = fmin(amin, area), armax = fmax(armax, ar);
    sa += area, sa2 += area * area;
    slv += ang < 5.0 ? 1u : 0u;
    equ += (lmax - lmin) <= 1e-9 * lmax ? 1u : 0u;
    atomicAdd(&s_hist[min((int)(ang * 0.5), QHIST - 1)], 1u);
  }
  // block reductions
  for (int o = 16; o > 0; o >>= 1) {
    angmin = fmin(angmin, __shfl_xor_sync(0xffffffffu, angmin, o));
    amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
    armax = fmax(armax, __shfl_xor_sync(0xffffffffu, armax, o));
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sa2 += __shfl_xor_sync(0xffffffffu, sa2, o);
    slv += __shfl_xor_sync(0xffffffffu, slv, o);
    equ += __shfl_xor_sync(0xffffffffu, equ, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    if (angmin < 1e300) atomic_min_pos(&mm[0], angmin);
    if (amin < 1e300) atomic_min_pos(&mm[1], amin);
    atomic_max_pos(&mm[2], armax);
    s_red[0][w] = sa, s_red[1][w] = sa2;
    atomicAdd(&s_cnt[0], (unsigned long long)slv);
    atomicAdd(&s_cnt[1], (unsigned long long)equ);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int k = 0; k < 8; ++k) x += s_red[0][k], y += s_red[1][k];
    part[2 * blockIdx.x] = x, part[2 * blockIdx.x + 1] = y;
    atomicAdd(&cnt[0], s_cnt[0]);
    atomicAdd(&cnt[1], s_cnt[1]);
  }
  if (threadIdx.x < QHIST && s_hist[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_hist[threadIdx.x]);
}

// one level of the radix select: histogram of the bits [lo, lo + width) of
// the values whose bits above lo + width equal prefix[r], for the two ranks
__global__ void __launch_bounds__(256) k_select_hist(const float* v, u64 T, int lo, int width, u32 pre0, u32 pre1,
                                                     int above, u32* h0, u32* h1) {
  extern __shared__ u32 s_h[];  // 2 << width counters
  const int nb = 1 << width;
  for (int k = threadIdx.x; k < 2 * nb; k += blockDim.x) s_h[k] = 0;
  __syncthreads();
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x) {
    const u32 bits = __float_as_uint(v[t]);
    const u32 top = above < 32 ? bits >> above : 0u;
    const u32 bin = (bits >> lo) & (u32)(nb - 1);
    if (top == pre0) atomicAdd(&s_h[bin], 1u);
    if (top == pre1) atomicAdd(&s_h[nb + bin], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    if (s_h[k]) atomicAdd(&h0[k], s_h[k]);
    if (s_h[nb + k]) atomicAdd(&h1[k], s_h[nb + k]);
  }
}

}  // namespace

int launch_quality(const double* xy, const int* tri, u64 T, float* ar, unsigned long long* mm,
                   unsigned long long* cnt, double* part, int nblocks, u32* hist, cudaStream_t st) {
  k_quality<<<nblocks, 256, 0, st>>>(xy, tri, T, ar, mm, cnt, part, hist);
  return 1;
}

int launch_select_hist(const float* v, u64 T, int lo, int width, u32 pre0, u32 pre1, int above, u32* h0, u32* h1,
                       cudaStream_t st) {
  const size_t sm = (size_t)2 << width << 2;
  k_select_hist<<<152 * 4, 256, sm, st>>>(v, T, lo, width, pre0, pre1, above, h0, h1);
  return 1;
}

}  // namespace sbmt
