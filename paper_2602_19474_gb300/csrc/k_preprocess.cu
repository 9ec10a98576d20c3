// k_preprocess.cu -- geometric preprocessing of the base mesh (Alg. 3,
// Steps 1-3).
//
// The base mesh T0 (the lattice cells meeting the image rectangle, Sec. 3.3)
// and the boundary go in; the preprocessed mesh T comes out.
//  - Region I (Steps 1 and 2, which commute): a lattice vertex snaps onto the
//    nearest boundary point closer than a; a vertex that did not snap and is
//    closer than c to the boundary moves away from its nearest boundary point
//    q along q -> v to distance c.  Both read the positions of T0.
//  - Region II (Step 3): a boundary point p closer than b to an edge e of T
//    (neither end of e at p) is a candidate (p, e).  It applies when e is p's
//    smallest candidate edge (smaller end id, then larger) and no smaller
//    point has a candidate on an edge of the triangles beside e; it inserts
//    p and splits each triangle (u, w, x) beside e = uw into (u, p, x) and
//    (p, w, x) (Fig. "b threshold split").
// Boundary points are the PSLG vertices (pixel corners, id y (W + 1) + x),
// boundary segments the boundary pixel edges.  The thresholds arrive in
// pixels.
//
// Every decision is the plain double-precision evaluation of its formula,
// each operation rounded once (the _rn intrinsics keep the compiler from
// fusing them).  This part runs FP64 at a small fraction of its FP32 rate,
// so candidates are screened first: by integer tests (corner flags, pixel
// labels) and in single precision with a margin that covers the rounding
// of the coordinates to float.  Only survivors reach the double test.
#include <algorithm>

#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

// a boundary point's smallest candidate edge (Step 3) and the cells beside it
struct PreCand {
  u32 u, w;            // the edge's ends, u < w
  u32 cell[2];         // the cells beside it, NONE where absent
  u32 cv[2][3];        // their corners A, B, C
  unsigned char k[2];  // the edge's local index in each cell (AB 0, BC 1, CA 2)
  unsigned char n;     // cells found (0: no candidate)
};

size_t pre_cand_bytes(u32 np) { return (size_t)std::max<u32>(np, 1) * sizeof(PreCand); }

namespace {

constexpr double SQRT3D = 1.7320508075688772935;

SBMT_DEV double dadd(double a, double b) { return __dadd_rn(a, b); }
SBMT_DEV double dsub(double a, double b) { return __dsub_rn(a, b); }
SBMT_DEV double dmul(double a, double b) { return __dmul_rn(a, b); }
SBMT_DEV double d2of(double dx, double dy) { return dadd(dmul(dx, dx), dmul(dy, dy)); }

// (double)c - 1/2 from its bits, without the double-precision pipe
SBMT_DEV double half_minus(int c) {
  const int n = 2 * c - 1;  // odd, so never 0
  const u32 m = (u32)abs(n);
  const int e = 31 - __clz((int)m);  // m = 1.f * 2^e; the value is m / 2
  const u64 frac = ((u64)m << (52 - e)) & ((1ull << 52) - 1);
  const u64 bits = ((u64)(n < 0) << 63) | ((u64)(1022 + e) << 52) | frac;
  return __longlong_as_double((long long)bits);
}


// y of lattice row j in pixels, (oy + 3 p j sqrt3) / S
SBMT_DEV double row_y(const GridP& g, i64 j) {
  return __ddiv_rn(dadd((double)g.oy, dmul((double)(3 * g.p * j), SQRT3D)), (double)g.S);
}

SBMT_DEV bool corner_flag(const PreArgs& a, int cx, int cy) {
  return (a.vrow[(i64)cy * a.wpr + (cx >> 5)] >> (cx & 31)) & 1u;
}

// squared distance from p to the segment u -> w: the projection parameter
// clamped to [0, 1], then the offset
SBMT_DEV double seg_d2(double px, double py, double2 u, double2 w) {
  const double ex = dsub(w.x, u.x), ey = dsub(w.y, u.y);
  const double qx = dsub(px, u.x), qy = dsub(py, u.y);
  const double t = fmin(fmax(__ddiv_rn(dadd(dmul(qx, ex), dmul(qy, ey)), d2of(ex, ey)), 0.0), 1.0);
  return d2of(dsub(qx, dmul(t, ex)), dsub(qy, dmul(t, ey)));
}
SBMT_DEV float seg_d2f(float px, float py, float2 u, float2 w) {
  const float ex = w.x - u.x, ey = w.y - u.y, qx = px - u.x, qy = py - u.y;
  const float t = fminf(fmaxf((qx * ex + qy * ey) / (ex * ex + ey * ey), 0.f), 1.f);
  const float dx = qx - t * ex, dy = qy - t * ey;
  return dx * dx + dy * dy;
}

// Step 3's candidate test of the point (px, py) against the edge u w
// (a float distance beyond the band dband around b decides; an end at p
// has float coordinates equal to p's, the only case that reads doubles
// before the band does)
// The point is the corner (pcx, pcy), at (pcx - 1/2, pcy - 1/2): exact in
// float, so its doubles are made only where doubles decide.
SBMT_DEV bool is_cand(const PreArgs& a, int pcx, int pcy, u32 u, u32 w) {
  const float pxf = (float)pcx - 0.5f, pyf = (float)pcy - 0.5f;
  const float2 fu = a.xyf[u], fw = a.xyf[w];
  const float d2f = seg_d2f(pxf, pyf, fu, fw);
  if (d2f > a.b_hi2) return false;
  const double2* xy = reinterpret_cast<const double2*>(a.xy);
  // an end at p: a vertex snapped to p, or (an exact coincidence) one whose
  // double coordinates equal p's
  const int p = pcy * (a.g.W + 1) + pcx;
  auto at_p = [&](u32 v, float2 f) {
    if (f.x != pxf || f.y != pyf) return false;
    if (a.status[v] == 1) return a.snap[v] == p;
    const double2 d = xy[v];
    return d.x == half_minus(pcx) && d.y == half_minus(pcy);
  };
  if (at_p(u, fu) || at_p(w, fw)) return false;
  if (d2f < a.b_lo2) return true;
  return seg_d2(half_minus(pcx), half_minus(pcy), xy[u], xy[w]) < a.B2;
}

// pixel index of the centroid coordinate ((c0 + c1) + c2) / 3: the floor of
// it plus 1/2.  The float estimate decides unless it lies within its error
// bound of an integer; then the double evaluation does.
SBMT_DEV int cen_floor(double c0, double c1, double c2, float f0, float f1, float f2) {
  const float s = ((f0 + f1) + f2) * (1.0f / 3.0f) + 0.5f;
  const float M = fmaxf(fmaxf(fabsf(f0), fabsf(f1)), fabsf(f2));
  const float eps = (M + 1.0f) * 0x1p-19f;
  const float fl = floorf(s);
  if (s - fl > eps && (fl + 1.0f) - s > eps) return (int)fl;
  return (int)floor(dadd(__ddiv_rn(dadd(dadd(c0, c1), c2), 3.0), 0.5));
}

template <typename T>
SBMT_DEV unsigned short pre_label(const PreArgs& a, int col, int row) {
  const int l = pix<T>(a.img, a.pitch, a.g.W, a.g.H, col, row);
  return l == OUTSIDE ? (unsigned short)0xFFFF : (unsigned short)l;
}

template <typename T>
SBMT_DEV unsigned short moved_label(const PreArgs& a, const double2* pd, const float2* pf) {
  const int col = cen_floor(pd[0].x, pd[1].x, pd[2].x, pf[0].x, pf[1].x, pf[2].x);
  const int row = cen_floor(pd[0].y, pd[1].y, pd[2].y, pf[0].y, pf[1].y, pf[2].y);
  return pre_label<T>(a, col, row);
}

// x table over m = 2i + j (the x of v(i, j) depends on m only), y of every
// vertex row, and the pixel rows of the centroids of unmoved up and down
// cells, per strip row
__global__ void __launch_bounds__(256) k_pre_rows(PreArgs a) {
  const GridP& g = a.g;
  const i64 stride = (i64)gridDim.x * blockDim.x, t0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  for (i64 k = t0; k < a.nm; k += stride) {
    const double x = __ddiv_rn((double)(g.ox + 3 * g.p * (a.m0 + k)), (double)g.S);
    a.tab[k] = x;
    a.tabf[k] = __double2float_rn(x);
  }
  for (i64 r = t0; r < g.nvrows; r += stride) {
    const double y = row_y(g, g.vj0 + r);
    a.ytab[r] = y;
    a.ytabf[r] = __double2float_rn(y);
  }
  for (i64 r = t0; r < g.nrows; r += stride) {
    const i64 j = g.j0 + r;
    const double y0 = row_y(g, j), y1 = row_y(g, j + 1);
    // up cells have two corners on row j, down cells two on row j + 1
    a.prow[2 * r] = (int)floor(dadd(__ddiv_rn(dadd(dadd(y0, y0), y1), 3.0), 0.5));
    a.prow[2 * r + 1] = (int)floor(dadd(__ddiv_rn(dadd(dadd(y0, y1), y1), 3.0), 0.5));
  }
}

// Step 1 for the vertex v: the boundary point nearest to v, if closer than
// a (ties: the smaller id).  Float distances decide unless the nearest is
// within the band of a or of the next one; then doubles do.  Returns true
// with (bx, by) on a snap.
SBMT_DEV bool step1(const PreArgs& a, double x, double y, float xf, float yf, int& bx, int& by) {
  const int W = a.g.W, H = a.g.H;
  const float Af = a.ascr;
  const int x0 = max(0, (int)ceilf(xf + 0.5f - Af)), x1 = min(W, (int)floorf(xf + 0.5f + Af));
  const int y0 = max(0, (int)ceilf(yf + 0.5f - Af)), y1 = min(H, (int)floorf(yf + 0.5f + Af));
  int nclose = 0;
  float b1 = 3.0e38f, b2 = 3.0e38f;  // the two smallest float squared distances
  for (int cy = y0; cy <= y1 && x0 <= x1; ++cy) {
    const u32* wrow = a.vrow + (i64)cy * a.wpr;
    for (int wx = x0 >> 5; wx <= (x1 >> 5); ++wx) {
      const int lo = max(x0 - 32 * wx, 0), hi = min(x1 - 32 * wx, 31);
      u32 bits = wrow[wx] & (0xFFFFFFFFu << lo) & (0xFFFFFFFFu >> (31 - hi));
      while (bits) {
        const int cx = 32 * wx + __ffs(bits) - 1;
        bits &= bits - 1;
        const float dx = xf - ((float)cx - 0.5f), dy = yf - ((float)cy - 0.5f), d2f = dx * dx + dy * dy;
        if (d2f > a.a_hi2) continue;
        ++nclose;
        if (d2f < b1) b2 = b1, b1 = d2f, bx = cx, by = cy;
        else if (d2f < b2) b2 = d2f;
      }
    }
  }
  if (nclose == 0) return false;
  if (b1 < a.a_lo2 && (nclose == 1 || sqrtf(b2) - sqrtf(b1) > 2.5f * a.dband)) return true;
  // doubles, in increasing corner id
  double best = 0.0;
  bx = -1;
  for (int cy = y0; cy <= y1; ++cy)
    for (int cx = x0; cx <= x1; ++cx) {
      if (!corner_flag(a, cx, cy)) continue;
      const double d2 = d2of(dsub(x, half_minus(cx)), dsub(y, half_minus(cy)));
      if (bx < 0 || d2 < best) best = d2, bx = cx, by = cy;
    }
  return best < dmul(a.A, a.A);
}

// Step 2's candidate edges: the boundary pixel edges between two pixels of
// the box m0..m1 x k0..k1 (pixel labels from get(m, kk)).  Horizontal edge
// (m, kk) at y = kk - 1/2 lies between pixels (m, kk - 1) and (m, kk), id
// kk W + m; vertical edge (m, kk) at x = m - 1/2 between (m - 1, kk) and
// (m, kk), id (H + 1) W + kk (W + 1) + m.  visit(horizontal, m, kk).
template <class G, class F>
SBMT_DEV void box_edges(int W, int H, int m0, int m1, int k0, int k1, G&& get, F&& visit) {
  for (int kk = k0; kk <= k1; ++kk)
    for (int m = m0; m <= m1; ++m) {
      const int l = get(m, kk);
      if (kk > k0 && m >= 0 && m < W && l != get(m, kk - 1)) visit(true, m, kk);
      if (m > m0 && kk >= 0 && kk < H && l != get(m - 1, kk)) visit(false, m, kk);
    }
}

// Step 2 for the vertex v: the nearest point q of the boundary pixel edges
// (ties: the smaller edge id); if it is closer than c, v moves to
// q + c (v - q) / |v - q|.  An edge within c of v lies between two pixels
// of the box around v.  With only_screen, returns whether the float
// distances leave a move possible (the nearest edge within the band of c);
// otherwise decides in doubles among the edges within two bands of the
// float minimum and returns whether v moved (to out).
template <typename T>
SBMT_DEV bool step2(const PreArgs& a, double x, double y, float xf, float yf, bool only_screen, double2& out) {
  const int W = a.g.W, H = a.g.H;
  const float Cf = a.cscr;
  const int m0 = max(-1, (int)ceilf(xf - Cf - 0.5f)), m1 = min(W, (int)floorf(xf + Cf + 0.5f));
  const int k0 = max(-1, (int)ceilf(yf - Cf - 0.5f)), k1 = min(H, (int)floorf(yf + Cf + 0.5f));
  auto fdist = [&](bool hor, int m, int kk) {
    const float dx = hor ? xf - fminf(fmaxf(xf, (float)m - 0.5f), (float)m + 0.5f) : xf - ((float)m - 0.5f);
    const float dy = hor ? yf - ((float)kk - 0.5f) : yf - fminf(fmaxf(yf, (float)kk - 0.5f), (float)kk + 0.5f);
    return dx * dx + dy * dy;
  };
  float minf = 3.0e38f;
  auto fvisit = [&](bool hor, int m, int kk) { minf = fminf(minf, fdist(hor, m, kk)); };
  double best = 0.0, bqx = 0.0, bqy = 0.0;
  i64 bid = -1;
  float lim = 0.0f;
  auto dvisit = [&](bool hor, int m, int kk) {
    if (fdist(hor, m, kk) > lim) return;
    const double qx = hor ? fmin(fmax(x, half_minus(m)), half_minus(m + 1)) : half_minus(m);
    const double qy = hor ? half_minus(kk) : fmin(fmax(y, half_minus(kk)), half_minus(kk + 1));
    const double d2 = d2of(dsub(x, qx), dsub(y, qy));
    const i64 id = hor ? (i64)kk * W + m : (i64)(H + 1) * W + (i64)kk * (W + 1) + m;
    if (bid < 0 || d2 < best || (d2 == best && id < bid)) best = d2, bid = id, bqx = qx, bqy = qy;
  };
  auto get = [&](int m, int kk) { return pix<T>(a.img, a.pitch, W, H, m, kk); };
  box_edges(W, H, m0, m1, k0, k1, get, fvisit);
  if (minf > a.c_hi2) return false;  // no boundary edge within c
  if (only_screen) return true;
  lim = (sqrtf(minf) + 2.0f * a.dband) * (sqrtf(minf) + 2.0f * a.dband) * 1.0001f;
  box_edges(W, H, m0, m1, k0, k1, get, dvisit);
  if (bid < 0 || !(best < dmul(a.C, a.C))) return false;
  const double t = __ddiv_rn(a.C, __dsqrt_rn(best));
  out = make_double2(dadd(bqx, dmul(t, dsub(x, bqx))), dadd(bqy, dmul(t, dsub(y, bqy))));
  return true;
}

// Region I, first pass: one block per vertex row.  A vertex whose nearby
// pixels carry one label stays; the others are queued in the row's own part
// of the queue (the row's vertex ids) for the second pass, which takes them
// densely, so that the few near the boundary do not hold up warps of
// vertices that stay.
constexpr int PV_U = 1;  // vertices per thread per iteration (2 measured slower)

template <typename T>
__global__ void __launch_bounds__(256) k_pre_vertex(PreArgs a) {
  __shared__ u32 nslow;
  if (threadIdx.x == 0) nslow = 0;
  __syncthreads();
  const GridP& g = a.g;
  const int r = blockIdx.x, W = g.W, H = g.H;
  const i64 j = g.vj0 + r, lo = g.vlo[r], n = g.vhi[r] - lo + 1, base = g.vbase[r];
  const double y = a.ytab[r];
  const float yf = a.ytabf[r];
  const float Af = a.ascr;
  // pixel rows whose squares reach within a of the row
  const int py0 = (int)ceilf(yf - Af - 0.5f), py1 = (int)floorf(yf + Af + 0.5f);
  const float invS = 1.0f / (float)g.S;
  double2* xy = reinterpret_cast<double2*>(a.xy);
  const int lane = threadIdx.x & 31;
  // one label over the pixels whose squares reach within a of v: no boundary
  // edge within a (c < a), no boundary point either (a PSLG vertex's four
  // pixels are among them), and v stays.  Boxes reaching past the image take
  // the general path.
  auto uniform_at = [&](i64 mi) {
    // x of v for the box: the exact numerator times 1/S in float (within a
    // few float roundings of the table's value; the box's margin covers them)
    const float xq = (float)(int)(g.ox + 3 * g.p * (a.m0 + mi)) * invS;
    const int px0 = (int)ceilf(xq - Af - 0.5f), px1 = (int)floorf(xq + Af + 0.5f);
    if (px0 < 0 || py0 < 0 || px1 >= W || py1 >= H) return false;
    const unsigned char* rowp = a.img + (i64)py0 * a.pitch;
    const T l0 = ((const T*)rowp)[px0];
    bool uniform = true;
    if (py1 - py0 < 3 && px1 - px0 < 4) {
      // a box of at most 3 x 4 pixels: all loads issued at once
      T pv[3][4];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          pv[rr][c] = (rr <= py1 - py0 && c <= px1 - px0) ? ((const T*)(rowp + rr * a.pitch))[px0 + c] : l0;
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int c = 0; c < 4; ++c) uniform &= pv[rr][c] == l0;
    } else {
      for (int yy = py0; yy <= py1 && uniform; ++yy, rowp += a.pitch)
        for (int xx = px0; xx <= px1; ++xx)
          if (((const T*)rowp)[xx] != l0) {
            uniform = false;
            break;
          }
    }
    return uniform;
  };
  // the screen's loads before any store; whole warps in every iteration
  for (i64 k0 = 0; k0 < n; k0 += PV_U * blockDim.x) {
    bool slow[PV_U];
#pragma unroll
    for (int u = 0; u < PV_U; ++u) {
      const i64 k = k0 + threadIdx.x + u * blockDim.x;
      slow[u] = k < n && !uniform_at(2 * (lo + k) + j - a.m0);
    }
#pragma unroll
    for (int u = 0; u < PV_U; ++u) {
      const i64 k = k0 + threadIdx.x + u * blockDim.x;
      if (k < n && !slow[u]) {
        const i64 mi = 2 * (lo + k) + j - a.m0;
        xy[base + k] = make_double2(a.tab[mi], y);
        a.xyf[base + k] = make_float2(a.tabf[mi], yf);
        a.status[base + k] = 0;
        a.snap[base + k] = -1;
      }
      const u32 m = __ballot_sync(0xFFFFFFFFu, slow[u]);
      if (m) {
        u32 q0 = 0;
        if (lane == 0) q0 = atomicAdd(&nslow, (u32)__popc(m));
        q0 = __shfl_sync(0xFFFFFFFFu, q0, 0);
        if (slow[u]) a.vq[base + q0 + __popc(m & ((1u << lane) - 1u))] = (u32)(base + k);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) a.vqn[r] = nslow;
}

// a vertex of the base mesh's outer boundary: one of the six cells around
// v(i, j) -- up cells 2i-2 and 2i and down cell 2i-1 of strip j, down cells
// 2i-1 and 2i+1 and up cell 2i of strip j-1 -- is not in the mesh.  Such a
// vertex snaps only onto an image corner or a border point at least h + a
// from both ends of its side: a neighbour lies within h of it and it within
// a of the point, so only a point nearer an image corner lets the moved
// outer boundary cut across the image's corner (and a point off the border
// would pull it inside).  It may be repelled.
SBMT_DEV bool outer_vertex(const GridP& g, i64 i, i64 j) {
  return !(cell_in(g, 2 * i - 2, j) && cell_in(g, 2 * i - 1, j) && cell_in(g, 2 * i, j) &&
           cell_in(g, 2 * i - 1, j - 1) && cell_in(g, 2 * i, j - 1) && cell_in(g, 2 * i + 1, j - 1));
}
SBMT_DEV bool border_safe(const PreArgs& a, int bx, int by) {
  const GridP& g = a.g;
  const bool onx = bx == 0 || bx == g.W, ony = by == 0 || by == g.H;
  if (onx && ony) return true;
  if (!onx && !ony) return false;
  const int side = onx ? min(by, g.H - by) : min(bx, g.W - bx);
  return (double)side >= dadd(__ddiv_rn((double)g.p, (double)g.q), a.A);
}

// Region I, second pass: the queued vertices, one block per vertex row at a
// time.  Step 1 in full; Step 2 only screened here: a vertex the float
// distances leave within reach of c goes to the third pass, so that the
// double-precision work of the moves runs in full warps.
constexpr int PR_CHUNK = 1024;

template <typename T>
__global__ void __launch_bounds__(128) k_pre_region1(PreArgs a) {
  __shared__ u32 rq[PR_CHUNK];
  __shared__ u32 nrq, rq0;
  const GridP& g = a.g;
  double2* xy = reinterpret_cast<double2*>(a.xy);
  u32 nsnap = 0;
  for (int r = blockIdx.x; r < g.nvrows; r += gridDim.x) {
    const u32 nq = a.vqn[r];
    const i64 base = g.vbase[r], j = g.vj0 + r, lo = g.vlo[r];
    const double y = a.ytab[r];
    const float yf = a.ytabf[r];
    for (u32 c0 = 0; c0 < nq; c0 += PR_CHUNK) {
      if (threadIdx.x == 0) nrq = 0;
      __syncthreads();
      const u32 c1 = min(nq, c0 + PR_CHUNK);
      for (u32 e = c0 + threadIdx.x; e < c1; e += blockDim.x) {
        const i64 v = a.vq[base + e], mi = 2 * (lo + (v - base)) + j - a.m0;
        const double x = a.tab[mi];
        const float xf = a.tabf[mi];
        int bx = -1, by = -1;
        if (step1(a, x, y, xf, yf, bx, by) && (!outer_vertex(g, lo + (v - base), j) || border_safe(a, bx, by))) {
          xy[v] = make_double2(half_minus(bx), half_minus(by));
          a.xyf[v] = make_float2((float)bx - 0.5f, (float)by - 0.5f);
          a.status[v] = 1;
          a.snap[v] = by * (g.W + 1) + bx;
          ++nsnap;
          continue;
        }
        double2 dummy;
        xy[v] = make_double2(x, y);
        a.xyf[v] = make_float2(xf, yf);
        a.status[v] = 0;
        a.snap[v] = -1;
        if (step2<T>(a, x, y, xf, yf, true, dummy)) rq[atomicAdd(&nrq, 1u)] = (u32)v;
      }
      __syncthreads();
      const u32 n = nrq;
      if (threadIdx.x == 0 && n) rq0 = atomicAdd(a.cnt + 6, n);
      __syncthreads();
      for (u32 e = threadIdx.x; e < n; e += blockDim.x) {
        a.rq[rq0 + e] = make_uint2(rq[e], (u32)r);
      }
      __syncthreads();
    }
  }
  nsnap = __reduce_add_sync(0xFFFFFFFFu, nsnap);
  if ((threadIdx.x & 31) == 0 && nsnap) atomicAdd(a.cnt + 3, nsnap);
}

// Region I, third pass: Step 2 in doubles for the vertices the float
// screen left within reach of c
template <typename T>
__global__ void __launch_bounds__(128) k_pre_repel(PreArgs a) {
  const GridP& g = a.g;
  const u32 n = a.cnt[6];
  double2* xy = reinterpret_cast<double2*>(a.xy);
  u32 nrep = 0;
  for (u32 e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const uint2 qe = a.rq[e];
    const int r = (int)qe.y;
    const i64 v = qe.x, mi = 2 * (g.vlo[r] + (v - g.vbase[r])) + (g.vj0 + r) - a.m0;
    double2 out;
    if (step2<T>(a, a.tab[mi], a.ytab[r], a.tabf[mi], a.ytabf[r], false, out)) {
      xy[v] = out;
      a.xyf[v] = make_float2(__double2float_rn(out.x), __double2float_rn(out.y));
      a.status[v] = 2;
      ++nrep;
    }
  }
  nrep = __reduce_add_sync(0xFFFFFFFFu, nrep);
  if ((threadIdx.x & 31) == 0 && nrep) atomicAdd(a.cnt + 4, nrep);
}

// population counts of a bit-plane; with wpr > 0 the plane has rows of wpr
// words and only the bits of corner columns 0..W count
__global__ void __launch_bounds__(256) k_popc(const u32* words, u64 n, int wpr, int W, u32* out) {
  for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (u64)gridDim.x * blockDim.x) {
    u32 b = words[w];
    if (wpr > 0) {
      const int c0 = 32 * (int)(w % (u64)wpr);
      if (W - c0 < 31) b &= (2u << (W - c0)) - 1u;
    }
    out[w] = __popc(b);
  }
}

// the boundary points in corner-id order
__global__ void __launch_bounds__(256) k_pre_points(PreArgs a, u64 nw, const u32* wscan) {
  const int W = a.g.W;
  for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (u64)gridDim.x * blockDim.x) {
    u32 b = a.vrow[w];
    const int cy = (int)(w / (u64)a.wpr), c0 = 32 * (int)(w % (u64)a.wpr);
    u32 o = wscan[w];
    while (b) {
      const int cx = c0 + __ffs(b) - 1;
      b &= b - 1;
      if (cx > W || o >= a.np) break;
      a.plist[o++] = (u32)cy * (u32)(W + 1) + (u32)cx;
    }
  }
}

// Step 3, one thread per boundary point p.
// First p's smallest candidate edge and the cells beside it: a candidate
// edge's moved ends lie within a of their lattice positions, so its lattice
// segment lies within a + b of p, and the cells visited are those whose
// lattice extent meets p's box of that half-width.
// Then the conflict test: p applies unless a smaller point has a candidate
// on an edge of a cell beside p's edge; such a point lies within b of the
// bounding box of those cells' moved corners.
__global__ void __launch_bounds__(128, 4) k_pre_step3(PreArgs a) {
  const GridP& g = a.g;
  const u64 V = (u64)g.nverts;
  const float R = a.reach;
  u32 found = 0;
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < a.np; t += gridDim.x * blockDim.x) {
    const u32 p = a.plist[t];
    const int pcx = (int)(p % (u32)(g.W + 1)), pcy = (int)(p / (u32)(g.W + 1));
    const float pxf = (float)pcx - 0.5f, pyf = (float)pcy - 0.5f;
    PreCand c;
    c.u = c.w = NONE, c.cell[0] = c.cell[1] = NONE, c.k[0] = c.k[1] = 0, c.n = 0;
    u64 best = ~0ull;
    // strip rows: row jj spans the lattice row coordinate [jj, jj + 1]
    const float ilo = (pyf - R - a.oyf) / a.rowh, ihi = (pyf + R - a.oyf) / a.rowh;
    const int jlo = max(g.j0, (int)floorf(ilo - 1e-6f * fabsf(ilo) - 0.01f));
    const int jhi = min(g.j0 + g.nrows - 1, (int)floorf(ihi + 1e-6f * fabsf(ihi) + 0.01f));
    for (int jj = jlo; jj <= jhi; ++jj) {
      const int r = jj - g.j0, rv = jj - g.vj0;
      const i64 clo = g.clo[r], vb0 = g.vbase[rv] - g.vlo[rv], vb1 = g.vbase[rv + 1] - g.vlo[rv + 1];
      const u32 cb = (u32)g.cbase[r];
      // cell cc of the row spans 2u in [cc, cc + 2], u = (x - ox) / h - jj / 2
      const float ulo = 2.0f * ((pxf - R - a.oxf) / a.hf) - (float)jj;
      const float uhi = 2.0f * ((pxf + R - a.oxf) / a.hf) - (float)jj;
      const i64 c0 = max(clo, (i64)(int)floorf(ulo - 2.0f - 1e-6f * fabsf(ulo) - 0.01f));
      const i64 c1 = min(g.chi[r], (i64)(int)floorf(uhi + 1e-6f * fabsf(uhi) + 0.01f));
      for (i64 cc = c0; cc <= c1; ++cc) {
        const i64 i = cc >> 1;
        const bool down = (cc & 1) != 0;
        const u32 v[3] = {(u32)(down ? vb0 + i + 1 : vb0 + i), (u32)(down ? vb1 + i + 1 : vb0 + i + 1),
                          (u32)(vb1 + i)};
        const float2 f[3] = {a.xyf[v[0]], a.xyf[v[1]], a.xyf[v[2]]};
        // the cell's moved bounding box against p's b-box
        const float bx0 = fminf(fminf(f[0].x, f[1].x), f[2].x), bx1 = fmaxf(fmaxf(f[0].x, f[1].x), f[2].x);
        const float by0 = fminf(fminf(f[0].y, f[1].y), f[2].y), by1 = fmaxf(fmaxf(f[0].y, f[1].y), f[2].y);
        if (bx0 > pxf + a.bscr || bx1 < pxf - a.bscr || by0 > pyf + a.bscr || by1 < pyf - a.bscr) continue;
        const u32 cid = cb + (u32)(cc - clo);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const u32 u = v[e], w = v[e == 2 ? 0 : e + 1];
          if (!is_cand(a, pcx, pcy, u, w)) continue;
          const u32 lo = min(u, w), hi = max(u, w);
          const u64 key = (u64)lo * V + hi;
          if (key < best) {
            best = key, c.u = lo, c.w = hi, c.n = 1;
            c.cell[0] = cid, c.k[0] = (unsigned char)e, c.cell[1] = NONE;
            c.cv[0][0] = v[0], c.cv[0][1] = v[1], c.cv[0][2] = v[2];
          } else if (key == best && c.n == 1) {
            c.n = 2, c.cell[1] = cid, c.k[1] = (unsigned char)e;
            c.cv[1][0] = v[0], c.cv[1][1] = v[1], c.cv[1][2] = v[2];
          }
        }
      }
    }
    bool ok = c.n != 0;
    found += ok;
    if (ok) {
      float bx0 = 3.0e38f, bx1 = -3.0e38f, by0 = 3.0e38f, by1 = -3.0e38f;
      for (int s = 0; s < c.n; ++s)
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const float2 f = a.xyf[c.cv[s][e]];
          bx0 = fminf(bx0, f.x), bx1 = fmaxf(bx1, f.x), by0 = fminf(by0, f.y), by1 = fmaxf(by1, f.y);
        }
      const int x0 = max(0, (int)ceilf(bx0 - a.bscr + 0.5f)), x1 = min(g.W, (int)floorf(bx1 + a.bscr + 0.5f));
      const int y0 = max(0, (int)ceilf(by0 - a.bscr + 0.5f)), y1 = min(pcy, (int)floorf(by1 + a.bscr + 0.5f));
      for (int cy = y0; cy <= y1 && ok; ++cy) {
        const int xe = cy == pcy ? min(x1, pcx - 1) : x1;  // ids below p only
        const u32* wrow = a.vrow + (i64)cy * a.wpr;
        for (int wx = x0 >> 5; wx <= (xe >> 5) && ok && x0 <= xe; ++wx) {
          // the flagged corners of this word within [x0, xe]
          u32 bits = wrow[wx];
          const int b0 = max(x0 - 32 * wx, 0), b1 = min(xe - 32 * wx, 31);
          bits &= (0xFFFFFFFFu << b0) & (0xFFFFFFFFu >> (31 - b1));
          while (bits && ok) {
            const int cx = 32 * wx + __ffs(bits) - 1;
            bits &= bits - 1;
            for (int s = 0; s < c.n && ok; ++s)
#pragma unroll
              for (int e = 0; e < 3; ++e)
                if (ok && is_cand(a, cx, cy, c.cv[s][e], c.cv[s][e == 2 ? 0 : e + 1])) ok = false;
          }
        }
      }
    }
    if (ok) {
      // the re-fan keeps both halves (u, p, x) and (p, w, x) of every cell
      // beside the edge strictly counter-clockwise
      const double2* X = reinterpret_cast<const double2*>(a.xy);
      const double2 P = make_double2((double)pcx - 0.5, (double)pcy - 0.5);
      auto orient = [](double2 p0, double2 p1, double2 p2) {
        return dsub(dmul(dsub(p1.x, p0.x), dsub(p2.y, p0.y)), dmul(dsub(p1.y, p0.y), dsub(p2.x, p0.x)));
      };
      for (int s = 0; s < c.n && ok; ++s) {
        const int e = c.k[s];
        const double2 U = X[c.cv[s][e]], Wv = X[c.cv[s][e == 2 ? 0 : e + 1]], Xv = X[c.cv[s][e == 0 ? 2 : e - 1]];
        ok = orient(U, P, Xv) > 0.0 && orient(P, Wv, Xv) > 0.0;
      }
    }
    a.appl[t] = ok ? 1u : 0u;
    if (ok) {
      a.cand[t] = c;
      for (int s = 0; s < c.n; ++s) atomicOr(a.sbit + (c.cell[s] >> 5), 1u << (c.cell[s] & 31));
    }
  }
  found = __reduce_add_sync(0xFFFFFFFFu, found);
  if ((threadIdx.x & 31) == 0 && found) atomicAdd(a.cnt + 5, found);
}

// output triangle index of cell cid: its id plus the split cells before it
SBMT_DEV u64 out_index(const PreArgs& a, u32 cid) {
  return (u64)cid + a.wpre[cid >> 5] + __popc(a.sbit[cid >> 5] & ((1u << (cid & 31)) - 1u));
}

// the preprocessed mesh: every cell that is not split, as its triangle
// (A, B, C), labelled by its centroid -- exactly for a cell with three
// unmoved corners (the column in integers, the row from the per-row table).
// One block per strip row at a time, each thread over four of the row's
// cells at once (their loads issued together).
constexpr int PE_CELLS = 4;

template <typename T>
__global__ void __launch_bounds__(256, 6) k_pre_emit(PreArgs a) {
  const GridP& g = a.g;
  const double2* xy = reinterpret_cast<const double2*>(a.xy);
  const int den = (int)(2 * g.S);
  const float inv_den = 1.0f / (float)den;
  for (int r = blockIdx.x; r < g.nrows; r += gridDim.x) {
    const i64 jr = g.j0 + (i64)r, clo = g.clo[r];
    const int nrc = (int)(g.chi[r] - clo + 1);
    const u32 cb = (u32)g.cbase[r];
    const int rv = (int)(jr - g.vj0);  // vertex rows rv (jr) and rv + 1 (jr + 1)
    const int vb0 = (int)(g.vbase[rv] - g.vlo[rv]), vb1 = (int)(g.vbase[rv + 1] - g.vlo[rv + 1]);
    const int prow0 = a.prow[2 * r], prow1 = a.prow[2 * r + 1];
    const int i0 = (int)(clo >> 1), par = (int)(clo & 1);
    // centroid x of cell c in units of 1/S: ox + 3p (c + jr + 1), so the
    // pixel column's numerator 2 xc + S grows by 6p per cell
    const int num0 = (int)(2 * (g.ox + 3 * g.p * (clo + jr + 1)) + g.S), dnum = (int)(6 * g.p);
    for (int kb = 0; kb < nrc; kb += PE_CELLS * blockDim.x) {
      int v0[PE_CELLS], v1[PE_CELLS], v2[PE_CELLS], praw[PE_CELLS];
      unsigned char mv[PE_CELLS];
      u32 o[PE_CELLS];
      bool act[PE_CELLS];
      // every load of the four cells first (a cell past the row's end reads
      // the row's last cell), then the split test and the writes
      u32 sw[PE_CELLS], wp[PE_CELLS], cidq[PE_CELLS];
#pragma unroll
      for (int q = 0; q < PE_CELLS; ++q) {
        const int k0q = kb + (int)threadIdx.x + q * (int)blockDim.x;
        act[q] = k0q < nrc;
        const int k = act[q] ? k0q : nrc - 1;
        const u32 cid = cb + (u32)k;
        cidq[q] = cid;
        sw[q] = a.sbit[cid >> 5], wp[q] = a.wpre[cid >> 5];
        const int c = par + k, i = i0 + (c >> 1);  // c: the cell index relative to 2 i0
        const bool down = (c & 1) != 0;
        v0[q] = down ? vb0 + i + 1 : vb0 + i;
        v1[q] = down ? vb1 + i + 1 : vb0 + i + 1;
        v2[q] = vb1 + i;
        mv[q] = a.status[v0[q]] | a.status[v1[q]] | a.status[v2[q]];
        // pixel column floor(num / 2S): a float estimate, corrected
        const int num = num0 + dnum * k;
        int col = (int)floorf((float)num * inv_den);
        while (col * den > num) --col;
        while ((col + 1) * den <= num) ++col;
        praw[q] = pix<T>(a.img, a.pitch, g.W, g.H, col, down ? prow1 : prow0);
      }
#pragma unroll
      for (int q = 0; q < PE_CELLS; ++q) {
        const u32 cid = cidq[q];
        if ((sw[q] >> (cid & 31)) & 1u) act[q] = false;  // split: the split kernel writes it
        o[q] = cid + wp[q] + __popc(sw[q] & ((1u << (cid & 31)) - 1u));
      }
#pragma unroll
      for (int q = 0; q < PE_CELLS; ++q) {
        if (!act[q]) continue;
        unsigned short lab;
        if (mv[q] == 0) {
          lab = praw[q] == OUTSIDE ? (unsigned short)0xFFFF : (unsigned short)praw[q];
        } else {
          const double2 pd[3] = {xy[v0[q]], xy[v1[q]], xy[v2[q]]};
          const float2 pf[3] = {a.xyf[v0[q]], a.xyf[v1[q]], a.xyf[v2[q]]};
          lab = moved_label<T>(a, pd, pf);
        }
        const u64 oo = o[q];
        a.tri[3 * oo] = v0[q], a.tri[3 * oo + 1] = v1[q], a.tri[3 * oo + 2] = v2[q];
        a.label[oo] = lab, a.code[oo] = 0;
      }
    }
  }
}

// the applied points: vertex V + rank at the corner, the elimination
// record, and the two halves of each split cell
template <typename T>
__global__ void __launch_bounds__(128) k_pre_split(PreArgs a) {
  const GridP& g = a.g;
  double2* xy = reinterpret_cast<double2*>(a.xy);
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < a.np; t += gridDim.x * blockDim.x) {
    if (!a.appl[t]) continue;
    const PreCand c = a.cand[t];
    const u32 p = a.plist[t], rank = a.ascan[t], q = (u32)g.nverts + rank;
    const int cx = (int)(p % (u32)(g.W + 1)), cy = (int)(p / (u32)(g.W + 1));
    const double2 pq = make_double2((double)cx - 0.5, (double)cy - 0.5);
    const float2 pqf = make_float2((float)cx - 0.5f, (float)cy - 0.5f);
    xy[q] = pq;
    a.elim[3 * (u64)rank] = (int)p, a.elim[3 * (u64)rank + 1] = (int)c.u, a.elim[3 * (u64)rank + 2] = (int)c.w;
    for (int s = 0; s < c.n; ++s) {
      const u32 cell = c.cell[s];
      const int k = c.k[s];
      const u32 u = c.cv[s][k], w = c.cv[s][(k + 1) % 3], x = c.cv[s][(k + 2) % 3];
      const u64 o = out_index(a, cell);
      const double2 du = xy[u], dw = xy[w], dx = xy[x];
      const float2 fu = a.xyf[u], fw = a.xyf[w], fx = a.xyf[x];
      // (u, p, x), then (p, w, x)
      a.tri[3 * o] = (int)u, a.tri[3 * o + 1] = (int)q, a.tri[3 * o + 2] = (int)x;
      a.tri[3 * o + 3] = (int)q, a.tri[3 * o + 4] = (int)w, a.tri[3 * o + 5] = (int)x;
      const double2 d0[3] = {du, pq, dx}, d1[3] = {pq, dw, dx};
      const float2 f0[3] = {fu, pqf, fx}, f1[3] = {pqf, fw, fx};
      a.label[o] = moved_label<T>(a, d0, f0);
      a.label[o + 1] = moved_label<T>(a, d1, f1);
      a.code[o] = 0, a.code[o + 1] = 0;
    }
  }
}

// status words: the eliminations and split cells, from the scans' totals
__global__ void k_pre_totals(PreArgs a, u64 nsw) {
  a.cnt[1] = a.ascan[a.np];
  a.cnt[2] = a.wpre[nsw];
}

unsigned grid_for(u64 n, int threads, unsigned cap) {
  return (unsigned)std::max<u64>(1, std::min<u64>((n + threads - 1) / threads, cap));
}

}  // namespace

int launch_preprocess(const PreArgs& a, u64 nw, u32* wpop, u32* wscan, u32* scr, cudaStream_t st) {
  int n = 0;
  const GridP& g = a.g;
  k_pre_rows<<<grid_for((u64)std::max<i64>(a.nm, std::max(g.nrows, g.nvrows)), 256, 1024), 256, 0, st>>>(a), ++n;
  if (a.dtype == 1) {
    k_pre_vertex<unsigned char><<<g.nvrows, 256, 0, st>>>(a);
    k_pre_region1<unsigned char><<<(unsigned)std::min(g.nvrows, 152 * 16), 128, 0, st>>>(a);
    k_pre_repel<unsigned char><<<152 * 8, 128, 0, st>>>(a);
  } else {
    k_pre_vertex<unsigned short><<<g.nvrows, 256, 0, st>>>(a);
    k_pre_region1<unsigned short><<<(unsigned)std::min(g.nvrows, 152 * 16), 128, 0, st>>>(a);
    k_pre_repel<unsigned short><<<152 * 8, 128, 0, st>>>(a);
  }
  n += 3;
  // the boundary points, in corner-id order
  k_popc<<<grid_for(nw, 256, 152 * 8), 256, 0, st>>>(a.vrow, nw, a.wpr, g.W, wpop), ++n;
  n += launch_scan(wpop, 1, wscan, (u32)nw, scr, st);
  k_pre_points<<<grid_for(nw, 256, 152 * 8), 256, 0, st>>>(a, nw, wscan), ++n;
  // Step 3
  const u64 nsw = ((u64)g.ncells + 31) / 32;
  if (cudaMemsetAsync(a.sbit, 0, (nsw + 1) * sizeof(u32), st) != cudaSuccess) return -1;
  k_pre_step3<<<grid_for(a.np, 128, 152 * 16), 128, 0, st>>>(a), ++n;
  n += launch_scan(a.appl, 1, a.ascan, a.np, scr, st);
  k_popc<<<grid_for(nsw, 256, 152 * 8), 256, 0, st>>>(a.sbit, nsw, 0, 0, a.spop), ++n;
  n += launch_scan(a.spop, 1, a.wpre, (u32)nsw, scr, st);
  // the preprocessed mesh
  if (a.dtype == 1) {
    k_pre_emit<unsigned char><<<(unsigned)std::min(g.nrows, 152 * 16), 256, 0, st>>>(a);
    k_pre_split<unsigned char><<<grid_for(a.np, 128, 152 * 16), 128, 0, st>>>(a);
  } else {
    k_pre_emit<unsigned short><<<(unsigned)std::min(g.nrows, 152 * 16), 256, 0, st>>>(a);
    k_pre_split<unsigned short><<<grid_for(a.np, 128, 152 * 16), 128, 0, st>>>(a);
  }
  n += 2;
  k_pre_totals<<<1, 1, 0, st>>>(a, nsw), ++n;
  return n;
}

}  // namespace sbmt
