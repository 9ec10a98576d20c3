// k_traverse.cu -- K2: analytic segment -> grid-triangle traversal, bucketed
// by cell id and by grid-edge id, and the frozen event registry.
//
// Alg. 1 (Sec. 3.3.1) classifies every segment/edge pair.  For the
// degeneracy-free grids accepted here (integer origin, h = p/q with p even and
// q odd) no grid vertex lies on a pixel line and no pixel corner on a grid
// edge, so a boundary segment meets a grid edge only in a proper crossing:
// one Alg. 1 "crosses e" event.  Instead of testing pairs (or querying a
// KD-tree, App. C) each segment is walked analytically: a horizontal run
// stays in one strip row and crosses the 60- and 120-degree lines, which
// repeat every 6p scaled units; a vertical run crosses one slanted edge and
// one horizontal edge per strip.  Every crossing is an event; every cell
// visited is a (cell, segment) pair.
//
// Events are numbered as the registry of Assumption "frozen registry"
// (Sec. 3.3.3): by grid-edge id, then by position along the edge, so that
// both cells sharing an edge name each crossing vertex identically with no
// atomics and no tolerance.
#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

SBMT_DEV bool vid_ok(const GridP& g, i64 i, i64 j) {
  if (j < g.vj0 || j >= g.vj0 + g.nvrows) return false;
  const int r = (int)(j - g.vj0);
  return i >= g.vlo[r] && i <= g.vhi[r];
}

// Walk one segment from its lower end along +x / +y, calling f.cell(c, j)
// for every cell entered and f.cross(edge, x, y) for every crossing, in order.
template <class F>
SBMT_DEV void walk_segment(const GridP& g, const Seg& s, F& f) {
  const i64 p = g.p, q = g.q, ox = g.ox, oy = g.oy, P6 = 6 * p;
  const i64 L = seg_len(s);
  if (seg_dir(s) == 0) {
    const i64 Y = 6 * q * s.cy - 3 * q;
    const i64 X0 = 6 * q * s.cx - 3 * q, X1 = X0 + 6 * q * L;
    const i64 j = strip_of(g, zq(Y));
    // at height Y the 60-degree lines sit at ox + 6p i + U sqrt3 and the
    // 120-degree lines at ox + 6p (k + j) - U sqrt3, U = (Y - oy) / 3; the
    // cell index is the number of lines of both families left of x
    const i64 U = (Y - oy) / 3;
    i64 c = zfloordiv(zq(X0 - ox, -U), P6) + zfloordiv(zq(X0 - ox - P6 * j, U), P6);
    const i64 cend = zfloordiv(zq(X1 - ox, -U), P6) + zfloordiv(zq(X1 - ox - P6 * j, U), P6);
    if (!f.cell(c, j)) return;
    while (c < cend) {
      const i64 i = c >> 1;
      if (!vid_ok(g, i + 1, j)) return f.fail();
      u32 e;
      Zq px;
      if ((c & 1) == 0) {  // up(i, j) is left through its 120-degree edge from v(i+1, j)
        e = 3u * vid(g, i + 1, j) + 2u;
        px = zq(ox + P6 * (i + 1 + j), -U);
      } else {  // down(i, j) is left through the 60-degree edge from v(i+1, j)
        e = 3u * vid(g, i + 1, j) + 1u;
        px = zq(ox + P6 * (i + 1), U);
      }
      if (!f.cross(e, px, zq(Y))) return;
      ++c;
      if (!f.cell(c, j)) return;
    }
    return;
  }
  const i64 X = 6 * q * s.cx - 3 * q;
  const i64 Y0 = 6 * q * s.cy - 3 * q, Y1 = Y0 + 6 * q * L;
  i64 j = strip_of(g, zq(Y0));
  const i64 U0 = (Y0 - oy) / 3;
  i64 c = zfloordiv(zq(X - ox, -U0), P6) + zfloordiv(zq(X - ox - P6 * j, U0), P6);
  if (!f.cell(c, j)) return;
  while (true) {
    // at the bottom of strip j the line x = X is inside up(ab, j); it leaves
    // that cell through the 60-degree edge from v(ab, j) left of the apex,
    // or the 120-degree edge from v(ab+1, j) right of it
    const i64 ab = ifloordiv(X - ox - 3 * p * j, P6);
    const i64 xab = ox + 3 * p * (2 * ab + j);
    Zq ys;
    u32 e;
    i64 upper;
    if (X - xab < 3 * p) {
      if (!vid_ok(g, ab, j)) return f.fail();
      ys = zq(oy, 3 * p * j + (X - xab));
      e = 3u * vid(g, ab, j) + 1u;
      upper = 2 * ab - 1;
    } else {
      if (!vid_ok(g, ab + 1, j)) return f.fail();
      ys = zq(oy, 3 * p * j + (xab + P6 - X));
      e = 3u * vid(g, ab + 1, j) + 2u;
      upper = 2 * ab + 1;
    }
    if (zcmp(ys, zq(Y0)) > 0) {
      if (zcmp(ys, zq(Y1)) >= 0) return;
      if (c != 2 * ab) return f.fail();
      if (!f.cross(e, zq(X), ys)) return;
      c = upper;
      if (!f.cell(c, j)) return;
    } else if (c != upper) {
      return f.fail();
    }
    // the horizontal edge on top of strip j, from v(ih, j+1)
    const Zq yt = zq(oy, 3 * p * (j + 1));
    if (zcmp(yt, zq(Y1)) >= 0) return;
    const i64 ih = ifloordiv(X - ox - 3 * p * (j + 1), P6);
    if (c != 2 * ih + 1 || !vid_ok(g, ih, j + 1)) return f.fail();
    e = 3u * vid(g, ih, j + 1) + 0u;
    if (!f.cross(e, zq(X), yt)) return;
    ++j;
    c = 2 * ih;
    if (!f.cell(c, j)) return;
  }
}

struct CountF {
  const GridP* g;
  u32 *pcnt, *ecnt, *err;
  u32 pb, pn, eb, en;
  unsigned long long np, ne;
  SBMT_DEV bool cell(i64 c, i64 j) {
    if (!cell_in(*g, c, j)) {
      fail();
      return false;
    }
    const u32 b = cell_id(*g, c, j) >> CB_LOG;
    if (b != pb) {
      if (pn) atomicAdd(pcnt + pb, pn);
      pb = b, pn = 0;
    }
    ++pn, ++np;
    return true;
  }
  SBMT_DEV bool cross(u32 e, Zq, Zq) {
    const u32 b = e >> EB_LOG;
    if (b != eb) {
      if (en) atomicAdd(ecnt + eb, en);
      eb = b, en = 0;
    }
    ++en, ++ne;
    return true;
  }
  SBMT_DEV void fail() { atomicOr(err, ERR_TRAVERSAL); }
  SBMT_DEV void flush() {
    if (pn) atomicAdd(pcnt + pb, pn);
    if (en) atomicAdd(ecnt + eb, en);
  }
};

struct EmitF {
  const GridP* g;
  u32 *pcur, *ecur, *err;
  Pair* pairs;
  Event* ev;
  u32 seg, cur, ev_in;
  SBMT_DEV bool cell(i64 c, i64 j) {
    if (!cell_in(*g, c, j)) {
      fail();
      return false;
    }
    cur = cell_id(*g, c, j);
    return true;
  }
  SBMT_DEV bool cross(u32 e, Zq px, Zq py) {
    const u32 slot = atomicAdd(ecur + (e >> EB_LOG), 1u);
    ev[slot] = Event{e, seg, 0u, 0u, (int)px.a, (int)px.b, (int)py.a, (int)py.b};
    const u32 ps = atomicAdd(pcur + (cur >> CB_LOG), 1u);
    pairs[ps] = Pair{cur, seg, ev_in, slot};
    ev_in = slot;
    return true;
  }
  SBMT_DEV void fail() {
    atomicOr(err, ERR_TRAVERSAL);
    cur = NONE;
  }
  SBMT_DEV void finish() {
    if (cur == NONE) return;
    const u32 ps = atomicAdd(pcur + (cur >> CB_LOG), 1u);
    pairs[ps] = Pair{cur, seg, ev_in, NONE};
  }
};

__global__ void k_traverse_count(GridP g, const Seg* segs, const u32* nseg, u32 cap, u32* pcnt, u32* ecnt,
                                 unsigned long long* totals, u32* err) {
  const u32 n = min(*nseg, cap);
  unsigned long long np = 0, ne = 0;
  for (u32 s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    CountF f{&g, pcnt, ecnt, err, NONE, 0u, NONE, 0u, 0ull, 0ull};
    walk_segment(g, segs[s], f);
    f.flush();
    np += f.np, ne += f.ne;
  }
  // warp-reduce the totals before the global atomics
  for (int o = 16; o; o >>= 1) {
    np += __shfl_down_sync(0xffffffffu, np, o);
    ne += __shfl_down_sync(0xffffffffu, ne, o);
  }
  if ((threadIdx.x & 31) == 0 && (np | ne)) {
    atomicAdd(totals + 0, np);
    atomicAdd(totals + 1, ne);
  }
}

__global__ void k_traverse_emit(GridP g, const Seg* segs, const u32* nseg, u32 cap, u32* pcur, u32* ecur,
                                Pair* pairs, Event* ev, u32* err) {
  const u32 n = min(*nseg, cap);
  for (u32 s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    EmitF f{&g, pcur, ecur, err, pairs, ev, s, NONE, NONE};
    walk_segment(g, segs[s], f);
    f.finish();
  }
}

SBMT_DEV Zq event_t(const Event& e) {
  // horizontal grid edges run +x from their lower endpoint, slanted ones +y
  return (e.edge % 3u == 0u) ? zq(e.xa, e.xb) : zq(e.ya, e.yb);
}

// The registry: one block per event bucket (2048 consecutive grid-edge ids).
// Events are counting-sorted by edge in shared memory; an event's vertex id
// is NVg + (events on lower edge ids) + (events on its edge nearer the
// edge's lower endpoint), compared exactly.
__global__ void __launch_bounds__(256) k_rank(GridP g, Event* ev, u32* elist, const u32* eoff, u32 NVg,
                                              double* xy) {
  constexpr int NEB = 1 << EB_LOG;
  __shared__ u32 s_cnt[NEB], s_off[NEB], s_cur[NEB];
  __shared__ u32 s_sh[8];
  const u32 lo = eoff[blockIdx.x], n = eoff[blockIdx.x + 1] - lo;
  if (n == 0) return;
  const u32 e0 = blockIdx.x << EB_LOG;
  for (int k = threadIdx.x; k < NEB; k += blockDim.x) s_cnt[k] = 0;
  __syncthreads();
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_cnt[ev[lo + i].edge - e0], 1u);
  __syncthreads();
  {
    constexpr int PER = NEB / 256;
    const int k0 = threadIdx.x * PER;
    u32 s = 0;
    for (int u = 0; u < PER; ++u) s += s_cnt[k0 + u];
    u32 tot;
    u32 run = block_exscan256(s, &tot, s_sh);
    for (int u = 0; u < PER; ++u) s_off[k0 + u] = run, s_cur[k0 + u] = run, run += s_cnt[k0 + u];
  }
  __syncthreads();
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
    const u32 slot = atomicAdd(&s_cur[ev[lo + i].edge - e0], 1u);
    elist[lo + slot] = i;
  }
  __syncthreads();
  const double invS = 1.0 / (double)g.S;
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
    const Event ei = ev[lo + i];
    const Zq ti = event_t(ei);
    const u32 k = ei.edge - e0, first = s_off[k], cnt = s_cnt[k];
    u32 rank = first;
    for (u32 q = 0; q < cnt; ++q) {
      const u32 j = elist[lo + first + q];
      if (j != i && zcmp(event_t(ev[lo + j]), ti) < 0) ++rank;
    }
    const u32 gid = NVg + lo + rank;
    ev[lo + i].gid = gid;
    double2 v;
    v.x = zdouble(zq(ei.xa, ei.xb)) * invS;
    v.y = zdouble(zq(ei.ya, ei.yb)) * invS;
    reinterpret_cast<double2*>(xy)[gid] = v;
  }
}

}  // namespace

void launch_traverse_count(const GridP& g, const Seg* segs, const u32* nseg, u32 seg_cap, u32* pcnt, u32* ecnt,
                           unsigned long long* totals, u32* err, cudaStream_t st) {
  const int blk = 256;
  const unsigned grd = (unsigned)std::max<u64>(1, std::min<u64>((seg_cap + blk - 1) / blk, 152u * 64u));
  k_traverse_count<<<grd, blk, 0, st>>>(g, segs, nseg, seg_cap, pcnt, ecnt, totals, err);
}

void launch_traverse_emit(const GridP& g, const Seg* segs, const u32* nseg, u32 seg_cap, u32* pcur, u32* ecur,
                          Pair* pairs, Event* events, u32* err, cudaStream_t st) {
  const int blk = 256;
  const unsigned grd = (unsigned)std::max<u64>(1, std::min<u64>((seg_cap + blk - 1) / blk, 152u * 64u));
  k_traverse_emit<<<grd, blk, 0, st>>>(g, segs, nseg, seg_cap, pcur, ecur, pairs, events, err);
}

void launch_rank_events(const GridP& g, Event* events, u32* elist, const u32* eoff, u32 nbe, u32 NVg, double* xy,
                        cudaStream_t st) {
  if (nbe == 0) return;
  k_rank<<<nbe, 256, 0, st>>>(g, events, elist, eoff, NVg, xy);
}

}  // namespace sbmt
