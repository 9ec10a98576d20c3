// k_cells.cu -- K3 classification, canonical key and lookup; K4 emission of
// the conforming mesh (uncut cells, Tier-T patches) and K4-G (Tier-G cells).
//
// Sec. 3.3.2: a cut base triangle K is described by the Alg. 1 events on its
// edges (bitmask AB=2, BC=4, CA=8 per segment, (m,n) = per-segment counts)
// and the boundary vertices inside it.  Sec. 3.3.3: its key kappa(K) is
// canonicalised under the three rotations of K and looked up in a
// single-valued table (Assumption "frozen registry and single-valued
// lookup"); Alg. 2 instantiates the stored template by mapping canonical
// labels to actual points, pre-composed with the rotation.  Lemma 3.1's regime
// (at most two chords, or one boundary vertex whose segments all leave K) is
// the table's domain ("Tier-T"); a cell outside it ("Tier-G": pixel-staircase
// runs shorter than the grid edge) takes the greedy triangulation of its
// local boundary graph: every vertex pair in order of exact length, kept when
// it crosses nothing.  Uncut cells keep their base triangle (A, B, C).
#include <algorithm>

#include "sbmt_launch.h"

namespace sbmt {

namespace {

// ---------------------------------------------------------------------------
// lookup table (App. G), canonical frame: labels 0,1,2 = A', B', C';
// 3..6 = E0..E3, the events read counter-clockwise from A'; 7 = P
// ---------------------------------------------------------------------------
enum { TA = 0, TB = 1, TC = 2, T0 = 3, T1 = 4, T2 = 5, T3 = 6, TP = 7 };
constexpr int NKEYS = 15;
// canonical code star<<10 | n(A'B')<<7 | n(B'C')<<4 | n(C'A')<<1 | dir of keys 1..15
__constant__ unsigned short c_key_code[NKEYS] = {
    (0 << 10) | (0 << 7) | (1 << 4) | (1 << 1) | 0,  // 1 single segment (b)
    (1 << 10) | (0 << 7) | (1 << 4) | (1 << 1) | 0,  // 2 (1,1) (a)
    (1 << 10) | (0 << 7) | (0 << 4) | (2 << 1) | 0,  // 3 (1,1) (c)
    (0 << 10) | (1 << 7) | (1 << 4) | (2 << 1) | 0,  // 4 (2,2) (b1)
    (0 << 10) | (0 << 7) | (2 << 4) | (2 << 1) | 1,  // 5 (2,2) (d3)
    (0 << 10) | (0 << 7) | (2 << 4) | (2 << 1) | 0,  // 6 (2,2) (a4)
    (1 << 10) | (0 << 7) | (0 << 4) | (3 << 1),      // 7..15: one vertex of degree 3-4,
    (1 << 10) | (0 << 7) | (1 << 4) | (2 << 1),      //   star from P
    (1 << 10) | (0 << 7) | (2 << 4) | (1 << 1),
    (1 << 10) | (1 << 7) | (1 << 4) | (1 << 1),
    (1 << 10) | (0 << 7) | (0 << 4) | (4 << 1),
    (1 << 10) | (0 << 7) | (1 << 4) | (3 << 1),
    (1 << 10) | (0 << 7) | (2 << 4) | (2 << 1),
    (1 << 10) | (0 << 7) | (3 << 4) | (1 << 1),
    (1 << 10) | (1 << 7) | (1 << 4) | (2 << 1),
};
// templates of the paper's keys 1..6, in App. G's order
__constant__ unsigned char c_tpl[6][5][3] = {
    // single segment (b): Q1 on B'C' (E0), Q2 on C'A' (E1)
    {{T1, T0, TC}, {T1, TA, TB}, {T0, T1, TB}, {0, 0, 0}, {0, 0, 0}},
    // (1,1) (a): Q2 on B'C' (E0), Q1 on C'A' (E1), P inside
    {{T1, TP, TC}, {TP, T0, TC}, {T1, TA, TP}, {TA, TB, TP}, {T0, TP, TB}},
    // (1,1) (c): Q1, Q2 on C'A', Q1 nearer C' (E0 = Q1, E1 = Q2)
    {{T0, TP, TC}, {TP, T0, T1}, {T1, TA, TP}, {TB, TC, TP}, {TA, TB, TP}},
    // (2,2) (b1): Q1 on A'B' (E0), Q3 on B'C' (E1), Q4 (E2) and Q2 (E3) on C'A'
    {{T0, T3, TA}, {T0, T2, T3}, {T0, T1, T2}, {T0, TB, T1}, {T2, T1, TC}},
    // (2,2) (d3): nested chords at C'; Q4 (E0), Q3 (E1) on B'C'; Q1 (E2), Q2 (E3) on C'A'
    {{TA, TB, T3}, {T3, TB, T0}, {T2, T3, T0}, {T2, T0, T1}, {T2, T1, TC}},
    // (2,2) (a4), drawn at A and turned so the cut corner is C': Q2 (E0), Q1 (E1)
    // on B'C'; Q3 (E2), Q4 (E3) on C'A'
    {{T2, T1, TC}, {T3, T1, T2}, {T1, T3, T0}, {T0, T3, TA}, {T0, TA, TB}},
};

SBMT_DEV int thm32_class(int m, int n) {
  // 1-based position of the sorted pair in Thm. 3.2's list, 0 if absent
  if (m > n) {
    int t = m;
    m = n, n = t;
  }
  const int lst[8] = {0 * 4 + 1, 0 * 4 + 2, 0 * 4 + 3, 1 * 4 + 1, 1 * 4 + 2, 2 * 4 + 2, 1 * 4 + 3, 2 * 4 + 3};
  for (int k = 0; k < 8; ++k)
    if (lst[k] == m * 4 + n) return k + 1;
  return 0;
}

// ---------------------------------------------------------------------------
// cell geometry
// ---------------------------------------------------------------------------
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
SBMT_DEV int local_edge(const CellGeo& cg, u32 e) {
  return cg.edge[0] == e ? 0 : cg.edge[1] == e ? 1 : cg.edge[2] == e ? 2 : -1;
}
// a number increasing counter-clockwise along local edge k (corner k -> k+1):
// up cells run AB +x, BC +y, CA -y; down cells AB +y, BC -x, CA -y
SBMT_DEV Zq ccw_pos(int down, int k, const Event& e) {
  if (k == 2) return zq(-e.ya, -e.yb);
  if (down == 0) return k == 0 ? zq(e.xa, e.xb) : zq(e.ya, e.yb);
  return k == 0 ? zq(e.ya, e.yb) : zq(-e.xa, -e.xb);
}
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

// label of the pixel holding the centroid of three global points
template <typename T>
SBMT_DEV unsigned short centroid_label(const GridP& g, const unsigned char* img, i64 pitch, const Pq& a,
                                       const Pq& b, const Pq& c) {
  const Zq sx = a.x + b.x + c.x, sy = a.y + b.y + c.y;
  // pixel column floor(x/S + 1/2) with x = sx / 3
  const i64 col = zfloordiv(Zq{2 * sx.a + 3 * g.S, 2 * sx.b}, 6 * g.S);
  const i64 row = zfloordiv(Zq{2 * sy.a + 3 * g.S, 2 * sy.b}, 6 * g.S);
  const int l = pix<T>(img, pitch, g.W, g.H, col, row);
  return l == OUTSIDE ? (unsigned short)0xFFFF : (unsigned short)l;
}
SBMT_DEV unsigned short label_of(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pq& a,
                                 const Pq& b, const Pq& c) {
  return dtype == 1 ? centroid_label<unsigned char>(g, img, pitch, a, b, c)
                    : centroid_label<unsigned short>(g, img, pitch, a, b, c);
}

// ---------------------------------------------------------------------------
// K3 classification of one cut cell from its (cell, segment) pairs
// ---------------------------------------------------------------------------
struct Klass {
  u32 code, ntri, nchain;
  bool tierG;
};

SBMT_DEV Klass classify_cell(const GridP& g, const CellGeo& cg, const Pair* P, u32 np, const Seg* segs,
                             const Event* ev, u32* err) {
  int nev[3] = {0, 0, 0};
  u32 mask = 0, nchain = 0;
  bool all_one_inside = true;
  int pin[2] = {-1, -1}, pout[2] = {-1, -1};  // local edges of the walk-order ends (Tier-T chords)
  u32 ein_ev[2] = {NONE, NONE}, eout_ev[2] = {NONE, NONE};
  int prev[2] = {0, 0}, mcount[2] = {0, 0};
  for (u32 k = 0; k < np; ++k) {
    const Pair pr = P[k];
    const Seg s = segs[pr.seg];
    int inside = 0, m = 0;
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e != NONE) {
        const int le = local_edge(cg, ev[e].edge);
        if (le < 0) {
          atomicOr(err, ERR_TRAVERSAL);
          continue;
        }
        nev[le]++;
        mask |= 2u << le;
        ++m;
        if (k < 2) (end == 0 ? pin[k] : pout[k]) = le;
        continue;
      }
      ++inside;
      // count each inside corner once: skip it if an earlier pair ends there
      const u32 id = corner_id(g, s, end);
      bool seen = false;
      for (u32 k2 = 0; k2 < k && !seen; ++k2) {
        const Pair q = P[k2];
        const Seg s2 = segs[q.seg];
        if (q.ev_in == NONE && corner_id(g, s2, 0) == id) seen = true;
        if (q.ev_out == NONE && corner_id(g, s2, 1) == id) seen = true;
      }
      if (!seen) ++nchain;
    }
    if (inside != 1) all_one_inside = false;
    if (k < 2) {
      ein_ev[k] = pr.ev_in, eout_ev[k] = pr.ev_out, prev[k] = seg_rev(s), mcount[k] = m;
    }
  }
  Klass r;
  r.nchain = nchain;
  r.ntri = 2 * nchain + 1 + (u32)(nev[0] + nev[1] + nev[2]);
  if (nchain) mask |= 1u;
  const int klass = np == 1 ? thm32_class(0, mcount[0]) : np == 2 ? thm32_class(mcount[0], mcount[1]) : 0;
  const bool chords = nchain == 0 && (np == 1 || np == 2);
  const bool star = nchain == 1 && all_one_inside && np >= 2 && np <= 4;
  if (!chords && !star) {
    r.tierG = true;
    r.code = (mask & 15u) | (63u << 6) | ((u32)klass << 12);
    return r;
  }
  int dir = 0;
  if (chords && np == 2) {
    int X[2];
    for (int k = 0; k < 2; ++k) X[k] = (pout[k] == (pin[k] + 1) % 3) ? pout[k] : pin[k];
    if (X[0] == X[1]) {
      // nested chords at corner X: the chord nearer X meets the edge ending
      // at X later in counter-clockwise order
      const int ein = (X[0] + 2) % 3, eout = X[0];
      Zq pos[2];
      for (int k = 0; k < 2; ++k) {
        const u32 e = pin[k] == ein ? ein_ev[k] : eout_ev[k];
        pos[k] = ccw_pos(cg.down, ein, ev[e]);
      }
      const int near = zcmp(pos[0], pos[1]) > 0 ? 0 : 1;
      // the chord's own direction: the walk runs in -> out, reversed if rev
      const int first = prev[near] ? pout[near] : pin[near];
      const int second = prev[near] ? pin[near] : pout[near];
      dir = (first == ein && second == eout) ? 1 : 0;
    }
  }
  const int st = star ? 1 : 0;
  int best = -1, sigma = 0;
  for (int rr = 0; rr < 3; ++rr) {
    const int code = (st << 10) | (nev[rr] << 7) | (nev[(rr + 1) % 3] << 4) | (nev[(rr + 2) % 3] << 1) | dir;
    if (best < 0 || code < best) best = code, sigma = rr;
  }
  int key = 0;
  for (int k = 0; k < NKEYS; ++k)
    if (c_key_code[k] == best) key = k + 1;
  if (key == 0) {  // structure in the regime but no table entry: treat as Tier-G
    r.tierG = true;
    r.code = (mask & 15u) | (63u << 6) | ((u32)klass << 12);
    return r;
  }
  r.tierG = false;
  r.code = (mask & 15u) | ((u32)sigma << 4) | ((u32)key << 6) | ((u32)klass << 12);
  return r;
}

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------
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

constexpr int KCAP = 2048;

__global__ void __launch_bounds__(256) k_classify(GridP g, const Pair* pairs, Pair* sorted, const u32* poff,
                                                  const Seg* segs, const Event* ev, CutRec* recs, u32* bstat,
                                                  u32* err) {
  __shared__ unsigned long long s_key[KCAP];
  __shared__ u32 s_sh[8];
  __shared__ u32 s_stat[4];
  const u32 b = blockIdx.x, lo = poff[b], n = poff[b + 1] - lo;
  if (threadIdx.x < 4) s_stat[threadIdx.x] = 0;
  if (n == 0) {
    if (threadIdx.x < 4) bstat[4 * b + threadIdx.x] = 0;
    return;
  }
  // 1. order the bucket's pairs by (cell, segment): rank sort
  const bool cached = n <= (u32)KCAP;
  if (cached)
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
      const Pair p = pairs[lo + i];
      s_key[i] = ((unsigned long long)p.cell << 32) | p.seg;
    }
  __syncthreads();
  for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
    const Pair p = pairs[lo + i];
    const unsigned long long ki = ((unsigned long long)p.cell << 32) | p.seg;
    u32 rank = 0;
    for (u32 k = 0; k < n; ++k) {
      unsigned long long kk;
      if (cached) kk = s_key[k];
      else {
        const Pair q = pairs[lo + k];
        kk = ((unsigned long long)q.cell << 32) | q.seg;
      }
      rank += kk < ki ? 1u : 0u;
    }
    sorted[lo + rank] = p;
  }
  __syncthreads();
  // 2. one record per cell: a pair starts a cell when its cell differs from
  //    the previous pair's
  u32 carry = 0, st_cut = 0, st_extra = 0, st_chain = 0, st_g = 0;
  int row = -1;
  for (u32 base = 0; base < n; base += blockDim.x) {
    const u32 i = base + threadIdx.x;
    bool start = false;
    Pair p{};
    if (i < n) {
      p = sorted[lo + i];
      start = (i == 0) || (sorted[lo + i - 1].cell != p.cell);
    }
    u32 tot;
    const u32 idx = block_exscan256(start ? 1u : 0u, &tot, s_sh);
    if (start) {
      u32 np = 1;
      while (i + np < n && sorted[lo + i + np].cell == p.cell) ++np;
      if (row < 0 || !(g.cbase[row] <= (i64)p.cell && (row + 1 == g.nrows || g.cbase[row + 1] > (i64)p.cell)))
        row = cell_row(g, p.cell);
      const CellGeo cg = cell_geo(g, p.cell, row);
      const Klass k = classify_cell(g, cg, sorted + lo + i, np, segs, ev, err);
      CutRec rec{p.cell, lo + i, np, k.code | (k.tierG ? (1u << 16) : 0u), k.ntri, k.nchain, 0u, 0u};
      recs[lo + carry + idx] = rec;
      st_cut += 1, st_extra += k.ntri - 1, st_chain += k.nchain, st_g += k.tierG ? 1u : 0u;
    }
    carry += tot;
  }
  atomicAdd(&s_stat[0], st_cut);
  atomicAdd(&s_stat[1], st_extra);
  atomicAdd(&s_stat[2], st_chain);
  atomicAdd(&s_stat[3], st_g);
  __syncthreads();
  if (threadIdx.x < 4) bstat[4 * b + threadIdx.x] = s_stat[threadIdx.x];
}

// exclusive scan over n strided values, one block of 1024 threads
__global__ void __launch_bounds__(1024) k_scan(const u32* in, int stride, u32* out, u32 n) {
  __shared__ u32 sh[1024];
  const u32 t = threadIdx.x;
  const u32 chunk = (n + 1023) / 1024;
  const u32 a = min(n, t * chunk), e = min(n, a + chunk);
  u32 s = 0;
  for (u32 i = a; i < e; ++i) s += in[(u64)i * stride];
  sh[t] = s;
  __syncthreads();
  for (u32 o = 1; o < 1024; o <<= 1) {
    const u32 v = t >= o ? sh[t - o] : 0u;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  u32 run = sh[t] - s;
  for (u32 i = a; i < e; ++i) {
    const u32 v = in[(u64)i * stride];
    out[i] = run;
    run += v;
  }
  if (t == 1023) out[n] = sh[1023];
}

// ---------------------------------------------------------------------------
// K4: emission
// ---------------------------------------------------------------------------
// Tier-T patch: events in counter-clockwise order from A, the template of the
// key read through sigma (Alg. 2 "instantiate by a single map")
SBMT_DEV void emit_tier_t(const GridP& g, const CellGeo& cg, const CutRec& rec, const Pair* P, const Seg* segs,
                          const Event* ev, const unsigned char* img, i64 pitch, int dtype, int* tri,
                          unsigned short* label, unsigned short* code, double* xy, u32* err) {
  // local vertices: 0..2 corners, then up to 4 events, then P
  Pq pt[8];
  u32 gid[8];
  for (int k = 0; k < 3; ++k) {
    pt[k] = lattice_pt(g, cg.ci[k], cg.cj[k]);
    gid[k] = vid(g, cg.ci[k], cg.cj[k]);
  }
  u32 evs[4];
  int evk[4];
  Zq evp[4];
  int ne = 0;
  u32 pcorner = NONE;
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e == NONE) {
        pcorner = corner_id(g, segs[pr.seg], end);
        continue;
      }
      if (ne >= 4) {
        atomicOr(err, ERR_COUNT);
        return;
      }
      const int le = local_edge(cg, ev[e].edge);
      if (le < 0) {
        atomicOr(err, ERR_TRAVERSAL);
        return;
      }
      evs[ne] = e, evk[ne] = le, evp[ne] = ccw_pos(cg.down, le, ev[e]);
      ++ne;
    }
  }
  // order events by (edge, counter-clockwise position)
  for (int a = 1; a < ne; ++a)
    for (int b = a; b > 0; --b) {
      const bool sw = evk[b] < evk[b - 1] || (evk[b] == evk[b - 1] && zcmp(evp[b], evp[b - 1]) < 0);
      if (!sw) break;
      u32 te = evs[b];
      evs[b] = evs[b - 1], evs[b - 1] = te;
      int tk = evk[b];
      evk[b] = evk[b - 1], evk[b - 1] = tk;
      Zq tp = evp[b];
      evp[b] = evp[b - 1], evp[b - 1] = tp;
    }
  for (int k = 0; k < ne; ++k) {
    const Event e = ev[evs[k]];
    pt[3 + k] = Pq{zq(e.xa, e.xb), zq(e.ya, e.yb)};
    gid[3 + k] = e.gid;
  }
  const int key = (int)((rec.code >> 6) & 63u), sigma = (int)((rec.code >> 4) & 3u);
  const int P_ = 3 + ne;
  if (rec.nchain == 1) {
    pt[P_] = corner_of_id(g, pcorner);
    gid[P_] = rec.chain_base;
    xy[2 * (i64)rec.chain_base] = zdouble(pt[P_].x) / (double)g.S;
    xy[2 * (i64)rec.chain_base + 1] = zdouble(pt[P_].y) / (double)g.S;
  }
  // canonical label -> local vertex
  int map[8];
  for (int k = 0; k < 3; ++k) map[k] = (sigma + k) % 3;
  int nin[3] = {0, 0, 0};
  for (int k = 0; k < ne; ++k) nin[evk[k]]++;
  int t = 0;
  for (int s = 0; s < 3; ++s) {
    const int e = (sigma + s) % 3;
    int first = 3;
    for (int u = 0; u < e; ++u) first += nin[u];
    for (int u = 0; u < nin[e]; ++u) map[3 + t++] = first + u;
  }
  for (int k = t; k < 4; ++k) map[3 + k] = -1;
  map[TP] = rec.nchain == 1 ? P_ : -1;
  const unsigned short cd = (unsigned short)(rec.code & 0xFFFFu);
  u32 out = rec.tri_off;
  auto put = [&](int la, int lb, int lc) {
    const int a = map[la], b = map[lb], c = map[lc];
    tri[3 * (i64)out] = (int)gid[a];
    tri[3 * (i64)out + 1] = (int)gid[b];
    tri[3 * (i64)out + 2] = (int)gid[c];
    label[out] = label_of(g, img, pitch, dtype, pt[a], pt[b], pt[c]);
    code[out] = cd;
    ++out;
  };
  if (key <= 6) {
    const int nt = key == 1 ? 3 : 5;
    for (int k = 0; k < nt; ++k) put(c_tpl[key - 1][k][0], c_tpl[key - 1][k][1], c_tpl[key - 1][k][2]);
  } else {
    // star from P over the boundary cycle read counter-clockwise from A'
    int cyc[8], nc = 0, ev_i = 0;
    for (int s = 0; s < 3; ++s) {
      cyc[nc++] = s;
      const int e = (sigma + s) % 3;
      for (int u = 0; u < nin[e]; ++u) cyc[nc++] = T0 + ev_i++;
    }
    for (int k = 0; k < nc; ++k) put(cyc[k], cyc[(k + 1) % nc], TP);
  }
  if (out != rec.tri_off + rec.ntri) atomicOr(err, ERR_COUNT);
}

__global__ void __launch_bounds__(256) k_emit(GridP g, const unsigned char* img, i64 pitch, int dtype,
                                              const Pair* sorted, const Seg* segs, const Event* ev, CutRec* recs,
                                              const u32* poff, const u32* bstat, const u32* extra_scan,
                                              const u32* chain_scan, u32 NVg, u32 NE, int* tri,
                                              unsigned short* label, unsigned short* code, double* xy, u32* glist,
                                              u32* nglist, u32* ngtri, u32* err) {
  constexpr int NB = 1 << CB_LOG;
  __shared__ u32 s_cnt[NB];
  __shared__ u32 s_off[NB];
  __shared__ u32 s_cb[NB];
  __shared__ u32 s_sh[8];
  const u32 b = blockIdx.x;
  const i64 c0 = (i64)b << CB_LOG;
  const int nc = (int)min((i64)NB, g.ncells - c0);
  const u32 ncut = bstat[4 * b], rec0 = poff[b];
  for (int k = threadIdx.x; k < NB; k += blockDim.x) s_cnt[k] = k < nc ? 1u : 0u;
  __syncthreads();
  for (u32 r = threadIdx.x; r < ncut; r += blockDim.x) {
    const CutRec rec = recs[rec0 + r];
    s_cnt[rec.cell - c0] = rec.ntri;
  }
  __syncthreads();
  // exclusive scan of the bucket's triangle counts (4 cells per thread) and
  // of the records' inside-vertex counts
  {
    const int k0 = threadIdx.x * 4;
    u32 v[4], s = 0;
    for (int u = 0; u < 4; ++u) v[u] = s_cnt[k0 + u], s += v[u];
    u32 tot;
    u32 run = block_exscan256(s, &tot, s_sh);
    for (int u = 0; u < 4; ++u) s_off[k0 + u] = run, run += v[u];
  }
  {
    u32 carry = 0;
    for (u32 base = 0; base < ncut; base += blockDim.x) {
      const u32 r = base + threadIdx.x;
      const u32 v = r < ncut ? recs[rec0 + r].nchain : 0u;
      u32 tot;
      const u32 ex = block_exscan256(v, &tot, s_sh);
      if (r < ncut) s_cb[r] = carry + ex;
      carry += tot;
    }
  }
  __syncthreads();
  const u32 T0_ = (u32)c0 + extra_scan[b];
  const u32 CB0 = NVg + NE + chain_scan[b];
  // uncut cells: the base triangle (A, B, C), untouched
  int row = cell_row(g, (u32)c0);
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    if (s_cnt[k] != 1u) continue;
    const u32 cid = (u32)(c0 + k);
    int r = row;
    while (r + 1 < g.nrows && g.cbase[r + 1] <= (i64)cid) ++r;
    const i64 j = g.j0 + r, c = g.clo[r] + ((i64)cid - g.cbase[r]);
    i64 ci[3], cj[3];
    cell_corners(c, j, ci, cj);
    const u32 o = T0_ + s_off[k];
    Pq pt[3];
    for (int u = 0; u < 3; ++u) {
      tri[3 * (i64)o + u] = (int)vid(g, ci[u], cj[u]);
      pt[u] = lattice_pt(g, ci[u], cj[u]);
    }
    label[o] = label_of(g, img, pitch, dtype, pt[0], pt[1], pt[2]);
    code[o] = 0;
  }
  // cut cells
  for (u32 r = threadIdx.x; r < ncut; r += blockDim.x) {
    CutRec rec = recs[rec0 + r];
    rec.tri_off = T0_ + s_off[rec.cell - c0];
    rec.chain_base = CB0 + s_cb[r];
    if (rec.code & (1u << 16)) {
      recs[rec0 + r] = rec;
      const u32 slot = atomicAdd(nglist, 1u);
      glist[slot] = rec0 + r;
      atomicAdd(ngtri, rec.ntri);
      continue;
    }
    const CellGeo cg = cell_geo(g, rec.cell, cell_row(g, rec.cell));
    emit_tier_t(g, cg, rec, sorted + rec.pair_lo, segs, ev, img, pitch, dtype, tri, label, code, xy, err);
  }
}

// ---------------------------------------------------------------------------
// K4-G: one warp per Tier-G cell
// ---------------------------------------------------------------------------
constexpr int GN = 64;                  // local vertices per cell
constexpr int GWARPS = 4;               // warps per block
constexpr int GCAND = GN * (GN - 1) / 2;
constexpr int GCANDP = 2048;            // power of two >= GCAND
constexpr int GEDGE = 3 * GN;
constexpr int GTRI = 2 * GN;

struct GShared {
  int xa[GN], xb[GN], ya[GN], yb[GN];  // cell-local exact coordinates
  u32 gid[GN];
  u32 corner[GN];
  u64 adj[GN];
  unsigned short cand[GCANDP];
  unsigned short edge[GEDGE];
  u32 tri[GTRI];
  int n, nedge, ntri, ok;
};

SBMT_DEV Pq lpt(const GShared& s, int k) { return Pq{zq(s.xa[k], s.xb[k]), zq(s.ya[k], s.yb[k])}; }
SBMT_DEV Zq len2(const GShared& s, int u, int v) {
  const Zq dx = zq(s.xa[v] - s.xa[u], s.xb[v] - s.xb[u]), dy = zq(s.ya[v] - s.ya[u], s.yb[v] - s.yb[u]);
  return dx * dx + dy * dy;
}
// candidate order: exact squared length, then (u, v)
SBMT_DEV bool cand_less(const GShared& s, unsigned short x, unsigned short y) {
  if (x == 0xFFFFu) return false;
  if (y == 0xFFFFu) return true;
  const int c = zcmp(len2(s, x >> 8, x & 255), len2(s, y >> 8, y & 255));
  if (c != 0) return c < 0;
  return x < y;
}
SBMT_DEV Zq dot3(const Pq& o, const Pq& p, const Pq& q) { return (p.x - o.x) * (q.x - o.x) + (p.y - o.y) * (q.y - o.y); }

// build the cell's local boundary graph (lane 0): corners, events in
// counter-clockwise order, inside vertices by corner id, constraint edges
SBMT_DEV void build_local_g(const GridP& g, const CellGeo& cg, const CutRec& rec, const Pair* P, const Seg* segs,
                            const Event* ev, GShared& s) {
  const Pq A = lattice_pt(g, cg.ci[0], cg.cj[0]);
  s.ok = 1;
  s.nedge = 0;
  for (int k = 0; k < GN; ++k) s.adj[k] = 0;
  for (int k = 0; k < 3; ++k) {
    const Pq p = lattice_pt(g, cg.ci[k], cg.cj[k]);
    s.xa[k] = (int)(p.x.a - A.x.a), s.xb[k] = (int)(p.x.b - A.x.b);
    s.ya[k] = (int)(p.y.a - A.y.a), s.yb[k] = (int)(p.y.b - A.y.b);
    s.gid[k] = vid(g, cg.ci[k], cg.cj[k]);
    s.corner[k] = NONE;
  }
  // events, sorted by (edge, position); their slots hold the event index
  int ne = 0;
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e == NONE) continue;
      if (3 + ne >= GN) {
        s.ok = 0;
        return;
      }
      if (local_edge(cg, ev[e].edge) < 0) {
        s.ok = 0;
        return;
      }
      s.corner[3 + ne] = e;  // temporarily: event index
      ++ne;
    }
  }
  for (int a = 1; a < ne; ++a)
    for (int b = a; b > 0; --b) {
      const Event x = ev[s.corner[3 + b]], y = ev[s.corner[3 + b - 1]];
      const int kx = local_edge(cg, x.edge), ky = local_edge(cg, y.edge);
      const bool sw = kx < ky || (kx == ky && zcmp(ccw_pos(cg.down, kx, x), ccw_pos(cg.down, ky, y)) < 0);
      if (!sw) break;
      const u32 t = s.corner[3 + b];
      s.corner[3 + b] = s.corner[3 + b - 1], s.corner[3 + b - 1] = t;
    }
  int nev[3] = {0, 0, 0};
  for (int k = 0; k < ne; ++k) {
    const Event e = ev[s.corner[3 + k]];
    nev[local_edge(cg, e.edge)]++;
    s.xa[3 + k] = (int)(e.xa - A.x.a), s.xb[3 + k] = (int)(e.xb - A.x.b);
    s.ya[3 + k] = (int)(e.ya - A.y.a), s.yb[3 + k] = (int)(e.yb - A.y.b);
    s.gid[3 + k] = e.gid;
  }
  // inside vertices: distinct corner ids, ascending
  int n = 3 + ne;
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    for (int end = 0; end < 2; ++end) {
      if ((end == 0 ? pr.ev_in : pr.ev_out) != NONE) continue;
      const u32 id = corner_id(g, segs[pr.seg], end);
      int pos = 3 + ne;
      while (pos < n && s.corner[pos] < id) ++pos;
      if (pos < n && s.corner[pos] == id) continue;
      if (n >= GN) {
        s.ok = 0;
        return;
      }
      for (int t = n; t > pos; --t) s.corner[t] = s.corner[t - 1];
      s.corner[pos] = id;
      ++n;
    }
  }
  if ((u32)(n - 3 - ne) != rec.nchain) {
    s.ok = 0;
    return;
  }
  for (int k = 3 + ne; k < n; ++k) {
    const Pq p = corner_of_id(g, s.corner[k]);
    s.xa[k] = (int)(p.x.a - A.x.a), s.xb[k] = (int)(p.x.b - A.x.b);
    s.ya[k] = (int)(p.y.a - A.y.a), s.yb[k] = (int)(p.y.b - A.y.b);
    s.gid[k] = rec.chain_base + (u32)(k - 3 - ne);
  }
  s.n = n;
  auto add_edge = [&](int u, int v) {
    if (u > v) {
      int t = u;
      u = v, v = t;
    }
    if ((s.adj[u] >> v) & 1ull) return;
    s.adj[u] |= 1ull << v, s.adj[v] |= 1ull << u;
    s.edge[s.nedge++] = (unsigned short)((u << 8) | v);
  };
  // boundary cycle A, events on AB, B, events on BC, C, events on CA
  {
    int cyc[GN], nc = 0, e = 3;
    for (int k = 0; k < 3; ++k) {
      cyc[nc++] = k;
      for (int t = 0; t < nev[k]; ++t) cyc[nc++] = e++;
    }
    for (int k = 0; k < nc; ++k) add_edge(cyc[k], cyc[(k + 1) % nc]);
  }
  // chain pieces
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    int ends[2];
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      int loc = -1;
      if (e != NONE) {
        for (int t = 0; t < ne; ++t)
          if (s.corner[3 + t] == e) loc = 3 + t;
      } else {
        const u32 id = corner_id(g, segs[pr.seg], end);
        for (int t = 3 + ne; t < n; ++t)
          if (s.corner[t] == id) loc = t;
      }
      ends[end] = loc;
    }
    if (ends[0] < 0 || ends[1] < 0) {
      s.ok = 0;
      return;
    }
    add_edge(ends[0], ends[1]);
  }
  // the chain vertices' coordinates are written by their cell
}

__global__ void __launch_bounds__(32 * GWARPS) k_tierg(GridP g, const unsigned char* img, i64 pitch, int dtype,
                                                       const Pair* sorted, const Seg* segs, const Event* ev,
                                                       const CutRec* recs, const u32* glist, const u32* nglist,
                                                       u32 NVg, u32 NE, int* tri, unsigned short* label,
                                                       unsigned short* code, double* xy, u32* err) {
  __shared__ GShared sm[GWARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  GShared& s = sm[w];
  const u32 total = *nglist;
  for (u32 item = blockIdx.x * GWARPS + w; item < total; item += gridDim.x * GWARPS) {
    const CutRec rec = recs[glist[item]];
    const CellGeo cg = cell_geo(g, rec.cell, cell_row(g, rec.cell));
    if (lane == 0) build_local_g(g, cg, rec, sorted + rec.pair_lo, segs, ev, s);
    __syncwarp();
    if (!s.ok) {
      if (lane == 0) atomicOr(err, ERR_CAPACITY);
      __syncwarp();
      continue;
    }
    const int n = s.n;
    const Pq A = lattice_pt(g, cg.ci[0], cg.cj[0]);
    // candidate pairs not joined by a constraint edge
    int m = 0;
    for (int u = 0; u < n; ++u)
      for (int vb = u + 1; vb < n; vb += 32) {
        const int v = vb + lane;
        const bool ok = v < n && !((s.adj[u] >> v) & 1ull);
        const u32 bal = __ballot_sync(0xffffffffu, ok);
        if (ok) s.cand[m + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)((u << 8) | v);
        m += __popc(bal);
      }
    int M = 1;
    while (M < m) M <<= 1;
    for (int k = m + lane; k < M; k += 32) s.cand[k] = 0xFFFFu;
    __syncwarp();
    // bitonic sort of the candidates
    for (int kk = 2; kk <= M; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < M; i += 32) {
          const int l = i ^ jj;
          if (l > i) {
            const unsigned short x = s.cand[i], y = s.cand[l];
            const bool up = (i & kk) == 0;
            if (up ? cand_less(s, y, x) : cand_less(s, x, y)) s.cand[i] = y, s.cand[l] = x;
          }
        }
        __syncwarp();
      }
    // greedy: keep a pair when its open segment holds no vertex and crosses
    // no kept edge
    const int nb = 3 + (int)(rec.ntri + 2 - 2 * rec.nchain - 3);  // boundary vertices
    const int max_edges = 3 * n - nb - 3;
    for (int ci = 0; ci < m && s.nedge < max_edges; ++ci) {
      const int u = s.cand[ci] >> 8, v = s.cand[ci] & 255;
      const Pq pu = lpt(s, u), pv = lpt(s, v);
      bool bad = false;
      for (int k = lane; k < n; k += 32) {
        if (k == u || k == v) continue;
        const Pq pk = lpt(s, k);
        if (orient3(pu, pv, pk) == 0 && zsign(dot3(pu, pv, pk)) > 0 && zsign(dot3(pv, pu, pk)) > 0) bad = true;
      }
      const int ned = s.nedge;
      for (int k = lane; k < ned && !bad; k += 32) {
        const int a = s.edge[k] >> 8, bb = s.edge[k] & 255;
        if (a == u || a == v || bb == u || bb == v) continue;
        const Pq pa = lpt(s, a), pb = lpt(s, bb);
        const int o1 = orient3(pu, pv, pa), o2 = orient3(pu, pv, pb);
        const int o3 = orient3(pa, pb, pu), o4 = orient3(pa, pb, pv);
        if (o1 * o2 < 0 && o3 * o4 < 0) bad = true;
      }
      if (!__any_sync(0xffffffffu, bad)) {
        if (lane == 0) {
          s.adj[u] |= 1ull << v, s.adj[v] |= 1ull << u;
          s.edge[s.nedge] = (unsigned short)((u << 8) | v);
          s.nedge = s.nedge + 1;
        }
      }
      __syncwarp();
    }
    // faces: 3-cycles with no vertex strictly inside
    if (lane == 0) s.ntri = 0;
    __syncwarp();
    for (int u = lane; u < n; u += 32) {
      for (u64 vs = s.adj[u] & ~((2ull << u) - 1ull); vs; vs &= vs - 1) {
        const int v = __ffsll((long long)vs) - 1;
        for (u64 ws = s.adj[u] & s.adj[v] & ~((2ull << v) - 1ull); ws; ws &= ws - 1) {
          const int x = __ffsll((long long)ws) - 1;
          const Pq a = lpt(s, u), b = lpt(s, v), c = lpt(s, x);
          const int o = orient3(a, b, c);
          if (o == 0) continue;
          bool empty = true;
          for (int k = 0; k < n && empty; ++k) {
            if (k == u || k == v || k == x) continue;
            const Pq pk = lpt(s, k);
            if (orient3(a, b, pk) == o && orient3(b, c, pk) == o && orient3(c, a, pk) == o) empty = false;
          }
          if (!empty) continue;
          const int slot = atomicAdd(&s.ntri, 1);
          if (slot < GTRI) s.tri[slot] = o > 0 ? ((u32)u << 16 | (u32)v << 8 | (u32)x) : ((u32)u << 16 | (u32)x << 8 | (u32)v);
        }
      }
    }
    __syncwarp();
    const int nt = min(s.ntri, GTRI);
    if (lane == 0) {
      if ((u32)s.ntri != rec.ntri) atomicOr(err, ERR_COUNT);
      for (int a = 1; a < nt; ++a)
        for (int b = a; b > 0 && s.tri[b] < s.tri[b - 1]; --b) {
          const u32 t = s.tri[b];
          s.tri[b] = s.tri[b - 1], s.tri[b - 1] = t;
        }
    }
    __syncwarp();
    const unsigned short cd = (unsigned short)(rec.code & 0xFFFFu);
    for (int k = lane; k < nt && k < (int)rec.ntri; k += 32) {
      const int a = (int)(s.tri[k] >> 16), b = (int)((s.tri[k] >> 8) & 255u), c = (int)(s.tri[k] & 255u);
      const u32 o = rec.tri_off + (u32)k;
      tri[3 * (i64)o] = (int)s.gid[a];
      tri[3 * (i64)o + 1] = (int)s.gid[b];
      tri[3 * (i64)o + 2] = (int)s.gid[c];
      const Pq pa = lpt(s, a), pb = lpt(s, b), pc = lpt(s, c);
      const Pq ga{pa.x + A.x, pa.y + A.y}, gb{pb.x + A.x, pb.y + A.y}, gc{pc.x + A.x, pc.y + A.y};
      label[o] = label_of(g, img, pitch, dtype, ga, gb, gc);
      code[o] = cd;
    }
    // coordinates of the cell's inside vertices
    const int nin = (int)rec.nchain;
    for (int k = lane; k < nin; k += 32) {
      const int loc = n - nin + k;
      const u32 id = s.gid[loc];
      xy[2 * (i64)id] = zdouble(zq(s.xa[loc] + A.x.a, s.xb[loc] + A.x.b)) / (double)g.S;
      xy[2 * (i64)id + 1] = zdouble(zq(s.ya[loc] + A.y.a, s.yb[loc] + A.y.b)) / (double)g.S;
    }
    __syncwarp();
  }
  (void)NVg;
  (void)NE;
}

__global__ void k_lattice_xy(GridP g, double* xy) {
  const double invS = 1.0 / (double)g.S;
  for (i64 id = (i64)blockIdx.x * blockDim.x + threadIdx.x; id < g.nverts; id += (i64)gridDim.x * blockDim.x) {
    int lo = 0, hi = g.nvrows - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (g.vbase[mid] <= id) lo = mid;
      else hi = mid - 1;
    }
    const i64 j = g.vj0 + lo, i = g.vlo[lo] + (id - g.vbase[lo]);
    const Pq p = lattice_pt(g, i, j);
    double2 v;
    v.x = zdouble(p.x) * invS;
    v.y = zdouble(p.y) * invS;
    reinterpret_cast<double2*>(xy)[id] = v;
  }
}

}  // namespace

void launch_classify(const GridP& g, const Pair* pairs, Pair* sorted, const u32* poff, u32 nbc, const Seg* segs,
                     const Event* events, CutRec* recs, u32* bstat, u32* err, cudaStream_t st) {
  if (nbc == 0) return;
  k_classify<<<nbc, 256, 0, st>>>(g, pairs, sorted, poff, segs, events, recs, bstat, err);
}

void launch_scan(const u32* in, int stride, u32* out, u32 n, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(in, stride, out, n);
}

void launch_emit(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                 const Seg* segs, const Event* events, CutRec* recs, const u32* poff, const u32* bstat,
                 const u32* extra_scan, const u32* chain_scan, u32 nbc, u32 NVg, u32 NE, int* tri,
                 unsigned short* label, unsigned short* code, double* xy, u32* glist, u32* nglist, u32* ngtri,
                 u32* err, cudaStream_t st) {
  if (nbc == 0) return;
  k_emit<<<nbc, 256, 0, st>>>(g, img, pitch, dtype, sorted, segs, events, recs, poff, bstat, extra_scan,
                              chain_scan, NVg, NE, tri, label, code, xy, glist, nglist, ngtri, err);
}

void launch_tierg(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                  const Seg* segs, const Event* events, const CutRec* recs, const u32* glist, const u32* nglist,
                  u32 NVg, u32 NE, int* tri, unsigned short* label, unsigned short* code, double* xy, u32* err,
                  cudaStream_t st) {
  k_tierg<<<152 * 4, 32 * GWARPS, 0, st>>>(g, img, pitch, dtype, sorted, segs, events, recs, glist, nglist, NVg, NE,
                                           tri, label, code, xy, err);
}

void launch_lattice_xy(const GridP& g, double* xy, cudaStream_t st) {
  if (g.nverts == 0) return;
  const unsigned grd = (unsigned)std::min<i64>((g.nverts + 255) / 256, 152 * 32);
  k_lattice_xy<<<grd, 256, 0, st>>>(g, xy);
}

}  // namespace sbmt
