// k_tierg.cu -- K4-G: cells outside the regime of Lemma 3.1 ("Tier-G").
//
// At grid edges h of a few pixels the pixel staircase puts several boundary
// vertices, or several chords, into one base triangle, outside the paper's
// finite table (Lemma 3.1 needs segments longer than the grid edge,
// Sec. 3.2).  Such a cell is triangulated by a deterministic Steiner-free
// rule: its local boundary graph (the cell's boundary split at the crossing
// events, plus the pieces of boundary segments inside it) is completed
// greedily -- every other vertex pair in order of exact squared length, ties
// by local index pair, kept when its open segment holds no vertex and crosses
// no kept edge.  A maximal plane straight-line graph on a point set
// triangulates its convex hull, so the result tiles the cell and embeds every
// boundary piece.  The faces are the 3-cycles with no vertex inside, listed
// with the smallest local index first, counter-clockwise, in sorted order.
//
// The cells are first ordered by vertex count, largest first.  Cells with at
// most TN vertices (nearly all of them at h = 2 px) run one thread each, on
// per-pair vertex sets; larger cells run one warp each with the state in
// shared memory (a small state up to WS vertices, a large one above).
#include <type_traits>

#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

constexpr int TN = TIERG_TN;  // thread path: local vertices per cell (16-bit vertex sets)
constexpr int WN = 64;  // warp path, large state
constexpr int WS = TIERG_WN;  // warp path, small state (16-bit vertex sets)
constexpr int WWARPS = 4;
constexpr int SW_BLOCKS = 6;  // small-state warp kernel: blocks per SM
constexpr int GORDER_W = 8;   // ordering kernel: cell buckets (warps) per block

SBMT_DEV constexpr int pow2_at_least(int x) {
  int m = 1;
  while (m < x) m <<= 1;
  return m;
}

// The state of one Tier-G cell.  The thread path (L false, N <= 16) keeps it
// in local memory and small -- 16-bit vertex sets, no edge list; the warp
// path (L true; N = 16 or 64) keeps it in shared memory, with the kept edges
// listed.  Cell-local coordinates keep full 32-bit
// components: a value near the cell can have components of order the image
// size (a point on a slanted grid edge has x = a + b sqrt3 with both large).
template <int N, bool L>
struct GStore {
  static constexpr int NCAND = N * (N - 1) / 2;
  static constexpr int NCANDP = L ? pow2_at_least(NCAND) : NCAND;
  using Adj = typename std::conditional<(N <= 16), unsigned short, u64>::type;
  int xa[N], xb[N], ya[N], yb[N];  // cell-local exact coordinates (a + b sqrt3)
  u32 gid[N];
  u32 ref[N];  // event index (events) or pixel-corner id (inside vertices) while building
  Adj adj[N];
  unsigned short edge[L ? 3 * N : 1];  // kept edges, warp path only (L)
  unsigned short cand[L ? NCANDP : 1];  // candidate order, warp path only (the thread path keeps it with the keys)
  u32 tri[2 * N];
  float fx[N], fy[N];  // the values rounded once from double, for the fast filters
  unsigned char em[N];  // the cell edges a vertex lies on (bit k: edge k)
  int n, nev, nedge, ntri, ok;
};
template <int N, bool L>
SBMT_DEV float sfx(const GStore<N, L>& s, int k) {
  return s.fx[k];
}
template <int N, bool L>
SBMT_DEV float sfy(const GStore<N, L>& s, int k) {
  return s.fy[k];
}

template <int G>
SBMT_DEV bool g_any(bool v) {
  if constexpr (G == 1) return v;
  else return __any_sync(0xffffffffu, v);
}
template <int G>
SBMT_DEV void g_sync() {
  if constexpr (G == 32) __syncwarp();
}

template <int N, bool L>
SBMT_DEV Pq lpt(const GStore<N, L>& s, int k) {
  return Pq{zq(s.xa[k], s.xb[k]), zq(s.ya[k], s.yb[k])};
}
template <int N, bool L>
SBMT_DEV Zq len2(const GStore<N, L>& s, int u, int v) {
  const Zq dx = zq((i64)s.xa[v] - s.xa[u], (i64)s.xb[v] - s.xb[u]);
  const Zq dy = zq((i64)s.ya[v] - s.ya[u], (i64)s.yb[v] - s.yb[u]);
  return dx * dx + dy * dy;
}
// candidate order: exact squared length, then the packed pair (u << 8 | v)
template <int N, bool L>
SBMT_DEV bool cand_less(const GStore<N, L>& s, unsigned short x, unsigned short y) {
  if (x == 0xFFFFu) return false;
  if (y == 0xFFFFu) return true;
  const int c = zcmp(len2(s, x >> 8, x & 255), len2(s, y >> 8, y & 255));
  if (c != 0) return c < 0;
  return x < y;
}
SBMT_DEV Zq dot3(const Pq& o, const Pq& p, const Pq& q) {
  return (p.x - o.x) * (q.x - o.x) + (p.y - o.y) * (q.y - o.y);
}

// Same order as cand_less, decided in single precision when the two lengths
// are far apart and exactly otherwise.  Coordinates are rounded from their
// exact values (error below |coordinate| 2^-24), so a key's error stays far
// below tol for cells of extent E (scaled units).
template <int N, bool L>
SBMT_DEV bool cand_less_fast(const GStore<N, L>& s, unsigned short x, unsigned short y, float tolc) {
  const int xu = x >> 8, xv = x & 255, yu = y >> 8, yv = y & 255;
  const float dx0 = sfx(s, xv) - sfx(s, xu), dy0 = sfy(s, xv) - sfy(s, xu);
  const float dx1 = sfx(s, yv) - sfx(s, yu), dy1 = sfy(s, yv) - sfy(s, yu);
  const float kx = dx0 * dx0 + dy0 * dy0, ky = dx1 * dx1 + dy1 * dy1;
  const float tol = 1e-5f * (kx + ky) + tolc;
  if (kx < ky - tol) return true;
  if (kx > ky + tol) return false;
  return cand_less(s, x, y);
}

// cand_less_fast with the sort's padding entries (0xFFFF) last
template <int N, bool L>
SBMT_DEV bool cand_less_sent(const GStore<N, L>& s, unsigned short x, unsigned short y, float tolc) {
  if (x == 0xFFFFu) return false;
  if (y == 0xFFFFu) return true;
  return cand_less_fast(s, x, y, tolc);
}

SBMT_DEV void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Build the local boundary graph (one thread): corners A, B, C; the events
// on AB, BC, CA in counter-clockwise order; the inside vertices by pixel-
// corner id; constraint edges = boundary cycle + one piece per pair.
template <int N, bool L>
SBMT_DEV void build_local(const GridP& g, const CellGeo& cg, const CutRec& rec, const Pair* P, const Seg* segs,
                          const Event* ev, GStore<N, L>& s) {
  s.ok = 0;
  s.nedge = 0;
  const Pq A = lattice_pt(g, cg.ci[0], cg.cj[0]);
  for (int k = 0; k < 3; ++k) {
    const Pq p = lattice_pt(g, cg.ci[k], cg.cj[k]);
    s.xa[k] = (int)(p.x.a - A.x.a), s.xb[k] = (int)(p.x.b - A.x.b);
    s.ya[k] = (int)(p.y.a - A.y.a), s.yb[k] = (int)(p.y.b - A.y.b);
    s.gid[k] = vid(g, cg.ci[k], cg.cj[k]);
    s.ref[k] = NONE;
  }
  // events: gather once, keyed by (local edge, counter-clockwise position)
  int ne = 0;
  int ek[N];
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e == NONE) continue;
      if (3 + ne >= N) return;
      const Event x = ev[e];
      const int le = local_edge(cg, x.edge);
      if (le < 0) return;
      const int t = 3 + ne;
      s.ref[t] = e, ek[t] = le, s.gid[t] = x.gid;
      s.xa[t] = (int)(x.xa - A.x.a), s.xb[t] = (int)(x.xb - A.x.b);
      s.ya[t] = (int)(x.ya - A.y.a), s.yb[t] = (int)(x.yb - A.y.b);
      ++ne;
    }
  }
  for (int a = 4; a < 3 + ne; ++a)
    for (int b = a; b > 3; --b) {
      const Zq pb = ccw_pos_xy(cg.down, ek[b], zq(s.xa[b], s.xb[b]), zq(s.ya[b], s.yb[b]));
      const Zq pa = ccw_pos_xy(cg.down, ek[b - 1], zq(s.xa[b - 1], s.xb[b - 1]), zq(s.ya[b - 1], s.yb[b - 1]));
      if (!(ek[b] < ek[b - 1] || (ek[b] == ek[b - 1] && zcmp(pb, pa) < 0))) break;
      int ti = ek[b];
      ek[b] = ek[b - 1], ek[b - 1] = ti;
      u32 tu = s.ref[b];
      s.ref[b] = s.ref[b - 1], s.ref[b - 1] = tu;
      tu = s.gid[b], s.gid[b] = s.gid[b - 1], s.gid[b - 1] = tu;
      ti = s.xa[b], s.xa[b] = s.xa[b - 1], s.xa[b - 1] = ti;
      ti = s.xb[b], s.xb[b] = s.xb[b - 1], s.xb[b - 1] = ti;
      ti = s.ya[b], s.ya[b] = s.ya[b - 1], s.ya[b - 1] = ti;
      ti = s.yb[b], s.yb[b] = s.yb[b - 1], s.yb[b - 1] = ti;
    }
  int nev[3] = {0, 0, 0};
  for (int t = 3; t < 3 + ne; ++t) nev[ek[t]]++;
  // inside vertices: distinct pixel-corner ids, ascending
  int n = 3 + ne;
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
    if (pr.ev_in != NONE && pr.ev_out != NONE) continue;
    const Seg sg = segs[pr.seg];
    for (int end = 0; end < 2; ++end) {
      if ((end == 0 ? pr.ev_in : pr.ev_out) != NONE) continue;
      const u32 id = corner_id(g, sg, end);
      int pos = 3 + ne;
      while (pos < n && s.ref[pos] < id) ++pos;
      if (pos < n && s.ref[pos] == id) continue;
      if (n >= N) return;
      for (int t = n; t > pos; --t) s.ref[t] = s.ref[t - 1];
      s.ref[pos] = id;
      ++n;
    }
  }
  if ((u32)(n - 3 - ne) != rec.nchain) return;
  for (int k = 3 + ne; k < n; ++k) {
    const Pq p = corner_of_id(g, s.ref[k]);
    s.xa[k] = (int)(p.x.a - A.x.a), s.xb[k] = (int)(p.x.b - A.x.b);
    s.ya[k] = (int)(p.y.a - A.y.a), s.yb[k] = (int)(p.y.b - A.y.b);
    s.gid[k] = rec.chain_base + (u32)(k - 3 - ne);
  }
  s.n = n, s.nev = ne;
  for (int k = 0; k < n; ++k) {
    s.em[k] = k < 3 ? (unsigned char)((1 << k) | (1 << (k == 0 ? 2 : k - 1))) : k < 3 + ne ? (unsigned char)(1 << ek[k]) : 0;
    s.adj[k] = 0;
    s.fx[k] = (float)zdouble(zq(s.xa[k], s.xb[k]));
    s.fy[k] = (float)zdouble(zq(s.ya[k], s.yb[k]));
  }
  bool room = true;
  auto add_edge = [&](int u, int v) {
    if (u > v) {
      const int t = u;
      u = v, v = t;
    }
    if ((s.adj[u] >> v) & 1ull) return;
    if (s.nedge >= 3 * N) {
      room = false;
      return;
    }
    s.adj[u] |= 1ull << v, s.adj[v] |= 1ull << u;
    if constexpr (L) s.edge[s.nedge] = (unsigned short)((u << 8) | v);
    ++s.nedge;
  };
  {  // boundary cycle A, events on AB, B, events on BC, C, events on CA
    int prev = 0, e = 3, first = 0;
    for (int k = 0; k < 3; ++k) {
      if (k) add_edge(prev, k), prev = k;
      for (int t = 0; t < nev[k]; ++t) add_edge(prev, e), prev = e++;
    }
    add_edge(prev, first);
  }
  for (u32 k = 0; k < rec.npairs; ++k) {  // boundary pieces
    const Pair pr = P[k];
    int loc[2] = {-1, -1};
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e != NONE) {
        for (int t = 3; t < 3 + ne; ++t)
          if (s.ref[t] == e) loc[end] = t;
      } else {
        const u32 id = corner_id(g, segs[pr.seg], end);
        for (int t = 3 + ne; t < n; ++t)
          if (s.ref[t] == id) loc[end] = t;
      }
    }
    if (loc[0] < 0 || loc[1] < 0) return;
    add_edge(loc[0], loc[1]);
  }
  s.ok = room ? 1 : 0;
}

// The greedy completion and face listing by a group of G lanes (G = 1: one
// thread; G = 32: a warp with the store in shared memory).
template <int G, int N, bool L, class O>
SBMT_DEV void greedy_faces(GStore<N, L>& s, int lane, int nb, const O& ori, float tolc) {
  const int n = s.n;
  // candidate pairs not joined by a constraint edge
  int m = 0;
  if constexpr (G == 1) {
    for (int u = 0; u < n; ++u)
      for (int v = u + 1; v < n; ++v)
        if (!((s.adj[u] >> v) & 1ull)) s.cand[m++] = (unsigned short)((u << 8) | v);
    // insertion sort by (exact length, pair)
    for (int a = 1; a < m; ++a) {
      const unsigned short x = s.cand[a];
      int b = a;
      while (b > 0 && cand_less_fast(s, x, s.cand[b - 1], tolc)) s.cand[b] = s.cand[b - 1], --b;
      s.cand[b] = x;
    }
  } else {
    for (int u = 0; u < n; ++u)
      for (int vb = u + 1; vb < n; vb += 32) {
        const int v = vb + lane;
        // a pair on one cell edge that is not a cycle edge has a vertex
        // between its ends and is always rejected: left out
        const bool ok = v < n && !((s.adj[u] >> v) & 1ull) && !(s.em[u] & s.em[v]);
        const u32 bal = __ballot_sync(0xffffffffu, ok);
        if (ok) s.cand[m + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)((u << 8) | v);
        m += __popc(bal);
      }
    int M = 1;
    while (M < m) M <<= 1;
    for (int k = m + lane; k < M; k += 32) s.cand[k] = 0xFFFFu;
    __syncwarp();
    for (int kk = 2; kk <= M; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < M; i += 32) {
          const int l = i ^ jj;
          if (l > i) {
            const unsigned short x = s.cand[i], y = s.cand[l];
            const bool up = (i & kk) == 0;
            if (up ? cand_less_sent(s, y, x, tolc) : cand_less_sent(s, x, y, tolc)) s.cand[i] = y, s.cand[l] = x;
          }
        }
        __syncwarp();
      }
  }
  // keep a pair when its open segment holds no vertex and crosses no kept edge
  const int max_edges = 3 * n - nb - 3;
  for (int ci = 0; ci < m && s.nedge < max_edges; ++ci) {
    const int u = s.cand[ci] >> 8, v = s.cand[ci] & 255;
    bool bad = false;
    for (int k = lane; k < n && !bad; k += G) {
      if (k == u || k == v || ori(u, v, k) != 0) continue;
      const Pq pu = lpt(s, u), pv = lpt(s, v), pk = lpt(s, k);
      if (zsign(dot3(pu, pv, pk)) > 0 && zsign(dot3(pv, pu, pk)) > 0) bad = true;
    }
    const int ned = s.nedge;
    for (int k = lane; k < ned && !bad; k += G) {
      const int a = s.edge[k] >> 8, b = s.edge[k] & 255;
      if (a == u || a == v || b == u || b == v) continue;
      const int o1 = ori(u, v, a), o2 = ori(u, v, b);
      if (o1 * o2 >= 0) continue;
      const int o3 = ori(a, b, u), o4 = ori(a, b, v);
      if (o3 * o4 < 0) bad = true;
    }
    if (!g_any<G>(bad) && lane == 0) {
      s.adj[u] |= 1ull << v, s.adj[v] |= 1ull << u;
      s.edge[s.nedge] = (unsigned short)((u << 8) | v);
      s.nedge = s.nedge + 1;
    }
    g_sync<G>();
  }
  // faces: 3-cycles with no vertex strictly inside
  if (lane == 0) s.ntri = 0;
  g_sync<G>();
  for (int u = lane; u < n; u += G) {
    for (u64 vs = s.adj[u] & ~((2ull << u) - 1ull); vs; vs &= vs - 1) {
      const int v = __ffsll((long long)vs) - 1;
      for (u64 ws = s.adj[u] & s.adj[v] & ~((2ull << v) - 1ull); ws; ws &= ws - 1) {
        const int x = __ffsll((long long)ws) - 1;
        const int o = ori(u, v, x);
        if (o == 0) continue;
        bool empty = true;
        for (int k = 0; k < n && empty; ++k) {
          if (k == u || k == v || k == x) continue;
          if (ori(u, v, k) == o && ori(v, x, k) == o && ori(x, u, k) == o) empty = false;
        }
        if (!empty) continue;
        int slot;
        if constexpr (G == 1) slot = s.ntri++;
        else slot = atomicAdd(&s.ntri, 1);
        if (slot < 2 * N)
          s.tri[slot] = o > 0 ? ((u32)u << 16 | (u32)v << 8 | (u32)x) : ((u32)u << 16 | (u32)x << 8 | (u32)v);
      }
    }
  }
  g_sync<G>();
  const int nt = min(s.ntri, 2 * N);
  if constexpr (G == 1) {
    for (int a = 1; a < nt; ++a)
      for (int b = a; b > 0 && s.tri[b] < s.tri[b - 1]; --b) {
        const u32 t = s.tri[b];
        s.tri[b] = s.tri[b - 1], s.tri[b - 1] = t;
      }
  } else {
    // by rank, the lanes together: the keys are distinct (each face once)
    constexpr int R = (2 * N + G - 1) / G;
    u32 key[R];
    int rank[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int k = lane + q * G;
      key[q] = k < nt ? s.tri[k] : 0u;
      rank[q] = 0;
      if (k < nt)
        for (int j = 0; j < nt; ++j) rank[q] += s.tri[j] < key[q] ? 1 : 0;
    }
    g_sync<G>();
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (lane + q * G < nt) s.tri[rank[q]] = key[q];
  }
  g_sync<G>();
}

// The same greedy rule for one thread, on vertex sets.  For every pair u < v
// two 16-bit sets record the vertices strictly left of the directed line
// u -> v and those on it; each orientation is decided in single precision
// when the determinant is clear of its rounding bound and exactly otherwise,
// so that it is the exact one.  A candidate is blocked by a collinear vertex between
// its ends or by a kept edge with one end on each side whose own line
// separates the candidate's ends; a 3-cycle is a face when no vertex lies on
// the inner side of all three of its edges.
template <int N, bool L>
SBMT_DEV int ori_filtered(const GStore<N, L>& s, int a, int b, int c, float tol) {
  const float fxa = sfx(s, a), fya = sfy(s, a);
  const float dx1 = sfx(s, b) - fxa, dy1 = sfy(s, b) - fya;
  const float dx2 = sfx(s, c) - fxa, dy2 = sfy(s, c) - fya;
  const float d = dx1 * dy2 - dy1 * dx2;
  if (d > tol) return 1;
  if (d < -tol) return -1;
  // three points of one cell edge (an exact line) need no exact test
  if (s.em[a] & s.em[b] & s.em[c]) return 0;
  return orient3(lpt(s, a), lpt(s, b), lpt(s, c));
}

// orientation decided in single precision when clear, exactly otherwise
template <int N, bool L>
struct OriFiltered {
  const GStore<N, L>* s;
  float tol;
  SBMT_DEV int operator()(int u, int v, int w) const { return ori_filtered(*s, u, v, w, tol); }
};

template <int N, bool L>
SBMT_DEV void greedy_faces_sets(GStore<N, L>& s, int nb, float tolc, float tolo) {
  static_assert(N <= 16 && !L, "vertex sets are 16 bits wide");
  constexpr int NPAIR = N * (N - 1) / 2;
  const int n = s.n;
  unsigned short Lm[NPAIR], Zm[NPAIR];
  auto pid = [](int u, int v) { return v * (v - 1) / 2 + u; };  // u < v
  // Per pair u < v, the vertices left of u -> v and those on its line,
  // gathered in registers and stored once (the coordinates of every w in
  // registers too).  Each orientation comes out exact whichever way round its
  // triple is taken (the filter decides only outside its rounding bound), so
  // deciding a triple once per pair gives the sets of deciding it once.
  float fxr[N], fyr[N];
#pragma unroll
  for (int w = 0; w < N; ++w) fxr[w] = w < n ? sfx(s, w) : 0.f, fyr[w] = w < n ? sfy(s, w) : 0.f;
  for (int v = 1; v < n; ++v)
    for (int u = 0; u < v; ++u) {
      const float xu = sfx(s, u), yu = sfy(s, u), dx1 = sfx(s, v) - xu, dy1 = sfy(s, v) - yu;
      unsigned lm = 0, zm = 0, und = 0;
#pragma unroll
      for (int w = 0; w < N; ++w) {
        if (w >= n || w == u || w == v) continue;
        const float d = dx1 * (fyr[w] - yu) - dy1 * (fxr[w] - xu);
        if (d > tolo) lm |= 1u << w;
        else if (!(d < -tolo)) und |= 1u << w;
      }
      for (; und; und &= und - 1) {  // within the rounding bound: exactly
        const int w = __ffs(und) - 1;
        const int o = (s.em[u] & s.em[v] & s.em[w]) ? 0 : orient3(lpt(s, u), lpt(s, v), lpt(s, w));
        if (o > 0) lm |= 1u << w;
        else if (o == 0) zm |= 1u << w;
      }
      Lm[pid(u, v)] = (unsigned short)lm, Zm[pid(u, v)] = (unsigned short)zm;
    }
  const unsigned valid = (1u << n) - 1u;
  auto Zset = [&](int u, int v) -> unsigned { return u < v ? Zm[pid(u, v)] : Zm[pid(v, u)]; };
  auto Lset = [&](int u, int v) -> unsigned {
    return u < v ? (unsigned)Lm[pid(u, v)] : (valid & ~((unsigned)Lm[pid(v, u)] | Zm[pid(v, u)]));
  };
  auto ori = [&](int u, int v, int w) -> int {
    if ((Zset(u, v) >> w) & 1u) return 0;
    return ((Lset(u, v) >> w) & 1u) ? 1 : -1;
  };
  // candidates in order of exact length, then (u, v).  A pair on one cell
  // edge that is not a cycle edge always has a vertex between its ends, so
  // it is left out; each candidate's single-precision key is taken once.
  int m = 0;
  u64 kc[NPAIR];  // the key's bits above the candidate (u << 8 | v): one word moves per shift
  for (int u = 0; u < n; ++u)
    for (int v = u + 1; v < n; ++v)
      if (!((s.adj[u] >> v) & 1ull) && !(s.em[u] & s.em[v])) {
        const unsigned short x = (unsigned short)((u << 8) | v);
        const float dx = sfx(s, v) - sfx(s, u), dy = sfy(s, v) - sfy(s, u);
        const float kx = dx * dx + dy * dy;
        int b = m++;
        // insertion: the same order as cand_less_fast, with the keys kept
        while (b > 0) {
          const u64 y = kc[b - 1];
          const float ky = __uint_as_float((u32)(y >> 32));
          const float tol = 1e-5f * (kx + ky) + tolc;
          const bool less =
              kx < ky - tol ? true : kx > ky + tol ? false : cand_less(s, x, (unsigned short)(y & 0xFFFFu));
          if (!less) break;
          kc[b] = y, --b;
        }
        kc[b] = (u64)__float_as_uint(kx) << 32 | x;
      }
  const int max_edges = 3 * n - nb - 3;
  for (int ci = 0; ci < m && s.nedge < max_edges; ++ci) {
    const int u = (int)((kc[ci] >> 8) & 255u), v = (int)(kc[ci] & 255u);
    bool bad = false;
    const unsigned zu = Zset(u, v);
    for (unsigned zc = zu & ~((1u << u) | (1u << v)); zc && !bad; zc &= zc - 1) {
      const int k = __ffs(zc) - 1;
      const Pq pu = lpt(s, u), pv = lpt(s, v), pk = lpt(s, k);
      if (zsign(dot3(pu, pv, pk)) > 0 && zsign(dot3(pv, pu, pk)) > 0) bad = true;
    }
    if (!bad) {
      // the complement of L and Z holds u and v themselves: drop them
      const unsigned lu = Lset(u, v), ru = valid & ~(lu | zu | (1u << u) | (1u << v));
      for (unsigned as = lu; as && !bad; as &= as - 1) {
        const int a = __ffs(as) - 1;
        for (unsigned bs = (unsigned)s.adj[a] & ru; bs && !bad; bs &= bs - 1) {
          const int b = __ffs(bs) - 1;
          if (ori(a, b, u) * ori(a, b, v) < 0) bad = true;
        }
      }
    }
    if (!bad) {
      s.adj[u] |= 1ull << v, s.adj[v] |= 1ull << u;
      ++s.nedge;
    }
  }
  s.ntri = 0;
  for (int u = 0; u < n; ++u)
    for (unsigned vs = (unsigned)s.adj[u] & ~((2u << u) - 1u); vs; vs &= vs - 1) {
      const int v = __ffs(vs) - 1;
      for (unsigned ws = (unsigned)(s.adj[u] & s.adj[v]) & ~((2u << v) - 1u); ws; ws &= ws - 1) {
        const int w = __ffs(ws) - 1;
        const int o = ori(u, v, w);
        if (o == 0) continue;
        unsigned inside;
        if (o > 0) {
          inside = Lset(u, v) & Lset(v, w) & Lset(w, u);
        } else {
          inside = (valid & ~(Lset(u, v) | Zset(u, v))) & (valid & ~(Lset(v, w) | Zset(v, w))) &
                   (valid & ~(Lset(w, u) | Zset(w, u)));
        }
        if (inside & ~((1u << u) | (1u << v) | (1u << w))) continue;
        if (s.ntri < 2 * N)
          s.tri[s.ntri] = o > 0 ? ((u32)u << 16 | (u32)v << 8 | (u32)w) : ((u32)u << 16 | (u32)w << 8 | (u32)v);
        ++s.ntri;
      }
    }
  const int nt = min(s.ntri, 2 * N);
  for (int a = 1; a < nt; ++a)
    for (int b = a; b > 0 && s.tri[b] < s.tri[b - 1]; --b) {
      const u32 t = s.tri[b];
      s.tri[b] = s.tri[b - 1], s.tri[b - 1] = t;
    }
}

template <int G, int N, bool L>
SBMT_DEV void write_patch(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const CellGeo& cg,
                          const CutRec& rec, const GStore<N, L>& s, int lane, int* tri, unsigned short* label,
                          unsigned short* code, double* xy, u32 xy0, u32* err) {
  const Pq A = lattice_pt(g, cg.ci[0], cg.cj[0]);
  const int nt = min(s.ntri, 2 * N);
  if (lane == 0 && (u32)s.ntri != rec.ntri) atomicOr(err, ERR_COUNT);
  const unsigned short cd = (unsigned short)(rec.code & 0xFFFFu);
  for (int k = lane; k < nt && k < (int)rec.ntri; k += G) {
    const int a = (int)(s.tri[k] >> 16), b = (int)((s.tri[k] >> 8) & 255u), c = (int)(s.tri[k] & 255u);
    const u32 o = rec.tri_off + (u32)k;
    tri[3 * (i64)o] = (int)s.gid[a];
    tri[3 * (i64)o + 1] = (int)s.gid[b];
    tri[3 * (i64)o + 2] = (int)s.gid[c];
    const Pq pa = lpt(s, a), pb = lpt(s, b), pc = lpt(s, c);
    label[o] = label_of(g, img, pitch, dtype, Pq{pa.x + A.x, pa.y + A.y}, Pq{pb.x + A.x, pb.y + A.y},
                        Pq{pc.x + A.x, pc.y + A.y});
    code[o] = cd;
  }
  // coordinates of the cell's inside vertices
  const int nin = (int)rec.nchain;
  const double invS = 1.0 / (double)g.S;
  for (int k = lane; k < nin; k += G) {
    const int loc = s.n - nin + k;
    double2 v;
    v.x = zdouble(zq((i64)s.xa[loc] + A.x.a, (i64)s.xb[loc] + A.x.b)) * invS;
    v.y = zdouble(zq((i64)s.ya[loc] + A.y.a, (i64)s.yb[loc] + A.y.b)) * invS;
    reinterpret_cast<double2*>(xy)[s.gid[loc] - xy0] = v;
  }
}

// the number of local vertices of a Tier-G cell: ntri = 2 n_in + n_b - 2
SBMT_DEV int local_count(const CutRec& rec) { return (int)(rec.ntri + 2 - rec.nchain); }
SBMT_DEV int boundary_count(const CutRec& rec) { return (int)(rec.ntri + 2 - 2 * rec.nchain); }

// Tier-G cells of the whole batch ordered by local vertex count, largest
// first.  bd->gcnt[n] holds the batch's number of Tier-G cells with n
// vertices (n > WS pooled at index WS + 1).  The cells of at most WS vertices
// form one order: those above TN run one warp each with the small state
// (slist), the others one thread each (olist), so that the lanes of a warp
// run cells of one size.  (Moving more of the largest cells to the warp
// kernel measured no faster on any workload tried, from 10^4 to 2 x 10^5
// Tier-G cells: a warp's greedy pass takes about as long per cell as a
// thread's.)  Cells above WS vertices go to the
// large-state warp kernel (wlist).  One warp per
// cell bucket scans the bucket's records (in cell order) and gives each
// Tier-G cell its output range from the scans the emission kernel uses: its
// triangles follow those of the bucket's earlier cells (one each when uncut,
// ntri each when cut) and its inside vertices those of the bucket's earlier
// cut cells.  In the compact format only the cut cells' triangles are listed.
// The lists hold (job, record) pairs.
template <bool ONE>
__global__ void __launch_bounds__(32 * GORDER_W) k_gorder_b(const __grid_constant__ Job one,
                                                            const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                            int njobs, BatchDev* bd, uint2* olist, uint2* slist,
                                                            uint2* wlist) {
  __shared__ u32 s_base[WS + 2];
  __shared__ u32 s_kw;
  __shared__ u32 s_wc[GORDER_W][WS + 2];  // per warp: its cells per size, then its first place among the block's
  __shared__ u32 s_blk[WS + 2];           // the block's first place per size (one atomic per size and block)
  if (threadIdx.x == 0) {
    u32 run = 0, big = 0;
    for (int n = WS; n >= 0; --n) {
      s_base[n] = run, run += bd->gcnt[n];
      if (n == TN + 1) big = run;  // the cells above TN
    }
    s_base[WS + 1] = 0;
    s_kw = big;
    if (blockIdx.x == 0) bd->nolist = run - big, bd->nslist = big;
  }
  for (int i = threadIdx.x; i < GORDER_W * (WS + 2); i += blockDim.x) (&s_wc[0][0])[i] = 0u;
  __syncthreads();
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 b = lb * GORDER_W + (u32)w;
  const bool live = b < J.nbc;  // a warp past the job's buckets still meets the block's barriers
  CutRec* recs = J.recs;
  const u32 n = live ? J.bcut[b] : 0u, rec0 = live ? J.bbase[b] : 0u;
  // the warp's Tier-G cells per size
  for (u32 base = 0; base < n; base += 32) {
    const u32 r = base + (u32)lane;
    CutRec rec{};
    if (r < n) rec = recs[rec0 + r];
    const bool tg = r < n && (rec.code & (1u << 16));
    const unsigned tmask = __ballot_sync(0xffffffffu, tg);
    if (tg) {
      const int nv = local_count(rec);
      const int key = nv > WS ? WS + 1 : nv;
      const unsigned peers = __match_any_sync(tmask, key);
      if (lane == __ffs(peers) - 1) s_wc[w][key] += (u32)__popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // per size: the warps' places within the block, and one atomic for the block
  if (threadIdx.x < WS + 2) {
    const int key = (int)threadIdx.x;
    u32 tot = 0;
    for (int q = 0; q < GORDER_W; ++q) {
      const u32 c = s_wc[q][key];
      s_wc[q][key] = tot, tot += c;
    }
    s_blk[key] = tot ? atomicAdd(key > WS ? &bd->nwlist : &bd->gcur[key], tot) : 0u;
  }
  __syncthreads();
  if (!live) return;
  const u32* extra_scan = J.extra_scan;
  const u32* cut_scan = J.cp.on ? J.cp.cut_scan : nullptr;
  const u32 CB0 = J.NVg + J.NE;
  const u32 kw = s_kw;
  u32 ct = 0, cc = 0;  // the bucket's earlier records: sum of (ntri - 1), of nchain
  for (u32 base = 0; base < n; base += 32) {
    const u32 r = base + (u32)lane;
    const bool valid = r < n;
    CutRec rec{};
    if (valid) rec = recs[rec0 + r];
    const u32 vt = valid ? rec.ntri - 1u : 0u, vc = valid ? rec.nchain : 0u;
    u32 it = vt, ic = vc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 t = __shfl_up_sync(0xffffffffu, it, o), c = __shfl_up_sync(0xffffffffu, ic, o);
      if (lane >= o) it += t, ic += c;
    }
    const u32 pt = ct + it - vt, pc = cc + ic - vc;
    ct += __shfl_sync(0xffffffffu, it, 31), cc += __shfl_sync(0xffffffffu, ic, 31);
    const bool tg = valid && (rec.code & (1u << 16));
    const unsigned tmask = __ballot_sync(0xffffffffu, tg);
    if (tg) {
      recs[rec0 + r].tri_off = cut_scan ? extra_scan[b] + cut_scan[b] + r + pt : rec.cell + extra_scan[b] + pt;
      recs[rec0 + r].chain_base = CB0 + J.chain_scan[b] + pc;
      const int nv = local_count(rec);
      const int key = nv > WS ? WS + 1 : nv;
      // the cells of one size take consecutive places, in the warp's order
      const unsigned peers = __match_any_sync(tmask, key);
      const int leader = __ffs(peers) - 1;
      u32 at = 0;
      if (lane == leader) at = s_blk[key] + s_wc[w][key], s_wc[w][key] += (u32)__popc(peers);
      at = __shfl_sync(peers, at, leader) + (u32)__popc(peers & ((1u << lane) - 1u));
      const uint2 e = make_uint2((u32)jk, rec0 + r);
      if (key > WS) {
        wlist[at] = e;
      } else {
        const u32 pos = s_base[key] + at;  // place in the order, largest first
        if (pos < kw) slist[pos] = e;
        else olist[pos - kw] = e;
      }
    }
    __syncwarp();
  }
}

SBMT_DEV void tierg_over(const Job& J, u32 cell) {
  atomicOr(jc(J, JC_ERR), ERR_CAPACITY);
  const u32 slot = atomicAdd(jc(J, JC_NOVER), 1u);
  if (slot < OVER_CAP) J.over[slot] = cell;
}

// one thread per Tier-G cell of at most TN vertices, in the order above
template <bool ONE>
__global__ void __launch_bounds__(64, 12) k_tierg_thread_b(const __grid_constant__ Job one,
                                                           const Job* __restrict__ jobs, const BatchDev* bd,
                                                           const uint2* olist) {
  const u32 total = bd->nolist;
  for (u32 item = blockIdx.x * blockDim.x + threadIdx.x; item < total; item += gridDim.x * blockDim.x) {
    const uint2 e = olist[item];
    const Job& J = ONE ? one : jobs[e.x];
    const GridP g = J.g;
    const CutRec rec = J.recs[e.y];
    const CellGeo cg = cell_geo(g, rec.cell, cell_row_near(g, rec.cell));
    GStore<TN, false> s;
    build_local(g, cg, rec, J.raw + rec.pair_lo, J.segs, J.ev, s);
    if (!s.ok) {
      tierg_over(J, rec.cell);
      continue;
    }
    // cell-local coordinates are bounded by the cell extent M = 6p scaled units
    const float M = (float)(6 * g.p);
    greedy_faces_sets<TN>(s, boundary_count(rec), 1e-4f * M * M, 8e-6f * M * M);
    write_patch<1, TN, false>(g, J.img, J.pitch, J.dtype, cg, rec, s, 0, J.tri, J.label, J.code, J.xy, J.cp.xy0,
                       jc(J, JC_ERR));
  }
}

// one warp per Tier-G cell, the state (N vertices at most) in shared memory
template <bool ONE, int N>
__global__ void __launch_bounds__(32 * WWARPS) k_tierg_warp_b(const __grid_constant__ Job one,
                                                              const Job* __restrict__ jobs, const u32* count,
                                                              const uint2* list) {
  __shared__ GStore<N, true> sm[WWARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  GStore<N, true>& s = sm[w];
  const u32 total = *count;
  for (u32 item = blockIdx.x * WWARPS + w; item < total; item += gridDim.x * WWARPS) {
    const uint2 e = list[item];
    const Job& J = ONE ? one : jobs[e.x];
    const GridP g = J.g;
    const CutRec rec = J.recs[e.y];
    const CellGeo cg = cell_geo(g, rec.cell, cell_row_near(g, rec.cell));
    // the lanes request the cell's pair records, events and segments into
    // L1 together, so that the one lane building the local graph finds them
    // there instead of waiting on each in turn
    const Pair* P = J.raw + rec.pair_lo;
    for (u32 k = (u32)lane; k < rec.npairs; k += 32) {
      const Pair pr = P[k];
      if (pr.ev_in != NONE) prefetch_l1(J.ev + pr.ev_in);
      if (pr.ev_out != NONE) prefetch_l1(J.ev + pr.ev_out);
      prefetch_l1(J.segs + pr.seg);
    }
    __syncwarp();
    if (lane == 0) build_local(g, cg, rec, P, J.segs, J.ev, s);
    __syncwarp();
    if (!s.ok) {
      if (lane == 0) tierg_over(J, rec.cell);
      __syncwarp();
      continue;
    }
    // cell-local coordinates are bounded by the cell extent M = 6p scaled units
    const float M = (float)(6 * g.p);
    greedy_faces<32, N, true>(s, lane, boundary_count(rec), OriFiltered<N, true>{&s, 8e-6f * M * M}, 1e-4f * M * M);
    write_patch<32, N, true>(g, J.img, J.pitch, J.dtype, cg, rec, s, lane, J.tri, J.label, J.code, J.xy, J.cp.xy0,
                             jc(J, JC_ERR));
    __syncwarp();
  }
}

// the status words of every job (error bits, cut cells, Tier-G cells, Tier-G
// triangles, cells over the Tier-G limit) into its mapped host slot
__global__ void k_status_b(const Job* __restrict__ jobs, int njobs, const BatchDev* bd) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < njobs; k += gridDim.x * blockDim.x) {
    const Job& J = jobs[k];
    for (int w = 0; w < 5; ++w) J.hinfo[w] = *jc(J, JC_ERR + w);
  }
  __threadfence_system();
}

}  // namespace

int launch_tierg_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, const BatchPtrs& bp,
                   int thread_blocks_per_sm, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_order,
                   cudaEvent_t ev_warp) {
  if (nblocks == 0) return 0;
  const Job none{};
  const Job& oj = one ? *one : none;
  if (one)
    k_gorder_b<true><<<nblocks, 32 * GORDER_W, 0, st>>>(oj, jobs, bpre, njobs, bp.bd, bp.olist, bp.slist, bp.wlist);
  else
    k_gorder_b<false><<<nblocks, 32 * GORDER_W, 0, st>>>(oj, jobs, bpre, njobs, bp.bd, bp.olist, bp.slist, bp.wlist);
  if (one) k_tierg_thread_b<true><<<152 * thread_blocks_per_sm, 64, 0, st>>>(oj, jobs, bp.bd, bp.olist);
  else k_tierg_thread_b<false><<<152 * thread_blocks_per_sm, 64, 0, st>>>(oj, jobs, bp.bd, bp.olist);
  // the warp kernels on their own stream when given one, beside the thread
  // kernel: the large-state cells (the largest of all) first
  if (st2) {
    if (cudaEventRecord(ev_order, st) != cudaSuccess || cudaStreamWaitEvent(st2, ev_order, 0) != cudaSuccess) return -1;
  }
  cudaStream_t ws = st2 ? st2 : st;
  if (one) {
    k_tierg_warp_b<true, WN><<<152 * 2, 32 * WWARPS, 0, ws>>>(oj, jobs, &bp.bd->nwlist, bp.wlist);
    k_tierg_warp_b<true, WS><<<152 * SW_BLOCKS, 32 * WWARPS, 0, ws>>>(oj, jobs, &bp.bd->nslist, bp.slist);
  } else {
    k_tierg_warp_b<false, WN><<<152 * 2, 32 * WWARPS, 0, ws>>>(oj, jobs, &bp.bd->nwlist, bp.wlist);
    k_tierg_warp_b<false, WS><<<152 * SW_BLOCKS, 32 * WWARPS, 0, ws>>>(oj, jobs, &bp.bd->nslist, bp.slist);
  }
  if (st2) {
    if (cudaEventRecord(ev_warp, st2) != cudaSuccess || cudaStreamWaitEvent(st, ev_warp, 0) != cudaSuccess) return -1;
  }
  return 4;
}

int tierg_init() {
  // each thread of the thread path keeps a cell's state in local memory:
  // give L1 the most room
  const bool ok = cudaFuncSetAttribute(k_tierg_thread_b<true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0) ==
                      cudaSuccess &&
                  cudaFuncSetAttribute(k_tierg_thread_b<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0) ==
                      cudaSuccess;
  return ok ? 0 : -1;
}

int launch_status_b(const Job* jobs, int njobs, const BatchPtrs& bp, cudaStream_t st) {
  k_status_b<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, njobs, bp.bd);
  return 1;
}

}  // namespace sbmt
