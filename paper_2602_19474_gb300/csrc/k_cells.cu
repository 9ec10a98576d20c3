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

#include "sbmt_cell.cuh"
#include "sbmt_keys.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

// ---------------------------------------------------------------------------
// K3 classification of one cut cell from its (cell, segment) pairs
// ---------------------------------------------------------------------------
struct Klass {
  u32 code, ntri, nchain;
  bool tierG;
};

SBMT_DEV Klass classify_cell(const GridP& g, const CellGeo& cg, const Pair* P, u32 np, const Seg* segs,
                             const Event* ev, u32* err) {
  int n0 = 0, n1 = 0, n2 = 0;  // events on AB, BC, CA
  u32 mask = 0, nchain = 0;
  bool all_one_inside = true;
  // the first two pairs (Tier-T chords): local edges of the walk-order ends,
  // their events, the segment's orientation, the pair's event count
  int pin0 = -1, pout0 = -1, pin1 = -1, pout1 = -1, rev0 = 0, rev1 = 0, m0 = 0, m1 = 0;
  u32 ein0 = NONE, eout0 = NONE, ein1 = NONE, eout1 = NONE;
  for (u32 k = 0; k < np; ++k) {
    const Pair pr = P[k];
    const Seg s = segs[pr.seg];
    int inside = 0, m = 0, lin = -1, lout = -1;
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e != NONE) {
        const int le = local_edge(cg, ev[e].edge);
        if (le < 0) {
          atomicOr(err, ERR_TRAVERSAL);
          continue;
        }
        n0 += le == 0, n1 += le == 1, n2 += le == 2;
        mask |= 2u << le;
        ++m;
        if (end == 0) lin = le;
        else lout = le;
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
    if (k == 0) pin0 = lin, pout0 = lout, ein0 = pr.ev_in, eout0 = pr.ev_out, rev0 = seg_rev(s), m0 = m;
    else if (k == 1) pin1 = lin, pout1 = lout, ein1 = pr.ev_in, eout1 = pr.ev_out, rev1 = seg_rev(s), m1 = m;
  }
  Klass r;
  r.nchain = nchain;
  r.ntri = 2 * nchain + 1 + (u32)(n0 + n1 + n2);
  if (nchain) mask |= 1u;
  const int klass = np == 1 ? thm32_class(0, m0) : np == 2 ? thm32_class(m0, m1) : 0;
  const bool chords = nchain == 0 && (np == 1 || np == 2);
  const bool star = nchain == 1 && all_one_inside && np >= 2 && np <= 4;
  if (!chords && !star) {
    r.tierG = true;
    r.code = (mask & 15u) | (63u << 6) | ((u32)klass << 12);
    return r;
  }
  int dir = 0;
  if (chords && np == 2) {
    const int X0 = (pout0 == (pin0 + 1) % 3) ? pout0 : pin0;
    const int X1 = (pout1 == (pin1 + 1) % 3) ? pout1 : pin1;
    if (X0 == X1) {
      // nested chords at corner X: the chord nearer X meets the edge ending
      // at X later in counter-clockwise order
      const int ein = (X0 + 2) % 3, eout = X0;
      const Zq pos0 = ccw_pos(cg.down, ein, ev[pin0 == ein ? ein0 : eout0]);
      const Zq pos1 = ccw_pos(cg.down, ein, ev[pin1 == ein ? ein1 : eout1]);
      const bool near0 = zcmp(pos0, pos1) > 0;
      const int pi = near0 ? pin0 : pin1, po = near0 ? pout0 : pout1, rv = near0 ? rev0 : rev1;
      // the chord's own direction: the walk runs in -> out, reversed if rev
      const int first = rv ? po : pi, second = rv ? pi : po;
      dir = (first == ein && second == eout) ? 1 : 0;
    }
  }
  // canonical rotation: the least code over the three rotations
  const int st = star ? 1 : 0;
  const int cr0 = (st << 10) | (n0 << 7) | (n1 << 4) | (n2 << 1) | dir;
  const int cr1 = (st << 10) | (n1 << 7) | (n2 << 4) | (n0 << 1) | dir;
  const int cr2 = (st << 10) | (n2 << 7) | (n0 << 4) | (n1 << 1) | dir;
  int best = cr0, sigma = 0;
  if (cr1 < best) best = cr1, sigma = 1;
  if (cr2 < best) best = cr2, sigma = 2;
  int key = 0;
  for (int k = 0; k < NKEYS; ++k)
    if (g_keys.code[k] == best) key = k + 1;
  if (key == 0) {  // structure in the regime but no table entry: treat as Tier-G
    r.tierG = true;
    r.code = (mask & 15u) | (63u << 6) | ((u32)klass << 12);
    return r;
  }
  r.tierG = false;
  r.code = (mask & 15u) | ((u32)sigma << 4) | ((u32)key << 6) | ((u32)klass << 12);
  return r;
}

// K3a: one warp per cell bucket (1024 consecutive cell ids), four buckets
// to a block.  The bucket's pairs are counting-sorted by cell in the warp's
// shared memory -- a histogram, a scan over the 1024 cells in 32 rounds of
// the warp, a scatter -- and each cut cell gets a record, in cell order, in
// a dense range of recs drawn from a counter (bbase[b], bcut[b] records).
// The warp's one array holds the counts, then their exclusive scan, then
// (after the scatter's increments) each cell's end, which is the next cell's
// start.  No block barrier: a bucket holds a few dozen pairs, and the warps
// of a block do not wait for one another.
constexpr int SORT_W = 4;  // buckets (warps) per block
template <bool ONE>
__global__ void __launch_bounds__(32 * SORT_W) k_sort_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                       const u32* __restrict__ bpre, int njobs) {
  constexpr int NB = 1 << CB_LOG;
  __shared__ __align__(16) u32 s_c[SORT_W][NB];
  __shared__ unsigned short s_cut[SORT_W][NB];
  __shared__ u32 s_kc[SORT_W][NCLS], s_kc2[SORT_W][NCLS], s_kb[SORT_W][NCLS];
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 b = lb * SORT_W + (u32)w;
  if (b >= J.nbc) return;
  const Pair* pairs = J.pairs;
  Pair* sorted = J.raw;
  u32* c = s_c[w];
  unsigned short* cut = s_cut[w];
  const u32 lo = J.poff[b], n = J.poff[b + 1] - lo;
  const i64 c0 = (i64)b << CB_LOG;
  if (n == 0) {
    if (lane == 0) J.bcut[b] = 0, J.bbase[b] = 0;
    return;
  }
  for (int k = lane; k < NB / 4; k += 32) reinterpret_cast<uint4*>(c)[k] = make_uint4(0u, 0u, 0u, 0u);
  if (lane < NCLS) s_kc[w][lane] = 0, s_kc2[w][lane] = 0;
  __syncwarp();
  for (u32 i = lane; i < n; i += 32) atomicAdd(&c[pairs[lo + i].cell - c0], 1u);
  __syncwarp();
  // exclusive scan of the counts, and the cut cells in order
  u32 carry = 0, ncut = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < NB / 32; ++r) {
    const u32 v = c[r * 32 + lane];
    u32 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= o) inc += y;
    }
    c[r * 32 + lane] = carry + inc - v;
    carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    const unsigned m = __ballot_sync(0xFFFFFFFFu, v != 0u);
    if (v) cut[ncut + __popc(m & lt)] = (unsigned short)(r * 32 + lane);
    ncut += __popc(m);
  }
  u32 base = 0;
  if (lane == 0) base = atomicAdd(jc(J, JC_NREC), ncut);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  __syncwarp();
  for (u32 i = lane; i < n; i += 32) {
    const Pair p = pairs[lo + i];
    sorted[lo + atomicAdd(&c[p.cell - c0], 1u)] = p;
  }
  __syncwarp();
  // records (a cell's start is the previous cell's end), and their class
  // counts; then their places in the class lists (the order within a class
  // is only the classification's work order)
  for (u32 r = lane; r < ncut; r += 32) {
    const int k = cut[r];
    const u32 st = k == 0 ? 0u : c[k - 1], cnt = c[k] - st;
    J.recs[base + r] = CutRec{(u32)(c0 + k), lo + st, cnt, 0u, 0u, 0u, 0u, 0u};
    atomicAdd(&s_kc[w][piece_class(cnt)], 1u);
  }
  __syncwarp();
  if (lane < NCLS && s_kc[w][lane]) s_kb[w][lane] = atomicAdd(jc(J, JC_KCNT + lane), s_kc[w][lane]);
  __syncwarp();
  for (u32 r = lane; r < ncut; r += 32) {
    const int k = cut[r];
    const u32 st = k == 0 ? 0u : c[k - 1], cls = (u32)piece_class(c[k] - st);
    J.klist[(size_t)cls * J.NP + s_kb[w][cls] + atomicAdd(&s_kc2[w][cls], 1u)] = base + r;
  }
  if (lane == 0) J.bcut[b] = ncut, J.bbase[b] = base;
}

// ---------------------------------------------------------------------------
// Tier-T patches (Alg. 2)
// ---------------------------------------------------------------------------
// From the cell's pairs: the events in counter-clockwise order from A (their
// vertex ids staged), the labels of the patch's triangles (staged), and the
// pixel corner of P (returned; NONE without P).  Points are kept relative to
// corner A, where they fit 32 bits.
SBMT_DEV u32 stage_tier_t(const GridP& g, const CellGeo& cg, const CutRec& rec, const Pair* P, const Seg* segs,
                          const Event* ev, const unsigned char* img, i64 pitch, int dtype, TStage* out, u32* err) {
  // events as (local edge, counter-clockwise position, index); absent ones
  // carry edge 3 and sort last
  u32 e_[4] = {NONE, NONE, NONE, NONE};
  int k_[4] = {3, 3, 3, 3};
  Zq p_[4] = {zq(0), zq(0), zq(0), zq(0)};
  int ne = 0;
  u32 pcorner = NONE;
  for (u32 k = 0; k < rec.npairs; ++k) {
    const Pair pr = P[k];
#pragma unroll
    for (int end = 0; end < 2; ++end) {
      const u32 e = end == 0 ? pr.ev_in : pr.ev_out;
      if (e == NONE) {
        pcorner = corner_id(g, segs[pr.seg], end);
        continue;
      }
      if (ne >= 4) {
        atomicOr(err, ERR_COUNT);
        return NONE;
      }
      const Event x = ev[e];
      const int le = local_edge(cg, x.edge);
      if (le < 0) {
        atomicOr(err, ERR_TRAVERSAL);
        return NONE;
      }
      const Zq pos = ccw_pos(cg.down, le, x);
      // slot ne, written through fixed indices
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t == ne) e_[t] = e, k_[t] = le, p_[t] = pos;
      ++ne;
    }
  }
  // sorting network on four by (edge, position)
  auto cswap = [&](int a, int b) {
    const bool sw = k_[b] < k_[a] || (k_[b] == k_[a] && k_[a] < 3 && zcmp(p_[b], p_[a]) < 0);
    if (sw) {
      const u32 te = e_[a];
      e_[a] = e_[b], e_[b] = te;
      const int tk = k_[a];
      k_[a] = k_[b], k_[b] = tk;
      const Zq tp = p_[a];
      p_[a] = p_[b], p_[b] = tp;
    }
  };
  cswap(0, 1), cswap(2, 3), cswap(0, 2), cswap(1, 3), cswap(1, 2);
  const Pq A = lattice_pt(g, cg.ci[0], cg.cj[0]);
  int4 lp[8];  // (x.a, x.b, y.a, y.b) relative to A
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Pq q = lattice_pt(g, cg.ci[k], cg.cj[k]);
    lp[k] = make_int4((int)(q.x.a - A.x.a), (int)(q.x.b - A.x.b), (int)(q.y.a - A.y.a), (int)(q.y.b - A.y.b));
  }
  TStage st;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (e_[k] != NONE) {
      const Event x = ev[e_[k]];
      lp[3 + k] = make_int4((int)(x.xa - A.x.a), (int)(x.xb - A.x.b), (int)(x.ya - A.y.a), (int)(x.yb - A.y.b));
      st.ev[k] = x.gid;
    } else {
      lp[3 + k] = lp[0];
      st.ev[k] = NONE;
    }
  }
  if (rec.nchain == 1) {
    const Pq q = corner_of_id(g, pcorner);
    lp[7] = make_int4((int)(q.x.a - A.x.a), (int)(q.x.b - A.x.b), (int)(q.y.a - A.y.a), (int)(q.y.b - A.y.b));
  } else {
    lp[7] = lp[0];
  }
  const int key = (int)((rec.code >> 6) & 63u), sigma = (int)((rec.code >> 4) & 3u);
  const unsigned long long w = g_keys.tris[(key - 1) * 3 + sigma];
  const int nt = (int)rec.ntri;
  const Zq Sx = zq(3 * A.x.a, 3 * A.x.b), Sy = zq(3 * A.y.a, 3 * A.y.b);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    unsigned short l = 0;
    if (k < nt) {
      const int4 a = lp[tri_label(w, k, 0)], b = lp[tri_label(w, k, 1)], c = lp[tri_label(w, k, 2)];
      const Zq sx = Sx + zq((i64)a.x + b.x + c.x, (i64)a.y + b.y + c.y);
      const Zq sy = Sy + zq((i64)a.z + b.z + c.z, (i64)a.w + b.w + c.w);
      l = label_at_sum(g, img, pitch, dtype, sx, sy);
    }
    st.lab[k] = l;
  }
  *out = st;
  return rec.nchain == 1 ? pcorner : NONE;
}

// K3b: one thread per cut cell (dense): classification (key, sigma, class,
// Tier-T / Tier-G, triangle and inside-vertex counts) added to the bucket's
// totals, for a Tier-T cell its staged patch, and a Tier-G cell counted
// (cells in ngcell, triangles in ngtri, cells per local vertex count in
// gcnt, counts above TIERG_WN pooled at TIERG_WN + 1).
// The records of every job form one work queue, handed out in chunks of
// CUT_CHUNK records of one job and one piece class (recpre[njobs + 1 + k]:
// the chunks before job k), so that a block works for one job at a time with
// its descriptor in shared memory and a warp's cells have as many boundary
// pieces; the Tier-G size counts are batch-wide, so that the Tier-G
// kernels take the largest cells of the whole batch first.
template <bool ONE>
__global__ void __launch_bounds__(128, 8) k_cutcells_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                       int njobs, BatchDev* bd) {
  __shared__ Job sJ;
  __shared__ u32 s_kc[NCLS];
  const u32* cpre = bd->recpre + njobs + 1;
  u32 nchunks = 0;
  if constexpr (ONE) {
    for (int q = 0; q < NCLS; ++q) nchunks += (*jc(one, JC_KCNT + q) + CUT_CHUNK - 1) / CUT_CHUNK;
    if (threadIdx.x < NCLS) s_kc[threadIdx.x] = *jc(one, JC_KCNT + threadIdx.x);
    __syncthreads();
  } else {
    nchunks = cpre[njobs];
  }
  int cur = -1;
  for (u32 c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const Job* jp = &one;
    u32 c0 = 0;
    if constexpr (!ONE) {
      const int jk = job_of(cpre, njobs, c);
      if (jk != cur) {
        __syncthreads();
        load_job(jobs, jk, &sJ);
        if (threadIdx.x < NCLS) s_kc[threadIdx.x] = *jc(sJ, JC_KCNT + threadIdx.x);
        __syncthreads();
        cur = jk;
      }
      jp = &sJ;
      c0 = cpre[jk];
    }
    const Job& J = *jp;
    // the job's chunks run class by class: this chunk's class and place
    u32 cc = c - c0;
    int q = 0;
    for (; q < NCLS - 1; ++q) {
      const u32 nq = (s_kc[q] + CUT_CHUNK - 1) / CUT_CHUNK;
      if (cc < nq) break;
      cc -= nq;
    }
    const u32 pos = cc * CUT_CHUNK + threadIdx.x;
    if (pos >= s_kc[q]) continue;
    const u32 ri = J.klist[(size_t)q * J.NP + pos];
    const GridP& g = J.g;
    u32* err = jc(J, JC_ERR);
    CutRec rec = J.recs[ri];
    const CellGeo cg = cell_geo(g, rec.cell, cell_row_near(g, rec.cell));
    const Pair* P = J.raw + rec.pair_lo;
    const Klass kl = classify_cell(g, cg, P, rec.npairs, J.segs, J.ev, err);
    rec.code = kl.code | (kl.tierG ? (1u << 16) : 0u);
    rec.ntri = kl.ntri, rec.nchain = kl.nchain;
    // until emission, a Tier-T record keeps P's pixel corner in tri_off
    if (!kl.tierG)
      rec.tri_off = stage_tier_t(g, cg, rec, P, J.segs, J.ev, J.img, J.pitch, J.dtype, J.stg + ri, err);
    J.recs[ri] = rec;
    const u32 b = rec.cell >> CB_LOG;
    atomicAdd(&j_bextra(J)[b], kl.ntri - 1);
    if (kl.nchain) atomicAdd(&j_bchain(J)[b], kl.nchain);
    if (kl.tierG) {
      // one atomic per warp for the job's cell and triangle counts, one per
      // distinct size for the batch's per-size counts (n = ntri + 2 - n_i)
      const unsigned act = __activemask();
      const int lane = threadIdx.x & 31, lead = __ffs(act) - 1;
      const u32 t = __reduce_add_sync(act, kl.ntri);
      if (lane == lead) atomicAdd(jc(J, JC_NGCELL), (u32)__popc(act)), atomicAdd(jc(J, JC_NGTRI), t);
      const u32 n = kl.ntri + 2 - kl.nchain, key = n > TIERG_WN ? TIERG_WN + 1 : n;
      const unsigned peers = __match_any_sync(act, key);
      if (lane == __ffs(peers) - 1) atomicAdd(&bd->gcnt[key], (u32)__popc(peers));
    }
  }
}

// the jobs' record counts into the batch's prefix (one block)
__global__ void __launch_bounds__(1024) k_rec_prefix(const Job* __restrict__ jobs, int njobs, BatchDev* bd) {
  __shared__ u32 sh[1024];
  u32 carry = 0;
  for (int base = 0; base < njobs; base += 1024) {
    const int k = base + (int)threadIdx.x;
    const u32 v = k < njobs ? *jc(jobs[k], JC_NREC) : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const u32 x = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0u;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (k < njobs) bd->recpre[k] = carry + sh[threadIdx.x] - v;
    carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) bd->recpre[njobs] = carry;
  // the same over the jobs' chunks of CUT_CHUNK records
  u32* cpre = bd->recpre + njobs + 1;
  carry = 0;
  for (int base = 0; base < njobs; base += 1024) {
    const int k = base + (int)threadIdx.x;
    u32 v = 0;
    if (k < njobs)
      for (int q = 0; q < NCLS; ++q) v += (*jc(jobs[k], JC_KCNT + q) + CUT_CHUNK - 1) / CUT_CHUNK;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const u32 x = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0u;
      __syncthreads();
      sh[threadIdx.x] += x;
      __syncthreads();
    }
    if (k < njobs) cpre[k] = carry + sh[threadIdx.x] - v;
    carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) cpre[njobs] = carry;
}

// ---------------------------------------------------------------------------
// K4: emission, one warp per cell bucket (1024 consecutive cell ids), four
// buckets to a block with no block barrier
// ---------------------------------------------------------------------------
// Every uncut cell writes its base triangle (A, B, C); every Tier-T cell its
// staged patch at its offset, with P's id and coordinates.  Tier-G cells are
// left to the Tier-G kernels, which run beside this one and take their output
// ranges from the same scans.
//
// A cell's first triangle is T0 + k + (the extra triangles, ntri - 1, of the
// bucket's cut cells before it), k its index in the bucket.  Two uncut cells
// sharing an edge carry one label: a boundary crossing the edge would cut
// both cells, and none lies along it.  So a maximal run of uncut cells within
// a strip row takes the label of its first cell, and one pixel is read per
// run.  The warp's steps:
//  1. the bucket's cut-cell records give each cell its extra triangles (a
//     word per cell in shared memory, 0 for an uncut cell);
//  2. lane l takes cells 32 l .. 32 l + 31: their cut and row-start bit
//     masks give the run starts, whose pixel loads are all issued before any
//     label is stored (the label goes into the run start's word);
//  3. 32 turns over chunks of 32 consecutive cells, lane l writing cell
//     32 t + l: the chunk's scan of extra triangles gives the offsets, the
//     latest run start at or before the cell (else the one carried from
//     earlier chunks) the label, so the warp's stores of neighbouring cells
//     are adjacent;
//  4. the cut cells, a lane per record, offsets from a scan over the records.
constexpr int EMIT_W = 4;  // buckets (warps) per block

template <bool ONE>
__global__ void __launch_bounds__(32 * EMIT_W, 8) k_emit_b(const __grid_constant__ Job one,
                                                           const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                           int njobs) {
  constexpr int NB = 1 << CB_LOG;
  static_assert(NB == 32 * 32, "a lane's range is one 32-bit mask");
  __shared__ __align__(16) u32 s_x[EMIT_W][NB];  // extra triangles per cell; a run start's label after step 2
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 b = lb * EMIT_W + (u32)w;
  if (b >= J.nbc) return;
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const GridP& g = J.g;
  const CompactOut& cp = J.cp;
  u32* xs = s_x[w];
  const i64 c0 = (i64)b << CB_LOG;
  const int nc = (int)min((i64)NB, g.ncells - c0);
  const u32 ncut = J.bcut[b], rec0 = J.bbase[b];
  const int row0 = cell_row_near(g, (u32)c0);
  // 1. extra triangles per cell
  for (int k = lane; k < NB / 4; k += 32) reinterpret_cast<uint4*>(xs)[k] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
  for (u32 r = lane; r < ncut; r += 32) {
    const CutRec rec = J.recs[rec0 + r];
    xs[rec.cell - c0] = rec.ntri - 1u;  // at least 2: a cut cell is never one triangle
  }
  __syncwarp();
  // 2. this lane's cells: cut, valid and row-start masks, run starts, labels
  const int k0 = 32 * lane;
  u32 cutm = 0, xsum = 0;  // cut cells, and their extra triangles
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint4 v = reinterpret_cast<const uint4*>(xs + k0)[i];
    cutm |= (v.x ? 1u : 0u) << (4 * i) | (v.y ? 2u : 0u) << (4 * i) | (v.z ? 4u : 0u) << (4 * i) |
            (v.w ? 8u : 0u) << (4 * i);
    xsum += v.x + v.y + v.z + v.w;
  }
  // the extra triangles of the cut cells before this lane's range
  u32 xinc = xsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(FULL, xinc, o);
    if (lane >= o) xinc += y;
  }
  const u32 xex = xinc - xsum;
  const int nv = max(0, min(32, nc - k0));
  const u32 validm = nv >= 32 ? FULL : (1u << nv) - 1u;
  int r = row0;  // strip row of the lane's first cell, then of each run start
  u32 rowm = 0;
  if (nv > 0) {
    const i64 cfirst = c0 + k0;
    r = advance_row(g, row0, (u32)cfirst);
    if (g.cbase[r] == cfirst) rowm |= 1u;
    for (int q = r + 1; q < g.nrows && g.cbase[q] < cfirst + nv; ++q) rowm |= 1u << (int)(g.cbase[q] - cfirst);
  }
  const u32 prev_last = __shfl_up_sync(FULL, cutm, 1) >> 31;
  const u32 prevm = (cutm << 1) | (lane == 0 ? 1u : prev_last);  // the bucket's first cell starts a run
  const u32 startm = ~cutm & validm & (prevm | rowm);
  {
    const i64 twoS = 2 * g.S;
    const float inv2S = 1.0f / (float)twoS;
    // four run starts at a time: their loads are in flight together
    for (u32 m = startm; m;) {
      int kk[4], lab[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        kk[q] = -1;
        if (!m) continue;
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const i64 cid = c0 + k0 + i;
        r = advance_row(g, r, (u32)cid);
        const i64 c = g.clo[r] + (cid - g.cbase[r]);
        const i64 xc = g.ox + 3 * g.p * (c + g.j0 + r + 1);
        const int prow = g.lrow[2 * r + (int)(c & 1)];
        const int num = (int)(2 * xc + g.S), den = (int)twoS;
        int pcol = (int)floorf((float)num * inv2S);
        while (pcol * den > num) --pcol;
        while ((pcol + 1) * den <= num) ++pcol;
        kk[q] = k0 + i;
        lab[q] = J.dtype == 1 ? pix<unsigned char>(J.img, J.pitch, g.W, g.H, pcol, prow)
                              : pix<unsigned short>(J.img, J.pitch, g.W, g.H, pcol, prow);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (kk[q] >= 0) xs[kk[q]] = lab[q] == OUTSIDE ? 0xFFFFu : (u32)lab[q];
    }
  }
  __syncwarp();
  // the label of the latest run start before this lane's range (every uncut
  // cell has a run start at or before it in the bucket)
  u32 carry;
  {
    const u32 mylast = startm ? xs[k0 + 31 - __clz(startm)] : 0u;
    const u32 below = __ballot_sync(FULL, startm != 0u) & ((1u << lane) - 1u);
    const u32 v = __shfl_sync(FULL, mylast, below ? 31 - __clz(below) : 0);
    carry = below ? v : 0u;
  }
  // 3. uncut cells, lane l writing cell 32 t + l of chunk t; a chunk's
  // extra triangles before it and its carried label come from lane t, so the
  // chunks do not wait on one another
  const u32 T0 = (u32)c0 + J.extra_scan[b];
  int rr = row0;           // strip row of this lane's cell, advanced chunk by chunk
  i64 rnext = rr + 1 < g.nrows ? g.cbase[rr + 1] : g.ncells;
  i64 clo_r = g.clo[rr], cb_r = g.cbase[rr];
  i64 vb0 = g.vbase[rr] - g.vlo[rr], vb1 = g.vbase[rr + 1] - g.vlo[rr + 1];
#pragma unroll 4
  for (int t = 0; t * 32 < nc; ++t) {
    const int k = 32 * t + lane;
    const u32 cm = __shfl_sync(FULL, cutm, t), sm = __shfl_sync(FULL, startm, t);
    const u32 ext = __shfl_sync(FULL, xex, t), ct = __shfl_sync(FULL, carry, t);
    const u32 xv = xs[k];
    const bool cut = (cm >> lane) & 1u;
    // a chunk without cut cells (most of them) needs no scan, one without
    // run starts no label from a lane
    u32 exinc = 0;  // the extra triangles of the chunk's cut cells before this cell
    if (cm) {
      const u32 ex = cut ? xv : 0u;
      u32 inc = ex;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
      }
      exinc = inc - ex;
    }
    const u32 off = T0 + (u32)k + ext + exinc;
    u32 lab = ct;
    if (sm) {
      const u32 upto = sm & (lane == 31 ? FULL : (2u << lane) - 1u);
      const u32 lv = __shfl_sync(FULL, xv, upto ? 31 - __clz(upto) : 0);
      if (upto) lab = lv;
    }
    if (cut || k >= nc) continue;
    const i64 cid = c0 + k;
    if (cid >= rnext) {
      while (cid >= rnext) ++rr, rnext = rr + 1 < g.nrows ? g.cbase[rr + 1] : g.ncells;
      clo_r = g.clo[rr], cb_r = g.cbase[rr];
      vb0 = g.vbase[rr] - g.vlo[rr], vb1 = g.vbase[rr + 1] - g.vlo[rr + 1];
    }
    if (cp.on) {  // the base triangle stays implicit: its cell's label and code
      cp.cell_label[cid] = (unsigned short)lab, cp.cell_code[cid] = 0;
      continue;
    }
    const i64 c = clo_r + (cid - cb_r), i = c >> 1;
    int a0, a1, a2;
    if ((c & 1) == 0) a0 = (int)(vb0 + i), a1 = (int)(vb0 + i + 1), a2 = (int)(vb1 + i);
    else a0 = (int)(vb0 + i + 1), a1 = (int)(vb1 + i + 1), a2 = (int)(vb1 + i);
    J.tri[3 * (i64)off] = a0;
    J.tri[3 * (i64)off + 1] = a1;
    J.tri[3 * (i64)off + 2] = a2;
    J.label[off] = (unsigned short)lab;
    J.code[off] = 0;
  }
  // 4. cut cells, a lane per record: offsets and inside-vertex ids from
  // scans over the records (in cell order)
  const u32 CB0 = J.NVg + J.NE + J.chain_scan[b];
  const double invS = 1.0 / (double)g.S;
  u32 ex_carry = 0, ch_carry = 0;
  int row = row0;
  for (u32 base = 0; base < ncut; base += 32) {
    const u32 ri = base + (u32)lane;
    const bool valid = ri < ncut;
    CutRec rec{};
    if (valid) rec = J.recs[rec0 + ri];
    const u32 ex = valid ? rec.ntri - 1u : 0u, ch = valid ? rec.nchain : 0u;
    u32 ie = ex, ic = ch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 ye = __shfl_up_sync(FULL, ie, o), yc = __shfl_up_sync(FULL, ic, o);
      if (lane >= o) ie += ye, ic += yc;
    }
    const u32 pe = ex_carry + ie - ex, cb = CB0 + ch_carry + ic - ch;
    ex_carry += __shfl_sync(FULL, ie, 31), ch_carry += __shfl_sync(FULL, ic, 31);
    if (!valid) continue;
    const u32 kl = rec.cell - (u32)c0;
    u32 off = T0 + kl + pe;
    if (cp.on) {
      // patch triangles before this cell: those of earlier buckets, then the
      // bucket's earlier cut cells (their extra triangles plus one each)
      const u32 gi = cp.cut_scan[b] + ri;
      off = J.extra_scan[b] + cp.cut_scan[b] + ri + pe;
      cp.patch_cell[gi] = rec.cell, cp.patch_off[gi] = off;
      cp.cell_label[rec.cell] = 0xFFFF, cp.cell_code[rec.cell] = (unsigned short)(rec.code & 0xFFFFu);
    }
    if (rec.code & (1u << 16)) continue;  // Tier-G
    row = advance_row(g, row, rec.cell);
    const CellGeo cg = cell_geo(g, rec.cell, row);
    const TStage st = J.stg[rec0 + ri];
    const unsigned long long wk = g_keys.tris[(((rec.code >> 6) & 63u) - 1) * 3 + ((rec.code >> 4) & 3u)];
    const u32 ga = vid(g, cg.ci[0], cg.cj[0]), gb = vid(g, cg.ci[1], cg.cj[1]), gc = vid(g, cg.ci[2], cg.cj[2]);
    auto gid = [&](int l) -> u32 {
      switch (l) {
        case 0: return ga;
        case 1: return gb;
        case 2: return gc;
        case 3: return st.ev[0];
        case 4: return st.ev[1];
        case 5: return st.ev[2];
        case 6: return st.ev[3];
        default: return cb;
      }
    };
    const unsigned short cd = (unsigned short)(rec.code & 0xFFFFu);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      if (q >= (int)rec.ntri) break;
      const u32 o = off + (u32)q;
      J.tri[3 * (i64)o] = (int)gid(tri_label(wk, q, 0));
      J.tri[3 * (i64)o + 1] = (int)gid(tri_label(wk, q, 1));
      J.tri[3 * (i64)o + 2] = (int)gid(tri_label(wk, q, 2));
      J.label[o] = st.lab[q];
      J.code[o] = cd;
    }
    if (rec.nchain == 1) {
      const Pq p = corner_of_id(g, rec.tri_off);
      double2 vv;
      vv.x = zdouble(p.x) * invS;
      vv.y = zdouble(p.y) * invS;
      reinterpret_cast<double2*>(J.xy)[cb - cp.xy0] = vv;
    }
  }
  if (cp.on && b == J.nbc - 1 && lane == 0)
    cp.patch_off[cp.cut_scan[J.nbc]] = J.extra_scan[J.nbc] + cp.cut_scan[J.nbc];
}

// lattice vertex coordinates.  Vertex v(i, j) has x = (ox + 3p m) / S with
// m = 2i + j, so every row reads its x values from one table over the m the
// image uses (the double arithmetic is done once per m, not per vertex;
// this part has little FP64 throughput); one block per vertex row.
__global__ void __launch_bounds__(256) k_lattice_tab_b(const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                       int njobs) {
  const int jk = job_of(bpre, njobs, blockIdx.x);
  const Job& J = jobs[jk];
  const double invS = 1.0 / (double)J.g.S;
  const i64 k = (i64)(blockIdx.x - bpre[jk]) * blockDim.x + threadIdx.x;
  if (k < J.nm) J.xtab[k] = (double)(J.g.ox + 3 * J.g.p * (J.m_lo + k)) * invS;
}

__global__ void __launch_bounds__(256) k_lattice_xy_b(const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                      int njobs) {
  const int jk = job_of(bpre, njobs, blockIdx.x);
  const Job& J = jobs[jk];
  const GridP& g = J.g;
  const int r = (int)(blockIdx.x - bpre[jk]);
  const i64 j = g.vj0 + r, lo = g.vlo[r], n = g.vhi[r] - lo + 1, base = g.vbase[r];
  const double y = zdouble(zq(g.oy, 3 * g.p * j)) * (1.0 / (double)g.S);
  const double* tx = J.xtab + (2 * lo + j - J.m_lo);
  double2* out = reinterpret_cast<double2*>(J.xy) + base;
  for (i64 k = threadIdx.x; k < n; k += blockDim.x) {
    double2 v;
    v.x = tx[2 * k];
    v.y = y;
    out[k] = v;
  }
}

}  // namespace

int launch_sort_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_sort_b<true><<<nblocks, 32 * SORT_W, 0, st>>>(*one, jobs, bpre, njobs);
  else k_sort_b<false><<<nblocks, 32 * SORT_W, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

int launch_cutcells_b(const Job* one, const Job* jobs, int njobs, const BatchPtrs& bp, int blocks_per_sm,
                      cudaStream_t st) {
  if (one) {
    k_cutcells_b<true><<<152 * blocks_per_sm, 128, 0, st>>>(*one, jobs, njobs, bp.bd);
    return 1;
  }
  k_rec_prefix<<<1, 1024, 0, st>>>(jobs, njobs, bp.bd);
  k_cutcells_b<false><<<152 * blocks_per_sm, 128, 0, st>>>(Job{}, jobs, njobs, bp.bd);
  return 2;
}

int launch_emit_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_emit_b<true><<<nblocks, 32 * EMIT_W, 0, st>>>(*one, jobs, bpre, njobs);
  else k_emit_b<false><<<nblocks, 32 * EMIT_W, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

int launch_lattice_b(const Job* jobs, const u32* bpre_tab, u32 nb_tab, const u32* bpre_xy, u32 nb_xy, int njobs,
                     cudaStream_t st) {
  int n = 0;
  if (nb_tab) k_lattice_tab_b<<<nb_tab, 256, 0, st>>>(jobs, bpre_tab, njobs), ++n;
  if (nb_xy) k_lattice_xy_b<<<nb_xy, 256, 0, st>>>(jobs, bpre_xy, njobs), ++n;
  return n;
}

}  // namespace sbmt
