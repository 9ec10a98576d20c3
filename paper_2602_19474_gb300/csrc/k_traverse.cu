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
#include "sbmt_walk.cuh"

namespace sbmt {

namespace {

SBMT_DEV bool vid_ok(const GridP& g, i64 i, i64 j) {
  if (j < g.vj0 || j >= g.vj0 + g.nvrows) return false;
  const int r = (int)(j - g.vj0);
  return i >= g.vlo[r] && i <= g.vhi[r];
}

// cell (c, j) of pair k
SBMT_DEV void walk_cell(const GridP& g, const SegWalk& w, u32 k, i64* c, i64* j) {
  if (w.dir == 0) {
    *c = w.c0 + k, *j = w.j;
    return;
  }
  const i64 v = (i64)k - 1 + (w.s0 ? 0 : 1);  // virtual crossing just before the cell
  if (v < 0) {
    *j = w.j, *c = 2 * strip_ab(g, w.X, w.j);
  } else if ((v & 1) == 0) {
    Zq ys;
    i64 ei, ej, up;
    int fam;
    *j = w.j + v / 2;
    strip_slant(g, w.X, *j, &ys, &ei, &ej, &fam, &up);
    *c = up;
  } else {
    *j = w.j + (v + 1) / 2;
    *c = 2 * strip_ab(g, w.X, *j);
  }
}

// grid edge (lattice index of its lower endpoint, family) and point of crossing k
SBMT_DEV void walk_cross(const GridP& g, const SegWalk& w, u32 k, i64* ei, i64* ej, int* fam, Zq* px, Zq* py) {
  const i64 P6 = 6 * g.p;
  if (w.dir == 0) {
    const i64 c = w.c0 + k, i = c >> 1;
    *ei = i + 1, *ej = w.j, *py = zq(w.Y);
    if ((c & 1) == 0) {  // up(i, j) is left through its 120-degree edge from v(i+1, j)
      *fam = 2, *px = zq(g.ox + P6 * (i + 1 + w.j), -w.U);
    } else {  // down(i, j) through the 60-degree edge from v(i+1, j)
      *fam = 1, *px = zq(g.ox + P6 * (i + 1), w.U);
    }
    return;
  }
  const i64 v = (i64)k + (w.s0 ? 0 : 1);
  *px = zq(w.X);
  if ((v & 1) == 0) {
    i64 up;
    strip_slant(g, w.X, w.j + v / 2, py, ei, ej, fam, &up);
  } else {
    const i64 jj = w.j + (v + 1) / 2;  // the horizontal edge on top of strip jj - 1
    *ej = jj, *ei = strip_ab(g, w.X, jj), *fam = 0, *py = zq(g.oy, 3 * g.p * jj);
  }
}

// the counting phase's results per job: PSLG vertices (u64), segments, error
// bits, pairs, into mapped host memory (8 words per job)
__global__ void k_counts_b(const Job* __restrict__ jobs, int njobs, u32* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < njobs; k += gridDim.x * blockDim.x) {
    const Job& J = jobs[k];
    const unsigned long long nv = *(const unsigned long long*)J.zero;
    out[8 * k + 0] = (u32)nv, out[8 * k + 1] = (u32)(nv >> 32);
    out[8 * k + 2] = *jc(J, JC_NSEG);
    out[8 * k + 3] = *jc(J, JC_ERR);
    out[8 * k + 4] = J.pbase[min(*jc(J, JC_NSEG), J.seg_cap)];
  }
  __threadfence_system();
}

constexpr u32 CH = 2;  // pairs per thread in the chunked walks

// atomicAdd(&cur[key], 1) for each active lane, one atomic per distinct key
// among them (neighbouring lanes mostly fill the same bucket)
SBMT_DEV u32 warp_inc(u32* cur, u32 key) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  u32 at = 0;
  if (lane == leader) at = atomicAdd(cur + key, (u32)__popc(peers));
  at = __shfl_sync(peers, at, leader);
  return at + (u32)__popc(peers & ((1u << lane) - 1u));
}

// first segment of every chunk of CH pairs: chunk c starts in the segment s
// with pbase[s] <= c CH < pbase[s + 1] (every segment has at least one pair)
__global__ void __launch_bounds__(256) k_chunk_map_b(const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                     int njobs) {
  const int k = job_of(bpre, njobs, blockIdx.x);
  const Job& J = jobs[k];
  const u32 s = (blockIdx.x - bpre[k]) * blockDim.x + threadIdx.x;
  if (s >= J.nseg) return;
  const u32 a = J.pbase[s], b = J.pbase[s + 1];
  for (u32 c = (a + CH - 1) / CH; c * CH < b; ++c) J.cstart[c] = s;
}

// Chunked walk over the global pair index range, done once: every pair is
// written at its global index (raw), every event at its fixed index (segment
// event base + k), and the pairs per cell bucket and events per event bucket
// are counted (one atomic per run of equal buckets).  k_scatter then places
// pairs and event indices into their buckets.
SBMT_DEV void walk_chunk(const GridP& g, const Seg* segs, const u32* pbase, const u32* cstart, u32 NP, u32* pbk,
                        u32* ebk, Pair* raw, Event* ev, u32* err, u64 t) {
  const u64 p0 = t * CH;
  if (p0 >= NP) return;
  const u32 p1 = (u32)((p0 + CH < (u64)NP) ? p0 + CH : (u64)NP);
  u32 s = cstart[t], k = (u32)p0 - pbase[s];
  SegWalk w = seg_setup(g, segs[s]);
  u32 pb = NONE, pn = 0, eb = NONE, en = 0;
  for (u32 p = (u32)p0; p < p1; ++p, ++k) {
    if (k > w.ncross) {
      ++s, k = 0;
      w = seg_setup(g, segs[s]);
    }
    i64 c, j;
    walk_cell(g, w, k, &c, &j);
    if (!cell_in(g, c, j)) {
      atomicOr(err, ERR_TRAVERSAL);
      return;
    }
    const u32 cid = cell_id(g, c, j);
    const u32 ebase = pbase[s] - s;
    if (k < w.ncross) {
      i64 ei, ej;
      int fam;
      Zq px, py;
      walk_cross(g, w, k, &ei, &ej, &fam, &px, &py);
      if (!vid_ok(g, ei, ej)) {
        atomicOr(err, ERR_TRAVERSAL);
        return;
      }
      const u32 e = 3u * vid(g, ei, ej) + (u32)fam;
      ev[ebase + k] = Event{e, s, 0u, 0u, (int)px.a, (int)px.b, (int)py.a, (int)py.b};
      const u32 b = e >> EB_LOG;
      if (b != eb) {
        if (en) atomicAdd(ebk + eb, en);
        eb = b, en = 0;
      }
      ++en;
    }
    raw[p] = Pair{cid, s, k > 0 ? ebase + k - 1 : NONE, k < w.ncross ? ebase + k : NONE};
    const u32 b = cid >> CB_LOG;
    if (b != pb) {
      if (pn) atomicAdd(pbk + pb, pn);
      pb = b, pn = 0;
    }
    ++pn;
  }
  if (pn) atomicAdd(pbk + pb, pn);
  if (en) atomicAdd(ebk + eb, en);
}

template <bool ONE>
__global__ void __launch_bounds__(256) k_walk_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                const u32* __restrict__ bpre, int njobs) {
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const GridP& g = J.g;
  walk_chunk(g, J.segs, J.pbase, J.cstart, J.NP, j_pcnt(J), j_ecnt(J), J.raw, J.ev, jc(J, JC_ERR),
             (u64)lb * blockDim.x + threadIdx.x);
}

// pairs into their cell buckets and event indices into their event buckets
// (pcur / ecur: bucket cursors, the exclusive scans of the counts)
__global__ void __launch_bounds__(256) k_scatter_b(const Job* __restrict__ jobs, const u32* __restrict__ bpre,
                                                   int njobs) {
  const int k = job_of(bpre, njobs, blockIdx.x);
  const Job& J = jobs[k];
  const u32 i = (blockIdx.x - bpre[k]) * blockDim.x + threadIdx.x;
  if (i < J.NP) {
    const Pair pr = J.raw[i];
    J.pairs[warp_inc(J.pcur, pr.cell >> CB_LOG)] = pr;
  }
  if (i < J.NE) J.eidx[warp_inc(J.ecur, J.ev[i].edge >> EB_LOG)] = i;
}

SBMT_DEV Zq event_t(const Event& e) {
  // horizontal grid edges run +x from their lower endpoint, slanted ones +y
  return (e.edge % 3u == 0u) ? zq(e.xa, e.xb) : zq(e.ya, e.yb);
}

// The registry: one block per event bucket (2048 consecutive grid-edge ids).
// An event's vertex id is NVg + (events on lower edge ids) + (events on its
// edge nearer the edge's lower endpoint), compared exactly.  A bucket of at
// most 256 events ranks each event against the others held in shared
// memory; a larger one counting-sorts its events by edge first.
// The registry, small buckets (at most RANK_SMALL events, nearly all of
// them): a 64-thread block per bucket, each event ranked by a count over
// the bucket's events held in shared memory.
SBMT_DEV void rank_small_bucket(const GridP& g, Event* ev, const u32* eidx, const u32* eoff, u32 bucket, u32 NVg,
                                double* xy, u32 xy0, u32* s_edge, int* s_ta, int* s_tb) {
  const u32 lo = eoff[bucket], n = eoff[bucket + 1] - lo;
  if (n == 0 || n > RANK_SMALL) return;
  const double invS = 1.0 / (double)g.S;
  u32 me[RANK_SMALL / 64];
#pragma unroll
  for (int u = 0; u < (int)(RANK_SMALL / 64); ++u) {
    const u32 i = threadIdx.x + 64u * u;
    if (i < n) {
      me[u] = eidx[lo + i];
      const Event x = ev[me[u]];
      const bool horiz = x.edge % 3u == 0u;
      s_edge[i] = x.edge, s_ta[i] = horiz ? x.xa : x.ya, s_tb[i] = horiz ? x.xb : x.yb;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < (int)(RANK_SMALL / 64); ++u) {
    const u32 i = threadIdx.x + 64u * u;
    if (i >= n) break;
    const u32 xe = s_edge[i];
    const Zq ti = zq(s_ta[i], s_tb[i]);
    u32 rank = 0;
    for (u32 q = 0; q < n; ++q) {
      const u32 eq = s_edge[q];
      if (eq < xe || (eq == xe && q != i && zcmp(zq(s_ta[q], s_tb[q]), ti) < 0)) ++rank;
    }
    const u32 gid = NVg + lo + rank;
    const Event x = ev[me[u]];
    ev[me[u]].gid = gid;
    double2 v;
    v.x = zdouble(zq(x.xa, x.xb)) * invS;
    v.y = zdouble(zq(x.ya, x.yb)) * invS;
    reinterpret_cast<double2*>(xy)[gid - xy0] = v;
  }
}

template <bool ONE>
__global__ void __launch_bounds__(64) k_rank_small_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                     const u32* __restrict__ bpre, int njobs) {
  __shared__ u32 s_edge[RANK_SMALL];
  __shared__ int s_ta[RANK_SMALL], s_tb[RANK_SMALL];
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const GridP& g = J.g;
  rank_small_bucket(g, J.ev, J.eidx, J.eoff, lb, J.NVg, J.xy, J.cp.xy0, s_edge, s_ta, s_tb);
}

// The registry, large buckets (grid-edge buckets along the image border
// collect thousands of events): a counting sort of the bucket's events by
// grid edge, then each event ranked among those of its own edge.  A short
// grid walks over all buckets and skips the small ones.
constexpr int NEB = 1 << EB_LOG;
SBMT_DEV void rank_large_bucket(const GridP& g, Event* ev, const u32* eidx, u32* elist, const u32* eoff, u32 b,
                                u32 NVg, double* xy, u32 xy0, u32* s_cnt, u32* s_off, u32* s_cur, u32* s_sh) {
  const double invS = 1.0 / (double)g.S;
  {
    const u32 lo = eoff[b], n = eoff[b + 1] - lo;
    if (n <= RANK_SMALL) return;
    const u32 e0 = b << EB_LOG;
    for (int k = threadIdx.x; k < NEB; k += blockDim.x) s_cnt[k] = 0;
    __syncthreads();
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&s_cnt[ev[eidx[lo + i]].edge - e0], 1u);
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
      const u32 slot = atomicAdd(&s_cur[ev[eidx[lo + i]].edge - e0], 1u);
      elist[lo + slot] = eidx[lo + i];
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < n; i += blockDim.x) {
      const u32 me = eidx[lo + i];
      const Event ei = ev[me];
      const Zq ti = event_t(ei);
      const u32 k = ei.edge - e0, first = s_off[k], cnt = s_cnt[k];
      u32 rank = first;
      for (u32 q = 0; q < cnt; ++q) {
        const u32 j = elist[lo + first + q];
        if (j != me && zcmp(event_t(ev[j]), ti) < 0) ++rank;
      }
      const u32 gid = NVg + lo + rank;
      ev[me].gid = gid;
      double2 v;
      v.x = zdouble(zq(ei.xa, ei.xb)) * invS;
      v.y = zdouble(zq(ei.ya, ei.yb)) * invS;
      reinterpret_cast<double2*>(xy)[gid - xy0] = v;
    }
    __syncthreads();
  }
}

// the large buckets of every job, from the batch's list (filled by the scan
// of the event bucket counts)
template <bool ONE>
__global__ void __launch_bounds__(256) k_rank_big_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                    const BatchDev* bd, const uint2* big) {
  __shared__ u32 s_cnt[NEB], s_off[NEB], s_cur[NEB];
  __shared__ u32 s_sh[8];
  __shared__ Job sJ;
  const u32 n = bd->nbig;
  for (u32 it = blockIdx.x; it < n; it += gridDim.x) {
    const uint2 e = big[it];
    const Job* jp = &one;
    if constexpr (!ONE) {
      __syncthreads();
      load_job(jobs, (int)e.x, &sJ);
      jp = &sJ;
    }
    const Job& J = *jp;
    const GridP& g = J.g;
    rank_large_bucket(g, J.ev, J.eidx, J.elist, J.eoff, e.y, J.NVg, J.xy, J.cp.xy0, s_cnt, s_off, s_cur, s_sh);
  }
}

}  // namespace

size_t walk_chunks(u32 NP) { return (NP + CH - 1) / CH; }

int launch_counts_b(const Job* jobs, int njobs, u32* out, cudaStream_t st) {
  k_counts_b<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, njobs, out);
  return 1;
}

int launch_chunk_map_b(const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  k_chunk_map_b<<<nblocks, 256, 0, st>>>(jobs, bpre, njobs);
  return 1;
}

int launch_walk_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_walk_b<true><<<nblocks, 256, 0, st>>>(*one, jobs, bpre, njobs);
  else k_walk_b<false><<<nblocks, 256, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

int launch_scatter_b(const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  k_scatter_b<<<nblocks, 256, 0, st>>>(jobs, bpre, njobs);
  return 1;
}

int launch_rank_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, const BatchPtrs& bp,
                  cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_a, cudaEvent_t ev_b) {
  if (nblocks == 0) return 0;
  if (st2) {
    if (cudaEventRecord(ev_a, st) != cudaSuccess || cudaStreamWaitEvent(st2, ev_a, 0) != cudaSuccess) return -1;
  }
  if (one) {
    k_rank_big_b<true><<<152 * 2, 256, 0, st2 ? st2 : st>>>(*one, jobs, bp.bd, bp.big);
    k_rank_small_b<true><<<nblocks, 64, 0, st>>>(*one, jobs, bpre, njobs);
  } else {
    k_rank_big_b<false><<<152 * 2, 256, 0, st2 ? st2 : st>>>(Job{}, jobs, bp.bd, bp.big);
    k_rank_small_b<false><<<nblocks, 64, 0, st>>>(Job{}, jobs, bpre, njobs);
  }
  if (st2) {
    if (cudaEventRecord(ev_b, st2) != cudaSuccess || cudaStreamWaitEvent(st, ev_b, 0) != cudaSuccess) return -1;
  }
  return 2;
}

}  // namespace sbmt
