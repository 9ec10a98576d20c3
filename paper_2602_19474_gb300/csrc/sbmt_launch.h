// sbmt_launch.h -- host-side launchers of the SBMT kernels (one per step of
// the hot path), called by the C interface in sbmt_api.cu.  Each returns the
// number of kernels it launched.
#pragma once
#include <cuda_runtime.h>

#include "sbmt_dev.cuh"

namespace sbmt {

// K1a: vertex flags of every pixel corner, bit-packed per corner row (vrow)
// and per corner column (vcol); counts the PSLG vertices into *nvtx.
int launch_corner_bits(const unsigned char* img, i64 pitch, int dtype, int W, int H, u32* vrow, int wpr,
                        u32* vcol, int wpc, unsigned long long* nvtx, cudaStream_t st);

// K1b: maximal boundary runs between PSLG vertices, compacted into segs.
int launch_segments(const unsigned char* img, i64 pitch, int dtype, int W, int H, const u32* vrow, int wpr,
                     const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, cudaStream_t st);

// K2: number of pairs (cells visited = crossings + 1) of every segment, in
// closed form; slots beyond the segment count get 0.
int launch_seg_count(const GridP& g, const Seg* segs, const u32* nseg, u32 cap, u32* npairs, cudaStream_t st);

// K2 walk, chunked over the global pair index (pbase = exclusive scan of
// npairs; cstart = first segment of every chunk, from launch_chunk_map over
// walk_chunks(NP) chunks): every pair at its global index in raw, every event
// at its fixed index, pairs per cell bucket counted into pbk and events per
// event bucket into ebk.  launch_scatter then moves the pairs into their cell
// buckets and the event indices into their event buckets (pcur / ecur: the
// buckets' cursors, starting at the exclusive scans of pbk / ebk).
size_t walk_chunks(u32 NP);
int launch_chunk_map(const u32* pbase, const u32* nseg, u32 cap, u32* cstart, cudaStream_t st);
int launch_walk(const GridP& g, const Seg* segs, const u32* pbase, const u32* cstart, u32 NP, u32* pbk, u32* ebk,
                Pair* raw, Event* events, u32* err, cudaStream_t st);
int launch_scatter(const Pair* raw, u32 NP, const Event* events, u32 NE, u32* pcur, u32* ecur, Pair* pairs,
                   u32* eidx, cudaStream_t st);

// frozen registry: rank the events of each event bucket (listed in eidx) by
// (grid-edge id, position), assign vertex ids NVg + rank, write coordinates.
// With st2 the few large buckets are ranked there beside the small ones
// (ev_a, ev_b fork and join); returns the kernels launched, -1 when an
// event call failed.
int launch_rank_events(const GridP& g, Event* events, const u32* eidx, u32* elist, const u32* eoff, u32 nbe,
                        u32 NVg, double* xy, u32 xy0, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_a,
                        cudaEvent_t ev_b);

// K3a: sort each cell bucket's pairs by cell into sorted; one record per cut
// cell, in cell order, in a dense range of recs drawn from *nrec (bucket b:
// bcut[b] records from bbase[b]).
int launch_sort(const Pair* pairs, Pair* sorted, const u32* poff, u32 nbc, CutRec* recs, u32* nrec, u32* bcut,
                 u32* bbase, cudaStream_t st);

// K3b: classify every cut cell (key, sigma, class, Tier-T / Tier-G, triangle
// and inside-vertex counts, added per bucket into bextra / bchain) and stage
// the patch of every Tier-T cell in stg (same index as its record).
int launch_cutcells(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                     const Seg* segs, const Event* events, CutRec* recs, const u32* nrec, u32* bextra, u32* bchain,
                     TStage* stg, u32* ngcell, u32* ngtri, u32* gcnt, u32* err, cudaStream_t st);

// exclusive scan of n u32 values with stride `stride` into out (n + 1
// entries, out[n] = total); inputs above 65536 values need scratch of
// scan_scratch_words(n) words
size_t scan_scratch_words(u32 n);
// exclusive scans of one or two arrays (in_b = nullptr for one) of at most
// SCAN_ONE values each in one launch, the results also copied to out2 when
// given (nullptr otherwise)
constexpr u32 SCAN_ONE = 1u << 14;
int launch_scan_pair(const u32* in_a, u32* out_a, u32* out2_a, u32 n_a, const u32* in_b, u32* out_b, u32* out2_b,
                     u32 n_b, cudaStream_t st);
int launch_scan(const u32* in, int stride, u32* out, u32 n, u32* scratch, cudaStream_t st);

// K4: per cell bucket, emit every uncut cell's base triangle and every
// Tier-T cell's staged patch (Alg. 2) with its inside vertex (Tier-G cells
// are skipped: k_cutcells queued them, the Tier-G kernels place them).
int launch_emit(const GridP& g, const unsigned char* img, i64 pitch, int dtype, CutRec* recs, const u32* bcut,
                 const u32* bbase, const u32* extra_scan, const u32* chain_scan, const TStage* stg, u32 nbc, u32 NVg,
                 u32 NE, int* tri, unsigned short* label, unsigned short* code, double* xy, const CompactOut& cp,
                 cudaStream_t st);

// K4-G: greedy Steiner-free triangulation of every queued Tier-G cell.  The
// cells are first ordered by local vertex count, largest first, into olist
// (gcnt: zeroed, 3 * (TIERG_TN + 2) words; its first TIERG_TN + 2 are the
// per-count totals k_cutcells gathered), each cell's output range taken from
// the scans (cut_scan for the compact format, else null; CB0 = the first
// inside-vertex id); one thread per cell of at most TIERG_TN vertices, one
// warp per larger cell (through wlist).  A cell over the per-cell limit
// sets ERR_CAPACITY, counts itself in *nover and lists its id in over
// (OVER_CAP at most).  With st2 the warp kernel runs there,
// after ev_order (recorded on st after the ordering), and st waits for it
// through ev_warp; without, everything runs on st.  Returns the kernels
// launched, or -1 when an event call failed.
int launch_tierg(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                  const Seg* segs, const Event* events, CutRec* recs, const u32* bcut, const u32* bbase, u32 nbc,
                  u32* gcnt, u32* olist, u32* wlist, u32* nwlist, const u32* extra_scan, const u32* chain_scan,
                  const u32* cut_scan, u32 CB0, int* tri, unsigned short* label, unsigned short* code, double* xy,
                  u32 xy0, u32* err, u32* nover, u32* over, cudaStream_t st, cudaStream_t st2,
                  cudaEvent_t ev_order, cudaEvent_t ev_warp);

// quality measures: per-triangle pass (mm: min angle, min area, max AR as
// double bits; cnt: slivers, equilateral; part: per-block area sums; ar:
// AR per triangle as float) and one level of the radix select of two ranks
int launch_quality(const double* xy, const int* tri, u64 T, float* ar, unsigned long long* mm,
                   unsigned long long* cnt, double* part, int nblocks, u32* hist, cudaStream_t st);
int launch_select_hist(const float* v, u64 T, int lo, int width, u32 pre0, u32 pre1, int above, u32* h0, u32* h1,
                       cudaStream_t st);

// projection of a float pixel field (row pitch fpitch bytes): per-triangle
// means into tri_value and bilinear vertex values into vertex_value (either
// may be null); scratch holds project_scratch_bytes(V) bytes (16-byte
// aligned) for the vertices' split coordinates; returns the number of
// kernels launched, -1 if T >= 2^32
size_t project_scratch_bytes(u64 V);
int launch_project(const double* xy, const int* tri, u64 T, u64 V, const float* f, i64 fpitch, int W, int H,
                   float* tri_value, float* vertex_value, void* scratch, cudaStream_t st);

// geometric preprocessing of the base mesh (Alg. 3, Steps 1-3), on the PSLG
// vertex flags vrow of launch_corner_bits.  Thresholds in pixels; the *scr
// fields are their screening radii (each plus the float rounding margin of
// the coordinates), bscr2 = bscr^2.  Scratch: tab / tabf (nm entries, the
// x table over m0 <= m < m0 + nm), prow (2 per strip row), xyf (float copy
// of the moved lattice positions), plist (np boundary points), cand
// (pre_cand_bytes(np)), appl / ascan (np and np + 1 words), sbit / spop /
// wpre (split-cell bit-plane of ncells / 32 + 1 words, its counts and their
// scan), ytab / ytabf / vqn (one per vertex row), vq / rq (nverts), cnt
// (7 zeroed words: error, eliminations, split cells, snapped, repelled,
// points with a candidate, the Step 2 queue length).  Outputs: xy (lattice vertices, then
// the inserted points), tri / label / code (ncells + split cells
// triangles), status and snap per lattice vertex, elim (3 per elimination).
struct PreCand;
struct PreArgs {
  GridP g;
  const unsigned char* img;
  i64 pitch;
  int dtype;
  const u32* vrow;
  int wpr;
  u32 np;
  double A, B2, C;
  float ascr, bscr, bscr2, cscr, reach;  // reach: a + b plus the margin
  // float decisions: dband bounds the error of a float distance; r_lo2 =
  // (r - dband)^2 (or -1), r_hi2 = (r + dband)^2 for r = a, b, c
  float dband, a_lo2, a_hi2, b_lo2, b_hi2, c_hi2;
  float oxf, oyf, hf, rowh;              // origin, h and the strip height in pixels
  i64 m0, nm;
  double* tab;
  float* tabf;
  double* ytab;  // y of every vertex row, and its float copy
  float* ytabf;
  u32* vq;       // Region I queue: vertex ids, in each row's own id range
  u32* vqn;      // queued vertices per vertex row
  uint2* rq;     // Step 2 queue: (vertex id, vertex row), nverts entries
  int* prow;
  float2* xyf;
  u32* plist;
  PreCand* cand;
  u32 *appl, *ascan, *sbit, *spop, *wpre, *cnt;
  double* xy;
  int* tri;
  unsigned short *label, *code;
  unsigned char* status;
  int *snap, *elim;
};
size_t pre_cand_bytes(u32 np);
// nw vrow words; wpop / wscan: nw and nw + 1 words; scr: scan scratch for
// the largest of nw, np and ncells / 32 + 1.  Returns the kernels launched,
// -1 if a CUDA call failed.
int launch_preprocess(const PreArgs& a, u64 nw, u32* wpop, u32* wscan, u32* scr, cudaStream_t st);

// heat diffusion on the triangles of label L (backward Euler, cotangent
// stiffness, lumped mass, preconditioned conjugate gradients to relative
// residual tol, at most maxit iterations per step): u (device, V doubles)
// receives the solution; peaks / iters (host, nsteps each, or null) the
// maximum of u and the iterations after each step.  scratch holds
// heat_scratch_bytes(T, V, maxit) bytes (256-byte aligned).  Synchronises
// with the device a few times per step; returns the kernels launched, -1 if
// a CUDA call failed, -2 if a step did not converge.
size_t heat_scratch_bytes(u64 T, u64 V, int maxit);
int heat_solve(const double* xy, const int* tri, const unsigned short* label, u64 T, u64 V, int L, double alpha,
               double dt, int nsteps, double x0, double y0, double sigma, double amp, double tol, int maxit,
               double* u, double* peaks, int* iters, void* scratch, cudaStream_t st);

// coordinates of the lattice vertices; tab: scratch of nm doubles for the x
// values (ox + 3p m) / S, m0 <= m < m0 + nm covering 2i + j of every vertex
int launch_lattice_xy(const GridP& g, double* xy, double* tab, i64 m0, i64 nm, cudaStream_t st);

}  // namespace sbmt
