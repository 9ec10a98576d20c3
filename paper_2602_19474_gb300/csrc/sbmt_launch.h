// sbmt_launch.h -- host-side launchers of the SBMT kernels (one per step of
// the hot path), called by the C interface in sbmt_api.cu.  Each returns the
// number of kernels it launched.
#pragma once
#include <cuda_runtime.h>

#include "sbmt_dev.cuh"

namespace sbmt {

// ---------------------------------------------------------------------------
// Batched launches.  A batch of images (one image is a batch of one) runs
// every stage of the path as one launch over a job table: job k is image k
// with its grid, its image and its buffers.  The blocks of a launch are split
// among the jobs by a prefix of per-job block counts (bpre, njobs + 1
// entries); block b works for the job k with bpre[k] <= b < bpre[k + 1].
// The stages whose work is only known on the device (cut cells, Tier-G
// cells, the large registry buckets) are persistent kernels that pull items
// from batch-wide work queues.
// ---------------------------------------------------------------------------
// counters of one job, in its zeroed block (words): the PSLG vertex count
// (u64 at 0), the status words at 8.. (see JC_*), then the per-bucket counts
constexpr int JC_NSEG = 8, JC_ERR = 10, JC_NREC = 11, JC_NGCELL = 12, JC_NGTRI = 13, JC_NOVER = 14;
// cut cells by their number of boundary pieces (1, 2, 3, 4, 5 or more), so
// that the classification's warps run cells of one shape: counts at JC_KCNT
constexpr int NCLS = 5, JC_KCNT = 16;
constexpr int JC_BUCKETS = 24;
SBMT_HD int piece_class(u32 npairs) { return npairs >= (u32)NCLS ? NCLS - 1 : (int)npairs - 1; }
struct __align__(16) Job {
  GridP g;
  const unsigned char* img;
  i64 pitch;
  int dtype;
  int wpr, wpc;
  u32* vrow;
  u32* vcol;
  u32* zero;  // counters (JC_*), then pcnt (nbc + 1), ecnt (nbe + 1), bextra (nbc + 1), bchain (nbc + 1)
  Seg* segs;
  u32 seg_cap;
  u32* npairs;  // seg_cap values
  u32* pbase;   // seg_cap + 1 values
  // known after the counting phase
  u32 nseg, NP, NE, NVg, nbc, nbe;
  u32* cstart;
  Pair* raw;     // pairs in walk order, later sorted by cell
  Pair* pairs;   // pairs in cell buckets
  Event* ev;
  u32* eidx;
  u32* elist;
  u32 *poff, *eoff, *pcur, *ecur;
  CutRec* recs;
  u32* klist;  // record indices by piece class: NCLS regions of NP entries
  u32 *bcut, *bbase, *extra_scan, *chain_scan, *cut_scan;
  TStage* stg;
  int* tri;
  unsigned short* label;
  unsigned short* code;
  double* xy;
  CompactOut cp;
  double* xtab;
  i64 m_lo, nm;
  u32* over;   // ids of cells over the Tier-G limit (OVER_CAP)
  u32* hinfo;  // host status words (mapped pinned memory), written at the end
};
SBMT_DEV u32* jc(const Job& J, int k) { return J.zero + k; }
SBMT_DEV u32* j_pcnt(const Job& J) { return J.zero + JC_BUCKETS; }
SBMT_DEV u32* j_ecnt(const Job& J) { return J.zero + JC_BUCKETS + J.nbc + 1; }
SBMT_DEV u32* j_bextra(const Job& J) { return J.zero + JC_BUCKETS + J.nbc + 1 + J.nbe + 1; }
SBMT_DEV u32* j_bchain(const Job& J) { return J.zero + JC_BUCKETS + 2 * (J.nbc + 1) + J.nbe + 1; }
inline size_t job_zero_words(u32 nbc, u32 nbe) { return JC_BUCKETS + 3 * ((size_t)nbc + 1) + (nbe + 1); }

// the job of a block-uniform kernel, copied once into shared memory so that
// its fields do not occupy registers for the whole kernel
SBMT_DEV void load_job(const Job* jobs, int k, Job* sj) {
  const int4* src = reinterpret_cast<const int4*>(jobs + k);
  int4* dst = reinterpret_cast<int4*>(sj);
  for (int i = threadIdx.x; i < (int)(sizeof(Job) / 16); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// The job of a block-uniform kernel.  A launch for one image (ONE) takes its
// job as a kernel parameter, whose fields the kernel reads as constant-bank
// operands; a batched launch finds the block's job from the block prefix
// and copies it into shared memory.  Declares J (the job), jk (its index)
// and lb (the block's index within the job).
#define SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)  \
  __shared__ Job sJ_;                                 \
  int jk = 0;                                         \
  u32 lb = blockIdx.x;                                \
  const Job* jp_ = &one;                              \
  if constexpr (!ONE) {                               \
    jk = job_of(bpre, njobs, blockIdx.x);             \
    load_job(jobs, jk, &sJ_);                         \
    jp_ = &sJ_;                                       \
    lb = blockIdx.x - bpre[jk];                       \
  }                                                   \
  const Job& J = *jp_;

// the job of block b: the last k with bpre[k] <= b
SBMT_DEV int job_of(const u32* bpre, int njobs, u32 b) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(bpre + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// batch-wide state of the persistent stages
struct BatchDev {
  u32 gcnt[TIERG_WN + 2];  // Tier-G cells per local vertex count (above TIERG_WN pooled)
  u32 gcur[TIERG_WN + 2];  // cursors while ordering
  u32 nolist, nwlist, nbig, err;
  u32 nslist;              // cells of the small-state warp list
  u32 recpre[1];           // 2 (njobs + 1) entries: prefix of the jobs' cut-cell records, then of
                           // their chunks of CUT_CHUNK records
};
inline size_t batch_dev_words(int njobs) { return sizeof(BatchDev) / 4 + 2 * ((size_t)njobs + 1); }
constexpr u32 CUT_CHUNK = 128;  // records per block and turn of the persistent cut-cell kernel
struct BatchPtrs {
  BatchDev* bd;
  uint2* olist;  // (job, record) of Tier-G cells of at most TIERG_TN vertices, largest first
  uint2* slist;  // (job, record) of Tier-G cells of TIERG_TN + 1 .. TIERG_WN vertices, largest first
  uint2* wlist;  // (job, record) of Tier-G cells above TIERG_WN vertices
  uint2* big;    // (job, event bucket) of registry buckets above RANK_SMALL events
};

// one prefix sum of a batched scan: out[i] = sum of in[0..i), out[n] = total,
// also into out2 when given; with big, the indices of values above big_thr
// are listed as (img, index) in big (count in *nbig)
struct ScanJob {
  const u32* in;
  u32* out;
  u32* out2;
  u32 n;             // values (the tiles cover n + 1 outputs)
  const u32* n_dev;  // or null: the number of values is min(*n_dev, n), known on the device only
  int img;
  u32 big_thr;
  uint2* big;
  u32* nbig;
  u32* err;  // the image's error word (ERR_TIMEOUT when a wait ran out)
};
constexpr int MSCAN_TILE = 2048;
inline u32 mscan_tiles(u32 n) { return (n + 1 + MSCAN_TILE - 1) / MSCAN_TILE; }
// single-pass scans of every job in one launch (tpre: prefix of the jobs'
// tiles; flags: tpre[nsj] words of zeroed scratch for the tiles' published
// sums, ticket: one zeroed word).  Each tile waits for its predecessor's
// prefix with a bounded wait (about one second), after which it records
// ERR_TIMEOUT and publishes an error mark.  stall_tile (NONE normally)
// names a tile that withholds its sums, so that the wait of its successor
// runs out -- the test of the bound.
int launch_mscan(const ScanJob* sj, const u32* tpre, int nsj, u32 ntiles, unsigned long long* flags, u32* ticket,
                 u32 stall_tile, cudaStream_t st);

// batched stages (jobs and the block prefix bpre in device memory; nblocks =
// bpre[njobs]); each returns the kernels it launched.  `one` is the host
// copy of the job when the launch has a single job (then passed as a kernel
// parameter), else null.
int launch_corner_bits_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
int launch_segments_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
// each segment's pair count (cells visited) into npairs, over the segments
// the device counted (a job's blocks stride over them)
int launch_seg_count_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
// per job {PSLG vertices (2 words), segments, error, pairs} into out (mapped
// host memory)
int launch_counts_b(const Job* jobs, int njobs, u32* out, cudaStream_t st);
int launch_chunk_map_b(const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
int launch_walk_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
int launch_scatter_b(const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
// registry: small buckets one block each (bpre over nbe), large ones from
// the batch's list on st2 (or st) beside them
int launch_rank_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, const BatchPtrs& bp,
                  cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_a, cudaEvent_t ev_b);
int launch_sort_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
// cut-cell classification, persistent over every job's records
int launch_cutcells_b(const Job* one, const Job* jobs, int njobs, const BatchPtrs& bp, int blocks_per_sm,
                      cudaStream_t st);
int launch_emit_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st);
int launch_lattice_b(const Job* jobs, const u32* bpre_tab, u32 nb_tab, const u32* bpre_xy, u32 nb_xy, int njobs,
                     cudaStream_t st);
// Tier-G: ordering (bpre over warps of buckets), then the persistent thread
// and warp kernels over the batch's lists (warp kernels on st2 when given).
// Cells of at most TIERG_TN vertices run one thread each, larger ones one warp
// each (a small-state kernel up to TIERG_WN vertices, a large-state one above).
int launch_tierg_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, const BatchPtrs& bp,
                   int thread_blocks_per_sm, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_order,
                   cudaEvent_t ev_warp);
// kernel attributes set once per device (outside any stream capture)
int tierg_init();
// status words of every job into its mapped host slot
int launch_status_b(const Job* jobs, int njobs, const BatchPtrs& bp, cudaStream_t st);

// K1a: vertex flags of every pixel corner, bit-packed per corner row (vrow)
// and per corner column (vcol); counts the PSLG vertices into *nvtx.
int launch_corner_bits(const unsigned char* img, i64 pitch, int dtype, int W, int H, u32* vrow, int wpr,
                        u32* vcol, int wpc, unsigned long long* nvtx, cudaStream_t st);

// K1b: maximal boundary runs between PSLG vertices, compacted into segs.
int launch_segments(const unsigned char* img, i64 pitch, int dtype, int W, int H, const u32* vrow, int wpr,
                     const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, cudaStream_t st);

// K2 walk, chunked over the global pair index: walk_chunks(NP) chunks of
// pairs, one thread each.
size_t walk_chunks(u32 NP);

// exclusive scan of n u32 values with stride `stride` into out (n + 1
// entries, out[n] = total); inputs above 65536 values need scratch of
// scan_scratch_words(n) words
size_t scan_scratch_words(u32 n);
int launch_scan(const u32* in, int stride, u32* out, u32 n, u32* scratch, cudaStream_t st);

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

// Region III (Alg. 2 on an arbitrary counter-clockwise mesh T, the
// preprocessed one): the image, T (nv vertices as double pairs, nt cells as
// vertex-id triples), the per-vertex cell lists (deg: nv counts, vptr:
// nv + 1 offsets, inc: 3 nt cell ids), per cell the triangle count, the
// events on the edges it owns (the smaller cell beside an edge), the inside
// vertices and the owned events per local edge (8 bits each), their
// exclusive scans (nt + 1 each), the output mesh, the Tier-G queue (nt
// entries) and its length, the error word and counters.
enum : u32 { R3_CAPACITY = 1u, R3_GEOMETRY = 2u, R3_COUNT = 4u };
struct R3Args {
  const unsigned char* img;
  i64 pitch;
  int dtype, W, H;
  const double* txy;
  const int* ttri;
  u32 nv;
  u64 nt;
  u32 *deg, *vptr, *inc;
  u32 *ntri, *nown, *nin, *own3;
  u32 *toff, *eoff, *ioff;
  u32 ne_total;
  double* xy;
  int* tri;
  unsigned short *label, *code;
  u32 *glist, *ng, *err, *ncut, *ngtri;  // glist: the Tier-G cells (bit 31: over 12 nodes), ng of them
  unsigned short* ulab;  // per cell: the label of an uncut cell's pixel box
  u32* cmark;            // candidate bit-plane, (nt + 31) / 32 words
  u32 *cand, *ncand;     // the candidates (nt entries) and their count
  u32* ngsmall;          // Tier-G cells done by one thread
  u32* cutl;             // the cut cells (nt entries), ncut of them
};
int launch_r3_adjacency(const R3Args& a, u32* scr, cudaStream_t st);
int launch_r3_count(const R3Args& a, cudaStream_t st);
int launch_r3_emit(const R3Args& a, cudaStream_t st);

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

}  // namespace sbmt
