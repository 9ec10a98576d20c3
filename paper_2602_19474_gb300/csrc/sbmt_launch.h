// sbmt_launch.h -- host-side launchers of the SBMT kernels (one per step of
// the hot path), called by the C interface in sbmt_api.cu.
#pragma once
#include <cuda_runtime.h>

#include "sbmt_dev.cuh"

namespace sbmt {

// K1a: vertex flags of every pixel corner, bit-packed per corner row (vrow)
// and per corner column (vcol); counts the PSLG vertices into *nvtx.
void launch_corner_bits(const unsigned char* img, i64 pitch, int dtype, int W, int H, u32* vrow, int wpr,
                        u32* vcol, int wpc, unsigned long long* nvtx, cudaStream_t st);

// K1b: maximal boundary runs between PSLG vertices, compacted into segs.
void launch_segments(const unsigned char* img, i64 pitch, int dtype, int W, int H, const u32* vrow, int wpr,
                     const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, cudaStream_t st);

// K2 count pass: per segment, the cells it visits and the grid edges it
// crosses, histogrammed into cell buckets and event buckets.
void launch_traverse_count(const GridP& g, const Seg* segs, const u32* nseg, u32 seg_cap, u32* pcnt, u32* ecnt,
                           unsigned long long* totals, u32* err, cudaStream_t st);

// K2 emit pass: writes pairs and events into their buckets.
void launch_traverse_emit(const GridP& g, const Seg* segs, const u32* nseg, u32 seg_cap, u32* pcur, u32* ecur,
                          Pair* pairs, Event* events, u32* err, cudaStream_t st);

// frozen registry: rank events by (grid-edge id, position) inside each event
// bucket, assign vertex ids NVg + rank, write their coordinates.
void launch_rank_events(const GridP& g, Event* events, u32* elist, const u32* eoff, u32 nbe, u32 NVg, double* xy,
                        cudaStream_t st);

// K3: sort each cell bucket's pairs by cell, classify every cut cell (key,
// sigma, class, Tier-T / Tier-G, triangle and inside-vertex counts).
void launch_classify(const GridP& g, const Pair* pairs, Pair* sorted, const u32* poff, u32 nbc, const Seg* segs,
                     const Event* events, CutRec* recs, u32* bstat, u32* err, cudaStream_t st);

// exclusive scan of n u32 values with stride `stride` into out (n + 1
// entries, out[n] = total), single block
void launch_scan(const u32* in, int stride, u32* out, u32 n, cudaStream_t st);

// K4: emit every uncut cell's base triangle and every Tier-T patch; queue
// the Tier-G cells.
void launch_emit(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                 const Seg* segs, const Event* events, CutRec* recs, const u32* poff, const u32* bstat,
                 const u32* extra_scan, const u32* chain_scan, u32 nbc, u32 NVg, u32 NE, int* tri,
                 unsigned short* label, unsigned short* code, double* xy, u32* glist, u32* nglist, u32* ngtri,
                 u32* err, cudaStream_t st);

// K4-G: greedy Steiner-free triangulation of every queued Tier-G cell (one
// thread per small cell; cells above the thread limit go to a warp each
// through wlist).
void launch_tierg(const GridP& g, const unsigned char* img, i64 pitch, int dtype, const Pair* sorted,
                  const Seg* segs, const Event* events, const CutRec* recs, const u32* glist, const u32* nglist,
                  u32* wlist, u32* nwlist, int* tri, unsigned short* label, unsigned short* code, double* xy,
                  u32* err, cudaStream_t st);

// coordinates of the lattice vertices
void launch_lattice_xy(const GridP& g, double* xy, cudaStream_t st);

}  // namespace sbmt
