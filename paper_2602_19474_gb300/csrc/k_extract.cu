// k_extract.cu -- K1: boundary extraction and compaction.
//
// The boundary is the set of unit pixel edges whose two pixels carry
// different labels (outside the image the label is OUTSIDE), the polygonal
// network taken as the "prescribed prior" of Sec. 3.1.  A pixel corner is a
// PSLG vertex unless none or exactly two collinear boundary edges meet there;
// a segment is a maximal straight run between two vertices (Sec. 3.2 takes
// segments of the 4-connected pixel contour).
//
// K1a marks vertex corners with warp ballots into two bit-planes, one packed
// along corner rows and one along corner columns (transposed through shared
// memory), so that K1b finds the end of every run with find-first-set over
// 32-bit words instead of walking pixel by pixel.
#include "sbmt_launch.h"
#include "sbmt_walk.cuh"

namespace sbmt {

namespace {

enum { BE_E = 1, BE_N = 2, BE_W = 4, BE_S = 8 };

template <typename T>
SBMT_DEV int corner_mask(const unsigned char* img, i64 pitch, int W, int H, int cx, int cy) {
  int a = pix<T>(img, pitch, W, H, cx - 1, cy - 1);
  int b = pix<T>(img, pitch, W, H, cx, cy - 1);
  int c = pix<T>(img, pitch, W, H, cx - 1, cy);
  int d = pix<T>(img, pitch, W, H, cx, cy);
  // E: edge to (cx+1, cy) between pixels (cx, cy-1) and (cx, cy); W: between
  // (cx-1, cy-1) and (cx-1, cy); N: edge to (cx, cy+1) between (cx-1, cy)
  // and (cx, cy); S: between (cx-1, cy-1) and (cx, cy-1)
  return (b != d ? BE_E : 0) | (a != c ? BE_W : 0) | (c != d ? BE_N : 0) | (a != b ? BE_S : 0);
}
SBMT_DEV bool vertex_mask(int m) { return m != 0 && m != (BE_E | BE_W) && m != (BE_N | BE_S); }

// 8 consecutive pixels of row y starting at column x0 (x0 a multiple of 8),
// OUTSIDE beyond the image; one vector load when the row is in range and
// aligned
template <typename T>
SBMT_DEV void load8(const unsigned char* img, i64 pitch, int W, int H, int x0, int y, int* out) {
  if (y < 0 || y >= H) {
    for (int k = 0; k < 8; ++k) out[k] = OUTSIDE;
    return;
  }
  const unsigned char* row = img + (i64)y * pitch;
  const T* p = (const T*)row + x0;
  if (x0 + 8 <= W && (((uintptr_t)p) & (8 * sizeof(T) - 1)) == 0) {
    if (sizeof(T) == 2) {
      const uint4 v = *(const uint4*)p;
      const u32 w[4] = {v.x, v.y, v.z, v.w};
      for (int k = 0; k < 4; ++k) out[2 * k] = (int)(w[k] & 0xFFFFu), out[2 * k + 1] = (int)(w[k] >> 16);
    } else {
      const uint2 v = *(const uint2*)p;
      const u32 w[2] = {v.x, v.y};
      for (int k = 0; k < 2; ++k)
        for (int b = 0; b < 4; ++b) out[4 * k + b] = (int)((w[k] >> (8 * b)) & 0xFFu);
    }
    return;
  }
  for (int k = 0; k < 8; ++k) out[k] = (x0 + k < W) ? (int)p[k] : OUTSIDE;
}

// K1a: a block covers 32 corner rows x 256 corner columns; each thread takes
// 8 consecutive corners of 4 rows.  The block's pixels (33 rows, the 256
// columns and a 16-byte halo chunk to their left) are first staged in shared
// memory with asynchronous 16-byte copies, every copy of the tile in flight
// at once; chunks that leave the image or are not 16-byte aligned are read
// pixel by pixel.  Vertex flags go to shared memory as one byte per (row, 8
// corners), then out as row words and transposed column words.
constexpr int CB_ROWS = 33;  // pixel rows r0 - 1 .. r0 + 31

template <typename T>
struct CornerTile {
  static constexpr int CHUNK = 16 / (int)sizeof(T);  // pixels per 16-byte chunk
  static constexpr int COLS = 256 + CHUNK;           // columns x0 - CHUNK .. x0 + 255
  static constexpr int NCH = COLS / CHUNK;           // chunks per row
  __align__(16) T px[CB_ROWS][COLS];
};

SBMT_DEV void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
SBMT_DEV void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
SBMT_DEV void corner_bits_tile(const unsigned char* img, i64 pitch, int W, int H, u32* vrow, int wpr, u32* vcol,
                               int wpc, unsigned long long* nvtx, int bx, int by, unsigned char (*fl)[33],
                               unsigned int& cnt, CornerTile<T>& tile) {
  using TT = CornerTile<T>;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int xb = bx * 256, r0 = by * 32;
  const int xs = xb - TT::CHUNK;  // first staged column
  if (threadIdx.x == 0) cnt = 0;
  // stage rows r0 - 1 .. r0 + 31, columns xs .. xb + 255 (in-image pixels only)
  for (int q = threadIdx.x; q < CB_ROWS * TT::NCH; q += blockDim.x) {
    const int tr = q / TT::NCH, ch = q - tr * TT::NCH;
    const int y = r0 - 1 + tr, x = xs + ch * TT::CHUNK;
    if (y < 0 || y >= H) continue;
    const T* src = (const T*)(img + (i64)y * pitch) + x;
    T* dst = &tile.px[tr][ch * TT::CHUNK];
    if (x >= 0 && x + TT::CHUNK <= W && (((uintptr_t)src) & 15) == 0) {
      cp_async16(dst, src);
    } else {
      for (int k = 0; k < TT::CHUNK; ++k)
        if (x + k >= 0 && x + k < W) dst[k] = src[k];
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // pixel (x, y) of the tile, OUTSIDE beyond the image
  auto P = [&](int x, int y) -> int {
    return (x < 0 || x >= W || y < 0 || y >= H) ? OUTSIDE : (int)tile.px[y - r0 + 1][x - xs];
  };
  u32 mycnt = 0;
  const int x0 = xb + lane * 8;  // first corner column of this thread
  // a tile whose pixels (rows r0 - 1 .. r0 + 31, columns xb - 1 .. xb + 255)
  // all lie in the image reads them without bounds checks
  const bool interior = xb >= 1 && xb + 255 < W && r0 >= 1 && r0 + 31 < H;
  for (int rr = 0; rr < 4; ++rr) {
    const int r = w * 4 + rr, cy = r0 + r;
    int lo[9], hi[9];  // pixel rows cy-1 and cy, columns x0-1 .. x0+7
    if (interior) {
#pragma unroll
      for (int k = 0; k < 9; ++k) lo[k] = tile.px[r][x0 - 1 + k - xs], hi[k] = tile.px[r + 1][x0 - 1 + k - xs];
    } else {
#pragma unroll
      for (int k = 0; k < 9; ++k) lo[k] = P(x0 - 1 + k, cy - 1), hi[k] = P(x0 - 1 + k, cy);
    }
    // the eight corners' masks as bit vectors: corner (x0 + k, cy) has pixels
    // a = lo[k], b = lo[k+1], c = hi[k], d = hi[k+1]; its E edge is b != d,
    // W a != c, N c != d, S a != b
    u32 vv = 0, nn = 0, ss = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) vv |= (lo[k] != hi[k] ? 1u : 0u) << k;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      nn |= (hi[k] != hi[k + 1] ? 1u : 0u) << k;
      ss |= (lo[k] != lo[k + 1] ? 1u : 0u) << k;
    }
    const u32 ee = vv >> 1, ww = vv & 0xFFu;
    // a vertex: some boundary edge, and not exactly two collinear ones
    u32 bits = (ee | ww | nn | ss) & ~(ee & ww & ~nn & ~ss) & ~(nn & ss & ~ee & ~ww) & 0xFFu;
    if (!interior) {
      const int room = W - x0 + 1;  // corners x0 + k <= W
      bits &= cy <= H ? (room >= 8 ? 0xFFu : room > 0 ? (1u << room) - 1u : 0u) : 0u;
    }
    fl[r][lane] = (unsigned char)bits;
    mycnt += __popc(bits);
  }
  atomicAdd(&cnt, mycnt);
  __syncthreads();
  // row words: row r, word k of the block = groups 4k .. 4k+3
  {
    const int r = threadIdx.x >> 3, k = threadIdx.x & 7, cy = r0 + r;
    const u32 word = (u32)fl[r][4 * k] | ((u32)fl[r][4 * k + 1] << 8) | ((u32)fl[r][4 * k + 2] << 16) |
                     ((u32)fl[r][4 * k + 3] << 24);
    const int wx = bx * 8 + k;
    if (cy <= H && wx < wpr) vrow[(i64)cy * wpr + wx] = word;
  }
  // column words: corner column c of the block, rows r0 .. r0+31
  {
    const int c = threadIdx.x, cx = bx * 256 + c;
    u32 word = 0;
    for (int r = 0; r < 32; ++r) word |= (u32)((fl[r][c >> 3] >> (c & 7)) & 1u) << r;
    if (cx <= W) vcol[(i64)cx * wpc + by] = word;
  }
  if (threadIdx.x == 0 && cnt) atomicAdd(nvtx, (unsigned long long)cnt);
}

template <typename T>
__global__ void __launch_bounds__(256) k_corner_bits(const unsigned char* img, i64 pitch, int W, int H, u32* vrow,
                                                     int wpr, u32* vcol, int wpc, unsigned long long* nvtx) {
  __shared__ unsigned char fl[32][33];
  __shared__ unsigned int cnt;
  __shared__ CornerTile<T> tile;
  corner_bits_tile<T>(img, pitch, W, H, vrow, wpr, vcol, wpc, nvtx, blockIdx.x, blockIdx.y, fl, cnt, tile);
}

// batched: job k's tiles are its blocks, row-major over (256-column, 32-row) tiles
template <bool ONE>
__global__ void __launch_bounds__(256) k_corner_bits_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                       const u32* __restrict__ bpre, int njobs) {
  __shared__ unsigned char fl[32][33];
  __shared__ unsigned int cnt;
  __shared__ union {
    CornerTile<unsigned char> t8;
    CornerTile<unsigned short> t16;
  } tile;
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const int W = J.g.W, H = J.g.H, gx = (W + 1 + 255) / 256;
  const int bx = (int)(lb % (u32)gx), by = (int)(lb / (u32)gx);
  unsigned long long* nvtx = (unsigned long long*)J.zero;
  if (J.dtype == 1)
    corner_bits_tile<unsigned char>(J.img, J.pitch, W, H, J.vrow, J.wpr, J.vcol, J.wpc, nvtx, bx, by, fl, cnt, tile.t8);
  else
    corner_bits_tile<unsigned short>(J.img, J.pitch, W, H, J.vrow, J.wpr, J.vcol, J.wpc, nvtx, bx, by, fl, cnt,
                                     tile.t16);
}

// first set bit at index >= from in a packed bit-plane line of nwords words;
// -1 if none
SBMT_DEV int next_set(const u32* line, int nwords, int from) {
  int w = from >> 5;
  if (w >= nwords) return -1;
  u32 word = line[w] & (0xffffffffu << (from & 31));
  while (true) {
    if (word) return (w << 5) + __ffs(word) - 1;
    if (++w >= nwords) return -1;
    word = line[w];
  }
}

SBMT_DEV u32 lab16(int l) { return l == OUTSIDE ? 0xFFFFu : (u32)l; }

// K1b: one thread per 32-corner word of a row bit-plane; every vertex starts
// its +x and +y runs.  Output slots are taken one atomic per warp.
template <typename T>
SBMT_DEV void segments_word(const unsigned char* img, i64 pitch, int W, int H, const u32* vrow, int wpr,
                            const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, i64 t) {
  const bool in = t < (i64)(H + 1) * wpr;
  const int cy = in ? (int)(t / wpr) : 0, w = in ? (int)(t % wpr) : 0;
  const u32 bits = in ? vrow[t] : 0u;
  u32 cnt = 0;
  for (u32 b = bits; b; b &= b - 1) {
    const int cx = (w << 5) + __ffs(b) - 1;
    const int m = corner_mask<T>(img, pitch, W, H, cx, cy);
    cnt += ((m & BE_E) != 0) + ((m & BE_N) != 0);
  }
  // warp-wide exclusive scan of the counts and one atomic for the warp
  const int lane = threadIdx.x & 31;
  u32 x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  const u32 wtot = __shfl_sync(0xffffffffu, x, 31);
  u32 wbase = 0;
  if (lane == 31 && wtot) wbase = atomicAdd(nseg, wtot);
  wbase = __shfl_sync(0xffffffffu, wbase, 31);
  u32 slot = wbase + x - cnt;
  for (u32 b = cnt ? bits : 0u; b; b &= b - 1) {
    const int cx = (w << 5) + __ffs(b) - 1;
    const int m = corner_mask<T>(img, pitch, W, H, cx, cy);
    if (m & BE_E) {
      const int end = next_set(vrow + (i64)cy * wpr, wpr, cx + 1);
      if (end < 0) {
        atomicOr(err, ERR_TRAVERSAL);
      } else if (slot < cap) {
        const int l0 = pix<T>(img, pitch, W, H, cx, cy - 1), l1 = pix<T>(img, pitch, W, H, cx, cy);
        // going +x the left side is above: forward when the upper label is lower
        const u32 rev = l1 < l0 ? 0u : 1u;
        const Seg sg{cx, cy, (u32)(end - cx) | (rev << 31), lab16(l0) | (lab16(l1) << 16)};
        segs[slot] = sg;
      }
      ++slot;
    }
    if (m & BE_N) {
      const int end = next_set(vcol + (i64)cx * wpc, wpc, cy + 1);
      if (end < 0) {
        atomicOr(err, ERR_TRAVERSAL);
      } else if (slot < cap) {
        const int l0 = pix<T>(img, pitch, W, H, cx - 1, cy), l1 = pix<T>(img, pitch, W, H, cx, cy);
        // going +y the left side is -x: forward when the left label is lower
        const u32 rev = l0 < l1 ? 0u : 1u;
        const Seg sg{cx, cy, (u32)(end - cy) | (1u << 30) | (rev << 31), lab16(l0) | (lab16(l1) << 16)};
        segs[slot] = sg;
      }
      ++slot;
    }
  }
}

template <typename T>
__global__ void k_segments(const unsigned char* img, i64 pitch, int W, int H, const u32* vrow, int wpr,
                           const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err) {
  segments_word<T>(img, pitch, W, H, vrow, wpr, vcol, wpc, segs, cap, nseg, err,
                   (i64)blockIdx.x * blockDim.x + threadIdx.x);
}

template <bool ONE>
__global__ void __launch_bounds__(256) k_segments_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                       const u32* __restrict__ bpre, int njobs) {
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const i64 t = (i64)lb * blockDim.x + threadIdx.x;
  u32* cnt = J.zero;
  const GridP& g = J.g;
  if (J.dtype == 1)
    segments_word<unsigned char>(J.img, J.pitch, g.W, g.H, J.vrow, J.wpr, J.vcol, J.wpc, J.segs, J.seg_cap,
                                 cnt + JC_NSEG, cnt + JC_ERR, t);
  else
    segments_word<unsigned short>(J.img, J.pitch, g.W, g.H, J.vrow, J.wpr, J.vcol, J.wpc, J.segs, J.seg_cap,
                                  cnt + JC_NSEG, cnt + JC_ERR, t);
}

// the cells each segment visits (its pairs), densely over the segments the
// device counted: a job's blocks stride over its segments
template <bool ONE>
__global__ void __launch_bounds__(256) k_seg_count_b(const __grid_constant__ Job one, const Job* __restrict__ jobs,
                                                     const u32* __restrict__ bpre, int njobs) {
  SBMT_BLOCK_JOB(ONE, one, jobs, bpre, njobs)
  const u32 nb = ONE ? gridDim.x : bpre[jk + 1] - bpre[jk];
  const u32 n = min(*jc(J, JC_NSEG), J.seg_cap);
  const GridP& g = J.g;
  for (u32 s = lb * blockDim.x + threadIdx.x; s < n; s += nb * blockDim.x) J.npairs[s] = seg_pairs(g, J.segs[s]);
}

}  // namespace

int launch_corner_bits(const unsigned char* img, i64 pitch, int dtype, int W, int H, u32* vrow, int wpr,
                        u32* vcol, int wpc, unsigned long long* nvtx, cudaStream_t st) {
  dim3 blk(256), grd((W + 1 + 255) / 256, (H + 1 + 31) / 32);
  if (dtype == 1)
    k_corner_bits<unsigned char><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, nvtx);
  else
    k_corner_bits<unsigned short><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, nvtx);
  return 1;
}

int launch_segments(const unsigned char* img, i64 pitch, int dtype, int W, int H, const u32* vrow, int wpr,
                     const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, cudaStream_t st) {
  const i64 n = (i64)(H + 1) * wpr;
  const int blk = 256;
  const unsigned grd = (unsigned)((n + blk - 1) / blk);
  if (dtype == 1)
    k_segments<unsigned char><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, segs, cap, nseg, err);
  else
    k_segments<unsigned short><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, segs, cap, nseg, err);
  return 1;
}

int launch_corner_bits_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_corner_bits_b<true><<<nblocks, 256, 0, st>>>(*one, jobs, bpre, njobs);
  else k_corner_bits_b<false><<<nblocks, 256, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

int launch_segments_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_segments_b<true><<<nblocks, 256, 0, st>>>(*one, jobs, bpre, njobs);
  else k_segments_b<false><<<nblocks, 256, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

int launch_seg_count_b(const Job* one, const Job* jobs, const u32* bpre, int njobs, u32 nblocks, cudaStream_t st) {
  if (nblocks == 0) return 0;
  if (one) k_seg_count_b<true><<<nblocks, 256, 0, st>>>(*one, jobs, bpre, njobs);
  else k_seg_count_b<false><<<nblocks, 256, 0, st>>>(Job{}, jobs, bpre, njobs);
  return 1;
}

}  // namespace sbmt
