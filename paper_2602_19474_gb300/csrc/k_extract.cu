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

template <typename T>
__global__ void __launch_bounds__(1024) k_corner_bits(const unsigned char* img, i64 pitch, int W, int H, u32* vrow,
                                                      int wpr, u32* vcol, int wpc, unsigned long long* nvtx) {
  __shared__ unsigned char fl[32][33];
  __shared__ unsigned int cnt;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int cx = blockIdx.x * 32 + tx, cy = blockIdx.y * 32 + ty;
  if (tx == 0 && ty == 0) cnt = 0;
  bool v = false;
  if (cx <= W && cy <= H) v = vertex_mask(corner_mask<T>(img, pitch, W, H, cx, cy));
  const u32 row_bits = __ballot_sync(0xffffffffu, v);
  fl[ty][tx] = v ? 1 : 0;
  __syncthreads();
  if (tx == 0 && cy <= H) {
    vrow[(i64)cy * wpr + blockIdx.x] = row_bits;
    atomicAdd(&cnt, (unsigned)__popc(row_bits));
  }
  // transposed read: this warp gathers corner column blockIdx.x * 32 + ty
  const bool v2 = fl[tx][ty] != 0;
  const u32 col_bits = __ballot_sync(0xffffffffu, v2);
  const int ccol = blockIdx.x * 32 + ty;
  if (tx == 0 && ccol <= W) vcol[(i64)ccol * wpc + blockIdx.y] = col_bits;
  __syncthreads();
  if (tx == 0 && ty == 0 && cnt) atomicAdd(nvtx, (unsigned long long)cnt);
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

template <typename T>
__global__ void k_segments(const unsigned char* img, i64 pitch, int W, int H, const u32* vrow, int wpr,
                           const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err) {
  const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (i64)(H + 1) * wpr) return;
  const int cy = (int)(t / wpr), w = (int)(t % wpr);
  const u32 bits = vrow[t];
  if (!bits) return;
  int cnt = 0;
  for (u32 b = bits; b; b &= b - 1) {
    const int cx = (w << 5) + __ffs(b) - 1;
    const int m = corner_mask<T>(img, pitch, W, H, cx, cy);
    cnt += ((m & BE_E) != 0) + ((m & BE_N) != 0);
  }
  if (!cnt) return;
  u32 slot = atomicAdd(nseg, (u32)cnt);
  for (u32 b = bits; b; b &= b - 1) {
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
        segs[slot] = Seg{cx, cy, (u32)(end - cx) | (rev << 31), lab16(l0) | (lab16(l1) << 16)};
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
        segs[slot] = Seg{cx, cy, (u32)(end - cy) | (1u << 30) | (rev << 31), lab16(l0) | (lab16(l1) << 16)};
      }
      ++slot;
    }
  }
}

}  // namespace

void launch_corner_bits(const unsigned char* img, i64 pitch, int dtype, int W, int H, u32* vrow, int wpr,
                        u32* vcol, int wpc, unsigned long long* nvtx, cudaStream_t st) {
  dim3 blk(32, 32), grd((W + 1 + 31) / 32, (H + 1 + 31) / 32);
  if (dtype == 1)
    k_corner_bits<unsigned char><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, nvtx);
  else
    k_corner_bits<unsigned short><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, nvtx);
}

void launch_segments(const unsigned char* img, i64 pitch, int dtype, int W, int H, const u32* vrow, int wpr,
                     const u32* vcol, int wpc, Seg* segs, u32 cap, u32* nseg, u32* err, cudaStream_t st) {
  const i64 n = (i64)(H + 1) * wpr;
  const int blk = 256;
  const unsigned grd = (unsigned)((n + blk - 1) / blk);
  if (dtype == 1)
    k_segments<unsigned char><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, segs, cap, nseg, err);
  else
    k_segments<unsigned short><<<grd, blk, 0, st>>>(img, pitch, W, H, vrow, wpr, vcol, wpc, segs, cap, nseg, err);
}

}  // namespace sbmt
