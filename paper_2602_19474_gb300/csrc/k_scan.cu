// k_scan.cu -- exclusive prefix sums of u32 counts (offsets of the output
// patches, of the (cell, segment) pairs and crossing events per segment, of
// the bucket ranges).  Small inputs scan in one block; large ones in three
// passes: tile sums, a scan of the tile sums, and the tiles with their
// offsets.
#include "sbmt_cell.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

constexpr int TILE = 2048;  // elements per tile (256 threads x 8)

// one block of 1024 threads: exclusive scan of n strided values, total at out[n]
__global__ void __launch_bounds__(1024) k_scan_small(const u32* in, int stride, u32* out, u32 n) {
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

__global__ void __launch_bounds__(256) k_tile_sums(const u32* in, int stride, u32 n, u32* part) {
  __shared__ u32 s_sh[8];
  const u64 base = (u64)blockIdx.x * TILE;
  u32 s = 0;
  for (int u = 0; u < 8; ++u) {
    const u64 i = base + (u64)threadIdx.x * 8 + u;
    if (i < n) s += in[i * stride];
  }
  u32 tot;
  block_exscan256(s, &tot, s_sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_tile_scan(const u32* in, int stride, u32 n, const u32* part_scan,
                                                   u32* out) {
  __shared__ u32 s_sh[8];
  const u64 base = (u64)blockIdx.x * TILE;
  u32 v[8], s = 0;
  for (int u = 0; u < 8; ++u) {
    const u64 i = base + (u64)threadIdx.x * 8 + u;
    v[u] = i < n ? in[i * stride] : 0u;
    s += v[u];
  }
  u32 tot;
  u32 run = block_exscan256(s, &tot, s_sh) + part_scan[blockIdx.x];
  for (int u = 0; u < 8; ++u) {
    const u64 i = base + (u64)threadIdx.x * 8 + u;
    if (i < n) out[i] = run;
    run += v[u];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 255) out[n] = run;
}

// one block of 1024 threads per array: exclusive scans of up to two arrays
// of at most SCAN_ONE values each (total at out[n]), the result written to
// out and, when given, to out2 as well (bucket cursors)
struct ScanJob {
  const u32* in;
  u32* out;
  u32* out2;
  u32 n;
};
__global__ void __launch_bounds__(1024) k_scan_jobs(ScanJob a, ScanJob b) {
  __shared__ u32 sh[1024];
  const ScanJob j = blockIdx.x == 0 ? a : b;
  const u32 t = threadIdx.x, n = j.n;
  const u32 chunk = (n + 1023) / 1024;
  const u32 lo = min(n, t * chunk), hi = min(n, lo + chunk);
  u32 s = 0;
  for (u32 i = lo; i < hi; ++i) s += j.in[i];
  sh[t] = s;
  __syncthreads();
  for (u32 o = 1; o < 1024; o <<= 1) {
    const u32 v = t >= o ? sh[t - o] : 0u;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  u32 run = sh[t] - s;
  for (u32 i = lo; i < hi; ++i) {
    const u32 v = j.in[i];
    j.out[i] = run;
    if (j.out2) j.out2[i] = run;
    run += v;
  }
  if (t == 1023) {
    j.out[n] = sh[1023];
    if (j.out2) j.out2[n] = sh[1023];
  }
}

}  // namespace

int launch_scan_pair(const u32* in_a, u32* out_a, u32* out2_a, u32 n_a, const u32* in_b, u32* out_b, u32* out2_b,
                     u32 n_b, cudaStream_t st) {
  k_scan_jobs<<<in_b ? 2 : 1, 1024, 0, st>>>(ScanJob{in_a, out_a, out2_a, n_a}, ScanJob{in_b, out_b, out2_b, n_b});
  return 1;
}

size_t scan_scratch_words(u32 n) { return n <= 16384 ? 0 : (size_t)((n + TILE - 1) / TILE) + 1; }

int launch_scan(const u32* in, int stride, u32* out, u32 n, u32* scratch, cudaStream_t st) {
  if (n <= 16384 || scratch == nullptr) {
    k_scan_small<<<1, 1024, 0, st>>>(in, stride, out, n);
    return 1;
  }
  const u32 tiles = (n + TILE - 1) / TILE;
  k_tile_sums<<<tiles, 256, 0, st>>>(in, stride, n, scratch);
  // scan of the tile sums in place (tiles <= 65536 for any n < 2^27)
  k_scan_small<<<1, 1024, 0, st>>>(scratch, 1, scratch, tiles);
  k_tile_scan<<<tiles, 256, 0, st>>>(in, stride, n, scratch, out);
  return 3;
}

}  // namespace sbmt
