// k_scan.cu -- exclusive prefix sums of u32 counts (offsets of the output
// patches, of the (cell, segment) pairs and crossing events per segment, of
// the bucket ranges).  The meshing path scans every array of a batch in one
// single-pass launch (k_mscan); the preprocessing and heat paths use the
// three-pass scan (one block for small inputs; else tile sums, a scan of the
// tile sums, and the tiles with their offsets).
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

// ---------------------------------------------------------------------------
// Batched single-pass scan: every tile of every scan job in one launch.
// Tiles take their order from a ticket counter (so a tile's predecessors
// were started before it), publish their sum, and look back over their
// predecessors' published sums (decoupled look-back): a tile's flag word is
// status << 32 | value, status 1 = the tile's own sum, 2 = the inclusive
// prefix through the tile, 3 = an error upstream.  Every wait is bounded by
// the global timer; a wait that runs out records ERR_TIMEOUT in the job's
// error word and publishes status 3, so that the tiles after it stop at once.
// ---------------------------------------------------------------------------
constexpr unsigned long long FLAG_AGG = 1ull << 32, FLAG_INC = 2ull << 32, FLAG_ERR = 3ull << 32;
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;  // one second

SBMT_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256) k_mscan(const ScanJob* __restrict__ sj, const u32* __restrict__ tpre,
                                               int nsj, unsigned long long* flags, u32* ticket, u32 stall_tile) {
  __shared__ u32 s_sh[8];
  __shared__ u32 s_tile, s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const u32 tile = s_tile;
  const int k = job_of(tpre, nsj, tile);
  const ScanJob J = sj[k];
  const u32 t = tile - tpre[k];
  const u64 base = (u64)t * MSCAN_TILE;
  const u32 n = J.n_dev ? min(*J.n_dev, J.n) : J.n;
  if (base > n) {
    // past the end of a scan whose length is known on the device only: no
    // output, and nothing after it waits for a value from here
    if (threadIdx.x == 0) atomicExch(flags + tile, FLAG_INC);
    return;
  }
  u32 v[8], s = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const u64 i = base + (u64)threadIdx.x * 8 + u;
    v[u] = i < n ? J.in[i] : 0u;
    s += v[u];
  }
  u32 tot;
  const u32 ex = block_exscan256(s, &tot, s_sh);
  if (threadIdx.x == 0) {
    const bool stall = tile == stall_tile;
    volatile unsigned long long* vf = flags;
    u32 prefix = 0;
    bool bad = false;
    if (t > 0) {
      if (!stall) atomicExch(flags + tile, FLAG_AGG | tot);
      unsigned long long t0 = 0;
      for (u32 p = tile - 1;;) {
        const unsigned long long f = vf[p];
        const unsigned long long st = f & (3ull << 32);
        if (st == 0) {
          const unsigned long long now = global_ns();
          if (t0 == 0) t0 = now;
          if (now - t0 > WAIT_LIMIT_NS) {
            bad = true;
            atomicOr(J.err, ERR_TIMEOUT);
            break;
          }
          __nanosleep(128);
          continue;
        }
        if (st == FLAG_ERR) {
          bad = true;
          break;
        }
        prefix += (u32)f;
        if (st == FLAG_INC) break;
        --p;  // an aggregate: keep looking back (tile 0 of a job always publishes its prefix)
        t0 = 0;
      }
    }
    if (!stall) atomicExch(flags + tile, bad ? FLAG_ERR : (FLAG_INC | (u32)(prefix + tot)));
    s_prefix = prefix;
  }
  __syncthreads();
  u32 run = s_prefix + ex;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const u64 i = base + (u64)threadIdx.x * 8 + u;
    if (i <= n) {
      J.out[i] = run;
      if (J.out2) J.out2[i] = run;
      if (J.big && i < n && v[u] > J.big_thr) J.big[atomicAdd(J.nbig, 1u)] = make_uint2((u32)J.img, (u32)i);
    }
    run += v[u];
  }
}

}  // namespace

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

int launch_mscan(const ScanJob* sj, const u32* tpre, int nsj, u32 ntiles, unsigned long long* flags, u32* ticket,
                 u32 stall_tile, cudaStream_t st) {
  if (ntiles == 0) return 0;
  k_mscan<<<ntiles, 256, 0, st>>>(sj, tpre, nsj, flags, ticket, stall_tile);
  return 1;
}

}  // namespace sbmt
