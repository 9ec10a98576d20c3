// k_heat.cu -- transient heat diffusion on a label region of a finished mesh
// (App. H): du/dt = alpha Lap u on the triangles of one label, u = 0 on the
// region's boundary, from a Gaussian pulse.
//
// Linear finite elements: the cotangent stiffness K (a triangle with angle
// theta_k at corner k couples the ends i, j of the opposite edge with
// -cot(theta_k) / 2 and adds cot(theta_k) / 2 to both diagonals), the lumped
// mass M (a third of each incident triangle's area), backward Euler in time:
// (M + alpha dt K) u_{n+1} = M u_n on the free vertices (those of the region
// not on a triangle of another label).  Each step is solved by conjugate
// gradients with the diagonal as preconditioner.  The operator is assembled
// once per call into sparse rows over the free vertices (from one record per
// region triangle), so that each product is a gather with no atomics.
// Double precision throughout.  The result does not depend on the order in
// which threads run: records are placed by a scan, each free vertex's mass
// and diagonal are gathered over its incident records in record order, the
// rows' entries are sorted by column, and every reduction is finished by
// the last block of its launch over the blocks' partial sums in block order.
#include <algorithm>
#include <vector>

#include "sbmt_dev.cuh"
#include "sbmt_launch.h"

namespace sbmt {

namespace {

constexpr int HB = 256;  // threads per block

// one region triangle: its corners and the weights cot(theta_k) / 2 of the
// edges opposite each corner
struct HeatTri {
  int v[3];
  int pad;
  double w[3];
  double third;  // a third of the triangle's area
};

__global__ void __launch_bounds__(HB) k_heat_flags(const int* tri, const unsigned short* label, u64 T, int L,
                                                   u32* flag) {
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x) {
    const u32 f = label[t] == (unsigned short)L ? 1u : 2u;
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicOr(flag + tri[3 * t + k], f);
  }
}

// free vertices (flag 1) as 0/1 for the scan that numbers them
__global__ void __launch_bounds__(HB) k_heat_free(u64 V, u32* flag) {
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x)
    flag[v] = flag[v] == 1u ? 1u : 0u;
}

// the free vertices in id order (fidx: exclusive scan of the 0/1 flags)
__global__ void __launch_bounds__(HB) k_heat_list(u64 V, const u32* free01, const u32* fidx, u32* list) {
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x)
    if (free01[v]) list[fidx[v]] = (u32)v;
}

// region triangles as 0/1 flags, for the scan that places their records
__global__ void __launch_bounds__(HB) k_heat_tflag(const unsigned short* label, u64 T, int L, u32* tf) {
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x)
    tf[t] = label[t] == (unsigned short)L ? 1u : 0u;
}

// the region's triangles: records (corners as free indices, -1 for
// boundary vertices) at their scan positions, in triangle order, and the
// number of records at each free vertex
__global__ void __launch_bounds__(HB) k_heat_setup(const double* xy, const int* tri, const unsigned short* label,
                                                   u64 T, int L, const u32* free01, const u32* fidx, const u32* tpos,
                                                   HeatTri* rec, u32* vcnt) {
  const double2* p = reinterpret_cast<const double2*>(xy);
  for (u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (u64)gridDim.x * blockDim.x) {
    if (label[t] != (unsigned short)L) continue;
    HeatTri h;
    double2 c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int v = tri[3 * t + k];
      c[k] = p[v];
      h.v[k] = free01[v] ? (int)fidx[v] : -1;
    }
    h.pad = 0;
    const double cross = fabs((c[1].x - c[0].x) * (c[2].y - c[0].y) - (c[1].y - c[0].y) * (c[2].x - c[0].x));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double2 a = c[k], b = c[(k + 1) % 3], d = c[(k + 2) % 3];
      const double dot = (b.x - a.x) * (d.x - a.x) + (b.y - a.y) * (d.y - a.y);
      h.w[k] = 0.5 * dot / cross;  // cot(theta_k) / 2 = (u . v) / (2 |u x v|)
    }
    h.third = cross / 6.0;  // a third of the area |u x v| / 2
    rec[tpos[t]] = h;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (h.v[k] >= 0) atomicAdd(vcnt + h.v[k], 1u);
  }
}

// each free vertex's incident records (record index * 4 + corner), placed
// at cursors from the scan of the counts; sorted afterwards
__global__ void __launch_bounds__(HB) k_heat_inc(const HeatTri* rec, u32 nr, u32* cur, u32* inc) {
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < nr; t += gridDim.x * blockDim.x) {
    const HeatTri h = rec[t];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (h.v[k] >= 0) inc[atomicAdd(cur + h.v[k], 1u)] = 4 * t + (u32)k;
  }
}

// per free vertex, in record order: the lumped mass (a third of each
// incident triangle's area |u x v| / 2) and the stiffness diagonal (the
// weights of the two edges at the vertex)
__global__ void __launch_bounds__(HB) k_heat_gather(const HeatTri* rec, u32 n, const u32* vptr, u32* inc,
                                                    double* mass, double* kdiag) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const u32 e0 = vptr[i], e1 = vptr[i + 1];
    for (u32 a = e0 + 1; a < e1; ++a)  // insertion sort: a vertex has few records
      for (u32 b = a; b > e0 && inc[b] < inc[b - 1]; --b) {
        const u32 t = inc[b];
        inc[b] = inc[b - 1], inc[b - 1] = t;
      }
    double m = 0.0, d = 0.0;
    for (u32 e = e0; e < e1; ++e) {
      const HeatTri h = rec[inc[e] >> 2];
      const int c = (int)(inc[e] & 3u);
      m += h.third;
      // the edges at corner c are those opposite corners c + 1 and c + 2
      d += h.w[(c + 1) % 3];
      d += h.w[(c + 2) % 3];
    }
    mass[i] = m;
    kdiag[i] = d;
  }
}

// A reduction slot: the blocks' partial sums and a counter of finished
// blocks (zeroed once; the last block resets it).
struct Red {
  double* part;
  u32* done;
};

// block sum of v into *out: each block writes its partial sum, and the last
// block to finish adds the partials in a fixed order (thread t sums partials
// t, t + HB, ..., then a fixed tree over the threads), so the sum is the same
// on every run, whatever order the blocks ran in
__device__ __forceinline__ double block_sum_fixed(double v, double* s) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  double b = 0.0;
  if (threadIdx.x < 32) {
    b = threadIdx.x < blockDim.x / 32 ? s[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
  }
  __syncthreads();
  return b;  // valid in thread 0
}

__device__ __forceinline__ void block_add(double v, double* out, Red red) {
  __shared__ double s[HB / 32];
  __shared__ bool last;
  const double b = block_sum_fixed(v, s);
  if (threadIdx.x == 0) {
    red.part[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(red.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double t = 0.0;
    for (u32 k = threadIdx.x; k < gridDim.x; k += blockDim.x) t += __ldcg(red.part + k);
    t = block_sum_fixed(t, s);
    if (threadIdx.x == 0) {
      *out = t;
      *red.done = 0;
    }
  }
  __syncthreads();
}

// the free vertices: the pulse, the operator's inverse diagonal
__global__ void __launch_bounds__(HB) k_heat_init(const double* xy, u32 n, const u32* list, const double* mass,
                                                  const double* kdiag, double tau, double x0, double y0,
                                                  double s2, double amp, double* x, double* dg, double* dinv) {
  const double2* p = reinterpret_cast<const double2*>(xy);
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 c = p[list[i]];
    const double dx = c.x - x0, dy = c.y - y0;
    x[i] = amp * exp(-(dx * dx + dy * dy) / (2.0 * s2));
    dg[i] = mass[i] + tau * kdiag[i];
    dinv[i] = 1.0 / dg[i];
  }
}

// q = M x
__global__ void __launch_bounds__(HB) k_heat_mass(u32 n, const double* mass, const double* x, double* q) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = mass[i] * x[i];
}

// the operator as sparse rows over the free vertices: two entries per
// region-triangle edge with both ends free, -tau cot/2 each (an edge shared
// by two region triangles gives two entries for the same neighbour, merged
// afterwards); the diagonal is kept apart
__global__ void __launch_bounds__(HB) k_heat_rowcount(const HeatTri* rec, u32 n, u32* cnt) {
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const HeatTri h = rec[t];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i = h.v[(k + 1) % 3], j = h.v[(k + 2) % 3];
      if (i >= 0 && j >= 0) atomicAdd(cnt + i, 1u), atomicAdd(cnt + j, 1u);
    }
  }
}
__global__ void __launch_bounds__(HB) k_heat_fill(const HeatTri* rec, u32 n, double tau, u32* cur, u32* col,
                                                  double* val) {
  for (u32 t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const HeatTri h = rec[t];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i = h.v[(k + 1) % 3], j = h.v[(k + 2) % 3];
      if (i < 0 || j < 0) continue;
      const double w = -tau * h.w[k];
      const u32 a = atomicAdd(cur + i, 1u), b = atomicAdd(cur + j, 1u);
      col[a] = (u32)j, val[a] = w;
      col[b] = (u32)i, val[b] = w;
    }
  }
}

// each row's entries of one column summed, in place at the row's start;
// mcnt: the merged counts
__global__ void __launch_bounds__(HB) k_heat_merge(u32 n, const u32* rowptr, u32* col, double* val, u32* mcnt) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const u32 e0 = rowptr[i], e1 = rowptr[i + 1];
    u32 m = 0;
    for (u32 e = e0; e < e1; ++e) {
      const u32 c = col[e];
      const double v = val[e];
      u32 k = 0;
      while (k < m && col[e0 + k] != c) ++k;
      if (k < m) {
        val[e0 + k] += v;
      } else {
        col[e0 + m] = c, val[e0 + m] = v;
        ++m;
      }
    }
    // the row's entries by column, so that each product sums them in one order
    for (u32 a = 1; a < m; ++a)
      for (u32 b = a; b > 0 && col[e0 + b] < col[e0 + b - 1]; --b) {
        const u32 tc = col[e0 + b];
        col[e0 + b] = col[e0 + b - 1], col[e0 + b - 1] = tc;
        const double tv = val[e0 + b];
        val[e0 + b] = val[e0 + b - 1], val[e0 + b - 1] = tv;
      }
    mcnt[i] = m;
  }
}

// q = (M + tau K) x over the free rows (dg: the diagonal M + tau diag K),
// and x . q added into *xq
__global__ void __launch_bounds__(HB) k_heat_apply(u32 n, const u32* rowptr, const u32* mcnt, const u32* col,
                                                   const double* val, const double* dg, const double* x, double* q,
                                                   double* xq, Red red) {
  double acc = 0.0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double xi = x[i];
    double y = dg[i] * xi;
    const u32 e0 = rowptr[i], e1 = e0 + mcnt[i];
    for (u32 e = e0; e < e1; ++e) y += val[e] * x[col[e]];
    q[i] = y;
    acc += xi * y;
  }
  block_add(acc, xq, red);
}

// u over the mesh: 0, then the free values at their vertices
__global__ void __launch_bounds__(HB) k_heat_zero(u64 V, double* u) {
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x) u[v] = 0.0;
}
__global__ void __launch_bounds__(HB) k_heat_put(u32 n, const u32* list, const double* x, double* u) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) u[list[i]] = x[i];
}

// CG scalars per iteration it: s[4 it + 0] = p.q, s[4 it + 1] = r.z,
// s[4 it + 2] = r.r (all zeroed before the solve)
__global__ void __launch_bounds__(HB) k_heat_dot(u64 V, const double* a, const double* b, double* out, Red red) {
  double acc = 0.0;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x)
    acc += a[v] * b[v];
  block_add(acc, out, red);
}

// r = b - q (q = A x), z = D^-1 r, p = z; r.z into rz, r.r into rr
__global__ void __launch_bounds__(HB) k_heat_start(u64 V, const double* b, const double* q, const double* dinv,
                                                   double* r, double* z, double* p, double* rz, double* rr, Red r1,
                                                   Red r2) {
  double a1 = 0.0, a2 = 0.0;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x) {
    const double rv = dinv[v] != 0.0 ? b[v] - q[v] : 0.0, zv = rv * dinv[v];
    r[v] = rv, z[v] = zv, p[v] = zv;
    a1 += rv * zv, a2 += rv * rv;
  }
  block_add(a1, rz, r1);
  block_add(a2, rr, r2);
}

// x += alpha p, r -= alpha q, z = D^-1 r, with alpha = rz / pq; the new
// r.z and r.r
__global__ void __launch_bounds__(HB) k_heat_update(u64 V, const double* sc, double* x, double* r, double* z,
                                                    const double* p, const double* q, const double* dinv,
                                                    double* rz_next, double* rr_next, Red r1, Red r2) {
  const double al = sc[0] != 0.0 ? sc[1] / sc[0] : 0.0;  // sc: {p.q, r.z} of this iteration
  double a1 = 0.0, a2 = 0.0;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x) {
    x[v] += al * p[v];
    const double rv = r[v] - al * q[v], zv = rv * dinv[v];
    r[v] = rv, z[v] = zv;
    a1 += rv * zv, a2 += rv * rv;
  }
  block_add(a1, rz_next, r1);
  block_add(a2, rr_next, r2);
}

// p = z + beta p, beta = rz_next / rz
__global__ void __launch_bounds__(HB) k_heat_dir(u64 V, const double* rz, const double* rz_next, const double* z,
                                                 double* p) {
  const double be = *rz != 0.0 ? *rz_next / *rz : 0.0;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x)
    p[v] = z[v] + be * p[v];
}

// per-block maxima of u (the host takes the largest)
__global__ void __launch_bounds__(HB) k_heat_max(u64 V, const double* u, double* out) {
  __shared__ double s[HB / 32];
  double m = -1.0e308;
  for (u64 v = (u64)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (u64)gridDim.x * blockDim.x)
    m = fmax(m, u[v]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x / 32); ++w) m = fmax(m, s[w]);
    out[blockIdx.x] = m;
  }
}

unsigned grid_v(u64 n) { return (unsigned)std::max<u64>(1, std::min<u64>((n + HB - 1) / HB, 152 * 8)); }

}  // namespace

constexpr int RED_BLOCKS = 152 * 8;  // the most blocks of a reducing launch (grid_v)

size_t heat_scratch_bytes(u64 T, u64 V, int maxit) {
  return 256 * 32 + T * (sizeof(HeatTri) + 6 * (4 + 8) + 4 + 4 + 12) + V * (4 + 4 + 4 + 4 + 4 + 4 + 4 + 8 * 10) +
         8 * 4 * (size_t)(maxit + 1) + 8 * 152 * 8 + 8 * 2 * RED_BLOCKS + 16 +
         4 * scan_scratch_words((u32)std::min<u64>(std::max(T, V), 0xFFFFFFFFu));
}

int heat_solve(const double* xy, const int* tri, const unsigned short* label, u64 T, u64 V, int L, double alpha,
               double dt, int nsteps, double x0, double y0, double sigma, double amp, double tol, int maxit,
               double* u, double* peaks, int* iters, void* scratch, cudaStream_t st) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* s = (char*)scratch;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = s + off;
    off = up(off + bytes);
    return p;
  };
  HeatTri* rec = (HeatTri*)take(T * sizeof(HeatTri));
  u32* flag = (u32*)take(4 * V);
  u32* fidx = (u32*)take(4 * (V + 1));
  u32* list = (u32*)take(4 * V);
  u32* tf = (u32*)take(4 * T);          // region triangles as 0/1
  u32* tpos = (u32*)take(4 * (T + 1));  // their scan: record positions
  u32* vcnt = (u32*)take(4 * V);        // records per free vertex
  u32* vptr = (u32*)take(4 * (V + 1));  // their scan
  u32* inc = (u32*)take(4 * 3 * T);     // incident records per free vertex
  double* mass = (double*)take(8 * V);
  double* kdiag = (double*)take(8 * V);
  double* dinv = (double*)take(8 * V);
  double* dg = (double*)take(8 * V);
  u32* rowptr = (u32*)take(4 * (V + 1));
  u32* mcnt = (u32*)take(4 * V);
  u32* col = (u32*)take(4 * 6 * T);
  double* val = (double*)take(8 * 6 * T);
  double* x = (double*)take(8 * V);
  double* b = (double*)take(8 * V);
  double* q = (double*)take(8 * V);
  double* r = (double*)take(8 * V);
  double* z = (double*)take(8 * V);
  double* p = (double*)take(8 * V);
  double* sc = (double*)take(8 * 4 * (size_t)(maxit + 1));  // 4 per iteration
  double* bmax = (double*)take(8 * 152 * 8);
  double* part = (double*)take(8 * 2 * RED_BLOCKS);
  u32* rdone = (u32*)take(16);
  u32* sscr = (u32*)take(4 * scan_scratch_words((u32)std::max(T, V)) + 4);
  const Red r1{part, rdone}, r2{part + RED_BLOCKS, rdone + 1};
  const unsigned gt = grid_v(T);
  const double tau = alpha * dt;
  int launches = 0;
  if (cudaMemsetAsync(flag, 0, 4 * V, st) || cudaMemsetAsync(rdone, 0, 16, st)) return -1;
  k_heat_flags<<<gt, HB, 0, st>>>(tri, label, T, L, flag);
  k_heat_free<<<grid_v(V), HB, 0, st>>>(V, flag);
  launches += 2 + launch_scan(flag, 1, fidx, (u32)V, sscr, st);
  k_heat_list<<<grid_v(V), HB, 0, st>>>(V, flag, fidx, list);
  k_heat_tflag<<<gt, HB, 0, st>>>(label, T, L, tf);
  launches += 2 + launch_scan(tf, 1, tpos, (u32)T, sscr, st);
  u32 n = 0, nr = 0;
  if (cudaMemcpyAsync(&n, fidx + V, 4, cudaMemcpyDeviceToHost, st) ||
      cudaMemcpyAsync(&nr, tpos + T, 4, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
    return -1;
  if (cudaMemsetAsync(vcnt, 0, 4 * (size_t)std::max<u32>(n, 1), st)) return -1;
  k_heat_setup<<<gt, HB, 0, st>>>(xy, tri, label, T, L, flag, fidx, tpos, rec, vcnt);
  const unsigned gv = grid_v(n);
  const unsigned gr = grid_v(nr);
  launches += 1;
  if (n > 0) {
    // the free vertices' incident records, sorted, then their mass and diagonal
    launches += launch_scan(vcnt, 1, vptr, n, sscr, st);
    if (cudaMemcpyAsync(mcnt, vptr, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st)) return -1;
    k_heat_inc<<<gr, HB, 0, st>>>(rec, nr, mcnt, inc);
    k_heat_gather<<<gv, HB, 0, st>>>(rec, n, vptr, inc, mass, kdiag);
    k_heat_init<<<gv, HB, 0, st>>>(xy, n, list, mass, kdiag, tau, x0, y0, sigma * sigma, amp, x, dg, dinv);
    launches += 3;
  }
  // the rows: counts (in flag, free now), their scan, then the entries at
  // cursors starting from the row offsets
  if (n > 0) {
    if (cudaMemsetAsync(flag, 0, 4 * (size_t)n, st)) return -1;
    k_heat_rowcount<<<gr, HB, 0, st>>>(rec, nr, flag);
    launches += 1 + launch_scan(flag, 1, rowptr, n, sscr, st);
    if (cudaMemcpyAsync(flag, rowptr, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st)) return -1;
    k_heat_fill<<<gr, HB, 0, st>>>(rec, nr, tau, flag, col, val);
    k_heat_merge<<<gv, HB, 0, st>>>(n, rowptr, col, val, mcnt);
    launches += 2;
  }
  bool converged = true;
  if (n == 0)
    for (int step = 0; step < nsteps; ++step) {
      if (iters) iters[step] = 0;
      if (peaks) peaks[step] = 0.0;
    }
  for (int step = 0; step < nsteps && n > 0; ++step) {
    // b = M x_n; start from x_n: r = b - A x_n
    if (cudaMemsetAsync(sc, 0, 8 * 4 * (size_t)(maxit + 1), st)) return -1;
    k_heat_mass<<<gv, HB, 0, st>>>(n, mass, x, b);
    k_heat_apply<<<gv, HB, 0, st>>>(n, rowptr, mcnt, col, val, dg, x, q, bmax, r1);
    k_heat_start<<<gv, HB, 0, st>>>(n, b, q, dinv, r, z, p, sc + 1, sc + 2, r1, r2);
    k_heat_dot<<<gv, HB, 0, st>>>(n, b, b, sc + 3, r1);
    launches += 4;
    double h2[2];
    if (cudaMemcpyAsync(h2, sc + 2, 16, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st)) return -1;
    const double stop = tol * tol * h2[1];
    double rr = h2[0];
    int it = 0;
    while (rr > stop && it < maxit) {
      double* s0 = sc + 4 * it;  // {p.q, r.z, r.r, -} of iteration it; the next iteration's at s0 + 4
      k_heat_apply<<<gv, HB, 0, st>>>(n, rowptr, mcnt, col, val, dg, p, q, s0, r1);
      k_heat_update<<<gv, HB, 0, st>>>(n, s0, x, r, z, p, q, dinv, s0 + 5, s0 + 6, r1, r2);
      k_heat_dir<<<gv, HB, 0, st>>>(n, s0 + 1, s0 + 5, z, p);
      launches += 3;
      ++it;
      // the residual, read back every eighth iteration
      if ((it & 7) == 0 || it == maxit) {
        if (cudaMemcpyAsync(&rr, sc + 4 * it + 2, 8, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
          return -1;
      }
    }
    if (iters) iters[step] = it;
    if (peaks) {
      k_heat_max<<<gv, HB, 0, st>>>(n, x, bmax);
      ++launches;
      std::vector<double> hb(gv);
      if (cudaMemcpyAsync(hb.data(), bmax, 8 * gv, cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
        return -1;
      peaks[step] = std::max(0.0, *std::max_element(hb.begin(), hb.end()));
    }
    if (rr > stop) {
      converged = false;
      break;
    }
  }
  k_heat_zero<<<grid_v(V), HB, 0, st>>>(V, u);
  k_heat_put<<<std::max(gv, 1u), HB, 0, st>>>(n, list, x, u);
  launches += 2;
  if (!converged) return -2;
  return launches;
}

}  // namespace sbmt
