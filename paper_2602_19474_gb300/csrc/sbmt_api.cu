// sbmt_api.cu -- the C interface (include/sbmt.h): context, buffers, grid
// tables and the ordered launch of the hot-path kernels on one stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <sys/stat.h>

#include "sbmt.h"
#include "sbmt_launch.h"

using namespace sbmt;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(SBMT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

// grid tables of Sec. 3.3's lattice, on the host: per strip row the range of
// cells meeting the closed image rectangle, per vertex row the range of
// lattice vertices they use
struct Tables {
  std::vector<i64> clo, chi, cbase, vlo, vhi, vbase;
  std::vector<int> lrow;  // per strip row: pixel rows of up-cell and down-cell centroids
  i64 j0 = 0, vj0 = 0, ncells = 0, nverts = 0;
};

int build_tables(const GridP& g, Tables& t) {
  const i64 p = g.p, q = g.q, ox = g.ox, oy = g.oy, P6 = 6 * p;
  const i64 xl = -3 * q, xr = 6 * q * g.W - 3 * q, yl = -3 * q, yr = 6 * q * g.H - 3 * q;
  const i64 j0 = strip_of(g, zq(yl)), j1 = strip_of(g, zq(yr));
  t.j0 = j0;
  const i64 nrows = j1 - j0 + 1;
  t.clo.resize(nrows), t.chi.resize(nrows), t.cbase.resize(nrows), t.lrow.resize(2 * nrows);
  i64 base = 0;
  for (i64 j = j0; j <= j1; ++j) {
    // centroid heights oy + (3pj + p) sqrt3 (up) and oy + (3pj + 2p) sqrt3
    // (down); pixel row = floor(y / S + 1/2)
    t.lrow[2 * (j - j0)] = (int)zfloordiv(Zq{2 * oy + g.S, 2 * (3 * p * j + p)}, 2 * g.S);
    t.lrow[2 * (j - j0) + 1] = (int)zfloordiv(Zq{2 * oy + g.S, 2 * (3 * p * j + 2 * p)}, 2 * g.S);
    const Zq yj = zq(oy, 3 * p * j), yj1 = zq(oy, 3 * p * (j + 1));
    // the band of the strip inside the rectangle is [ya, yb]; an up cell is
    // widest at ya, a down cell at yb; da, db = the slant offsets there
    const Zq da = zcmp(yj, zq(yl)) >= 0 ? zq(0) : Zq{-3 * p * j, (yl - oy) / 3};
    const Zq db = zcmp(yj1, zq(yr)) <= 0 ? zq(0) : Zq{3 * p * (j + 1), -(yr - oy) / 3};
    const i64 iu_hi = zfloordiv(zq(xr - ox - 3 * p * j) - da, P6);
    const i64 iu_lo = -zfloordiv(zq(-(xl - ox - 3 * p * j - P6)) - da, P6);
    const i64 id_hi = zfloordiv(zq(xr - ox - 3 * p * (j + 1)) - db, P6);
    const i64 id_lo = -zfloordiv(zq(-(xl - ox - 3 * p * (j + 3))) - db, P6);
    i64 lo = INT64_MAX, hi = INT64_MIN;
    if (iu_lo <= iu_hi) lo = std::min(lo, 2 * iu_lo), hi = std::max(hi, 2 * iu_hi);
    if (id_lo <= id_hi) lo = std::min(lo, 2 * id_lo + 1), hi = std::max(hi, 2 * id_hi + 1);
    if (lo > hi) return fail(SBMT_EINTERNAL, "empty cell row %lld", (long long)j);
    // the union of both families must be contiguous: every even c in
    // [lo, hi] an up cell, every odd c a down cell
    auto fl2 = [](i64 x) { return x >> 1; };
    auto ce2 = [](i64 x) { return -((-x) >> 1); };
    const bool even_ok = ce2(lo) > fl2(hi) || (iu_lo <= ce2(lo) && iu_hi >= fl2(hi));
    const bool odd_ok = ce2(lo - 1) > fl2(hi - 1) || (id_lo <= ce2(lo - 1) && id_hi >= fl2(hi - 1));
    if (!even_ok || !odd_ok) return fail(SBMT_EINTERNAL, "cell row %lld not contiguous", (long long)j);
    t.clo[j - j0] = lo, t.chi[j - j0] = hi, t.cbase[j - j0] = base;
    base += hi - lo + 1;
  }
  t.ncells = base;
  // vertex rows j0 .. j1 + 1: row j holds the bottom vertices of strip j and
  // the top vertices of strip j - 1
  t.vj0 = j0;
  const i64 nv = nrows + 1;
  t.vlo.assign(nv, INT64_MAX), t.vhi.assign(nv, INT64_MIN), t.vbase.resize(nv);
  for (i64 r = 0; r < nrows; ++r) {
    const i64 lo = t.clo[r], hi = t.chi[r];
    // up(i): bottom i, i+1, top i; down(i): bottom i+1, top i, i+1
    const i64 bmin = (lo & 1) ? (lo >> 1) + 1 : (lo >> 1), bmax = (hi >> 1) + 1;
    const i64 tmin = lo >> 1, tmax = (hi & 1) ? (hi >> 1) + 1 : (hi >> 1);
    t.vlo[r] = std::min(t.vlo[r], bmin), t.vhi[r] = std::max(t.vhi[r], bmax);
    t.vlo[r + 1] = std::min(t.vlo[r + 1], tmin), t.vhi[r + 1] = std::max(t.vhi[r + 1], tmax);
  }
  for (i64 r = 1; r < nrows; ++r) {
    // the two contributions to an inner row overlap (cells of adjacent strips share it)
    const i64 lo = t.clo[r], hi = t.chi[r];
    const i64 bmin = (lo & 1) ? (lo >> 1) + 1 : (lo >> 1), bmax = (hi >> 1) + 1;
    const i64 tmin = t.clo[r - 1] >> 1, tmax = (t.chi[r - 1] & 1) ? (t.chi[r - 1] >> 1) + 1 : (t.chi[r - 1] >> 1);
    if (bmin > tmax + 1 || tmin > bmax + 1) return fail(SBMT_EINTERNAL, "vertex row %lld split", (long long)r);
  }
  base = 0;
  for (i64 r = 0; r < nv; ++r) t.vbase[r] = base, base += t.vhi[r] - t.vlo[r] + 1;
  t.nverts = base;
  return SBMT_OK;
}

// device memory or an event shared by the meshes of one batch, released
// with the last of them
struct Shared {
  void* ptr = nullptr;
  cudaEvent_t ev = nullptr;
  int refs = 0;
};

struct MeshRec {
  sbmt_mesh id = 0;
  cudaEvent_t done = nullptr;   // completion of the mesh's work
  Shared* done_sh = nullptr;    // the batch's completion event (done is its event)
  bool own_done = false;        // done is this mesh's own pooled event
  Shared* out_sh = nullptr;     // the batch's output block holding this mesh
  void* out_block = nullptr;    // this mesh's own output block (preprocessed meshes)
  double* xy = nullptr;
  int* tri = nullptr;
  unsigned short* label = nullptr;
  unsigned short* code = nullptr;
  int64_t nv = 0, nt = 0, ncells = 0, nseg_total = 0, ne_total = 0, nc_total = 0, nvg = 0;
  size_t bytes = 0;  // device bytes of the mesh's outputs (and kept stages)
  // SBMT_COMPACT: per-cell labels and codes, the cut cells' patch list
  int format = SBMT_EXPLICIT;
  unsigned short* cell_label = nullptr;
  unsigned short* cell_code = nullptr;
  u32* patch_cell = nullptr;
  u32* patch_off = nullptr;
  u32* h_info = nullptr;  // pinned: err, ncut, ntierg, tierg triangles, cells over the Tier-G limit
  u32* over_cells = nullptr;  // device: ids of the cells over the Tier-G limit (OVER_CAP at most)
  int W = 0, H = 0;
  // kept intermediates (SBMT_KEEP_STAGES)
  bool keep = false;
  Seg* segs = nullptr;
  u32 nseg = 0;
  Event* ev = nullptr;
  u32 ne = 0;
  CutRec* recs = nullptr;
  u32* bcut = nullptr;
  u32* bbase = nullptr;
  u32 nbc = 0;
  std::vector<void*> scratch;  // device memory freed with the mesh
  // preprocessed meshes (Alg. 3): the counts are known once the work is done
  // (h_info: err, eliminations, split cells, snapped, repelled, points with
  // a candidate)
  bool pre = false, settled = false;
  // Region III meshes (Alg. 2 on a preprocessed mesh): h_info holds the
  // error bits, cut cells, Tier-G cells and Tier-G triangles
  bool r3 = false;
  unsigned char* pstatus = nullptr;
  int* psnap = nullptr;
  int* pelim = nullptr;
  double thr[3] = {0, 0, 0};
  int64_t npts = 0;
};

}  // namespace

// stages of the hot path, in launch order (for the per-stage timing)
enum {
  KN_CORNER,
  KN_SEG,
  KN_TCOUNT,
  KN_SCAN,
  KN_TEMIT,
  KN_RANK,
  KN_SORT,
  KN_CUTCELLS,
  KN_EMIT,
  KN_TIERG,
  KN_XY,
  KN_PRE,
  KN_HEAT,
  KN_R3,
  KN_COUNT
};
const char* const kKernelNames[KN_COUNT] = {"k_corner_bits", "k_segments", "k_seg_count", "k_scan",
                                            "k_walk", "k_rank", "k_sort", "k_cutcells", "k_emit",
                                            "k_tierg", "k_lattice_xy", "k_preprocess", "k_heat",
                                            "k_region3"};

// The context's stream of work with its side streams, scratch arena, staging
// buffers and tracing events.
struct Lane {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the Tier-G kernels (and the registry's large buckets) run on side
  // streams beside the main kernels, forked from and joined back into the
  // lane's stream
  cudaStream_t side = nullptr, side2 = nullptr;  // side2: the Tier-G warp kernel
  cudaEvent_t fork = nullptr, join = nullptr, order = nullptr, warp = nullptr, lat = nullptr;
  // per-call scratch: bump allocation in stream-ordered chunks
  std::vector<std::pair<char*, size_t>> chunks;
  size_t chunk_used = 0, call_bytes = 0;
  // pinned staging of the job tables, reused once its last copy is done
  char* stage = nullptr;
  size_t stage_cap = 0;
  cudaEvent_t stage_ev = nullptr;
  // mapped pinned memory receiving the counting phase's results
  u32* cnt_h = nullptr;
  u32* cnt_d = nullptr;
  size_t cnt_cap = 0;
  // the emission phase as a CUDA graph (updated in place call to call)
  cudaGraphExec_t gexec = nullptr;
  bool capturing = false;
  // tracing: events around each kernel launch, resolved lazily
  struct Mark {
    int k, kernels;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Mark> pending;
};

// launch parameters of the batched path (chosen per size class by the tuner)
struct Tune {
  int cut_blocks_per_sm = 8;     // persistent cut-cell kernel, 128 threads a block
  int tierg_blocks_per_sm = 24;  // persistent Tier-G thread kernel, 64 threads a block
  int fork = 1;                  // Tier-G and the large registry buckets on side streams
  int graph = 0;                 // the emission phase captured into a CUDA graph
};

struct sbmt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;   // one API call at a time
  std::mutex reg;  // meshes, ids, events, pinned slots, tables
  std::map<sbmt_mesh, MeshRec*> meshes;
  sbmt_mesh next = 1;
  Lane main;
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[KN_COUNT] = {};
  int64_t prof_n[KN_COUNT] = {};
  // grid tables per (W, H, h, origin), kept on the device; entries uploaded
  // together share one device block
  struct TableEntry {
    Tables host;
    i64* dev = nullptr;
    Shared* block = nullptr;
    uint64_t last_use = 0;
  };
  std::map<std::array<i64, 6>, TableEntry> tables;
  uint64_t tick = 0;
  // pinned slots for the per-mesh status words (mapped: kernels write them)
  std::vector<std::pair<u32*, u32*>> pinned_slabs;  // host, device
  std::vector<u32*> pinned_free;
  // tuning: the launch parameters in use, and per size class those chosen
  // by mesh_autotune (also read from and written to the tuning file)
  Tune tune;
  std::map<std::string, Tune> tuned;
  bool tuned_loaded = false;
};

namespace {

cudaEvent_t take_event(std::vector<cudaEvent_t>& pool) {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// a context-level event (mesh completion); callers hold ctx->reg
cudaEvent_t pool_event(sbmt_ctx* c) { return take_event(c->ev_pool); }

void prof_collect_lane(sbmt_ctx* c, Lane* L) {
  for (auto& mk : L->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(mk.b) == cudaSuccess && cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
      c->prof_ms[mk.k] += ms;
      c->prof_n[mk.k] += mk.kernels;
    }
    L->ev_pool.push_back(mk.a), L->ev_pool.push_back(mk.b);
  }
  L->pending.clear();
}
void prof_collect(sbmt_ctx* c) { prof_collect_lane(c, &c->main); }

// brackets one launcher call with events on the lane's stream when tracing
// (not while the lane's stream is being captured into a graph)
struct ProfScope {
  Lane* L;
  cudaStream_t s;
  int k, kernels = 0;
  cudaEvent_t a = nullptr;
  ProfScope(sbmt_ctx* c, Lane* L_, int k_, cudaStream_t s_) : L(L_), s(s_), k(k_) {
    if (c->prof && !L->capturing && (a = take_event(L->ev_pool))) cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = take_event(L->ev_pool);
    cudaEventRecord(b, s);
    L->pending.push_back({k, kernels, a, b});
  }
};
#define TRACE_ON(kn, strm, call)           \
  do {                                     \
    ProfScope ps_(ctx, lane, kn, strm);    \
    ps_.kernels = (call);                  \
  } while (0)
#define TRACE(kn, call) TRACE_ON(kn, lane->stream, call)

// scratch arena: every call bumps through the lane's chunks; a call that
// needed more than one chunk leaves a single chunk of its total size for the
// next call (frees and allocations are ordered on the lane's stream)
template <typename T>
int aalloc(Lane* L, T** p, size_t count) {
  const size_t bytes = (std::max<size_t>(count * sizeof(T), 16) + 255) & ~(size_t)255;
  L->call_bytes += bytes;
  if (L->chunks.empty() || L->chunk_used + bytes > L->chunks.back().second) {
    const size_t want = std::max<size_t>(bytes, L->chunks.empty() ? ((size_t)64 << 20) : 2 * L->chunks.back().second);
    void* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, want, L->stream);
    if (e != cudaSuccess) return fail(SBMT_ENOMEM, "scratch chunk of %zu bytes: %s", want, cudaGetErrorString(e));
    L->chunks.push_back({(char*)v, want});
    L->chunk_used = 0;
  }
  *p = (T*)(L->chunks.back().first + L->chunk_used);
  L->chunk_used += bytes;
  return SBMT_OK;
}
void arena_begin(Lane* L) {
  L->call_bytes = 0;
  L->chunk_used = 0;
  // keep only the first chunk's position: reuse from the start
  while (L->chunks.size() > 1) {
    cudaFreeAsync(L->chunks.back().first, L->stream);
    L->chunks.pop_back();
  }
}
void arena_end(Lane* L) {
  if (L->chunks.size() <= 1) return;
  const size_t total = L->call_bytes + ((size_t)16 << 20);
  for (auto& c : L->chunks) cudaFreeAsync(c.first, L->stream);
  L->chunks.clear();
  void* v = nullptr;
  if (cudaMallocAsync(&v, total, L->stream) == cudaSuccess) L->chunks.push_back({(char*)v, total});
}
void lane_release(Lane* L) {
  for (auto& c : L->chunks) cudaFreeAsync(c.first, L->stream);
  L->chunks.clear();
  cudaStreamSynchronize(L->stream);
  for (cudaEvent_t e : L->ev_pool) cudaEventDestroy(e);
  L->ev_pool.clear();
  if (L->gexec) cudaGraphExecDestroy(L->gexec), L->gexec = nullptr;
  if (L->stage) cudaFreeHost(L->stage), L->stage = nullptr;
  if (L->cnt_h) cudaFreeHost(L->cnt_h), L->cnt_h = nullptr;
  if (L->own_stream) cudaStreamDestroy(L->stream);
  if (L->side) cudaStreamSynchronize(L->side), cudaStreamDestroy(L->side);
  if (L->side2) cudaStreamSynchronize(L->side2), cudaStreamDestroy(L->side2);
  for (cudaEvent_t e : {L->fork, L->join, L->order, L->warp, L->lat, L->stage_ev})
    if (e) cudaEventDestroy(e);
}

// the lane's second and third streams, made on first use (highest priority:
// the Tier-G kernels' largest cells are the long pole of the call)
int lane_side(Lane* L) {
  if (L->side && L->side2) return SBMT_OK;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  for (cudaStream_t* s : {&L->side, &L->side2})
    if (!*s && cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, hi) != cudaSuccess) {
      *s = nullptr;
      return fail(SBMT_ECUDA, "side stream");
    }
  for (cudaEvent_t* e : {&L->fork, &L->join, &L->order, &L->warp, &L->lat})
    if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
      *e = nullptr;
      return fail(SBMT_ECUDA, "fork/join events");
    }
  return SBMT_OK;
}

// pinned staging of `bytes` for a host-to-device copy on the lane's stream;
// waits until the previous copy from it is done
int stage_begin(Lane* L, size_t bytes, char** out) {
  if (!L->stage_ev && cudaEventCreateWithFlags(&L->stage_ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(SBMT_ECUDA, "staging event");
  if (cudaEventSynchronize(L->stage_ev) != cudaSuccess) return fail(SBMT_ECUDA, "staging wait");
  if (bytes > L->stage_cap) {
    if (L->stage) cudaFreeHost(L->stage), L->stage = nullptr, L->stage_cap = 0;
    const size_t want = std::max<size_t>(bytes, (size_t)1 << 20) * 2;
    if (cudaMallocHost(&L->stage, want) != cudaSuccess) return fail(SBMT_ENOMEM, "pinned staging of %zu bytes", want);
    L->stage_cap = want;
  }
  *out = L->stage;
  return SBMT_OK;
}
int stage_copy(Lane* L, void* dst, size_t bytes) {
  if (cudaMemcpyAsync(dst, L->stage, bytes, cudaMemcpyHostToDevice, L->stream) != cudaSuccess ||
      cudaEventRecord(L->stage_ev, L->stream) != cudaSuccess)
    return fail(SBMT_ECUDA, "job table upload");
  return SBMT_OK;
}
// mapped pinned words for the counting phase's results
int lane_counts(Lane* L, size_t words) {
  if (words <= L->cnt_cap) return SBMT_OK;
  if (L->cnt_h) cudaFreeHost(L->cnt_h), L->cnt_h = nullptr, L->cnt_cap = 0;
  const size_t want = std::max<size_t>(words, 4096) * 2;
  if (cudaHostAlloc(&L->cnt_h, want * sizeof(u32), cudaHostAllocMapped) != cudaSuccess)
    return fail(SBMT_ENOMEM, "pinned counts");
  if (cudaHostGetDevicePointer(&L->cnt_d, L->cnt_h, 0) != cudaSuccess) return fail(SBMT_ECUDA, "mapped counts");
  L->cnt_cap = want;
  return SBMT_OK;
}

// callers hold ctx->reg
u32* pinned_slot(sbmt_ctx* ctx) {
  if (ctx->pinned_free.empty()) {
    u32* slab = nullptr;
    u32* dslab = nullptr;
    if (cudaHostAlloc(&slab, 1024 * 8 * sizeof(u32), cudaHostAllocMapped) != cudaSuccess) return nullptr;
    if (cudaHostGetDevicePointer(&dslab, slab, 0) != cudaSuccess) {
      cudaFreeHost(slab);
      return nullptr;
    }
    ctx->pinned_slabs.push_back({slab, dslab});
    for (int k = 1023; k >= 0; --k) ctx->pinned_free.push_back(slab + 8 * k);
  }
  u32* p = ctx->pinned_free.back();
  ctx->pinned_free.pop_back();
  std::memset(p, 0, 8 * sizeof(u32));
  return p;
}
// the device address of a pinned slot; callers hold ctx->reg
u32* pinned_dev(sbmt_ctx* ctx, u32* host) {
  for (auto& s : ctx->pinned_slabs)
    if (host >= s.first && host < s.first + 1024 * 8) return s.second + (host - s.first);
  return nullptr;
}

// grid tables for a batch of configurations, built once and kept on the
// device.  The entries a call adds are built on the host and uploaded
// together, in one block shared by them.  An evicted entry may still be
// read by work in flight, so eviction waits for the device; entries the
// call uses are never evicted by it.
int get_tables_many(sbmt_ctx* ctx, Lane* lane, const std::vector<GridP>& G, std::vector<const Tables*>& host,
                    std::vector<const i64*>& dev) {
  const size_t n = G.size();
  host.assign(n, nullptr), dev.assign(n, nullptr);
  std::vector<std::array<i64, 6>> keys(n);
  std::vector<size_t> missing;
  std::map<std::array<i64, 6>, size_t> first_missing;
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    ++ctx->tick;
    for (size_t k = 0; k < n; ++k) {
      const GridP& g = G[k];
      keys[k] = {g.W, g.H, g.p, g.q, g.ox, g.oy};
      auto it = ctx->tables.find(keys[k]);
      if (it != ctx->tables.end()) {
        it->second.last_use = ctx->tick;
      } else if (!first_missing.count(keys[k])) {
        first_missing[keys[k]] = k;
        missing.push_back(k);
      }
    }
    if (ctx->tables.size() + missing.size() > 1024) {  // evict the least recently used entries
      cudaDeviceSynchronize();
      std::vector<std::pair<uint64_t, std::array<i64, 6>>> age;
      for (auto& kv : ctx->tables)
        if (kv.second.last_use != ctx->tick) age.push_back({kv.second.last_use, kv.first});
      std::sort(age.begin(), age.end());
      for (size_t a = 0; a < age.size() && ctx->tables.size() + missing.size() > 1024; ++a) {
        auto it = ctx->tables.find(age[a].second);
        Shared* b = it->second.block;
        if (--b->refs == 0) cudaFree(b->ptr), delete b;
        ctx->tables.erase(it);
      }
    }
  }
  if (!missing.empty()) {
    std::vector<Tables> built(missing.size());
    std::vector<size_t> off(missing.size());
    size_t words = 0;
    for (size_t u = 0; u < missing.size(); ++u) {
      if (int rc = build_tables(G[missing[u]], built[u])) return rc;
      const Tables& tb = built[u];
      off[u] = words;
      words += (6 * tb.clo.size() + 3 * tb.vlo.size()) + (tb.lrow.size() + 1) / 2;
      words = (words + 7) & ~(size_t)7;
    }
    std::vector<i64> all(std::max<size_t>(words, 1));
    for (size_t u = 0; u < missing.size(); ++u) {
      const Tables& tb = built[u];
      i64* o = all.data() + off[u];
      for (const std::vector<i64>* v : {&tb.clo, &tb.chi, &tb.cbase, &tb.vlo, &tb.vhi, &tb.vbase}) {
        std::copy(v->begin(), v->end(), o);
        o += v->size();
      }
      std::memcpy(o, tb.lrow.data(), tb.lrow.size() * sizeof(int));
    }
    Shared* blk = new Shared();
    if (cudaMallocAsync(&blk->ptr, all.size() * sizeof(i64), lane->stream) != cudaSuccess) {
      delete blk;
      return fail(SBMT_ENOMEM, "table allocation");
    }
    // from pageable memory the copy has read `all` when the call returns
    if (cudaMemcpyAsync(blk->ptr, all.data(), all.size() * sizeof(i64), cudaMemcpyHostToDevice, lane->stream) !=
        cudaSuccess) {
      cudaFreeAsync(blk->ptr, lane->stream);
      delete blk;
      return fail(SBMT_ECUDA, "table upload");
    }
    std::lock_guard<std::mutex> lk(ctx->reg);
    for (size_t u = 0; u < missing.size(); ++u) {
      sbmt_ctx::TableEntry te;
      te.host = std::move(built[u]);
      te.dev = (i64*)blk->ptr + off[u];
      te.block = blk;
      te.last_use = ctx->tick;
      blk->refs++;
      ctx->tables.emplace(keys[missing[u]], std::move(te));
    }
  }
  std::lock_guard<std::mutex> lk(ctx->reg);
  for (size_t k = 0; k < n; ++k) {
    auto it = ctx->tables.find(keys[k]);
    host[k] = &it->second.host;
    dev[k] = it->second.dev;
  }
  return SBMT_OK;
}

int get_tables(sbmt_ctx* ctx, Lane* lane, const GridP& g, const Tables** host, const i64** dev) {
  std::vector<GridP> G{g};
  std::vector<const Tables*> h;
  std::vector<const i64*> d;
  if (int rc = get_tables_many(ctx, lane, G, h, d)) return rc;
  *host = h[0], *dev = d[0];
  return SBMT_OK;
}

// the device tables of one configuration into its grid
void set_grid_tables(GridP& g, const Tables& tb, const i64* dt) {
  const i64 nrows = (i64)tb.clo.size(), nvr = (i64)tb.vlo.size();
  g.j0 = (int)tb.j0, g.nrows = (int)nrows, g.vj0 = (int)tb.vj0, g.nvrows = (int)nvr;
  g.clo = dt, g.chi = dt + nrows, g.cbase = dt + 2 * nrows;
  g.vlo = dt + 3 * nrows, g.vhi = dt + 3 * nrows + nvr, g.vbase = dt + 3 * nrows + 2 * nvr;
  g.lrow = (const int*)(dt + 3 * nrows + 3 * nvr);
  g.ncells = tb.ncells, g.nverts = tb.nverts;
}

template <typename T>
int dalloc(Lane* L, T** p, size_t count, std::vector<void*>& track) {
  void* v = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMallocAsync(&v, bytes, L->stream);
  if (e != cudaSuccess) return fail(SBMT_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
  track.push_back(v);
  *p = (T*)v;
  return SBMT_OK;
}

void free_list(cudaStream_t st, std::vector<void*>& v) {
  for (void* p : v) cudaFreeAsync(p, st);
  v.clear();
}

// frees a mesh's memory, ordered on st after the mesh's own work; callers
// hold ctx->reg
void destroy_mesh(sbmt_ctx* ctx, MeshRec* m, cudaStream_t st) {
  if (m->done) cudaEventSynchronize(m->done);
  free_list(st, m->scratch);
  if (m->out_block) cudaFreeAsync(m->out_block, st);
  if (m->out_sh && --m->out_sh->refs == 0) cudaFreeAsync(m->out_sh->ptr, st), delete m->out_sh;
  if (m->own_done && m->done) ctx->ev_pool.push_back(m->done);
  if (m->done_sh && --m->done_sh->refs == 0) ctx->ev_pool.push_back(m->done_sh->ev), delete m->done_sh;
  if (m->h_info) ctx->pinned_free.push_back(m->h_info);
  delete m;
}

// pre: mesh_preprocess's parameters; base: the general path's base mesh
// (any integer origin, no thresholds)
int check_params(const sbmt_image* img, const sbmt_params* pr, bool pre = false, bool base = false) {
  if (!img || !pr || !img->data) return fail(SBMT_EINVAL, "null image or params");
  if (img->width < 1 || img->height < 1 || img->width > 32768 || img->height > 32768)
    return fail(SBMT_EINVAL, "image size %dx%d outside 1..32768", img->width, img->height);
  if (img->dtype != SBMT_U8 && img->dtype != SBMT_U16) return fail(SBMT_EINVAL, "dtype %d", img->dtype);
  if (img->pitch_bytes < (int64_t)img->width * img->dtype) return fail(SBMT_EINVAL, "pitch too small");
  // the kernels read a device image in place with 2-byte loads for u16
  // pixels: an odd pitch or base address would be a misaligned access (a
  // host image is copied into an aligned buffer first)
  if (img->on_device && img->dtype == SBMT_U16 && ((img->pitch_bytes & 1) || ((uintptr_t)img->data & 1)))
    return fail(SBMT_EINVAL, "a device u16 image needs an even pitch and an even address");
  if (base) {
    if (pr->format != SBMT_EXPLICIT) return fail(SBMT_EINVAL, "a degenerate origin is meshed in the explicit format");
  } else if (pre) {
    if (pr->mode != SBMT_PREPROCESS || pr->format != SBMT_EXPLICIT)
      return fail(SBMT_EINVAL, "mesh_preprocess takes mode SBMT_PREPROCESS and the explicit format");
  } else {
    if (pr->mode == SBMT_PREPROCESS) return fail(SBMT_EPROTO, "SBMT_PREPROCESS is available through mesh_bitmap");
    if (pr->mode != SBMT_PLAIN || (pr->format != SBMT_EXPLICIT && pr->format != SBMT_COMPACT))
      return fail(SBMT_EINVAL, "mode/format");
  }
  if (pr->h_num < 2 || pr->h_num > 1024 || (pr->h_num & 1) || pr->h_den < 1 || pr->h_den > 63 ||
      !(pr->h_den & 1))
    return fail(SBMT_EINVAL, "h = %d/%d outside the degeneracy-free class (even h_num <= 1024, odd h_den < 64)",
                pr->h_num, pr->h_den);
  if (pr->origin2x < -65536 || pr->origin2x > 65536 || pr->origin2y < -65536 || pr->origin2y > 65536)
    return fail(SBMT_EINVAL, "origin outside +-32768 px");
  if (!base && ((pr->origin2x & 1) || (pr->origin2y & 1)))
    return fail(SBMT_EINVAL, "origin (%d/2, %d/2) on a pixel line: mesh_bitmap meshes it (the general path); "
                "mesh_batch and mesh_preprocess take integer origins", pr->origin2x, pr->origin2y);
  return SBMT_OK;
}

GridP grid_of(const sbmt_image& img, const sbmt_params& pr) {
  GridP g{};
  g.W = img.width, g.H = img.height;
  g.p = pr.h_num, g.q = pr.h_den, g.S = 6 * g.q;
  g.ox = 3 * g.q * (i64)pr.origin2x, g.oy = 3 * g.q * (i64)pr.origin2y;
  return g;
}

// room for the boundary segments of an image before they are counted: a
// quarter of its pixel corners (real images hold a few percent), at most the
// bound of two per corner; an image with more is counted exactly and redone
u32 seg_cap_guess(int W, int H) {
  const u64 corners = (u64)(W + 1) * (u64)(H + 1);
  return (u32)std::min<u64>(2 * corners, corners / 4 + 4096);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RunOpts {
  bool fork = true;    // Tier-G and the large registry buckets on side streams
  bool graph = false;  // the emission phase captured into a CUDA graph
  bool stall = false;  // test of the device wait bound (SBMT_DEBUG_STALL_SCAN)
  int cut_blocks_per_sm = 8, tierg_blocks_per_sm = 24;
};

// per-stage block prefix over the jobs
template <class F>
std::vector<u32> prefix_of(int n, F blocks) {
  std::vector<u32> p(n + 1, 0);
  for (int k = 0; k < n; ++k) p[k + 1] = p[k] + (u32)blocks(k);
  return p;
}

// The whole path for a batch of images (one image is a batch of one), on
// one lane: a counting phase (segments and pairs per image, one launch per
// stage over all images), one host synchronisation to size the buffers, and
// an emission phase (one launch per stage, the variable-size stages
// persistent over batch-wide work queues), optionally as a CUDA graph.
int mesh_run(sbmt_ctx* ctx, Lane* lane, const sbmt_image* imgs, int n, const sbmt_params* prs, int nprs,
             sbmt_mesh* out, const RunOpts& opt) {
  if (n == 0) return SBMT_OK;
  for (int k = 0; k < n; ++k)
    if (int rc = check_params(imgs + k, prs + (nprs == 1 ? 0 : k))) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = lane->stream;
  std::vector<GridP> G(n);
  for (int k = 0; k < n; ++k) G[k] = grid_of(imgs[k], prs[nprs == 1 ? 0 : k]);
  std::vector<const Tables*> TB;
  std::vector<const i64*> DT;
  if (int rc = get_tables_many(ctx, lane, G, TB, DT)) return rc;
  for (int k = 0; k < n; ++k) {
    if (TB[k]->ncells >= (1ll << 31) || 3 * TB[k]->nverts >= (1ll << 32))
      return fail(SBMT_EINVAL, "mesh too large (%lld cells)", (long long)TB[k]->ncells);
    set_grid_tables(G[k], *TB[k], DT[k]);
  }
  std::vector<MeshRec*> M(n, nullptr);
  arena_begin(lane);
  auto bail = [&](int code) {
    arena_end(lane);
    std::lock_guard<std::mutex> lk(ctx->reg);
    for (MeshRec* m : M)
      if (m) destroy_mesh(ctx, m, st);
    return code;
  };
  std::vector<Job> J(n);
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    for (int k = 0; k < n; ++k) {
      const sbmt_params& pr = prs[nprs == 1 ? 0 : k];
      MeshRec* m = M[k] = new MeshRec();
      m->W = G[k].W, m->H = G[k].H, m->keep = (pr.flags & SBMT_KEEP_STAGES) != 0, m->format = pr.format;
      m->h_info = pinned_slot(ctx);
      if (!m->h_info) break;
      std::memset(&J[k], 0, sizeof(Job));
      J[k].hinfo = pinned_dev(ctx, m->h_info);
    }
  }
  for (int k = 0; k < n; ++k)
    if (!M[k] || !M[k]->h_info) return bail(fail(SBMT_ENOMEM, "pinned status words"));
  int rc;
  // images on the device, grids, bucket counts
  for (int k = 0; k < n; ++k) {
    const sbmt_image& img = imgs[k];
    Job& j = J[k];
    j.g = G[k], j.dtype = img.dtype;
    if (img.on_device) {
      j.img = (const unsigned char*)img.data, j.pitch = img.pitch_bytes;
    } else {
      unsigned char* d;
      j.pitch = (i64)img.width * img.dtype;
      if ((rc = aalloc(lane, &d, (size_t)j.pitch * img.height))) return bail(rc);
      if (cudaMemcpy2DAsync(d, j.pitch, img.data, img.pitch_bytes, j.pitch, img.height, cudaMemcpyHostToDevice, st))
        return bail(fail(SBMT_ECUDA, "image upload"));
      j.img = d;
    }
    j.wpr = (G[k].W + 1 + 31) / 32, j.wpc = (G[k].H + 1 + 31) / 32;
    j.nbc = (u32)((G[k].ncells + (1 << CB_LOG) - 1) >> CB_LOG);
    j.nbe = (u32)((3 * G[k].nverts + (1 << EB_LOG) - 1) >> EB_LOG);
    j.NVg = (u32)G[k].nverts;
  }
  // ---------------- counting phase ----------------
  std::vector<u32> cap(n);
  for (int k = 0; k < n; ++k) cap[k] = seg_cap_guess(G[k].W, G[k].H);
  if ((rc = lane_counts(lane, 8 * (size_t)n))) return bail(rc);
  for (int attempt = 0;; ++attempt) {
    std::vector<size_t> zoff(n);
    size_t zw = 0;
    for (int k = 0; k < n; ++k) zoff[k] = zw, zw += (job_zero_words(J[k].nbc, J[k].nbe) + 63) & ~(size_t)63;
    const std::vector<u32> tpre = prefix_of(n, [&](int k) { return mscan_tiles(cap[k]); });
    const u32 ntiles = tpre[n];
    u32* zero;
    const size_t zall = zw + 2 * (size_t)ntiles + 64;
    if ((rc = aalloc(lane, &zero, zall))) return bail(rc);
    CK(cudaMemsetAsync(zero, 0, zall * sizeof(u32), st));
    unsigned long long* flags = (unsigned long long*)(zero + zw);
    u32* ticket = zero + zw + 2 * (size_t)ntiles;
    std::vector<ScanJob> sj(n);
    for (int k = 0; k < n; ++k) {
      Job& j = J[k];
      MeshRec* m = M[k];
      const int W = G[k].W, H = G[k].H;
      j.zero = zero + zoff[k];
      if ((rc = aalloc(lane, &j.vrow, (size_t)j.wpr * (H + 1)))) return bail(rc);
      if ((rc = aalloc(lane, &j.vcol, (size_t)j.wpc * (W + 1)))) return bail(rc);
      free_list(st, m->scratch);
      if ((rc = m->keep ? dalloc(lane, &j.segs, cap[k], m->scratch) : aalloc(lane, &j.segs, cap[k]))) return bail(rc);
      if ((rc = aalloc(lane, &j.npairs, cap[k])) || (rc = aalloc(lane, &j.pbase, (size_t)cap[k] + 1))) return bail(rc);
      j.seg_cap = cap[k];
      sj[k] = ScanJob{j.npairs, j.pbase, nullptr, cap[k], j.zero + JC_NSEG, k, 0, nullptr, nullptr, j.zero + JC_ERR};
    }
    const std::vector<u32> pc = prefix_of(n, [&](int k) {
      return (u32)(((G[k].W + 1 + 255) / 256) * ((G[k].H + 1 + 31) / 32));
    });
    const std::vector<u32> ps = prefix_of(n, [&](int k) {
      return (u32)(((i64)(G[k].H + 1) * J[k].wpr + 255) / 256);
    });
    // the pair counts: a job's blocks stride over its segments, about 1216
    // blocks over the batch, at least one and at most enough for its room
    const std::vector<u32> pq = prefix_of(n, [&](int k) {
      return std::max<u32>(1, std::min<u32>((cap[k] + 255) / 256, std::max<u32>(1, 1216 / (u32)n)));
    });
    // the job table, the scan jobs and the block prefixes in one upload
    const size_t b_jobs = up256(n * sizeof(Job)), b_sj = up256(n * sizeof(ScanJob)), b_pre = up256((n + 1) * 4);
    const size_t bytes = b_jobs + b_sj + 4 * b_pre;
    char *hs, *ds;
    if ((rc = aalloc(lane, &ds, bytes)) || (rc = stage_begin(lane, bytes, &hs))) return bail(rc);
    std::memcpy(hs, J.data(), n * sizeof(Job));
    std::memcpy(hs + b_jobs, sj.data(), n * sizeof(ScanJob));
    std::memcpy(hs + b_jobs + b_sj, pc.data(), (n + 1) * 4);
    std::memcpy(hs + b_jobs + b_sj + b_pre, ps.data(), (n + 1) * 4);
    std::memcpy(hs + b_jobs + b_sj + 2 * b_pre, tpre.data(), (n + 1) * 4);
    std::memcpy(hs + b_jobs + b_sj + 3 * b_pre, pq.data(), (n + 1) * 4);
    if ((rc = stage_copy(lane, ds, bytes))) return bail(rc);
    const Job* djobs = (const Job*)ds;
    const ScanJob* dsj = (const ScanJob*)(ds + b_jobs);
    const u32* dpc = (const u32*)(ds + b_jobs + b_sj);
    const u32* dps = (const u32*)(ds + b_jobs + b_sj + b_pre);
    const u32* dtp = (const u32*)(ds + b_jobs + b_sj + 2 * b_pre);
    const u32* dpq = (const u32*)(ds + b_jobs + b_sj + 3 * b_pre);
    // the test of the wait bound: the second tile of the first image's scan
    // withholds its sums, so that the third tile's wait runs out
    const u32 stall = (opt.stall && tpre[1] >= 3) ? 1u : NONE;
    // a single image's job goes to the kernels as a parameter
    const Job* one_a = n == 1 ? &J[0] : nullptr;
    TRACE(KN_CORNER, launch_corner_bits_b(one_a, djobs, dpc, n, pc[n], st));
    TRACE(KN_SEG, launch_segments_b(one_a, djobs, dps, n, ps[n], st));
    TRACE(KN_TCOUNT, launch_seg_count_b(one_a, djobs, dpq, n, pq[n], st));
    TRACE(KN_SCAN, launch_mscan(dsj, dtp, n, ntiles, flags, ticket, stall, st));
    TRACE(KN_TCOUNT, launch_counts_b(djobs, n, lane->cnt_d, st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    bool redo = false;
    for (int k = 0; k < n; ++k) {
      const u32 err = lane->cnt_h[8 * k + 3], ns = lane->cnt_h[8 * k + 2];
      if (err & ERR_TIMEOUT) return bail(fail(SBMT_ETIMEDOUT, "a device wait ran out while counting (image %d)", k));
      if (err) return bail(fail(SBMT_EINTERNAL, "device check failed during extraction (0x%x, image %d)", err, k));
      if (ns > cap[k]) cap[k] = ns, redo = true;
    }
    if (!redo) break;
    if (attempt > 0) return bail(fail(SBMT_EINTERNAL, "segment count above its exact size"));
  }
  // ---------------- sizes ----------------
  std::vector<u64> T(n), V(n);
  u64 np_all = 0, nbe_all = 0;
  for (int k = 0; k < n; ++k) {
    Job& j = J[k];
    const u32* c = lane->cnt_h + 8 * k;
    const u64 NC = (u64)c[0] | ((u64)c[1] << 32), NP = c[4];
    j.nseg = c[2], j.NP = (u32)NP, j.NE = (u32)(NP - c[2]);
    V[k] = (u64)j.NVg + j.NE + NC, T[k] = (u64)G[k].ncells + 2 * NC + 2 * (u64)j.NE;
    if (V[k] >= (1ull << 31) || T[k] >= (1ull << 31) || NP >= (1ull << 31))
      return bail(fail(SBMT_EINVAL, "mesh too large (%llu triangles)", (unsigned long long)T[k]));
    MeshRec* m = M[k];
    m->nv = (int64_t)V[k], m->nt = (int64_t)T[k], m->ncells = G[k].ncells;
    m->nseg_total = j.nseg, m->ne_total = j.NE, m->nc_total = (int64_t)NC, m->nvg = j.NVg;
    np_all += NP, nbe_all += j.nbe;
  }
  // ---------------- emission-phase buffers ----------------
  std::vector<size_t> ooff(n);
  size_t obytes = 0;
  struct OutLay {
    size_t tri, lab, code, cl, cc, pc, po, ov;
  };
  std::vector<OutLay> L(n);
  for (int k = 0; k < n; ++k) {
    Job& j = J[k];
    MeshRec* m = M[k];
    const bool compact = m->format == SBMT_COMPACT;
    const u64 NP = j.NP, nxy = compact ? V[k] - j.NVg : V[k], ntr = compact ? (T[k] - (u64)G[k].ncells) + NP : T[k];
    OutLay& l = L[k];
    l.tri = up256(16 * nxy), l.lab = up256(l.tri + 12 * ntr), l.code = up256(l.lab + 2 * ntr);
    l.cl = up256(l.code + 2 * ntr), l.cc = up256(l.cl + (compact ? 2 * (size_t)G[k].ncells : 0));
    l.pc = up256(l.cc + (compact ? 2 * (size_t)G[k].ncells : 0));
    l.po = up256(l.pc + (compact ? 4 * NP : 0));
    l.ov = up256(l.po + (compact ? 4 * (NP + 1) : 0));
    ooff[k] = obytes;
    obytes += up256(l.ov + 4 * (size_t)OVER_CAP);
    m->bytes = up256(l.ov + 4 * (size_t)OVER_CAP);
  }
  Shared* osh = new Shared();
  if (cudaMallocAsync(&osh->ptr, std::max<size_t>(obytes, 256), st) != cudaSuccess) {
    delete osh;
    return bail(fail(SBMT_ENOMEM, "output allocation of %zu bytes", obytes));
  }
  osh->refs = n;
  for (int k = 0; k < n; ++k) M[k]->out_sh = osh;
  for (int k = 0; k < n; ++k) {
    Job& j = J[k];
    MeshRec* m = M[k];
    char* ob = (char*)osh->ptr + ooff[k];
    const OutLay& l = L[k];
    m->xy = (double*)ob, m->tri = (int*)(ob + l.tri), m->label = (unsigned short*)(ob + l.lab);
    m->code = (unsigned short*)(ob + l.code), m->over_cells = (u32*)(ob + l.ov);
    j.xy = m->xy, j.tri = m->tri, j.label = m->label, j.code = m->code, j.over = m->over_cells;
    const u32 NP = j.NP, NE = j.NE, nbc = j.nbc, nbe = j.nbe;
    if ((rc = aalloc(lane, &j.cstart, walk_chunks(NP) + 1)) || (rc = aalloc(lane, &j.raw, NP)) ||
        (rc = aalloc(lane, &j.pairs, NP)) || (rc = aalloc(lane, &j.eidx, NE)) || (rc = aalloc(lane, &j.elist, NE)) ||
        (rc = aalloc(lane, &j.poff, nbc + 1)) || (rc = aalloc(lane, &j.eoff, nbe + 1)) ||
        (rc = aalloc(lane, &j.pcur, nbc + 1)) || (rc = aalloc(lane, &j.ecur, nbe + 1)) ||
        (rc = aalloc(lane, &j.extra_scan, nbc + 1)) || (rc = aalloc(lane, &j.chain_scan, nbc + 1)) ||
        (rc = aalloc(lane, &j.stg, NP)) || (rc = aalloc(lane, &j.klist, (size_t)NCLS * NP)))
      return bail(rc);
    if (m->keep) {
      if ((rc = dalloc(lane, &j.ev, NE, m->scratch)) || (rc = dalloc(lane, &j.recs, NP, m->scratch)) ||
          (rc = dalloc(lane, &j.bcut, nbc + 1, m->scratch)) || (rc = dalloc(lane, &j.bbase, nbc + 1, m->scratch)))
        return bail(rc);
    } else {
      if ((rc = aalloc(lane, &j.ev, NE)) || (rc = aalloc(lane, &j.recs, NP)) || (rc = aalloc(lane, &j.bcut, nbc + 1)) ||
          (rc = aalloc(lane, &j.bbase, nbc + 1)))
        return bail(rc);
    }
    j.cp = CompactOut{0, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (m->format == SBMT_COMPACT) {
      m->cell_label = (unsigned short*)(ob + l.cl), m->cell_code = (unsigned short*)(ob + l.cc);
      m->patch_cell = (u32*)(ob + l.pc), m->patch_off = (u32*)(ob + l.po);
      if ((rc = aalloc(lane, &j.cut_scan, nbc + 1))) return bail(rc);
      j.cp = CompactOut{1, j.NVg, m->cell_label, m->cell_code, m->patch_cell, m->patch_off, j.cut_scan};
      if (nbc == 0) CK(cudaMemsetAsync(m->patch_off, 0, sizeof(u32), st));
    }
    // x of lattice vertex v(i, j) is indexed by m = 2i + j
    const Tables& tb = *TB[k];
    i64 m_lo = 0, m_hi = -1;
    for (size_t r = 0; r < tb.vlo.size(); ++r) {
      const i64 a = 2 * tb.vlo[r] + tb.vj0 + (i64)r, b = 2 * tb.vhi[r] + tb.vj0 + (i64)r;
      if (r == 0 || a < m_lo) m_lo = a;
      if (r == 0 || b > m_hi) m_hi = b;
    }
    j.m_lo = m_lo, j.nm = std::max<i64>(1, m_hi - m_lo + 1);
    if ((rc = aalloc(lane, &j.xtab, (size_t)j.nm))) return bail(rc);
    if (m->keep) {
      m->segs = j.segs, m->nseg = j.nseg, m->ev = j.ev, m->ne = j.NE, m->recs = j.recs, m->bcut = j.bcut;
      m->bbase = j.bbase, m->nbc = nbc;
    }
  }
  // batch-wide state, work lists and the scans' flags
  BatchPtrs bp{};
  if ((rc = aalloc(lane, &bp.olist, std::max<u64>(np_all, 1))) || (rc = aalloc(lane, &bp.slist, std::max<u64>(np_all, 1))) ||
      (rc = aalloc(lane, &bp.wlist, std::max<u64>(np_all, 1))) ||
      (rc = aalloc(lane, &bp.big, std::max<u64>(nbe_all, 1))))
    return bail(rc);
  std::vector<ScanJob> sj1(2 * n), sj2;
  const size_t bdw = (batch_dev_words(n) + 63) & ~(size_t)63;
  std::vector<u32> t1pre(2 * n + 1, 0), t2pre;
  for (int k = 0; k < n; ++k) {
    t1pre[2 * k + 1] = t1pre[2 * k] + mscan_tiles(J[k].nbc);
    t1pre[2 * k + 2] = t1pre[2 * k + 1] + mscan_tiles(J[k].nbe);
  }
  std::vector<int> sj2_job;
  for (int k = 0; k < n; ++k) {
    const int per = M[k]->format == SBMT_COMPACT ? 3 : 2;
    for (int u = 0; u < per; ++u) sj2_job.push_back(k);
  }
  const int n2 = (int)sj2_job.size();
  t2pre.assign(n2 + 1, 0);
  for (int u = 0; u < n2; ++u) t2pre[u + 1] = t2pre[u] + mscan_tiles(J[sj2_job[u]].nbc);
  const u32 nt1 = t1pre[2 * n], nt2 = t2pre[n2];
  u32* zb;
  const size_t zball = bdw + 2 * ((size_t)nt1 + nt2) + 64;
  if ((rc = aalloc(lane, &zb, zball))) return bail(rc);
  CK(cudaMemsetAsync(zb, 0, zball * sizeof(u32), st));
  bp.bd = (BatchDev*)zb;
  unsigned long long* flags1 = (unsigned long long*)(zb + bdw);
  unsigned long long* flags2 = flags1 + nt1;
  u32* tickets = zb + bdw + 2 * ((size_t)nt1 + nt2);
  for (int k = 0; k < n; ++k) {
    Job& j = J[k];
    u32* z = j.zero;
    u32* pcnt = z + JC_BUCKETS;
    u32* ecnt = pcnt + j.nbc + 1;
    sj1[2 * k] = ScanJob{pcnt, j.poff, j.pcur, j.nbc, nullptr, k, 0, nullptr, nullptr, z + JC_ERR};
    sj1[2 * k + 1] = ScanJob{ecnt, j.eoff, j.ecur, j.nbe, nullptr, k, RANK_SMALL, bp.big, &bp.bd->nbig, z + JC_ERR};
  }
  for (int u = 0, k = -1, w = 0; u < n2; ++u) {
    if (sj2_job[u] != k) k = sj2_job[u], w = 0;
    Job& j = J[k];
    u32* z = j.zero;
    u32* bextra = z + JC_BUCKETS + (j.nbc + 1) + (j.nbe + 1);  // after pcnt and ecnt
    u32* bchain = bextra + j.nbc + 1;
    if (w == 0) sj2.push_back(ScanJob{bextra, j.extra_scan, nullptr, j.nbc, nullptr, k, 0, nullptr, nullptr, z + JC_ERR});
    else if (w == 1) sj2.push_back(ScanJob{bchain, j.chain_scan, nullptr, j.nbc, nullptr, k, 0, nullptr, nullptr, z + JC_ERR});
    else sj2.push_back(ScanJob{j.bcut, j.cut_scan, nullptr, j.nbc, nullptr, k, 0, nullptr, nullptr, z + JC_ERR});
    ++w;
  }
  // block prefixes of the emission phase
  const std::vector<u32> p_cm = prefix_of(n, [&](int k) { return (J[k].nseg + 255) / 256; });
  const std::vector<u32> p_walk = prefix_of(n, [&](int k) { return (u32)((walk_chunks(J[k].NP) + 255) / 256); });
  const std::vector<u32> p_sc = prefix_of(n, [&](int k) { return (std::max(J[k].NP, J[k].NE) + 255) / 256; });
  const std::vector<u32> p_rk = prefix_of(n, [&](int k) { return J[k].nbe; });
  const std::vector<u32> p_so = prefix_of(n, [&](int k) { return (J[k].nbc + 3) / 4; });  // the emission: 4 buckets a block
  const std::vector<u32> p_sw = prefix_of(n, [&](int k) { return (J[k].nbc + 3) / 4; });  // the sort: 4 buckets a block
  const std::vector<u32> p_go = prefix_of(n, [&](int k) { return (J[k].nbc + 7) / 8; });
  const std::vector<u32> p_lt = prefix_of(n, [&](int k) {
    return M[k]->format == SBMT_COMPACT ? 0u : (u32)((J[k].nm + 255) / 256);
  });
  const std::vector<u32> p_lx = prefix_of(n, [&](int k) {
    return M[k]->format == SBMT_COMPACT ? 0u : (u32)G[k].nvrows;
  });
  // upload: jobs, scan jobs of both scans, and the prefixes
  const std::vector<const std::vector<u32>*> pres = {&p_cm, &p_walk, &p_sc, &p_rk, &p_so, &p_go, &p_lt, &p_lx,
                                                    &t1pre, &t2pre, &p_sw};
  const size_t b_jobs = up256(n * sizeof(Job)), b_s1 = up256(sj1.size() * sizeof(ScanJob)),
               b_s2 = up256(std::max<size_t>(sj2.size(), 1) * sizeof(ScanJob));
  std::vector<size_t> poffs;
  size_t bytes = b_jobs + b_s1 + b_s2;
  for (auto* p : pres) poffs.push_back(bytes), bytes += up256(p->size() * 4);
  char *hs, *ds;
  if ((rc = aalloc(lane, &ds, bytes)) || (rc = stage_begin(lane, bytes, &hs))) return bail(rc);
  std::memcpy(hs, J.data(), n * sizeof(Job));
  std::memcpy(hs + b_jobs, sj1.data(), sj1.size() * sizeof(ScanJob));
  if (!sj2.empty()) std::memcpy(hs + b_jobs + b_s1, sj2.data(), sj2.size() * sizeof(ScanJob));
  for (size_t u = 0; u < pres.size(); ++u) std::memcpy(hs + poffs[u], pres[u]->data(), pres[u]->size() * 4);
  if ((rc = stage_copy(lane, ds, bytes))) return bail(rc);
  const Job* dj = (const Job*)ds;
  const ScanJob* ds1 = (const ScanJob*)(ds + b_jobs);
  const ScanJob* ds2 = (const ScanJob*)(ds + b_jobs + b_s1);
  auto dpre = [&](int u) { return (const u32*)(ds + poffs[u]); };
  // ---------------- emission phase ----------------
  const Job* one = n == 1 ? &J[0] : nullptr;
  const bool fork = opt.fork;
  if (fork && (rc = lane_side(lane))) return bail(rc);
  cudaGraph_t graph = nullptr;
  if (opt.graph) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bail(fail(SBMT_ECUDA, "graph capture"));
    lane->capturing = true;
  }
  int kerr = 0;
  // the lattice coordinates need only the grid: written on a side stream
  // beside the compute-bound walk and registry (its writes are the only
  // bandwidth-bound work there); the Tier-G join below waits for it
  if (fork) {
    if (cudaEventRecord(lane->lat, st) != cudaSuccess || cudaStreamWaitEvent(lane->side2, lane->lat, 0) != cudaSuccess)
      kerr = 1;
    TRACE_ON(KN_XY, lane->side2, launch_lattice_b(dj, dpre(6), p_lt[n], dpre(7), p_lx[n], n, lane->side2));
  }
  TRACE(KN_TCOUNT, launch_chunk_map_b(dj, dpre(0), n, p_cm[n], st));
  TRACE(KN_TEMIT, launch_walk_b(one, dj, dpre(1), n, p_walk[n], st));
  TRACE(KN_SCAN, launch_mscan(ds1, dpre(8), 2 * n, nt1, flags1, tickets, NONE, st));
  TRACE(KN_TEMIT, launch_scatter_b(dj, dpre(2), n, p_sc[n], st));
  int nrk = 0;
  TRACE(KN_RANK, nrk = launch_rank_b(one, dj, dpre(3), n, p_rk[n], bp, st, fork ? lane->side : nullptr, lane->fork,
                                     lane->join));
  if (nrk < 0) kerr = 1;
  TRACE(KN_SORT, launch_sort_b(one, dj, dpre(10), n, p_sw[n], st));
  TRACE(KN_CUTCELLS, launch_cutcells_b(one, dj, n, bp, opt.cut_blocks_per_sm, st));
  TRACE(KN_SCAN, launch_mscan(ds2, dpre(9), n2, nt2, flags2, tickets + 1, NONE, st));
  // Tier-G beside the emission: both read the scans and the records, and
  // write disjoint parts of the output
  cudaStream_t gst = st;
  if (fork) {
    if (cudaEventRecord(lane->fork, st) != cudaSuccess || cudaStreamWaitEvent(lane->side, lane->fork, 0) != cudaSuccess)
      kerr = 1;
    gst = lane->side;
  }
  int ntg = 0;
  TRACE_ON(KN_TIERG, gst,
           ntg = launch_tierg_b(one, dj, dpre(5), n, p_go[n], bp, opt.tierg_blocks_per_sm, gst,
                                fork ? lane->side2 : nullptr, lane->order, lane->warp));
  if (ntg < 0) kerr = 1;
  if (fork && cudaEventRecord(lane->join, lane->side) != cudaSuccess) kerr = 1;
  TRACE(KN_EMIT, launch_emit_b(one, dj, dpre(4), n, p_so[n], st));
  if (!fork) TRACE(KN_XY, launch_lattice_b(dj, dpre(6), p_lt[n], dpre(7), p_lx[n], n, st));
  if (fork && cudaStreamWaitEvent(st, lane->join, 0) != cudaSuccess) kerr = 1;
  launch_status_b(dj, n, bp, st);
  if (opt.graph) {
    lane->capturing = false;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (ce != cudaSuccess || kerr) {
      if (graph) cudaGraphDestroy(graph);
      return bail(fail(SBMT_ECUDA, "graph capture: %s", cudaGetErrorString(ce)));
    }
    bool ok = false;
    if (lane->gexec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(lane->gexec, graph, &info) == cudaSuccess;
      if (!ok) cudaGetLastError(), cudaGraphExecDestroy(lane->gexec), lane->gexec = nullptr;
    }
    if (!ok && cudaGraphInstantiate(&lane->gexec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      lane->gexec = nullptr;
      return bail(fail(SBMT_ECUDA, "graph instantiation"));
    }
    cudaGraphDestroy(graph);
    CK(cudaGraphLaunch(lane->gexec, st));
  }
  if (kerr) return bail(fail(SBMT_ECUDA, "stream events"));
  CK(cudaGetLastError());
  arena_end(lane);
  std::lock_guard<std::mutex> lk(ctx->reg);
  Shared* dsh = new Shared();
  dsh->ev = pool_event(ctx);
  if (!dsh->ev || cudaEventRecord(dsh->ev, st) != cudaSuccess) {
    if (dsh->ev) ctx->ev_pool.push_back(dsh->ev);
    delete dsh;
    for (MeshRec* m : M) destroy_mesh(ctx, m, st);
    return fail(SBMT_ECUDA, "event record");
  }
  dsh->refs = n;
  for (int k = 0; k < n; ++k) {
    MeshRec* m = M[k];
    m->done_sh = dsh, m->done = dsh->ev;
    m->id = ctx->next++;
    ctx->meshes[m->id] = m;
    out[k] = m->id;
  }
  return SBMT_OK;
}

// ---------------------------------------------------------------------------
// Tuning of the batched path.  A batch's size class is its image count,
// total pixels (both log2) and largest grid edge h (log2, rounded).  For a
// class, mesh_autotune times the path under candidate launch parameters
// (persistent blocks per SM of the cut-cell and Tier-G kernels, Tier-G on
// side streams or not, the emission phase as a CUDA graph or not) by
// coordinate descent from the defaults, keeps the fastest and appends it to
// the tuning file (SBMT_TUNE_FILE, else $HOME/.cache/sbmt_tune.txt), which
// later contexts read.  Meshes are identical under every choice: only
// launch shapes and stream placement change.
// ---------------------------------------------------------------------------
std::string size_class(const sbmt_image* imgs, int n, const sbmt_params* prs, int nprs) {
  u64 px = 0;
  double hmax = 0;
  for (int k = 0; k < n; ++k) {
    const sbmt_params& pr = prs[nprs == 1 ? 0 : k];
    px += (u64)imgs[k].width * (u64)imgs[k].height;
    hmax = std::max(hmax, (double)pr.h_num / (double)std::max(1, pr.h_den));
  }
  auto lg = [](u64 v) {
    int l = 0;
    while (v > 1) v >>= 1, ++l;
    return l;
  };
  char buf[64];
  std::snprintf(buf, sizeof buf, "n%d_p%d_h%d", lg((u64)std::max(n, 1)), lg(std::max<u64>(px, 1)),
                (int)std::lround(std::log2(std::max(hmax, 1e-9))));
  return buf;
}

std::string tune_path() {
  if (const char* e = std::getenv("SBMT_TUNE_FILE")) return e;
  const char* home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/sbmt_tune.txt";
}

void tune_load(sbmt_ctx* ctx) {
  if (ctx->tuned_loaded) return;
  ctx->tuned_loaded = true;
  FILE* f = std::fopen(tune_path().c_str(), "r");
  if (!f) return;
  char key[64];
  Tune t;
  while (std::fscanf(f, "%63s %d %d %d %d", key, &t.cut_blocks_per_sm, &t.tierg_blocks_per_sm, &t.fork, &t.graph) ==
         5) {
    const bool ok = t.cut_blocks_per_sm >= 1 && t.cut_blocks_per_sm <= 16 && t.tierg_blocks_per_sm >= 1 &&
                    t.tierg_blocks_per_sm <= 32 && (t.fork == 0 || t.fork == 1) && (t.graph == 0 || t.graph == 1);
    if (ok) ctx->tuned[key] = t;  // later lines win
  }
  std::fclose(f);
}

void tune_save(const std::string& key, const Tune& t) {
  const std::string path = tune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) {
    // the cache directory, made when missing (one level)
    mkdir(path.substr(0, slash).c_str(), 0755);
  }
  if (FILE* f = std::fopen(path.c_str(), "a")) {
    std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), t.cut_blocks_per_sm, t.tierg_blocks_per_sm, t.fork, t.graph);
    std::fclose(f);
  }
}

// launch parameters for a batch: the tuned ones of its size class, else the
// context's defaults; callers hold ctx->mu
Tune tune_for(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* prs, int nprs) {
  tune_load(ctx);
  auto it = ctx->tuned.find(size_class(imgs, n, prs, nprs));
  return it != ctx->tuned.end() ? it->second : ctx->tune;
}

RunOpts opts_of(const Tune& t) {
  RunOpts o;
  o.fork = t.fork != 0, o.graph = t.graph != 0;
  o.cut_blocks_per_sm = t.cut_blocks_per_sm, o.tierg_blocks_per_sm = t.tierg_blocks_per_sm;
  return o;
}

// Alg. 3's thresholds in pixels: a, b, c are relative to the reference edge
// sqrt(0.45) px, so each is scaled by h / sqrt(0.45); they must lie in the
// admissible range b < a/2, c < a/sqrt2, and a < h/2
int pre_thresholds(const sbmt_params* pr, double* A, double* B, double* C) {
  const double h = (double)pr->h_num / (double)pr->h_den;
  const double s = h / std::sqrt(0.45);
  *A = pr->a * s, *B = pr->b * s, *C = pr->c * s;
  if (!(*B < *A / 2 && *C < *A / std::sqrt(2.0) && *A < h / 2 && *A > 0 && *B >= 0 && *C >= 0))
    return fail(SBMT_EINVAL, "thresholds (%g, %g, %g) outside the admissible range", pr->a, pr->b, pr->c);
  return SBMT_OK;
}

// the preprocessed mesh of one image (Alg. 3), enqueued on one lane
// base_only: the unmoved base mesh (no thresholds: nothing snaps, moves or
// splits), for the general path
int pre_one(sbmt_ctx* ctx, Lane* lane, const sbmt_image* img, const sbmt_params* pr, sbmt_mesh* out,
            bool base_only = false) {
  int rc = check_params(img, pr, !base_only, base_only);
  if (rc) return rc;
  double A = 0.0, B = 0.0, C = 0.0;
  if (!base_only && (rc = pre_thresholds(pr, &A, &B, &C))) return rc;
  cudaStream_t st = lane->stream;
  CK(cudaSetDevice(ctx->device));
  GridP g{};
  g.W = img->width, g.H = img->height;
  g.p = pr->h_num, g.q = pr->h_den, g.S = 6 * g.q;
  g.ox = 3 * g.q * (i64)pr->origin2x, g.oy = 3 * g.q * (i64)pr->origin2y;
  const Tables* tbp;
  const i64* dt;
  if ((rc = get_tables(ctx, lane, g, &tbp, &dt))) return rc;
  const Tables& tb = *tbp;
  if (tb.ncells >= (1ll << 31) || 3 * tb.nverts >= (1ll << 31))
    return fail(SBMT_EINVAL, "mesh too large (%lld cells)", (long long)tb.ncells);
  MeshRec* m = new MeshRec();
  m->W = g.W, m->H = g.H, m->pre = true;
  std::vector<void*> tmp;
  arena_begin(lane);
  auto bail = [&](int code) {
    free_list(st, tmp);
    arena_end(lane);
    std::lock_guard<std::mutex> lk(ctx->reg);
    destroy_mesh(ctx, m, st);
    return code;
  };
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    m->h_info = pinned_slot(ctx);
  }
  if (!m->h_info) return bail(fail(SBMT_ENOMEM, "pinned info"));
  const unsigned char* dimg;
  i64 pitch;
  if (img->on_device) {
    dimg = (const unsigned char*)img->data;
    pitch = img->pitch_bytes;
  } else {
    unsigned char* d;
    pitch = (i64)img->width * img->dtype;
    if ((rc = aalloc(lane, &d, (size_t)pitch * img->height))) return bail(rc);
    if (cudaMemcpy2DAsync(d, pitch, img->data, img->pitch_bytes, pitch, img->height, cudaMemcpyHostToDevice, st))
      return bail(fail(SBMT_ECUDA, "image upload"));
    dimg = d;
  }
  const i64 nrows = (i64)tb.clo.size(), nvr = (i64)tb.vlo.size();
  g.j0 = (int)tb.j0, g.nrows = (int)nrows, g.vj0 = (int)tb.vj0, g.nvrows = (int)nvr;
  g.clo = dt, g.chi = dt + nrows, g.cbase = dt + 2 * nrows;
  g.vlo = dt + 3 * nrows, g.vhi = dt + 3 * nrows + nvr, g.vbase = dt + 3 * nrows + 2 * nvr;
  g.lrow = (const int*)(dt + 3 * nrows + 3 * nvr);
  g.ncells = tb.ncells, g.nverts = tb.nverts;
  // counters: the PSLG vertex count (u64), then the six status words
  u32* zero;
  if ((rc = aalloc(lane, &zero, 16))) return bail(rc);
  CK(cudaMemsetAsync(zero, 0, 16 * sizeof(u32), st));
  unsigned long long* cnt64 = (unsigned long long*)zero;
  const int W = g.W, H = g.H;
  const int wpr = (W + 1 + 31) / 32, wpc = (H + 1 + 31) / 32;
  u32 *vrow, *vcol;
  if ((rc = aalloc(lane, &vrow, (size_t)wpr * (H + 1)))) return bail(rc);
  if ((rc = aalloc(lane, &vcol, (size_t)wpc * (W + 1)))) return bail(rc);
  TRACE(KN_CORNER, launch_corner_bits(dimg, pitch, img->dtype, W, H, vrow, wpr, vcol, wpc, cnt64, st));
  unsigned long long h64 = 0;
  CK(cudaMemcpyAsync(&h64, cnt64, sizeof h64, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const u64 NP = h64, V = (u64)tb.nverts, NCELL = (u64)tb.ncells;
  if (V + NP >= (1ull << 31) || NCELL + 2 * NP >= (1ull << 31))
    return bail(fail(SBMT_EINVAL, "mesh too large (%llu cells)", (unsigned long long)NCELL));
  // x of lattice vertex v(i, j) is indexed by m = 2i + j
  i64 m_lo = 0, m_hi = -1;
  for (i64 r = 0; r < nvr; ++r) {
    const i64 a = 2 * tb.vlo[r] + tb.vj0 + r, b = 2 * tb.vhi[r] + tb.vj0 + r;
    if (r == 0 || a < m_lo) m_lo = a;
    if (r == 0 || b > m_hi) m_hi = b;
  }
  const u64 nm = (u64)std::max<i64>(1, m_hi - m_lo + 1);
  const u64 nw = (u64)wpr * (H + 1), nsw = (NCELL + 31) / 32;
  PreArgs a{};
  a.g = g, a.img = dimg, a.pitch = pitch, a.dtype = img->dtype, a.vrow = vrow, a.wpr = wpr, a.np = (u32)NP;
  a.m0 = m_lo, a.nm = (i64)nm;
  u32 *wpop, *wscan, *scr;
  const size_t scr_words =
      std::max({scan_scratch_words((u32)nw), scan_scratch_words((u32)NP), scan_scratch_words((u32)nsw)}) + 1;
  if ((rc = aalloc(lane, &a.tab, nm)) || (rc = aalloc(lane, &a.tabf, nm)) ||
      (rc = aalloc(lane, &a.prow, 2 * (size_t)nrows)) || (rc = aalloc(lane, &a.xyf, V)) ||
      (rc = aalloc(lane, &wpop, nw)) || (rc = aalloc(lane, &wscan, nw + 1)) ||
      (rc = aalloc(lane, &a.plist, std::max<u64>(NP, 1))) || (rc = aalloc(lane, &a.appl, std::max<u64>(NP, 1))) ||
      (rc = aalloc(lane, &a.ascan, NP + 1)) || (rc = aalloc(lane, &a.sbit, nsw + 1)) ||
      (rc = aalloc(lane, &a.spop, nsw + 1)) || (rc = aalloc(lane, &a.wpre, nsw + 1)) ||
      (rc = aalloc(lane, &scr, scr_words)) || (rc = aalloc(lane, &a.ytab, (size_t)nvr)) ||
      (rc = aalloc(lane, &a.ytabf, (size_t)nvr)) || (rc = aalloc(lane, &a.vq, std::max<u64>(V, 1))) ||
      (rc = aalloc(lane, &a.vqn, (size_t)nvr)) || (rc = aalloc(lane, &a.rq, std::max<u64>(V, 1))))
    return bail(rc);
  char* candb;
  if ((rc = aalloc(lane, &candb, pre_cand_bytes((u32)NP)))) return bail(rc);
  a.cand = (PreCand*)candb;
  a.cnt = zero + 8;
  // thresholds and their float screens.  A float copy of a coordinate is
  // within 2^-24 of its magnitude (at most M) of the double; a distance is
  // 1-Lipschitz in the points, and its float evaluation adds a few 2^-24 of
  // the local lengths (at most 2h + a + b): dband bounds the difference
  // between a float distance and the double one, twice over
  const double h = (double)g.p / (double)g.q;
  const double M = std::max(W, H) + h + 2 + std::abs(pr->origin2x) / 2 + std::abs(pr->origin2y) / 2;
  const double dband = std::ldexp(M + 1, -21) + std::ldexp(2 * h + A + B + 1, -19);
  const double marg = dband + 1.0 / 256.0;
  auto lo2 = [&](double r) { return r > dband ? (float)((r - dband) * (r - dband)) : -1.0f; };
  auto hi2 = [&](double r) { return (float)((r + dband) * (r + dband)); };
  a.dband = (float)dband, a.a_lo2 = lo2(A), a.a_hi2 = hi2(A), a.b_lo2 = lo2(B), a.b_hi2 = hi2(B), a.c_hi2 = hi2(C);
  a.A = A, a.B2 = B * B, a.C = C;
  a.ascr = (float)(A + marg), a.cscr = (float)(C + marg), a.bscr = (float)(B + marg);
  a.bscr2 = (float)((B + marg) * (B + marg));
  a.reach = (float)(A + B + marg);
  a.oxf = (float)(pr->origin2x / 2), a.oyf = (float)(pr->origin2y / 2);
  a.hf = (float)h, a.rowh = (float)(h * std::sqrt(3.0) / 2.0);
  // outputs: at most one inserted vertex and two extra triangles per point
  const u64 nxy = V + NP, ntr = NCELL + 2 * NP;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_tri = up(16 * nxy), off_lab = up(off_tri + 12 * ntr), off_code = up(off_lab + 2 * ntr);
  const size_t off_st = up(off_code + 2 * ntr), off_sn = up(off_st + V), off_el = up(off_sn + 4 * V);
  const size_t total = off_el + 12 * std::max<u64>(NP, 1) + 256;
  m->bytes = total;
  if (cudaMallocAsync(&m->out_block, total, st) != cudaSuccess)
    return bail(fail(SBMT_ENOMEM, "output allocation of %zu bytes", total));
  char* ob = (char*)m->out_block;
  m->xy = (double*)ob, m->tri = (int*)(ob + off_tri);
  m->label = (unsigned short*)(ob + off_lab), m->code = (unsigned short*)(ob + off_code);
  m->pstatus = (unsigned char*)(ob + off_st), m->psnap = (int*)(ob + off_sn), m->pelim = (int*)(ob + off_el);
  a.xy = m->xy, a.tri = m->tri, a.label = m->label, a.code = m->code;
  a.status = m->pstatus, a.snap = m->psnap, a.elim = m->pelim;
  m->nv = (int64_t)V, m->nt = (int64_t)NCELL, m->ncells = (int64_t)NCELL, m->nvg = (int64_t)V;
  m->thr[0] = A, m->thr[1] = B, m->thr[2] = C, m->npts = (int64_t)NP;
  int nk = 0;
  TRACE(KN_PRE, nk = launch_preprocess(a, nw, wpop, wscan, scr, st));
  if (nk < 0) return bail(fail(SBMT_ECUDA, "preprocess launch"));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(m->h_info, a.cnt, 6 * sizeof(u32), cudaMemcpyDeviceToHost, st));
  free_list(st, tmp);
  arena_end(lane);
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    m->done = pool_event(ctx);
    m->own_done = true;
  }
  if (!m->done) return bail(fail(SBMT_ECUDA, "event create"));
  CK(cudaEventRecord(m->done, st));
  std::lock_guard<std::mutex> lk(ctx->reg);
  m->id = ctx->next++;
  ctx->meshes[m->id] = m;
  *out = m->id;
  return SBMT_OK;
}

// a preprocessed mesh's vertex and triangle counts, once its work is done
int settle(MeshRec* m) {
  if (!m->pre || m->settled) return SBMT_OK;
  CK(cudaEventSynchronize(m->done));
  m->nv = m->nvg + (int64_t)m->h_info[1];
  m->nt = m->ncells + (int64_t)m->h_info[2];
  m->settled = true;
  return SBMT_OK;
}

// Region III: Alg. 2 on the counter-clockwise mesh (txy, ttri) against the
// boundary of the device image; registers the result in *out.  One host
// synchronisation (the output sizes), then the emission.
int r3_one(sbmt_ctx* ctx, Lane* lane, const unsigned char* dimg, i64 pitch, int dtype, int W, int H,
           const double* txy, const int* ttri, i64 nv, i64 nt, sbmt_mesh* out) {
  if (nv < 3 || nt < 1 || nv >= (1ll << 31) || 3 * nt >= (1ll << 31))
    return fail(SBMT_EINVAL, "mesh of %lld vertices and %lld cells", (long long)nv, (long long)nt);
  cudaStream_t st = lane->stream;
  MeshRec* m = new MeshRec();
  m->W = W, m->H = H, m->r3 = true;
  std::vector<void*> tmp;
  arena_begin(lane);
  auto bail = [&](int code) {
    free_list(st, tmp);
    arena_end(lane);
    std::lock_guard<std::mutex> lk(ctx->reg);
    destroy_mesh(ctx, m, st);
    return code;
  };
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    m->h_info = pinned_slot(ctx);
  }
  if (!m->h_info) return bail(fail(SBMT_ENOMEM, "pinned info"));
  int rc;
  R3Args a{};
  a.img = dimg, a.pitch = pitch, a.dtype = dtype, a.W = W, a.H = H;
  a.txy = txy, a.ttri = ttri, a.nv = (u32)nv, a.nt = (u64)nt;
  u32 *cnt, *scr;
  const size_t scr_words = std::max(scan_scratch_words((u32)nv), scan_scratch_words((u32)nt)) + 1;
  if ((rc = aalloc(lane, &a.deg, nv)) || (rc = aalloc(lane, &a.vptr, nv + 1)) || (rc = aalloc(lane, &a.inc, 3 * nt)) ||
      (rc = aalloc(lane, &a.ntri, nt)) || (rc = aalloc(lane, &a.nown, nt)) || (rc = aalloc(lane, &a.nin, nt)) ||
      (rc = aalloc(lane, &a.own3, nt)) || (rc = aalloc(lane, &a.toff, nt + 1)) || (rc = aalloc(lane, &a.eoff, nt + 1)) ||
      (rc = aalloc(lane, &a.ioff, nt + 1)) || (rc = aalloc(lane, &a.glist, nt)) || (rc = aalloc(lane, &cnt, 8)) ||
      (rc = aalloc(lane, &scr, scr_words)) || (rc = aalloc(lane, &a.ulab, nt)) ||
      (rc = aalloc(lane, &a.cmark, (nt + 31) / 32)) || (rc = aalloc(lane, &a.cand, nt)) ||
      (rc = aalloc(lane, &a.cutl, nt)))
    return bail(rc);
  a.err = cnt, a.ncut = cnt + 1, a.ng = cnt + 2, a.ngtri = cnt + 3, a.ncand = cnt + 4, a.ngsmall = cnt + 5;
  CK(cudaMemsetAsync(a.deg, 0, sizeof(u32) * (size_t)nv, st));
  CK(cudaMemsetAsync(cnt, 0, 8 * sizeof(u32), st));
  int nk = 0;
  TRACE(KN_R3, nk = launch_r3_adjacency(a, scr, st));
  TRACE(KN_R3, nk = launch_r3_count(a, st));
  TRACE(KN_R3, nk = launch_scan(a.ntri, 1, a.toff, (u32)nt, scr, st));
  TRACE(KN_R3, nk = launch_scan(a.nown, 1, a.eoff, (u32)nt, scr, st));
  TRACE(KN_R3, nk = launch_scan(a.nin, 1, a.ioff, (u32)nt, scr, st));
  (void)nk;
  CK(cudaGetLastError());
  u32* h = m->h_info;
  CK(cudaMemcpyAsync(h + 4, a.toff + nt, sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + 5, a.eoff + nt, sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + 6, a.ioff + nt, sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h, cnt, sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h[0]) {
    const u32 e = h[0];
    return bail(fail((e & R3_CAPACITY) ? SBMT_ECAPACITY : SBMT_EINTERNAL,
                     "retriangulation: %s (error bits 0x%x)",
                     (e & R3_CAPACITY) ? "a cell over the per-cell limits (16 events per edge, 16 boundary "
                                         "vertices, 48 nodes)"
                                       : "an inconsistent mesh (a cell not counter-clockwise, an edge in three cells)",
                     e));
  }
  const u64 NT = h[4], NE = h[5], NI = h[6], NV = (u64)nv + NE + NI;
  if (NV >= (1ull << 31) || NT >= (1ull << 31)) return bail(fail(SBMT_EINVAL, "mesh too large"));
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_tri = up(16 * NV), off_lab = up(off_tri + 12 * NT), off_code = up(off_lab + 2 * NT);
  const size_t total = off_code + 2 * NT + 256;
  m->bytes = total;
  if (cudaMallocAsync(&m->out_block, total, st) != cudaSuccess)
    return bail(fail(SBMT_ENOMEM, "output allocation of %zu bytes", total));
  char* ob = (char*)m->out_block;
  m->xy = (double*)ob, m->tri = (int*)(ob + off_tri);
  m->label = (unsigned short*)(ob + off_lab), m->code = (unsigned short*)(ob + off_code);
  CK(cudaMemcpyAsync(m->xy, txy, 16 * (size_t)nv, cudaMemcpyDeviceToDevice, st));
  a.ne_total = (u32)NE;
  a.xy = m->xy, a.tri = m->tri, a.label = m->label, a.code = m->code;
  TRACE(KN_R3, nk = launch_r3_emit(a, st));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h, cnt, 6 * sizeof(u32), cudaMemcpyDeviceToHost, st));
  free_list(st, tmp);
  arena_end(lane);
  m->nv = (int64_t)NV, m->nt = (int64_t)NT, m->ncells = nt, m->nvg = nv;
  m->ne_total = (int64_t)NE, m->nc_total = (int64_t)NI;
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    m->done = pool_event(ctx);
    m->own_done = true;
  }
  if (!m->done) return bail(fail(SBMT_ECUDA, "event create"));
  CK(cudaEventRecord(m->done, st));
  std::lock_guard<std::mutex> lk(ctx->reg);
  m->id = ctx->next++;
  ctx->meshes[m->id] = m;
  *out = m->id;
  return SBMT_OK;
}

// the image on the device for a call that reads it twice: a device image as
// it is, a host image uploaded into *owned (freed by the caller on st)
int device_image(const sbmt_image* img, cudaStream_t st, sbmt_image* dev, void** owned) {
  *dev = *img;
  *owned = nullptr;
  if (img->on_device) return SBMT_OK;
  const size_t pitch = (size_t)img->width * img->dtype;
  if (cudaMallocAsync(owned, pitch * img->height, st) != cudaSuccess) return fail(SBMT_ENOMEM, "image upload");
  if (cudaMemcpy2DAsync(*owned, pitch, img->data, img->pitch_bytes, pitch, img->height, cudaMemcpyHostToDevice, st))
    return fail(SBMT_ECUDA, "image upload");
  dev->data = *owned, dev->pitch_bytes = (int64_t)pitch, dev->on_device = 1;
  return SBMT_OK;
}

// Alg. 3 in full: Regions I-II (mesh_preprocess), the barrier, Region III.
// base_only: the general path of a degenerate origin -- the unmoved base
// mesh, then Region III (Alg. 2 cell by cell, with Alg. 1's vertex-on-segment
// and overlap incidences that a lattice on the pixel lines creates)
int preprocess_mesh(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* pr, sbmt_mesh* out,
                    bool base_only = false) {
  int rc = check_params(img, pr, !base_only, base_only);
  if (rc) return rc;
  Lane* lane = &ctx->main;
  cudaStream_t st = lane->stream;
  CK(cudaSetDevice(ctx->device));
  sbmt_image dev;
  void* owned = nullptr;
  if ((rc = device_image(img, st, &dev, &owned))) {
    if (owned) cudaFreeAsync(owned, st);
    return rc;
  }
  sbmt_mesh tid = 0;
  rc = pre_one(ctx, lane, &dev, pr, &tid, base_only);
  MeshRec* tm = nullptr;
  if (rc == SBMT_OK) {
    std::lock_guard<std::mutex> lk(ctx->reg);
    tm = ctx->meshes[tid];
  }
  if (rc == SBMT_OK && (rc = settle(tm)) == SBMT_OK && tm->h_info[0])
    rc = fail(SBMT_EINTERNAL, "preprocessing reported error bits 0x%x", tm->h_info[0]);
  if (rc == SBMT_OK)
    rc = r3_one(ctx, lane, (const unsigned char*)dev.data, dev.pitch_bytes, dev.dtype, dev.width, dev.height, tm->xy,
                tm->tri, tm->nv, tm->nt, out);
  if (tm) {
    std::lock_guard<std::mutex> lk(ctx->reg);
    ctx->meshes.erase(tid);
    destroy_mesh(ctx, tm, st);
  }
  if (owned) cudaFreeAsync(owned, st);
  return rc;
}

}  // namespace

extern "C" {

const char* sbmt_last_error(void) { return g_last_error.c_str(); }

int mesh_create(sbmt_ctx** out, int device, size_t pool_bytes, void* cuda_stream) {
  if (!out) return fail(SBMT_EINVAL, "null ctx pointer");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(SBMT_ECUDA, "no CUDA device");
  if (device < 0 || device >= n) return fail(SBMT_EINVAL, "device %d of %d", device, n);
  CK(cudaSetDevice(device));
  if (tierg_init()) return fail(SBMT_ECUDA, "kernel attributes");
  sbmt_ctx* ctx = new sbmt_ctx();
  ctx->device = device;
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return fail(SBMT_ECUDA, "stream create");
    }
    ctx->main.own_stream = true;
  }
  ctx->main.stream = ctx->stream;
  // keep freed stream-ordered memory cached for the next call
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    u64 thr = pool_bytes ? (u64)pool_bytes : ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  *out = ctx;
  return SBMT_OK;
}

int mesh_bitmap(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* params, sbmt_mesh* out) {
  if (!ctx || !out || !params) return fail(SBMT_EINVAL, "null ctx, params or out");
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (params->mode == SBMT_PREPROCESS) return preprocess_mesh(ctx, img, params, out);
  if (params->mode == SBMT_PLAIN && ((params->origin2x & 1) || (params->origin2y & 1)))
    return preprocess_mesh(ctx, img, params, out, true);
  RunOpts o = opts_of(tune_for(ctx, img, 1, params, 1));
  o.stall = (params->flags & SBMT_DEBUG_STALL_SCAN) != 0;
  return mesh_run(ctx, &ctx->main, img, 1, params, 1, out, o);
}

int mesh_preprocess(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* params, sbmt_mesh* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  std::lock_guard<std::mutex> lk(ctx->mu);
  return pre_one(ctx, &ctx->main, img, params, out);
}

int mesh_retriangulate(sbmt_ctx* ctx, const sbmt_image* img, sbmt_mesh base, sbmt_mesh* out) {
  if (!ctx || !out || !img || !img->data) return fail(SBMT_EINVAL, "null ctx, image or out");
  if (img->width < 1 || img->height < 1 || img->width > 32768 || img->height > 32768 ||
      (img->dtype != SBMT_U8 && img->dtype != SBMT_U16) || img->pitch_bytes < (int64_t)img->width * img->dtype)
    return fail(SBMT_EINVAL, "image");
  if (img->on_device && img->dtype == SBMT_U16 && ((img->pitch_bytes & 1) || ((uintptr_t)img->data & 1)))
    return fail(SBMT_EINVAL, "a device u16 image needs an even pitch and an even address");
  std::lock_guard<std::mutex> lk(ctx->mu);
  MeshRec* tm;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    auto it = ctx->meshes.find(base);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh %llu", (unsigned long long)base);
    tm = it->second;
  }
  if (tm->format != SBMT_EXPLICIT) return fail(SBMT_EINVAL, "the base mesh must be explicit");
  CK(cudaSetDevice(ctx->device));
  Lane* lane = &ctx->main;
  cudaStream_t st = lane->stream;
  CK(cudaStreamWaitEvent(st, tm->done, 0));
  if (int rc = settle(tm)) return rc;
  sbmt_image dev;
  void* owned = nullptr;
  int rc = device_image(img, st, &dev, &owned);
  if (rc == SBMT_OK)
    rc = r3_one(ctx, lane, (const unsigned char*)dev.data, dev.pitch_bytes, dev.dtype, dev.width, dev.height, tm->xy,
                tm->tri, tm->nv, tm->nt, out);
  if (owned) cudaFreeAsync(owned, st);
  return rc;
}

int mesh_import(sbmt_ctx* ctx, const double* xy, int64_t n_vertices, const int32_t* tri, int64_t n_triangles,
                sbmt_mesh* out) {
  // the arrays first (host logic only), then the context
  if (!xy || !tri) return fail(SBMT_EINVAL, "null xy or tri");
  if (n_vertices < 3 || n_triangles < 1 || n_vertices >= (1ll << 31) || 3 * n_triangles >= (1ll << 31))
    return fail(SBMT_EINVAL, "mesh of %lld vertices and %lld triangles", (long long)n_vertices,
                (long long)n_triangles);
  constexpr double kMaxCoord = 16777216.0;  // 2^24 px: every pixel-line index fits an int
  for (int64_t i = 0; i < 2 * n_vertices; ++i)
    if (!(std::fabs(xy[i]) <= kMaxCoord))
      return fail(SBMT_EINVAL, "vertex %lld: coordinate not finite or beyond 2^24 px", (long long)(i / 2));
  for (int64_t t = 0; t < n_triangles; ++t) {
    const int32_t u = tri[3 * t], v = tri[3 * t + 1], w = tri[3 * t + 2];
    if (u < 0 || v < 0 || w < 0 || u >= n_vertices || v >= n_vertices || w >= n_vertices)
      return fail(SBMT_EINVAL, "triangle %lld: vertex id out of range", (long long)t);
    if (u == v || v == w || w == u) return fail(SBMT_EINVAL, "triangle %lld: repeated vertex id", (long long)t);
  }
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->main.stream;
  MeshRec* m = new MeshRec();
  auto bail = [&](int code) {
    std::lock_guard<std::mutex> rl(ctx->reg);
    destroy_mesh(ctx, m, st);
    return code;
  };
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    m->h_info = pinned_slot(ctx);
  }
  if (!m->h_info) return bail(fail(SBMT_ENOMEM, "pinned info"));
  std::memset(m->h_info, 0, 8 * sizeof(u32));
  const size_t NV = (size_t)n_vertices, NT = (size_t)n_triangles;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_tri = up(16 * NV), off_lab = up(off_tri + 12 * NT), off_code = up(off_lab + 2 * NT);
  const size_t total = off_code + 2 * NT + 256;
  if (cudaMallocAsync(&m->out_block, total, st) != cudaSuccess)
    return bail(fail(SBMT_ENOMEM, "mesh allocation of %zu bytes", total));
  char* ob = (char*)m->out_block;
  m->xy = (double*)ob, m->tri = (int*)(ob + off_tri);
  m->label = (unsigned short*)(ob + off_lab), m->code = (unsigned short*)(ob + off_code);
  if (cudaMemcpyAsync(m->xy, xy, 16 * NV, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(m->tri, tri, 12 * NT, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(m->label, 0xFF, 2 * NT, st) != cudaSuccess || cudaMemsetAsync(m->code, 0, 2 * NT, st) != cudaSuccess)
    return bail(fail(SBMT_ECUDA, "mesh upload"));
  m->bytes = total;
  m->nv = m->nvg = (int64_t)NV, m->nt = m->ncells = (int64_t)NT;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    m->done = pool_event(ctx);
    m->own_done = true;
  }
  if (!m->done) return bail(fail(SBMT_ECUDA, "event create"));
  CK(cudaEventRecord(m->done, st));
  // the caller's arrays may be pinned (a truly asynchronous copy): done
  // with them before returning
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(SBMT_ECUDA, "mesh upload"));
  std::lock_guard<std::mutex> rl(ctx->reg);
  m->id = ctx->next++;
  ctx->meshes[m->id] = m;
  *out = m->id;
  return SBMT_OK;
}

int mesh_preprocess_info(sbmt_ctx* ctx, sbmt_mesh mesh, sbmt_pre_info* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  MeshRec* m;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->meshes.find(mesh);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh %llu", (unsigned long long)mesh);
    m = it->second;
  }
  if (!m->pre) return fail(SBMT_EINVAL, "not a preprocessed mesh");
  if (int rc = settle(m)) return rc;
  std::memset(out, 0, sizeof *out);
  out->n_lattice_vertices = m->nvg, out->n_points = m->npts;
  out->n_snapped = m->h_info[3], out->n_repelled = m->h_info[4], out->n_candidate_points = m->h_info[5];
  out->n_eliminated = m->h_info[1], out->n_split_cells = m->h_info[2];
  out->a_px = m->thr[0], out->b_px = m->thr[1], out->c_px = m->thr[2];
  out->status = m->pstatus, out->snap = m->psnap, out->elim = m->pelim;
  return SBMT_OK;
}

int mesh_batch(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
               sbmt_mesh* out) {
  if (!ctx || !imgs || !params || !out || n < 0 || (n_params != 1 && n_params != n))
    return fail(SBMT_EINVAL, "bad batch arguments");
  std::lock_guard<std::mutex> lk(ctx->mu);
  RunOpts o = opts_of(tune_for(ctx, imgs, n, params, n_params));
  o.stall = n > 0 && (params[0].flags & SBMT_DEBUG_STALL_SCAN) != 0;
  return mesh_run(ctx, &ctx->main, imgs, n, params, n_params, out, o);
}

int mesh_autotune(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                  int repeats) {
  if (!ctx || !imgs || !params || n < 1 || (n_params != 1 && n_params != n) || repeats < 1)
    return fail(SBMT_EINVAL, "bad autotune arguments");
  std::lock_guard<std::mutex> lk(ctx->mu);
  tune_load(ctx);
  std::vector<sbmt_mesh> ids(n);
  // the wall time of the call and its device work, best of `repeats`
  auto time_of = [&](const Tune& t, double* best) -> int {
    *best = 1e30;
    for (int r = 0; r <= repeats; ++r) {  // the first run warms the tables and the arena
      const auto t0 = std::chrono::steady_clock::now();
      int rc = mesh_run(ctx, &ctx->main, imgs, n, params, n_params, ids.data(), opts_of(t));
      if (rc) return rc;
      if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail(SBMT_ECUDA, "autotune run");
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      {
        std::lock_guard<std::mutex> rl(ctx->reg);
        for (sbmt_mesh id : ids) {
          auto it = ctx->meshes.find(id);
          if (it != ctx->meshes.end()) destroy_mesh(ctx, it->second, ctx->stream), ctx->meshes.erase(it);
        }
      }
      if (r > 0) *best = std::min(*best, ms);
    }
    return SBMT_OK;
  };
  Tune cur = ctx->tune;
  double cur_ms;
  if (int rc = time_of(cur, &cur_ms)) return rc;
  const std::vector<int> cut_c = {4, 8, 12, 16}, tg_c = {8, 16, 24, 32};
  for (int pass = 0; pass < 2; ++pass) {
    for (int axis = 0; axis < 4; ++axis) {
      std::vector<Tune> cands;
      if (axis == 0)
        for (int v : cut_c) cands.push_back(cur), cands.back().cut_blocks_per_sm = v;
      if (axis == 1)
        for (int v : tg_c) cands.push_back(cur), cands.back().tierg_blocks_per_sm = v;
      if (axis == 2) cands.push_back(cur), cands.back().fork ^= 1;
      if (axis == 3) cands.push_back(cur), cands.back().graph ^= 1;
      for (const Tune& t : cands) {
        if (t.cut_blocks_per_sm == cur.cut_blocks_per_sm && t.tierg_blocks_per_sm == cur.tierg_blocks_per_sm &&
            t.fork == cur.fork && t.graph == cur.graph)
          continue;
        double ms;
        if (int rc = time_of(t, &ms)) return rc;
        if (ms < 0.97 * cur_ms) cur = t, cur_ms = ms;
      }
    }
  }
  const std::string key = size_class(imgs, n, params, n_params);
  ctx->tuned[key] = cur;
  tune_save(key, cur);
  return SBMT_OK;
}

int mesh_tuning(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                int32_t* out4) {
  if (!ctx || !imgs || !params || !out4 || n < 1 || (n_params != 1 && n_params != n))
    return fail(SBMT_EINVAL, "bad arguments");
  std::lock_guard<std::mutex> lk(ctx->mu);
  const Tune t = tune_for(ctx, imgs, n, params, n_params);
  out4[0] = t.cut_blocks_per_sm, out4[1] = t.tierg_blocks_per_sm, out4[2] = t.fork, out4[3] = t.graph;
  return SBMT_OK;
}

int mesh_set_tuning(sbmt_ctx* ctx, const sbmt_image* imgs, int n, const sbmt_params* params, int n_params,
                    const int32_t* in4) {
  if (!ctx || !imgs || !params || !in4 || n < 1 || (n_params != 1 && n_params != n))
    return fail(SBMT_EINVAL, "bad arguments");
  if (in4[0] < 1 || in4[0] > 16 || in4[1] < 1 || in4[1] > 32 || (in4[2] != 0 && in4[2] != 1) ||
      (in4[3] != 0 && in4[3] != 1))
    return fail(SBMT_EINVAL, "tuning values out of range");
  std::lock_guard<std::mutex> lk(ctx->mu);
  tune_load(ctx);
  Tune t;
  t.cut_blocks_per_sm = in4[0], t.tierg_blocks_per_sm = in4[1], t.fork = in4[2], t.graph = in4[3];
  ctx->tuned[size_class(imgs, n, params, n_params)] = t;
  return SBMT_OK;
}

int mesh_check(const sbmt_image* img, const sbmt_params* params) { return check_params(img, params); }

int mesh_footprint(sbmt_ctx* ctx, sbmt_mesh mesh, size_t* bytes) {
  if (!ctx || !bytes) return fail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->meshes.find(mesh);
  if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
  const MeshRec* m = it->second;
  size_t b = m->bytes;
  if (m->keep) b += (size_t)m->nseg * sizeof(Seg) + (size_t)m->ne * sizeof(Event) + 8 * ((size_t)m->nbc + 1) +
                    (size_t)(m->nseg_total + m->ne_total) * sizeof(CutRec);
  *bytes = b;
  return SBMT_OK;
}

int mesh_query(sbmt_ctx* ctx, sbmt_mesh mesh, int wait_ms, sbmt_mesh_view* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  MeshRec* m;
  {
    // the registry lock only: a query does not wait for another thread's
    // call in progress on the same context
    std::lock_guard<std::mutex> lk(ctx->reg);
    auto it = ctx->meshes.find(mesh);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh %llu", (unsigned long long)mesh);
    m = it->second;
  }
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    const cudaError_t q = cudaEventQuery(m->done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return fail(SBMT_ECUDA, "mesh work failed: %s", cudaGetErrorString(q));
    if (wait_ms == 0) return SBMT_EPENDING;
    if (wait_ms > 0 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(wait_ms))
      return SBMT_ETIMEDOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  int rc = settle(m);
  if (rc) return rc;
  std::memset(out, 0, sizeof *out);
  out->n_vertices = m->nv, out->n_triangles = m->nt, out->n_cells = m->ncells;
  if (m->r3) {
    // h_info: error bits, cut cells, Tier-G cells (all queued), Tier-G
    // triangles, candidates, Tier-G cells done by one thread
    out->n_cut_cells = m->h_info[1], out->n_tierG_cells = m->h_info[2];
    out->n_tierG_triangles = m->h_info[3];
    out->n_events = m->ne_total, out->n_inside_vertices = m->nc_total, out->n_lattice_vertices = m->nvg;
    out->xy = m->xy, out->tri = m->tri, out->label = m->label, out->code = m->code;
    out->format = SBMT_EXPLICIT;
    const u32 e = m->h_info[0];
    out->status = e == 0 ? SBMT_OK : (e & R3_CAPACITY) ? SBMT_ECAPACITY : SBMT_EINTERNAL;
    if (out->status) fail(out->status, "device reported error bits 0x%x", e);
    return out->status;
  }
  if (m->pre) {
    out->n_cut_cells = m->h_info[2], out->n_lattice_vertices = m->nvg;
    out->xy = m->xy, out->tri = m->tri, out->label = m->label, out->code = m->code;
    out->format = SBMT_EXPLICIT;
    out->status = m->h_info[0] == 0 ? SBMT_OK : SBMT_EINTERNAL;
    if (out->status) fail(out->status, "device reported error bits 0x%x", m->h_info[0]);
    return out->status;
  }
  out->n_cut_cells = m->h_info[1], out->n_tierG_cells = m->h_info[2];
  out->n_segments = m->nseg_total, out->n_events = m->ne_total, out->n_inside_vertices = m->nc_total;
  out->n_lattice_vertices = m->nvg, out->n_tierG_triangles = m->h_info[3];
  out->xy = m->xy, out->tri = m->tri, out->label = m->label, out->code = m->code;
  out->format = m->format;
  if (m->format == SBMT_COMPACT) {
    out->n_patch_triangles = (m->nt - m->ncells) + (int64_t)m->h_info[1];
    out->cell_label = m->cell_label, out->cell_code = m->cell_code;
    out->patch_cell = m->patch_cell, out->patch_off = m->patch_off;
  }
  const u32 e = m->h_info[0];
  out->status = e == 0 ? SBMT_OK : (e & ERR_CAPACITY) ? SBMT_ECAPACITY : SBMT_EINTERNAL;
  if (out->status) fail(out->status, "device reported error bits 0x%x", e);
  return out->status;
}

int mesh_release(sbmt_ctx* ctx, sbmt_mesh mesh) {
  if (!ctx) return fail(SBMT_EINVAL, "null ctx");
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::lock_guard<std::mutex> rl(ctx->reg);
  auto it = ctx->meshes.find(mesh);
  if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
  destroy_mesh(ctx, it->second, ctx->stream);
  ctx->meshes.erase(it);
  return SBMT_OK;
}

int mesh_destroy(sbmt_ctx* ctx) {
  if (!ctx) return fail(SBMT_EINVAL, "null ctx");
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::lock_guard<std::mutex> rl(ctx->reg);
    for (auto& kv : ctx->meshes) destroy_mesh(ctx, kv.second, ctx->stream);
    ctx->meshes.clear();
    cudaDeviceSynchronize();
    prof_collect(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (auto& kv : ctx->tables) {
      Shared* b = kv.second.block;
      if (--b->refs == 0) cudaFreeAsync(b->ptr, ctx->stream), delete b;
    }
    ctx->tables.clear();
    lane_release(&ctx->main);
    for (auto& slab : ctx->pinned_slabs) cudaFreeHost(slab.first);
  }
  delete ctx;
  return SBMT_OK;
}

int mesh_quality(sbmt_ctx* ctx, sbmt_mesh mesh, sbmt_quality* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  MeshRec* m;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    auto it = ctx->meshes.find(mesh);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
    m = it->second;
  }
  if (m->format != SBMT_EXPLICIT) return fail(SBMT_EINVAL, "quality needs the explicit format");
  if (int rc0 = settle(m)) return rc0;
  CK(cudaSetDevice(ctx->device));
  std::memset(out, 0, sizeof *out);
  const u64 T = (u64)m->nt;
  out->triangles = (int64_t)T;
  if (T == 0) return SBMT_OK;
  Lane* lane = &ctx->main;
  cudaStream_t st = lane->stream;
  CK(cudaStreamWaitEvent(st, m->done, 0));
  constexpr int NBLK = 152 * 8;
  arena_begin(lane);
  float* ar;
  unsigned long long* mm;
  double* part;
  u32* hist;
  int rc;
  if ((rc = aalloc(lane, &ar, T)) || (rc = aalloc(lane, &mm, 8)) || (rc = aalloc(lane, &part, 2 * NBLK)) ||
      (rc = aalloc(lane, &hist, 32 + 2 * 4096))) {
    arena_end(lane);
    return rc;
  }
  unsigned long long* cnt = mm + 3;
  u32* h0 = hist + 32;
  u32* h1 = h0 + 4096;
  const unsigned long long init[5] = {0x7FF0000000000000ull, 0x7FF0000000000000ull, 0ull, 0ull, 0ull};
  std::vector<double> hpart(2 * NBLK);
  unsigned long long hmm[5];
  u32 hh[32];
  CK(cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(hist, 0, 32 * sizeof(u32), st));
  launch_quality(m->xy, m->tri, T, ar, mm, cnt, part, NBLK, hist, st);
  CK(cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hpart.data(), part, hpart.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hh, hist, sizeof hh, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  auto dbl = [](unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
  };
  out->min_angle_deg = dbl(hmm[0]), out->min_area = dbl(hmm[1]), out->ar_max = dbl(hmm[2]);
  out->slivers = (int64_t)hmm[3], out->equilateral = (int64_t)hmm[4];
  double sa = 0.0, sa2 = 0.0;
  for (int b = 0; b < NBLK; ++b) sa += hpart[2 * b], sa2 += hpart[2 * b + 1];
  out->area_mean = sa / (double)T;
  out->area_var = std::max(0.0, sa2 / (double)T - out->area_mean * out->area_mean);
  for (int k = 0; k < 30; ++k) out->angle_hist[k] = hh[k];
  // nearest-rank percentiles: a radix select over the float bits in three
  // levels, both ranks at once
  u64 rank[2] = {(T + 1) / 2, (u64)std::ceil(0.95 * (double)T)};
  rank[1] = std::max<u64>(1, std::min<u64>(rank[1], T));
  u32 pre[2] = {0, 0};
  const int lo_of[3] = {20, 10, 0}, width_of[3] = {12, 10, 10};
  std::vector<u32> a0(4096), a1(4096);
  for (int lev = 0; lev < 3; ++lev) {
    const int lo = lo_of[lev], width = width_of[lev], nb = 1 << width;
    CK(cudaMemsetAsync(h0, 0, 2 * 4096 * sizeof(u32), st));
    launch_select_hist(ar, T, lo, width, pre[0], pre[1], lo + width, h0, h1, st);
    CK(cudaMemcpyAsync(a0.data(), h0, nb * sizeof(u32), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(a1.data(), h1, nb * sizeof(u32), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int r = 0; r < 2; ++r) {
      const std::vector<u32>& h = r == 0 ? a0 : a1;
      u64 cum = 0;
      int bin = nb - 1;
      for (int k = 0; k < nb; ++k) {
        if (cum + h[k] >= rank[r]) {
          bin = k;
          break;
        }
        cum += h[k];
      }
      rank[r] -= cum;
      pre[r] = (pre[r] << width) | (u32)bin;
    }
  }
  float f[2];
  std::memcpy(&f[0], &pre[0], 4);
  std::memcpy(&f[1], &pre[1], 4);
  out->ar_median = f[0], out->ar_p95 = f[1];
  arena_end(lane);
  return SBMT_OK;
}

int mesh_project(sbmt_ctx* ctx, sbmt_mesh mesh, const sbmt_image* field, float* tri_value, float* vertex_value) {
  if (!ctx || !field) return fail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  MeshRec* m;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    auto it = ctx->meshes.find(mesh);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
    m = it->second;
  }
  if (m->format != SBMT_EXPLICIT) return fail(SBMT_EINVAL, "projection needs the explicit format");
  if (int rc0 = settle(m)) return rc0;
  if (field->dtype != SBMT_F32 || field->width != m->W || field->height != m->H || !field->data)
    return fail(SBMT_EINVAL, "field must be a %dx%d SBMT_F32 image", m->W, m->H);
  if (field->pitch_bytes < 4 * (int64_t)field->width || (field->pitch_bytes & 3))
    return fail(SBMT_EINVAL, "field pitch");
  if ((u64)m->nt >= (1ull << 32)) return fail(SBMT_EINVAL, "mesh too large to project");
  if (!tri_value && !vertex_value) return SBMT_OK;
  CK(cudaSetDevice(ctx->device));
  Lane* lane = &ctx->main;
  cudaStream_t st = lane->stream;
  CK(cudaStreamWaitEvent(st, m->done, 0));
  arena_begin(lane);
  const float* f = (const float*)field->data;
  i64 pitch = field->pitch_bytes;
  if (!field->on_device) {
    float* d;
    int rc;
    pitch = 4 * (i64)field->width;
    if ((rc = aalloc(lane, &d, (size_t)field->width * field->height))) {
      arena_end(lane);
      return rc;
    }
    if (cudaMemcpy2DAsync(d, pitch, field->data, field->pitch_bytes, pitch, field->height, cudaMemcpyHostToDevice,
                          st) != cudaSuccess) {
      arena_end(lane);
      return fail(SBMT_ECUDA, "field upload");
    }
    f = d;
  }
  unsigned char* scratch = nullptr;
  if (tri_value) {
    int rc;
    if ((rc = aalloc(lane, &scratch, project_scratch_bytes((u64)m->nv)))) {
      arena_end(lane);
      return rc;
    }
  }
  launch_project(m->xy, m->tri, (u64)m->nt, (u64)m->nv, f, pitch, m->W, m->H, tri_value, vertex_value, scratch, st);
  const cudaError_t e = cudaGetLastError();
  arena_end(lane);
  if (e != cudaSuccess) return fail(SBMT_ECUDA, "projection launch: %s", cudaGetErrorString(e));
  // the mesh's completion now includes the projection (an event of its own:
  // a batch's meshes share their completion event)
  if (!m->own_done) {
    std::lock_guard<std::mutex> rl(ctx->reg);
    cudaEvent_t e = pool_event(ctx);
    if (!e) return fail(SBMT_ECUDA, "event create");
    m->done = e, m->own_done = true;
  }
  CK(cudaEventRecord(m->done, st));
  return SBMT_OK;
}

int mesh_heat(sbmt_ctx* ctx, sbmt_mesh mesh, const sbmt_heat_params* hp, double* u, double* peaks,
              int32_t* iterations) {
  if (!ctx || !hp || !u) return fail(SBMT_EINVAL, "null argument");
  if (hp->steps < 0 || !(hp->dt > 0) || !(hp->alpha >= 0) || !(hp->sigma > 0) || !(hp->tol > 0) ||
      hp->max_iterations < 1 || hp->label < 0 || hp->label > 0xFFFF)
    return fail(SBMT_EINVAL, "heat parameters");
  std::lock_guard<std::mutex> lk(ctx->mu);
  MeshRec* m;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    auto it = ctx->meshes.find(mesh);
    if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
    m = it->second;
  }
  if (m->format != SBMT_EXPLICIT) return fail(SBMT_EINVAL, "heat diffusion needs the explicit format");
  if (int rc0 = settle(m)) return rc0;
  if (m->nt >= (1ll << 32) || m->nv >= (1ll << 31)) return fail(SBMT_EINVAL, "mesh too large");
  CK(cudaSetDevice(ctx->device));
  Lane* lane = &ctx->main;
  cudaStream_t st = lane->stream;
  CK(cudaStreamWaitEvent(st, m->done, 0));
  arena_begin(lane);
  char* scratch;
  int rc = aalloc(lane, &scratch, heat_scratch_bytes((u64)m->nt, (u64)m->nv, hp->max_iterations));
  if (rc) {
    arena_end(lane);
    return rc;
  }
  int n = 0;
  TRACE(KN_HEAT, n = heat_solve(m->xy, m->tri, m->label, (u64)m->nt, (u64)m->nv, hp->label, hp->alpha, hp->dt,
                                hp->steps, hp->x0, hp->y0, hp->sigma, hp->amplitude, hp->tol, hp->max_iterations, u,
                                peaks, iterations, scratch, st));
  arena_end(lane);
  if (n == -2) return fail(SBMT_ETIMEDOUT, "a step did not reach the residual within %d iterations", hp->max_iterations);
  if (n < 0) return fail(SBMT_ECUDA, "heat solve: %s", cudaGetErrorString(cudaGetLastError()));
  CK(cudaGetLastError());
  return SBMT_OK;
}

int mesh_profile(sbmt_ctx* ctx, int enable) {
  if (!ctx) return fail(SBMT_EINVAL, "null ctx");
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->prof = enable != 0;
  return SBMT_OK;
}

int mesh_profile_read(sbmt_ctx* ctx, int reset, int cap, const char** names, double* ms, int64_t* launches,
                      int* n) {
  if (!ctx || !n) return fail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  prof_collect(ctx);
  *n = KN_COUNT;
  for (int k = 0; k < KN_COUNT && k < cap; ++k) {
    if (names) names[k] = kKernelNames[k];
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < KN_COUNT; ++k) ctx->prof_ms[k] = 0, ctx->prof_n[k] = 0;
  return SBMT_OK;
}

int mesh_stage(sbmt_ctx* ctx, sbmt_mesh mesh, int stage, void* host_out, int64_t cap, int64_t* n) {
  if (!ctx || !n) return fail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->meshes.find(mesh);
  if (it == ctx->meshes.end()) return fail(SBMT_ENOENT, "unknown mesh");
  MeshRec* m = it->second;
  if (stage == 4) {  // cells over the Tier-G limit, for every mesh (none in a preprocessed one)
    CK(cudaEventSynchronize(m->done));
    const u32 cnt = m->pre ? 0u : m->h_info[4], kept = std::min<u32>(cnt, OVER_CAP);
    std::vector<u32> ids(kept);
    if (kept) CK(cudaMemcpy(ids.data(), m->over_cells, kept * sizeof(u32), cudaMemcpyDeviceToHost));
    std::sort(ids.begin(), ids.end());
    *n = (int64_t)cnt;
    int64_t* o = (int64_t*)host_out;
    for (int64_t k = 0; k < std::min<int64_t>(cap, (int64_t)kept); ++k) o[k] = (int64_t)ids[k];
    return SBMT_OK;
  }
  if (!m->keep) return fail(SBMT_EINVAL, "mesh made without SBMT_KEEP_STAGES");
  CK(cudaEventSynchronize(m->done));
  if (stage == 1) {
    std::vector<Seg> s(m->nseg);
    CK(cudaMemcpy(s.data(), m->segs, s.size() * sizeof(Seg), cudaMemcpyDeviceToHost));
    *n = (int64_t)s.size();
    int32_t* o = (int32_t*)host_out;
    for (int64_t k = 0; k < std::min<int64_t>(cap, *n); ++k) {
      const Seg& x = s[k];
      const int32_t rec[8] = {x.cx, x.cy, seg_dir(x), seg_len(x), (int32_t)(x.lab & 0xFFFF),
                              (int32_t)(x.lab >> 16), seg_rev(x), 0};
      std::memcpy(o + 8 * k, rec, sizeof rec);
    }
    return SBMT_OK;
  }
  if (stage == 2) {
    std::vector<Event> e(m->ne);
    std::vector<Seg> s(m->nseg);
    CK(cudaMemcpy(e.data(), m->ev, e.size() * sizeof(Event), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.data(), m->segs, s.size() * sizeof(Seg), cudaMemcpyDeviceToHost));
    std::sort(e.begin(), e.end(), [](const Event& a, const Event& b) { return a.gid < b.gid; });
    *n = (int64_t)e.size();
    int64_t* o = (int64_t*)host_out;
    for (int64_t k = 0; k < std::min<int64_t>(cap, *n); ++k) {
      const Seg& x = s[e[k].seg];
      const int64_t rec[4] = {(int64_t)e[k].edge, (int64_t)e[k].gid, (int64_t)x.cy * (m->W + 1) + x.cx,
                              (int64_t)seg_dir(x)};
      std::memcpy(o + 4 * k, rec, sizeof rec);
    }
    return SBMT_OK;
  }
  if (stage == 3) {
    std::vector<u32> bs(m->nbc), po(m->nbc);
    CK(cudaMemcpy(bs.data(), m->bcut, bs.size() * sizeof(u32), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(po.data(), m->bbase, po.size() * sizeof(u32), cudaMemcpyDeviceToHost));
    u64 nr = 0;
    for (u32 b = 0; b < m->nbc; ++b) nr = std::max<u64>(nr, (u64)po[b] + bs[b]);
    std::vector<CutRec> r(nr);
    CK(cudaMemcpy(r.data(), m->recs, r.size() * sizeof(CutRec), cudaMemcpyDeviceToHost));
    int64_t k = 0;
    int64_t* o = (int64_t*)host_out;
    for (u32 b = 0; b < m->nbc; ++b)
      for (u32 u = 0; u < bs[b]; ++u, ++k) {
        const CutRec& c = r[po[b] + u];
        if (k < cap) {
          const int64_t rec[5] = {(int64_t)c.cell, (int64_t)(c.code & 0xFFFF), (int64_t)c.ntri, (int64_t)c.nchain,
                                  (int64_t)((c.code >> 16) & 1)};
          std::memcpy(o + 5 * k, rec, sizeof rec);
        }
      }
    *n = k;
    return SBMT_OK;
  }
  return fail(SBMT_EINVAL, "unknown stage %d", stage);
}

}  // extern "C"
