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

struct MeshRec {
  sbmt_mesh id = 0;
  cudaEvent_t done = nullptr;
  void* out_block = nullptr;
  double* xy = nullptr;
  int* tri = nullptr;
  unsigned short* label = nullptr;
  unsigned short* code = nullptr;
  int64_t nv = 0, nt = 0, ncells = 0, nseg_total = 0, ne_total = 0, nc_total = 0, nvg = 0;
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
  unsigned char* pstatus = nullptr;
  int* psnap = nullptr;
  int* pelim = nullptr;
  double thr[3] = {0, 0, 0};
  int64_t npts = 0;
};

}  // namespace

// kernels of the hot path, in launch order (for the per-kernel timing)
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
  KN_COUNT
};
const char* const kKernelNames[KN_COUNT] = {"k_corner_bits", "k_segments", "k_seg_count", "k_scan",
                                            "k_walk", "k_rank", "k_sort", "k_cutcells", "k_emit",
                                            "k_tierg", "k_lattice_xy", "k_preprocess", "k_heat"};

// One stream of work: the context's own stream, or one of the extra streams
// a batch spreads its images over.  Each lane has its own scratch arena and
// its own tracing events, so lanes run on separate host threads.
struct Lane {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the Tier-G kernels run on a second stream beside the emission kernel,
  // forked from and joined back into the lane's stream
  cudaStream_t side = nullptr, side2 = nullptr;  // side2: the Tier-G warp kernel
  cudaEvent_t fork = nullptr, join = nullptr, order = nullptr, warp = nullptr;
  // per-call scratch: bump allocation in stream-ordered chunks
  std::vector<std::pair<char*, size_t>> chunks;
  size_t chunk_used = 0, call_bytes = 0;
  // tracing: events around each kernel launch, resolved lazily
  struct Mark {
    int k, kernels;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Mark> pending;
};

// images a batch meshes at once, each on its own lane (SBMT_BATCH_LANES
// overrides, 1..32)
int batch_lanes() {
  static const int n = [] {
    const char* e = std::getenv("SBMT_BATCH_LANES");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 && v <= 32 ? v : 12;
  }();
  return n;
}

struct sbmt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::mutex mu;   // one API call at a time
  std::mutex reg;  // meshes, ids, events, pinned slots, tables: shared by the lanes of a batch
  std::map<sbmt_mesh, MeshRec*> meshes;
  sbmt_mesh next = 1;
  Lane main;
  std::vector<Lane*> extra;
  bool in_batch = false;  // lanes share the tables: no eviction while set
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[KN_COUNT] = {};
  int64_t prof_n[KN_COUNT] = {};
  // grid tables per (W, H, h, origin), kept on the device
  struct TableEntry {
    Tables host;
    i64* dev = nullptr;
    cudaEvent_t ready = nullptr;  // recorded after the upload
    uint64_t last_use = 0;
  };
  std::map<std::array<i64, 6>, TableEntry> tables;
  uint64_t tick = 0;
  // pinned slots for the per-mesh status words
  std::vector<u32*> pinned_slabs;
  std::vector<u32*> pinned_free;
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
void prof_collect(sbmt_ctx* c) {
  prof_collect_lane(c, &c->main);
  for (Lane* L : c->extra) prof_collect_lane(c, L);
}

// brackets one kernel launch with events on the lane's stream when tracing
struct ProfScope {
  Lane* L;
  cudaStream_t s;
  int k, kernels = 0;
  cudaEvent_t a = nullptr;
  ProfScope(sbmt_ctx* c, Lane* L_, int k_, cudaStream_t s_) : L(L_), s(s_), k(k_) {
    if (c->prof && (a = take_event(L->ev_pool))) cudaEventRecord(a, s);
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
  if (L->own_stream) cudaStreamDestroy(L->stream);
  if (L->side) cudaStreamSynchronize(L->side), cudaStreamDestroy(L->side);
  if (L->side2) cudaStreamSynchronize(L->side2), cudaStreamDestroy(L->side2);
  for (cudaEvent_t e : {L->fork, L->join, L->order, L->warp})
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
  for (cudaEvent_t* e : {&L->fork, &L->join, &L->order, &L->warp})
    if (!*e && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
      *e = nullptr;
      return fail(SBMT_ECUDA, "fork/join events");
    }
  return SBMT_OK;
}

// callers hold ctx->reg
u32* pinned_slot(sbmt_ctx* ctx) {
  if (ctx->pinned_free.empty()) {
    u32* slab = nullptr;
    if (cudaMallocHost(&slab, 1024 * 8 * sizeof(u32)) != cudaSuccess) return nullptr;
    ctx->pinned_slabs.push_back(slab);
    for (int k = 1023; k >= 0; --k) ctx->pinned_free.push_back(slab + 8 * k);
  }
  u32* p = ctx->pinned_free.back();
  ctx->pinned_free.pop_back();
  std::memset(p, 0, 8 * sizeof(u32));
  return p;
}

// grid tables for one configuration, built once and kept on the device.
// The host build and the upload run outside ctx->reg, so the lanes of a
// batch build different tables at once; a lane that finds an entry another
// lane is still uploading waits for its event.  An evicted entry may still be
// read by work in flight on any lane, so eviction waits for the device, and
// is put off while a batch runs.
int get_tables(sbmt_ctx* ctx, Lane* lane, const GridP& g, const Tables** host, const i64** dev) {
  const std::array<i64, 6> key{g.W, g.H, g.p, g.q, g.ox, g.oy};
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    auto it = ctx->tables.find(key);
    if (it != ctx->tables.end()) {
      it->second.last_use = ++ctx->tick;
      *host = &it->second.host;
      *dev = it->second.dev;
      if (cudaStreamWaitEvent(lane->stream, it->second.ready, 0) != cudaSuccess)
        return fail(SBMT_ECUDA, "table wait");
      return SBMT_OK;
    }
    if (ctx->tables.size() >= 1024 && !ctx->in_batch) {  // evict the least recently used entry
      auto old = ctx->tables.begin();
      for (auto jt = ctx->tables.begin(); jt != ctx->tables.end(); ++jt)
        if (jt->second.last_use < old->second.last_use) old = jt;
      cudaDeviceSynchronize();
      cudaFree(old->second.dev);
      cudaEventDestroy(old->second.ready);
      ctx->tables.erase(old);
    }
  }
  sbmt_ctx::TableEntry te;
  int rc = build_tables(g, te.host);
  if (rc) return rc;
  const Tables& tb = te.host;
  const i64 nrows = (i64)tb.clo.size(), nvr = (i64)tb.vlo.size();
  std::vector<i64> all;
  all.insert(all.end(), tb.clo.begin(), tb.clo.end());
  all.insert(all.end(), tb.chi.begin(), tb.chi.end());
  all.insert(all.end(), tb.cbase.begin(), tb.cbase.end());
  all.insert(all.end(), tb.vlo.begin(), tb.vlo.end());
  all.insert(all.end(), tb.vhi.begin(), tb.vhi.end());
  all.insert(all.end(), tb.vbase.begin(), tb.vbase.end());
  const size_t nl = all.size();
  all.resize(nl + nrows);
  std::memcpy(all.data() + nl, tb.lrow.data(), tb.lrow.size() * sizeof(int));
  (void)nvr;
  if (cudaMallocAsync(&te.dev, all.size() * sizeof(i64), lane->stream) != cudaSuccess)
    return fail(SBMT_ENOMEM, "table allocation");
  // from pageable memory the copy has read `all` when the call returns
  if (cudaMemcpyAsync(te.dev, all.data(), all.size() * sizeof(i64), cudaMemcpyHostToDevice, lane->stream) ||
      cudaEventCreateWithFlags(&te.ready, cudaEventDisableTiming) || cudaEventRecord(te.ready, lane->stream))
    return fail(SBMT_ECUDA, "table upload");
  std::lock_guard<std::mutex> lk(ctx->reg);
  auto ins = ctx->tables.try_emplace(key, std::move(te));
  auto it = ins.first;
  if (!ins.second) {
    // another lane built the same tables meanwhile: use those
    cudaFreeAsync(te.dev, lane->stream);
    cudaEventDestroy(te.ready);
    if (cudaStreamWaitEvent(lane->stream, it->second.ready, 0) != cudaSuccess) return fail(SBMT_ECUDA, "table wait");
  }
  it->second.last_use = ++ctx->tick;
  *host = &it->second.host;
  *dev = it->second.dev;
  return SBMT_OK;
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
  if (m->done) ctx->ev_pool.push_back(m->done);
  if (m->h_info) ctx->pinned_free.push_back(m->h_info);
  delete m;
}

int check_params(const sbmt_image* img, const sbmt_params* pr, bool pre = false) {
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
  if (pre) {
    if (pr->mode != SBMT_PREPROCESS || pr->format != SBMT_EXPLICIT)
      return fail(SBMT_EINVAL, "mesh_preprocess takes mode SBMT_PREPROCESS and the explicit format");
  } else {
    if (pr->mode == SBMT_PREPROCESS) return fail(SBMT_EPROTO, "SBMT_PREPROCESS is not available");
    if (pr->mode != SBMT_PLAIN || (pr->format != SBMT_EXPLICIT && pr->format != SBMT_COMPACT))
      return fail(SBMT_EINVAL, "mode/format");
  }
  if (pr->h_num < 2 || pr->h_num > 1024 || (pr->h_num & 1) || pr->h_den < 1 || pr->h_den > 63 ||
      !(pr->h_den & 1))
    return fail(SBMT_EINVAL, "h = %d/%d outside the degeneracy-free class (even h_num <= 1024, odd h_den < 64)",
                pr->h_num, pr->h_den);
  if ((pr->origin2x & 1) || (pr->origin2y & 1) || pr->origin2x < -65536 || pr->origin2x > 65536 ||
      pr->origin2y < -65536 || pr->origin2y > 65536)
    return fail(SBMT_EINVAL, "origin must be integer pixels within +-32768");
  return SBMT_OK;
}

// the whole path for one image, enqueued on one lane
// fork: run the Tier-G kernels on the lane's second stream beside the
// emission (single meshes; a batch's lanes already fill the device)
int mesh_one(sbmt_ctx* ctx, Lane* lane, const sbmt_image* img, const sbmt_params* pr, sbmt_mesh* out, bool fork) {
  int rc = check_params(img, pr);
  if (rc) return rc;
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
  if (tb.ncells >= (1ll << 31) || 3 * tb.nverts >= (1ll << 32))
    return fail(SBMT_EINVAL, "mesh too large (%lld cells)", (long long)tb.ncells);
  MeshRec* m = new MeshRec();
  m->W = g.W, m->H = g.H;
  m->keep = (pr->flags & SBMT_KEEP_STAGES) != 0;
  std::vector<void*> tmp;  // device memory freed at the end of the call
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
  // image on the device
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

  // every counter of the call, zeroed by one memset: the vertex count (u64),
  // the u32 counters (err, cut cells, Tier-G cells and their triangles next
  // to each other: the mesh's status words), the bucket counts of pairs and
  // events, the buckets' extra triangles and inside vertices, the Tier-G
  // per-size counts
  const u32 nbc = (u32)((tb.ncells + (1 << CB_LOG) - 1) >> CB_LOG);
  const u32 nbe = (u32)((3 * tb.nverts + (1 << EB_LOG) - 1) >> EB_LOG);
  const size_t zwords = 16 + (nbc + 1) + (nbe + 1) + 2 * ((size_t)nbc + 1) + 3 * (TIERG_TN + 2);
  u32* zero;
  if ((rc = aalloc(lane, &zero, zwords))) return bail(rc);
  CK(cudaMemsetAsync(zero, 0, zwords * sizeof(u32), st));
  unsigned long long* cnt64 = (unsigned long long*)zero;
  u32* cnt32 = zero + 8;
  u32 *nseg = cnt32 + 0, *nwlist = cnt32 + 1, *err = cnt32 + 2, *nrec = cnt32 + 3, *nglist = cnt32 + 4,
      *ngtri = cnt32 + 5, *nover = cnt32 + 6;
  u32* pcnt = zero + 16;
  u32* ecnt = pcnt + nbc + 1;
  u32* bextra = ecnt + nbe + 1;
  u32* bchain = bextra + nbc + 1;
  u32* gcnt = bchain + nbc + 1;

  // K1a
  const int W = g.W, H = g.H;
  const int wpr = (W + 1 + 31) / 32, wpc = (H + 1 + 31) / 32;
  u32 *vrow, *vcol;
  if ((rc = aalloc(lane, &vrow, (size_t)wpr * (H + 1)))) return bail(rc);
  if ((rc = aalloc(lane, &vcol, (size_t)wpc * (W + 1)))) return bail(rc);
  TRACE(KN_CORNER, launch_corner_bits(dimg, pitch, img->dtype, W, H, vrow, wpr, vcol, wpc, cnt64 + 0, st));
  unsigned long long h64[4];
  CK(cudaMemcpyAsync(h64, cnt64, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const u64 NC = h64[0];
  // K1b: every vertex starts at most two runs (+x and +y)
  const u32 seg_cap = (u32)std::max<u64>(2 * NC, 1);
  Seg* segs;
  if ((rc = m->keep ? dalloc(lane, &segs, seg_cap, m->scratch) : aalloc(lane, &segs, seg_cap))) return bail(rc);
  TRACE(KN_SEG, launch_segments(dimg, pitch, img->dtype, W, H, vrow, wpr, vcol, wpc, segs, seg_cap, nseg, err, st));
  // K2: pairs per segment in closed form and their scan -> fixed pair and
  // event indices of every segment
  u32 *npairs, *pbase, *sscr;
  const size_t scr_words = std::max({scan_scratch_words(seg_cap), scan_scratch_words(nbc), scan_scratch_words(nbe)});
  if ((rc = aalloc(lane, &npairs, seg_cap))) return bail(rc);
  if ((rc = aalloc(lane, &pbase, (size_t)seg_cap + 1))) return bail(rc);
  if ((rc = aalloc(lane, &sscr, scr_words + 1))) return bail(rc);
  TRACE(KN_TCOUNT, launch_seg_count(g, segs, nseg, seg_cap, npairs, st));
  TRACE(KN_SCAN, launch_scan(npairs, 1, pbase, seg_cap, sscr, st));
  u32 h32[4];
  CK(cudaMemcpyAsync(h32, cnt32, 4 * sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h32 + 3, pbase + seg_cap, sizeof(u32), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h32[2]) return bail(fail(SBMT_EINTERNAL, "device check failed during extraction (0x%x)", h32[2]));
  const u32 nsegs = h32[0];
  if (nsegs > seg_cap) return bail(fail(SBMT_EINTERNAL, "segment count %u above bound %u", nsegs, seg_cap));
  const u64 NP = h32[3], NE = NP - nsegs;
  const u64 NVg = (u64)tb.nverts;
  const u64 V = NVg + NE + NC, T = (u64)tb.ncells + 2 * NC + 2 * NE;
  if (V >= (1ull << 31) || T >= (1ull << 31) || NP >= (1ull << 31))
    return bail(fail(SBMT_EINVAL, "mesh too large (%llu triangles)", (unsigned long long)T));
  // buckets: pairs by cell id, events by grid-edge id
  u32 *poff, *eoff, *pcur, *ecur;
  if ((rc = aalloc(lane, &poff, nbc + 1))) return bail(rc);
  if ((rc = aalloc(lane, &eoff, nbe + 1))) return bail(rc);
  if ((rc = aalloc(lane, &pcur, nbc + 1))) return bail(rc);
  if ((rc = aalloc(lane, &ecur, nbe + 1))) return bail(rc);
  Pair *pairs, *sorted;
  Event* ev;
  CutRec* recs;
  u32 *bcut, *bbase, *extra_scan, *chain_scan, *olist, *wlist, *elist, *eidx;
  TStage* stg;
  u32* cstart;
  if ((rc = aalloc(lane, &cstart, walk_chunks((u32)NP) + 1))) return bail(rc);
  if ((rc = aalloc(lane, &pairs, NP))) return bail(rc);
  if ((rc = aalloc(lane, &sorted, NP))) return bail(rc);
  if ((rc = m->keep ? dalloc(lane, &ev, NE, m->scratch) : aalloc(lane, &ev, NE))) return bail(rc);
  if ((rc = aalloc(lane, &eidx, NE))) return bail(rc);
  // K2: one walk (pairs in their global order, in the sorted buffer for now;
  // events at their fixed indices; bucket counts), then the bucket scans and
  // the scatter into buckets
  TRACE(KN_TCOUNT, launch_chunk_map(pbase, nseg, seg_cap, cstart, st));
  TRACE(KN_TEMIT, launch_walk(g, segs, pbase, cstart, (u32)NP, pcnt, ecnt, sorted, ev, err, st));
  if (nbc <= SCAN_ONE && nbe <= SCAN_ONE) {
    TRACE(KN_SCAN, launch_scan_pair(pcnt, poff, pcur, nbc, ecnt, eoff, ecur, nbe, st));
  } else {
    TRACE(KN_SCAN, launch_scan(pcnt, 1, poff, nbc, sscr, st));
    TRACE(KN_SCAN, launch_scan(ecnt, 1, eoff, nbe, sscr, st));
    CK(cudaMemcpyAsync(pcur, poff, (nbc + 1) * sizeof(u32), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ecur, eoff, (nbe + 1) * sizeof(u32), cudaMemcpyDeviceToDevice, st));
  }
  TRACE(KN_TEMIT, launch_scatter(sorted, (u32)NP, ev, (u32)NE, pcur, ecur, pairs, eidx, st));
  if ((rc = m->keep ? dalloc(lane, &recs, NP, m->scratch) : aalloc(lane, &recs, NP))) return bail(rc);
  if ((rc = m->keep ? dalloc(lane, &bcut, nbc + 1, m->scratch) : aalloc(lane, &bcut, nbc + 1))) return bail(rc);
  if ((rc = m->keep ? dalloc(lane, &bbase, nbc + 1, m->scratch) : aalloc(lane, &bbase, nbc + 1))) return bail(rc);
  if ((rc = aalloc(lane, &extra_scan, nbc + 1))) return bail(rc);
  if ((rc = aalloc(lane, &chain_scan, nbc + 1))) return bail(rc);
  if ((rc = aalloc(lane, &stg, NP))) return bail(rc);
  if ((rc = aalloc(lane, &wlist, NP))) return bail(rc);
  if ((rc = aalloc(lane, &olist, NP))) return bail(rc);
  if ((rc = aalloc(lane, &elist, NE))) return bail(rc);
  // outputs.  The compact format stores the vertices after the lattice, the
  // per-cell label and code, and the patch triangles of the cut cells (at
  // most the extra triangles plus one per cut cell, and cut cells <= pairs).
  const bool compact = pr->format == SBMT_COMPACT;
  m->format = pr->format;
  const u64 nxy = compact ? V - NVg : V, ntr = compact ? (T - (u64)tb.ncells) + NP : T;
  const size_t bxy = 16 * nxy, btri = 12 * ntr, blab = 2 * ntr, bcode = 2 * ntr;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_tri = up(bxy), off_lab = up(off_tri + btri), off_code = up(off_lab + blab);
  const size_t off_cl = up(off_code + bcode), off_cc = up(off_cl + (compact ? 2 * (size_t)tb.ncells : 0));
  const size_t off_pc = up(off_cc + (compact ? 2 * (size_t)tb.ncells : 0));
  const size_t off_po = up(off_pc + (compact ? 4 * NP : 0));
  const size_t off_ov = up(off_po + (compact ? 4 * (NP + 1) : 0));
  const size_t total = off_ov + 4 * (size_t)OVER_CAP + 256;
  if (cudaMallocAsync(&m->out_block, total, st) != cudaSuccess)
    return bail(fail(SBMT_ENOMEM, "output allocation of %zu bytes", total));
  char* ob = (char*)m->out_block;
  m->xy = (double*)ob;
  m->tri = (int*)(ob + off_tri);
  m->label = (unsigned short*)(ob + off_lab);
  m->code = (unsigned short*)(ob + off_code);
  m->over_cells = (u32*)(ob + off_ov);
  CompactOut cp{0, 0, nullptr, nullptr, nullptr, nullptr, nullptr};
  u32* cut_scan = nullptr;
  if (compact) {
    m->cell_label = (unsigned short*)(ob + off_cl), m->cell_code = (unsigned short*)(ob + off_cc);
    m->patch_cell = (u32*)(ob + off_pc), m->patch_off = (u32*)(ob + off_po);
    if ((rc = aalloc(lane, &cut_scan, nbc + 1))) return bail(rc);
    cp = CompactOut{1, (u32)NVg, m->cell_label, m->cell_code, m->patch_cell, m->patch_off, cut_scan};
    if (nbc == 0) CK(cudaMemsetAsync(m->patch_off, 0, sizeof(u32), st));
  }
  m->nv = (int64_t)V, m->nt = (int64_t)T, m->ncells = tb.ncells;
  m->nseg_total = nsegs, m->ne_total = (int64_t)NE, m->nc_total = (int64_t)NC, m->nvg = (int64_t)NVg;
  // registry, K3, scans, K4, K4-G, lattice coordinates
  if (fork && (rc = lane_side(lane))) return bail(rc);
  int nrk = 0;
  TRACE(KN_RANK, nrk = launch_rank_events(g, ev, eidx, elist, eoff, nbe, (u32)NVg, m->xy, cp.xy0, st,
                                          fork ? lane->side : nullptr, lane->fork, lane->join));
  if (nrk < 0) return bail(fail(SBMT_ECUDA, "registry stream events"));
  TRACE(KN_SORT, launch_sort(pairs, sorted, poff, nbc, recs, nrec, bcut, bbase, st));
  TRACE(KN_CUTCELLS, launch_cutcells(g, dimg, pitch, img->dtype, sorted, segs, ev, recs, nrec, bextra, bchain, stg,
                                     nglist, ngtri, gcnt, err, st));
  if (nbc <= SCAN_ONE) {
    TRACE(KN_SCAN, launch_scan_pair(bextra, extra_scan, nullptr, nbc, bchain, chain_scan, nullptr, nbc, st));
  } else {
    TRACE(KN_SCAN, launch_scan(bextra, 1, extra_scan, nbc, sscr, st));
    TRACE(KN_SCAN, launch_scan(bchain, 1, chain_scan, nbc, sscr, st));
  }
  if (compact) {
    if (nbc <= SCAN_ONE) {
      TRACE(KN_SCAN, launch_scan_pair(bcut, cut_scan, nullptr, nbc, nullptr, nullptr, nullptr, 0, st));
    } else {
      TRACE(KN_SCAN, launch_scan(bcut, 1, cut_scan, nbc, sscr, st));
    }
  }
  // Tier-G beside the emission: both read the scans and the records, and
  // write disjoint parts of the output
  cudaStream_t gst = st;
  if (fork) {
    if ((rc = lane_side(lane))) return bail(rc);
    CK(cudaEventRecord(lane->fork, st));
    CK(cudaStreamWaitEvent(lane->side, lane->fork, 0));
    gst = lane->side;
  }
  int ntg = 0;
  TRACE_ON(KN_TIERG, gst,
           ntg = launch_tierg(g, dimg, pitch, img->dtype, sorted, segs, ev, recs, bcut, bbase, nbc, gcnt, olist, wlist,
                        nwlist, extra_scan, chain_scan, compact ? cut_scan : nullptr, (u32)(NVg + NE), m->tri,
                        m->label, m->code, m->xy, cp.xy0, err, nover, m->over_cells, gst,
                        fork ? lane->side2 : nullptr, lane->order, lane->warp));
  if (ntg < 0) return bail(fail(SBMT_ECUDA, "Tier-G stream events"));
  if (fork) CK(cudaEventRecord(lane->join, lane->side));
  TRACE(KN_EMIT, launch_emit(g, dimg, pitch, img->dtype, recs, bcut, bbase, extra_scan, chain_scan, stg, nbc,
                             (u32)NVg, (u32)NE, m->tri, m->label, m->code, m->xy, cp, st));
  // x of lattice vertex v(i, j) is indexed by m = 2i + j
  i64 m_lo = 0, m_hi = -1;
  for (i64 r = 0; r < nvr; ++r) {
    const i64 a = 2 * tb.vlo[r] + tb.vj0 + r, b = 2 * tb.vhi[r] + tb.vj0 + r;
    if (r == 0 || a < m_lo) m_lo = a;
    if (r == 0 || b > m_hi) m_hi = b;
  }
  double* xtab;
  if ((rc = aalloc(lane, &xtab, (size_t)std::max<i64>(1, m_hi - m_lo + 1)))) return bail(rc);
  if (!compact) TRACE(KN_XY, launch_lattice_xy(g, m->xy, xtab, m_lo, m_hi - m_lo + 1, st));
  if (fork) CK(cudaStreamWaitEvent(st, lane->join, 0));
  CK(cudaGetLastError());
  // the status words: err, cut cells, Tier-G cells, Tier-G triangles, cells
  // over the Tier-G limit
  CK(cudaMemcpyAsync(m->h_info, err, 5 * sizeof(u32), cudaMemcpyDeviceToHost, st));
  if (m->keep) {
    // sorted pairs are needed by nobody after emission; keep what mesh_stage reads
    m->segs = segs, m->nseg = nsegs, m->ev = ev, m->ne = (u32)NE, m->recs = recs, m->bcut = bcut;
    m->bbase = bbase, m->nbc = nbc;
  }
  free_list(st, tmp);
  arena_end(lane);
  {
    std::lock_guard<std::mutex> lk(ctx->reg);
    m->done = pool_event(ctx);
  }
  if (!m->done) return bail(fail(SBMT_ECUDA, "event create"));
  CK(cudaEventRecord(m->done, st));
  std::lock_guard<std::mutex> lk(ctx->reg);
  m->id = ctx->next++;
  ctx->meshes[m->id] = m;
  *out = m->id;
  return SBMT_OK;
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
int pre_one(sbmt_ctx* ctx, Lane* lane, const sbmt_image* img, const sbmt_params* pr, sbmt_mesh* out) {
  int rc = check_params(img, pr, true);
  if (rc) return rc;
  double A, B, C;
  if ((rc = pre_thresholds(pr, &A, &B, &C))) return rc;
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

}  // namespace

extern "C" {

const char* sbmt_last_error(void) { return g_last_error.c_str(); }

int mesh_create(sbmt_ctx** out, int device, size_t pool_bytes, void* cuda_stream) {
  if (!out) return fail(SBMT_EINVAL, "null ctx pointer");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(SBMT_ECUDA, "no CUDA device");
  if (device < 0 || device >= n) return fail(SBMT_EINVAL, "device %d of %d", device, n);
  CK(cudaSetDevice(device));
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
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  std::lock_guard<std::mutex> lk(ctx->mu);
  return mesh_one(ctx, &ctx->main, img, params, out, true);
}

int mesh_preprocess(sbmt_ctx* ctx, const sbmt_image* img, const sbmt_params* params, sbmt_mesh* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  std::lock_guard<std::mutex> lk(ctx->mu);
  return pre_one(ctx, &ctx->main, img, params, out);
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
  CK(cudaSetDevice(ctx->device));
  const int K = std::min(n, batch_lanes());
  while ((int)ctx->extra.size() < K - 1) {
    Lane* L = new Lane();
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete L;
      return fail(SBMT_ECUDA, "stream create");
    }
    L->own_stream = true;
    ctx->extra.push_back(L);
  }
  std::vector<Lane*> lanes{&ctx->main};
  for (int k = 0; k < K - 1; ++k) lanes.push_back(ctx->extra[k]);
  // the extra lanes start after the work already on the context stream
  cudaEvent_t start;
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    start = pool_event(ctx);
  }
  CK(cudaEventRecord(start, ctx->stream));
  for (int k = 1; k < K; ++k) CK(cudaStreamWaitEvent(lanes[k]->stream, start, 0));
  // largest images first, each lane taking the next image when it is free
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (i64)imgs[a].width * imgs[a].height > (i64)imgs[b].width * imgs[b].height;
  });
  std::vector<char> made(n, 0);
  std::atomic<int> next{0};
  std::atomic<int> first_rc{0};
  std::mutex msg_mu;
  std::string msg;
  ctx->in_batch = true;
  auto work = [&](Lane* L) {
    cudaSetDevice(ctx->device);
    for (int i; (i = next.fetch_add(1)) < n;) {
      if (first_rc.load()) break;
      const int k = order[i];
      const int rc = mesh_one(ctx, L, imgs + k, params + (n_params == 1 ? 0 : k), out + k, false);
      if (rc) {
        std::lock_guard<std::mutex> ml(msg_mu);
        if (!first_rc.load()) first_rc = rc, msg = sbmt_last_error();
        break;
      }
      made[k] = 1;
    }
  };
  std::vector<std::thread> threads;
  for (int k = 1; k < K; ++k) threads.emplace_back(work, lanes[k]);
  work(lanes[0]);
  for (auto& t : threads) t.join();
  ctx->in_batch = false;
  // later work on the context stream sees every mesh of the batch
  for (int k = 1; k < K; ++k) {
    cudaEvent_t e;
    {
      std::lock_guard<std::mutex> rl(ctx->reg);
      e = pool_event(ctx);
    }
    CK(cudaEventRecord(e, lanes[k]->stream));
    CK(cudaStreamWaitEvent(ctx->stream, e, 0));
    std::lock_guard<std::mutex> rl(ctx->reg);
    ctx->ev_pool.push_back(e);
  }
  {
    std::lock_guard<std::mutex> rl(ctx->reg);
    ctx->ev_pool.push_back(start);
  }
  if (first_rc.load()) {
    std::lock_guard<std::mutex> rl(ctx->reg);
    for (int k = 0; k < n; ++k) {
      if (!made[k]) continue;
      auto it = ctx->meshes.find(out[k]);
      if (it != ctx->meshes.end()) destroy_mesh(ctx, it->second, ctx->stream), ctx->meshes.erase(it);
    }
    return fail(first_rc.load(), "%s", msg.c_str());
  }
  return SBMT_OK;
}

int mesh_query(sbmt_ctx* ctx, sbmt_mesh mesh, int wait_ms, sbmt_mesh_view* out) {
  if (!ctx || !out) return fail(SBMT_EINVAL, "null ctx or out");
  MeshRec* m;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
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
    for (auto& kv : ctx->tables) cudaFreeAsync(kv.second.dev, ctx->stream), cudaEventDestroy(kv.second.ready);
    for (Lane* L : ctx->extra) lane_release(L), delete L;
    lane_release(&ctx->main);
    for (u32* slab : ctx->pinned_slabs) cudaFreeHost(slab);
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
  // the mesh's completion now includes the projection
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
