// sbmt_server.cu -- serving: a request loop over meshing requests of
// different sizes, built on the C interface (mesh_batch, mesh_query,
// mesh_release).
//
// Requests are admitted by device memory: before its boundary is counted a
// request reserves an upper bound of what meshing it can hold on the device
// (from W, H and h alone), and once its batch's counting phase is done the
// reservation becomes the exact size of its mesh.  Admitted requests are
// meshed in batches (one mesh_batch call: every stage one launch over all of
// them).  Continuous batching: each worker owns a context with its own
// stream and host thread and takes the next batch from the queue as soon as
// its previous batch's counting phase is done, so arrivals join the next
// launch while earlier batches still emit on the device, and the workers'
// batches overlap on the GPU.  Bitmaps given as device pointers and every
// finished mesh stay on the device.  Meshes do not depend on how requests
// were grouped: each is the mesh of its own image (Sec. 3.5's corollary,
// every cell's patch is independent of the others).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sbmt.h"

namespace {

using Clock = std::chrono::steady_clock;

thread_local std::string g_srv_err;
int sfail(int code, const char* msg) {
  g_srv_err = msg;
  return code;
}

enum { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2 };

struct Req {
  uint64_t id = 0;
  sbmt_image img{};
  sbmt_params pr{};
  std::vector<unsigned char> host;  // copy of a host image
  size_t bound = 0, reserved = 0;
  int state = RQ_QUEUED;
  int status = SBMT_EPENDING;
  int worker = -1;
  sbmt_mesh mesh = 0;
  sbmt_mesh_view view{};
  int batch_size = 0;
  bool cancelled = false;
  int starved = 0;  // admission checks failed while nothing else held memory
  Clock::time_point t_submit, t_admit, t_done;
};

struct Batch {
  cudaEvent_t done = nullptr;
  std::vector<std::shared_ptr<Req>> reqs;
};

// An upper bound of the device bytes meshing one image can hold, before its
// boundary is counted: every pixel edge a boundary edge, every corner a
// boundary vertex, and every boundary edge crossing as many grid edges as
// its length allows (a unit pixel edge meets at most 3 + 2.31/h grid edges),
// times the bytes per segment, event, (cell, segment) pair and triangle of
// the path, plus the image, the corner bit-planes and the per-cell tables.
size_t request_bound(const sbmt_image& img, const sbmt_params& pr) {
  const double W = img.width, H = img.height, h = (double)pr.h_num / (double)pr.h_den;
  const double edges = 2 * W * H + W + H, corners = (W + 1) * (H + 1);
  const double events = edges * (3.0 + 2.31 / h);
  const double cells = 2.0 * (W + h) * (H + h) / (h * h * 0.8660254) + 4 * (W + H) / h + 64;
  const double segs = std::min(2 * corners, edges);
  const double pairs = segs + events;
  const double tri = cells + 2 * corners + 2 * events, vert = cells + events + corners;
  const double bytes = W * H * img.dtype + corners / 4 + 24 * segs + 96 * pairs + 40 * events + 16 * pairs +
                       16 * tri + 16 * vert + 32 * cells / 1024 + (1 << 20);
  return (size_t)std::min(bytes, 1e18);
}

}  // namespace

struct sbmt_server {
  int device = 0;
  sbmt_server_config cfg{};
  size_t budget = 0, reserved = 0, peak = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::map<uint64_t, std::shared_ptr<Req>> reqs;
  uint64_t next_id = 1;
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_cancelled = 0, n_batches = 0, n_admit_checks = 0;
  bool stop = false;
  struct Worker {
    sbmt_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::thread th;
  };
  std::vector<Worker> workers;
  // batches on the device, in launch order, with their worker
  std::deque<std::pair<int, Batch>> inflight;
  std::thread harvester;
  bool workers_done = false;
};

namespace {

// the bytes of finished meshes, or of reservations, are given back under s->mu
void give_back(sbmt_server* s, Req& r) {
  s->reserved -= std::min(s->reserved, r.reserved);
  r.reserved = 0;
}

// The harvester thread: finished batches' meshes, their views and status.
// It queries events and meshes only (mesh_query does not wait for a
// worker's call in progress on the same context), so a request is seen
// finished within microseconds of its batch.
void harvest_loop(sbmt_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<std::pair<int, Batch>> ready;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto it = s->inflight.begin(); it != s->inflight.end();) {
        const cudaError_t q = cudaEventQuery(it->second.done);
        if (q == cudaErrorNotReady) {
          ++it;
          continue;
        }
        ready.push_back(std::move(*it));
        it = s->inflight.erase(it);
      }
      if (ready.empty() && s->workers_done && s->inflight.empty()) return;
    }
    if (ready.empty()) {
      std::this_thread::sleep_for(std::chrono::microseconds(10));
      continue;
    }
    const auto now = Clock::now();
    for (auto& wb : ready) {
      sbmt_ctx* ctx = s->workers[wb.first].ctx;
      Batch& b = wb.second;
      std::vector<int> rcs;
      for (auto& r : b.reqs) {
        sbmt_mesh_view v{};
        rcs.push_back(mesh_query(ctx, r->mesh, -1, &v));
        r->view = v;
      }
      cudaEventDestroy(b.done);
      std::vector<sbmt_mesh> drop;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t k = 0; k < b.reqs.size(); ++k) {
          Req& r = *b.reqs[k];
          r.status = rcs[k], r.state = RQ_DONE, r.t_done = now;
          if (rcs[k] == SBMT_OK) ++s->n_completed;
          else ++s->n_failed;
          if (r.cancelled || rcs[k] != SBMT_OK) {
            drop.push_back(r.mesh);
            r.mesh = 0;
            give_back(s, r);
            if (r.cancelled) s->reqs.erase(r.id);
          }
        }
      }
      for (sbmt_mesh m : drop) mesh_release(ctx, m);
    }
    s->cv_done.notify_all();
  }
}

// free device memory as the admission check sees it (fault injection on
// the host: every oom_every-th check reports none)
size_t free_device_bytes(sbmt_server* s) {
  ++s->n_admit_checks;
  if (s->cfg.oom_every > 0 && s->n_admit_checks % s->cfg.oom_every == 0) return 0;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
  return fr;
}

void worker_loop(sbmt_server* s, int wi) {
  sbmt_server::Worker& w = s->workers[wi];
  cudaSetDevice(s->device);
  const int maxb = s->cfg.max_batch > 0 ? s->cfg.max_batch : 64;
  while (true) {
    std::vector<std::shared_ptr<Req>> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->queue.empty()) return;
      if (s->queue.empty()) {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      } else {
        // admission: requests in arrival order while their bounds fit the
        // budget and the free device memory; one that can never fit fails
        size_t take = 0;
        bool checked = false;
        size_t fr = 0;
        while (!s->queue.empty() && (int)batch.size() < maxb) {
          std::shared_ptr<Req> r = s->queue.front();
          if (r->cancelled) {
            s->queue.pop_front();
            continue;
          }
          if (r->bound > s->budget) {
            s->queue.pop_front();
            r->state = RQ_DONE, r->status = SBMT_ENOMEM, r->t_done = Clock::now();
            ++s->n_failed;
            s->cv_done.notify_all();
            continue;
          }
          if (!checked) fr = free_device_bytes(s), checked = true;
          if (s->reserved + r->bound > s->budget || take + r->bound > fr) {
            // with nothing else holding memory the free memory will not grow:
            // after many such checks (about a tenth of a second) it fails
            if (s->reserved == 0 && batch.empty() && ++r->starved > 1000) {
              s->queue.pop_front();
              r->state = RQ_DONE, r->status = SBMT_ENOMEM, r->t_done = Clock::now();
              ++s->n_failed;
              s->cv_done.notify_all();
            }
            break;
          }
          s->queue.pop_front();
          s->reserved += r->bound, r->reserved = r->bound, take += r->bound;
          s->peak = std::max(s->peak, s->reserved);
          r->state = RQ_RUNNING, r->worker = wi, r->t_admit = Clock::now();
          batch.push_back(r);
        }
      }
    }
    if (batch.empty()) {
      // nothing admitted (memory): try again in a moment
      std::this_thread::sleep_for(std::chrono::microseconds(50));
      continue;
    }
    const int n = (int)batch.size();
    std::vector<sbmt_image> im(n);
    std::vector<sbmt_params> pr(n);
    std::vector<sbmt_mesh> ids(n, 0);
    for (int k = 0; k < n; ++k) im[k] = batch[k]->img, pr[k] = batch[k]->pr;
    int rc = mesh_batch(w.ctx, im.data(), n, pr.data(), n, ids.data());
    std::vector<int> rcs(n, rc);
    if (rc != SBMT_OK && n > 1) {
      // isolate the failing request: each alone
      for (int k = 0; k < n; ++k) rcs[k] = mesh_batch(w.ctx, &im[k], 1, &pr[k], 1, &ids[k]);
    }
    Batch b;
    cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    cudaEventRecord(b.done, w.stream);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      ++s->n_batches;
      for (int k = 0; k < n; ++k) {
        Req& r = *batch[k];
        r.batch_size = n;
        if (rcs[k] != SBMT_OK) {
          r.state = RQ_DONE, r.status = rcs[k], r.t_done = Clock::now();
          ++s->n_failed;
          give_back(s, r);
          continue;
        }
        r.mesh = ids[k];
        // the exact device bytes of the mesh replace the bound
        size_t exact = 0;
        if (mesh_footprint(w.ctx, ids[k], &exact) == SBMT_OK && exact <= r.reserved) {
          s->reserved -= r.reserved - exact;
          r.reserved = exact;
        }
        b.reqs.push_back(batch[k]);
      }
    }
    s->cv_done.notify_all();
    if (b.reqs.empty()) {
      cudaEventDestroy(b.done);
      continue;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->inflight.push_back({wi, std::move(b)});
  }
}

}  // namespace

extern "C" {

const char* sbmt_server_last_error(void) { return g_srv_err.c_str(); }

int mesh_bound(const sbmt_image* img, const sbmt_params* params, size_t* bytes) {
  if (!bytes) return sfail(SBMT_EINVAL, "null argument");
  if (int rc = mesh_check(img, params)) return sfail(rc, sbmt_last_error());
  *bytes = request_bound(*img, *params);
  return SBMT_OK;
}

int server_create(sbmt_server** out, int device, const sbmt_server_config* cfg) {
  if (!out) return sfail(SBMT_EINVAL, "null server pointer");
  sbmt_server* s = new sbmt_server();
  s->device = device;
  if (cfg) s->cfg = *cfg;
  if (s->cfg.max_batch < 0 || s->cfg.workers < 0 || s->cfg.oom_every < 0) {
    delete s;
    return sfail(SBMT_EINVAL, "negative server setting");
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete s;
    return sfail(SBMT_ECUDA, "no such device");
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete s;
    return sfail(SBMT_ECUDA, "device memory query failed");
  }
  s->budget = s->cfg.hbm_budget ? s->cfg.hbm_budget : (size_t)(0.9 * (double)fr);
  const int nw = s->cfg.workers > 0 ? s->cfg.workers : 2;
  s->workers.resize(nw);
  for (auto& w : s->workers) {
    if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
        mesh_create(&w.ctx, device, 0, w.stream) != SBMT_OK) {
      for (auto& x : s->workers) {
        if (x.ctx) mesh_destroy(x.ctx);
        if (x.stream) cudaStreamDestroy(x.stream);
      }
      delete s;
      return sfail(SBMT_ECUDA, "worker context");
    }
  }
  for (int k = 0; k < nw; ++k) s->workers[k].th = std::thread(worker_loop, s, k);
  s->harvester = std::thread(harvest_loop, s);
  *out = s;
  return SBMT_OK;
}

int server_submit(sbmt_server* s, const sbmt_image* img, const sbmt_params* params, uint64_t* id) {
  if (!s || !img || !params || !id) return sfail(SBMT_EINVAL, "null argument");
  if (int rc = mesh_check(img, params)) return sfail(rc, sbmt_last_error());
  auto r = std::make_shared<Req>();
  r->img = *img, r->pr = *params;
  if (!img->on_device) {
    // the caller may reuse a host image once submit returns: keep a copy
    const size_t row = (size_t)img->width * img->dtype;
    r->host.resize(row * img->height);
    for (int y = 0; y < img->height; ++y)
      std::memcpy(r->host.data() + row * y, (const unsigned char*)img->data + (size_t)img->pitch_bytes * y, row);
    r->img.data = r->host.data(), r->img.pitch_bytes = (int64_t)row;
  }
  r->bound = request_bound(*img, *params);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return sfail(SBMT_EINVAL, "server stopping");
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    ++s->n_submitted;
    *id = r->id;
  }
  s->cv_work.notify_one();
  return SBMT_OK;
}

int server_wait(sbmt_server* s, uint64_t id, int wait_ms, sbmt_mesh_view* view, sbmt_request_info* info) {
  if (!s) return sfail(SBMT_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(SBMT_ENOENT, "unknown request");
  std::shared_ptr<Req> r = it->second;
  auto ready = [&] { return r->state == RQ_DONE; };
  if (!ready()) {
    if (wait_ms == 0) return SBMT_EPENDING;
    if (wait_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready)) return SBMT_ETIMEDOUT;
  }
  if (info) {
    info->status = r->status;
    info->batch_size = r->batch_size;
    info->queued_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
    info->total_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->t_admit.time_since_epoch().count() == 0) info->queued_ms = info->total_ms;
  }
  if (view) *view = r->view;
  return r->status == SBMT_OK ? SBMT_OK : sfail(r->status, "request failed");
}

int server_cancel(sbmt_server* s, uint64_t id) {
  if (!s) return sfail(SBMT_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(SBMT_ENOENT, "unknown request");
  Req& r = *it->second;
  if (r.state == RQ_QUEUED) {
    r.cancelled = true;
    r.state = RQ_DONE, r.status = SBMT_ECANCELED, r.t_done = Clock::now();
    ++s->n_cancelled;
    s->cv_done.notify_all();
    return SBMT_OK;
  }
  if (r.state == RQ_RUNNING) {
    // released as soon as its batch is done
    r.cancelled = true;
    ++s->n_cancelled;
    return SBMT_OK;
  }
  return sfail(SBMT_EINVAL, "request already finished");
}

int server_release(sbmt_server* s, uint64_t id) {
  if (!s) return sfail(SBMT_EINVAL, "null server");
  std::shared_ptr<Req> r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(SBMT_ENOENT, "unknown request");
    r = it->second;
    if (r->state != RQ_DONE) return sfail(SBMT_EPENDING, "request not finished");
    s->reqs.erase(it);
    give_back(s, *r);
  }
  if (r->mesh) mesh_release(s->workers[r->worker].ctx, r->mesh);
  return SBMT_OK;
}

int server_stats(sbmt_server* s, sbmt_server_stats* out) {
  if (!s || !out) return sfail(SBMT_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->n_submitted, out->completed = s->n_completed, out->failed = s->n_failed;
  out->cancelled = s->n_cancelled, out->batches = s->n_batches, out->queued = (int64_t)s->queue.size();
  out->reserved_bytes = (int64_t)s->reserved, out->peak_reserved_bytes = (int64_t)s->peak;
  out->budget_bytes = (int64_t)s->budget;
  return SBMT_OK;
}

int server_destroy(sbmt_server* s) {
  if (!s) return sfail(SBMT_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // queued requests are dropped
    for (auto& r : s->queue)
      if (r->state == RQ_QUEUED) r->state = RQ_DONE, r->status = SBMT_ECANCELED;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& w : s->workers)
    if (w.th.joinable()) w.th.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->workers_done = true;
  }
  if (s->harvester.joinable()) s->harvester.join();
  for (auto& w : s->workers) {
    mesh_destroy(w.ctx);
    cudaStreamDestroy(w.stream);
  }
  delete s;
  return SBMT_OK;
}

}  // extern "C"
