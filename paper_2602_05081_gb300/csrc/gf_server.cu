// gf_server.cu -- render server: continuous batching of scattering renders
// over resident fields (the gf_server_* entry points of include/gf.h).
//
// Host side, native C++.  A scheduler thread owns the device work:
//   admit   requests leave the arrival queue in order when a slot is free and
//           their framebuffer fits the device pool (first-fit allocator);
//   batch   every admitted request with pixels left gets an equal share of
//           the launch's sample budget (water-filling: requests that need
//           less than the share free the rest for the others), as its next
//           contiguous pixel range;
//   launch  one k_render_server launch renders every range of the batch, in
//           units of up to 8 consecutive samples of one pixel (so a 64-spp
//           request spreads over 8 times as many lanes as pixels), summed in
//           64-bit fixed point per pixel;
//           two launches stay in flight on two streams, so the blocks of the
//           next launch fill the SMs that the previous launch's tail frees;
//   retire  when a launch's event completes, its ranges are done; a request
//           whose last range is done has its sums turned into the image (sum
//           / spp) and copied to the caller's buffer, then releases its
//           memory and slot.
// Requests that arrive while launches run join the next launch: the batch is
// re-formed at every launch (iteration-level scheduling), never drained.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gf_host.h"
#include "gf_pool.h"

using namespace gf;

namespace {

constexpr int kBatches = 2;        // launches in flight
constexpr size_t kHead = 1024;     // counter | error word | work counters
constexpr size_t kErrOff = 256, kStatsOff = 512;
constexpr int kMinRangePix = 32;
constexpr int kUnitSamples = 8;    // samples per work unit of a lane

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Req {
  uint64_t ticket = 0;
  gf_request r{};
  ServerReqDev dev{};
  int state = GF_REQ_QUEUED;
  int status = GF_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t npix = 0, next_pix = 0, outstanding = 0, launches = 0;
  size_t fb_off = 0, fb_bytes = 0;  // pool block: fixed-point sums, then the float image
  float* fb = nullptr;
  bool copying = false;
  cudaEvent_t copy_ev = nullptr;
};

struct Batch {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  unsigned char* host = nullptr;  // pinned mirror of dev
  unsigned char* dev = nullptr;   // [head | items | reqs]
  size_t items_off = 0, reqs_off = 0;
  DevField* fields = nullptr;     // the assets' views; err/stats -> this batch's head
  float4* store = nullptr;        // per-warp chord store of the launch
  bool busy = false;
  std::vector<Req*> members;
};

gf_status status_of_err(int err) {
  if (err & (ERR_STACK | ERR_WINDOW | ERR_POINTS)) return GF_EOVERFLOW;
  if (err & ERR_GUARD) return GF_ETIMEOUT;
  if (err & ERR_INDEX) return GF_ECUDA;
  return GF_EINVAL;
}

}  // namespace

struct gf_server {
  Ctx ctx;
  DevMem mem;                   // device buffers, through the context's allocator
  std::vector<DevField> views;  // per asset, as given (host copies)
  std::vector<const Field*> fields;
  gf_server_opts opts{};
  int64_t max_n = 0;
  int64_t grid = 1;
  float* pool_mem = nullptr;
  Pool pool;
  Batch batches[kBatches];
  cudaStream_t copy_stream = nullptr;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::vector<Req*> running;  // admitted, in admission order
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  gf_server_stats st{};

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }

  void fail_req(Req* r, int status) {
    if (r->state == GF_REQ_DONE || r->state == GF_REQ_FAILED) return;
    r->status = status;
    if (r->outstanding > 0 || r->copying) return;  // finished when its launches retire
    if (r->state == GF_REQ_RUNNING) release(r);
    r->state = GF_REQ_FAILED;
    r->t_done = now_ms();
    st.failed += 1;
    cv_done.notify_all();
  }

  void release(Req* r) {
    pool.release(r->fb_off, r->fb_bytes);
    running.erase(std::find(running.begin(), running.end(), r));
  }

  // admit from the head of the queue while a slot and pool memory are free
  void admit() {
    while (!queue.empty() && (int)running.size() < opts.max_inflight) {
      Req* r = queue.front();
      size_t off = 0;
      if (!pool.alloc(r->fb_bytes, off)) break;
      queue.pop_front();
      r->fb_off = off;
      unsigned char* base = reinterpret_cast<unsigned char*>(pool_mem) + off;
      r->dev.acc = reinterpret_cast<unsigned long long*>(base);
      r->fb = reinterpret_cast<float*>(base + align256((size_t)r->npix * 8));
      r->state = GF_REQ_RUNNING;
      r->t_admit = now_ms();
      running.push_back(r);
      st.max_inflight_seen = std::max(st.max_inflight_seen, (int)running.size());
      st.max_bytes_seen = std::max(st.max_bytes_seen, (int64_t)pool.used());
    }
  }

  // form and launch one batch on b; false if no admitted request has pixels left
  bool launch(Batch& b) {
    std::vector<Req*> act;
    for (Req* r : running)
      if (r->status == GF_OK && r->next_pix < r->npix) act.push_back(r);
    if (act.empty()) return false;
    // equal shares of the sample budget, water-filled over the demands
    const size_t n = act.size();
    std::vector<int64_t> demand(n), give(n, 0);
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) {
      demand[i] = (act[i]->npix - act[i]->next_pix) * (int64_t)act[i]->dev.P.spp;
      order[i] = i;
    }
    std::sort(order.begin(), order.end(), [&](size_t a, size_t c) { return demand[a] < demand[c]; });
    int64_t budget = opts.batch_samples;
    for (size_t k = 0; k < n; ++k) {
      const size_t i = order[k];
      const int64_t share = budget / (int64_t)(n - k);
      give[i] = std::min(demand[i], std::max<int64_t>(share, 1));
      budget -= give[i];
      if (budget < 0) budget = 0;
    }
    ServerItem* items = reinterpret_cast<ServerItem*>(b.host + b.items_off);
    ServerReqDev* rq = reinterpret_cast<ServerReqDev*>(b.host + b.reqs_off);
    int total = 0;
    b.members.clear();
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < n; ++i) {
      Req* r = act[i];
      const int64_t spp = r->dev.P.spp;
      int64_t pix = (give[i] + spp - 1) / spp;
      pix = std::max<int64_t>(kMinRangePix, (pix + kMinRangePix - 1) / kMinRangePix * kMinRangePix);
      pix = std::min(pix, r->npix - r->next_pix);
      items[i].req = (int)i;
      items[i].pix0 = (int)r->next_pix;
      items[i].npix = (int)pix;
      items[i].base = total;
      total += (int)(pix * r->dev.nchunk);
      // the request's sums start at zero, before its first range is rendered
      if (r->launches == 0 && e == cudaSuccess)
        e = cudaMemsetAsync(r->dev.acc, 0, (size_t)r->npix * 8, b.stream);
      rq[i] = r->dev;
      r->next_pix += pix;
      r->outstanding += 1;
      r->launches += 1;
      b.members.push_back(r);
    }
    std::memset(b.host, 0, kHead);
    const size_t up = b.reqs_off + n * sizeof(ServerReqDev);
    ServerLaunch L;
    L.fields = b.fields;
    L.max_n = max_n;
    L.items = reinterpret_cast<const ServerItem*>(b.dev + b.items_off);
    L.n_items = (int)n;
    L.total = total;
    L.reqs = reinterpret_cast<const ServerReqDev*>(b.dev + b.reqs_off);
    L.counter = reinterpret_cast<int*>(b.dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.dev, b.host, up, cudaMemcpyHostToDevice, b.stream);
    if (e == cudaSuccess) e = cudaEventRecord(b.start, b.stream);
    if (e == cudaSuccess) e = launch_render_server(L, std::min<int64_t>(grid, (total + 127) / 128), b.store, b.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b.host + kErrOff, b.dev + kErrOff, kHead - kErrOff, cudaMemcpyDeviceToHost,
                          b.stream);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, b.stream);
    b.busy = true;
    st.launches += 1;
    st.items += (int64_t)n;
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      b.busy = false;
      for (Req* r : b.members) {
        r->outstanding -= 1;
        fail_req(r, GF_ECUDA);
      }
      b.members.clear();
    }
    return true;
  }

  void finish_copy(Req* r) {
    r->copying = false;
    release(r);
    if (r->status != GF_OK) {
      r->state = GF_REQ_FAILED;
      st.failed += 1;
    } else {
      r->state = GF_REQ_DONE;
      st.completed += 1;
    }
    r->t_done = now_ms();
    cv_done.notify_all();
  }

  void retire(Batch& b, bool ok) {
    b.busy = false;
    int err = 0;
    if (ok) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, b.start, b.done) == cudaSuccess) st.busy_ms += ms;
      std::memcpy(&err, b.host + kErrOff, sizeof(int));
      unsigned long long w[kNumStats];
      std::memcpy(w, b.host + kStatsOff, sizeof(w));
      st.work.rays += w[ST_RAYS];
      st.work.chords += w[ST_CHORDS];
      st.work.evals += w[ST_EVALS];
      st.work.nodes += w[ST_NODES];
      st.work.points += w[ST_POINTS];
      st.work.windows += w[ST_WINDOWS];
      st.work.steps += w[ST_STEPS];
      st.work.leaves += w[ST_LEAVES];
    }
    const int status = !ok ? GF_ECUDA : err ? status_of_err(err) : GF_OK;
    for (Req* r : b.members) {
      r->outstanding -= 1;
      if (status != GF_OK && r->status == GF_OK) r->status = status;
      if (r->outstanding > 0) continue;
      if (r->status != GF_OK) {
        if (r->state == GF_REQ_RUNNING) {
          release(r);
          r->state = GF_REQ_FAILED;
          r->t_done = now_ms();
          st.failed += 1;
          cv_done.notify_all();
        }
        continue;
      }
      if (r->next_pix < r->npix) continue;
      // last range done: sums -> image, copied out, then release
      cudaError_t e = launch_fix_to_image(r->dev.acc, r->npix, r->dev.P.spp, r->fb, copy_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->r.out, r->fb, (size_t)r->npix * 4, cudaMemcpyDefault, copy_stream);
      if (e == cudaSuccess) e = cudaEventRecord(r->copy_ev, copy_stream);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        r->status = GF_ECUDA;
        finish_copy(r);
        continue;
      }
      r->copying = true;
    }
    b.members.clear();
  }

  bool any_busy() const {
    for (const Batch& b : batches)
      if (b.busy) return true;
    return false;
  }

  void run() {
    cudaSetDevice(ctx.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progress = false;
      for (Batch& b : batches) {
        if (!b.busy) continue;
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaSuccess) {
          retire(b, true);
          progress = true;
        } else if (q != cudaErrorNotReady) {
          (void)cudaGetLastError();
          retire(b, false);
          progress = true;
        }
      }
      for (size_t i = 0; i < running.size();) {
        Req* r = running[i];
        if (r->copying) {
          const cudaError_t q = cudaEventQuery(r->copy_ev);
          if (q != cudaErrorNotReady) {
            if (q != cudaSuccess) {
              (void)cudaGetLastError();
              r->status = GF_ECUDA;
            }
            finish_copy(r);  // removes r from running
            progress = true;
            continue;
          }
        }
        ++i;
      }
      if (stop) {
        while (!queue.empty()) {
          Req* r = queue.front();
          queue.pop_front();
          r->state = GF_REQ_FAILED;
          r->status = GF_ESTATE;
          r->t_done = now_ms();
          st.failed += 1;
        }
        cv_done.notify_all();
      }
      admit();
      for (Batch& b : batches) {
        if (b.busy) continue;
        if (launch(b)) progress = true;
        break;  // at most one new launch per round: retire first
      }
      if (stop && queue.empty() && running.empty() && !any_busy()) break;
      if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
  }
};

namespace {

gf_status fail_cuda(cudaError_t e, const char* where) {
  (void)cudaGetLastError();
  return report(e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

void free_server(gf_server* S) {
  cudaDeviceSynchronize();  // no launch or copy of the server is in flight
  for (Batch& b : S->batches) {
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.start) cudaEventDestroy(b.start);
    if (b.done) cudaEventDestroy(b.done);
    if (b.host) cudaFreeHost(b.host);  // pinned host mirror (host memory)
  }
  for (auto& kv : S->reqs)
    if (kv.second->copy_ev) cudaEventDestroy(kv.second->copy_ev);
  if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
  S->mem.release_all();  // pool, batch buffers, field views, chord stores
  delete S;
}

}  // namespace

extern "C" {

gf_status gf_server_create(gf_ctx* ctx, gf_field* const* fields, int n_fields,
                           const gf_server_opts* opts, gf_server** out) {
  if (!ctx || !fields || !opts || !out) return report(GF_EINVAL, "null argument");
  *out = nullptr;
  if (n_fields < 1 || n_fields > 64) return report(GF_EINVAL, "n_fields in [1, 64]");
  if (opts->max_inflight < 1 || opts->max_inflight > 1024) return report(GF_EINVAL, "max_inflight in [1, 1024]");
  if (opts->max_queue < 1) return report(GF_EINVAL, "max_queue >= 1");
  if (opts->mem_budget < 256) return report(GF_EINVAL, "mem_budget too small");
  if (opts->batch_samples < 0 || opts->batch_samples > (1ll << 30))
    return report(GF_EINVAL, "batch_samples in [0, 2^30]");
  for (int i = 0; i < n_fields; ++i) {
    if (!fields[i]) return report(GF_EINVAL, "null field");
    if (!fields[i]->f.built) return report(GF_ESTATE, "field not built");
    if (fields[i]->f.camera_lod)
      return report(GF_ESTATE, "field has a camera LoD selection (requests carry their cameras)");
    if (fields[i]->f.ctx.device != ctx->c.device) return report(GF_EINVAL, "field of another device");
  }
  cudaError_t e = cudaSetDevice(ctx->c.device);
  if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
  gf_server* S = new gf_server;
  S->ctx = ctx->c;
  S->mem.ctx = ctx->c;
  S->opts = *opts;
  S->opts.mem_budget = opts->mem_budget & ~size_t(255);
  for (int i = 0; i < n_fields; ++i) {
    S->fields.push_back(&fields[i]->f);
    S->views.push_back(fields[i]->f.dev);
    S->max_n = std::max(S->max_n, fields[i]->f.n);
  }
  if ((e = server_grid(S->ctx.sm_count, S->grid)) != cudaSuccess) {
    free_server(S);
    return fail_cuda(e, "occupancy");
  }
  // about four units of kUnitSamples samples per resident lane
  if (S->opts.batch_samples == 0) S->opts.batch_samples = S->grid * 128 * 4 * kUnitSamples;
  if ((e = S->mem.get(&S->pool_mem, S->opts.mem_budget, nullptr)) != cudaSuccess) {
    free_server(S);
    return fail_cuda(e, "framebuffer pool");
  }
  S->pool.init(S->opts.mem_budget);
  if ((e = cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    free_server(S);
    return fail_cuda(e, "copy stream");
  }
  const size_t items_off = kHead;
  const size_t reqs_off = align256(items_off + (size_t)S->opts.max_inflight * sizeof(ServerItem));
  const size_t bytes = reqs_off + (size_t)S->opts.max_inflight * sizeof(ServerReqDev);
  for (Batch& b : S->batches) {
    b.items_off = items_off;
    b.reqs_off = reqs_off;
    if ((e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&b.start)) != cudaSuccess || (e = cudaEventCreate(&b.done)) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&b.host, bytes, cudaHostAllocDefault)) != cudaSuccess ||
        (e = S->mem.get(&b.dev, bytes, b.stream)) != cudaSuccess ||
        (e = S->mem.get(&b.fields, sizeof(DevField) * n_fields, b.stream)) != cudaSuccess ||
        (e = S->mem.get(&b.store, scatter_store_bytes(S->grid), b.stream)) != cudaSuccess) {
      free_server(S);
      return fail_cuda(e, "server buffers");
    }
    std::vector<DevField> v = S->views;
    for (DevField& d : v) {
      d.err = reinterpret_cast<int*>(b.dev + kErrOff);
      d.stats = reinterpret_cast<unsigned long long*>(b.dev + kStatsOff);
    }
    if ((e = cudaMemcpy(b.fields, v.data(), sizeof(DevField) * n_fields, cudaMemcpyHostToDevice)) !=
        cudaSuccess) {
      free_server(S);
      return fail_cuda(e, "field views");
    }
  }
  S->t0 = std::chrono::steady_clock::now();
  S->worker = std::thread([S] { S->run(); });
  for (const Field* f : S->fields) ++const_cast<Field*>(f)->server_refs;
  *out = S;
  return GF_OK;
}

gf_status gf_server_submit(gf_server* S, const gf_request* rq, uint64_t* ticket) {
  if (!S || !rq || !ticket) return report(GF_EINVAL, "null argument");
  if (rq->asset < 0 || rq->asset >= (int)S->fields.size()) return report(GF_EINVAL, "bad asset index");
  if (!rq->out) return report(GF_EINVAL, "out null");
  if (rq->opts.integrator != GF_INTEG_SCATTER) return report(GF_EINVAL, "the server renders GF_INTEG_SCATTER");
  if (rq->opts.free_flight != GF_FLIGHT_DELTA) return report(GF_EINVAL, "the server renders GF_FLIGHT_DELTA");
  if (!lod_ok(&rq->lod) || !lod_ok(&rq->lod_nee)) return report(GF_EINVAL, "bad lod descriptor");
  auto r = std::make_unique<Req>();
  gf_status s = camera_params(&rq->camera, &rq->opts, rq->seed, *S->fields[rq->asset], r->dev.P);
  if (s != GF_OK) return s;
  r->dev.P.lod = lod_dev(rq->lod);
  r->dev.P.lod_nee = lod_dev(rq->lod_nee);
  r->dev.asset = rq->asset;
  r->r = *rq;
  r->npix = (int64_t)rq->camera.width * rq->camera.height;
  r->fb_bytes = align256((size_t)r->npix * 8) + align256((size_t)r->npix * 4);
  r->dev.chunk = std::min(r->dev.P.spp, kUnitSamples);
  r->dev.nchunk = (r->dev.P.spp + r->dev.chunk - 1) / r->dev.chunk;
  if (r->fb_bytes > S->opts.mem_budget) return report(GF_EINVAL, "framebuffer larger than the pool");
  if (r->npix > (1ll << 30)) return report(GF_EINVAL, "image too large");
  cudaError_t e = cudaSetDevice(S->ctx.device);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->copy_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return fail_cuda(e, "request event");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    cudaEventDestroy(r->copy_ev);
    return report(GF_ESTATE, "server stopping");
  }
  if ((int)S->queue.size() >= S->opts.max_queue) {
    cudaEventDestroy(r->copy_ev);
    return report(GF_EOVERFLOW, "request queue full");
  }
  r->ticket = S->next_ticket++;
  r->t_submit = S->now_ms();
  *ticket = r->ticket;
  S->queue.push_back(r.get());
  S->reqs.emplace(r->ticket, std::move(r));
  S->st.submitted += 1;
  S->cv_work.notify_all();
  return GF_OK;
}

static void fill_result(const Req& r, gf_result* out) {
  out->state = r.state;
  out->status = r.status;
  out->t_submit_ms = r.t_submit;
  out->t_admit_ms = r.t_admit;
  out->t_done_ms = r.t_done;
  out->launches = r.launches;
}

gf_status gf_server_poll(gf_server* S, uint64_t ticket, gf_result* out) {
  if (!S || !out) return report(GF_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return report(GF_EINVAL, "unknown ticket");
  fill_result(*it->second, out);
  return GF_OK;
}

gf_status gf_server_wait(gf_server* S, uint64_t ticket, double timeout_ms, gf_result* out) {
  if (!S || !out) return report(GF_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return report(GF_EINVAL, "unknown ticket");
  Req* r = it->second.get();
  const auto until = std::chrono::steady_clock::now() +
                     std::chrono::microseconds((int64_t)(std::max(0.0, timeout_ms) * 1000.0));
  const bool fin = S->cv_done.wait_until(lk, until, [r] {
    return r->state == GF_REQ_DONE || r->state == GF_REQ_FAILED;
  });
  fill_result(*r, out);
  if (!fin) return report(GF_ETIMEOUT, "request not finished");
  return GF_OK;
}

gf_status gf_server_get_stats(gf_server* S, gf_server_stats* out) {
  if (!S || !out) return report(GF_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  return GF_OK;
}

gf_status gf_server_destroy(gf_server* S) {
  if (!S) return report(GF_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (const Field* f : S->fields) --const_cast<Field*>(f)->server_refs;
  cudaSetDevice(S->ctx.device);
  free_server(S);
  return GF_OK;
}

}  // extern "C"
