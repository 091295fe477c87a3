// Serving: continuous batching of fidelity(+gradient) solves on one GPU.
//
// Requests are admitted in arrival order while a slot is free and the device
// memory they need fits the budget.  Each slot owns a worker thread and a CUDA
// stream and runs one request's solve at a time, so the kernels of all admitted
// requests overlap on the device; a request that arrives while others run starts
// as soon as a slot and memory free up, without waiting for the running ones to
// finish.  A system has at most one request in the server at a time (the slot runs
// it with its own context and may prepare it).  Results are bitwise independent of what else runs: every
// solve uses only its own buffers and fixed-order reductions.
#include <cstdio>
#include "sg_internal.h"
#include "batcher.h"
#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

namespace {

constexpr int kServerMaxBatch = 16;

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Req {
  uint64_t ticket = 0;
  sg_system* sys = nullptr;
  sg_evolve_opts opts{};
  std::vector<long long> cols;
  std::vector<double> target;
  int kind = SG_FID_AVG;
  int want_grad = 1;
  size_t mem = 0;
  int state = 0;                 // 0 queued, 1 running, 2 done, 3 cancelled
  sg_status status = SG_OK;
  double F[2] = {0, 0};
  std::vector<double> gp, gh;
  double submit_s = 0, start_s = 0, done_s = 0;
  std::string error;
  std::string shape;             // requests of one shape may share batched launches
};

// The step shape of a request: everything its on-chip launches' plan and kernels
// depend on (modes and level counts, terms and their operators, drives and their
// envelope kinds, columns, precision, frame, step), not the parameter values or T.
std::string shape_key(const sg_system* sys, const sg_evolve_opts& o, const std::vector<long long>& cols, int kind,
                      int want_grad) {
  std::string k;
  auto add = [&](long long v) { k += std::to_string(v); k += ','; };
  add((long long)sys->modes.size());
  for (const HostMode& m : sys->modes) { add(m.kind); add(m.d); add(m.coupler); add((long long)m.local.size()); }
  add((long long)sys->couplings.size());
  for (const HostCoupling& c : sys->couplings) { add(c.a); add(c.op_a); add(c.b); add(c.op_b); }
  add((long long)sys->drives.size());
  for (const HostDrive& d : sys->drives) { add(d.mode); add(d.op); add(d.kind); add(d.nseg); }
  add((long long)sys->collapses.size());
  for (long long c : cols) add(c);
  add(o.precision); add(o.frame); add(o.solver); add(o.compensation); add(o.basis); add(kind); add(want_grad);
  char dt[40];
  std::snprintf(dt, sizeof dt, "%.17g", o.dt);
  k += dt;
  return k;
}

size_t estimate_bytes(const sg_system* sys, const sg_evolve_opts& o, int want_grad) {
  long long D = 1;
  for (const HostMode& m : sys->modes) D *= m.d;
  const double N = o.T / o.dt;
  size_t row = 0;
  for (const HostMode& m : sys->modes) row += (size_t)m.d * m.d;
  row += 2 * sys->couplings.size() * (size_t)SG_MAXD * SG_MAXD;
  const size_t slab = (size_t)D * o.ncols * sizeof(double2);
  size_t b = (size_t)(3.0 * N) * row * (sizeof(double2) + sizeof(float2)) + 8 * slab + (1u << 20);
  if (want_grad) {
    const size_t K = std::max<size_t>(1, (size_t)std::lround(std::sqrt(N)));
    b += (size_t)(N / K + 2) * slab + (K + 1) * slab + 10 * slab;
    b += (size_t)(3.0 * N) * sizeof(double) * std::max<size_t>(1, sys->drives.size());
  }
  return b;
}

}  // namespace

struct sg_server {
  sg_ctx* ctx = nullptr;
  size_t budget = 0;
  int max_slots = 1;
  // packing: a slot takes up to max_batch queued requests of one shape and runs them
  // together, their on-chip launches batched by the slot's batcher on its own stream;
  // bctx[w] holds the streams of the slot's other members
  int max_batch = 1;
  std::vector<OcBatcher*> batchers;
  std::vector<std::vector<sg_ctx*>> bctx;
  long long batches = 0, batched_requests = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Req*> queue;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  // systems with a request queued or running: a slot swaps the system's context and
  // may prepare it, so one system has at most one request in the server at a time
  std::map<const sg_system*, int> inflight;
  uint64_t next_ticket = 1;
  size_t mem_in_use = 0;
  int active = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<sg_ctx*> wctx;
  uint64_t submitted = 0, completed = 0, cancelled = 0, rejected = 0;
  std::vector<double> latencies;
  double first_start = -1, last_done = 0;
  double busy_accum = 0, busy_since = -1;

  // One request's solve on context c (its stream), through batcher bt when non-null.
  void run_one(sg_ctx* c, Req* r, OcBatcher* bt) {
    if (bt) onchip_batcher_bind(bt);
    sg_ctx* saved = r->sys->ctx;
    r->sys->ctx = c;
    sg_status rc = SG_OK;
    if (!r->sys->prepared) rc = sg_prepare_impl(r->sys);
    int np = 0, nh = 0;
    sg_param_counts(r->sys, &np, &nh);
    r->gp.assign(std::max(1, np), 0.0);
    r->gh.assign(std::max(1, nh), 0.0);
    if (rc == SG_OK)
      rc = sg_fidelity_impl(r->sys, &r->opts, r->target.data(), r->kind, r->F, nullptr,
                            r->want_grad != 0, r->gp.data(), r->gh.data(), 0);
    onchip_batcher_release();                   // every exit path leaves the batch
    r->sys->ctx = saved;
    r->status = rc;
    if (rc != SG_OK) r->error = c->last_error;
  }

  void worker(int w) {
    sg_ctx* c = wctx[w];
    for (;;) {
      std::vector<Req*> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
          if (stop) return true;
          return !queue.empty() && mem_in_use + queue.front()->mem <= budget;
        });
        if (stop) return;
        Req* r0 = queue.front();
        queue.pop_front();
        batch.push_back(r0);
        mem_in_use += r0->mem;
        // same-shape requests queued behind it join its batch while memory allows,
        // those with the step count closest to its own first (a shared launch runs
        // to its longest member's end)
        if (max_batch > 1) {
          std::vector<std::pair<double, Req*>> cand;
          const double n0 = r0->opts.T / r0->opts.dt;
          for (Req* r : queue)
            if (r->shape == r0->shape) cand.push_back({std::fabs(r->opts.T / r->opts.dt - n0), r});
          std::stable_sort(cand.begin(), cand.end(),
                           [](const std::pair<double, Req*>& a, const std::pair<double, Req*>& b) {
                             return a.first < b.first;
                           });
          for (const auto& c : cand) {
            if ((int)batch.size() >= max_batch) break;
            if (mem_in_use + c.second->mem > budget) continue;
            batch.push_back(c.second);
            mem_in_use += c.second->mem;
            queue.erase(std::find(queue.begin(), queue.end(), c.second));
          }
        }
        const double t = now_s(t0);
        if (active == 0) busy_since = t;
        active += (int)batch.size();
        if (first_start < 0) first_start = t;
        for (Req* r : batch) { r->state = 1; r->start_s = t; }
        if (batch.size() > 1) { ++batches; batched_requests += (long long)batch.size(); }
      }
      if (batch.size() == 1) {
        run_one(c, batch[0], nullptr);
      } else {
        OcBatcher* bt = batchers[w];
        onchip_batcher_join(bt, (int)batch.size());
        std::vector<std::thread> th;
        for (size_t i = 1; i < batch.size(); ++i)
          th.emplace_back([this, w, i, bt, &batch] {
            cudaSetDevice(bctx[w][i - 1]->device);
            run_one(bctx[w][i - 1], batch[i], bt);
          });
        run_one(c, batch[0], bt);
        for (auto& t : th) t.join();
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        const double t = now_s(t0);
        for (Req* r : batch) {
          r->done_s = t;
          r->state = 2;
          mem_in_use -= r->mem;
          --active;
          ++completed;
          inflight.erase(r->sys);
          latencies.push_back(r->done_s - r->submit_s);
        }
        if (active == 0 && busy_since >= 0) { busy_accum += t - busy_since; busy_since = -1; }
        last_done = t;
      }
      cv.notify_all();
      done_cv.notify_all();
    }
  }
};

extern "C" {

sg_status sg_server_create(sg_ctx* ctx, size_t mem_budget_bytes, int max_slots, sg_server** out) {
  if (!ctx || !out) return SG_E_INVALID;
  if (max_slots < 1 || max_slots > 64) return sg_fail(ctx, SG_E_INVALID, "max_slots must be 1..64");
  if (mem_budget_bytes == 0) return sg_fail(ctx, SG_E_INVALID, "memory budget must be > 0");
  sg_server* s = new sg_server();
  s->ctx = ctx;
  s->budget = mem_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  cudaSetDevice(ctx->device);
  for (int w = 0; w < max_slots; ++w) {
    sg_ctx* c = new sg_ctx();
    c->device = ctx->device;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      for (sg_ctx* x : s->wctx) { cudaStreamDestroy(x->stream); delete x; }
      delete s;
      return sg_fail(ctx, SG_E_CUDA, "cudaStreamCreate failed");
    }
    s->wctx.push_back(c);
  }
  for (int w = 0; w < max_slots; ++w)
    s->workers.emplace_back([s, w] { cudaSetDevice(s->wctx[w]->device); s->worker(w); });
  *out = s;
  return SG_OK;
}

sg_status sg_server_destroy(sg_server* srv) {
  if (!srv) return SG_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  for (auto& t : srv->workers) t.join();
  for (sg_ctx* c : srv->wctx) { cudaStreamSynchronize(c->stream); cudaStreamDestroy(c->stream); delete c; }
  for (auto& v : srv->bctx)
    for (sg_ctx* c : v) { cudaStreamSynchronize(c->stream); cudaStreamDestroy(c->stream); delete c; }
  for (OcBatcher* b : srv->batchers) onchip_batcher_destroy(b);
  delete srv;
  return SG_OK;
}

sg_status sg_server_set_batch(sg_server* srv, int max_batch) {
  if (!srv) return SG_E_INVALID;
  if (max_batch < 1 || max_batch > kServerMaxBatch)
    return sg_fail(srv->ctx, SG_E_INVALID, "max_batch must be 1.." + std::to_string(kServerMaxBatch));
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->submitted > srv->completed + srv->cancelled + srv->rejected)
    return sg_fail(srv->ctx, SG_E_STATE, "set the batch size while no request is queued or running");
  cudaSetDevice(srv->ctx->device);
  if (srv->batchers.empty()) srv->batchers.assign(srv->max_slots, nullptr);
  srv->bctx.resize(srv->max_slots);
  for (int w = 0; w < srv->max_slots; ++w) {
    if (max_batch > 1 && !srv->batchers[w]) {
      srv->batchers[w] = onchip_batcher_create(srv->ctx->device);
      if (!srv->batchers[w]) return sg_fail(srv->ctx, SG_E_CUDA, "stream creation for the batched launches failed");
    }
    while ((int)srv->bctx[w].size() < max_batch - 1) {
      sg_ctx* c = new sg_ctx();
      c->device = srv->ctx->device;
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return sg_fail(srv->ctx, SG_E_CUDA, "cudaStreamCreate failed");
      }
      srv->bctx[w].push_back(c);
    }
  }
  srv->max_batch = max_batch;
  return SG_OK;
}

sg_status sg_server_submit(sg_server* srv, const sg_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return SG_E_INVALID;
  if (!req->sys || !req->target_re_im) return sg_fail(srv->ctx, SG_E_INVALID, "request needs a system and a target");
  auto r = std::make_unique<Req>();
  r->sys = req->sys;
  r->opts = req->opts;
  r->kind = req->kind;
  r->want_grad = req->want_grad;
  const int nq = (int)req->sys->modes.size();
  int nqb = 0;
  for (const HostMode& m : req->sys->modes) nqb += m.coupler ? 0 : 1;
  if (nq < 1 || nq > SG_MAXQ || nqb < 1 || nqb > 12)
    return sg_fail(srv->ctx, SG_E_INVALID, "request system needs 1..12 qubit modes");
  if (req->opts.col_index) {
    r->cols.assign(req->opts.col_index, req->opts.col_index + req->opts.ncols);
  } else {
    // every computational state: qubit modes in {0, 1} (first qubit most significant),
    // couplers in level 0
    for (int j = 0; j < (1 << nqb); ++j) {
      long long row = 0;
      int b = nqb - 1;
      for (const HostMode& m : req->sys->modes) row = row * m.d + (m.coupler ? 0 : (j >> b--) & 1);
      r->cols.push_back(row);
    }
    r->opts.ncols = (int)r->cols.size();
  }
  r->opts.col_index = r->cols.data();
  const size_t dc = (size_t)1 << nqb;
  r->target.assign(req->target_re_im, req->target_re_im + 2 * dc * dc);
  r->mem = estimate_bytes(req->sys, r->opts, req->want_grad);
  r->shape = shape_key(req->sys, r->opts, r->cols, r->kind, r->want_grad);
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->inflight.count(req->sys))
    return sg_fail(srv->ctx, SG_E_STATE, "this system already has a request queued or running in the server; "
                                         "give each concurrent request its own system");
  ++srv->submitted;
  if (r->mem > srv->budget) {
    ++srv->rejected;
    return sg_fail(srv->ctx, SG_E_NOMEM_RETRY, "request alone exceeds the memory budget");
  }
  srv->inflight[req->sys] = 1;
  r->ticket = srv->next_ticket++;
  r->submit_s = now_s(srv->t0);
  *ticket = r->ticket;
  srv->queue.push_back(r.get());
  srv->reqs[r->ticket] = std::move(r);
  srv->cv.notify_all();
  return SG_OK;
}

static sg_status fill_result(Req* r, sg_result* out) {
  if (!out) return SG_OK;
  out->status = r->status;
  out->F[0] = r->F[0];
  out->F[1] = r->F[1];
  out->grad_pulse = r->gp.data();
  out->grad_ham = r->gh.data();
  int np = 0, nh = 0;
  sg_param_counts(r->sys, &np, &nh);
  out->n_pulse = np;
  out->n_ham = nh;
  out->submit_s = r->submit_s;
  out->start_s = r->start_s;
  out->done_s = r->done_s;
  std::snprintf(out->error, sizeof out->error, "%s", r->error.c_str());
  return SG_OK;
}

sg_status sg_server_poll(sg_server* srv, uint64_t ticket, sg_result* out) {
  if (!srv) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return sg_fail(srv->ctx, SG_E_NOTFOUND, "unknown ticket");
  Req* r = it->second.get();
  if (r->state == 3) return SG_E_CANCELLED;
  if (r->state != 2) return SG_E_PENDING;
  return fill_result(r, out);
}

sg_status sg_server_wait(sg_server* srv, uint64_t ticket, sg_result* out) {
  if (!srv) return SG_E_INVALID;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return sg_fail(srv->ctx, SG_E_NOTFOUND, "unknown ticket");
  Req* r = it->second.get();
  srv->done_cv.wait(lk, [&] { return r->state >= 2; });
  if (r->state == 3) return SG_E_CANCELLED;
  return fill_result(r, out);
}

sg_status sg_server_cancel(sg_server* srv, uint64_t ticket) {
  if (!srv) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return sg_fail(srv->ctx, SG_E_NOTFOUND, "unknown ticket");
  Req* r = it->second.get();
  if (r->state != 0) return r->state == 3 ? SG_OK : sg_fail(srv->ctx, SG_E_STATE, "request already started");
  srv->queue.erase(std::remove(srv->queue.begin(), srv->queue.end(), r), srv->queue.end());
  srv->inflight.erase(r->sys);
  r->state = 3;
  ++srv->cancelled;
  srv->done_cv.notify_all();
  return SG_OK;
}

sg_status sg_server_stats(sg_server* srv, sg_stats* out) {
  if (!srv || !out) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->cancelled = srv->cancelled;
  out->rejected = srv->rejected;
  double span = srv->first_start >= 0 ? srv->last_done - srv->first_start : 0.0;
  out->solves_per_s = span > 0 ? srv->completed / span : 0.0;
  std::vector<double> l = srv->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(l.size() - 1, std::ceil(p * l.size()) - 1);
    return l[i];
  };
  out->p50_s = pct(0.50);
  out->p99_s = pct(0.99);
  double busy = srv->busy_accum;
  double nowt = now_s(srv->t0);
  if (srv->busy_since >= 0) busy += nowt - srv->busy_since;
  out->gpu_busy_frac = srv->first_start >= 0 ? busy / std::max(1e-9, nowt - srv->first_start) : 0.0;
  out->mem_in_use = srv->mem_in_use;
  out->mem_budget = srv->budget;
  out->active_slots = srv->active;
  out->max_slots = srv->max_slots;
  out->batches = srv->batches;
  out->batched_requests = srv->batched_requests;
  long long bl = 0, bm = 0;
  for (OcBatcher* b : srv->batchers) {
    if (!b) continue;
    long long l = 0, m = 0;
    onchip_batcher_stats(b, &l, &m);
    bl += l;
    bm += m;
  }
  out->batched_launches = bl;
  out->batched_launch_members = bm;
  return SG_OK;
}

}  // extern "C"
