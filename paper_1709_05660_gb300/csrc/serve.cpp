// Continuous-batching server for Newton-step requests (the serving form of
// the solver): worker threads with their own CUDA streams pick the oldest
// runnable request - an instance not already running, admitted by planned
// device bytes against the budget (evicting idle instances to the host when
// the oldest waiting request does not fit) - and run one fsi_newton_step on
// that instance's resident hierarchy.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fsi.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Instance {
  fsi_ctx* ctx = nullptr;
  int64_t bytes = 0;
  bool busy = false;
  int64_t n = 0;
  int failed = 0;                  // error of an earlier step that freed the instance
  bool batchable = false;          // mixed precision with >= 2 levels: may share a factorisation launch
  // eviction under memory pressure: a steady instance that is idle and has no
  // queued request may be evicted (state kept on the host, hierarchy freed)
  // and is rebuilt from that state when its next request is admitted
  bool steady = false;
  bool evicted = false;
  std::vector<double> saved_y;
  fsi_problem_desc desc{};
  fsi_solver_opts opts{};
  uint64_t last_use = 0;
  bool free_after = false;         // its last request was cancelled while a step ran
};

struct Ticket {
  uint64_t id = 0;
  fsi_request req{};
  std::vector<double> noise;       // copy of the first request's noise
  std::vector<double> dx;          // kept update (keep_dx)
  fsi_result res{};
  Clock::time_point t_submit, t_start, t_end;
  int state = 0;                   // 0 queued, 1 running, 2 done
  int64_t planned = 0;             // planned bytes when the request creates the instance
  int64_t reserved = 0;            // bytes reserved at admission (new or evicted instance)
};

double ms(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct fsi_server {
  int64_t budget = 0;
  int64_t resident = 0;
  int max_batch = 4;                   // requests that may share one Schwarz factorisation launch
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Ticket*> queue;
  std::map<uint64_t, std::unique_ptr<Ticket>> tickets;
  std::map<uint64_t, Instance> inst;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;   // one per worker; destroyed after the instances
  uint64_t next = 1;
  uint64_t use_clock = 0;
  int64_t evictions = 0;
  bool evict = true;                   // evict idle instances when a request does not fit
  int running = 0;
  bool stop = false;

  // device bytes a ticket needs to be admitted: the planned size of a new
  // instance, the size of an evicted one, nothing for a resident one
  int64_t need(const Ticket* t, std::map<uint64_t, Instance>::iterator f) {
    if (f == inst.end()) return t->planned;
    const Instance& in = f->second;
    if (in.ctx || in.failed) return 0;
    return in.evicted ? in.bytes : t->planned;
  }

  bool has_queued(uint64_t id) {
    for (Ticket* q : queue)
      if (q->req.instance == id) return true;
    return false;
  }

  // evicts least recently used idle steady instances without queued requests
  // until `bytes` more fit in the budget (caller holds mu); false if not
  bool make_room(int64_t bytes) {
    while (budget > 0 && resident + bytes > budget) {
      Instance* lru = nullptr;
      for (auto& kv : inst) {
        Instance& in = kv.second;
        if (!in.ctx || in.busy || !in.steady || has_queued(kv.first)) continue;
        if (!lru || in.last_use < lru->last_use) lru = &in;
      }
      if (!lru) return false;
      lru->saved_y.assign(lru->n, 0.0);
      if (fsi_get_state(lru->ctx, lru->saved_y.data()) != FSI_OK) return false;
      fsi_destroy(lru->ctx);
      lru->ctx = nullptr;
      lru->evicted = true;
      resident -= lru->bytes;
      ++evictions;
    }
    return true;
  }

  // first runnable ticket in arrival order (caller holds mu); with
  // batch_only, only requests of resident batchable instances qualify
  Ticket* pick(bool batch_only = false) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Ticket* t = *it;
      auto f = inst.find(t->req.instance);
      if (f != inst.end() && f->second.busy) continue;                 // in order per instance
      if (batch_only && (f == inst.end() || !f->second.ctx || !f->second.batchable)) continue;
      bool earlier_same = false;                                       // an older request of it waits
      for (auto jt = queue.begin(); jt != it; ++jt)
        if ((*jt)->req.instance == t->req.instance) { earlier_same = true; break; }
      if (earlier_same) continue;
      const int64_t nb = need(t, f);
      if (nb > 0 && budget > 0 && resident + nb > budget) {   // admission
        // evict only on behalf of the oldest waiting request, so that later
        // small requests cannot evict instances ahead of it
        if (!evict || it != queue.begin() || !make_room(nb)) continue;
      }
      queue.erase(it);
      return t;
    }
    return nullptr;
  }

  // marks a picked ticket running (caller holds mu)
  void claim(Ticket* t) {
    auto f = inst.find(t->req.instance);
    t->reserved = need(t, f);
    auto& in = inst[t->req.instance];
    in.busy = true;
    resident += t->reserved;   // reserve before building
    t->state = 1;
    t->t_start = Clock::now();
    ++running;
  }

  // first request of an instance: build its hierarchy and initial state
  // an evicted instance: rebuilt from its descriptor and saved state
  int build(Ticket* t, Instance* in, cudaStream_t stream) {
    const bool again = in->evicted;
    if (!again) {
      in->desc = t->req.desc;
      in->opts = t->req.opts;
    }
    int rc = fsi_build_hierarchy(&in->desc, &in->opts, stream, &in->ctx);
    if (rc == FSI_OK) {
      int64_t nl[16], hb = 0;
      fsi_get_sizes(in->ctx, nl, nullptr, &hb);
      in->n = nl[in->desc.levels - 1];
      in->bytes = hb;
      in->batchable = in->opts.precision == FSI_MIXED && in->desc.levels >= 2;
      in->steady = in->desc.transient == 0;
      if (again) {
        rc = fsi_set_state(in->ctx, in->saved_y.data(), nullptr, nullptr, 0.0);
      } else {
        std::vector<double> y(in->n);
        rc = fsi_initial_state(in->ctx, t->noise.data(), y.data());
        if (rc == FSI_OK) rc = fsi_set_state(in->ctx, y.data(), nullptr, nullptr, 0.0);
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    resident += (rc == FSI_OK ? in->bytes : 0) - t->reserved;
    t->reserved = 0;
    t->planned = 0;
    if (rc == FSI_OK) {
      in->evicted = false;
      in->saved_y.clear();
    }
    if (rc != FSI_OK && in->ctx) {
      fsi_destroy(in->ctx);
      in->ctx = nullptr;
    }
    return rc;
  }

  // records a finished step and frees / keeps its instance
  void finish(Ticket* t, Instance* in, int rc, double rel, const fsi_solve_stats& st, std::vector<double>& dx) {
    {
      std::lock_guard<std::mutex> lk(mu);
      t->t_end = Clock::now();
      t->res.status = rc;
      t->res.iters = st.iters;
      t->res.rel_step = rel;
      t->res.rel_res = st.rel_res;
      t->res.n = in->n;
      t->res.queue_ms = ms(t->t_submit, t->t_start);
      t->res.run_ms = ms(t->t_start, t->t_end);
      t->res.latency_ms = ms(t->t_submit, t->t_end);
      if (t->req.keep_dx) t->dx.swap(dx);
      t->noise.clear();
      in->last_use = ++use_clock;
      // a step that did not converge leaves the instance (and its state) in
      // place; other failures free it and are remembered, so the instance's
      // queued requests complete with the same error; the last request
      // forgets the instance
      if (t->req.last || in->free_after || (rc != FSI_OK && rc != FSI_E_NOT_CONVERGED)) {
        if (in->ctx) {
          fsi_destroy(in->ctx);
          in->ctx = nullptr;
          resident -= in->bytes;
        }
        if (t->req.last || in->free_after) {
          inst.erase(t->req.instance);
        } else {
          in->failed = rc;
          in->busy = false;
        }
      } else {
        in->busy = false;
      }
      t->state = 2;
      --running;
    }
    cv.notify_all();
    done_cv.notify_all();
  }

  void run_single(Ticket* t, cudaStream_t stream) {
    Instance* in;
    {
      std::lock_guard<std::mutex> lk(mu);
      in = &inst[t->req.instance];
    }
    int rc = FSI_OK;
    if (in->failed) {
      // an earlier step of this instance failed and freed it: complete the
      // request at once with that step's error instead of rebuilding it
      rc = in->failed;
    } else if (!in->ctx) {
      rc = build(t, in, stream);
    }
    fsi_solve_stats st{};
    double rel = 0.0;
    std::vector<double> dx;
    if (rc == FSI_OK) {
      // the step runs on this worker's stream, whichever worker built the
      // instance, so instances served by different workers overlap on the
      // device (the ctx is idle here: its previous step has completed)
      rc = fsi_set_stream(in->ctx, stream);
      dx.assign(t->req.keep_dx ? in->n : 0, 0.0);
      if (rc == FSI_OK) rc = fsi_newton_step(in->ctx, t->req.keep_dx ? dx.data() : nullptr, &rel, &st);
    }
    finish(t, in, rc, rel, st, dx);
  }

  // steps of several resident instances: each assembles, the Schwarz blocks
  // of all of them are factored by one launch (fsi_factor_schwarz_batch;
  // bit-identical to factoring them one by one), then each solves and
  // updates; on a factorisation error every instance factors alone, so the
  // error is reported for the instance it belongs to
  void run_batch(const std::vector<Ticket*>& batch, cudaStream_t stream) {
    const size_t k = batch.size();
    std::vector<Instance*> in(k);
    {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t i = 0; i < k; ++i) in[i] = &inst[batch[i]->req.instance];
    }
    std::vector<int> rc(k, FSI_OK);
    std::vector<fsi_ctx*> ok;
    for (size_t i = 0; i < k; ++i) {
      rc[i] = fsi_set_stream(in[i]->ctx, stream);
      if (rc[i] == FSI_OK) rc[i] = fsi_assemble_jacobian(in[i]->ctx, nullptr);
      if (rc[i] == FSI_OK) ok.push_back(in[i]->ctx);
    }
    if (!ok.empty() && fsi_factor_schwarz_batch(ok.data(), (int)ok.size()) != FSI_OK)
      for (size_t i = 0; i < k; ++i)
        if (rc[i] == FSI_OK) rc[i] = fsi_factor_schwarz(in[i]->ctx);
    for (size_t i = 0; i < k; ++i) {
      fsi_solve_stats st{};
      double rel = 0.0;
      std::vector<double> dx(batch[i]->req.keep_dx ? in[i]->n : 0, 0.0);
      if (rc[i] == FSI_OK)
        rc[i] = fsi_newton_solve_update(in[i]->ctx, batch[i]->req.keep_dx ? dx.data() : nullptr, &rel, &st);
      finish(batch[i], in[i], rc[i], rel, st, dx);
    }
  }

  void work(int slot) {
    cudaStream_t stream = streams[slot];
    while (true) {
      std::vector<Ticket*> batch;
      {
        std::unique_lock<std::mutex> lk(mu);
        Ticket* t = nullptr;
        cv.wait(lk, [&] { return stop || (t = pick()) != nullptr; });
        if (!t) break;
        claim(t);
        batch.push_back(t);
        auto f = inst.find(t->req.instance);
        if (max_batch > 1 && f != inst.end() && f->second.ctx && f->second.batchable) {
          // other resident batchable instances with a runnable request join
          while ((int)batch.size() < max_batch) {
            Ticket* u = pick(true);
            if (!u) break;
            claim(u);
            batch.push_back(u);
          }
        }
      }
      if (batch.size() == 1) run_single(batch[0], stream);
      else run_batch(batch, stream);
    }
  }
};

extern "C" {

int fsi_server_create(int64_t hbm_budget_bytes, int max_slots, fsi_server** out) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes < 0) return FSI_E_INVALID;
  fsi_server* s = new fsi_server();
  s->budget = hbm_budget_bytes;
  s->streams.assign(max_slots, nullptr);
  for (int i = 0; i < max_slots; ++i)
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
      delete s;
      return FSI_E_CUDA;
    }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s, i] { s->work(i); });
  *out = s;
  return FSI_OK;
}

int fsi_serve_submit(fsi_server* s, const fsi_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return FSI_E_INVALID;
  std::unique_ptr<Ticket> t(new Ticket());
  t->req = *req;
  t->t_submit = Clock::now();
  bool known;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    known = s->inst.count(req->instance) != 0;
    for (Ticket* q : s->queue)
      if (q->req.instance == req->instance) known = true;
  }
  if (!known) {
    // new instance: validate the descriptor and plan its size on the host
    fsi_ctx* plan = nullptr;
    int rc = fsi_plan_hierarchy(&req->desc, &req->opts, &plan);
    if (rc != FSI_OK) return rc;
    int64_t nl[16], hb = 0;
    fsi_get_sizes(plan, nl, nullptr, &hb);
    const int64_t n = nl[req->desc.levels - 1];
    fsi_destroy(plan);
    if (s->budget > 0 && hb > s->budget) return FSI_E_INVALID;
    if (!req->noise) return FSI_E_INVALID;
    t->planned = hb;
    t->noise.assign(req->noise, req->noise + n);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  t->id = s->next++;
  *ticket = t->id;
  s->queue.push_back(t.get());
  s->tickets[t->id] = std::move(t);
  s->cv.notify_all();
  return FSI_OK;
}

int fsi_serve_poll(fsi_server* s, uint64_t ticket, fsi_result* out, double* dx_out) {
  if (!s) return FSI_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return FSI_E_INVALID;
  Ticket* t = it->second.get();
  if (t->state != 2) return FSI_PENDING;
  if (out) *out = t->res;
  if (dx_out && !t->dx.empty()) std::memcpy(dx_out, t->dx.data(), t->dx.size() * sizeof(double));
  s->tickets.erase(it);
  return FSI_OK;
}

int fsi_serve_drain(fsi_server* s) {
  if (!s) return FSI_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  s->done_cv.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
  return FSI_OK;
}

int fsi_serve_cancel(fsi_server* s, uint64_t ticket) {
  if (!s) return FSI_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return FSI_E_INVALID;
    Ticket* t = it->second.get();
    if (t->state != 0) return FSI_PENDING;   // running or done: not cancelled
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if (*q == t) {
        s->queue.erase(q);
        break;
      }
    // the instance's other queued requests, in arrival order
    Ticket* first = nullptr;
    Ticket* final_ = nullptr;
    for (Ticket* q : s->queue)
      if (q->req.instance == t->req.instance) {
        if (!first) first = q;
        final_ = q;
      }
    // a cancelled first request hands the noise of the initial state (and
    // the planned size) to the next one, which then builds the instance
    if (!t->noise.empty() && first) {
      first->noise.swap(t->noise);
      first->planned = t->planned;
    }
    // a cancelled last request: the instance ends after its latest queued
    // request, else after the step that runs now, else at once
    if (t->req.last) {
      if (final_) {
        final_->req.last = 1;
      } else {
        auto f = s->inst.find(t->req.instance);
        if (f != s->inst.end()) {
          Instance& in = f->second;
          if (in.busy) {
            in.free_after = true;
          } else {
            if (in.ctx) {
              fsi_destroy(in.ctx);
              s->resident -= in.bytes;
            }
            s->inst.erase(f);
          }
        }
      }
    }
    t->state = 2;
    t->t_start = t->t_end = Clock::now();
    t->res = fsi_result{};
    t->res.status = FSI_E_CANCELLED;
    t->res.queue_ms = ms(t->t_submit, t->t_end);
    t->res.latency_ms = t->res.queue_ms;
    t->noise.clear();
  }
  s->cv.notify_all();
  s->done_cv.notify_all();
  return FSI_OK;
}

int fsi_server_set_batching(fsi_server* s, int max_batch) {
  if (!s || max_batch < 1 || max_batch > 64) return FSI_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  s->max_batch = max_batch;
  return FSI_OK;
}

int64_t fsi_server_resident_bytes(const fsi_server* s) { return s ? s->resident : 0; }

int fsi_server_set_eviction(fsi_server* s, int on) {
  if (!s) return FSI_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  s->evict = on != 0;
  return FSI_OK;
}

int64_t fsi_server_evictions(fsi_server* s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->evictions;
}

int fsi_server_destroy(fsi_server* s) {
  if (!s) return FSI_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv.notify_all();
  for (auto& w : s->workers) w.join();
  for (auto& kv : s->inst)
    if (kv.second.ctx) fsi_destroy(kv.second.ctx);
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamDestroy(st);
  delete s;
  return FSI_OK;
}

}  // extern "C"
