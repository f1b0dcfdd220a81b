// Continuous-batching solver service (included by context.cu, which owns the
// kernels).  A scheduler thread admits requests under an HBM budget (one device
// slab, first-fit free list with adjacent-block coalescing), and advances all
// admitted requests together in steps: every step launches, per quartet class,
// ONE kernel whose job table holds the next chunk of work items of every
// active request of that class, so requests that arrive while others run share
// the device.  Requests finish independently; host waits are bounded.
#pragma once
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "arena.h"

namespace {

enum JobState { kQueued = 0, kActive, kDraining, kDone, kCancelled, kFailed };

struct SvcJob {
  uint64_t ticket = 0;
  ltjk_request req{};
  int state = kQueued;
  int status = LTJK_OK;
  bool prologue_done = false, cancel_req = false;
  size_t off = 0, bytes = 0;
  bool has_mem = false;
  std::vector<int> cur64, cur32;  // cursor per ClassWork entry of the context
  cudaEvent_t ev = nullptr;       // recorded after the job's last launch
  double t_submit = 0, t_done = 0;
  JKArgs a{};
  double *Jq = nullptr, *Kq = nullptr;
  const double *scale = nullptr;  // per-density scales of the prologue
  int lane = 0;                   // stream set: 0 bulk, 1 fast (small requests)
};

// One set of streams: a prologue/epilogue stream and the side streams its
// class launches run on (fork before a step, join before an epilogue).
struct StreamSet {
  cudaStream_t st = nullptr;
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSideStreams] = {};
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ltjk_service {
  int device = 0;
  // Two stream sets: bulk (lowest priority) for large requests, which advance
  // step_items work items per class per step, and fast (highest priority) for
  // requests of at most kFastFlops algorithmic flops (about 10 ms of work
  // alone), which issue all their work in one step.  The block scheduler starts the fast set's CTAs ahead of the
  // bulk set's pending ones, and a fast request's epilogue joins only the
  // fast streams, so a small request does not queue behind the steps already
  // issued for large ones.
  StreamSet set[2];
  static constexpr double kFastFlops = 2e10;
  Arena arena;
  std::thread thr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SvcJob *> queue;
  std::vector<SvcJob *> active;
  std::map<uint64_t, std::unique_ptr<SvcJob>> jobs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int fail_next_admission = 0;
  // work items per request per class per step, and steps queued on the
  // device ahead of the host: a request that arrives waits for the steps
  // already queued, so both bound its first-step delay (2048 and 8 let a
  // small request behind a large one wait up to 70x its own service time)
  int step_items = 1024;
  static constexpr int kRunAhead = kSideStreams;
  // statistics
  std::vector<double> lat;
  uint64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, steps = 0, launches = 0;
  double t_first_submit = -1, t_last_done = 0;
  std::deque<cudaEvent_t> inflight;  // step events, at most two steps ahead of the device
  std::vector<cudaEvent_t> event_pool;

  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }
  void put_event(cudaEvent_t e) {
    if (e) event_pool.push_back(e);
  }
  void run();
  int step(std::vector<SvcJob *> &run_jobs, const StreamSet &S, int cap);
};

namespace {

size_t job_bytes(const ltjk_request &r) {
  const size_t n = (size_t)r.ctx->nao * r.ctx->nao * r.n;
  if (r.kind == LTJK_REQ_JK) return jk_scratch_bytes(r.ctx, r.n);
  return 4 * n * sizeof(double);  // P, Q, P + P^T, Q + Q^T, q-innermost
}

// Bounded host wait on an event (polling); never blocks forever.
int wait_event(cudaEvent_t e, double timeout_s) {
  const double t0 = now_s();
  for (;;) {
    cudaError_t q = cudaEventQuery(e);
    if (q == cudaSuccess) return LTJK_OK;
    if (q != cudaErrorNotReady) return set_error(LTJK_ECUDA, "event: %s", cudaGetErrorString(q));
    if (now_s() - t0 > timeout_s) return set_error(LTJK_ETIMEDOUT, "device did not finish in %.1f s", timeout_s);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

}  // namespace

// One step of one stream set: per (precision, mode, quartet class) one launch
// over the next chunk (at most cap items per job; cap 0: all remaining) of
// every runnable job of the set.  Returns the number of launches.
int ltjk_service::step(std::vector<SvcJob *> &run, const StreamSet &S, int cap) {
  const ProgramSet *ps;
  if (program_set(&ps)) return -1;
  int nl = 0;
  for (int mode = 0; mode < 2; ++mode)
    for (int prec = 0; prec < 3; ++prec)
      for (int q = 0; q < kNumPairClass * kNumPairClass; ++q) {
        JobTable T;
        T.njobs = 0;
        T.total = 0;
        const ClassProg *prog = nullptr;
        auto flush = [&]() {
          if (T.total == 0) return;
          const DevProgs &PR = run[0]->req.ctx->progs;
          // a class always runs on the same side stream: launches of one class
          // stay ordered, different classes overlap, and no step waits for
          // the previous one to drain
          cudaStream_t st = S.side[q % kSideStreams];
          if (mode == 0) {
            if (prec == 0 && !ieee64_class(prog->la, prog->lb, prog->lc, prog->ld))
              launch_jk<dflt>(*prog, PR, T, st);
            else if (prec == 1)
              launch_jk<float>(*prog, PR, T, st);
            else
              launch_jk<double>(*prog, PR, T, st);
          } else {
            if (prec == 0)
              launch_class<dflt, kGrad>(PR, grad_launch(*prog, sizeof(dflt)), T, st);
            else if (prec == 1)
              launch_class<float, kGrad>(PR, grad_launch(*prog, sizeof(float)), T, st);
            else
              launch_class<double, kGrad>(PR, grad_launch(*prog, sizeof(double)), T, st);
          }
          ++nl;
          T.njobs = 0;
          T.total = 0;
        };
        for (SvcJob *j : run) {
          if ((j->req.kind == LTJK_REQ_JK) != (mode == 0)) continue;
          ltjk_ctx *c = j->req.ctx;
          const bool native = c->opts.precision == LTJK_FP64_NATIVE;
          if ((prec == 0 && native) || (prec == 2 && !native)) continue;
          for (size_t w = 0; w < c->work.size(); ++w) {
            ClassWork &cw = *c->work[w];
            if (quartet_index(cw.la, cw.lb, cw.lc, cw.ld, 0) != q) continue;
            int &cur = prec != 1 ? j->cur64[w] : j->cur32[w];
            const int n = prec != 1 ? cw.n64 : cw.n32;
            if (cur >= n) continue;
            const int take = cap > 0 ? std::min(cap, n - cur) : n - cur;
            prog = &ps->progs[quartet_index(cw.la, cw.lb, cw.lc, cw.ld, mode)];
            JobDesc &D = T.j[T.njobs++];
            D.B = c->basis();
            D.a = j->a;
            D.items = (prec != 1 ? cw.items64.as<WorkItem>() : cw.items32.as<WorkItem>()) + cur;
            D.nitems = take;
            D.first = T.total;
            T.total += take;
            cur += take;
            if (T.njobs == kMaxJobs) flush();
          }
        }
        flush();
      }
  return nl;
}

void ltjk_service::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<SvcJob *> admitted, run_jobs;
    {
      std::unique_lock<std::mutex> g(mu);
      if (active.empty() && queue.empty()) {
        if (stop) break;
        cv_work.wait_for(g, std::chrono::milliseconds(2));
        continue;
      }
      // admission, first come first served, as memory allows
      while (!queue.empty()) {
        SvcJob *j = queue.front();
        if (j->cancel_req) {
          queue.pop_front();
          j->state = kCancelled;
          j->status = LTJK_ECANCELLED;
          ++cancelled;
          cv_done.notify_all();
          continue;
        }
        if (fail_next_admission > 0) {  // injected allocation failure (tests)
          --fail_next_admission;
          queue.pop_front();
          j->state = kFailed;
          j->status = LTJK_ENOMEM;
          ++failed;
          cv_done.notify_all();
          continue;
        }
        if (!arena.alloc(j->bytes, &j->off)) break;
        j->has_mem = true;
        queue.pop_front();
        j->state = kActive;
        active.push_back(j);
        admitted.push_back(j);
      }
      for (SvcJob *j : active)
        if (j->state == kActive && !j->cancel_req) run_jobs.push_back(j);
    }
    // prologues of newly admitted jobs
    for (SvcJob *j : admitted) {
      ltjk_ctx *c = j->req.ctx;
      const size_t NN = (size_t)c->nao * c->nao, n = NN * j->req.n;
      double *mem = reinterpret_cast<double *>(arena.base + j->off);
      const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
      j->cur64.assign(c->work.size(), 0);
      j->cur32.assign(c->work.size(), 0);
      // small requests by the flop model (item counts say little: small
      // molecules get one ket per work item)
      const double work = j->req.kind == LTJK_REQ_JK
                              ? c->stats.eri_flops_per_build + 20.0 * c->stats.cart_integrals_kept * j->req.n
                              : c->stats.grad_eri_flops + c->stats.cart_integrals_kept * (2.0 * j->req.n + 18.0);
      j->lane = work <= kFastFlops ? 1 : 0;
      cudaStream_t st = set[j->lane].st;
      JKArgs a{};
      if (j->req.kind == LTJK_REQ_JK) {
        if (jk_prologue(c, j->req.D, mem, j->req.n, j->req.J != nullptr, j->req.K != nullptr, st, &a) != LTJK_OK)
          j->status = LTJK_ECUDA;
        j->Jq = mem + 2 * n;
        j->Kq = mem + 3 * n;
        j->scale = a.scale;
        g_launches -= 2;  // counted below with the others
      } else {
        double *Pq = mem, *Qq = Pq + n, *Ps = Qq + n, *Qs = Ps + n;
        to_qinner<<<blocks, 256, 0, st>>>(j->req.P, Pq, Ps, nullptr, nullptr, j->req.n, c->nao);
        to_qinner<<<blocks, 256, 0, st>>>(j->req.Q, Qq, Qs, nullptr, nullptr, j->req.n, c->nao);
        cudaMemsetAsync(j->req.grad, 0, sizeof(double) * 3 * c->natoms, st);
        a.P = Pq; a.Q = Qq; a.S = Ps; a.D = Qs; a.cJ = j->req.cJ; a.cK = j->req.cK; a.grad = j->req.grad;
      }
      a.nd = j->req.n;
      j->a = a;
      g_launches += 2;
      launches += 2;
      run_jobs.push_back(j);
    }
    for (int l = 0; l < 2; ++l) {  // their layout copies (on st) precede their class launches
      bool any = false;
      for (SvcJob *j : admitted) any |= j->lane == l;
      if (!any) continue;
      cudaEventRecord(set[l].fork_ev, set[l].st);
      for (int k = 0; k < kSideStreams; ++k) cudaStreamWaitEvent(set[l].side[k], set[l].fork_ev, 0);
    }
    // bulk steps run at most kRunAhead ahead of the device; the check never
    // blocks, so admission, fast requests and completions keep moving while
    // the bulk queue is full
    while (!inflight.empty() && cudaEventQuery(inflight.front()) != cudaErrorNotReady) {
      put_event(inflight.front());
      inflight.pop_front();
    }
    const bool bulk_ok = inflight.size() < (size_t)kRunAhead;
    int nl = 0, nl_bulk = 0;
    {
      std::vector<SvcJob *> part[2];
      for (SvcJob *j : run_jobs) part[j->lane].push_back(j);
      if (!part[1].empty()) nl += step(part[1], set[1], 0);
      if (!part[0].empty() && bulk_ok) nl += (nl_bulk = step(part[0], set[0], step_items));
    }
    if (nl > 0) {
      ++steps;
      launches += nl;
    }
    // jobs with every item issued: epilogue and completion event
    std::vector<SvcJob *> to_finish;
    {
      std::lock_guard<std::mutex> g(mu);
      for (SvcJob *j : active) {
        if (j->state != kActive) continue;
        bool all = true;
        if (!j->cancel_req) {
          ltjk_ctx *c = j->req.ctx;
          for (size_t w = 0; w < c->work.size() && all; ++w)
            all = j->cur64[w] >= c->work[w]->n64 && j->cur32[w] >= c->work[w]->n32;
        }
        if (all) to_finish.push_back(j);
      }
    }
    for (int l = 0; l < 2; ++l) {  // the set's class launches so far precede its epilogues
      bool any = false;
      for (SvcJob *j : to_finish) any |= j->lane == l;
      if (!any) continue;
      for (int k = 0; k < kSideStreams; ++k) {
        cudaEventRecord(set[l].join_ev[k], set[l].side[k]);
        cudaStreamWaitEvent(set[l].st, set[l].join_ev[k], 0);
      }
    }
    for (SvcJob *j : to_finish) {
      cudaStream_t st = set[j->lane].st;
      if (!j->cancel_req && j->req.kind == LTJK_REQ_JK) {
        ltjk_ctx *c = j->req.ctx;
        const size_t n = (size_t)c->nao * c->nao * j->req.n;
        const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)num_sms() * 16);
        from_qinner<<<blocks, 256, 0, st>>>(j->Jq, j->Kq, j->req.J, j->req.K, j->req.n, c->nao, j->scale);
        g_launches += 1;
        launches += 1;
      }
      j->ev = get_event();
      cudaEventRecord(j->ev, st);
      std::lock_guard<std::mutex> g(mu);
      j->state = kDraining;
    }
    // keep the host a bounded number of bulk steps ahead of the device
    if (nl_bulk > 0) {
      cudaEvent_t se = get_event();
      cudaEventRecord(se, set[0].side[steps % kSideStreams]);
      inflight.push_back(se);
    }
    if (nl == 0 && to_finish.empty() && admitted.empty())
      std::this_thread::sleep_for(std::chrono::microseconds(50));  // waiting on the device
    // completions
    {
      std::lock_guard<std::mutex> g(mu);
      const double t = now_s();
      for (auto it = active.begin(); it != active.end();) {
        SvcJob *j = *it;
        if (j->state == kDraining) {
          cudaError_t q = cudaEventQuery(j->ev);
          if (q != cudaErrorNotReady) {
            if (q != cudaSuccess) {
              j->state = kFailed;
              j->status = LTJK_ECUDA;
              ++failed;
            } else if (j->cancel_req) {
              j->state = kCancelled;
              j->status = LTJK_ECANCELLED;
              ++cancelled;
            } else {
              j->state = kDone;
              j->status = LTJK_OK;
              j->t_done = t;
              lat.push_back(t - j->t_submit);
              ++completed;
              t_last_done = t;
            }
            put_event(j->ev);
            j->ev = nullptr;
            if (j->has_mem) arena.release(j->off, j->bytes);
            j->has_mem = false;
            it = active.erase(it);
            cv_done.notify_all();
            continue;
          }
        }
        ++it;
      }
    }
  }
  for (cudaEvent_t e : inflight) {
    wait_event(e, 600.0);
    cudaEventDestroy(e);
  }
  inflight.clear();
}

extern "C" {

int ltjk_service_create(size_t hbm_budget_bytes, int device, ltjk_service **out) {
  if (!out || hbm_budget_bytes < (1u << 20)) return set_error(LTJK_EINVAL, "service_create: budget below 1 MiB");
  *out = nullptr;
  auto s = std::make_unique<ltjk_service>();
  s->device = device;
  CUDA_TRY(cudaSetDevice(device));
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, hbm_budget_bytes);
  if (e != cudaSuccess) return set_error(LTJK_ENOMEM, "service arena of %zu bytes: %s", hbm_budget_bytes, cudaGetErrorString(e));
  s->arena.init(static_cast<char *>(p), hbm_budget_bytes);
  int prio_low = 0, prio_high = 0;
  e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  for (int l = 0; l < 2 && e == cudaSuccess; ++l) {
    StreamSet &S = s->set[l];
    const int prio = l == 1 ? prio_high : prio_low;
    e = cudaStreamCreateWithPriority(&S.st, cudaStreamNonBlocking, prio);
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithPriority(&S.side[k], cudaStreamNonBlocking, prio);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.join_ev[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.fork_ev, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cudaFree(p);
    return set_error(LTJK_ECUDA, "stream: %s", cudaGetErrorString(e));
  }
  ltjk_service *raw = s.get();
  s->thr = std::thread([raw]() { raw->run(); });
  *out = s.release();
  return LTJK_OK;
}

int ltjk_service_submit(ltjk_service *s, const ltjk_request *r, uint64_t *ticket) {
  if (!s || !r || !ticket) return set_error(LTJK_EINVAL, "service_submit: null argument");
  if (!r->ctx) return set_error(LTJK_EINVAL, "service_submit: null context");
  if (r->ctx->device != s->device) return set_error(LTJK_EINVAL, "service_submit: context on another device");
  if (r->n < 1 || r->n > 4096) return set_error(LTJK_EINVAL, "service_submit: n %d not in 1..4096", r->n);
  if (r->kind == LTJK_REQ_JK) {
    if (!r->D || (!r->J && !r->K)) return set_error(LTJK_EINVAL, "service_submit: J/K request needs D and J or K");
  } else if (r->kind == LTJK_REQ_GRAD) {
    if (!r->P || !r->Q || !r->grad) return set_error(LTJK_EINVAL, "service_submit: gradient request needs P, Q, grad");
    for (int sh = 0; sh < r->ctx->nshells; ++sh)
      if (r->ctx->sh_l[sh] > kMaxLGrad)
        return set_error(LTJK_EUNSUPPORTED, "service_submit: gradient of a context with l = %d above "
                         "LTJK_MAX_L_GRAD = %d", r->ctx->sh_l[sh], kMaxLGrad);
  } else {
    return set_error(LTJK_EINVAL, "service_submit: unknown request kind %d", r->kind);
  }
  auto j = std::make_unique<SvcJob>();
  j->req = *r;
  j->bytes = job_bytes(*r);
  if (!s->arena.could_fit(j->bytes))
    return set_error(LTJK_EBUDGET, "request needs %zu bytes (%zu rounded to the arena's %zu-byte blocks), "
                     "usable budget is %zu", j->bytes, Arena::rounded(j->bytes), Arena::kAlign, s->arena.size);
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return set_error(LTJK_EINVAL, "service is shutting down");
  j->ticket = s->next_ticket++;
  j->t_submit = now_s();
  if (s->t_first_submit < 0) s->t_first_submit = j->t_submit;
  *ticket = j->ticket;
  s->queue.push_back(j.get());
  s->jobs[j->ticket] = std::move(j);
  ++s->submitted;
  s->cv_work.notify_one();
  return LTJK_OK;
}

int ltjk_service_poll(ltjk_service *s, uint64_t ticket, int *done) {
  if (!s || !done) return set_error(LTJK_EINVAL, "service_poll: null argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return set_error(LTJK_EINVAL, "service_poll: unknown ticket");
  const int st = it->second->state;
  *done = st == kDone || st == kCancelled || st == kFailed;
  return *done ? it->second->status : LTJK_OK;
}

int ltjk_service_wait(ltjk_service *s, uint64_t ticket, double timeout_s) {
  if (!s) return set_error(LTJK_EINVAL, "service_wait: null service");
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return set_error(LTJK_EINVAL, "service_wait: unknown ticket");
  SvcJob *j = it->second.get();
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(std::max(0.0, timeout_s)));
  while (!(j->state == kDone || j->state == kCancelled || j->state == kFailed)) {
    if (s->cv_done.wait_until(g, deadline) == std::cv_status::timeout &&
        !(j->state == kDone || j->state == kCancelled || j->state == kFailed))
      return set_error(LTJK_ETIMEDOUT, "service_wait: ticket %llu not done after %.3f s",
                       (unsigned long long)ticket, timeout_s);
  }
  if (j->status != LTJK_OK) {
    if (j->status == LTJK_ECANCELLED) return set_error(LTJK_ECANCELLED, "request was cancelled");
    if (j->status == LTJK_ENOMEM) return set_error(LTJK_ENOMEM, "request admission failed");
    return set_error(j->status, "request failed");
  }
  return LTJK_OK;
}

int ltjk_service_cancel(ltjk_service *s, uint64_t ticket) {
  if (!s) return set_error(LTJK_EINVAL, "service_cancel: null service");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return set_error(LTJK_EINVAL, "service_cancel: unknown ticket");
  it->second->cancel_req = true;
  s->cv_work.notify_one();
  return LTJK_OK;
}

int ltjk_service_stats(ltjk_service *s, ltjk_svc_stats *o) {
  if (!s || !o) return set_error(LTJK_EINVAL, "service_stats: null argument");
  std::lock_guard<std::mutex> g(s->mu);
  *o = ltjk_svc_stats{};
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->cancelled = s->cancelled;
  o->failed = s->failed;
  std::vector<double> l = s->lat;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) { return l.empty() ? 0.0 : 1e3 * l[std::min(l.size() - 1, (size_t)std::floor(p * (l.size() - 1) + 0.5))]; };
  o->p50_ms = pct(0.50);
  o->p99_ms = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  o->mean_ms = l.empty() ? 0.0 : 1e3 * sum / l.size();
  const double span = s->t_last_done - s->t_first_submit;
  o->throughput_rps = (s->completed && span > 0) ? s->completed / span : 0.0;
  o->bytes_in_use = s->arena.used;
  o->bytes_peak = s->arena.peak;
  o->budget = s->arena.size;
  o->steps = s->steps;
  o->launches = s->launches;
  o->active = (int)s->active.size();
  o->queued = (int)s->queue.size();
  return LTJK_OK;
}

int ltjk_service_fail_next_admission(ltjk_service *s, int count) {
  if (!s || count < 0) return set_error(LTJK_EINVAL, "service_fail_next_admission: bad argument");
  std::lock_guard<std::mutex> g(s->mu);
  s->fail_next_admission = count;
  return LTJK_OK;
}

int ltjk_service_destroy(ltjk_service *s) {
  if (!s) return set_error(LTJK_EINVAL, "service_destroy: null service");
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (SvcJob *j : s->queue) j->cancel_req = true;
    s->cv_work.notify_all();
  }
  if (s->thr.joinable()) s->thr.join();
  cudaSetDevice(s->device);
  for (int l = 0; l < 2; ++l)
    if (s->set[l].st) cudaStreamSynchronize(s->set[l].st);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  for (auto &kv : s->jobs)
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
  for (int l = 0; l < 2; ++l) {
    StreamSet &S = s->set[l];
    for (int k = 0; k < kSideStreams; ++k) {
      if (S.side[k]) cudaStreamDestroy(S.side[k]);
      if (S.join_ev[k]) cudaEventDestroy(S.join_ev[k]);
    }
    if (S.fork_ev) cudaEventDestroy(S.fork_ev);
    if (S.st) cudaStreamDestroy(S.st);
  }
  cudaFree(s->arena.base);
  delete s;
  return LTJK_OK;
}

}  // extern "C"
