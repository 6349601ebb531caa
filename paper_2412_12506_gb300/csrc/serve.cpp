// Serving engine (include/ldgmg_serve.h): a cache of problem classes
// (operator + hierarchy) admitted by device footprint, and continuous
// batching of queued solves onto worker threads with one CUDA stream each.
//
// All scheduling state lives under one mutex.  Scheduling is event driven:
// every event that can make progress possible (a submit, a finished build, a
// finished solve) calls plan() with the mutex held.  plan() (0) rebuilds
// classes marked for an FP64 V-cycle once no running call reads them, (1)
// fails the queues of classes whose build failed, (2) admits classes with
// queued requests in the order of their oldest request, evicting idle
// classes least-recently-used first while the footprint does not fit, and
// (3) hands work to idle workers, oldest waiting request first: a large
// class's call takes as many of its own requests as one solve call takes; a
// small class's request starts a grouped call (ldgmg_solve_group) that takes
// the oldest queued requests of every ready small class.
#include "ldgmg_serve.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

void ldgmg_set_error(const std::string& msg);

namespace {

using Clock = std::chrono::steady_clock;

ldgmg_status serr(ldgmg_status s, const std::string& m) {
  ldgmg_set_error(m);
  return s;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct ClassKey {
  int dim, n, p, stokes;
  double tau0, taup;
  uint64_t mu_hash;
  bool operator<(const ClassKey& o) const {
    return std::tie(dim, n, p, stokes, tau0, taup, mu_hash) <
           std::tie(o.dim, o.n, o.p, o.stokes, o.tau0, o.taup, o.mu_hash);
  }
};

struct Req {
  uint64_t id = 0;
  std::vector<double> rhs;
  double* x_host = nullptr;
  double tol = 0.0;
  ldgmg_result res{};
  bool done = false;
};

struct Class {
  ClassKey key{};
  std::vector<double> mu;   // empty: mu == 1
  int b = 0;
  int64_t N = 0;
  enum State { EMPTY, BUILDING, READY, FAILED } state = EMPTY;
  ldgmg_status fail_status = LDGMG_OK;
  ldgmg_op* op = nullptr;
  ldgmg_hier* h = nullptr;
  int rmax = 1;             // right-hand sides per solve call of this class
  int prec = -1;            // V-cycle precision of this class (-1: the server's); LDGMG_FP64 after a fallback
  bool small = false;       // solved in grouped calls together with other small classes
  int users = 0;            // requests of running calls that read the class (grouped calls may share it)
  bool rebuild_fp64 = false;   // rebuild with an FP64 V-cycle once no call reads it
  size_t est = 0, bytes = 0;
  double last_use = 0.0;
  std::deque<std::shared_ptr<Req>> queue;
};

struct Job {
  Class* c = nullptr;                 // per-class call
  bool grouped = false;               // grouped call: cls[r] is the class of reqs[r]
  std::vector<Class*> cls;
  std::vector<std::shared_ptr<Req>> reqs;
};

size_t esize(int prec) { return prec == LDGMG_FP64 ? 8 : (prec == LDGMG_FP32 ? 4 : 2); }

// V-cycle precision a class is built with
int class_prec(const ldgmg_server_opts& o, const Class& c) { return c.prec >= 0 ? c.prec : o.setup.vcycle_precision; }

// simulate = 1: the solve outcome of a class (the injected non-convergence of
// a reduced-precision class, see simulate_notconv_n)
ldgmg_status simulated_status(const ldgmg_server_opts& o, const Class& c) {
  return o.simulate_notconv_n > 0 && c.key.n == o.simulate_notconv_n && class_prec(o, c) != LDGMG_FP64
             ? LDGMG_ENOTCONV
             : LDGMG_OK;
}

}  // namespace

struct ldgmg_server {
  ldgmg_server_opts o{};
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_done, cv_work, cv_build;
  bool stop = false;
  std::map<ClassKey, std::unique_ptr<Class>> classes;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
  uint64_t next_id = 1;
  uint64_t outstanding = 0;   // submitted, not yet done
  std::deque<Class*> build_q;
  std::deque<Job> work_q;
  int idle_workers = 0;
  // small lane: with grouped calls on, one more worker takes grouped calls
  // only, so small requests never wait behind large solves
  bool has_lane = false, lane_idle = false;
  std::deque<Job> lane_q;
  size_t reserved = 0;        // estimates of building classes + measured bytes of resident ones
  ldgmg_server_stats st{};
  std::thread builder;
  std::vector<std::thread> workers;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Device footprint of a class before it is built (admission); replaced by the
// measured ldgmg_*_device_bytes once it is.  Block rows per level times stored
// blocks per row times block bytes, for A, the smoother (B and B^T, or D),
// level vectors, the FP64 outer operator and Krylov space, the bottom
// pseudo-inverse and (tensor-core classes) the operand images of x, plus 10%.
size_t estimate(const ldgmg_server_opts& o, const Class& c) {
  const ClassKey& k = c.key;
  const int d = k.dim;
  const double b = c.b;
  int per_row = 2 * d + 1;                        // face-neighbour stencil
  if (k.stokes == 1) per_row = d == 2 ? 7 : 13;   // stress form couples diagonal neighbours
  const int sai_rows = o.setup.sai_level == 2 ? (d == 2 ? 13 : 25) : per_row;
  const int prec = c.prec >= 0 ? c.prec : o.setup.vcycle_precision;
  const double es = double(esize(prec));
  const int rmax = c.rmax;
  const double vs = prec == LDGMG_FP64 ? 8.0 : 4.0;
  double total = 0.0;
  total += double(c.N) * per_row * b * b * 8.0 * 2.0;   // FP64 A (+ double-FP32 copy)
  int n = k.n;
  double Nl = double(c.N);
  while (true) {
    const bool bottom = !(n % 2 == 0 && n > 1);
    total += Nl * per_row * b * b * es;
    if (!bottom) total += Nl * b * b * es * (o.setup.smoother == LDGMG_SAI ? 2.0 * sai_rows : 1.0);
    total += 3.0 * Nl * b * vs * rmax;
    if (bottom) {
      total += (Nl * b) * (Nl * b) * 8.0;
      break;
    }
    n /= 2;
    Nl /= double(1 << d);
  }
  total += double(c.N) * b * 8.0 * rmax * 8.0;           // CG vectors and staging
  const bool tc = rmax > 1 && (c.b == 16 || c.b == 64) && vs == 4.0 && o.setup.smoother != LDGMG_GS;
  if (tc) total += double(c.N) * b * 4.0 * double((rmax + 7) / 8 * 8);   // tensor-core operand images of x
  if (k.stokes >= 0) total += double(c.N) * b * 8.0 * (2.0 * o.setup.restart + 1.0);
  return size_t(total * 1.1);
}

void free_class(Class* c) {
  if (c->h) ldgmg_hier_free(c->h);
  if (c->op) ldgmg_op_free(c->op);
  c->h = nullptr;
  c->op = nullptr;
}

void complete(ldgmg_server* s, const std::shared_ptr<Req>& r) {
  r->done = true;
  s->outstanding--;
  s->st.completed++;
}

// Requests queued on a failed (or refused) class complete with its status.
void fail_queue(ldgmg_server* s, Class* c) {
  while (!c->queue.empty()) {
    auto r = c->queue.front();
    c->queue.pop_front();
    r->res.status = c->fail_status;
    r->res.t_start = r->res.t_end = s->now();
    r->res.relres = std::numeric_limits<double>::quiet_NaN();
    complete(s, r);
  }
}

// Called with s->mu held; the caller wakes waiters (cv_done) afterwards.
void plan(ldgmg_server* s) {
  // (0) classes marked for an FP64 rebuild that no running call reads any more
  for (auto& kv : s->classes) {
    Class* c = kv.second.get();
    if (c->state == Class::READY && c->rebuild_fp64 && c->users == 0) {
      free_class(c);
      s->reserved -= c->bytes;
      c->bytes = 0;
      c->prec = LDGMG_FP64;
      c->rebuild_fp64 = false;
      c->state = Class::EMPTY;
      s->st.classes_resident--;
      s->st.precision_fallbacks++;
    }
  }
  // (1) failed builds: their queued requests complete with the build status
  for (auto& kv : s->classes) {
    Class* c = kv.second.get();
    if (c->state == Class::FAILED) fail_queue(s, c);
  }
  // (2) admission, oldest waiting request first
  std::vector<Class*> want;
  for (auto& kv : s->classes) {
    Class* c = kv.second.get();
    if (c->state == Class::EMPTY && !c->queue.empty()) want.push_back(c);
  }
  std::sort(want.begin(), want.end(),
            [](Class* a, Class* b) { return a->queue.front()->res.t_submit < b->queue.front()->res.t_submit; });
  for (Class* c : want) {
    c->est = estimate(s->o, *c);
    if (c->est > s->o.hbm_budget) {
      // larger than the whole budget on its own: refused, never built
      c->state = Class::FAILED;
      c->fail_status = LDGMG_ENOMEM;
      s->st.build_failures++;
      fail_queue(s, c);
      continue;
    }
    while (s->reserved + c->est > s->o.hbm_budget) {
      Class* victim = nullptr;
      for (auto& kv : s->classes) {
        Class* v = kv.second.get();
        if (v->state == Class::READY && v->users == 0 && v->queue.empty() && (!victim || v->last_use < victim->last_use))
          victim = v;
      }
      if (!victim) break;
      free_class(victim);
      s->reserved -= victim->bytes;
      victim->bytes = 0;
      victim->state = Class::EMPTY;
      s->st.evictions++;
      s->st.classes_resident--;
    }
    if (s->reserved + c->est > s->o.hbm_budget) break;   // wait for room, keep order
    c->state = Class::BUILDING;
    s->reserved += c->est;
    s->build_q.push_back(c);
    s->cv_build.notify_one();
  }
  // (3) dispatch to idle workers, oldest waiting request first.  A small
  // class's request starts a grouped call that takes the oldest queued
  // requests of all ready small classes; any other class runs one call at a
  // time with as many of its own requests as one call takes.
  auto ready = [](const Class* c) { return c->state == Class::READY && !c->rebuild_fp64 && !c->queue.empty(); };
  auto grouped_job = [&]() {
    Job j;
    j.grouped = true;
    std::vector<Class*> cand;
    for (auto& kv : s->classes)
      if (kv.second->small && ready(kv.second.get())) cand.push_back(kv.second.get());
    while (j.reqs.size() < size_t(s->o.group_max)) {
      Class* o = nullptr;
      for (Class* c : cand)
        if (!c->queue.empty() && (!o || c->queue.front()->res.t_submit < o->queue.front()->res.t_submit)) o = c;
      if (!o) break;
      j.reqs.push_back(o->queue.front());
      j.cls.push_back(o);
      o->queue.pop_front();
      o->users++;
    }
    return j;
  };
  if (s->has_lane && s->lane_idle) {
    Job j = grouped_job();
    if (!j.reqs.empty()) {
      s->lane_idle = false;
      s->lane_q.push_back(std::move(j));
      s->cv_work.notify_all();
    }
  }
  while (s->idle_workers > 0) {
    Class* best = nullptr;
    for (auto& kv : s->classes) {
      Class* c = kv.second.get();
      if (!ready(c) || (!c->small && c->users > 0)) continue;
      if (!best || c->queue.front()->res.t_submit < best->queue.front()->res.t_submit) best = c;
    }
    if (!best) break;
    Job j;
    if (best->small) {
      j = grouped_job();
    } else {
      j.c = best;
      const size_t cap = size_t(best->rmax);
      const double tol = best->queue.front()->tol;
      while (!best->queue.empty() && j.reqs.size() < cap && best->queue.front()->tol == tol) {
        j.reqs.push_back(best->queue.front());
        best->queue.pop_front();
      }
      best->users++;
    }
    s->idle_workers--;
    s->work_q.push_back(std::move(j));
    s->cv_work.notify_all();
  }
  s->st.bytes_resident = s->reserved;
  s->st.bytes_peak = std::max(s->st.bytes_peak, s->reserved);
}

void builder_loop(ldgmg_server* s) {
  cudaStream_t st = nullptr;
  if (!s->o.simulate) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv_build.wait(lk, [&] { return s->stop || !s->build_q.empty(); });
    if (s->build_q.empty()) break;
    Class* c = s->build_q.front();
    s->build_q.pop_front();
    const ClassKey k = c->key;
    const std::vector<double> mu = c->mu;
    ldgmg_setup_opts so = s->o.setup;
    so.max_rhs = c->rmax;
    if (c->prec >= 0) so.vcycle_precision = c->prec;
    const bool simulate = s->o.simulate != 0;
    lk.unlock();
    ldgmg_op* op = nullptr;
    ldgmg_hier* h = nullptr;
    ldgmg_status status = LDGMG_OK;
    size_t bytes = 0;
    if (!simulate) {
      ldgmg_mesh mesh{k.dim, k.n, 1};
      const double* m = mu.empty() ? nullptr : mu.data();
      status = k.stokes < 0 ? ldgmg_assemble(&mesh, k.p, m, k.tau0, &op)
                            : ldgmg_assemble_stokes(&mesh, k.p, m, k.stokes, k.tau0, k.taup, &op);
      if (status == LDGMG_OK) status = ldgmg_setup(op, &so, st, &h);
      if (status == LDGMG_OK) {
        size_t a = 0, b = 0;
        ldgmg_op_device_bytes(op, &a);
        ldgmg_hier_device_bytes(h, &b);
        bytes = a + b;
      } else {
        if (h) ldgmg_hier_free(h);
        if (op) ldgmg_op_free(op);
        h = nullptr;
        op = nullptr;
      }
    }
    lk.lock();
    s->reserved -= c->est;
    if (status == LDGMG_OK) {
      c->op = op;
      c->h = h;
      c->bytes = simulate ? c->est : bytes;
      s->reserved += c->bytes;
      c->state = Class::READY;
      c->last_use = s->now();
      s->st.builds++;
      s->st.classes_resident++;
    } else {
      c->state = Class::FAILED;
      c->fail_status = status;
      s->st.build_failures++;
    }
    plan(s);
    s->cv_done.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

// A grouped call: every request on its own class's hierarchy, one
// ldgmg_solve_group call.  Called without the mutex; fills iters / relres /
// status per request.
void run_grouped(ldgmg_server* s, ldgmg_group** grp, const Job& j, cudaStream_t st, std::vector<int>& iters,
                 std::vector<double>& relres, std::vector<ldgmg_status>& sts) {
  const int R = int(j.reqs.size());
  if (s->o.simulate) {
    std::this_thread::sleep_for(std::chrono::duration<double>(s->o.simulate_solve_s));
    for (int r = 0; r < R; ++r) sts[r] = simulated_status(s->o, *j.cls[r]);
    return;
  }
  if (!*grp && ldgmg_group_create(grp) != LDGMG_OK) {
    std::fill(sts.begin(), sts.end(), LDGMG_ENOMEM);
    return;
  }
  std::vector<ldgmg_hier*> hs(R);
  std::vector<const double*> bs(R);
  std::vector<double*> xs(R);
  std::vector<double> tols(R);
  for (int r = 0; r < R; ++r) {
    hs[r] = j.cls[r]->h;
    bs[r] = j.reqs[r]->rhs.data();
    xs[r] = j.reqs[r]->x_host;
    tols[r] = j.reqs[r]->tol;
  }
  const ldgmg_status unset = ldgmg_status(-1);
  std::fill(sts.begin(), sts.end(), unset);
  const ldgmg_status all =
      ldgmg_solve_group(*grp, R, hs.data(), bs.data(), xs.data(), tols.data(), iters.data(), relres.data(), sts.data(), st);
  for (auto& v : sts)
    if (v == unset) v = all;     // the call failed before solving
}

void worker_loop(ldgmg_server* s, int wid, bool lane) {
  cudaStream_t st = nullptr;
  ldgmg_group* grp = nullptr;     // grouped-call work space of this worker
  double *hb = nullptr, *hx = nullptr;   // pinned staging for the stacked right-hand sides
  size_t cap = 0;
  const bool simulate = s->o.simulate != 0;
  if (!simulate) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    std::deque<Job>& q = lane ? s->lane_q : s->work_q;
    s->cv_work.wait(lk, [&] { return s->stop || !q.empty(); });
    if (q.empty()) break;
    Job j = std::move(q.front());
    q.pop_front();
    Class* c = j.c;
    const double t_start = s->now();
    lk.unlock();
    if (j.grouped) {
      const int R = int(j.reqs.size());
      std::vector<int> iters(R, 0);
      std::vector<double> relres(R, std::numeric_limits<double>::quiet_NaN());
      std::vector<ldgmg_status> sts(R, LDGMG_OK);
      run_grouped(s, &grp, j, st, iters, relres, sts);
      lk.lock();
      const double t_end = s->now();
      int served = 0;
      // requests whose reduced-precision solve did not converge go back to the
      // front of their class's queue (in order); the class is rebuilt with an
      // FP64 V-cycle once no running call reads it
      for (int r = R - 1; r >= 0; --r) {
        Class* k = j.cls[size_t(r)];
        auto& q = j.reqs[size_t(r)];
        if (sts[r] == LDGMG_ENOTCONV && class_prec(s->o, *k) != LDGMG_FP64) {
          k->queue.push_front(q);
          k->rebuild_fp64 = true;
          continue;
        }
        q->res.status = sts[r];
        q->res.iters = iters[r];
        q->res.relres = relres[r];
        q->res.t_start = t_start;
        q->res.t_end = t_end;
        q->res.batch = R;
        q->res.worker = wid;
        complete(s, q);
        ++served;
      }
      for (Class* k : j.cls) {
        k->users--;
        k->last_use = t_end;
      }
      s->st.solve_calls++;
      s->st.group_calls++;
      s->st.group_requests += uint64_t(served);
      s->st.max_batch_seen = std::max(s->st.max_batch_seen, R);
      if (lane) s->lane_idle = true;
      else s->idle_workers++;
      plan(s);
      s->cv_done.notify_all();
      continue;
    }
    const int R = int(j.reqs.size());
    const size_t n = size_t(c->N) * c->b;
    std::vector<int> iters(R, 0);
    std::vector<double> relres(R, std::numeric_limits<double>::quiet_NaN());
    ldgmg_status status = LDGMG_OK;
    if (simulate) {
      std::this_thread::sleep_for(std::chrono::duration<double>(s->o.simulate_solve_s));
      status = simulated_status(s->o, *c);
    } else {
      if (cap < n * R) {
        if (hb) cudaFreeHost(hb);
        if (hx) cudaFreeHost(hx);
        hb = hx = nullptr;
        cap = 0;
        if (cudaMallocHost((void**)&hb, n * R * sizeof(double)) == cudaSuccess &&
            cudaMallocHost((void**)&hx, n * R * sizeof(double)) == cudaSuccess)
          cap = n * R;
      }
      if (cap < n * R) {
        status = LDGMG_ENOMEM;
      } else {
        for (int r = 0; r < R; ++r) std::memcpy(hb + r * n, j.reqs[r]->rhs.data(), n * sizeof(double));
        status = ldgmg_solve(c->h, hb, j.reqs[0]->tol, hx, R, iters.data(), relres.data(), st);
        for (int r = 0; r < R; ++r) std::memcpy(j.reqs[r]->x_host, hx + r * n, n * sizeof(double));
      }
    }
    lk.lock();
    const double t_end = s->now();
    if (status == LDGMG_ENOTCONV && class_prec(s->o, *c) != LDGMG_FP64) {
      // A reduced-precision V-cycle too inexact for this class (large
      // coefficient contrast): rebuild the class once with an FP64 V-cycle
      // and solve these requests again, ahead of the class's later ones.
      for (int r = R - 1; r >= 0; --r) c->queue.push_front(j.reqs[size_t(r)]);
      free_class(c);
      s->reserved -= c->bytes;
      c->bytes = 0;
      c->prec = LDGMG_FP64;
      c->state = Class::EMPTY;
      c->users--;
      s->st.classes_resident--;
      s->st.precision_fallbacks++;
      s->st.solve_calls++;
      s->idle_workers++;
      plan(s);
      s->cv_done.notify_all();
      continue;
    }
    for (int r = 0; r < R; ++r) {
      auto& q = j.reqs[r];
      q->res.status = status;
      q->res.iters = iters[r];
      q->res.relres = relres[r];
      q->res.t_start = t_start;
      q->res.t_end = t_end;
      q->res.batch = R;
      q->res.worker = wid;
      complete(s, q);
    }
    c->users--;
    c->last_use = t_end;
    s->st.solve_calls++;
    s->st.max_batch_seen = std::max(s->st.max_batch_seen, R);
    s->idle_workers++;
    plan(s);
    s->cv_done.notify_all();
  }
  lk.unlock();
  if (grp) ldgmg_group_free(grp);
  if (hb) cudaFreeHost(hb);
  if (hx) cudaFreeHost(hx);
  if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

ldgmg_status ldgmg_server_create(const ldgmg_server_opts* o, ldgmg_server** out) {
  if (!o || !out) return serr(LDGMG_EINVAL, "null argument");
  *out = nullptr;
  if (o->workers < 1 || o->workers > 16) return serr(LDGMG_EINVAL, "workers must be in 1..16");
  if (o->max_batch < 1 || o->max_batch > 64) return serr(LDGMG_EINVAL, "max_batch must be in 1..64");
  if (o->simulate && !(o->simulate_solve_s >= 0.0)) return serr(LDGMG_EINVAL, "simulate_solve_s");
  if (o->group_max < 0 || o->group_max > 65536) return serr(LDGMG_EINVAL, "group_max must be in 0..65536");
  auto* s = new (std::nothrow) ldgmg_server();
  if (!s) return serr(LDGMG_ENOMEM, "host allocation");
  s->o = *o;
  if (s->o.group_max == 0) s->o.group_max = 512;
  s->t0 = Clock::now();
  if (s->o.hbm_budget == 0) {
    if (s->o.simulate) {
      s->o.hbm_budget = size_t(1) << 30;
    } else {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        delete s;
        return serr(LDGMG_ECUDA, "cudaMemGetInfo");
      }
      s->o.hbm_budget = size_t(double(fr) * 0.9);
    }
  }
  s->st.hbm_budget = s->o.hbm_budget;
  s->idle_workers = o->workers;
  s->has_lane = s->lane_idle = o->group_dofs > 0;
  s->builder = std::thread(builder_loop, s);
  for (int w = 0; w < o->workers; ++w) s->workers.emplace_back(worker_loop, s, w, false);
  if (s->has_lane) s->workers.emplace_back(worker_loop, s, o->workers, true);
  *out = s;
  return LDGMG_OK;
}

ldgmg_status ldgmg_server_submit(ldgmg_server* s, const ldgmg_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket) return serr(LDGMG_EINVAL, "null argument");
  if (q->dim != 2 && q->dim != 3) return serr(LDGMG_EINVAL, "dim must be 2 or 3");
  if (q->n < 1 || q->n > 4096 || q->p < 1 || q->p > 5) return serr(LDGMG_EINVAL, "n or p out of range");
  if (q->stokes < -1 || q->stokes > 1) return serr(LDGMG_EINVAL, "stokes must be -1, 0 or 1");
  if (!q->rhs_host || !q->x_host) return serr(LDGMG_EINVAL, "rhs_host and x_host are required");
  if (!(q->tol > 0.0)) return serr(LDGMG_EINVAL, "tol must be positive");
  int64_t N = 1;
  int bs = 1;
  for (int t = 0; t < q->dim; ++t) {
    N *= q->n;
    bs *= q->p + 1;
  }
  const int b = (q->stokes >= 0 ? q->dim + 1 : 1) * bs;
  ClassKey k{q->dim, q->n, q->p, q->stokes, q->tau0, q->stokes >= 0 ? q->taup : 0.0,
             q->mu_host ? fnv1a(q->mu_host, size_t(N) * sizeof(double)) : 0};
  auto r = std::make_shared<Req>();
  r->rhs.assign(q->rhs_host, q->rhs_host + size_t(N) * b);
  r->x_host = q->x_host;
  r->tol = q->tol;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return serr(LDGMG_EINVAL, "server is shutting down");
  auto it = s->classes.find(k);
  if (it == s->classes.end()) {
    auto c = std::make_unique<Class>();
    c->key = k;
    if (q->mu_host) c->mu.assign(q->mu_host, q->mu_host + N);
    c->b = b;
    c->N = N;
    // Scalar classes take up to max_batch right-hand sides per call (tensor
    // cores where the hierarchy supports them, else the CUDA-core kernels),
    // capped so that a call holds at most 2^22 dofs; GMRES classes take one.
    // Small scalar classes (at most group_dofs unknowns, CG) take one
    // right-hand side per hierarchy and are solved in grouped calls.
    const int64_t cap = std::max<int64_t>(1, (int64_t(1) << 22) / (N * b));
    const int kr = s->o.setup.krylov;
    c->small = q->stokes < 0 && size_t(N) * size_t(b) <= s->o.group_dofs &&
               (kr == LDGMG_KRYLOV_AUTO || kr == LDGMG_KRYLOV_CG);
    c->rmax = q->stokes < 0 && !c->small ? int(std::min<int64_t>(s->o.max_batch, cap)) : 1;
    it = s->classes.emplace(k, std::move(c)).first;
  }
  r->id = s->next_id++;
  r->res.t_submit = s->now();
  r->res.relres = std::numeric_limits<double>::quiet_NaN();
  it->second->queue.push_back(r);
  s->tickets.emplace(r->id, r);
  s->outstanding++;
  s->st.submitted++;
  *ticket = r->id;
  plan(s);
  s->cv_done.notify_all();   // plan may have completed requests (refused classes)
  return LDGMG_OK;
}

ldgmg_status ldgmg_server_wait(ldgmg_server* s, uint64_t ticket, ldgmg_result* out) {
  if (!s || !out) return serr(LDGMG_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return serr(LDGMG_EINVAL, "unknown ticket");
  auto r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  *out = r->res;
  s->tickets.erase(ticket);
  return LDGMG_OK;
}

ldgmg_status ldgmg_server_get_stats(ldgmg_server* s, ldgmg_server_stats* out) {
  if (!s || !out) return serr(LDGMG_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return LDGMG_OK;
}

double ldgmg_server_clock(const ldgmg_server* s) { return s ? s->now() : 0.0; }

void ldgmg_server_destroy(ldgmg_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
    s->stop = true;
  }
  s->cv_build.notify_all();
  s->cv_work.notify_all();
  if (s->builder.joinable()) s->builder.join();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  for (auto& kv : s->classes) free_class(kv.second.get());
  delete s;
}

}  // extern "C"
