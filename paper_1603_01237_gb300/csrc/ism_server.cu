// ism_server.cu -- a request loop that serves ISM solves of different sizes concurrently on one GPU,
// with continuous batching.
//
// The paper runs one control problem at a time over N processors.  A solver service receives many
// problems of different Hilbert dimensions, step counts and N.  Each submitted request (problem,
// options, initial controls, iteration count) is copied and queued; `slots` worker threads each own a
// CUDA stream and take requests in arrival order.
//
// Continuous batching.  Requests that can share launches -- the structured kinds (tridiagonal, bit-flip)
// in mixed precision with the Chebyshev step and one local step -- are grouped by (kind, d, N,
// objective): a worker opens a shared plan of `group_capacity` rows (each row its own Hamiltonian,
// states, step count, control time and step size), admits every queued request of that group, and
// runs ISM passes over the active rows.  Between passes it retires the requests that have done their
// iterations (the last row moves into the hole, so the active rows stay contiguous) and admits
// requests that arrived meanwhile into the free rows: a request joins while others are half-way
// through their solves.  Each pass records J at the rows' current controls; a request's final pass
// only evaluates (its step size is set to 0).  Every kernel treats the rows independently and the
// warp-wide term and step counts add exact no-ops, so a request's result is the same alone and in
// the mix, bit for bit.  Other requests (FP64, the grid, Pauli and dense kinds, Crank-Nicolson,
// several local steps) run on a plan of their own, as a whole solve.
//
// Admission by device footprint: a shared plan (or a request's own plan) starts only when its bytes
// fit in what the budget has left; plans allocate and free stream-ordered.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "ism.h"
#include "ism_launch.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  long long id = 0;
  ism_problem prob{};
  ism_options opt{};
  std::vector<double> H0, H1, H0i, H1i, psi_i, psi_f, O, alpha, u, J;
  int iters = 0;
  size_t bytes = 0;
  bool batchable = false;
  bool h1diag = true;
  int passes = 0;          // passes done in a shared plan (J recorded for each)
  int state = ISM_REQ_QUEUED;
  int status = ISM_OK;
  std::string message;
  double t_submit = 0, t_start = 0, t_done = 0;
};

template <class T>
std::vector<T> copy_of(const T* p, size_t n) {
  return p ? std::vector<T>(p, p + n) : std::vector<T>();
}

// The requests that can share a plan: same kind, d, N, objective (and, for the tridiagonal kind, whether
// H1 has a diagonal, which selects the kernel variant).
struct GroupKey {
  int kind, d, N, obj;
  bool h1diag;
};
GroupKey key_of(const Request* r) { return GroupKey{r->prob.kind, r->prob.d, r->prob.N, r->prob.objective, r->h1diag}; }
bool in_group(const Request* a, const GroupKey& k) {
  return a->batchable && a->prob.kind == k.kind && a->prob.d == k.d && a->prob.N == k.N && a->prob.objective == k.obj &&
         a->h1diag == k.h1diag;
}

// step size of a request's next pass: 0 once it has done its iterations (the pass evaluates J only)
double rho_next(const Request* r) { return r->passes < r->iters ? r->opt.rho : 0.0; }

}  // namespace

struct ism_server_s {
  ism_server_options o{};
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv;         // queue, budget or state changed
  std::deque<Request*> queue;
  std::unordered_map<long long, std::unique_ptr<Request>> all;
  long long next_id = 0;
  size_t used = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  long long st_passes = 0, st_rows = 0, st_max_rows = 0, st_groups = 0, st_single = 0;

  int capacity() const { return o.group_capacity > 0 ? o.group_capacity : 64; }
  int max_steps(const Request* r) const { return std::max(r->prob.Nt, o.group_max_steps > 0 ? o.group_max_steps : 50000); }

  void finish(Request* r, int rc, const std::string& msg) {
    r->status = rc;
    r->message = msg;
    r->state = rc == ISM_OK ? ISM_REQ_DONE : ISM_REQ_FAILED;
    r->t_done = now_ms();
  }

  // A worker's own plan for a request that cannot share launches: the whole solve at once.
  void run_single(Request* r, cudaStream_t st) {
    ism_plan_t plan = nullptr;
    int rc = ism_plan(&r->prob, &r->opt, st, &plan);
    if (rc == ISM_OK) rc = ism_iterate(plan, r->iters, r->u.data(), r->J.data(), nullptr);
    std::string msg = rc == ISM_OK ? std::string() : std::string(ism_last_error());
    if (plan) ism_plan_destroy(plan);
    std::lock_guard<std::mutex> lk(mu);
    used -= r->bytes;
    ++st_single;
    finish(r, rc, msg);
  }

  // Take the queued requests of group k that fit (Nt <= Ntmax), up to `room`; mu held.
  void take_group(const GroupKey& k, int Ntmax, int room, std::vector<Request*>* out) {
    for (auto it = queue.begin(); it != queue.end() && room > 0;) {
      if (in_group(*it, k) && (*it)->prob.Nt <= Ntmax) {
        (*it)->state = ISM_REQ_RUNNING;
        (*it)->t_start = now_ms();
        out->push_back(*it);
        it = queue.erase(it);
        --room;
      } else {
        ++it;
      }
    }
  }

  // A shared plan: passes over the active rows, retiring and admitting between passes.
  void run_group(std::vector<Request*> rows, int Ntmax, int cap, size_t gbytes, cudaStream_t st) {
    const GroupKey key = key_of(rows.front());   // the requests themselves may be released once finished
    ism_plan_t plan = nullptr;
    int rc = ism::het_create(key.kind, key.d, key.N, key.obj, key.h1diag, Ntmax, cap, st, &plan, nullptr);
    std::string msg = rc == ISM_OK ? std::string() : std::string(ism_last_error());
    auto fail_all = [&](std::vector<Request*>& rs) {
      std::lock_guard<std::mutex> lk(mu);
      for (Request* q : rs) finish(q, rc, msg);
      rs.clear();
    };
    for (size_t i = 0; i < rows.size() && rc == ISM_OK; ++i) {
      rc = ism::het_set_row(plan, (int)i, rows[i]->prob, rows[i]->u.data(), rho_next(rows[i]));
      if (rc != ISM_OK) msg = ism_last_error();
    }
    std::vector<double> J(cap);
    while (rc == ISM_OK && !rows.empty()) {
      const int A = (int)rows.size();
      rc = ism::het_step(plan, A, J.data());
      if (rc != ISM_OK) { msg = ism_last_error(); break; }
      std::vector<int> done;
      for (int i = 0; i < A && rc == ISM_OK; ++i) {
        Request* q = rows[i];
        q->J[q->passes] = J[i];
        ++q->passes;
        if (q->passes == q->iters + 1) {
          rc = ism::het_get_u(plan, i, q->u.data(), q->prob.Nt);
          done.push_back(i);
        } else if (q->passes == q->iters) {
          rc = ism::het_set_rho(plan, i, 0.0);   // the next pass evaluates J[u^(iters)] only
        }
      }
      if (rc != ISM_OK) { msg = ism_last_error(); break; }
      // retire: the last active row moves into each hole (from the highest hole down)
      std::vector<Request*> finished;
      for (int k = (int)done.size() - 1; k >= 0 && rc == ISM_OK; --k) {
        const int i = done[k], last = (int)rows.size() - 1;
        finished.push_back(rows[i]);
        if (i != last) {
          rc = ism::het_set_row(plan, i, rows[last]->prob, nullptr, rho_next(rows[last]));
          if (rc == ISM_OK) rc = ism::het_move_u(plan, last, i);
          rows[i] = rows[last];
        }
        rows.pop_back();
      }
      if (rc != ISM_OK) { msg = ism_last_error(); rows.insert(rows.end(), finished.begin(), finished.end()); break; }
      std::vector<Request*> joined;
      {
        std::lock_guard<std::mutex> lk(mu);
        for (Request* q : finished) finish(q, ISM_OK, std::string());
        ++st_passes;
        st_rows += A;
        st_max_rows = std::max<long long>(st_max_rows, A);
        take_group(key, Ntmax, cap - (int)rows.size(), &joined);   // continuous batching
      }
      cv.notify_all();
      for (Request* q : joined) {
        const int i = (int)rows.size();
        rows.push_back(q);
        if (rc == ISM_OK) {
          rc = ism::het_set_row(plan, i, q->prob, q->u.data(), rho_next(q));
          if (rc != ISM_OK) msg = ism_last_error();
        }
      }
    }
    if (rc != ISM_OK) fail_all(rows);
    if (plan) ism_plan_destroy(plan);
    {
      std::lock_guard<std::mutex> lk(mu);
      used -= gbytes;
    }
    cv.notify_all();
  }

  void work() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
      Request* r = nullptr;
      int Ntmax = 0, cap = 0;
      size_t need = 0;
      std::vector<Request*> group;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] {
          if (stop) return true;
          if (queue.empty()) return false;
          Request* f = queue.front();
          need = f->bytes;
          if (f->batchable) {   // the shared plan's footprint: as many rows as the whole budget holds
            Ntmax = max_steps(f);
            for (cap = capacity(); cap >= 1; cap /= 2) {
              size_t gb = 0;
              if (ism::het_create(f->prob.kind, f->prob.d, f->prob.N, f->prob.objective, f->h1diag, Ntmax, cap,
                                  nullptr, nullptr, &gb) == ISM_OK &&
                  gb + (1u << 20) <= o.hbm_budget_bytes) {
                need = gb + (1u << 20);
                break;
              }
            }
            if (cap < 1) f->batchable = false;   // not even one row fits: a plan of its own
          }
          return used + need <= o.hbm_budget_bytes;
        });
        if (stop) break;
        r = queue.front();
        used += need;
        if (r->batchable) {   // the group's queued requests, taken under this lock
          take_group(key_of(r), Ntmax, cap, &group);
          ++st_groups;
        } else {
          queue.pop_front();
          r->state = ISM_REQ_RUNNING;
          r->t_start = now_ms();
        }
      }
      cv.notify_all();
      if (r->batchable) run_group(std::move(group), Ntmax, cap, need, st);
      else run_single(r, st);
      cv.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

namespace {

// Copies the request's problem, options and controls and queues it; returns its id.  Host
// allocations here may throw std::bad_alloc, which the extern "C" caller turns into ISM_ENOMEM.
long long enqueue_copy(ism_server_s* S, const ism_problem& p, const ism_options& opt, const double* u0, int iters,
                       size_t bytes) {
  auto r = std::make_unique<Request>();
  const int d = p.d;
  const int B = p.batch < 1 ? 1 : p.batch;
  const bool gp = p.kind == ISM_H_GRID_GP || p.kind == ISM_H_GRID_GP_DOUBLE_WELL;
  int q = 0;
  while (q < 30 && (1 << q) < d) ++q;
  const size_t nH0 = gp ? (p.kind == ISM_H_GRID_GP_DOUBLE_WELL ? 4 : 3) : p.kind == ISM_H_DENSE ? (size_t)d * d : p.kind == ISM_H_TRIDIAG ? 2 * (size_t)d - 1 : (size_t)d;
  const size_t m = p.kind == ISM_H_PAULI && p.controls > 1 ? (size_t)p.controls : 1;
  const size_t nH1 = gp ? 0
                     : p.kind == ISM_H_DENSE   ? (size_t)d * d
                     : p.kind == ISM_H_TRIDIAG ? 2 * (size_t)d - 1
                     : p.kind == ISM_H_PAULI   ? 2 * m * q
                                               : (size_t)q;
  r->H0 = copy_of(p.H0, nH0);
  r->H1 = copy_of(p.H1, nH1);
  if (p.kind == ISM_H_DENSE) {   // imaginary parts of a complex Hermitian H
    r->H0i = copy_of(p.H0_imag, nH0);
    r->H1i = copy_of(p.H1_imag, nH1);
  }
  r->psi_i = copy_of(p.psi_i, 2 * (size_t)d);
  if (p.objective == ISM_OBJ_OVERLAP) r->psi_f = copy_of(p.psi_f, 2 * (size_t)d);
  else r->O = copy_of(p.O, (size_t)d * d);
  r->alpha = copy_of(p.alpha, (size_t)p.Nt);
  r->prob = p;
  r->prob.H0 = r->H0.empty() ? nullptr : r->H0.data();
  r->prob.H1 = r->H1.empty() ? nullptr : r->H1.data();
  r->prob.H0_imag = r->H0i.empty() ? nullptr : r->H0i.data();
  r->prob.H1_imag = r->H1i.empty() ? nullptr : r->H1i.data();
  r->prob.psi_i = r->psi_i.data();
  r->prob.psi_f = r->psi_f.empty() ? nullptr : r->psi_f.data();
  r->prob.O = r->O.empty() ? nullptr : r->O.data();
  r->prob.alpha = r->alpha.empty() ? nullptr : r->alpha.data();
  r->opt = opt;
  r->batchable = ism::het_batchable(p, opt) && S->o.group_capacity >= 0;
  r->h1diag = r->batchable ? ism::het_h1diag(p) : true;
  r->u.assign(u0, u0 + (size_t)B * p.Nt * m);
  r->J.assign((size_t)B * ((size_t)iters + 1), 0.0);
  r->iters = iters;
  r->bytes = bytes;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(S->mu);
  const long long rid = S->next_id++;
  r->id = rid;
  Request* raw = r.get();
  S->all.emplace(rid, std::move(r));
  try {
    S->queue.push_back(raw);
  } catch (...) {
    S->all.erase(rid);
    throw;
  }
  return rid;
}

}  // namespace

extern "C" {

int ism_server_create(const ism_server_options* opt, ism_server_t* out) {
  if (!opt || !out) return ism::set_error(ISM_EINVAL, "null argument");
  if (opt->slots < 1 || opt->slots > 64 || opt->hbm_budget_bytes == 0)
    return ism::set_error(ISM_EINVAL, "slots must be 1..64 and the budget > 0");
  if (opt->group_capacity > 4096 || opt->group_max_steps < 0)
    return ism::set_error(ISM_EINVAL, "group_capacity must be <= 4096 and group_max_steps >= 0");
  auto* S = new (std::nothrow) ism_server_s();
  if (!S) return ism::set_error(ISM_ENOMEM, "host memory for the server");
  S->o = *opt;
  cudaGetDevice(&S->dev);
  try {
    for (int i = 0; i < opt->slots; ++i) S->workers.emplace_back([S] { S->work(); });
  } catch (...) {
    // a worker thread could not be started: stop the ones that did and report it
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return ism::set_error(ISM_ENOMEM, "could not start the server's worker threads");
  }
  *out = S;
  return ISM_OK;
}

int ism_server_submit(ism_server_t S, const ism_problem* prob, const ism_options* opt, const double* u0, int iters,
                      long long* id) {
  if (!S || !prob || !opt || !u0 || !id || iters < 0) return ism::set_error(ISM_EINVAL, "null argument or iters < 0");
  size_t bytes = 0;
  int rc = ism_plan_footprint(prob, opt, &bytes);
  if (rc != ISM_OK) return rc;
  const int B = prob->batch < 1 ? 1 : prob->batch;
  bytes += 16 * (size_t)B * ((size_t)iters + 1) + (1u << 20);   // history buffers and slack
  if (bytes > S->o.hbm_budget_bytes)
    return ism::set_error(ISM_ENOMEM, "the request's device footprint exceeds the server's whole budget");
  try {
    *id = enqueue_copy(S, *prob, *opt, u0, iters, bytes);
  } catch (const std::bad_alloc&) {
    return ism::set_error(ISM_ENOMEM, "host memory for the request's copy of its problem");
  } catch (...) {
    return ism::set_error(ISM_EINVAL, "the request could not be queued");
  }
  S->cv.notify_all();
  return ISM_OK;
}

int ism_server_poll(ism_server_t S, long long id, int wait, int* state, double* u_out, double* J_hist,
                    double* times_ms) {
  if (!S || !state) return ism::set_error(ISM_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return ism::set_error(ISM_EINVAL, "unknown request id");
  Request* r = it->second.get();
  if (wait) S->cv.wait(lk, [&] { return r->state == ISM_REQ_DONE || r->state == ISM_REQ_FAILED; });
  *state = r->state;
  if (times_ms) {
    times_ms[0] = r->t_start > 0 ? r->t_start - r->t_submit : -1.0;
    times_ms[1] = r->t_done > 0 ? r->t_done - r->t_start : -1.0;
    times_ms[2] = r->t_done > 0 ? r->t_done - r->t_submit : -1.0;
  }
  if (r->state == ISM_REQ_DONE) {
    if (u_out) std::memcpy(u_out, r->u.data(), r->u.size() * sizeof(double));
    if (J_hist) std::memcpy(J_hist, r->J.data(), r->J.size() * sizeof(double));
  }
  if (r->state == ISM_REQ_FAILED) return ism::set_error(r->status, r->message.c_str());
  return ISM_OK;
}

int ism_server_release(ism_server_t S, long long id) {
  if (!S) return ism::set_error(ISM_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return ism::set_error(ISM_EINVAL, "unknown request id");
  const int st = it->second->state;
  if (st != ISM_REQ_DONE && st != ISM_REQ_FAILED) return ism::set_error(ISM_EINVAL, "the request has not finished");
  S->all.erase(it);
  return ISM_OK;
}

int ism_server_stats(ism_server_t S, long long* out) {
  if (!S || !out) return ism::set_error(ISM_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->st_passes;
  out[1] = S->st_rows;
  out[2] = S->st_max_rows;
  out[3] = S->st_groups;
  out[4] = S->st_single;
  return ISM_OK;
}

int ism_server_destroy(ism_server_t S) {
  if (!S) return ISM_OK;
  {
    // finish the requests already admitted; drop the queued ones
    std::unique_lock<std::mutex> lk(S->mu);
    for (Request* r : S->queue) {
      r->state = ISM_REQ_FAILED;
      r->status = ISM_EINVAL;
      r->message = "server destroyed before the request started";
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return ISM_OK;
}

}  // extern "C"
