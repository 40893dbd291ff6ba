// ism_server.cu -- a request loop that serves ISM solves of different sizes concurrently on one GPU.
//
// The paper runs one control problem at a time over N processors.  A solver service receives many
// problems of different Hilbert dimensions, step counts and N.  Here each submitted request (problem,
// options, initial controls, iteration count) is copied and queued; `slots` worker threads each own
// a CUDA stream and take requests in arrival order.  A request is admitted when its plan's device
// footprint (ism_plan_footprint) fits in the remaining budget, so that requests arriving while
// others run start as soon as a slot and memory are free; its plan (states, controls, adjoints,
// trajectories) stays resident on the device for the whole solve, and the solves of different
// slots overlap on the GPU.  Plans allocate and free stream-ordered, so admitting or retiring a
// request does not stall the others.  A request's result does not depend on what else runs: every
// kernel reads only its own plan.
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
  std::vector<double> H0, H1, psi_i, psi_f, O, alpha, u, J;
  int iters = 0;
  size_t bytes = 0;
  int state = ISM_REQ_QUEUED;
  int status = ISM_OK;
  std::string message;
  double t_submit = 0, t_start = 0, t_done = 0;
};

template <class T>
std::vector<T> copy_of(const T* p, size_t n) {
  return p ? std::vector<T>(p, p + n) : std::vector<T>();
}

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

  void work() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || (!queue.empty() && used + queue.front()->bytes <= o.hbm_budget_bytes); });
        if (stop) break;
        r = queue.front();
        queue.pop_front();
        used += r->bytes;
        r->state = ISM_REQ_RUNNING;
        r->t_start = now_ms();
      }
      cv.notify_all();
      ism_plan_t plan = nullptr;
      int rc = ism_plan(&r->prob, &r->opt, st, &plan);
      if (rc == ISM_OK) rc = ism_iterate(plan, r->iters, r->u.data(), r->J.data(), nullptr);
      std::string msg = rc == ISM_OK ? std::string() : std::string(ism_last_error());
      if (plan) ism_plan_destroy(plan);
      {
        std::lock_guard<std::mutex> lk(mu);
        used -= r->bytes;
        r->status = rc;
        r->message = msg;
        r->state = rc == ISM_OK ? ISM_REQ_DONE : ISM_REQ_FAILED;
        r->t_done = now_ms();
      }
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
  r->psi_i = copy_of(p.psi_i, 2 * (size_t)d);
  if (p.objective == ISM_OBJ_OVERLAP) r->psi_f = copy_of(p.psi_f, 2 * (size_t)d);
  else r->O = copy_of(p.O, (size_t)d * d);
  r->alpha = copy_of(p.alpha, (size_t)p.Nt);
  r->prob = p;
  r->prob.H0 = r->H0.empty() ? nullptr : r->H0.data();
  r->prob.H1 = r->H1.empty() ? nullptr : r->H1.data();
  r->prob.psi_i = r->psi_i.data();
  r->prob.psi_f = r->psi_f.empty() ? nullptr : r->psi_f.data();
  r->prob.O = r->O.empty() ? nullptr : r->O.data();
  r->prob.alpha = r->alpha.empty() ? nullptr : r->alpha.data();
  r->opt = opt;
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
