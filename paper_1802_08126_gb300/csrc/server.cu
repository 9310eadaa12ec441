// Serving loop: continuous batching of time-global solves on one GPU.
//
// Requests (any grid, N_t, coefficient, precision) enter a queue.  One worker thread owns the
// device work: at every iteration boundary it admits queued requests while the device memory
// they need (estimated before creation) fits the budget and an active slot is free, creates
// their problems (state stays resident on the device), and then launches one CUDA graph that
// holds one Uzawa iteration of every active problem (each problem's captured iteration as a
// child graph).  Every few launches it reads all done flags; finished solves are copied to
// host memory, their device memory is released, waiters are woken, and the graph is rebuilt
// for the new active set.  Requests that arrive while others run are therefore admitted as
// slots and memory free up, and their iterations overlap with the others' on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pt_internal.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  unsigned long long ticket = 0;
  pt_grid grid{};
  int N = 0;
  double T = 0.0;
  pt_coeff coeff{};
  pt_options opt{};
  std::vector<double> f, u0, steps;
  bool seeded = false;
  unsigned long long seed = 0;
  double tol = 0.0;
  int max_it = 0;
  size_t est_bytes = 0;
  long long dofs = 0;
  double t_submit = 0.0, t_done = 0.0;
  pt_problem* prob = nullptr;
  std::vector<double> u;
  int iters = 0;
  pt_status status = PT_OK;
  bool done = false;
  bool failed = false;
  std::string error;
};

}  // namespace

struct pt_server {
  int device = 0;
  size_t budget = 0;
  int max_active = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::map<unsigned long long, Request*> all;
  bool stop = false;
  unsigned long long next_ticket = 1;
  size_t used = 0;
  // device side (worker thread only)
  cudaStream_t st = nullptr;
  cudaGraph_t parent = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  pt::SolveState** dstates = nullptr;
  int* ddone = nullptr;
  int* hdone = nullptr;
  int cap = 0;
  // statistics
  std::vector<double> lat_ms;
  double dofs_done = 0.0, t_first = 0.0, t_last = 0.0;
  int completed = 0;
};

namespace {

void release(Request* r) {
  if (r->prob) pt_problem_destroy(r->prob);
  r->prob = nullptr;
}

// Create and start the solve of an admitted request (worker thread, device current).
bool start(Request* r) {
  pt_problem* p = nullptr;
  pt_status s = pt_problem_create(&r->grid, r->N, r->T, &r->coeff, r->seeded ? nullptr : r->f.data(), 0,
                                  r->u0.empty() ? nullptr : r->u0.data(), 0, &r->opt, &p);
  if (s == PT_OK && r->seeded)
    s = pt_problem_set_rhs_uniform(p, r->seed, r->u0.empty() ? nullptr : r->u0.data(), 0);
  if (s == PT_OK) s = pt::problem_begin(p, r->tol, r->max_it);
  if (s != PT_OK) {
    r->failed = true;
    r->status = s;
    r->error = pt_last_error();
    if (p) pt_problem_destroy(p);
    return false;
  }
  r->prob = p;
  return true;
}

cudaError_t rebuild(pt_server* sv) {
  if (sv->exec) cudaGraphExecDestroy(sv->exec);
  if (sv->parent) cudaGraphDestroy(sv->parent);
  sv->exec = nullptr;
  sv->parent = nullptr;
  sv->kernels = 0;
  if (sv->active.empty()) return cudaSuccess;
  if ((int)sv->active.size() > sv->cap) {
    if (sv->dstates) cudaFree(sv->dstates);
    if (sv->ddone) cudaFree(sv->ddone);
    if (sv->hdone) cudaFreeHost(sv->hdone);
    sv->cap = std::max<int>((int)sv->active.size(), 2 * sv->cap);
    cudaError_t e = cudaMalloc(&sv->dstates, sizeof(pt::SolveState*) * sv->cap);
    if (e == cudaSuccess) e = cudaMalloc(&sv->ddone, sizeof(int) * sv->cap);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->hdone, sizeof(int) * sv->cap);
    if (e != cudaSuccess) return e;
  }
  std::vector<pt::SolveState*> states;
  cudaError_t e = cudaGraphCreate(&sv->parent, 0);
  for (Request* r : sv->active) {
    if (e != cudaSuccess) break;
    unsigned long long k = 0;
    cudaGraph_t child = pt::problem_graph(r->prob, &k);
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, sv->parent, nullptr, 0, child);
    sv->kernels += k;
    states.push_back(pt::problem_state(r->prob));
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sv->dstates, states.data(), sizeof(pt::SolveState*) * states.size(), cudaMemcpyHostToDevice,
                        sv->st);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sv->exec, sv->parent, 0);
  return e;
}

void finish(pt_server* sv, Request* r) {
  int iters = 0;
  pt_status status = PT_OK;
  pt_status s = pt::problem_result(r->prob, &iters, &status);
  r->u.assign((size_t)r->dofs, 0.0);
  if (s == PT_OK) s = pt_problem_get_state(r->prob, r->u.data(), nullptr, 0);
  if (s != PT_OK) {
    r->failed = true;
    r->status = s;
    r->error = pt_last_error();
  } else {
    r->iters = iters;
    r->status = status;
  }
  release(r);
  r->t_done = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->used -= r->est_bytes;
  r->done = true;
  sv->lat_ms.push_back(1e3 * (r->t_done - r->t_submit));
  sv->dofs_done += (double)r->dofs;
  sv->t_last = r->t_done;
  sv->completed += 1;
  sv->cv_done.notify_all();
}

void worker(pt_server* sv) {
  cudaSetDevice(sv->device);
  cudaStreamCreateWithFlags(&sv->st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (sv->active.empty())
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->pending.empty(); });
      if (sv->stop && sv->pending.empty() && sv->active.empty()) break;
      while (!sv->pending.empty() && (int)(sv->active.size() + admit.size()) < sv->max_active) {
        Request* r = sv->pending.front();
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const bool fits = sv->used + r->est_bytes <= sv->budget && r->est_bytes + (size_t)(1u << 30) <= free_b;
        if (!fits && !(sv->active.empty() && admit.empty())) break;  // wait for memory to free up
        sv->pending.pop_front();
        sv->used += r->est_bytes;
        admit.push_back(r);
      }
    }
    bool changed = false;
    for (Request* r : admit) {
      if (start(r)) {
        sv->active.push_back(r);
        changed = true;
      } else {
        r->t_done = now_s();
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= r->est_bytes;
        r->done = true;
        sv->cv_done.notify_all();
      }
    }
    if (sv->active.empty()) continue;
    if (changed && rebuild(sv) != cudaSuccess) {
      cudaGetLastError();
      for (Request* r : sv->active) {
        r->failed = true;
        r->status = PT_ECUDA;
        r->error = "graph build failed";
        release(r);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= r->est_bytes;
        r->done = true;
      }
      sv->active.clear();
      sv->cv_done.notify_all();
      continue;
    }
    // a few iterations of every active solve, then read the done flags
    for (int k = 0; k < 4; ++k) {
      cudaGraphLaunch(sv->exec, sv->st);
      pt::note_launch((int)sv->kernels);
    }
    const int na = (int)sv->active.size();
    pt::launch_gather_done(sv->dstates, na, sv->ddone, sv->st);
    cudaMemcpyAsync(sv->hdone, sv->ddone, sizeof(int) * na, cudaMemcpyDeviceToHost, sv->st);
    cudaStreamSynchronize(sv->st);
    std::vector<Request*> still;
    bool any = false;
    for (int i = 0; i < na; ++i) {
      if (sv->hdone[i]) {
        finish(sv, sv->active[i]);
        any = true;
      } else {
        still.push_back(sv->active[i]);
      }
    }
    if (any) {
      sv->active.swap(still);
      if (rebuild(sv) != cudaSuccess) cudaGetLastError();
    }
  }
  if (sv->exec) cudaGraphExecDestroy(sv->exec);
  if (sv->parent) cudaGraphDestroy(sv->parent);
  if (sv->dstates) cudaFree(sv->dstates);
  if (sv->ddone) cudaFree(sv->ddone);
  if (sv->hdone) cudaFreeHost(sv->hdone);
  cudaStreamDestroy(sv->st);
}

pt_status sfail(pt_status s, const char* m) {
  pt::set_last_error(m);
  return s;
}

}  // namespace

extern "C" {

pt_status pt_server_create(size_t hbm_budget, int max_active, pt_server** out) {
  pt::set_last_error("");
  if (!out) return sfail(PT_EINVAL, "out is NULL");
  *out = nullptr;
  pt_server* sv = new pt_server();
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return sfail(PT_ECUDA, "cudaGetDevice failed");
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete sv;
    return sfail(PT_ECUDA, "cudaMemGetInfo failed");
  }
  sv->budget = hbm_budget > 0 ? std::min(hbm_budget, free_b) : (size_t)(0.85 * (double)free_b);
  sv->max_active = max_active > 0 ? max_active : 256;
  sv->worker = std::thread(worker, sv);
  *out = sv;
  return PT_OK;
}

pt_status pt_server_submit(pt_server* sv, const pt_grid* grid, int N_t, double T, const pt_coeff* coeff,
                           const double* f, unsigned long long f_seed, const double* u0,
                           const pt_options* opts, double tol, int max_it, unsigned long long* ticket) {
  pt::set_last_error("");
  if (!sv || !grid || !coeff || !ticket) return sfail(PT_EINVAL, "NULL argument");
  if (max_it < 0 || !(tol >= 0.0)) return sfail(PT_EINVAL, "need max_it >= 0 and tol >= 0");
  if (grid->dim < 1 || grid->dim > 3 || N_t < 1) return sfail(PT_EINVAL, "bad grid or N_t");
  Request* r = new Request();
  r->grid = *grid;
  r->N = N_t;
  r->T = T;
  r->coeff = *coeff;
  if (opts) r->opt = *opts;
  r->opt.stream = nullptr;
  if (r->opt.tau_steps) {  // the request outlives the caller's array
    r->steps.assign(r->opt.tau_steps, r->opt.tau_steps + N_t);
    r->opt.tau_steps = r->steps.data();
  }
  long long ns = 1;
  for (int d = 0; d < grid->dim; ++d) ns *= grid->n[d];
  r->dofs = ns * N_t;
  if (f) {
    r->f.assign(f, f + r->dofs);
  } else {
    r->seeded = true;
    r->seed = f_seed;
  }
  if (u0) r->u0.assign(u0, u0 + ns);
  r->tol = tol;
  r->max_it = max_it;
  r->est_bytes = pt::estimate_problem_bytes(grid, N_t, &r->opt);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete r;
      return sfail(PT_EBUSY, "server is shutting down");
    }
    if (r->est_bytes > sv->budget) {
      delete r;
      return sfail(PT_ENOMEM, "request needs more device memory than the server budget");
    }
    r->ticket = sv->next_ticket++;
    if (sv->t_first == 0.0) sv->t_first = r->t_submit;
    sv->all[r->ticket] = r;
    sv->pending.push_back(r);
    *ticket = r->ticket;
  }
  sv->cv_work.notify_one();
  return PT_OK;
}

pt_status pt_server_wait(pt_server* sv, unsigned long long ticket, int timeout_ms, double* u_out, int* iters,
                         pt_status* solve_status) {
  pt::set_last_error("");
  if (!sv) return sfail(PT_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return sfail(PT_EINVAL, "unknown ticket");
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0)
    sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return sfail(PT_ETIMEOUT, "request not finished within the timeout");
  sv->all.erase(it);
  lk.unlock();
  pt_status ret = PT_OK;
  if (r->failed) {
    pt::set_last_error(r->error.c_str());
    ret = r->status;
  } else {
    if (u_out) std::copy(r->u.begin(), r->u.end(), u_out);
    if (iters) *iters = r->iters;
    if (solve_status) *solve_status = r->status;
  }
  delete r;
  return ret;
}

pt_status pt_server_stats(pt_server* sv, double* p50_ms, double* p99_ms, double* dofs_per_s, int* completed) {
  if (!sv) return sfail(PT_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::vector<double> v = sv->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    return v[i];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (dofs_per_s) *dofs_per_s = sv->t_last > sv->t_first ? sv->dofs_done / (sv->t_last - sv->t_first) : 0.0;
  if (completed) *completed = sv->completed;
  return PT_OK;
}

void pt_server_destroy(pt_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& kv : sv->all) {
    release(kv.second);
    delete kv.second;
  }
  delete sv;
}

}  // extern "C"
