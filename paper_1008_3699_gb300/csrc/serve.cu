// Continuous-batching solve server (no counterpart in the paper: a serving
// pattern around the library's solvers).
//
// serve_submit copies a request (matrix, right-hand side, method) and queues
// it; worker threads ("slots"), each with a CUDA stream of its own, take the
// first queued request whose estimated device memory fits the remaining
// budget (free device memory at start unless given), so a request that
// arrives while others run is admitted as soon as a slot and memory free up,
// and the solves of several requests overlap on the device. A request keeps
// its factors and vectors resident for its whole solve and releases them at
// the end. serve_poll returns NDIAG_EBUSY until the request has finished, then
// its status, solver info, queue/run/latency times and (optionally) x.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

using Clock = std::chrono::steady_clock;

namespace {

struct Job {
  uint64_t ticket = 0;
  ndiag_request req{};
  std::vector<double> diags, b, x;
  size_t mem = 0;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  ndiag_result res{};
};

// Device bytes of one solve: the fp64 matrix, the sweep-precision matrix and
// scaled sets, about twelve vectors and the line tables / scratch.
size_t estimate_bytes(const ndiag_request& r, int64_t N) {
  const size_t cs = r.precision == NDIAG_FP64 ? 8 : (r.precision == NDIAG_FP32 ? 4 : 2);
  const size_t s = (size_t)r.stencil;
  size_t b = (size_t)N * (s * 8 + s * (r.precision == NDIAG_FP64 ? 0 : 4) + 3 * s * cs + 12 * 8);
  return b + (64u << 20);
}

}  // namespace

struct ndiag_server {
  std::mutex mu, mu9;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  size_t budget = 0, in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int running = 0, max_running = 0, device = 0;
  int64_t solved = 0;
};

namespace {

void run_job(Job& j, cudaStream_t s) {
  const ndiag_request& r = j.req;
  ndiag_result& out = j.res;
  ndiag* h = nullptr;
  ndiag_status st = ndiag_create(&h, r.dim, r.n, r.stencil, j.diags.data(), r.sub, r.precision, s);
  double* dev = nullptr;
  int64_t N = 0;
  if (st == NDIAG_OK) {
    N = ndiag_cells(h);
    dev = (double*)nd::dev_alloc(sizeof(double) * 2 * (size_t)N, s);
    if (!dev) st = NDIAG_ENOMEM;
  }
  // the full factor of every subdomain block: on 9-point matrices it needs about a
  // third fewer BiCGSTAB iterations than D-ILU; on 5/7-point ones it is the same factor
  if (st == NDIAG_OK && r.precond == NDIAG_PREC_ILU0) st = ilu0_factor(h, NDIAG_DECOMPOSED_FULL);
  if (st == NDIAG_OK) {
    cudaMemcpyAsync(dev, j.b.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(dev + N, 0, sizeof(double) * N, s);
    double om[8];
    for (double& v : om) v = r.omega > 0.0 ? r.omega : 1.0;
    st = krylov_solve(h, r.method, r.precond, NDIAG_DECOMPOSED, om, r.rtol, r.maxit, dev, dev + N, &out.info);
    j.x.resize((size_t)N);
    if (cudaMemcpyAsync(j.x.data(), dev + N, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      if (st == NDIAG_OK) st = NDIAG_EDEVICE;
    }
  }
  if (dev) nd::dev_free(dev, sizeof(double) * 2 * (size_t)N, s);
  if (h) ndiag_destroy(h);
  cudaStreamSynchronize(s);
  out.status = st;
  out.cells = N;
}

void worker(ndiag_server* S) {
  cudaSetDevice(S->device);
  nd::use_plain_allocator_on_this_thread(true);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] {
        if (S->stop && S->queue.empty()) return true;
        for (auto& q : S->queue)
          if (q->mem + S->in_use <= S->budget || S->in_use == 0) return true;
        return false;
      });
      if (S->stop && S->queue.empty()) break;
      // first queued request that fits; a request larger than the whole budget runs alone
      for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
        if ((*it)->mem + S->in_use <= S->budget || S->in_use == 0) {
          j = *it;
          S->queue.erase(it);
          break;
        }
      if (!j) continue;
      S->in_use += j->mem;
      ++S->running;
      S->max_running = std::max(S->max_running, S->running);
    }
    j->t_start = Clock::now();
    if (j->req.stencil == 9 && nd::sweep9_needs_residency(j->req.n[1], j->req.sub[1])) {
      // tall 9-point subdomains keep the CTAs of an x-interface in step
      // through global memory and need all of them resident: one such solve
      // at a time
      std::lock_guard<std::mutex> lk9(S->mu9);
      run_job(*j, s);
    } else {
      run_job(*j, s);
    }
    j->t_end = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= j->mem;
      --S->running;
      ++S->solved;
      auto sec = [](Clock::duration d) { return std::chrono::duration<double>(d).count(); };
      j->res.queue_s = sec(j->t_start - j->t_submit);
      j->res.run_s = sec(j->t_end - j->t_start);
      j->res.latency_s = sec(j->t_end - j->t_submit);
      j->done = true;
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  cudaStreamDestroy(s);
}

}  // namespace

extern "C" {

ndiag_status ndiag_server_create(ndiag_server** out, int slots, size_t mem_budget) {
  if (!out) return NDIAG_EINVAL;
  *out = nullptr;
  if (slots < 1 || slots > 64) return NDIAG_EINVAL;
  ndiag_server* S = new ndiag_server();
  cudaGetDevice(&S->device);
  if (mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return NDIAG_EDEVICE;
    }
    mem_budget = fr / 10 * 8;
  }
  S->budget = mem_budget;
  for (int k = 0; k < slots; ++k) S->workers.emplace_back(worker, S);
  *out = S;
  return NDIAG_OK;
}

ndiag_status serve_submit(ndiag_server* S, const ndiag_request* r, uint64_t* ticket) {
  if (!S || !r || !ticket || !r->diags || !r->b) return NDIAG_EINVAL;
  const bool ok = (r->dim == 2 && (r->stencil == 5 || r->stencil == 9)) || (r->dim == 3 && r->stencil == 7);
  if (!ok || !(r->rtol > 0.0) || r->maxit < 1) return NDIAG_EINVAL;
  int64_t N = 1;
  for (int a = 0; a < r->dim; ++a) {
    if (r->n[a] < 1) return NDIAG_EINVAL;
    N *= r->n[a];
  }
  auto j = std::make_shared<Job>();
  j->req = *r;
  j->diags.assign(r->diags, r->diags + (size_t)r->stencil * (size_t)N);
  j->b.assign(r->b, r->b + (size_t)N);
  j->req.diags = nullptr;
  j->req.b = nullptr;
  j->mem = estimate_bytes(*r, N);
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return NDIAG_EBUSY;
    j->ticket = S->next_ticket++;
    S->jobs[j->ticket] = j;
    S->queue.push_back(j);
    *ticket = j->ticket;
  }
  S->cv_work.notify_all();
  return NDIAG_OK;
}

ndiag_status serve_poll(ndiag_server* S, uint64_t ticket, ndiag_result* out, double* x) {
  if (!S || !out) return NDIAG_EINVAL;
  std::shared_ptr<Job> j;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return NDIAG_EINVAL;
    if (!it->second->done) return NDIAG_EBUSY;
    j = it->second;
    S->jobs.erase(it);
  }
  *out = j->res;
  if (x && !j->x.empty()) std::memcpy(x, j->x.data(), sizeof(double) * j->x.size());
  return NDIAG_OK;
}

ndiag_status ndiag_server_wait(ndiag_server* S, uint64_t ticket, double timeout_s) {
  if (!S) return NDIAG_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return NDIAG_EINVAL;
  std::shared_ptr<Job> j = it->second;
  const bool done = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->done; });
  return done ? NDIAG_OK : NDIAG_EBUSY;
}

ndiag_status ndiag_server_stats(ndiag_server* S, ndiag_server_stats_t* out) {
  if (!S || !out) return NDIAG_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  out->queued = (int)S->queue.size();
  out->running = S->running;
  out->max_running = S->max_running;
  out->solved = S->solved;
  out->budget_bytes = (int64_t)S->budget;
  out->in_use_bytes = (int64_t)S->in_use;
  return NDIAG_OK;
}

void ndiag_server_destroy(ndiag_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (std::thread& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
