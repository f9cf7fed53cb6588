// Serving runtime: environment solves of mixed (cell, D, chi) as they arrive.
//
// A scheduler thread admits pending solves first-fit in arrival order while
// the sum of the admitted solves' device footprints (ctm_footprint) stays
// within the HBM budget and fewer than max_concurrent run. Every admitted
// solve gets its own host thread and its own context (own CUDA stream, own
// resident C, T, X, W), so the kernels of concurrent solves overlap on the
// device; a finished solve returns its footprint to the budget, and the
// scheduler admits the next ones (continuous batching). Results (corner
// spectra, optional bond energies, timings) stay with the server until the
// caller collects them with ctm_server_result.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ctm.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  ctm_solve_spec spec{};
  std::vector<std::vector<char>> A;    // owned copies of the tensors
  std::vector<const void*> Aptr;
  std::vector<char> op;
  size_t footprint = 0;
  double t_submit = 0, t_start = 0, t_end = 0;
  bool done = false;
  ctm_status status = CTM_OK;
  int iters = 0;
  double delta = 0;
  std::vector<double> spectra;         // [4][S][chi]
  std::vector<double> energies;        // [S][2 directions][re, im]
  std::string msg;
};

}  // namespace

struct ctm_server {
  int device = 0;
  size_t budget = 0, used = 0;
  int max_conc = 1, running = 0;
  std::mutex m;
  std::condition_variable cv_sched, cv_done;
  std::deque<Job*> pending;
  std::map<uint64_t, Job*> jobs;
  std::vector<std::thread> workers;
  std::thread scheduler;
  bool stop = false;
  uint64_t next_id = 1;
  std::vector<double> latencies;       // submit -> end of finished solves
  double first_submit = -1, last_end = 0;
  std::string msg;
};

namespace {

void run_job(ctm_server* sv, Job* j) {
  cudaSetDevice(sv->device);
  const ctm_solve_spec& s = j->spec;
  ctm_opts o = s.opts;
  o.stream = nullptr;   // a private stream per solve
  ctm_ctx* ctx = nullptr;
  ctm_status st = ctm_init(&ctx, s.Lx, s.Ly, j->Aptr.data(), nullptr, s.dtype, s.d, s.D, s.chi, &o);
  int it = 0;
  double delta = 0;
  std::vector<double> spectra, energies;
  std::string msg;
  if (st == CTM_OK) {
    st = ctm_converge(ctx, s.tol, s.max_iter, &it, &delta);
    if (st == CTM_ENOCONV) st = CTM_OK;   // reported through iters / delta
    const int S = s.Lx * s.Ly;
    spectra.assign((size_t)4 * S * s.chi, 0.0);
    for (int lab = 0; lab < 4 && st == CTM_OK; ++lab)
      for (int y = 0; y < s.Ly && st == CTM_OK; ++y)
        for (int x = 0; x < s.Lx && st == CTM_OK; ++x)
          st = ctm_spectrum(ctx, x, y, lab + 1,
                            spectra.data() + ((size_t)lab * S + y * s.Lx + x) * s.chi);
    if (!j->op.empty()) {
      energies.assign((size_t)S * 4, 0.0);
      for (int y = 0; y < s.Ly && st == CTM_OK; ++y)
        for (int x = 0; x < s.Lx && st == CTM_OK; ++x)
          for (int dir = 0; dir < 2 && st == CTM_OK; ++dir)
            st = ctm_expect(ctx, j->op.data(), x, y, dir,
                            energies.data() + ((size_t)(y * s.Lx + x) * 2 + dir) * 2);
    }
    if (st != CTM_OK) msg = ctm_last_error(ctx);
    ctm_free(ctx);
  } else {
    msg = ctm_last_error(nullptr);
  }
  std::lock_guard<std::mutex> lk(sv->m);
  j->status = st;
  j->iters = it;
  j->delta = delta;
  j->spectra.swap(spectra);
  j->energies.swap(energies);
  j->msg = msg;
  j->t_end = now_ms();
  j->done = true;
  sv->used -= j->footprint;
  sv->running -= 1;
  sv->latencies.push_back(j->t_end - j->t_submit);
  sv->last_end = std::max(sv->last_end, j->t_end);
  sv->cv_done.notify_all();
  sv->cv_sched.notify_all();
}

void schedule(ctm_server* sv) {
  std::unique_lock<std::mutex> lk(sv->m);
  while (true) {
    // first fit in arrival order
    auto fits = [&]() -> std::deque<Job*>::iterator {
      if (sv->running >= sv->max_conc) return sv->pending.end();
      for (auto it = sv->pending.begin(); it != sv->pending.end(); ++it)
        if (sv->used + (*it)->footprint <= sv->budget) return it;
      return sv->pending.end();
    };
    sv->cv_sched.wait(lk, [&] { return sv->stop || fits() != sv->pending.end(); });
    if (sv->stop) return;
    auto it = fits();
    Job* j = *it;
    sv->pending.erase(it);
    sv->used += j->footprint;
    sv->running += 1;
    j->t_start = now_ms();
    sv->workers.emplace_back(run_job, sv, j);
  }
}

}  // namespace

extern "C" ctm_status ctm_server_create(ctm_server** out, size_t hbm_budget, int max_concurrent) {
  if (!out || max_concurrent < 1) return CTM_EINVAL;
  ctm_server* sv = new ctm_server;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return CTM_ECUDA;
  }
  if (hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      delete sv;
      return CTM_ECUDA;
    }
    hbm_budget = free_b / 10 * 9;
  }
  sv->budget = hbm_budget;
  sv->max_conc = max_concurrent;
  sv->scheduler = std::thread(schedule, sv);
  *out = sv;
  return CTM_OK;
}

extern "C" ctm_status ctm_server_submit(ctm_server* sv, const ctm_solve_spec* spec,
                                        uint64_t* ticket) {
  if (!sv || !spec || !ticket || !spec->A || spec->Lx < 1 || spec->Ly < 1 || spec->d < 1 ||
      spec->D < 1 || spec->chi < 1 || spec->max_iter < 1 ||
      (spec->dtype != CTM_F64 && spec->dtype != CTM_C128))
    return CTM_EINVAL;
  Job* j = new Job;
  j->spec = *spec;
  const int S = spec->Lx * spec->Ly;
  const size_t es = spec->dtype == CTM_C128 ? 16 : 8;
  const size_t nA = (size_t)spec->d * spec->D * spec->D * spec->D * spec->D * es;
  j->A.resize(S);
  for (int i = 0; i < S; ++i) {
    if (!spec->A[i]) {
      delete j;
      return CTM_EINVAL;
    }
    j->A[i].assign(static_cast<const char*>(spec->A[i]), static_cast<const char*>(spec->A[i]) + nA);
    j->Aptr.push_back(j->A[i].data());
  }
  j->spec.A = nullptr;
  if (spec->op) {
    const size_t n = (size_t)spec->d * spec->d * spec->d * spec->d * es;
    j->op.assign(static_cast<const char*>(spec->op), static_cast<const char*>(spec->op) + n);
  }
  j->spec.op = nullptr;
  if (ctm_footprint(spec->Lx, spec->Ly, spec->d, spec->D, spec->chi, spec->dtype, &spec->opts,
                    &j->footprint) != CTM_OK) {
    delete j;
    return CTM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->m);
  if (j->footprint > sv->budget) {
    delete j;
    sv->msg = "solve does not fit the HBM budget of the server";
    return CTM_ENOMEM;
  }
  j->id = sv->next_id++;
  j->t_submit = now_ms();
  if (sv->first_submit < 0) sv->first_submit = j->t_submit;
  sv->jobs[j->id] = j;
  sv->pending.push_back(j);
  *ticket = j->id;
  sv->cv_sched.notify_all();
  return CTM_OK;
}

extern "C" ctm_status ctm_server_result(ctm_server* sv, uint64_t ticket, ctm_solve_result* res,
                                        double* spectra, double* energies) {
  if (!sv || !res) return CTM_EINVAL;
  std::unique_lock<std::mutex> lk(sv->m);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return CTM_EINVAL;
  Job* j = it->second;
  sv->cv_done.wait(lk, [&] { return j->done; });
  res->status = j->status;
  res->iters = j->iters;
  res->delta = j->delta;
  res->queue_ms = j->t_start - j->t_submit;
  res->run_ms = j->t_end - j->t_start;
  res->footprint = j->footprint;
  if (spectra && !j->spectra.empty())
    memcpy(spectra, j->spectra.data(), j->spectra.size() * sizeof(double));
  if (energies && !j->energies.empty())
    memcpy(energies, j->energies.data(), j->energies.size() * sizeof(double));
  sv->msg = j->msg;
  sv->jobs.erase(it);
  delete j;
  return res->status;
}

extern "C" ctm_status ctm_server_stats(ctm_server* sv, double* p50_ms, double* p99_ms,
                                       double* solves_per_s, int* completed) {
  if (!sv) return CTM_EINVAL;
  std::lock_guard<std::mutex> lk(sv->m);
  std::vector<double> l = sv->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    // nearest rank
    size_t r = (size_t)std::ceil(q * (double)l.size());
    if (r < 1) r = 1;
    return l[std::min(r, l.size()) - 1];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (completed) *completed = (int)l.size();
  if (solves_per_s)
    *solves_per_s = (l.empty() || sv->last_end <= sv->first_submit)
                        ? 0.0
                        : 1000.0 * (double)l.size() / (sv->last_end - sv->first_submit);
  return CTM_OK;
}

extern "C" const char* ctm_server_last_error(const ctm_server* sv) {
  return sv ? sv->msg.c_str() : "";
}

extern "C" void ctm_server_free(ctm_server* sv) {
  if (!sv) return;
  {
    std::unique_lock<std::mutex> lk(sv->m);
    // admit nothing more, let the admitted solves finish, drop the pending
    sv->stop = true;
    sv->cv_sched.notify_all();
    sv->cv_done.wait(lk, [&] { return sv->running == 0; });
    for (Job* j : sv->pending) {
      sv->jobs.erase(j->id);
      delete j;
    }
    sv->pending.clear();
  }
  sv->scheduler.join();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->jobs) delete kv.second;
  delete sv;
}
