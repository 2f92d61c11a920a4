// Request server: continuous batching of independent solves on one GPU (fmg_eig_serve).
//
// One host thread runs the loop.  Requests that have arrived wait in a FIFO queue.  Whenever
// fewer than max_inflight cohorts are resident, the queue's front request and the queued
// requests with the same shared settings (up to max_batch, while their hierarchies fit what
// is left of the device-memory budget) are admitted as a cohort: one batch handle, built with
// stream-ordered allocation on its own stream and launched directly.  Its FMG stages run
// every step of a level as one launch over the cohort's instances with that level (see
// engine.h), and after the stage that finishes some instances their eigenvalues are copied to
// pinned host memory and an event is recorded.  Cohorts admitted later run on other streams
// and overlap on the GPU with the ones already there.  A request's latency is read from the
// GPU clock (the event of its copy against an event recorded when serving started).  When
// all of a cohort's instances are done its outputs are collected and its memory returns to
// the device pool for the next admissions.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "engine.h"

namespace fmg {
namespace {

struct StageMark {
  cudaEvent_t ev = nullptr;
  int first = 0, count = 0;
  bool seen = false;
};

struct Cohort {
  fmg_eig_handle* h = nullptr;
  int id = 0;
  std::vector<int> req;  // req[b]: request index of the handle's sorted instance b
  std::vector<StageMark> marks;
  double* plam = nullptr;  // pinned region receiving the eigenvalues (nb)
  size_t bytes = 0;
  double admit_s = 0.0;
  int pending = 0;
  bool failed = false;
};

using Clock = std::chrono::steady_clock;

double since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Upper bound of a cohort's device bytes: the sum of its instances' single-instance
// footprints (the per-level arrays scale with the instance count, shared tables are counted
// once per instance instead of once per cohort).
struct Footprints {
  std::map<std::tuple<int, int, int, int>, size_t> cache;
  size_t of(const fmg_eig_problem& p) {
    const auto key = std::make_tuple(p.dim, p.coarse_cells, p.levels, p.precision);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const size_t b = estimate_bytes(&p, 1) + ((size_t)1 << 16);
    cache[key] = b;
    return b;
  }
};

}  // namespace
}  // namespace fmg

using namespace fmg;

extern "C" size_t fmg_eig_estimate_bytes(const fmg_eig_problem* probs, int32_t count) {
  return estimate_bytes(probs, count);
}

extern "C" int fmg_eig_serve(const fmg_eig_serve_config* cfg, const fmg_eig_request* reqs,
                             int32_t n, fmg_eig_result* results, fmg_eig_serve_stats* stats) {
  if (!cfg || !reqs || n < 1 || !results || cfg->max_batch < 1 || cfg->max_inflight < 1 ||
      !(cfg->batch_window_s >= 0.0))
    return FMG_EINVAL;
  for (int i = 0; i < n; ++i) {
    const int v = validate(&reqs[i].problem);
    if (v != FMG_OK) return v;
    if (!(reqs[i].arrival_s >= 0.0) || (i > 0 && reqs[i].arrival_s < reqs[i - 1].arrival_s))
      return FMG_EINVAL;
    const fmg_eig_problem& p = reqs[i].problem;
    const size_t m = (size_t)((p.coarse_cells << (p.levels - 1)) - 1);
    if (reqs[i].u && reqs[i].u_len != (p.dim == 2 ? m * m : m * m * m)) return FMG_EINVAL;
  }
  int dev = 0;
  size_t free_b = 0, total_b = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  const double budget = cfg->hbm_budget_bytes > 0.0 ? cfg->hbm_budget_bytes : 0.8 * (double)free_b;
  Footprints fp;
  for (int i = 0; i < n; ++i)
    if ((double)fp.of(reqs[i].problem) > budget) return FMG_EINVAL;  // could never be admitted

  // keep released cohort memory in the device pool for the next admissions
  cudaMemPool_t pool = nullptr;
  uint64_t old_threshold = 0, keep = UINT64_MAX;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold) != cudaSuccess ||
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  double* plam_all = nullptr;
  cudaStream_t ref_stream = nullptr;
  cudaEvent_t ev_ref = nullptr;
  int rc = FMG_OK;
  if (cudaMallocHost(&plam_all, sizeof(double) * n) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ref_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&ev_ref) != cudaSuccess || cudaEventRecord(ev_ref, ref_stream) != cudaSuccess ||
      cudaEventSynchronize(ev_ref) != cudaSuccess) {
    cudaGetLastError();
    rc = FMG_ECUDA;
  }
  const Clock::time_point t0 = Clock::now();

  for (int i = 0; i < n; ++i) {
    memset(&results[i], 0, sizeof(results[i]));
    results[i].status = FMG_ECUDA;
    results[i].cohort = -1;
  }
  std::deque<int> queue;
  std::vector<Cohort> inflight;
  int next = 0, done = 0, cohorts = 0, max_cohort = 0, max_inflight_seen = 0;
  size_t plam_next = 0;
  double used = 0.0, peak = 0.0;
  CreateOptions opt;
  opt.graph = false;
  opt.component_setup = false;
  opt.async_alloc = true;
  opt.tune = 1;

  auto finish = [&](Cohort& c) {
    fmg_eig_handle* h = c.h;
    const int nb = h->nb, L = h->levels();
    std::vector<int> st((size_t)L * nb, 1);
    bool ok = !c.failed;
    if (ok) {
      bool any_u = false;
      for (int b = 0; b < nb; ++b) any_u |= reqs[c.req[b]].u != nullptr;
      if (any_u) enqueue_outputs(h, h->stream);
      ok = cudaMemcpyAsync(st.data(), h->status, sizeof(int) * L * nb, cudaMemcpyDeviceToHost,
                           h->stream) == cudaSuccess;
      for (int b = 0; ok && b < nb; ++b) {
        const fmg_eig_request& r = reqs[c.req[b]];
        if (r.u)
          ok = cudaMemcpyAsync(r.u, h->uout + h->uoff[b], sizeof(double) * r.u_len,
                               cudaMemcpyDeviceToHost, h->stream) == cudaSuccess;
      }
      ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
    }
    for (int b = 0; b < nb; ++b) {
      fmg_eig_result& o = results[c.req[b]];
      if (!ok) {
        o.status = FMG_ECUDA;
        continue;
      }
      int code = FMG_OK;
      for (int k = 1; k <= h->probs[b].levels; ++k)
        if (st[(size_t)(k - 1) * nb + b] != 0) code = FMG_ENOCONV;
      o.status = code;
    }
    if (!ok) cudaGetLastError();
    for (StageMark& m : c.marks) cudaEventDestroy(m.ev);
    delete h;  // stream-ordered release: does not wait for other cohorts
    used -= (double)c.bytes;
  };

  while (rc == FMG_OK && done < n) {
    bool progress = false;
    const double now = since(t0);
    while (next < n && reqs[next].arrival_s <= now) {
      queue.push_back(next++);
      progress = true;
    }
    // completions, in stage order per cohort
    for (Cohort& c : inflight) {
      for (StageMark& m : c.marks) {
        if (m.seen) continue;
        const cudaError_t q = cudaEventQuery(m.ev);
        if (q == cudaErrorNotReady) break;
        m.seen = true;
        progress = true;
        float ms = 0.f;
        if (q != cudaSuccess || cudaEventElapsedTime(&ms, ev_ref, m.ev) != cudaSuccess) {
          cudaGetLastError();
          c.failed = true;
          ms = (float)(since(t0) * 1e3);
        }
        for (int b = m.first; b < m.first + m.count; ++b) {
          const int i = c.req[b];
          fmg_eig_result& o = results[i];
          o.lambda = c.plam[b];
          o.done_s = ms * 1e-3;
          o.latency_s = o.done_s - reqs[i].arrival_s;
          o.admit_s = c.admit_s;
          o.cohort = c.id;
          ++done;
          --c.pending;
        }
      }
    }
    for (size_t j = 0; j < inflight.size();) {
      if (inflight[j].pending == 0) {
        finish(inflight[j]);
        inflight.erase(inflight.begin() + j);
      } else {
        ++j;
      }
    }
    // admissions
    while (!queue.empty() && (int)inflight.size() < cfg->max_inflight) {
      const fmg_eig_problem& front = reqs[queue.front()].problem;
      std::vector<int> pick;
      double bytes = 0.0;
      int same = 0;
      for (int i : queue)
        if (same_shared_settings(reqs[i].problem, front)) ++same;
      // a short window lets more requests of this kind join a cohort
      if (same < cfg->max_batch && next < n &&
          since(t0) - reqs[queue.front()].arrival_s < cfg->batch_window_s)
        break;
      for (int i : queue) {
        if ((int)pick.size() >= cfg->max_batch) break;
        if (!same_shared_settings(reqs[i].problem, front)) continue;
        const double b = (double)fp.of(reqs[i].problem);
        if (used + bytes + b > budget) continue;
        pick.push_back(i);
        bytes += b;
      }
      if (pick.empty() || pick[0] != queue.front()) break;  // wait for memory (FIFO front first)
      std::vector<fmg_eig_problem> ps;
      for (int i : pick) ps.push_back(reqs[i].problem);
      fmg_eig_handle* h = nullptr;
      const int crc = create_handle(ps.data(), (int)ps.size(), opt, &h);
      if (crc == FMG_ENOMEM && !inflight.empty()) break;  // retry once memory is released
      std::deque<int> rest;
      for (int i : queue)
        if (std::find(pick.begin(), pick.end(), i) == pick.end()) rest.push_back(i);
      queue.swap(rest);
      progress = true;
      if (crc != FMG_OK) {  // fails alone as well: report it on these requests
        for (int i : pick) {
          results[i].status = crc;
          results[i].done_s = since(t0);
          results[i].latency_s = results[i].done_s - reqs[i].arrival_s;
          ++done;
        }
        continue;
      }
      Cohort c;
      c.h = h;
      c.id = cohorts++;
      c.req.resize(h->nb);
      for (int b = 0; b < h->nb; ++b) c.req[b] = pick[h->order[b]];
      c.plam = plam_all + plam_next;
      plam_next += h->nb;
      c.bytes = h->bytes;
      c.admit_s = since(t0);
      c.pending = h->nb;
      bool launch_ok = true;
      const StageHook hook = [&](int, int first, int count) {
        StageMark m;
        m.first = first;
        m.count = count;
        launch_ok = launch_ok && cudaEventCreate(&m.ev) == cudaSuccess &&
                    cudaMemcpyAsync(c.plam + first, h->lam + first, sizeof(double) * count,
                                    cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
                    cudaEventRecord(m.ev, h->stream) == cudaSuccess;
        c.marks.push_back(m);
      };
      launch_ok = upload_params(h, h->stream) == cudaSuccess;
      enqueue_fmg(h, h->stream, &hook);
      if (!launch_ok || cudaGetLastError() != cudaSuccess) {
        rc = FMG_ECUDA;
        c.failed = true;
      }
      used += (double)c.bytes;
      peak = std::max(peak, used);
      max_cohort = std::max(max_cohort, h->nb);
      inflight.push_back(std::move(c));
      max_inflight_seen = std::max(max_inflight_seen, (int)inflight.size());
      if (rc != FMG_OK) break;
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // drain (error paths): wait for and release everything still resident
  for (Cohort& c : inflight) {
    cudaStreamSynchronize(c.h->stream);
    c.failed = true;
    finish(c);
  }
  inflight.clear();
  cudaMemPoolTrimTo(pool, 0);
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold);
  if (plam_all) cudaFreeHost(plam_all);
  if (ev_ref) cudaEventDestroy(ev_ref);
  if (ref_stream) cudaStreamDestroy(ref_stream);
  cudaGetLastError();

  int conv = FMG_OK;
  std::vector<double> lat;
  double first_arrival = reqs[0].arrival_s, last_done = 0.0;
  int completed = 0;
  for (int i = 0; i < n; ++i) {
    if (results[i].status == FMG_OK || results[i].status == FMG_ENOCONV) {
      ++completed;
      lat.push_back(results[i].latency_s);
      last_done = std::max(last_done, results[i].done_s);
    }
    if (results[i].status == FMG_ENOCONV && conv == FMG_OK) conv = FMG_ENOCONV;
    if (results[i].status != FMG_OK && results[i].status != FMG_ENOCONV && rc == FMG_OK)
      rc = results[i].status;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    std::sort(lat.begin(), lat.end());
    auto rank = [&](double q) {
      if (lat.empty()) return 0.0;
      size_t r = (size_t)ceil(q * lat.size());
      r = r < 1 ? 1 : (r > lat.size() ? lat.size() : r);
      return lat[r - 1];
    };
    stats->p50_s = rank(0.50);
    stats->p99_s = rank(0.99);
    double sum = 0.0;
    for (double v : lat) sum += v;
    stats->mean_s = lat.empty() ? 0.0 : sum / lat.size();
    stats->max_s = lat.empty() ? 0.0 : lat.back();
    stats->makespan_s = last_done - first_arrival;
    stats->solves_per_s = stats->makespan_s > 0 ? completed / stats->makespan_s : 0.0;
    stats->peak_bytes = peak;
    stats->budget_bytes = budget;
    stats->cohorts = cohorts;
    stats->max_cohort = max_cohort;
    stats->max_inflight_seen = max_inflight_seen;
    stats->completed = completed;
  }
  return rc != FMG_OK ? rc : conv;
}
