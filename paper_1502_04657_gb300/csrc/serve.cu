// Request server: continuous batching of independent solves on one GPU (fmg_eig_serve).
//
// One host thread runs the loop.  Requests that have arrived wait in a FIFO queue.  Whenever
// fewer than max_inflight cohorts are in flight, the queue's front request and the queued
// requests with the same shared settings (up to max_batch, while their hierarchies fit what
// is left of the device-memory budget) are admitted as a cohort: one batch handle on its own
// stream, whose FMG stages run every step of a level as one launch over the cohort's
// instances with that level (see engine.h).  Cohorts admitted later run on other streams and
// overlap on the GPU with the ones already there.
//
// The handle of a cohort is recorded once as a CUDA graph that, after the stage which
// finishes some instances, copies their eigenvalues to pinned host memory and records an
// event.  A request's latency is read from the GPU clock: the event of its copy against an
// event recorded when serving started.  When a cohort is done its hierarchy stays resident in
// a pool keyed by its settings and sorted level counts; a later cohort with the same key
// uploads its own parameters and replays the graph (no allocation, no capture, no per-kernel
// launches).  Pooled hierarchies count against the budget and are released oldest first
// (stream-ordered frees, which wait for no other cohort) when an admission needs room.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "engine.h"

namespace fmg {
namespace {

struct Cohort {
  fmg_eig_handle* h = nullptr;
  std::string key;
  int id = 0;
  std::vector<int> req;  // req[b]: request index of the handle's sorted instance b
  std::vector<char> seen;
  size_t bytes = 0;
  double admit_s = 0.0;
  int pending = 0;
  bool failed = false;
};

struct Pooled {
  fmg_eig_handle* h;
  size_t bytes;
  uint64_t stamp;  // release order (oldest first)
};

using Clock = std::chrono::steady_clock;

double since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Upper bound of a cohort's device bytes: the sum of its instances' single-instance
// footprints (the per-level arrays scale with the instance count, shared tables are counted
// once per instance instead of once per cohort).
struct Footprints {
  std::map<std::tuple<int, int, int, int, int>, size_t> cache;
  size_t of(const fmg_eig_problem& p) {
    const auto key = std::make_tuple(p.dim, p.coarse_cells, p.levels, p.precision, p.operator_form);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const size_t b = estimate_bytes(&p, 1) + ((size_t)1 << 16);
    cache[key] = b;
    return b;
  }
};

// Pinned eigenvalue slots of the pooled graphs (each graph copies to fixed addresses): a bump
// arena with per-size free lists for the slots of released hierarchies.
struct PinnedSlots {
  double* base = nullptr;
  size_t cap = 0, next = 0;
  std::map<int, std::vector<double*>> free_by_size;
  double* take(int n) {
    auto it = free_by_size.find(n);
    if (it != free_by_size.end() && !it->second.empty()) {
      double* p = it->second.back();
      it->second.pop_back();
      return p;
    }
    if (next + n > cap) return nullptr;
    double* p = base + next;
    next += n;
    return p;
  }
  void give(double* p, int n) { free_by_size[n].push_back(p); }
};

// the settings every instance of a cohort shares, and its sorted level counts
std::string cohort_key(const fmg_eig_problem& p, const std::vector<int>& levels_desc) {
  std::string k;
  auto put = [&k](const void* v, size_t n) { k.append(static_cast<const char*>(v), n); };
  const int32_t ints[] = {p.dim, p.coarse_cells, p.nu_pre, p.nu_post, p.vcycles, p.corrections,
                          p.smoother, p.precision, p.operator_form, p.scf_max_iter, p.flags};
  put(ints, sizeof(ints));
  put(&p.box_len, sizeof(double));
  put(&p.scf_tol, sizeof(double));
  for (int l : levels_desc) put(&l, sizeof(int));
  return k;
}

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

  // keep released hierarchies' memory in the device pool for the next admissions
  cudaMemPool_t pool = nullptr;
  uint64_t old_threshold = 0, keep = UINT64_MAX;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
      cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold) != cudaSuccess ||
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    cudaGetLastError();
    return FMG_ECUDA;
  }
  PinnedSlots slots;
  slots.cap = std::max<size_t>((size_t)1 << 20, 4 * (size_t)n);
  cudaStream_t ref_stream = nullptr;
  cudaEvent_t ev_ref = nullptr;
  int rc = FMG_OK;
  if (cudaMallocHost(&slots.base, sizeof(double) * slots.cap) != cudaSuccess ||
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
  std::map<std::string, std::vector<Pooled>> pooled;
  uint64_t stamp = 0;
  int next = 0, done = 0, cohorts = 0, max_cohort = 0, max_inflight_seen = 0, reused = 0,
      evicted = 0;
  double used = 0.0, peak = 0.0;  // bytes of in-flight and pooled hierarchies
  CreateOptions opt;
  opt.component_setup = false;
  opt.async_alloc = true;
  opt.tune = 1;

  auto release = [&](fmg_eig_handle* h, size_t bytes) {
    slots.give(h->opt.stage_lam, h->nb);
    delete h;  // stream-ordered frees: do not wait for other cohorts
    used -= (double)bytes;
  };
  // release the oldest pooled hierarchy; false when none is left
  auto evict_oldest = [&]() {
    std::string best_key;
    size_t best_i = 0;
    uint64_t best = UINT64_MAX;
    for (auto& kv : pooled)
      for (size_t i = 0; i < kv.second.size(); ++i)
        if (kv.second[i].stamp < best) {
          best = kv.second[i].stamp;
          best_key = kv.first;
          best_i = i;
        }
    if (best == UINT64_MAX) return false;
    Pooled p = pooled[best_key][best_i];
    pooled[best_key].erase(pooled[best_key].begin() + best_i);
    release(p.h, p.bytes);
    ++evicted;
    return true;
  };
  auto by_levels = [&](std::vector<int>& v) {  // the order a handle sorts its instances in
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
      return reqs[a].problem.levels > reqs[b].problem.levels;
    });
  };
  auto levels_of = [&](const std::vector<int>& v) {
    std::vector<int> lv;
    for (int i : v) lv.push_back(reqs[i].problem.levels);
    return lv;
  };

  auto finish = [&](Cohort& c) {
    fmg_eig_handle* h = c.h;
    const int nb = h->nb, L = h->levels();
    std::vector<int> st((size_t)L * nb, 1), wf(nb, 0);
    bool ok = !c.failed;
    if (ok) {
      bool any_u = false;
      for (int b = 0; b < nb; ++b) any_u |= reqs[c.req[b]].u != nullptr;
      if (any_u) enqueue_outputs(h, h->stream);
      ok = cudaMemcpyAsync(st.data(), h->status, sizeof(int) * L * nb, cudaMemcpyDeviceToHost,
                           h->stream) == cudaSuccess &&
           cudaMemcpyAsync(wf.data(), h->wait_fail, sizeof(int) * nb, cudaMemcpyDeviceToHost,
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
      o.status = instance_code(st.data(), wf.data(), nb, b, h->probs[b].levels);
    }
    if (!ok) {
      cudaGetLastError();
      release(h, c.bytes);
      return;
    }
    pooled[c.key].push_back({h, c.bytes, stamp++});  // resident for the next such cohort
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
      const auto& marks = c.h->marks;
      for (size_t m = 0; m < marks.size(); ++m) {
        if (c.seen[m]) continue;
        const cudaError_t q = cudaEventQuery(marks[m].ev);
        if (q == cudaErrorNotReady) break;
        c.seen[m] = 1;
        progress = true;
        float ms = 0.f;
        if (q != cudaSuccess || cudaEventElapsedTime(&ms, ev_ref, marks[m].ev) != cudaSuccess) {
          cudaGetLastError();
          c.failed = true;
          ms = (float)(since(t0) * 1e3);
        }
        for (int b = marks[m].first; b < marks[m].first + marks[m].count; ++b) {
          const int i = c.req[b];
          fmg_eig_result& o = results[i];
          o.lambda = c.h->opt.stage_lam[b];
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
      int same = 0;
      for (int i : queue)
        if (same_shared_settings(reqs[i].problem, front)) ++same;
      // a short window lets more requests of this kind join a cohort
      if (same < cfg->max_batch && next < n &&
          since(t0) - reqs[queue.front()].arrival_s < cfg->batch_window_s)
        break;
      std::vector<int> pick;
      for (int i : queue) {
        if ((int)pick.size() >= cfg->max_batch) break;
        if (same_shared_settings(reqs[i].problem, front)) pick.push_back(i);
      }
      std::vector<int> sorted = pick;
      by_levels(sorted);
      fmg_eig_handle* h = nullptr;
      size_t bytes = 0;
      auto pit = pooled.find(cohort_key(front, levels_of(sorted)));
      if (pit != pooled.end() && !pit->second.empty()) {  // replay a pooled hierarchy
        h = pit->second.back().h;
        bytes = pit->second.back().bytes;
        pit->second.pop_back();
        for (int b = 0; b < h->nb; ++b) {
          h->probs[b] = reqs[sorted[b]].problem;
          h->order[b] = b;
        }
        fill_params(h);
        ++reused;
      } else {
        double need = 0.0;
        for (int i : pick) need += (double)fp.of(reqs[i].problem);
        while (used + need > budget && evict_oldest()) {
        }
        if (used + need > budget) {  // shrink to what fits (FIFO front first)
          std::vector<int> fit;
          double b2 = 0.0;
          for (int i : pick) {
            const double b = (double)fp.of(reqs[i].problem);
            if (used + b2 + b <= budget) {
              fit.push_back(i);
              b2 += b;
            }
          }
          if (fit.empty() || fit[0] != queue.front()) break;  // wait for memory
          pick = fit;
          sorted = pick;
          by_levels(sorted);
        }
        std::vector<fmg_eig_problem> ps;
        for (int i : sorted) ps.push_back(reqs[i].problem);
        opt.stage_lam = slots.take((int)ps.size());
        while (!opt.stage_lam && evict_oldest()) opt.stage_lam = slots.take((int)ps.size());
        if (!opt.stage_lam) break;  // every slot is in flight: wait
        const int crc = create_handle(ps.data(), (int)ps.size(), opt, &h);
        if (crc != FMG_OK) {
          slots.give(opt.stage_lam, (int)ps.size());
          if (crc == FMG_ENOMEM && (!inflight.empty() || evict_oldest())) break;  // retry later
          std::deque<int> rest;
          for (int i : queue)
            if (std::find(pick.begin(), pick.end(), i) == pick.end()) rest.push_back(i);
          queue.swap(rest);
          for (int i : pick) {  // fails alone as well: report it on these requests
            results[i].status = crc;
            results[i].done_s = since(t0);
            results[i].latency_s = results[i].done_s - reqs[i].arrival_s;
            ++done;
          }
          progress = true;
          continue;
        }
        bytes = h->bytes;
        used += (double)bytes;
      }
      std::deque<int> rest;
      for (int i : queue)
        if (std::find(pick.begin(), pick.end(), i) == pick.end()) rest.push_back(i);
      queue.swap(rest);
      progress = true;
      Cohort c;
      c.h = h;
      c.key = cohort_key(front, levels_of(sorted));
      c.id = cohorts++;
      c.req = sorted;
      c.seen.assign(h->marks.size(), 0);
      c.bytes = bytes;
      c.admit_s = since(t0);
      c.pending = h->nb;
      if (upload_params(h, h->stream) != cudaSuccess ||
          cudaGraphLaunch(h->exec, h->stream) != cudaSuccess) {
        cudaGetLastError();
        rc = FMG_ECUDA;
        c.failed = true;
      }
      peak = std::max(peak, used);
      max_cohort = std::max(max_cohort, h->nb);
      inflight.push_back(std::move(c));
      max_inflight_seen = std::max(max_inflight_seen, (int)inflight.size());
      if (rc != FMG_OK) break;
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // drain (error paths): wait for and release everything still in flight
  for (Cohort& c : inflight) {
    cudaStreamSynchronize(c.h->stream);
    c.failed = true;
    finish(c);
  }
  inflight.clear();
  for (auto& kv : pooled)
    for (Pooled& p : kv.second) release(p.h, p.bytes);
  pooled.clear();
  cudaDeviceSynchronize();  // the frees above are stream-ordered
  cudaMemPoolTrimTo(pool, 0);
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &old_threshold);
  if (slots.base) cudaFreeHost(slots.base);
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
    stats->reused = reused;
    stats->evicted = evicted;
  }
  return rc != FMG_OK ? rc : conv;
}
