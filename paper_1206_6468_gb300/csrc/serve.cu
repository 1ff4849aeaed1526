// Continuous-batching server over batch contexts (host code only).
//
// Requests arrive over time; each runs the sweep of Section 3.2 until its own
// bound stops moving (relative change below a tolerance) or a sweep limit,
// then leaves with its posteriors.  A request joins the batch of its model as
// soon as it has arrived and the batch has room for its frames (the batch's
// frame store is its HBM budget); every tick runs one sweep over all jobs of
// every non-empty batch.  The posterior factorises over jobs, so a request's
// results do not depend on the requests it shares a batch with.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "../../include/nfhmm.h"
#include "nfhmm_kernels.h"

namespace {

struct Active {
  int req;
  long long id;
  double prev_bound;
  int sweeps;
};

int fail(int code, const std::string& m) {
  nfhmm::set_last_error(m);
  return code;
}

}  // namespace

extern "C" {

int nfhmm_serve(nfhmm_ctx** batches, int n_batches, const nfhmm_request* reqs, int n_reqs,
                const nfhmm_serve_opts* opts, nfhmm_result* results) {
  if (!batches || !reqs || !opts || !results || n_batches < 1 || n_reqs < 0)
    return fail(NFHMM_EINVAL, "NULL argument or empty batch list");
  for (int b = 0; b < n_batches; ++b)
    if (!batches[b]) return fail(NFHMM_EINVAL, "NULL batch context");
  if (!(opts->rel_tol >= 0.0) || opts->max_sweeps < 1 || opts->min_sweeps < 1 ||
      opts->min_sweeps > opts->max_sweeps)
    return fail(NFHMM_EINVAL, "need rel_tol >= 0 and 1 <= min_sweeps <= max_sweeps");
  for (int r = 0; r < n_reqs; ++r) {
    if (reqs[r].model < 0 || reqs[r].model >= n_batches || reqs[r].T < 1 || !reqs[r].V)
      return fail(NFHMM_EINVAL, "request " + std::to_string(r) + ": bad model, T or V");
    results[r] = nfhmm_result{-1.0, -1.0, 0, 0.0, NFHMM_ESTATE};
  }
  for (int b = 0; b < n_batches; ++b) {
    int nj = 0;
    int rc = nfhmm_batch_info(batches[b], &nj, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (rc) return rc;
    if (nj != 0) return fail(NFHMM_EINVAL, "batches must start empty");
  }
  // arrival order per model
  std::vector<int> order(n_reqs);
  for (int r = 0; r < n_reqs; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return reqs[a].arrival_s < reqs[b].arrival_s; });
  std::vector<std::deque<int>> queue(n_batches);
  for (int r : order) queue[reqs[r].model].push_back(r);
  std::vector<std::vector<Active>> active(n_batches);
  std::vector<int> capacity_of(n_batches), max_jobs_of(n_batches);
  for (int b = 0; b < n_batches; ++b) {
    long long cap = 0, mj = 0;
    int rc = nfhmm_query(batches[b], NFHMM_Q_FRAME_CAPACITY, &cap);
    if (!rc) rc = nfhmm_query(batches[b], NFHMM_Q_MAX_JOBS, &mj);
    if (rc) return rc;
    capacity_of[b] = (int)cap;
    max_jobs_of[b] = (int)mj;
  }

  using clk = std::chrono::steady_clock;
  const auto t_start = clk::now();
  auto now = [&]() { return std::chrono::duration<double>(clk::now() - t_start).count(); };
  auto arrived = [&](int r) { return !opts->realtime || reqs[r].arrival_s <= now(); };
  int done = 0;
  std::vector<double> bounds;
  while (done < n_reqs) {
    // admission: in arrival order while the batch has room, all of a
    // batch's newcomers in one call
    for (int b = 0; b < n_batches; ++b) {
      int nj = 0, held = 0;
      int rc = nfhmm_batch_info(batches[b], &nj, &held, nullptr, nullptr, nullptr, nullptr);
      if (rc) return rc;
      const int cap_jobs = max_jobs_of[b], cap_frames = capacity_of[b];
      std::vector<int> take;
      std::vector<int> fr;
      std::vector<const float*> vs;
      while (!queue[b].empty() && arrived(queue[b].front())) {
        const int r = queue[b].front();
        if (reqs[r].T > cap_frames) {   // can never fit
          results[r].status = NFHMM_EFULL;
          results[r].done_s = now();
          queue[b].pop_front();
          ++done;
          continue;
        }
        if (nj + (int)take.size() + 1 > cap_jobs || held + reqs[r].T > cap_frames) break;
        held += reqs[r].T;
        take.push_back(r);
        fr.push_back(reqs[r].T);
        vs.push_back(reqs[r].V);
        queue[b].pop_front();
      }
      if (take.empty()) continue;
      std::vector<long long> ids(take.size());
      rc = nfhmm_batch_add_many(batches[b], (int)take.size(), fr.data(), vs.data(), 0, ids.data());
      if (rc == NFHMM_EINVAL) {
        // a bad spectrogram among them: add one by one to find it
        for (size_t i = 0; i < take.size(); ++i) {
          const int r = take[i];
          long long id = -1;
          const int rc1 = nfhmm_batch_add(batches[b], reqs[r].T, reqs[r].V, 0, &id);
          if (rc1) {
            results[r].status = rc1;
            results[r].done_s = now();
            ++done;
            continue;
          }
          results[r].admit_s = now();
          active[b].push_back(Active{r, id, 0.0, 0});
        }
        continue;
      }
      if (rc) return rc;
      const double ta = now();
      for (size_t i = 0; i < take.size(); ++i) {
        results[take[i]].admit_s = ta;
        active[b].push_back(Active{take[i], ids[i], 0.0, 0});
      }
    }
    bool any = false;
    for (int b = 0; b < n_batches; ++b) any = any || !active[b].empty();
    if (!any) {
      // idle: wait for the next arrival
      double next = 1e300;
      for (int b = 0; b < n_batches; ++b)
        if (!queue[b].empty()) next = std::min(next, reqs[queue[b].front()].arrival_s);
      if (next == 1e300) break;
      const double wait = next - now();
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
      continue;
    }
    // one sweep of every non-empty batch, all in flight together, then the
    // per-job bounds of each
    for (int b = 0; b < n_batches; ++b) {
      if (active[b].empty()) continue;
      const int rc = nfhmm_vi_sweep_async(batches[b], 1, 1);
      if (rc) return rc;
    }
    for (int b = 0; b < n_batches; ++b) {
      if (active[b].empty()) continue;
      bounds.assign(active[b].size(), 0.0);
      int rc = nfhmm_job_bounds(batches[b], bounds.data());
      if (rc) return rc;
      // job order in the batch is admission order, as in active[b]
      std::vector<Active> keep;
      std::vector<long long> leaving;
      for (size_t j = 0; j < active[b].size(); ++j) {
        Active& a = active[b][j];
        a.sweeps += 1;
        const double L = bounds[j];
        const bool conv = a.sweeps >= opts->min_sweeps && a.sweeps >= 2 &&
                          std::abs(L - a.prev_bound) < opts->rel_tol * std::abs(L);
        a.prev_bound = L;
        if (conv || a.sweeps >= opts->max_sweeps) {
          const nfhmm_request& q = reqs[a.req];
          if (q.dhat_out) {
            rc = nfhmm_job_posteriors(batches[b], a.id, q.dhat_out, 0);
            if (rc) return rc;
          }
          nfhmm_result& res = results[a.req];
          res.sweeps = a.sweeps;
          res.bound = L;
          res.status = NFHMM_OK;
          res.done_s = now();
          ++done;
          leaving.push_back(a.id);
        } else {
          keep.push_back(a);
        }
      }
      if (!leaving.empty()) {
        rc = nfhmm_batch_remove_many(batches[b], (int)leaving.size(), leaving.data());
        if (rc) return rc;
      }
      active[b].swap(keep);
    }
  }
  return NFHMM_OK;
}

}  // extern "C"
