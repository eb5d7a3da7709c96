// server.cu -- continuous-batching request loop (sw_server_* in lagmean.h).
//
// One host thread per server.  Each round it (1) admits queued jobs in
// arrival order while the job-state bytes (sw_state_bytes) fit in the budget
// and a slot is free, creating the job's handle from its initial condition
// and opening its interval; (2) groups the active jobs by compatible block
// shapes and stepper (all grids 64..512 together, every larger size in a
// group of its own size; one stepper per group) and advances each group as
// one sw_batch by the largest step count no member overshoots (at most
// chunk_steps); (3) completes the jobs whose interval has ended: lmean_end
// into the caller's host buffers, handle released.
// Without a caller stream every group has a stream of its own (its jobs'
// handles are created on it), so the groups' steps overlap on the device: a
// 2048^2 group and a batch of small grids run side by side.  Steps are
// enqueued asynchronously; the loop waits only when it completes a job.
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

#include "../../include/lagmean.h"

namespace lm {
void set_handleless_error(const std::string& msg);
}

namespace {

struct Job {
  sw_job j;
  double t_submit = 0, t_admit = 0;
  int64_t bytes = 0;
  sw_handle* h = nullptr;
  int64_t remaining = 0;
};

struct Group {
  std::vector<sw_handle*> members;
  sw_batch* batch = nullptr;
};

// batch group of a job: sizes 64..512 share one group; every stepper has its
// own groups (a batch runs one stepper)
int group_key(const sw_params& p) { return ((p.N >= 64 && p.N <= 512) ? 0 : p.N) * 4 + p.stepper; }

}  // namespace

struct sw_server {
  sw_server_params p{};
  int device = 0;
  cudaStream_t stream = nullptr;  // the caller's stream for every group, or null
  std::map<int, cudaStream_t> gstreams;  // per group key, without a caller stream
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::vector<Job> active;
  std::vector<sw_job_done> done;
  std::map<int, Group> groups;
  sw_server_stats st{};
  bool stop = false;
  std::thread th;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  void finish(Job& jb, int status) {
    sw_job_done d{};
    d.tag = jb.j.tag;
    d.status = status;
    d.t_submit = jb.t_submit;
    d.t_admit = jb.t_admit;
    d.t_done = now();
    d.bytes = jb.bytes;
    std::lock_guard<std::mutex> lk(mu);
    done.push_back(d);
    if (status == SW_OK) {
      st.completed++;
      st.grid_point_steps += (int64_t)jb.j.params.N * jb.j.params.N * jb.j.lm.n_steps;
    } else {
      st.failed++;
    }
    st.bytes_in_use -= jb.bytes;
    cv_done.notify_all();
  }

  void set_active_count() {
    std::lock_guard<std::mutex> lk(mu);
    st.active = (int64_t)active.size();
  }

  void drop_groups() {
    for (auto& kv : groups)
      if (kv.second.batch) sw_batch_destroy(kv.second.batch);
    groups.clear();
  }

  // admit queued jobs that fit
  void admit() {
    for (;;) {
      Job jb;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (stop || queue.empty() || (int)active.size() >= p.max_active) return;
        if (st.bytes_in_use + queue.front().bytes > p.hbm_budget) return;
        jb = queue.front();
        queue.pop_front();
        st.queued = (int64_t)queue.size();
        st.bytes_in_use += jb.bytes;
        st.peak_bytes = std::max(st.peak_bytes, st.bytes_in_use);
      }
      jb.t_admit = now();
      cudaStream_t js = stream;
      int rc = SW_OK;
      if (!js) {
        auto it = gstreams.find(group_key(jb.j.params));
        if (it == gstreams.end()) {
          cudaStream_t ns = nullptr;
          if (cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            rc = SW_ECUDA;
          } else {
            it = gstreams.emplace(group_key(jb.j.params), ns).first;
          }
        }
        if (rc == SW_OK) js = it->second;
      }
      if (rc == SW_OK) rc = sw_create(&jb.j.params, jb.j.ic_uvh, 0, js, &jb.h);
      if (rc == SW_OK) rc = lmean_begin(jb.h, &jb.j.lm);
      if (rc != SW_OK) {
        if (jb.h) sw_destroy(jb.h);
        jb.h = nullptr;
        finish(jb, rc);
        continue;
      }
      jb.remaining = jb.j.lm.n_steps;
      active.push_back(jb);  // `active` belongs to the loop thread
      set_active_count();
    }
  }

  // (re)build the batch groups whose membership changed (a batch must be
  // destroyed before any of its members; destroying it waits for its stream)
  int regroup() {
    std::map<int, std::vector<sw_handle*>> want;
    for (auto& jb : active) want[group_key(jb.j.params)].push_back(jb.h);
    for (auto it = groups.begin(); it != groups.end();) {
      auto w = want.find(it->first);
      if (w == want.end() || w->second != it->second.members) {
        if (it->second.batch) sw_batch_destroy(it->second.batch);
        it = groups.erase(it);
      } else {
        ++it;
      }
    }
    for (auto& kv : want) {
      if (groups.count(kv.first)) continue;
      Group g;
      g.members = kv.second;
      int rc = sw_batch_create(g.members.data(), (int)g.members.size(), &g.batch);
      if (rc != SW_OK) return rc;
      groups[kv.first] = g;
    }
    return SW_OK;
  }

  // destroy the batch that holds handle h (before h itself is destroyed)
  void drop_group_of(sw_handle* h) {
    for (auto it = groups.begin(); it != groups.end(); ++it)
      for (sw_handle* m : it->second.members)
        if (m == h) {
          if (it->second.batch) sw_batch_destroy(it->second.batch);
          groups.erase(it);
          return;
        }
  }

  void round() {
    if (regroup() != SW_OK) {
      // cannot batch: fail every active job
      drop_groups();
      std::vector<Job> act;
      act.swap(active);
      set_active_count();
      for (auto& jb : act) {
        sw_destroy(jb.h);
        finish(jb, SW_ECUDA);
      }
      return;
    }
    for (auto& kv : groups) {
      int64_t k = p.chunk_steps;
      for (auto& jb : active)
        if (group_key(jb.j.params) == kv.first) k = std::min(k, jb.remaining);
      if (k <= 0) continue;
      int rc = sw_batch_step(kv.second.batch, k);
      for (auto& jb : active)
        if (group_key(jb.j.params) == kv.first) jb.remaining = rc == SW_OK ? jb.remaining - k : -1;
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      st.rounds++;
    }
    // complete finished jobs
    for (size_t i = 0; i < active.size();) {
      Job& jb = active[i];
      if (jb.remaining > 0) {
        ++i;
        continue;
      }
      int rc = jb.remaining == 0 ? lmean_end(jb.h, &jb.j.out) : SW_ECUDA;
      Job fin = jb;
      active.erase(active.begin() + i);
      set_active_count();
      // the batch that holds this handle must go before the handle; the
      // other groups keep their batches and their work in flight
      drop_group_of(fin.h);
      sw_destroy(fin.h);
      finish(fin, rc);
    }
  }

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait_for(lk, std::chrono::milliseconds(5),
                         [&] { return stop || !queue.empty() || !active.empty(); });
        if (stop) break;
      }
      admit();
      if (active.empty()) continue;
      round();
    }
    drop_groups();
    for (auto& jb : active)
      if (jb.h) sw_destroy(jb.h);
    active.clear();
    for (auto& kv : gstreams) cudaStreamDestroy(kv.second);
    gstreams.clear();
  }
};

extern "C" int sw_server_create(const sw_server_params* p, sw_server** out) {
  if (!out) return SW_EINVAL;
  *out = nullptr;
  if (!p || p->max_active < 1 || p->chunk_steps < 1 || p->hbm_budget <= 0 || p->reserved != 0 ||
      (p->precision != SW_PREC_FP32 && p->precision != SW_PREC_FP64)) {
    lm::set_handleless_error("sw_server_create: invalid parameters");
    return SW_EINVAL;
  }
  sw_server* s = new (std::nothrow) sw_server();
  if (!s) return SW_ENOMEM;
  s->p = *p;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  s->stream = (cudaStream_t)p->stream;
  if (e != cudaSuccess) {
    lm::set_handleless_error(std::string("sw_server_create: ") + cudaGetErrorString(e));
    delete s;
    return SW_ECUDA;
  }
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return SW_OK;
}

extern "C" int sw_server_submit(sw_server* s, const sw_job* job) {
  if (!s || !job || !job->ic_uvh) return SW_EINVAL;
  if (job->params.precision != s->p.precision || job->out.on_device != 0) return SW_EINVAL;
  const int64_t bytes = sw_state_bytes(&job->params);
  if (bytes <= 0 || bytes > s->p.hbm_budget || job->lm.n_steps < 1) return SW_EINVAL;
  Job jb;
  jb.j = *job;
  jb.bytes = bytes;
  jb.t_submit = s->now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return SW_ESTATE;
    s->queue.push_back(jb);
    s->st.submitted++;
    s->st.queued = (int64_t)s->queue.size();
  }
  s->cv_work.notify_one();
  return SW_OK;
}

extern "C" int sw_server_poll(sw_server* s, sw_job_done* done, int max, int* n, int wait_ms) {
  if (!s || !n || (max > 0 && !done)) return SW_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  const int k = std::min<int>(max, (int)s->done.size());
  for (int i = 0; i < k; ++i) done[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *n = k;
  return SW_OK;
}

extern "C" int sw_server_stats_get(sw_server* s, sw_server_stats* st) {
  if (!s || !st) return SW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  return SW_OK;
}

extern "C" double sw_server_clock(sw_server* s) { return s ? s->now() : 0.0; }

extern "C" void sw_server_destroy(sw_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  delete s;
}
