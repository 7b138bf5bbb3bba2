// Serving form: a queue of tessellation jobs, admitted under a device-memory
// budget and advanced together in batched launches by one scheduler thread.
//
// Threads.  Callers submit, wait and read statistics from any thread; those
// calls touch only host records under the server mutex.  Every CUDA call and
// every lf_mesh belongs to the scheduler thread.  A job's operator is built on
// the submitting thread, so host preparation of new jobs overlaps the batches
// that run on the device.

#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
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

#include "../../include/lf.h"
#include "lf_internal.h"

namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return static_cast<int64_t>(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

struct Job {
  int64_t id = 0;
  int64_t n_v = 0;
  std::vector<int64_t> rp;          // operator (off-diagonal), dropped at admission
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<int32_t> seeds;
  std::vector<double> V;            // geometry, kept only for Lloyd rounds or the dual mesh
  std::vector<int32_t> F;
  int32_t n_iters = 0;
  int32_t lloyd_rounds = 0, lloyd_done = 0;
  bool want_dual = false;
  std::vector<int32_t> dual;        // oriented triangles, 3 seed ids each
  bool dual_ready = false;
  uint64_t skeleton_before = 0;     // nnz-updates of the finished rounds
  lf_params prm{};
  int64_t bytes_est = 0;
  int64_t arrival_ns = 0, admit_ns = 0, finish_ns = 0;
  int32_t state = LF_JOB_QUEUED;
  int32_t status = LF_OK;
  int64_t steps_done = 0;
  uint64_t skeleton_total = 0;
  int64_t device_bytes = 0;
  lf_mesh mesh = nullptr;           // scheduler thread only
  std::vector<int32_t> labels;
};
using JobPtr = std::shared_ptr<Job>;

}  // namespace

struct lf_server_s {
  lf_server_params sp{};
  lf_device dev{};
  int device = 0;
  cudaStream_t stream = nullptr;

  std::mutex mu;
  std::condition_variable cv_work;   // scheduler: new work or stop
  std::condition_variable cv_done;   // waiters: a job finished
  std::deque<JobPtr> queue;
  std::vector<JobPtr> running;       // admitted (the scheduler owns their meshes)
  int64_t admitting = 0;             // taken from the queue, being created on the device
  std::unordered_map<int64_t, JobPtr> jobs;
  int64_t next_id = 1;
  bool stop = false;
  lf_server_stats_t st{};
  std::thread thr;
};

namespace {

lf_status server_fail(lf_status s, const std::string& msg) {
  lf::set_last_error(msg);
  return s;
}

// Device bytes reserved for the running jobs: each counts the larger of its
// estimate and what it holds now (its buffers may have grown).
int64_t reserved_bytes(const lf_server_s* s) {
  int64_t b = 0;
  for (const auto& j : s->running) b += std::max(j->bytes_est, j->device_bytes);
  return b;
}

void retire(lf_server_s* s, const JobPtr& j, int32_t state, int32_t status) {
  if (j->mesh) {
    lf_destroy_mesh(j->mesh);
    j->mesh = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  j->state = state;
  j->status = status;
  j->finish_ns = now_ns();
  if (state == LF_JOB_DONE) {
    ++s->st.done;
    s->st.skeleton_total += j->skeleton_total;
  } else {
    ++s->st.failed;
  }
  s->running.erase(std::remove(s->running.begin(), s->running.end(), j), s->running.end());
  s->cv_done.notify_all();
}

void scheduler(lf_server_s* s) {
  cudaSetDevice(s->device);
  std::vector<JobPtr> admit;
  for (;;) {
    admit.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->running.empty(); });
      if (s->stop) break;
      // admission in arrival order, under the job-count and memory limits
      int64_t used = reserved_bytes(s);
      while (!s->queue.empty() && static_cast<int64_t>(s->running.size() + admit.size()) < s->sp.max_active) {
        JobPtr j = s->queue.front();
        if (j->bytes_est > s->sp.hbm_budget_bytes) {
          s->queue.pop_front();
          j->state = LF_JOB_FAILED;
          j->status = LF_ERR_OOM;
          j->finish_ns = now_ns();
          ++s->st.failed;
          s->cv_done.notify_all();
          continue;
        }
        if (used + j->bytes_est > s->sp.hbm_budget_bytes) break;
        used += j->bytes_est;
        s->queue.pop_front();
        admit.push_back(j);
        ++s->admitting;
      }
    }
    // create and seed the admitted jobs (outside the lock: the upload is long)
    for (const JobPtr& j : admit) {
      lf::TraceRange trace("lf_server admit");
      lf_mesh m = nullptr;
      lf_status r = lf::create_from_offdiag(&s->dev, j->n_v, j->rp, j->col, j->val, j->prm, &m);
      if (r == LF_OK && !j->V.empty())
        r = lf::attach_geometry(m, j->V.data(), j->n_v, j->F.data(), static_cast<int64_t>(j->F.size() / 3));
      if (r == LF_OK) r = lf_seed(m, j->seeds.data(), static_cast<int32_t>(j->seeds.size()));
      std::vector<int64_t>().swap(j->rp);
      std::vector<int32_t>().swap(j->col);
      std::vector<double>().swap(j->val);
      std::vector<double>().swap(j->V);
      std::vector<int32_t>().swap(j->F);
      std::lock_guard<std::mutex> lk(s->mu);
      j->mesh = m;
      j->admit_ns = now_ns();
      j->state = LF_JOB_RUNNING;
      s->running.push_back(j);
      --s->admitting;
      if (r != LF_OK) {
        j->status = r;                 // retired below, before any step
      } else {
        lf_stats_t stt;
        if (lf_stats(m, &stt) == LF_OK) j->device_bytes = stt.device_bytes;
      }
      s->st.peak_running = std::max<int64_t>(s->st.peak_running, static_cast<int64_t>(s->running.size()));
      s->st.peak_bytes = std::max(s->st.peak_bytes, reserved_bytes(s));
    }
    std::vector<JobPtr> batch;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      batch = s->running;
    }
    for (const JobPtr& j : batch)
      if (j->status != LF_OK) retire(s, j, LF_JOB_FAILED, j->status);
    batch.erase(std::remove_if(batch.begin(), batch.end(), [](const JobPtr& j) { return j->status != LF_OK; }),
                batch.end());
    if (batch.empty()) continue;

    // one chunk of steps for every running job
    std::vector<lf_mesh> ms;
    std::vector<int32_t> cnt;
    std::vector<int64_t> before;
    for (const JobPtr& j : batch) {
      ms.push_back(j->mesh);
      cnt.push_back(static_cast<int32_t>(std::min<int64_t>(s->sp.chunk_steps, j->n_iters - j->steps_done)));
      before.push_back(j->steps_done);
    }
    const int64_t t0 = now_ns();
    const lf_status r = lf_step_batch(ms.data(), static_cast<int32_t>(ms.size()), cnt.data());
    const int64_t t1 = now_ns();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.busy_ns += t1 - t0;
      ++s->st.batches;
    }
    for (size_t a = 0; a < batch.size(); ++a) {
      const JobPtr& j = batch[a];
      lf_stats_t stt;
      lf_status rs = lf_stats(j->mesh, &stt);
      if (rs == LF_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        j->steps_done = stt.steps;
        j->skeleton_total = j->skeleton_before + stt.skeleton_total;
        j->device_bytes = stt.device_bytes;
      }
      if (rs != LF_OK || (r != LF_OK && j->steps_done < before[a] + cnt[a])) {
        retire(s, j, LF_JOB_FAILED, rs != LF_OK ? rs : r);
        continue;
      }
      if (j->steps_done >= j->n_iters && j->lloyd_done < j->lloyd_rounds) {
        // a Lloyd-like round: new seeds and a fresh field; the round's steps
        // then run in the following batches
        const uint64_t sk = j->skeleton_total;
        rs = lf_lloyd(j->mesh, 1, 0, nullptr);
        if (rs != LF_OK) {
          retire(s, j, LF_JOB_FAILED, rs);
          continue;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        j->skeleton_before = sk;
        j->steps_done = 0;
        ++j->lloyd_done;
        continue;
      }
      if (j->steps_done >= j->n_iters) {
        if (j->want_dual) {
          int64_t n = 0;
          rs = lf_extract_dual(j->mesh, nullptr, 0, &n);
          std::vector<int32_t> tris(static_cast<size_t>(3 * n));
          if (rs == LF_OK && n > 0) rs = lf_extract_dual(j->mesh, tris.data(), n, &n);
          if (rs != LF_OK) {
            retire(s, j, LF_JOB_FAILED, rs);
            continue;
          }
          std::lock_guard<std::mutex> lk(s->mu);
          j->dual.swap(tris);
          j->dual_ready = true;
        }
        std::vector<int32_t> lab(static_cast<size_t>(j->n_v));
        rs = lf_labels(j->mesh, lab.data(), nullptr);
        if (rs == LF_OK) {
          std::lock_guard<std::mutex> lk(s->mu);
          j->labels.swap(lab);
        }
        retire(s, j, rs == LF_OK ? LF_JOB_DONE : LF_JOB_FAILED, rs);
      }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.peak_bytes = std::max(s->st.peak_bytes, reserved_bytes(s));
  }
  // stopping: nothing left runs
  std::vector<JobPtr> left;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    left = s->running;
  }
  for (const JobPtr& j : left) retire(s, j, LF_JOB_FAILED, LF_ERR_STATE);
  std::lock_guard<std::mutex> lk(s->mu);
  for (const JobPtr& j : s->queue) {
    j->state = LF_JOB_FAILED;
    j->status = LF_ERR_STATE;
    j->finish_ns = now_ns();
    ++s->st.failed;
  }
  s->queue.clear();
  s->cv_done.notify_all();
}

void fill_info(const Job& j, lf_job_info* info) {
  if (!info) return;
  info->state = j.state;
  info->status = j.status;
  info->n_v = j.n_v;
  info->steps = j.n_iters;
  info->steps_done = j.steps_done;
  info->arrival_ns = j.arrival_ns;
  info->admit_ns = j.admit_ns;
  info->finish_ns = j.finish_ns;
  info->skeleton_total = j.skeleton_total;
  info->device_bytes = j.device_bytes;
  info->lloyd_rounds = j.lloyd_rounds;
  info->lloyd_done = j.lloyd_done;
  info->dual_triangles = j.dual_ready ? static_cast<int64_t>(j.dual.size() / 3) : -1;
}

bool finished(const Job& j) { return j.state == LF_JOB_DONE || j.state == LF_JOB_FAILED; }

}  // namespace

extern "C" {

void lf_server_default_params(lf_server_params* p) {
  if (!p) return;
  p->hbm_budget_bytes = 150000000000LL;
  p->max_active = lf::kMaxJobs;
  p->chunk_steps = 256;
}

lf_status lf_server_create(const lf_device* dev, const lf_server_params* sp, lf_server* out) {
  if (!out) return server_fail(LF_ERR_INVALID, "out is null");
  *out = nullptr;
  lf_server_params p;
  lf_server_default_params(&p);
  if (sp) p = *sp;
  if (p.hbm_budget_bytes < 1) return server_fail(LF_ERR_INVALID, "hbm_budget_bytes must be positive");
  if (p.max_active < 1 || p.max_active > lf::kMaxJobs) return server_fail(LF_ERR_INVALID, "max_active must be in [1, 64]");
  if (p.chunk_steps < 1) return server_fail(LF_ERR_INVALID, "chunk_steps must be >= 1");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  cudaStream_t stream = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return server_fail(LF_ERR_CUDA, std::string("lf_server_create: ") + cudaGetErrorString(e));
  }
  lf_server s = new (std::nothrow) lf_server_s();
  if (!s) {
    cudaStreamDestroy(stream);
    return server_fail(LF_ERR_OOM, "host allocation");
  }
  s->sp = p;
  if (dev) s->dev = *dev;
  s->dev.cuda_stream = stream;
  s->device = device;
  s->stream = stream;
  try {
    s->thr = std::thread(scheduler, s);
  } catch (...) {
    cudaStreamDestroy(stream);
    delete s;
    return server_fail(LF_ERR_OOM, "cannot start the scheduler thread");
  }
  *out = s;
  return LF_OK;
}

lf_status lf_server_submit(lf_server s, const double* V, int64_t n_v, const int32_t* F, int64_t n_f,
                           const int32_t* seeds, int32_t k, int32_t n_iters, int32_t lloyd_rounds,
                           int32_t extract_dual, const lf_params* params, int64_t arrival_ns, int64_t* job_id) {
  if (!s || !job_id) return server_fail(LF_ERR_INVALID, "null server or job_id");
  lf_params prm;
  lf_default_params(&prm);
  if (params) prm = *params;
  std::string why;
  if (!lf::params_valid(prm, why) || !lf::mesh_ok(n_v, V, n_f, F, why) || !lf::seeds_ok(n_v, seeds, k, why))
    return server_fail(LF_ERR_INVALID, why);
  if (n_iters < 0 || lloyd_rounds < 0) return server_fail(LF_ERR_INVALID, "n_iters and lloyd_rounds must be >= 0");
  auto j = std::make_shared<Job>();
  try {
    if (!lf::cotan_offdiag(n_v, V, n_f, F, j->rp, j->col, j->val, why)) return server_fail(LF_ERR_INVALID, why);
    j->seeds.assign(seeds, seeds + k);
    if (lloyd_rounds > 0 || extract_dual) {
      j->V.assign(V, V + 3 * n_v);
      j->F.assign(F, F + 3 * n_f);
    }
  } catch (const std::bad_alloc&) {
    return server_fail(LF_ERR_OOM, "host allocation");
  }
  j->n_v = n_v;
  j->n_iters = n_iters;
  j->lloyd_rounds = lloyd_rounds;
  j->want_dual = extract_dual != 0;
  j->prm = prm;
  j->bytes_est = lf::device_bytes_estimate(n_v, static_cast<int64_t>(j->col.size()), prm);
  if (!j->V.empty()) j->bytes_est += lf::geometry_bytes_estimate(n_v, n_f, k);
  j->arrival_ns = arrival_ns > 0 ? arrival_ns : now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return server_fail(LF_ERR_STATE, "the server is shutting down");
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    ++s->st.submitted;
  }
  s->cv_work.notify_one();
  *job_id = j->id;
  return LF_OK;
}

lf_status lf_server_wait(lf_server s, int64_t job_id, double timeout_s, lf_job_info* info, int32_t* labels,
                         int32_t release) {
  if (!s) return server_fail(LF_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return server_fail(LF_ERR_INVALID, "unknown job id");
  JobPtr j = it->second;
  if (timeout_s > 0.0) {
    const auto dur = std::chrono::duration<double>(std::min(timeout_s, 1e7));
    s->cv_done.wait_for(lk, dur, [&] { return finished(*j); });
  }
  fill_info(*j, info);
  if (!finished(*j)) return LF_ERR_TIMEOUT;
  if (j->state == LF_JOB_DONE && labels && !j->labels.empty())
    std::memcpy(labels, j->labels.data(), sizeof(int32_t) * j->labels.size());
  const lf_status r = j->state == LF_JOB_DONE ? LF_OK : static_cast<lf_status>(j->status);
  if (release) s->jobs.erase(job_id);
  return r;
}

lf_status lf_server_dual_mesh(lf_server s, int64_t job_id, int32_t* tris, int64_t cap, int64_t* n_tris) {
  if (!s || !n_tris) return server_fail(LF_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return server_fail(LF_ERR_INVALID, "unknown job id");
  const Job& j = *it->second;
  if (!j.dual_ready) return server_fail(LF_ERR_STATE, "no dual mesh for this job (not asked for, or not finished)");
  const int64_t n = static_cast<int64_t>(j.dual.size() / 3);
  *n_tris = n;
  if (!tris) return LF_OK;
  if (cap < n) return server_fail(LF_ERR_CAPACITY, "tris holds fewer than *n_tris triangles");
  if (n > 0) std::memcpy(tris, j.dual.data(), sizeof(int32_t) * 3 * static_cast<size_t>(n));
  return LF_OK;
}

lf_status lf_server_drain(lf_server s, double timeout_s) {
  if (!s) return server_fail(LF_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->queue.empty() && s->running.empty() && s->admitting == 0; };
  if (timeout_s > 0.0) s->cv_done.wait_for(lk, std::chrono::duration<double>(std::min(timeout_s, 1e7)), idle);
  return idle() ? LF_OK : LF_ERR_TIMEOUT;
}

lf_status lf_server_stats(lf_server s, lf_server_stats_t* out) {
  if (!s || !out) return server_fail(LF_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->queued = static_cast<int64_t>(s->queue.size());
  out->running = static_cast<int64_t>(s->running.size()) + s->admitting;
  out->bytes_in_use = reserved_bytes(s);
  return LF_OK;
}

void lf_server_destroy(lf_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->thr.joinable()) s->thr.join();
  cudaStreamSynchronize(s->stream);
  cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
