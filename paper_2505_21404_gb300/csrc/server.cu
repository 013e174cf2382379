// Serving loop: PINN solve jobs (a problem, initial parameters, collocation
// data and a number of D-NGD iterations) are submitted from any thread and
// run by one worker thread that owns the device work.
//
// * Admission: a job is admitted when a slot is free and its device footprint
//   (dngd_workspace_bytes + its resident inputs) fits in what is left of the
//   HBM budget; a job that can never fit is rejected (DNGD_ERR_BUDGET).
//   Admission is first come, first served.
// * Continuous batching: every admitted job has its own context and stream
//   and always has its next iteration in flight (graph-captured step followed
//   by the device-side line search and update), so iterations of jobs that
//   arrived at different times overlap on the device; a finished job frees its
//   memory and slot for the next queued job at once.
// * State: parameters, points and targets stay on the device from admission
//   to completion; the result is copied back once.
// * Isolation: a job whose step fails (non-SPD, non-finite, timeout) is marked
//   FAILED and freed; no other job is touched.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  dngd_problem_desc desc;
  std::vector<double> theta, X, target;  // host copies until admission; theta holds the result when done
  int n_steps = 0;
  int state = DNGD_JOB_QUEUED;
  int steps_done = 0;
  dngd_status status = DNGD_OK;
  size_t bytes = 0;
  bool cancel = false;
  double loss = 0.0;
  double submit_t = 0.0, start_t = 0.0, end_t = 0.0;
  // device side (worker thread only)
  dngd_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  double *d_theta = nullptr, *d_X = nullptr, *d_target = nullptr, *d_delta = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool in_flight = false;
  int retries = 0;          // consecutive failed factorisations
  int64_t n = 0;
  int m = 0;
};

// Host copy of a caller's buffer: a plain memcpy from host memory (so a
// submission never waits behind work queued on the legacy stream), a
// synchronous device-to-host copy from device memory.
bool copy_in(void* dst, const void* src, size_t bytes) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, src) != cudaSuccess) {
    cudaGetLastError();
    a.type = cudaMemoryTypeUnregistered;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess;
  memcpy(dst, src, bytes);
  return false;
}

// The converse for results: memcpy into host memory, a synchronous
// host-to-device copy into device memory.
bool copy_out(void* dst, const void* src, size_t bytes) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, dst) != cudaSuccess) {
    cudaGetLastError();
    a.type = cudaMemoryTypeUnregistered;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess;
  memcpy(dst, src, bytes);
  return false;
}

}  // namespace

struct dngd_server {
  dngd_server_cfg cfg;
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job*> queue;
  std::vector<Job*> running;
  std::unordered_map<uint64_t, Job*> jobs;
  std::thread worker;
  std::atomic<bool> stop{false};
  uint64_t next_id = 1;
  int device = 0;
  std::vector<float> lat_ms;
  long long steps_total = 0;
  double t_first = 0.0, t_last = 0.0;
  int admitted = 0, rejected = 0, done = 0, failed = 0;
  double etas[64];
  int k = 31;

  void loop();
  bool admit_one();
  void release(Job* j, int state, dngd_status st);
};

void dngd_server::release(Job* j, int state, dngd_status st) {
  if (j->ctx) {
    cudaStreamSynchronize(j->st);
    if (state == DNGD_JOB_DONE) {
      cudaMemcpyAsync(j->theta.data(), j->d_theta, sizeof(double) * j->n, cudaMemcpyDeviceToHost, j->st);
      cudaStreamSynchronize(j->st);
    }
    dngd_destroy(j->ctx);
    j->ctx = nullptr;
  }
  for (double* p : {j->d_theta, j->d_X, j->d_target, j->d_delta})
    if (p) cudaFree(p);
  j->d_theta = j->d_X = j->d_target = j->d_delta = nullptr;
  if (j->ev0) cudaEventDestroy(j->ev0);
  if (j->ev1) cudaEventDestroy(j->ev1);
  j->ev0 = j->ev1 = nullptr;
  if (j->st) cudaStreamDestroy(j->st);
  j->st = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  used -= j->bytes;
  j->state = state;
  j->status = st;
  j->end_t = now_s();
  j->X.clear();
  j->X.shrink_to_fit();
  j->target.clear();
  j->target.shrink_to_fit();
  running.erase(std::remove(running.begin(), running.end(), j), running.end());
  if (state == DNGD_JOB_DONE) ++done;
  else ++failed;
  cv.notify_all();
}

// Admit the head of the queue if it fits (worker thread).  Returns true if a
// job was admitted or rejected.
bool dngd_server::admit_one() {
  Job* j = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (queue.empty()) return false;
    Job* h = queue.front();
    if (h->cancel) {
      queue.pop_front();
      h->state = DNGD_JOB_CANCELLED;
      cv.notify_all();
      return true;
    }
    if (h->bytes > budget) {
      queue.pop_front();
      h->state = DNGD_JOB_FAILED;
      h->status = DNGD_ERR_BUDGET;
      ++rejected;
      cv.notify_all();
      return true;
    }
    if ((int)running.size() >= cfg.max_slots || used + h->bytes > budget) return false;
    queue.pop_front();
    used += h->bytes;
    running.push_back(h);
    h->state = DNGD_JOB_RUNNING;
    h->start_t = now_s();
    ++admitted;
    j = h;
  }
  dngd_status s = DNGD_OK;
  if (cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking) != cudaSuccess) s = DNGD_ERR_CUDA;
  if (!s) s = dngd_create(&j->ctx, &j->desc, j->st);
  auto dal = [&](double** p, size_t cnt) {
    if (!s && cudaMalloc(p, sizeof(double) * cnt) != cudaSuccess) s = DNGD_ERR_OOM;
  };
  dal(&j->d_theta, j->n);
  dal(&j->d_X, j->X.size());
  dal(&j->d_target, j->m);
  dal(&j->d_delta, j->n);
  // the inputs go up on the job's own stream, ahead of its first step there
  // (the job streams are non-blocking: a copy on the legacy stream would not
  // be ordered before that step)
  if (!s && (cudaMemcpyAsync(j->d_theta, j->theta.data(), sizeof(double) * j->n, cudaMemcpyHostToDevice, j->st) ||
             cudaMemcpyAsync(j->d_X, j->X.data(), sizeof(double) * j->X.size(), cudaMemcpyHostToDevice, j->st) ||
             cudaMemcpyAsync(j->d_target, j->target.data(), sizeof(double) * j->m, cudaMemcpyHostToDevice, j->st)))
    s = DNGD_ERR_CUDA;
  if (!s && (cudaEventCreate(&j->ev0) || cudaEventCreate(&j->ev1))) s = DNGD_ERR_CUDA;
  if (s) release(j, DNGD_JOB_FAILED, s);
  return true;
}

void dngd_server::loop() {
  cudaSetDevice(device);
  while (!stop.load()) {
    bool busy = false;
    while (admit_one()) busy = true;
    std::vector<Job*> run;
    {
      std::lock_guard<std::mutex> lk(mu);
      run = running;
    }
    for (Job* j : run) {
      if (j->in_flight) {
        if (cudaEventQuery(j->ev1) == cudaErrorNotReady) continue;
        j->in_flight = false;
        busy = true;
        dngd_step_info info;
        dngd_status s = dngd_step_wait(j->ctx, &info);
        if (s == DNGD_ERR_NOT_SPD && ++j->retries <= 3) {
          // theta was left unchanged; the next iteration re-runs the shift
          // search synchronously
          j->in_flight = false;
        } else if (s && s != DNGD_ERR_NO_CONVERGE) {
          release(j, DNGD_JOB_FAILED, s);
          continue;
        } else {
          j->retries = 0;
        }
        if (s == DNGD_ERR_NOT_SPD) goto launch;
        {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, j->ev0, j->ev1);
        {
          std::lock_guard<std::mutex> lk(mu);
          lat_ms.push_back(ms);
          ++steps_total;
          t_last = now_s();
          j->steps_done++;
          j->loss = info.loss;
        }
        if (j->steps_done >= j->n_steps || j->cancel) {
          release(j, j->cancel ? DNGD_JOB_CANCELLED : DNGD_JOB_DONE, DNGD_OK);
          continue;
        }
        }
      }
    launch:
      if (!j->in_flight) {
        if (j->cancel) {
          release(j, DNGD_JOB_CANCELLED, DNGD_OK);
          continue;
        }
        busy = true;
        cudaEventRecord(j->ev0, j->st);
        dngd_status s = dngd_step_async(j->ctx, j->d_theta, j->d_X, j->d_target, j->d_delta);
        if (s == DNGD_ERR_NO_CONVERGE) s = DNGD_OK;
        if (!s) s = dngd_line_search_async(j->ctx, j->d_theta, j->d_X, j->d_target, j->d_delta, etas, k);
        if (s) {
          release(j, DNGD_JOB_FAILED, s);
          continue;
        }
        cudaEventRecord(j->ev1, j->st);
        j->in_flight = true;
      }
    }
    if (!busy) {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
  // shut down: finish what is in flight, free everything
  std::vector<Job*> run;
  {
    std::lock_guard<std::mutex> lk(mu);
    run = running;
  }
  for (Job* j : run) release(j, DNGD_JOB_CANCELLED, DNGD_OK);
}

extern "C" {

dngd_status dngd_server_create(dngd_server** out, const dngd_server_cfg* cfg) {
  if (!out || !cfg || cfg->max_slots < 1) return DNGD_ERR_INVALID_ARG;
  dngd_server* s = new dngd_server();
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete s;
    return DNGD_ERR_CUDA;
  }
  s->budget = cfg->hbm_budget_bytes ? (size_t)cfg->hbm_budget_bytes : (size_t)(0.8 * (double)fr);
  s->k = cfg->line_search_points > 0 && cfg->line_search_points <= 64 ? cfg->line_search_points : 31;
  for (int j = 0; j < s->k; ++j) s->etas[j] = 1.0 / (double)(1ull << j);
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return DNGD_OK;
}

dngd_status dngd_server_destroy(dngd_server* s) {
  if (!s) return DNGD_ERR_INVALID_ARG;
  s->stop.store(true);
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return DNGD_OK;
}

dngd_status dngd_submit(dngd_server* s, const dngd_job_desc* job, uint64_t* job_id) {
  if (!s || !job || !job_id || !job->theta0 || !job->X || !job->target || job->n_steps < 1)
    return DNGD_ERR_INVALID_ARG;
  if (job->desc.solver != DNGD_DENSE) return DNGD_ERR_INVALID_ARG;
  const int64_t n = dngd_num_params(&job->desc);
  if (n < 1) return DNGD_ERR_INVALID_ARG;
  size_t ws = 0;
  dngd_status st = dngd_workspace_bytes(&job->desc, &ws);
  if (st) return st;
  Job* j = new Job();
  j->desc = job->desc;
  j->n = n;
  int m = 0;
  for (int c = 0; c < job->desc.n_classes; ++c) m += job->desc.classes[c].count;
  j->m = m;
  const int d = job->desc.widths[0];
  // host copies (the caller may free its buffers after this call)
  j->theta.resize(n);
  j->X.resize((size_t)m * d);
  j->target.resize(m);
  if (copy_in(j->theta.data(), job->theta0, sizeof(double) * n) ||
      copy_in(j->X.data(), job->X, sizeof(double) * m * d) || copy_in(j->target.data(), job->target, sizeof(double) * m)) {
    delete j;
    return DNGD_ERR_CUDA;
  }
  j->n_steps = job->n_steps;
  j->bytes = ws + sizeof(double) * ((size_t)2 * n + (size_t)m * d + m) + ((size_t)8 << 20);
  j->submit_t = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  j->id = s->next_id++;
  if (s->t_first == 0.0) s->t_first = j->submit_t;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return DNGD_OK;
}

dngd_status dngd_poll(dngd_server* s, uint64_t job_id, dngd_job_state* out, double* theta_out) {
  if (!s || !out) return DNGD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return DNGD_ERR_INVALID_ARG;
  Job* j = it->second;
  out->state = j->state;
  out->steps_done = j->steps_done;
  out->status = j->status;
  out->loss = j->loss;
  out->queue_s = (j->start_t > 0 ? j->start_t : now_s()) - j->submit_t;
  out->run_s = j->start_t > 0 ? ((j->end_t > 0 ? j->end_t : now_s()) - j->start_t) : 0.0;
  if (theta_out && j->state == DNGD_JOB_DONE)
    if (copy_out(theta_out, j->theta.data(), sizeof(double) * j->n)) return DNGD_ERR_CUDA;
  return DNGD_OK;
}

dngd_status dngd_cancel(dngd_server* s, uint64_t job_id) {
  if (!s) return DNGD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return DNGD_ERR_INVALID_ARG;
  it->second->cancel = true;
  s->cv.notify_all();
  return DNGD_OK;
}

dngd_status dngd_server_stats(dngd_server* s, dngd_serving_stats* out) {
  if (!s || !out) return DNGD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->steps_total = s->steps_total;
  const double span = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
  out->steps_per_s = span > 0 ? (double)s->steps_total / span : 0.0;
  std::vector<float> v = s->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) -> double {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
    return v[i];
  };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  out->admitted = s->admitted;
  out->rejected = s->rejected;
  out->done = s->done;
  out->failed = s->failed;
  out->running = (int)s->running.size();
  out->queued = (int)s->queue.size();
  out->hbm_used_bytes = s->used;
  out->hbm_budget_bytes = s->budget;
  return DNGD_OK;
}

dngd_status dngd_server_drain(dngd_server* s, double timeout_s) {
  if (!s) return DNGD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  while (!(s->queue.empty() && s->running.empty())) {
    if (s->cv.wait_until(lk, until) == std::cv_status::timeout) return DNGD_ERR_TIMEOUT;
  }
  return DNGD_OK;
}

}  // extern "C"
