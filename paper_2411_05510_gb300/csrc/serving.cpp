// Serving: continuous batching of SSI solves.
//
// ssi_submit queues a job and returns.  A scheduler thread owns every CUDA call of the
// serving path:
//   * completion: a running job whose completion event has fired is finished (its
//     device status word and latency are recorded, its slot is freed);
//   * admission: queued jobs are scanned in arrival order; a job is admitted as soon
//     as a slot is free and the HBM budget can hold the slot's buffers for it (a
//     later, smaller job may pass an earlier one that does not fit yet);
//   * each admitted job runs on its slot's own stream, so work of different jobs
//     overlaps on the device; its results are copied to pinned host staging and
//     then to host memory owned by the context until ssi_release.
// Slot buffers (covariances, sketches, workspace) stay resident between jobs and
// grow only when a larger job needs them.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "common.cuh"
#include "pipeline.h"

namespace ssi {

namespace {
using Clock = std::chrono::steady_clock;

enum class JobState { Queued, Running, Done, Failed };

struct Job {
  uint64_t id = 0;
  ssi_job_desc desc{};
  std::vector<int32_t> lags, orders;
  JobPlan plan;
  JobState state = JobState::Queued;
  ssi_status result = SSI_OK;
  std::string error;
  Clock::time_point t_submit, t_done;
  int slot = -1;
  std::vector<ssi_pole> poles;
  std::vector<float> phi;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  JobBuffers B;
  void* d_out = nullptr;  // poles then phi
  size_t d_out_cap = 0;
  void* h_out = nullptr;  // pinned staging
  size_t h_out_cap = 0;
  int* h_status = nullptr;
  Job* job = nullptr;
};
}  // namespace

struct Serving {
  ssi_ctx* ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Job*> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<Slot> slots;
  std::thread th;
  bool stop = false;
  int max_queue = 1024;
  uint64_t next_id = 1;
};

namespace {

size_t out_bytes(const JobPlan& p) {
  return (size_t)p.n_slots * sizeof(ssi_pole) + (size_t)p.phi_floats * sizeof(float) + 256;
}

// bytes a slot must add to run `p`
size_t extra_bytes(const Slot& s, const JobPlan& p) {
  size_t need = 0;
  if (s.B.buf_cap < p.buf_bytes) need += p.buf_bytes + (1u << 20);
  if (s.B.ws.cap < p.ws_bytes) need += p.ws_bytes + (1u << 20);
  if (s.d_out_cap < out_bytes(p)) need += out_bytes(p);
  return need;
}

ssi_status launch_job(Serving* sv, Slot& s, Job* j) {
  ssi_ctx* ctx = sv->ctx;
  SSI_TRY(buffers_reserve(ctx, s.B, j->plan, s.stream));
  const size_t ob = out_bytes(j->plan);
  if (s.d_out_cap < ob) {
    if (s.d_out) ctx_free(ctx, s.d_out, s.d_out_cap);
    s.d_out = nullptr;
    s.d_out_cap = 0;
    SSI_TRY(ctx_alloc(ctx, &s.d_out, ob));
    s.d_out_cap = ob;
  }
  if (s.h_out_cap < ob) {
    if (s.h_out) cudaFreeHost(s.h_out);
    s.h_out = nullptr;
    SSI_CUDA(cudaMallocHost(&s.h_out, ob));
    s.h_out_cap = ob;
  }
  ssi_pole* d_poles = static_cast<ssi_pole*>(s.d_out);
  float* d_phi = reinterpret_cast<float*>(static_cast<char*>(s.d_out) +
                                          ((j->plan.n_slots * sizeof(ssi_pole) + 255) & ~size_t(255)));
  SSI_CUDA(cudaMemsetAsync(d_poles, 0, j->plan.n_slots * sizeof(ssi_pole), s.stream));
  SSI_TRY(run_job(ctx, &j->desc, j->plan, s.B, d_poles, d_phi, nullptr, s.stream));
  SSI_CUDA(cudaMemcpyAsync(s.h_out, s.d_out, ob, cudaMemcpyDeviceToHost, s.stream));
  SSI_CUDA(cudaMemcpyAsync(s.h_status, s.B.status, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
  SSI_CUDA(cudaMemsetAsync(s.B.status, 0, sizeof(int), s.stream));
  SSI_CUDA(cudaEventRecord(s.done, s.stream));
  return SSI_OK;
}

void finish_job(Slot& s, Job* j) {
  const size_t pole_bytes = j->plan.n_slots * sizeof(ssi_pole);
  j->poles.resize(j->plan.n_slots);
  std::memcpy(j->poles.data(), s.h_out, pole_bytes);
  j->phi.resize(j->plan.phi_floats);
  std::memcpy(j->phi.data(), static_cast<char*>(s.h_out) + ((pole_bytes + 255) & ~size_t(255)),
              j->plan.phi_floats * sizeof(float));
  const int st = *s.h_status;
  if (st & DEV_TIMEOUT) {
    j->result = SSI_E_TIMEOUT;
    j->error = "a device-side bounded wait ran out";
  }
  j->state = j->result == SSI_OK ? JobState::Done : JobState::Failed;
  j->t_done = Clock::now();
}

void scheduler(Serving* sv) {
  cudaSetDevice(sv->ctx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    bool progressed = false;
    int running = 0;
    // completions
    for (auto& s : sv->slots) {
      if (!s.job) continue;
      const cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) {
        ++running;
        continue;
      }
      Job* j = s.job;
      if (q != cudaSuccess) {
        j->result = SSI_E_CUDA;
        j->error = cudaGetErrorString(q);
        j->state = JobState::Failed;
        j->t_done = Clock::now();
      } else {
        finish_job(s, j);
      }
      s.job = nullptr;
      j->slot = -1;
      progressed = true;
      sv->cv_done.notify_all();
    }
    // admissions (arrival order, a job that does not fit yet does not block later ones)
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      Slot* free_slot = nullptr;
      for (auto& s : sv->slots)
        if (!s.job) {
          free_slot = &s;
          break;
        }
      if (!free_slot) break;
      Job* j = *it;
      size_t need = extra_bytes(*free_slot, j->plan);
      size_t in_use;
      {
        std::lock_guard<std::mutex> g(sv->ctx->mem_mu);
        in_use = sv->ctx->in_use;
      }
      if (in_use + need > sv->ctx->budget) {
        if (running == 0) {
          // nothing will free memory: release idle slot buffers and retry this job once
          for (auto& s : sv->slots)
            if (!s.job) {
              buffers_free(sv->ctx, s.B);
              if (s.d_out) ctx_free(sv->ctx, s.d_out, s.d_out_cap);
              s.d_out = nullptr;
              s.d_out_cap = 0;
            }
          need = extra_bytes(*free_slot, j->plan);
          std::lock_guard<std::mutex> g(sv->ctx->mem_mu);
          in_use = sv->ctx->in_use;
        }
        if (in_use + need > sv->ctx->budget) {
          if (running == 0) {
            j->result = SSI_E_NOMEM;
            j->error = "job does not fit the HBM budget";
            j->state = JobState::Failed;
            j->t_done = Clock::now();
            it = sv->queue.erase(it);
            sv->cv_done.notify_all();
            progressed = true;
            continue;
          }
          ++it;
          continue;
        }
      }
      ssi_status st = launch_job(sv, *free_slot, j);
      if (st != SSI_OK) {
        j->result = st;
        j->error = ssi_last_error();
        j->state = JobState::Failed;
        j->t_done = Clock::now();
        sv->cv_done.notify_all();
      } else {
        j->state = JobState::Running;
        j->slot = (int)(free_slot - sv->slots.data());
        free_slot->job = j;
        ++running;
      }
      it = sv->queue.erase(it);
      progressed = true;
    }
    if (running == 0 && sv->queue.empty()) {
      sv->cv_sched.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
    } else if (!progressed) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

ssi_status serving_start(ssi_ctx* ctx, int max_slots, int max_queue) {
  Serving* sv = new Serving();
  sv->ctx = ctx;
  sv->max_queue = max_queue;
  sv->slots.resize(max_slots);
  for (auto& s : sv->slots) {
    SSI_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    SSI_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    SSI_CUDA(cudaMallocHost(&s.h_status, sizeof(int)));
    *s.h_status = 0;
  }
  ctx->serving = sv;
  sv->th = std::thread(scheduler, sv);
  return SSI_OK;
}

}  // namespace

void serving_destroy(ssi_ctx* ctx) {
  Serving* sv = ctx->serving;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->stop = true;
  }
  sv->cv_sched.notify_all();
  if (sv->th.joinable()) sv->th.join();
  for (auto& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    buffers_free(ctx, s.B);
    if (s.d_out) ctx_free(ctx, s.d_out, s.d_out_cap);
    if (s.h_out) cudaFreeHost(s.h_out);
    if (s.h_status) cudaFreeHost(s.h_status);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  delete sv;
  ctx->serving = nullptr;
}

}  // namespace ssi

using namespace ssi;

extern "C" ssi_status ssi_serve_config(ssi_ctx* ctx, int max_slots, int max_queue) {
  SSI_CHECK(ctx, "ssi_serve_config: null context");
  SSI_CHECK(max_slots >= 1 && max_slots <= 64 && max_queue >= 1, "ssi_serve_config: bad limits");
  SSI_CUDA(cudaSetDevice(ctx->device));
  serving_destroy(ctx);
  ctx->inflight.store(max_slots);
  return serving_start(ctx, max_slots, max_queue);
}

extern "C" ssi_status ssi_submit(ssi_ctx* ctx, const ssi_job_desc* job, uint64_t* job_id) {
  SSI_CHECK(ctx && job_id, "ssi_submit: null pointer");
  SSI_TRY(validate_job(job));
  if (!ctx->serving) SSI_TRY(ssi_serve_config(ctx, 4, 1024));
  Serving* sv = ctx->serving;
  auto j = std::make_unique<Job>();
  j->desc = *job;
  j->lags.assign(job->lags, job->lags + job->n_lags);
  j->orders.assign(job->orders, job->orders + job->n_orders);
  j->desc.lags = j->lags.data();
  j->desc.orders = j->orders.data();
  j->plan = plan_job(&j->desc, ctx);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(sv->mu);
  if ((int)sv->queue.size() >= sv->max_queue) {
    set_error("ssi_submit: queue full (%d jobs)", sv->max_queue);
    return SSI_E_BUSY;
  }
  j->id = sv->next_id++;
  *job_id = j->id;
  sv->queue.push_back(j.get());
  sv->jobs[j->id] = std::move(j);
  sv->cv_sched.notify_all();
  return SSI_OK;
}

extern "C" ssi_status ssi_poll(ssi_ctx* ctx, uint64_t job_id, int timeout_ms, const ssi_pole** poles,
                               const float** phi, int64_t* n_slots, double* latency_us) {
  SSI_CHECK(ctx && ctx->serving, "ssi_poll: serving not started");
  Serving* sv = ctx->serving;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) {
    set_error("ssi_poll: unknown job %llu", (unsigned long long)job_id);
    return SSI_E_NOTFOUND;
  }
  Job* j = it->second.get();
  auto finished = [&] { return j->state == JobState::Done || j->state == JobState::Failed; };
  if (!finished()) {
    if (timeout_ms == 0) {
      set_error("ssi_poll: job %llu not finished", (unsigned long long)job_id);
      return SSI_E_TIMEOUT;
    }
    if (timeout_ms < 0) {
      sv->cv_done.wait(lk, finished);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
      set_error("ssi_poll: job %llu not finished after %d ms", (unsigned long long)job_id, timeout_ms);
      return SSI_E_TIMEOUT;
    }
  }
  if (latency_us)
    *latency_us = std::chrono::duration<double, std::micro>(j->t_done - j->t_submit).count();
  if (j->state == JobState::Failed) {
    set_error("job %llu failed: %s", (unsigned long long)job_id, j->error.c_str());
    return j->result;
  }
  if (poles) *poles = j->poles.data();
  if (phi) *phi = j->phi.data();
  if (n_slots) *n_slots = j->plan.n_slots;
  return SSI_OK;
}

extern "C" ssi_status ssi_release(ssi_ctx* ctx, uint64_t job_id) {
  SSI_CHECK(ctx && ctx->serving, "ssi_release: serving not started");
  Serving* sv = ctx->serving;
  std::lock_guard<std::mutex> g(sv->mu);
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) {
    set_error("ssi_release: unknown job %llu", (unsigned long long)job_id);
    return SSI_E_NOTFOUND;
  }
  if (it->second->state == JobState::Queued || it->second->state == JobState::Running) {
    set_error("ssi_release: job %llu still in flight", (unsigned long long)job_id);
    return SSI_E_BUSY;
  }
  sv->jobs.erase(it);
  return SSI_OK;
}
