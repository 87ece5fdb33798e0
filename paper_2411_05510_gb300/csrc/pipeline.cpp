// One complete solve (stages a-d) of one record, enqueued on one stream, and the
// planning of its device memory.  Used directly by ssi_solve and by the serving
// scheduler (serving.cpp).
#include <algorithm>
#include <string>
#include <vector>

#include "common.cuh"
#include "pipeline.h"

namespace ssi {

ssi_status validate_job(const ssi_job_desc* j) {
  SSI_CHECK(j, "job: null descriptor");
  SSI_CHECK(j->Y, "job: null record");
  SSI_CHECK(j->l >= 1 && j->l <= 1024, "job: l=%d out of range", j->l);
  SSI_CHECK(j->fs > 0, "job: fs must be positive");
  SSI_CHECK(j->n_lags >= 1 && j->n_lags <= 64 && j->lags, "job: 1 <= n_lags <= 64");
  SSI_CHECK(j->n_orders >= 1 && j->n_orders <= 512 && j->orders, "job: 1 <= n_orders <= 512");
  SSI_CHECK(j->k >= 2 && j->oversample >= 0 && j->q >= 0, "job: bad k / oversample / q");
  SSI_CHECK(j->k <= 512 && j->k + j->oversample <= 16384,
            "job: need k <= 512 and k + oversample <= 16384");
  SSI_CHECK(j->prec == SSI_PREC_FP32 || j->prec == SSI_PREC_SPLIT_BF16, "job: bad precision");
  SSI_CHECK(j->small == SSI_SMALL_FP32 || j->small == SSI_SMALL_FP64,
            "job: bad small-problem precision");
  for (int t = 0; t < j->n_lags; ++t) {
    SSI_CHECK(j->lags[t] >= 2, "job: lag %d < 2", j->lags[t]);
    SSI_CHECK(t == 0 || j->lags[t] > j->lags[t - 1], "job: lags must ascend");
    SSI_CHECK((int64_t)j->l * j->lags[t] >= j->k + j->oversample, "job: l*i < k + oversample");
  }
  const int max_lag = 2 * j->lags[j->n_lags - 1] - 1;
  SSI_CHECK(j->N > max_lag, "job: N=%lld must exceed 2*max(lags)-1=%d", (long long)j->N, max_lag);
  SSI_CHECK(j->N < (1LL << 31) - 1024, "job: N too large");
  for (int m = 0; m < j->n_orders; ++m) {
    SSI_CHECK(j->orders[m] >= 2 && j->orders[m] % 2 == 0 && j->orders[m] <= j->k,
              "job: order %d must be even and in [2, k]", j->orders[m]);
    SSI_CHECK(j->orders[m] <= 512, "job: order %d > 512 not supported", j->orders[m]);
    SSI_CHECK(m == 0 || j->orders[m] > j->orders[m - 1], "job: orders must ascend");
  }
  return SSI_OK;
}

std::string job_shape_key(const ssi_job_desc* j) {
  std::string key = std::to_string(j->l) + ":" + std::to_string(j->N) + ":" + std::to_string(j->k) +
                    ":" + std::to_string(j->oversample) + ":" + std::to_string(j->prec) + ":" +
                    std::to_string(j->small) + ":";
  for (int t = 0; t < j->n_lags; ++t) key += std::to_string(j->lags[t]) + ",";
  return key;
}

JobPlan plan_job(const ssi_job_desc* j, ssi_ctx* ctx, const std::array<int, 4>* tune) {
  const int num_sms = ctx->num_sms;
  std::array<int, 4> tv{0, 0, 0, 0};
  if (tune) {
    tv = *tune;
  } else {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    auto it = ctx->tuned.find(job_shape_key(j));
    if (it != ctx->tuned.end()) tv = it->second;
  }
  JobPlan p{};
  p.max_lag = 2 * j->lags[j->n_lags - 1] - 1;
  p.cov = cov_plan(j->l, j->N, p.max_lag, (ssi_precision)j->prec, num_sms, SIZE_MAX, tv[0]);
  size_t ws = p.cov.ws_bytes;
  // the RSVDs of several lags run at once, each in its own region of the scratch
  size_t rs_total = 0;
  for (int t = 0; t < j->n_lags; ++t) {
    p.rs.push_back(rsvd_plan(j->l, j->lags[t], j->k, j->oversample, j->q, num_sms, tv[1], tv[2],
                             tv[3]));
    p.rs_off.push_back(rs_total);
    rs_total += (p.rs.back().ws_bytes + 255) & ~size_t(255);
  }
  ws = std::max(ws, rs_total);
  std::vector<int> lags(j->lags, j->lags + j->n_lags), orders(j->orders, j->orders + j->n_orders);
  p.rz = realize_plan(j->n_lags, lags.data(), j->l, j->k, orders.data(), j->n_orders);
  if (j->small == SSI_SMALL_FP64)
    p.rz.ws_bytes = realize64_ws_bytes(j->n_lags, lags.data(), j->l, j->k, orders.data(), j->n_orders);
  ws = std::max(ws, p.rz.ws_bytes);
  p.ws_bytes = ws;
  WsPlan b;
  b.add<int>(64);                                              // device status words
  b.add<double>((size_t)p.max_lag * j->l * j->l);             // R
  const size_t esz = j->small == SSI_SMALL_FP64 ? sizeof(double) : sizeof(float);
  for (int t = 0; t < j->n_lags; ++t) b.add<char>(esz * j->l * j->lags[t] * j->k);   // U_t
  b.add<char>(esz * j->n_lags * j->k);                                                 // S
  if (j->y_on_host) b.add<float>((size_t)j->l * j->N);        // device copy of Y
  p.buf_bytes = b.bytes;
  p.n_slots = p.rz.slots_per_lag * j->n_lags;
  p.phi_floats = p.n_slots * 2 * j->l;
  return p;
}

namespace {

// the job's buffers carved out of B.buf (the same layout on every call of a plan)
struct JobCarve {
  int* status;
  double* R;
  std::vector<void*> U;
  char* S;
  float* Ydev;
  size_t esz;
};

ssi_status carve_job(const ssi_job_desc* j, const JobPlan& p, JobBuffers& B, JobCarve& c) {
  Workspace carve;
  carve.base = static_cast<char*>(B.buf);
  carve.cap = B.buf_cap;
  // the status words first: their address must not depend on the job's sizes, because
  // they are cleared only when the buffer is allocated and then reset by each read
  c.status = carve.take<int>(64);
  c.R = carve.take<double>((size_t)p.max_lag * j->l * j->l);
  const bool s64 = j->small == SSI_SMALL_FP64;
  c.esz = s64 ? sizeof(double) : sizeof(float);
  c.U.assign(j->n_lags, nullptr);
  for (int t = 0; t < j->n_lags; ++t) c.U[t] = carve.take<char>(c.esz * j->l * j->lags[t] * j->k);
  c.S = carve.take<char>(c.esz * j->n_lags * j->k);
  c.Ydev = j->y_on_host ? carve.take<float>((size_t)j->l * j->N) : nullptr;
  if (!c.R || !c.S || !c.status || (j->y_on_host && !c.Ydev)) {
    set_error("solve: job buffers too small");
    return SSI_E_NOMEM;
  }
  return SSI_OK;
}

}  // namespace

ssi_status run_job(ssi_ctx* ctx, const ssi_job_desc* j, const JobPlan& p, JobBuffers& B,
                   ssi_pole* poles, float* phi, double* S_out, cudaStream_t stream,
                   RealizePrep** defer) {
  JobCarve c;
  SSI_TRY(carve_job(j, p, B, c));
  int* status = c.status;
  double* R = c.R;
  const bool s64 = j->small == SSI_SMALL_FP64;
  const size_t esz = c.esz;
  std::vector<void*>& U = c.U;
  char* S = c.S;
  B.status = status;
  const float* Y = j->Y;
  if (j->y_on_host) {
    SSI_CUDA(cudaMemcpyAsync(c.Ydev, j->Y, sizeof(float) * (size_t)j->l * j->N,
                             cudaMemcpyHostToDevice, stream));
    Y = c.Ydev;
  }
  if (!B.status_cleared) {
    SSI_CUDA(cudaMemsetAsync(status, 0, 64 * sizeof(int), stream));
    B.status_cleared = true;
  }
  SSI_TRY(covariances_ws(ctx, B.ws, p.cov, Y, (ssi_precision)j->prec, R, status, stream));
  if (j->n_lags == 1) {
    SSI_TRY(toeplitz_rsvd_ws(ctx, B.ws, p.rs[0], R, j->seed, (ssi_precision)j->prec, s64, U[0], S,
                             s64, status, stream, false));
  } else {
    // the lags' RSVDs are independent (Sec. 2.3): fork them over LAG_STREAMS streams, each
    // lag in its own scratch region, and join before the realisations
    const int n_str = std::min(j->n_lags, LAG_STREAMS);
    if (!B.fork) {
      SSI_CUDA(cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
      for (int a = 0; a < LAG_STREAMS; ++a) {
        SSI_CUDA(cudaStreamCreateWithFlags(&B.lag_stream[a], cudaStreamNonBlocking));
        SSI_CUDA(cudaEventCreateWithFlags(&B.join[a], cudaEventDisableTiming));
      }
    }
    SSI_CUDA(cudaEventRecord(B.fork, stream));
    for (int a = 0; a < n_str; ++a) SSI_CUDA(cudaStreamWaitEvent(B.lag_stream[a], B.fork, 0));
    for (int t = 0; t < j->n_lags; ++t) {
      Workspace sub;
      sub.base = B.ws.base + p.rs_off[t];
      sub.cap = p.rs[t].ws_bytes;
      SSI_TRY(toeplitz_rsvd_ws(ctx, sub, p.rs[t], R, j->seed, (ssi_precision)j->prec, s64, U[t],
                               S + esz * t * j->k, s64, status, B.lag_stream[t % n_str], true));
    }
    for (int a = 0; a < n_str; ++a) {
      SSI_CUDA(cudaEventRecord(B.join[a], B.lag_stream[a]));
      SSI_CUDA(cudaStreamWaitEvent(stream, B.join[a], 0));
    }
  }
  std::vector<int> lags(j->lags, j->lags + j->n_lags), orders(j->orders, j->orders + j->n_orders);
  if (s64) {
    SSI_CHECK(!defer, "solve: deferred realisations need FP32 small problems");
    std::vector<const double*> Ud(j->n_lags);
    for (int t = 0; t < j->n_lags; ++t) Ud[t] = static_cast<const double*>(U[t]);
    SSI_TRY(realize64_ws(ctx, B.ws, j->n_lags, lags.data(), j->l, j->k, Ud.data(), orders.data(),
                         j->n_orders, p.rz.slots_per_lag, 1.0 / j->fs, poles, phi, status, stream));
  } else {
    std::vector<const float*> Uc(j->n_lags);
    for (int t = 0; t < j->n_lags; ++t) Uc[t] = static_cast<const float*>(U[t]);
    SSI_TRY(realize_ws(ctx, B.ws, p.rz, lags.data(), Uc.data(), orders.data(), 1.0 / j->fs, poles,
                       phi, status, stream, defer));
    if (defer) return SSI_OK;
  }
  return finish_job(ctx, j, p, B, poles, phi, S_out, stream);
}

ssi_status finish_job(ssi_ctx* ctx, const ssi_job_desc* j, const JobPlan& p, JobBuffers& B,
                      ssi_pole* poles, float* phi, double* S_out, cudaStream_t stream) {
  JobCarve c;
  SSI_TRY(carve_job(j, p, B, c));
  std::vector<int> orders(j->orders, j->orders + j->n_orders);
  SSI_TRY(stabilize_ws(ctx, B.ws, j->n_lags, j->n_orders, orders.data(), j->l, poles, phi, &j->stab,
                       stream));
  if (S_out) {
    if (j->small == SSI_SMALL_FP64)
      SSI_CUDA(cudaMemcpyAsync(S_out, c.S, sizeof(double) * (size_t)j->n_lags * j->k,
                               cudaMemcpyDeviceToDevice, stream));
    else
      SSI_TRY(convert_f2d(reinterpret_cast<const float*>(c.S), (long long)j->n_lags * j->k, S_out,
                          stream));
  }
  return SSI_OK;
}

ssi_status buffers_reserve(ssi_ctx* ctx, JobBuffers& B, const JobPlan& p, cudaStream_t stream) {
  if (B.buf_cap < p.buf_bytes) {
    if (B.buf) {
      SSI_CUDA(cudaStreamSynchronize(stream));
      ctx_free(ctx, B.buf, B.buf_cap);
      B.buf = nullptr;
      B.buf_cap = 0;
    }
    size_t want = (p.buf_bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
    SSI_TRY(ctx_alloc(ctx, &B.buf, want));
    B.buf_cap = want;
    B.status_cleared = false;
  }
  return ws_reserve(ctx, B.ws, p.ws_bytes, stream);
}

void buffers_free(ssi_ctx* ctx, JobBuffers& B) {
  for (int a = 0; a < LAG_STREAMS; ++a) {
    if (B.lag_stream[a]) {
      cudaStreamSynchronize(B.lag_stream[a]);
      cudaStreamDestroy(B.lag_stream[a]);
    }
    if (B.join[a]) cudaEventDestroy(B.join[a]);
  }
  if (B.fork) cudaEventDestroy(B.fork);
  if (B.buf) ctx_free(ctx, B.buf, B.buf_cap);
  if (B.ws.base) ctx_free(ctx, B.ws.base, B.ws.cap);
  B = JobBuffers{};
}

// State of ssi_solve_batch kept in the context between calls: one set of job buffers per
// job of the largest batch so far, the streams the jobs' front stages run on, and the
// device table of the batched eig launches.
constexpr int BATCH_STREAMS = 4;
struct BatchState {
  std::vector<JobBuffers*> bufs;
  cudaStream_t stream[BATCH_STREAMS] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[BATCH_STREAMS] = {};
  void* table = nullptr;
  size_t table_cap = 0;
};

JobBuffers& ctx_solve_buffers(ssi_ctx* ctx) {
  if (!ctx->solve) ctx->solve = new JobBuffers();
  return *ctx->solve;
}

void solve_buffers_destroy(ssi_ctx* ctx) {
  if (ctx->solve) {
    buffers_free(ctx, *ctx->solve);
    delete ctx->solve;
    ctx->solve = nullptr;
  }
  if (BatchState* bs = ctx->batch) {
    for (JobBuffers* b : bs->bufs) {
      buffers_free(ctx, *b);
      delete b;
    }
    for (int a = 0; a < BATCH_STREAMS; ++a) {
      if (bs->stream[a]) {
        cudaStreamSynchronize(bs->stream[a]);
        cudaStreamDestroy(bs->stream[a]);
      }
      if (bs->join[a]) cudaEventDestroy(bs->join[a]);
    }
    if (bs->fork) cudaEventDestroy(bs->fork);
    if (bs->table) ctx_free(ctx, bs->table, bs->table_cap);
    delete bs;
    ctx->batch = nullptr;
  }
}

}  // namespace ssi

using namespace ssi;

extern "C" ssi_status ssi_job_sizes(const ssi_job_desc* job, int64_t* n_slots, int64_t* phi_floats) {
  SSI_TRY(validate_job(job));
  int64_t s = 0;
  for (int m = 0; m < job->n_orders; ++m) s += job->orders[m] / 2;
  s *= job->n_lags;
  if (n_slots) *n_slots = s;
  if (phi_floats) *phi_floats = s * 2 * job->l;
  return SSI_OK;
}

extern "C" ssi_status ssi_solve(ssi_ctx* ctx, const ssi_job_desc* job, ssi_pole* poles, float* phi,
                                double* S_out, void* stream) {
  SSI_CHECK(ctx && poles && phi, "ssi_solve: null pointer");
  SSI_TRY(validate_job(job));
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  JobPlan p = plan_job(job, ctx);
  JobBuffers& B = ctx_solve_buffers(ctx);
  SSI_TRY(buffers_reserve(ctx, B, p, s));
  return run_job(ctx, job, p, B, poles, phi, S_out, s);
}

extern "C" ssi_status ssi_sync_status(ssi_ctx* ctx, void* stream) {
  SSI_CHECK(ctx, "ssi_sync_status: null context");
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SSI_CUDA(cudaStreamSynchronize(s));
  ssi_status st = check_dev_status(ctx->dev_status, s);
  if (st != SSI_OK) return st;
  JobBuffers& B = ctx_solve_buffers(ctx);
  if (B.status) return check_dev_status(B.status, s);
  return SSI_OK;
}

extern "C" ssi_status ssi_solve_batch(ssi_ctx* ctx, int n_jobs, const ssi_job_desc* jobs,
                                      ssi_pole* const* poles, float* const* phi,
                                      double* const* S_out, void* stream) {
  SSI_CHECK(ctx && jobs && poles && phi, "ssi_solve_batch: null pointer");
  SSI_CHECK(n_jobs >= 1 && n_jobs <= SSI_BATCH_MAX, "ssi_solve_batch: 1 <= n_jobs <= %d",
            SSI_BATCH_MAX);
  for (int i = 0; i < n_jobs; ++i) {
    SSI_TRY(validate_job(&jobs[i]));
    SSI_CHECK(poles[i] && phi[i], "ssi_solve_batch: null output of job %d", i);
    SSI_CHECK(jobs[i].small == SSI_SMALL_FP32,
              "ssi_solve_batch: job %d has FP64 small problems (the batched eig is FP32)", i);
  }
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!ctx->batch) ctx->batch = new BatchState();
  BatchState& bs = *ctx->batch;
  if (!bs.fork) {
    SSI_CUDA(cudaEventCreateWithFlags(&bs.fork, cudaEventDisableTiming));
    for (int a = 0; a < BATCH_STREAMS; ++a) {
      SSI_CUDA(cudaStreamCreateWithFlags(&bs.stream[a], cudaStreamNonBlocking));
      SSI_CUDA(cudaEventCreateWithFlags(&bs.join[a], cudaEventDisableTiming));
    }
  }
  while ((int)bs.bufs.size() < n_jobs) bs.bufs.push_back(new JobBuffers());
  std::vector<JobPlan> plans(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    plans[i] = plan_job(&jobs[i], ctx);
    SSI_TRY(buffers_reserve(ctx, *bs.bufs[i], plans[i], s));
  }
  // each job's covariances, RSVD and factorisations on one of the batch streams (jobs i,
  // i + 4, ... one after another), forked from and joined back to the caller's stream
  const int n_str = std::min(n_jobs, BATCH_STREAMS);
  SSI_CUDA(cudaEventRecord(bs.fork, s));
  for (int a = 0; a < n_str; ++a) SSI_CUDA(cudaStreamWaitEvent(bs.stream[a], bs.fork, 0));
  std::vector<RealizePrep*> preps(n_jobs, nullptr);
  ssi_status st = SSI_OK;
  for (int i = 0; i < n_jobs && st == SSI_OK; ++i)
    st = run_job(ctx, &jobs[i], plans[i], *bs.bufs[i], poles[i], phi[i],
                 S_out ? S_out[i] : nullptr, bs.stream[i % n_str], &preps[i]);
  for (int a = 0; a < n_str; ++a) {
    cudaEventRecord(bs.join[a], bs.stream[a]);
    cudaStreamWaitEvent(s, bs.join[a], 0);
  }
  // one launch of each eig kernel over every job's realisations, then each job's stability
  if (st == SSI_OK) {
    const size_t need = realize_batch_table_bytes(preps.data(), n_jobs);
    if (bs.table_cap < need) {
      if (bs.table) {
        cudaStreamSynchronize(s);
        ctx_free(ctx, bs.table, bs.table_cap);
        bs.table = nullptr;
        bs.table_cap = 0;
      }
      st = ctx_alloc(ctx, &bs.table, need);
      if (st == SSI_OK) bs.table_cap = need;
    }
  }
  if (st == SSI_OK) st = realize_batch_launch(ctx, preps.data(), n_jobs, bs.table, bs.table_cap, s);
  for (int i = 0; i < n_jobs && st == SSI_OK; ++i)
    st = finish_job(ctx, &jobs[i], plans[i], *bs.bufs[i], poles[i], phi[i],
                    S_out ? S_out[i] : nullptr, s);
  for (RealizePrep* r : preps)
    if (r) realize_prep_free(r);
  return st;
}

