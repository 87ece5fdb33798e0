// Autotuner of the plan choices of one job shape (the batching pattern's tile shapes).
//
// Four choices of a solve are made by cost models when nothing else is known: the lag
// GEMM's time split (samples per FP32 partial sum; the model minimises whole waves of
// work units), the Toeplitz GEMMs' reduction splits (the model maximises wave efficiency),
// the K x K Jacobi's block width (columns per block of the parallel ordering, which
// trades grid barriers against the work of one outer round) and the sketch QR's grid (row
// chunks per CTA: the rows are cut into one chunk per SM, and fewer CTAs meet at cheaper
// barriers but each does more work, and above two chunks per CTA the rows no longer fit
// shared memory).  ssi_autotune times real solves of the job on the calling thread: for
// each choice in turn (coordinate descent), every candidate runs one untimed and two
// timed solves with the context's stage profiler on, and the candidate with the smallest
// time of its own stage is kept.  The QR grid is tuned for the shared device only
// (ssi_set_concurrency > 1): a cooperative grid of every SM cannot start while another
// solve's kernels hold SMs, so its candidates are grids of at most half the SMs (2 and 4
// chunks per CTA); a solve alone on the device always takes the whole-device grid (one
// chunk per CTA: 3.7 ms per solve on the benchmark's shape, against 5.2 ms with two).  (A
// score of time x CTAs, tried first, picked 8 chunks per CTA: 20.8 ms per solve instead of
// 3.7, a QR that holds few SMs but stays on the solve's critical path for longer.)  The
// four values are stored in the context under the job's shape (channels, samples, lags,
// k, oversampling, precisions) and every later plan of that shape, by ssi_solve or the
// serving loop, uses them.
#include <algorithm>
#include <array>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "pipeline.h"

namespace ssi {
namespace {

// Candidate samples per split of the lag GEMM: the model's choice and the split lengths
// that give whole waves of units near it, plus the longest allowed split.
std::vector<int> cov_candidates(const ssi_job_desc* j, int num_sms) {
  const int max_lag = 2 * j->lags[j->n_lags - 1] - 1;
  const CovPlan base = cov_plan(j->l, j->N, max_lag, (ssi_precision)j->prec, num_sms);
  std::vector<int> c{base.rows_per_split};
  for (double f : {0.5, 0.75, 1.5, 2.0}) {
    const int64_t r = std::min<int64_t>(16384, std::max<int64_t>(512, (int64_t)(base.rows_per_split * f)));
    c.push_back((int)round_up(r, 32));
  }
  c.push_back(16384);
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  return c;
}

std::vector<int> split_candidates(const ssi_job_desc* j, int num_sms) {
  const RsvdPlan base = rsvd_plan(j->l, j->lags[0], j->k, j->oversample, j->q, num_sms);
  std::vector<int> c{base.tg_splits};
  for (int s : {2, 3, 4, 6, 8, 12, 16}) c.push_back(s);
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  return c;
}

std::vector<int> block_candidates(const ssi_job_desc* j) {
  if (j->small == SSI_SMALL_FP64) return {1, 2, 3, 4, 6};
  return {6, 8, 10, 12, 14, 16, 20, 28};
}

std::vector<int> qr_candidates(bool shared) {
  if (shared) return {2, 4};
  return {1};
}

}  // namespace
}  // namespace ssi

using namespace ssi;

extern "C" ssi_status ssi_autotune(ssi_ctx* ctx, const ssi_job_desc* job, ssi_tuning* out) {
  SSI_CHECK(ctx && job, "ssi_autotune: null pointer");
  SSI_TRY(validate_job(job));
  SSI_CUDA(cudaSetDevice(ctx->device));
  int64_t n_slots = 0, phi_floats = 0;
  SSI_TRY(ssi_job_sizes(job, &n_slots, &phi_floats));
  void* poles = nullptr;
  void* phi = nullptr;
  const size_t pb = (size_t)n_slots * sizeof(ssi_pole), fb = (size_t)phi_floats * sizeof(float);
  SSI_TRY(ctx_alloc(ctx, &poles, pb));
  ssi_status st = ctx_alloc(ctx, &phi, fb);
  cudaStream_t s = nullptr;
  if (st == SSI_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
  }
  const bool prof_was = ctx->prof_on;
  std::array<int, 4> best{0, 0, 0, 0};
  double best_ms[4] = {0, 0, 0, 0};
  // stage time per solve of a candidate: one untimed solve, then two profiled ones
  auto time_stage = [&](const std::array<int, 4>& tv, int which, double* ms_out) -> ssi_status {
    const JobPlan p = plan_job(job, ctx, &tv);
    JobBuffers& B = ctx_solve_buffers(ctx);
    SSI_TRY(buffers_reserve(ctx, B, p, s));
    SSI_TRY(run_job(ctx, job, p, B, static_cast<ssi_pole*>(poles), static_cast<float*>(phi), nullptr, s));
    SSI_CUDA(cudaStreamSynchronize(s));
    double drop[ST_COUNT];
    SSI_TRY(ssi_profile_read(ctx, drop, nullptr, ST_COUNT, nullptr));
    ctx->prof_on = true;
    for (int r = 0; r < 2; ++r)
      SSI_TRY(run_job(ctx, job, p, B, static_cast<ssi_pole*>(poles), static_cast<float*>(phi), nullptr, s));
    ctx->prof_on = false;
    double ms[ST_COUNT];
    SSI_TRY(ssi_profile_read(ctx, ms, nullptr, ST_COUNT, nullptr));
    SSI_TRY(check_dev_status(ctx_solve_buffers(ctx).status, s));
    const double t = which == 0   ? ms[ST_SPLIT] + ms[ST_LAG_GEMM] + ms[ST_LAG_REDUCE]
                     : which == 1 ? ms[ST_SKETCH_GEMM]
                     : which == 2 ? ms[ST_SMALL_SVD]
                                  : ms[ST_QR];
    *ms_out = t / 2.0;
    return SSI_OK;
  };
  if (st == SSI_OK) {
    ctx->prof_on = false;
    const std::vector<int> cand[4] = {cov_candidates(job, ctx->num_sms),
                                      split_candidates(job, ctx->num_sms), block_candidates(job),
                                      qr_candidates(ctx->inflight > 1)};
    for (int which = 0; which < 4 && st == SSI_OK; ++which) {
      double bt = 1e300;
      int bv = 0;
      for (int v : cand[which]) {
        std::array<int, 4> tv = best;
        tv[which] = v;
        double t = 0.0;
        st = time_stage(tv, which, &t);
        if (st != SSI_OK) break;
        if (t < bt) {
          bt = t;
          bv = v;
        }
      }
      best[which] = bv;
      best_ms[which] = bt;
    }
  }
  ctx->prof_on = prof_was;
  if (s) cudaStreamDestroy(s);
  ctx_free(ctx, poles, pb);
  ctx_free(ctx, phi, fb);
  if (st != SSI_OK) return st;
  {
    std::lock_guard<std::mutex> g(ctx->tune_mu);
    ctx->tuned[job_shape_key(job)] = best;
  }
  if (out) {
    out->cov_rows_per_split = best[0];
    out->sketch_splits = best[1];
    out->jacobi_block = best[2];
    out->qr_chunks_per_cta = best[3];
    for (int i = 0; i < 4; ++i) out->stage_ms[i] = best_ms[i];
  }
  return SSI_OK;
}

extern "C" ssi_status ssi_tuning_get(ssi_ctx* ctx, const ssi_job_desc* job, ssi_tuning* out) {
  SSI_CHECK(ctx && job && out, "ssi_tuning_get: null pointer");
  SSI_TRY(validate_job(job));
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  auto it = ctx->tuned.find(job_shape_key(job));
  if (it == ctx->tuned.end()) {
    set_error("ssi_tuning_get: no tuned choices for this job shape");
    return SSI_E_NOTFOUND;
  }
  out->cov_rows_per_split = it->second[0];
  out->sketch_splits = it->second[1];
  out->jacobi_block = it->second[2];
  out->qr_chunks_per_cta = it->second[3];
  for (int i = 0; i < 4; ++i) out->stage_ms[i] = 0.0;
  return SSI_OK;
}

extern "C" ssi_status ssi_tuning_set(ssi_ctx* ctx, const ssi_job_desc* job, const ssi_tuning* in) {
  SSI_CHECK(ctx && job && in, "ssi_tuning_set: null pointer");
  SSI_TRY(validate_job(job));
  SSI_CHECK(in->cov_rows_per_split >= 0 && in->sketch_splits >= 0 && in->jacobi_block >= 0 &&
                in->qr_chunks_per_cta >= 0,
            "ssi_tuning_set: negative choice");
  std::lock_guard<std::mutex> g(ctx->tune_mu);
  ctx->tuned[job_shape_key(job)] = {in->cov_rows_per_split, in->sketch_splits, in->jacobi_block,
                                    in->qr_chunks_per_cta};
  return SSI_OK;
}
