// Job planning and execution shared by ssi_solve and the serving scheduler.
#pragma once

#include <vector>

#include "common.cuh"

namespace ssi {

struct JobPlan {
  int max_lag;
  CovPlan cov;
  std::vector<RsvdPlan> rs;
  RealizePlan rz;
  size_t ws_bytes;     // scratch (shared by the stages, which run in sequence)
  std::vector<size_t> rs_off;   // per-lag RSVD scratch offsets (several lags run at once)
  size_t buf_bytes;    // R, U per lag, S, device Y copy, status word
  int64_t n_slots, phi_floats;
};

constexpr int LAG_STREAMS = 4;   // the per-lag RSVDs of a multi-lag solve run on this many streams

struct JobBuffers {
  void* buf = nullptr;
  size_t buf_cap = 0;
  Workspace ws;
  int* status = nullptr;
  bool status_cleared = false;
  // streams and fork/join events of the per-lag fan-out (created on first use)
  cudaStream_t lag_stream[LAG_STREAMS] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[LAG_STREAMS] = {};
};

ssi_status validate_job(const ssi_job_desc* j);
// tune: plan choices (lag-GEMM samples per split, Toeplitz splits, Jacobi block; 0 = the
// model's); nullptr = the context's autotuned choices for the job's shape, if any
JobPlan plan_job(const ssi_job_desc* j, ssi_ctx* ctx, const std::array<int, 4>* tune = nullptr);
std::string job_shape_key(const ssi_job_desc* j);
ssi_status buffers_reserve(ssi_ctx* ctx, JobBuffers& B, const JobPlan& p, cudaStream_t stream);
void buffers_free(ssi_ctx* ctx, JobBuffers& B);
// defer (FP32 small problems only): stop after the realisations' factorisations and
// return their pending eig launches in *defer; finish_job then runs what follows them
// (stability, singular values out) once the eig launches are made
ssi_status run_job(ssi_ctx* ctx, const ssi_job_desc* j, const JobPlan& p, JobBuffers& B,
                   ssi_pole* poles, float* phi, double* S_out, cudaStream_t stream,
                   RealizePrep** defer = nullptr);
ssi_status finish_job(ssi_ctx* ctx, const ssi_job_desc* j, const JobPlan& p, JobBuffers& B,
                      ssi_pole* poles, float* phi, double* S_out, cudaStream_t stream);
JobBuffers& ctx_solve_buffers(ssi_ctx* ctx);

}  // namespace ssi
