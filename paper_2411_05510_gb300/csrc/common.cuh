// Internal declarations shared by the libssi translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <cstdio>
#include <atomic>
#include <string>
#include <mutex>
#include <tuple>
#include <vector>
#include <map>
#include <array>

#include "../../include/ssi.h"

namespace ssi {

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
ssi_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SSI_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return ::ssi::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SSI_CHECK(cond, ...)                                                  \
  do {                                                                        \
    if (!(cond)) { ::ssi::set_error(__VA_ARGS__); return SSI_E_INVALID; }     \
  } while (0)

#define SSI_TRY(call)                                                         \
  do {                                                                        \
    ssi_status s_ = (call);                                                   \
    if (s_ != SSI_OK) return s_;                                              \
  } while (0)

// device status word bits (written by kernels, read by the host)
enum : int {
  DEV_TIMEOUT = 1,        // a bounded wait ran out
  DEV_NOTCONVERGED = 2,   // an iteration hit its cap
  DEV_BADSHAPE = 4,       // a kernel met a shape it cannot handle
};

// ---------------------------------------------------------------------------
// workspace: a bump allocator over one device buffer owned by the context
// ---------------------------------------------------------------------------
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  void reset() { off = 0; }
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// byte-size accumulator that mirrors Workspace::take for planning
struct WsPlan {
  size_t bytes = 0;
  template <typename T>
  void add(size_t count) { bytes += (count * sizeof(T) + 255) & ~size_t(255); }
};

struct Serving;     // serving.cpp
struct JobBuffers;  // pipeline.h
struct BatchState;  // pipeline.cpp

}  // namespace ssi

namespace ssi {
// stage ids of the optional per-stage timers (ssi_profile / ssi_profile_read)
enum Stage : int {
  ST_SPLIT = 0, ST_LAG_GEMM = 1, ST_LAG_REDUCE = 2, ST_SKETCH_GEMM = 3, ST_QR = 4, ST_SMALL_SVD = 5,
  ST_GRAM = 6, ST_EIG = 7, ST_STAB = 8, ST_OTHER = 9, ST_EIG_VEC = 10, ST_CLUSTER = 11, ST_COUNT = 12
};
}  // namespace ssi

struct ssi_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;
  size_t in_use = 0;
  std::mutex mem_mu;
  ssi::Workspace ws;        // workspace of the direct (non-serving) calls
  ssi::Workspace ws_aux;    // second workspace of the direct calls (clustering's medoid tiles)
  int* dev_status = nullptr;  // device status word of the direct calls
  ssi::Serving* serving = nullptr;
  ssi::JobBuffers* solve = nullptr;  // buffers of ssi_solve
  ssi::BatchState* batch = nullptr;  // buffers, streams and tables of ssi_solve_batch
  std::atomic<int> inflight{1};        // solves expected to share the device at once
  std::atomic<long long> launches{0};  // kernels launched through this context
  bool prof_on = false;               // per-stage CUDA-event timers
  std::mutex prof_mu;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> prof_recs;
  // autotuned plan choices per job shape (ssi_autotune): lag-GEMM samples per split,
  // Toeplitz GEMM splits, Jacobi columns per block, QR row chunks per CTA (0 = the
  // model's choice)
  std::mutex tune_mu;
  std::map<std::string, std::array<int, 4>> tuned;
};

namespace ssi {

// memory accounting against the context budget
ssi_status ctx_alloc(ssi_ctx* ctx, void** p, size_t bytes);
void ctx_free(ssi_ctx* ctx, void* p, size_t bytes);
// grow `ws` to at least `bytes` (synchronises `stream` before freeing the old buffer)
ssi_status ws_reserve(ssi_ctx* ctx, Workspace& ws, size_t bytes, cudaStream_t stream);
// read and clear a device status word (synchronises `stream`)
ssi_status check_dev_status(int* dev_status, cudaStream_t stream);

// ---------------------------------------------------------------------------
// stage entry points with explicit workspace (used by the ABI wrappers, by
// ssi_solve and by the serving scheduler)
// ---------------------------------------------------------------------------
struct CovPlan {
  int l, l_pad, max_lag, n_nt, nb;    // channel padding, N tiles of the tensor-core kernel
  int64_t N, n_rows;
  int64_t ldy;                        // floats between channels of Y (N unless a caller sets it)
  int rows_per_split, n_split;
  size_t ws_bytes;
};
// max_ws: largest workspace the plan may need (the time split is coarsened to fit);
// rows > 0: samples per time split chosen by the caller (the autotuner) instead of the model
CovPlan cov_plan(int l, int64_t N, int max_lag, ssi_precision prec, int num_sms,
                 size_t max_ws = SIZE_MAX, int64_t rows = 0);
// acc == nullptr: R = covariances of Y; otherwise acc (double-float hi/lo pairs, same
// layout as R) += acc_sign * the unnormalised lag sums sum_t y_{t+k} y_t^T and R is unused
// (accumulation over segments)
ssi_status covariances_ws(ssi_ctx* ctx, Workspace& ws, const CovPlan& plan, const float* Y,
                          ssi_precision prec, double* R, int* dev_status, cudaStream_t stream,
                          float acc_sign = 0.f, float2* acc = nullptr);

struct RsvdPlan {
  int l, l_pad, i, k, K, Kp, q, L, L_pad;
  int tg_splits;        // reduction splits of the Toeplitz GEMMs
  int tg_mt;            // 128-row M tiles per CTA of the Toeplitz GEMMs (1 or 2)
  int jacobi_block;     // columns per block of the K x K Jacobi (0: the model's choice)
  int qr_cpc;           // QR row chunks per CTA (0: the model's choice)
  size_t ws_bytes;
};
// splits > 0 / jacobi_block > 0 / qr_cpc > 0: values chosen by the caller (the autotuner)
RsvdPlan rsvd_plan(int l, int i, int k, int oversample, int q, int num_sms, int splits = 0,
                   int jacobi_block = 0, int qr_cpc = 0);
// shared_device: other work (another lag of the same solve) runs beside this one, so the
// QR takes the half-device grid
// small64: FP64 Jacobi and U = Q U~ in FP64 (U, S double); otherwise FP32, written as
// double when out64 (U, S float otherwise)
ssi_status toeplitz_rsvd_ws(ssi_ctx* ctx, Workspace& ws, const RsvdPlan& plan, const double* R,
                            uint64_t seed, ssi_precision prec, bool small64, void* U, void* S,
                            bool out64, int* dev_status, cudaStream_t stream, bool shared_device);
ssi_status convert_f2d(const float* x, long long n, double* y, cudaStream_t stream);
ssi_status convert_d2f(const double* x, long long n, float* y, cudaStream_t stream);

struct RealizePlan {
  int n_lags, l, k, n_orders, max_order;
  int64_t slots_per_lag;
  size_t ws_bytes;
};
RealizePlan realize_plan(int n_lags, const int* lags, int l, int k, const int* orders,
                         int n_orders);
// A realisation prepared but not launched (csrc/realize.cu): with `defer`, realize_ws
// runs the Gram matrices and factorisations and returns the eig launches' parameters in
// *defer (free with realize_prep_free); realize_batch_launch then runs the
// eigen-decompositions of several jobs in one launch each (k_eig, k_eig_vectors), with
// their parameter blocks and item tables in `table` (realize_batch_table_bytes).
struct RealizePrep;
ssi_status realize_ws(ssi_ctx* ctx, Workspace& ws, const RealizePlan& plan, const int* lags,
                      const float* const* U, const int* orders, double dt, ssi_pole* poles,
                      float* phi, int* dev_status, cudaStream_t stream,
                      RealizePrep** defer = nullptr);
ssi_status realize_batch_launch(ssi_ctx* ctx, RealizePrep* const* preps, int n, void* table,
                                size_t table_cap, cudaStream_t stream);
size_t realize_batch_table_bytes(RealizePrep* const* preps, int n);
void realize_prep_free(RealizePrep* p);

// FP64 small problems (csrc/eig64.cu): U per lag is (l*i) x k FP64
size_t realize64_ws_bytes(int n_lags, const int* lags, int l, int k, const int* orders, int n_orders);
ssi_status realize64_ws(ssi_ctx* ctx, Workspace& ws, int n_lags, const int* lags, int l, int k,
                        const double* const* U, const int* orders, int n_orders, int64_t slots_per_lag,
                        double dt, ssi_pole* poles, float* phi, int* dev_status, cudaStream_t stream);
ssi_status lag_factor64_launch(const double* GH, int k, int n_lags, double* RM, double* Fs, int* status,
                               cudaStream_t stream);

ssi_status stabilize_ws(ssi_ctx* ctx, Workspace& ws, int n_lags, int n_orders, const int* orders,
                        int l, ssi_pole* poles, const float* phi, const ssi_stab_params* p,
                        cudaStream_t stream);
size_t stabilize_ws_bytes(int n_lags, int n_orders);

ssi_status gaussian_omega_launch(int rows, int cols, int ld, uint64_t seed, float* out,
                                 __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t stream);

// per-stage timing scope: records a CUDA event pair around the enclosed launches when the
// context's timers are on (host-side bookkeeping only; no synchronisation)
struct ProfScope {
  ssi_ctx* ctx;
  int stage;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  ProfScope(ssi_ctx* c, int st, cudaStream_t strm) : ctx(c), stage(st), s(strm) {
    if (ctx && ctx->prof_on) {
      cudaEventCreate(&e0);
      cudaEventRecord(e0, s);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEvent_t e1;
      cudaEventCreate(&e1);
      cudaEventRecord(e1, s);
      std::lock_guard<std::mutex> g(ctx->prof_mu);
      ctx->prof_recs.emplace_back(stage, e0, e1);
    }
  }
};
inline void count_launches(ssi_ctx* ctx, int n) {
  if (ctx) ctx->launches += n;
}

// shared launch helpers
int device_sms(int device);
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

}  // namespace ssi
