// Sliding-window output covariances for continuous monitoring.
//
// The monitored bridge of Sec. 3.2 is recorded without a break in two-hour files and
// identified file after file over a month (Sec. 3.2.2); the related work of Sec. 1 follows
// time-varying modes with sliding data windows.  Recomputing R_1..R_K of a whole window
// after every new block costs O(l^2 W K); this object keeps the unnormalised lag sums
//     S_k = sum over pairs (t, t+k) inside the window of y_{t+k} y_t^T
// and updates them with the pairs that enter and leave, at O(l^2 (B + K) K) per block of
// B samples.  Both updates are differences of two whole-segment lag sums, which the stage
// (a) kernels add straight into S (their reduction's accumulate mode; S is double-float,
// hi + lo FP32 pairs, ~2^-48 relative, so the per-element update needs no FP64):
//   entering pairs, t + k in [e, e+B):   F([e-T, e+B)) - F([e-T, e))
//   leaving pairs,  t in [s, s+D):       F([s, s+D+T)) - F([s+D, s+D+T))
// where F(seg) = sum over the pairs inside seg, e / s are the window's
// end / start and T = K + 1 >= K (every pair with one end in the block has its other end
// within K samples).  R_k of the window is S_k / (n - k).
//
// Samples live in a device ring of W + B_max columns per channel; segments are gathered
// into a contiguous buffer by 2D copies.
#include "common.cuh"

#include <algorithm>

struct ssi_cov_stream {
  ssi_ctx* ctx = nullptr;
  int l = 0, K = 0;
  int64_t W = 0, Bmax = 0, C = 0;
  ssi_precision prec = SSI_PREC_SPLIT_BF16;
  float* ring = nullptr;      // l x C
  float* seg = nullptr;       // l x (Bmax + K + 1)
  float2* S = nullptr;        // K x l x l lag sums, double-float (hi, lo)
  int64_t start = 0, n = 0;   // absolute index of the window's first sample; samples held
  size_t bytes_ring = 0, bytes_seg = 0, bytes_S = 0;
  ssi::Workspace ws;
};

namespace ssi {
namespace {

// R_k = S_k / (n - k): one block per (lag k, eight channels a), the reciprocal once per
// block (FP64 divisions are slow here).
__global__ void __launch_bounds__(256) k_stream_normalise(const float2* __restrict__ S, int l, long long n,
                                                          double* __restrict__ R) {
  __shared__ double s_inv;
  const int k = blockIdx.y + 1;
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_inv = 1.0 / (double)(n - k);
  __syncthreads();
  if (a >= l) return;
  const long long row = ((long long)(k - 1) * l + a) * l;
  for (int b = lane; b < l; b += 32) {
    const float2 v = S[row + b];
    R[row + b] = ((double)v.x + (double)v.y) * s_inv;
  }
}

// Copy absolute samples [a, a + len) of every channel from the ring into dst
// (l x len, channel-major).
ssi_status ring_gather(ssi_cov_stream* st, int64_t a, int64_t len, float* dst, cudaStream_t s) {
  int64_t done = 0;
  while (done < len) {
    const int64_t pos = (a + done) % st->C;
    const int64_t w = std::min(len - done, st->C - pos);
    SSI_CUDA(cudaMemcpy2DAsync(dst + done, (size_t)len * sizeof(float), st->ring + pos,
                               (size_t)st->C * sizeof(float), (size_t)w * sizeof(float), (size_t)st->l,
                               cudaMemcpyDeviceToDevice, s));
    done += w;
  }
  return SSI_OK;
}

// S += sign * F(absolute samples [a, a + len)).
ssi_status segment_acc(ssi_cov_stream* st, int64_t a, int64_t len, double sign, cudaStream_t s) {
  SSI_TRY(ring_gather(st, a, len, st->seg, s));
  ssi_ctx* ctx = st->ctx;
  CovPlan plan = cov_plan(st->l, len, st->K, st->prec, ctx->num_sms);
  SSI_TRY(ws_reserve(ctx, st->ws, plan.ws_bytes, s));
  st->ws.reset();
  return covariances_ws(ctx, st->ws, plan, st->seg, st->prec, nullptr, ctx->dev_status, s,
                        (float)sign, st->S);
}

void stream_free(ssi_cov_stream* st) {
  ctx_free(st->ctx, st->ring, st->bytes_ring);
  ctx_free(st->ctx, st->seg, st->bytes_seg);
  ctx_free(st->ctx, st->S, st->bytes_S);
  if (st->ws.base) ctx_free(st->ctx, st->ws.base, st->ws.cap);
  delete st;
}

}  // namespace
}  // namespace ssi

extern "C" ssi_status ssi_cov_stream_create(ssi_ctx* ctx, int l, int max_lag, int64_t window,
                                            int64_t max_block, ssi_precision prec,
                                            ssi_cov_stream** out) {
  using namespace ssi;
  if (out) *out = nullptr;
  SSI_CHECK(ctx && out, "ssi_cov_stream_create: null pointer");
  SSI_CHECK(l >= 1 && l <= 1024, "ssi_cov_stream_create: l=%d out of range [1, 1024]", l);
  SSI_CHECK(max_lag >= 1, "ssi_cov_stream_create: need max_lag >= 1");
  SSI_CHECK(max_block >= 1 && window >= (int64_t)max_lag + 1,
            "ssi_cov_stream_create: need max_block >= 1 and window > max_lag");
  SSI_CHECK(window + max_block < (1LL << 31) - 1024, "ssi_cov_stream_create: window too large");
  SSI_CHECK(prec == SSI_PREC_FP32 || prec == SSI_PREC_SPLIT_BF16, "ssi_cov_stream_create: bad precision");
  SSI_CUDA(cudaSetDevice(ctx->device));
  ssi_cov_stream* st = new ssi_cov_stream;
  st->ctx = ctx;
  st->l = l;
  st->K = max_lag;
  st->W = window;
  st->Bmax = max_block;
  st->C = window + max_block;
  st->prec = prec;
  st->bytes_ring = sizeof(float) * (size_t)l * st->C;
  st->bytes_seg = sizeof(float) * (size_t)l * (max_block + max_lag + 1 + max_lag + 1);
  st->bytes_S = sizeof(float2) * (size_t)max_lag * l * l;
  ssi_status rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->ring), st->bytes_ring);
  if (rc == SSI_OK) rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->seg), st->bytes_seg);
  if (rc == SSI_OK) rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->S), st->bytes_S);
  if (rc != SSI_OK) {
    stream_free(st);
    return rc;
  }
  *out = st;
  return SSI_OK;
}

extern "C" ssi_status ssi_cov_stream_push(ssi_cov_stream* st, const float* Y, int64_t B, void* stream) {
  using namespace ssi;
  SSI_CHECK(st && Y, "ssi_cov_stream_push: null pointer");
  SSI_CHECK(B >= 1 && B <= st->Bmax, "ssi_cov_stream_push: need 1 <= B <= max_block (%lld)",
            (long long)st->Bmax);
  SSI_CHECK(st->n > 0 || B >= (int64_t)st->K + 1,
            "ssi_cov_stream_push: the first block needs more than max_lag samples");
  SSI_CUDA(cudaSetDevice(st->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t T = (int64_t)st->K + 1;
  const int64_t e = st->start + st->n;   // absolute index of the first new sample
  // the block into the ring (the window occupies at most W of the W + B_max columns)
  int64_t done = 0;
  while (done < B) {
    const int64_t pos = (e + done) % st->C;
    const int64_t w = std::min(B - done, st->C - pos);
    SSI_CUDA(cudaMemcpy2DAsync(st->ring + pos, (size_t)st->C * sizeof(float), Y + done,
                               (size_t)B * sizeof(float), (size_t)w * sizeof(float), (size_t)st->l,
                               cudaMemcpyDeviceToDevice, s));
    done += w;
  }
  if (st->n == 0) {
    SSI_CUDA(cudaMemsetAsync(st->S, 0, st->bytes_S, s));
    SSI_TRY(segment_acc(st, e, B, 1.0, s));
  } else {
    // entering pairs: F([e-T, e+B)) - F([e-T, e)); n >= T since the first block
    SSI_TRY(segment_acc(st, e - T, T + B, 1.0, s));
    SSI_TRY(segment_acc(st, e - T, T, -1.0, s));
  }
  st->n += B;
  if (st->n > st->W) {
    // leaving pairs: F([s, s+D+T)) - F([s+D, s+D+T)); the window keeps W >= T samples
    const int64_t D = st->n - st->W;
    SSI_TRY(segment_acc(st, st->start, D + T, -1.0, s));
    SSI_TRY(segment_acc(st, st->start + D, T, 1.0, s));
    st->start += D;
    st->n = st->W;
  }
  return SSI_OK;
}

extern "C" ssi_status ssi_cov_stream_covariances(ssi_cov_stream* st, double* R, int64_t* n_samples,
                                                 void* stream) {
  using namespace ssi;
  SSI_CHECK(st && R, "ssi_cov_stream_covariances: null pointer");
  SSI_CHECK(st->n > st->K, "ssi_cov_stream_covariances: the window holds no more than max_lag samples");
  SSI_CUDA(cudaSetDevice(st->ctx->device));
  count_launches(st->ctx, 1);
  k_stream_normalise<<<dim3((unsigned)ceil_div(st->l, 8), (unsigned)st->K), 256, 0,
                       static_cast<cudaStream_t>(stream)>>>(st->S, st->l, st->n, R);
  SSI_CUDA(cudaGetLastError());
  if (n_samples) *n_samples = st->n;
  return SSI_OK;
}

extern "C" ssi_status ssi_cov_stream_destroy(ssi_cov_stream* st) {
  using namespace ssi;
  if (!st) return SSI_OK;
  SSI_CUDA(cudaSetDevice(st->ctx->device));
  SSI_CUDA(cudaDeviceSynchronize());
  stream_free(st);
  return SSI_OK;
}
