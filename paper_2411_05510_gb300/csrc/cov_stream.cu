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
// Samples live in a device ring of W + B_max columns per channel.  A segment that lies in
// one piece of the ring is read in place (the stage (a) kernels take a channel stride);
// one that wraps is gathered into a contiguous buffer by 2D copies.
//
// Rounding: each update adds and subtracts segment sums whose rounding errors do not
// cancel, so the error of S would grow with the number of updates.  Every W samples
// pushed (and on ssi_cov_stream_refresh) S is therefore rebuilt from the window held in
// the ring, which resets it to the error of one whole-window computation.
//
// The workspace is reserved at creation for the largest segment and for a whole window,
// so a push or a rebuild never grows it; a push that fails part way (a CUDA error) leaves
// the object marked inconsistent, and every later call but destroy is refused.
#include "common.cuh"

#include <algorithm>

struct ssi_cov_stream {
  ssi_ctx* ctx = nullptr;
  int l = 0, K = 0;
  int64_t W = 0, Bmax = 0, C = 0;
  ssi_precision prec = SSI_PREC_SPLIT_BF16;
  float* ring = nullptr;      // l x C
  float* seg = nullptr;       // l x seg_cap, seg_cap = Bmax + 2 (K + 1)
  float2* S = nullptr;        // K x l x l lag sums, double-float (hi, lo)
  int64_t start = 0, n = 0;   // absolute index of the window's first sample; samples held
  int64_t since_rebuild = 0;  // samples pushed since S was last rebuilt from the ring
  int64_t seg_cap = 0;        // columns of the gather buffer
  bool broken = false;        // a push or rebuild failed part way: S no longer matches the window
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

// S += sign * F(Y), Y an l x len record with channel stride ldy (len > max_lag).
ssi_status lag_sums_acc(ssi_cov_stream* st, const float* Y, int64_t len, int64_t ldy, double sign,
                        cudaStream_t s) {
  ssi_ctx* ctx = st->ctx;
  CovPlan plan = cov_plan(st->l, len, st->K, st->prec, ctx->num_sms, st->ws.cap);
  if (plan.ws_bytes > st->ws.cap) {
    set_error("cov_stream: a segment of %lld samples needs more than the reserved workspace",
              (long long)len);
    return SSI_E_NOMEM;
  }
  plan.ldy = ldy;
  st->ws.reset();
  return covariances_ws(ctx, st->ws, plan, Y, st->prec, nullptr, ctx->dev_status, s, (float)sign,
                        st->S);
}

// S += sign * F(absolute samples [a, a + len)): in place when the segment does not wrap,
// else gathered (len <= seg_cap).
ssi_status segment_acc(ssi_cov_stream* st, int64_t a, int64_t len, double sign, cudaStream_t s) {
  const int64_t pos = a % st->C;
  if (pos + len <= st->C) return lag_sums_acc(st, st->ring + pos, len, st->C, sign, s);
  SSI_TRY(ring_gather(st, a, len, st->seg, s));
  return lag_sums_acc(st, st->seg, len, len, sign, s);
}

// S = F(window), from the samples in the ring.  A window that wraps around the ring is
// A (older, to the ring's end) followed by B (from column 0): F(A B) = F(A) + F(B) + the
// pairs across the seam, which are F(a B') - F(a) - F(B') for a = the last T samples of A
// and B' = the first T of B (every pair spans at most K < T samples); a piece shorter
// than T is taken whole into the gathered seam segment instead.  Every segment is longer
// than max_lag.
ssi_status rebuild(ssi_cov_stream* st, cudaStream_t s) {
  const int64_t T = (int64_t)st->K + 1;
  const int64_t a0 = st->start, n = st->n, pos = a0 % st->C;
  st->since_rebuild = 0;
  SSI_CUDA(cudaMemsetAsync(st->S, 0, st->bytes_S, s));
  if (pos + n <= st->C) return lag_sums_acc(st, st->ring + pos, n, st->C, 1.0, s);
  if (n <= st->seg_cap) return segment_acc(st, a0, n, 1.0, s);
  const int64_t lenA = st->C - pos, lenB = n - lenA;
  const int64_t seam = a0 + lenA;   // absolute index of B's first sample
  const int64_t ta = std::min(lenA, T), tb = std::min(lenB, T);
  if (lenA >= T) SSI_TRY(segment_acc(st, a0, lenA, 1.0, s));
  if (lenB >= T) SSI_TRY(segment_acc(st, seam, lenB, 1.0, s));
  // the seam segment: (a or all of A) followed by (B' or all of B)
  SSI_TRY(segment_acc(st, seam - ta, ta + tb, 1.0, s));
  if (lenA >= T) SSI_TRY(segment_acc(st, seam - ta, ta, -1.0, s));
  if (lenB >= T) SSI_TRY(segment_acc(st, seam, tb, -1.0, s));
  st->since_rebuild = 0;
  return SSI_OK;
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
  st->seg_cap = max_block + 2 * ((int64_t)max_lag + 1);
  st->bytes_seg = sizeof(float) * (size_t)l * st->seg_cap;
  st->bytes_S = sizeof(float2) * (size_t)max_lag * l * l;
  ssi_status rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->ring), st->bytes_ring);
  if (rc == SSI_OK) rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->seg), st->bytes_seg);
  if (rc == SSI_OK) rc = ctx_alloc(ctx, reinterpret_cast<void**>(&st->S), st->bytes_S);
  if (rc == SSI_OK) {
    // the workspace of the largest segment of a push and of a whole window, reserved now
    // so that no push or rebuild has to grow it (segments in between fit by the planner)
    const int64_t T = (int64_t)max_lag + 1;
    size_t cap = 0;
    for (int64_t len : {T, max_block + T, st->seg_cap, window})
      cap = std::max(cap, cov_plan(l, len, max_lag, prec, ctx->num_sms).ws_bytes);
    rc = ws_reserve(ctx, st->ws, cap, nullptr);
  }
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
  SSI_CHECK(!st->broken, "ssi_cov_stream_push: the stream is inconsistent after a failed call");
  SSI_CUDA(cudaSetDevice(st->ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st->broken = true;   // until every step below has been enqueued
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
  st->since_rebuild += B;
  if (st->since_rebuild >= st->W) SSI_TRY(rebuild(st, s));
  st->broken = false;
  return SSI_OK;
}

extern "C" ssi_status ssi_cov_stream_refresh(ssi_cov_stream* st, void* stream) {
  using namespace ssi;
  SSI_CHECK(st, "ssi_cov_stream_refresh: null pointer");
  SSI_CHECK(!st->broken, "ssi_cov_stream_refresh: the stream is inconsistent after a failed call");
  SSI_CHECK(st->n > st->K, "ssi_cov_stream_refresh: the window holds no more than max_lag samples");
  SSI_CUDA(cudaSetDevice(st->ctx->device));
  st->broken = true;
  SSI_TRY(rebuild(st, static_cast<cudaStream_t>(stream)));
  st->broken = false;
  return SSI_OK;
}

extern "C" ssi_status ssi_cov_stream_covariances(ssi_cov_stream* st, double* R, int64_t* n_samples,
                                                 void* stream) {
  using namespace ssi;
  SSI_CHECK(st && R, "ssi_cov_stream_covariances: null pointer");
  SSI_CHECK(!st->broken, "ssi_cov_stream_covariances: the stream is inconsistent after a failed call");
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
