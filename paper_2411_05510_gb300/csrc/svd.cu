// Small SVD of the RSVD (Sec. 2.2: "P = U~ Sigma V^T", Algorithm 1 line 5).
//
// With P^T = Q2 R2 (QR of the K x L_cols matrix's transpose), the left singular
// vectors of P are the right singular vectors of R2.  One-sided (Hestenes) Jacobi
// on B = R2^T: rotating the columns of B until they are mutually orthogonal gives
// B V = W Sigma, hence R2 = V Sigma W^T and U~ = W (the normalised columns of B),
// Sigma = their norms; V itself is never needed.
// One CTA of 1024 threads; B is held column by column in shared memory when
// K^2 floats fit, else in global memory.  Pairs follow the circle (round-robin)
// ordering, one pair per warp at a time.  Sweeps stop when every pair satisfies
// |b_p^T b_q| <= tol ||b_p|| ||b_q|| or after max_sweeps (status bit set).
#include "common.cuh"

namespace ssi {

namespace {

constexpr int JT = 1024;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// B: column c of B at B + c*ldb (length K).  Output: Ut (K x K row-major, column j =
// singular vector of rank j), S (K, descending).
__global__ void __launch_bounds__(JT, 1)
    k_jacobi_svd(const float* __restrict__ R2, int K, float* __restrict__ Bglobal, float tol,
                 int max_sweeps, float* __restrict__ Ut, float* __restrict__ Sout, int* status) {
  extern __shared__ float smem_f[];
  const bool in_smem = Bglobal == nullptr;
  float* B = in_smem ? smem_f : Bglobal;
  __shared__ float s_norm[512];
  __shared__ int s_rank[512];
  __shared__ int s_rot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = JT / 32;
  // B = R2^T: column c of B is row c of R2
  for (int e = tid; e < K * K; e += JT) B[e] = R2[e];
  __syncthreads();
  const int n_pad = K + (K & 1);
  const int half = n_pad / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < n_pad - 1; ++rnd) {
      // circle method: position 0 fixed, others rotate by rnd
      for (int pi = warp; pi < half; pi += nw) {
        int a = pi, b = n_pad - 1 - pi;
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + rnd) % (n_pad - 1); };
        int p = pos(a), q = pos(b);
        if (p >= K || q >= K) continue;
        if (p > q) { int t = p; p = q; q = t; }
        float* bp = B + (size_t)p * K;
        float* bq = B + (size_t)q * K;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int r = lane; r < K; r += 32) {
          const float x = bp[r], y = bq[r];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (fabsf(ga) > tol * sqrtf(al * be) && al > 0.f && be > 0.f) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t);
          const float s = c * t;
          for (int r = lane; r < K; r += 32) {
            const float x = bp[r], y = bq[r];
            bp[r] = c * x - s * y;
            bq[r] = s * x + c * y;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  if (sweep == max_sweeps && tid == 0) atomicOr(status, DEV_NOTCONVERGED);
  // norms and ranks
  for (int c = warp; c < K; c += nw) {
    float s = 0.f;
    for (int r = lane; r < K; r += 32) s = fmaf(B[(size_t)c * K + r], B[(size_t)c * K + r], s);
    s = warp_sum(s);
    if (lane == 0) s_norm[c] = sqrtf(s);
  }
  __syncthreads();
  for (int c = tid; c < K; c += JT) {
    int rank = 0;
    const float v = s_norm[c];
    for (int d = 0; d < K; ++d) {
      const float u = s_norm[d];
      rank += (u > v) || (u == v && d < c);
    }
    s_rank[c] = rank;
    Sout[rank] = v;
  }
  __syncthreads();
  for (int e = tid; e < K * K; e += JT) {
    const int c = e / K, r = e % K;
    const float nv = s_norm[c];
    Ut[(size_t)r * K + s_rank[c]] = nv > 0.f ? B[(size_t)c * K + r] / nv : 0.f;
  }
}

}  // namespace

size_t jacobi_ws_bytes(int K) {
  WsPlan w;
  if ((size_t)K * K * sizeof(float) > 200 * 1024) w.add<float>((size_t)K * K);
  return w.bytes;
}

ssi_status jacobi_launch(Workspace& ws, const float* R2, int K, float* Ut, float* S, int* status,
                         cudaStream_t stream) {
  if (K > 512) {
    set_error("jacobi: K=%d > 512", K);
    return SSI_E_INVALID;
  }
  const size_t bytes = (size_t)K * K * sizeof(float);
  float* Bg = nullptr;
  size_t smem = 0;
  if (bytes > 200 * 1024) {
    Bg = ws.take<float>((size_t)K * K);
    if (!Bg) {
      set_error("jacobi: workspace too small");
      return SSI_E_NOMEM;
    }
  } else {
    smem = bytes;
    SSI_CUDA(cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(200 * 1024)));
  }
  k_jacobi_svd<<<1, JT, smem, stream>>>(R2, K, Bg, 2e-6f, 30, Ut, S, status);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace ssi
