// Small SVD of the RSVD (Sec. 2.2: P = U~ Sigma V^T, Algorithm 1).
//
// With P^T = Q2 R2 (QR of the K x L_cols matrix's transpose), the left singular
// vectors of P are the right singular vectors of R2.  One-sided (Hestenes) Jacobi
// on B = R2^T: rotating the columns of B until they are mutually orthogonal gives
// B V = W Sigma, hence R2 = V Sigma W^T and U~ = W (the normalised columns of B),
// Sigma = their norms; V itself is never needed.
// One CTA of 512 threads; B is held column by column in shared memory when it fits,
// else in global memory.  Pairs follow the circle (round-robin) ordering, four pairs
// per warp (eight lanes each).  The column stride is = 8 (mod 32) floats, so the four
// groups of a warp, which hold consecutive pair indices, read distinct banks.  Sweeps stop when every pair satisfies
// |b_p^T b_q| <= tol ||b_p|| ||b_q|| or after max_sweeps (status bit set).
#include "common.cuh"

namespace ssi {

namespace {

constexpr int JT = 512;

__host__ __device__ inline int col_stride(int K) { return ((K + 23) / 32) * 32 + 8; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// B: column c of B at B + c*ldb (length K).  Output: Ut (K x K row-major, column j =
// singular vector of rank j), S (K, descending).
template <int RJ8>   // K <= 8 * RJ8
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
  const int KS = col_stride(K);
  for (int e = tid; e < K * K; e += JT) B[(e / K) * KS + e % K] = R2[e];
  __syncthreads();
  const int n_pad = K + (K & 1);
  const int half = n_pad / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < n_pad - 1; ++rnd) {
      // circle method: position 0 fixed, others rotate by rnd.  Eight lanes per pair
      // (four pairs per warp): short reductions, many pairs in flight per warp.
      const int g = lane >> 3, gl = lane & 7;
      const unsigned gmask = 0xFFu << (8 * g);
      // the loop bound depends on the warp only, so all 32 lanes run the same iterations
      // (the group reductions below shuffle across the whole warp)
      for (int base = warp * 4; base < half; base += nw * 4) {
        const int pi = base + g;
        const bool live = pi < half;
        int p = 0, q = 0;
        if (live) {
          // (x - 1 + rnd) mod (n_pad - 1) with both terms below the modulus: one subtraction
          const int a = pi, b = n_pad - 1 - pi, m1 = n_pad - 1;
          int va = a - 1 + rnd, vb = b - 1 + rnd;
          if (va >= m1) va -= m1;
          if (vb >= m1) vb -= m1;
          p = (a == 0) ? 0 : 1 + va;
          q = (b == 0) ? 0 : 1 + vb;
          if (p > q) { const int t = p; p = q; q = t; }
        }
        const bool act = live && p < K && q < K;
        float* bp = B + (size_t)p * KS;
        float* bq = B + (size_t)q * KS;
        float xv[RJ8], yv[RJ8];
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int t = 0; t < RJ8; ++t) {
          const int r = gl + 8 * t;
          xv[t] = (act && r < K) ? bp[r] : 0.f;
          yv[t] = (act && r < K) ? bq[r] : 0.f;
          al = fmaf(xv[t], xv[t], al);
          be = fmaf(yv[t], yv[t], be);
          ga = fmaf(xv[t], yv[t], ga);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        (void)gmask;
        if (act && fabsf(ga) > tol * sqrtf(al * be) && al > 0.f && be > 0.f) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + t * t);
          const float s = c * t;
#pragma unroll
          for (int u = 0; u < RJ8; ++u) {
            const int r = gl + 8 * u;
            if (r < K) {
              bp[r] = c * xv[u] - s * yv[u];
              bq[r] = s * xv[u] + c * yv[u];
            }
          }
          if (gl == 0) s_rot = 1;
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
    for (int r = lane; r < K; r += 32) s = fmaf(B[(size_t)c * KS + r], B[(size_t)c * KS + r], s);
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
    Ut[(size_t)r * K + s_rank[c]] = nv > 0.f ? B[(size_t)c * KS + r] / nv : 0.f;
  }
}

}  // namespace

constexpr size_t JACOBI_SMEM_MAX = 216 * 1024;

size_t jacobi_ws_bytes(int K) {
  WsPlan w;
  if ((size_t)K * col_stride(K) * sizeof(float) > JACOBI_SMEM_MAX) w.add<float>((size_t)K * col_stride(K));
  return w.bytes;
}

ssi_status jacobi_launch(Workspace& ws, const float* R2, int K, float* Ut, float* S, int* status,
                         cudaStream_t stream) {
  if (K > 512) {
    set_error("jacobi: K=%d > 512", K);
    return SSI_E_INVALID;
  }
  const size_t bytes = (size_t)K * col_stride(K) * sizeof(float);
  float* Bg = nullptr;
  size_t smem = 0;
  if (bytes > JACOBI_SMEM_MAX) {
    Bg = ws.take<float>((size_t)K * col_stride(K));
    if (!Bg) {
      set_error("jacobi: workspace too small");
      return SSI_E_NOMEM;
    }
  } else {
    smem = bytes;
    SSI_CUDA(cudaFuncSetAttribute(k_jacobi_svd<29>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)JACOBI_SMEM_MAX));
  }
  if (K <= 232)
    k_jacobi_svd<29><<<1, JT, smem, stream>>>(R2, K, Bg, 1e-5f, 30, Ut, S, status);
  else
    k_jacobi_svd<64><<<1, JT, smem, stream>>>(R2, K, Bg, 1e-5f, 30, Ut, S, status);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace ssi
