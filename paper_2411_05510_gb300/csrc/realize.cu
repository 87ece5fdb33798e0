// Stage (c): realisation of every (lag, order) of a stabilization diagram (Sec. 2.1).
//
// Paper: O = U S^{1/2}, C = O[:l], A = (O^to)^+ O^bo, A = Psi M Psi^{-1},
// lambda = ln(mu)/dt, f = |lambda|/(2 pi), xi = -Re(lambda)/|lambda|, Phi = C Psi.
//
// GPU formulation (same results, better conditioned):
//   * S^{1/2} is a similarity transform of A, so A~_n = (U^to_n)^+ U^bo_n has the same
//     eigenvalues and Phi = U[:l, :n] Psi~.  U^to has nearly orthonormal columns, so the
//     normal equations are well conditioned in FP32.
//   * Nested orders: with G = U^to^T U^to = R^T R (Cholesky) and H = U^to^T U^bo,
//     A~_n = (R^{-1})[:n,:n] (R^{-T} H)[:n,:n] for every order n, so one k x k
//     factorisation per lag serves all orders.
// Kernels:
//   k_gram_gh     split-row partial sums of G and H (FP32 within a chunk)
//   k_gram_reduce FP64 sum of the chunks
//   k_lag_factor  one CTA per lag: Cholesky of G, R^{-1}, M = R^{-T} H
//   k_eig         one CTA per (lag, order): A~_n in shared memory, Householder
//                 Hessenberg reduction, Francis double-shift QR to real Schur form
//                 (iteration cap 30 n, status flag when hit), complex eigenvectors
//                 by back substitution on the quasi-triangular factor, back
//                 transformation through the logged reflectors, Phi = U[:l,:n] Psi~,
//                 pole parameters, MPC and MPD.  Largest orders are scheduled first.
#include <cfloat>

#include "common.cuh"

namespace ssi {

namespace {

constexpr int MAX_LAGS = 64;
constexpr int EIG_THREADS = 256;
constexpr int GR_ROWS = 512;      // rows per Gram chunk
constexpr int SMEM_N_MAX = 224;   // largest order whose A fits shared memory

constexpr int WN = 32;                       // window of the bulge chase
constexpr int WB = WN - 3;                   // bulge steps per window
__device__ __forceinline__ int warp_id_of(int tid) { return tid >> 5; }   // reflectors staged per chunk in the back transformation

struct LagTable {
  int n_lags;
  int l, k;
  int i[MAX_LAGS];
  const float* U[MAX_LAGS];
};

// ------------------------------------------------------------------ Gram matrices
// partial[t][chunk][which][a][b], which 0: G = sum_r U[r][a] U[r][b], 1: H = sum_r U[r][a] U[r+l][b],
// r in the chunk, r < L - l.
__global__ void __launch_bounds__(256)
    k_gram_gh(LagTable lt, int n_chunks, float* __restrict__ partial) {
  __shared__ float As[32][64 + 4];
  __shared__ float Bs[32][64 + 4];
  const int k = lt.k, l = lt.l;
  const int tiles = (k + 63) / 64;
  const int ta = blockIdx.x / tiles, tb = blockIdx.x % tiles;
  const int chunk = blockIdx.y;
  const int t = blockIdx.z >> 1, which = blockIdx.z & 1;
  const int L = l * lt.i[t];
  const int r_end_all = L - l;
  const int r0 = chunk * GR_ROWS;
  const int r1 = min(r_end_all, r0 + GR_ROWS);
  const float* U = lt.U[t];
  const int a0 = ta * 64, b0 = tb * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  const int shift = which ? l : 0;
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int rr = e / 64, c = e % 64;
      const int r = rb + rr;
      const bool in = r < r1;
      As[rr][c] = (in && a0 + c < k) ? U[(size_t)r * k + a0 + c] : 0.f;
      Bs[rr][c] = (in && b0 + c < k) ? U[(size_t)(r + shift) * k + b0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) { a[x] = As[rr][ty * 4 + x]; b[x] = Bs[rr][tx * 4 + x]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  float* out = partial + ((((size_t)t * n_chunks + chunk) * 2 + which) * k) * k;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int a = a0 + ty * 4 + x, b = b0 + tx * 4 + y;
      if (a < k && b < k) out[(size_t)a * k + b] = acc[x][y];
    }
}

__global__ void k_gram_reduce(const float* __restrict__ partial, int n_lags, int n_chunks, int k,
                              float* __restrict__ GH) {
  const long long per = 2LL * k * k;
  const long long total = (long long)n_lags * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / per);
    const long long w = e % per;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += (double)partial[((size_t)t * n_chunks + c) * per + w];
    GH[e] = (float)s;
  }
}

// ------------------------------------------------------------------ per-lag factorisation
// GH[t] = [G | H] (2 x k x k); out RM[t] = [Rinv | M] (2 x k x k).
__global__ void __launch_bounds__(1024)
    k_lag_factor(const float* __restrict__ GH, int k, float* __restrict__ RM, int* status) {
  extern __shared__ float sR[];   // k x k, Cholesky factor (upper)
  const int t = blockIdx.x;
  const float* G = GH + (size_t)t * 2 * k * k;
  const float* H = G + (size_t)k * k;
  float* Rinv = RM + (size_t)t * 2 * k * k;
  float* M = Rinv + (size_t)k * k;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int e = tid; e < k * k; e += nth) sR[e] = G[e];
  __syncthreads();
  __shared__ float s_d;
  float gmax = 0.f;
  for (int j = 0; j < k; ++j) gmax = fmaxf(gmax, G[(size_t)j * k + j]);
  const float floor_v = fmaxf(gmax * 1e-10f, FLT_MIN);
  // right-looking Cholesky on the upper triangle: row j of R
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      float d = sR[j * k + j];
      if (!(d > floor_v)) {
        atomicOr(status, DEV_NOTCONVERGED);
        d = floor_v;
      }
      s_d = sqrtf(d);
      sR[j * k + j] = s_d;
    }
    __syncthreads();
    const float d = s_d;
    for (int c = j + 1 + tid; c < k; c += nth) sR[j * k + c] /= d;
    __syncthreads();
    // trailing update of the upper triangle: G[a][c] -= R[j][a] R[j][c], j < a <= c
    const int m = k - j - 1;
    for (int e = tid; e < m * m; e += nth) {
      const int a = j + 1 + e / m, c = j + 1 + e % m;
      if (c >= a) sR[a * k + c] -= sR[j * k + a] * sR[j * k + c];
    }
    __syncthreads();
  }
  // Rinv by column back substitution and M = R^{-T} H by forward substitution; one warp
  // per column, the column held in registers across the lanes (entry j on lane j % 32)
  const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
  constexpr int KJ = 8;   // k <= 256
  for (int c = warp; c < k; c += nwarps) {
    float x[KJ];
#pragma unroll
    for (int q = 0; q < KJ; ++q) x[q] = 0.f;
    for (int r = c; r >= 0; --r) {
      float part = 0.f;
#pragma unroll
      for (int q = 0; q < KJ; ++q) {
        const int j = lane + 32 * q;
        if (j > r && j <= c) part = fmaf(sR[r * k + j], x[q], part);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const float v = ((r == c) ? 1.f - part : -part) / sR[r * k + r];
      if (lane == (r & 31)) x[r >> 5] = v;
    }
#pragma unroll
    for (int q = 0; q < KJ; ++q) {
      const int j = lane + 32 * q;
      if (j < k) Rinv[(size_t)j * k + c] = (j <= c) ? x[q] : 0.f;
    }
  }
  for (int c = warp; c < k; c += nwarps) {
    float x[KJ];
#pragma unroll
    for (int q = 0; q < KJ; ++q) x[q] = 0.f;
    for (int r = 0; r < k; ++r) {
      float part = 0.f;
#pragma unroll
      for (int q = 0; q < KJ; ++q) {
        const int j = lane + 32 * q;
        if (j < r) part = fmaf(sR[j * k + r], x[q], part);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const float v = (H[(size_t)r * k + c] - part) / sR[r * k + r];
      if (lane == (r & 31)) x[r >> 5] = v;
    }
#pragma unroll
    for (int q = 0; q < KJ; ++q) {
      const int j = lane + 32 * q;
      if (j < k) M[(size_t)j * k + c] = x[q];
    }
  }
}

// ------------------------------------------------------------------ eig per realisation
struct EigParams {
  LagTable lt;
  int n_orders;
  int orders[512];
  long long slot_off[512];   // offset of order m's first pole slot within a lag
  long long slots_per_lag;
  const float* RM;           // [t][2][k][k]
  float* work;               // per-realisation scratch
  long long work_off[512];   // offset of order m's scratch within a lag's scratch
  long long work_per_lag;
  int xbuf_off;              // floats: start of the per-warp eigenvector buffers in shared memory
  int log_off;               // floats: start of the reflector staging buffer in shared memory
  int nmax;                  // largest order of the launch
  double dt;
  ssi_pole* poles;
  float* phi;
  int* status;
};

// scratch of one realisation of order n: Hessenberg v's (n*n), reflector log, X (n*n)
// scratch of one realisation of order n: Hessenberg reflectors (n*n), the log of window
// transformations (zlog_cap(n) entries of ZREC floats), eigenvector matrix X (n*n)
constexpr int ZREC = 32 * 32 + 8;   // one window: b, e, then the 32 x 32 factor row-major
__host__ __device__ inline long long zlog_cap(int n) { return (long long)n * n / 16 + 2LL * n + 64; }
__host__ __device__ inline long long eig_work_floats(int n, int) {
  return (long long)n * n + zlog_cap(n) * ZREC + (long long)n * n + 64;
}

__device__ __forceinline__ float sgnf(float a, float b) { return b >= 0.f ? fabsf(a) : -fabsf(a); }

__global__ void __launch_bounds__(EIG_THREADS)
    k_eig(EigParams p) {
  extern __shared__ float smem[];
  // work item: largest orders first
  const int item = blockIdx.x;
  const int mi = p.n_orders - 1 - (item / p.lt.n_lags);
  const int t = item % p.lt.n_lags;
  const int n = p.orders[mi];
  const int k = p.lt.k, l = p.lt.l;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ld = n + 1;   // padded leading dimension against bank conflicts
  float* work = p.work + (size_t)t * p.work_per_lag + p.work_off[mi];
  float* hv = work;                           // Hessenberg reflectors: n x n (v, beta in [j*n + n-1])
  float* zlog = hv + (size_t)n * n;           // window transformations of the QR sweeps
  float* X = zlog + zlog_cap(n) * ZREC;       // eigenvector matrix, n x (2 m)
  float* A = smem;                            // n x (n+1), orders <= SMEM_N_MAX
  __shared__ float sh[16];
  __shared__ int shi[16];
  __shared__ int s_pos[256];                  // position p of the 2x2 block of pole j
  __shared__ float s_mur[256], s_mui[256];
  const float* Rinv = p.RM + (size_t)t * 2 * k * k;
  const float* M = Rinv + (size_t)k * k;
  const float* U = p.lt.U[t];
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  float* phi_out = p.phi + ((size_t)t * p.slots_per_lag + p.slot_off[mi]) * 2 * l;
  const int n_slots = n / 2;

  // ---- 1. A~_n = Rinv[:n,:n] M[:n,:n] (Rinv upper triangular); 1 x 4 strips per thread
  {
    const int n4 = (n + 3) / 4;
    for (int e = tid; e < n * n4; e += nth) {
      const int r = e / n4, c0 = (e % n4) * 4;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      const float* rrow = Rinv + (size_t)r * k;
      for (int j = r; j < n; ++j) {
        const float a = rrow[j];
        const float* mrow = M + (size_t)j * k + c0;
        s0 = fmaf(a, mrow[0], s0);
        if (c0 + 1 < n) s1 = fmaf(a, mrow[1], s1);
        if (c0 + 2 < n) s2 = fmaf(a, mrow[2], s2);
        if (c0 + 3 < n) s3 = fmaf(a, mrow[3], s3);
      }
      A[r * ld + c0] = s0;
      if (c0 + 1 < n) A[r * ld + c0 + 1] = s1;
      if (c0 + 2 < n) A[r * ld + c0 + 2] = s2;
      if (c0 + 3 < n) A[r * ld + c0 + 3] = s3;
    }
  }
  __syncthreads();

  // ---- 2. Householder reduction to upper Hessenberg form (v kept in shared memory and
  //         logged to global memory for the back transformation)
  float* sv = smem + p.xbuf_off;   // n floats (the eigenvector buffers are not in use yet)
  __shared__ float s_part[EIG_THREADS / 32];
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    float* v = hv + (size_t)j * n;
    float ss = 0.f;
    for (int r = tid; r < len; r += nth) {
      const float x = A[(j + 1 + r) * ld + j];
      ss = fmaf(x, x, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) s_part[tid >> 5] = ss;
    __syncthreads();
    if (tid == 0) {
      float tot = 0.f;
      for (int w2 = 0; w2 < nth / 32; ++w2) tot += s_part[w2];
      const float x0 = A[(j + 1) * ld + j];
      const float nx = sqrtf(tot);
      const float alpha = x0 >= 0.f ? -nx : nx;
      const float vv = tot - x0 * x0 + (x0 - alpha) * (x0 - alpha);
      sh[0] = alpha;
      sh[1] = (nx > 0.f && vv > 0.f) ? 2.f / vv : 0.f;
      sh[2] = x0 - alpha;
    }
    __syncthreads();
    const float beta = sh[1];
    for (int r = tid; r < len; r += nth) {
      const float vr = (r == 0) ? sh[2] : A[(j + 1 + r) * ld + j];
      sv[r] = vr;
      v[r] = vr;
    }
    if (tid == 0) v[n - 1] = beta;   // v has len <= n-2 entries; beta stored at the end
    __syncthreads();
    if (beta != 0.f) {
      float* __restrict__ Ar = A;
      const float* __restrict__ vr = sv;
      // left: A[j+1:, c] -= beta v (v^T A[j+1:, c]) for c > j (column j is set below)
      for (int c = j + 1 + tid; c < n; c += nth) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int r = 0;
        for (; r + 3 < len; r += 4) {
          s0 = fmaf(vr[r], Ar[(j + 1 + r) * ld + c], s0);
          s1 = fmaf(vr[r + 1], Ar[(j + 2 + r) * ld + c], s1);
          s2 = fmaf(vr[r + 2], Ar[(j + 3 + r) * ld + c], s2);
          s3 = fmaf(vr[r + 3], Ar[(j + 4 + r) * ld + c], s3);
        }
        for (; r < len; ++r) s0 = fmaf(vr[r], Ar[(j + 1 + r) * ld + c], s0);
        const float sc = (s0 + s1 + s2 + s3) * beta;
#pragma unroll 4
        for (r = 0; r < len; ++r) Ar[(j + 1 + r) * ld + c] -= sc * vr[r];
      }
      __syncthreads();
      // right: A[r, j+1:] -= beta (A[r, j+1:] v) v^T for all rows
      for (int r = tid; r < n; r += nth) {
        float* __restrict__ row = Ar + r * ld + j + 1;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int c = 0;
        for (; c + 3 < len; c += 4) {
          s0 = fmaf(row[c], vr[c], s0);
          s1 = fmaf(row[c + 1], vr[c + 1], s1);
          s2 = fmaf(row[c + 2], vr[c + 2], s2);
          s3 = fmaf(row[c + 3], vr[c + 3], s3);
        }
        for (; c < len; ++c) s0 = fmaf(row[c], vr[c], s0);
        const float sc = (s0 + s1 + s2 + s3) * beta;
#pragma unroll 4
        for (c = 0; c < len; ++c) row[c] -= sc * vr[c];
      }
      __syncthreads();
      for (int r = 1 + tid; r <= len; r += nth) A[(j + r) * ld + j] = (r == 1) ? sh[0] : 0.f;
    }
    __syncthreads();
  }

  // ---- 3b. Francis double-shift QR to real Schur form (full T), windowed.
  //  The bulge of each sweep is chased by warp 0 inside a window of WN rows/columns;
  //  in-window rows and columns are updated at once and the window's transformations
  //  accumulate in Zb (WN x WN).  After each window all threads apply Zb to the rows
  //  right of the window (H[b:e, e:n] = Zb^T H[b:e, e:n]) and to the rows above it
  //  (H[0:b, b:e] = H[0:b, b:e] Zb), and Zb is logged for the back transformation of
  //  the eigenvectors.  Same arithmetic as the unwindowed sweep.
  float* Zbuf = smem + p.log_off;     // 2 buffers of WN x (WN + 4) (16-byte aligned rows)
  __shared__ int s_ctl[8];            // 0 b, 1 e, 2 kend, 3 state (0 run, 1 done, 2 failed), 4 pending buf, 5 pb, 6 pe
  __shared__ float s_sh[3];           // shift vector of the first step of the sweep
  if (tid == 0) {
    s_ctl[3] = 0;
    s_ctl[4] = -1;
    s_ctl[7] = 0;   // windows logged
  }
  __syncthreads();
  {
    // warp-0 state (identical in every lane)
    float anorm = 0.f;
    int nn = n - 1, its = 0, total_its = 0, ll = 0, m = 0, b = 0, fail = 0, blk = 0;
    bool in_sweep = false;
    if (warp_id_of(tid) == 0) {
      for (int e2 = tid; e2 < n * n; e2 += 32) {
        const int r = e2 / n, c = e2 % n;
        if (c >= r - 1) anorm += fabsf(A[r * ld + c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) anorm += __shfl_xor_sync(0xffffffffu, anorm, o);
    }
    const int itmax = 30 * max(10, n);
    while (true) {
      const int cur = blk & 1;
      float* Zb = Zbuf + cur * WN * (WN + 4);
      if (tid < 32) {
        const int lane0 = tid;
        // start a sweep when none is running: deflation and shift selection
        while (!in_sweep && nn >= 0 && !fail) {
          int l2 = 0;
          for (int base = nn; base >= 1; base -= 32) {
            const int cand = base - lane0;
            bool small = false;
            if (cand >= 1) {
              float sd = fabsf(A[(cand - 1) * ld + cand - 1]) + fabsf(A[cand * ld + cand]);
              if (sd == 0.f) sd = anorm;
              small = fabsf(A[cand * ld + cand - 1]) <= FLT_EPSILON * sd;
            }
            const unsigned msk = __ballot_sync(0xffffffffu, small);
            if (msk) {
              l2 = base - (__ffs(msk) - 1);
              break;
            }
          }
          __syncwarp();
          if (l2 >= 1 && lane0 == 0) A[l2 * ld + l2 - 1] = 0.f;
          __syncwarp();
          if (l2 == nn) { nn -= 1; its = 0; continue; }
          if (l2 == nn - 1) { nn -= 2; its = 0; continue; }
          if (total_its >= itmax) { fail = 1; break; }
          float x = A[nn * ld + nn], y = A[(nn - 1) * ld + nn - 1];
          float w = A[nn * ld + nn - 1] * A[(nn - 1) * ld + nn];
          if (its == 10 || its == 20) {
            const float s = fabsf(A[nn * ld + nn - 1]) + fabsf(A[(nn - 1) * ld + nn - 2]);
            x = y = 0.75f * s;
            w = -0.4375f * s * s;
          }
          ++its;
          ++total_its;
          // start of the bulge: the largest mm in [l2, nn-2] where two consecutive
          // subdiagonals are negligible relative to the shift vector (mm = l2 always
          // qualifies); lanes test 32 candidates at a time
          int mm = l2;
          for (int base = nn - 2; base >= l2; base -= 32) {
            const int cand = base - lane0;
            bool ok = false;
            if (cand >= l2) {
              if (cand == l2) {
                ok = true;
              } else {
                const float z = A[cand * ld + cand];
                const float r2 = x - z, s2 = y - z;
                float p0 = (r2 * s2 - w) / A[(cand + 1) * ld + cand] + A[cand * ld + cand + 1];
                float q0 = A[(cand + 1) * ld + cand + 1] - z - r2 - s2;
                float r0 = A[(cand + 2) * ld + cand + 1];
                const float sc = fabsf(p0) + fabsf(q0) + fabsf(r0);
                p0 /= sc; q0 /= sc; r0 /= sc;
                const float u = fabsf(A[cand * ld + cand - 1]) * (fabsf(q0) + fabsf(r0));
                const float v = fabsf(p0) * (fabsf(A[(cand - 1) * ld + cand - 1]) + fabsf(z) +
                                             fabsf(A[(cand + 1) * ld + cand + 1]));
                ok = u <= FLT_EPSILON * v;
              }
            }
            const unsigned msk = __ballot_sync(0xffffffffu, ok);
            if (msk) {
              mm = base - (__ffs(msk) - 1);
              break;
            }
          }
          float pp, qq, rr;
          {
            const float z = A[mm * ld + mm];
            const float r2 = x - z, s2 = y - z;
            pp = (r2 * s2 - w) / A[(mm + 1) * ld + mm] + A[mm * ld + mm + 1];
            qq = A[(mm + 1) * ld + mm + 1] - z - r2 - s2;
            rr = A[(mm + 2) * ld + mm + 1];
            const float sc = fabsf(pp) + fabsf(qq) + fabsf(rr);
            pp /= sc; qq /= sc; rr /= sc;
          }
          __syncwarp();
          for (int r = mm + 2 + lane0; r <= nn; r += 32) {
            A[r * ld + r - 2] = 0.f;
            if (r != mm + 2) A[r * ld + r - 3] = 0.f;
          }
          __syncwarp();
          ll = l2;
          m = mm;
          b = mm;
          if (lane0 == 0) { s_sh[0] = pp; s_sh[1] = qq; s_sh[2] = rr; }
          in_sweep = true;
        }
        __syncwarp();
        if (lane0 == 0) {
          if (fail) s_ctl[3] = 2;
          else if (!in_sweep) s_ctl[3] = 1;
        }
        if (in_sweep) {
          // ---- chase one window: steps kk in [b, kend), window [b, e)
          const int kend = min(b + WB, nn);
          const int e = min(b + WN, n);
          const int w = e - b;
          for (int q = 0; q < WN; ++q) Zb[lane0 * (WN + 4) + q] = (q == lane0) ? 1.f : 0.f;
          __syncwarp();
          for (int kk = b; kk < kend; ++kk) {
            const bool three = kk != nn - 1;
            float pp, qq, rr, xs = 1.f;
            bool go = true;
            if (kk == m) {
              pp = s_sh[0]; qq = s_sh[1]; rr = s_sh[2];
            } else {
              pp = A[kk * ld + kk - 1];
              qq = A[(kk + 1) * ld + kk - 1];
              rr = three ? A[(kk + 2) * ld + kk - 1] : 0.f;
              xs = fabsf(pp) + fabsf(qq) + fabsf(rr);
              if (xs != 0.f) {
                const float ix = __fdividef(1.f, xs);
                pp *= ix; qq *= ix; rr *= ix;
              } else {
                go = false;
              }
            }
            float s = 0.f, is = 0.f;
            if (go) {
              const float ss = pp * pp + qq * qq + rr * rr;
              go = ss > 0.f;
              if (go) {
                const float rs = rsqrtf(ss);
                s = sgnf(ss * rs, pp);
                is = sgnf(rs, pp);
              }
            }
            __syncwarp();
            if (go) {
              if (lane0 == 0) {
                if (kk == m) {
                  if (ll != m) A[kk * ld + kk - 1] = -A[kk * ld + kk - 1];
                } else {
                  A[kk * ld + kk - 1] = -s * xs;
                }
              }
              pp += s;
              const float ip = __fdividef(1.f, pp);
              const float w0 = pp * is, w1 = qq * is, w2 = three ? rr * is : 0.f;
              const float u1 = qq * ip, u2 = three ? rr * ip : 0.f;
              // row modification inside the window: columns kk .. e-1
              {
                const int j = b + lane0;
                if (j >= kk && j < e) {
                  const float a0 = A[kk * ld + j], a1 = A[(kk + 1) * ld + j];
                  const float a2 = three ? A[(kk + 2) * ld + j] : 0.f;
                  const float t = a0 + u1 * a1 + u2 * a2;
                  A[kk * ld + j] = a0 - t * w0;
                  A[(kk + 1) * ld + j] = a1 - t * w1;
                  if (three) A[(kk + 2) * ld + j] = a2 - t * w2;
                }
              }
              __syncwarp();
              // column modification inside the window: rows b .. min(nn, kk+3)
              {
                const int i2 = b + lane0;
                if (i2 <= min(nn, kk + 3)) {
                  const float b0 = A[i2 * ld + kk], b1 = A[i2 * ld + kk + 1];
                  const float b2 = three ? A[i2 * ld + kk + 2] : 0.f;
                  const float t = w0 * b0 + w1 * b1 + w2 * b2;
                  A[i2 * ld + kk] = b0 - t;
                  A[i2 * ld + kk + 1] = b1 - t * u1;
                  if (three) A[i2 * ld + kk + 2] = b2 - t * u2;
                }
                // the same transformation accumulated in Zb (window coordinates)
                const int kl = kk - b;
                float* zr = Zb + lane0 * (WN + 4);
                const float z0 = zr[kl], z1 = zr[kl + 1];
                const float z2 = three ? zr[kl + 2] : 0.f;
                const float t = w0 * z0 + w1 * z1 + w2 * z2;
                zr[kl] = z0 - t;
                zr[kl + 1] = z1 - t * u1;
                if (three) zr[kl + 2] = z2 - t * u2;
              }
            }
            __syncwarp();
          }
          if (lane0 == 0) {
            s_ctl[0] = b;
            s_ctl[1] = e;
            s_ctl[2] = kend;
          }
          b = kend;
          if (b > nn - 1) in_sweep = false;
          (void)w;
        }
        __syncwarp();
      }
      __syncthreads();
      const int state = s_ctl[3];
      if (state != 0) break;
      // ---- apply the window's Zb outside the window (all threads)
      {
        const int bb = s_ctl[0], ee = s_ctl[1], ww = ee - bb;
        float* ZT = Zbuf + (cur ^ 1) * WN * (WN + 4);   // the other buffer: Zb transposed, ld WN+4
        for (int e2 = tid; e2 < WN * WN; e2 += nth) {
          const int i2 = e2 / WN, j2 = e2 % WN;
          ZT[i2 * (WN + 4) + j2] = Zb[j2 * (WN + 4) + i2];
        }
        __syncthreads();
        const int n_right = n - ee;
        const int t = tid;
        if (t < n_right || t - n_right < bb) {
          const bool right = t < n_right;
          const int c = ee + t, r = t - n_right;
          float in[WN];
#pragma unroll
          for (int j2 = 0; j2 < WN; ++j2)
            in[j2] = (j2 < ww) ? (right ? A[(bb + j2) * ld + c] : A[r * ld + bb + j2]) : 0.f;
          // four outputs at a time: four independent accumulation chains
          for (int i0 = 0; i0 < ww; i0 += 4) {
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4* zt = reinterpret_cast<const float4*>(ZT + (i0 + u) * (WN + 4));
              float a = 0.f;
#pragma unroll
              for (int q4 = 0; q4 < WN / 4; ++q4) {
                const float4 z = zt[q4];
                a = fmaf(z.x, in[4 * q4], a);
                a = fmaf(z.y, in[4 * q4 + 1], a);
                a = fmaf(z.z, in[4 * q4 + 2], a);
                a = fmaf(z.w, in[4 * q4 + 3], a);
              }
              acc[u] = a;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (i0 + u < ww) {
                if (right) A[(bb + i0 + u) * ld + c] = acc[u];
                else A[r * ld + bb + i0 + u] = acc[u];
              }
            }
          }
        }
        // log the window: (b, e) and Zb
        const int widx = s_ctl[7];
        if (widx < zlog_cap(n)) {
          float* rec = zlog + (size_t)widx * ZREC;
          for (int e2 = tid; e2 < WN * WN; e2 += nth)
            rec[8 + e2] = Zb[(e2 / WN) * (WN + 4) + (e2 % WN)];
          if (tid == 0) {
            rec[0] = __int_as_float(bb);
            rec[1] = __int_as_float(ee);
          }
        }
        __syncthreads();
        if (tid == 0) s_ctl[7] = widx + 1;
      }
      __syncthreads();
      ++blk;
    }
    if (tid == 0) {
      shi[4] = (s_ctl[3] == 2 || s_ctl[7] > zlog_cap(n)) ? 1 : 0;
      shi[5] = min((long long)s_ctl[7], zlog_cap(n));
    }
    (void)total_its;
  }
  __syncthreads();
  const bool failed = shi[4] != 0;

  // ---- 4. complex eigenvalues (2x2 blocks), ranked by frequency
  __shared__ int s_npole;
  if (tid == 0) {
    int np = 0;
    if (!failed) {
      for (int r = 0; r + 1 < n;) {
        if (A[(r + 1) * ld + r] != 0.f) {
          const float a = A[r * ld + r], b = A[r * ld + r + 1];
          const float c = A[(r + 1) * ld + r], d = A[(r + 1) * ld + r + 1];
          const float hm = 0.5f * (a - d);
          const float disc = hm * hm + b * c;
          if (disc < 0.f && np < 256) {
            s_pos[np] = r;
            s_mur[np] = 0.5f * (a + d);
            s_mui[np] = sqrtf(-disc);
            ++np;
          }
          r += 2;
        } else {
          r += 1;
        }
      }
    }
    s_npole = np;
  }
  __syncthreads();
  const int npole = s_npole;
  // rank by |lambda| (frequency); ties by position
  __shared__ int s_rank[256];
  __shared__ float s_f[256];
  for (int j = tid; j < npole; j += nth) {
    const double mr = s_mur[j], mu_i = s_mui[j];
    const double lr = 0.5 * log(mr * mr + mu_i * mu_i) / p.dt, li = atan2(mu_i, mr) / p.dt;
    s_f[j] = (float)sqrt(lr * lr + li * li);
  }
  __syncthreads();
  for (int j = tid; j < npole; j += nth) {
    int rk = 0;
    for (int o = 0; o < npole; ++o) rk += (s_f[o] < s_f[j]) || (s_f[o] == s_f[j] && o < j);
    s_rank[j] = rk;
  }
  __syncthreads();

  // ---- 5. eigenvectors of the quasi-triangular T: one warp per eigenvalue, column 2*rank
  //         (real part) and 2*rank+1 (imaginary part) of X
  const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
  const int ncx = 2 * npole;   // columns of X
  float* xr = smem + p.xbuf_off + warp * 2 * p.nmax;   // this warp's vector (shared memory)
  float* xi = xr + p.nmax;
  for (int j = warp; j < npole; j += nwarps) {
    const int pos = s_pos[j];
    const float mr = s_mur[j], mu_i = s_mui[j];
    for (int r = lane; r < n; r += 32) { xr[r] = 0.f; xi[r] = 0.f; }
    __syncwarp();
    if (lane == 0) {
      // eigenvector of the 2x2 block: (b01, mu - b00)
      xr[pos] = A[pos * ld + pos + 1];
      xi[pos] = 0.f;
      xr[pos + 1] = mr - A[pos * ld + pos];
      xi[pos + 1] = mu_i;
    }
    __syncwarp();
    const float tiny = FLT_EPSILON * sh[8] + FLT_MIN;
    for (int r = pos - 1; r >= 0;) {
      const bool pair = (r >= 1) && A[r * ld + r - 1] != 0.f;
      const int top = pair ? r - 1 : r;
      // s_row = sum_{c > r} T[row][c] x[c], c up to pos+1, for row in {top, r}
      float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f;
      for (int c = r + 1 + lane; c <= pos + 1; c += 32) {
        const float vr = xr[c], vi = xi[c];
        const float t1 = A[r * ld + c];
        s1r = fmaf(t1, vr, s1r);
        s1i = fmaf(t1, vi, s1i);
        if (pair) {
          const float t0 = A[top * ld + c];
          s0r = fmaf(t0, vr, s0r);
          s0i = fmaf(t0, vi, s0i);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1r += __shfl_xor_sync(0xffffffffu, s1r, o);
        s1i += __shfl_xor_sync(0xffffffffu, s1i, o);
        s0r += __shfl_xor_sync(0xffffffffu, s0r, o);
        s0i += __shfl_xor_sync(0xffffffffu, s0i, o);
      }
      if (lane == 0) {
        if (!pair) {
          // (T[r][r] - mu) x_r = -s1
          float dr = A[r * ld + r] - mr, di = -mu_i;
          if (fabsf(dr) + fabsf(di) < tiny) dr = tiny;
          const float den = dr * dr + di * di;
          xr[r] = -(s1r * dr + s1i * di) / den;
          xi[r] = -(s1i * dr - s1r * di) / den;
        } else {
          // [[a - mu, b], [c, d - mu]] [x_top; x_r] = -[s0; s1]
          const float ar = A[top * ld + top] - mr, ai = -mu_i;
          const float br = A[top * ld + r];
          const float cr = A[r * ld + top];
          const float dr = A[r * ld + r] - mr, di = -mu_i;
          // det = (a-mu)(d-mu) - b c
          float detr = ar * dr - ai * di - br * cr;
          float deti = ar * di + ai * dr;
          if (fabsf(detr) + fabsf(deti) < tiny) detr = tiny;
          const float den = detr * detr + deti * deti;
          // x_top = (-(s0)(d-mu) + b s1) / det ; x_r = (-(a-mu) s1 + c s0) / det
          const float n0r = -(s0r * dr - s0i * di) + br * s1r;
          const float n0i = -(s0r * di + s0i * dr) + br * s1i;
          const float n1r = -(ar * s1r - ai * s1i) + cr * s0r;
          const float n1i = -(ar * s1i + ai * s1r) + cr * s0i;
          xr[top] = (n0r * detr + n0i * deti) / den;
          xi[top] = (n0i * detr - n0r * deti) / den;
          xr[r] = (n1r * detr + n1i * deti) / den;
          xi[r] = (n1i * detr - n1r * deti) / den;
        }
      }
      __syncwarp();
      r = top - 1;
    }
    // column 2*rank (real part) and 2*rank+1 (imaginary part) of X (n x ncx, global)
    float* xc = X + 2 * s_rank[j];
    for (int r = lane; r < n; r += 32) {
      xc[(size_t)r * ncx] = xr[r];
      xc[(size_t)r * ncx + 1] = xi[r];
    }
    __syncwarp();
  }
  __syncthreads();

  // ---- 6. back transformation Psi~ = Q_hess Zb_1 ... Zb_B x (X in shared memory; T is
  //         no longer needed): windows in reverse order, then the Hessenberg reflectors
  float* Xs = A;
  for (int e = tid; e < n * ncx; e += nth) Xs[e] = X[e];
  {
    float* Zs = smem + p.log_off;   // two staged window factors, WN x (WN + 4) each
    const int n_win = shi[5];
    auto stage = [&](int wdx, int buf) {
      const float* rec = zlog + (size_t)wdx * ZREC;
      float* dst = Zs + buf * WN * (WN + 4);
      for (int e2 = tid; e2 < WN * WN; e2 += nth) dst[(e2 / WN) * (WN + 4) + (e2 % WN)] = rec[8 + e2];
    };
    if (n_win > 0) stage(n_win - 1, 0);
    for (int wdx = n_win - 1, buf = 0; wdx >= 0; --wdx, buf ^= 1) {
      __syncthreads();
      if (wdx > 0) stage(wdx - 1, buf ^ 1);   // next factor, overlapped with this product
      const float* rec = zlog + (size_t)wdx * ZREC;
      const int bb = __float_as_int(rec[0]), ee = __float_as_int(rec[1]), ww = ee - bb;
      const float* Zc = Zs + buf * WN * (WN + 4);
      for (int col = tid; col < ncx; col += nth) {
        float in[WN];
#pragma unroll
        for (int j2 = 0; j2 < WN; ++j2) in[j2] = (j2 < ww) ? Xs[(bb + j2) * ncx + col] : 0.f;
        for (int i0 = 0; i0 < ww; i0 += 4) {
          float acc[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4* zr = reinterpret_cast<const float4*>(Zc + (i0 + u) * (WN + 4));
            float a = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < WN / 4; ++q4) {
              const float4 z = zr[q4];
              a = fmaf(z.x, in[4 * q4], a);
              a = fmaf(z.y, in[4 * q4 + 1], a);
              a = fmaf(z.z, in[4 * q4 + 2], a);
              a = fmaf(z.w, in[4 * q4 + 3], a);
            }
            acc[u] = a;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (i0 + u < ww) Xs[(bb + i0 + u) * ncx + col] = acc[u];
        }
      }
    }
    __syncthreads();
    float* sv3 = Zs;   // Hessenberg reflector staging (n floats)
    for (int j = n - 3; j >= 0; --j) {
      const int len = n - j - 1;
      __syncthreads();
      for (int c = tid; c < len; c += nth) sv3[c] = hv[(size_t)j * n + c];
      __syncthreads();
      const float beta = hv[(size_t)j * n + n - 1];
      if (beta == 0.f) continue;
      for (int col = tid; col < ncx; col += nth) {
        float sacc = 0.f;
        for (int r = 0; r < len; ++r) sacc = fmaf(sv3[r], Xs[(j + 1 + r) * ncx + col], sacc);
        sacc *= beta;
        for (int r = 0; r < len; ++r) Xs[(j + 1 + r) * ncx + col] -= sacc * sv3[r];
      }
    }
  }
  __syncthreads();

  // ---- 7. Phi = U[:l, :n] Psi~, normalisation, pole parameters
  for (int j = warp; j < n_slots; j += nwarps) {
    ssi_pole rec;
    rec.lag = p.lt.i[t];
    rec.order = n;
    rec.index = j;
    float* ph = phi_out + (size_t)j * 2 * l;
    if (failed || j >= npole) {
      if (lane == 0) {
        rec.f_hz = 0.f; rec.xi = 0.f; rec.mu_re = 0.f; rec.mu_im = 0.f; rec.mpc = 0.f; rec.mpd = 0.f;
        rec.flags = failed ? SSI_POLE_NOTCONV : 0u;
        poles[j] = rec;
      }
      for (int c = lane; c < 2 * l; c += 32) ph[c] = 0.f;
      continue;
    }
    // the pole of rank j
    int src = 0;
    for (int o = 0; o < npole; ++o) if (s_rank[o] == j) src = o;
    const float* xr = Xs + 2 * j;
    // phi_c = sum_a U[c][a] psi_a, complex: lanes split a (coalesced rows of U, psi held in
    // registers), a warp reduction per channel
    constexpr int NA = (SMEM_N_MAX + 31) / 32;
    float xre[NA], xim[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int a = lane + 32 * q;
      xre[q] = (a < n) ? xr[a * ncx] : 0.f;
      xim[q] = (a < n) ? xr[a * ncx + 1] : 0.f;
    }
    float nrm2 = 0.f, best = -1.f, bre = 1.f, bim = 0.f;
    for (int c = 0; c < l; ++c) {
      const float* wrow = U + (size_t)c * k;
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        const int a = lane + 32 * q;
        const float u = (a < n) ? wrow[a] : 0.f;
        sr = fmaf(u, xre[q], sr);
        si = fmaf(u, xim[q], si);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == (c & 31)) {
        ph[2 * c] = sr;
        ph[2 * c + 1] = si;
        const float m2 = sr * sr + si * si;
        nrm2 += m2;
        if (m2 > best) { best = m2; bre = sr; bim = si; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const float orr = __shfl_xor_sync(0xffffffffu, bre, o);
      const float oi = __shfl_xor_sync(0xffffffffu, bim, o);
      if (ob > best) { best = ob; bre = orr; bim = oi; }
    }
    __syncwarp();
    // scale by conj(largest)/|largest| / ||phi||
    const float bm = sqrtf(fmaxf(best, 0.f));
    const float inv = (nrm2 > 0.f && bm > 0.f) ? rsqrtf(nrm2) / bm : 0.f;
    const float cr = bre * inv, ci = -bim * inv;
    float sxx = 0.f, syy = 0.f, sxy = 0.f;
    for (int c = lane; c < l; c += 32) {
      const float a = ph[2 * c], b = ph[2 * c + 1];
      const float re = a * cr - b * ci, im = a * ci + b * cr;
      ph[2 * c] = re;
      ph[2 * c + 1] = im;
      sxx = fmaf(re, re, sxx);
      syy = fmaf(im, im, syy);
      sxy = fmaf(re, im, sxy);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
      syy += __shfl_xor_sync(0xffffffffu, syy, o);
      sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
    }
    const float tr = sxx + syy;
    const float dd = sqrtf((sxx - syy) * (sxx - syy) + 4.f * sxy * sxy);
    const float mpc = tr > 0.f ? (dd / tr) * (dd / tr) : 0.f;
    const float th = 0.5f * atan2f(2.f * sxy, sxx - syy);
    const float v1x = cosf(th), v1y = sinf(th);
    __syncwarp();
    float wsum = 0.f, asum = 0.f;
    for (int c = lane; c < l; c += 32) {
      const float re = ph[2 * c], im = ph[2 * c + 1];
      const float m = sqrtf(re * re + im * im);
      if (m > 0.f) {
        const float cosang = fminf(1.f, fabsf(re * v1x + im * v1y) / m);
        wsum += m;
        asum += m * acosf(cosang);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
      asum += __shfl_xor_sync(0xffffffffu, asum, o);
    }
    if (lane == 0) {
      const double mr = s_mur[src], mu_i = s_mui[src];
      const double lr = 0.5 * log(mr * mr + mu_i * mu_i) / p.dt, li = atan2(mu_i, mr) / p.dt;
      const double lam = sqrt(lr * lr + li * li);
      rec.f_hz = (float)(lam / (2.0 * 3.14159265358979323846));
      rec.xi = lam > 0 ? (float)(-lr / lam) : 0.f;
      rec.mu_re = (float)mr;
      rec.mu_im = (float)mu_i;
      rec.mpc = mpc;
      rec.mpd = wsum > 0.f ? (asum / wsum) / 1.5707963267948966f : 0.f;
      rec.flags = SSI_POLE_VALID;
      poles[j] = rec;
    }
  }
}

}  // namespace

RealizePlan realize_plan(int n_lags, const int* lags, int l, int k, const int* orders, int n_orders) {
  RealizePlan r{};
  r.n_lags = n_lags;
  r.l = l;
  r.k = k;
  r.n_orders = n_orders;
  r.max_order = 0;
  r.slots_per_lag = 0;
  long long work = 0;
  int max_i = 0;
  for (int m = 0; m < n_orders; ++m) {
    r.max_order = std::max(r.max_order, orders[m]);
    r.slots_per_lag += orders[m] / 2;
    work += eig_work_floats(orders[m], l) + 64;
  }
  for (int t = 0; t < n_lags; ++t) max_i = std::max(max_i, lags[t]);
  const int n_chunks = (int)ceil_div((int64_t)l * (max_i - 1), GR_ROWS);
  (void)SMEM_N_MAX;
  WsPlan w;
  w.add<float>((size_t)n_lags * std::max(n_chunks, 1) * 2 * k * k);  // Gram partials
  w.add<float>((size_t)n_lags * 2 * k * k);                          // G | H
  w.add<float>((size_t)n_lags * 2 * k * k);                          // Rinv | M
  w.add<float>((size_t)n_lags * work);                               // eig scratch
  r.ws_bytes = w.bytes;
  return r;
}

ssi_status realize_ws(ssi_ctx* ctx, Workspace& ws, const RealizePlan& r, const int* lags,
                      const float* const* U, const int* orders, double dt, ssi_pole* poles,
                      float* phi, int* dev_status, cudaStream_t stream) {
  ws.reset();
  SSI_CHECK(r.n_lags <= MAX_LAGS, "realize: at most %d lags per call", MAX_LAGS);
  SSI_CHECK(r.n_orders <= 512, "realize: at most 512 orders per call");
  LagTable lt{};
  lt.n_lags = r.n_lags;
  lt.l = r.l;
  lt.k = r.k;
  int max_i = 0;
  for (int t = 0; t < r.n_lags; ++t) {
    lt.i[t] = lags[t];
    lt.U[t] = U[t];
    max_i = std::max(max_i, lags[t]);
  }
  const int n_chunks = std::max(1, (int)ceil_div((int64_t)r.l * (max_i - 1), GR_ROWS));
  const int k = r.k;
  float* partial = ws.take<float>((size_t)r.n_lags * n_chunks * 2 * k * k);
  float* GH = ws.take<float>((size_t)r.n_lags * 2 * k * k);
  float* RM = ws.take<float>((size_t)r.n_lags * 2 * k * k);
  EigParams ep{};
  long long work = 0;
  for (int m = 0; m < r.n_orders; ++m) {
    ep.orders[m] = orders[m];
    ep.work_off[m] = work;
    work += eig_work_floats(orders[m], r.l) + 64;
  }
  float* eigw = ws.take<float>((size_t)r.n_lags * work);
  if (!partial || !GH || !RM || !eigw) {
    set_error("realize: workspace too small");
    return SSI_E_NOMEM;
  }
  const int tiles = (int)ceil_div(k, 64);
  dim3 g1((unsigned)(tiles * tiles), (unsigned)n_chunks, (unsigned)(2 * r.n_lags));
  count_launches(ctx, 4);
  {
  ProfScope ps(ctx, ST_GRAM, stream);
  k_gram_gh<<<g1, 256, 0, stream>>>(lt, n_chunks, partial);
  SSI_CUDA(cudaGetLastError());
  k_gram_reduce<<<ctx->num_sms * 4, 256, 0, stream>>>(partial, r.n_lags, n_chunks, k, GH);
  SSI_CUDA(cudaGetLastError());
  const size_t fsmem = (size_t)k * k * sizeof(float);
  SSI_CHECK(fsmem <= 220 * 1024, "realize: k=%d too large for the per-lag factorisation", k);
  SSI_CUDA(cudaFuncSetAttribute(k_lag_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(220 * 1024)));
  k_lag_factor<<<r.n_lags, 1024, fsmem, stream>>>(GH, k, RM, dev_status);
  SSI_CUDA(cudaGetLastError());
  }
  ep.lt = lt;
  ep.n_orders = r.n_orders;
  long long so = 0;
  for (int m = 0; m < r.n_orders; ++m) {
    ep.slot_off[m] = so;
    so += orders[m] / 2;
  }
  ep.slots_per_lag = so;
  ep.RM = RM;
  ep.work = eigw;
  ep.work_per_lag = work;
  ep.dt = dt;
  ep.poles = poles;
  ep.phi = phi;
  ep.status = dev_status;
  const int nsm_max = std::min(r.max_order, SMEM_N_MAX);
  ep.nmax = nsm_max;
  ep.xbuf_off = (int)round_up((int64_t)nsm_max * (nsm_max + 1), 32);
  ep.log_off = (int)round_up((int64_t)ep.xbuf_off + (int64_t)(EIG_THREADS / 32) * 2 * nsm_max, 32);
  const size_t esmem = ((size_t)ep.log_off + (size_t)std::max(2 * WN * (WN + 4), SMEM_N_MAX)) * sizeof(float);
  SSI_CUDA(cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esmem));
  ProfScope ps_eig(ctx, ST_EIG, stream);
  k_eig<<<r.n_lags * r.n_orders, EIG_THREADS, esmem, stream>>>(ep);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace ssi

extern "C" ssi_status ssi_realize_batch(ssi_ctx* ctx, int n_lags, const int* lags,
                                        const float* const* U, int l, int k, const int* orders,
                                        int n_orders, double dt, ssi_pole* poles, float* phi,
                                        void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && lags && U && orders && poles && phi, "ssi_realize_batch: null pointer");
  SSI_CHECK(n_lags >= 1 && n_lags <= MAX_LAGS, "ssi_realize_batch: 1 <= n_lags <= %d", MAX_LAGS);
  SSI_CHECK(n_orders >= 1 && n_orders <= 512, "ssi_realize_batch: 1 <= n_orders <= 512");
  SSI_CHECK(l >= 1 && k >= 2 && dt > 0, "ssi_realize_batch: bad l/k/dt");
  SSI_CHECK(k <= 224, "ssi_realize_batch: k=%d > 224 not supported", k);
  for (int t = 0; t < n_lags; ++t) {
    SSI_CHECK(lags[t] >= 2, "ssi_realize_batch: lag %d < 2", lags[t]);
    SSI_CHECK(U[t], "ssi_realize_batch: null U[%d]", t);
    SSI_CHECK((int64_t)l * lags[t] >= k, "ssi_realize_batch: l*i < k");
  }
  for (int m = 0; m < n_orders; ++m) {
    SSI_CHECK(orders[m] >= 2 && orders[m] % 2 == 0 && orders[m] <= k,
              "ssi_realize_batch: order %d must be even and in [2, k]", orders[m]);
    SSI_CHECK(orders[m] <= SMEM_N_MAX, "ssi_realize_batch: order %d > %d not supported", orders[m],
              SMEM_N_MAX);
    SSI_CHECK(m == 0 || orders[m] > orders[m - 1], "ssi_realize_batch: orders must ascend");
  }
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RealizePlan plan = realize_plan(n_lags, lags, l, k, orders, n_orders);
  SSI_TRY(ws_reserve(ctx, ctx->ws, plan.ws_bytes, s));
  SSI_TRY(realize_ws(ctx, ctx->ws, plan, lags, U, orders, dt, poles, phi, ctx->dev_status, s));
  return check_dev_status(ctx->dev_status, s);
}
