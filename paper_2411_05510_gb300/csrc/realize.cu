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
  // Rinv by column back substitution: thread c owns column c
  for (int c = tid; c < k; c += nth) {
    for (int r = k - 1; r >= 0; --r) {
      if (r > c) { Rinv[(size_t)r * k + c] = 0.f; continue; }
      float s = (r == c) ? 1.f : 0.f;
      for (int j = r + 1; j <= c; ++j) s -= sR[r * k + j] * Rinv[(size_t)j * k + c];
      Rinv[(size_t)r * k + c] = s / sR[r * k + r];
    }
  }
  // M = R^{-T} H: forward substitution R^T M = H, thread c owns column c
  for (int c = tid; c < k; c += nth) {
    for (int r = 0; r < k; ++r) {
      float s = H[(size_t)r * k + c];
      for (int j = 0; j < r; ++j) s -= sR[j * k + r] * M[(size_t)j * k + c];
      M[(size_t)r * k + c] = s / sR[r * k + r];
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
  int nmax;                  // largest order of the launch
  double dt;
  ssi_pole* poles;
  float* phi;
  int* status;
};

// scratch of one realisation of order n: Hessenberg v's (n*n), reflector log, X (n*n)
__host__ __device__ inline long long qr_log_cap(int n) { return 3LL * n * n + 64LL * n + 64; }
__host__ __device__ inline long long eig_work_floats(int n) {
  return (long long)n * n + 8 * qr_log_cap(n) + (long long)n * n + 2LL * n + 64;
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
  float* qlog = hv + (size_t)n * n;           // QR reflector log, 8 floats per entry
  float* X = qlog + 8 * qr_log_cap(n);        // eigenvector matrix, n x (2 m)
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

  // ---- 1. A~_n = Rinv[:n,:n] M[:n,:n]
  for (int e = tid; e < n * n; e += nth) {
    const int r = e / n, c = e % n;
    float s = 0.f;
    for (int j = r; j < n; ++j) s = fmaf(Rinv[(size_t)r * k + j], M[(size_t)j * k + c], s);
    A[r * ld + c] = s;
  }
  __syncthreads();

  // ---- 2. Householder reduction to upper Hessenberg form
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    float* v = hv + (size_t)j * n;
    // norm of A[j+1:, j] (thread 0; len <= 224)
    if (tid == 0) {
      float ss = 0.f;
      for (int r = 0; r < len; ++r) ss = fmaf(A[(j + 1 + r) * ld + j], A[(j + 1 + r) * ld + j], ss);
      const float x0 = A[(j + 1) * ld + j];
      const float nx = sqrtf(ss);
      const float alpha = x0 >= 0.f ? -nx : nx;
      const float vv = ss - x0 * x0 + (x0 - alpha) * (x0 - alpha);
      sh[0] = alpha;
      sh[1] = (nx > 0.f && vv > 0.f) ? 2.f / vv : 0.f;
      sh[2] = x0 - alpha;
    }
    __syncthreads();
    const float beta = sh[1];
    for (int r = tid; r < len; r += nth) v[r] = (r == 0) ? sh[2] : A[(j + 1 + r) * ld + j];
    if (tid == 0) v[n - 1] = beta;   // v has len <= n-2 entries; beta stored at the end
    __syncthreads();
    if (beta != 0.f) {
      // left: A[j+1:, c] -= beta v (v^T A[j+1:, c]) for c >= j
      for (int c = j + tid; c < n; c += nth) {
        float s = 0.f;
        for (int r = 0; r < len; ++r) s = fmaf(v[r], A[(j + 1 + r) * ld + c], s);
        s *= beta;
        for (int r = 0; r < len; ++r) A[(j + 1 + r) * ld + c] -= s * v[r];
      }
      __syncthreads();
      // right: A[r, j+1:] -= beta (A[r, j+1:] v) v^T for all rows
      for (int r = tid; r < n; r += nth) {
        float s = 0.f;
        for (int c = 0; c < len; ++c) s = fmaf(A[r * ld + j + 1 + c], v[c], s);
        s *= beta;
        for (int c = 0; c < len; ++c) A[r * ld + j + 1 + c] -= s * v[c];
      }
      __syncthreads();
      if (tid == 0) {
        A[(j + 1) * ld + j] = sh[0];
        for (int r = 2; r <= len; ++r) A[(j + r) * ld + j] = 0.f;
      }
    }
    __syncthreads();
  }

  // ---- 3. Francis double-shift QR (real Schur form, full T updated), reflectors logged
  // shi[0]: nn, shi[1]: l, shi[2]: m, shi[3]: done flag, shi[4]: failed, shi[5]: log count
  if (tid == 0) {
    float anorm = 0.f;
    for (int r = 0; r < n; ++r)
      for (int c = max(r - 1, 0); c < n; ++c) anorm += fabsf(A[r * ld + c]);
    sh[8] = anorm;
    shi[0] = n - 1;
    shi[4] = 0;
    shi[5] = 0;
  }
  __syncthreads();
  const long long log_cap = qr_log_cap(n);
  int its = 0, total_its = 0;
  const int itmax = 30 * max(10, n);
  while (true) {
    // thread 0: deflation search and shift selection
    if (tid == 0) {
      int nn = shi[0];
      const float anorm = sh[8];
      shi[3] = 0;
      while (nn >= 0) {
        int ll;
        for (ll = nn; ll >= 1; --ll) {
          float s = fabsf(A[(ll - 1) * ld + ll - 1]) + fabsf(A[ll * ld + ll]);
          if (s == 0.f) s = anorm;
          if (fabsf(A[ll * ld + ll - 1]) <= FLT_EPSILON * s) {
            A[ll * ld + ll - 1] = 0.f;
            break;
          }
        }
        if (ll < 1) ll = 0;
        if (ll == nn) { nn -= 1; its = 0; continue; }
        if (ll == nn - 1) { nn -= 2; its = 0; continue; }
        // a QR sweep is needed on rows ll..nn
        if (total_its >= itmax) { shi[4] = 1; nn = -1; break; }
        float x = A[nn * ld + nn], y = A[(nn - 1) * ld + nn - 1];
        float w = A[nn * ld + nn - 1] * A[(nn - 1) * ld + nn];
        if (its == 10 || its == 20) {
          const float s = fabsf(A[nn * ld + nn - 1]) + fabsf(A[(nn - 1) * ld + nn - 2]);
          x = y = 0.75f * s;
          w = -0.4375f * s * s;
        }
        ++its;
        ++total_its;
        int m;
        float pp = 0.f, qq = 0.f, rr = 0.f;
        for (m = nn - 2; m >= ll; --m) {
          const float z = A[m * ld + m];
          const float r2 = x - z, s2 = y - z;
          pp = (r2 * s2 - w) / A[(m + 1) * ld + m] + A[m * ld + m + 1];
          qq = A[(m + 1) * ld + m + 1] - z - r2 - s2;
          rr = A[(m + 2) * ld + m + 1];
          const float s = fabsf(pp) + fabsf(qq) + fabsf(rr);
          pp /= s; qq /= s; rr /= s;
          if (m == ll) break;
          const float u = fabsf(A[m * ld + m - 1]) * (fabsf(qq) + fabsf(rr));
          const float v = fabsf(pp) * (fabsf(A[(m - 1) * ld + m - 1]) + fabsf(z) + fabsf(A[(m + 1) * ld + m + 1]));
          if (u <= FLT_EPSILON * v) break;
        }
        for (int r = m + 2; r <= nn; ++r) {
          A[r * ld + r - 2] = 0.f;
          if (r != m + 2) A[r * ld + r - 3] = 0.f;
        }
        shi[1] = ll;
        shi[2] = m;
        sh[0] = pp; sh[1] = qq; sh[2] = rr;
        shi[3] = 1;
        break;
      }
      shi[0] = nn;
    }
    __syncthreads();
    if (!shi[3]) break;   // converged (nn < 0) or failed
    const int ll = shi[1], m = shi[2], nn = shi[0];
    // bulge chase k = m .. nn-1
    for (int kk = m; kk <= nn - 1; ++kk) {
      if (tid == 0) {
        float pp, qq, rr, x;
        bool go = true;
        if (kk == m) {
          pp = sh[0]; qq = sh[1]; rr = sh[2];
          x = 1.f;
        } else {
          pp = A[kk * ld + kk - 1];
          qq = A[(kk + 1) * ld + kk - 1];
          rr = (kk != nn - 1) ? A[(kk + 2) * ld + kk - 1] : 0.f;
          x = fabsf(pp) + fabsf(qq) + fabsf(rr);
          if (x != 0.f) { pp /= x; qq /= x; rr /= x; } else go = false;
        }
        float s = 0.f;
        if (go) {
          s = sgnf(sqrtf(pp * pp + qq * qq + rr * rr), pp);
          if (s == 0.f) go = false;
        }
        if (go) {
          if (kk == m) {
            if (ll != m) A[kk * ld + kk - 1] = -A[kk * ld + kk - 1];
          } else {
            A[kk * ld + kk - 1] = -s * x;
          }
          pp += s;
          sh[4] = pp / s;        // w0
          sh[5] = qq / s;        // w1
          sh[6] = rr / s;        // w2
          sh[9] = qq / pp;       // u1
          sh[10] = rr / pp;      // u2
          shi[6] = 1;
          const int cnt = shi[5];
          if (cnt < log_cap) {
            float* e = qlog + 8LL * cnt;
            e[0] = sh[4]; e[1] = sh[5]; e[2] = sh[6]; e[3] = sh[9]; e[4] = sh[10];
            e[5] = __int_as_float(kk);
            e[6] = __int_as_float(kk != nn - 1 ? 3 : 2);
            e[7] = 0.f;
          }
          shi[5] = cnt + 1;
        } else {
          shi[6] = 0;
        }
      }
      __syncthreads();
      if (shi[6]) {
        const float w0 = sh[4], w1 = sh[5], w2 = sh[6], u1 = sh[9], u2 = sh[10];
        const bool three = kk != nn - 1;
        // row modification over all columns j >= kk (full Schur form)
        for (int j = kk + tid; j < n; j += nth) {
          float s = A[kk * ld + j] + u1 * A[(kk + 1) * ld + j];
          if (three) s += u2 * A[(kk + 2) * ld + j];
          A[kk * ld + j] -= s * w0;
          A[(kk + 1) * ld + j] -= s * w1;
          if (three) A[(kk + 2) * ld + j] -= s * w2;
        }
        __syncthreads();
        // column modification over rows 0 .. min(nn, kk+3)
        const int imax = min(nn, kk + 3);
        for (int i2 = tid; i2 <= imax; i2 += nth) {
          float s = w0 * A[i2 * ld + kk] + w1 * A[i2 * ld + kk + 1];
          if (three) s += w2 * A[i2 * ld + kk + 2];
          A[i2 * ld + kk] -= s;
          A[i2 * ld + kk + 1] -= s * u1;
          if (three) A[i2 * ld + kk + 2] -= s * u2;
        }
      }
      __syncthreads();
    }
  }
  const bool failed = shi[4] != 0 || shi[5] > log_cap;
  const int n_log = min((long long)shi[5], log_cap);

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

  // ---- 6. back transformation: Psi~ = Z x, reflectors applied in reverse order
  float* Xs = A;   // T is no longer needed: X moves to shared memory (n x ncx)
  for (int e = tid; e < n * ncx; e += nth) Xs[e] = X[e];
  __syncthreads();
  for (int col = tid; col < ncx; col += nth) {
    for (int q = n_log - 1; q >= 0; --q) {
      const float* e = qlog + 8LL * q;
      const float w0 = e[0], w1 = e[1], w2 = e[2], u1 = e[3], u2 = e[4];
      const int kk = __float_as_int(e[5]);
      const bool three = __float_as_int(e[6]) == 3;
      float s = Xs[kk * ncx + col] + u1 * Xs[(kk + 1) * ncx + col];
      if (three) s += u2 * Xs[(kk + 2) * ncx + col];
      Xs[kk * ncx + col] -= s * w0;
      Xs[(kk + 1) * ncx + col] -= s * w1;
      if (three) Xs[(kk + 2) * ncx + col] -= s * w2;
    }
    for (int j = n - 3; j >= 0; --j) {
      const float* v = hv + (size_t)j * n;
      const float beta = v[n - 1];
      if (beta == 0.f) continue;
      const int len = n - j - 1;
      float s = 0.f;
      for (int r = 0; r < len; ++r) s = fmaf(v[r], Xs[(j + 1 + r) * ncx + col], s);
      s *= beta;
      for (int r = 0; r < len; ++r) Xs[(j + 1 + r) * ncx + col] -= s * v[r];
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
    // phi_c = sum_a U[c][a] x_a, complex; track the norm and the largest component
    float nrm2 = 0.f, best = -1.f, bre = 1.f, bim = 0.f;
    for (int c = lane; c < l; c += 32) {
      float sr = 0.f, si = 0.f;
      const float* urow = U + (size_t)c * k;
      for (int a = 0; a < n; ++a) {
        const float u = urow[a];
        sr = fmaf(u, xr[a * ncx], sr);
        si = fmaf(u, xr[a * ncx + 1], si);
      }
      ph[2 * c] = sr;
      ph[2 * c + 1] = si;
      const float m2 = sr * sr + si * si;
      nrm2 += m2;
      if (m2 > best) { best = m2; bre = sr; bim = si; }
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
    work += eig_work_floats(orders[m]) + (orders[m] > SMEM_N_MAX ? (long long)orders[m] * (orders[m] + 1) : 0) + 64;
  }
  for (int t = 0; t < n_lags; ++t) max_i = std::max(max_i, lags[t]);
  const int n_chunks = (int)ceil_div((int64_t)l * (max_i - 1), GR_ROWS);
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
    work += eig_work_floats(orders[m]) + (orders[m] > SMEM_N_MAX ? (long long)orders[m] * (orders[m] + 1) : 0) + 64;
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
  const size_t esmem = ((size_t)ep.xbuf_off + (size_t)(EIG_THREADS / 32) * 2 * nsm_max) * sizeof(float);
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
  SSI_CHECK(k <= 232, "ssi_realize_batch: k=%d > 232 not supported", k);
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
