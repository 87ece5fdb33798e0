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
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <vector>

#include "blackwell.cuh"
#include "common.cuh"

namespace ssi {

namespace {

constexpr int MAX_LAGS = 64;
constexpr int EIG_THREADS = 512;
constexpr int GR_ROWS = 512;      // rows per Gram chunk
constexpr int SMEM_N_MAX = 224;   // largest order whose A fits shared memory
constexpr int N_MAX = 512;        // largest order (larger ones keep A in global scratch)

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
constexpr int FACTOR_SMEM_K = 224;   // largest k whose factor fits shared memory
// GH[t] = [G | H] (2 x k x k); out RM[t] = [Rinv | M] (2 x k x k) with G = R^T R and
// M = R^{-T} H.  One CTA per lag, R in shared memory (row stride k + 1):
//   1. right-looking Cholesky on the upper triangle (warp 0 scales row j, then all
//      threads update the trailing triangle);
//   2. R^{-1} in place, column by column (column j from the inverted leading block and
//      a copy of R's column j);
//   3. M = R^{-T} H = (R^{-1})^T H with 4 x 4 outputs per thread.
// GLOBAL: k > FACTOR_SMEM_K (FP32) or FP64, the same layout in the lag's global scratch
// (L2-resident); a separate instantiation keeps shared-memory instructions for the common
// case.  T: float (the default small-problem arithmetic) or double.
template <typename T> __device__ __forceinline__ T min_normal();
template <> __device__ __forceinline__ float min_normal<float>() { return FLT_MIN; }
template <> __device__ __forceinline__ double min_normal<double>() { return DBL_MIN; }

template <bool GLOBAL, typename T>
__global__ void __launch_bounds__(1024)
    k_lag_factor(const T* __restrict__ GH, int k, T* __restrict__ RM, T* Rglobal, int* status) {
  extern __shared__ __align__(16) unsigned char s_R_raw[];  // k x (k+1), then a column buffer of k
  T* sR = GLOBAL ? Rglobal + (size_t)blockIdx.x * ((size_t)k * (k + 1) + k)
                 : reinterpret_cast<T*>(s_R_raw);
  const int ldr = k + 1;
  T* col = sR + (size_t)k * ldr;
  const int t = blockIdx.x;
  const T* G = GH + (size_t)t * 2 * k * k;
  const T* H = G + (size_t)k * k;
  T* Rinv = RM + (size_t)t * 2 * k * k;
  T* M = Rinv + (size_t)k * k;
  const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5, lane = tid & 31,
            nwarps = nth >> 5;
  __shared__ T s_red[32];
  T gmax = 0;
  for (int e = tid; e < k * k; e += nth) {
    const int r = e / k, c = e % k;
    const T v = G[e];
    sR[r * ldr + c] = v;
    if (r == c) gmax = fmax(gmax, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  if (lane == 0) s_red[warp] = gmax;
  __syncthreads();
  if (tid == 0) {
    T g = 0;
    for (int w2 = 0; w2 < nwarps; ++w2) g = fmax(g, s_red[w2]);
    s_red[0] = g;
  }
  __syncthreads();
  const T floor_v = fmax(s_red[0] * (T)1e-10, min_normal<T>());
  // 1. Cholesky: row j of R
  for (int j = 0; j < k; ++j) {
    if (warp == 0) {
      T d = sR[j * ldr + j];
      if (!(d > floor_v)) {
        if (lane == 0) atomicOr(status, DEV_NOTCONVERGED);
        d = floor_v;
      }
      d = sqrt(d);
      const T id = T(1) / d;
      for (int c = j + 1 + lane; c < k; c += 32) sR[j * ldr + c] *= id;
      if (lane == 0) sR[j * ldr + j] = d;
    }
    __syncthreads();
    // G[a][c] -= R[j][a] R[j][c], j < a <= c: warps along rows, lanes along columns
    for (int a = j + 1 + warp; a < k; a += nwarps) {
      const T ra = sR[j * ldr + a];
      for (int c = a + lane; c < k; c += 32) sR[a * ldr + c] -= ra * sR[j * ldr + c];
    }
    __syncthreads();
  }
  // 2. R^{-1} in place: column j = -(1/R[j][j]) Rinv[0:j, 0:j] R[0:j, j], Rinv[j][j] = 1/R[j][j]
  for (int j = 0; j < k; ++j) {
    for (int i = tid; i < j; i += nth) col[i] = sR[i * ldr + j];
    __syncthreads();
    const T inv = T(1) / sR[j * ldr + j];
    for (int i = tid; i < j; i += nth) {
      T a0 = 0, a1 = 0;
      int m = i;
      for (; m + 1 < j; m += 2) {
        a0 = fma(sR[i * ldr + m], col[m], a0);
        a1 = fma(sR[i * ldr + m + 1], col[m + 1], a1);
      }
      if (m < j) a0 = fma(sR[i * ldr + m], col[m], a0);
      sR[i * ldr + j] = -(a0 + a1) * inv;
    }
    __syncthreads();
    if (tid == 0) sR[j * ldr + j] = inv;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nth) {
    const int r = e / k, c = e % k;
    Rinv[e] = (c >= r) ? sR[r * ldr + c] : T(0);
  }
  // 3. M[j][c] = sum_{r <= j} Rinv[r][j] H[r][c]
  const int k4 = (k + 3) / 4;
  for (int task = tid; task < k4 * k4; task += nth) {
    const int j0 = 4 * (task / k4), c0 = 4 * (task % k4);
    T acc[4][4] = {};
    const int rmax = min(j0 + 3, k - 1);
    for (int r = 0; r <= rmax; ++r) {
      T ri[4], hv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ri[u] = (j0 + u < k && r <= j0 + u) ? sR[r * ldr + j0 + u] : T(0);
        hv[u] = (c0 + u < k) ? __ldg(H + (size_t)r * k + c0 + u) : T(0);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[a][u] = fma(ri[a], hv[u], acc[a][u]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + a < k && c0 + u < k) M[(size_t)(j0 + a) * k + c0 + u] = acc[a][u];
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
  double dt;
  ssi_pole* poles;
  float* phi;
  int* status;
  int vec_blocks[512];       // eigenvector blocks of order m (k_eig_vectors)
  int vec_blocks_per_lag;
};

// scratch of one realisation of order n: a header (poles, windows, failure flag), the
// Householder vectors of the Hessenberg reduction (n*n), the eigenvectors of T (n*n) and the
// log of the QR iteration's window factors (zlog_cap(n) records of ZREC floats: b, e, then
// the WN x WN factor row-major)
constexpr int EIG_HDR = 64;
constexpr int ZREC = WN * WN + 8;
__host__ __device__ inline long long zlog_cap(int n) { return (long long)n * n / 16 + 2LL * n + 64; }
// (a multiple of 8 floats, so that every realisation's window records stay 16-byte aligned
// for the cp.async copies of the eigenvector kernel)
__host__ __device__ inline long long eig_work_floats(int n, int) {
  return EIG_HDR + 2LL * n * n + zlog_cap(n) * ZREC + 64 +
         (n > SMEM_N_MAX ? (((long long)n * (n + 1) + 7) & ~7LL) : 0LL);   // A of the larger orders
}
// shared-memory layout of one k_eig CTA of order n (in floats): A when n <= SMEM_N_MAX,
// then the vector buffers (8 warps x 2n floats; before the eigenvectors they hold the
// Hessenberg vector and the helpers' transposed window factor), then the two window
// factors of the QR iteration
__host__ __device__ inline int eig_xbuf_off(int n) {
  return n <= SMEM_N_MAX ? ((n * (n + 1) + 31) / 32) * 32 : 0;
}
__host__ __device__ inline int eig_log_off(int n) {
  const int vb = 16 * n > WN * (WN + 4) ? 16 * n : WN * (WN + 4);
  return ((eig_xbuf_off(n) + vb + 31) / 32) * 32;
}
__host__ __device__ inline int eig_smem_floats(int n) { return eig_log_off(n) + 2 * WN * (WN + 4); }
constexpr int VEC_COLS = 32;   // columns of X per eigenvector block (16 poles)

// Bounded wait (2 s of %globaltimer) of a whole warp until *x >= v; the result is the
// same in every lane.  On timeout the status word gets DEV_TIMEOUT from the caller.
__device__ __forceinline__ bool warp_wait_geq(volatile int* x, int v) {
  bool ok = true;
  if (*x < v) {
    const uint64_t t0 = bw::global_ns();
    while (*x < v) {
      if (bw::global_ns() - t0 > 2000000000ull) {
        ok = false;
        break;
      }
      __nanosleep(32);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  __threadfence_block();
  return ok;
}

constexpr int NCH = 6;        // chaser warps: bulges chased at once in a multi-bulge sweep
constexpr int NMIN_MB = 30;   // active blocks below this size are swept with one bulge

// barrier of the chaser warps only (named barrier 2)
__device__ __forceinline__ void chaser_sync() {
  asm volatile("bar.sync 2, %0;" ::"n"(NCH * 32) : "memory");
}

// barrier of the helper warps only (named barrier 1; barrier 0 is __syncthreads)
__device__ __forceinline__ void helper_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

__device__ __forceinline__ float sgnf(float a, float b) { return b >= 0.f ? fabsf(a) : -fabsf(a); }

// One Householder reflector of the Hessenberg reduction applied from both sides,
// H = (I - beta v v^T) H (I - beta v v^T) on rows/columns j+1.., with v in registers: entry c
// on lane c % 32, slot c / 32 (the same layout serves the rows of the left update and the
// columns of the right update); a warp owns HB whole columns (rows) at a time, forms their
// dot products, reduces the HB sums together (independent shuffle trees, so their
// latencies overlap), and updates the elements it still holds in registers.  NV slots
// cover reflectors of up to 32 NV entries.
constexpr int HB = 4;
template <int NV>
__device__ __forceinline__ void hess_update(float* A, int ld, int n, int j, int len, float beta,
                                            const float* sv, int hw, int hl, int hnw) {
  float vreg[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const int c = hl + 32 * q;
    vreg[q] = (c < len) ? sv[c] : 0.f;
  }
  // left: A[j+1:, c] -= beta v (v^T A[j+1:, c]) for c > j (column j is already final)
  for (int c0 = j + 1 + HB * hw; c0 < n; c0 += HB * hnw) {
    float a[HB][NV];
    float dot[HB];
#pragma unroll
    for (int b = 0; b < HB; ++b) {
      dot[b] = 0.f;
      const bool ok = c0 + b < n;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int r = hl + 32 * q;
        a[b][q] = (ok && r < len) ? A[(j + 1 + r) * ld + c0 + b] : 0.f;
        dot[b] = fmaf(a[b][q], vreg[q], dot[b]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int b = 0; b < HB; ++b) dot[b] += __shfl_xor_sync(0xffffffffu, dot[b], o);
#pragma unroll
    for (int b = 0; b < HB; ++b) {
      if (c0 + b >= n) break;
      const float sc = dot[b] * beta;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int r = hl + 32 * q;
        if (r < len) A[(j + 1 + r) * ld + c0 + b] = fmaf(-sc, vreg[q], a[b][q]);
      }
    }
  }
  __syncthreads();
  // right: A[r, j+1:] -= beta (A[r, j+1:] v) v^T for all rows
  for (int r0 = HB * hw; r0 < n; r0 += HB * hnw) {
    float a[HB][NV];
    float dot[HB];
#pragma unroll
    for (int b = 0; b < HB; ++b) {
      dot[b] = 0.f;
      const bool ok = r0 + b < n;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int c = hl + 32 * q;
        a[b][q] = (ok && c < len) ? A[(r0 + b) * ld + j + 1 + c] : 0.f;
        dot[b] = fmaf(a[b][q], vreg[q], dot[b]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int b = 0; b < HB; ++b) dot[b] += __shfl_xor_sync(0xffffffffu, dot[b], o);
#pragma unroll
    for (int b = 0; b < HB; ++b) {
      if (r0 + b >= n) break;
      const float sc = dot[b] * beta;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int c = hl + 32 * q;
        if (c < len) A[(r0 + b) * ld + j + 1 + c] = fmaf(-sc, vreg[q], a[b][q]);
      }
    }
  }
}

// BIG: orders above SMEM_N_MAX, A in the realisation's global scratch (a separate
// instantiation, so that the shared-memory kernel of the smaller orders is unchanged).
// Work items count from item_base: largest orders first.  The parameters of the
// realisation(s) are in device memory: one block P[0] when `items` is null (the CTA's item
// is its index), or one block per job of a batch, the CTA's (job, order index, lag) then
// read from `items`.
template <bool BIG>
__global__ void __launch_bounds__(EIG_THREADS, 1)
    k_eig(const EigParams* __restrict__ P, const int4* __restrict__ items, int item_base) {
  extern __shared__ float smem[];
  int job = 0, mi, t;
  if (items) {
    const int4 it = items[blockIdx.x + item_base];
    job = it.x;
    mi = it.y;
    t = it.z;
  } else {
    // work item: largest orders first
    const int item = blockIdx.x + item_base;
    mi = P[0].n_orders - 1 - (item / P[0].lt.n_lags);
    t = item % P[0].lt.n_lags;
  }
  const EigParams& p = P[job];
  const int n = p.orders[mi];
  const int k = p.lt.k, l = p.lt.l;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ld = n + 1;   // padded leading dimension against bank conflicts
  float* work = p.work + (size_t)t * p.work_per_lag + p.work_off[mi];
  int* hdr = reinterpret_cast<int*>(work);    // 0 poles, 1 windows, 2 failed
  float* hv = work + EIG_HDR;                 // Hessenberg reflectors: n x n (v, beta in [j*n + n-1])
  float* X = hv + (size_t)n * n;              // eigenvectors of T, n x (2 m)
  float* zlog = X + (size_t)n * n;            // window factors of the QR iteration
  // A (n x (n+1)): shared memory up to SMEM_N_MAX, else the realisation's global scratch
  // (L2-resident), same code either way
  float* A = BIG ? zlog + zlog_cap(n) * ZREC : smem;
  const int xbuf_off = eig_xbuf_off(n), log_off = eig_log_off(n);
  __shared__ float sh[16];
  __shared__ int shi[16];
  __shared__ int s_pos[256];                  // position p of the 2x2 block of pole j
  __shared__ float s_mur[256], s_mui[256];
  const float* Rinv = p.RM + (size_t)t * 2 * k * k;
  const float* M = Rinv + (size_t)k * k;
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  const int n_slots = n / 2;

  // ---- 1. A~_n = Rinv[:n,:n] M[:n,:n] (Rinv upper triangular); 4 x 4 tiles per thread
  {
    const int n4 = (n + 3) / 4;
    for (int tt = tid; tt < n4 * n4; tt += nth) {
      const int r0 = 4 * (tt / n4), c0 = 4 * (tt % n4);
      float acc[4][4] = {};
      for (int j = r0; j < n; ++j) {
        float ri[4], mv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ri[u] = (r0 + u < n && j >= r0 + u) ? Rinv[(size_t)(r0 + u) * k + j] : 0.f;
          mv[u] = (c0 + u < n) ? M[(size_t)j * k + c0 + u] : 0.f;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[a][u] = fmaf(ri[a], mv[u], acc[a][u]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (r0 + a < n && c0 + u < n) A[(r0 + a) * ld + c0 + u] = acc[a][u];
    }
  }
  __syncthreads();

  // ---- 2. Householder reduction to upper Hessenberg form (v kept in shared memory and
  //         logged to global memory for the back transformation)
  float* sv = smem + xbuf_off;   // n floats (the vector buffers are not in use yet)
  __shared__ float s_part[EIG_THREADS / 32];
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;
    float* v = hv + (size_t)j * n;
    const float x0 = A[(j + 1) * ld + j];   // read by every thread before the barrier
    float ss = 0.f;
    for (int r = tid; r < len; r += nth) {
      const float x = A[(j + 1 + r) * ld + j];
      ss = fmaf(x, x, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0) s_part[tid >> 5] = ss;
    __syncthreads();
    // every thread forms the reflector (the same in every thread: no second barrier)
    float tot = 0.f;
    for (int w2 = 0; w2 < nth / 32; ++w2) tot += s_part[w2];
    const float nx = sqrtf(tot);
    const float alpha = x0 >= 0.f ? -nx : nx;
    const float vv = tot - x0 * x0 + (x0 - alpha) * (x0 - alpha);
    const float beta = (nx > 0.f && vv > 0.f) ? 2.f / vv : 0.f;
    // v to shared and global memory; column j takes its final value (alpha, then zeros)
    // from the thread that read the entry
    for (int r = tid; r < len; r += nth) {
      const float vr = (r == 0) ? x0 - alpha : A[(j + 1 + r) * ld + j];
      sv[r] = vr;
      v[r] = vr;
      if (beta != 0.f) A[(j + 1 + r) * ld + j] = (r == 0) ? alpha : 0.f;
    }
    if (tid == 0) v[n - 1] = beta;   // v has len <= n-2 entries; beta stored at the end
    __syncthreads();
    if (beta != 0.f) {
      // as many 32-entry register slots as this reflector has entries: the instruction
      // count of an update scales with the slots, and the reflectors shrink (the
      // global-memory kernel keeps one variant)
      const int hw = tid >> 5, hl = tid & 31, hnw = nth >> 5;
      switch (BIG ? 0 : (len + 31) / 32) {
        case 1: hess_update<1>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 2: hess_update<2>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 3: hess_update<3>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 4: hess_update<4>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 5: hess_update<5>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 6: hess_update<6>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        case 7: hess_update<7>(A, ld, n, j, len, beta, sv, hw, hl, hnw); break;
        default: hess_update<((BIG ? N_MAX : SMEM_N_MAX) + 31) / 32>(A, ld, n, j, len, beta, sv, hw,
                                                                    hl, hnw);
      }
    }
    __syncthreads();
  }

  // ---- 3b. Francis double-shift QR iteration to real Schur form T = Z^T H Z (Martin,
  //  Peters and Wilkinson's algorithm for real Hessenberg matrices, with their
  //  exceptional shifts after 10 and 20 iterations), windowed and pipelined.
  //  Warp 0 (the chaser) chases the bulge of each sweep inside windows of WN rows/columns,
  //  updating in-window rows and columns at once and accumulating the window's
  //  transformations in Zb (WN x WN).  The helpers (warps 1-15 except those sharing warp
  //  0's scheduler: warps 4, 8, 12) apply each posted Zb to the rest of the matrix -- the
  //  rows of the window right of it (H[b:e, e:n] = Zb^T H[b:e, e:n]) and the columns of
  //  the window above it (H[0:b, b:e] = H[0:b, b:e] Zb) -- and log it to global memory
  //  for the back transformation of the eigenvectors, while the chaser is in the next
  //  window.  The next window overlaps the rows of the previous one in
  //  three rows, so the chaser first does the previous window's right update in the
  //  columns of the next window itself (the helpers skip them).  A sweep starts only when
  //  every window has been applied.  Same arithmetic as the unwindowed sweep.  Hand-offs
  //  are shared counters with bounded waits.
  float* Zbuf = smem + log_off;       // 2 window factors, WN x (WN + 4) each (16-byte aligned rows)
  float* ZT = smem + xbuf_off;        // the helpers' transposed factor (vector buffers idle here)
  __shared__ volatile int s_posted, s_taken, s_applied, s_state, s_go, s_nwin;
  __shared__ int s_desc[2][4];        // per factor buffer: b, e, kend, end of the chaser's columns
  __shared__ float s_sh[3];           // shift vector of the first step of the sweep
  if (tid == 0) {
    s_posted = 0;
    s_taken = 0;
    s_applied = 0;
    s_state = 0;   // 0 running, 1 done, 2 failed
    s_go = 0;
    s_nwin = 0;
  }
  __syncthreads();
  if (warp_id_of(tid) < NCH) {
    // ---------------------------------------------------------------- chasers
    const int cw = warp_id_of(tid), lane0 = tid & 31;
    __shared__ int s_sw[8];              // sweep: 0 go, 1 nbs, 2 l, 3 nn, 4 m, 5 fail
    __shared__ int s_wok[2];             // per window parity: hand-off waits succeeded
    __shared__ float s_tr[NCH], s_det[NCH];
    float anorm = 0.f;
    if (cw == 0) {
      for (int e2 = lane0; e2 < n * n; e2 += 32) {
        const int r = e2 / n, c = e2 % n;
        if (c >= r - 1) anorm += fabsf(A[r * ld + c]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) anorm += __shfl_xor_sync(0xffffffffu, anorm, o);
      if (lane0 == 0) sh[8] = anorm;
    }
    // warp 0's iteration state; the sweep parameters reach the other chasers via s_sw
    int nn = n - 1, its = 0, total_its = 0, fail = 0, wdx = 0;
    int ll = 0, m = 0, nbs = 1, k0 = 0, b = 0;
    bool in_sweep = false, cont = false;
    const int itmax = 30 * max(10, n);
    while (true) {
      if (!in_sweep) {
        if (cw == 0) {
          // every posted window must be applied before the matrix is read outside a window
          if (!warp_wait_geq(&s_applied, wdx)) fail = 2;
          int l2 = 0, mm = 0, nb_new = 1;
          while (!in_sweep && nn >= 0 && !fail) {
            l2 = 0;
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
            const bool excep = its == 10 || its == 20;
            ++its;
            ++total_its;
            if (NCH > 1 && nn - l2 + 1 >= NMIN_MB) {
              // several bulges: shift pair q = the trailing 2x2 diagonal block q (trace and
              // determinant); bulges enter at the top of the active block
              nb_new = NCH;
              if (lane0 < NCH) {
                const int q = lane0, r0 = nn - 2 * q - 1;
                float tr, de;
                if (excep) {
                  const float s0 = fabsf(A[nn * ld + nn - 1]) + fabsf(A[(nn - 1) * ld + nn - 2]);
                  tr = 1.5f * s0;
                  de = s0 * s0;
                } else {
                  const float a = A[r0 * ld + r0], bq = A[r0 * ld + r0 + 1];
                  const float c = A[(r0 + 1) * ld + r0], d = A[(r0 + 1) * ld + r0 + 1];
                  tr = a + d;
                  de = a * d - bq * c;
                }
                s_tr[q] = tr;
                s_det[q] = de;
              }
              mm = l2;
            } else {
              nb_new = 1;
              float x = A[nn * ld + nn], y = A[(nn - 1) * ld + nn - 1];
              float w = A[nn * ld + nn - 1] * A[(nn - 1) * ld + nn];
              if (excep) {
                const float s0 = fabsf(A[nn * ld + nn - 1]) + fabsf(A[(nn - 1) * ld + nn - 2]);
                x = y = 0.75f * s0;
                w = -0.4375f * s0 * s0;
              }
            // start of the bulge: the largest mm in [l2, nn-2] where two consecutive
            // subdiagonals are negligible relative to the shift vector (mm = l2 always
            // qualifies); lanes test 32 candidates at a time
            mm = l2;
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
              if (lane0 == 0) { s_sh[0] = pp; s_sh[1] = qq; s_sh[2] = rr; }
            }
            __syncwarp();
            for (int r = mm + 2 + lane0; r <= nn; r += 32) {
              A[r * ld + r - 2] = 0.f;
              if (r != mm + 2) A[r * ld + r - 3] = 0.f;
            }
            __syncwarp();
            in_sweep = true;
          }
          if (lane0 == 0) {
            s_sw[0] = (in_sweep && !fail) ? 1 : 0;
            s_sw[1] = nb_new;
            s_sw[2] = l2;
            s_sw[3] = nn;
            s_sw[4] = mm;
            s_sw[5] = fail;
          }
        }
        chaser_sync();
        if (!s_sw[0]) {
          fail = s_sw[5];
          break;
        }
        nbs = s_sw[1];
        ll = s_sw[2];
        nn = s_sw[3];
        m = s_sw[4];
        k0 = m;     // leading bulge position at the first chain step
        b = m;
        in_sweep = true;
        cont = false;
        chaser_sync();   // s_sw is rewritten only after every chaser has read it
      }
      const int cur = wdx & 1;
      float* Zb = Zbuf + cur * WN * (WN + 4);
      const int e = min(b + WN, n);
      // hand-off checks and the identity factor (warp 0), then the previous window's left
      // transformation on its rows in the columns of this window (every chaser)
      if (cw == 0) {
        bool ok = warp_wait_geq(&s_taken, wdx - 1);
        if (ok && cont) ok = warp_wait_geq(&s_applied, wdx - 1);
        for (int q = 0; q < WN; ++q) Zb[lane0 * (WN + 4) + q] = (q == lane0) ? 1.f : 0.f;
        if (lane0 == 0) s_wok[cur] = ok ? 1 : 0;   // rewritten two windows later, after
      }                                              // every chaser passed the next barrier
      chaser_sync();
      if (!s_wok[cur]) {
        fail = 2;
        break;
      }
      if (cont) {
        // H[pb:pe, pe:pc] = Zp^T H[pb:pe, pe:pc]: lane = column, chaser cw = output rows
        // [RPW cw, RPW cw + RPW); every chaser reads the block before any writes it
        constexpr int RPW = (WN + NCH - 1) / NCH;
        const int pb = s_desc[cur ^ 1][0], pe = s_desc[cur ^ 1][1], pc = s_desc[cur ^ 1][3];
        const int pw = pe - pb;
        const float* Zp = Zbuf + (cur ^ 1) * WN * (WN + 4);
        const int c = pe + lane0;
        const bool mine = c < pc;
        const int i0 = cw * RPW;
        float out[RPW];
#pragma unroll
        for (int r = 0; r < RPW; ++r) out[r] = 0.f;
#pragma unroll 4
        for (int j2 = 0; j2 < pw; ++j2) {
          const float a = mine ? A[(pb + j2) * ld + c] : 0.f;
          const float* zr = Zp + j2 * (WN + 4) + i0;
#pragma unroll
          for (int r = 0; r < RPW; ++r)
            if (i0 + r < WN) out[r] = fmaf(zr[r], a, out[r]);
        }
        chaser_sync();
        if (mine) {
#pragma unroll
          for (int r = 0; r < RPW; ++r)
            if (i0 + r < pw) A[(pb + i0 + r) * ld + c] = out[r];
        }
        chaser_sync();
      }
      int kend;       // positions chased in this window end before kend (single bulge)
      bool next;      // the sweep continues in another window
      int nb_next;    // start row of the next window
      if (nbs == 1) {
        kend = min(b + WB, nn);
        if (cw == 0) {
            for (int kk = b; kk < kend; ++kk) {
              const bool three = kk != nn - 1;
              // loads that do not depend on this step's reflector, issued together: the
              // previous step's column update was published by its closing __syncwarp
              const int j = b + lane0;
              const bool row_lane = j >= kk && j < e;
              float a0 = 0.f, a1 = 0.f, a2 = 0.f;
              if (row_lane) {
                a0 = A[kk * ld + j];
                a1 = A[(kk + 1) * ld + j];
                a2 = three ? A[(kk + 2) * ld + j] : 0.f;
              }
              const int kl = kk - b;
              float* zr = Zb + lane0 * (WN + 4);
              const float z0 = zr[kl], z1 = zr[kl + 1];
              const float z2 = three ? zr[kl + 2] : 0.f;
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
              float w0 = 0.f, w1 = 0.f, w2 = 0.f, u1 = 0.f, u2 = 0.f;
              if (go) {
                pp += s;
                const float ip = __fdividef(1.f, pp);
                w0 = pp * is;
                w1 = qq * is;
                w2 = three ? rr * is : 0.f;
                u1 = qq * ip;
                u2 = three ? rr * ip : 0.f;
                // row modification inside the window: columns kk .. e-1
                if (row_lane) {
                  const float t = a0 + u1 * a1 + u2 * a2;
                  A[kk * ld + j] = a0 - t * w0;
                  A[(kk + 1) * ld + j] = a1 - t * w1;
                  if (three) A[(kk + 2) * ld + j] = a2 - t * w2;
                }
                // the same transformation accumulated in Zb (window coordinates)
                const float t = w0 * z0 + w1 * z1 + w2 * z2;
                zr[kl] = z0 - t;
                zr[kl + 1] = z1 - t * u1;
                if (three) zr[kl + 2] = z2 - t * u2;
              }
              __syncwarp();
              if (go) {
                // A[kk][kk-1]: read by every lane above, by no lane from here on in this step
                if (lane0 == 0) {
                  if (kk == m) {
                    if (ll != m) A[kk * ld + kk - 1] = -A[kk * ld + kk - 1];
                  } else {
                    A[kk * ld + kk - 1] = -s * xs;
                  }
                }
                // column modification inside the window: rows b .. min(nn, kk+3)
                const int i2 = b + lane0;
                if (i2 <= min(nn, kk + 3)) {
                  const float b0 = A[i2 * ld + kk], b1 = A[i2 * ld + kk + 1];
                  const float b2 = three ? A[i2 * ld + kk + 2] : 0.f;
                  const float t = w0 * b0 + w1 * b1 + w2 * b2;
                  A[i2 * ld + kk] = b0 - t;
                  A[i2 * ld + kk + 1] = b1 - t * u1;
                  if (three) A[i2 * ld + kk + 2] = b2 - t * u2;
                }
              }
              __syncwarp();
            }
        }
        next = kend <= nn - 1;
        nb_next = kend;
      } else {
        // ---- chain of nbs bulges: bulge j at position k0 - 3 j, active while in [ll, nn-1].
        //  One chain step: every chaser computes its bulge's reflector and applies it to the
        //  rows (the rows of different bulges are disjoint), then, after a barrier, to the
        //  columns (disjoint too); left and right transformations commute, so this equals
        //  the bulges moving one after another.
        float w0 = 0.f, w1 = 0.f, w2 = 0.f, u1 = 0.f, u2 = 0.f;
        while (true) {
          // the lowest active bulge must stay inside the window
          const int lead = min(k0, nn - 1);
          const int jl = (k0 - lead + 2) / 3;               // first bulge at or above nn-1
          const int klead = k0 - 3 * jl;
          if (jl >= nbs || klead < ll) break;               // every bulge has left
          if (min(klead + 3, nn) >= e) break;               // window full
          const int k = k0 - 3 * cw;
          const bool act = cw < nbs && k >= ll && k <= nn - 1;
          const bool three = k != nn - 1;
          bool go = false;
          float s = 0.f, xs = 1.f;
          if (act) {
            const int j = b + lane0;
            const bool row_lane = j >= k && j < e;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            if (row_lane) {
              a0 = A[k * ld + j];
              a1 = A[(k + 1) * ld + j];
              a2 = three ? A[(k + 2) * ld + j] : 0.f;
            }
            const int kl = k - b;
            float* zr = Zb + lane0 * (WN + 4);
            const float z0 = zr[kl], z1 = zr[kl + 1];
            const float z2 = three ? zr[kl + 2] : 0.f;
            float pp, qq, rr;
            if (k == ll) {
              // bulge entry: first column of (H - s1 I)(H - s2 I) from this bulge's shifts
              const float tr = s_tr[cw], de = s_det[cw];
              const float h00 = A[ll * ld + ll], h01 = A[ll * ld + ll + 1];
              const float h10 = A[(ll + 1) * ld + ll], h11 = A[(ll + 1) * ld + ll + 1];
              const float h21 = A[(ll + 2) * ld + ll + 1];
              pp = h00 * h00 + h01 * h10 - tr * h00 + de;
              qq = h10 * (h00 + h11 - tr);
              rr = three ? h21 * h10 : 0.f;
            } else {
              pp = A[k * ld + k - 1];
              qq = A[(k + 1) * ld + k - 1];
              rr = three ? A[(k + 2) * ld + k - 1] : 0.f;
            }
            xs = fabsf(pp) + fabsf(qq) + fabsf(rr);
            if (xs != 0.f) {
              const float ix = __fdividef(1.f, xs);
              pp *= ix; qq *= ix; rr *= ix;
              const float ss = pp * pp + qq * qq + rr * rr;
              if (ss > 0.f) {
                go = true;
                const float rs = rsqrtf(ss);
                s = sgnf(ss * rs, pp);
                const float is = sgnf(rs, pp);
                pp += s;
                const float ip = __fdividef(1.f, pp);
                w0 = pp * is;
                w1 = qq * is;
                w2 = three ? rr * is : 0.f;
                u1 = qq * ip;
                u2 = three ? rr * ip : 0.f;
              }
            }
            if (go) {
              if (row_lane) {
                const float t = a0 + u1 * a1 + u2 * a2;
                A[k * ld + j] = a0 - t * w0;
                A[(k + 1) * ld + j] = a1 - t * w1;
                if (three) A[(k + 2) * ld + j] = a2 - t * w2;
              }
              const float t = w0 * z0 + w1 * z1 + w2 * z2;
              zr[kl] = z0 - t;
              zr[kl + 1] = z1 - t * u1;
              if (three) zr[kl + 2] = z2 - t * u2;
            }
            __syncwarp();
            // column k-1 below the subdiagonal is now annihilated: store it (the next bulge
            // of the chain reaches position k within this sweep and reads these entries)
            if (go && k != ll) {
              if (lane0 == 0) A[k * ld + k - 1] = -s * xs;
              if (lane0 == 1) A[(k + 1) * ld + k - 1] = 0.f;
              if (lane0 == 2 && three) A[(k + 2) * ld + k - 1] = 0.f;
            }
          }
          chaser_sync();
          if (act && go) {
            const int i2 = b + lane0;
            if (i2 <= min(nn, k + 3)) {
              const float b0 = A[i2 * ld + k], b1 = A[i2 * ld + k + 1];
              const float b2 = three ? A[i2 * ld + k + 2] : 0.f;
              const float t = w0 * b0 + w1 * b1 + w2 * b2;
              A[i2 * ld + k] = b0 - t;
              A[i2 * ld + k + 1] = b1 - t * u1;
              if (three) A[i2 * ld + k + 2] = b2 - t * u2;
            }
          }
          chaser_sync();
          ++k0;
        }
        const int ktr = k0 - 3 * (nbs - 1);
        next = ktr <= nn - 1;
        nb_next = max(ll, ktr);
        kend = nb_next;
      }
      // post the window
      if (cw == 0) {
        if (lane0 == 0) {
          s_desc[cur][0] = b;
          s_desc[cur][1] = e;
          s_desc[cur][2] = kend;
          s_desc[cur][3] = next ? min(nb_next + WN, n) : e;
        }
        __syncwarp();
        __threadfence_block();
        if (lane0 == 0) s_posted = wdx + 1;
      }
      ++wdx;
      b = nb_next;
      in_sweep = next;
      cont = next;
    }
    if (cw == 0) {
      __syncwarp();
      if (lane0 == 0) {
        s_nwin = wdx;
        s_state = fail ? 2 : 1;
        if (fail == 2) atomicOr(p.status, DEV_TIMEOUT);
      }
    }
    (void)total_its;
  } else {
    // ---------------------------------------------------------------- helpers
    const int nh = nth - 32 * NCH;
    const int h = tid - 32 * NCH;
    for (int v = 0;; ++v) {
      if (h == 0) {
        int go = 0;
        const uint64_t t0 = bw::global_ns();
        while (true) {
          if (s_posted > v) { go = 1; break; }
          if (s_state != 0) break;
          if (bw::global_ns() - t0 > 2000000000ull) {
            atomicOr(p.status, DEV_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
        s_go = go;
      }
      helper_sync(nh);
      if (!s_go) break;
      __threadfence_block();
      const int cur = v & 1;
      const int bb = s_desc[cur][0], ee = s_desc[cur][1], cs = s_desc[cur][3];
      const int ww = ee - bb;
      const float* Zb = Zbuf + cur * WN * (WN + 4);
      for (int e2 = h; e2 < WN * WN; e2 += nh) {
        const int i2 = e2 / WN, j2 = e2 % WN;
        ZT[i2 * (WN + 4) + j2] = Zb[j2 * (WN + 4) + i2];
      }
      helper_sync(nh);
      if (h == 0) s_taken = v + 1;
      // log the factor (row-major Zb, from the transposed copy)
      if (v < zlog_cap(n)) {
        float* rec = zlog + (size_t)v * ZREC;
        for (int e2 = h; e2 < WN * WN; e2 += nh) rec[8 + e2] = ZT[(e2 % WN) * (WN + 4) + e2 / WN];
        if (h == 0) {
          rec[0] = __int_as_float(bb);
          rec[1] = __int_as_float(ee);
        }
      }
      const int n_right = n - cs, n_top = bb;
      for (int task = h; task < n_right + n_top; task += nh) {
        const bool right = task < n_right;
        // right: column cs + task of rows [bb, ee); top: row task - n_right, columns [bb, ee)
        float* base = right ? A + bb * ld + cs + task : A + (task - n_right) * ld + bb;
        const int stride = right ? ld : 1;
        float in[WN];
#pragma unroll
        for (int j2 = 0; j2 < WN; ++j2) in[j2] = (j2 < ww) ? base[j2 * stride] : 0.f;
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
          for (int u = 0; u < 4; ++u)
            if (i0 + u < ww) base[(i0 + u) * stride] = acc[u];
        }
      }
      helper_sync(nh);
      if (h == 0) {
        __threadfence_block();
        s_applied = v + 1;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    shi[4] = (s_state == 2 || s_nwin > zlog_cap(n)) ? 1 : 0;
    shi[5] = s_nwin;
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
  const int warp = tid >> 5, lane = tid & 31;
  const int ncx = 2 * npole;   // columns of X
  constexpr int VEC_WARPS = 8;  // warps with a vector buffer (shared memory)
  float* xr = smem + xbuf_off + (warp % VEC_WARPS) * 2 * n;
  float* xi = xr + n;
  for (int j = warp; j < npole && warp < VEC_WARPS; j += VEC_WARPS) {
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
    const float tiny = FLT_EPSILON * sh[8] + FLT_MIN;   // sh[8] = ||H||_1 (entrywise)
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

  // ---- 6. pole records, largest frequency last; MPC and MPD follow with the mode shapes
  //         (k_eig_vectors)
  __shared__ int s_src[256];
  for (int j = tid; j < npole; j += nth) s_src[s_rank[j]] = j;
  __syncthreads();
  for (int j = tid; j < n_slots; j += nth) {
    ssi_pole rec;
    rec.lag = p.lt.i[t];
    rec.order = n;
    rec.index = j;
    rec.mpc = 0.f;
    rec.mpd = 0.f;
    if (failed || j >= npole) {
      rec.f_hz = 0.f; rec.xi = 0.f; rec.mu_re = 0.f; rec.mu_im = 0.f;
      rec.flags = failed ? SSI_POLE_NOTCONV : 0u;
    } else {
      const int src = s_src[j];
      const double mr = s_mur[src], mu_i = s_mui[src];
      const double lr = 0.5 * log(mr * mr + mu_i * mu_i) / p.dt, li = atan2(mu_i, mr) / p.dt;
      const double lam = sqrt(lr * lr + li * li);
      rec.f_hz = (float)(lam / (2.0 * 3.14159265358979323846));
      rec.xi = lam > 0 ? (float)(-lr / lam) : 0.f;
      rec.mu_re = (float)mr;
      rec.mu_im = (float)mu_i;
      rec.flags = SSI_POLE_VALID;
    }
    poles[j] = rec;
  }
  if (tid == 0) {
    hdr[0] = failed ? 0 : npole;
    hdr[1] = shi[5];
    hdr[2] = failed ? 1 : 0;
  }
  (void)k;
  (void)l;
}

// ------------------------------------------------------------------ mode shapes
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(bw::smem_u32(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(bw::smem_u32(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One CTA per (lag, order, block of VEC_COLS columns of X = 16 poles), largest orders
// first.  The block of X (eigenvectors of T) is carried back to eigenvectors of A~:
// the logged window factors in reverse order (X[b:e] = Zb X[b:e]), then the Hessenberg
// reflectors in reverse order; then Phi = U[:l, :n] X, its normalisation (unit norm,
// largest component real), MPC and MPD of every pole of the block.  Window records and
// reflectors stream through shared-memory rings filled by cp.async, several ahead.
constexpr int VEC_THREADS = 256;
constexpr int XLD = VEC_COLS + 1;   // shared-memory row stride of the X block
constexpr int ZRING = 4;            // window records in flight
constexpr int VRING = 4;            // Hessenberg reflectors in flight

__global__ void __launch_bounds__(VEC_THREADS)
    k_eig_vectors(const EigParams* __restrict__ P, const int4* __restrict__ items) {
  extern __shared__ float vsm[];
  int job = 0, t, q, mi;
  if (items) {
    // a batch: (job, order index, lag, column block) from the table
    const int4 it = items[blockIdx.x];
    job = it.x;
    mi = it.y;
    t = it.z;
    q = it.w;
  } else {
    // block -> (lag, order, column block), largest orders first
    const EigParams& p0 = P[0];
    t = blockIdx.x % p0.lt.n_lags;
    q = blockIdx.x / p0.lt.n_lags;   // block index within the lag, largest orders first
    mi = p0.n_orders - 1;
    while (mi > 0 && q >= p0.vec_blocks[mi]) {
      q -= p0.vec_blocks[mi];
      --mi;
    }
  }
  const EigParams& p = P[job];
  const int n = p.orders[mi];
  const int k = p.lt.k, l = p.lt.l;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = VEC_THREADS / 32;
  const float* work = p.work + (size_t)t * p.work_per_lag + p.work_off[mi];
  const int* hdr = reinterpret_cast<const int*>(work);
  const float* hv = work + EIG_HDR;
  const float* X = hv + (size_t)n * n;
  const float* zlog = X + (size_t)n * n;
  const int npole = hdr[0], n_win = min(hdr[1], (int)zlog_cap(n));
  const int ncx = 2 * npole;
  const int c0 = q * VEC_COLS;                   // first column of this block
  const int nc = max(0, min(VEC_COLS, ncx - c0));
  const int slot0 = c0 / 2;
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  float* phi_out = p.phi + ((size_t)t * p.slots_per_lag + p.slot_off[mi]) * 2 * l;
  const float* U = p.lt.U[t];
  const int n_slots_blk = min(VEC_COLS / 2, n / 2 - slot0);
  if (nc == 0) {
    // no pole of this block has a shape: zero their mode shapes
    for (int e = tid; e < n_slots_blk * 2 * l; e += VEC_THREADS)
      phi_out[(size_t)slot0 * 2 * l + e] = 0.f;
    return;
  }
  float* Xs = vsm;                                         // n x XLD
  float* Zs = Xs + (((size_t)n * XLD + 3) & ~size_t(3));   // ZRING window records
  float* vs = Zs + ZRING * ZREC;                           // VRING reflectors of N_MAX
  for (int e = tid; e < n * VEC_COLS; e += VEC_THREADS) {
    const int r = e / VEC_COLS, c = e % VEC_COLS;
    Xs[r * XLD + c] = (c < nc) ? X[(size_t)r * ncx + c0 + c] : 0.f;
  }
  // 1. window factors in reverse order; warp w owns rows 4w..4w+3 of the window, lane the
  //    column.  Record w goes to ring slot w % ZRING, ZRING - 1 records ahead; a slot is
  //    refilled only after the barrier that follows every thread's last use of it.
  {
    auto issue = [&](int w) {
      if (w >= 0) {
        const float* src = zlog + (size_t)w * ZREC;
        float* dst = Zs + (w % ZRING) * ZREC;
        for (int e = tid; e < ZREC / 4; e += VEC_THREADS) cp_async16(dst + 4 * e, src + 4 * e);
      }
      cp_async_commit();
    };
    for (int a = 1; a < ZRING; ++a) issue(n_win - a);
    for (int w = n_win - 1; w >= 0; --w) {
      cp_async_wait<ZRING - 2>();   // record w has landed (the newer ZRING - 2 may not)
      __syncthreads();
      issue(w - (ZRING - 1));       // into the slot of record w + 1, done by every thread
      const float* rec = Zs + (w % ZRING) * ZREC;
      const float* Zc = rec + 8;
      const int bb = __float_as_int(rec[0]), ee = __float_as_int(rec[1]), ww = ee - bb;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int i0 = 4 * warp;
      for (int j4 = 0; j4 < ww; j4 += 4) {
        float xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = (j4 + u < ww) ? Xs[(bb + j4 + u) * XLD + lane] : 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 z = *reinterpret_cast<const float4*>(Zc + (i0 + r) * WN + j4);
          acc[r] = fmaf(z.x, xv[0], fmaf(z.y, xv[1], fmaf(z.z, xv[2], fmaf(z.w, xv[3], acc[r]))));
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + r < ww) Xs[(bb + i0 + r) * XLD + lane] = acc[r];
    }
    cp_async_wait<0>();
  }
  __syncthreads();
  // 2. Hessenberg reflectors in reverse order: 8 threads per column split the rows; row j
  //    of the reflector log goes to ring slot j % VRING, VRING - 1 reflectors ahead
  {
    const int c = tid & 31, g = tid >> 5;   // column, row group
    __shared__ float s_part[VEC_THREADS];
    auto issue = [&](int j) {
      if (j >= 0)
        for (int r = tid; r < n; r += VEC_THREADS)
          cp_async4(vs + (j % VRING) * N_MAX + r, hv + (size_t)j * n + r);
      cp_async_commit();
    };
    for (int a = 0; a < VRING - 1; ++a) issue(n - 3 - a);
    for (int j = n - 3; j >= 0; --j) {
      cp_async_wait<VRING - 2>();   // reflector j has landed
      __syncthreads();
      issue(j - (VRING - 1));       // into the slot of reflector j + 1, done by every thread
      const float* v = vs + (j % VRING) * N_MAX;
      const int len = n - j - 1;
      const float beta = v[n - 1];
      float part = 0.f;
      if (beta != 0.f)
        for (int r = g; r < len; r += 8) part = fmaf(v[r], Xs[(j + 1 + r) * XLD + c], part);
      s_part[tid] = part;
      __syncthreads();
      if (beta != 0.f) {
        float dot = 0.f;
#pragma unroll
        for (int g2 = 0; g2 < 8; ++g2) dot += s_part[g2 * 32 + c];
        const float sc = dot * beta;
        for (int r = g; r < len; r += 8) Xs[(j + 1 + r) * XLD + c] -= sc * v[r];
      }
    }
    cp_async_wait<0>();
  }
  __syncthreads();
  // 3. Phi = U[:l, :n] X for the block: thread per channel, all columns in registers
  for (int ch = tid; ch < l; ch += VEC_THREADS) {
    float acc[VEC_COLS];
#pragma unroll
    for (int c = 0; c < VEC_COLS; ++c) acc[c] = 0.f;
    const float* urow = U + (size_t)ch * k;
    for (int a = 0; a < n; ++a) {
      const float u = __ldg(urow + a);
      const float* xr = Xs + a * XLD;
#pragma unroll
      for (int c = 0; c < VEC_COLS; ++c) acc[c] = fmaf(u, xr[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < VEC_COLS; ++c)
      if (c < nc) phi_out[(size_t)(slot0 + c / 2) * 2 * l + 2 * ch + (c & 1)] = acc[c];
  }
  // slots of the block without a pole
  for (int e = tid; e < (n_slots_blk - nc / 2) * 2 * l; e += VEC_THREADS)
    phi_out[(size_t)(slot0 + nc / 2) * 2 * l + e] = 0.f;
  __syncthreads();
  // 4. per pole: scale by conj(largest)/|largest| / ||phi||, MPC, MPD
  for (int jj = warp; jj < nc / 2; jj += nwarps) {
    const int j = slot0 + jj;
    float* ph = phi_out + (size_t)j * 2 * l;
    float nrm2 = 0.f, best = -1.f, bre = 1.f, bim = 0.f;
    for (int c = lane; c < l; c += 32) {
      const float sr = ph[2 * c], si = ph[2 * c + 1];
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
      poles[j].mpc = mpc;
      poles[j].mpd = wsum > 0.f ? (asum / wsum) / 1.5707963267948966f : 0.f;
    }
  }
}

}  // namespace

// The per-lag factorisation in FP64 (the FP64 realisation path, csrc/eig64.cu); R in the
// lags' global scratch Fs (k (k + 1) + k doubles per lag).
ssi_status lag_factor64_launch(const double* GH, int k, int n_lags, double* RM, double* Fs, int* status,
                               cudaStream_t stream) {
  k_lag_factor<true, double><<<n_lags, 1024, 0, stream>>>(GH, k, RM, Fs, status);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

// a prepared realisation: the parameter block of its eigen-decompositions (host copy and
// device copy in the job's scratch) and its largest order
struct RealizePrep {
  EigParams ep;
  EigParams* dev;
  int max_order;
};

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
  WsPlan w;
  w.add<float>((size_t)n_lags * std::max(n_chunks, 1) * 2 * k * k);  // Gram partials
  w.add<float>((size_t)n_lags * 2 * k * k);                          // G | H
  w.add<float>((size_t)n_lags * 2 * k * k);                          // Rinv | M
  w.add<float>((size_t)n_lags * work);                               // eig scratch
  if (k > FACTOR_SMEM_K) w.add<float>((size_t)n_lags * ((size_t)k * (k + 1) + k));  // factors
  w.add<EigParams>(1);                                               // eig launch parameters
  r.ws_bytes = w.bytes;
  return r;
}

ssi_status realize_ws(ssi_ctx* ctx, Workspace& ws, const RealizePlan& r, const int* lags,
                      const float* const* U, const int* orders, double dt, ssi_pole* poles,
                      float* phi, int* dev_status, cudaStream_t stream, RealizePrep** defer) {
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
  EigParams* ep_dev = ws.take<EigParams>(1);
  float* Rg = (k > FACTOR_SMEM_K) ? ws.take<float>((size_t)r.n_lags * ((size_t)k * (k + 1) + k))
                                  : nullptr;
  if (!partial || !GH || !RM || !eigw || !ep_dev || (k > FACTOR_SMEM_K && !Rg)) {
    set_error("realize: workspace too small");
    return SSI_E_NOMEM;
  }
  const int tiles = (int)ceil_div(k, 64);
  dim3 g1((unsigned)(tiles * tiles), (unsigned)n_chunks, (unsigned)(2 * r.n_lags));
  count_launches(ctx, 3);   // Gram, its reduction, the factorisation (the eig launches count their own)
  {
  ProfScope ps(ctx, ST_GRAM, stream);
  k_gram_gh<<<g1, 256, 0, stream>>>(lt, n_chunks, partial);
  SSI_CUDA(cudaGetLastError());
  k_gram_reduce<<<ctx->num_sms * 4, 256, 0, stream>>>(partial, r.n_lags, n_chunks, k, GH);
  SSI_CUDA(cudaGetLastError());
  const size_t fsmem = Rg ? 0 : ((size_t)k * (k + 1) + k) * sizeof(float);
  if (Rg) {
    k_lag_factor<true, float><<<r.n_lags, 1024, 0, stream>>>(GH, k, RM, Rg, dev_status);
  } else {
    SSI_CUDA(cudaFuncSetAttribute(k_lag_factor<false, float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(220 * 1024)));
    k_lag_factor<false, float><<<r.n_lags, 1024, fsmem, stream>>>(GH, k, RM, nullptr, dev_status);
  }
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
  int vec_total = 0;
  for (int m = 0; m < r.n_orders; ++m) {
    ep.vec_blocks[m] = (int)ceil_div(orders[m], VEC_COLS);
    vec_total += ep.vec_blocks[m];
  }
  ep.vec_blocks_per_lag = vec_total;
  // the parameter block in device memory, behind the factorisations on the stream (a
  // pageable source is staged before the call returns)
  SSI_CUDA(cudaMemcpyAsync(ep_dev, &ep, sizeof(EigParams), cudaMemcpyHostToDevice, stream));
  RealizePrep* prep = new RealizePrep{ep, ep_dev, r.max_order};
  if (defer) {
    *defer = prep;
    return SSI_OK;
  }
  const ssi_status st = realize_batch_launch(ctx, &prep, 1, nullptr, 0, stream);
  delete prep;
  return st;
}

// Launches of the eigen-decompositions.  The CTAs' layouts differ by order, so each launch
// reserves its largest; orders above SMEM_N_MAX run in their own launch, first.  One
// realisation (n == 1) indexes its items by CTA.  A batch lists every job's (job, order
// index, lag[, column block]) in `table` (device memory of realize_batch_table_bytes),
// largest orders first across the jobs, after the jobs' parameter blocks.
ssi_status realize_batch_launch(ssi_ctx* ctx, RealizePrep* const* preps, int n, void* table,
                                size_t table_cap, cudaStream_t stream) {
  SSI_CHECK(n >= 1, "realize: no realisation to launch");
  int esmem_s = 0, esmem_b = 0, max_order = 0;
  // items as (job, order index, lag, order); vector blocks as (job, order index, lag,
  // column block), with their orders alongside for the sort
  std::vector<int4> small, big, vec;
  std::vector<int> vec_order;
  for (int j = 0; j < n; ++j) {
    const EigParams& ep = preps[j]->ep;
    max_order = std::max(max_order, preps[j]->max_order);
    for (int m = 0; m < ep.n_orders; ++m) {
      const int o = ep.orders[m];
      if (o > SMEM_N_MAX) esmem_b = std::max(esmem_b, eig_smem_floats(o));
      else esmem_s = std::max(esmem_s, eig_smem_floats(o));
      for (int t = 0; t < ep.lt.n_lags; ++t) {
        (o > SMEM_N_MAX ? big : small).push_back(make_int4(j, m, t, o));
        for (int q = 0; q < ep.vec_blocks[m]; ++q) {
          vec.push_back(make_int4(j, m, t, q));
          vec_order.push_back(o);
        }
      }
    }
  }
  const int n_small = (int)small.size(), n_big = (int)big.size(), n_vec = (int)vec.size();
  const EigParams* P = preps[0]->dev;
  const int4 *t_eig = nullptr, *t_vec = nullptr;
  if (n > 1) {
    // largest orders first across the jobs (stable among equal orders)
    auto by_order = [](const int4& a, const int4& b) { return a.w > b.w; };
    std::stable_sort(small.begin(), small.end(), by_order);
    std::stable_sort(big.begin(), big.end(), by_order);
    std::vector<int> idx(vec.size());
    for (size_t e = 0; e < idx.size(); ++e) idx[e] = (int)e;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return vec_order[a] > vec_order[b]; });
    // the batch's parameter blocks side by side, then the eig items (big, then small: one
    // table serves both launches) and the vector blocks
    const size_t need = realize_batch_table_bytes(preps, n);
    SSI_CHECK(table && table_cap >= need, "realize: batch table too small");
    std::vector<char> host(need);
    size_t off = 0;
    for (int j = 0; j < n; ++j, off += sizeof(EigParams))
      std::memcpy(host.data() + off, &preps[j]->ep, sizeof(EigParams));
    char* base = static_cast<char*>(table);
    P = reinterpret_cast<const EigParams*>(base);
    t_eig = reinterpret_cast<const int4*>(base + off);
    for (const int4& v : big) { std::memcpy(host.data() + off, &v, sizeof(int4)); off += sizeof(int4); }
    for (const int4& v : small) { std::memcpy(host.data() + off, &v, sizeof(int4)); off += sizeof(int4); }
    t_vec = reinterpret_cast<const int4*>(base + off);
    for (int e : idx) { std::memcpy(host.data() + off, &vec[e], sizeof(int4)); off += sizeof(int4); }
    SSI_CUDA(cudaMemcpyAsync(table, host.data(), off, cudaMemcpyHostToDevice, stream));
  }
  SSI_CUDA(cudaFuncSetAttribute(k_eig<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(std::max(esmem_s, 1) * sizeof(float))));
  SSI_CUDA(cudaFuncSetAttribute(k_eig<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(std::max(esmem_b, 1) * sizeof(float))));
  const size_t vsmem =
      ((((size_t)max_order * XLD + 3) & ~size_t(3)) + ZRING * ZREC + VRING * N_MAX) * sizeof(float);
  SSI_CUDA(cudaFuncSetAttribute(k_eig_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem));
  {
    ProfScope ps_eig(ctx, ST_EIG, stream);
    if (n_big > 0) {
      count_launches(ctx, 1);
      k_eig<true><<<n_big, EIG_THREADS, (size_t)esmem_b * sizeof(float), stream>>>(P, t_eig, 0);
      SSI_CUDA(cudaGetLastError());
    }
    if (n_small > 0) {
      count_launches(ctx, 1);
      k_eig<false><<<n_small, EIG_THREADS, (size_t)esmem_s * sizeof(float), stream>>>(P, t_eig,
                                                                                      n_big);
      SSI_CUDA(cudaGetLastError());
    }
  }
  ProfScope ps_vec(ctx, ST_EIG_VEC, stream);
  count_launches(ctx, 1);
  k_eig_vectors<<<n_vec, VEC_THREADS, vsmem, stream>>>(P, t_vec);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

size_t realize_batch_table_bytes(RealizePrep* const* preps, int n) {
  size_t items = 0;
  for (int j = 0; j < n; ++j) {
    const EigParams& ep = preps[j]->ep;
    for (int m = 0; m < ep.n_orders; ++m) items += (size_t)ep.lt.n_lags * (1 + ep.vec_blocks[m]);
  }
  return (size_t)n * sizeof(EigParams) + items * sizeof(int4);
}

void realize_prep_free(RealizePrep* p) { delete p; }

}  // namespace ssi

extern "C" ssi_status ssi_realize_batch(ssi_ctx* ctx, int n_lags, const int* lags,
                                        const double* const* U, int l, int k, const int* orders,
                                        int n_orders, double dt, ssi_small_precision small,
                                        ssi_pole* poles, float* phi, void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && lags && U && orders && poles && phi, "ssi_realize_batch: null pointer");
  SSI_CHECK(n_lags >= 1 && n_lags <= MAX_LAGS, "ssi_realize_batch: 1 <= n_lags <= %d", MAX_LAGS);
  SSI_CHECK(n_orders >= 1 && n_orders <= 512, "ssi_realize_batch: 1 <= n_orders <= 512");
  SSI_CHECK(l >= 1 && k >= 2 && dt > 0, "ssi_realize_batch: bad l/k/dt");
  SSI_CHECK(k <= N_MAX, "ssi_realize_batch: k=%d > %d not supported", k, N_MAX);
  SSI_CHECK(small == SSI_SMALL_FP32 || small == SSI_SMALL_FP64,
            "ssi_realize_batch: bad small-problem precision");
  for (int t = 0; t < n_lags; ++t) {
    SSI_CHECK(lags[t] >= 2, "ssi_realize_batch: lag %d < 2", lags[t]);
    SSI_CHECK(U[t], "ssi_realize_batch: null U[%d]", t);
    SSI_CHECK((int64_t)l * lags[t] >= k, "ssi_realize_batch: l*i < k");
  }
  for (int m = 0; m < n_orders; ++m) {
    SSI_CHECK(orders[m] >= 2 && orders[m] % 2 == 0 && orders[m] <= k,
              "ssi_realize_batch: order %d must be even and in [2, k]", orders[m]);
    SSI_CHECK(orders[m] <= N_MAX, "ssi_realize_batch: order %d > %d not supported", orders[m],
              N_MAX);
    SSI_CHECK(m == 0 || orders[m] > orders[m - 1], "ssi_realize_batch: orders must ascend");
  }
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RealizePlan plan = realize_plan(n_lags, lags, l, k, orders, n_orders);
  if (small == SSI_SMALL_FP64) {
    SSI_TRY(ws_reserve(ctx, ctx->ws, realize64_ws_bytes(n_lags, lags, l, k, orders, n_orders), s));
    SSI_TRY(realize64_ws(ctx, ctx->ws, n_lags, lags, l, k, U, orders, n_orders, plan.slots_per_lag,
                         dt, poles, phi, ctx->dev_status, s));
    return check_dev_status(ctx->dev_status, s);
  }
  // FP32: U rounded once into the auxiliary workspace, then the FP32 path
  size_t u_floats = 0;
  for (int t = 0; t < n_lags; ++t) u_floats += (size_t)round_up((int64_t)l * lags[t] * k, 64);
  SSI_TRY(ws_reserve(ctx, ctx->ws_aux, u_floats * sizeof(float), s));
  std::vector<const float*> U32(n_lags);
  size_t off = 0;
  for (int t = 0; t < n_lags; ++t) {
    float* dst = reinterpret_cast<float*>(ctx->ws_aux.base) + off;
    SSI_TRY(convert_d2f(U[t], (long long)l * lags[t] * k, dst, s));
    U32[t] = dst;
    off += (size_t)round_up((int64_t)l * lags[t] * k, 64);
  }
  SSI_TRY(ws_reserve(ctx, ctx->ws, plan.ws_bytes, s));
  SSI_TRY(realize_ws(ctx, ctx->ws, plan, lags, U32.data(), orders, dt, poles, phi, ctx->dev_status, s));
  return check_dev_status(ctx->dev_status, s);
}
