// Stage (c) in FP64: realisation of every (lag, order) with FP64 least squares and an FP64
// eigensolver (Sec. 2.1: A = (O^to)^+ O^bo, A = Psi M Psi^{-1}, lambda = ln(mu)/dt,
// f = |lambda|/(2 pi), xi = -Re(lambda)/|lambda|, Phi = C Psi).
//
// The formulation is the FP32 path's (csrc/realize.cu): S^{1/2} is a similarity transform
// and is dropped, and one Cholesky factorisation per lag, G = U^to^T U^to = R^T R, serves
// every order through A~_n = (R^{-1})[:n,:n] (R^{-T} H)[:n,:n], H = U^to^T U^bo.
// Kernels:
//   k_gram64      FP64 partial sums of G and H over row chunks
//   k_gram_reduce64  fixed-order sum of the chunks
//   (the factorisation is the FP32 path's k_lag_factor in FP64)
//   k_eig64       one CTA per (lag, order), largest orders first: A~_n, Householder
//                 Hessenberg reduction, double-shift Francis QR to the real Schur form T
//                 (Martin, Peters and Wilkinson's HQR with full-matrix updates), with the
//                 3-element reflector of every bulge step logged; eigenvalues from the
//                 diagonal blocks; pole records
//   k_eigvec64    one CTA per (lag, order, 16 poles): eigenvectors of T by back
//                 substitution, the logged reflectors in reverse, the Hessenberg
//                 reflectors in reverse, Phi = U[:l,:n] x, its normalisation, MPC, MPD
// FP64 instructions issue at about one warp instruction per 16 clocks per SM on this
// part whatever the number of active lanes, so the scalar work of each bulge step is
// done once (warp 0) and broadcast, and the vector kernels put one pole in each lane.
#include <cfloat>

#include <algorithm>

#include "common.cuh"
#include "dfloat.cuh"

namespace ssi {

namespace {

constexpr int MAX_LAGS64 = 64;
struct Lag64Table {
  int n_lags;
  int l, k;
  int i[MAX_LAGS64];
  const double* U[MAX_LAGS64];
};

constexpr int E64_THREADS = 256;
constexpr int V64_POLES = 16;         // poles per eigenvector CTA (one per lane)
constexpr int G64_ROWS = 1024;        // rows per Gram chunk

// scratch of one realisation (doubles): header, T (n x n), Hessenberg reflectors (n x n),
// eigenvalues by frequency rank (mu_re, mu_im, position; 3 x n/2), reflector log
// (log_cap records of 6: k, x, y, z, q, r)
constexpr int H64 = 8;
__host__ __device__ inline long long log_cap64(int n) { return 2LL * n * n + 64; }
__host__ __device__ inline long long eig64_doubles(int n) {
  return H64 + 2LL * n * n + 3LL * (n / 2) + 6LL * log_cap64(n) + 8;
}

// ------------------------------------------------------------------ Gram matrices (FP64)
// partial[t][chunk][which][a][b]: which 0: G = sum_r U[r][a] U[r][b]; 1: H = sum_r U[r][a]
// U[r+l][b]; r in the chunk, r < L - l.  32 x 32 output tile per CTA, 2 x 2 per thread.
__global__ void __launch_bounds__(256) k_gram64(Lag64Table lt, int n_chunks, double* __restrict__ partial) {
  __shared__ double As[32][33];
  __shared__ double Bs[32][33];
  const int k = lt.k, l = lt.l;
  const int tiles = (k + 31) / 32;
  const int ta = blockIdx.x / tiles, tb = blockIdx.x % tiles;
  const int chunk = blockIdx.y;
  const int t = blockIdx.z >> 1, which = blockIdx.z & 1;
  const int L = l * lt.i[t];
  const int r_end = L - l;
  const int r0 = chunk * G64_ROWS, r1 = min(r_end, r0 + G64_ROWS);
  const double* U = lt.U[t];
  const int a0 = ta * 32, b0 = tb * 32;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int shift = which ? l : 0;
  double acc[2][2] = {{0, 0}, {0, 0}};
  for (int rb = r0; rb < r1; rb += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int rr = e / 32, c = e % 32;
      const int r = rb + rr;
      const bool in = r < r1;
      As[rr][c] = (in && a0 + c < k) ? U[(size_t)r * k + a0 + c] : 0.0;
      Bs[rr][c] = (in && b0 + c < k) ? U[(size_t)(r + shift) * k + b0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const double x0 = As[rr][ty * 2], x1 = As[rr][ty * 2 + 1];
      const double y0 = Bs[rr][tx * 2], y1 = Bs[rr][tx * 2 + 1];
      acc[0][0] = fma(x0, y0, acc[0][0]);
      acc[0][1] = fma(x0, y1, acc[0][1]);
      acc[1][0] = fma(x1, y0, acc[1][0]);
      acc[1][1] = fma(x1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  double* out = partial + (((size_t)t * n_chunks + chunk) * 2 + which) * (size_t)k * k;
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const int a = a0 + ty * 2 + x, b = b0 + tx * 2 + y;
      if (a < k && b < k) out[(size_t)a * k + b] = acc[x][y];
    }
}

__global__ void k_gram_reduce64(const double* __restrict__ partial, int n_lags, int n_chunks, int k,
                                double* __restrict__ GH) {
  const long long per = 2LL * k * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * n_lags;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / per, r = e % per;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += partial[((size_t)t * n_chunks + c) * per + r];
    GH[e] = s;
  }
}

// ------------------------------------------------------------------ eig per realisation
struct Eig64Params {
  Lag64Table lt;
  int n_orders;
  int orders[512];
  long long slot_off[512];
  long long slots_per_lag;
  const double* RM;          // [t][2][k][k]: Rinv | M
  double* work;
  long long work_off[512];
  long long work_per_lag;
  double dt;
  ssi_pole* poles;
  float* phi;
  int* status;
  int vec_blocks[512];       // eigenvector CTAs of order m
};

struct Step {
  float2 x, y, z, q, r;   // the bulge reflector in double-float
  int k, three;
};

// Element (i, j) of A during the QR iteration, as a double-float (hi, lo) pair: the full
// row-major matrix in the realisation's scratch (L2), or, for orders up to E64_BAND_N,
// the band j >= i - 3 that the iteration can touch (upper Hessenberg plus the bulge's two
// extra subdiagonals), packed row by row in shared memory.
struct FullA {
  float2* A;
  int ld;
  __device__ __forceinline__ float2& operator()(int i, int j) const { return A[(size_t)i * ld + j]; }
};
struct BandA {
  float2* P;
  const int* base;   // offset of row i's first stored column, max(i - 3, 0)
  __device__ __forceinline__ float2& operator()(int i, int j) const {
    return P[base[i] + j - (i > 3 ? i - 3 : 0)];
  }
};
__host__ __device__ inline int band_doubles(int n) {
  int tot = 0;
  for (int i = 0; i < n; ++i) tot += n - (i > 3 ? i - 3 : 0);
  return tot;
}
constexpr int E64_BAND_N = 224;   // largest order whose band fits in shared memory
constexpr float DF_EPS = 1.42e-14f;   // negligibility threshold of the double-float iteration (2^-46)

// exponent e with 2^e <= x < 2^(e+1)
__device__ __forceinline__ int pow2_exp(float x) {
  int e = 0;
  frexpf(x, &e);
  return e - 1;
}

// Double-shift QR iteration (Martin, Peters and Wilkinson's HQR, full-matrix updates so
// that A ends as the real Schur form T), in double-float arithmetic on the FP32 pipes:
// the scalar work of each bulge step is one thread's chain of dependent operations, which
// FP64 would issue at many clocks per instruction on this part.  One bulge chase step =
// one reflector logged (as doubles).  Returns through *npole_out, *nlog_out,
// *failed_out; eigenvalues of the complex pairs in s_mur/s_mui/s_pos (FP64, from the 2 x 2
// blocks).
template <class Acc>
__device__ void hqr_df(const Acc& A, int n, float anorm, double* lg, float2* s_sc, int* s_i, Step& s_st,
                       double* s_mur, double* s_mui, int* s_pos, int* npole_out, int* nlog_out,
                       int* failed_out) {
  using namespace dfl;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int npole = 0, nlog = 0, failed = 0;
  const long long cap = log_cap64(n);
  int nn = n - 1, its = 0, total = 0;
  const int max_total = 30 * n;
  while (nn >= 0) {
    // deflation: the largest l <= nn with a negligible subdiagonal A[l][l-1] (l = 0 if none)
    if (warp == 0) {
      int lsel = 0;
      for (int base = nn; base >= 1 && lsel == 0; base -= 32) {
        const int lq = base - lane;
        bool small = false;
        if (lq >= 1) {
          float sdiag = absf(A(lq - 1, lq - 1)) + absf(A(lq, lq));
          if (sdiag == 0.f) sdiag = anorm;
          small = absf(A(lq, lq - 1)) <= DF_EPS * sdiag;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, small);
        if (bal) lsel = base - (__ffs(bal) - 1);   // lowest lane = largest l
      }
      if (lane == 0) {
        if (lsel >= 1) A(lsel, lsel - 1) = make_float2(0.f, 0.f);
        s_i[0] = lsel;
      }
    }
    __syncthreads();
    const int l0 = s_i[0];
    if (l0 == nn) {   // one real eigenvalue
      nn -= 1;
      its = 0;
      continue;
    }
    if (l0 == nn - 1) {   // a 2 x 2 block: a complex pair or two real eigenvalues
      if (tid == 0) {
        const double a = to_double(A(nn - 1, nn - 1)), b = to_double(A(nn - 1, nn));
        const double c = to_double(A(nn, nn - 1)), d = to_double(A(nn, nn));
        const double h = 0.5 * (a - d);
        const double disc = h * h + b * c;
        if (disc < 0.0 && npole < 256) {
          s_mur[npole] = 0.5 * (a + d);
          s_mui[npole] = sqrt(-disc);
          s_pos[npole] = nn - 1;
        }
        s_i[1] = disc < 0.0 ? 1 : 0;
      }
      __syncthreads();
      npole += s_i[1];
      nn -= 2;
      its = 0;
      continue;
    }
    if (total >= max_total || nlog + n > cap) {
      failed = 1;
      break;
    }
    // shifts (trace and determinant of the trailing 2 x 2 block; exceptional shifts after
    // 10 and 20 iterations without deflation) and the start m of the bulge
    if (warp == 0) {
      float2 tr, det;
      const float2 a = A(nn - 1, nn - 1), b = A(nn - 1, nn);
      const float2 c = A(nn, nn - 1), d = A(nn, nn);
      if (its == 10 || its == 20) {
        const float2 sx = make_float2(absf(c) + absf(A(nn - 1, nn - 2)), 0.f);
        tr = dmulf(sx, 1.5f);
        det = dmul(sx, sx);
      } else {
        tr = dadd(a, d);
        det = dsub(dmul(a, d), dmul(b, c));
      }
      int msel = l0;
      for (int base = nn - 2; base >= l0 && msel == l0; base -= 32) {
        const int m = base - lane;
        bool ok = false;
        if (m > l0) {
          // the test only compares magnitudes: FP32 on the leading parts is enough
          const float hmm = A(m, m).x, h10 = A(m + 1, m).x;
          float pp = hmm * hmm + A(m, m + 1).x * h10 - tr.x * hmm + det.x;
          float qq = h10 * (hmm + A(m + 1, m + 1).x - tr.x);
          float rr = h10 * A(m + 2, m + 1).x;
          const float sc = fabsf(pp) + fabsf(qq) + fabsf(rr);
          if (sc > 0.f) {
            const int e = pow2_exp(sc);
            pp = ldexpf(pp, -e); qq = ldexpf(qq, -e); rr = ldexpf(rr, -e);
          }
          const float u = absf(A(m, m - 1)) * (fabsf(qq) + fabsf(rr));
          const float v = fabsf(pp) * (absf(A(m - 1, m - 1)) + fabsf(hmm) + absf(A(m + 1, m + 1)));
          ok = u <= DF_EPS * v;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (bal) msel = base - (__ffs(bal) - 1);
      }
      if (lane == 0) {
        s_i[2] = msel;
        s_sc[3] = tr;
        s_sc[4] = det;
      }
    }
    __syncthreads();
    const int m = s_i[2];
    const float2 tr = s_sc[3], det = s_sc[4];
    ++its;
    ++total;
    // chase the bulge from m to nn
    for (int kk = m; kk <= nn - 1; ++kk) {
      if (tid == 0) {
        const bool three = kk != nn - 1;
        float2 pp, qq, rr;
        if (kk == m) {
          const float2 hmm = A(m, m), h10 = A(m + 1, m);
          pp = dadd(dsub(dadd(dmul(hmm, hmm), dmul(A(m, m + 1), h10)), dmul(tr, hmm)), det);
          qq = dmul(h10, dsub(dadd(hmm, A(m + 1, m + 1)), tr));
          rr = dmul(h10, A(m + 2, m + 1));
        } else {
          pp = A(kk, kk - 1);
          qq = A(kk + 1, kk - 1);
          rr = three ? A(kk + 2, kk - 1) : make_float2(0.f, 0.f);
        }
        if (!three) rr = make_float2(0.f, 0.f);
        const float xs = absf(pp) + absf(qq) + absf(rr);
        Step st{};
        st.k = kk;
        st.three = three ? 1 : 0;
        if (xs > 0.f) {
          const int e = pow2_exp(xs);   // exact rescaling by a power of two
          pp = ldexp2(pp, -e);
          qq = ldexp2(qq, -e);
          rr = ldexp2(rr, -e);
          float2 s = dsqrt(dadd(dadd(dmul(pp, pp), dmul(qq, qq)), dmul(rr, rr)));
          if (pp.x < 0.f) s = dneg(s);
          if (kk != m) {
            A(kk, kk - 1) = ldexp2(dneg(s), e);
            A(kk + 1, kk - 1) = make_float2(0.f, 0.f);
            if (three) A(kk + 2, kk - 1) = make_float2(0.f, 0.f);
          } else if (l0 != m) {
            A(kk, kk - 1) = dneg(A(kk, kk - 1));
          }
          pp = dadd(pp, s);
          const float2 one = make_float2(1.f, 0.f);
          const float2 is = ddiv(one, s), ip = ddiv(one, pp);
          st.x = dmul(pp, is);
          st.y = dmul(qq, is);
          st.z = dmul(rr, is);
          st.q = dmul(qq, ip);
          st.r = dmul(rr, ip);
        } else {
          st.x = make_float2(0.f, 0.f);   // nothing to annihilate: identity step
        }
        s_st = st;
      }
      __syncthreads();
      const Step st = s_st;
      if (st.x.x != 0.f) {
        // rows kk.. of the whole matrix (columns kk .. n-1)
        for (int j = kk + tid; j < n; j += E64_THREADS) {
          const float2 a0 = A(kk, j), a1 = A(kk + 1, j);
          float2 pj = dadd(a0, dmul(st.q, a1));
          if (st.three) {
            const float2 a2 = A(kk + 2, j);
            pj = dadd(pj, dmul(st.r, a2));
            A(kk + 2, j) = dsub(a2, dmul(pj, st.z));
          }
          A(kk, j) = dsub(a0, dmul(pj, st.x));
          A(kk + 1, j) = dsub(a1, dmul(pj, st.y));
        }
        __syncthreads();
        // columns kk.. of rows 0 .. min(nn, kk + 3)
        const int imax = min(nn, kk + 3);
        for (int i = tid; i <= imax; i += E64_THREADS) {
          const float2 a0 = A(i, kk), a1 = A(i, kk + 1);
          float2 pi = dadd(dmul(st.x, a0), dmul(st.y, a1));
          if (st.three) {
            const float2 a2 = A(i, kk + 2);
            pi = dadd(pi, dmul(st.z, a2));
            A(i, kk + 2) = dsub(a2, dmul(pi, st.r));
          }
          A(i, kk) = dsub(a0, pi);
          A(i, kk + 1) = dsub(a1, dmul(pi, st.q));
        }
        if (tid == 0) {
          double* rec = lg + 6LL * nlog;
          rec[0] = (double)(kk + (st.three ? 0 : 4096));
          rec[1] = to_double(st.x);
          rec[2] = to_double(st.y);
          rec[3] = to_double(st.z);
          rec[4] = to_double(st.q);
          rec[5] = to_double(st.r);
        }
        ++nlog;
      }
      __syncthreads();
    }
  }
  *npole_out = npole;
  *nlog_out = nlog;
  *failed_out = failed;
}

// BAND: orders up to E64_BAND_N run the QR iteration on the band in shared memory; larger
// ones on the full matrix in the scratch.  The Hessenberg reduction runs on the full matrix
// in the scratch for every order (it streams rows and columns, so L2 latency overlaps).
template <bool BAND>
__global__ void __launch_bounds__(E64_THREADS, 1) k_eig64(Eig64Params p, int item_base) {
  extern __shared__ double smem64[];
  const int item = blockIdx.x + item_base;
  const int mi = p.n_orders - 1 - (item / p.lt.n_lags);
  const int t = item % p.lt.n_lags;
  const int n = p.orders[mi];
  const int k = p.lt.k;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* work = p.work + (size_t)t * p.work_per_lag + p.work_off[mi];
  int* hdr = reinterpret_cast<int*>(work);
  double* Tg = work + H64;                     // A, then T, n x n
  double* hv = Tg + (size_t)n * n;             // Hessenberg reflectors
  double* ev = hv + (size_t)n * n;             // eigenvalues by rank: 3 x n/2
  double* lg = ev + 3 * (n / 2);               // reflector log
  double* A = Tg;
  const int ld = n;
  const double* Rinv = p.RM + (size_t)t * 2 * k * k;
  const double* M = Rinv + (size_t)k * k;
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  __shared__ double s_v[512 + 8];              // Hessenberg vector (n <= 512)
  __shared__ double s_sc[8];
  __shared__ float2 s_sc2[8];
  __shared__ int s_i[8];
  __shared__ Step s_st;
  __shared__ double s_mur[256], s_mui[256];
  __shared__ int s_pos[256], s_rank[256];
  __shared__ double s_f[256];
  __shared__ int s_base[E64_BAND_N + 1];

  // ---- 1. A~_n = Rinv[:n,:n] M[:n,:n], Rinv upper triangular
  for (int e = tid; e < n * n; e += E64_THREADS) {
    const int r = e / n, c = e % n;
    double s = 0.0;
    for (int j = r; j < n; ++j) s = fma(Rinv[(size_t)r * k + j], M[(size_t)j * k + c], s);
    A[r * ld + c] = s;
  }
  if (tid == 0) s_sc[7] = 0.0;
  __syncthreads();
  // ||A||_1 entrywise, for the negligibility tests of the QR iteration
  {
    double a = 0.0;
    for (int e = tid; e < n * n; e += E64_THREADS) a += fabs(A[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) atomicAdd(&s_sc[7], a);
  }
  __syncthreads();
  const double anorm = s_sc[7];

  // ---- 2. Householder Hessenberg reduction: reflector j zeroes A[j+2:, j]
  for (int j = 0; j + 2 < n; ++j) {
    const int len = n - j - 1;   // rows j+1 .. n-1
    if (warp == 0) {
      double ss = 0.0;
      for (int r = 1 + lane; r < len; r += 32) {
        const double v = A[(j + 1 + r) * ld + j];
        ss = fma(v, v, ss);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) {
        const double alpha = A[(j + 1) * ld + j];
        double tau = 0.0, beta = alpha, scal = 0.0;
        if (ss > 0.0) {
          const double nrm = sqrt(alpha * alpha + ss);
          beta = alpha >= 0.0 ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        s_sc[0] = tau;
        s_sc[1] = beta;
        s_sc[2] = scal;
      }
    }
    __syncthreads();
    const double tau = s_sc[0], scal = s_sc[2];
    for (int r = tid; r < len; r += E64_THREADS) {
      const double v = r == 0 ? 1.0 : A[(j + 1 + r) * ld + j] * scal;
      s_v[r] = v;
      hv[(size_t)j * n + r] = v;
    }
    if (tid == 0) hv[(size_t)j * n + n - 1] = tau;
    __syncthreads();
    if (tau != 0.0) {
      // left: A[j+1:, c] -= tau v (v^T A[j+1:, c]), c > j; one thread per column
      for (int c = j + 1 + tid; c < n; c += E64_THREADS) {
        double s = 0.0;
        for (int r = 0; r < len; ++r) s = fma(s_v[r], A[(j + 1 + r) * ld + c], s);
        s *= tau;
        for (int r = 0; r < len; ++r) A[(j + 1 + r) * ld + c] -= s * s_v[r];
      }
      if (tid == 0) A[(j + 1) * ld + j] = s_sc[1];
      for (int r = 1 + tid; r < len; r += E64_THREADS) A[(j + 1 + r) * ld + j] = 0.0;
      __syncthreads();
      // right: A[r, j+1:] -= tau (A[r, j+1:] v) v^T, every row; one warp per row
      for (int r = warp; r < n; r += E64_THREADS / 32) {
        double s = 0.0;
        for (int c = lane; c < len; c += 32) s = fma(A[r * ld + j + 1 + c], s_v[c], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s *= tau;
        for (int c = lane; c < len; c += 32) A[r * ld + j + 1 + c] -= s * s_v[c];
      }
    }
    __syncthreads();
  }

  // ---- 3. double-shift QR iteration to the real Schur form, in double-float: the band
  //         (shared memory) or the whole matrix (the scratch, converted in place)
  int npole = 0, nlog = 0, failed = 0;
  if (BAND) {
    if (tid == 0) {
      int off = 0;
      for (int i = 0; i < n; ++i) {
        s_base[i] = off;
        off += n - (i > 3 ? i - 3 : 0);
      }
      s_base[n] = off;
    }
    __syncthreads();
    const BandA B{reinterpret_cast<float2*>(smem64), s_base};
    for (int i = warp; i < n; i += E64_THREADS / 32) {
      const int j0 = i > 3 ? i - 3 : 0;
      for (int j = j0 + lane; j < n; j += 32) B(i, j) = dfl::from_double(A[i * ld + j]);
    }
    __syncthreads();
    hqr_df(B, n, (float)anorm, lg, s_sc2, s_i, s_st, s_mur, s_mui, s_pos, &npole, &nlog, &failed);
    __syncthreads();
    for (int i = warp; i < n; i += E64_THREADS / 32) {
      const int j0 = i > 3 ? i - 3 : 0;
      for (int j = j0 + lane; j < n; j += 32) A[i * ld + j] = dfl::to_double(B(i, j));
    }
  } else {
    float2* A2 = reinterpret_cast<float2*>(A);   // same 8 bytes per element, in place
    for (int e = tid; e < n * n; e += E64_THREADS) A2[e] = dfl::from_double(A[e]);
    __syncthreads();
    const FullA F{A2, ld};
    hqr_df(F, n, (float)anorm, lg, s_sc2, s_i, s_st, s_mur, s_mui, s_pos, &npole, &nlog, &failed);
    __syncthreads();
    for (int e = tid; e < n * n; e += E64_THREADS) A[e] = dfl::to_double(A2[e]);
  }
  if (failed && tid == 0) atomicOr(p.status, DEV_NOTCONVERGED);
  npole = min(npole, 256);
  __syncthreads();

  // ---- 4. poles by frequency
  for (int j = tid; j < npole; j += E64_THREADS) {
    const double mr = s_mur[j], mu_i = s_mui[j];
    const double lr = 0.5 * log(mr * mr + mu_i * mu_i) / p.dt, li = atan2(mu_i, mr) / p.dt;
    s_f[j] = sqrt(lr * lr + li * li);
  }
  __syncthreads();
  for (int j = tid; j < npole; j += E64_THREADS) {
    int rk = 0;
    for (int o = 0; o < npole; ++o) rk += (s_f[o] < s_f[j]) || (s_f[o] == s_f[j] && o < j);
    s_rank[j] = rk;
    ev[3 * rk] = s_mur[j];
    ev[3 * rk + 1] = s_mui[j];
    ev[3 * rk + 2] = (double)s_pos[j];
  }
  __syncthreads();
  const int n_slots = n / 2;
  for (int j = tid; j < n_slots; j += E64_THREADS) {
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
      const double mr = ev[3 * j], mu_i = ev[3 * j + 1];
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
    hdr[1] = nlog;
    hdr[2] = failed;
  }
}

// ------------------------------------------------------------------ mode shapes
// One CTA of one warp per (lag, order, block of 16 poles), largest orders first.  Lane j
// carries pole j of the block through every step (complex arithmetic in the lane); the
// loops are uniform across the lanes and every operand they share (rows of T, log
// records, Hessenberg reflectors, rows of U) is first staged in shared memory by the
// whole warp with coalesced loads:
//   1. x = eigenvector of T for mu_j in FP64: x = (b, mu - a) on its 2 x 2 block, then
//      quasi-triangular back substitution upwards (a lane's entries above its own block
//      start as zero, so the shared row loop serves every lane).  This step divides by
//      T_rr - mu, which is small where another eigenvalue lies close, so it keeps FP64;
//   2. in FP32: the logged bulge reflectors in reverse order, then the Hessenberg
//      reflectors in reverse order (x becomes an eigenvector of A~_n).  They are
//      orthogonal transformations, so FP32 adds a relative error of ~1e-7 to x, which
//      changes 1 - MAC against any shape by ~1e-14 (MAC is quadratic in the error);
//   3. in FP32: Phi = U[:l, :n] x, scaled to unit norm with its largest component real
//      positive, MPC and MPD (the shapes are written in FP32 in every mode).
constexpr int V64_LOGCHUNK = 256;   // log records staged at a time

__global__ void __launch_bounds__(32) k_eigvec64(Eig64Params p) {
  extern __shared__ double vsm64[];
  const int t = blockIdx.x % p.lt.n_lags;
  int q = blockIdx.x / p.lt.n_lags;
  int mi = p.n_orders - 1;
  while (mi > 0 && q >= p.vec_blocks[mi]) {
    q -= p.vec_blocks[mi];
    --mi;
  }
  const int n = p.orders[mi];
  const int k = p.lt.k, l = p.lt.l;
  const int lane = threadIdx.x;
  const double* work = p.work + (size_t)t * p.work_per_lag + p.work_off[mi];
  const int* hdr = reinterpret_cast<const int*>(work);
  const double* T = work + H64;
  const double* hv = T + (size_t)n * n;
  const double* ev = hv + (size_t)n * n;
  const double* lg = ev + 3 * (n / 2);
  const int npole = hdr[0], nlog = hdr[1];
  const int j0 = q * V64_POLES;
  const int nj = max(0, min(V64_POLES, npole - j0));
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  float* phi_out = p.phi + ((size_t)t * p.slots_per_lag + p.slot_off[mi]) * 2 * l;
  const double* U = p.lt.U[t];
  const int n_slots_blk = min(V64_POLES, n / 2 - j0);
  // slots of the block without a pole: zero mode shapes
  for (int jj = nj; jj < n_slots_blk; ++jj)
    for (int e = lane; e < 2 * l; e += 32) phi_out[(size_t)(j0 + jj) * 2 * l + e] = 0.f;
  if (nj == 0) return;
  // shared memory: x (re, im) of the 16 poles in FP64, column-interleaved [r][lane]; two
  // staged rows of n doubles; the staged log records (doubles); x again in FP32
  const int ldx = V64_POLES + 1;
  double* xr = vsm64;                                   // n x ldx
  double* xi = xr + (size_t)n * ldx;                    // n x ldx
  double* row0 = xi + (size_t)n * ldx;                  // n
  double* row1 = row0 + n;                              // n
  double* logs = row1 + n;                              // 6 x V64_LOGCHUNK
  float* fr = reinterpret_cast<float*>(logs + 6 * V64_LOGCHUNK);   // n x ldx
  float* fi = fr + (size_t)n * ldx;                                // n x ldx
  float* frow = reinterpret_cast<float*>(row0);                    // n floats (staging)
  const bool act = lane < nj;
  const int ln = act ? lane : 0;
  const double mr = ev[3 * (j0 + ln)], mu_i = ev[3 * (j0 + ln) + 1];
  const int pos = act ? (int)ev[3 * (j0 + ln) + 2] : -1;
  int maxpos = pos;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxpos = max(maxpos, __shfl_xor_sync(0xffffffffu, maxpos, o));
  for (int r = 0; r < n; ++r) {
    if (lane < V64_POLES) {
      xr[r * ldx + lane] = 0.0;
      xi[r * ldx + lane] = 0.0;
    }
  }
  __syncwarp();
  if (act) {
    xr[pos * ldx + lane] = T[(size_t)pos * n + pos + 1];
    xr[(pos + 1) * ldx + lane] = mr - T[(size_t)pos * n + pos];
    xi[(pos + 1) * ldx + lane] = mu_i;
  }
  double tnorm = 0.0;
  for (int r = lane; r <= maxpos + 1; r += 32) tnorm = fmax(tnorm, fabs(T[(size_t)r * n + r]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  const double tiny = DBL_EPSILON * fmax(tnorm, 1e-300);
  __syncwarp();
  // 1. back substitution (FP64), rows maxpos-1 .. 0 (row blocks are the same for every lane)
  for (int r = maxpos - 1; r >= 0;) {
    const bool pair = (r >= 1) && T[(size_t)r * n + r - 1] != 0.0;
    const int top = pair ? r - 1 : r;
    const int c0 = top, c1 = maxpos + 1;   // columns staged
    for (int c = c0 + lane; c <= c1; c += 32) {
      row1[c] = T[(size_t)r * n + c];
      if (pair) row0[c] = T[(size_t)top * n + c];
    }
    __syncwarp();
    if (act && r < pos) {
      double s0r = 0.0, s0i = 0.0, s1r = 0.0, s1i = 0.0;
      for (int c = r + 1; c <= c1; ++c) {
        const double vr = xr[c * ldx + lane], vi = xi[c * ldx + lane];
        s1r = fma(row1[c], vr, s1r);
        s1i = fma(row1[c], vi, s1i);
        if (pair) {
          s0r = fma(row0[c], vr, s0r);
          s0i = fma(row0[c], vi, s0i);
        }
      }
      if (!pair) {
        double dr = row1[r] - mr, di = -mu_i;
        if (fabs(dr) + fabs(di) < tiny) dr = tiny;
        const double den = 1.0 / (dr * dr + di * di);
        xr[r * ldx + lane] = -(s1r * dr + s1i * di) * den;
        xi[r * ldx + lane] = -(s1i * dr - s1r * di) * den;
      } else {
        // s0 collected row `top` from column r + 1 on; row top's column r belongs to the
        // 2 x 2 system
        const double ar = row0[top] - mr, ai = -mu_i;
        const double br = row0[r];
        const double cr = row1[top];
        const double dr = row1[r] - mr, di = -mu_i;
        double detr = ar * dr - ai * di - br * cr;
        double deti = ar * di + ai * dr;
        if (fabs(detr) + fabs(deti) < tiny) detr = tiny;
        const double den = 1.0 / (detr * detr + deti * deti);
        const double n0r = -(s0r * dr - s0i * di) + br * s1r;
        const double n0i = -(s0r * di + s0i * dr) + br * s1i;
        const double n1r = -(ar * s1r - ai * s1i) + cr * s0r;
        const double n1i = -(ar * s1i + ai * s1r) + cr * s0i;
        xr[top * ldx + lane] = (n0r * detr + n0i * deti) * den;
        xi[top * ldx + lane] = (n0i * detr - n0r * deti) * den;
        xr[r * ldx + lane] = (n1r * detr + n1i * deti) * den;
        xi[r * ldx + lane] = (n1i * detr - n1r * deti) * den;
      }
    }
    __syncwarp();
    r = top - 1;
  }
  // x to FP32, scaled by its largest entry (the FP64 back substitution may grow it far
  // beyond the FP32 range's comfort: only the direction matters)
  {
    double big = 0.0;
    if (lane < V64_POLES)
      for (int r = 0; r < n; ++r)
        big = fmax(big, fmax(fabs(xr[r * ldx + lane]), fabs(xi[r * ldx + lane])));
    const double sc = big > 0.0 ? 1.0 / big : 0.0;
    if (lane < V64_POLES)
      for (int r = 0; r < n; ++r) {
        fr[r * ldx + lane] = (float)(xr[r * ldx + lane] * sc);
        fi[r * ldx + lane] = (float)(xi[r * ldx + lane] * sc);
      }
  }
  __syncwarp();
  // 2a. bulge reflectors in reverse (FP32): x[k..k+2] -= (x, y, z) (x_k + q x_{k+1} + r x_{k+2})
  for (int e1 = nlog; e1 > 0; e1 -= V64_LOGCHUNK) {
    const int e0 = max(0, e1 - V64_LOGCHUNK);
    for (int u = lane; u < 6 * (e1 - e0); u += 32) logs[u] = lg[6LL * e0 + u];
    __syncwarp();
    if (lane < V64_POLES) {
      for (int e = e1 - 1; e >= e0; --e) {
        const double* rec = logs + 6 * (e - e0);
        int kk = (int)rec[0];
        const bool three = kk < 4096;
        if (!three) kk -= 4096;
        const float ax = (float)rec[1], ay = (float)rec[2], az = (float)rec[3];
        const float bq = (float)rec[4], br = (float)rec[5];
        float* x0r = fr + kk * ldx + lane;
        float* x0i = fi + kk * ldx + lane;
        float tr = fmaf(bq, x0r[ldx], x0r[0]);
        float ti = fmaf(bq, x0i[ldx], x0i[0]);
        if (three) {
          tr = fmaf(br, x0r[2 * ldx], tr);
          ti = fmaf(br, x0i[2 * ldx], ti);
        }
        x0r[0] = fmaf(-ax, tr, x0r[0]);
        x0i[0] = fmaf(-ax, ti, x0i[0]);
        x0r[ldx] = fmaf(-ay, tr, x0r[ldx]);
        x0i[ldx] = fmaf(-ay, ti, x0i[ldx]);
        if (three) {
          x0r[2 * ldx] = fmaf(-az, tr, x0r[2 * ldx]);
          x0i[2 * ldx] = fmaf(-az, ti, x0i[2 * ldx]);
        }
      }
    }
    __syncwarp();
  }
  // 2b. Hessenberg reflectors in reverse (FP32): x[j+1:] -= tau v (v^T x[j+1:])
  for (int j = n - 3; j >= 0; --j) {
    const double* v = hv + (size_t)j * n;
    const int len = n - j - 1;
    for (int c = lane; c < len; c += 32) frow[c] = (float)v[c];
    const float tau = (float)v[n - 1];
    __syncwarp();
    if (tau != 0.f && lane < V64_POLES) {
      float dr = 0.f, di = 0.f;
      for (int r = 0; r < len; ++r) {
        dr = fmaf(frow[r], fr[(j + 1 + r) * ldx + lane], dr);
        di = fmaf(frow[r], fi[(j + 1 + r) * ldx + lane], di);
      }
      dr *= tau;
      di *= tau;
      for (int r = 0; r < len; ++r) {
        fr[(j + 1 + r) * ldx + lane] = fmaf(-dr, frow[r], fr[(j + 1 + r) * ldx + lane]);
        fi[(j + 1 + r) * ldx + lane] = fmaf(-di, frow[r], fi[(j + 1 + r) * ldx + lane]);
      }
    }
    __syncwarp();
  }
  // 3. Phi = U[:l, :n] x (row ch of U staged), normalisation, MPC, MPD: one pole per lane.
  //    The unnormalised components are kept in the output and rescaled in place.
  float* ph = phi_out + (size_t)(j0 + ln) * 2 * l;
  float nrm2 = 0.f, best = -1.f, bre = 1.f, bim = 0.f;
  for (int ch = 0; ch < l; ++ch) {
    for (int a = lane; a < n; a += 32) frow[a] = (float)U[(size_t)ch * k + a];
    __syncwarp();
    if (act) {
      float sr = 0.f, si = 0.f;
      for (int a = 0; a < n; ++a) {
        sr = fmaf(frow[a], fr[a * ldx + lane], sr);
        si = fmaf(frow[a], fi[a * ldx + lane], si);
      }
      const float m2 = sr * sr + si * si;
      nrm2 += m2;
      if (m2 > best) { best = m2; bre = sr; bim = si; }
      ph[2 * ch] = sr;
      ph[2 * ch + 1] = si;
    }
    __syncwarp();
  }
  if (act) {
    const float bm = sqrtf(fmaxf(best, 0.f));
    const float inv = (nrm2 > 0.f && bm > 0.f) ? rsqrtf(nrm2) / bm : 0.f;
    const float cr = bre * inv, ci = -bim * inv;
    float sxx = 0.f, syy = 0.f, sxy = 0.f;
    for (int ch = 0; ch < l; ++ch) {
      const float sr = ph[2 * ch], si = ph[2 * ch + 1];
      const float re = sr * cr - si * ci, im = sr * ci + si * cr;
      ph[2 * ch] = re;
      ph[2 * ch + 1] = im;
      sxx = fmaf(re, re, sxx);
      syy = fmaf(im, im, syy);
      sxy = fmaf(re, im, sxy);
    }
    const float tr = sxx + syy;
    const float dd = sqrtf((sxx - syy) * (sxx - syy) + 4.f * sxy * sxy);
    const float mpc = tr > 0.f ? (dd / tr) * (dd / tr) : 0.f;
    const float th = 0.5f * atan2f(2.f * sxy, sxx - syy);
    const float v1x = cosf(th), v1y = sinf(th);
    float wsum = 0.f, asum = 0.f;
    for (int ch = 0; ch < l; ++ch) {
      const float re = ph[2 * ch], im = ph[2 * ch + 1];
      const float mg = sqrtf(re * re + im * im);
      if (mg > 0.f) {
        const float cosang = fminf(1.f, fabsf(re * v1x + im * v1y) / mg);
        wsum += mg;
        asum += mg * acosf(cosang);
      }
    }
    poles[j0 + lane].mpc = mpc;
    poles[j0 + lane].mpd = wsum > 0.f ? (asum / wsum) / 1.5707963267948966f : 0.f;
  }
}

}  // namespace

size_t realize64_ws_bytes(int n_lags, const int* lags, int l, int k, const int* orders, int n_orders) {
  long long work = 0;
  int max_i = 0;
  for (int m = 0; m < n_orders; ++m) work += eig64_doubles(orders[m]) + 8;
  for (int t = 0; t < n_lags; ++t) max_i = std::max(max_i, lags[t]);
  const int n_chunks = (int)ceil_div((int64_t)l * (max_i - 1), G64_ROWS);
  WsPlan w;
  w.add<double>((size_t)n_lags * std::max(n_chunks, 1) * 2 * k * k);   // Gram partials
  w.add<double>((size_t)n_lags * 2 * k * k);                           // G | H
  w.add<double>((size_t)n_lags * 2 * k * k);                           // Rinv | M
  w.add<double>((size_t)n_lags * ((size_t)k * (k + 1) + k));           // factor scratch
  w.add<double>((size_t)n_lags * work);                                // eig scratch
  return w.bytes;
}

ssi_status realize64_ws(ssi_ctx* ctx, Workspace& ws, int n_lags, const int* lags, int l, int k,
                        const double* const* U, const int* orders, int n_orders, int64_t slots_per_lag,
                        double dt, ssi_pole* poles, float* phi, int* dev_status, cudaStream_t stream) {
  ws.reset();
  int max_i = 0;
  for (int t = 0; t < n_lags; ++t) max_i = std::max(max_i, lags[t]);
  const int n_chunks = std::max(1, (int)ceil_div((int64_t)l * (max_i - 1), G64_ROWS));
  double* partial = ws.take<double>((size_t)n_lags * n_chunks * 2 * k * k);
  double* GH = ws.take<double>((size_t)n_lags * 2 * k * k);
  double* RM = ws.take<double>((size_t)n_lags * 2 * k * k);
  double* Fs = ws.take<double>((size_t)n_lags * ((size_t)k * (k + 1) + k));
  Eig64Params ep{};
  long long work = 0;
  for (int m = 0; m < n_orders; ++m) {
    ep.orders[m] = orders[m];
    ep.work_off[m] = work;
    work += eig64_doubles(orders[m]) + 8;
  }
  double* eigw = ws.take<double>((size_t)n_lags * work);
  if (!partial || !GH || !RM || !Fs || !eigw) {
    set_error("realize64: workspace too small");
    return SSI_E_NOMEM;
  }
  Lag64Table lt{};
  lt.n_lags = n_lags;
  lt.l = l;
  lt.k = k;
  for (int t = 0; t < n_lags; ++t) {
    lt.i[t] = lags[t];
    lt.U[t] = U[t];
  }
  {
    ProfScope ps(ctx, ST_GRAM, stream);
    const int tiles = (int)ceil_div(k, 32);
    dim3 g1((unsigned)(tiles * tiles), (unsigned)n_chunks, (unsigned)(2 * n_lags));
    k_gram64<<<g1, 256, 0, stream>>>(lt, n_chunks, partial);
    SSI_CUDA(cudaGetLastError());
    k_gram_reduce64<<<ctx->num_sms * 4, 256, 0, stream>>>(partial, n_lags, n_chunks, k, GH);
    SSI_CUDA(cudaGetLastError());
    SSI_TRY(lag_factor64_launch(GH, k, n_lags, RM, Fs, dev_status, stream));
    count_launches(ctx, 3);
  }
  ep.lt = lt;
  ep.n_orders = n_orders;
  long long off = 0;
  for (int m = 0; m < n_orders; ++m) {
    ep.slot_off[m] = off;
    off += orders[m] / 2;
    ep.vec_blocks[m] = (int)ceil_div(orders[m] / 2, V64_POLES);
  }
  ep.slots_per_lag = slots_per_lag;
  ep.RM = RM;
  ep.work = eigw;
  ep.work_per_lag = work;
  ep.dt = dt;
  ep.poles = poles;
  ep.phi = phi;
  ep.status = dev_status;
  // largest orders first; the ones above E64_BAND_N run the QR iteration on the full
  // matrix in the scratch (L2), the others on its band in shared memory
  int n_big = 0, nmax_band = 0;
  for (int m = 0; m < n_orders; ++m) {
    if (orders[m] > E64_BAND_N) ++n_big;
    else nmax_band = std::max(nmax_band, orders[m]);
  }
  {
    ProfScope ps(ctx, ST_EIG, stream);
    if (n_big > 0) {
      k_eig64<false><<<n_lags * n_big, E64_THREADS, 0, stream>>>(ep, 0);
      SSI_CUDA(cudaGetLastError());
    }
    if (n_orders > n_big) {
      const size_t smem = (size_t)band_doubles(nmax_band) * sizeof(double);
      SSI_CUDA(cudaFuncSetAttribute(k_eig64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)std::max<size_t>(smem, 1024)));
      k_eig64<true><<<n_lags * (n_orders - n_big), E64_THREADS, smem, stream>>>(ep, n_lags * n_big);
      SSI_CUDA(cudaGetLastError());
    }
    count_launches(ctx, (n_big > 0) + (n_orders > n_big));
  }
  {
    ProfScope ps(ctx, ST_EIG_VEC, stream);
    int total = 0, nmax = 0;
    for (int m = 0; m < n_orders; ++m) {
      total += ep.vec_blocks[m];
      nmax = std::max(nmax, orders[m]);
    }
    const size_t vsmem =
        ((size_t)2 * nmax * (V64_POLES + 1) + 2 * (size_t)nmax + 6 * V64_LOGCHUNK) * sizeof(double) +
        (size_t)2 * nmax * (V64_POLES + 1) * sizeof(float);
    SSI_CUDA(cudaFuncSetAttribute(k_eigvec64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem));
    k_eigvec64<<<n_lags * total, 32, vsmem, stream>>>(ep);
    SSI_CUDA(cudaGetLastError());
    count_launches(ctx, 1);
  }
  return SSI_OK;
}

}  // namespace ssi
