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
constexpr int E64_SMEM_N = 160;       // largest order whose A (FP64) stays in shared memory
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
  double x, y, z, q, r;
  int k, three;
};

template <bool BIG>
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
  double* Tg = work + H64;                     // T, n x n
  double* hv = Tg + (size_t)n * n;             // Hessenberg reflectors
  double* ev = hv + (size_t)n * n;             // eigenvalues by rank: 3 x n/2
  double* lg = ev + 3 * (n / 2);               // reflector log
  double* A = BIG ? Tg : smem64;
  const int ld = n;
  const double* Rinv = p.RM + (size_t)t * 2 * k * k;
  const double* M = Rinv + (size_t)k * k;
  ssi_pole* poles = p.poles + (size_t)t * p.slots_per_lag + p.slot_off[mi];
  __shared__ double s_v[512 + 8];              // Hessenberg vector (n <= 512)
  __shared__ double s_sc[8];
  __shared__ int s_i[8];
  __shared__ Step s_st;
  __shared__ double s_mur[256], s_mui[256];
  __shared__ int s_pos[256], s_rank[256];
  __shared__ double s_f[256];

  // ---- 1. A~_n = Rinv[:n,:n] M[:n,:n], Rinv upper triangular
  for (int e = tid; e < n * n; e += E64_THREADS) {
    const int r = e / n, c = e % n;
    double s = 0.0;
    for (int j = r; j < n; ++j) s = fma(Rinv[(size_t)r * k + j], M[(size_t)j * k + c], s);
    A[r * ld + c] = s;
  }
  __syncthreads();
  // ||A||_1 entrywise, for the negligibility tests of the QR iteration
  if (tid == 0) s_sc[7] = 0.0;
  __syncthreads();
  {
    double a = 0.0;
    for (int e = tid; e < n * n; e += E64_THREADS) a += fabs(A[(e / n) * ld + e % n]);
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
      if (tid == 0) {
        A[(j + 1) * ld + j] = s_sc[1];
      }
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

  // ---- 3. double-shift QR iteration to the real Schur form (full-matrix updates)
  int npole = 0;
  int nlog = 0;
  int failed = 0;
  {
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
            double sdiag = fabs(A[(lq - 1) * ld + lq - 1]) + fabs(A[lq * ld + lq]);
            if (sdiag == 0.0) sdiag = anorm;
            small = fabs(A[lq * ld + lq - 1]) <= DBL_EPSILON * sdiag;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, small);
          if (bal) lsel = base - (__ffs(bal) - 1);   // lowest lane = largest l
        }
        if (lane == 0) {
          if (lsel >= 1) A[lsel * ld + lsel - 1] = 0.0;
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
          const double a = A[(nn - 1) * ld + nn - 1], b = A[(nn - 1) * ld + nn];
          const double c = A[nn * ld + nn - 1], d = A[nn * ld + nn];
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
      // shifts (trace and determinant of the trailing 2 x 2 block; exceptional shifts
      // after 10 and 20 iterations without deflation) and the start m of the bulge
      if (warp == 0) {
        double tr, det;
        const double a = A[(nn - 1) * ld + nn - 1], b = A[(nn - 1) * ld + nn];
        const double c = A[nn * ld + nn - 1], d = A[nn * ld + nn];
        if (its == 10 || its == 20) {
          const double s = fabs(c) + fabs(A[(nn - 1) * ld + nn - 2]);
          tr = 1.5 * s;
          det = s * s;
        } else {
          tr = a + d;
          det = a * d - b * c;
        }
        int msel = l0;
        for (int base = nn - 2; base >= l0 && msel == l0; base -= 32) {
          const int m = base - lane;
          bool ok = false;
          if (m > l0) {
            const double hmm = A[m * ld + m], h10 = A[(m + 1) * ld + m];
            double pp = hmm * hmm + A[m * ld + m + 1] * h10 - tr * hmm + det;
            double qq = h10 * (hmm + A[(m + 1) * ld + m + 1] - tr);
            double rr = h10 * A[(m + 2) * ld + m + 1];
            const double sc = fabs(pp) + fabs(qq) + fabs(rr);
            if (sc > 0.0) { pp /= sc; qq /= sc; rr /= sc; }
            const double u = fabs(A[m * ld + m - 1]) * (fabs(qq) + fabs(rr));
            const double v = fabs(pp) * (fabs(A[(m - 1) * ld + m - 1]) + fabs(hmm) +
                                         fabs(A[(m + 1) * ld + m + 1]));
            ok = u <= DBL_EPSILON * v;
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
      const double tr = s_sc[3], det = s_sc[4];
      ++its;
      ++total;
      // chase the bulge from m to nn
      for (int kk = m; kk <= nn - 1; ++kk) {
        if (tid == 0) {
          const bool three = kk != nn - 1;
          double pp, qq, rr;
          if (kk == m) {
            const double hmm = A[m * ld + m], h10 = A[(m + 1) * ld + m];
            pp = hmm * hmm + A[m * ld + m + 1] * h10 - tr * hmm + det;
            qq = h10 * (hmm + A[(m + 1) * ld + m + 1] - tr);
            rr = h10 * A[(m + 2) * ld + m + 1];
          } else {
            pp = A[kk * ld + kk - 1];
            qq = A[(kk + 1) * ld + kk - 1];
            rr = three ? A[(kk + 2) * ld + kk - 1] : 0.0;
          }
          if (!three) rr = 0.0;
          const double xs = fabs(pp) + fabs(qq) + fabs(rr);
          Step st{};
          st.k = kk;
          st.three = three ? 1 : 0;
          if (xs > 0.0) {
            pp /= xs;
            qq /= xs;
            rr /= xs;
            const double s = copysign(sqrt(pp * pp + qq * qq + rr * rr), pp);
            if (kk != m) {
              A[kk * ld + kk - 1] = -s * xs;
              A[(kk + 1) * ld + kk - 1] = 0.0;
              if (three) A[(kk + 2) * ld + kk - 1] = 0.0;
            } else if (l0 != m) {
              A[kk * ld + kk - 1] = -A[kk * ld + kk - 1];
            }
            pp += s;
            st.x = pp / s;
            st.y = qq / s;
            st.z = rr / s;
            st.q = qq / pp;
            st.r = rr / pp;
          } else {
            st.x = 0.0;   // nothing to annihilate: identity step
          }
          s_st = st;
        }
        __syncthreads();
        const Step st = s_st;
        if (st.x != 0.0) {
          // rows kk.. of the whole matrix (columns kk .. n-1)
          for (int j = kk + tid; j < n; j += E64_THREADS) {
            double pj = A[kk * ld + j] + st.q * A[(kk + 1) * ld + j];
            if (st.three) pj += st.r * A[(kk + 2) * ld + j];
            A[kk * ld + j] -= pj * st.x;
            A[(kk + 1) * ld + j] -= pj * st.y;
            if (st.three) A[(kk + 2) * ld + j] -= pj * st.z;
          }
          __syncthreads();
          // columns kk.. of rows 0 .. min(nn, kk + 3)
          const int imax = min(nn, kk + 3);
          for (int i = tid; i <= imax; i += E64_THREADS) {
            double pi = st.x * A[i * ld + kk] + st.y * A[i * ld + kk + 1];
            if (st.three) pi += st.z * A[i * ld + kk + 2];
            A[i * ld + kk] -= pi;
            A[i * ld + kk + 1] -= pi * st.q;
            if (st.three) A[i * ld + kk + 2] -= pi * st.r;
          }
          if (tid == 0) {
            double* rec = lg + 6LL * nlog;
            rec[0] = (double)(kk + (st.three ? 0 : 4096));
            rec[1] = st.x;
            rec[2] = st.y;
            rec[3] = st.z;
            rec[4] = st.q;
            rec[5] = st.r;
          }
          ++nlog;
        }
        __syncthreads();
      }
    }
  }
  if (failed && tid == 0) atomicOr(p.status, DEV_NOTCONVERGED);
  npole = min(npole, 256);

  // ---- 4. T to the scratch (the eigenvector kernel reads it); poles by frequency
  if (!BIG)
    for (int e = tid; e < n * n; e += E64_THREADS) Tg[e] = A[(e / n) * ld + e % n];
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

// ------------------------------------------------------------------ mode shapes (FP64)
// One CTA of one warp per (lag, order, block of 16 poles), largest orders first.  Lane j
// carries pole j of the block through every step (complex arithmetic in the lane):
//   1. x = eigenvector of T for mu_j: x = (b, mu - a) on its 2 x 2 block, then quasi-
//      triangular back substitution upwards;
//   2. the logged bulge reflectors in reverse order, then the Hessenberg reflectors in
//      reverse order (x becomes an eigenvector of A~_n);
//   3. Phi = U[:l, :n] x, scaled to unit norm with its largest component real positive,
//      MPC and MPD.
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
  // x of pole (lane): xr, xi at vsm64[lane * n + r], vsm64[(16 + lane) * n + r]
  double* xr = vsm64 + (size_t)lane * n;
  double* xi = vsm64 + (size_t)(V64_POLES + lane) * n;
  const bool act = lane < nj;
  if (act) {
    const double mr = ev[3 * (j0 + lane)], mu_i = ev[3 * (j0 + lane) + 1];
    const int pos = (int)ev[3 * (j0 + lane) + 2];
    for (int r = 0; r < n; ++r) { xr[r] = 0.0; xi[r] = 0.0; }
    xr[pos] = T[(size_t)pos * n + pos + 1];
    xr[pos + 1] = mr - T[(size_t)pos * n + pos];
    xi[pos + 1] = mu_i;
    double tnorm = 0.0;
    for (int r = 0; r <= pos + 1; ++r) tnorm = fmax(tnorm, fabs(T[(size_t)r * n + r]));
    const double tiny = DBL_EPSILON * fmax(tnorm, 1e-300);
    for (int r = pos - 1; r >= 0;) {
      const bool pair = (r >= 1) && T[(size_t)r * n + r - 1] != 0.0;
      const int top = pair ? r - 1 : r;
      double s0r = 0.0, s0i = 0.0, s1r = 0.0, s1i = 0.0;
      for (int c = r + 1; c <= pos + 1; ++c) {
        const double vr = xr[c], vi = xi[c];
        const double t1 = T[(size_t)r * n + c];
        s1r = fma(t1, vr, s1r);
        s1i = fma(t1, vi, s1i);
        if (pair) {
          const double t0 = T[(size_t)top * n + c];
          s0r = fma(t0, vr, s0r);
          s0i = fma(t0, vi, s0i);
        }
      }
      if (!pair) {
        double dr = T[(size_t)r * n + r] - mr, di = -mu_i;
        if (fabs(dr) + fabs(di) < tiny) dr = tiny;
        const double den = 1.0 / (dr * dr + di * di);
        xr[r] = -(s1r * dr + s1i * di) * den;
        xi[r] = -(s1i * dr - s1r * di) * den;
      } else {
        const double ar = T[(size_t)top * n + top] - mr, ai = -mu_i;
        const double br = T[(size_t)top * n + r];
        const double cr = T[(size_t)r * n + top];
        const double dr = T[(size_t)r * n + r] - mr, di = -mu_i;
        double detr = ar * dr - ai * di - br * cr;
        double deti = ar * di + ai * dr;
        if (fabs(detr) + fabs(deti) < tiny) detr = tiny;
        const double den = 1.0 / (detr * detr + deti * deti);
        const double n0r = -(s0r * dr - s0i * di) + br * s1r;
        const double n0i = -(s0r * di + s0i * dr) + br * s1i;
        const double n1r = -(ar * s1r - ai * s1i) + cr * s0r;
        const double n1i = -(ar * s1i + ai * s1r) + cr * s0i;
        xr[top] = (n0r * detr + n0i * deti) * den;
        xi[top] = (n0i * detr - n0r * deti) * den;
        xr[r] = (n1r * detr + n1i * deti) * den;
        xi[r] = (n1i * detr - n1r * deti) * den;
      }
      r = top - 1;
    }
    // bulge reflectors in reverse: x[k..k+2] -= (x, y, z) (x_k + q x_{k+1} + r x_{k+2})
    for (int e = nlog - 1; e >= 0; --e) {
      const double* rec = lg + 6LL * e;
      int kk = (int)rec[0];
      const bool three = kk < 4096;
      if (!three) kk -= 4096;
      const double ax = rec[1], ay = rec[2], az = rec[3], bq = rec[4], br = rec[5];
      double tr = xr[kk] + bq * xr[kk + 1];
      double ti = xi[kk] + bq * xi[kk + 1];
      if (three) {
        tr += br * xr[kk + 2];
        ti += br * xi[kk + 2];
      }
      xr[kk] -= ax * tr;
      xi[kk] -= ax * ti;
      xr[kk + 1] -= ay * tr;
      xi[kk + 1] -= ay * ti;
      if (three) {
        xr[kk + 2] -= az * tr;
        xi[kk + 2] -= az * ti;
      }
    }
    // Hessenberg reflectors in reverse: x[j+1:] -= tau v (v^T x[j+1:])
    for (int j = n - 3; j >= 0; --j) {
      const double* v = hv + (size_t)j * n;
      const double tau = v[n - 1];
      if (tau == 0.0) continue;
      const int len = n - j - 1;
      double dr = 0.0, di = 0.0;
      for (int r = 0; r < len; ++r) {
        dr = fma(v[r], xr[j + 1 + r], dr);
        di = fma(v[r], xi[j + 1 + r], di);
      }
      dr *= tau;
      di *= tau;
      for (int r = 0; r < len; ++r) {
        xr[j + 1 + r] -= dr * v[r];
        xi[j + 1 + r] -= di * v[r];
      }
    }
  }
  __syncwarp();
  // Phi = U[:l, :n] x, normalisation, MPC, MPD: one pole per lane.  The unnormalised
  // components are kept in the output (FP32) and rescaled in place.
  if (act) {
    float* ph = phi_out + (size_t)(j0 + lane) * 2 * l;
    double nrm2 = 0.0, best = -1.0, bre = 1.0, bim = 0.0;
    for (int ch = 0; ch < l; ++ch) {
      double sr = 0.0, si = 0.0;
      const double* urow = U + (size_t)ch * k;
      for (int a = 0; a < n; ++a) {
        const double u = urow[a];
        sr = fma(u, xr[a], sr);
        si = fma(u, xi[a], si);
      }
      const double m2 = sr * sr + si * si;
      nrm2 += m2;
      if (m2 > best) { best = m2; bre = sr; bim = si; }
      ph[2 * ch] = (float)sr;
      ph[2 * ch + 1] = (float)si;
    }
    const double bm = sqrt(fmax(best, 0.0));
    const double inv = (nrm2 > 0.0 && bm > 0.0) ? 1.0 / (sqrt(nrm2) * bm) : 0.0;
    const double cr = bre * inv, ci = -bim * inv;
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int ch = 0; ch < l; ++ch) {
      const double sr = ph[2 * ch], si = ph[2 * ch + 1];
      const double re = sr * cr - si * ci, im = sr * ci + si * cr;
      ph[2 * ch] = (float)re;
      ph[2 * ch + 1] = (float)im;
      sxx = fma(re, re, sxx);
      syy = fma(im, im, syy);
      sxy = fma(re, im, sxy);
    }
    const double tr = sxx + syy;
    const double dd = sqrt((sxx - syy) * (sxx - syy) + 4.0 * sxy * sxy);
    const double mpc = tr > 0.0 ? (dd / tr) * (dd / tr) : 0.0;
    const double th = 0.5 * atan2(2.0 * sxy, sxx - syy);
    const double v1x = cos(th), v1y = sin(th);
    double wsum = 0.0, asum = 0.0;
    for (int ch = 0; ch < l; ++ch) {
      const double re = ph[2 * ch], im = ph[2 * ch + 1];
      const double mg = sqrt(re * re + im * im);
      if (mg > 0.0) {
        const double cosang = fmin(1.0, fabs(re * v1x + im * v1y) / mg);
        wsum += mg;
        asum += mg * acos(cosang);
      }
    }
    poles[j0 + lane].mpc = (float)mpc;
    poles[j0 + lane].mpd = wsum > 0.0 ? (float)((asum / wsum) / 1.5707963267948966) : 0.f;
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
  // largest orders first; the ones above E64_SMEM_N keep A in the scratch (L2)
  int n_big = 0;
  for (int m = 0; m < n_orders; ++m) n_big += orders[m] > E64_SMEM_N;
  {
    ProfScope ps(ctx, ST_EIG, stream);
    if (n_big > 0) {
      k_eig64<true><<<n_lags * n_big, E64_THREADS, 0, stream>>>(ep, 0);
      SSI_CUDA(cudaGetLastError());
    }
    if (n_orders > n_big) {
      int nmax_small = 0;
      for (int m = 0; m < n_orders; ++m)
        if (orders[m] <= E64_SMEM_N) nmax_small = std::max(nmax_small, orders[m]);
      const size_t smem = (size_t)nmax_small * nmax_small * sizeof(double);
      SSI_CUDA(cudaFuncSetAttribute(k_eig64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)std::max<size_t>(smem, 1024)));
      k_eig64<false><<<n_lags * (n_orders - n_big), E64_THREADS, smem, stream>>>(ep, n_lags * n_big);
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
    const size_t vsmem = (size_t)2 * V64_POLES * (nmax + 1) * sizeof(double);
    SSI_CUDA(cudaFuncSetAttribute(k_eigvec64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsmem));
    k_eigvec64<<<n_lags * total, 32, vsmem, stream>>>(ep);
    SSI_CUDA(cudaGetLastError());
    count_launches(ctx, 1);
  }
  return SSI_OK;
}

}  // namespace ssi
