// Economy QR of a tall-skinny FP32 matrix (the sketch re-orthonormalisation of Sec. 2.2,
// "(Q, R) = qr(Y, 0)" of Algorithm 1).
//
// One cooperative persistent kernel.  The rows are cut into a fixed number of chunks
// (one per SM of the device) and each CTA owns one or two consecutive chunks: one when
// the solve has the device to itself, two when several solves share it (half the
// SMs, so that two solves' QR grids run side by side).  Every reduction is taken over
// per-chunk partials in a fixed order, so the result does not depend on the grid.
// Columns are processed in panels of 32:
//   pass 1:  W  = Y_j - Q_{<j} (Q_{<j}^T Y_j);   W  = W R1^{-1},  R1 = chol(W^T W)
//   pass 2:  W' = W   - Q_{<j} (Q_{<j}^T W);     Q_j = W' R2^{-1}, R2 = chol(W'^T W')
// (block classical Gram-Schmidt with re-orthogonalisation, each panel made
// orthonormal by Cholesky-QR).  The first-pass Gram matrices are accumulated in
// double-FP32 (error-free products with fma, two-sum accumulation) and reduced in FP64.
// The 32x32 Cholesky factors run redundantly in every CTA: in FP32 by the whole CTA, and
// for the first pass in FP64 when the FP32 pivots show cond(G) above ~1e5, so a panel
// with condition number up to ~1e7 is orthonormalised to FP32 precision.  Grid-wide
// reductions use a two-phase barrier (partials -> sliced sums -> broadcast); every barrier
// wait is bounded and sets the status word when it runs out.
// R = [C1 + C2 R1 | R2 R1] per panel is written when requested.
#include <cooperative_groups.h>

#include "common.cuh"
#include "blackwell.cuh"

namespace ssi {

namespace {

constexpr int PB = 32;          // panel width
constexpr int QR_THREADS = 256;
constexpr uint64_t BAR_NS = 2000000000ull;

struct QrParams {
  float* A;            // rows x ld, first ncols columns are factorised in place (-> Q)
  int rows, ncols, ld;
  float* Rout;         // optional ncols x ncols row-major (upper triangular)
  float* red_c;        // [P][ncols*PB] projection partials
  float* fin_c;        // [ncols*PB] reduced projection
  double* red_g;       // [P][PB*PB] Gram partials (hi), [P][PB*PB] (lo) after
  double* fin_g;       // [PB*PB]
  unsigned* bar;       // [0] monotonic arrival counter of the grid barrier (zeroed per launch)
  int* status;
  int* abort_flag;
  int lds;             // leading dimension of the rows staged in shared memory (0: not staged)
  int n_chunks;        // row chunks (partials per reduction)
  int chunks_per_cta;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Grid barrier on a monotonic arrival counter (zeroed before the launch): barrier k of the
// launch is passed once the counter reaches k x gridDim.x.  One atomic per CTA, nothing
// to reset; a CTA that passes early cannot disturb the count of the barrier others still
// wait at.  The wait is bounded.
struct GridBar {
  unsigned n;   // barriers this CTA has entered in this launch
};

__device__ bool grid_sync(const QrParams& p, GridBar& gb) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    gb.n += 1;
    const unsigned target = gb.n * gridDim.x;
    __threadfence();
    const unsigned arrived = atomicAdd(&p.bar[0], 1u) + 1u;
    if (arrived < target) {
      const uint64_t t0 = bw::global_ns();
      while (*(volatile unsigned*)&p.bar[0] < target) {
        if (*(volatile int*)p.abort_flag) { ok = 0; break; }
        if (bw::global_ns() - t0 > BAR_NS) {
          atomicOr(p.status, DEV_TIMEOUT);
          atomicExch(p.abort_flag, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Sum over the C per-chunk partials of entries [e0, e1) (stride `stride` between
// partials).  Each entry is summed by RED_PER threads, thread q taking partials
// q, q + RED_PER, ... in order, and their sums are added in order: the same rounding
// whatever the grid and however the entries are split between CTAs.
constexpr int RED_PER = 8;
constexpr int RED_AHEAD = 20;   // >= 152 / RED_PER
template <typename T>
__device__ void slice_reduce(const T* part, size_t stride, int C, int e0, int e1, T* out) {
  __shared__ double red[QR_THREADS];
  const int E = e1 - e0;
  if (E <= 0) return;
  constexpr int EPP = QR_THREADS / RED_PER;   // entries per pass
  const int tid = threadIdx.x;
  const int sub = tid % RED_PER;
  for (int base = 0; base < E; base += EPP) {
    const int le = base + tid / RED_PER;
    double s = 0.0;
    if (le < E) {
      // up to RED_AHEAD partials loaded ahead of their adds (one L2 round trip for one
      // chunk per SM; same order of addition)
      for (int cb = sub; cb < C; cb += RED_AHEAD * RED_PER) {
        T v[RED_AHEAD];
#pragma unroll
        for (int u = 0; u < RED_AHEAD; ++u) {
          const int c = cb + u * RED_PER;
          v[u] = (c < C) ? part[(size_t)c * stride + e0 + le] : T(0);
        }
#pragma unroll
        for (int u = 0; u < RED_AHEAD; ++u) s += (double)v[u];
      }
    }
    red[tid] = s;
    __syncthreads();
    if (sub == 0 && le < E) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < RED_PER; ++q) t += red[tid + q];
      out[e0 + le] = (T)t;
    }
    __syncthreads();
  }
}

// FP32 Cholesky of a w x w Gram matrix by the whole CTA, on an FP32 copy of its upper
// triangle in buf (PB x PB, shared memory).  Two columns per step: every thread forms
// both pivots itself, warp 0 writes rows j and j+1 of R, and the warps apply the rank-2
// update to the trailing triangle (rows by warp, columns by lane); one barrier per step.
// Writes R (FP64, upper, zero elsewhere) and 1 / R[j][j].  Returns min_j pivot_j /
// max_j G[j][j], an estimate of 1 / cond(G) that decides whether the FP32 factor is
// accurate enough (the same in every thread).
__device__ float chol_cta_f32(const double* G, int w, double* R, double* rdiag, float* buf) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = QR_THREADS / 32;
  for (int e = tid; e < PB * PB; e += QR_THREADS) {
    const int a = e / PB, c = e % PB;
    buf[e] = (a < w && c < w && a <= c) ? (float)G[e] : 0.f;
    R[e] = 0.0;
  }
  __syncthreads();
  float gmax = 0.f, dmin = 3.0e38f;
  for (int j = 0; j < w; ++j) gmax = fmaxf(gmax, buf[j * PB + j]);
  // two columns per barrier: rows j and j+1 of R and the rank-2 update of the trailing
  // triangle; row j+1 after the rank-1 step of column j is formed where it is needed,
  // u[c] = G[j+1][c] - G[j][j+1] G[j][c] / d_j
  for (int j = 0; j < w; j += 2) {
    const bool two = j + 1 < w;
    const float d0 = buf[j * PB + j];
    const float rs0 = rsqrtf(fmaxf(d0, 1e-30f)), q0 = rs0 * rs0;
    const float g01 = two ? buf[j * PB + j + 1] : 0.f;
    const float d1 = two ? fmaf(-g01 * q0, g01, buf[(j + 1) * PB + j + 1]) : 1.f;
    const float rs1 = rsqrtf(fmaxf(d1, 1e-30f)), q1 = rs1 * rs1;
    dmin = fminf(dmin, two ? fminf(d0, d1) : d0);
    if (warp == 0 && lane < w) {
      const float g0l = buf[j * PB + lane];
      if (lane >= j) R[j * PB + lane] = (double)(g0l * rs0);   // lane == j: sqrt(d0)
      if (lane == j) rdiag[j] = (double)rs0;
      if (two && lane >= j + 1) {
        const float ul = (lane == j + 1) ? d1 : fmaf(-g01 * q0, g0l, buf[(j + 1) * PB + lane]);
        R[(j + 1) * PB + lane] = (double)(ul * rs1);   // lane == j+1: sqrt(d1)
        if (lane == j + 1) rdiag[j + 1] = (double)rs1;
      }
    }
    // G[a][c] -= G[j][a] G[j][c] / d0 + u[a] u[c] / d1 for j+2 <= a <= c: a lane's rows are
    // loaded first, then updated, so their shared-memory round trips overlap
    const int c = lane;
    if (two && c >= j + 2 && c < w) {
      const float g0c = buf[j * PB + c];
      const float uc = fmaf(-g01 * q0, g0c, buf[(j + 1) * PB + c]);
      const float g0cq = g0c * q0, ucq = uc * q1;
      constexpr int RPWARP = PB / (QR_THREADS / 32);
      float g0a[RPWARP], g1a[RPWARP], gac[RPWARP];
#pragma unroll
      for (int k = 0; k < RPWARP; ++k) {
        const int a = j + 2 + warp + k * nwarps;
        g0a[k] = (a <= c) ? buf[j * PB + a] : 0.f;
        g1a[k] = (a <= c) ? buf[(j + 1) * PB + a] : 0.f;
        gac[k] = (a <= c) ? buf[a * PB + c] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < RPWARP; ++k) {
        const int a = j + 2 + warp + k * nwarps;
        if (a <= c) {
          const float ua = fmaf(-g01 * q0, g0a[k], g1a[k]);
          buf[a * PB + c] = fmaf(-ua, ucq, fmaf(-g0a[k], g0cq, gac[k]));
        }
      }
    }
    __syncthreads();
  }
  return (w == 0) ? 1.f : (gmax > 0.f ? dmin / gmax : 0.f);
}

// Cholesky of the w x w Gram matrix G (FP64, upper triangle used) by the whole CTA.  Per
// step j, thread 0 forms 1/R[j][j] (reciprocal square root: FP32 seed and two Newton
// steps in FP64, since FP64 division and square root are long instruction sequences on
// this part); then, between the same two barriers, row j of R is written
// (R[j][c] = G[j][c] / R[j][j]) and the trailing upper triangle is updated from the
// unscaled row (G[a][c] -= G[j][a] G[j][c] / R[j][j]^2).  Warps take rows, lanes
// columns.  Writes R (upper, zero elsewhere) and 1 / R[j][j].
__device__ void chol_cta(double* G, int w, double* R, double* rdiag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = QR_THREADS / 32;
  __shared__ double s_floor;
  if (tid == 0) {
    double gmax = 0.0;
    for (int j = 0; j < w; ++j) gmax = fmax(gmax, G[j * PB + j]);
    s_floor = fmax(gmax * 1e-14, 1e-300);
  }
  for (int e = tid; e < PB * PB; e += QR_THREADS) R[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < w; ++j) {
    if (tid == 0) {
      const double d = fmax(G[j * PB + j], s_floor);
      double y = (double)rsqrtf((float)d);
      y = y * (1.5 - 0.5 * d * y * y);
      y = y * (1.5 - 0.5 * d * y * y);
      rdiag[j] = y;
      R[j * PB + j] = d * y;
    }
    __syncthreads();
    const double rs = rdiag[j], rs2 = rs * rs;
    if (warp == 0 && lane > j && lane < w) R[j * PB + lane] = G[j * PB + lane] * rs;
    const int c = lane;
    if (c > j && c < w) {
      const double gjc = G[j * PB + c] * rs2;
      for (int a = j + 1 + warp; a <= c; a += nwarps) G[a * PB + c] -= G[j * PB + a] * gjc;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(QR_THREADS, 1)   // one CTA per SM (cooperative grid)
    k_qr_bcgs2(QrParams p) {
  extern __shared__ float s_rows[];     // this CTA's rows (when they fit), leading dim p.lds
  __shared__ double sG[PB * PB];
  __shared__ double sR[2][PB * PB];     // R1, R2 of the current panel
  __shared__ double sRd[PB];            // 1 / R[j][j] of the current factor
  __shared__ float sRf[PB * PB];        // current factor in FP32
  __shared__ float sRdf[PB];
  GridBar gb;
  gb.n = 0;

  const int P = gridDim.x;
  const int C = p.n_chunks;
  const int rows_per = (p.rows + C - 1) / C;            // rows of a chunk
  const int c0 = blockIdx.x * p.chunks_per_cta;         // this CTA's chunks [c0, c1)
  const int c1 = min(C, c0 + p.chunks_per_cta);
  const int r0 = min(p.rows, c0 * rows_per);
  const int r1 = min(p.rows, c1 * rows_per);
  const int nr = max(0, r1 - r0);
  const int tid = threadIdx.x;
  // local rows: shared memory when they fit, else the matrix itself
  float* Ab = p.lds ? s_rows : p.A + (size_t)r0 * p.ld;
  const int ldb = p.lds ? p.lds : p.ld;
  // the reduced projection C (j0 x PB), 16-byte aligned for float4 rows
  float* sC = p.lds ? s_rows + (((size_t)rows_per * p.chunks_per_cta * p.lds + 3) & ~size_t(3))
                    : nullptr;
  if (p.lds) {
    for (int e = tid; e < nr * p.ncols; e += QR_THREADS) {
      const int rr = e / p.ncols, c = e % p.ncols;
      Ab[rr * ldb + c] = p.A[(size_t)(r0 + rr) * p.ld + c];
    }
    __syncthreads();
  }

  for (int j0 = 0; j0 < p.ncols; j0 += PB) {
    const int w = min(PB, p.ncols - j0);
    for (int pass = 0; pass < 2; ++pass) {
      if (j0 > 0) {
        // ---- C = Q[:, :j0]^T W, partial over this CTA's rows
        const int nC = j0 * PB;
        // 4 x 4 outputs per thread: rows a0..a0+3 of Q^T, columns b0..b0+3 of the panel;
        // one partial per chunk
        const int n_tiles = (j0 / 4) * (PB / 4);
        for (int tc = tid; tc < n_tiles * (c1 - c0); tc += QR_THREADS) {
          const int ch = tc / n_tiles, tt = tc % n_tiles;
          float* myC = p.red_c + (size_t)(c0 + ch) * p.ncols * PB;
          const int lr0 = ch * rows_per, lr1 = min(nr, lr0 + rows_per);
          const int a0 = 4 * (tt / (PB / 4)), b0 = 4 * (tt % (PB / 4));
          float acc[4][4] = {};
          for (int rr = lr0; rr < lr1; ++rr) {
            const float* row = Ab + rr * ldb;
            float qa[4], wb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              qa[u] = row[a0 + u];
              wb[u] = (b0 + u < w) ? row[j0 + b0 + u] : 0.f;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[i][u] = fmaf(qa[i], wb[u], acc[i][u]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int u = 0; u < 4; ++u) myC[(a0 + i) * PB + b0 + u] = acc[i][u];
        }
        if (!grid_sync(p, gb)) return;
        {
          const int per_cta = (nC + P - 1) / P;
          const int e0 = blockIdx.x * per_cta, e1 = min(nC, e0 + per_cta);
          slice_reduce<float>(p.red_c, (size_t)p.ncols * PB, C, e0, e1, p.fin_c);
        }
        if (!grid_sync(p, gb)) return;
        const float* C = p.fin_c;
        if (sC) {
          for (int e = tid; e < nC; e += QR_THREADS) sC[e] = p.fin_c[e];
          __syncthreads();
          C = sC;
        }
        // ---- W -= Q[:, :j0] C on local rows: UR_ROWS rows x 4 columns per thread (three
        //      rows keep 200 of the 256 threads busy on a 74-row chunk)
        constexpr int UR_ROWS = 3;
        for (int tt = tid; tt < ((nr + UR_ROWS - 1) / UR_ROWS) * (PB / 4); tt += QR_THREADS) {
          const int r0 = UR_ROWS * (tt / (PB / 4)), b0 = 4 * (tt % (PB / 4));
          float acc[UR_ROWS][4] = {};
          for (int a = 0; a < j0; ++a) {
            float qv[UR_ROWS], cv[4];
#pragma unroll
            for (int i = 0; i < UR_ROWS; ++i) qv[i] = (r0 + i < nr) ? Ab[(r0 + i) * ldb + a] : 0.f;
            {
              const float4 c4 = *reinterpret_cast<const float4*>(C + a * PB + b0);
              cv[0] = c4.x;
              cv[1] = c4.y;
              cv[2] = c4.z;
              cv[3] = c4.w;
            }
#pragma unroll
            for (int i = 0; i < UR_ROWS; ++i)
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[i][u] = fmaf(qv[i], cv[u], acc[i][u]);
          }
#pragma unroll
          for (int i = 0; i < UR_ROWS; ++i)
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (r0 + i < nr && b0 + u < w) Ab[(r0 + i) * ldb + j0 + b0 + u] -= acc[i][u];
        }
        if (p.Rout && blockIdx.x == 0) {
          // R[:j0, j0+b] accumulates C1 + C2 R1
          for (int e = tid; e < j0 * PB; e += QR_THREADS) {
            const int a = e / PB, b = e % PB;
            if (b >= w) continue;
            if (pass == 0) {
              p.Rout[(size_t)a * p.ncols + j0 + b] = C[e];
            } else {
              float s = 0.f;
              for (int c = 0; c <= b; ++c) s = fmaf(C[a * PB + c], (float)sR[0][c * PB + b], s);
              p.Rout[(size_t)a * p.ncols + j0 + b] += s;
            }
          }
        }
        __syncthreads();
      }
      // ---- Gram G = W^T W over each chunk's rows: the 36 upper 4 x 4 tiles of the 32 x 32
      // panel Gram (the lower triangle is never read).  Four adjacent lanes per (chunk,
      // tile) take every fourth row and are merged by shuffles in a fixed order, so a
      // chunk's sum is the same whatever the number of chunks per CTA.  First pass
      // (the panel may be ill-conditioned): double-FP32, exact products by fma and sums by
      // two-sum.  Second pass (the panel is orthonormal to ~1e-4, G close to I): FP32.
      {
        const int nch = c1 - c0;
        constexpr int RG = 4;
        const int rg = tid % RG;
        // every lane runs the same number of iterations (the merge below shuffles across
        // the whole warp); slots past the last (chunk, tile) accumulate nothing
        const int n_combo = 36 * nch;
        const int n_iter = (n_combo + QR_THREADS / RG - 1) / (QR_THREADS / RG);
        for (int it = 0; it < n_iter; ++it) {
          const int combo = tid / RG + it * (QR_THREADS / RG);
          const bool valid = combo < n_combo;
          const int ch = valid ? combo / 36 : 0;
          int t = valid ? combo % 36 : 0, ta = 0;
          while (t >= 8 - ta) { t -= 8 - ta; ++ta; }
          const int a0 = 4 * ta, b0 = 4 * (ta + t);
          const int lr0 = ch * rows_per, lr1 = valid ? min(nr, lr0 + rows_per) : lr0;
          double* myG = p.red_g + (size_t)(c0 + ch) * PB * PB;
          float sh[4][4] = {}, sl[4][4] = {};
          for (int rr = lr0 + rg; rr < lr1; rr += RG) {
            float xa[4], yb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              xa[u] = (a0 + u < w) ? Ab[rr * ldb + j0 + a0 + u] : 0.f;
              yb[u] = (b0 + u < w) ? Ab[rr * ldb + j0 + b0 + u] : 0.f;
            }
            if (pass == 0) {
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const float pr = xa[i] * yb[u];
                  const float pe = fmaf(xa[i], yb[u], -pr);
                  float s2, e2;
                  two_sum(sh[i][u], pr, s2, e2);
                  sh[i][u] = s2;
                  sl[i][u] += e2 + pe;
                }
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int u = 0; u < 4; ++u) sh[i][u] = fmaf(xa[i], yb[u], sh[i][u]);
            }
          }
#pragma unroll
          for (int o = 1; o < RG; o <<= 1)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float h2 = __shfl_xor_sync(0xffffffffu, sh[i][u], o);
                const float l2 = __shfl_xor_sync(0xffffffffu, sl[i][u], o);
                float s2, e2;
                two_sum(sh[i][u], h2, s2, e2);
                sh[i][u] = s2;
                sl[i][u] += l2 + e2;
              }
          if (valid && rg == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int u = 0; u < 4; ++u)
                myG[(a0 + i) * PB + b0 + u] =
                    (a0 + i <= b0 + u) ? (double)sh[i][u] + (double)sl[i][u] : 0.0;
          }
        }
        if (!grid_sync(p, gb)) return;
        {
          const int per_cta = (PB * PB + P - 1) / P;
          const int e0 = blockIdx.x * per_cta, e1 = min(PB * PB, e0 + per_cta);
          slice_reduce<double>(p.red_g, (size_t)PB * PB, C, e0, e1, p.fin_g);
        }
        if (!grid_sync(p, gb)) return;
      }
      // ---- Cholesky (FP64, whole CTA, every CTA) and W <- W R^{-1} row by row (FP32)
      for (int e = tid; e < PB * PB; e += QR_THREADS) {
        const int a = e / PB, b = e % PB;
        sG[e] = (a < w && b < w && a <= b) ? p.fin_g[e] : 0.0;
      }
      __syncthreads();
      // FP32 Cholesky by the CTA; the first pass falls back to the FP64 factorisation
      // when a pivot is below 1e-5 of the largest diagonal (cond(G) above ~1e5, where the
      // FP32 factor would be too inaccurate for the second pass to repair).  Every CTA
      // factors the same G, so every CTA takes the same branch.
      {
        const float ratio = chol_cta_f32(sG, w, sR[pass], sRd, sRf);
        const bool f32ok = (pass == 1) || ratio >= 1e-5f;
        if (!f32ok) chol_cta(sG, w, sR[pass], sRd);
      }
      for (int e = tid; e < PB * PB; e += QR_THREADS) sRf[e] = (float)sR[pass][e];
      for (int e = tid; e < PB; e += QR_THREADS) sRdf[e] = (float)sRd[e];
      __syncthreads();
      for (int rr = tid; rr < nr; rr += QR_THREADS) {
        float x[PB];
#pragma unroll
        for (int b = 0; b < PB; ++b) x[b] = (b < w) ? Ab[rr * ldb + j0 + b] : 0.f;
        // solve x_new R = x (forward substitution over columns)
#pragma unroll
        for (int b = 0; b < PB; ++b) {
          float s = x[b];
#pragma unroll
          for (int a = 0; a < b; ++a) s = fmaf(-x[a], sRf[a * PB + b], s);
          x[b] = s * sRdf[b];
        }
#pragma unroll
        for (int b = 0; b < PB; ++b)
          if (b < w) Ab[rr * ldb + j0 + b] = x[b];
      }
      __syncthreads();
    }
    if (p.Rout && blockIdx.x == 0) {
      // diagonal block R2 R1
      for (int e = tid; e < PB * PB; e += QR_THREADS) {
        const int a = e / PB, b = e % PB;
        if (a >= w || b >= w) continue;
        double s = 0.0;
        for (int c = a; c <= b; ++c) s += sR[1][a * PB + c] * sR[0][c * PB + b];
        p.Rout[(size_t)(j0 + a) * p.ncols + j0 + b] = (float)s;
      }
    }
    __syncthreads();
  }
  if (p.lds) {
    for (int e = tid; e < nr * p.ncols; e += QR_THREADS) {
      const int rr = e / p.ncols, c = e % p.ncols;
      p.A[(size_t)(r0 + rr) * p.ld + c] = Ab[rr * ldb + c];
    }
  }
}

}  // namespace

size_t qr_ws_bytes(int ncols, int num_sms) {
  WsPlan w;
  w.add<float>((size_t)num_sms * ncols * PB);
  w.add<float>((size_t)ncols * PB);
  w.add<double>((size_t)num_sms * PB * PB);
  w.add<double>((size_t)PB * PB);
  w.add<unsigned>(64);
  return w.bytes;
}

// QR of A (rows x ncols, leading dimension ld) in place; optional R (ncols x ncols).
ssi_status qr_launch(ssi_ctx* ctx, Workspace& ws, float* A, int rows, int ncols, int ld, float* Rout,
                     int* status, cudaStream_t stream, bool shared_device, int chunks_per_cta) {
  if (rows < ncols) {
    set_error("qr: rows (%d) < columns (%d)", rows, ncols);
    return SSI_E_INVALID;
  }
  QrParams p{};
  p.A = A;
  p.rows = rows;
  p.ncols = ncols;
  p.ld = ld;
  p.Rout = Rout;
  // chunks: one per SM (fixed for the device and the shape, so the result is too); a CTA
  // per chunk when the solve has the device to itself, and when several solves (or
  // several lags of one solve) share it, a CTA per two chunks or the autotuner's choice
  // for that case.  The grouping changes which CTA sums a chunk, not the order of any sum.
  const int C = std::max(1, std::min<int>(ctx->num_sms, (int)ceil_div(rows, 32)));
  const bool shared = ctx->inflight > 1 || shared_device;
  const int cpc = !shared ? 1 : chunks_per_cta > 0 ? std::min(chunks_per_cta, C) : 2;
  const int P = (int)ceil_div(C, cpc);
  p.n_chunks = C;
  p.chunks_per_cta = cpc;
  const int rows_per = (int)ceil_div(rows, C) * cpc;   // rows of a CTA
  const int lds = ncols | 1;   // odd leading dimension: rows of a warp fall in distinct banks
  size_t smem = ((size_t)rows_per * lds + 4 + (size_t)ncols * PB) * sizeof(float);
  if (smem > 192 * 1024) {
    smem = 0;   // rows stay in global memory
  } else {
    p.lds = lds;
  }
  SSI_CUDA(cudaFuncSetAttribute(k_qr_bcgs2, cudaFuncAttributeMaxDynamicSharedMemorySize, 192 * 1024));
  p.red_c = ws.take<float>((size_t)ctx->num_sms * ncols * PB);
  p.fin_c = ws.take<float>((size_t)ncols * PB);
  p.red_g = ws.take<double>((size_t)ctx->num_sms * PB * PB);
  p.fin_g = ws.take<double>((size_t)PB * PB);
  unsigned* bar = ws.take<unsigned>(64);
  if (!p.red_c || !p.fin_c || !p.red_g || !p.fin_g || !bar) {
    set_error("qr: workspace too small");
    return SSI_E_NOMEM;
  }
  p.bar = bar;
  p.abort_flag = reinterpret_cast<int*>(bar + 8);
  p.status = status;
  SSI_CUDA(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), stream));
  if (Rout) SSI_CUDA(cudaMemsetAsync(Rout, 0, sizeof(float) * ncols * ncols, stream));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(QR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SSI_CUDA(cudaLaunchKernelEx(&cfg, k_qr_bcgs2, p));
  return SSI_OK;
}

}  // namespace ssi
