// Economy QR of a tall-skinny FP32 matrix (the sketch re-orthonormalisation of Sec. 2.2,
// "(Q, R) = qr(Y, 0)" of Algorithm 1).
//
// One cooperative persistent kernel.  Each CTA owns a contiguous block of rows;
// columns are processed in panels of 32:
//   pass 1:  W  = Y_j - Q_{<j} (Q_{<j}^T Y_j);   W  = W R1^{-1},  R1 = chol(W^T W)
//   pass 2:  W' = W   - Q_{<j} (Q_{<j}^T W);     Q_j = W' R2^{-1}, R2 = chol(W'^T W')
// (block classical Gram-Schmidt with re-orthogonalisation, each panel made
// orthonormal by Cholesky-QR).  The Gram matrices are accumulated in double-FP32
// (error-free products with fma, two-sum accumulation) and reduced in FP64, the
// 32x32 Cholesky runs in FP64 redundantly in every CTA, so a panel with condition
// number up to ~1e7 is orthonormalised to FP32 precision.  Grid-wide reductions
// use a two-phase barrier (partials -> sliced sums -> broadcast); every barrier
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
  unsigned* bar;       // [2] arrival counter, generation
  int* status;
  int* abort_flag;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct GridBar {
  unsigned gen;
};

__device__ bool grid_sync(const QrParams& p, GridBar& gb) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned arrived = atomicAdd(&p.bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&p.bar[0], 0u);
      __threadfence();
      atomicAdd(&p.bar[1], 1u);
    } else {
      const uint64_t t0 = bw::global_ns();
      while (*(volatile unsigned*)&p.bar[1] == gb.gen) {
        if (*(volatile int*)p.abort_flag) { ok = 0; break; }
        if (bw::global_ns() - t0 > BAR_NS) {
          atomicOr(p.status, DEV_TIMEOUT);
          atomicExch(p.abort_flag, 1);
          ok = 0;
          break;
        }
      }
    }
    gb.gen += 1;
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// In-place FP64 Cholesky of the w x w matrix G (row-major, lower part used), executed by
// one warp; returns the upper factor R (R^T R = G) in Rm and its inverse in Ri.
__device__ void chol_inv_warp(const double* G, int w, double* Rm, double* Ri, int lane) {
  // R computed row by row: R[j][j] = sqrt(G[j][j] - sum_k<j R[k][j]^2),
  // R[j][c] = (G[j][c] - sum_k<j R[k][j] R[k][c]) / R[j][j]
  double gmax = 0.0;
  for (int j = 0; j < w; ++j) gmax = fmax(gmax, G[j * PB + j]);
  const double floor_v = fmax(gmax * 1e-14, 1e-300);
  for (int j = 0; j < w; ++j) {
    double d = G[j * PB + j];
    for (int k = 0; k < j; ++k) d -= Rm[k * PB + j] * Rm[k * PB + j];
    d = sqrt(fmax(d, floor_v));
    __syncwarp();
    for (int c = lane; c < w; c += 32) {
      if (c == j) Rm[j * PB + j] = d;
      else if (c > j) {
        double s = G[j * PB + c];
        for (int k = 0; k < j; ++k) s -= Rm[k * PB + j] * Rm[k * PB + c];
        Rm[j * PB + c] = s / d;
      } else {
        Rm[j * PB + c] = 0.0;
      }
    }
    __syncwarp();
  }
  // inverse of the upper triangular R by column back substitution: lane = column
  for (int c = lane; c < w; c += 32) {
    for (int r = w - 1; r >= 0; --r) {
      double s = (r == c) ? 1.0 : 0.0;
      for (int k = r + 1; k <= c; ++k) s -= Rm[r * PB + k] * Ri[k * PB + c];
      Ri[r * PB + c] = (r <= c) ? s / Rm[r * PB + r] : 0.0;
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(QR_THREADS)
    k_qr_bcgs2(QrParams p) {
  __shared__ double sG[PB * PB];
  __shared__ double sR[2][PB * PB];     // R1, R2 of the current panel
  __shared__ double sRi[PB * PB];
  __shared__ float sRif[PB * PB];
  __shared__ float sW[64][PB + 1];      // staging for local row updates
  GridBar gb;
  gb.gen = *(volatile unsigned*)&p.bar[1];

  const int P = gridDim.x;
  const int rows_per = (p.rows + P - 1) / P;
  const int r0 = blockIdx.x * rows_per;
  const int r1 = min(p.rows, r0 + rows_per);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;

  for (int j0 = 0; j0 < p.ncols; j0 += PB) {
    const int w = min(PB, p.ncols - j0);
    for (int pass = 0; pass < 2; ++pass) {
      if (j0 > 0) {
        // ---- C = Q[:, :j0]^T W, partial over this CTA's rows
        const int nC = j0 * PB;
        float* myC = p.red_c + (size_t)blockIdx.x * p.ncols * PB;
        for (int e = tid; e < nC; e += QR_THREADS) {
          const int a = e / PB, b = e % PB;
          float s = 0.f;
          if (b < w)
            for (int r = r0; r < r1; ++r) s = fmaf(p.A[(size_t)r * p.ld + a], p.A[(size_t)r * p.ld + j0 + b], s);
          myC[e] = s;
        }
        if (!grid_sync(p, gb)) return;
        for (int e = blockIdx.x * QR_THREADS + tid; e < nC; e += P * QR_THREADS) {
          float s = 0.f;
          for (int c = 0; c < P; ++c) s += p.red_c[(size_t)c * p.ncols * PB + e];
          p.fin_c[e] = s;
        }
        if (!grid_sync(p, gb)) return;
        // ---- W -= Q[:, :j0] C on local rows
        for (int rb = r0; rb < r1; rb += 64) {
          const int nr = min(64, r1 - rb);
          for (int e = tid; e < nr * PB; e += QR_THREADS) {
            const int rr = e / PB, b = e % PB;
            float s = 0.f;
            if (b < w) {
              const float* qrow = p.A + (size_t)(rb + rr) * p.ld;
              for (int a = 0; a < j0; ++a) s = fmaf(qrow[a], p.fin_c[a * PB + b], s);
            }
            sW[rr][b] = s;
          }
          __syncthreads();
          for (int e = tid; e < nr * PB; e += QR_THREADS) {
            const int rr = e / PB, b = e % PB;
            if (b < w) p.A[(size_t)(rb + rr) * p.ld + j0 + b] -= sW[rr][b];
          }
          __syncthreads();
        }
        if (p.Rout && blockIdx.x == 0) {
          // R[:j0, j0+b] accumulates C1 + C2 R1 (pass 1 adds C2 * R1 later)
          for (int e = tid; e < j0 * PB; e += QR_THREADS) {
            const int a = e / PB, b = e % PB;
            if (b >= w) continue;
            if (pass == 0) {
              p.Rout[(size_t)a * p.ncols + j0 + b] = p.fin_c[e];
            } else {
              float s = 0.f;
              for (int c = 0; c <= b; ++c) s = fmaf(p.fin_c[a * PB + c], (float)sR[0][c * PB + b], s);
              p.Rout[(size_t)a * p.ncols + j0 + b] += s;
            }
          }
        }
      }
      // ---- Gram G = W^T W in double-FP32 over local rows
      {
        double* myG = p.red_g + (size_t)blockIdx.x * PB * PB;
        for (int e = tid; e < PB * PB; e += QR_THREADS) {
          const int a = e / PB, b = e % PB;
          float sh = 0.f, sl = 0.f;
          if (a < w && b < w && a <= b) {
            for (int r = r0; r < r1; ++r) {
              const float x = p.A[(size_t)r * p.ld + j0 + a];
              const float y = p.A[(size_t)r * p.ld + j0 + b];
              const float pr = x * y;
              const float pe = fmaf(x, y, -pr);
              float s, e2;
              two_sum(sh, pr, s, e2);
              sh = s;
              sl += e2 + pe;
            }
          }
          myG[e] = (double)sh + (double)sl;
        }
        if (!grid_sync(p, gb)) return;
        for (int e = blockIdx.x * QR_THREADS + tid; e < PB * PB; e += P * QR_THREADS) {
          double s = 0.0;
          for (int c = 0; c < P; ++c) s += p.red_g[(size_t)c * PB * PB + e];
          p.fin_g[e] = s;
        }
        if (!grid_sync(p, gb)) return;
      }
      // ---- Cholesky (FP64, one warp, every CTA) and W <- W R^{-1}
      for (int e = tid; e < PB * PB; e += QR_THREADS) {
        const int a = e / PB, b = e % PB;
        const double g = (a <= b) ? p.fin_g[a * PB + b] : p.fin_g[b * PB + a];
        sG[e] = (a < w && b < w) ? g : 0.0;
        sR[pass][e] = 0.0;
        sRi[e] = 0.0;
      }
      __syncthreads();
      if (warp == 0) chol_inv_warp(sG, w, sR[pass], sRi, lane);
      __syncthreads();
      for (int e = tid; e < PB * PB; e += QR_THREADS) sRif[e] = (float)sRi[e];
      __syncthreads();
      for (int rb = r0; rb < r1; rb += 64) {
        const int nr = min(64, r1 - rb);
        for (int e = tid; e < nr * PB; e += QR_THREADS) {
          const int rr = e / PB, b = e % PB;
          sW[rr][b] = (b < w) ? p.A[(size_t)(rb + rr) * p.ld + j0 + b] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < nr * PB; e += QR_THREADS) {
          const int rr = e / PB, b = e % PB;
          if (b >= w) continue;
          float s = 0.f;
          for (int a = 0; a <= b; ++a) s = fmaf(sW[rr][a], sRif[a * PB + b], s);
          p.A[(size_t)(rb + rr) * p.ld + j0 + b] = s;
        }
        __syncthreads();
      }
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
      for (int e = tid; e < PB * p.ncols; e += QR_THREADS) {
        const int a = e / p.ncols, b = e % p.ncols;
        if (a < w && b < j0) p.Rout[(size_t)(j0 + a) * p.ncols + b] = 0.f;
      }
    }
    __syncthreads();
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
                     int* status, cudaStream_t stream) {
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
  int per_sm = 0;
  SSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_bcgs2, QR_THREADS, 0));
  int P = std::min<int>(ctx->num_sms * std::max(per_sm, 1), ctx->num_sms);
  P = std::max(1, std::min<int>(P, (int)ceil_div(rows, 32)));
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
  cfg.dynamicSmemBytes = 0;
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
