// Stages (a2)-(b): the block-Toeplitz matrix T_{1|i} (Eq. Toeplitz, block (a,b) = R_{i+a-b})
// kept implicit, and its randomized SVD (Sec. 2.2, Algorithm 1 with oversampling and
// power iterations).
//
// Layout (padded): every l x l covariance becomes an l_pad x l_pad block (l_pad = multiple
// of 64, zero padding), so T_pad is (i*l_pad)^2 and a 64-row tile never straddles a
// block.  The sketch bases X live as L_pad x Kp row-major matrices.
//
// k_toeplitz_gemm_tc<MODE>: D = T X (MODE 0) or D = T^T X (MODE 1) on tcgen05.  The
// A operand is never formed: for each 64-row half of a 128-row M tile and each
// 32-column K stage, the lag index i + a - b selects the covariance block and TMA
// loads the tile straight from the BF16 covariance store.  For T the tile is K-major
// (64-byte swizzle, 32 columns), for T^T the same bytes are read MN-major (128-byte
// swizzle), so one store serves both products.  X is MN-major.  Split-BF16: three
// MMAs per k-step.  A CTA takes MT (1 or 2) M tiles against one N tile of X: with two,
// a stage brings 64 KB for twelve 128 x 256 x 16 MMAs instead of 48 KB for six, which
// is what keeps the tensor pipe fed from L2.  When the accumulators of a unit use at
// most half of TMEM, two sets let the epilogue of one unit overlap the MMAs of the
// next; otherwise the epilogue (a few hundred cycles against the unit's thousands of
// MMA cycles) runs between units.  A unit is (M tile group, N tile, K split); FP32
// partials per split are summed by k_sum_splits.
#include "common.cuh"
#include "blackwell.cuh"

namespace ssi {

// qr.cu / svd.cu
size_t qr_ws_bytes(int ncols, int num_sms);
ssi_status qr_launch(ssi_ctx* ctx, Workspace& ws, float* A, int rows, int ncols, int ld,
                     float* Rout, int* status, cudaStream_t stream, bool shared_device,
                     int chunks_per_cta = 0);
size_t jacobi_ws_bytes(int K, int num_sms, bool fp64);
ssi_status jacobi_launch64(Workspace& ws, const float* R2, int K, double* Ut, double* S, int* status,
                           int num_sms, int block, cudaStream_t stream);
ssi_status jacobi_launch(Workspace& ws, const float* R2, int K, float* Ut, float* S, int* status,
                         int num_sms, int block, cudaStream_t stream);

namespace {

constexpr int SBK = 32;                 // K rows per stage
constexpr int BOX_BYTES = 4096;         // 64 x 32 bf16 box
constexpr int TG_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ float gaussian_at(uint32_t r, uint32_t c, uint64_t seed) {
  uint32_t x0 = r, x1 = c, x2 = 0, x3 = 0;
  philox4x32_10(x0, x1, x2, x3, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const float u0 = ((float)x0 + 0.5f) * 2.3283064365386963e-10f;
  const float u1 = ((float)x1 + 0.5f) * 2.3283064365386963e-10f;
  return sqrtf(-2.f * logf(u0)) * cospif(2.f * u1);
}

// Omega: plain (rows x cols, ld) when `plain` != null; padded Toeplitz-column layout
// (row b*l_pad + c <- real row b*l + c, zero for c >= l or col >= cols) otherwise.
__global__ void k_omega(int rows, int cols, int ld, uint64_t seed, float* __restrict__ plain,
                        int l, int l_pad, int n_rows_pad, float* __restrict__ f32,
                        __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long total = plain ? (long long)rows * ld : (long long)n_rows_pad * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int rp = (int)(e / ld), col = (int)(e % ld);
    float z = 0.f;
    if (plain) {
      if (col < cols) z = gaussian_at((uint32_t)rp, (uint32_t)col, seed);
      plain[e] = z;
      continue;
    }
    const int b = rp / l_pad, c = rp % l_pad;
    if (c < l && col < cols) z = gaussian_at((uint32_t)(b * l + c), (uint32_t)col, seed);
    if (f32) f32[e] = z;
    if (hi) {
      const __nv_bfloat16 h = __float2bfloat16_rn(z);
      hi[e] = h;
      lo[e] = __float2bfloat16_rn(z - __bfloat162float(h));
    }
  }
}

// covariance store: R (n_lag x l x l, fp64) -> padded n_lag x l_pad x l_pad (bf16 hi/lo or fp32)
__global__ void k_r_store(const double* __restrict__ R, int n_lag, int l, int l_pad,
                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                          float* __restrict__ f32) {
  const long long total = (long long)n_lag * l_pad * l_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int cb = (int)(e % l_pad);
    const int ca = (int)((e / l_pad) % l_pad);
    const int k = (int)(e / ((long long)l_pad * l_pad));
    const float x = (ca < l && cb < l) ? (float)R[((long long)k * l + ca) * l + cb] : 0.f;
    if (f32) f32[e] = x;
    if (hi) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      hi[e] = h;
      lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ hi,
                          __nv_bfloat16* __restrict__ lo) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float v = x[e];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Sum of the per-split FP32 partials of a sketch product: Knuth's two-sum in FP32 (hi +
// lo, about twice FP32 precision) in a fixed split order, eight partials loaded ahead of
// their adds; FP64 arithmetic on this part runs at a small fraction of the FP32 rate.
__global__ void k_sum_splits(const float* __restrict__ part, int n_split, long long stride,
                             float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < stride;
       e += (long long)gridDim.x * blockDim.x) {
    float hi = 0.f, lo = 0.f;
    for (int sp = 0; sp < n_split; sp += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (sp + u < n_split) ? __ldcs(part + (sp + u) * stride + e) : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float s2 = hi + v[u];
        const float bb = s2 - hi;
        lo += (hi - (s2 - bb)) + (v[u] - bb);
        hi = s2;
      }
    }
    out[e] = hi + lo;
  }
}

struct TgParams {
  int i, l_pad, L_pad;
  int n_mt, n_nt, n_split, krows;
  int ld;                 // Kp
  long long split_stride;
};

// ------------------------------------------------------------------ tcgen05 Toeplitz GEMM
template <int MODE, int NB, int MT, int STAGES>
__global__ void __launch_bounds__(TG_THREADS, 1)
    k_toeplitz_gemm_tc(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                       const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                       TgParams p, float* __restrict__ partial, int* __restrict__ status) {
  constexpr int NT = 64 * NB;
  constexpr int A_BYTES = 2 * BOX_BYTES;          // one M tile: two 64-row boxes
  constexpr int B_BYTES = NB * BOX_BYTES;
  constexpr int STAGE_BYTES = MT * 2 * A_BYTES + 2 * B_BYTES;
  constexpr int ACC = MT * NT;                    // TMEM columns of one unit's accumulators
  constexpr int NBUF = 2 * ACC <= 512 ? 2 : 1;
  constexpr uint32_t IDESC = bw::idesc_bf16(128, NT, MODE, 1);
  constexpr uint32_t TMEM_COLS = (NBUF * ACC <= 32) ? 32 : (NBUF * ACC <= 64) ? 64
                                 : (NBUF * ACC <= 128) ? 128 : (NBUF * ACC <= 256) ? 256 : 512;
  static_assert(NBUF * ACC <= 512, "accumulators exceed TMEM");
  static_assert(4 * MT + 2 * NB <= 32, "one lane per box");

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // [0,S) full, [S,2S) empty, [2S,2S+2) tmem full, [2S+2,2S+4) tmem empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = bw::smem_u32(smem);
  const uint32_t bar_base = bw::smem_u32(bars);
  auto full_bar = [&](int s) { return bar_base + 8u * s; };
  auto empty_bar = [&](int s) { return bar_base + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar_base + 8u * (2 * STAGES + 2 + b); };
  // accumulator set of the uc-th unit of this CTA, and how often that set was used before
  auto acc_buf = [](int uc) { return NBUF == 2 ? (uc & 1) : 0; };
  auto acc_use = [](int uc) { return NBUF == 2 ? (uc >> 1) : uc; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      bw::mbar_init(full_bar(s), 1);
      bw::mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      bw::mbar_init(tfull_bar(b), 1);
      bw::mbar_init(tempty_bar(b), 4);
    }
    *abort_flag = 0;
    bw::fence_mbar_init();
    bw::tma_prefetch_desc(&tA_hi);
    bw::tma_prefetch_desc(&tA_lo);
    bw::tma_prefetch_desc(&tB_hi);
    bw::tma_prefetch_desc(&tB_lo);
  }
  if (warp == 1) {
    bw::tmem_alloc(bw::smem_u32(tmem_slot), TMEM_COLS);
    bw::tmem_relinquish();
  }
  bw::tc_fence_before();
  __syncthreads();
  bw::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int n_units = p.n_mt * p.n_nt * p.n_split;
  auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
    if (bw::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = bw::global_ns();
    while (true) {
      if (bw::mbar_try_wait(bar, parity)) return true;
      if (*abort_flag) return false;
      if (bw::global_ns() - t0 > WAIT_NS) {
        atomicOr(status, DEV_TIMEOUT);
        *abort_flag = 1;
        return false;
      }
    }
  };
  auto unit_krange = [&](int u, int& j_begin, int& n_st) {
    const int sp = (u / p.n_mt) / p.n_nt;
    j_begin = sp * p.krows;
    const int j_end = min(p.L_pad, j_begin + p.krows);
    n_st = (j_end - j_begin) / SBK;
  };

  if (warp == 0) {
    // Lane 0 takes the barrier waits and the transaction count; each box of a stage
    // (A: MT tiles x 2 halves x hi/lo, B: NB atoms x hi/lo) is issued by its own lane.
    int g = 0;
    int armed_phase[STAGES];
    for (int s = 0; s < STAGES; ++s) armed_phase[s] = -1;
    bool ok = true;
    const bool lo_half = (lane & 1) != 0;
    const bool a_box = lane < 4 * MT;
    const bool b_box = lane >= 4 * MT && lane < 4 * MT + 2 * NB;
    const CUtensorMap* a_map = lo_half ? &tA_lo : &tA_hi;
    const CUtensorMap* b_map = lo_half ? &tB_lo : &tB_hi;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int mt = u % p.n_mt;
      const int nt = (u / p.n_mt) % p.n_nt;
      int j_begin, n_st;
      unit_krange(u, j_begin, n_st);
      const int m0 = mt * 128 * MT;
      for (int st = 0; st < n_st; ++st, ++g) {
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1;
        int okw = 1;
        if (lane == 0) {
          okw = wait(empty_bar(s), ph ^ 1) ? 1 : 0;
          if (okw) {
            bw::mbar_arrive_expect_tx(full_bar(s), (uint32_t)STAGE_BYTES);
            armed_phase[s] = (int)ph;
          }
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) { ok = false; break; }
        const uint32_t sb = smem_base + s * STAGE_BYTES;
        const int j0 = j_begin + st * SBK;
        if (a_box) {
          const int t = lane >> 2, h = (lane >> 1) & 1;
          const int mrow = m0 + 128 * t + 64 * h;
          int lag, x, y;
          if (MODE == 0) {
            const int a = mrow / p.l_pad, c0 = mrow % p.l_pad;
            const int b = j0 / p.l_pad, d0 = j0 % p.l_pad;
            lag = p.i + a - b;
            x = d0;
            y = (lag - 1) * p.l_pad + c0;
          } else {
            const int a = j0 / p.l_pad, c0 = j0 % p.l_pad;
            const int b = mrow / p.l_pad, d0 = mrow % p.l_pad;
            lag = p.i + a - b;
            x = d0;
            y = (lag - 1) * p.l_pad + c0;
          }
          bw::tma_load_2d(sb + t * 2 * A_BYTES + (lo_half ? A_BYTES : 0) + h * BOX_BYTES, a_map,
                          full_bar(s), x, y);
        } else if (b_box) {
          const int bb = (lane - 4 * MT) >> 1;
          const int x = nt * NT + bb * 64;
          bw::tma_load_2d(sb + MT * 2 * A_BYTES + (lo_half ? B_BYTES : 0) + bb * BOX_BYTES, b_map,
                          full_bar(s), x, j0);
        }
      }
    }
    if (lane == 0 && *abort_flag) {
      for (int s = 0; s < STAGES; ++s) {
        if (armed_phase[s] < 0) continue;
        const uint64_t t0 = bw::global_ns();
        while (!bw::mbar_try_wait(full_bar(s), (uint32_t)armed_phase[s]) &&
               bw::global_ns() - t0 < 50000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0, uc = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, ++uc) {
        int j_begin, n_st;
        unit_krange(u, j_begin, n_st);
        const int buf = acc_buf(uc);
        if (!wait(tempty_bar(buf), (acc_use(uc) & 1) ^ 1)) { ok = false; break; }
        bw::tc_fence_after();
        const uint32_t d = tmem_base + buf * ACC;
        for (int st = 0; st < n_st; ++st, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (!wait(full_bar(s), ph)) { ok = false; break; }
          bw::tc_fence_after();
          const uint32_t sb = smem_base + s * STAGE_BYTES;
#pragma unroll
          for (int kk = 0; kk < SBK / 16; ++kk) {
            const uint32_t sbb = sb + MT * 2 * A_BYTES;
            const uint64_t bh = bw::smem_desc(sbb + kk * 2048, BOX_BYTES, 1024, bw::SMEM_SW128);
            const uint64_t bl = bw::smem_desc(sbb + B_BYTES + kk * 2048, BOX_BYTES, 1024, bw::SMEM_SW128);
#pragma unroll
            for (int t = 0; t < MT; ++t) {
              const uint32_t sa = sb + t * 2 * A_BYTES;
              uint64_t ah, al;
              if (MODE == 0) {
                ah = bw::smem_desc(sa + kk * 32, 16, 512, bw::SMEM_SW64);
                al = bw::smem_desc(sa + A_BYTES + kk * 32, 16, 512, bw::SMEM_SW64);
              } else {
                ah = bw::smem_desc(sa + kk * 2048, BOX_BYTES, 1024, bw::SMEM_SW128);
                al = bw::smem_desc(sa + A_BYTES + kk * 2048, BOX_BYTES, 1024, bw::SMEM_SW128);
              }
              const uint32_t dt = d + t * NT;
              bw::umma_bf16(dt, ah, bh, IDESC, (st > 0 || kk > 0) ? 1u : 0u);
              bw::umma_bf16(dt, ah, bl, IDESC, 1u);
              bw::umma_bf16(dt, al, bh, IDESC, 1u);
            }
          }
          bw::umma_commit(empty_bar(s));
        }
        if (!ok) break;
        bw::umma_commit(tfull_bar(buf));
      }
    }
  } else {
    const int quarter = warp & 3;
    int uc = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, ++uc) {
      const int mt = u % p.n_mt;
      const int nt = (u / p.n_mt) % p.n_nt;
      const int sp = (u / p.n_mt) / p.n_nt;
      const int buf = acc_buf(uc);
      bool ok = true;
      if (lane == 0) ok = wait(tfull_bar(buf), acc_use(uc) & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      bw::tc_fence_after();
#pragma unroll 1
      for (int t = 0; t < MT; ++t) {
        const int row = mt * 128 * MT + 128 * t + quarter * 32 + lane;
        const bool valid = row < p.L_pad;   // the last M tile may hang over the matrix
        float* dst = partial + (long long)sp * p.split_stride + (long long)(valid ? row : 0) * p.ld + nt * NT;
#pragma unroll 1
        for (int cb = 0; cb < NT / 32; ++cb) {
          uint32_t r[32];
          bw::tmem_ld_32x32(tmem_base + ((uint32_t)(quarter * 32) << 16) + buf * ACC + t * NT + cb * 32, r);
          bw::tmem_ld_wait();
          if (valid) {
            float4* d4 = reinterpret_cast<float4*>(dst + cb * 32);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              d4[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                  __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
          }
        }
      }
      bw::tc_fence_before();
      __syncwarp();
      if (lane == 0) bw::mbar_arrive(tempty_bar(buf));
    }
  }
  bw::tc_fence_before();
  __syncthreads();
  bw::tc_fence_after();
  if (warp == 1) bw::tmem_dealloc(tmem_base, TMEM_COLS);
}

// ------------------------------------------------------------------ CUDA-core Toeplitz GEMM
template <int MODE>
__global__ void __launch_bounds__(256)
    k_toeplitz_gemm_fp32(const float* __restrict__ R32, const float* __restrict__ X, TgParams p,
                         float* __restrict__ partial) {
  constexpr int TK = 32;
  __shared__ float As[TK][64 + 4];
  __shared__ float Bs[TK][64 + 4];
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64, sp = blockIdx.z;
  const int j_begin = sp * p.krows, j_end = min(p.L_pad, j_begin + p.krows);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  const size_t blk = (size_t)p.l_pad * p.l_pad;
  for (int j0 = j_begin; j0 < j_end; j0 += TK) {
    for (int e = threadIdx.x; e < 64 * TK; e += 256) {
      // A tile (64 rows m, TK cols j)
      int r, j;
      if (MODE == 0) { r = e / TK; j = e % TK; } else { j = e / 64; r = e % 64; }
      const int m = m0 + r, jj = j0 + j;
      int lag, ca, cb;
      if (MODE == 0) {
        lag = p.i + m / p.l_pad - jj / p.l_pad;
        ca = m % p.l_pad;
        cb = jj % p.l_pad;
      } else {
        lag = p.i + jj / p.l_pad - m / p.l_pad;
        ca = jj % p.l_pad;
        cb = m % p.l_pad;
      }
      As[j][r] = R32[(size_t)(lag - 1) * blk + (size_t)ca * p.l_pad + cb];
    }
    for (int e = threadIdx.x; e < 64 * TK; e += 256) {
      const int j = e / 64, c = e % 64;
      Bs[j][c] = X[(size_t)(j0 + j) * p.ld + n0 + c];
    }
    __syncthreads();
#pragma unroll 8
    for (int j = 0; j < TK; ++j) {
      float a[4], b[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) { a[x] = As[j][ty * 4 + x]; b[x] = Bs[j][tx * 4 + x]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  float* out = partial + (long long)sp * p.split_stride;
#pragma unroll
  for (int x = 0; x < 4; ++x)
    *reinterpret_cast<float4*>(out + (size_t)(m0 + ty * 4 + x) * p.ld + n0 + tx * 4) =
        make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
}

// U[b*l + c][j] = sum_a Q[b*l_pad + c][a] Ut[a][j], j < k; accumulated in Ut's precision
template <typename TU, typename TO>
__global__ void k_form_u(const float* __restrict__ Q, int ldq, const TU* __restrict__ Ut, int K,
                         int k, int l, int l_pad, int i, TO* __restrict__ U) {
  const long long total = (long long)l * i * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % k);
    const int rr = (int)(e / k);
    const int b = rr / l, c = rr % l;
    const float* q = Q + (size_t)(b * l_pad + c) * ldq;
    TU s = 0;
    for (int a = 0; a < K; ++a) s = fma((TU)q[a], Ut[(size_t)a * K + j], s);
    U[e] = (TO)s;
  }
}

// The FP32 form of k_form_u as a tiled product: a CTA computes 64 rows x 64 columns of U
// from 32-deep slabs of Q and Ut staged in shared memory, 4 x 4 outputs per thread.  Each
// output is still one FMA chain over a = 0, 1, ..., K - 1 in order, so the result is the
// same as the one-output-per-thread form; the slabs make every Q and Ut element serve 64
// outputs instead of one.
template <typename TO>
__global__ void __launch_bounds__(256)
    k_form_u_tiled(const float* __restrict__ Q, int ldq, const float* __restrict__ Ut, int K, int k,
                   int l, int l_pad, int i, TO* __restrict__ U) {
  constexpr int TA = 32;
  __shared__ __align__(16) float As[TA][64 + 4];   // As[a][r] = Q[row of r0 + r][a0 + a]
  __shared__ __align__(16) float Bs[TA][64 + 4];   // Bs[a][c] = Ut[a0 + a][j0 + c]
  const int L = l * i;
  const int j0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int a0 = 0; a0 < K; a0 += TA) {
    for (int e = tid; e < 64 * TA; e += 256) {
      const int r = e / TA, a = e % TA;
      const int rr = r0 + r;
      float v = 0.f;
      if (rr < L && a0 + a < K) {
        const int b = rr / l, c = rr % l;
        v = Q[(size_t)(b * l_pad + c) * ldq + a0 + a];
      }
      As[a][r] = v;
    }
    for (int e = tid; e < 64 * TA; e += 256) {
      const int a = e / 64, c = e % 64;
      Bs[a][c] = (a0 + a < K && j0 + c < k) ? Ut[(size_t)(a0 + a) * K + j0 + c] : 0.f;
    }
    __syncthreads();
    const int na = min(TA, K - a0);
    for (int a = 0; a < na; ++a) {
      const float4 qa = *reinterpret_cast<const float4*>(&As[a][ty * 4]);
      const float4 ub = *reinterpret_cast<const float4*>(&Bs[a][tx * 4]);
      const float q4[4] = {qa.x, qa.y, qa.z, qa.w}, u4[4] = {ub.x, ub.y, ub.z, ub.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(q4[x], u4[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int rr = r0 + ty * 4 + x;
    if (rr >= L) continue;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int j = j0 + tx * 4 + y;
      if (j < k) U[(size_t)rr * k + j] = (TO)acc[x][y];
    }
  }
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ x, long long n, TO* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (TO)x[e];
}

template <int NB, int MT>
constexpr int tg_stage_bytes() {
  return MT * 4 * BOX_BYTES + 2 * NB * BOX_BYTES;
}

template <int NB, int MT>
constexpr int tg_stages() {
  return (200 * 1024) / tg_stage_bytes<NB, MT>() > 6 ? 6 : (200 * 1024) / tg_stage_bytes<NB, MT>();
}

template <int MODE, int NB, int MT>
ssi_status launch_tg(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh,
                     const CUtensorMap& bl, const TgParams& p, float* partial, int* status, int grid,
                     cudaStream_t stream) {
  constexpr int STAGES = tg_stages<NB, MT>();
  constexpr int STAGE_BYTES = tg_stage_bytes<NB, MT>();
  const size_t smem = 1024 + (size_t)STAGES * STAGE_BYTES + 8 * (2 * STAGES + 4) + 16;
  auto kern = k_toeplitz_gemm_tc<MODE, NB, MT, STAGES>;
  SSI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, TG_THREADS, smem, stream>>>(ah, al, bh, bl, p, partial, status);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

template <int MODE>
ssi_status launch_tg_nb(int nb, int mt, const CUtensorMap& ah, const CUtensorMap& al,
                        const CUtensorMap& bh, const CUtensorMap& bl, const TgParams& p,
                        float* partial, int* status, int grid, cudaStream_t stream) {
  if (mt == 2) {
    switch (nb) {
      case 1: return launch_tg<MODE, 1, 2>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 2: return launch_tg<MODE, 2, 2>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 3: return launch_tg<MODE, 3, 2>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 4: return launch_tg<MODE, 4, 2>(ah, al, bh, bl, p, partial, status, grid, stream);
      default: break;
    }
  } else {
    switch (nb) {
      case 1: return launch_tg<MODE, 1, 1>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 2: return launch_tg<MODE, 2, 1>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 3: return launch_tg<MODE, 3, 1>(ah, al, bh, bl, p, partial, status, grid, stream);
      case 4: return launch_tg<MODE, 4, 1>(ah, al, bh, bl, p, partial, status, grid, stream);
      default: break;
    }
  }
  set_error("toeplitz gemm: unsupported tiling (N atoms %d, M tiles %d)", nb, mt);
  return SSI_E_INVALID;
}

// Reduction splits of the Toeplitz products: the count in [2, 16] whose units
// (n_tiles per split) fill the SMs' waves best, the smallest such count on ties; each
// split covers a multiple of SBK rows.
int toeplitz_splits(int L_pad, int n_tiles, int num_sms) {
  int best = 1;
  double best_eff = -1.0;
  for (int S = 2; S <= 16; ++S) {
    const int krows = (int)round_up(ceil_div(L_pad, S), SBK);
    const int S_eff = (int)ceil_div(L_pad, krows);
    const long long units = (long long)n_tiles * S_eff;
    const double waves = (double)units / num_sms;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 1e-3) {
      best_eff = eff;
      best = S_eff;
    }
  }
  return best;
}

int grid_1d(long long n, int threads, int num_sms) {
  return (int)std::max<long long>(1, std::min<long long>(ceil_div(n, threads), (long long)num_sms * 8));
}

}  // namespace

ssi_status convert_f2d(const float* x, long long n, double* y, cudaStream_t stream) {
  k_convert<float, double><<<grid_1d(n, 256, 152), 256, 0, stream>>>(x, n, y);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

ssi_status convert_d2f(const double* x, long long n, float* y, cudaStream_t stream) {
  k_convert<double, float><<<grid_1d(n, 256, 152), 256, 0, stream>>>(x, n, y);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

ssi_status gaussian_omega_launch(int rows, int cols, int ld, uint64_t seed, float* out,
                                 __nv_bfloat16*, __nv_bfloat16*, cudaStream_t stream) {
  k_omega<<<grid_1d((long long)rows * ld, 256, 152), 256, 0, stream>>>(rows, cols, ld, seed, out, 1, 1,
                                                                       0, nullptr, nullptr, nullptr);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

RsvdPlan rsvd_plan(int l, int i, int k, int oversample, int q, int num_sms, int splits_req,
                   int jacobi_block, int qr_cpc) {
  RsvdPlan r{};
  r.l = l;
  r.i = i;
  r.k = k;
  r.q = q;
  r.K = k + oversample;
  r.l_pad = (int)round_up(l, 64);
  r.L = l * i;
  r.L_pad = r.l_pad * i;
  const int n_nt = (int)ceil_div(round_up(r.K, 64), 256);
  r.Kp = (int)round_up(r.K, 64 * n_nt);
  // two M tiles per CTA halve the operand bytes per MMA of X; small T keeps one so that
  // the units still fill the SMs
  r.tg_mt = r.L_pad >= 2048 ? 2 : 1;
  const int n_mt = (int)ceil_div(r.L_pad, 128 * r.tg_mt);
  int S = splits_req > 0 ? std::min(splits_req, 64) : toeplitz_splits(r.L_pad, n_mt * n_nt, num_sms);
  const int krows = (int)round_up(ceil_div(r.L_pad, S), SBK);
  S = (int)ceil_div(r.L_pad, krows);
  r.tg_splits = S;
  r.jacobi_block = jacobi_block;
  r.qr_cpc = qr_cpc;
  const int n_lag = 2 * i - 1;
  const size_t rblk = (size_t)n_lag * r.l_pad * r.l_pad;
  const size_t xsz = (size_t)r.L_pad * r.Kp;
  WsPlan w;
  w.add<__nv_bfloat16>(rblk);   // R hi
  w.add<__nv_bfloat16>(rblk);   // R lo
  w.add<float>(rblk);           // R fp32
  w.add<__nv_bfloat16>(xsz);    // X hi
  w.add<__nv_bfloat16>(xsz);    // X lo
  w.add<float>(xsz);            // Y (product / QR in place)
  w.add<float>(xsz);            // Q kept for U = Q U~
  w.add<float>((size_t)S * xsz);  // split partials
  w.add<float>((size_t)r.K * r.K);  // R2
  w.add<float>((size_t)r.K * r.K);  // U~
  w.add<float>((size_t)r.K);        // sigma
  w.add<double>((size_t)r.K * r.K); // U~ (FP64 small problems)
  w.add<double>((size_t)r.K);       // sigma (FP64 small problems)
  w.bytes += qr_ws_bytes(r.K, num_sms) +
             std::max(jacobi_ws_bytes(r.K, num_sms, false), jacobi_ws_bytes(r.K, num_sms, true)) + 4096;
  r.ws_bytes = w.bytes;
  return r;
}

ssi_status toeplitz_rsvd_ws(ssi_ctx* ctx, Workspace& ws, const RsvdPlan& r, const double* R,
                            uint64_t seed, ssi_precision prec, bool small64, void* U, void* S,
                            bool out64, int* dev_status, cudaStream_t stream, bool shared_device) {
  ws.reset();
  const bool tc = prec == SSI_PREC_SPLIT_BF16;
  const int n_lag = 2 * r.i - 1;
  const size_t rblk = (size_t)n_lag * r.l_pad * r.l_pad;
  const size_t xsz = (size_t)r.L_pad * r.Kp;
  const int n_nt = (int)ceil_div(round_up(r.K, 64), 256);
  const int nb = r.Kp / 64 / n_nt;
  TgParams p{};
  p.i = r.i;
  p.l_pad = r.l_pad;
  p.L_pad = r.L_pad;
  p.n_mt = (int)ceil_div(r.L_pad, 128 * r.tg_mt);
  p.n_nt = n_nt;
  p.krows = (int)round_up(ceil_div(r.L_pad, r.tg_splits), SBK);
  p.n_split = (int)ceil_div(r.L_pad, p.krows);
  p.ld = r.Kp;
  p.split_stride = (long long)xsz;

  __nv_bfloat16* Rh = ws.take<__nv_bfloat16>(rblk);
  __nv_bfloat16* Rl = ws.take<__nv_bfloat16>(rblk);
  float* R32 = ws.take<float>(rblk);
  __nv_bfloat16* Xh = ws.take<__nv_bfloat16>(xsz);
  __nv_bfloat16* Xl = ws.take<__nv_bfloat16>(xsz);
  float* Yb = ws.take<float>(xsz);
  float* Qs = ws.take<float>(xsz);
  float* part = ws.take<float>((size_t)p.n_split * xsz);
  float* R2 = ws.take<float>((size_t)r.K * r.K);
  float* Ut = ws.take<float>((size_t)r.K * r.K);
  float* sig = ws.take<float>((size_t)r.K);
  double* Ut64 = ws.take<double>((size_t)r.K * r.K);
  double* sig64 = ws.take<double>((size_t)r.K);
  if (!Rh || !Rl || !R32 || !Xh || !Xl || !Yb || !Qs || !part || !R2 || !Ut || !sig || !Ut64 ||
      !sig64) {
    set_error("toeplitz_rsvd: workspace too small");
    return SSI_E_NOMEM;
  }
  const int nsm = ctx->num_sms;
  count_launches(ctx, 4);   // covariance store, Omega, U = Q U~, small SVD
  {
    ProfScope ps_pre(ctx, ST_OTHER, stream);
    k_r_store<<<grid_1d((long long)rblk, 256, nsm), 256, 0, stream>>>(R, n_lag, r.l, r.l_pad,
                                                                        tc ? Rh : nullptr, Rl,
                                                                        tc ? nullptr : R32);
    SSI_CUDA(cudaGetLastError());
    // Omega in the padded column layout of T
    k_omega<<<grid_1d((long long)xsz, 256, nsm), 256, 0, stream>>>(0, r.K, r.Kp, seed, nullptr, r.l,
                                                                     r.l_pad, r.L_pad, Yb,
                                                                     tc ? Xh : nullptr, Xl);
    SSI_CUDA(cudaGetLastError());
  }

  CUtensorMap tAn_h, tAn_l, tAt_h, tAt_l, tX_h, tX_l;
  if (tc) {
    const uint64_t rrows = (uint64_t)n_lag * r.l_pad;
    if (!make_tmap_bf16_2d(&tAn_h, Rh, rrows, r.l_pad, r.l_pad, 32, 64, CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_tmap_bf16_2d(&tAn_l, Rl, rrows, r.l_pad, r.l_pad, 32, 64, CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_tmap_bf16_2d(&tAt_h, Rh, rrows, r.l_pad, r.l_pad, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tmap_bf16_2d(&tAt_l, Rl, rrows, r.l_pad, r.l_pad, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tmap_bf16_2d(&tX_h, Xh, r.L_pad, r.Kp, r.Kp, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tmap_bf16_2d(&tX_l, Xl, r.L_pad, r.Kp, r.Kp, 64, 32, CU_TENSOR_MAP_SWIZZLE_128B))
      return SSI_E_CUDA;
  }
  const int units = p.n_mt * p.n_nt * p.n_split;
  const int grid_tc = std::min(units, nsm);

  // one product D = T X (mode 0) or T^T X (mode 1) of the current basis into Yb
  auto product = [&](int mode) -> ssi_status {
    count_launches(ctx, tc ? 3 : 2);
    if (tc) {
      ProfScope ps0(ctx, ST_OTHER, stream);
      // the basis sits in Yb (fp32): split it into the bf16 operand pair
      k_to_bf16<<<grid_1d((long long)xsz, 256, nsm), 256, 0, stream>>>(Yb, (long long)xsz, Xh, Xl);
      SSI_CUDA(cudaGetLastError());
    }
    if (tc) {
      ProfScope ps(ctx, ST_SKETCH_GEMM, stream);
      if (mode == 0)
        SSI_TRY(launch_tg_nb<0>(nb, r.tg_mt, tAn_h, tAn_l, tX_h, tX_l, p, part, dev_status, grid_tc,
                                stream));
      else
        SSI_TRY(launch_tg_nb<1>(nb, r.tg_mt, tAt_h, tAt_l, tX_h, tX_l, p, part, dev_status, grid_tc,
                                stream));
    } else {
      ProfScope ps(ctx, ST_SKETCH_GEMM, stream);
      dim3 g((unsigned)(r.L_pad / 64), (unsigned)(r.Kp / 64), (unsigned)p.n_split);
      if (mode == 0) k_toeplitz_gemm_fp32<0><<<g, 256, 0, stream>>>(R32, Yb, p, part);
      else k_toeplitz_gemm_fp32<1><<<g, 256, 0, stream>>>(R32, Yb, p, part);
      SSI_CUDA(cudaGetLastError());
    }
    ProfScope ps2(ctx, ST_SKETCH_GEMM, stream);
    k_sum_splits<<<grid_1d((long long)xsz, 256, nsm), 256, 0, stream>>>(part, p.n_split,
                                                                         (long long)xsz, Yb);
    SSI_CUDA(cudaGetLastError());
    return SSI_OK;
  };
  const size_t ws_mark = ws.off;
  auto qr = [&](float* Rout) -> ssi_status {
    ws.off = ws_mark;
    ProfScope ps(ctx, ST_QR, stream);
    count_launches(ctx, 1);
    return qr_launch(ctx, ws, Yb, r.L_pad, r.K, r.Kp, Rout, dev_status, stream, shared_device,
                     r.qr_cpc);
  };

  // Y = T Omega; Q = qr(Y)
  SSI_TRY(product(0));
  SSI_TRY(qr(nullptr));
  for (int it = 0; it < r.q; ++it) {
    SSI_TRY(product(1));     // Z = T^T Q
    SSI_TRY(qr(nullptr));
    SSI_TRY(product(0));     // Y = T Q_z
    SSI_TRY(qr(nullptr));
  }
  SSI_CUDA(cudaMemcpyAsync(Qs, Yb, xsz * sizeof(float), cudaMemcpyDeviceToDevice, stream));
  SSI_TRY(product(1));       // P^T = T^T Q
  SSI_TRY(qr(R2));           // P^T = Q2 R2
  ws.off = ws_mark;
  {
    ProfScope ps(ctx, ST_SMALL_SVD, stream);
    if (small64)
      SSI_TRY(jacobi_launch64(ws, R2, r.K, Ut64, sig64, dev_status, nsm, r.jacobi_block, stream));
    else
      SSI_TRY(jacobi_launch(ws, R2, r.K, Ut, sig, dev_status, nsm, r.jacobi_block, stream));
  }
  ProfScope ps_u(ctx, ST_OTHER, stream);
  const int gu = grid_1d((long long)r.L * r.k, 256, nsm), gs = grid_1d(r.k, 256, nsm);
  const dim3 gt((unsigned)ceil_div(r.k, 64), (unsigned)ceil_div(r.L, 64));
  if (small64) {
    k_form_u<double, double><<<gu, 256, 0, stream>>>(Qs, r.Kp, Ut64, r.K, r.k, r.l, r.l_pad, r.i,
                                                     static_cast<double*>(U));
    SSI_CUDA(cudaGetLastError());
    SSI_CUDA(cudaMemcpyAsync(S, sig64, sizeof(double) * r.k, cudaMemcpyDeviceToDevice, stream));
  } else if (out64) {
    k_form_u_tiled<double><<<gt, 256, 0, stream>>>(Qs, r.Kp, Ut, r.K, r.k, r.l, r.l_pad, r.i,
                                                   static_cast<double*>(U));
    SSI_CUDA(cudaGetLastError());
    k_convert<float, double><<<gs, 256, 0, stream>>>(sig, r.k, static_cast<double*>(S));
  } else {
    k_form_u_tiled<float><<<gt, 256, 0, stream>>>(Qs, r.Kp, Ut, r.K, r.k, r.l, r.l_pad, r.i,
                                                  static_cast<float*>(U));
    SSI_CUDA(cudaGetLastError());
    SSI_CUDA(cudaMemcpyAsync(S, sig, sizeof(float) * r.k, cudaMemcpyDeviceToDevice, stream));
  }
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace ssi

extern "C" ssi_status ssi_gaussian_omega(ssi_ctx* ctx, int rows, int cols, uint64_t seed, float* omega,
                                         void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && omega, "ssi_gaussian_omega: null pointer");
  SSI_CHECK(rows > 0 && cols > 0, "ssi_gaussian_omega: empty shape");
  SSI_CUDA(cudaSetDevice(ctx->device));
  return gaussian_omega_launch(rows, cols, cols, seed, omega, nullptr, nullptr,
                               static_cast<cudaStream_t>(stream));
}

extern "C" ssi_status ssi_toeplitz_rsvd(ssi_ctx* ctx, const double* R, int l, int i, int k,
                                        int oversample, int q, uint64_t seed, ssi_precision prec,
                                        ssi_small_precision small, double* U, double* S,
                                        void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && R && U && S, "ssi_toeplitz_rsvd: null pointer");
  SSI_CHECK(l >= 1 && l <= 1024, "ssi_toeplitz_rsvd: l=%d out of range", l);
  SSI_CHECK(i >= 2, "ssi_toeplitz_rsvd: need i >= 2");
  SSI_CHECK(k >= 1 && oversample >= 0 && q >= 0, "ssi_toeplitz_rsvd: bad k/oversample/q");
  SSI_CHECK(k + oversample <= 16384 && (int64_t)(k + oversample) <= (int64_t)l * i,
            "ssi_toeplitz_rsvd: need k + oversample <= min(l*i, 16384)");
  SSI_CHECK(prec == SSI_PREC_FP32 || prec == SSI_PREC_SPLIT_BF16, "ssi_toeplitz_rsvd: bad precision");
  SSI_CHECK(small == SSI_SMALL_FP32 || small == SSI_SMALL_FP64,
            "ssi_toeplitz_rsvd: bad small-problem precision");
  SSI_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RsvdPlan plan = rsvd_plan(l, i, k, oversample, q, ctx->num_sms);
  SSI_TRY(ws_reserve(ctx, ctx->ws, plan.ws_bytes, s));
  SSI_TRY(toeplitz_rsvd_ws(ctx, ctx->ws, plan, R, seed, prec, small == SSI_SMALL_FP64, U, S, true,
                           ctx->dev_status, s, false));
  return check_dev_status(ctx->dev_status, s);
}
