// Stage (a): output covariances R_k = 1/(N-k) sum_t y_{t+k} y_t^T, k = 1..max_lag (Sec. 2.1).
//
// Tensor-core path (SSI_PREC_SPLIT_BF16):
//   1. k_split_transpose: Y (l x N fp32, channel-major) -> Yhi, Ylo (N x l_pad bf16,
//      time-major), y = hi + lo.
//   2. k_lag_gemm_tc: persistent tcgen05 kernel.  Stack every lag into one GEMM:
//      row (k, c) of A at time t is Y[t+k][c], B is Y[t][c'], the reduction runs over
//      time.  A work unit is (256 rows of (lag, channel) = four 64-channel atoms,
//      one N tile of channels, one time split).  TMA loads each atom as a
//      64-channel x 32-sample box of the time-major record at a time offset of
//      t + k (no alignment constraint on the time coordinate, zero fill past N), so
//      the lag shift costs nothing.  Both operands are MN-major 128B-swizzled.
//      Three BF16 MMAs per k-step (hi*hi, hi*lo, lo*hi) accumulate in FP32 in TMEM.
//   3. k_reduce_partials: FP64 sum of the per-split FP32 partials, scaled by 1/(N-k).
// CUDA-core path (SSI_PREC_FP32): k_lag_gemm_fp32 writes the same partials.
#include "common.cuh"
#include "blackwell.cuh"

namespace ssi {

namespace {

constexpr int BT = 32;            // time rows per pipeline stage
constexpr int ATOM_BYTES = BT * 128;  // one 64-channel x BT box, bf16
constexpr int A_ATOMS = 4;        // two M tiles of 128 rows per CTA
constexpr int TC_THREADS = 192;   // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr uint64_t WAIT_NS = 2000000000ull;  // bounded waits: 2 s
constexpr int UR = 4;             // ring of work-unit indices from the producer to the MMA
                                  // issuer and the epilogue

struct LagGemmParams {
  int n_atoms;          // max_lag * l_pad / 64
  int n_mp;             // ceil(n_atoms / 4)
  int n_nt;             // N tiles over l_pad
  int n_split;
  int rows_per_split;   // multiple of BT
  int N;
  int l_pad;
  int ld_out;           // l_pad
  long long split_stride;  // floats between splits in the partial buffer
  int* unit_counter;    // zero before the launch: units handed out beyond the first wave
};

// ------------------------------------------------------------------ split/transpose
__global__ void k_split_transpose(const float* __restrict__ Y, long long ldy, int l, int N, int n_rows,
                                  int l_pad, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo) {
  __shared__ float tile[32][33];
  const int t0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, t = t0 + threadIdx.x;
    tile[r][threadIdx.x] = (c < l && t < N) ? Y[(size_t)c * ldy + t] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int t = t0 + r, c = c0 + threadIdx.x;
    if (t < n_rows) {
      const float x = tile[threadIdx.x][r];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const __nv_bfloat16 g = __float2bfloat16_rn(x - __bfloat162float(h));
      hi[(size_t)t * l_pad + c] = h;
      lo[(size_t)t * l_pad + c] = g;
    }
  }
}

// ------------------------------------------------------------------ tensor-core lag GEMM
template <int NB, int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_lag_gemm_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                  LagGemmParams p, float* __restrict__ partial, int* __restrict__ status) {
  constexpr int NT = 64 * NB;                       // N tile (columns of TMEM per accumulator)
  constexpr int A_BYTES = A_ATOMS * ATOM_BYTES;     // per operand half (hi or lo)
  constexpr int B_BYTES = NB * ATOM_BYTES;
  constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  constexpr uint32_t IDESC = bw::idesc_bf16(128, NT, 1, 1);

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars[0..S) full, [S..2S) empty, [2S] tmem_full, [2S+1] tmem_empty,
  // [2S+2..2S+2+UR) unit_full, [2S+2+UR..2S+2+2UR) unit_empty
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2 + 2 * UR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* s_unit = abort_flag + 1;   // UR entries

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = bw::smem_u32(smem);
  const uint32_t bar_base = bw::smem_u32(bars);
  auto full_bar = [&](int s) { return bar_base + 8u * s; };
  auto empty_bar = [&](int s) { return bar_base + 8u * (STAGES + s); };
  const uint32_t tfull_bar = bar_base + 8u * (2 * STAGES);
  const uint32_t tempty_bar = bar_base + 8u * (2 * STAGES + 1);
  auto unit_full = [&](int r) { return bar_base + 8u * (2 * STAGES + 2 + r); };
  auto unit_empty = [&](int r) { return bar_base + 8u * (2 * STAGES + 2 + UR + r); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      bw::mbar_init(full_bar(s), 1);
      bw::mbar_init(empty_bar(s), 1);
    }
    bw::mbar_init(tfull_bar, 1);
    bw::mbar_init(tempty_bar, 4);
    for (int r = 0; r < UR; ++r) {
      bw::mbar_init(unit_full(r), 1);
      bw::mbar_init(unit_empty(r), 5);   // the MMA issuer and the four epilogue warps
    }
    *abort_flag = 0;
    bw::fence_mbar_init();
    bw::tma_prefetch_desc(&tm_hi);
    bw::tma_prefetch_desc(&tm_lo);
  }
  if (warp == 1) {
    bw::tmem_alloc(bw::smem_u32(tmem_slot), 512);
    bw::tmem_relinquish();
  }
  bw::tc_fence_before();
  __syncthreads();
  bw::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int n_units = p.n_mp * p.n_nt * p.n_split;
  auto fail = [&]() {
    atomicOr(status, DEV_TIMEOUT);
    *abort_flag = 1;
  };
  // bounded wait that also gives up as soon as another role has aborted
  auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
    if (bw::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = bw::global_ns();
    while (true) {
      if (bw::mbar_try_wait(bar, parity)) return true;
      if (*abort_flag) return false;
      if (bw::global_ns() - t0 > WAIT_NS) {
        fail();
        return false;
      }
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // Lane 0 takes the barrier waits and the transaction count; the boxes of a stage
    // (2 per A atom, 2 per B atom) are issued by one lane each, so that their issue
    // does not serialise on one thread.
    int g = 0;
    int armed_phase[STAGES];
    for (int s = 0; s < STAGES; ++s) armed_phase[s] = -1;
    bool ok = true;
    // dynamic schedule: the first unit is blockIdx.x, later ones come from a global
    // counter, claimed one unit ahead so that the atomic's latency is hidden; a CTA
    // that starts late (the SMs busy with other work) simply takes fewer units
    int u = blockIdx.x;
    int u_next = n_units;
    if (lane == 0 && u < n_units) u_next = (int)gridDim.x + atomicAdd(p.unit_counter, 1);
    for (int uc = 0; ok; ++uc) {
      const int r = uc % UR;
      int okl = 1;
      if (lane == 0) {
        okl = wait(unit_empty(r), ((uc / UR) & 1) ^ 1) ? 1 : 0;
        if (okl) {
          s_unit[r] = (u < n_units) ? u : -1;
          bw::mbar_arrive(unit_full(r));
        }
      }
      okl = __shfl_sync(0xffffffffu, okl, 0);
      if (!okl) { ok = false; break; }
      if (u >= n_units) break;
      const int mp = u % p.n_mp;
      const int v = u / p.n_mp;
      const int nt = v % p.n_nt;
      const int sp = v / p.n_nt;
      const int t0 = sp * p.rows_per_split;
      const int t1 = min(p.N, t0 + p.rows_per_split);
      const int n_st = (t1 - t0 + BT - 1) / BT;
      const int cpl = p.l_pad / 64;
      const int n_valid = min(A_ATOMS, p.n_atoms - mp * A_ATOMS);
      // this lane's box: A atom (lane / 2) for lanes < 2 A_ATOMS, B atom for the next 2 NB
      const bool lo_half = (lane & 1) != 0;
      const bool a_box = lane < 2 * n_valid;
      const bool b_box = lane >= 2 * A_ATOMS && lane < 2 * A_ATOMS + 2 * NB;
      int box_ch = 0, box_lag = 0;
      uint32_t box_off = 0;
      if (a_box) {
        const int atom = mp * A_ATOMS + (lane >> 1);
        box_lag = atom / cpl + 1;
        box_ch = (atom % cpl) * 64;
        box_off = (lo_half ? A_BYTES : 0) + (lane >> 1) * ATOM_BYTES;
      } else if (b_box) {
        const int bb = (lane - 2 * A_ATOMS) >> 1;
        box_ch = nt * NT + bb * 64;
        box_off = 2 * A_BYTES + (lo_half ? B_BYTES : 0) + bb * ATOM_BYTES;
      }
      const CUtensorMap* box_map = lo_half ? &tm_lo : &tm_hi;
      for (int st = 0; st < n_st; ++st, ++g) {
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1;
        int okw = 1;
        if (lane == 0) {
          okw = wait(empty_bar(s), ph ^ 1) ? 1 : 0;
          if (okw) {
            const uint32_t bytes = (uint32_t)(2 * n_valid + 2 * NB) * ATOM_BYTES;
            bw::mbar_arrive_expect_tx(full_bar(s), bytes);
            armed_phase[s] = (int)ph;
          }
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) { ok = false; break; }
        if (a_box || b_box)
          bw::tma_load_2d(smem_base + s * STAGE_BYTES + box_off, box_map, full_bar(s), box_ch,
                          t0 + st * BT + box_lag);
      }
      if (lane == 0) {
        u = u_next;
        if (u < n_units) u_next = (int)gridDim.x + atomicAdd(p.unit_counter, 1);
      }
      u = __shfl_sync(0xffffffffu, u, 0);
    }
    if (lane == 0 && *abort_flag) {
      // do not leave the CTA while TMA writes into its shared memory are in flight
      for (int s = 0; s < STAGES; ++s) {
        if (armed_phase[s] < 0) continue;
        const uint64_t t0 = bw::global_ns();
        while (!bw::mbar_try_wait(full_bar(s), (uint32_t)armed_phase[s]) &&
               bw::global_ns() - t0 < 50000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int uc = 0; ok; ++uc) {
        const int r = uc % UR;
        if (!wait(unit_full(r), (uc / UR) & 1)) { ok = false; break; }
        const int u = s_unit[r];
        bw::mbar_arrive(unit_empty(r));
        if (u < 0) break;
        const int v = u / p.n_mp;
        const int sp = v / p.n_nt;
        const int t0 = sp * p.rows_per_split;
        const int t1 = min(p.N, t0 + p.rows_per_split);
        const int n_st = (t1 - t0 + BT - 1) / BT;
        if (!wait(tempty_bar, (uc & 1) ^ 1)) { ok = false; break; }
        bw::tc_fence_after();
        for (int st = 0; st < n_st; ++st, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (!wait(full_bar(s), ph)) { ok = false; break; }
          bw::tc_fence_after();
          const uint32_t sb = smem_base + s * STAGE_BYTES;
#pragma unroll
          for (int kk = 0; kk < BT / 16; ++kk) {
            const uint32_t koff = kk * 2048;
            const uint64_t bh = bw::smem_desc(sb + 2 * A_BYTES + koff, ATOM_BYTES, 1024, bw::SMEM_SW128);
            const uint64_t bl = bw::smem_desc(sb + 2 * A_BYTES + B_BYTES + koff, ATOM_BYTES, 1024, bw::SMEM_SW128);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              const uint32_t aoff = mt * 2 * ATOM_BYTES + koff;
              const uint64_t ah = bw::smem_desc(sb + aoff, ATOM_BYTES, 1024, bw::SMEM_SW128);
              const uint64_t al = bw::smem_desc(sb + A_BYTES + aoff, ATOM_BYTES, 1024, bw::SMEM_SW128);
              const uint32_t d = tmem_base + mt * NT;
              bw::umma_bf16(d, ah, bh, IDESC, (st > 0 || kk > 0) ? 1u : 0u);
              bw::umma_bf16(d, ah, bl, IDESC, 1u);
              bw::umma_bf16(d, al, bh, IDESC, 1u);
            }
          }
          bw::umma_commit(empty_bar(s));
        }
        if (!ok) break;
        bw::umma_commit(tfull_bar);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int quarter = warp & 3;   // TMEM lane quarter this warp may access
    for (int uc = 0;; ++uc) {
      int u = -1;
      if (lane == 0) {
        const int r = uc % UR;
        if (wait(unit_full(r), (uc / UR) & 1)) {
          u = s_unit[r];
          bw::mbar_arrive(unit_empty(r));
        }
      }
      u = __shfl_sync(0xffffffffu, u, 0);
      if (u < 0) break;
      const int mp = u % p.n_mp;
      const int v = u / p.n_mp;
      const int nt = v % p.n_nt;
      const int sp = v / p.n_nt;
      bool ok = true;
      if (lane == 0) ok = wait(tfull_bar, uc & 1);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) break;
      bw::tc_fence_after();
      float* out = partial + (long long)sp * p.split_stride;
#pragma unroll 1
      for (int mt = 0; mt < 2; ++mt) {
        const int row_in_tile = quarter * 32 + lane;
        const int atom = mp * A_ATOMS + mt * 2 + row_in_tile / 64;
        const bool valid = atom < p.n_atoms;
        const long long orow = (long long)atom * 64 + (row_in_tile & 63);
        float* dst = out + orow * p.ld_out + nt * NT;
#pragma unroll 1
        for (int cb = 0; cb < NT / 32; ++cb) {
          uint32_t r[32];
          const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + mt * NT + cb * 32;
          bw::tmem_ld_32x32(taddr, r);
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
      if (lane == 0) bw::mbar_arrive(tempty_bar);
    }
  }

  bw::tc_fence_before();
  __syncthreads();
  bw::tc_fence_after();
  if (warp == 1) bw::tmem_dealloc(tmem_base, 512);
}

// ------------------------------------------------------------------ CUDA-core lag GEMM
// One CTA: one lag, a 64 x 64 block of (c, c'), one time split.  FP32 FMA.
__global__ void __launch_bounds__(256)
    k_lag_gemm_fp32(const float* __restrict__ Y, long long ldy, int l, int N, int l_pad, int max_lag,
                    int rows_per_split, long long split_stride, float* __restrict__ partial) {
  constexpr int TK = 32;
  __shared__ float As[TK][64 + 4];
  __shared__ float Bs[TK][64 + 4];
  const int nb = (l + 63) / 64;
  int bid = blockIdx.x;
  const int cb2 = bid % nb; bid /= nb;
  const int cb1 = bid % nb; bid /= nb;
  const int lag = bid + 1;
  const int sp = blockIdx.y;
  const int c0 = cb1 * 64, d0 = cb2 * 64;
  const int t_begin = sp * rows_per_split;
  const int t_end = min(N - lag, t_begin + rows_per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int t = t_begin; t < t_end; t += TK) {
    for (int e = threadIdx.x; e < 64 * TK; e += 256) {
      const int r = e / TK, j = e % TK;
      const int tt = t + j;
      const bool in = tt < t_end;
      As[j][r] = (in && c0 + r < l) ? Y[(size_t)(c0 + r) * ldy + tt + lag] : 0.f;
      Bs[j][r] = (in && d0 + r < l) ? Y[(size_t)(d0 + r) * ldy + tt] : 0.f;
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
  float* out = partial + (long long)sp * split_stride;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int c = c0 + ty * 4 + x;
    if (c >= l_pad) continue;
    float4 v = make_float4(acc[x][0], acc[x][1], acc[x][2], acc[x][3]);
    const int d = d0 + tx * 4;
    if (d + 3 < l_pad)
      *reinterpret_cast<float4*>(out + ((long long)(lag - 1) * l_pad + c) * l_pad + d) = v;
  }
}

// ------------------------------------------------------------------ split reduction
// Sum of the per-split FP32 partials with Knuth's two-sum: hi + lo carries the running
// sum to about twice FP32 precision using FP32 adds only (FP64 runs at a small fraction
// of the FP32 rate on this part); the order over splits is fixed, so the result is
// deterministic.  Eight partials are loaded ahead of their adds.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

__global__ void k_reduce_partials(const float* __restrict__ partial, int n_split,
                                  long long split_stride, int l, int l_pad, int max_lag, int N,
                                  double* __restrict__ R) {
  const long long total = (long long)max_lag * l * l;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % l);
    const int a = (int)((e / l) % l);
    const int k = (int)(e / ((long long)l * l)) + 1;
    const float* src = partial + ((long long)(k - 1) * l_pad + a) * l_pad + b;
    float hi = 0.f, lo = 0.f;
    int sp = 0;
    for (; sp + 8 <= n_split; sp += 8) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldcs(src + (long long)(sp + u) * split_stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) two_sum_acc(hi, lo, x[u]);
    }
    for (; sp < n_split; ++sp) two_sum_acc(hi, lo, __ldcs(src + (long long)sp * split_stride));
    R[e] = ((double)hi + (double)lo) / (double)(N - k);
  }
}

// Accumulating variant, S += acc_sign * (sum of the per-split partials), for callers that
// add unnormalised lag sums over segments.  S is kept in double-float (hi, lo FP32 pairs,
// ~2^-48 relative), so the update runs on the FP32 pipes: the split sum (hi, lo) is added
// with Knuth's two-sum and renormalised.  One block per (lag k, eight channels a), one
// warp per a, lanes over b (no per-element index division); splits in the same order.
__global__ void __launch_bounds__(256) k_accumulate_partials(const float* __restrict__ partial,
                                                             int n_split, long long split_stride,
                                                             int l, int l_pad, float acc_sign,
                                                             float2* __restrict__ S) {
  const int k = blockIdx.y + 1;
  const int a = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= l) return;
  const float* src = partial + ((long long)(k - 1) * l_pad + a) * l_pad;
  float2* dst = S + ((long long)(k - 1) * l + a) * l;
  for (int b = lane; b < l; b += 32) {
    float hi = 0.f, lo = 0.f;
    int sp = 0;
    for (; sp + 8 <= n_split; sp += 8) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldcs(src + b + (long long)(sp + u) * split_stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) two_sum_acc(hi, lo, x[u]);
    }
    for (; sp < n_split; ++sp) two_sum_acc(hi, lo, __ldcs(src + b + (long long)sp * split_stride));
    if (acc_sign < 0.f) {
      hi = -hi;
      lo = -lo;
    }
    const float2 v = dst[b];
    const float s = __fadd_rn(v.x, hi);
    const float bb = __fsub_rn(s, v.x);
    const float err = __fadd_rn(__fsub_rn(v.x, __fsub_rn(s, bb)), __fsub_rn(hi, bb));
    const float t = __fadd_rn(__fadd_rn(v.y, lo), err);
    const float h2 = __fadd_rn(s, t);
    dst[b] = make_float2(h2, __fsub_rn(t, __fsub_rn(h2, s)));
  }
}

template <int NB>
constexpr int tc_stages() {
  return (225 * 1024) / ((2 * A_ATOMS + 2 * NB) * ATOM_BYTES) > 4
             ? 4
             : (225 * 1024) / ((2 * A_ATOMS + 2 * NB) * ATOM_BYTES);
}

template <int NB>
ssi_status launch_tc(const CUtensorMap& thi, const CUtensorMap& tlo, const LagGemmParams& p,
                     float* partial, int* status, int grid, cudaStream_t stream) {
  constexpr int STAGES = tc_stages<NB>();
  constexpr int STAGE_BYTES = (2 * A_ATOMS + 2 * NB) * ATOM_BYTES;
  const size_t smem = 1024 + (size_t)STAGES * STAGE_BYTES + 8 * (2 * STAGES + 2 + 2 * UR) + 8 + 4 * UR;
  auto kern = k_lag_gemm_tc<NB, STAGES>;
  SSI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, TC_THREADS, smem, stream>>>(thi, tlo, p, partial, status);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace

CovPlan cov_plan(int l, int64_t N, int max_lag, ssi_precision prec, int num_sms, size_t max_ws,
                 int64_t rows_req) {
  CovPlan c{};
  c.ldy = N;
  c.l = l;
  c.N = N;
  c.max_lag = max_lag;
  const int l64 = (int)round_up(l, 64);
  c.n_nt = (int)ceil_div(l64, 256);
  c.l_pad = (int)round_up(l, 64 * c.n_nt);
  c.nb = c.l_pad / 64 / c.n_nt;
  // time split: the persistent grid takes units dynamically, so its critical path is
  // (waves of units) x (samples per unit + the unit's epilogue, which costs about as much
  // as 512 samples of MMAs whatever the tile).  Choose the split length (a multiple of
  // BT, 512..16384 samples per FP32 partial sum) that minimises it; on ties the longer
  // split wins (fewer partials to write and reduce).
  const int n_atoms = max_lag * c.l_pad / 64;
  const int n_mp = (int)ceil_div(n_atoms, A_ATOMS);
  const int64_t units_per_split = (int64_t)n_mp * c.n_nt;
  // splits whose workspace exceeds max_ws are skipped (the fewest splits are kept if none
  // fits; the caller then sees ws_bytes above its cap)
  c.n_rows = std::max<int64_t>(N, 64);
  auto ws_of = [&](int64_t n_sp) {
    WsPlan w;
    if (prec == SSI_PREC_SPLIT_BF16) {
      w.add<__nv_bfloat16>((size_t)c.n_rows * c.l_pad);
      w.add<__nv_bfloat16>((size_t)c.n_rows * c.l_pad);
    }
    w.add<float>((size_t)n_sp * max_lag * c.l_pad * c.l_pad);
    if (prec == SSI_PREC_SPLIT_BF16) w.add<int>(64);   // the lag GEMM's unit counter
    return w.bytes;
  };
  int64_t best_rows = 0, best_cost = 0;
  const int64_t s_lo = std::max<int64_t>(1, ceil_div(N, 16384));
  const int64_t s_hi = std::max<int64_t>(s_lo, ceil_div(N, 512));
  if (rows_req > 0) {
    // the caller's split length, kept within the FP32 partial-sum bound of 16384 samples
    const int64_t rows = std::min<int64_t>(16384, std::max<int64_t>(512, round_up(rows_req, BT)));
    if (ws_of(ceil_div(N, rows)) <= max_ws) best_rows = rows;
  }
  const bool fixed = best_rows > 0;
  for (int64_t sp = s_lo; sp <= s_hi && !fixed; ++sp) {
    const int64_t rows = std::max<int64_t>(512, round_up(ceil_div(N, sp), BT));
    const int64_t n_sp = ceil_div(N, rows);
    if (sp > s_lo && ws_of(n_sp) > max_ws) continue;
    const int64_t waves = ceil_div(units_per_split * n_sp, (int64_t)std::max(1, num_sms));
    const int64_t cost = waves * (rows + 512);
    if (best_rows == 0 || cost < best_cost || (cost == best_cost && rows > best_rows)) {
      best_rows = rows;
      best_cost = cost;
    }
  }
  c.rows_per_split = (int)best_rows;
  c.n_split = (int)ceil_div(N, best_rows);
  c.ws_bytes = ws_of(c.n_split);
  return c;
}

ssi_status covariances_ws(ssi_ctx* ctx, Workspace& ws, const CovPlan& c, const float* Y,
                          ssi_precision prec, double* R, int* dev_status, cudaStream_t stream,
                          float acc_sign, float2* acc) {
  const dim3 red_grid((unsigned)ceil_div(c.l, 8), (unsigned)c.max_lag);
  ws.reset();
  const long long split_stride = (long long)c.max_lag * c.l_pad * c.l_pad;
  if (prec == SSI_PREC_SPLIT_BF16) {
    __nv_bfloat16* hi = ws.take<__nv_bfloat16>((size_t)c.n_rows * c.l_pad);
    __nv_bfloat16* lo = ws.take<__nv_bfloat16>((size_t)c.n_rows * c.l_pad);
    float* partial = ws.take<float>((size_t)c.n_split * split_stride);
    int* counter = ws.take<int>(64);
    if (!hi || !lo || !partial || !counter) {
      set_error("covariances: workspace too small");
      return SSI_E_NOMEM;
    }
    {
      ProfScope ps(ctx, ST_SPLIT, stream);
      dim3 blk(32, 8), grd((unsigned)ceil_div(c.n_rows, 32), c.l_pad / 32);
      k_split_transpose<<<grd, blk, 0, stream>>>(Y, c.ldy, c.l, (int)c.N, (int)c.n_rows, c.l_pad, hi, lo);
      SSI_CUDA(cudaGetLastError());
    }
    CUtensorMap thi, tlo;
    if (!make_tmap_bf16_2d(&thi, hi, (uint64_t)c.n_rows, c.l_pad, c.l_pad, 64, BT,
                           CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_tmap_bf16_2d(&tlo, lo, (uint64_t)c.n_rows, c.l_pad, c.l_pad, 64, BT,
                           CU_TENSOR_MAP_SWIZZLE_128B))
      return SSI_E_CUDA;
    LagGemmParams p{};
    p.n_atoms = c.max_lag * c.l_pad / 64;
    p.n_mp = (int)ceil_div(p.n_atoms, A_ATOMS);
    p.n_nt = c.n_nt;
    p.n_split = c.n_split;
    p.rows_per_split = c.rows_per_split;
    p.N = (int)c.N;
    p.l_pad = c.l_pad;
    p.ld_out = c.l_pad;
    p.split_stride = split_stride;
    p.unit_counter = counter;
    SSI_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), stream));
    const int n_units = p.n_mp * p.n_nt * p.n_split;
    const int grid = std::min(n_units, ctx->num_sms);
    {
      ProfScope ps(ctx, ST_LAG_GEMM, stream);
      ssi_status st;
      switch (c.nb) {
        case 1: st = launch_tc<1>(thi, tlo, p, partial, dev_status, grid, stream); break;
        case 2: st = launch_tc<2>(thi, tlo, p, partial, dev_status, grid, stream); break;
        case 3: st = launch_tc<3>(thi, tlo, p, partial, dev_status, grid, stream); break;
        case 4: st = launch_tc<4>(thi, tlo, p, partial, dev_status, grid, stream); break;
        default: set_error("covariances: unsupported channel tiling"); return SSI_E_INVALID;
      }
      SSI_TRY(st);
    }
    {
      ProfScope ps(ctx, ST_LAG_REDUCE, stream);
      if (!acc)
        k_reduce_partials<<<ctx->num_sms * 8, 256, 0, stream>>>(partial, c.n_split, split_stride, c.l,
                                                                c.l_pad, c.max_lag, (int)c.N, R);
      else
        k_accumulate_partials<<<red_grid, 256, 0, stream>>>(partial, c.n_split, split_stride, c.l,
                                                            c.l_pad, acc_sign, acc);
      SSI_CUDA(cudaGetLastError());
    }
    count_launches(ctx, 3);
  } else {
    float* partial = ws.take<float>((size_t)c.n_split * split_stride);
    if (!partial) { set_error("covariances: workspace too small"); return SSI_E_NOMEM; }
    const int nb = (c.l + 63) / 64;
    {
      ProfScope ps(ctx, ST_LAG_GEMM, stream);
      dim3 grd((unsigned)(c.max_lag * nb * nb), (unsigned)c.n_split);
      k_lag_gemm_fp32<<<grd, 256, 0, stream>>>(Y, c.ldy, c.l, (int)c.N, c.l_pad, c.max_lag,
                                               c.rows_per_split, split_stride, partial);
      SSI_CUDA(cudaGetLastError());
    }
    {
      ProfScope ps(ctx, ST_LAG_REDUCE, stream);
      if (!acc)
        k_reduce_partials<<<ctx->num_sms * 8, 256, 0, stream>>>(partial, c.n_split, split_stride, c.l,
                                                                c.l_pad, c.max_lag, (int)c.N, R);
      else
        k_accumulate_partials<<<red_grid, 256, 0, stream>>>(partial, c.n_split, split_stride, c.l,
                                                            c.l_pad, acc_sign, acc);
      SSI_CUDA(cudaGetLastError());
    }
    count_launches(ctx, 2);
  }
  return SSI_OK;
}

}  // namespace ssi

extern "C" ssi_status ssi_covariances(ssi_ctx* ctx, const float* Y, int l, int64_t N, int max_lag,
                                      ssi_precision prec, double* R, void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx, "ssi_covariances: null context");
  SSI_CHECK(Y && R, "ssi_covariances: null pointer");
  SSI_CHECK(l >= 1 && l <= 1024, "ssi_covariances: l=%d out of range [1, 1024]", l);
  SSI_CHECK(max_lag >= 1 && (int64_t)max_lag < N, "ssi_covariances: need 1 <= max_lag < N");
  SSI_CHECK(N < (1LL << 31) - 1024, "ssi_covariances: N too large");
  SSI_CHECK(prec == SSI_PREC_FP32 || prec == SSI_PREC_SPLIT_BF16, "ssi_covariances: bad precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SSI_CUDA(cudaSetDevice(ctx->device));
  CovPlan plan = cov_plan(l, N, max_lag, prec, ctx->num_sms);
  SSI_TRY(ws_reserve(ctx, ctx->ws, plan.ws_bytes, s));
  SSI_TRY(covariances_ws(ctx, ctx->ws, plan, Y, prec, R, ctx->dev_status, s));
  return SSI_OK;
}

// ---------------------------------------------------------------------------------------
// Covariances without any device allocation.
//
// Some callers cannot allocate device memory at the time they need covariances: code
// running inside a CUDA-graph capture that must not add allocation nodes, plugins of a
// host framework that owns every device allocation, or processes that run under a fixed
// memory reservation.  For them this variant keeps its scratch (the per-time-chunk FP32
// partial sums of the CUDA-core lag GEMM) in one file-scope device array of
// NOALLOC_SCRATCH_FLOATS floats (16 MiB), which every GPU that loads the library holds
// until the process exits.  Inputs and outputs still come from the caller.
// ---------------------------------------------------------------------------------------
namespace ssi {
namespace {

constexpr size_t NOALLOC_SCRATCH_FLOATS = size_t(4) << 20;   // 16 MiB
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

// Device address of the scratch array on the current device.  Host code cannot use the
// array's name as an address; it asks the runtime on every call (a host-side lookup), so
// that the address stays right after the device's context has been torn down and
// recreated, e.g. by cudaDeviceReset.
ssi_status noalloc_scratch(float** out) {
  void* p = nullptr;
  SSI_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = static_cast<float*>(p);
  return SSI_OK;
}

}  // namespace
}  // namespace ssi

extern "C" ssi_status ssi_covariances_noalloc(const float* Y, int l, int64_t N, int max_lag,
                                              double* R, void* stream) {
  using namespace ssi;
  SSI_CHECK(Y && R, "ssi_covariances_noalloc: null pointer");
  SSI_CHECK(l >= 1 && l <= 1024, "ssi_covariances_noalloc: l=%d out of range [1, 1024]", l);
  SSI_CHECK(max_lag >= 1 && (int64_t)max_lag < N, "ssi_covariances_noalloc: need 1 <= max_lag < N");
  SSI_CHECK(N < (1LL << 31) - 1024, "ssi_covariances_noalloc: N too large");
  int device = 0;
  SSI_CUDA(cudaGetDevice(&device));
  const int l_pad = (int)round_up(l, 64);
  const size_t per_split = (size_t)max_lag * l_pad * l_pad;
  if (per_split > NOALLOC_SCRATCH_FLOATS) {
    set_error("ssi_covariances_noalloc: max_lag * roundup(l, 64)^2 = %zu floats exceeds the "
              "fixed scratch of %zu floats; use ssi_covariances",
              per_split, NOALLOC_SCRATCH_FLOATS);
    return SSI_E_INVALID;
  }
  float* scratch = nullptr;
  SSI_TRY(noalloc_scratch(&scratch));
  // as many time chunks as fit the scratch, at most one per 512 samples and 64 in all
  int64_t n_split = (int64_t)(NOALLOC_SCRATCH_FLOATS / per_split);
  n_split = std::min<int64_t>(n_split, std::min<int64_t>(64, ceil_div(N, 512)));
  n_split = std::max<int64_t>(1, n_split);
  const int rows_per_split = (int)round_up(ceil_div(N, n_split), 32);
  n_split = ceil_div(N, rows_per_split);
  const int nb = (l + 63) / 64;
  const int num_sms = device_sms(device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every partial entry read by the reduction is written by the GEMM, so nothing needs
  // clearing between calls
  dim3 grd((unsigned)(max_lag * nb * nb), (unsigned)n_split);
  k_lag_gemm_fp32<<<grd, 256, 0, s>>>(Y, (long long)N, l, (int)N, l_pad, max_lag, rows_per_split,
                                      (long long)per_split, scratch);
  SSI_CUDA(cudaGetLastError());
  k_reduce_partials<<<num_sms * 4, 256, 0, s>>>(scratch, (int)n_split, (long long)per_split, l,
                                                l_pad, max_lag, (int)N, R);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}
