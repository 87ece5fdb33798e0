// Small SVD of the RSVD (Sec. 2.2: P = U~ Sigma V^T, Algorithm 1).
//
// With P^T = Q2 R2 (QR of the K x L_cols matrix's transpose), the left singular
// vectors of P are the right singular vectors of R2.  One-sided (Hestenes) Jacobi
// on B = R2^T: rotating the columns of B until they are mutually orthogonal gives
// B V = W Sigma, hence R2 = V Sigma W^T and U~ = W (the normalised columns of B),
// Sigma = their norms; V itself is never needed.
//
// Parallel block ordering on a cooperative grid of C CTAs.  The K columns are cut into
// 2C blocks of bw columns; in each outer round every CTA holds two blocks and rotates
// every column of the one against every column of the other (bw inner rounds of bw
// disjoint pairs, one warp per pair), and in the first outer round of a sweep also the
// pairs inside each of its two blocks.  The blocks move between CTAs by the circle
// (round-robin) schedule of 2C players, so one sweep (2C - 1 outer rounds) meets every
// column pair once.  The blocks of a round are staged in shared memory when they fit;
// the global copy of B is the exchange medium, and a bounded grid barrier separates the
// rounds.  Sweeps stop when no pair of a sweep had |b_p^T b_q| > tol ||b_p|| ||b_q||, or
// after max_sweeps (status bit set).  Every reduction runs in a fixed order, so the
// result does not depend on timing.
//
// When the grid is small enough for one thread-block cluster (C <= 8 CTAs), the rounds
// run in k_cluster_jacobi instead: the same schedule and the same rotations in the same
// order (so the same result), but the blocks stay in shared memory for the whole launch.
// Between rounds each CTA copies the two blocks of its next round out of the shared
// memory of the CTAs that hold them (distributed shared memory, double-buffered), and
// the CTAs meet at the cluster's hardware barrier instead of a barrier on a global
// counter.
//
// The scalar type is FP32 (the default small-problem arithmetic) or FP64.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include <cooperative_groups.h>

#include "blackwell.cuh"
#include "common.cuh"

namespace cg = cooperative_groups;

namespace ssi {

namespace {

constexpr int BJ_THREADS = 512;
constexpr int BJ_WARPS = BJ_THREADS / 32;
constexpr uint64_t BJ_BAR_NS = 2000000000ull;
constexpr size_t BJ_SMEM_MAX = 200 * 1024;

template <typename T>
struct BjParams {
  const float* R2;      // K x K row-major: column c of B = R2^T is row c of R2
  int K, ldb;           // B in global memory, column c at B + c * ldb
  T* B;
  int n_blk, bw;        // 2C blocks of bw columns (the last ones may be short or empty)
  T tol;
  int max_sweeps;
  int* flags;           // [max_sweeps] "some pair was rotated", zeroed before the launch
  unsigned* bar;        // [0] grid barrier counter, [8] abort flag; zeroed before the launch
  T* norms;             // K column norms
  T* Ut;                // K x K row-major: column j = singular vector of rank j
  T* S;                 // K singular values, descending
  int* status;
  int ldk;              // leading dimension of a staged column (0: blocks stay in global)
};

// Grid barrier on a monotonic arrival counter: barrier j of the launch passes once the
// counter reaches j x gridDim.x.  The wait is bounded; on timeout the status word gets
// DEV_TIMEOUT and every CTA leaves through the abort flag.
template <typename T>
__device__ bool bj_grid_sync(const BjParams<T>& p, unsigned& n_bar) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    n_bar += 1;
    const unsigned target = n_bar * gridDim.x;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(p.bar + 8);
    __threadfence();
    const unsigned arrived = atomicAdd(&p.bar[0], 1u) + 1u;
    if (arrived < target) {
      const uint64_t t0 = bw::global_ns();
      while (*(volatile unsigned*)&p.bar[0] < target) {
        if (*abort_flag) { ok = 0; break; }
        if (bw::global_ns() - t0 > BJ_BAR_NS) {
          atomicOr(p.status, DEV_TIMEOUT);
          atomicExch(reinterpret_cast<int*>(p.bar + 8), 1);
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

__device__ __forceinline__ float bj_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double bj_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float bj_pow2_inv(float m) { return ldexpf(1.f, -ilogbf(m)); }
__device__ __forceinline__ double bj_pow2_inv(double m) { return ldexp(1.0, -ilogb(m)); }

// Rotation of columns x, y with a = x.x, b = y.y, g = x.y that makes them orthogonal
// (Hestenes): with d = (b - a) / 2, t = tan(theta) = sign(d) g / (|d| + hypot(d, g)),
// c = 1 / sqrt(1 + t^2), s = c t.  Written with D = |d| + hypot(d, g) and
// h = hypot(D, g): c = D / h, s = sign(d) g / h -- two square roots and one division on
// the critical path.  d and g are first scaled by a power of two near 1 / max(a, b)
// (exact), so the squares neither overflow nor lose the larger term.
template <typename T>
__device__ __forceinline__ void rotation(T a, T b, T g, T& c, T& s) {
  const T sc = bj_pow2_inv(a > b ? a : b);
  const T d = (b - a) * (sc * T(0.5)), gs = g * sc;
  const T r = bj_sqrt(fma(d, d, gs * gs));
  const T D = fabs(d) + r;
  const T inv = T(1) / bj_sqrt(fma(D, D, gs * gs));
  c = D * inv;
  s = (d >= T(0) ? gs : -gs) * inv;
}

// One Jacobi rotation of columns x and y (length K) by one warp; returns whether it
// rotated (the same in every lane).  Columns of up to 32 * BJ_REG entries (8 FP32 or 4
// FP64 registers a lane per column) stay in registers between the dot products and the
// update.
template <typename T>
__device__ __forceinline__ bool rotate_pair(T* x, T* y, int K, T tol, int lane) {
  constexpr int BJ_REG = sizeof(T) == 8 ? 4 : 8;
  T a = 0, b = 0, g = 0;
  const bool in_reg = K <= 32 * BJ_REG;
  T xr[BJ_REG], yr[BJ_REG];
  if (in_reg) {
#pragma unroll
    for (int q = 0; q < BJ_REG; ++q) {
      const int r = lane + 32 * q;
      xr[q] = r < K ? x[r] : T(0);
      yr[q] = r < K ? y[r] : T(0);
    }
#pragma unroll
    for (int q = 0; q < BJ_REG; ++q) {
      a = fma(xr[q], xr[q], a);
      b = fma(yr[q], yr[q], b);
      g = fma(xr[q], yr[q], g);
    }
  } else {
    for (int r = lane; r < K; r += 32) {
      const T xv = x[r], yv = y[r];
      a = fma(xv, xv, a);
      b = fma(yv, yv, b);
      g = fma(xv, yv, g);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  // rotate when |g| > tol sqrt(a b), i.e. g^2 > tol^2 a b (a, b > 0)
  if (!(a > T(0) && b > T(0)) || !(g * g > (tol * tol) * (a * b))) return false;
  T c, s;
  rotation(a, b, g, c, s);
  if (in_reg) {
#pragma unroll
    for (int q = 0; q < BJ_REG; ++q) {
      const int r = lane + 32 * q;
      if (r < K) {
        x[r] = c * xr[q] - s * yr[q];
        y[r] = s * xr[q] + c * yr[q];
      }
    }
  } else {
    for (int r = lane; r < K; r += 32) {
      const T xv = x[r], yv = y[r];
      x[r] = c * xv - s * yv;
      y[r] = s * xv + c * yv;
    }
  }
  return true;
}

// player at position pos of round r of the circle schedule of np players (np even)
__device__ __forceinline__ int circle_player(int pos, int r, int np) {
  if (pos == 0) return 0;
  int v = pos - 1 + r;
  v %= (np - 1);
  return 1 + v;
}

template <typename T>
__global__ void __launch_bounds__(BJ_THREADS, 1) k_block_jacobi(BjParams<T> p) {
  extern __shared__ __align__(16) unsigned char bj_smem_raw[];
  T* smem = reinterpret_cast<T*>(bj_smem_raw);
  __shared__ int s_rot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = p.K, bw = p.bw, np = p.n_blk;
  unsigned n_bar = 0;
  // B = R2^T in T precision: column c of B is row c of R2
  for (long long e = (long long)blockIdx.x * BJ_THREADS + tid; e < (long long)K * K;
       e += (long long)gridDim.x * BJ_THREADS) {
    const int c = (int)(e / K), r = (int)(e % K);
    p.B[(size_t)c * p.ldb + r] = (T)p.R2[e];
  }
  if (!bj_grid_sync(p, n_bar)) return;
  const bool staged = p.ldk > 0;
  T* sA = smem;
  T* sB = smem + (size_t)bw * p.ldk;
  int sweep = 0;
  bool converged = false;
  for (; sweep < p.max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    bool rot = false;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      const int pa = circle_player(blockIdx.x, rnd, np);
      const int pb = circle_player(np - 1 - blockIdx.x, rnd, np);
      const int a0 = pa * bw, b0 = pb * bw;
      const int na = max(0, min(bw, K - a0)), nb = max(0, min(bw, K - b0));
      T* A = staged ? sA : p.B + (size_t)a0 * p.ldb;
      T* Bk = staged ? sB : p.B + (size_t)b0 * p.ldb;
      const int ld = staged ? p.ldk : p.ldb;
      if (staged) {
        for (int e = tid; e < na * K; e += BJ_THREADS)
          sA[(size_t)(e / K) * ld + e % K] = p.B[(size_t)(a0 + e / K) * p.ldb + e % K];
        for (int e = tid; e < nb * K; e += BJ_THREADS)
          sB[(size_t)(e / K) * ld + e % K] = p.B[(size_t)(b0 + e / K) * p.ldb + e % K];
      }
      __syncthreads();
      if (rnd == 0) {
        // pairs inside each of the two blocks: circle schedule of bw (even) players, both
        // blocks at once (pairs 0..half-1 in A, half..2 half-1 in B)
        const int bwe = bw + (bw & 1), half = bwe / 2;
        for (int ir = 0; ir < bwe - 1; ++ir) {
          for (int q = warp; q < 2 * half; q += BJ_WARPS) {
            const int which = q / half, j = q % half;
            int u = circle_player(j, ir, bwe), v = circle_player(bwe - 1 - j, ir, bwe);
            const int ncol = which ? nb : na;
            if (u < ncol && v < ncol) {
              T* base = which ? Bk : A;
              rot |= rotate_pair(base + (size_t)u * ld, base + (size_t)v * ld, K, p.tol, lane);
            }
          }
          __syncthreads();
        }
      }
      // every column of block A against every column of block B: bw inner rounds of bw
      // disjoint pairs (j, (j + ir) mod bw)
      for (int ir = 0; ir < bw; ++ir) {
        for (int j = warp; j < bw; j += BJ_WARPS) {
          const int v = (j + ir) % bw;
          if (j < na && v < nb)
            rot |= rotate_pair(A + (size_t)j * ld, Bk + (size_t)v * ld, K, p.tol, lane);
        }
        __syncthreads();
      }
      if (staged) {
        for (int e = tid; e < na * K; e += BJ_THREADS)
          p.B[(size_t)(a0 + e / K) * p.ldb + e % K] = sA[(size_t)(e / K) * ld + e % K];
        for (int e = tid; e < nb * K; e += BJ_THREADS)
          p.B[(size_t)(b0 + e / K) * p.ldb + e % K] = sB[(size_t)(e / K) * ld + e % K];
      }
      if (rnd == np - 2) {
        if (rot && lane == 0) s_rot = 1;
        __syncthreads();
        if (tid == 0 && s_rot) atomicOr(&p.flags[sweep], 1);
      }
      if (!bj_grid_sync(p, n_bar)) return;
    }
    converged = *(volatile int*)&p.flags[sweep] == 0;
  }
  if (!converged && blockIdx.x == 0 && tid == 0) atomicOr(p.status, DEV_NOTCONVERGED);
  // column norms, then each column's rank among them, S and the normalised columns
  for (int c = blockIdx.x * BJ_WARPS + warp; c < K; c += gridDim.x * BJ_WARPS) {
    T s = 0;
    for (int r = lane; r < K; r += 32) {
      const T v = p.B[(size_t)c * p.ldb + r];
      s = fma(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) p.norms[c] = bj_sqrt(s);
  }
  if (!bj_grid_sync(p, n_bar)) return;
  for (int c = blockIdx.x * BJ_WARPS + warp; c < K; c += gridDim.x * BJ_WARPS) {
    const T v = p.norms[c];
    int rank = 0;
    for (int d = lane; d < K; d += 32) {
      const T u = p.norms[d];
      rank += (u > v) || (u == v && d < c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0) p.S[rank] = v;
    const T inv = v > T(0) ? T(1) / v : T(0);
    for (int r = lane; r < K; r += 32) p.Ut[(size_t)r * K + rank] = p.B[(size_t)c * p.ldb + r] * inv;
  }
}

// position of player P at round r of the circle schedule (the inverse of circle_player)
__device__ __forceinline__ int circle_pos(int P, int r, int np) {
  if (P == 0) return 0;
  int v = (P - 1 - r) % (np - 1);
  if (v < 0) v += np - 1;
  return 1 + v;
}

constexpr int BJ_CLUSTER_MAX = 8;   // portable cluster size

// The block ordering of k_block_jacobi on one cluster of C = gridDim.x CTAs (grid =
// cluster).  Shared memory holds two buffers of two blocks (bw x ldk each); round g
// computes on buffer g & 1 and then pulls the next round's blocks into the other one.
// A peer reads buffer g & 1 of this CTA only between the barriers that close rounds g
// and g + 1, and this CTA rewrites it only after the barrier closing round g + 1, so one
// cluster barrier per round suffices.  Every CTA takes the same number of barriers: the
// end of a sweep is decided from every CTA's rotation flag, read after the barrier.
template <typename T>
__global__ void __launch_bounds__(BJ_THREADS, 1) k_cluster_jacobi(BjParams<T> p) {
  extern __shared__ __align__(16) unsigned char bj_smem_raw[];
  T* smem = reinterpret_cast<T*>(bj_smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  __shared__ int s_rot;
  __shared__ int s_flag[2];
  __shared__ T s_norm[2][64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = p.K, bw = p.bw, np = p.n_blk, C = np / 2;
  const int me = (int)cl.block_rank();
  const int ld = p.ldk;
  const size_t slot = (size_t)bw * ld;
  auto buf = [&](int b, int s) { return smem + (size_t)(2 * b + s) * slot; };
  auto ncols = [&](int P) { return max(0, min(bw, K - P * bw)); };
  // round 0: the CTA's two blocks straight from R2 (column c of B = row c of R2)
  for (int s = 0; s < 2; ++s) {
    const int P = circle_player(s ? np - 1 - me : me, 0, np);
    const int c0 = P * bw, nc = ncols(P);
    T* dst = buf(0, s);
    for (int e = tid; e < nc * K; e += BJ_THREADS)
      dst[(size_t)(e / K) * ld + e % K] = (T)p.R2[(size_t)(c0 + e / K) * K + e % K];
  }
  if (tid == 0) {
    s_flag[0] = 0;
    s_flag[1] = 0;
  }
  __syncthreads();
  int cur = 0, pa = 0, pb = 0;
  int sweep = 0;
  bool converged = false;
  for (; sweep < p.max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    bool rot = false;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      pa = circle_player(me, rnd, np);
      pb = circle_player(np - 1 - me, rnd, np);
      const int na = ncols(pa), nb = ncols(pb);
      T* A = buf(cur, 0);
      T* Bk = buf(cur, 1);
      if (rnd == 0) {
        const int bwe = bw + (bw & 1), half = bwe / 2;
        for (int ir = 0; ir < bwe - 1; ++ir) {
          for (int q = warp; q < 2 * half; q += BJ_WARPS) {
            const int which = q / half, j = q % half;
            int u = circle_player(j, ir, bwe), v = circle_player(bwe - 1 - j, ir, bwe);
            const int ncol = which ? nb : na;
            if (u < ncol && v < ncol) {
              T* base = which ? Bk : A;
              rot |= rotate_pair(base + (size_t)u * ld, base + (size_t)v * ld, K, p.tol, lane);
            }
          }
          __syncthreads();
        }
      }
      for (int ir = 0; ir < bw; ++ir) {
        for (int j = warp; j < bw; j += BJ_WARPS) {
          const int v = (j + ir) % bw;
          if (j < na && v < nb)
            rot |= rotate_pair(A + (size_t)j * ld, Bk + (size_t)v * ld, K, p.tol, lane);
        }
        __syncthreads();
      }
      const bool last = rnd == np - 2;
      if (last) {
        if (rot && lane == 0) s_rot = 1;
        __syncthreads();
        if (tid == 0) s_flag[sweep & 1] = s_rot;
      }
      cl.sync();
      if (last) {
        int any = 0;
        for (int r = 0; r < C; ++r) any |= *cl.map_shared_rank(&s_flag[sweep & 1], r);
        converged = any == 0;
        if (converged || sweep + 1 == p.max_sweeps) break;   // the blocks stay where they are
      }
      // pull the next round's two blocks (round rnd + 1, modulo np - 1)
      const int r1 = rnd + 1;
      for (int s = 0; s < 2; ++s) {
        const int P = circle_player(s ? np - 1 - me : me, r1, np);
        const int pos = circle_pos(P, rnd, np);
        const int holder = pos < C ? pos : np - 1 - pos, hs = pos < C ? 0 : 1;
        const uint4* src = reinterpret_cast<const uint4*>(cl.map_shared_rank(buf(cur, hs), holder));
        uint4* dst = reinterpret_cast<uint4*>(buf(cur ^ 1, s));
        const int n16 = (int)((size_t)ncols(P) * ld * sizeof(T) / 16);
        for (int e = tid; e < n16; e += BJ_THREADS) dst[e] = src[e];
      }
      __syncthreads();
      cur ^= 1;
    }
  }
  if (!converged && me == 0 && tid == 0) atomicOr(p.status, DEV_NOTCONVERGED);
  // column norms of the CTA's two blocks (players pa and pb of the last round)
  for (int q = warp; q < 2 * bw; q += BJ_WARPS) {
    const int s = q / bw, j = q % bw, P = s ? pb : pa;
    if (j >= ncols(P)) continue;
    const T* col = buf(cur, s) + (size_t)j * ld;
    T v = 0;
    for (int r = lane; r < K; r += 32) v = fma(col[r], col[r], v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      s_norm[s][j] = bj_sqrt(v);
      p.norms[P * bw + j] = bj_sqrt(v);
    }
  }
  __threadfence();
  cl.sync();
  for (int q = warp; q < 2 * bw; q += BJ_WARPS) {
    const int s = q / bw, j = q % bw, P = s ? pb : pa;
    if (j >= ncols(P)) continue;
    const int c = P * bw + j;
    const T v = s_norm[s][j];
    int rank = 0;
    for (int d = lane; d < K; d += 32) {
      const T u = *(volatile T*)&p.norms[d];
      rank += (u > v) || (u == v && d < c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0) p.S[rank] = v;
    const T inv = v > T(0) ? T(1) / v : T(0);
    const T* col = buf(cur, s) + (size_t)j * ld;
    for (int r = lane; r < K; r += 32) p.Ut[(size_t)r * K + rank] = col[r] * inv;
  }
  // no CTA leaves while a peer may still read its shared memory
  cl.sync();
}

// Grid of the block ordering: C CTAs, 2C blocks of bw columns.  FP32 rounds are short
// and latency-bound, so fewer, wider blocks (about 14 columns) keep the barrier count
// low; FP64 work is bound by the FP64 pipes (two FMA per clock per SM), so it spreads
// over more SMs with narrow blocks.
struct BjGrid {
  int C, bw;
};

BjGrid bj_grid(int K, bool fp64, int num_sms, int block = 0) {
  const int target_bw = block > 0 ? block : (fp64 ? 2 : 14);
  int C = std::max(1, (int)ceil_div(K, 2 * target_bw));
  C = std::min(C, num_sms);
  int bw = (int)ceil_div(K, 2 * C);
  return {C, bw};
}

template <typename T>
size_t bj_smem(int K, int bw) {
  const int ldk = (int)round_up(K, 2);
  return (size_t)2 * bw * ldk * sizeof(T);
}

template <typename T>
size_t bj_ws_bytes_t(int K, int num_sms) {
  const BjGrid g = bj_grid(K, sizeof(T) == 8, num_sms);
  WsPlan w;
  w.add<T>((size_t)K * round_up(K, 4));   // B
  w.add<T>((size_t)K);                     // norms
  w.add<int>(256);                         // sweep flags
  w.add<unsigned>(64);                     // barrier
  (void)g;
  return w.bytes;
}

// Whether a cluster of C CTAs with `smem` bytes of dynamic shared memory each can be
// resident on this device (asked once per shape and device).
template <typename T>
bool cluster_fits(int C, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, std::pair<int, size_t>>, bool> known;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, std::make_pair(C, smem));
  auto it = known.find(key);
  if (it != known.end()) return it->second;
  bool ok = cudaFuncSetAttribute(k_cluster_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)BJ_SMEM_MAX) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(BJ_THREADS);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, k_cluster_jacobi<T>, &cfg) == cudaSuccess && n > 0;
  }
  cudaGetLastError();   // a refused query leaves no sticky error behind
  known[key] = ok;
  return ok;
}

template <typename T>
ssi_status bj_launch(Workspace& ws, const float* R2, int K, T* Ut, T* S, int* status, int num_sms,
                     int block, T tol, int max_sweeps, cudaStream_t stream) {
  const BjGrid g = bj_grid(K, sizeof(T) == 8, num_sms, block);
  BjParams<T> p{};
  p.R2 = R2;
  p.K = K;
  p.ldb = (int)round_up(K, 4);
  p.B = ws.take<T>((size_t)K * p.ldb);
  p.norms = ws.take<T>((size_t)K);
  p.flags = ws.take<int>(256);
  p.bar = ws.take<unsigned>(64);
  if (!p.B || !p.norms || !p.flags || !p.bar) {
    set_error("jacobi: workspace too small");
    return SSI_E_NOMEM;
  }
  p.n_blk = 2 * g.C;
  p.bw = g.bw;
  p.tol = tol;
  p.max_sweeps = std::min(max_sweeps, 256);
  p.Ut = Ut;
  p.S = S;
  p.status = status;
  size_t smem = bj_smem<T>(K, g.bw);
  if (smem > BJ_SMEM_MAX) {
    smem = 0;
    p.ldk = 0;   // the blocks stay in global memory (L2-resident)
  } else {
    p.ldk = (int)round_up(K, 2);
  }
  if (g.C <= BJ_CLUSTER_MAX && g.bw <= 64) {
    // one cluster: four blocks (two buffers of two) in shared memory, 16-byte rows
    const int ldk = (int)round_up(K, 4);
    const size_t csmem = (size_t)4 * g.bw * ldk * sizeof(T);
    if (csmem <= BJ_SMEM_MAX && cluster_fits<T>(g.C, csmem)) {
      p.ldk = ldk;
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(g.C);
      cfg.blockDim = dim3(BJ_THREADS);
      cfg.dynamicSmemBytes = csmem;
      cfg.stream = stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = g.C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      SSI_CUDA(cudaLaunchKernelEx(&cfg, k_cluster_jacobi<T>, p));
      return SSI_OK;
    }
  }
  SSI_CUDA(cudaMemsetAsync(p.flags, 0, 256 * sizeof(int), stream));
  SSI_CUDA(cudaMemsetAsync(p.bar, 0, 64 * sizeof(unsigned), stream));
  SSI_CUDA(cudaFuncSetAttribute(k_block_jacobi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)BJ_SMEM_MAX));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(g.C);
  cfg.blockDim = dim3(BJ_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SSI_CUDA(cudaLaunchKernelEx(&cfg, k_block_jacobi<T>, p));
  return SSI_OK;
}

}  // namespace

size_t jacobi_ws_bytes(int K, int num_sms, bool fp64) {
  return fp64 ? bj_ws_bytes_t<double>(K, num_sms) : bj_ws_bytes_t<float>(K, num_sms);
}

// FP32: stop at |b_p^T b_q| <= 1e-5 ||b_p|| ||b_q|| (30 sweeps at most); FP64: 1e-13
// (the rounding of an FP64 dot product of length K is about sqrt(K) 1e-16).
ssi_status jacobi_launch(Workspace& ws, const float* R2, int K, float* Ut, float* S, int* status,
                         int num_sms, int block, cudaStream_t stream) {
  return bj_launch<float>(ws, R2, K, Ut, S, status, num_sms, block, 1e-5f, 30, stream);
}

ssi_status jacobi_launch64(Workspace& ws, const float* R2, int K, double* Ut, double* S, int* status,
                           int num_sms, int block, cudaStream_t stream) {
  return bj_launch<double>(ws, R2, K, Ut, S, status, num_sms, block, 1e-13, 40, stream);
}

}  // namespace ssi
