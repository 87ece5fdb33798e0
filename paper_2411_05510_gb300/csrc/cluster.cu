// Two-stage clustering of the stable poles of a stabilization diagram (Sec. 2.3,
// "3D clustering"; Sec. 3.1).
//
// Stage I.  Every pole that passes the hard criteria and is stable along orders or lags
// gets the feature vector x = (d_f, d_xi, 1 - MAC, 1 - MPC, MPD).  The first three are
// taken against the pole's nearest HC-passing neighbour, nearest in d_f + d_xi + (1 - MAC),
// among the poles of the previous order of the same lag and of the same order of the
// previous lag (the neighbourhoods of Eq. (stabcriteria3D)); d = |a - b| / max(a, b).
// Fuzzy C-means with two clusters (Bezdek's alternation, started from the feature-wise
// minimum and maximum) splits the poles; the cluster whose centroid lies nearer the
// origin is the possibly physical one, and a pole is kept when its membership of that
// cluster is at least 1/2.
// Stage II.  Single linkage in d_f + d_xi + (1 - MAC) over the kept poles, cut at tau:
// the clusters are the connected components of the graph that joins two poles at
// distance <= tau.  Clusters of at least min_size poles are the modes; a mode reports the
// mean frequency and damping of its poles, its size and its medoid (the member with the
// smallest sum of distances to the others, ties to the earlier pole).
//
// Every decision (nearest neighbour, link) is taken on FP64 distances, the medoid on sums
// of double-float-accurate distances (~1e-13 relative).  MACs are
// first screened in FP32 (lanes over channels, FP32 FMA): the FP32 MAC of unit vectors
// differs from the exact one by at most eps = 2 (5 gamma + 4 u), gamma = (2 ceil(l/32) + 5) u,
// u = 2^-24 (the per-lane FMA chain plus the shuffle tree; the bound is relative to
// |a| |b| and does not depend on the normalisation).  Only candidates within that bound
// of a decision are recomputed with FP64 accumulation, so the decisions are those of the
// FP64 definition.
//
// Kernels, in launch order:
//   k_features      one warp per slot: Stage I features of the candidates (two passes,
//                   FP32 screening then FP64 among the screened neighbours)
//   k_fcm           cooperative persistent kernel: candidate min/max, the C-means
//                   iterations with a fixed-order reduction over fixed 128-slot chunks
//                   (bit-identical for any grid size), memberships, the ordered list of
//                   kept poles
//   k_prelink       join each kept pole to its Stage I nearest neighbour when that one is
//                   kept and within tau (an exact Stage II link found for free)
//   k_compress      point every kept pole at its root
//   k_link          tiles of 32 x 32 kept-pole pairs: screen by d_f + d_xi, skip pairs
//                   already connected, decide d <= tau, join components (lock-free union-
//                   find whose roots are the smallest index of their component)
//   k_label         component root and size of every kept pole
//   k_modes_scan    one CTA: components in index order, those with >= min_size poles
//   k_mode_members  one CTA per mode: its members in index order, mean f and xi
//   k_medoid_prep   one warp per member: FP64 reciprocals of f, xi and |phi|^2
//   k_medoid_tiles  each pair of a mode once, in 32 x 32 tiles: distances with double-
//                   float cross products and an FP64 finish of 32 partners side by side,
//                   row and column sums per tile
//   k_medoid_finish one thread per member: its sum over the tiles, in order
//   k_medoid_pick   one CTA per mode: first minimum
//   k_relabel       (per-slot labels asked for) the slot of each kept pole's component root
#include "common.cuh"
#include "blackwell.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ssi {
namespace {

constexpr int CL_THREADS = 256;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int FCM_THREADS = 128;       // C-means CTA: one slot of its chunk per thread
constexpr int FCM_WARPS = FCM_THREADS / 32;
constexpr int FCM_CH = 128;            // slots per C-means chunk (fixes the reduction order)
constexpr int FCM_NV = 13;             // per chunk: sum w0 x (5), sum w0, sum w1 x (5), sum w1, max |du|
constexpr int FCM_STRIDE = 16;
constexpr int FCM_RED_PER = 8;         // threads per value of the cross-chunk reduction
constexpr uint64_t CL_BAR_NS = 2000000000ull;
constexpr int UNION_LIMIT = 1 << 20;
constexpr int SCAN_THREADS = 1024;

struct Grid {
  int n_lags, n_orders, l;
  long long slots_per_lag;
  long long slot_off[512];
  int nslot[512];
};

// device-side results read back by the host
struct Hdr {
  int n_cand, n_kept, iters, converged, phys, n_comp, n_modes, pad;
  double V[2][5];
};

__device__ __forceinline__ double rel_diff(double a, double b) { return fabs(a - b) / fmax(a, b); }

// FP32 screen of d_f + d_xi: within 3 ulp (relative) of the FP64 value of the same
// FP32 inputs (one subtraction, one division per term, one addition).
__device__ __forceinline__ float rel_sum32(float fa, float fb, float xa, float xb) {
  return fabsf(fa - fb) / fmaxf(fa, fb) + fabsf(xa - xb) / fmaxf(xa, xb);
}

__device__ __forceinline__ bool pole_live(uint32_t fl) {
  return (fl & SSI_POLE_VALID) && (fl & SSI_POLE_HC);
}

__device__ __forceinline__ void slot_cell(const Grid& g, long long e, int& t, int& m) {
  t = (int)(e / g.slots_per_lag);
  const long long w = e - (long long)t * g.slots_per_lag;
  int lo = 0, hi = g.n_orders - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.slot_off[mid] <= w) lo = mid; else hi = mid - 1;
  }
  m = lo;
}

// MAC of two complex l-vectors (interleaved re/im), FP32 accumulation; every lane
// returns the same value.
__device__ __forceinline__ float mac32(const float2* __restrict__ a, const float2* __restrict__ b,
                                       int l, int lane) {
  float dr = 0.f, di = 0.f, na = 0.f, nb = 0.f;
  for (int c = lane; c < l; c += 32) {
    const float2 x = a[c], y = b[c];
    dr = fmaf(x.x, y.x, fmaf(x.y, y.y, dr));
    di = fmaf(x.x, y.y, fmaf(-x.y, y.x, di));
    na = fmaf(x.x, x.x, fmaf(x.y, x.y, na));
    nb = fmaf(y.x, y.x, fmaf(y.y, y.y, nb));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const float den = na * nb;
  return den > 0.f ? (dr * dr + di * di) / den : 0.f;
}

// The same with FP64 accumulation (the products of FP32 inputs are exact in FP64).
__device__ __forceinline__ double mac64(const float2* __restrict__ a, const float2* __restrict__ b,
                                        int l, int lane) {
  double dr = 0.0, di = 0.0, na = 0.0, nb = 0.0;
  for (int c = lane; c < l; c += 32) {
    const float2 x = a[c], y = b[c];
    const double xr = x.x, xi = x.y, yr = y.x, yi = y.y;
    dr += xr * yr + xi * yi;
    di += xr * yi - xi * yr;
    na += xr * xr + xi * xi;
    nb += yr * yr + yi * yi;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const double den = na * nb;
  return den > 0.0 ? (dr * dr + di * di) / den : 0.0;
}

// ---------------------------------------------------------------------------------
// Stage I features
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(CL_THREADS) k_features(const ssi_pole* __restrict__ poles,
                                                         const float* __restrict__ phi, Grid g,
                                                         float E, double* __restrict__ feat,
                                                         unsigned char* __restrict__ cand,
                                                         int* __restrict__ nbr,
                                                         double* __restrict__ ndist) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long n = g.slots_per_lag * g.n_lags;
  const size_t pstride = (size_t)g.l;   // float2 per slot
  const float2* ph = reinterpret_cast<const float2*>(phi);
  for (long long e = warp0; e < n; e += nwarps) {
    const ssi_pole q = poles[e];
    const bool is_c = pole_live(q.flags) && (q.flags & (SSI_POLE_ORDER | SSI_POLE_LAG));
    if (!is_c) {
      if (lane == 0) cand[e] = 0;
      continue;
    }
    int t, m;
    slot_cell(g, e, t, m);
    long long nb_base[2];
    int nb_cnt[2];
    int nn = 0;
    if (m > 0) {
      nb_base[nn] = (long long)t * g.slots_per_lag + g.slot_off[m - 1];
      nb_cnt[nn++] = g.nslot[m - 1];
    }
    if (t > 0) {
      nb_base[nn] = (long long)(t - 1) * g.slots_per_lag + g.slot_off[m];
      nb_cnt[nn++] = g.nslot[m];
    }
    const double fq = q.f_hz, xq = q.xi;
    const float2* pq = ph + (size_t)e * pstride;
    // Pass 1 (FP32 only): the smallest screened total t32 = s32 + (1 - MAC32), which is
    // within E of the FP64 total.  Lanes take 32 neighbours at a time for the scalar
    // part; the warp then computes the MACs of the survivors in order.  A neighbour is
    // skipped only when s32 alone exceeds best32 + 3 E.
    float best32 = INFINITY;
    for (int c = 0; c < nn; ++c) {
      for (int j0 = 0; j0 < nb_cnt[c]; j0 += 32) {
        const int j = j0 + lane;
        bool ok = j < nb_cnt[c];
        float s32 = 0.f;
        if (ok) {
          const ssi_pole o = poles[nb_base[c] + j];
          ok = pole_live(o.flags);
          if (ok) {
            s32 = rel_sum32(q.f_hz, o.f_hz, q.xi, o.xi);
            ok = s32 <= best32 + 3.f * E;
          }
        }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        while (bal) {
          const int jj = __ffs(bal) - 1;
          bal &= bal - 1;
          const float sj = __shfl_sync(0xffffffffu, s32, jj);
          if (sj > best32 + 3.f * E) continue;
          const float mc = mac32(pq, ph + (size_t)(nb_base[c] + j0 + jj) * pstride, g.l, lane);
          best32 = fminf(best32, sj + (1.f - mc));
        }
      }
    }
    if (!(best32 < INFINITY)) {
      if (lane == 0) cand[e] = 0;
      continue;
    }
    // Pass 2: FP64 totals of the neighbours whose screened total lies within 2 E of
    // best32 (the FP64 minimum is among them); first minimum in scan order.
    double best = INFINITY, bf = 0.0, bx = 0.0, bm = 0.0;
    long long barg = -1;
    for (int c = 0; c < nn; ++c) {
      for (int j0 = 0; j0 < nb_cnt[c]; j0 += 32) {
        const int j = j0 + lane;
        bool ok = j < nb_cnt[c];
        float s32 = 0.f;
        if (ok) {
          const ssi_pole o = poles[nb_base[c] + j];
          ok = pole_live(o.flags);
          if (ok) {
            s32 = rel_sum32(q.f_hz, o.f_hz, q.xi, o.xi);
            ok = s32 <= best32 + 3.f * E;
          }
        }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        while (bal) {
          const int jj = __ffs(bal) - 1;
          bal &= bal - 1;
          const float sj = __shfl_sync(0xffffffffu, s32, jj);
          const long long o_e = nb_base[c] + j0 + jj;
          const float2* po = ph + (size_t)o_e * pstride;
          const float mc = mac32(pq, po, g.l, lane);
          if (sj + (1.f - mc) > best32 + 2.f * E) continue;
          const ssi_pole o = poles[o_e];
          const double dfj = rel_diff(fq, (double)o.f_hz), dxj = rel_diff(xq, (double)o.xi);
          const double dm = 1.0 - mac64(pq, po, g.l, lane);
          const double tot = (dfj + dxj) + dm;
          if (tot < best) {
            best = tot;
            bf = dfj;
            bx = dxj;
            bm = dm;
            barg = o_e;
          }
        }
      }
    }
    if (lane == 0) {
      double* x = feat + (size_t)e * 5;
      x[0] = bf;
      x[1] = bx;
      x[2] = bm;
      x[3] = 1.0 - (double)q.mpc;
      x[4] = (double)q.mpd;
      cand[e] = 1;
      nbr[e] = (int)barg;
      ndist[e] = best;
    }
  }
}

// ---------------------------------------------------------------------------------
// Stage I fuzzy C-means (cooperative)
// ---------------------------------------------------------------------------------
struct FcmParams {
  const double* feat;
  const unsigned char* cand;
  long long n;            // slots
  int n_chunks;
  int max_iter;
  double m, tol;
  double* u;              // n x 2
  double* part;           // 2 x n_chunks x FCM_STRIDE
  double* mm;             // n_chunks x FCM_STRIDE: min (5), max (5), count
  int* kcount;            // n_chunks
  double* membership;     // per slot (optional)
  int* label_out;         // per slot (optional): -1 here, kept poles relabelled later
  int* kept_slot;         // n
  int* parent;            // n
  int* slot2kept;         // n: position in the kept list, or -1
  Hdr* hdr;
  unsigned* bar;
  int* abort_flag;
  int* status;
};

__device__ bool fcm_grid_sync(const FcmParams& p, unsigned& nbar) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    nbar += 1;
    const unsigned target = nbar * gridDim.x;
    __threadfence();
    const unsigned arrived = atomicAdd(p.bar, 1u) + 1u;
    if (arrived < target) {
      const uint64_t t0 = bw::global_ns();
      while (*(volatile unsigned*)p.bar < target) {
        if (*(volatile int*)p.abort_flag) { ok = 0; break; }
        if (bw::global_ns() - t0 > CL_BAR_NS) {
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

enum RedOp { RED_SUM = 0, RED_MIN = 1, RED_MAX = 2 };

__device__ __forceinline__ double red_apply(int op, double a, double b) {
  return op == RED_SUM ? a + b : (op == RED_MIN ? fmin(a, b) : fmax(a, b));
}

// Block-wide reduction of NV values (op[k] per value) in a fixed order: a shuffle tree
// within each warp, then the warps in order.  The result is in out[0..NV) (shared).
template <int NV, int NW = CL_WARPS>
__device__ void block_reduce(double (&v)[NV], const int (&op)[NV], double* sh, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v[k] = red_apply(op[k], v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[w * NV + k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int k = threadIdx.x;
    double a = sh[k];
    for (int ww = 1; ww < NW; ++ww) a = red_apply(op[k], a, sh[ww * NV + k]);
    out[k] = a;
  }
  __syncthreads();
}

__device__ __forceinline__ double fcm_pow(double r, double e) { return e == 2.0 ? r * r : pow(r, e); }

__global__ void __launch_bounds__(FCM_THREADS) k_fcm(FcmParams p) {
  __shared__ double sh[FCM_WARPS * FCM_STRIDE];
  __shared__ double sred[FCM_NV * FCM_RED_PER];
  __shared__ double sres[FCM_STRIDE];
  __shared__ double sV[2][5];
  __shared__ double sdelta;
  __shared__ int sdone;
  __shared__ int sw[FCM_WARPS + 1];
  unsigned nbar = 0;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const double inf = INFINITY;

  // phase 0: candidate count and feature-wise min / max per chunk
  for (int c = blockIdx.x; c < p.n_chunks; c += gridDim.x) {
    double v[11];
    int op[11];
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      v[d] = inf; op[d] = RED_MIN;
      v[5 + d] = -inf; op[5 + d] = RED_MAX;
    }
    v[10] = 0.0; op[10] = RED_SUM;
    for (int r = 0; r < FCM_CH / FCM_THREADS; ++r) {
      const long long e = (long long)c * FCM_CH + r * FCM_THREADS + tid;
      if (e < p.n && p.cand[e]) {
        v[10] += 1.0;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          const double x = p.feat[e * 5 + d];
          v[d] = fmin(v[d], x);
          v[5 + d] = fmax(v[5 + d], x);
        }
      }
    }
    block_reduce<11, FCM_WARPS>(v, op, sh, sres);
    if (tid < 11) p.mm[(size_t)c * FCM_STRIDE + tid] = sres[tid];
  }
  if (!fcm_grid_sync(p, nbar)) return;
  if (tid < 11) {
    const int k = tid;
    double a = p.mm[k];
    for (int c = 1; c < p.n_chunks; ++c) {
      const double b = p.mm[(size_t)c * FCM_STRIDE + k];
      a = k < 5 ? fmin(a, b) : (k < 10 ? fmax(a, b) : a + b);
    }
    sres[k] = a;
  }
  __syncthreads();
  const int n_cand = (int)sres[10];
  if (tid < 10) sV[tid / 5][tid % 5] = sres[tid];
  __syncthreads();
  if (n_cand == 0) {
    if (blockIdx.x == 0 && tid == 0) {
      p.hdr->n_cand = 0;
      p.hdr->n_kept = 0;
      p.hdr->iters = 0;
      p.hdr->converged = 1;
      p.hdr->phys = 0;
    }
    for (long long e = (long long)blockIdx.x * FCM_THREADS + tid; e < p.n; e += (long long)gridDim.x * FCM_THREADS) {
      if (p.membership) p.membership[e] = -1.0;
      if (p.label_out) p.label_out[e] = -1;
    }
    return;
  }

  // C-means iterations
  const double e_u = 2.0 / (p.m - 1.0);
  int it = 0, converged = 0;
  for (it = 1; it <= p.max_iter; ++it) {
    double* part = p.part + (size_t)(it & 1) * p.n_chunks * FCM_STRIDE;
    for (int c = blockIdx.x; c < p.n_chunks; c += gridDim.x) {
      double v[FCM_NV];
      int op[FCM_NV];
#pragma unroll
      for (int k = 0; k < FCM_NV; ++k) { v[k] = 0.0; op[k] = RED_SUM; }
      op[FCM_NV - 1] = RED_MAX;
      for (int r = 0; r < FCM_CH / FCM_THREADS; ++r) {
        const long long e = (long long)c * FCM_CH + r * FCM_THREADS + tid;
        if (e >= p.n || !p.cand[e]) continue;
        double x[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) x[d] = p.feat[e * 5 + d];
        double dist[2];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          double s = 0.0;
#pragma unroll
          for (int d = 0; d < 5; ++d) {
            const double z = __dsub_rn(x[d], sV[cc][d]);
            s = __dadd_rn(s, __dmul_rn(z, z));
          }
          dist[cc] = sqrt(s);
        }
        double un[2];
        if (dist[0] == 0.0) {
          un[0] = 1.0; un[1] = 0.0;
        } else if (dist[1] == 0.0) {
          un[0] = 0.0; un[1] = 1.0;
        } else {
#pragma unroll
          for (int cc = 0; cc < 2; ++cc)
            un[cc] = 1.0 / (fcm_pow(dist[cc] / dist[0], e_u) + fcm_pow(dist[cc] / dist[1], e_u));
        }
        double u0 = 0.5, u1 = 0.5;
        if (it > 1) {
          u0 = p.u[e * 2];
          u1 = p.u[e * 2 + 1];
        }
        v[FCM_NV - 1] = fmax(v[FCM_NV - 1], fmax(fabs(un[0] - u0), fabs(un[1] - u1)));
        p.u[e * 2] = un[0];
        p.u[e * 2 + 1] = un[1];
        const double w0 = fcm_pow(un[0], p.m), w1 = fcm_pow(un[1], p.m);
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          v[d] += w0 * x[d];
          v[6 + d] += w1 * x[d];
        }
        v[5] += w0;
        v[11] += w1;
      }
      block_reduce<FCM_NV, FCM_WARPS>(v, op, sh, sres);
      if (tid < FCM_NV) part[(size_t)c * FCM_STRIDE + tid] = sres[tid];
    }
    if (!fcm_grid_sync(p, nbar)) return;
    // every CTA: the chunk partials in a fixed order (thread k*FCM_RED_PER + q sums
    // chunks q, q + FCM_RED_PER, ... of value k; the FCM_RED_PER sums are added in order)
    {
      const int k = tid / FCM_RED_PER, q = tid % FCM_RED_PER;
      double a = 0.0;
      if (k < FCM_NV) {
        const bool mx = (k == FCM_NV - 1);
        for (int c = q; c < p.n_chunks; c += FCM_RED_PER) {
          const double b = part[(size_t)c * FCM_STRIDE + k];
          a = mx ? fmax(a, b) : a + b;
        }
        sred[tid] = a;
      }
      __syncthreads();
      if (tid < FCM_NV) {
        const bool mx = (tid == FCM_NV - 1);
        double s = sred[tid * FCM_RED_PER];
        for (int qq = 1; qq < FCM_RED_PER; ++qq) {
          const double b = sred[tid * FCM_RED_PER + qq];
          s = mx ? fmax(s, b) : s + b;
        }
        sres[tid] = s;
      }
      __syncthreads();
      if (tid < 10) {
        // a cluster whose memberships are all zero keeps its centroid (the update is 0/0)
        const int cc = tid / 5, d = tid % 5;
        if (sres[cc * 6 + 5] > 0.0) sV[cc][d] = sres[cc * 6 + d] / sres[cc * 6 + 5];
      }
      if (tid == 0) {
        sdelta = sres[FCM_NV - 1];
        sdone = sdelta < p.tol;
      }
      __syncthreads();
    }
    if (sdone) {
      converged = 1;
      break;
    }
  }
  if (it > p.max_iter) it = p.max_iter;
  // the physical cluster: the centroid nearer the origin (ties to the first)
  double nrm[2];
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 5; ++d) s = __dadd_rn(s, __dmul_rn(sV[cc][d], sV[cc][d]));
    nrm[cc] = sqrt(s);
  }
  const int phys = nrm[1] < nrm[0] ? 1 : 0;

  // kept poles: per-chunk counts, then the ordered list
  for (int c = blockIdx.x; c < p.n_chunks; c += gridDim.x) {
    int cnt = 0;
    for (int r = 0; r < FCM_CH / FCM_THREADS; ++r) {
      const long long e = (long long)c * FCM_CH + r * FCM_THREADS + tid;
      if (e < p.n && p.cand[e] && p.u[e * 2 + phys] >= 0.5) ++cnt;
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) sw[wid] = cnt;
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int w = 0; w < FCM_WARPS; ++w) s += sw[w];
      p.kcount[c] = s;
    }
    __syncthreads();
  }
  if (!fcm_grid_sync(p, nbar)) return;
  for (int c = blockIdx.x; c < p.n_chunks; c += gridDim.x) {
    // kept poles of the chunks before this one (integer sum: any order)
    int before = 0;
    for (int cc = tid; cc < c; cc += FCM_THREADS) before += p.kcount[cc];
    for (int o = 16; o; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    if (lane == 0) sw[wid] = before;
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int w = 0; w < FCM_WARPS; ++w) s += sw[w];
      sw[FCM_WARPS] = s;
    }
    __syncthreads();
    int base = sw[FCM_WARPS];
    __syncthreads();
    for (int r = 0; r < FCM_CH / FCM_THREADS; ++r) {
      const long long e = (long long)c * FCM_CH + r * FCM_THREADS + tid;
      const bool in = e < p.n;
      const bool is_c = in && p.cand[e];
      const double P = is_c ? p.u[e * 2 + phys] : -1.0;
      const bool keep = is_c && P >= 0.5;
      if (in && p.membership) p.membership[e] = P;
      if (in && p.label_out) p.label_out[e] = -1;
      if (in && !keep) p.slot2kept[e] = -1;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) sw[wid] = __popc(bal);
      __syncthreads();
      int off = base;
      for (int w = 0; w < wid; ++w) off += sw[w];
      int tot = 0;
      for (int w = 0; w < FCM_WARPS; ++w) tot += sw[w];
      if (keep) {
        const int pos = off + __popc(bal & ((1u << lane) - 1u));
        p.kept_slot[pos] = (int)e;
        p.parent[pos] = pos;
        p.slot2kept[e] = pos;
      }
      base += tot;
      __syncthreads();
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    int nk = 0;
    for (int c = 0; c < p.n_chunks; ++c) nk += p.kcount[c];
    p.hdr->n_cand = n_cand;
    p.hdr->n_kept = nk;
    p.hdr->iters = it;
    p.hdr->converged = converged;
    p.hdr->phys = phys;
    for (int cc = 0; cc < 2; ++cc)
      for (int d = 0; d < 5; ++d) p.hdr->V[cc][d] = sV[cc][d];
  }
}

// ---------------------------------------------------------------------------------
// Stage II: single linkage as connected components
// ---------------------------------------------------------------------------------
// Every parent index is <= its child's, so a root is the smallest index of its tree.
// Only non-roots are shortened (to an ancestor), so a concurrent hook is never undone.
__device__ __forceinline__ int uf_find(int* parent, int x) {
  volatile int* pv = parent;
  int cur = pv[x];
  if (cur != x) {
    int prev = x, next;
    while (cur > (next = pv[cur])) {
      pv[prev] = next;
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

__device__ void uf_union(int* parent, int a, int b, int* status) {
  int ra = uf_find(parent, a), rb = uf_find(parent, b);
  for (int guard = 0; ra != rb; ++guard) {
    if (guard >= UNION_LIMIT) {
      atomicOr(status, DEV_TIMEOUT);
      return;
    }
    if (ra < rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    // hook the larger root under the smaller one
    const int old = atomicCAS(&parent[ra], ra, rb);
    if (old == ra) return;
    ra = uf_find(parent, old);
    rb = uf_find(parent, rb);
  }
}

struct LinkParams {
  const ssi_pole* poles;
  const float2* phi;
  int l;
  const int* kept_slot;
  const int* n_kept;     // device
  int* parent;
  double tau, eps;
  float tau32;           // FP32 screen of d_f + d_xi <= tau
  float tau_lo, tau_hi;  // FP32 distances <= tau_lo link, > tau_hi do not
  long long n_tiles;
  int nb;                // tiles per side
  int* status;
};

__device__ __forceinline__ void tile_rc(long long t, int nb, int& bi, int& bj) {
  // row bi holds tiles (bi, bi..nb-1); start(bi) = bi*nb - bi*(bi-1)/2
  const double B = 2.0 * nb + 1.0;
  int r = (int)((B - sqrt(fmax(B * B - 8.0 * (double)t, 0.0))) * 0.5);
  r = max(0, min(r, nb - 1));
  auto start = [nb](long long b) { return b * nb - b * (b - 1) / 2; };
  while (r > 0 && start(r) > t) --r;
  while (r + 1 < nb && start(r + 1) <= t) ++r;
  bi = r;
  bj = (int)(r + (t - start(r)));
}

__global__ void __launch_bounds__(CL_THREADS) k_link(LinkParams p) {
  __shared__ int s_slot[2][32];
  __shared__ float s_f[2][32], s_x[2][32];
  __shared__ int s_tile[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nk = *p.n_kept;
  for (long long t = blockIdx.x; t < p.n_tiles; t += gridDim.x) {
    // one thread maps the tile index (an FP64 square root) for the block
    if (threadIdx.x == 0) tile_rc(t, p.nb, s_tile[0], s_tile[1]);
    __syncthreads();
    const int bi = s_tile[0], bj = s_tile[1];
    if (threadIdx.x < 64) {
      const int side = threadIdx.x >> 5, k = threadIdx.x & 31;
      const int idx = (side ? bj : bi) * 32 + k;
      if (idx < nk) {
        const int e = p.kept_slot[idx];
        s_slot[side][k] = e;
        s_f[side][k] = p.poles[e].f_hz;
        s_x[side][k] = p.poles[e].xi;
      } else {
        s_slot[side][k] = -1;
      }
    }
    __syncthreads();
    const int b = bj * 32 + lane;
    for (int rr = 0; rr < 4; ++rr) {
      const int ar = wid * 4 + rr;
      const int a = bi * 32 + ar;
      if (a >= nk) break;                         // warp-uniform
      bool need = b < nk && b > a;
      float s = 0.f;
      if (need) {
        s = rel_sum32(s_f[0][ar], s_f[1][lane], s_x[0][ar], s_x[1][lane]);
        need = s <= p.tau32;
        // already connected: nothing to decide (each lane looks up its own pair)
        if (need) need = uf_find(p.parent, a) != uf_find(p.parent, b);
      }
      unsigned bal = __ballot_sync(0xffffffffu, need);
      while (bal) {
        const int j = __ffs(bal) - 1;
        bal &= bal - 1;
        const float sj = __shfl_sync(0xffffffffu, s, j);
        const int bb = bj * 32 + j;
        const float2* pa = p.phi + (size_t)s_slot[0][ar] * p.l;
        const float2* pb = p.phi + (size_t)s_slot[1][j] * p.l;
        const float d32 = sj + (1.f - mac32(pa, pb, p.l, lane));
        bool link = d32 <= p.tau_lo;
        if (!link && d32 <= p.tau_hi) {
          // inconclusive in FP32: the FP64 distance decides
          const double s64 = rel_diff(s_f[0][ar], s_f[1][j]) + rel_diff(s_x[0][ar], s_x[1][j]);
          link = s64 + (1.0 - mac64(pa, pb, p.l, lane)) <= p.tau;
        }
        if (link && lane == 0) uf_union(p.parent, a, bb, p.status);
      }
    }
  }
}

// Stage I already found each candidate's nearest neighbour and its FP64 distance (the
// Stage II metric): kept pairs within tau are joined first, which connects most of each
// mode's poles at linear cost.  Then every pole points at its root.
__global__ void k_prelink(const int* __restrict__ kept_slot, const int* __restrict__ n_kept,
                          const int* __restrict__ nbr, const double* __restrict__ ndist,
                          const int* __restrict__ slot2kept, double tau, int* parent, int* status) {
  const int nk = *n_kept;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
    const int e = kept_slot[i];
    if (!(ndist[e] <= tau)) continue;
    const int j = slot2kept[nbr[e]];
    if (j >= 0) uf_union(parent, i, j, status);
  }
}

__global__ void k_compress(int* parent, const int* __restrict__ n_kept) {
  const int nk = *n_kept;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
    const int r = uf_find(parent, i);
    parent[i] = r;
  }
}

__global__ void k_relabel(const int* __restrict__ kept_slot, const int* __restrict__ lab,
                          const int* __restrict__ n_kept, int32_t* __restrict__ label) {
  const int nk = *n_kept;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x)
    label[kept_slot[i]] = kept_slot[lab[i]];
}

__global__ void k_label(int* parent, const int* __restrict__ n_kept, int* __restrict__ lab,
                        int* __restrict__ size) {
  const int nk = *n_kept;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
    const int r = uf_find(parent, i);
    lab[i] = r;
    atomicAdd(&size[r], 1);
  }
}

// One CTA: components in index order; those of >= min_size poles become modes.
__global__ void __launch_bounds__(SCAN_THREADS) k_modes_scan(const int* __restrict__ lab,
                                                             const int* __restrict__ size,
                                                             int min_size, Hdr* hdr,
                                                             int* __restrict__ mode_root,
                                                             int* __restrict__ mode_off) {
  __shared__ int sw[2][SCAN_THREADS / 32];
  __shared__ int s_base[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = SCAN_THREADS / 32;
  const int nk = hdr->n_kept;
  if (threadIdx.x == 0) {
    s_base[0] = 0;
    s_base[1] = 0;
  }
  int n_comp = 0;
  __syncthreads();
  for (int i0 = 0; i0 < nk; i0 += SCAN_THREADS) {
    const int i = i0 + threadIdx.x;
    const bool root = i < nk && lab[i] == i;
    const int sz = root ? size[i] : 0;
    const bool mode = root && sz >= min_size;
    const unsigned bm = __ballot_sync(0xffffffffu, mode);
    const unsigned br = __ballot_sync(0xffffffffu, root);
    // sizes of the modes before this thread (warp inclusive scan)
    int ssz = mode ? sz : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ssz, o);
      if (lane >= o) ssz += y;
    }
    if (lane == 31) {
      sw[0][wid] = __popc(bm);
      sw[1][wid] = ssz;
    }
    __syncthreads();
    int mb = s_base[0], sb = s_base[1];
    for (int w = 0; w < wid; ++w) {
      mb += sw[0][w];
      sb += sw[1][w];
    }
    if (mode) {
      const int id = mb + __popc(bm & ((1u << lane) - 1u));
      mode_root[id] = i;
      mode_off[id] = sb + ssz - sz;
    }
    if (lane == 0) n_comp += __popc(br);
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < nw; ++w) {
        s_base[0] += sw[0][w];
        s_base[1] += sw[1][w];
      }
    }
    __syncthreads();
  }
  // components: sum of the per-warp counts
  for (int o = 16; o; o >>= 1) n_comp += __shfl_xor_sync(0xffffffffu, n_comp, o);
  __shared__ int s_comp[SCAN_THREADS / 32];
  if (lane == 0) s_comp[wid] = n_comp;
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < nw; ++w) c += s_comp[w];
    hdr->n_comp = c;
    hdr->n_modes = s_base[0];
    mode_off[s_base[0]] = s_base[1];
  }
}

// One CTA per mode: members in index order; mean f and xi (fixed-order sums).
__global__ void __launch_bounds__(CL_THREADS) k_mode_members(
    const ssi_pole* __restrict__ poles, const int* __restrict__ kept_slot,
    const int* __restrict__ lab, const Hdr* __restrict__ hdr, const int* __restrict__ mode_root,
    const int* __restrict__ mode_off, int* __restrict__ members, int* __restrict__ member_mode,
    double* __restrict__ mode_fx) {
  __shared__ int sw[CL_WARPS];
  __shared__ double sh[CL_WARPS * 2];
  __shared__ double sres[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int md = blockIdx.x;
  const int root = mode_root[md];
  const int nk = hdr->n_kept;
  int base = mode_off[md];
  double sf = 0.0, sx = 0.0;
  for (int i0 = root; i0 < nk; i0 += CL_THREADS) {
    const int i = i0 + threadIdx.x;
    const bool mem = i < nk && lab[i] == root;
    const unsigned bal = __ballot_sync(0xffffffffu, mem);
    if (lane == 0) sw[wid] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int w = 0; w < wid; ++w) off += sw[w];
    int tot = 0;
    for (int w = 0; w < CL_WARPS; ++w) tot += sw[w];
    if (mem) {
      const int pos = off + __popc(bal & ((1u << lane) - 1u));
      members[pos] = i;
      member_mode[pos] = md;
      const ssi_pole q = poles[kept_slot[i]];
      sf += (double)q.f_hz;
      sx += (double)q.xi;
    }
    base += tot;
    __syncthreads();
  }
  double v[2] = {sf, sx};
  const int op[2] = {RED_SUM, RED_SUM};
  block_reduce<2>(v, op, sh, sres);
  if (threadIdx.x == 0) {
    const double cnt = (double)(mode_off[md + 1] - mode_off[md]);
    mode_fx[md * 2] = sres[0] / cnt;
    mode_fx[md * 2 + 1] = sres[1] / cnt;
  }
}

struct MedoidParams {
  const ssi_pole* poles;
  const float2* phi;
  int l;
  const int* kept_slot;
  const int* members;
  const int* member_mode;
  const int* mode_off;
  int n_members;
  double* inv;        // per member: 1/f, 1/xi, 1/|phi|^2 (FP64)
  double* sum;        // per member: sum of distances to the other members
  int* medoid;        // per mode: slot of the medoid
};

// Error-free transformations in FP32 (Knuth's two-sum; the product split by an FMA).
// Intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
// (hi, lo) += a * b
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  float s, e;
  two_sum(hi, p, s, e);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
// One warp per member: 1/f, 1/xi and 1/|phi|^2 in FP64 (exact products, FP64 sum).
__global__ void __launch_bounds__(CL_THREADS) k_medoid_prep(MedoidParams p) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long q = warp0; q < p.n_members; q += nwarps) {
    const int e = p.kept_slot[p.members[q]];
    const float2* pa = p.phi + (size_t)e * p.l;
    double na = 0.0;
    for (int c = lane; c < p.l; c += 32) {
      const float2 x = pa[c];
      na += (double)x.x * x.x + (double)x.y * x.y;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) na += __shfl_xor_sync(0xffffffffu, na, o);
    if (lane == 0) {
      const ssi_pole qa = p.poles[e];
      p.inv[q * 3] = 1.0 / (double)qa.f_hz;
      p.inv[q * 3 + 1] = 1.0 / (double)qa.xi;
      p.inv[q * 3 + 2] = na > 0.0 ? 1.0 / na : 0.0;
    }
  }
}

// (hi, lo) summed over the warp (butterfly: every lane gets the total)
__device__ __forceinline__ void df_warp_allsum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(l2, e));
  }
}

// Each pair of a mode once.  A work item is a tile pair (ti <= tj) of 32 x 32 members of
// one mode; warp w takes rows 4w..4w+3 of the tile, and for each row the 32 partners'
// cross products (double-float, lanes over channels; lane j keeps partner j's), then the
// 32 distances in FP64 side by side.  A row's sum over the tile goes to P[a][tj], a
// column's sum over the tile (from shared memory, rows in order) to P[b][ti]; on a
// diagonal tile, pairs a < b only, and member x gets its row and column sums together in
// P[x][ti].  Every (member, tile) entry of P is written once, so sum[a] = sum over t of
// P[a][t] in t order is deterministic.
struct MedoidTiles {
  const int4* items;        // (mode, ti, tj, 0)
  int n_items;
  const long long* pbase;   // per mode: first entry of its P block (members x tiles)
  double* P;
};

__global__ void __launch_bounds__(CL_THREADS) k_medoid_tiles(MedoidParams p, MedoidTiles mt) {
  __shared__ double s_col[32][33];
  __shared__ double s_row[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int item = blockIdx.x; item < mt.n_items; item += gridDim.x) {
    const int4 it = mt.items[item];
    const int md = it.x, ti = it.y, tj = it.z;
    const int b0 = p.mode_off[md], sm = p.mode_off[md + 1] - b0;
    const int nt = (sm + 31) / 32;
    const bool diag = ti == tj;
    double* P = mt.P + mt.pbase[md];
    __syncthreads();
    for (int rr = 0; rr < 4; ++rr) {
      const int r = wid * 4 + rr;
      const int ra = ti * 32 + r;                  // member index within the mode
      double d = 0.0;
      if (ra < sm) {                               // warp-uniform
        const int qa = b0 + ra;
        const int ea = p.kept_slot[p.members[qa]];
        const float2* pa = p.phi + (size_t)ea * p.l;
        float kr_h = 0.f, kr_l = 0.f, ki_h = 0.f, ki_l = 0.f;
        for (int jj = 0; jj < 32; ++jj) {
          const int cb = tj * 32 + jj;
          if (cb >= sm || (diag && cb <= ra)) continue;   // warp-uniform
          const float2* pb = p.phi + (size_t)p.kept_slot[p.members[b0 + cb]] * p.l;
          float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
          for (int c = lane; c < p.l; c += 32) {
            const float2 x = pa[c], y = pb[c];
            df_fma(rh, rl, x.x, y.x);
            df_fma(rh, rl, x.y, y.y);
            df_fma(ih, il, x.x, y.y);
            df_fma(ih, il, -x.y, y.x);
          }
          df_warp_allsum(rh, rl);
          df_warp_allsum(ih, il);
          if (lane == jj) {
            kr_h = rh; kr_l = rl; ki_h = ih; ki_l = il;
          }
        }
        const int cb = tj * 32 + lane;
        if (cb < sm && !(diag && cb <= ra)) {
          const int qb = b0 + cb;
          const ssi_pole pola = p.poles[ea];
          const ssi_pole polb = p.poles[p.kept_slot[p.members[qb]]];
          const double dr = (double)kr_h + (double)kr_l, di = (double)ki_h + (double)ki_l;
          const double sdist =
              fabs((double)pola.f_hz - (double)polb.f_hz) * fmin(p.inv[qa * 3], p.inv[qb * 3]) +
              fabs((double)pola.xi - (double)polb.xi) * fmin(p.inv[qa * 3 + 1], p.inv[qb * 3 + 1]);
          const double mac = (dr * dr + di * di) * p.inv[qa * 3 + 2] * p.inv[qb * 3 + 2];
          d = sdist + (1.0 - mac);
        }
      }
      s_col[r][lane] = d;
      double rs = d;
#pragma unroll
      for (int o = 16; o; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
      if (lane == 0) {
        if (diag) s_row[r] = rs;
        else if (ra < sm) P[(long long)ra * nt + tj] = rs;
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int c = threadIdx.x;
      const int cb = tj * 32 + c;
      if (cb < sm) {
        double cs = 0.0;
        for (int r = 0; r < 32; ++r) cs += s_col[r][c];
        P[(long long)cb * nt + ti] = diag ? s_row[c] + cs : cs;
      }
    }
  }
}

// One thread per member: its sum over the tiles of its mode, in tile order.
__global__ void k_medoid_finish(MedoidParams p, MedoidTiles mt) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < p.n_members;
       q += (long long)gridDim.x * blockDim.x) {
    const int md = p.member_mode[q];
    const int b0 = p.mode_off[md], sm = p.mode_off[md + 1] - b0;
    const int nt = (sm + 31) / 32;
    const double* P = mt.P + mt.pbase[md] + (long long)(q - b0) * nt;
    double sum = 0.0;
    for (int t = 0; t < nt; ++t) sum += P[t];
    p.sum[q] = sum;
  }
}

// One CTA per mode: the member with the smallest sum, ties to the earlier one.
__global__ void __launch_bounds__(CL_THREADS) k_medoid_pick(MedoidParams p) {
  __shared__ double s_val[CL_WARPS];
  __shared__ int s_arg[CL_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int md = blockIdx.x;
  const int b0 = p.mode_off[md], b1 = p.mode_off[md + 1];
  double best = INFINITY;
  int arg = 0x7fffffff;
  for (int q = b0 + threadIdx.x; q < b1; q += CL_THREADS) {
    const double v = p.sum[q];
    if (v < best) {            // q ascends within the thread
      best = v;
      arg = q;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int a2 = __shfl_xor_sync(0xffffffffu, arg, o);
    if (v2 < best || (v2 == best && a2 < arg)) {
      best = v2;
      arg = a2;
    }
  }
  if (lane == 0) {
    s_val[wid] = best;
    s_arg[wid] = arg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bv = INFINITY;
    int ba = 0x7fffffff;
    for (int w = 0; w < CL_WARPS; ++w) {
      if (s_val[w] < bv || (s_val[w] == bv && s_arg[w] < ba)) {
        bv = s_val[w];
        ba = s_arg[w];
      }
    }
    p.medoid[md] = p.kept_slot[p.members[ba < b1 ? ba : b0]];
  }
}

}  // namespace

namespace {

double mac_screen_eps(int l) {
  const double u = std::ldexp(1.0, -24);
  const double gamma = (2.0 * (double)((l + 31) / 32) + 5.0) * u;
  return 2.0 * (5.0 * gamma + 4.0 * u);
}

}  // namespace

ssi_status cluster_run(ssi_ctx* ctx, int n_lags, int n_orders, const int* orders, int l,
                       const ssi_pole* poles, const float* phi, const ssi_cluster_params* cp,
                       ssi_mode* modes, int max_modes, int* n_modes_out, double* features,
                       double* membership, int32_t* label, ssi_cluster_info* info,
                       cudaStream_t stream) {
  Grid g{};
  g.n_lags = n_lags;
  g.n_orders = n_orders;
  g.l = l;
  long long so = 0;
  for (int m = 0; m < n_orders; ++m) {
    g.slot_off[m] = so;
    g.nslot[m] = orders[m] / 2;
    so += orders[m] / 2;
  }
  g.slots_per_lag = so;
  const long long n = so * n_lags;
  SSI_CHECK(n <= (1ll << 30), "ssi_cluster: too many pole slots");
  const int n_chunks = (int)ceil_div(n, FCM_CH);
  const double eps = mac_screen_eps(l);
  // bound on |t32 - t64| for a screened distance t = d_f + d_xi + (1 - MAC): the MAC
  // bound plus the FP32 rounding of d_f + d_xi (<= 2, 3 ulp) and of the final sum
  const float E32 = (float)(eps + 1e-6);

  // workspace
  WsPlan wp;
  if (!features) wp.add<double>((size_t)n * 5);
  wp.add<unsigned char>((size_t)n);
  wp.add<double>((size_t)n * 2);
  wp.add<double>((size_t)2 * n_chunks * FCM_STRIDE);
  wp.add<double>((size_t)n_chunks * FCM_STRIDE);
  wp.add<int>((size_t)n_chunks);
  for (int k = 0; k < 7; ++k) wp.add<int>((size_t)n + 1);   // kept, parent, lab, size, roots, offsets, members
  wp.add<int>((size_t)n + 1);                               // member_mode
  wp.add<double>((size_t)n * 2);                            // mode f / xi
  wp.add<double>((size_t)n * 4);                            // medoid reciprocals, sums
  wp.add<int>((size_t)n + 1);                               // medoid
  wp.add<int>((size_t)n);                                   // nearest neighbour
  wp.add<double>((size_t)n);                                // its distance
  wp.add<int>((size_t)n);                                   // slot -> kept index
  wp.add<Hdr>(1);
  wp.add<unsigned>(64);
  SSI_TRY(ws_reserve(ctx, ctx->ws, wp.bytes, stream));
  Workspace& ws = ctx->ws;
  ws.reset();
  double* feat = features ? features : ws.take<double>((size_t)n * 5);
  unsigned char* cand = ws.take<unsigned char>((size_t)n);
  double* u = ws.take<double>((size_t)n * 2);
  double* part = ws.take<double>((size_t)2 * n_chunks * FCM_STRIDE);
  double* mm = ws.take<double>((size_t)n_chunks * FCM_STRIDE);
  int* kcount = ws.take<int>((size_t)n_chunks);
  int* kept = ws.take<int>((size_t)n + 1);
  int* parent = ws.take<int>((size_t)n + 1);
  int* lab = ws.take<int>((size_t)n + 1);
  int* csize = ws.take<int>((size_t)n + 1);
  int* mode_root = ws.take<int>((size_t)n + 1);
  int* mode_off = ws.take<int>((size_t)n + 1);
  int* members = ws.take<int>((size_t)n + 1);
  int* member_mode = ws.take<int>((size_t)n + 1);
  double* mode_fx = ws.take<double>((size_t)n * 2);
  double* sums = ws.take<double>((size_t)n * 4);
  int* medoid = ws.take<int>((size_t)n + 1);
  int* nbr = ws.take<int>((size_t)n);
  double* ndist = ws.take<double>((size_t)n);
  int* slot2kept = ws.take<int>((size_t)n);
  Hdr* hdr = ws.take<Hdr>(1);
  unsigned* bar = ws.take<unsigned>(64);
  if (!feat || !cand || !u || !part || !mm || !kcount || !kept || !parent || !lab || !csize ||
      !mode_root || !mode_off || !members || !member_mode || !mode_fx || !sums || !medoid || !hdr ||
      !bar || !nbr || !ndist || !slot2kept) {
    set_error("ssi_cluster: workspace too small");
    return SSI_E_NOMEM;
  }
  ProfScope ps(ctx, ST_CLUSTER, stream);

  // Stage I features
  if (features) SSI_CUDA(cudaMemsetAsync(features, 0, sizeof(double) * (size_t)n * 5, stream));
  {
    const int blocks = (int)std::min<long long>(ceil_div(n * 32, CL_THREADS), (long long)ctx->num_sms * 16);
    count_launches(ctx, 1);
    k_features<<<std::max(blocks, 1), CL_THREADS, 0, stream>>>(poles, phi, g, E32, feat, cand, nbr,
                                                               ndist);
    SSI_CUDA(cudaGetLastError());
  }
  // Stage I C-means and the kept list
  SSI_CUDA(cudaMemsetAsync(bar, 0, 64 * sizeof(unsigned), stream));
  SSI_CUDA(cudaMemsetAsync(hdr, 0, sizeof(Hdr), stream));
  {
    FcmParams fp{};
    fp.feat = feat;
    fp.cand = cand;
    fp.n = n;
    fp.n_chunks = n_chunks;
    fp.max_iter = cp->fcm_max_iter;
    fp.m = cp->fcm_m;
    fp.tol = cp->fcm_tol;
    fp.u = u;
    fp.part = part;
    fp.mm = mm;
    fp.kcount = kcount;
    fp.membership = membership;
    fp.label_out = label;
    fp.kept_slot = kept;
    fp.parent = parent;
    fp.slot2kept = slot2kept;
    fp.hdr = hdr;
    fp.bar = bar;
    fp.abort_flag = reinterpret_cast<int*>(bar + 8);
    fp.status = ctx->dev_status;
    // every chunk its own CTA where they fit at once (the cooperative launch needs all CTAs
    // resident); solves sharing the device get their share of it
    int occ = 0;
    SSI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fcm, FCM_THREADS, 0));
    const int inflight = std::max(1, ctx->inflight.load());
    const int resident = std::max(1, ctx->num_sms * std::max(1, occ) / inflight);
    const int grid = std::max(1, std::min(n_chunks, resident));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(FCM_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launches(ctx, 1);
    SSI_CUDA(cudaLaunchKernelEx(&cfg, k_fcm, fp));
  }
  Hdr h{};
  SSI_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, stream));
  SSI_TRY(check_dev_status(ctx->dev_status, stream));
  const int nk = h.n_kept;
  int n_modes = 0;
  std::vector<int> med;
  std::vector<double> fx;
  std::vector<int> off;
  if (nk > 0) {
    // Stage II: links, components, modes
    const int nb = (int)ceil_div(nk, 32);
    LinkParams lp{};
    lp.poles = poles;
    lp.phi = reinterpret_cast<const float2*>(phi);
    lp.l = l;
    lp.kept_slot = kept;
    lp.n_kept = &hdr->n_kept;
    lp.parent = parent;
    lp.tau = cp->tau;
    lp.eps = eps;
    lp.tau32 = std::nextafter((float)((cp->tau + 1e-12) / (1.0 - 1e-6)), INFINITY);
    lp.tau_lo = std::nextafter((float)(cp->tau - 2.0 * E32), -INFINITY);
    lp.tau_hi = std::nextafter((float)(cp->tau + 2.0 * E32), INFINITY);
    lp.nb = nb;
    lp.n_tiles = (long long)nb * (nb + 1) / 2;
    lp.status = ctx->dev_status;
    const int lblocks = (int)std::min<long long>(lp.n_tiles, (long long)ctx->num_sms * 8);
    SSI_CUDA(cudaMemsetAsync(csize, 0, sizeof(int) * (size_t)nk, stream));
    const int pb = (int)std::min<long long>(ceil_div(nk, 256), (long long)ctx->num_sms * 4);
    count_launches(ctx, 5);
    k_prelink<<<pb, 256, 0, stream>>>(kept, &hdr->n_kept, nbr, ndist, slot2kept, cp->tau, parent,
                                      ctx->dev_status);
    SSI_CUDA(cudaGetLastError());
    k_compress<<<pb, 256, 0, stream>>>(parent, &hdr->n_kept);
    SSI_CUDA(cudaGetLastError());
    k_link<<<lblocks, CL_THREADS, 0, stream>>>(lp);
    SSI_CUDA(cudaGetLastError());
    const int lb = (int)std::min<long long>(ceil_div(nk, 256), (long long)ctx->num_sms * 4);
    k_label<<<lb, 256, 0, stream>>>(parent, &hdr->n_kept, lab, csize);
    SSI_CUDA(cudaGetLastError());
    k_modes_scan<<<1, SCAN_THREADS, 0, stream>>>(lab, csize, cp->min_size, hdr, mode_root, mode_off);
    SSI_CUDA(cudaGetLastError());
    SSI_CUDA(cudaMemcpyAsync(&h, hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, stream));
    SSI_CUDA(cudaStreamSynchronize(stream));
    n_modes = h.n_modes;
    if (n_modes > 0) {
      count_launches(ctx, 3);
      k_mode_members<<<n_modes, CL_THREADS, 0, stream>>>(poles, kept, lab, hdr, mode_root, mode_off,
                                                         members, member_mode, mode_fx);
      SSI_CUDA(cudaGetLastError());
      off.resize(n_modes + 1);
      SSI_CUDA(cudaMemcpyAsync(off.data(), mode_off, sizeof(int) * (n_modes + 1),
                               cudaMemcpyDeviceToHost, stream));
      SSI_CUDA(cudaStreamSynchronize(stream));
      MedoidParams mp{};
      mp.poles = poles;
      mp.phi = reinterpret_cast<const float2*>(phi);
      mp.l = l;
      mp.kept_slot = kept;
      mp.members = members;
      mp.member_mode = member_mode;
      mp.mode_off = mode_off;
      mp.n_members = off[n_modes];
      mp.inv = sums;
      mp.sum = sums + (size_t)3 * n;
      mp.medoid = medoid;
      const int mblocks = (int)std::min<long long>(ceil_div((long long)mp.n_members * 32, CL_THREADS),
                                                   (long long)ctx->num_sms * 16);
      count_launches(ctx, 1);
      k_medoid_prep<<<std::max(mblocks, 1), CL_THREADS, 0, stream>>>(mp);
      SSI_CUDA(cudaGetLastError());
      // tile pairs of every mode, and each mode's block of per-(member, tile) partials
      std::vector<int4> items;
      std::vector<long long> pbase(n_modes);
      long long ptot = 0;
      for (int md = 0; md < n_modes; ++md) {
        const int sm = off[md + 1] - off[md];
        const int nt = (sm + 31) / 32;
        pbase[md] = ptot;
        ptot += (long long)sm * nt;
        for (int ti = 0; ti < nt; ++ti)
          for (int tj = ti; tj < nt; ++tj) items.push_back(make_int4(md, ti, tj, 0));
      }
      WsPlan tp;
      tp.add<int4>(items.size());
      tp.add<long long>((size_t)n_modes);
      tp.add<double>((size_t)ptot);
      SSI_TRY(ws_reserve(ctx, ctx->ws_aux, tp.bytes, stream));
      ctx->ws_aux.reset();
      MedoidTiles mt{};
      int4* d_items = ctx->ws_aux.take<int4>(items.size());
      long long* d_pbase = ctx->ws_aux.take<long long>((size_t)n_modes);
      mt.P = ctx->ws_aux.take<double>((size_t)ptot);
      if (!d_items || !d_pbase || !mt.P) {
        set_error("ssi_cluster: medoid workspace too small");
        return SSI_E_NOMEM;
      }
      SSI_CUDA(cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(),
                               cudaMemcpyHostToDevice, stream));
      SSI_CUDA(cudaMemcpyAsync(d_pbase, pbase.data(), sizeof(long long) * n_modes,
                               cudaMemcpyHostToDevice, stream));
      mt.items = d_items;
      mt.n_items = (int)items.size();
      mt.pbase = d_pbase;
      const int tblocks = (int)std::min<long long>((long long)items.size(), (long long)ctx->num_sms * 8);
      count_launches(ctx, 1);
      k_medoid_tiles<<<std::max(tblocks, 1), CL_THREADS, 0, stream>>>(mp, mt);
      SSI_CUDA(cudaGetLastError());
      k_medoid_finish<<<(int)std::min<long long>(ceil_div(mp.n_members, 256), (long long)ctx->num_sms * 4),
                        256, 0, stream>>>(mp, mt);
      SSI_CUDA(cudaGetLastError());
      // the host vectors above must outlive the copies
      SSI_CUDA(cudaStreamSynchronize(stream));
      k_medoid_pick<<<n_modes, CL_THREADS, 0, stream>>>(mp);
      SSI_CUDA(cudaGetLastError());
      med.resize(n_modes);
      fx.resize((size_t)n_modes * 2);
      SSI_CUDA(cudaMemcpyAsync(med.data(), medoid, sizeof(int) * n_modes, cudaMemcpyDeviceToHost, stream));
      SSI_CUDA(cudaMemcpyAsync(fx.data(), mode_fx, sizeof(double) * 2 * n_modes,
                               cudaMemcpyDeviceToHost, stream));
      SSI_CUDA(cudaStreamSynchronize(stream));
    }
    if (label) {
      // kept poles: the slot of the first pole of their component
      count_launches(ctx, 1);
      const int kb = (int)std::min<long long>(ceil_div(nk, 256), (long long)ctx->num_sms * 4);
      k_relabel<<<kb, 256, 0, stream>>>(kept, lab, &hdr->n_kept, label);
      SSI_CUDA(cudaGetLastError());
    }
  }
  // modes sorted by mean frequency (stable: component order on ties)
  std::vector<int> ord(n_modes);
  for (int i = 0; i < n_modes; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fx[2 * a] < fx[2 * b]; });
  for (int i = 0; i < n_modes && i < max_modes; ++i) {
    const int md = ord[i];
    modes[i].f_hz = fx[2 * md];
    modes[i].xi = fx[2 * md + 1];
    modes[i].size = off[md + 1] - off[md];
    modes[i].medoid_slot = med[md];
  }
  if (n_modes_out) *n_modes_out = n_modes;
  if (info) {
    info->n_candidates = h.n_cand;
    info->n_kept = h.n_kept;
    info->n_components = nk > 0 ? h.n_comp : 0;
    info->n_modes = n_modes;
    info->fcm_iterations = h.iters;
    info->fcm_converged = h.converged;
    info->physical = h.phys;
    info->reserved = 0;
    for (int c = 0; c < 2; ++c)
      for (int d = 0; d < 5; ++d) info->centroids[c][d] = h.V[c][d];
  }
  return check_dev_status(ctx->dev_status, stream);
}

}  // namespace ssi

extern "C" ssi_status ssi_cluster(ssi_ctx* ctx, int n_lags, int n_orders, const int* orders, int l,
                                  const ssi_pole* poles, const float* phi,
                                  const ssi_cluster_params* params, ssi_mode* modes, int max_modes,
                                  int* n_modes, double* features, double* membership,
                                  int32_t* label, ssi_cluster_info* info, void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && orders && poles && phi && params && n_modes, "ssi_cluster: null pointer");
  SSI_CHECK(max_modes >= 0 && (modes || max_modes == 0), "ssi_cluster: bad modes buffer");
  SSI_CHECK(n_lags >= 1 && l >= 1 && l <= 4096, "ssi_cluster: bad n_lags / l");
  SSI_CHECK(n_orders >= 1 && n_orders <= 512, "ssi_cluster: 1 <= n_orders <= 512");
  for (int m = 0; m < n_orders; ++m)
    SSI_CHECK(orders[m] >= 2 && orders[m] % 2 == 0, "ssi_cluster: orders must be even and >= 2");
  SSI_CHECK(params->tau >= 0.0 && params->min_size >= 1, "ssi_cluster: need tau >= 0, min_size >= 1");
  SSI_CHECK(params->fcm_m > 1.0 && params->fcm_tol > 0.0 && params->fcm_max_iter >= 1,
            "ssi_cluster: need fcm_m > 1, fcm_tol > 0, fcm_max_iter >= 1");
  SSI_CHECK((reinterpret_cast<uintptr_t>(phi) & 7) == 0, "ssi_cluster: phi must be 8-byte aligned");
  SSI_CUDA(cudaSetDevice(ctx->device));
  *n_modes = 0;
  return cluster_run(ctx, n_lags, n_orders, orders, l, poles, phi, params, modes, max_modes, n_modes,
                     features, membership, label, info, static_cast<cudaStream_t>(stream));
}
