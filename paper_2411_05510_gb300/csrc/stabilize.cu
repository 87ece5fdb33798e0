// Stage (d): hard criteria and the soft criteria of the 2D / 3D stabilization diagram
// (Sec. 2.1 "HC" and "SC", Sec. 2.3 Eq. (stabcriteria3D)).
//   HC: xi <= xi_max (and xi > 0, |mu| < 1), MPC > mpc_min, MPD < mpd_max.
//   SC: pole i at (lag t, order m) is stable along orders when SOME HC-passing pole j at
//       (t, m-1) has |f_i - f_j|/max(f_i, f_j) <= a_f, |xi_i - xi_j|/max(xi_i, xi_j) <= a_xi
//       and 1 - MAC(phi_i, phi_j) <= a_mac; along lags likewise with (t-1, m).
// k_hard_criteria writes the HC bits of every slot; k_soft_criteria then runs one warp per
// HC-passing pole, scanning the neighbour cells (frequency and damping first, the complex
// MAC dot product of length l only for candidates that pass both).
#include "common.cuh"

namespace ssi {

namespace {

struct StabParams {
  int n_lags, n_orders, l;
  long long slots_per_lag;
  long long slot_off[512];
  int nslot[512];
  double xi_max, mpc_min, mpd_max, a_f, a_xi, a_mac;
  int use_lag;
};

__global__ void k_hard_criteria(ssi_pole* __restrict__ poles, long long n, StabParams p) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    ssi_pole q = poles[e];
    uint32_t f = q.flags & (SSI_POLE_VALID | SSI_POLE_NOTCONV);
    if (f & SSI_POLE_VALID) {
      const double mod = sqrt((double)q.mu_re * q.mu_re + (double)q.mu_im * q.mu_im);
      if (!(q.xi <= p.xi_max) || !(q.xi > 0.0) || !(mod < 1.0)) f |= SSI_POLE_HC_XI;
      if (!(q.mpc > p.mpc_min)) f |= SSI_POLE_HC_MPC;
      if (!(q.mpd < p.mpd_max)) f |= SSI_POLE_HC_MPD;
      if (!(f & (SSI_POLE_HC_XI | SSI_POLE_HC_MPC | SSI_POLE_HC_MPD))) f |= SSI_POLE_HC;
    }
    poles[e].flags = f;
  }
}

__device__ bool pair_ok(const ssi_pole& a, const float* pa, const ssi_pole& b, const float* pb, int l,
                        const StabParams& p, int lane) {
  const double fa = a.f_hz, fb = b.f_hz, xa = a.xi, xb = b.xi;
  const bool pre = fabs(fa - fb) / fmax(fa, fb) <= p.a_f && fabs(xa - xb) / fmax(xa, xb) <= p.a_xi;
  if (!pre) return false;
  // MAC = |a^H b|^2 / (|a|^2 |b|^2)
  float dr = 0.f, di = 0.f, na = 0.f, nb = 0.f;
  for (int c = lane; c < l; c += 32) {
    const float ar = pa[2 * c], ai = pa[2 * c + 1], br = pb[2 * c], bi = pb[2 * c + 1];
    dr += ar * br + ai * bi;
    di += ar * bi - ai * br;
    na += ar * ar + ai * ai;
    nb += br * br + bi * bi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
  }
  const double den = (double)na * (double)nb;
  const double mac = den > 0 ? ((double)dr * dr + (double)di * di) / den : 0.0;
  return 1.0 - mac <= p.a_mac;
}

__global__ void k_soft_criteria(ssi_pole* __restrict__ poles, const float* __restrict__ phi,
                                long long n, StabParams p) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = warp0; e < n; e += nwarps) {
    const ssi_pole q = poles[e];
    if (!(q.flags & SSI_POLE_HC)) continue;
    const int t = (int)(e / p.slots_per_lag);
    const long long w = e % p.slots_per_lag;
    int m = 0;
    while (m + 1 < p.n_orders && p.slot_off[m + 1] <= w) ++m;
    const float* pq = phi + (size_t)e * 2 * p.l;
    uint32_t add = 0;
    // previous order, same lag
    if (m > 0) {
      const long long base = (long long)t * p.slots_per_lag + p.slot_off[m - 1];
      for (int j = 0; j < p.nslot[m - 1]; ++j) {
        const ssi_pole o = poles[base + j];
        if (!(o.flags & SSI_POLE_HC)) continue;
        if (pair_ok(q, pq, o, phi + (size_t)(base + j) * 2 * p.l, p.l, p, lane)) {
          add |= SSI_POLE_ORDER;
          break;
        }
      }
    }
    // previous lag, same order
    if (p.use_lag && t > 0) {
      const long long base = (long long)(t - 1) * p.slots_per_lag + p.slot_off[m];
      for (int j = 0; j < p.nslot[m]; ++j) {
        const ssi_pole o = poles[base + j];
        if (!(o.flags & SSI_POLE_HC)) continue;
        if (pair_ok(q, pq, o, phi + (size_t)(base + j) * 2 * p.l, p.l, p, lane)) {
          add |= SSI_POLE_LAG;
          break;
        }
      }
    }
    if (lane == 0 && add) poles[e].flags = q.flags | add;
  }
}

}  // namespace

size_t stabilize_ws_bytes(int, int) { return 0; }

ssi_status stabilize_ws(ssi_ctx* ctx, Workspace&, int n_lags, int n_orders, const int* orders, int l,
                        ssi_pole* poles, const float* phi, const ssi_stab_params* sp,
                        cudaStream_t stream) {
  SSI_CHECK(n_orders >= 1 && n_orders <= 512, "stabilize: 1 <= n_orders <= 512");
  StabParams p{};
  p.n_lags = n_lags;
  p.n_orders = n_orders;
  p.l = l;
  long long so = 0;
  for (int m = 0; m < n_orders; ++m) {
    p.slot_off[m] = so;
    p.nslot[m] = orders[m] / 2;
    so += orders[m] / 2;
  }
  p.slots_per_lag = so;
  p.xi_max = sp->xi_max;
  p.mpc_min = sp->mpc_min;
  p.mpd_max = sp->mpd_max;
  p.a_f = sp->a_f;
  p.a_xi = sp->a_xi;
  p.a_mac = sp->a_mac;
  p.use_lag = sp->use_lag_axis ? 1 : 0;
  const long long n = so * n_lags;
  if (n == 0) return SSI_OK;
  const int blocks = (int)std::min<long long>(ceil_div(n, 256), (long long)ctx->num_sms * 8);
  ProfScope ps(ctx, ST_STAB, stream);
  count_launches(ctx, 2);
  k_hard_criteria<<<blocks, 256, 0, stream>>>(poles, n, p);
  SSI_CUDA(cudaGetLastError());
  const int blocks2 = (int)std::min<long long>(ceil_div(n * 32, 256), (long long)ctx->num_sms * 16);
  k_soft_criteria<<<blocks2, 256, 0, stream>>>(poles, phi, n, p);
  SSI_CUDA(cudaGetLastError());
  return SSI_OK;
}

}  // namespace ssi

extern "C" ssi_status ssi_stabilize(ssi_ctx* ctx, int n_lags, int n_orders, const int* orders, int l,
                                    ssi_pole* poles, const float* phi, const ssi_stab_params* params,
                                    void* stream) {
  using namespace ssi;
  SSI_CHECK(ctx && orders && poles && phi && params, "ssi_stabilize: null pointer");
  SSI_CHECK(n_lags >= 1 && l >= 1, "ssi_stabilize: bad n_lags / l");
  for (int m = 0; m < n_orders; ++m)
    SSI_CHECK(orders[m] >= 2 && orders[m] % 2 == 0, "ssi_stabilize: orders must be even and >= 2");
  SSI_CUDA(cudaSetDevice(ctx->device));
  return stabilize_ws(ctx, ctx->ws, n_lags, n_orders, orders, l, poles, phi, params,
                      static_cast<cudaStream_t>(stream));
}
