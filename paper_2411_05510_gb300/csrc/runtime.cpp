// Host runtime of libssi: contexts, device-memory accounting against the HBM budget,
// workspaces, error reporting, tensor-map encoding, and the parameter rules of Sec. 3.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace ssi {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

ssi_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e), cudaGetErrorString(e), what,
            file, line);
  return SSI_E_CUDA;
}

int device_sms(int device) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  return n > 0 ? n : 1;
}

ssi_status ctx_alloc(ssi_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return SSI_OK;
  {
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    if (ctx->in_use + bytes > ctx->budget) {
      set_error("HBM budget exceeded: %zu in use + %zu requested > %zu budget", ctx->in_use, bytes,
                ctx->budget);
      return SSI_E_NOMEM;
    }
    ctx->in_use += bytes;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    ctx->in_use -= bytes;
    *p = nullptr;
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return SSI_E_NOMEM;
  }
  return SSI_OK;
}

void ctx_free(ssi_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> g(ctx->mem_mu);
  ctx->in_use -= bytes;
}

ssi_status ws_reserve(ssi_ctx* ctx, Workspace& ws, size_t bytes, cudaStream_t stream) {
  if (bytes <= ws.cap) return SSI_OK;
  if (ws.base) {
    SSI_CUDA(cudaStreamSynchronize(stream));
    ctx_free(ctx, ws.base, ws.cap);
    ws.base = nullptr;
    ws.cap = 0;
  }
  size_t want = (bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
  void* p = nullptr;
  SSI_TRY(ctx_alloc(ctx, &p, want));
  ws.base = static_cast<char*>(p);
  ws.cap = want;
  ws.off = 0;
  return SSI_OK;
}

ssi_status check_dev_status(int* dev_status, cudaStream_t stream) {
  int h = 0;
  SSI_CUDA(cudaMemcpyAsync(&h, dev_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SSI_CUDA(cudaStreamSynchronize(stream));
  if (h == 0) return SSI_OK;
  SSI_CUDA(cudaMemsetAsync(dev_status, 0, sizeof(int), stream));
  if (h & DEV_TIMEOUT) {
    set_error("a device-side bounded wait ran out (status 0x%x)", h);
    return SSI_E_TIMEOUT;
  }
  if (h & DEV_NOTCONVERGED) {
    set_error("a device iteration hit its cap (status 0x%x)", h);
    return SSI_E_NOTCONVERGED;
  }
  set_error("a kernel reported an unsupported shape (status 0x%x)", h);
  return SSI_E_INVALID;
}

bool make_tmap_bf16_2d(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols,
                       uint64_t pitch_elems, uint32_t box_cols, uint32_t box_rows,
                       CUtensorMapSwizzle swizzle) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {pitch_elems * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): rows=%llu cols=%llu pitch=%llu box=%ux%u", (int)r,
              (unsigned long long)rows, (unsigned long long)cols, (unsigned long long)pitch_elems,
              box_cols, box_rows);
    return false;
  }
  return true;
}

void serving_destroy(ssi_ctx* ctx);  // serving.cpp
void solve_buffers_destroy(ssi_ctx* ctx);  // pipeline.cpp

}  // namespace ssi

using namespace ssi;

extern "C" {

const char* ssi_last_error(void) { return g_err; }

int ssi_version(void) { return 100; }

ssi_status ssi_create(ssi_ctx** out, int device, size_t hbm_budget_bytes) {
  SSI_CHECK(out, "ssi_create: null output pointer");
  *out = nullptr;
  int n = 0;
  SSI_CUDA(cudaGetDeviceCount(&n));
  SSI_CHECK(device >= 0 && device < n, "ssi_create: device %d not present (%d devices)", device, n);
  SSI_CUDA(cudaSetDevice(device));
  int major = 0, minor = 0;
  SSI_CUDA(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
  SSI_CUDA(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
  if (major != 10 || minor != 3) {
    set_error("ssi_create: libssi is built for sm_103a; device %d is sm_%d%d", device, major, minor);
    return SSI_E_CUDA;
  }
  ssi_ctx* ctx = new (std::nothrow) ssi_ctx();
  if (!ctx) return SSI_E_NOMEM;
  ctx->device = device;
  ctx->num_sms = device_sms(device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : free_b / 2;
  void* p = nullptr;
  ssi_status st = ctx_alloc(ctx, &p, 256);
  if (st != SSI_OK) {
    delete ctx;
    return st;
  }
  ctx->dev_status = static_cast<int*>(p);
  cudaMemset(ctx->dev_status, 0, 256);
  *out = ctx;
  return SSI_OK;
}

void ssi_destroy(ssi_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  serving_destroy(ctx);
  cudaDeviceSynchronize();
  solve_buffers_destroy(ctx);
  if (ctx->ws.base) ctx_free(ctx, ctx->ws.base, ctx->ws.cap);
  if (ctx->ws_aux.base) ctx_free(ctx, ctx->ws_aux.base, ctx->ws_aux.cap);
  ctx_free(ctx, ctx->dev_status, 256);
  delete ctx;
}

size_t ssi_memory_in_use(const ssi_ctx* ctx) { return ctx ? ctx->in_use : 0; }

ssi_status ssi_set_concurrency(ssi_ctx* ctx, int solves_in_flight) {
  SSI_CHECK(ctx, "ssi_set_concurrency: null context");
  SSI_CHECK(solves_in_flight >= 1, "ssi_set_concurrency: solves_in_flight < 1");
  ctx->inflight.store(solves_in_flight);
  return SSI_OK;
}

ssi_status ssi_profile(ssi_ctx* ctx, int enable) {
  SSI_CHECK(ctx, "ssi_profile: null context");
  std::lock_guard<std::mutex> g(ctx->prof_mu);
  ctx->prof_on = enable != 0;
  return SSI_OK;
}

ssi_status ssi_profile_read(ssi_ctx* ctx, double* ms, int64_t* counts, int n, int64_t* launches) {
  SSI_CHECK(ctx, "ssi_profile_read: null context");
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> recs;
  {
    std::lock_guard<std::mutex> g(ctx->prof_mu);
    recs.swap(ctx->prof_recs);
  }
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = 0.0;
    if (counts) counts[i] = 0;
  }
  ssi_status st = SSI_OK;
  for (auto& r : recs) {
    const int id = std::get<0>(r);
    cudaEvent_t e0 = std::get<1>(r), e1 = std::get<2>(r);
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaEventElapsedTime", __FILE__, __LINE__);
    if (id >= 0 && id < n) {
      if (ms) ms[id] += t;
      if (counts) counts[id] += 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (launches) *launches = ctx->launches.exchange(0);
  return st;
}

ssi_status ssi_rank_rule(int64_t T_size, double* kbar_percent, int64_t* k) {
  SSI_CHECK(T_size > 0, "ssi_rank_rule: T_size must be positive");
  double kbar = 30.0 - 0.00156 * (double)T_size;
  if (kbar < 25.0) kbar = 25.0;
  if (kbar_percent) *kbar_percent = kbar;
  if (k) *k = (int64_t)std::ceil(kbar * (double)T_size / 100.0 - 1e-9);
  return SSI_OK;
}

ssi_status ssi_lag_rule(double fs, double f0, double beta, int* jb, int* jb_min, int* jb_max) {
  SSI_CHECK(fs > 0 && f0 > 0 && beta >= 1.0, "ssi_lag_rule: need fs > 0, f0 > 0, beta >= 1");
  const int j = (int)std::ceil(10.0 * fs / (2.0 * f0) - 1e-9);
  const int jmin = (int)std::ceil(9.0 * fs / (2.0 * f0) - 1e-9);
  const int jmax = (int)std::ceil(beta * jmin - 1e-9);
  if (jb) *jb = j;
  if (jb_min) *jb_min = jmin;
  if (jb_max) *jb_max = jmax;
  return SSI_OK;
}

double ssi_time_lag(int jb, double fs) { return (2.0 * jb - 1.0) / fs; }

int64_t ssi_pole_slots(int n_orders, const int* orders) {
  int64_t s = 0;
  for (int m = 0; m < n_orders; ++m) s += orders[m] / 2;
  return s;
}

}  // extern "C"
