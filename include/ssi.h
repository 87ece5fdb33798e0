/*
 * ssi.h -- C ABI of libssi, a GB300 (sm_103a) implementation of the hot path of
 * covariance-driven stochastic subspace identification with randomized SVD
 * (RSVD-CoV-SSI, arXiv 2411.05510).
 *
 * Conventions shared by every entry point
 *   - Every call returns an ssi_status; nothing throws across the ABI.
 *     ssi_last_error() returns a thread-local message for the last failure.
 *   - "device" pointers are CUDA device memory owned by the caller unless a
 *     comment says otherwise; "host" pointers are ordinary host memory.
 *   - Device work is enqueued on `stream` (a cudaStream_t passed as void*,
 *     NULL = legacy default stream) and is asynchronous: outputs are valid once
 *     the stream has been synchronised.  Entry points do not synchronise the
 *     stream unless stated.
 *   - Scratch memory comes from the context's workspace, which grows on demand
 *     within the context's HBM budget (SSI_E_NOMEM beyond it).  One context must
 *     not run two calls at the same time from different host threads, except
 *     through the serving calls (ssi_submit / ssi_poll), which are thread safe.
 *   - Matrices are row-major unless stated.
 *   - Invalid shapes or parameters return SSI_E_INVALID before any work is
 *     enqueued.  A CUDA error returns SSI_E_CUDA.  A device-side bounded wait
 *     that ran out returns SSI_E_TIMEOUT (checked at the next synchronising
 *     call); per-realisation non-convergence of eig(A) is reported per pole
 *     (SSI_POLE_NOTCONV) and does not fail the call.
 */
#ifndef SSI_H
#define SSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SSI_OK = 0,
  SSI_E_INVALID = 1,       /* bad argument or shape */
  SSI_E_NOMEM = 2,         /* HBM budget or device allocation exhausted */
  SSI_E_CUDA = 3,          /* CUDA runtime / driver error */
  SSI_E_TIMEOUT = 4,       /* a bounded device wait ran out, or ssi_poll timed out */
  SSI_E_NOTCONVERGED = 5,  /* an iteration hit its cap */
  SSI_E_BUSY = 6,          /* serving: no free slot / budget right now */
  SSI_E_NOTFOUND = 7       /* serving: unknown job id */
} ssi_status;

/* Arithmetic of the two dense contractions (lag GEMMs and Toeplitz sketch GEMMs). */
typedef enum {
  SSI_PREC_FP32 = 0,       /* plain FP32 FMA on the CUDA cores */
  SSI_PREC_SPLIT_BF16 = 1  /* tcgen05 tensor cores, x = hi + lo in BF16, products
                              hi*hi + hi*lo + lo*hi accumulated in FP32 */
} ssi_precision;

/* Arithmetic of the small dense problems of every lag: the K x K SVD of the range
 * finder (Sec. 2.2), the least squares for A and eig(A) (Sec. 2.1).  The sketch and QR
 * passes of the range finder are FP32 in both modes. */
typedef enum {
  SSI_SMALL_FP32 = 0,      /* FP32 with FP64 reductions (the fast mode) */
  SSI_SMALL_FP64 = 1       /* FP64 throughout: FP64 one-sided Jacobi (stops at 1e-13
                              relative off-orthogonality), U = Q U~ in FP64, FP64 Gram,
                              Cholesky and A~_n, FP64 Hessenberg + double-shift QR */
} ssi_small_precision;

typedef struct ssi_ctx ssi_ctx;

/* Context bound to CUDA device `device`.  hbm_budget_bytes caps the device memory
 * the context may hold (0 = half of the free memory at creation). */
ssi_status ssi_create(ssi_ctx** ctx, int device, size_t hbm_budget_bytes);
/* Frees the context and everything it owns; waits for its outstanding work. */
void ssi_destroy(ssi_ctx* ctx);
/* Thread-local description of the last failure on this thread ("" if none). */
const char* ssi_last_error(void);
/* Library version, 100*major + minor. */
int ssi_version(void);
/* Device memory currently held by the context (bytes). */
size_t ssi_memory_in_use(const ssi_ctx* ctx);

/* Concurrency hint: how many solves are expected on the device at once (several
 * contexts, or the slots of this context's serving loop).  With more than one, the
 * cooperative QR of the range finder (Sec. 2.2) takes half the SMs, two row chunks per
 * CTA, so that two solves' QR grids execute side by side and other SMs stay free for a
 * third solve's GEMMs and eigenproblems; with one it takes every SM.  Results are
 * bit-identical either way (the QR reductions run over fixed row chunks in a fixed
 * order).  Default 1; ssi_serve_config sets it to max_slots.  Takes effect for launches
 * made after the call.  SSI_E_INVALID for a null context or solves_in_flight < 1. */
ssi_status ssi_set_concurrency(ssi_ctx* ctx, int solves_in_flight);

/* Instrumentation.  ssi_profile(ctx, 1) makes the direct (non-serving) calls of the
 * context record a CUDA event pair around each stage on the call's stream; this adds
 * no synchronisation.  ssi_profile_read synchronises on the recorded events and
 * returns, per stage id, the summed device time in ms and the number of scopes since
 * the previous read, plus the number of kernels the context launched (also reset).
 * Stage ids: 0 split/transpose, 1 lag GEMM, 2 lag reduction, 3 Toeplitz sketch GEMMs,
 * 4 QR, 5 small SVD, 6 Gram/factorisation, 7 eig (Hessenberg, QR iteration, Schur
 * vectors), 8 stability, 9 other, 10 eigenvector back transformation and mode shapes,
 * 11 clustering;
 * stages with ids >= n are not reported. */
ssi_status ssi_profile(ssi_ctx* ctx, int enable);
ssi_status ssi_profile_read(ssi_ctx* ctx, double* ms, int64_t* counts, int n, int64_t* launches);

/* ------------------------------------------------------------------------------
 * Stage (a): output covariances, Sec. 2.1 ("R_1 .. R_{2jb-1} derived directly
 * from the records").
 *   R_k = 1/(N-k) * sum_{t=0}^{N-k-1} y_{t+k} y_t^T,  k = 1..max_lag.
 * Y       device, float32, l x N, channel-major (row c holds channel c, samples
 *         contiguous).
 * R       device, float64, max_lag x l x l; R_k at offset (k-1)*l*l, entry
 *         [a][b] = E[y_{t+k,a} y_{t,b}].
 * prec    SSI_PREC_SPLIT_BF16 (tensor cores) or SSI_PREC_FP32 (CUDA cores).
 *         Both accumulate FP32 partial sums over time chunks and add the chunks
 *         in FP64.
 * Limits: 1 <= l <= 1024, 1 <= max_lag < N, N < 2^31.
 * ---------------------------------------------------------------------------- */
ssi_status ssi_covariances(ssi_ctx* ctx, const float* Y, int l, int64_t N, int max_lag,
                           ssi_precision prec, double* R, void* stream);

/* ------------------------------------------------------------------------------
 * Sliding-window covariances for continuous monitoring (Sec. 3.2.2 identifies a
 * continuously recorded bridge window after window; Sec. 1 cites sliding-window SSI).
 * The object holds the last `window` samples of an l-channel stream and the
 * unnormalised lag sums S_k over the pairs inside them.  A push of B samples adds the
 * pairs that enter and, once the window is full, removes the B oldest samples' pairs,
 * each as the difference of two segment covariances of about B + max_lag samples
 * (cost O(l^2 (B + max_lag) max_lag) instead of O(l^2 window max_lag)).
 * ssi_cov_stream_covariances writes R_k = S_k / (n - k), k = 1..max_lag, for the n
 * samples in the window, in the layout of ssi_covariances.
 * create   window > max_lag, 1 <= max_block; l and precision as ssi_covariances.
 *          Allocates l x (window + max_block) floats of ring, the sums, a segment
 *          buffer and the stage (a) workspace from the context's budget.
 * push     Y: device, l x B channel-major, B <= max_block; the first push needs
 *          B > max_lag.  Asynchronous on `stream`; Y may be reused once the stream
 *          has passed the call.
 * covariances  R: device, max_lag x l x l; *n_samples (host, optional): n.
 *          SSI_E_INVALID while the window holds no more than max_lag samples.
 * refresh  rebuilds the sums from the samples held in the ring (one whole-window
 *          computation).  The updates add and subtract segment sums whose rounding does
 *          not cancel; push rebuilds by itself after every `window` samples pushed, so
 *          the error stays within that of a few whole-window computations however long
 *          the stream runs.
 * destroy  synchronises the device, then frees the object's memory; call it before
 *          ssi_destroy of its context.
 * The workspace of the largest segment and of a whole window is reserved at creation,
 * so push and refresh never allocate.  A push or refresh that fails part way (a CUDA
 * error) marks the object inconsistent: later calls other than destroy return
 * SSI_E_INVALID.
 * Pushes and reads of one object must be ordered (one stream, or synchronised).
 * ---------------------------------------------------------------------------- */
typedef struct ssi_cov_stream ssi_cov_stream;
ssi_status ssi_cov_stream_create(ssi_ctx* ctx, int l, int max_lag, int64_t window,
                                 int64_t max_block, ssi_precision prec, ssi_cov_stream** out);
ssi_status ssi_cov_stream_push(ssi_cov_stream* st, const float* Y, int64_t B, void* stream);
ssi_status ssi_cov_stream_covariances(ssi_cov_stream* st, double* R, int64_t* n_samples,
                                      void* stream);
ssi_status ssi_cov_stream_refresh(ssi_cov_stream* st, void* stream);
ssi_status ssi_cov_stream_destroy(ssi_cov_stream* st);

/* ------------------------------------------------------------------------------
 * Covariances without device allocation (no counterpart in the paper: an
 * interface for callers that cannot allocate device memory when they need the
 * covariances, e.g. code inside a CUDA-graph capture that must not add allocation
 * nodes, plugins of a framework that owns all device memory, or processes under a
 * fixed memory reservation).
 * Same result as ssi_covariances with SSI_PREC_FP32 (same definition of R_k, same
 * argument layout), computed on the CUDA cores of the current device.  It calls no
 * cudaMalloc / cudaFree and needs no context: its scratch is one file-scope device
 * array of 16 MiB (4 Mi floats) that every GPU loading the library holds until the
 * process exits.
 * Limits: max_lag * roundup(l, 64)^2 <= 4 Mi floats (SSI_E_INVALID beyond, with a
 * message), plus the limits of ssi_covariances.
 * Every call looks up the array's device address on the current device (a host-side
 * runtime query; the address is not cached, so it stays valid across cudaDeviceReset).
 * The first call on a device also loads the library's device code there, so make it
 * before any stream capture on that device.
 * Every call shares the one array: calls whose work overlaps on the GPU (different
 * streams, or several host threads) race and must be serialised by the caller.
 * ---------------------------------------------------------------------------- */
ssi_status ssi_covariances_noalloc(const float* Y, int l, int64_t N, int max_lag, double* R,
                                   void* stream);

/* ------------------------------------------------------------------------------
 * Gaussian test matrix Omega of Sec. 2.2 (Eq. Y = A Omega, Algorithm 1).
 * omega   device, float32, rows x cols row-major.  Entry (r, c) comes from the
 *         Philox4x32-10 counter (r, c, 0, 0) with key (seed & 0xffffffff,
 *         seed >> 32): outputs x0, x1 -> u = (x + 0.5)/2^32,
 *         z = sqrt(-2 ln u0) cos(2 pi u1).
 * ---------------------------------------------------------------------------- */
ssi_status ssi_gaussian_omega(ssi_ctx* ctx, int rows, int cols, uint64_t seed, float* omega,
                              void* stream);

/* ------------------------------------------------------------------------------
 * Stages (a)+(b): block-Toeplitz T_{1|i} (Eq. Toeplitz: block (a,b) = R_{i+a-b})
 * and its randomized SVD (Sec. 2.2, Algorithm 1, with oversampling and power
 * iterations re-orthonormalised by QR after every product).
 * T is never formed: its tiles are read from the covariances by lag index.
 *   Omega = gaussian(L, k+oversample, seed);  Q = qr(T Omega);
 *   repeat q times: Q = qr(T qr(T^T Q));      P = Q^T T;
 *   (U~, S) = svd(P);                          U = Q U~[:, :k].
 * R       device, float64, (2i-1) x l x l as produced by ssi_covariances (more
 *         lags may be present; only R_1..R_{2i-1} are read).
 * small   arithmetic of the K x K SVD and of U = Q U~ (SSI_SMALL_FP32: FP32 Jacobi,
 *         stopping at 1e-5 relative off-orthogonality; SSI_SMALL_FP64: FP64 Jacobi,
 *         1e-13).  The Jacobi sweeps run on a cooperative grid (parallel block
 *         ordering), so they take several SMs for as long as they run.
 * U       device, float64, L x k row-major, L = l*i (left singular vectors).
 * S       device, float64, k singular values, descending.
 * Limits: i >= 2, 1 <= k, k + oversample <= min(L, 16384), l <= 1024.  (K = L with
 *         q = 0 makes Q span the whole column space: U and S are then the SVD of T.)
 * ---------------------------------------------------------------------------- */
ssi_status ssi_toeplitz_rsvd(ssi_ctx* ctx, const double* R, int l, int i, int k, int oversample,
                             int q, uint64_t seed, ssi_precision prec, ssi_small_precision small,
                             double* U, double* S, void* stream);

/* ------------------------------------------------------------------------------
 * Stage (c): realisation for every (lag, order) of a stabilization diagram,
 * Sec. 2.1 (O = U S^{1/2}; C = first l rows; A = O^to+ O^bo; A = Psi M Psi^-1;
 * lambda = ln(mu)/dt; f = |lambda|/(2 pi); xi = -Re(lambda)/|lambda|; Phi = C Psi).
 * The S^{1/2} column scaling is a similarity transform of A and is not applied:
 * eig((U^to)+ U^bo) equals eig((O^to)+ O^bo) and C Psi = U[:l,:n] Psi~.
 * One pole per complex-conjugate eigenvalue pair (Im mu > 0); real eigenvalues
 * give no pole.
 *
 * lags     host, n_lags block counts i_t (each >= 2), n_lags <= 64.
 * U        host array of n_lags device pointers; U[t] is (l*lags[t]) x k float64, row-
 *          major (as written by ssi_toeplitz_rsvd).
 * small    SSI_SMALL_FP32: U is rounded to FP32 and the Gram matrices, Cholesky factor,
 *          A~_n and eig run in FP32 (FP64 chunk sums); SSI_SMALL_FP64: all of them in
 *          FP64.  Pole records are written in FP32 either way (f, xi and mu are rounded
 *          once, about 6e-8 relative).
 * orders   host, n_orders even model orders, ascending, 2 <= order <= min(k, 512),
 *          n_orders <= 512; k <= 512.  Orders up to 224 (FP32) or 160 (FP64) keep A
 *          in shared memory; larger ones run the same kernel with A in the
 *          realisation's global scratch (slower: every access goes to L2).
 * poles    device, ssi_pole_slots(n_orders, orders) * n_lags records.  Slot
 *          (t, m, j) = t*slots_per_lag + sum_{m'<m} orders[m']/2 + j; the poles of
 *          one realisation come first, ascending in frequency; unused slots have
 *          flags == 0.
 * phi      device, float32 complex (re, im interleaved), l values per slot,
 *          unit 2-norm, largest-modulus component real and positive.
 * ---------------------------------------------------------------------------- */
typedef struct {
  float f_hz;      /* natural frequency [Hz] */
  float xi;        /* damping ratio */
  float mu_re;     /* discrete eigenvalue */
  float mu_im;
  float mpc;       /* modal phase collinearity in [0, 1] */
  float mpd;       /* mean phase deviation in [0, 1] (degrees / 90) */
  int32_t lag;     /* block count i of the Toeplitz matrix */
  int32_t order;   /* model order n */
  uint32_t flags;  /* SSI_POLE_* bits */
  int32_t index;   /* pole index within its realisation */
} ssi_pole;

#define SSI_POLE_HC_XI    1u   /* fails xi <= xi_max (or xi <= 0, |mu| >= 1) */
#define SSI_POLE_HC_MPC   2u   /* fails MPC > mpc_min */
#define SSI_POLE_HC_MPD   4u   /* fails MPD < mpd_max */
#define SSI_POLE_HC       8u   /* passes every hard criterion */
#define SSI_POLE_ORDER   16u   /* stable along model orders */
#define SSI_POLE_LAG     32u   /* stable along time lags */
#define SSI_POLE_VALID   64u   /* slot holds a pole */
#define SSI_POLE_NOTCONV 128u  /* eig(A) of this realisation hit its iteration cap */

/* Number of pole slots of one lag: sum over orders of order/2. */
int64_t ssi_pole_slots(int n_orders, const int* orders);

ssi_status ssi_realize_batch(ssi_ctx* ctx, int n_lags, const int* lags, const double* const* U,
                             int l, int k, const int* orders, int n_orders, double dt,
                             ssi_small_precision small, ssi_pole* poles, float* phi, void* stream);

/* ------------------------------------------------------------------------------
 * Stage (d): hard criteria and the soft criteria of Eq. (stabcriteria3D).
 * HC: xi <= xi_max (and xi > 0, |mu| < 1), MPC > mpc_min, MPD < mpd_max.
 * SC: a pole passing HC at (lag t, order m) gets SSI_POLE_ORDER if some
 * HC-passing pole at (t, m-1) has |df|/max(f) <= a_f, |dxi|/max(xi) <= a_xi and
 * 1 - MAC <= a_mac; SSI_POLE_LAG likewise with (t-1, m) when use_lag_axis.
 * Indices m-1 and t-1 are the previous entries of the order and lag grids.
 * poles / phi  device, as written by ssi_realize_batch (flags updated in place).
 * ---------------------------------------------------------------------------- */
typedef struct {
  double xi_max, mpc_min, mpd_max;   /* e.g. 0.10, 0.6, 0.5 */
  double a_f, a_xi, a_mac;           /* e.g. 0.01, 0.03, 0.02 */
  int32_t use_lag_axis;              /* 1: 3D diagram, 0: orders only */
  int32_t reserved;
} ssi_stab_params;

ssi_status ssi_stabilize(ssi_ctx* ctx, int n_lags, int n_orders, const int* orders, int l,
                         ssi_pole* poles, const float* phi, const ssi_stab_params* params,
                         void* stream);

/* ------------------------------------------------------------------------------
 * Stage (e): two-stage clustering of the stable poles (Sec. 2.3 "3D clustering",
 * Sec. 3.1) into modes.
 * Stage I: every pole with SSI_POLE_VALID, SSI_POLE_HC and SSI_POLE_ORDER or
 * SSI_POLE_LAG (a candidate) gets x = (d_f, d_xi, 1 - MAC, 1 - MPC, MPD), the first three
 * against its nearest HC-passing neighbour in d_f + d_xi + (1 - MAC) among the poles of
 * (t, m-1) and (t-1, m), first minimum in slot order, d = |a - b| / max(a, b).  Fuzzy
 * C-means with two clusters, fuzzifier fcm_m, from the feature-wise minimum and
 * maximum, stops when no membership changes by fcm_tol or more (or after fcm_max_iter
 * iterations).  The physical cluster is the one whose centroid is nearer the origin;
 * a candidate is kept when its membership P of it is >= 1/2.
 * Stage II: single linkage in d_f + d_xi + (1 - MAC) over the kept poles, cut at tau:
 * connected components of the graph joining poles at distance <= tau.  Components of
 * >= min_size poles are the modes, sorted by mean frequency.  Decisions are taken on
 * FP64 distances.
 * poles / phi   device, as written by ssi_realize_batch or ssi_solve and flagged by
 *               ssi_stabilize (phi 8-byte aligned); not modified.
 * modes         host, max_modes entries; *n_modes receives the number of modes (may
 *               exceed max_modes: only the first max_modes are written).
 * features      optional device, 5 doubles per slot: the Stage I features of the
 *               candidates, zero elsewhere.
 * membership    optional device, one double per slot: P of the candidates, -1 elsewhere.
 * label         optional device, one int32 per slot: for a kept pole the slot of the
 *               first kept pole of its component, -1 elsewhere.
 * info          optional host: counts, C-means iterations and centroids.
 * Synchronises `stream` (the mode table is returned on the host); uses the context's
 * workspace.  SSI_E_INVALID for bad shapes or parameters, SSI_E_TIMEOUT if the C-means
 * grid barrier gave up.
 * ---------------------------------------------------------------------------- */
typedef struct {
  double tau;              /* Stage II cut distance, e.g. 0.05 */
  int32_t min_size;        /* smallest component reported as a mode, e.g. 10 */
  int32_t fcm_max_iter;    /* C-means iteration cap, e.g. 500 */
  double fcm_m;            /* fuzzifier, > 1; e.g. 2 */
  double fcm_tol;          /* membership change that ends the iteration, e.g. 1e-10 */
} ssi_cluster_params;

typedef struct {
  double f_hz;             /* mean natural frequency of the members [Hz] */
  double xi;               /* mean damping ratio of the members */
  int32_t size;            /* number of member poles */
  int32_t medoid_slot;     /* slot of the medoid (smallest sum of distances to the others,
                              ties to the earlier pole); its phi is the mode shape */
} ssi_mode;

typedef struct {
  int32_t n_candidates;    /* poles entering Stage I */
  int32_t n_kept;          /* poles kept by Stage I */
  int32_t n_components;    /* Stage II components before the size cut */
  int32_t n_modes;
  int32_t fcm_iterations;
  int32_t fcm_converged;   /* 0 if fcm_max_iter was reached */
  int32_t physical;        /* index (0 or 1) of the physical C-means cluster */
  int32_t reserved;
  double centroids[2][5];  /* final C-means centroids */
} ssi_cluster_info;

ssi_status ssi_cluster(ssi_ctx* ctx, int n_lags, int n_orders, const int* orders, int l,
                       const ssi_pole* poles, const float* phi, const ssi_cluster_params* params,
                       ssi_mode* modes, int max_modes, int* n_modes, double* features,
                       double* membership, int32_t* label, ssi_cluster_info* info, void* stream);

/* ------------------------------------------------------------------------------
 * One complete solve (stages a-d) of one record: covariances up to 2*max(lags)-1,
 * then per lag the Toeplitz RSVD, then the realisations of every (lag, order)
 * and the stability checks.  All work is ordered after earlier work on `stream`, and
 * later work on `stream` is ordered after all of it; nothing is synchronised.  With
 * several lags the per-lag RSVDs (independent once R exists, Sec. 2.3) run on up to
 * four internal streams of the context, forked from and joined back to `stream`
 * through events.  Y may be device memory (y_on_host = 0) or host memory
 * (y_on_host = 1, pinned for overlap), in which case it is copied in on `stream`.
 * ---------------------------------------------------------------------------- */
typedef struct {
  const float* Y;          /* l x N, channel-major */
  int32_t y_on_host;
  int32_t l;
  int64_t N;
  double fs;               /* sampling frequency [Hz] */
  int32_t n_lags;
  const int32_t* lags;     /* host, ascending */
  int32_t n_orders;
  const int32_t* orders;   /* host, ascending, even */
  int32_t k, oversample, q;
  int32_t prec;            /* ssi_precision of the lag and sketch GEMMs */
  uint64_t seed;
  ssi_stab_params stab;
  int32_t small;           /* ssi_small_precision of the K x K SVD, A and eig(A) */
  int32_t reserved;
} ssi_job_desc;

/* Output sizes of a job: total pole slots and the matching phi length (floats). */
ssi_status ssi_job_sizes(const ssi_job_desc* job, int64_t* n_slots, int64_t* phi_floats);

/* poles/phi: device buffers of ssi_job_sizes() size.  S_out (optional, device, float64):
 * n_lags x k singular values.  Limits: k <= 512, k + oversample <= 16384, orders <= 512.
 * A range finder wider than the orders need is k = max order, oversample = K - k. */
ssi_status ssi_solve(ssi_ctx* ctx, const ssi_job_desc* job, ssi_pole* poles, float* phi,
                     double* S_out, void* stream);

/* ------------------------------------------------------------------------------
 * Several jobs in one call, their eigen-decompositions in one launch (the batching
 * pattern: "jobs of different sizes in one launch"; the paper solves one record at a
 * time and has no counterpart).  Each job's covariances, range finder and per-lag
 * factorisations run as in ssi_solve, on up to four internal streams forked from
 * `stream`. Then one k_eig launch (plus one for orders above 224, if any) and one
 * k_eig_vectors launch take every (job, lag, order) realisation of the batch, largest
 * orders first across the jobs. Then each job's stability criteria run on `stream`.
 * Results are identical to n_jobs separate ssi_solve calls: the same kernels compute
 * every item in the same arithmetic. Jobs may differ in channels, record length, lags,
 * orders, k and GEMM precision; all must use SSI_SMALL_FP32 (the FP64 eigensolver runs
 * one job at a time), else SSI_E_INVALID. poles[i], phi[i]: device buffers of
 * ssi_job_sizes(&jobs[i]) size; S_out (optional) per job as in ssi_solve.
 * 1 <= n_jobs <= SSI_BATCH_MAX. Buffers are kept in the context for the next call; like
 * ssi_solve, one call at a time per context.
 * ---------------------------------------------------------------------------- */
#define SSI_BATCH_MAX 64
ssi_status ssi_solve_batch(ssi_ctx* ctx, int n_jobs, const ssi_job_desc* jobs,
                           ssi_pole* const* poles, float* const* phi, double* const* S_out,
                           void* stream);

/* ------------------------------------------------------------------------------
 * Autotuner of a job shape's plan choices (the batching pattern: tile and split shapes
 * picked from timed candidates; the paper has no counterpart).  Four choices are made
 * by cost models otherwise: the lag GEMM's samples per time split, the Toeplitz GEMMs'
 * reduction splits, the K x K Jacobi's columns per block and the sketch QR's row chunks
 * per CTA.  ssi_autotune runs solves of `job` (its record included) on an internal
 * stream, one choice at a time, each candidate once untimed and twice timed by the stage
 * profiler, keeps the fastest (the QR grid is tuned for the shared device only: 2 or 4
 * chunks per CTA when the context expects several solves at once; a solve alone takes the
 * whole-device grid), and stores the four values in the context under
 * the job's shape (l, N, lags, k, oversample, precisions); later ssi_solve calls and
 * serving jobs of that shape use them.  The results change only by rounding (the split
 * and block structure orders the sums; the QR grid changes none of its sums).
 * Synchronous; call it before serving starts.  ssi_tuning_get returns the stored values
 * (SSI_E_NOTFOUND if the shape was never tuned); ssi_tuning_set stores values, e.g. those
 * tuned on another context (0 = the model's choice).
 * ---------------------------------------------------------------------------- */
typedef struct {
  int32_t cov_rows_per_split;   /* lag GEMM: samples per FP32 partial sum */
  int32_t sketch_splits;        /* Toeplitz GEMMs: reduction splits */
  int32_t jacobi_block;         /* K x K Jacobi: columns per block */
  int32_t qr_chunks_per_cta;    /* sketch QR under concurrency: row chunks (one per SM) per CTA */
  double stage_ms[4];           /* ms per solve of each stage with the chosen value */
} ssi_tuning;
ssi_status ssi_autotune(ssi_ctx* ctx, const ssi_job_desc* job, ssi_tuning* out);
ssi_status ssi_tuning_get(ssi_ctx* ctx, const ssi_job_desc* job, ssi_tuning* out);
ssi_status ssi_tuning_set(ssi_ctx* ctx, const ssi_job_desc* job, const ssi_tuning* in);

/* Synchronise `stream` and report device-side status raised by earlier asynchronous
 * calls of this context on it (SSI_E_TIMEOUT for a bounded wait that ran out,
 * SSI_E_NOTCONVERGED for an iteration cap).  Clears the status. */
ssi_status ssi_sync_status(ssi_ctx* ctx, void* stream);

/* ------------------------------------------------------------------------------
 * Serving: continuous batching of solves.  ssi_submit copies the descriptor
 * (and the host record, when y_on_host) and returns at once; a scheduler thread
 * admits queued jobs when a slot and enough of the HBM budget are free, runs
 * each admitted job on its own stream so their kernels overlap, and keeps the
 * job's covariances, sketches and results resident until ssi_release.
 * ssi_submit returns SSI_E_BUSY when the queue is full.
 * ssi_poll waits up to timeout_ms (0 = just test, <0 = forever) for job_id and
 * then returns host pointers owned by the context (valid until ssi_release):
 * the pole records and phi values, and the job's latency in microseconds from
 * submission to completion.
 * ---------------------------------------------------------------------------- */
ssi_status ssi_serve_config(ssi_ctx* ctx, int max_slots, int max_queue);
ssi_status ssi_submit(ssi_ctx* ctx, const ssi_job_desc* job, uint64_t* job_id);
ssi_status ssi_poll(ssi_ctx* ctx, uint64_t job_id, int timeout_ms, const ssi_pole** poles,
                    const float** phi, int64_t* n_slots, double* latency_us);
ssi_status ssi_release(ssi_ctx* ctx, uint64_t job_id);

/* ------------------------------------------------------------------------------
 * Parameter rules of Sec. 3 (host functions, no device work).
 * Eq. (empirical_formula): kbar(T) = max(30 - 0.00156 T, 25) percent; k = ceil(kbar T / 100).
 * Eq. (jb), Eq. (jb_3D): jb = ceil(10 fs/(2 f0)), jb_min = ceil(9 fs/(2 f0)),
 * jb_max = ceil(beta jb_min); int() is read as the ceiling.
 * Eq. (tlag): tau = (2 jb - 1)/fs.
 * ---------------------------------------------------------------------------- */
ssi_status ssi_rank_rule(int64_t T_size, double* kbar_percent, int64_t* k);
ssi_status ssi_lag_rule(double fs, double f0, double beta, int* jb, int* jb_min, int* jb_max);
double ssi_time_lag(int jb, double fs);

#ifdef __cplusplus
}
#endif

#endif /* SSI_H */
