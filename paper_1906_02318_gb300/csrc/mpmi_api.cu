// C-ABI entry points of the MPMI-SC tick library (declared in include/mpmi.h).
//
// Host side: handle lifecycle, argument checks, the float64 fit, the safety-set
// preprocessing and the launch of the fused tick kernel.  Every step of a tick
// (sampling, lifting, prediction, safety, cost, argmin, decode) runs on the GPU
// in tick_kernel.cuh; the host only marshals arguments.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"
#include "tick_dispatch.cuh"

namespace mpmi {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

int fail(int code, const std::string& msg) {
  g_error = msg;
  return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(MPMI_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MPMI_CUDA(call, what)                  \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)


static bool budget_ok(mpmi_ctx* ctx, uint64_t bytes) {
  return ctx->budget == 0 || ctx->used + bytes <= ctx->budget;
}

// ---- kernel dispatch -------------------------------------------------------
static TickKernel pick_tick(int kind, int lanes, int cands, bool traj, bool noise) {
  return noise ? pick_tick_noise(kind, lanes, cands, traj)
               : pick_variant<false>(kind, lanes, cands, traj);
}

// Default launch shape (lanes, candidates per thread, block).  A tick is one
// warp's serial chain of H steps until the candidates fill the GPU several times
// over, so few candidates take more lanes each.  Measured on GB300 (race car,
// H = 60, CUDA events, L2 flushed): N = 1024 16 lanes 28 us; N = 4096 8 lanes
// 38 us against 47 (2 lanes) and 69 (1 lane); N = 8192 2 lanes 47 us against 62
// (8 lanes) and 69; N = 16384 2 lanes 60 us against 69 (1 lane); N = 32768 1 lane
// 103 us against 110 (2 lanes); from ~48k slots two candidates per thread.  The
// two-lane shape keeps two warps per SM sub-partition while they fit one wave
// (two 128-thread blocks per SM), hiding each other's latency.  Balance bot
// N <= 4096 with 4 lanes 12.6 against 13.4..14.1 us, else one lane.  Blocks of
// 128 threads (one warp per SM sub-partition per block) measured never slower
// than 64 or 256 (bot N = 8192..65536, race car N = 16384..65536), and fewer
// blocks stage K and the track grid fewer times.
constexpr int kDefaultBlock = 128;

// Threads per block the library picks for a shape.  The race car's one-lane
// shapes: where the warp-tiles fit one block of at most eight warps per SM,
// blocks of ceil(tiles / SMs) warps, one per SM, load the SMs more evenly than
// two four-warp blocks on some SMs and one on the rest (measured 4-10 % faster
// from 20k to 76k slots); everything else kDefaultBlock.
static int default_block(int kind, int lanes, int cands, long long n_slots, int sms) {
  if (kind == kCar && lanes == 1) {
    const long long tiles = (n_slots + 32LL * cands - 1) / (32LL * cands);
    const long long w = (tiles + sms - 1) / sms;
    if (w > 4 && w <= kMaxBlock / 32) return (int)(32 * w);
  }
  return kDefaultBlock;
}

static void default_shape(int kind, int n_slots, int sms, int* lanes, int* cands, int* block) {
  *cands = 1;
  if (kind == kCar) {
    const long long n = n_slots;
    if (n * 16 <= (long long)sms * 128) *lanes = 16;      // at most one warp per sub-partition
    else if (n * 8 <= (long long)sms * 256) *lanes = 8;   // up to ~2 warps per sub-partition
    else if (n <= (long long)sms * 128) *lanes = 2;       // two-lane warps fit one wave
    else {
      *lanes = 1;
      *cands = n > 48 * 1024 ? 2 : 1;
    }
  } else {
    *lanes = (kind == kBot && (long long)n_slots * 4 <= (long long)sms * 128) ? 4 : 1;
  }
  *block = default_block(kind, *lanes, *cands, n_slots, sms);
}

TickArgs make_tick_args(const mpmi_session* s, uint64_t tick) {
  const mpmi_model* m = s->model;
  TickArgs a;
  memset(&a, 0, sizeof(a));
  a.K = m->K32_dev;
  a.Ks = m->K32_dev + (size_t)m->n * m->n;
  a.Kp = m->K32_dev + 2 * (size_t)m->n * m->n;
  a.safety = m->dev_safety;
  a.kind = m->kind;
  a.n_samples = s->cfg.n_samples;
  a.n_slots = s->n_slots;
  a.horizon = s->cfg.horizon;
  a.include_user = s->cfg.include_user;
  a.sampler = s->cfg.sampler;
  for (int j = 0; j < MPMI_MAX_NU; ++j) {
    a.in_lo[j] = (float)s->cfg.input_lo[j];
    a.in_w[j] = (float)(s->cfg.input_hi[j] - s->cfg.input_lo[j]);
    a.in_lo64[j] = s->cfg.input_lo[j];
    a.in_hi64[j] = s->cfg.input_hi[j];
  }
  a.grid_g = s->grid_g;
  a.key0 = (uint32_t)(s->cfg.seed & 0xFFFFFFFFull);
  a.key1 = (uint32_t)(s->cfg.seed >> 32);
  a.t_lo = (uint32_t)(tick & 0xFFFFFFFFull);
  a.t_hi = (uint32_t)(tick >> 32);
  a.stream = s->cfg.stream_id;
  a.tick = tick;
  a.scratch = s->scratch_dev;
  for (int j = 0; j < MPMI_MAX_NX; ++j) a.noise_sigma[j] = s->noise_sigma[j];
  a.n_noise = s->n_noise;
  a.withhold_staging = s->withhold_staging;
  if (s->rollout == MPMI_ROLLOUT_FACTORED) {
    // read-outs: the position when a track is set, then every bounded coordinate
    a.ck = s->ck_dev;
    const DevSafety& ds = m->dev_safety;
    int r = 0;
    if (ds.has_track) {
      a.ro_idx[r++] = 0;
      a.ro_idx[r++] = 1;
    }
    for (int j = ds.has_track ? 2 : 0; j < m->nx; ++j)
      if (!isinf(ds.lo[j]) || !isinf(ds.hi[j])) a.ro_idx[r++] = j;
    a.ro_n = r;
  }
  return a;
}

// Persistent grid: no more blocks than are resident at once, and no more than
// the warp-tiles need.  Occupancy is cached per dynamic shared-memory size.
// Launch shape for a launch that evaluates few candidates (a screened list): more
// lanes per candidate shorten the serial H-step chain each candidate carries.
static void small_shape(int kind, int list_lanes, int* lanes, int* cands, int* block) {
  *cands = 1;
  *block = 128;
  *lanes = kind == kCar ? (list_lanes == 16 ? 16 : 8) : (kind == kBot ? 4 : 1);
}

// ---- persistent host ticks ----------------------------------------------------
// The resident kernel (persistent.cu) takes commands from the session's mailbox.
// Word 0 holds the number of the last command posted; the host posts command q
// by a compare-and-swap from q - 1, which fails only if the kernel has marked
// the word as exited after its idle limit (then the host waits for the exit and
// relaunches).  A stop request is a flag or-ed into the word; the kernel still
// finishes a command posted before it.

// Stops the resident kernel, if any, and waits for it to exit.
static int persist_stop(mpmi_session* s) {
  if (!s->persist_running) return MPMI_OK;
  __atomic_fetch_or(&s->mbox_host[0], kCmdStop, __ATOMIC_SEQ_CST);
  s->persist_running = false;
  MPMI_CUDA(cudaEventSynchronize(s->persist_done), "waiting for the resident tick kernel to stop");
  return MPMI_OK;
}

// Launches the resident kernel; commands numbered above `start` are new to it.
static int persist_start(mpmi_session* s, cudaStream_t st, unsigned long long start) {
  MPMI_CUDA(cudaEventSynchronize(s->persist_done), "waiting for the previous resident kernel");
  __atomic_store_n(&s->mbox_host[0], start, __ATOMIC_SEQ_CST);
  for (int j = 0; j < kCmdWords; ++j) s->cmd_init[j] = 0;
  s->cmd_init[0] = start;
  MPMI_CUDA(cudaMemcpyAsync(s->cmd_dev, s->cmd_init, sizeof(s->cmd_init),
                            cudaMemcpyHostToDevice, s->persist_stream),
            "initialising the resident kernel's command copy");
  // order behind a launched tick that may still be finishing and behind earlier
  // work on the caller's stream
  if (s->tail_pending) {
    MPMI_CUDA(cudaStreamWaitEvent(s->persist_stream, s->done, 0), "cudaStreamWaitEvent");
    s->tail_pending = false;
  }
  MPMI_CUDA(cudaEventRecord(s->done, st), "cudaEventRecord");
  MPMI_CUDA(cudaStreamWaitEvent(s->persist_stream, s->done, 0), "cudaStreamWaitEvent");
  TickArgs a = make_tick_args(s, 0);
  a.result = s->result_map;
  a.seq_out = s->seq_map;
  PersistArgs p;
  p.mbox = s->mbox_map;
  p.cmd = s->cmd_dev;
  p.start_seq = start;
  p.idle_ns = s->persist_idle_ns;
  const int rc = launch_persistent(s, a, p);
  if (rc != MPMI_OK) return rc;
  MPMI_CUDA(cudaEventRecord(s->persist_done, s->persist_stream), "cudaEventRecord");
  s->persist_running = true;
  return MPMI_OK;
}

// Posts command `seq` (mailbox words 1.. already written), relaunching the
// resident kernel where it is not running.
static int persist_post(mpmi_session* s, cudaStream_t st, unsigned long long seq) {
  for (int attempt = 0; attempt < 3; ++attempt) {
    if (!s->persist_running) {
      const int rc = persist_start(s, st, seq - 1);
      if (rc != MPMI_OK) return rc;
    }
    unsigned long long expect = seq - 1;
    if (__atomic_compare_exchange_n(&s->mbox_host[0], &expect, seq, false, __ATOMIC_SEQ_CST,
                                    __ATOMIC_SEQ_CST))
      return MPMI_OK;
    // the kernel exited after its idle limit just before the command
    s->persist_running = false;
  }
  return fail(MPMI_E_CUDA, "persistent tick: the resident kernel keeps exiting before a command");
}

// Waits for the completion word of the tick in flight (zero-copy ticks): true
// once it holds the tick's number, false after `limit`.
static bool poll_published(const mpmi_session* s, std::chrono::nanoseconds limit) {
  const volatile unsigned long long* w = s->seq_host;
  const auto t0 = std::chrono::steady_clock::now();
  for (unsigned long i = 0;; ++i) {
    if (*w == s->seq) {
      std::atomic_thread_fence(std::memory_order_acquire);
      return true;
    }
    if ((i & 1023) == 1023 && std::chrono::steady_clock::now() - t0 > limit) return false;
  }
}

// The result of a tick posted to the resident kernel: polls for the idle limit
// plus a second, then stops the kernel (which finishes the command first) and
// looks once more.
static int persist_wait(mpmi_session* s) {
  if (poll_published(s, std::chrono::nanoseconds(s->persist_idle_ns) + std::chrono::seconds(1)))
    return MPMI_OK;
  const int rc = persist_stop(s);
  if (poll_published(s, std::chrono::nanoseconds(0))) return MPMI_OK;
  if (rc != MPMI_OK) return rc;
  return fail(MPMI_E_TIMEOUT, "persistent tick: no result within the idle limit plus a second");
}

// A host tick (results through select_input) may start once the previous one
// has finished: wait for it if it is still in flight.
int host_tick_begin(mpmi_session* s) {
  if (!s->in_flight) return MPMI_OK;
  if (s->persist_posted) {
    const int rc = persist_wait(s);
    if (rc != MPMI_OK) return rc;
  } else {
    MPMI_CUDA(cudaEventSynchronize(s->done), "waiting for the previous tick");
  }
  s->in_flight = false;
  s->persist_posted = false;
  return MPMI_OK;
}

// After a host tick's launches on st: the event select_input falls back to.
int host_tick_end(mpmi_session* s, cudaStream_t st) {
  MPMI_CUDA(cudaEventRecord(s->done, st), "cudaEventRecord");
  s->in_flight = true;
  return MPMI_OK;
}

int launch_tick_args(mpmi_session* s, TickArgs& a, bool traj, cudaStream_t st, int n_hint,
                     int list_lanes) {
  // a launched tick shares the session's reduction record with the resident kernel
  if (s->persist_running) {
    const int rc = persist_stop(s);
    if (rc != MPMI_OK) return rc;
  }
  if (s->tail_pending) {
    // the previous host tick's kernel may still be finishing: order behind it
    const cudaError_t e = cudaStreamWaitEvent(st, s->done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    s->tail_pending = false;
  }
  int lanes = s->lanes, cands = s->cands, block = s->block;
  // a device-side list short enough that 8 lanes per candidate still fit one wave;
  // n_hint < 0: a list of unknown length (grid for every slot, idle blocks leave)
  const bool small = a.slot_list != nullptr &&
                     (n_hint < 0 || (n_hint > 0 && (long long)n_hint * 8 <=
                                                       (long long)s->ctx->sm_count * 512));
  if (s->rollout == MPMI_ROLLOUT_TENSOR) {
    if (a.n_noise > 0 && a.tick >= (1ull << 48))
      return fail(MPMI_E_INVALID_ARG, "ticks with noise must stay below 2^48");
    return launch_tensor(s, a, traj, st, n_hint);
  }
  if (s->rollout == MPMI_ROLLOUT_FACTORED) {
    if (traj) return fail(MPMI_E_UNSUPPORTED, "the factorised rollout records no trajectories");
    if (a.n_noise > 0) return fail(MPMI_E_UNSUPPORTED, "the factorised rollout has no noise");
    return launch_factored(s, a, st, n_hint);
  }
  if (small) small_shape(s->model->kind, list_lanes, &lanes, &cands, &block);
  const bool noise = a.n_noise > 0;
  if (noise && a.tick >= (1ull << 48))
    return fail(MPMI_E_INVALID_ARG, "ticks with noise must stay below 2^48");
  TickKernel k = pick_tick(s->model->kind, lanes, cands, traj, noise);
  if (!k.fn) return fail(MPMI_E_UNSUPPORTED, "tick kernel not compiled for this launch shape");
  const size_t smem = k.k_smem + (a.safety.has_track ? (size_t)a.safety.track.blob_bytes : 0);
  const int t = (traj ? 1 : 0) + (small ? 2 : 0) + (noise ? 4 : 0) + (small && lanes == 16 ? 8 : 0);
  if (s->max_grid[t] == 0 || s->grid_smem[t] != smem) {
    // static (lane exchange) plus dynamic shared memory may pass the 48 KB default
    if (smem > 0) {
      cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(k.k_smem + kMaxTrackBytes));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    }
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (nb < 1) return fail(MPMI_E_UNSUPPORTED, "tick kernel cannot be resident with this block");
    s->max_grid[t] = nb * s->ctx->sm_count;
    s->grid_smem[t] = smem;
  }
  const int wpb = block / 32;
  const int per_warp = 32 / lanes * cands;
  const int n_work = (n_hint > 0 && n_hint < s->n_slots) ? n_hint : s->n_slots;
  const int n_wtiles = (n_work + per_warp - 1) / per_warp;
  int grid = (n_wtiles + wpb - 1) / wpb;
  if (grid > s->max_grid[t]) grid = s->max_grid[t];
  k.launch(a, grid, block, smem, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tick kernel launch");
  return MPMI_OK;
}

static int check_finite(const double* v, int n, const char* what) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return fail(MPMI_E_NONFINITE, std::string(what) + " holds NaN/Inf");
  return MPMI_OK;
}

static int grid_points(int n, int nu) {
  if (n <= 0) return 0;
  int g = (int)llround(pow((double)n, 1.0 / nu));
  for (int c = g > 2 ? g - 2 : 1; c <= g + 2; ++c) {
    long long p = 1;
    for (int j = 0; j < nu; ++j) p *= c;
    if (p == n) return c;
  }
  return -1;
}

static void free_model_device(mpmi_model* m) {
  cudaFree(m->K32_dev);
  cudaFree(m->track_dev);
  m->K32_dev = nullptr;
  m->track_dev = nullptr;
}

// 16-byte words of the pair layout of K for a basis (0 where no shape uses it).
static size_t kpair_words(int kind) {
  return kind == kCar ? (size_t)KPair<kCar>::WORDS : 0;
}

// K in float32: row-major, then with each row's columns in staging order (the
// layout the row-split shared-memory shapes copy in one piece), then the pair
// layout of the one-lane shared-memory shapes (race car).
static int model_upload(mpmi_ctx* ctx, mpmi_model* m) {
  const size_t nn = (size_t)m->n * m->n;
  const size_t np = 4 * kpair_words(m->kind);
  const size_t bytes = sizeof(float) * (2 * nn + np);
  if (!budget_ok(ctx, bytes)) return fail(MPMI_E_OOM, "model exceeds the memory budget");
  std::vector<float> k32(2 * nn + np);
  for (size_t i = 0; i < nn; ++i) k32[i] = (float)m->K64[i];
  for (int r = 0; r < m->n; ++r)
    for (int p = 0; p < m->n; ++p)
      k32[nn + (size_t)r * m->n + p] = (float)m->K64[(size_t)r * m->n + staged_col(m->kind, m->n, p)];
  for (size_t i = 0; i < np; ++i) {
    const int stride = KPair<kCar>::STRIDE;
    const int e = (int)(i & 3), w = (int)(i / 4) % stride, p = (int)(i / 4) / stride;
    k32[2 * nn + i] = kpair_value(m->kind, m->n, k32.data(), p, w, e);
  }
  if (cudaMalloc(&m->K32_dev, bytes) != cudaSuccess)
    return fail(MPMI_E_OOM, "cudaMalloc of K failed");
  MPMI_CUDA(cudaMemcpy(m->K32_dev, k32.data(), bytes, cudaMemcpyHostToDevice), "upload K");
  m->bytes += bytes;
  ctx->used += bytes;
  return MPMI_OK;
}

// Test hook: the raw Philox4x32-10 words of n (counter, key) records, each six
// words c0 c1 c2 c3 k0 k1, through the same device function the sampler uses.
static __global__ void philox_words_kernel(const uint32_t* __restrict__ in, int64_t n,
                                           uint32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t* r = in + 6 * i;
  const U32x4 w = philox4x32_10(U32x4{r[0], r[1], r[2], r[3]}, r[4], r[5]);
  out[4 * i + 0] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}

}  // namespace mpmi

using namespace mpmi;

extern "C" {

const char* mpmi_last_error(void) { return g_error.c_str(); }

const char* mpmi_version(void) { return "mpmi-gb300 1.0 (sm_103a)"; }

int mpmi_create(int32_t device, uint64_t mem_budget_bytes, mpmi_ctx** out) {
  if (!out) return fail(MPMI_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(MPMI_E_INVALID_ARG, "no such CUDA device");
  DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaDeviceProp prop;
  MPMI_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  if (prop.major < 10) return fail(MPMI_E_UNSUPPORTED, "library is built for sm_103a");
  mpmi_ctx* c = new mpmi_ctx();
  c->device = device;
  c->budget = mem_budget_bytes;
  c->sm_count = prop.multiProcessorCount;
  *out = c;
  return MPMI_OK;
}

void mpmi_destroy(mpmi_ctx* ctx) { delete ctx; }

uint64_t mpmi_memory_in_use(const mpmi_ctx* ctx) { return ctx ? ctx->used : 0; }

int mpmi_fit_model(mpmi_ctx* ctx, const mpmi_basis_desc* basis, const double* x,
                   const double* u, const double* x_next, int64_t m, mpmi_model** out,
                   double* residual_out) {
  if (!ctx || !basis || !x || !u || !x_next || !out)
    return fail(MPMI_E_INVALID_ARG, "fit_model: NULL argument");
  *out = nullptr;
  const int kind = basis_kind(basis->basis, basis->nx, basis->nu);
  if (kind < 0) return fail(MPMI_E_UNSUPPORTED, "fit_model: basis/dimensions not compiled");
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m <= 0) return fail(MPMI_E_INVALID_ARG, "fit_model: no transitions");
  int rc;
  if ((rc = check_finite(x, (int)(m * nx), "fit_model: x")) != MPMI_OK) return rc;
  if ((rc = check_finite(u, (int)(m * nu), "fit_model: u")) != MPMI_OK) return rc;
  if ((rc = check_finite(x_next, (int)(m * nx), "fit_model: x_next")) != MPMI_OK) return rc;
  std::vector<double> K;
  std::string err;
  double res = 0.0;
  rc = fit_householder(kind, x, u, x_next, m, &K, &res, &err);
  if (rc != MPMI_OK) return fail(rc, err);
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  mpmi_model* md = new mpmi_model();
  md->ctx = ctx;
  md->basis = basis->basis;
  md->kind = kind;
  md->n = n; md->nx = nx; md->nu = nu; md->np = np;
  md->K64 = K;
  if ((rc = model_upload(ctx, md)) != MPMI_OK) {
    free_model_device(md);
    delete md;
    return rc;
  }
  if (residual_out) *residual_out = res;
  *out = md;
  return MPMI_OK;
}

int mpmi_fit_operator(const mpmi_basis_desc* basis, const double* x, const double* u,
                      const double* x_next, int64_t m, double* K_out, double* residual_out) {
  if (!basis || !x || !u || !x_next || !K_out)
    return fail(MPMI_E_INVALID_ARG, "fit_operator: NULL argument");
  const int kind = basis_kind(basis->basis, basis->nx, basis->nu);
  if (kind < 0) return fail(MPMI_E_UNSUPPORTED, "fit_operator: basis/dimensions not compiled");
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m <= 0) return fail(MPMI_E_INVALID_ARG, "fit_operator: no transitions");
  int rc;
  if ((rc = check_finite(x, (int)(m * nx), "fit_operator: x")) != MPMI_OK) return rc;
  if ((rc = check_finite(u, (int)(m * nu), "fit_operator: u")) != MPMI_OK) return rc;
  if ((rc = check_finite(x_next, (int)(m * nx), "fit_operator: x_next")) != MPMI_OK) return rc;
  std::vector<double> K;
  std::string err;
  double res = 0.0;
  rc = fit_householder(kind, x, u, x_next, m, &K, &res, &err);
  if (rc != MPMI_OK) return fail(rc, err);
  memcpy(K_out, K.data(), sizeof(double) * K.size());
  if (residual_out) *residual_out = res;
  return MPMI_OK;
}

int mpmi_fit_operator_sparse(const mpmi_basis_desc* basis, const double* x, const double* u,
                             const double* x_next, int64_t m, double gamma, double rho,
                             int32_t iters, double* K_out, uint8_t* support_out,
                             double* residual_out) {
  if (!basis || !x || !u || !x_next || !K_out)
    return fail(MPMI_E_INVALID_ARG, "fit_operator_sparse: NULL argument");
  const int kind = basis_kind(basis->basis, basis->nx, basis->nu);
  if (kind < 0) return fail(MPMI_E_UNSUPPORTED, "fit_operator_sparse: basis/dimensions not compiled");
  if (!(gamma >= 0.0) || !std::isfinite(gamma))
    return fail(MPMI_E_INVALID_ARG, "fit_operator_sparse: gamma must be finite and >= 0");
  if (!(rho > 0.0) || !std::isfinite(rho))
    return fail(MPMI_E_INVALID_ARG, "fit_operator_sparse: rho must be finite and > 0");
  if (iters < 1) return fail(MPMI_E_INVALID_ARG, "fit_operator_sparse: iters must be >= 1");
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (m <= 0) return fail(MPMI_E_INVALID_ARG, "fit_operator_sparse: no transitions");
  int rc;
  if ((rc = check_finite(x, (int)(m * nx), "fit_operator_sparse: x")) != MPMI_OK) return rc;
  if ((rc = check_finite(u, (int)(m * nu), "fit_operator_sparse: u")) != MPMI_OK) return rc;
  if ((rc = check_finite(x_next, (int)(m * nx), "fit_operator_sparse: x_next")) != MPMI_OK)
    return rc;
  std::vector<double> K;
  std::vector<unsigned char> sup;
  std::string err;
  double res = 0.0;
  rc = fit_sparse(kind, x, u, x_next, m, gamma, rho, iters, &K, &sup, &res, &err);
  if (rc != MPMI_OK) return fail(rc, err);
  memcpy(K_out, K.data(), sizeof(double) * K.size());
  if (support_out)
    for (int j = 0; j < n; ++j) support_out[j] = sup[j];
  if (residual_out) *residual_out = res;
  return MPMI_OK;
}

int mpmi_debug_track_query(const double* track_xy, int32_t n_track, double half_width,
                           const float* points, int64_t n_points, uint8_t* on_road) {
  if (!track_xy || (n_points > 0 && (!points || !on_road)) || n_points < 0)
    return fail(MPMI_E_INVALID_ARG, "debug_track_query: NULL argument or negative count");
  if (n_track < 3 || n_track > MPMI_MAX_TRACK_VERTICES)
    return fail(MPMI_E_INVALID_ARG, "debug_track_query: n_track out of range");
  if (!(half_width > 0.0) || !std::isfinite(half_width))
    return fail(MPMI_E_INVALID_ARG, "debug_track_query: half width must be > 0");
  std::string err;
  const int rc = track_query_host(track_xy, n_track, half_width, points, n_points, on_road, &err);
  return rc == MPMI_OK ? MPMI_OK : fail(rc, err);
}

int mpmi_model_from_operator(mpmi_ctx* ctx, const mpmi_basis_desc* basis, const double* K,
                             mpmi_model** out) {
  if (!ctx || !basis || !K || !out) return fail(MPMI_E_INVALID_ARG, "NULL argument");
  *out = nullptr;
  const int kind = basis_kind(basis->basis, basis->nx, basis->nu);
  if (kind < 0) return fail(MPMI_E_UNSUPPORTED, "basis/dimensions not compiled");
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  int rc = check_finite(K, n * n, "K");
  if (rc != MPMI_OK) return rc;
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  mpmi_model* md = new mpmi_model();
  md->ctx = ctx;
  md->basis = basis->basis;
  md->kind = kind;
  md->n = n; md->nx = nx; md->nu = nu; md->np = np;
  md->K64.assign(K, K + n * n);
  // rows of held input features must be unit rows (the input is held over the
  // horizon); rounding-level deviations are set exact, anything else is refused
  for (int j = 0; j < n; ++j) {
    if (!held_feature(kind, j)) continue;
    for (int k = 0; k < n; ++k) {
      const double want = k == j ? 1.0 : 0.0;
      if (fabs(md->K64[(size_t)j * n + k] - want) > 1e-6) {
        delete md;
        return fail(MPMI_E_INVALID_ARG,
                    "model_from_operator: row " + std::to_string(j) +
                        " belongs to a held input feature and must be a unit row "
                        "(the input is held over the horizon)");
      }
      md->K64[(size_t)j * n + k] = want;
    }
  }
  if ((rc = model_upload(ctx, md)) != MPMI_OK) {
    free_model_device(md);
    delete md;
    return rc;
  }
  *out = md;
  return MPMI_OK;
}

int mpmi_model_get_operator(const mpmi_model* model, double* K_out, int32_t* n_out) {
  if (!model) return fail(MPMI_E_INVALID_ARG, "model is NULL");
  if (n_out) *n_out = model->n;
  if (K_out) memcpy(K_out, model->K64.data(), sizeof(double) * model->K64.size());
  return MPMI_OK;
}

void mpmi_model_free(mpmi_model* model) {
  if (!model) return;
  DeviceGuard guard(model->ctx->device);
  free_model_device(model);
  model->ctx->used -= model->bytes;
  delete model;
}

int mpmi_set_safety_set(mpmi_model* model, const mpmi_safety_spec* spec) {
  if (!model || !spec) return fail(MPMI_E_INVALID_ARG, "set_safety_set: NULL argument");
  if (!(spec->inflation >= 0.0) || !isfinite(spec->inflation))
    return fail(MPMI_E_INVALID_ARG, "set_safety_set: inflation must be finite and >= 0");
  DevSafety ds;
  memset(&ds, 0, sizeof(ds));
  for (int j = 0; j < MPMI_MAX_NX; ++j) {
    const double lo = spec->state_lo[j], hi = spec->state_hi[j];
    if (isnan(lo) || isnan(hi)) return fail(MPMI_E_INVALID_ARG, "set_safety_set: NaN bound");
    if (j >= model->nx) {
      ds.lo[j] = -INFINITY;
      ds.hi[j] = INFINITY;
      continue;
    }
    ds.lo[j] = (float)(lo + spec->inflation);
    ds.hi[j] = (float)(hi - spec->inflation);
  }
  TrackGrid grid;
  const bool has_track = spec->track_xy != nullptr;
  if (has_track) {
    if (model->kind != kCar)
      return fail(MPMI_E_UNSUPPORTED, "set_safety_set: track test is compiled for the race car");
    if (spec->track_x != 0 || spec->track_y != 1)
      return fail(MPMI_E_UNSUPPORTED, "set_safety_set: track position must be state (0, 1)");
    if (spec->n_track < 3 || spec->n_track > MPMI_MAX_TRACK_VERTICES)
      return fail(MPMI_E_INVALID_ARG, "set_safety_set: n_track out of range");
    if (!(spec->track_half_width > 0.0) || !isfinite(spec->track_half_width))
      return fail(MPMI_E_INVALID_ARG, "set_safety_set: track half width must be > 0");
    std::string err;
    int rc = build_track_grid(spec->track_xy, spec->n_track,
                              spec->track_half_width - spec->inflation, &grid, &err);
    if (rc != MPMI_OK) return fail(rc, err);
  }
  mpmi_ctx* ctx = model->ctx;
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  // ticks in flight may still read the previous grid
  MPMI_CUDA(cudaDeviceSynchronize(), "set_safety_set: waiting for ticks in flight");
  cudaFree(model->track_dev);
  model->track_dev = nullptr;
  model->bytes -= model->track_bytes;
  ctx->used -= model->track_bytes;
  model->track_bytes = 0;
  if (has_track) {
    const uint64_t total = grid.blob.size();
    if (!budget_ok(ctx, total)) return fail(MPMI_E_OOM, "track grid exceeds the memory budget");
    if (cudaMalloc(&model->track_dev, total) != cudaSuccess)
      return fail(MPMI_E_OOM, "cudaMalloc of the track grid failed");
    MPMI_CUDA(cudaMemcpy(model->track_dev, grid.blob.data(), total, cudaMemcpyHostToDevice),
              "upload the track grid");
    model->track_bytes = total;
    model->bytes += total;
    ctx->used += total;
    const double w = spec->track_half_width - spec->inflation;
    ds.has_track = 1;
    ds.track.blob = model->track_dev;
    ds.track.blob_bytes = (int)total;
    ds.track.off_list = grid.off_list;
    ds.track.off_seg = grid.off_seg;
    ds.track.off_inv = grid.off_inv;
    ds.track.gx0 = (float)grid.gx0;
    ds.track.gy0 = (float)grid.gy0;
    ds.track.inv_h = (float)(1.0 / grid.h);
    ds.track.gnx = grid.gnx;
    ds.track.gny = grid.gny;
    ds.track.w2 = (float)(w * w);
    model->track_host.assign(spec->track_xy, spec->track_xy + 2 * spec->n_track);
  } else {
    model->track_host.clear();
  }
  model->spec = *spec;
  model->spec.track_xy = nullptr;
  model->dev_safety = ds;
  model->has_safety = true;
  return MPMI_OK;
}

int mpmi_session_open(mpmi_ctx* ctx, const mpmi_model* model, const mpmi_session_config* cfg,
                      mpmi_session** out) {
  if (!ctx || !model || !cfg || !out) return fail(MPMI_E_INVALID_ARG, "session_open: NULL argument");
  *out = nullptr;
  if (model->ctx != ctx) return fail(MPMI_E_INVALID_ARG, "session_open: model from another context");
  if (!model->has_safety)
    return fail(MPMI_E_INVALID_ARG, "session_open: call set_safety_set on the model first");
  if (cfg->n_samples < 0) return fail(MPMI_E_INVALID_ARG, "session_open: n_samples < 0");
  if (cfg->horizon < 1 || cfg->horizon > MPMI_MAX_HORIZON)
    return fail(MPMI_E_INVALID_ARG, "session_open: horizon out of range 1..511");
  if (cfg->include_user != 0 && cfg->include_user != 1)
    return fail(MPMI_E_INVALID_ARG, "session_open: include_user must be 0 or 1");
  const long long slots = (long long)cfg->n_samples + cfg->include_user;
  if (slots < 1 || slots > MPMI_MAX_SLOTS)
    return fail(MPMI_E_INVALID_ARG, "session_open: number of slots out of range");
  if (cfg->sampler < MPMI_SAMPLER_UNIFORM || cfg->sampler > MPMI_SAMPLER_EXTERNAL)
    return fail(MPMI_E_INVALID_ARG, "session_open: unknown sampler");
  for (int j = 0; j < model->nu; ++j) {
    if (!isfinite(cfg->input_lo[j]) || !isfinite(cfg->input_hi[j]) ||
        !(cfg->input_lo[j] < cfg->input_hi[j]))
      return fail(MPMI_E_INVALID_ARG, "session_open: input box must be finite with lo < hi");
  }
  int gg = 0;
  if (cfg->sampler == MPMI_SAMPLER_GRID) {
    gg = grid_points(cfg->n_samples, model->nu);
    if (gg <= 0) return fail(MPMI_E_INVALID_ARG, "session_open: grid sampling needs N = G^M");
  }
  int lanes = cfg->lanes, cands = cfg->cands_per_thread, block = cfg->block;
  if (lanes == 0 && cands == 0 && block == 0) {
    // a shape the autotuner measured for this configuration, if any
    for (const auto& t : ctx->tuned)
      if (t.kind == model->kind && t.n_slots == (int)slots && t.horizon == cfg->horizon) {
        lanes = t.lanes;
        cands = t.cands;
        block = t.block;
        break;
      }
  }
  if (lanes == 0 && cands > 1) lanes = 1;  // several candidates per thread need one lane
  if (lanes == 0) {
    int dl, dc, db;
    default_shape(model->kind, (int)slots, ctx->sm_count, &dl, &dc, &db);
    lanes = dl;
    if (cands == 0) cands = dc;
  } else {
    if (cands == 0) cands = (lanes == 1 && model->kind == kCar && slots > 48 * 1024) ? 2 : 1;
  }
  if (block == 0) block = default_block(model->kind, lanes, cands, slots, ctx->sm_count);
  if (block % 32 != 0 || block < 32 || block > kMaxBlock)
    return fail(MPMI_E_INVALID_ARG, "session_open: block must be a multiple of 32 in 32..256");
  if (!pick_tick(model->kind, lanes, cands, false, false).fn)
    return fail(MPMI_E_UNSUPPORTED, "session_open: launch shape (lanes, candidates per thread) "
                                    "not compiled for this basis");
  const uint64_t bytes = sizeof(TickScratch) + sizeof(mpmi_result) + 16 * sizeof(double);
  if (!budget_ok(ctx, bytes)) return fail(MPMI_E_OOM, "session exceeds the memory budget");
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  mpmi_session* s = new mpmi_session();
  s->ctx = ctx;
  s->model = model;
  s->cfg = *cfg;
  s->n_slots = (int)slots;
  s->lanes = lanes;
  s->cands = cands;
  s->block = block;
  s->grid_g = gg;
  auto cleanup = [&](int code, const char* msg) {
    cudaFree(s->scratch_dev);
    cudaFree(s->result_dev);
    cudaFree(s->in_dev);
    cudaFreeHost(s->in_host);
    cudaFreeHost(s->result_host);
    cudaFreeHost(s->seq_host);
    if (s->done) cudaEventDestroy(s->done);
    delete s;
    return fail(code, msg);
  };
  if (cudaMalloc(&s->scratch_dev, sizeof(TickScratch)) != cudaSuccess ||
      cudaMalloc(&s->result_dev, sizeof(mpmi_result)) != cudaSuccess ||
      cudaMalloc(&s->in_dev, 16 * sizeof(double)) != cudaSuccess)
    return cleanup(MPMI_E_OOM, "session_open: cudaMalloc failed");
  if (cudaMallocHost(&s->in_host, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&s->result_host, sizeof(mpmi_result)) != cudaSuccess)
    return cleanup(MPMI_E_OOM, "session_open: pinned allocation failed");
  if (cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(MPMI_E_CUDA, "session_open: cudaEventCreate failed");
  // host ticks read x_t, u_h from the pinned staging buffer and write the result
  // into pinned memory directly (zero-copy over the host link) where the device
  // can map host memory; otherwise they copy both ways
  {
    int can_map = 0;
    if (cudaDeviceGetAttribute(&can_map, cudaDevAttrCanMapHostMemory, ctx->device) == cudaSuccess &&
        can_map && cudaMallocHost(&s->seq_host, sizeof(unsigned long long)) == cudaSuccess &&
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->in_map), s->in_host, 0) ==
            cudaSuccess &&
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->result_map), s->result_host, 0) ==
            cudaSuccess &&
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->seq_map), s->seq_host, 0) ==
            cudaSuccess) {
      s->zero_copy = true;
      *s->seq_host = 0;
    }
    cudaGetLastError();
  }
  TickScratch init;
  memset(&init, 0, sizeof(init));
  init.key = ~0ull;
  if (cudaMemcpy(s->scratch_dev, &init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(s->result_dev, 0, sizeof(mpmi_result)) != cudaSuccess ||
      cudaMemset(s->in_dev, 0, 16 * sizeof(double)) != cudaSuccess)
    return cleanup(MPMI_E_CUDA, "session_open: initialising device state failed");
  memset(s->in_host, 0, 16 * sizeof(double));
  s->bytes = bytes;
  ctx->used += bytes;
  *out = s;
  return MPMI_OK;
}

void mpmi_session_close(mpmi_session* s) {
  if (!s) return;
  DeviceGuard guard(s->ctx->device);
  persist_stop(s);
  if (s->in_flight || s->tail_pending) cudaEventSynchronize(s->done);
  if (s->ck_dev) {
    cudaDeviceSynchronize();
    cudaFree(s->ck_dev);
    s->ctx->used -= s->ck_bytes;
  }
  cudaFree(s->scratch_dev);
  cudaFree(s->result_dev);
  cudaFree(s->in_dev);
  cudaFreeHost(s->in_host);
  cudaFreeHost(s->result_host);
  cudaFreeHost(s->seq_host);
  cudaEventDestroy(s->done);
  if (s->mbox_host) cudaFreeHost(s->mbox_host);
  if (s->cmd_dev) cudaFree(s->cmd_dev);
  if (s->persist_stream) cudaStreamDestroy(s->persist_stream);
  if (s->persist_done) cudaEventDestroy(s->persist_done);
  s->ctx->used -= s->bytes;
  delete s;
}

int mpmi_session_launch_shape(const mpmi_session* s, int32_t* lanes, int32_t* cands,
                              int32_t* block) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "session is NULL");
  if (lanes) *lanes = s->lanes;
  if (cands) *cands = s->cands;
  if (block) *block = s->block;
  return MPMI_OK;
}

int mpmi_session_set_noise(mpmi_session* s, const double* sigma, int32_t count) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "session is NULL");
  if (s->in_flight)
    return fail(MPMI_E_INVALID_ARG, "set_noise: a tick is in flight (call select_input first)");
  if (count < 0 || count > s->model->nx)
    return fail(MPMI_E_INVALID_ARG, "set_noise: count must be 0..the model's state dimension");
  if (count > 0 && !sigma) return fail(MPMI_E_INVALID_ARG, "set_noise: sigma is NULL");
  for (int j = 0; j < count; ++j) {
    if (!std::isfinite(sigma[j])) return fail(MPMI_E_NONFINITE, "set_noise: sigma not finite");
    if (sigma[j] < 0.0) return fail(MPMI_E_INVALID_ARG, "set_noise: sigma must be >= 0");
  }
  for (int j = 0; j < MPMI_MAX_NX; ++j) s->noise_sigma[j] = j < count ? (float)sigma[j] : 0.f;
  s->n_noise = count;
  return MPMI_OK;
}

int mpmi_session_set_rollout(mpmi_session* s, int32_t mode) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "session is NULL");
  if (mode != MPMI_ROLLOUT_FULL && mode != MPMI_ROLLOUT_FACTORED && mode != MPMI_ROLLOUT_TENSOR)
    return fail(MPMI_E_INVALID_ARG, "set_rollout: unknown mode");
  if (mode == MPMI_ROLLOUT_TENSOR && s->model->kind != kCar)
    return fail(MPMI_E_UNSUPPORTED, "set_rollout: the tensor-core rollout is compiled for the race car");
  if (s->in_flight)
    return fail(MPMI_E_INVALID_ARG, "set_rollout: a tick is in flight (call select_input first)");
  if (mode == s->rollout) return MPMI_OK;
  mpmi_ctx* ctx = s->ctx;
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  const int prc = persist_stop(s);  // the device-wide waits below would wait for it
  if (prc != MPMI_OK) return prc;
  if (mode == MPMI_ROLLOUT_FULL || mode == MPMI_ROLLOUT_TENSOR) {
    // device-resident ticks may still read the rows
    MPMI_CUDA(cudaDeviceSynchronize(), "set_rollout: waiting for ticks in flight");
    cudaFree(s->ck_dev);
    ctx->used -= s->ck_bytes;
    s->ck_dev = nullptr;
    s->ck_bytes = 0;
    s->rollout = mode;
    return MPMI_OK;
  }
  const mpmi_model* m = s->model;
  const uint64_t bytes = (uint64_t)s->cfg.horizon * m->nx * m->n * sizeof(float);
  if (!budget_ok(ctx, bytes)) return fail(MPMI_E_OOM, "set_rollout: exceeds the memory budget");
  float* ck = nullptr;
  if (cudaMalloc(&ck, bytes) != cudaSuccess)
    return fail(MPMI_E_OOM, "set_rollout: cudaMalloc failed");
  int rc = compute_powers(m->kind, m->K32_dev, s->cfg.horizon, ck, 0);
  if (rc == MPMI_OK) {
    const cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) rc = cuda_fail(e, "set_rollout: powers of K");
  }
  if (rc != MPMI_OK) {
    cudaFree(ck);
    return rc;
  }
  s->ck_dev = ck;
  s->ck_bytes = bytes;
  ctx->used += bytes;
  s->fact_grid = 0;
  s->rollout = mode;
  return MPMI_OK;
}

int mpmi_session_set_persistent(mpmi_session* s, int32_t on, double idle_ms) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "session is NULL");
  if (!(idle_ms == 0.0 || (idle_ms >= 1.0 && idle_ms <= 60000.0)))
    return fail(MPMI_E_INVALID_ARG, "set_persistent: idle_ms must be 0 or in 1..60000");
  DeviceGuard guard(s->ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  if (!on) {
    s->persist = false;
    return persist_stop(s);  // a command in flight is finished and published first
  }
  if (!s->zero_copy)
    return fail(MPMI_E_UNSUPPORTED, "set_persistent: the device cannot map host memory");
  int atomics = 0, coop = 0;
  if (cudaDeviceGetAttribute(&atomics, cudaDevAttrHostNativeAtomicSupported, s->ctx->device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPMI_E_CUDA, "set_persistent: device attributes");
  }
  if (!atomics)
    return fail(MPMI_E_UNSUPPORTED, "set_persistent: no native atomics on host memory");
  if (!coop) return fail(MPMI_E_UNSUPPORTED, "set_persistent: no cooperative launch");
  if (!persist_supported(s->model->kind, s->lanes, s->cands))
    return fail(MPMI_E_UNSUPPORTED, "set_persistent: no persistent form of this launch shape");
  if (!s->mbox_host) {
    const size_t bytes = kCmdWords * sizeof(unsigned long long);
    if (!budget_ok(s->ctx, bytes)) return fail(MPMI_E_OOM, "set_persistent: exceeds the memory budget");
    bool ok = cudaMallocHost(&s->mbox_host, bytes) == cudaSuccess &&
              cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->mbox_map), s->mbox_host, 0) ==
                  cudaSuccess &&
              cudaMalloc(&s->cmd_dev, bytes) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->persist_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->persist_done, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (s->mbox_host) cudaFreeHost(s->mbox_host);
      if (s->cmd_dev) cudaFree(s->cmd_dev);
      if (s->persist_stream) cudaStreamDestroy(s->persist_stream);
      if (s->persist_done) cudaEventDestroy(s->persist_done);
      s->mbox_host = nullptr;
      s->mbox_map = nullptr;
      s->cmd_dev = nullptr;
      s->persist_stream = nullptr;
      s->persist_done = nullptr;
      return fail(MPMI_E_OOM, "set_persistent: allocating the mailbox failed");
    }
    memset(s->mbox_host, 0, bytes);
    s->bytes += bytes;
    s->ctx->used += bytes;
  }
  const unsigned long long idle_ns =
      (unsigned long long)((idle_ms == 0.0 ? 1000.0 : idle_ms) * 1e6);
  if (s->persist_running && idle_ns != s->persist_idle_ns) {
    const int rc = persist_stop(s);  // the next tick relaunches with the new limit
    if (rc != MPMI_OK) return rc;
  }
  s->persist_idle_ns = idle_ns;
  s->persist = true;
  return MPMI_OK;
}

static int check_ext(const mpmi_session* s, const float* candidates_dev) {
  if (s->cfg.sampler == MPMI_SAMPLER_EXTERNAL && s->cfg.n_samples > 0 && !candidates_dev)
    return fail(MPMI_E_INVALID_ARG, "EXTERNAL sampler needs candidates_dev");
  if (s->cfg.sampler != MPMI_SAMPLER_EXTERNAL && candidates_dev)
    return fail(MPMI_E_INVALID_ARG, "candidates_dev given but the sampler is not EXTERNAL");
  return MPMI_OK;
}

int mpmi_evaluate_candidates(mpmi_session* s, const double* x_t, const double* u_h,
                             const float* candidates_dev, uint64_t tick, void* stream) {
  if (!s || !x_t || !u_h) return fail(MPMI_E_INVALID_ARG, "evaluate_candidates: NULL argument");
  const mpmi_model* m = s->model;
  int rc;
  if ((rc = check_finite(x_t, m->nx, "x_t")) != MPMI_OK) return rc;
  if ((rc = check_finite(u_h, m->nu, "u_h")) != MPMI_OK) return rc;
  if ((rc = check_ext(s, candidates_dev)) != MPMI_OK) return rc;
  DeviceGuard guard(s->ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = host_tick_begin(s)) != MPMI_OK) return rc;
  if (s->persist && s->rollout == MPMI_ROLLOUT_FULL && s->n_noise == 0 &&
      s->cfg.sampler != MPMI_SAMPLER_EXTERNAL) {
    // hand the tick to the resident kernel: mailbox words, then the number
    unsigned long long* mb = s->mbox_host;
    double xw[MPMI_MAX_NX] = {0, 0, 0, 0, 0, 0, 0, 0}, uw[MPMI_MAX_NU] = {0, 0, 0, 0};
    memcpy(xw, x_t, sizeof(double) * m->nx);
    memcpy(uw, u_h, sizeof(double) * m->nu);
    mb[1] = tick;
    memcpy(mb + 2, xw, sizeof(xw));
    memcpy(mb + 10, uw, sizeof(uw));
    if ((rc = persist_post(s, st, s->seq + 1)) != MPMI_OK) return rc;
    ++s->seq;
    s->persist_posted = true;
    s->in_flight = true;
    return MPMI_OK;
  }
  memcpy(s->in_host, x_t, sizeof(double) * m->nx);
  memcpy(s->in_host + 8, u_h, sizeof(double) * m->nu);
  TickArgs a = make_tick_args(s, tick);
  a.ext = candidates_dev;
  if (s->zero_copy) {
    a.x_t = s->in_map;
    a.u_h = s->in_map + 8;
    a.result = s->result_map;
    a.seq_out = s->seq_map;
    a.seq = ++s->seq;
    if ((rc = launch_tick_args(s, a, false, st, 0)) != MPMI_OK) return rc;
  } else {
    MPMI_CUDA(cudaMemcpyAsync(s->in_dev, s->in_host, 12 * sizeof(double),
                              cudaMemcpyHostToDevice, st),
              "copy x_t/u_h to the device");
    a.x_t = s->in_dev;
    a.u_h = s->in_dev + 8;
    a.result = s->result_dev;
    if ((rc = launch_tick_args(s, a, false, st, 0)) != MPMI_OK) return rc;
    MPMI_CUDA(cudaMemcpyAsync(s->result_host, s->result_dev, sizeof(mpmi_result),
                              cudaMemcpyDeviceToHost, st), "copy the result to the host");
  }
  return host_tick_end(s, st);
}

int mpmi_select_input(mpmi_session* s, mpmi_result* out) {
  if (!s || !out) return fail(MPMI_E_INVALID_ARG, "select_input: NULL argument");
  if (!s->in_flight) return fail(MPMI_E_NOT_READY, "select_input: no tick in flight");
  DeviceGuard guard(s->ctx->device);
  if (s->persist_posted) {
    const int rc = persist_wait(s);
    s->in_flight = false;
    s->persist_posted = false;
    if (rc != MPMI_OK) return rc;
    *out = *s->result_host;
    if (out->status == MPMI_TIMEOUT)
      return fail(MPMI_E_TIMEOUT, "select_input: a block of the resident tick kernel timed out "
                                  "staging shared memory; the result is not a selection");
    return MPMI_OK;
  }
  bool seen = false;
  if (s->zero_copy) {
    // the decoding block stores the tick's sequence number after the result
    // (system-scope fence between): poll it for up to a second, then fall back
    // to the event, which also reports a failed launch
    const volatile unsigned long long* w = s->seq_host;
    const auto t0 = std::chrono::steady_clock::now();
    for (unsigned long i = 0;; ++i) {
      if (*w == s->seq) {
        seen = true;
        break;
      }
      if ((i & 1023) == 1023 &&
          std::chrono::steady_clock::now() - t0 > std::chrono::seconds(1))
        break;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
  }
  if (!seen) MPMI_CUDA(cudaEventSynchronize(s->done), "waiting for the tick");
  s->tail_pending = seen;
  s->in_flight = false;
  *out = *s->result_host;
  if (out->status == MPMI_TIMEOUT)
    return fail(MPMI_E_TIMEOUT, "select_input: a block of the tick kernel timed out staging "
                                "shared memory; the result is not a selection");
  return MPMI_OK;
}

int mpmi_debug_withhold_staging(mpmi_session* s, int32_t on) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "session is NULL");
  s->withhold_staging = on ? 1 : 0;
  // a resident kernel keeps the staging it started with: the next tick relaunches
  DeviceGuard guard(s->ctx->device);
  return persist_stop(s);
}

static int evaluate_device(mpmi_session* s, const double* x_t_dev, const double* u_h_dev,
                           const float* candidates_dev, uint64_t tick, mpmi_result* result_dev,
                           int32_t* ttv_dev, float* cost_dev, float* traj_dev, void* stream) {
  if (!s || !x_t_dev || !u_h_dev || !result_dev)
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_device: NULL argument");
  int rc;
  if ((rc = check_ext(s, candidates_dev)) != MPMI_OK) return rc;
  DeviceGuard guard(s->ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  TickArgs a = make_tick_args(s, tick);
  a.x_t = x_t_dev;
  a.u_h = u_h_dev;
  a.ext = candidates_dev;
  a.result = result_dev;
  a.ttv_out = ttv_dev;
  a.cost_out = cost_dev;
  a.traj_out = traj_dev;
  return launch_tick_args(s, a, traj_dev != nullptr, (cudaStream_t)stream, 0);
}

int mpmi_evaluate_candidates_device(mpmi_session* s, const double* x_t_dev, const double* u_h_dev,
                                    const float* candidates_dev, uint64_t tick,
                                    mpmi_result* result_dev, int32_t* ttv_dev, float* cost_dev,
                                    void* stream) {
  return evaluate_device(s, x_t_dev, u_h_dev, candidates_dev, tick, result_dev, ttv_dev,
                         cost_dev, nullptr, stream);
}

int mpmi_debug_trajectories(mpmi_session* s, const double* x_t_dev, const double* u_h_dev,
                            const float* candidates_dev, uint64_t tick, mpmi_result* result_dev,
                            int32_t* ttv_dev, float* cost_dev, float* traj_dev, void* stream) {
  if (!traj_dev) return fail(MPMI_E_INVALID_ARG, "debug_trajectories: traj_dev is NULL");
  return evaluate_device(s, x_t_dev, u_h_dev, candidates_dev, tick, result_dev, ttv_dev,
                         cost_dev, traj_dev, stream);
}

int mpmi_tune_launch_shape(mpmi_ctx* ctx, const mpmi_model* model,
                           const mpmi_session_config* cfg, const double* x_t,
                           const double* u_h, int32_t reps, mpmi_tune_result* out) {
  if (!ctx || !model || !cfg || !x_t || !u_h || !out)
    return fail(MPMI_E_INVALID_ARG, "tune_launch_shape: NULL argument");
  if (reps < 1 || reps > 1000)
    return fail(MPMI_E_INVALID_ARG, "tune_launch_shape: reps must be in 1..1000");
  if (cfg->sampler == MPMI_SAMPLER_EXTERNAL)
    return fail(MPMI_E_UNSUPPORTED, "tune_launch_shape: tune with a built-in sampler");
  int rc;
  if ((rc = check_finite(x_t, model->nx, "x_t")) != MPMI_OK) return rc;
  if ((rc = check_finite(u_h, model->nu, "u_h")) != MPMI_OK) return rc;
  DeviceGuard guard(ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  const long long slots = (long long)cfg->n_samples + cfg->include_user;
  int dl = 0, dc = 0, db = 0;
  default_shape(model->kind, (int)slots, ctx->sm_count, &dl, &dc, &db);
  double* in_dev = nullptr;
  mpmi_result* res_dev = nullptr;
  // one start and one end event per timed tick: the ticks are queued back to back
  // and read after one synchronisation, so a tick's time never includes the
  // host's launch of the next one
  std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
  auto cleanup = [&]() {
    cudaFree(in_dev);
    cudaFree(res_dev);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  double in_host[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  memcpy(in_host, x_t, sizeof(double) * model->nx);
  memcpy(in_host + 8, u_h, sizeof(double) * model->nu);
  bool events_ok = true;
  for (cudaEvent_t& e : ev) events_ok = events_ok && cudaEventCreate(&e) == cudaSuccess;
  if (!events_ok || cudaMalloc(&in_dev, sizeof(in_host)) != cudaSuccess ||
      cudaMalloc(&res_dev, sizeof(mpmi_result)) != cudaSuccess ||
      cudaMemcpy(in_dev, in_host, sizeof(in_host), cudaMemcpyHostToDevice) != cudaSuccess) {
    cleanup();
    return fail(MPMI_E_OOM, "tune_launch_shape: device buffers");
  }
  mpmi_tune_result best;
  memset(&best, 0, sizeof(best));
  best.us = INFINITY;
  best.default_us = NAN;
  std::vector<float> t(reps);
  static const int kLanes[] = {1, 2, 4, 8, 16, 32};
  // every block size the built-in rule can pick is among these, so the default
  // shape is always timed
  static const int kBlocks[] = {64, 128, 160, 192, 224, 256};
  for (int lanes : kLanes) {
    for (int cands = 1; cands <= 2; ++cands) {
      if (!pick_tick(model->kind, lanes, cands, false, false).fn) continue;
      for (int block : kBlocks) {
        mpmi_session_config c = *cfg;
        c.lanes = lanes;
        c.cands_per_thread = cands;
        c.block = block;
        mpmi_session* s = nullptr;
        rc = mpmi_session_open(ctx, model, &c, &s);
        if (rc == MPMI_E_UNSUPPORTED) continue;  // not resident with this block
        if (rc != MPMI_OK) {
          cleanup();
          return rc;
        }
        for (int r = -2; r < reps && rc == MPMI_OK; ++r) {
          TickArgs a = make_tick_args(s, (uint64_t)(r + 2));
          a.x_t = in_dev;
          a.u_h = in_dev + 8;
          a.result = res_dev;
          if (r >= 0) cudaEventRecord(ev[2 * r], 0);
          rc = launch_tick_args(s, a, false, 0, 0);
          if (rc != MPMI_OK) break;
          if (r >= 0) cudaEventRecord(ev[2 * r + 1], 0);
        }
        if (rc == MPMI_OK) {
          if (cudaEventSynchronize(ev[2 * (size_t)reps - 1]) != cudaSuccess)
            rc = fail(MPMI_E_CUDA, "tune_launch_shape: timing the ticks");
          for (int r = 0; r < reps && rc == MPMI_OK; ++r)
            if (cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]) != cudaSuccess)
              rc = fail(MPMI_E_CUDA, "tune_launch_shape: timing a tick");
        }
        mpmi_session_close(s);
        if (rc == MPMI_E_UNSUPPORTED) {  // this block size cannot be resident: skip it
          rc = MPMI_OK;
          continue;
        }
        if (rc != MPMI_OK) {
          cleanup();
          return rc;
        }
        std::vector<float> sorted(t);
        std::sort(sorted.begin(), sorted.end());
        const double us = 1e3 * sorted[reps / 2];
        best.n_tried += 1;
        const bool is_default = lanes == dl && cands == dc && block == db;
        if (is_default) best.default_us = us;
        // event times are quantised: a tie goes to the default shape
        if (us < best.us || (us == best.us && is_default)) {
          best.us = us;
          best.lanes = lanes;
          best.cands = cands;
          best.block = block;
        }
      }
    }
  }
  cleanup();
  if (best.n_tried == 0) return fail(MPMI_E_UNSUPPORTED, "tune_launch_shape: no shape runs");
  bool replaced = false;
  for (auto& e : ctx->tuned)
    if (e.kind == model->kind && e.n_slots == (int)slots && e.horizon == cfg->horizon) {
      e.lanes = best.lanes;
      e.cands = best.cands;
      e.block = best.block;
      replaced = true;
    }
  if (!replaced)
    ctx->tuned.push_back({model->kind, (int)slots, cfg->horizon, best.lanes, best.cands, best.block});
  *out = best;
  return MPMI_OK;
}

int mpmi_sample_candidates(mpmi_session* s, const double* u_h_dev, const float* candidates_dev,
                           uint64_t tick, float* out_dev, void* stream) {
  if (!s || !out_dev) return fail(MPMI_E_INVALID_ARG, "sample_candidates: NULL argument");
  if (s->cfg.include_user && !u_h_dev)
    return fail(MPMI_E_INVALID_ARG, "sample_candidates: u_h_dev needed when slot 0 is u_h");
  int rc;
  if ((rc = check_ext(s, candidates_dev)) != MPMI_OK) return rc;
  DeviceGuard guard(s->ctx->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  TickArgs a = make_tick_args(s, tick);
  a.u_h = u_h_dev;
  a.ext = candidates_dev;
  const int block = 256, grid = (s->n_slots + block - 1) / block;
  cudaStream_t st = (cudaStream_t)stream;
  switch (s->model->nu) {
    case 1: sample_kernel<1><<<grid, block, 0, st>>>(a, out_dev); break;
    case 2: sample_kernel<2><<<grid, block, 0, st>>>(a, out_dev); break;
    default: return fail(MPMI_E_UNSUPPORTED, "sample_candidates: input dimension");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sample kernel launch");
  return MPMI_OK;
}

int mpmi_debug_philox(const uint32_t* records_dev, int64_t n, uint32_t* words_dev,
                      void* stream) {
  if (n < 0 || n > (int64_t(1) << 30))
    return fail(MPMI_E_INVALID_ARG, "debug_philox: n out of range");
  if (n == 0) return MPMI_OK;
  if (!records_dev || !words_dev) return fail(MPMI_E_INVALID_ARG, "debug_philox: NULL argument");
  if ((reinterpret_cast<uintptr_t>(records_dev) | reinterpret_cast<uintptr_t>(words_dev)) & 3)
    return fail(MPMI_E_INVALID_ARG, "debug_philox: buffers must be 4-byte aligned");
  const int block = 256;
  const int64_t grid = (n + block - 1) / block;
  philox_words_kernel<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(records_dev, n,
                                                                            words_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "philox kernel launch");
  return MPMI_OK;
}

}  // extern "C"
