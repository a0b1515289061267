// Continuous-batching tick server: many control sessions of one model, each with
// its own N, H, sampler stream and tick counter, evaluated together in one
// persistent launch that is replayed from a CUDA graph.
//
// Device side: the batch table lists the requests; their warp-tiles form one index
// space (prefix sums in tile_begin).  Persistent warps stride over it; each
// warp-tile runs the same per-tile code as the single-session tick (run_tile),
// then folds its key and counts into the session's reduction record; the warp
// that completes a session's last tile decodes its result.  A session's outcome
// is therefore bit-identical whether it is served alone or in a mix.
//
// Host side: admission (a free session slot and room in the context's memory
// budget), kBuffers batch buffers, each with one captured graph (table upload,
// kernel, result download) and a stream of its own, so a batch costs one graph
// launch and up to max_in_flight batches of the model run at once while the
// requests for the next one are staged.  A session has at most one request
// staged or on the GPU, so batches in flight touch disjoint reduction records;
// batches are collected in the order they complete.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "tick_kernel.cuh"

namespace mpmi {

// One request in a batch; field names follow TickArgs so run_tile and the
// decode read either.
struct SessionTick {
  int include_user, sampler, grid_g, n_slots;
  float in_lo[MPMI_MAX_NU], in_w[MPMI_MAX_NU];
  double in_lo64[MPMI_MAX_NU], in_hi64[MPMI_MAX_NU];
  uint32_t key0, key1, t_lo, t_hi, stream, pad0;
  const float* ext;
  int horizon, n_tiles, tile_begin, pad1;
  const int* slot_list;
  const int* n_list;
  int32_t* ttv_out;
  float* cost_out;
  float* traj_out;
  const double* u_h;  // device address of u_h_buf below
  mpmi_result* result;
  unsigned long long tick, result_flags;
  TickScratch* scratch;
  double x_t_buf[MPMI_MAX_NX];
  double u_h_buf[MPMI_MAX_NU];
};

struct ServeHeader {
  int n_requests;
  int total_tiles;
  int pad[2];
};

struct ServeArgs {
  const float* K;
  const float* Ks;  // K with each row's columns in staging order
  const float* Kp;  // the free rows of K in pairs (KPair layout; race car)
  DevSafety safety;
  const ServeHeader* table;  // header followed by SessionTick entries
};

template <int KIND, int L, int C, bool KSMEM>
__global__ void __launch_bounds__(kMaxBlock, 1) serve_kernel(const __grid_constant__ ServeArgs sa) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU;
  constexpr int R = N / L, GPW = 32 / L;
  constexpr int S = (N % 32 == 0) ? N + 4 : ((N % 4 == 0) ? N : N + (4 - N % 4));
  constexpr int NW = kMaxBlock / 32;
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  constexpr int KWORDS = ksmem_words<KIND, L, KSMEM, true>();
  constexpr bool PK = pair_k<KIND, L, KSMEM, true>();
  extern __shared__ uint4 s_dyn[];
  __shared__ __align__(16) float s_x[(L > 1) ? NW : 1][2][GPW][S];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = lane % L;
  // the grid covers the largest batch; a block past the batch's warp-tiles leaves
  // before staging anything, so that a small batch holds few SMs and batches in
  // flight at the same time share the device
  if ((long long)blockIdx.x * (blockDim.x >> 5) >= (long long)sa.table->total_tiles) return;

  if constexpr (PK) {
    const uint4* src = reinterpret_cast<const uint4*>(sa.Kp);
    for (int i = tid; i < KWORDS; i += blockDim.x) s_dyn[i] = __ldg(&src[i]);
  } else if constexpr (KSMEM) {
    stage_k<N>(sa.Ks, s_dyn, tid, blockDim.x);
  }
  TrackView tv{nullptr, nullptr, nullptr, nullptr};
  if constexpr (B::TRACK) {
    if (sa.safety.has_track) {
      uint4* dst = s_dyn + KWORDS;
      const int words = sa.safety.track.blob_bytes >> 4;
      for (int i = tid; i < words; i += blockDim.x) dst[i] = __ldg(&sa.safety.track.blob[i]);
      const char* base = reinterpret_cast<const char*>(dst);
      tv.cells = reinterpret_cast<const uint32_t*>(base);
      tv.list = reinterpret_cast<const uint16_t*>(base + sa.safety.track.off_list);
      tv.seg = reinterpret_cast<const float4*>(base + sa.safety.track.off_seg);
      tv.inv = reinterpret_cast<const float*>(base + sa.safety.track.off_inv);
    }
  }
  const float4* sK4 = reinterpret_cast<const float4*>(s_dyn);
  float kr[KSMEM ? 1 : R][KSMEM ? 1 : N];
  if constexpr (!KSMEM) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float* row = sa.K + (q * R + r) * N;
#pragma unroll
      for (int k = 0; k < N; ++k) kr[r][k] = __ldg(row + k);
    }
  }
  if constexpr (KSMEM || B::TRACK) __syncthreads();

  const ServeHeader* hdr = sa.table;
  const int n_req = hdr->n_requests, total = hdr->total_tiles;
  const SessionTick* ent = reinterpret_cast<const SessionTick*>(hdr + 1);
  const int wpb = blockDim.x >> 5;
  int cur = -1;
  float xs[NX], uh[NU], sn = 0.f, cs = 1.f;
  for (int gwt = blockIdx.x * wpb + warp; gwt < total; gwt += gridDim.x * wpb) {
    // the request this warp-tile belongs to (warp-uniform binary search)
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ent[mid].tile_begin <= gwt) lo = mid;
      else hi = mid - 1;
    }
    const SessionTick& st = ent[lo];
    if (lo != cur) {
#pragma unroll
      for (int j = 0; j < NX; ++j) xs[j] = __double2float_rn(st.x_t_buf[j]);
#pragma unroll
      for (int j = 0; j < NU; ++j) uh[j] = __double2float_rn(st.u_h_buf[j]);
      if constexpr (ANG >= 0) sincosf(xs[ANG], &sn, &cs);
      cur = lo;
    }
    unsigned long long best = ~0ull;
    unsigned int n_safe = 0, n_exec = 0;
    run_tile<KIND, L, C, KSMEM, false, false, true>(st, dyn_of(st), sa.safety, gwt - st.tile_begin, st.n_slots, xs, uh,
                                       sn, cs, kr, sK4, tv, &s_x[L > 1 ? warp : 0][0][0][0],
                                       best, n_safe, n_exec);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, best, o);
      best = other < best ? other : best;
      n_exec += __shfl_xor_sync(kFull, n_exec, o);
      n_safe += __shfl_xor_sync(kFull, n_safe, o);
    }
    if (lane == 0) {
      TickScratch* sc = st.scratch;
      atomicMin(&sc->key, best);
      atomicAdd(&sc->counts, ((unsigned long long)n_safe << 40) + n_exec);
      // acquire-release on the tile counter orders this warp's atomics before the
      // increment and lets the last warp see every other warp's
      unsigned int prev;
      asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&sc->done) : "memory");
      if (prev == (unsigned int)st.n_tiles - 1) {
        // this warp finished the session's last tile: decode and reset its record
        const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&sc->key);
        const unsigned long long cnt =
            *reinterpret_cast<volatile unsigned long long*>(&sc->counts);
        write_result<NU>(st, k, cnt, uh);
        sc->key = ~0ull;
        sc->counts = 0ull;
        sc->done = 0u;
      }
    }
    __syncwarp();
  }
}

struct ServeKernel {
  const void* fn = nullptr;
  void (*launch)(const ServeArgs&, int, int, size_t, cudaStream_t) = nullptr;
  size_t k_smem = 0;
  int per_warp = 32;
  int lanes = 1, cands = 1;
};

template <int KIND, int L, int C, bool KSMEM>
static void launch_serve(const ServeArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  serve_kernel<KIND, L, C, KSMEM><<<grid, block, smem, st>>>(a);
}

template <int KIND, int L, int C, bool KSMEM>
static ServeKernel make_serve() {
  ServeKernel k;
  k.fn = reinterpret_cast<const void*>(&serve_kernel<KIND, L, C, KSMEM>);
  k.launch = &launch_serve<KIND, L, C, KSMEM>;
  k.k_smem = (size_t)ksmem_words<KIND, L, KSMEM, true>() * 16;
  k.per_warp = 32 / L * C;
  k.lanes = L;
  k.cands = C;
  return k;
}

// The server's shapes per basis; the first is the initial one (one candidate per
// thread: the balance bot keeps K in registers, the race car in shared memory, as
// the single-session tick does by default), the others are for the autotuner.
static std::vector<ServeKernel> serve_shapes(int kind) {
  switch (kind) {
    case kBot:
      return {make_serve<kBot, 1, 1, false>(), make_serve<kBot, 1, 2, false>(),
              make_serve<kBot, 2, 1, false>(), make_serve<kBot, 4, 1, false>()};
    case kCar:
      return {make_serve<kCar, 1, 1, true>(), make_serve<kCar, 1, 2, true>(),
              make_serve<kCar, 2, 1, true>(), make_serve<kCar, 8, 1, false>()};
    case kLin11: return {make_serve<kLin11, 1, 1, false>()};
    case kLin22: return {make_serve<kLin22, 1, 1, false>()};
    case kLin41: return {make_serve<kLin41, 1, 1, false>()};
  }
  return {};
}

static ServeKernel pick_serve(int kind) {
  const std::vector<ServeKernel> v = serve_shapes(kind);
  return v.empty() ? ServeKernel{} : v[0];
}

}  // namespace mpmi

// ---------------------------------------------------------------- host side
constexpr int kServeBuffers = 5;                      // batch buffers
constexpr int kServeMaxInFlight = kServeBuffers - 1;  // one is always free for staging

struct mpmi_server {
  mpmi_ctx* ctx = nullptr;
  const mpmi_model* model = nullptr;
  int max_sessions = 0;
  std::vector<mpmi_session_config> cfg;
  std::vector<char> used;
  // per session slot: 0 idle, 1 staged in the stage buffer, 2 on the GPU
  std::vector<char> state;
  mpmi::TickScratch* scratch = nullptr;  // one record per session slot
  // batch buffers
  mpmi::ServeHeader* table_host[kServeBuffers] = {};  // pinned
  mpmi::ServeHeader* table_dev[kServeBuffers] = {};
  mpmi_result* res_dev[kServeBuffers] = {};
  mpmi_result* res_host[kServeBuffers] = {};         // pinned
  std::vector<int> slots[kServeBuffers];
  cudaGraphExec_t graph[kServeBuffers] = {};
  cudaStream_t bstream[kServeBuffers] = {};  // each buffer's batches run here
  cudaEvent_t start[kServeBuffers] = {};     // before the graph (timing)
  cudaEvent_t done[kServeBuffers] = {};      // after the graph
  cudaEvent_t after[kServeBuffers] = {};     // the caller's stream at launch
  bool flying[kServeBuffers] = {};
  unsigned long long seq[kServeBuffers] = {};  // launch order
  unsigned long long next_seq = 0;
  cudaStream_t capture = nullptr;
  int stage = 0;  // buffer receiving requests (never in flight)
  int max_in_flight = kServeMaxInFlight;
  size_t table_bytes = 0, smem = 0;
  int grid = 0, block = 128;
  mpmi::ServeKernel kern;
  uint64_t per_session_bytes = 0, bytes = 0;
};

namespace mpmi {

static int sfail(cudaError_t e, const char* what) {
  return fail(MPMI_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define SRV_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return sfail(e_, what); \
  } while (0)

static int build_graph(mpmi_server* s, int b) {
  ServeArgs a;
  memset(&a, 0, sizeof(a));
  a.K = s->model->K32_dev;
  a.Ks = s->model->K32_dev + (size_t)s->model->n * s->model->n;
  a.Kp = s->model->K32_dev + 2 * (size_t)s->model->n * s->model->n;
  a.safety = s->model->dev_safety;
  a.table = s->table_dev[b];
  cudaGraph_t g = nullptr;
  SRV_CUDA(cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaMemcpyAsync(s->table_dev[b], s->table_host[b], s->table_bytes, cudaMemcpyHostToDevice,
                  s->capture);
  s->kern.launch(a, s->grid, s->block, s->smem, s->capture);
  cudaMemcpyAsync(s->res_host[b], s->res_dev[b], sizeof(mpmi_result) * s->max_sessions,
                  cudaMemcpyDeviceToHost, s->capture);
  cudaError_t e = cudaStreamEndCapture(s->capture, &g);
  if (e != cudaSuccess) return sfail(e, "end capture");
  e = cudaGraphInstantiate(&s->graph[b], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return sfail(e, "graph instantiate");
  return MPMI_OK;
}

static int n_flying(const mpmi_server* s) {
  int n = 0;
  for (int b = 0; b < kServeBuffers; ++b) n += s->flying[b] ? 1 : 0;
  return n;
}

static void server_release_device(mpmi_server* s) {
  for (int b = 0; b < kServeBuffers; ++b) {
    if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
    for (cudaEvent_t e : {s->start[b], s->done[b], s->after[b]})
      if (e) cudaEventDestroy(e);
    if (s->bstream[b]) cudaStreamDestroy(s->bstream[b]);
    cudaFreeHost(s->table_host[b]);
    cudaFreeHost(s->res_host[b]);
    cudaFree(s->table_dev[b]);
    cudaFree(s->res_dev[b]);
  }
  cudaFree(s->scratch);
  if (s->capture) cudaStreamDestroy(s->capture);
}

}  // namespace mpmi

using namespace mpmi;

extern "C" {

int mpmi_server_create(mpmi_ctx* ctx, const mpmi_model* model, int32_t max_sessions,
                       mpmi_server** out) {
  if (!ctx || !model || !out) return fail(MPMI_E_INVALID_ARG, "server: NULL argument");
  *out = nullptr;
  if (!model->has_safety) return fail(MPMI_E_INVALID_ARG, "server: set_safety_set first");
  if (max_sessions < 1 || max_sessions > 65536)
    return fail(MPMI_E_INVALID_ARG, "server: max_sessions out of range");
  ServeKernel kern = pick_serve(model->kind);
  if (!kern.fn) return fail(MPMI_E_UNSUPPORTED, "server: basis not compiled");
  mpmi_server* s = new mpmi_server();
  s->ctx = ctx;
  s->model = model;
  s->max_sessions = max_sessions;
  s->kern = kern;
  s->cfg.resize(max_sessions);
  s->used.assign(max_sessions, 0);
  s->state.assign(max_sessions, 0);
  s->table_bytes = sizeof(ServeHeader) + sizeof(SessionTick) * (size_t)max_sessions;
  s->smem = kern.k_smem + (model->dev_safety.has_track ? (size_t)model->dev_safety.track.blob_bytes : 0);
  s->per_session_bytes =
      sizeof(TickScratch) + kServeBuffers * (sizeof(SessionTick) + sizeof(mpmi_result));
  const uint64_t fixed =
      kServeBuffers * (s->table_bytes + sizeof(mpmi_result) * (size_t)max_sessions) +
      sizeof(TickScratch) * (size_t)max_sessions;
  if (ctx->budget && ctx->used + fixed > ctx->budget) {
    delete s;
    return fail(MPMI_E_OOM, "server: tables exceed the memory budget");
  }
  bool ok = cudaMalloc(&s->scratch, sizeof(TickScratch) * max_sessions) == cudaSuccess &&
            cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) == cudaSuccess;
  for (int b = 0; b < kServeBuffers && ok; ++b)
    ok = cudaMallocHost(&s->table_host[b], s->table_bytes) == cudaSuccess &&
         cudaMalloc(&s->table_dev[b], s->table_bytes) == cudaSuccess &&
         cudaMalloc(&s->res_dev[b], sizeof(mpmi_result) * max_sessions) == cudaSuccess &&
         cudaMallocHost(&s->res_host[b], sizeof(mpmi_result) * max_sessions) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->bstream[b], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreate(&s->start[b]) == cudaSuccess &&
         cudaEventCreate(&s->done[b]) == cudaSuccess &&
         cudaEventCreateWithFlags(&s->after[b], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    server_release_device(s);
    delete s;
    return fail(MPMI_E_OOM, "server: allocation failed");
  }
  std::vector<TickScratch> init(max_sessions);
  for (auto& r : init) {
    memset(&r, 0, sizeof(r));
    r.key = ~0ull;
  }
  cudaMemcpy(s->scratch, init.data(), sizeof(TickScratch) * max_sessions, cudaMemcpyHostToDevice);
  for (int b = 0; b < kServeBuffers; ++b) {
    memset(s->table_host[b], 0, s->table_bytes);
    cudaMemset(s->table_dev[b], 0, s->table_bytes);
  }
  // persistent grid: every block resident at once
  if (s->smem > 0)
    cudaFuncSetAttribute(kern.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern.fn, s->block, s->smem);
  s->grid = (nb < 1 ? 1 : nb) * ctx->sm_count;
  for (int b = 0; b < kServeBuffers; ++b) {
    int rc = build_graph(s, b);
    if (rc != MPMI_OK) {
      server_release_device(s);
      delete s;
      return rc;
    }
  }
  s->bytes = fixed;
  ctx->used += fixed;
  *out = s;
  return MPMI_OK;
}

void mpmi_server_free(mpmi_server* s) {
  if (!s) return;
  for (int b = 0; b < kServeBuffers; ++b)
    if (s->flying[b]) cudaEventSynchronize(s->done[b]);
  server_release_device(s);
  for (int i = 0; i < s->max_sessions; ++i)
    if (s->used[i]) s->ctx->used -= s->per_session_bytes;
  s->ctx->used -= s->bytes;
  delete s;
}

int mpmi_server_admit(mpmi_server* s, const mpmi_session_config* cfg, int32_t* slot_out) {
  if (!s || !cfg || !slot_out) return fail(MPMI_E_INVALID_ARG, "server_admit: NULL argument");
  const mpmi_model* m = s->model;
  if (cfg->horizon < 1 || cfg->horizon > MPMI_MAX_HORIZON || cfg->n_samples < 0 ||
      (cfg->include_user != 0 && cfg->include_user != 1))
    return fail(MPMI_E_INVALID_ARG, "server_admit: bad N, H or include_user");
  const long long slots = (long long)cfg->n_samples + cfg->include_user;
  if (slots < 1 || slots > MPMI_MAX_SLOTS)
    return fail(MPMI_E_INVALID_ARG, "server_admit: slot count out of range");
  if (cfg->sampler != MPMI_SAMPLER_UNIFORM)
    return fail(MPMI_E_UNSUPPORTED, "server_admit: served sessions draw uniform samples");
  for (int j = 0; j < m->nu; ++j)
    if (!isfinite(cfg->input_lo[j]) || !isfinite(cfg->input_hi[j]) ||
        !(cfg->input_lo[j] < cfg->input_hi[j]))
      return fail(MPMI_E_INVALID_ARG, "server_admit: bad input box");
  int free_slot = -1;
  for (int i = 0; i < s->max_sessions; ++i)
    if (!s->used[i]) {
      free_slot = i;
      break;
    }
  if (free_slot < 0) return fail(MPMI_E_OOM, "server_admit: every session slot is taken");
  mpmi_ctx* ctx = s->ctx;
  if (ctx->budget && ctx->used + s->per_session_bytes > ctx->budget)
    return fail(MPMI_E_OOM, "server_admit: the context's memory budget is exhausted");
  s->used[free_slot] = 1;
  s->cfg[free_slot] = *cfg;
  ctx->used += s->per_session_bytes;
  *slot_out = free_slot;
  return MPMI_OK;
}

int mpmi_server_release(mpmi_server* s, int32_t slot) {
  if (!s || slot < 0 || slot >= s->max_sessions || !s->used[slot])
    return fail(MPMI_E_INVALID_ARG, "server_release: no such session");
  if (s->state[slot] == 1)
    return fail(MPMI_E_NOT_READY, "server_release: session has a staged request");
  if (s->state[slot] == 2) return fail(MPMI_E_NOT_READY, "server_release: session is on the GPU");
  s->used[slot] = 0;
  s->ctx->used -= s->per_session_bytes;
  return MPMI_OK;
}

int mpmi_server_submit(mpmi_server* s, int32_t n, const int32_t* slots, const double* x_t,
                       const double* u_h, const uint64_t* ticks) {
  if (!s || n < 0 || (n > 0 && (!slots || !x_t || !u_h || !ticks)))
    return fail(MPMI_E_INVALID_ARG, "server_submit: NULL argument");
  const mpmi_model* m = s->model;
  ServeHeader* hdr = s->table_host[s->stage];
  SessionTick* ent = reinterpret_cast<SessionTick*>(hdr + 1);
  const char* dev_base = reinterpret_cast<const char*>(s->table_dev[s->stage]);
  for (int r = 0; r < n; ++r) {
    const int sl = slots[r];
    if (sl < 0 || sl >= s->max_sessions || !s->used[sl])
      return fail(MPMI_E_INVALID_ARG, "server_submit: no such session");
    if (s->state[sl] == 1) return fail(MPMI_E_INVALID_ARG, "server_submit: session already staged");
    if (s->state[sl] == 2)
      return fail(MPMI_E_INVALID_ARG,
                  "server_submit: session's previous request is on the GPU (collect it first)");
    for (int j = 0; j < m->nx; ++j)
      if (!isfinite(x_t[(size_t)r * m->nx + j])) return fail(MPMI_E_NONFINITE, "server_submit: x_t");
    for (int j = 0; j < m->nu; ++j)
      if (!isfinite(u_h[(size_t)r * m->nu + j])) return fail(MPMI_E_NONFINITE, "server_submit: u_h");
  }
  for (int r = 0; r < n; ++r) {
    const int sl = slots[r];
    const mpmi_session_config& c = s->cfg[sl];
    const int i = hdr->n_requests;
    SessionTick& e = ent[i];
    memset(&e, 0, sizeof(e));
    e.include_user = c.include_user;
    e.sampler = c.sampler;
    e.n_slots = c.n_samples + c.include_user;
    for (int j = 0; j < MPMI_MAX_NU; ++j) {
      e.in_lo[j] = (float)c.input_lo[j];
      e.in_w[j] = (float)(c.input_hi[j] - c.input_lo[j]);
      e.in_lo64[j] = c.input_lo[j];
      e.in_hi64[j] = c.input_hi[j];
    }
    e.key0 = (uint32_t)(c.seed & 0xFFFFFFFFull);
    e.key1 = (uint32_t)(c.seed >> 32);
    e.t_lo = (uint32_t)(ticks[r] & 0xFFFFFFFFull);
    e.t_hi = (uint32_t)(ticks[r] >> 32);
    e.stream = c.stream_id;
    e.horizon = c.horizon;
    e.n_tiles = (e.n_slots + s->kern.per_warp - 1) / s->kern.per_warp;
    e.tile_begin = hdr->total_tiles;
    e.tick = ticks[r];
    e.scratch = s->scratch + sl;
    e.result = s->res_dev[s->stage] + i;
    for (int j = 0; j < m->nx; ++j) e.x_t_buf[j] = x_t[(size_t)r * m->nx + j];
    for (int j = 0; j < m->nu; ++j) e.u_h_buf[j] = u_h[(size_t)r * m->nu + j];
    e.u_h = reinterpret_cast<const double*>(
        dev_base + sizeof(ServeHeader) + sizeof(SessionTick) * (size_t)i +
        offsetof(SessionTick, u_h_buf));
    hdr->n_requests += 1;
    hdr->total_tiles += e.n_tiles;
    s->slots[s->stage].push_back(sl);
    s->state[sl] = 1;
  }
  return MPMI_OK;
}

int mpmi_server_launch(mpmi_server* s, void* stream, int32_t* n_launched) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "server_launch: NULL argument");
  const int b = s->stage;
  const int n = s->table_host[b]->n_requests;
  if (n_launched) *n_launched = 0;
  if (n == 0) return MPMI_OK;
  if (n_flying(s) >= s->max_in_flight)
    return fail(MPMI_E_NOT_READY, "server_launch: the most batches allowed in flight are on the "
                                  "GPU (collect one first)");
  // the batch follows the work queued so far on the caller's stream, and runs
  // on its buffer's own stream so that it overlaps the batches in flight
  cudaStream_t st = (cudaStream_t)stream;
  SRV_CUDA(cudaEventRecord(s->after[b], st), "server event");
  SRV_CUDA(cudaStreamWaitEvent(s->bstream[b], s->after[b], 0), "server stream wait");
  SRV_CUDA(cudaEventRecord(s->start[b], s->bstream[b]), "server event");
  SRV_CUDA(cudaGraphLaunch(s->graph[b], s->bstream[b]), "server graph launch");
  SRV_CUDA(cudaEventRecord(s->done[b], s->bstream[b]), "server event");
  if (n_launched) *n_launched = n;
  s->flying[b] = true;
  s->seq[b] = s->next_seq++;
  for (int sl : s->slots[b]) s->state[sl] = 2;
  // the next buffer not in flight receives the requests (one always is: at most
  // kServeBuffers - 1 batches fly)
  int nb = b;
  for (int i = 1; i < kServeBuffers; ++i) {
    const int c = (b + i) % kServeBuffers;
    if (!s->flying[c]) {
      nb = c;
      break;
    }
  }
  s->stage = nb;
  s->table_host[nb]->n_requests = 0;
  s->table_host[nb]->total_tiles = 0;
  s->slots[nb].clear();
  return MPMI_OK;
}

int mpmi_server_set_max_in_flight(mpmi_server* s, int32_t n) {
  if (!s || n < 1 || n > kServeMaxInFlight)
    return fail(MPMI_E_INVALID_ARG, "server_set_max_in_flight: n must be in 1.." +
                                        std::to_string(kServeMaxInFlight));
  s->max_in_flight = n;
  return MPMI_OK;
}

int mpmi_server_in_flight(const mpmi_server* s, int32_t* n_out) {
  if (!s || !n_out) return fail(MPMI_E_INVALID_ARG, "server_in_flight: NULL argument");
  *n_out = n_flying(s);
  return MPMI_OK;
}

// The in-flight batch to collect: the earliest launched among those finished,
// else the earliest launched (-1 if none flies).  *finished tells which.
static int next_batch(const mpmi_server* s, bool* finished, cudaError_t* err) {
  int oldest = -1, first_done = -1;
  *err = cudaSuccess;
  for (int b = 0; b < kServeBuffers; ++b) {
    if (!s->flying[b]) continue;
    if (oldest < 0 || s->seq[b] < s->seq[oldest]) oldest = b;
    const cudaError_t e = cudaEventQuery(s->done[b]);
    if (e == cudaSuccess) {
      if (first_done < 0 || s->seq[b] < s->seq[first_done]) first_done = b;
    } else if (e != cudaErrorNotReady) {
      *err = e;
      return b;
    }
  }
  *finished = first_done >= 0;
  return first_done >= 0 ? first_done : oldest;
}

int mpmi_server_poll(mpmi_server* s, int32_t* done) {
  if (!s || !done) return fail(MPMI_E_INVALID_ARG, "server_poll: NULL argument");
  bool finished = false;
  cudaError_t e;
  const int b = next_batch(s, &finished, &e);
  if (e != cudaSuccess) return sfail(e, "server_poll");
  *done = (b >= 0 && finished) ? 1 : 0;
  return MPMI_OK;
}

int mpmi_server_collect(mpmi_server* s, mpmi_result* out, int32_t* slots_out, int32_t* n_out) {
  if (!s || !out || !n_out) return fail(MPMI_E_INVALID_ARG, "server_collect: NULL argument");
  bool finished = false;
  cudaError_t e;
  const int b = next_batch(s, &finished, &e);
  if (e != cudaSuccess) return sfail(e, "server_collect");
  if (b < 0) return fail(MPMI_E_NOT_READY, "server_collect: no batch in flight");
  if (!finished) SRV_CUDA(cudaEventSynchronize(s->done[b]), "server_collect");
  const int n = (int)s->slots[b].size();
  memcpy(out, s->res_host[b], sizeof(mpmi_result) * n);
  if (slots_out) memcpy(slots_out, s->slots[b].data(), sizeof(int32_t) * n);
  *n_out = n;
  for (int sl : s->slots[b]) s->state[sl] = 0;
  s->slots[b].clear();
  s->table_host[b]->n_requests = 0;
  s->table_host[b]->total_tiles = 0;
  s->flying[b] = false;
  return MPMI_OK;
}

}  // extern "C"

namespace mpmi {

// Switches the server to launch shape k with `block` threads per block and
// re-captures both batch graphs.  UNSUPPORTED if the shape cannot be resident.
static int server_set_shape(mpmi_server* s, const ServeKernel& k, int block) {
  const size_t smem =
      k.k_smem + (s->model->dev_safety.has_track ? (size_t)s->model->dev_safety.track.blob_bytes : 0);
  if (smem > 0 &&
      cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return fail(MPMI_E_UNSUPPORTED, "server: shape cannot take its shared memory");
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, block, smem) != cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    return fail(MPMI_E_UNSUPPORTED, "server: shape cannot be resident");
  }
  s->kern = k;
  s->block = block;
  s->smem = smem;
  s->grid = nb * s->ctx->sm_count;
  for (int b = 0; b < kServeBuffers; ++b) {
    if (s->graph[b]) cudaGraphExecDestroy(s->graph[b]);
    s->graph[b] = nullptr;
    const int rc = build_graph(s, b);
    if (rc != MPMI_OK) return rc;
  }
  return MPMI_OK;
}

}  // namespace mpmi

extern "C" {

int mpmi_server_tune(mpmi_server* s, int32_t n, const mpmi_session_config* cfgs,
                     const double* x_t, const double* u_h, int32_t reps,
                     mpmi_tune_result* out) {
  if (!s || !cfgs || !x_t || !u_h || !out || n < 1)
    return fail(MPMI_E_INVALID_ARG, "server_tune: NULL argument or n < 1");
  if (reps < 1 || reps > 100) return fail(MPMI_E_INVALID_ARG, "server_tune: reps must be in 1..100");
  if (n_flying(s) > 0 || s->table_host[s->stage]->n_requests > 0)
    return fail(MPMI_E_NOT_READY, "server_tune: a batch is staged or in flight");
  std::vector<int32_t> slots;
  auto release_all = [&]() {
    for (int32_t sl : slots) mpmi_server_release(s, sl);
  };
  for (int i = 0; i < n; ++i) {
    int32_t sl = -1;
    const int rc = mpmi_server_admit(s, &cfgs[i], &sl);
    if (rc != MPMI_OK) {
      release_all();
      return rc;
    }
    slots.push_back(sl);
  }
  std::vector<mpmi_result> res(n);
  std::vector<int32_t> got(n);
  std::vector<uint64_t> ticks(n);
  std::vector<float> t(reps);
  const ServeKernel initial = s->kern;
  const int initial_block = s->block;
  ServeKernel best_k = initial;
  int best_block = initial_block;
  mpmi_tune_result best;
  memset(&best, 0, sizeof(best));
  best.us = INFINITY;
  best.default_us = NAN;
  int rc = MPMI_OK;
  static const int kBlocks[] = {64, 128, 256};
  for (const ServeKernel& k : serve_shapes(s->model->kind)) {
    for (int block : kBlocks) {
      rc = server_set_shape(s, k, block);
      if (rc == MPMI_E_UNSUPPORTED) {
        rc = MPMI_OK;
        continue;
      }
      if (rc != MPMI_OK) break;
      for (int r = -1; r < reps && rc == MPMI_OK; ++r) {
        for (int i = 0; i < n; ++i) ticks[i] = (uint64_t)(r + 1) * (uint64_t)n + (uint64_t)i;
        rc = mpmi_server_submit(s, n, slots.data(), x_t, u_h, ticks.data());
        if (rc != MPMI_OK) break;
        int32_t launched = 0, n_out = 0;
        const int b = s->stage;  // the buffer this batch launches from
        rc = mpmi_server_launch(s, nullptr, &launched);
        if (rc != MPMI_OK) break;
        rc = mpmi_server_collect(s, res.data(), got.data(), &n_out);
        if (rc != MPMI_OK) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->start[b], s->done[b]) != cudaSuccess) {
          rc = fail(MPMI_E_CUDA, "server_tune: timing a batch");
          break;
        }
        if (r >= 0) t[r] = ms;
      }
      if (rc != MPMI_OK) break;
      std::vector<float> sorted(t);
      std::sort(sorted.begin(), sorted.end());
      const double us = 1e3 * sorted[reps / 2];
      best.n_tried += 1;
      const bool is_default = k.fn == initial.fn && block == initial_block;
      if (is_default) best.default_us = us;
      // event times are quantised: a tie goes to the initial shape
      if (us < best.us || (us == best.us && is_default)) {
        best.us = us;
        best_k = k;
        best_block = block;
      }
    }
    if (rc != MPMI_OK) break;
  }
  // keep the winner (or go back to the initial shape after a failure)
  const int rc2 = rc == MPMI_OK ? server_set_shape(s, best_k, best_block)
                                : server_set_shape(s, initial, initial_block);
  release_all();
  if (rc != MPMI_OK) return rc;
  if (rc2 != MPMI_OK) return rc2;
  best.lanes = best_k.lanes;
  best.cands = best_k.cands;
  best.block = best_block;
  *out = best;
  return MPMI_OK;
}

int mpmi_server_staged(const mpmi_server* s, int32_t* n_out) {
  if (!s || !n_out) return fail(MPMI_E_INVALID_ARG, "server_staged: NULL argument");
  *n_out = s->table_host[s->stage]->n_requests;
  return MPMI_OK;
}

}  // extern "C"
