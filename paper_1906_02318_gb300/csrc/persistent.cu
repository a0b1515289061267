// A persistent tick kernel for host ticks.
//
// A control loop ticks at 60-100 Hz and the host waits for each result, so a
// host tick is dominated by fixed costs: the launch, the first memory round
// trips, staging K and the track grid.  In persistent mode the session keeps one
// cooperative grid resident on its own stream.  K and the track grid are staged
// once; block 0 polls a mailbox in pinned host memory (coherent with the GPU over
// the host link), copies each new command (x_t, u_h, tick) into a device-side
// record and releases it to the other blocks; every block then runs exactly the
// tick of tick_kernel (same warp-tile code, same reduction, same decode), and the
// last block publishes the result and the command's number into pinned memory.
// Every wait is bounded: a grid that sees no command for the idle limit stops
// (the host relaunches it on the next tick), and the other blocks follow block
// 0's verdict within a longer bound.
#include <cuda_runtime.h>

#include "internal.h"
#include "tick_kernel.cuh"

namespace mpmi {

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Block 0: the next command number from the host's mailbox word, or 0 to halt.
// A pending command is always taken before a stop request; with no command for
// idle_ns the kernel marks the word as exited, by a compare-and-swap that fails
// (and the loop goes on) if the host posted a command in the meantime.
__device__ __forceinline__ unsigned long long relay_wait(const PersistArgs& p,
                                                         unsigned long long last) {
  const unsigned long long t0 = global_ns();
  while (true) {
    const unsigned long long w = ld_acquire_sys(p.mbox);
    if ((w & kCmdSeqMask) > last) return w & kCmdSeqMask;
    if (w & kCmdStop) return 0;
    if (global_ns() - t0 > p.idle_ns) {
      const unsigned long long old = atomicCAS_system(p.mbox, last, kCmdExit | last);
      if (old == last) return 0;
    }
  }
}

// Other blocks: block 0's relay of the command number, or 0 to halt.  Block 0
// halts by setting a separate word and never overwrites a relayed number, so a
// block that polls late still takes the last command before it halts (after
// seeing the halt word, the number block 0 stored before it is visible).  No
// relay within twice the idle limit plus a second also halts.
__device__ __forceinline__ unsigned long long follow_wait(const PersistArgs& p,
                                                          unsigned long long last) {
  const unsigned long long t0 = global_ns();
  const unsigned long long limit = 2 * p.idle_ns + 1000000000ull;
  while (true) {
    unsigned long long c = ld_acquire_gpu(p.cmd);
    if (c > last) return c;
    if (ld_acquire_gpu(p.cmd + kCmdHalt) != 0) {
      c = ld_acquire_gpu(p.cmd);
      return c > last ? c : 0;
    }
    if (global_ns() - t0 > limit) return 0;
  }
}

template <int KIND, int L, int C, bool KSMEM>
__global__ void __launch_bounds__(kMaxBlock)
    tick_persistent(const __grid_constant__ TickArgs a, const __grid_constant__ PersistArgs p) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU;
  constexpr int R = N / L;
  constexpr int GPW = 32 / L;
  constexpr int S = (N % 32 == 0) ? N + 4 : ((N % 4 == 0) ? N : N + (4 - N % 4));
  constexpr int NW = kMaxBlock / 32;
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  constexpr int KWORDS = ksmem_words<KIND, L, KSMEM, true>();
  constexpr bool PK = pair_k<KIND, L, KSMEM, true>();

  extern __shared__ uint4 s_dyn[];
  __shared__ __align__(16) float s_x[(L > 1) ? NW : 1][2][GPW][S];
  __shared__ uint64_t s_bar;
  // this tick's command: [0] number, [1] tick, [2, 2 + 8) x_t, [10, 10 + 4) u_h
  __shared__ unsigned long long s_cmd[kCmdPayload];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = lane % L;
  const int n_eval = a.n_slots;

  // once per residency: K and the track grid into shared memory (bulk copies on
  // an mbarrier, bounded wait), or this lane's rows of K into registers
  const bool track_on = B::TRACK && a.safety.has_track;
  const bool staging = KSMEM || track_on;
  if (staging) {
    if (tid == 0) bar_init(&s_bar);
    __syncthreads();
    if (tid == 0)
      stage_issue(&s_bar, s_dyn, a.Ks, (KSMEM && !PK) ? N : 0, N, KSmem<N>::S4,
                  a.safety.track.blob, track_on ? a.safety.track.blob_bytes : 0,
                  a.withhold_staging != 0, a.Kp, PK ? (int)KPair<KIND>::BYTES : 0);
  }
  TrackView tv{nullptr, nullptr, nullptr, nullptr};
  if constexpr (B::TRACK) {
    if (a.safety.has_track) {
      const char* base = reinterpret_cast<const char*>(s_dyn + KWORDS);
      tv.cells = reinterpret_cast<const uint32_t*>(base);
      tv.list = reinterpret_cast<const uint16_t*>(base + a.safety.track.off_list);
      tv.seg = reinterpret_cast<const float4*>(base + a.safety.track.off_seg);
      tv.inv = reinterpret_cast<const float*>(base + a.safety.track.off_inv);
    }
  }
  const float4* sK4 = reinterpret_cast<const float4*>(s_dyn);
  float kr[KSMEM ? 1 : R][KSMEM ? 1 : N];
  if constexpr (!KSMEM) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float* row = a.K + (q * R + r) * N;
#pragma unroll
      for (int k = 0; k < N; ++k) kr[r][k] = __ldg(row + k);
    }
  }
  bool failed = false;
  if (staging) {
    // a block whose staging never lands skips its candidates in every tick and
    // flags each result, as the launched tick does
    bool ok = bar_wait(&s_bar, 0);
    if (!ok) ok = bar_wait(&s_bar, 0);
    failed = __syncthreads_or(!ok) != 0;
  }

  unsigned long long last = p.start_seq;
  if (blockIdx.x == 0 && tid == 0) {
    // a clean reduction record for the first command (the other blocks touch it
    // only after the release of that command's number)
    TickScratch* sc = a.scratch;
    sc->key = ~0ull;
    sc->counts = 0ull;
    sc->error = 0u;
    sc->done = 0u;
  }
  while (true) {
    // thread 0 takes the next command: block 0 from the host's mailbox (and
    // relays it to the device copy), the other blocks from that copy.  The
    // words are read after the acquiring load of the command number, by the
    // same thread (independent loads, in flight together).
    if (tid == 0) {
      const bool relay = blockIdx.x == 0;
      const unsigned long long v = relay ? relay_wait(p, last) : follow_wait(p, last);
      if (v != 0) {
        const volatile unsigned long long* src = relay ? p.mbox : p.cmd;
        unsigned long long w[kCmdPayload];
#pragma unroll
        for (int j = 1; j < kCmdPayload; ++j) w[j] = src[j];
#pragma unroll
        for (int j = 1; j < kCmdPayload; ++j) s_cmd[j] = w[j];
        if (relay) {
#pragma unroll
          for (int j = 1; j < kCmdPayload; ++j) p.cmd[j] = w[j];
          st_release_gpu(p.cmd, v);
        }
      } else if (relay) {
        st_release_gpu(p.cmd + kCmdHalt, 1ull);
      }
      s_cmd[0] = v;
    }
    __syncthreads();
    const unsigned long long v = s_cmd[0];
    if (v == 0) break;
    last = v;

    TickDyn d;
    d.tick = s_cmd[1];
    d.t_lo = (uint32_t)(d.tick & 0xFFFFFFFFull);
    d.t_hi = (uint32_t)(d.tick >> 32);
    d.seq = v;
    d.u_h = reinterpret_cast<const double*>(&s_cmd[10]);
    const double* x64 = reinterpret_cast<const double*>(&s_cmd[2]);
    float xs[NX], uh[NU];
#pragma unroll
    for (int j = 0; j < NX; ++j) xs[j] = __double2float_rn(x64[j]);
#pragma unroll
    for (int j = 0; j < NU; ++j) uh[j] = __double2float_rn(d.u_h[j]);
    float sn = 0.f, cs = 1.f;
    if constexpr (ANG >= 0) sincosf(xs[ANG], &sn, &cs);

    unsigned long long best = ~0ull;
    unsigned int n_safe = 0, n_exec = 0;
    const int wpb = blockDim.x >> 5;
    constexpr int PER_WARP = GPW * C;
    const int n_wtiles = failed ? 0 : (n_eval + PER_WARP - 1) / PER_WARP;
    for (int wt = blockIdx.x * wpb + warp; wt < n_wtiles; wt += gridDim.x * wpb)
      run_tile<KIND, L, C, KSMEM, false, false, true>(a, d, a.safety, wt, n_eval, xs, uh, sn, cs,
                                                     kr, sK4, tv, &s_x[L > 1 ? warp : 0][0][0][0],
                                                     best, n_safe, n_exec);
    session_epilogue<NU>(a, d, best, n_safe, n_exec, uh, failed);
    __syncthreads();
  }
}

struct PersistKernel {
  const void* fn = nullptr;
  size_t k_smem = 0;
};

template <int KIND, int L, int C, bool KSMEM>
static PersistKernel make_persist() {
  PersistKernel k;
  k.fn = reinterpret_cast<const void*>(&tick_persistent<KIND, L, C, KSMEM>);
  k.k_smem = (size_t)ksmem_words<KIND, L, KSMEM, true>() * 16;
  return k;
}

// The same launch shapes as the tick kernel (tick_dispatch.cuh).
static PersistKernel pick_persist(int kind, int lanes, int cands) {
  switch (kind) {
    case kBot:
      if (lanes == 1 && cands == 1) return make_persist<kBot, 1, 1, false>();
      if (lanes == 1 && cands == 2) return make_persist<kBot, 1, 2, false>();
      if (lanes == 2 && cands == 1) return make_persist<kBot, 2, 1, false>();
      if (lanes == 4 && cands == 1) return make_persist<kBot, 4, 1, false>();
      break;
    case kCar:
      if (lanes == 1 && cands == 1) return make_persist<kCar, 1, 1, true>();
      if (lanes == 1 && cands == 2) return make_persist<kCar, 1, 2, true>();
      if (lanes == 2 && cands == 1) return make_persist<kCar, 2, 1, true>();
      if (lanes == 4 && cands == 1) return make_persist<kCar, 4, 1, true>();
      if (lanes == 8 && cands == 1) return make_persist<kCar, 8, 1, false>();
      if (lanes == 16 && cands == 1) return make_persist<kCar, 16, 1, false>();
      break;
    case kLin11: if (lanes == 1 && cands == 1) return make_persist<kLin11, 1, 1, false>(); break;
    case kLin22: if (lanes == 1 && cands == 1) return make_persist<kLin22, 1, 1, false>(); break;
    case kLin41: if (lanes == 1 && cands == 1) return make_persist<kLin41, 1, 1, false>(); break;
  }
  return PersistKernel{};
}

bool persist_supported(int kind, int lanes, int cands) {
  return pick_persist(kind, lanes, cands).fn != nullptr;
}

int launch_persistent(mpmi_session* s, const TickArgs& a, const PersistArgs& pa) {
  const PersistKernel k = pick_persist(s->model->kind, s->lanes, s->cands);
  if (!k.fn) return fail(MPMI_E_UNSUPPORTED, "persistent tick not compiled for this launch shape");
  const size_t smem = k.k_smem + (a.safety.has_track ? (size_t)a.safety.track.blob_bytes : 0);
  if (smem > 0) {
    const cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(k.k_smem + kMaxTrackBytes));
    if (e != cudaSuccess) return fail(MPMI_E_CUDA, "cudaFuncSetAttribute (persistent)");
  }
  const int per_warp = 32 / s->lanes * s->cands;
  const int n_wtiles = (s->n_slots + per_warp - 1) / per_warp;
  // at most one block per SM (below), so the block is widened from the session's
  // until those blocks cover every warp-tile at once; the block size changes no
  // result (the reduction is a minimum and integer sums)
  int block = s->block;
  const int want_wpb = (n_wtiles + s->ctx->sm_count - 1) / s->ctx->sm_count;
  while (block < kMaxBlock && block / 32 < want_wpb) block += 32;
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, block, smem);
  if (e != cudaSuccess || nb < 1) {
    block = s->block;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.fn, block, smem);
  }
  if (e != cudaSuccess || nb < 1)
    return fail(MPMI_E_UNSUPPORTED, "persistent tick cannot be resident");
  const int wpb = block / 32;
  int grid = (n_wtiles + wpb - 1) / wpb;
  // at most one block per SM (warps stride over the warp-tiles), so that a
  // resident grid leaves room beside it for other kernels and other sessions'
  // resident grids
  if (grid > s->ctx->sm_count) grid = s->ctx->sm_count;
  if (grid > nb * s->ctx->sm_count) grid = nb * s->ctx->sm_count;
  if (grid < 1) grid = 1;
  // every block must be resident at once (they wait on block 0's relay)
  void* args[] = {const_cast<TickArgs*>(&a), const_cast<PersistArgs*>(&pa)};
  e = cudaLaunchCooperativeKernel(k.fn, dim3(grid), dim3(block), args, smem, s->persist_stream);
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("persistent tick launch: ") + cudaGetErrorString(e));
  return MPMI_OK;
}

}  // namespace mpmi
