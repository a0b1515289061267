// The race car's rollout on the 5th-generation tensor cores (tcgen05).
//
// Batched over a tile of candidates, Alg. 2's prediction step is a matrix
// product: with the lifted states of 128 candidates as the rows of Z (128 x 32),
// one step is Z <- Z K^T (Sec. IV-A: one matrix-matrix product per step for a
// batch).  A CTA of 320 threads keeps two tiles in flight, one per half: half h
// is candidate warps 4h .. 4h + 3 (thread i of them = candidate i = TMEM lane
// i) and warp 8 + h, which issues the half's MMAs.  Each half owns 128 TMEM
// columns: the accumulator (64) and its A operand as TF32 hi and lo rows (32
// each), so the operand the threads write never passes through shared memory;
// the halves share K (the B operand) and the track grid in shared memory and
// synchronise on their own named barriers, so one half's MMAs overlap the other
// half's CUDA-core work.  Per step, in each half:
//   1. wait for the step's MMAs, read both column halves of the thread's row
//      with tcgen05.ld and add them (A_hi K_hi^T + A_lo K_hi^T + A_hi K_lo^T),
//      restore the held features exactly (their rows of K are unit rows), add
//      the noise z_i if enabled;
//   2. write the new z into the thread's TMEM lane as TF32 hi = trunc(z) and
//      lo = trunc(z - hi) rows with tcgen05.st, then one barrier of the half,
//      which also ORs the candidates still alive;
//   3. one lane of the issuing warp issues the next step's tcgen05.mma
//      kind::tf32 (A from TMEM, B from K-major shared-memory tiles of 8-row x
//      16-byte core matrices) over the four K blocks of 8: A_hi [K_hi; K_lo]^T
//      (N = 64, the K_lo tile directly follows K_hi, so one operand covers both)
//      into the half's accumulator columns 0..63, then A_lo K_hi^T (N = 32) into
//      its columns 0..31 -- eight MMAs in all -- and commits to the half's
//      mbarrier;
//   4. while those MMAs run, the candidates run the safety test on the z of
//      this step.
// The next step is issued before this step's safety test has ended, so its
// launch depends on the candidates alive one step earlier: a tile whose last
// candidate fails at step t computes step t + 1 and then stops.
// The split and the dropped lo*lo leave a few float32 roundings of error per
// product (see tf32_trunc; 2.9e-5 relative after 60 steps against float64), so
// results agree with the oracle under the same tolerance as the float32 FMA
// chain but are not bit-identical to the CUDA-core shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>

#include "internal.h"
#include "tcgen05.cuh"
#include "tick_kernel.cuh"

namespace mpmi {

constexpr int kTcM = 128;                  // candidates per tile = TMEM lanes
constexpr int kTcHalves = 2;               // tiles in flight per CTA
constexpr int kTcHalfThreads = kTcM + 32;  // a half: its candidates and its MMA-issuing warp
constexpr int kTcThreads = kTcHalves * kTcHalfThreads;
// TMEM columns of one half: the accumulator (64), then its A operand as TF32 hi
// and lo rows (32 each); four halves fill an SM's 512 columns
constexpr int kTcHalfCols = 128;
constexpr int kTcTmemCols = kTcHalfCols * kTcHalves;

// x rounded to TF32 (round to nearest, ties away from zero; NaN and infinity
// preserved), one conversion instruction: the split of K, once per CTA.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x truncated to TF32 (the 13 low mantissa bits cleared): one integer
// instruction, the split of z every step.  z - trunc(z) is exact in float32, so
// hi = trunc(z), lo = trunc(z - hi) leave |z - hi - lo| <= 2^-20 |z|; with K
// split to nearest and lo*lo dropped, a product is off by at most ~2^-19 |z||K|
// (measured: 2.9e-5 worst relative trajectory error after 60 steps against
// float64, against 2.1e-5 with both halves of z rounded to nearest, whose two
// conversions per element ran on a narrower pipe: 1.30 against 1.01 ms at a
// million candidates).  A NaN stays a NaN in hi or lo.
__device__ __forceinline__ uint32_t tf32_trunc(float x) {
  return __float_as_uint(x) & 0xFFFFE000u;
}

// Byte offset of element (row, k) in a K-major tile of 32-bit elements: core
// matrices of 8 rows x 16 bytes, the 8 k-chunks of a row group adjacent (128 B
// apart, the descriptor's leading byte offset), row groups 1024 B apart (its
// stride byte offset).
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)((((row >> 3) * 8 + (k >> 2)) * 128) + (row & 7) * 16 + (k & 3) * 4);
}

// Instruction descriptor, kind::tf32: D float32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t idesc_tf32(uint32_t n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}
constexpr uint32_t kIdescTf32 = idesc_tf32(32);
constexpr uint32_t kIdescTf32N64 = idesc_tf32(64);

// D (TMEM) (+)= A B^T with A read from TMEM (lane i = row i, K elements in
// consecutive columns) and B from shared memory (descriptor).
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint32_t a_tmem, uint64_t bd,
                                         uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// Dynamic shared memory: K_hi | K_lo (4 KB each), then the track grid, shared by
// the halves.
constexpr int kTcKBytes = 32 * 32 * 4;
constexpr int kTcFixedSmem = 2 * kTcKBytes;

// Barrier of one half (named barrier 1 + h, its 160 threads; immediate ids, so
// the kernel reserves three barriers).
__device__ __forceinline__ void half_sync(int h) {
  static_assert(kTcHalves == 2, "one named barrier per half");
  if (h == 0) asm volatile("bar.sync 1, %0;" ::"n"(kTcHalfThreads) : "memory");
  else asm volatile("bar.sync 2, %0;" ::"n"(kTcHalfThreads) : "memory");
}
// The same barrier, returning whether `v` holds for any thread of the half.
__device__ __forceinline__ bool half_any(int h, bool v) {
  uint32_t r;
  if (h == 0)
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kTcHalfThreads)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, 2, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kTcHalfThreads)
        : "memory");
  return r != 0u;
}

template <int KIND, bool TRAJ>
__global__ void __launch_bounds__(kTcThreads, 2) tc_tick_kernel(const __grid_constant__ TickArgs a) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU, NP = B::NP;
  static_assert(N == 32, "the tensor-core rollout is laid out for n = 32");
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  extern __shared__ __align__(1024) unsigned char s_tc[];
  const int tid = threadIdx.x, warp = tid >> 5;
  // threads [0, 256): candidates, half h = tid / 128, row r = TMEM lane; warps 8
  // and 9: the MMA-issuing warps of halves 0 and 1
  const bool issuer = tid >= kTcHalves * kTcM;
  const int h = issuer ? (tid - kTcHalves * kTcM) / 32 : tid / kTcM;
  const int r = tid % kTcM;
  unsigned char* bhi = s_tc;
  unsigned char* blo = bhi + kTcKBytes;
  uint4* blob = reinterpret_cast<uint4*>(s_tc + kTcFixedSmem);
  __shared__ uint64_t s_bar_stage, s_bar_mma[kTcHalves];
  __shared__ uint32_t s_tmem;
  // a half's failed MMA waits, by step parity: written after a step's wait and
  // read after the half's next barrier, so a thread already past that barrier
  // writes the other slot while a slower one still reads this one
  __shared__ int s_fail[kTcHalves][2];

  if (fallback_not_needed(a)) return;
  const int n_eval = a.n_list ? *a.n_list : a.n_slots;
  const int H = a.horizon;
  const bool track_on = B::TRACK && a.safety.has_track;

  if (tid == 0) {
    bar_init(&s_bar_stage);
#pragma unroll
    for (int i = 0; i < kTcHalves; ++i) {
      bar_init(&s_bar_mma[i]);
      s_fail[i][0] = s_fail[i][1] = 0;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "n"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem + (uint32_t)(kTcHalfCols * h);  // this half's columns
  if (tid == 0 && track_on)
    stage_issue(&s_bar_stage, blob, nullptr, 0, 0, 0, a.safety.track.blob,
                a.safety.track.blob_bytes, a.withhold_staging != 0);
  // K split into TF32 hi and lo rows (row r of K = row r of the B operand)
  if (tid < N) {
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
      const float4 kv = __ldg(reinterpret_cast<const float4*>(a.K + tid * N) + c);
      const float kk[4] = {kv.x, kv.y, kv.z, kv.w};
      uint32_t hh[4], ll[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hh[e] = tf32_rna(kk[e]);
        ll[e] = tf32_rna(kk[e] - __uint_as_float(hh[e]));
      }
      *reinterpret_cast<uint4*>(bhi + tile_off(tid, 4 * c)) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
      *reinterpret_cast<uint4*>(blo + tile_off(tid, 4 * c)) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
    }
    // the MMAs of both halves read these tiles through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  TrackView tv{nullptr, nullptr, nullptr, nullptr};
  if (track_on) {
    const char* base = reinterpret_cast<const char*>(blob);
    tv.cells = reinterpret_cast<const uint32_t*>(base);
    tv.list = reinterpret_cast<const uint16_t*>(base + a.safety.track.off_list);
    tv.seg = reinterpret_cast<const float4*>(base + a.safety.track.off_seg);
    tv.inv = reinterpret_cast<const float*>(base + a.safety.track.off_inv);
  }
  float xs[NX], uh[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xs[j] = __double2float_rn(a.x_t[j]);
#pragma unroll
  for (int j = 0; j < NU; ++j) uh[j] = __double2float_rn(a.u_h[j]);
  float sn = 0.f, cs = 1.f;
  if constexpr (ANG >= 0) sincosf(xs[ANG], &sn, &cs);
  bool failed = false;
  if (track_on) {
    bool ok = bar_wait(&s_bar_stage, 0);
    if (!ok) ok = bar_wait(&s_bar_stage, 0);
    failed = __syncthreads_or(!ok) != 0;
  } else {
    __syncthreads();  // the K tiles are written
  }

  const uint32_t b_hi = smem_u32(bhi);
  const uint32_t a_hi = tmem + 64, a_lo = tmem + 96;  // A operand columns (lane 0)
  const uint32_t taddr = tmem + ((uint32_t)((warp % 4) * 32) << 16);  // this warp's lanes
  // this thread's z as TF32 hi and lo rows of the half's A operand in TMEM
  const auto write_rows = [&](const float* z) {
#pragma unroll
    for (int c = 0; c < N / 8; ++c) {
      uint32_t hh[8], ll[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        hh[e] = tf32_trunc(z[8 * c + e]);
        ll[e] = tf32_trunc(z[8 * c + e] - __uint_as_float(hh[e]));
      }
      tmem_st8(taddr + 64 + 8 * c, hh);
      tmem_st8(taddr + 96 + 8 * c, ll);
    }
    tmem_st_wait();
  };
  // one step's MMAs (thread 0 of the half): columns 0..31 A_hi K_hi^T + A_lo
  // K_hi^T, columns 32..63 A_hi K_lo^T (B rows 32..63 are the K_lo tile, which
  // directly follows K_hi); their completion arrives on the half's mbarrier
  const auto issue_step = [&]() {
#pragma unroll
    for (int kb = 0; kb < N / 8; ++kb)
      mma_tf32(tmem, a_hi + 8 * kb, mat_desc(b_hi + kb * 256, 128, 1024), kIdescTf32N64,
               kb ? 1u : 0u);
#pragma unroll
    for (int kb = 0; kb < N / 8; ++kb)
      mma_tf32(tmem, a_lo + 8 * kb, mat_desc(b_hi + kb * 256, 128, 1024), kIdescTf32, 1u);
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&s_bar_mma[h]))
        : "memory");
  };

  uint32_t phase = 0;
  unsigned long long best = ~0ull;
  unsigned int n_safe = 0, n_exec = 0;
  const int n_tiles = failed ? 0 : (n_eval + kTcM - 1) / kTcM;
  // half h of CTA b takes tiles b + h * grid, b + (h + 2) * grid, ...: with fewer
  // tiles than CTAs only the first halves work, one tile per SM
  const int tile0 = blockIdx.x + h * gridDim.x, tile_step = gridDim.x * kTcHalves;
  if (issuer) {
    // the half's MMA-issuing warp: the same tiles and steps as its candidates,
    // meeting them at each of the half's barriers; lane 0 issues, so no
    // candidate waits while the MMAs are handed to the tensor core
    const bool lead = (tid & 31) == 0;
    for (int tile = tile0; tile < n_tiles; tile += tile_step) {
      tc_fence_before();
      half_sync(h);
      tc_fence_after();
      if (lead) issue_step();
      for (int t = 1; t <= H; ++t) {
        tc_fence_before();
        const bool any = half_any(h, false);
        tc_fence_after();
        if (s_fail[h][t & 1] || !any) break;
        if (t < H && lead) issue_step();
      }
    }
  }
  for (int tile = issuer ? n_tiles : tile0; tile < n_tiles; tile += tile_step) {
    const int pos = tile * kTcM + r;
    const bool valid = pos < n_eval;
    const int slot = (valid && a.slot_list) ? a.slot_list[pos] : pos;
    float xi[NU];
    if (valid) {
      candidate_value<NU>(a, slot, uh, xi);
    } else {
#pragma unroll
      for (int j = 0; j < NU; ++j) xi[j] = uh[j];
    }
    float cost = 0.f;
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      const float d = __fsub_rn(xi[j], uh[j]);
      cost = __fmaf_rn(d, d, cost);
    }
    float p[NP];
    monomials32<KIND>(xi, p);
    float z[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float av, bv[kMaxP];
      feature_split<float>(KIND, j, xs, sn, cs, &av, bv);
#pragma unroll
      for (int k = 0; k < NP; ++k) av = __fmaf_rn(p[k], bv[k], av);
      z[j] = av;
    }
    float* traj = nullptr;
    if constexpr (TRAJ) {
      if (valid) {
        traj = a.traj_out + (size_t)slot * (H + 1) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) traj[j] = z[j];
      }
    }
    int ttv = 0;
    bool alive = valid;
    // step 1's MMAs; every earlier use of the half's tiles and accumulator has
    // ended (the previous tile waited for its last MMAs and read them back)
    write_rows(z);
    tc_fence_before();
    half_sync(h);
    tc_fence_after();
    for (int t = 1; t <= H; ++t) {
      // (1) step t's accumulator -> z (tcgen05.ld is warp-aligned: the warp decides as one)
      const bool done = __all_sync(kFull, bar_wait(&s_bar_mma[h], phase));
      phase ^= 1u;
      tc_fence_after();
      if (done) {
        // the two column halves, 16 columns at a time
#pragma unroll
        for (int c = 0; c < N / 16; ++c) {
          uint32_t zn[16], zl[16];
          tmem_ld16_nowait(taddr + 16 * c, zn);
          tmem_ld16_nowait(taddr + 32 + 16 * c, zl);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (!held_feature(KIND, 16 * c + e))
              z[16 * c + e] = __fadd_rn(__uint_as_float(zn[e]), __uint_as_float(zl[e]));
        }
      } else {
        s_fail[h][t & 1] = 1;
      }
      if (a.n_noise > 0 && alive) add_noise<NX>(a, dyn_of(a), slot, t, z);
      if constexpr (TRAJ) {
        if (traj != nullptr && alive) {
#pragma unroll
          for (int j = 0; j < N; ++j) traj[(size_t)t * N + j] = z[j];
        }
      }
      // (2) the next step's A rows; the half's barrier also ORs the candidates
      // alive after step t - 1 and orders every thread's TMEM reads before the
      // next MMAs overwrite the accumulator
      if (t < H) write_rows(z);
      tc_fence_before();
      const bool any = half_any(h, alive);
      tc_fence_after();
      if (s_fail[h][t & 1] || !any) break;  // uniform over the half; no MMA in flight
      // (3) the issuing warp starts step t + 1 on the tensor cores while (4) the
      // candidates test step t
      bool ok = box_ok<NX>(a.safety, z);
      if constexpr (B::TRACK) {
        if (track_on) ok = ok && track_ok<1>(a.safety.track, tv, z[0], z[1], 0, alive && ok);
      }
      if (alive) {
        if (ok) ttv = t;
        else alive = false;
      }
    }
    if (s_fail[h][0] | s_fail[h][1]) {
      failed = true;
      break;
    }
    if (valid) {
      const unsigned long long key = ((unsigned long long)(H - ttv) << 55) |
                                     ((unsigned long long)__float_as_uint(cost) << 23) |
                                     (unsigned long long)slot;
      best = key < best ? key : best;
      n_exec += (unsigned int)min(ttv + 1, H);
      n_safe += ttv == H;
      if (a.ttv_out) a.ttv_out[slot] = ttv;
      if (a.cost_out) a.cost_out[slot] = cost;
    }
  }
  tc_fence_before();
  failed = __syncthreads_or(failed) != 0;  // a half's failed wait flags the whole block
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "n"(kTcTmemCols)
                 : "memory");
  session_epilogue<NU, TickArgs, kTcThreads / 32>(a, best, n_safe, n_exec, uh, failed);
}

template <bool TRAJ>
static const void* tc_fn() {
  return reinterpret_cast<const void*>(&tc_tick_kernel<kCar, TRAJ>);
}

// The tensor-core rollout's CTAs per SM and the dynamic shared memory that keeps
// it there.  TMEM is not a scheduling resource: a CTA placed on an SM whose 512
// columns are taken would wait in tcgen05.alloc until a CTA there ends.  So the
// shared memory asked for is raised until no more CTAs than the TMEM holds fit
// by shared memory (2 CTAs of 256 columns).  (The occupancy calculator answers
// one CTA for this kernel whatever its shared memory, while two run side by
// side.)  Returns the CTAs per SM, 0 on an error.
static int tc_resident(const void* fn, size_t need, int device, size_t* smem_out) {
  int per_sm = 0, reserved = 0;
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) !=
          cudaSuccess)
    return 0;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
  constexpr int kTmemCtas = 512 / kTcTmemCols;
  const size_t fixed = fa.sharedSizeBytes + (size_t)reserved;
  // smallest request with kTmemCtas + 1 CTAs over the SM's shared memory
  const size_t floor_req = (size_t)per_sm / (kTmemCtas + 1) + 1 > fixed
                               ? ((size_t)per_sm / (kTmemCtas + 1) + 1 - fixed + 127) / 128 * 128
                               : 0;
  const size_t smem = std::max(need, floor_req);
  int nb = (int)((size_t)per_sm / (smem + fixed));
  nb = std::min(nb, kTmemCtas);
  nb = std::min(nb, 2048 / kTcThreads);
  if (fa.numRegs > 0) nb = std::min(nb, 65536 / (fa.numRegs * kTcThreads));
  *smem_out = smem;
  return nb;
}

int launch_tensor(mpmi_session* s, TickArgs& a, bool traj, cudaStream_t st, int n_hint) {
  if (s->model->kind != kCar)
    return fail(MPMI_E_UNSUPPORTED, "the tensor-core rollout is compiled for the race car");
  const void* fn = traj ? tc_fn<true>() : tc_fn<false>();
  const size_t smem =
      kTcFixedSmem + (a.safety.has_track ? (size_t)a.safety.track.blob_bytes : 0);
  const int t = traj ? 1 : 0;
  if (s->tc_grid[t] == 0 || s->tc_smem[t] != smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kTcFixedSmem + kMaxTrackBytes));
    if (e != cudaSuccess) return fail(MPMI_E_CUDA, "cudaFuncSetAttribute (tensor)");
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTcThreads, smem);
    if (e != cudaSuccess || nb < 1)
      return fail(MPMI_E_UNSUPPORTED, "tensor-core tick cannot be resident");
    size_t req = smem;
    nb = std::max(1, tc_resident(fn, smem, s->ctx->device, &req));
    s->tc_grid[t] = nb * s->ctx->sm_count;
    s->tc_smem[t] = smem;
    s->tc_req[t] = req;
  }
  const int n_work = (n_hint > 0 && n_hint < s->n_slots) ? n_hint : s->n_slots;
  // one CTA per tile while the tiles do not fill the resident CTAs' first halves
  int grid = (n_work + kTcM - 1) / kTcM;
  if (grid > s->tc_grid[t]) grid = s->tc_grid[t];
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  const cudaError_t e =
      cudaLaunchKernel(fn, dim3(grid), dim3(kTcThreads), args, s->tc_req[t], st);
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("tensor-core tick launch: ") + cudaGetErrorString(e));
  return MPMI_OK;
}

}  // namespace mpmi
