// The race car's rollout on the 5th-generation tensor cores (tcgen05).
//
// Batched over a tile of candidates, Alg. 2's prediction step is a matrix
// product: with the lifted states of 128 candidates as the rows of Z (128 x 32),
// one step is Z <- Z K^T (Sec. IV-A: one matrix-matrix product per step for a
// batch).  A CTA of 128 threads owns one tile at a time, thread i = candidate i =
// TMEM lane i:
//   1. thread i writes its z as two TF32 rows (hi = rna(z), lo = rna(z - hi)) into
//      the K-major shared-memory tiles A_hi, A_lo (8-row x 16-byte core
//      matrices, no swizzle);
//   2. one thread issues tcgen05.mma kind::tf32 over the four K blocks of 8:
//      A_hi [K_hi; K_lo]^T (N = 64, the K_lo tile directly follows K_hi, so one
//      operand covers both) into accumulator columns 0..63, then A_lo K_hi^T
//      (N = 32) into columns 0..31 -- eight MMAs in all -- and commits to an
//      mbarrier;
//   3. every thread reads its row of both column halves back with tcgen05.ld,
//      adds them (A_hi K_hi^T + A_lo K_hi^T + A_hi K_lo^T), restores the held
//      features exactly (their rows of K are unit rows), adds the noise z_i if
//      enabled, and runs the safety test.
// Dropping lo*lo leaves an error of the order of float32 rounding (measured:
// 4e-7 relative per product against float64, 1e-5 after 60 steps like the
// float32 FMA chain), so results agree with the oracle under the same
// tolerance but are not bit-identical to the CUDA-core shapes.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"
#include "tcgen05.cuh"
#include "tick_kernel.cuh"

namespace mpmi {

constexpr int kTcM = 128;  // candidates per tile = threads per CTA = TMEM lanes

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
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

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// Dynamic shared memory: A_hi | A_lo (16 KB each) | K_hi | K_lo (4 KB each) | track grid.
constexpr int kTcTileBytes = kTcM * 32 * 4;
constexpr int kTcKBytes = 32 * 32 * 4;
constexpr int kTcFixedSmem = 2 * kTcTileBytes + 2 * kTcKBytes;

template <int KIND, bool TRAJ>
__global__ void __launch_bounds__(kTcM) tc_tick_kernel(const __grid_constant__ TickArgs a) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU, NP = B::NP;
  static_assert(N == 32, "the tensor-core rollout is laid out for n = 32");
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  extern __shared__ __align__(1024) unsigned char s_tc[];
  unsigned char* ahi = s_tc;
  unsigned char* alo = s_tc + kTcTileBytes;
  unsigned char* bhi = s_tc + 2 * kTcTileBytes;
  unsigned char* blo = bhi + kTcKBytes;
  uint4* blob = reinterpret_cast<uint4*>(s_tc + kTcFixedSmem);
  __shared__ uint64_t s_bar_stage, s_bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5;
  if (fallback_not_needed(a)) return;
  const int n_eval = a.n_list ? *a.n_list : a.n_slots;
  const int H = a.horizon;
  const bool track_on = B::TRACK && a.safety.has_track;

  if (tid == 0) {
    bar_init(&s_bar_stage);
    bar_init(&s_bar_mma);
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
                     smem_u32(&s_tmem))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0 && track_on)
    stage_issue(&s_bar_stage, blob, nullptr, 0, 0, 0, a.safety.track.blob,
                a.safety.track.blob_bytes, a.withhold_staging != 0);
  // K split into TF32 hi and lo rows (row r of K = row r of the B operand)
  if (tid < N) {
#pragma unroll
    for (int c = 0; c < N / 4; ++c) {
      const float4 kv = __ldg(reinterpret_cast<const float4*>(a.K + tid * N) + c);
      const float kk[4] = {kv.x, kv.y, kv.z, kv.w};
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        h[e] = tf32_rna(kk[e]);
        l[e] = tf32_rna(kk[e] - __uint_as_float(h[e]));
      }
      *reinterpret_cast<uint4*>(bhi + tile_off(tid, 4 * c)) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4*>(blo + tile_off(tid, 4 * c)) = make_uint4(l[0], l[1], l[2], l[3]);
    }
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
  }

  const uint32_t a_hi = smem_u32(ahi), a_lo = smem_u32(alo);
  const uint32_t b_hi = smem_u32(bhi), b_lo = smem_u32(blo);
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  unsigned long long best = ~0ull;
  unsigned int n_safe = 0, n_exec = 0;
  const int n_tiles = failed ? 0 : (n_eval + kTcM - 1) / kTcM;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int pos = tile * kTcM + tid;
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
    for (int t = 1; t <= H; ++t) {
      // (1) this candidate's row of A_hi, A_lo
#pragma unroll
      for (int c = 0; c < N / 4; ++c) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          h[e] = tf32_rna(z[4 * c + e]);
          l[e] = tf32_rna(z[4 * c + e] - __uint_as_float(h[e]));
        }
        *reinterpret_cast<uint4*>(ahi + tile_off(tid, 4 * c)) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(alo + tile_off(tid, 4 * c)) = make_uint4(l[0], l[1], l[2], l[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // (2) Z K^T as hi*hi + hi*lo + lo*hi over the four K blocks of 8
      if (tid == 0) {
        // columns 0..31: A_hi K_hi^T + A_lo K_hi^T; columns 32..63: A_hi K_lo^T (B rows
        // 32..63 are the K_lo tile, which directly follows K_hi)
#pragma unroll
        for (int kb = 0; kb < N / 8; ++kb)
          mma_tf32(tmem, mat_desc(a_hi + kb * 256, 128, 1024), mat_desc(b_hi + kb * 256, 128, 1024),
                   kIdescTf32N64, kb ? 1u : 0u);
#pragma unroll
        for (int kb = 0; kb < N / 8; ++kb)
          mma_tf32(tmem, mat_desc(a_lo + kb * 256, 128, 1024), mat_desc(b_hi + kb * 256, 128, 1024),
                   kIdescTf32, 1u);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&s_bar_mma))
            : "memory");
      }
      // tcgen05.ld is warp-aligned: the warp decides as one
      const bool done = __all_sync(kFull, bar_wait(&s_bar_mma, phase));
      phase ^= 1u;
      if (!done) s_fail = 1;
      tc_fence_after();
      // (3) the new z: the accumulator row, held features restored exactly
      if (done) {
        float zn[N], zl[N];
        tmem_ld32(taddr, zn);
        tmem_ld32(taddr + 32, zl);
#pragma unroll
        for (int j = 0; j < N; ++j)
          if (!held_feature(KIND, j)) z[j] = __fadd_rn(zn[j], zl[j]);
      }
      if (a.n_noise > 0 && alive) add_noise<NX>(a, dyn_of(a), slot, t, z);
      if constexpr (TRAJ) {
        if (traj != nullptr && alive) {
#pragma unroll
          for (int j = 0; j < N; ++j) traj[(size_t)t * N + j] = z[j];
        }
      }
      bool ok = box_ok<NX>(a.safety, z);
      if constexpr (B::TRACK) {
        if (track_on) ok = ok && track_ok<1>(a.safety.track, tv, z[0], z[1], 0, alive && ok);
      }
      if (alive) {
        if (ok) ttv = t;
        else alive = false;
      }
      // every thread is done with the accumulator and the A tiles before the
      // next step overwrites them
      tc_fence_before();
      const bool any = __syncthreads_or(alive) != 0;
      tc_fence_after();
      if (s_fail) break;
      if (!any) break;
    }
    if (s_fail) {
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
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
  session_epilogue<NU>(a, best, n_safe, n_exec, uh, failed);
}

template <bool TRAJ>
static const void* tc_fn() {
  return reinterpret_cast<const void*>(&tc_tick_kernel<kCar, TRAJ>);
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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTcM, smem);
    if (e != cudaSuccess || nb < 1)
      return fail(MPMI_E_UNSUPPORTED, "tensor-core tick cannot be resident");
    s->tc_grid[t] = nb * s->ctx->sm_count;
    s->tc_smem[t] = smem;
  }
  const int n_work = (n_hint > 0 && n_hint < s->n_slots) ? n_hint : s->n_slots;
  int grid = (n_work + kTcM - 1) / kTcM;
  if (grid > s->tc_grid[t]) grid = s->tc_grid[t];
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kTcM), args, smem, st);
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("tensor-core tick launch: ") + cudaGetErrorString(e));
  return MPMI_OK;
}

}  // namespace mpmi
