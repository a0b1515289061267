// Factorised read-out rollout: an ablation of Alg. 2's prediction step.
//
// The candidate's input is held over the horizon and the lifting is affine in
// the input monomials, z_0 = a(x_t) + sum_k p_k(xi) b_k(x_t) (Sec. IV-A), so
// every predicted state coordinate j is
//     z_t[j] = e_j K^t a + sum_k p_k(xi) e_j K^t b_k,
// exact in real arithmetic.  Only the coordinates the safety test reads (those
// with a finite bound, and the position when a track is set) are needed.  Once
// per session `powers_kernel` forms the rows C K^t (C = the n_x state rows) for
// t = 1..H; per tick every block folds them with the split of the lifting at
// x_t into the table V[t][r] = (e_r K^t a, e_r K^t b_1, ...), after which a
// candidate-step costs (1 + P) FMAs per read-out coordinate instead of the n^2
// of z <- K z, and the steps of a candidate no longer depend on each other: the
// warp tests 32 of them at once.  Rounding differs from the full rollout.  The per-step noise of
// Alg. 2 enters after K and does not factor, so noisy sessions cannot use this.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"
#include "tick_kernel.cuh"

namespace mpmi {

constexpr int kFactBlock = 128;
constexpr int kFactCands = 8;  // candidates per warp-tile (lanes 0..7 draw them)

// Rows P_t = C K^t, t = 1..H: P_1 is the first NX rows of K and P_t = P_{t-1} K
// (each entry one FMA chain over i = 0..n-1).  One block of NX * N threads;
// out[((t - 1) NX + r) N + j].
template <int N, int NX>
__global__ void __launch_bounds__(256) powers_kernel(const float* K, int H, float* out) {
  __shared__ float sK[N][N];
  __shared__ float buf[2][NX][N];
  const int tid = threadIdx.x;
  for (int i = tid; i < N * N; i += blockDim.x) sK[i / N][i % N] = K[i];
  const int r = tid / N, j = tid % N;
  const bool act = tid < NX * N;
  if (act) {
    buf[0][r][j] = K[r * N + j];
    out[r * N + j] = K[r * N + j];
  }
  __syncthreads();
  for (int t = 2; t <= H; ++t) {
    const int src = t & 1, dst = src ^ 1;
    if (act) {
      float acc = 0.f;
      for (int i = 0; i < N; ++i) acc = __fmaf_rn(buf[src][r][i], sK[i][j], acc);
      buf[dst][r][j] = acc;
      out[((size_t)(t - 1) * NX + r) * N + j] = acc;
    }
    __syncthreads();
  }
}

// One tick in the factorised form.  Dynamic shared memory: [track grid (race
// car)] [V: H x ro_n float4, (a, b_1, b_2, b_3) coefficients per read-out].
template <int KIND>
__global__ void __launch_bounds__(256) factored_kernel(const __grid_constant__ TickArgs a) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU, NP = B::NP;
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  extern __shared__ uint4 s_dyn[];
  __shared__ float s_f[N][4];  // split of the lifting at x_t: a_j, b_1j, b_2j, b_3j

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (fallback_not_needed(a)) return;
  const int n_eval = a.n_list ? *a.n_list : a.n_slots;
  const int H = a.horizon, ro_n = a.ro_n;

  // the track grid arrives by bulk copy while the table V is built
  __shared__ uint64_t s_bar;
  const bool track_on = B::TRACK && a.safety.has_track;
  if (track_on) {
    if (tid == 0) bar_init(&s_bar);
    __syncthreads();
    if (tid == 0)
      stage_issue(&s_bar, s_dyn, nullptr, 0, 0, 0, a.safety.track.blob, a.safety.track.blob_bytes,
                  a.withhold_staging != 0);
  }
  TrackView tv{nullptr, nullptr, nullptr, nullptr};
  int track_words = 0;
  if constexpr (B::TRACK) {
    if (a.safety.has_track) {
      track_words = a.safety.track.blob_bytes >> 4;
      const char* base = reinterpret_cast<const char*>(s_dyn);
      tv.cells = reinterpret_cast<const uint32_t*>(base);
      tv.list = reinterpret_cast<const uint16_t*>(base + a.safety.track.off_list);
      tv.seg = reinterpret_cast<const float4*>(base + a.safety.track.off_seg);
      tv.inv = reinterpret_cast<const float*>(base + a.safety.track.off_inv);
    }
  }
  float4* V = reinterpret_cast<float4*>(s_dyn + track_words);

  float xs[NX], uh[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xs[j] = __double2float_rn(a.x_t[j]);
#pragma unroll
  for (int j = 0; j < NU; ++j) uh[j] = __double2float_rn(a.u_h[j]);
  float sn = 0.f, cs = 1.f;
  if constexpr (ANG >= 0) sincosf(xs[ANG], &sn, &cs);
  for (int j = tid; j < N; j += blockDim.x) {
    float av, bv[kMaxP];
    feature_split<float>(KIND, j, xs, sn, cs, &av, bv);
    s_f[j][0] = av;
#pragma unroll
    for (int k = 0; k < 3; ++k) s_f[j][1 + k] = k < NP ? bv[k] : 0.f;
  }
  __syncthreads();
  // V[t][r] = (P_t row ro_idx[r]) . (a, b_1, b_2, b_3)
  for (int e = tid; e < H * ro_n; e += blockDim.x) {
    const int t = e / ro_n, r = e - t * ro_n;
    const float* prow = a.ck + ((size_t)t * NX + a.ro_idx[r]) * N;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f;
#pragma unroll 8
    for (int j = 0; j < N; ++j) {
      const float pj = __ldg(prow + j);
      v0 = __fmaf_rn(pj, s_f[j][0], v0);
      v1 = __fmaf_rn(pj, s_f[j][1], v1);
      v2 = __fmaf_rn(pj, s_f[j][2], v2);
      v3 = __fmaf_rn(pj, s_f[j][3], v3);
    }
    V[e] = make_float4(v0, v1, v2, v3);
  }
  bool failed = false;
  if (track_on) {
    bool ok = bar_wait(&s_bar, 0);
    if (!ok) ok = bar_wait(&s_bar, 0);
    failed = __syncthreads_or(!ok) != 0;
  } else {
    __syncthreads();
  }

  // bounds of the read-out coordinates, in registers
  float lo[NX], hi[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    lo[r] = r < ro_n ? a.safety.lo[a.ro_idx[r]] : -INFINITY;
    hi[r] = r < ro_n ? a.safety.hi[a.ro_idx[r]] : INFINITY;
  }
  const bool track = B::TRACK && a.safety.has_track;  // read-outs 0, 1 are the position

  unsigned long long best = ~0ull;
  unsigned int n_safe = 0, n_exec = 0;
  const int wpb = blockDim.x >> 5;
  // Time-parallel: the read-outs of different steps do not depend on each other,
  // so a warp takes kFactCands candidates one after the other and tests 32 steps
  // of a candidate at once (lane l: step t0 + l + 1); a ballot gives the first
  // violation.
  const int n_wtiles = failed ? 0 : (n_eval + kFactCands - 1) / kFactCands;
  for (int wt = blockIdx.x * wpb + warp; wt < n_wtiles; wt += gridDim.x * wpb) {
    // lanes 0..kFactCands-1 draw and score one candidate each
    const int pos = wt * kFactCands + lane;
    const bool valid = lane < kFactCands && pos < n_eval;
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
    int my_ttv = 0;
    for (int c = 0; c < kFactCands; ++c) {
      if (!__shfl_sync(kFull, (int)valid, c)) continue;  // uniform over the warp
      float pc[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) pc[k] = __shfl_sync(kFull, p[k], c);
      int ttv = H;
      for (int t0 = 0; t0 < H; t0 += 32) {
        const int t = t0 + lane + 1;
        bool ok = true;
        if (t <= H) {
          const float4* Vt = V + (t - 1) * ro_n;
          float px = 0.f, py = 0.f;
#pragma unroll
          for (int r = 0; r < NX; ++r) {
            if (r < ro_n) {
              const float4 w = Vt[r];
              float v = __fmaf_rn(pc[0], w.y, w.x);
              if constexpr (NP > 1) v = __fmaf_rn(pc[1], w.z, v);
              if constexpr (NP > 2) v = __fmaf_rn(pc[2], w.w, v);
              ok = ok && (v > lo[r]) && (v < hi[r]);
              if (r == 0) px = v;
              if (r == 1) py = v;
            }
          }
          if constexpr (B::TRACK) {
            if (track) ok = ok && track_ok<1>(a.safety.track, tv, px, py, 0, ok);
          }
        }
        const unsigned bad = __ballot_sync(kFull, !ok);
        if (bad) {
          ttv = t0 + __ffs(bad) - 1;
          break;
        }
      }
      if (lane == c) my_ttv = ttv;
    }
    if (valid) {
      const unsigned long long key = ((unsigned long long)(H - my_ttv) << 55) |
                                     ((unsigned long long)__float_as_uint(cost) << 23) |
                                     (unsigned long long)slot;
      best = key < best ? key : best;
      n_exec += (unsigned int)min(my_ttv + 1, H);
      n_safe += my_ttv == H;
      if (a.ttv_out) a.ttv_out[slot] = my_ttv;
      if (a.cost_out) a.cost_out[slot] = cost;
    }
  }
  session_epilogue<NU>(a, best, n_safe, n_exec, uh, failed);
}

template <int KIND>
static const void* factored_fn() {
  return reinterpret_cast<const void*>(&factored_kernel<KIND>);
}

static const void* pick_factored(int kind) {
  switch (kind) {
    case kBot: return factored_fn<kBot>();
    case kCar: return factored_fn<kCar>();
    case kLin11: return factored_fn<kLin11>();
    case kLin22: return factored_fn<kLin22>();
    case kLin41: return factored_fn<kLin41>();
  }
  return nullptr;
}

int compute_powers(int kind, const float* K, int H, float* out, cudaStream_t st) {
  switch (kind) {
    case kBot: powers_kernel<12, 4><<<1, 4 * 12, 0, st>>>(K, H, out); break;
    case kCar: powers_kernel<32, 6><<<1, 6 * 32, 0, st>>>(K, H, out); break;
    case kLin11: powers_kernel<2, 1><<<1, 32, 0, st>>>(K, H, out); break;
    case kLin22: powers_kernel<4, 2><<<1, 32, 0, st>>>(K, H, out); break;
    case kLin41: powers_kernel<5, 4><<<1, 32, 0, st>>>(K, H, out); break;
    default: return fail(MPMI_E_UNSUPPORTED, "powers: unknown basis");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPMI_E_CUDA, std::string("powers kernel: ") + cudaGetErrorString(e));
  return MPMI_OK;
}

int launch_factored(mpmi_session* s, TickArgs& a, cudaStream_t st, int n_hint) {
  const void* fn = pick_factored(s->model->kind);
  if (!fn) return fail(MPMI_E_UNSUPPORTED, "factored kernel not compiled for this basis");
  const size_t track = a.safety.has_track ? (size_t)a.safety.track.blob_bytes : 0;
  const size_t smem = track + (size_t)a.horizon * a.ro_n * sizeof(float4);
  if (s->fact_grid == 0 || s->fact_smem != smem) {
    if (smem > 0) {
      const size_t cap = kMaxTrackBytes + (size_t)MPMI_MAX_HORIZON * MPMI_MAX_NX * sizeof(float4);
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)cap);
      if (e != cudaSuccess) return fail(MPMI_E_CUDA, "cudaFuncSetAttribute (factored)");
    }
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kFactBlock, smem);
    if (e != cudaSuccess || nb < 1)
      return fail(MPMI_E_UNSUPPORTED, "factored kernel cannot be resident");
    s->fact_grid = nb * s->ctx->sm_count;
    s->fact_smem = smem;
  }
  const int n_work = (n_hint > 0 && n_hint < s->n_slots) ? n_hint : s->n_slots;
  const int n_wtiles = (n_work + kFactCands - 1) / kFactCands;
  int grid = (n_wtiles + kFactBlock / 32 - 1) / (kFactBlock / 32);
  if (grid > s->fact_grid) grid = s->fact_grid;
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kFactBlock), args, smem, st);
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("factored kernel launch: ") + cudaGetErrorString(e));
  return MPMI_OK;
}

}  // namespace mpmi
