// The fused MPMI-SC tick (Alg. 2) as one kernel launch.
//
// Per candidate slot: draw the candidate (Alg. 2 first step), lift it
// (Sec. IV-A), predict z <- K z for up to H steps with the safety test after
// every step and exit at the first violation (Alg. 2's while-loop, Sec. V-C.1),
// score ||xi - u_h||^2 (Sec. IV-D), and fold (H - ttv, cost, slot) into one
// 64-bit key whose minimum over all candidates is the least-intervention safe
// input or, if none is safe, the longest survivor.  The block that finishes
// last decodes the minimum into the tick's result on the device.
//
// Work layout: L lanes of a warp share one candidate.  Lane q of a group holds
// rows [qR, qR + R) of K in registers (R = n / L) and computes those rows of
// K z; the group exchanges the new z through a per-warp shared-memory buffer
// (double-buffered by step parity, one __syncwarp per step).  L = 1 keeps a
// whole candidate in one thread; with L = 1 a thread may also carry C
// candidates, and K may sit in shared memory instead of registers (KSMEM).
// Warps are persistent: warp w of the grid takes the warp-tiles (32 C / L
// candidates each) w, w + W, w + 2W, ... so K is loaded once per thread (or
// block) and the race-car track grid once per block.
#pragma once

#include <stdint.h>

#include "internal.h"
#include "philox.cuh"

namespace mpmi {

constexpr int kMaxBlock = 256;
constexpr unsigned kFull = 0xffffffffu;

// ---- shared-memory staging by the bulk-copy engine (TMA, non-tensor form) ----
// Thread 0 initialises an mbarrier, announces the byte count and issues
// cp.async.bulk copies global -> shared that complete on it; every thread waits
// on phase 0 before reading the staged data.  Each wait is bounded by
// kWaitCycles SM clocks (about a second); a block whose wait runs out skips its
// candidates and flags the tick instead of hanging.
constexpr long long kWaitCycles = 1ll << 31;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// bytes: a multiple of 16; dst and src 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}

// true once phase `parity` of the barrier has completed, false after kWaitCycles
// (a phase already complete costs one try, no clock reads)
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  if (bar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (bar_try(bar, parity)) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel on the stream still runs;
// grid_dep_wait() returns once that kernel has completed and its memory is
// visible (at once for a kernel launched without the attribute), and
// grid_dep_release() lets the next such kernel start launching.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Issues the copies of one staging (thread 0): K with padded rows (k_rows > 0,
// row r of n floats to word r * s4) and then `blob_bytes` of blob.
// With kp_bytes > 0 K is one contiguous blob (the pair layout) copied first instead.
__device__ __forceinline__ void stage_issue(uint64_t* bar, uint4* dst, const float* K, int k_rows,
                                            int k_cols, int s4, const uint4* blob, int blob_bytes,
                                            bool withhold, const float* Kp = nullptr,
                                            int kp_bytes = 0) {
  const uint32_t row_bytes = (uint32_t)k_cols * 4u;
  bar_expect(bar, (uint32_t)k_rows * row_bytes + (uint32_t)kp_bytes + (uint32_t)blob_bytes);
  if (withhold) return;
  for (int r = 0; r < k_rows; ++r) bulk_g2s(dst + r * s4, K + (size_t)r * k_cols, row_bytes, bar);
  if (kp_bytes > 0) bulk_g2s(dst, Kp, (uint32_t)kp_bytes, bar);
  uint4* bd = dst + k_rows * s4 + kp_bytes / 16;
  for (int off = 0; off < blob_bytes; off += 32768) {
    const int b = blob_bytes - off < 32768 ? blob_bytes - off : 32768;
    bulk_g2s(reinterpret_cast<char*>(bd) + off, reinterpret_cast<const char*>(blob) + off,
             (uint32_t)b, bar);
  }
}

// K staged in shared memory (KSMEM shapes): row r starts at 16-byte word r * S4,
// rows padded by four floats so that the L lanes of a group, which read L
// different rows at once, fall into different banks.  Within a row the columns
// are in staging order (staged_col): the free columns ascending, then the held
// ones ascending, so a prediction step reads only the free columns' words.
template <int N>
struct KSmem {
  static constexpr int S4 = (N + 4) / 4;    // 16-byte words per padded row
  static constexpr int WORDS = N * S4;
  static constexpr size_t BYTES = (size_t)WORDS * 16;
};

// Number of free (not held) columns of a basis.
MPMI_HD constexpr int free_cols(int kind, int n) {
  int nf = 0;
  for (int k = 0; k < n; ++k) nf += held_feature(kind, k) ? 0 : 1;
  return nf;
}

// Column of K at position p of a row in staging order, in closed form so that
// the unrolled step loops index z with constants (checked against held_feature
// below).  Bot: held 4, 11; race car: held 6, 7, 30, 31; linear bases: the held
// inputs already come last.
MPMI_HD constexpr int staged_col(int kind, int n, int p) {
  return kind == kBot   ? (p < 4 ? p : (p < 10 ? p + 1 : (p == 10 ? 4 : 11)))
         : kind == kCar ? (p < 6 ? p : (p < 28 ? p + 2 : (p < 30 ? p - 22 : p)))
                        : (n > 0 ? p : -1);
}

// staged_col lists the free columns ascending, then the held ones ascending.
constexpr bool staged_order_ok(int kind, int n) {
  const int nf = free_cols(kind, n);
  for (int p = 0; p < n; ++p) {
    const int c = staged_col(kind, n, p);
    if (c < 0 || c >= n || held_feature(kind, c) != (p >= nf)) return false;
    if (p > 0 && p != nf && staged_col(kind, n, p - 1) >= c) return false;
  }
  return true;
}
static_assert(staged_order_ok(kBot, 12) && staged_order_ok(kCar, 32) &&
                  staged_order_ok(kLin11, 2) && staged_order_ok(kLin22, 4) &&
                  staged_order_ok(kLin41, 5),
              "staging order");

// The i-th free (not held) feature of a basis, ascending, or the i-th held one,
// in closed form so that unrolled loops index z with constants (checked against
// held_feature below).  Bot: held 4, 11; race car: held 6, 7, 30, 31; linear
// bases: the held inputs come last.
MPMI_HD constexpr int nth_feature(int kind, int n, int i, bool held) {
  return kind == kBot   ? (held ? (i == 0 ? 4 : 11) : (i < 4 ? i : i + 1))
         : kind == kCar ? (held ? (i < 2 ? 6 + i : 28 + i) : (i < 6 ? i : i + 2))
                        : (held ? free_cols(kind, n) + i : i);
}

constexpr bool nth_feature_ok(int kind, int n) {
  const int nf = free_cols(kind, n);
  for (int i = 0; i < n; ++i) {
    const bool held = i >= nf;
    const int k = nth_feature(kind, n, held ? i - nf : i, held);
    if (k < 0 || k >= n || held_feature(kind, k) != held) return false;
    if (i > 0 && i != nf && nth_feature(kind, n, held ? i - nf - 1 : i - 1, held) >= k)
      return false;
  }
  return true;
}
static_assert(nth_feature_ok(kBot, 12) && nth_feature_ok(kCar, 32) && nth_feature_ok(kLin11, 2) &&
                  nth_feature_ok(kLin22, 4) && nth_feature_ok(kLin41, 5),
              "free and held feature order");

// K for the one- and two-lane shapes with K in shared memory, rows in pairs: the
// free rows go two at a time (free features 2p and 2p + 1) through packed
// two-wide FMAs (fma.rn.f32x2), each half of which is the same fused multiply-add
// of its own row's chain.  Pair p starts at 16-byte word p * STRIDE and holds WPP
// words: word j < NF / 2 is {K[r0][c], K[r1][c], K[r0][c'], K[r1][c']} for the
// free columns c = 2j-th and c' = (2j + 1)-th, ascending; the last NH / 2 words
// hold the held columns the same way; one word of padding follows, so that the
// two lanes of a two-lane group, which read pairs 2i and 2i + 1 at once, hit
// different banks.  One LDS.128 thus feeds two packed FMAs, and each packed FMA
// advances two rows' chains at once (the rows' FMA chains, not the FMA pipe,
// limit a step with one warp per sub-partition).  The model builds this copy on
// the host (model_upload); the kernels stage it verbatim.
template <int KIND>
struct KPair {
  static constexpr int N = BasisTraits<KIND>::N;
  static constexpr int NF = free_cols(KIND, N);
  static constexpr int NH = N - NF;
  static constexpr bool OK = (NF % 4 == 0) && (NH % 2 == 0) && NF >= 2 && (NF / 2) % 2 == 0;
  static constexpr int PAIRS = NF / 2;
  static constexpr int WPP = NF / 2 + NH / 2;  // 16-byte words per pair of rows
  static constexpr int STRIDE = WPP + 1;       // with the padding word
  static constexpr int WORDS = PAIRS * STRIDE;
  static constexpr size_t BYTES = (size_t)WORDS * 16;
};

// Whether a shape stages K in the pair layout: one or two lanes, K in shared
// memory, and the held rows copied (HELD; the no-allocation variant computes
// every row from the caller's K and keeps the row layout).
template <int KIND, int L, bool KSMEM, bool HELD>
MPMI_HD constexpr bool pair_k() {
  return KSMEM && (L == 1 || L == 2) && HELD && KPair<KIND>::OK;
}

// 16-byte words of K a shape stages in shared memory (the track grid follows).
template <int KIND, int L, bool KSMEM, bool HELD>
MPMI_HD constexpr int ksmem_words() {
  return !KSMEM ? 0 : (pair_k<KIND, L, KSMEM, HELD>() ? KPair<KIND>::WORDS
                                                       : KSmem<BasisTraits<KIND>::N>::WORDS);
}

// Float of the pair layout at (pair p, word w < STRIDE, element e) for a
// row-major K (0 in the padding word).
MPMI_HD float kpair_value(int kind, int n, const float* K, int p, int w, int e) {
  const int nf = free_cols(kind, n);
  if (2 * w >= n) return 0.f;
  const int r = nth_feature(kind, n, 2 * p + (e & 1), false);
  const int i = 2 * w + (e >> 1);
  const int c = i < nf ? nth_feature(kind, n, i, false) : nth_feature(kind, n, i - nf, true);
  return K[(size_t)r * n + c];
}

// K already in staging order (the model's staging copy) into padded rows.
template <int N>
__device__ __forceinline__ void stage_k(const float* Ks, uint4* dst, int tid, int nthreads) {
  constexpr int W = N / 4;
  const uint4* src = reinterpret_cast<const uint4*>(Ks);
  for (int i = tid; i < N * W; i += nthreads) dst[(i / W) * KSmem<N>::S4 + i % W] = __ldg(&src[i]);
}

// K in row-major column order (a caller's buffer) into padded rows in staging
// order, one float at a time.
template <int KIND>
__device__ __forceinline__ void stage_k_gather(const float* K, uint4* dst, int tid, int nthreads) {
  constexpr int N = BasisTraits<KIND>::N;
  float* d = reinterpret_cast<float*>(dst);
  for (int i = tid; i < N * N; i += nthreads) {
    const int r = i / N, p = i % N;
    d[r * 4 * KSmem<N>::S4 + p] = __ldg(K + r * N + staged_col(KIND, N, p));
  }
}

// Parameter records that carry a completion word for zero-copy host ticks.
template <class P, class = void>
struct HasSeq {
  static constexpr bool value = false;
};
template <class P>
struct HasSeq<P, decltype((void)sizeof(((P*)nullptr)->seq_out), void())> {
  static constexpr bool value = true;
};

// Parameter records that carry a screened tick's first result (TickArgs).
template <class P, class = void>
struct HasSkip {
  static constexpr bool value = false;
};
template <class P>
struct HasSkip<P, decltype((void)sizeof(((P*)nullptr)->skip_if_safe), void())> {
  static constexpr bool value = true;
};

// A screened tick's fallback launch (skip_if_safe set) has nothing to do when the
// kept slots held a safe candidate or were already every slot of the tick.
template <class P>
__device__ __forceinline__ bool fallback_not_needed(const P& a) {
  if (a.skip_if_safe == nullptr) return false;
  const mpmi_result* p = a.skip_if_safe;
  return p->status == MPMI_SAFE || p->n_slots >= a.n_slots;
}

// The values that change from tick to tick: the Philox counter words of the
// tick, the tick itself, u_h (float64, device) and the completion number of a
// zero-copy host tick.  Normally the launch's parameters; a persistent kernel
// takes them from its command record.
struct TickDyn {
  uint32_t t_lo, t_hi;
  unsigned long long tick, seq;
  const double* u_h;
};

template <class P>
__device__ __forceinline__ TickDyn dyn_of(const P& a) {
  TickDyn d;
  d.t_lo = a.t_lo;
  d.t_hi = a.t_hi;
  d.tick = a.tick;
  d.u_h = a.u_h;
  if constexpr (HasSeq<P>::value) d.seq = a.seq;
  else d.seq = 0;
  return d;
}

// Alg. 2 first step: the input held by candidate `slot` in the tick whose
// counter words are (t_lo, t_hi).
template <int NU, class P>
__device__ __forceinline__ void candidate_value(const P& a, uint32_t t_lo, uint32_t t_hi,
                                                int slot, const float* uh32, float* xi) {
  if (a.include_user && slot == 0) {
#pragma unroll
    for (int j = 0; j < NU; ++j) xi[j] = uh32[j];
    return;
  }
  const int i = slot - a.include_user;
  if (a.sampler == MPMI_SAMPLER_UNIFORM) {
    const U32x4 w = philox4x32_10(U32x4{(uint32_t)i, t_lo, t_hi, a.stream}, a.key0, a.key1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      const float u = (float)(ws[j] >> 8) * 0x1p-24f;  // exact: 24-bit integer
      xi[j] = __fadd_rn(a.in_lo[j], __fmul_rn(a.in_w[j], u));
    }
  } else if (a.sampler == MPMI_SAMPLER_GRID) {
    int rem = i;
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      const int gj = rem % a.grid_g;
      rem /= a.grid_g;
      const double span = __dsub_rn(a.in_hi64[j], a.in_lo64[j]);
      const double v = __dadd_rn(
          __ddiv_rn(__dmul_rn((double)gj + 0.5, span), (double)a.grid_g), a.in_lo64[j]);
      xi[j] = __double2float_rn(v);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NU; ++j) xi[j] = a.ext[(size_t)i * NU + j];
  }
}

template <int NU, class P>
__device__ __forceinline__ void candidate_value(const P& a, int slot, const float* uh32,
                                                float* xi) {
  candidate_value<NU>(a, a.t_lo, a.t_hi, slot, uh32, xi);
}

// Two standard normals from two Philox words (Box & Muller, Ann. Math. Stat. 29,
// 1958): u1 = ((w_a >> 8) + 1) 2^-24 in (0, 1], u2 = (w_b >> 8) 2^-24 in [0, 1),
// both exact in binary32; n = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1) {
  const float u1 = (float)((wa >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(wb >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.f * logf(u1));
  float s, c;
  sincospif(2.f * u2, &s, &c);
  n0 = r * c;
  n1 = r * s;
}

// Alg. 2's noise z_i after prediction step t of candidate `slot`: the state
// coordinates j < n_noise get sigma_j n_j.  Block b (coordinates 4b..4b+3) is
// one Philox call with counter (slot, tick lo, (tick hi mod 2^16) + 2^16 t +
// 2^25 b, stream); its words pair as (w0, w1) -> 4b, 4b+1 and (w2, w3) -> 4b+2,
// 4b+3.  Since t >= 1 these counters never meet a candidate counter.
template <int NX, class P>
__device__ __forceinline__ void add_noise(const P& a, TickDyn d, int slot, int t, float* z) {
  constexpr int NB = (NX + 3) / 4;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (4 * b < a.n_noise) {
      const uint32_t c2 = (d.t_hi & 0xFFFFu) + ((uint32_t)t << 16) + ((uint32_t)b << 25);
      const U32x4 w = philox4x32_10(U32x4{(uint32_t)slot, d.t_lo, c2, a.stream}, a.key0, a.key1);
      float n[4];
      box_muller(w.x, w.y, n[0], n[1]);
      box_muller(w.z, w.w, n[2], n[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * b + j < NX) z[4 * b + j] = __fmaf_rn(a.noise_sigma[4 * b + j], n[j], z[4 * b + j]);
    }
  }
}

// Input monomials p_k(xi) of the split lifting, float32.
template <int KIND>
__device__ __forceinline__ void monomials32(const float* xi, float* p) {
  if constexpr (KIND == kCar) {
    p[0] = xi[0];
    p[1] = xi[1];
    p[2] = __fmul_rn(xi[0], xi[0]);
  } else {
#pragma unroll
    for (int k = 0; k < BasisTraits<KIND>::NP; ++k) p[k] = xi[k];
  }
}

// isSafe on the box part: lo < x_j < hi for every state coordinate (NaN fails).
template <int NX>
__device__ __forceinline__ bool box_ok(const DevSafety& s, const float* z) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < NX; ++j) ok = ok & (z[j] > s.lo[j]) & (z[j] < s.hi[j]);
  return ok;
}

// Shared-memory view of the staged track grid.
struct TrackView {
  const uint32_t* cells;
  const uint16_t* list;
  const float4* seg;
  const float* inv;
};

// isSafe on the track part, shared by the L lanes of a group: lane q tests list
// entries q, q + L, ... (nearest first, stops at the first hit); the group ORs
// through one warp vote.  Non-short-circuit boolean operators keep the tests
// independent (fewer dependent branches on the step's critical path).
template <int L>
__device__ __forceinline__ bool track_ok(const DevTrack& tr, const TrackView& v, float px,
                                         float py, int q, bool active) {
  bool ok = false;
  if (active) {
    const float fx = (px - tr.gx0) * tr.inv_h;
    const float fy = (py - tr.gy0) * tr.inv_h;
    if ((fx >= 0.f) & (fx < (float)tr.gnx) & (fy >= 0.f) & (fy < (float)tr.gny)) {
      const uint32_t c = v.cells[(int)fy * tr.gnx + (int)fx];
      const uint32_t cls = c & 3u;
      if (cls == kCellInside) {
        ok = true;
      } else if (cls == kCellBoundary) {
        const int off = (int)((c >> 2) & 0x3FFFFFu), cnt = (int)(c >> 24);
        // J independent segment tests per lane and round, J L >= 16 entries per
        // round for the group (lists hold ~7-15; entries past the list end
        // repeat its last entry); the OR over the list is unchanged
        constexpr int J = L >= 16 ? 1 : (L >= 8 ? 2 : 4);
        for (int i0 = q; i0 < cnt; i0 += J * L) {
          bool hit = false;
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const int s = v.list[off + min(i0 + j * L, cnt - 1)];
            const float4 sg = v.seg[s];
            const float rx = px - sg.x, ry = py - sg.y;
            const float t = fminf(fmaxf((rx * sg.z + ry * sg.w) * v.inv[s], 0.f), 1.f);
            const float ex = rx - t * sg.z, ey = ry - t * sg.w;
            hit = hit | (ex * ex + ey * ey < tr.w2);
          }
          if (hit) {
            ok = true;
            break;
          }
        }
      }
    }
  }
  if constexpr (L > 1) {
    // OR over the group's L lanes: one warp vote, then the group's bits
    const unsigned int votes = __ballot_sync(kFull, ok);
    const int base = (int)(threadIdx.x & 31) & ~(L - 1);
    ok = ((votes >> base) & ((L == 32) ? kFull : ((1u << L) - 1u))) != 0u;
  }
  return ok;
}

// Decode of the winning key into the tick's result record.
template <int NU, class P>
__device__ __forceinline__ void write_result(const P& a, TickDyn d, unsigned long long k,
                                             unsigned long long cnt, const float* uh,
                                             bool timed_out = false) {
  const int pick = (int)(k & 0x7FFFFFull);
  const int hm = (int)(k >> 55);
  mpmi_result r;
  float xb[NU];
  candidate_value<NU>(a, d.t_lo, d.t_hi, pick, uh, xb);
#pragma unroll
  for (int j = 0; j < MPMI_MAX_NU; ++j) r.u_r[j] = 0.0;
#pragma unroll
  for (int j = 0; j < NU; ++j)
    r.u_r[j] = (a.include_user && pick == 0) ? d.u_h[j] : (double)xb[j];
  r.index = pick;
  r.status = timed_out ? MPMI_TIMEOUT : (hm == 0 ? MPMI_SAFE : MPMI_FALLBACK);
  r.n_safe = (int32_t)(cnt >> 40);
  r.ttv = a.horizon - hm;
  r.cost = __uint_as_float((unsigned int)((k >> 23) & 0xFFFFFFFFull));
  r.n_slots = a.n_list ? *a.n_list : a.n_slots;
  r.executed_steps = cnt & ((1ull << 40) - 1);
  if constexpr (HasSkip<P>::value) {
    // a fallback launch reports the steps of the whole screened tick
    if (a.skip_if_safe != nullptr) r.executed_steps += a.skip_if_safe->executed_steps;
  }
  r.tick = d.tick;
  r.reserved = a.result_flags;
  *a.result = r;
  if constexpr (HasSeq<P>::value) {
    const bool final_result =
        !a.seq_if_final || r.status == MPMI_SAFE || r.n_slots >= a.n_slots;
    if (a.seq_out != nullptr && final_result) {  // the host polls this word instead of an event
      __threadfence_system();
      *reinterpret_cast<volatile unsigned long long*>(a.seq_out) = d.seq;
    }
  }
}

template <int NU, class P>
__device__ __forceinline__ void write_result(const P& a, unsigned long long k,
                                             unsigned long long cnt, const float* uh,
                                             bool timed_out = false) {
  write_result<NU>(a, dyn_of(a), k, cnt, uh, timed_out);
}

// One word (positions 4 w .. 4 w + 3) of a row of K in staging order: its part of
// the FMA chain of that row of K z.
template <int KIND>
__device__ __forceinline__ void fma_word(const float4 kv, const float* z, int w, float& v) {
  constexpr int N = BasisTraits<KIND>::N;
  v = __fmaf_rn(kv.x, z[staged_col(KIND, N, 4 * w)], v);
  v = __fmaf_rn(kv.y, z[staged_col(KIND, N, 4 * w + 1)], v);
  v = __fmaf_rn(kv.z, z[staged_col(KIND, N, 4 * w + 2)], v);
  v = __fmaf_rn(kv.w, z[staged_col(KIND, N, 4 * w + 3)], v);
}

// One warp-tile: the PER_WARP = 32 C / L candidate positions wt * PER_WARP ...
// of a tick (Alg. 2 for each: sample, lift, predict with early exit, test,
// score), folded into the caller's running key minimum and counts.  P is the
// tick's parameter record (TickArgs, or a served session's record).  HELD: the
// operator's held-feature rows are exact unit rows (true for every model the
// library built), so the one-lane shapes copy those coordinates instead of
// recomputing them -- bit for bit the same z for finite states.
//
// Row order of z <- K z: every shape sums row r as one FMA chain, first over the
// held columns (ascending), then over the others (ascending).  With HELD the held
// coordinates of z stay at their lifted values for the whole horizon (the input
// is held, Sec. VII-B), so the first part of the chain is the same number at
// every step: it is summed once per candidate (hc) and each step continues the
// chain from it -- the same rounding as summing it every step.
template <int KIND, int L, int C, bool KSMEM, bool TRAJ, bool NOISE, bool HELD, class P,
          class KR>
__device__ __forceinline__ void run_tile(const P& a, TickDyn d, const DevSafety& safety,
                                         int wt, int n_eval,
                                         const float* xs, const float* uh, float sn, float cs,
                                         const KR& kr, const float4* sK4, const TrackView& tv,
                                         float* xbuf, unsigned long long& best,
                                         unsigned int& n_safe, unsigned int& n_exec) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU, NP = B::NP;
  constexpr int R = N / L;
  constexpr int GPW = 32 / L;
  constexpr int S = (N % 32 == 0) ? N + 4 : ((N % 4 == 0) ? N : N + (4 - N % 4));
  constexpr int NF = free_cols(KIND, N);  // free columns: staged words [0, NF / 4)
  static_assert(!KSMEM || NF % 4 == 0, "K in shared memory needs whole words of free columns");
  // Every launch shape sums each row of K z in the same order (one FMA chain,
  // held columns first; see above), so all shapes produce bit-identical
  // trajectories and decisions.
  constexpr int PER_WARP = GPW * C;
  const int lane = threadIdx.x & 31, q = lane % L, g = lane / L;
  const int H = a.horizon;
  int slot[C];
  bool valid[C], alive[C];
  float cost[C];
  int ttv[C];
  float z[C][N];
  float* traj[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int pos = wt * PER_WARP + c * GPW + g;
    valid[c] = pos < n_eval;
    slot[c] = (valid[c] && a.slot_list) ? a.slot_list[pos] : pos;
    float xi[NU];
    if (valid[c]) {
      candidate_value<NU>(a, d.t_lo, d.t_hi, slot[c], uh, xi);
    } else {
#pragma unroll
      for (int j = 0; j < NU; ++j) xi[j] = uh[j];
    }
    cost[c] = 0.f;
#pragma unroll
    for (int j = 0; j < NU; ++j) {
      const float d = __fsub_rn(xi[j], uh[j]);
      cost[c] = __fmaf_rn(d, d, cost[c]);
    }
    // lift: z_0 = a(x_t) + sum_k p_k(xi) b_k(x_t)
    float p[NP];
    monomials32<KIND>(xi, p);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float av, bv[kMaxP];
      feature_split<float>(KIND, j, xs, sn, cs, &av, bv);
#pragma unroll
      for (int k = 0; k < NP; ++k) av = __fmaf_rn(p[k], bv[k], av);
      z[c][j] = av;
    }
    traj[c] = nullptr;
    if constexpr (TRAJ) {
      if (valid[c] && q == 0) {
        traj[c] = a.traj_out + (size_t)slot[c] * (H + 1) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) traj[c][j] = z[c][j];
      }
    }
    ttv[c] = 0;
    alive[c] = valid[c];
  }

  // the held columns' share of each row this lane computes (HELD only)
  constexpr int HR = (L == 1) ? N : R;  // rows per candidate held in hc
  constexpr bool PK = pair_k<KIND, L, KSMEM, HELD>();
  using KP = KPair<KIND>;
  float hc[HELD && !PK ? C : 1][HELD && !PK ? HR : 1];
  // with two lanes, lane q takes the pairs q, q + 2, ...: MYP pairs; pair i of
  // this lane is pair_of(i)
  constexpr int MYP = PK ? KP::PAIRS / L : 1;
  const auto pair_of = [q](int i) { return L == 1 ? i : q + L * i; };
  float2 hp[PK ? C : 1][MYP];  // the held columns' share, two rows per pair
  if constexpr (PK) {
    // held words of pair p: columns (held 2j, held 2j + 1) of both rows
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int pp = 0; pp < MYP; ++pp) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < KP::NH / 2; ++j) {
          const float4 w = sK4[pair_of(pp) * KP::STRIDE + KP::NF / 2 + j];
          const float z0 = z[c][nth_feature(KIND, N, 2 * j, true)];
          const float z1 = z[c][nth_feature(KIND, N, 2 * j + 1, true)];
          v = __ffma2_rn(make_float2(w.x, w.y), make_float2(z0, z0), v);
          v = __ffma2_rn(make_float2(w.z, w.w), make_float2(z1, z1), v);
        }
        hp[c][pp] = v;
      }
    }
  } else if constexpr (HELD) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int r = 0; r < HR; ++r) {
        if (L == 1 && held_feature(KIND, r)) continue;  // copied, never summed
        float v = 0.f;
        if constexpr (KSMEM) {
          const float4* row = sK4 + ((L == 1) ? r : (q + L * r)) * KSmem<N>::S4;
#pragma unroll
          for (int w = NF / 4; w < N / 4; ++w) fma_word<KIND>(row[w], z[c], w, v);
        } else {
#pragma unroll
          for (int k = 0; k < N; ++k)
            if (held_feature(KIND, k)) v = __fmaf_rn(kr[r][k], z[c][k], v);
        }
        hc[c][r] = v;
      }
    }
  }

  // this lane's first PREG pairs' free words stay in registers for the whole
  // horizon (fewer shared-memory wavefronts per step; the registers a single
  // candidate per thread leaves free)
  constexpr int PREG = (PK && C == 1) ? 2 : 0;
  float4 kreg[PREG > 0 ? PREG : 1][PREG > 0 ? KP::NF / 2 : 1];
  if constexpr (PREG > 0) {
#pragma unroll
    for (int pp = 0; pp < PREG; ++pp)
#pragma unroll
      for (int j = 0; j < KP::NF / 2; ++j) kreg[pp][j] = sK4[pair_of(pp) * KP::STRIDE + j];
  }
  for (int t = 1; t <= H; ++t) {
    if constexpr (PK) {
      // z <- K z with the free rows in pairs (see KPair): per pair one chain of
      // packed FMAs, continuing from the held columns' share, over the free
      // columns ascending; the held rows are copied.  With two lanes each lane
      // computes its pairs and the group exchanges the new free coordinates
      // through the warp's buffer (double-buffered by step parity).
      asm volatile("" ::: "memory");
      float2 nv[C][MYP];
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int pp = 0; pp < MYP; ++pp) nv[c][pp] = hp[c][pp];
      // one packed FMA of pair pp, candidate c, over free word j (two columns)
      const auto pair_word = [&](int pp, int j) {
        const float4 w = pp < PREG ? kreg[pp < PREG ? pp : 0][j]
                                   : sK4[pair_of(pp) * KP::STRIDE + j];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float z0 = z[c][nth_feature(KIND, N, 2 * j, false)];
          const float z1 = z[c][nth_feature(KIND, N, 2 * j + 1, false)];
          nv[c][pp] = __ffma2_rn(make_float2(w.x, w.y), make_float2(z0, z0), nv[c][pp]);
          nv[c][pp] = __ffma2_rn(make_float2(w.z, w.w), make_float2(z1, z1), nv[c][pp]);
        }
      };
      // Each pair's chain runs over the free words in ascending order either way;
      // only the interleaving of the chains differs.  One lane: word-major (all
      // 14 chains advance together, hiding the packed FMA's latency); two lanes:
      // pair-major (measured faster there, 60.0 against 61.0 us at N = 16384).
      if constexpr (L == 1) {
#pragma unroll
        for (int j = 0; j < KP::NF / 2; ++j)
#pragma unroll
          for (int pp = 0; pp < MYP; ++pp) pair_word(pp, j);
      } else {
#pragma unroll
        for (int pp = 0; pp < MYP; ++pp)
#pragma unroll
          for (int j = 0; j < KP::NF / 2; ++j) pair_word(pp, j);
      }
      if constexpr (L == 1) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
          for (int pp = 0; pp < MYP; ++pp) {
            z[c][nth_feature(KIND, N, 2 * pp, false)] = nv[c][pp].x;
            z[c][nth_feature(KIND, N, 2 * pp + 1, false)] = nv[c][pp].y;
          }
      } else {
        // the group's new free coordinates in free-feature order
        float* buf = xbuf + ((t & 1) * GPW + g) * S;
#pragma unroll
        for (int pp = 0; pp < MYP; ++pp)
          *reinterpret_cast<float2*>(buf + 2 * pair_of(pp)) = nv[0][pp];
        __syncwarp();
#pragma unroll
        for (int w4 = 0; w4 < KP::NF / 4; ++w4) {
          const float4 v = *reinterpret_cast<const float4*>(buf + 4 * w4);
          z[0][nth_feature(KIND, N, 4 * w4, false)] = v.x;
          z[0][nth_feature(KIND, N, 4 * w4 + 1, false)] = v.y;
          z[0][nth_feature(KIND, N, 4 * w4 + 2, false)] = v.z;
          z[0][nth_feature(KIND, N, 4 * w4 + 3, false)] = v.w;
        }
      }
    } else if constexpr (KSMEM && L == 1) {
      // z <- K z with K read from shared memory (one broadcast LDS.128 feeds 4 C
      // FMAs).  The empty asm keeps the compiler from hoisting the loop-invariant
      // K loads out of the step loop (1024 values would not fit in registers).
      asm volatile("" ::: "memory");
      float acc[C][N];
#pragma unroll
      for (int r = 0; r < N; ++r) {
        if (HELD && held_feature(KIND, r)) {  // unit row: the feature is held
#pragma unroll
          for (int c = 0; c < C; ++c) acc[c][r] = z[c][r];
          continue;
        }
        float av[C];
        if constexpr (HELD) {
#pragma unroll
          for (int c = 0; c < C; ++c) av[c] = hc[c][r];
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c) av[c] = 0.f;
#pragma unroll
          for (int w = NF / 4; w < N / 4; ++w) {
            const float4 kv = sK4[r * KSmem<N>::S4 + w];
#pragma unroll
            for (int c = 0; c < C; ++c) fma_word<KIND>(kv, z[c], w, av[c]);
          }
        }
#pragma unroll
        for (int w = 0; w < NF / 4; ++w) {
          const float4 kv = sK4[r * KSmem<N>::S4 + w];
#pragma unroll
          for (int c = 0; c < C; ++c) fma_word<KIND>(kv, z[c], w, av[c]);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c][r] = av[c];
      }
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int r = 0; r < N; ++r) z[c][r] = acc[c][r];
    } else if constexpr (L == 1) {
      float zn[C][N];
#pragma unroll
      for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int r = 0; r < N; ++r) {
          if (HELD && held_feature(KIND, r)) {  // unit row: the feature is held
            zn[c][r] = z[c][r];
            continue;
          }
          float v = 0.f;
          if constexpr (HELD) {
            v = hc[c][r];
          } else {
#pragma unroll
            for (int k = 0; k < N; ++k)
              if (held_feature(KIND, k)) v = __fmaf_rn(kr[r][k], z[c][k], v);
          }
#pragma unroll
          for (int k = 0; k < N; ++k)
            if (!held_feature(KIND, k)) v = __fmaf_rn(kr[r][k], z[c][k], v);
          zn[c][r] = v;
        }
      }
#pragma unroll
      for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < N; ++j) z[c][j] = zn[c][j];
    } else {
      // L lanes per candidate: this lane's rows, then exchange through shared
      // memory.  K in registers: rows [qR, qR + R).  K in shared memory: rows
      // q, q + L, ..., so the L rows read at once are consecutive padded rows in
      // distinct banks.
      float zn[R];
      if constexpr (KSMEM) {
        asm volatile("" ::: "memory");
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float4* row = sK4 + (q + L * r) * KSmem<N>::S4;
          float v = 0.f;
          if constexpr (HELD) {
            v = hc[0][r];
          } else {
#pragma unroll
            for (int w = NF / 4; w < N / 4; ++w) fma_word<KIND>(row[w], z[0], w, v);
          }
#pragma unroll
          for (int w = 0; w < NF / 4; ++w) fma_word<KIND>(row[w], z[0], w, v);
          zn[r] = v;
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float v = 0.f;
          if constexpr (HELD) {
            v = hc[0][r];
          } else {
#pragma unroll
            for (int k = 0; k < N; ++k)
              if (held_feature(KIND, k)) v = __fmaf_rn(kr[r][k], z[0][k], v);
          }
#pragma unroll
          for (int k = 0; k < N; ++k)
            if (!held_feature(KIND, k)) v = __fmaf_rn(kr[r][k], z[0][k], v);
          zn[r] = v;
        }
      }
      float* buf = xbuf + ((t & 1) * GPW + g) * S;
      if constexpr (KSMEM) {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[q + L * r] = zn[r];
      } else if constexpr (R % 4 == 0) {
#pragma unroll
        for (int r = 0; r < R; r += 4)
          *reinterpret_cast<float4*>(buf + q * R + r) =
              make_float4(zn[r], zn[r + 1], zn[r + 2], zn[r + 3]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[q * R + r] = zn[r];
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < N; k += 4) {
        const float4 v = *reinterpret_cast<const float4*>(buf + k);
        z[0][k] = v.x; z[0][k + 1] = v.y; z[0][k + 2] = v.z; z[0][k + 3] = v.w;
      }
    }
    if constexpr (NOISE) {
#pragma unroll
      for (int c = 0; c < C; ++c)
        if (alive[c]) add_noise<NX>(a, d, slot[c], t, z[c]);
    }
    bool any_alive = false;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if constexpr (TRAJ) {
        if (traj[c] != nullptr && alive[c]) {
#pragma unroll
          for (int j = 0; j < N; ++j) traj[c][(size_t)t * N + j] = z[c][j];
        }
      }
      bool ok = box_ok<NX>(safety, z[c]);
      if constexpr (B::TRACK) {
        if (safety.has_track) {  // uniform over the grid
          const bool on_road =
              track_ok<L>(safety.track, tv, z[c][0], z[c][1], q, alive[c] && ok);
          ok = ok && on_road;
        }
      }
      if (alive[c]) {
        if (ok) ttv[c] = t;
        else alive[c] = false;
      }
      any_alive = any_alive || alive[c];
    }
    if (!__any_sync(kFull, any_alive)) break;
  }

#pragma unroll
  for (int c = 0; c < C; ++c) {
    if (valid[c]) {
      // selection key: (H - ttv) | cost bits | slot -> lexicographic minimum
      const unsigned long long key = ((unsigned long long)(H - ttv[c]) << 55) |
                                     ((unsigned long long)__float_as_uint(cost[c]) << 23) |
                                     (unsigned long long)slot[c];
      best = key < best ? key : best;
      if (q == 0) {
        n_exec += (unsigned int)min(ttv[c] + 1, H);
        n_safe += ttv[c] == H;
        if (a.ttv_out) a.ttv_out[slot[c]] = ttv[c];
        if (a.cost_out) a.cost_out[slot[c]] = cost[c];
      }
    }
  }
}

// End of a tick launch: warp -> block -> grid reduction of the selection key
// and the counts into the session's reduction record (one atomicMin/atomicAdd per
// block); the block that finishes last decodes the result and resets the record.
// MAXW: the most warps a launch's blocks have.
template <int NU, class P, int MAXW = kMaxBlock / 32>
__device__ __forceinline__ void session_epilogue(const P& a, TickDyn d,
                                                 unsigned long long best, unsigned int n_safe,
                                                 unsigned int n_exec, const float* uh,
                                                 bool failed = false,
                                                 unsigned int n_blocks = 0) {
  __shared__ unsigned long long s_key[MAXW];
  __shared__ unsigned long long s_cnt[MAXW];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wpb = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(kFull, best, o);
    best = other < best ? other : best;
    n_exec += __shfl_xor_sync(kFull, n_exec, o);
    n_safe += __shfl_xor_sync(kFull, n_safe, o);
  }
  if (lane == 0) {
    s_key[warp] = best;
    s_cnt[warp] = ((unsigned long long)n_safe << 40) + n_exec;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long bk = s_key[0], bc = s_cnt[0];
    for (int w = 1; w < wpb; ++w) {
      bk = s_key[w] < bk ? s_key[w] : bk;
      bc += s_cnt[w];
    }
    TickScratch* sc = a.scratch;
    atomicMin(&sc->key, bk);
    atomicAdd(&sc->counts, bc);
    if (failed) atomicOr(&sc->error, 1u);
    // acquire-release on the block counter: this block's atomics above are
    // visible before the increment, and the last block sees every other block's
    unsigned int prev;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&sc->done) : "memory");
    s_last = (prev == (n_blocks ? n_blocks : gridDim.x) - 1);
  }
  __syncthreads();
  if (s_last && tid == 0) {
    TickScratch* sc = a.scratch;
    const unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&sc->key);
    const unsigned long long cnt = *reinterpret_cast<volatile unsigned long long*>(&sc->counts);
    const unsigned int err = *reinterpret_cast<volatile unsigned int*>(&sc->error);
    // reset the record before publishing: a persistent kernel's next tick may
    // start as soon as the result is visible (the publish of a zero-copy tick
    // sits behind a system-scope fence, which orders these stores too)
    sc->key = ~0ull;
    sc->counts = 0ull;
    sc->error = 0u;
    sc->done = 0u;
    write_result<NU>(a, d, k, cnt, uh, err != 0u);
  }
}

template <int NU, class P, int MAXW = kMaxBlock / 32>
__device__ __forceinline__ void session_epilogue(const P& a, unsigned long long best,
                                                 unsigned int n_safe, unsigned int n_exec,
                                                 const float* uh, bool failed = false,
                                                 unsigned int n_blocks = 0) {
  session_epilogue<NU, P, MAXW>(a, dyn_of(a), best, n_safe, n_exec, uh, failed, n_blocks);
}

// Template parameters of the tick kernel:
//   L        lanes per candidate (K rows split across the lanes, see above);
//   C        candidates per thread (L = 1 only): more independent FMA chains;
//   KSMEM    K staged once per block in shared memory and read with broadcast
//            LDS.128 (L = 1 only) instead of held in registers: frees the
//            registers of a large K (race car, n = 32) for occupancy;
//   TRAJ     record every predicted z_t (parity checks);
//   PARTIALS no-allocation variant: each block stores its partial (key,
//            counts) in a.partials and the last block folds them, instead of
//            atomics on a session's reduction record;
//   NOISE    add Alg. 2's Gaussian noise z_i after every prediction step.
template <int KIND, int L, int C, bool KSMEM, bool TRAJ, bool PARTIALS = false,
          bool NOISE = false>
__global__ void __launch_bounds__(kMaxBlock) tick_kernel(const __grid_constant__ TickArgs a) {
  using B = BasisTraits<KIND>;
  constexpr int N = B::N, NX = B::NX, NU = B::NU;
  static_assert(N % L == 0, "lanes must divide the lifted dimension");
  static_assert(32 % L == 0, "lanes must divide the warp");
  static_assert(C == 1 || L == 1, "several candidates per thread need L = 1");
  static_assert(!KSMEM || N % 4 == 0, "K in shared memory needs n % 4 == 0");
  constexpr int R = N / L;              // rows of K per lane
  constexpr int GPW = 32 / L;           // candidate groups per warp
  constexpr int S = (N % 32 == 0) ? N + 4 : ((N % 4 == 0) ? N : N + (4 - N % 4));
  constexpr int NW = kMaxBlock / 32;
  constexpr int ANG = (KIND == kBot) ? 0 : ((KIND == kCar) ? 2 : -1);
  constexpr int KWORDS = ksmem_words<KIND, L, KSMEM, !PARTIALS>();  // 16-byte words of K
  constexpr bool PK = pair_k<KIND, L, KSMEM, !PARTIALS>();

  extern __shared__ uint4 s_dyn[];  // [K in staging order (KSMEM)] [track blob (race car)]
  __shared__ __align__(16) float s_x[(L > 1) ? NW : 1][2][GPW][S];
  __shared__ unsigned long long s_key[NW];
  __shared__ unsigned long long s_cnt[NW];
  __shared__ int s_last;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = lane % L;
  // a screened tick's launches run as a chain of programmatic dependents: this
  // one was allowed to launch early, so wait for the previous kernel's results
  // (the kept-slot list, the first result, the reset reduction record), then let
  // the next launch start
  if (a.chained) {
    grid_dep_wait();
    grid_dep_release();
  }
  // The session's reduction record is usually cold in L2 (other work ran since
  // the last tick): start fetching it now, so that the epilogue's atomics do
  // not wait for HBM on the tick's critical path.
  if constexpr (!PARTIALS) {
    if (tid == 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.scratch));
  }
  // a fallback launch has nothing to do when the screened result is already safe
  if (fallback_not_needed(a)) return;
  // number of candidates this launch evaluates (all slots, or a device-side list)
  const int n_eval = a.n_list ? *a.n_list : a.n_slots;
  // A launch over a device-side list is sized for the longest list; the blocks
  // past the ones the list's warp-tiles need leave at once (no staging, no
  // atomics) and the epilogue waits for the needed blocks only.  Launches over
  // all slots are sized exactly, so there every block is needed.
  unsigned int n_active = gridDim.x;
  if constexpr (!PARTIALS) {
    const int wpb0 = blockDim.x >> 5;
    const long long tiles = ((long long)n_eval + GPW * C - 1) / (GPW * C);
    const long long need = (tiles + wpb0 - 1) / wpb0;
    n_active = (unsigned int)(need < 1 ? 1 : (need < (long long)gridDim.x ? need : gridDim.x));
    if (blockIdx.x >= n_active) return;
  }

  // stage K (KSMEM) and the track grid (race car) while the per-tick state is
  // prepared: bulk copies on an mbarrier (plain loads in the no-allocation
  // variant, whose K pointer comes from the caller with no alignment promise)
  __shared__ uint64_t s_bar;
  constexpr bool BULK = !PARTIALS;
  const bool track_on = B::TRACK && a.safety.has_track;
  const bool staging = KSMEM || track_on;
  if constexpr (BULK) {
    if (staging) {
      if (tid == 0) bar_init(&s_bar);
      __syncthreads();
      if (tid == 0)
        stage_issue(&s_bar, s_dyn, a.Ks, (KSMEM && !PK) ? N : 0, N, KSmem<N>::S4,
                    a.safety.track.blob, track_on ? a.safety.track.blob_bytes : 0,
                    a.withhold_staging != 0, a.Kp, PK ? (int)KPair<KIND>::BYTES : 0);
    }
  } else {
    if constexpr (KSMEM) stage_k_gather<KIND>(a.K, s_dyn, tid, blockDim.x);
    if (track_on) {
      const int words = a.safety.track.blob_bytes >> 4;
      for (int i = tid; i < words; i += blockDim.x) s_dyn[KWORDS + i] = __ldg(&a.safety.track.blob[i]);
    }
  }
  TrackView tv{nullptr, nullptr, nullptr, nullptr};
  if constexpr (B::TRACK) {
    if (a.safety.has_track) {
      uint4* dst = s_dyn + KWORDS;
      const char* base = reinterpret_cast<const char*>(dst);
      tv.cells = reinterpret_cast<const uint32_t*>(base);
      tv.list = reinterpret_cast<const uint16_t*>(base + a.safety.track.off_list);
      tv.seg = reinterpret_cast<const float4*>(base + a.safety.track.off_seg);
      tv.inv = reinterpret_cast<const float*>(base + a.safety.track.off_inv);
    }
  }
  const float4* sK4 = reinterpret_cast<const float4*>(s_dyn);
  // per-tick state: x_t and u_h in float32, the basis angle's sine and cosine
  float xs[NX], uh[NU];
#pragma unroll
  for (int j = 0; j < NX; ++j) xs[j] = __double2float_rn(a.x_t[j]);
#pragma unroll
  for (int j = 0; j < NU; ++j) uh[j] = __double2float_rn(a.u_h[j]);
  float sn = 0.f, cs = 1.f;
  if constexpr (ANG >= 0) sincosf(xs[ANG], &sn, &cs);
  // this lane's rows of K (registers)
  float kr[KSMEM ? 1 : R][KSMEM ? 1 : N];
  if constexpr (!KSMEM) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float* row = a.K + (q * R + r) * N;
      if constexpr (N % 4 == 0) {
#pragma unroll
        for (int k = 0; k < N; k += 4) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(row + k));
          kr[r][k] = v.x; kr[r][k + 1] = v.y; kr[r][k + 2] = v.z; kr[r][k + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k) kr[r][k] = __ldg(row + k);
      }
    }
  }
  bool failed = false;
  if constexpr (BULK) {
    if (staging) {
      // a wait that runs out is retried once (copies may still be in flight), then
      // the whole block agrees to skip its candidates
      bool ok = bar_wait(&s_bar, 0);
      if (!ok) ok = bar_wait(&s_bar, 0);
      failed = __syncthreads_or(!ok) != 0;
    }
  } else {
    if constexpr (KSMEM || B::TRACK) __syncthreads();
  }

  unsigned long long best = ~0ull;
  unsigned int n_safe = 0, n_exec = 0;
  const int wpb = blockDim.x >> 5;
  constexpr int PER_WARP = GPW * C;  // candidate slots per warp-tile
  const int n_wtiles = failed ? 0 : (n_eval + PER_WARP - 1) / PER_WARP;
  for (int wt = blockIdx.x * wpb + warp; wt < n_wtiles; wt += gridDim.x * wpb)
    run_tile<KIND, L, C, KSMEM, TRAJ, NOISE, !PARTIALS>(a, dyn_of(a), a.safety, wt, n_eval, xs, uh, sn, cs, kr, sK4, tv,
                                      &s_x[L > 1 ? warp : 0][0][0][0], best, n_safe, n_exec);

  if constexpr (!PARTIALS) {
    session_epilogue<NU>(a, best, n_safe, n_exec, uh, failed, n_active);
  } else {
    // warp -> block reduction, then per-block partials folded by the last block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, best, o);
      best = other < best ? other : best;
      n_exec += __shfl_xor_sync(kFull, n_exec, o);
      n_safe += __shfl_xor_sync(kFull, n_safe, o);
    }
    if (lane == 0) {
      s_key[warp] = best;
      s_cnt[warp] = ((unsigned long long)n_safe << 40) + n_exec;
    }
    __syncthreads();
    {
      unsigned long long* pk = a.partials;
      unsigned long long* pc = a.partials + a.partials_cap;
      unsigned long long* blocks_done = a.partials + 2 * a.partials_cap;
      if (tid == 0) {
        unsigned long long bk = s_key[0], bc = s_cnt[0];
        for (int w = 1; w < wpb; ++w) {
          bk = s_key[w] < bk ? s_key[w] : bk;
          bc += s_cnt[w];
        }
        pk[blockIdx.x] = bk;
        pc[blockIdx.x] = bc;
        __threadfence();
        const unsigned long long prev = atomicAdd(blocks_done, 1ull);
        s_last = (prev == (unsigned long long)gridDim.x - 1);
      }
      __syncthreads();
      if (!s_last) return;
      __threadfence();
      unsigned long long k = ~0ull, cc = 0ull;
      for (int b = tid; b < (int)gridDim.x; b += blockDim.x) {
        const unsigned long long kb = *reinterpret_cast<volatile unsigned long long*>(pk + b);
        k = kb < k ? kb : k;
        cc += *reinterpret_cast<volatile unsigned long long*>(pc + b);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(kFull, k, o);
        k = other < k ? other : k;
        cc += __shfl_xor_sync(kFull, cc, o);
      }
      __syncthreads();
      if (lane == 0) {
        s_key[warp] = k;
        s_cnt[warp] = cc;
      }
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < wpb; ++w) {
          k = s_key[w] < k ? s_key[w] : k;
          cc += s_cnt[w];
        }
        write_result<NU>(a, k, cc, uh);
        *blocks_done = 0ull;
      }
    }
  }
}

// Alg. 2 first step alone (parity of the candidate stream).
template <int NU>
__global__ void sample_kernel(const __grid_constant__ TickArgs a, float* out) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= a.n_slots) return;
  float uh[NU];
#pragma unroll
  for (int j = 0; j < NU; ++j) uh[j] = a.include_user ? __double2float_rn(a.u_h[j]) : 0.f;
  float xi[NU];
  candidate_value<NU>(a, slot, uh, xi);
#pragma unroll
  for (int j = 0; j < NU; ++j) out[(size_t)slot * NU + j] = xi[j];
}

}  // namespace mpmi
