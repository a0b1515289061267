// Learned candidate screener (not in the paper): training kernels (float32),
// tensor-core inference (tcgen05, bfloat16 operands, float32 accumulation in
// TMEM), per-tick track features, and the screened tick (score -> threshold ->
// compaction -> exact rollout on the kept slots -> on-device fallback to the full
// evaluation).
//
// Network: 12 -> 128 -> 128 -> 1, GELU in its tanh form (Hendrycks & Gimpel),
// sigmoid output trained on ttv / H with the mean squared error and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"
#include "tcgen05.cuh"
#include "tick_kernel.cuh"

namespace mpmi {

constexpr int kH = 128, kIn = 12, kInP = 16;
constexpr int oW1 = 0, ob1 = kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH,
              ob3 = ow3 + kH, kP = ob3 + 1;
static_assert(kP == MPMI_SCREENER_PARAMS, "packed weight layout");
// histograms of the screened tick over cost bins: float32 bits of a cost >= 0
// shifted right by kBinShift (sign 0, exponent, three mantissa bits) < kBins
constexpr int kBins = 2048;
constexpr int kBinShift = 20;
constexpr float kGeluC = 0.7978845608028654f, kGeluA = 0.044715f;

// bfloat16 inference copy of the weights, laid out as the tensor cores' B operands:
// K-major tiles of 8-row x 16-byte core matrices without swizzle (bf_off), row j
// = unit j of the layer, K = its inputs (layer 1 padded from 12 to 16).  Staged
// verbatim into shared memory by every scoring block.
struct InferW {
  __nv_bfloat16 W1[kH * kInP];  // 128 x 16: 2 core matrices per 8-row group
  __nv_bfloat16 W2[kH * kH];    // 128 x 128: 16 core matrices per 8-row group
  float b1[kH], b2[kH], w3[kH];
  float b3, pad[3];
};
static_assert(sizeof(InferW) % 16 == 0, "InferW is staged with 16-byte copies");

// Byte offset of element (row, k) in a K-major bfloat16 tile with kc 8-element
// chunks per row: core matrix (row / 8, k / 8) holds 8 rows x 16 bytes; the
// chunks of a row group lie 128 B apart (the descriptor's leading byte offset),
// the row groups kc * 128 B apart (its stride byte offset).
__host__ __device__ constexpr uint32_t bf_off(int row, int k, int kc) {
  return (uint32_t)((((row >> 3) * kc + (k >> 3)) * 128) + (row & 7) * 16 + (k & 7) * 2);
}

struct ScreenScratch {
  unsigned int hist[kBins];       // all slots per cost bin
  unsigned int hist_safe[kBins];  // predicted-safe slots per cost bin
  unsigned int done;  // score blocks finished
  int bstar;          // threshold bin
  int n_list;         // kept slots
  int pad;
};

// ---------------------------------------------------------------- float32 training
__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.f + tanhf(kGeluC * (z + kGeluA * z * z * z)));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float t = tanhf(kGeluC * (z + kGeluA * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * (1.f + 3.f * kGeluA * z * z);
}

// Forward pass, one sample per thread; activations stored feature-major ([unit][B])
// so consecutive threads write consecutive addresses.  "aug" arrays carry a final
// row of ones, which turns the bias gradients into one more column of the GEMMs.
__global__ void __launch_bounds__(128) mlp_forward(const float* __restrict__ P,
                                                   const float* __restrict__ feats, int B,
                                                   float* faug, float* z1, float* h1aug,
                                                   float* z2, float* h2aug, float* y) {
  extern __shared__ float sP[];
  for (int i = threadIdx.x; i < kP; i += blockDim.x) sP[i] = P[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float f[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) {
    f[k] = feats[(size_t)b * kIn + k];
    faug[(size_t)k * B + b] = f[k];
  }
  faug[(size_t)kIn * B + b] = 1.f;
  float h1[kH];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float z = sP[ob1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) z = fmaf(sP[oW1 + j * kIn + k], f[k], z);
    z1[(size_t)j * B + b] = z;
    h1[j] = gelu_f(z);
    h1aug[(size_t)j * B + b] = h1[j];
  }
  h1aug[(size_t)kH * B + b] = 1.f;
  float z3 = sP[ob3];
  for (int j = 0; j < kH; ++j) {
    float z = sP[ob2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) z = fmaf(sP[oW2 + j * kH + k], h1[k], z);
    z2[(size_t)j * B + b] = z;
    const float h = gelu_f(z);
    h2aug[(size_t)j * B + b] = h;
    z3 = fmaf(sP[ow3 + j], h, z3);
  }
  h2aug[(size_t)kH * B + b] = 1.f;
  y[b] = 1.f / (1.f + expf(-z3));
}

// Backward pass to the pre-activation deltas; accumulates the mean squared error.
__global__ void __launch_bounds__(128) mlp_backward(const float* __restrict__ P,
                                                    const float* __restrict__ target, int B,
                                                    const float* z1, const float* z2,
                                                    const float* y, float* d1, float* d2,
                                                    float* d3, float* loss) {
  extern __shared__ float sW[];  // W2 (kH x kH) then w3 (kH)
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) sW[i] = P[oW2 + i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) sW[kH * kH + i] = P[ow3 + i];
  __shared__ float s_loss[4];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.f;
  if (b < B) {
    const float yv = y[b], t = target[b];
    const float dz3 = (2.f / (float)B) * (yv - t) * yv * (1.f - yv);
    sq = (yv - t) * (yv - t) / (float)B;
    d3[b] = dz3;
    float dv[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      dv[j] = dz3 * sW[kH * kH + j] * gelu_grad_f(z2[(size_t)j * B + b]);
      d2[(size_t)j * B + b] = dv[j];
    }
    for (int k = 0; k < kH; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < kH; ++j) acc = fmaf(sW[j * kH + k], dv[j], acc);
      d1[(size_t)k * B + b] = acc * gelu_grad_f(z1[(size_t)k * B + b]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) s_loss[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_loss[w];
    atomicAdd(loss, s);
  }
}

// C[m][n] = sum_b A[m][b] Bm[n][b]  (A: M x K, Bm: N x K, both row-major over b).
__global__ void __launch_bounds__(256) gemm_nt(const float* __restrict__ A, int M,
                                               const float* __restrict__ Bm, int N, int K,
                                               float* C) {
  __shared__ float sA[32][33], sB[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r, n = n0 + r, k = k0 + tx;
      sA[r][tx] = (m < M && k < K) ? A[(size_t)m * K + k] : 0.f;
      sB[r][tx] = (n < N && k < K) ? Bm[(size_t)n * K + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float bv = sB[tx][kk];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(sA[ty + 8 * i][kk], bv, acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 8 * i, n = n0 + tx;
    if (m < M && n < N) C[(size_t)m * N + n] = acc[i];
  }
}

// Packs the three gradient GEMM outputs into the weight layout.
__global__ void pack_grad(const float* dW1a, const float* dW2a, const float* dw3a, float* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kP) return;
  float v;
  if (i < ob1) v = dW1a[(i / kIn) * (kIn + 1) + i % kIn];
  else if (i < oW2) v = dW1a[(i - ob1) * (kIn + 1) + kIn];
  else if (i < ob2) v = dW2a[((i - oW2) / kH) * (kH + 1) + (i - oW2) % kH];
  else if (i < ow3) v = dW2a[(i - ob2) * (kH + 1) + kH];
  else if (i < ob3) v = dw3a[i - ow3];
  else v = dw3a[kH];
  g[i] = v;
}

__global__ void adam(float* P, const float* g, float* m, float* v, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kP) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

__global__ void to_infer(const float* P, InferW* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned char* w1 = reinterpret_cast<unsigned char*>(w->W1);
  unsigned char* w2 = reinterpret_cast<unsigned char*>(w->W2);
  if (i < kH * kInP) {
    const int j = i / kInP, k = i % kInP;
    *reinterpret_cast<__nv_bfloat16*>(w1 + bf_off(j, k, kInP / 8)) =
        __float2bfloat16_rn(k < kIn ? P[oW1 + j * kIn + k] : 0.f);
  }
  if (i < kH * kH) {
    const int j = i / kH, k = i % kH;
    *reinterpret_cast<__nv_bfloat16*>(w2 + bf_off(j, k, kH / 8)) =
        __float2bfloat16_rn(P[oW2 + j * kH + k]);
  }
  if (i < kH) {
    w->b1[i] = P[ob1 + i];
    w->b2[i] = P[ob2 + i];
    w->w3[i] = P[ow3 + i];
  }
  if (i == 0) w->b3 = P[ob3];
}

// ---------------------------------------------------------------- inference (tensor cores)
// One CTA of 256 threads scores a tile of 128 rows on the 5th-generation tensor
// cores.  Warps w and w + 4 read TMEM lanes 32 (w % 4) .. + 31, so row i of the
// tile (TMEM lane i) has two threads: the first half of the block takes inputs
// 0..7 and accumulator columns 0..63 of each row, the second half inputs 8..15
// and columns 64..127.
//   1. each thread writes its 8 inputs (bfloat16; 12 inputs padded to 16) into row
//      i of the K-major tile A1;
//   2. one thread issues tcgen05.mma kind::f16 (M = N = 128, K = 16): A1 W1^T into
//      128 TMEM columns, and commits to an mbarrier;
//   3. each thread reads its 64 columns of row i back (tcgen05.ld), adds b1,
//      applies GELU and writes them into row i of the bfloat16 tile A2 (K = 128);
//   4. one thread issues eight K = 16 MMAs, A2 W2^T, into the same columns;
//   5. each thread reads its 64 columns, adds b2, applies GELU and takes the dot
//      product with its half of w3; the two halves are added in order, then b3
//      and the sigmoid.
// The weights' rounding to bfloat16 and the float32 accumulation are those of
// the network's inference form; GELU uses the hardware tanh approximation.
constexpr int kTileRows = 128;
constexpr int kScoreThreads = 2 * kTileRows;
constexpr uint32_t kOffA1 = 38912;                 // after the staged InferW (38,416 B)
constexpr uint32_t kOffA2 = kOffA1 + kTileRows * kInP * 2;
constexpr int kScoreSmem = (int)(kOffA2 + kTileRows * kH * 2);  // 75,776 B
static_assert(sizeof(InferW) <= kOffA1 && kOffA1 % 1024 == 0 && kOffA2 % 1024 == 0,
              "shared-memory layout of a scoring block");
constexpr int kTmemCols = 128;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float gelu_fast(float z) {
  return 0.5f * z * (1.f + tanh_approx(kGeluC * (z + kGeluA * z * z * z)));
}

// Instruction descriptor, kind::f16: D float32, A and B bfloat16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24 (M = N = 128).
constexpr uint32_t kIdescBf16 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(kIdescBf16), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Generic-proxy writes to shared memory become visible to the tensor cores, and
// every thread's earlier tcgen05 reads are ordered before the next MMA.
__device__ __forceinline__ void tc_handoff() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Waits for the MMAs committed to `bar` (phase `phase`), bounded; the CTA agrees.
__device__ __forceinline__ bool mma_wait(uint64_t* bar, uint32_t phase) {
  bool ok = bar_wait(bar, phase);
  if (!ok) ok = bar_wait(bar, phase);
  const bool all = __syncthreads_and(ok) != 0;
  tc_fence_after();
  return all;
}

// Per scoring block: TMEM for the accumulator and the mbarrier of the MMAs.
struct ScoreCtx {
  unsigned char* smem;  // staged InferW | A1 | A2
  uint32_t tmem;
  uint64_t* bar;
  uint32_t phase;
  bool ok;
};

// Row of the tile (TMEM lane) and half of the row's columns this thread takes.
__device__ __forceinline__ int score_row() {
  return (int)(((threadIdx.x >> 5) & 3) * 32 + (threadIdx.x & 31));
}
__device__ __forceinline__ int score_half() { return (int)(threadIdx.x >> 7); }

// The weights pass through registers on their way to shared memory: a thread
// issues its loads (weights_load), the block does other work while they are in
// flight, then stores them (weights_store; the first MMA hand-off makes them
// visible).  Plain loads: every block reads the same 38 KB, which the L2 serves
// to plain loads faster than to one bulk copy per block (measured: 1.3 TB/s
// with 304 blocks copying at once).
constexpr int kW16 = (int)(sizeof(InferW) / 16);
constexpr int kWPerThread = (kW16 + kScoreThreads - 1) / kScoreThreads;
struct WeightRegs {
  uint4 v[kWPerThread];
};
__device__ __forceinline__ void weights_load(const InferW* w, WeightRegs& r) {
  const uint4* src = reinterpret_cast<const uint4*>(w);
#pragma unroll
  for (int j = 0; j < kWPerThread; ++j) {
    const int i = (int)threadIdx.x + j * kScoreThreads;
    if (i < kW16) r.v[j] = __ldg(&src[i]);
  }
}
__device__ __forceinline__ void weights_store(const WeightRegs& r, unsigned char* smem) {
  uint4* dst = reinterpret_cast<uint4*>(smem);
#pragma unroll
  for (int j = 0; j < kWPerThread; ++j) {
    const int i = (int)threadIdx.x + j * kScoreThreads;
    if (i < kW16) dst[i] = r.v[j];
  }
}

// Allocates the accumulator and initialises the MMA barrier (all threads; ends
// synced).  The weights go into shared memory separately (weights_load/store).
__device__ void score_begin(unsigned char* smem, uint64_t* bar, uint32_t* s_tmem, ScoreCtx* c) {
  if (threadIdx.x == 0) bar_init(bar);
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)), "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c->smem = smem;
  c->tmem = *s_tmem;
  c->bar = bar;
  c->phase = 0;
  c->ok = true;
}

// Frees the accumulator (all threads, after the last tile).
__device__ void score_end(const ScoreCtx& c) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem),
                 "n"(kTmemCols)
                 : "memory");
}

// The network's output for this thread's row of the tile; f8 holds the row's
// inputs 8 h .. 8 h + 7 (h = score_half(); inputs 12..15 are zero).  Called by
// all 256 threads of the block; both threads of a row get the output.  After a
// wait that runs out the block stops using the tensor cores (c->ok = false) and
// every row scores 1.
__device__ float score_tile(ScoreCtx* c, const float* f8) {
  __shared__ float s_part[2][kTileRows];
  if (!c->ok) return 1.f;
  const int warp = (int)(threadIdx.x >> 5), row = score_row(), h = score_half();
  unsigned char* a1 = c->smem + kOffA1;
  unsigned char* a2 = c->smem + kOffA2;
  const InferW* sw = reinterpret_cast<const InferW*>(c->smem);
  *reinterpret_cast<uint4*>(a1 + bf_off(row, 8 * h, kInP / 8)) =
      make_uint4(pack_bf16(f8[0], f8[1]), pack_bf16(f8[2], f8[3]), pack_bf16(f8[4], f8[5]),
                 pack_bf16(f8[6], f8[7]));
  tc_handoff();
  const uint32_t sa1 = smem_u32(a1), sa2 = smem_u32(a2);
  const uint32_t sw1 = smem_u32(sw->W1), sw2 = smem_u32(sw->W2);
  if (threadIdx.x == 0) {
    mma_bf16(c->tmem, mat_desc(sa1, 128, 256), mat_desc(sw1, 128, 256), 0u);
    mma_commit(c->bar);
  }
  c->ok = mma_wait(c->bar, c->phase);
  c->phase ^= 1u;
  if (!c->ok) return 1.f;
  const int col0 = 64 * h;
  const uint32_t taddr = c->tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)col0;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float v[32];
    tmem_ld32(taddr + 32 * q, v);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int j = col0 + 32 * q + 8 * m;
      float g[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) g[e] = gelu_fast(v[8 * m + e] + sw->b1[j + e]);
      *reinterpret_cast<uint4*>(a2 + bf_off(row, j, kH / 8)) =
          make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                     pack_bf16(g[6], g[7]));
    }
  }
  tc_handoff();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int kb = 0; kb < kH / 16; ++kb)
      mma_bf16(c->tmem, mat_desc(sa2 + kb * 256, 128, 2048), mat_desc(sw2 + kb * 256, 128, 2048),
               kb ? 1u : 0u);
    mma_commit(c->bar);
  }
  c->ok = mma_wait(c->bar, c->phase);
  c->phase ^= 1u;
  if (!c->ok) return 1.f;
  float p = 0.f;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float v[32];
    tmem_ld32(taddr + 32 * q, v);
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int j = col0 + 32 * q + e;
      p = fmaf(sw->w3[j], gelu_fast(v[e] + sw->b2[j]), p);
    }
  }
  s_part[h][row] = p;
  __syncthreads();
  const float y = 1.f / (1.f + __expf(-((s_part[0][row] + s_part[1][row]) + sw->b3)));
  __syncthreads();  // s_part is rewritten by the next tile
  return y;
}

// Scores arbitrary feature rows (batch x 12), 128 rows per block and tile.
__global__ void __launch_bounds__(kScoreThreads) score_rows(const InferW* w, const float* feats,
                                                            int B, float* out) {
  extern __shared__ __align__(1024) unsigned char s_score[];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  ScoreCtx c;
  WeightRegs wr;
  weights_load(w, wr);
  score_begin(s_score, &s_bar, &s_tmem, &c);
  weights_store(wr, s_score);
  const int row = score_row(), h = score_half();
  const int tiles = (B + kTileRows - 1) / kTileRows;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int r = t * kTileRows + row;
    float f8[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = 8 * h + e;
      f8[e] = (r < B && k < kIn) ? feats[(size_t)r * kIn + k] : 0.f;
    }
    const float y = score_tile(&c, f8);
    if (h == 0 && r < B) out[r] = c.ok ? y : __int_as_float(0x7fc00000);  // NaN: the wait ran out
  }
  score_end(c);
}

// ---------------------------------------------------------------- track features
struct FeatureSrc {
  DevTrack track;
  const float* look;  // per segment start vertex: curvature 5, 10, 20, 40 m ahead
  float half_width;
};

// The 10 per-tick inputs (plus the nearest segment and its distance) for the
// state x_t, computed by the whole block; result in s_feat[0..12).
__device__ void block_tick_features(const FeatureSrc& fs, const double* x_t, float* s_feat) {
  __shared__ float s_d[32];
  __shared__ int s_i[32];
  __shared__ float4 s_win[2];  // the nearest segment and its look-ahead curvatures
  __shared__ float s_winv;     // and its 1 / |d|^2
  const char* base = reinterpret_cast<const char*>(fs.track.blob);
  const float4* seg = reinterpret_cast<const float4*>(base + fs.track.off_seg);
  const float* inv = reinterpret_cast<const float*>(base + fs.track.off_inv);
  const float4* look4 = reinterpret_cast<const float4*>(fs.look);
  const int S = (fs.track.off_inv - fs.track.off_seg) / 16;
  // every load the features need is issued before any of them is used: the
  // state, and for each of this thread's segments its geometry and its row of
  // the look-ahead table (the winner keeps them, so no load follows the search)
  const double x0 = x_t[0], x1 = x_t[1], x2 = x_t[2], x3 = x_t[3], x4 = x_t[4], x5 = x_t[5];
  const float px = (float)x0, py = (float)x1;
  float best = INFINITY;
  int bi = 0x7fffffff;
  float4 bseg = make_float4(0.f, 0.f, 0.f, 0.f), blook = bseg;
  float binv = 0.f;
  // two segments per round, both loaded before either is used
  for (int i0 = threadIdx.x; i0 < S; i0 += 2 * blockDim.x) {
    float4 sg[2], lk[2];
    float iv[2];
    int idx[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      idx[e] = i0 + e * (int)blockDim.x;
      const int j = idx[e] < S ? idx[e] : i0;
      sg[e] = seg[j];
      iv[e] = inv[j];
      lk[e] = look4[j];
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (idx[e] >= S) continue;
      const float rx = px - sg[e].x, ry = py - sg[e].y;
      const float t = fminf(fmaxf((rx * sg[e].z + ry * sg[e].w) * iv[e], 0.f), 1.f);
      const float ex = rx - t * sg[e].z, ey = ry - t * sg[e].w;
      const float d2 = ex * ex + ey * ey;
      if (d2 < best || (d2 == best && idx[e] < bi)) {
        best = d2;
        bi = idx[e];
        bseg = sg[e];
        blook = lk[e];
        binv = iv[e];
      }
    }
  }
  const int own = bi;  // this thread's candidate
  float gbest = best;
  int gbi = bi;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, gbest, o);
    const int oi = __shfl_xor_sync(0xffffffffu, gbi, o);
    if (ob < gbest || (ob == gbest && oi < gbi)) {
      gbest = ob;
      gbi = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_d[warp] = gbest;
    s_i[warp] = gbi;
  }
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
    if (s_d[w] < gbest || (s_d[w] == gbest && s_i[w] < gbi)) {
      gbest = s_d[w];
      gbi = s_i[w];
    }
  if (own == gbi) {  // exactly one thread holds the nearest segment
    s_win[0] = bseg;
    s_win[1] = blook;
    s_winv = binv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float4 sg = s_win[0];
    const float4 lk = s_win[1];
    const float rx = px - sg.x, ry = py - sg.y;
    const float t = fminf(fmaxf((rx * sg.z + ry * sg.w) * s_winv, 0.f), 1.f);
    const float len = sqrtf(sg.z * sg.z + sg.w * sg.w);
    const float tx = sg.z / len, ty = sg.w / len;
    const float ex = rx - t * sg.z, ey = ry - t * sg.w;
    const float e_y = (ex * (-ty) + ey * tx) / fs.half_width;
    float se, ce;
    sincosf((float)x2 - atan2f(ty, tx), &se, &ce);
    s_feat[0] = e_y;
    s_feat[1] = se;
    s_feat[2] = ce;
    s_feat[3] = (float)x3 / 25.f;
    s_feat[4] = (float)x4 / 5.f;
    s_feat[5] = (float)x5 / 2.f;
    s_feat[6] = 10.f * lk.x;
    s_feat[7] = 10.f * lk.y;
    s_feat[8] = 10.f * lk.z;
    s_feat[9] = 10.f * lk.w;
    s_feat[10] = (float)gbi;
    s_feat[11] = sqrtf(gbest);
  }
  __syncthreads();
}

__global__ void tick_features(FeatureSrc fs, const double* x_t, float* out) {
  __shared__ float s_feat[12];
  block_tick_features(fs, x_t, s_feat);
  if (threadIdx.x < 12) out[threadIdx.x] = s_feat[threadIdx.x];
}

// The 12 inputs of every slot of a tick (training data, parity).
__global__ void slot_features(TickArgs a, FeatureSrc fs, float* out) {
  __shared__ float s_feat[12];
  block_tick_features(fs, a.x_t, s_feat);
  float uh[2] = {__double2float_rn(a.u_h[0]), __double2float_rn(a.u_h[1])};
  for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < a.n_slots;
       slot += gridDim.x * blockDim.x) {
    float xi[2];
    candidate_value<2>(a, slot, uh, xi);
#pragma unroll
    for (int k = 0; k < 10; ++k) out[(size_t)slot * kIn + k] = s_feat[k];
    out[(size_t)slot * kIn + 10] = xi[0] / 0.4f;
    out[(size_t)slot * kIn + 11] = xi[1];
  }
}

// ---------------------------------------------------------------- screened tick
// Which slots a screened tick rolls out: a prefix of the cost order, cut between
// two cost bins (bin = float32 bits of the cost >> kBinShift: the exponent and
// the top three mantissa bits, monotone in the cost), so that every slot left
// out costs strictly more than every slot kept.  The prefix is the shortest one
// that holds at least k slots and -- with the network (tau > 0) -- at least m
// slots the network predicts safe (score >= tau).  Whatever the scores, the kept
// slots either contain the least-cost safe candidate of the whole tick or are all
// unsafe (then the full evaluation runs): the selection is always the exhaustive
// one.  The network only decides how far down the cost order to go.

// One histogram: the first bin at which the inclusive count reaches `target`, or
// kBins - 1 if it never does (whole block; s_hist in shared memory).
__device__ int first_bin_reaching(const unsigned int* s_hist, unsigned int target,
                                  unsigned int* s_run, int* s_bin) {
  constexpr int kRun = kBins / 128;
  unsigned int run = 0;
  if (threadIdx.x < 128)
    for (int i = 0; i < kRun; ++i) run += s_hist[threadIdx.x * kRun + i];
  if (threadIdx.x < 128) s_run[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive prefix of the run sums: 4 runs per lane, then a warp scan
    unsigned int v[4], tot = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      v[j] = s_run[threadIdx.x * 4 + j];
      tot += v[j];
    }
    unsigned int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int n = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)threadIdx.x >= o) incl += n;
    }
    unsigned int before = incl - tot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      s_run[threadIdx.x * 4 + j] = before;  // exclusive prefix of run j
      before += v[j];
    }
  }
  if (threadIdx.x == 0) *s_bin = kBins - 1;  // never reached: keep everything
  __syncthreads();
  if (threadIdx.x < 128) {
    unsigned int cum = s_run[threadIdx.x];
    if (cum < target) {
      for (int i = 0; i < kRun; ++i) {
        cum += s_hist[threadIdx.x * kRun + i];
        if (cum >= target) {
          *s_bin = threadIdx.x * kRun + i;  // the only run that crosses the target
          break;
        }
      }
    }
  }
  __syncthreads();
  const int b = *s_bin;
  __syncthreads();
  return b;
}

// End of a scoring launch (every thread of the block): this block's histograms
// into the tick's; the last block finds the threshold bin (the larger of the bin
// reaching k slots and, with s_safe, the bin reaching m predicted-safe slots),
// then clears the histograms and the list counter for the next tick.  s_all may
// be null when k <= m: a prefix holding m predicted-safe slots holds at least k
// slots, so the predicted-safe bin alone is the threshold.
__device__ void screen_finish(unsigned int* s_all, unsigned int* s_safe, int k, int m,
                              ScreenScratch* ss) {
  __shared__ int s_last, s_bin;
  __shared__ unsigned int s_run[128];
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) {
    if (s_all && s_all[i]) atomicAdd(&ss->hist[i], s_all[i]);
    if (s_safe && s_safe[i]) atomicAdd(&ss->hist_safe[i], s_safe[i]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&ss->done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) {
    if (s_all) s_all[i] = *reinterpret_cast<volatile unsigned int*>(&ss->hist[i]);
    if (s_safe) s_safe[i] = *reinterpret_cast<volatile unsigned int*>(&ss->hist_safe[i]);
  }
  __syncthreads();
  int b = 0;
  if (s_all) b = first_bin_reaching(s_all, (unsigned int)k, s_run, &s_bin);
  if (s_safe) {
    const int bs = first_bin_reaching(s_safe, (unsigned int)m, s_run, &s_bin);
    b = bs > b ? bs : b;
  }
  if (threadIdx.x == 0) {
    ss->bstar = b;
    ss->n_list = 0;
    ss->done = 0;
  }
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) {
    ss->hist[i] = 0;
    ss->hist_safe[i] = 0;
  }
}

// Cost of a candidate against the user's input: the same float32 operations as
// the rollout's cost (so a kept slot's bin follows its selection cost).
__device__ __forceinline__ float screen_cost_of(const float* x, const float* uh) {
  const float d0 = __fsub_rn(x[0], uh[0]), d1 = __fsub_rn(x[1], uh[1]);
  return __fmaf_rn(d1, d1, __fmul_rn(d0, d0));
}

// Scores every slot with the network (tau > 0), 128 slots per block and tile,
// writes its key (the cost's float32 bits) and builds the histograms of all slots
// and of the predicted-safe slots over the cost bins (screen_finish).
__global__ void __launch_bounds__(kScoreThreads) screen_score(TickArgs a, FeatureSrc fs,
                                                          const InferW* w, float tau, int k,
                                                          int m, unsigned int* keys,
                                                          ScreenScratch* ss) {
  extern __shared__ __align__(1024) unsigned char s_score[];
  __shared__ unsigned int s_hist[kBins];
  __shared__ unsigned int s_hsafe[kBins];
  __shared__ float s_feat[12];
  __shared__ uint64_t s_bar;
  __shared__ uint32_t s_tmem;
  grid_dep_release();  // the compaction may launch now; it waits for this kernel
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) {
    s_hist[i] = 0;
    s_hsafe[i] = 0;
  }
  ScoreCtx c;
  WeightRegs wr;
  weights_load(w, wr);  // in flight while the accumulator and the features are prepared
  score_begin(s_score, &s_bar, &s_tmem, &c);
  block_tick_features(fs, a.x_t, s_feat);  // ends with __syncthreads
  weights_store(wr, s_score);
  float uh[2] = {__double2float_rn(a.u_h[0]), __double2float_rn(a.u_h[1])};
  // the first half of the block feeds the per-tick inputs 0..7; the second half
  // inputs 8..11 (two per-tick, the candidate's two) and writes the keys
  const int row = score_row(), h = score_half();
  const int tiles = (a.n_slots + kTileRows - 1) / kTileRows;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int r = t * kTileRows + row;
    const bool live = r < a.n_slots;
    float f8[8], x[2] = {0.f, 0.f};
    if (h == 0) {
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) f8[mm] = s_feat[mm];
    } else {
      candidate_value<2>(a, live ? r : 0, uh, x);
      f8[0] = s_feat[8];
      f8[1] = s_feat[9];
      f8[2] = x[0] / 0.4f;
      f8[3] = x[1];
#pragma unroll
      for (int mm = 4; mm < 8; ++mm) f8[mm] = 0.f;
    }
    const float y = score_tile(&c, f8);
    if (h == 1) {  // whole warps
      unsigned int key = 0u;
      if (live) {
        key = __float_as_uint(screen_cost_of(x, uh));
        keys[r] = key;
      }
      // one shared-memory atomic per distinct bin of the warp (neighbouring slots'
      // costs share few bins), for all slots (only when k > m) and for the
      // predicted-safe ones
      const unsigned int bin = live ? key >> kBinShift : 0xFFFFFFFFu;
      if (k > m) {
        const unsigned int same = __match_any_sync(kFull, bin);
        if (live && (threadIdx.x & 31) == (unsigned int)(__ffs(same) - 1))
          atomicAdd(&s_hist[bin], (unsigned int)__popc(same));
      }
      const bool safe = live && y >= tau;
      const unsigned int sbin = safe ? bin : 0xFFFFFFFFu;
      const unsigned int ssame = __match_any_sync(kFull, sbin);
      if (safe && (threadIdx.x & 31) == (unsigned int)(__ffs(ssame) - 1))
        atomicAdd(&s_hsafe[bin], (unsigned int)__popc(ssame));
    }
  }
  score_end(c);
  screen_finish(k > m ? s_hist : nullptr, s_hsafe, k, m, ss);
}

// Cost order alone (tau <= 0; no network): warps take 16-slot tiles, lanes
// l and l + 4 k of a group compute the same two slots and one lane per slot
// writes its key (a small kernel keeps the instruction footprint of this path low).
__global__ void __launch_bounds__(128) screen_cost(TickArgs a, int k, unsigned int* keys,
                                                  ScreenScratch* ss) {
  __shared__ unsigned int s_hist[kBins];
  grid_dep_release();  // the compaction may launch now; it waits for this kernel
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
  float uh[2] = {__double2float_rn(a.u_h[0]), __double2float_rn(a.u_h[1])};
  const int tiles = (a.n_slots + 15) / 16;
  for (int t = blockIdx.x * wpb + warp; t < tiles; t += gridDim.x * wpb) {
    if (q != 0) continue;
    const int rr[2] = {16 * t + g, 16 * t + g + 8};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int r = rr[e];
      if (r >= a.n_slots) continue;
      float x[2];
      candidate_value<2>(a, r, uh, x);
      const unsigned int key = __float_as_uint(screen_cost_of(x, uh));
      keys[r] = key;
      atomicAdd(&s_hist[key >> kBinShift], 1u);
    }
  }
  screen_finish(s_hist, nullptr, k, 0, ss);
}

// Keeps the slots whose cost bin is at or below the threshold (warp-aggregated append).
__global__ void screen_compact(const unsigned int* keys, int n_slots, ScreenScratch* ss,
                               int* list) {
  grid_dep_wait();     // the screen's keys and threshold
  grid_dep_release();  // the rollout of the kept slots may launch now
  const int bstar = ss->bstar;
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_slots;
       base += gridDim.x * blockDim.x) {
    const int slot = base + lane;
    const bool keep = slot < n_slots && (int)(keys[slot] >> kBinShift) <= bstar;
    const unsigned int m = __ballot_sync(0xffffffffu, keep);
    int at = 0;
    if (lane == 0 && m) at = atomicAdd(&ss->n_list, __popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (keep) list[at + __popc(m & ((1u << lane) - 1))] = slot;
  }
}

}  // namespace mpmi

// ---------------------------------------------------------------- host side
struct mpmi_screener {
  mpmi_ctx* ctx = nullptr;
  const mpmi_model* model = nullptr;
  float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
  int step = 0;
  mpmi::InferW* infer = nullptr;
  bool stale = true;
  float* look = nullptr;
  float half_width = 0.f;
  int max_batch = 0, max_slots = 0;
  float* act = nullptr;      // training activations
  float* gemm_out = nullptr; // gradient GEMM outputs
  unsigned int* keys = nullptr;
  int* list = nullptr;
  mpmi::ScreenScratch* ss = nullptr;
  uint64_t bytes = 0;
  // optional phase timing of screened ticks: events around the screen, the
  // compaction, the kept rollout and the fallback launch
  bool timing = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace mpmi {

static int cfail(cudaError_t e, const char* what) {
  return fail(MPMI_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define SCR_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cfail(e_, what); \
  } while (0)

static FeatureSrc feature_src(const mpmi_screener* s) {
  FeatureSrc fs;
  fs.track = s->model->dev_safety.track;
  fs.look = s->look;
  fs.half_width = s->half_width;
  return fs;
}

// Curvature ahead (float64 on the host): signed Menger curvature of every vertex
// and, per vertex, the curvature at the first vertex 5, 10, 20, 40 m of arc ahead.
static std::vector<float> lookahead(const std::vector<double>& xy) {
  const int S = (int)xy.size() / 2;
  std::vector<double> kappa(S), seg(S);
  for (int i = 0; i < S; ++i) {
    const int p = (i + S - 1) % S, n = (i + 1) % S;
    const double ax = xy[2 * i] - xy[2 * p], ay = xy[2 * i + 1] - xy[2 * p + 1];
    const double bx = xy[2 * n] - xy[2 * i], by = xy[2 * n + 1] - xy[2 * i + 1];
    const double cx = xy[2 * n] - xy[2 * p], cy = xy[2 * n + 1] - xy[2 * p + 1];
    const double cross = ax * by - ay * bx;
    kappa[i] = 2.0 * cross / (sqrt(ax * ax + ay * ay) * sqrt(bx * bx + by * by) *
                              sqrt(cx * cx + cy * cy));
    seg[i] = sqrt(bx * bx + by * by);
  }
  const double ahead[4] = {5.0, 10.0, 20.0, 40.0};
  std::vector<float> out(4 * (size_t)S);
  for (int i = 0; i < S; ++i)
    for (int m = 0; m < 4; ++m) {
      double acc = 0.0;
      int j = i;
      do {
        acc += seg[j % S];
        ++j;
      } while (acc < ahead[m]);
      out[4 * (size_t)i + m] = (float)kappa[j % S];
    }
  return out;
}

static int refresh_infer(mpmi_screener* s, cudaStream_t st) {
  if (!s->stale) return MPMI_OK;
  to_infer<<<(kH * kH + 255) / 256, 256, 0, st>>>(s->params, s->infer);
  SCR_CUDA(cudaGetLastError(), "to_infer launch");
  s->stale = false;
  return MPMI_OK;
}

static int gradients(mpmi_screener* s, const float* feats, const float* target, int B,
                     float* grad, float* loss, cudaStream_t st) {
  float* A = s->act;
  const size_t Bz = (size_t)B;
  float* faug = A;
  float* z1 = faug + (kIn + 1) * Bz;
  float* h1aug = z1 + kH * Bz;
  float* z2 = h1aug + (kH + 1) * Bz;
  float* h2aug = z2 + kH * Bz;
  float* y = h2aug + (kH + 1) * Bz;
  float* d1 = y + Bz;
  float* d2 = d1 + kH * Bz;
  float* d3 = d2 + kH * Bz;
  float* dW2a = s->gemm_out;
  float* dW1a = dW2a + kH * (kH + 1);
  float* dw3a = dW1a + kH * (kIn + 1);
  const int fwd_smem = kP * sizeof(float), bwd_smem = (kH * kH + kH) * sizeof(float);
  SCR_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st), "clear loss");
  mlp_forward<<<(B + 127) / 128, 128, fwd_smem, st>>>(s->params, feats, B, faug, z1, h1aug, z2,
                                                      h2aug, y);
  mlp_backward<<<(B + 127) / 128, 128, bwd_smem, st>>>(s->params, target, B, z1, z2, y, d1, d2,
                                                       d3, loss);
  gemm_nt<<<dim3((kH + 1 + 31) / 32, kH / 32), 256, 0, st>>>(d2, kH, h1aug, kH + 1, B, dW2a);
  gemm_nt<<<dim3((kIn + 1 + 31) / 32, kH / 32), 256, 0, st>>>(d1, kH, faug, kIn + 1, B, dW1a);
  gemm_nt<<<dim3((kH + 1 + 31) / 32, 1), 256, 0, st>>>(d3, 1, h2aug, kH + 1, B, dw3a);
  pack_grad<<<(kP + 255) / 256, 256, 0, st>>>(dW1a, dW2a, dw3a, grad);
  SCR_CUDA(cudaGetLastError(), "screener gradient launches");
  return MPMI_OK;
}

}  // namespace mpmi

using namespace mpmi;

namespace mpmi {

static int screened_checks(const mpmi_session* session, const mpmi_screener* s, int32_t k,
                           float tau, int32_t m) {
  if (session->model != s->model) return fail(MPMI_E_INVALID_ARG, "screener: another model");
  if (session->cfg.sampler == MPMI_SAMPLER_EXTERNAL)
    return fail(MPMI_E_UNSUPPORTED, "evaluate_screened: sampled candidates only");
  if (session->n_slots > s->max_slots)
    return fail(MPMI_E_INVALID_ARG, "evaluate_screened: session has more slots than max_slots");
  if (k < 1) return fail(MPMI_E_INVALID_ARG, "evaluate_screened: k must be >= 1");
  if (tau > 0.f && m < 1)
    return fail(MPMI_E_INVALID_ARG, "evaluate_screened: m must be >= 1 with the network");
  return MPMI_OK;
}

// The screened tick's launches on stream st for the tick described by a (its
// x_t, u_h and result pointers set; with a.seq_out the launch whose result is
// final also stores a.seq there).
static int screened_chain(mpmi_session* session, mpmi_screener* s, const TickArgs& a, int32_t k,
                          float tau, int32_t m, int32_t* list_dev, int32_t* n_list_dev,
                          cudaStream_t st) {
  int rc = refresh_infer(s, st);
  if (rc != MPMI_OK) return rc;
  TickArgs sa = a;
  sa.seq_out = nullptr;  // the screen writes no result
  if (s->timing) SCR_CUDA(cudaEventRecord(s->ev[0], st), "cudaEventRecord");
  // at most two blocks per SM: with the network each holds 128 TMEM columns and
  // the staged weights; more blocks would only repeat the per-tick features
  if (tau > 0.f) {
    const int tiles = (session->n_slots + kTileRows - 1) / kTileRows;
    const int blocks = tiles < 2 * s->ctx->sm_count ? tiles : 2 * s->ctx->sm_count;
    screen_score<<<blocks, kScoreThreads, kScoreSmem, st>>>(sa, feature_src(s), s->infer, tau,
                                                            k, m, s->keys, s->ss);
  } else {
    const int tiles = (session->n_slots + 15) / 16;
    int blocks = (tiles + 3) / 4;
    if (blocks > 2 * s->ctx->sm_count) blocks = 2 * s->ctx->sm_count;
    screen_cost<<<blocks, 128, 0, st>>>(sa, k, s->keys, s->ss);
  }
  if (s->timing) SCR_CUDA(cudaEventRecord(s->ev[1], st), "cudaEventRecord");
  int cb = (session->n_slots + 255) / 256;
  if (cb > 4 * s->ctx->sm_count) cb = 4 * s->ctx->sm_count;
  {
    // the compaction, the rollout and the fallback run as programmatic
    // dependents: each may launch while its predecessor runs and waits for it
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cb);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SCR_CUDA(cudaLaunchKernelEx(&cfg, screen_compact, (const unsigned int*)s->keys,
                                (int)session->n_slots, s->ss, s->list),
             "screen_compact launch");
  }
  SCR_CUDA(cudaGetLastError(), "screen launches");
  if (s->timing) SCR_CUDA(cudaEventRecord(s->ev[2], st), "cudaEventRecord");
  // exact rollout on the kept slots (their number is known only on the device)
  TickArgs r = a;
  r.slot_list = s->list;
  r.n_list = &s->ss->n_list;
  r.result_flags = 1;
  r.chained = 1;
  r.seq_if_final = 1;
  // with the network the kept slots are mostly predicted safe and run the whole
  // horizon, so sixteen lanes per race-car candidate shorten the chain; in cost
  // order most kept slots leave early and eight lanes keep fewer warps
  rc = launch_tick_args(session, r, false, st, -1, tau > 0.f ? 16 : 0);
  if (rc != MPMI_OK) return rc;
  if (s->timing) SCR_CUDA(cudaEventRecord(s->ev[3], st), "cudaEventRecord");
  if (list_dev)
    SCR_CUDA(cudaMemcpyAsync(list_dev, s->list, sizeof(int) * session->n_slots,
                             cudaMemcpyDeviceToDevice, st), "copy list");
  if (n_list_dev)
    SCR_CUDA(cudaMemcpyAsync(n_list_dev, &s->ss->n_list, sizeof(int), cudaMemcpyDeviceToDevice,
                             st), "copy list size");
  // full evaluation only when the kept slots hold no safe candidate and were not
  // already every slot; its result counts the steps of both launches
  TickArgs f = a;
  f.skip_if_safe = a.result;
  f.result_flags = 3;
  f.chained = 1;
  rc = launch_tick_args(session, f, false, st, 0);
  if (rc == MPMI_OK && s->timing) SCR_CUDA(cudaEventRecord(s->ev[4], st), "cudaEventRecord");
  return rc;
}

}  // namespace mpmi

extern "C" {

int mpmi_screener_create(mpmi_ctx* ctx, const mpmi_model* model, const float* weights,
                         int32_t max_batch, int32_t max_slots, mpmi_screener** out) {
  if (!ctx || !model || !weights || !out) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  *out = nullptr;
  if (model->kind != kCar || !model->has_safety || !model->dev_safety.has_track)
    return fail(MPMI_E_UNSUPPORTED, "screener: needs a race-car model with a track");
  if (max_batch < 1 || max_slots < 1 || max_slots > MPMI_MAX_SLOTS)
    return fail(MPMI_E_INVALID_ARG, "screener: max_batch and max_slots must be positive");
  for (int i = 0; i < kP; ++i)
    if (!isfinite(weights[i])) return fail(MPMI_E_NONFINITE, "screener: non-finite weight");
  mpmi_screener* s = new mpmi_screener();
  s->ctx = ctx;
  s->model = model;
  s->max_batch = max_batch;
  s->max_slots = max_slots;
  s->half_width = (float)(model->spec.track_half_width - model->spec.inflation);
  std::vector<float> look = lookahead(model->track_host);
  const size_t act_floats = (size_t)max_batch * (2 * (kIn + 1) + 4 * kH + 2 * (kH + 1) + 2);
  const size_t gemm_floats = kH * (kH + 1) + kH * (kIn + 1) + (kH + 1);
  const uint64_t bytes = 4 * kP * sizeof(float) + sizeof(InferW) + look.size() * sizeof(float) +
                         act_floats * sizeof(float) + gemm_floats * sizeof(float) +
                         (size_t)max_slots * (sizeof(unsigned int) + sizeof(int)) +
                         sizeof(ScreenScratch);
  if (ctx->budget && ctx->used + bytes > ctx->budget) {
    delete s;
    return fail(MPMI_E_OOM, "screener exceeds the memory budget");
  }
  bool ok = cudaMalloc(&s->params, kP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->adam_m, kP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->adam_v, kP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->grad, kP * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->infer, sizeof(InferW)) == cudaSuccess &&
            cudaMalloc(&s->look, look.size() * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->act, act_floats * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->gemm_out, gemm_floats * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->keys, (size_t)max_slots * sizeof(unsigned int)) == cudaSuccess &&
            cudaMalloc(&s->list, (size_t)max_slots * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&s->ss, sizeof(ScreenScratch)) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(s->params, weights, kP * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(s->adam_m, 0, kP * sizeof(float)) == cudaSuccess &&
         cudaMemset(s->adam_v, 0, kP * sizeof(float)) == cudaSuccess &&
         cudaMemcpy(s->look, look.data(), look.size() * sizeof(float), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemset(s->ss, 0, sizeof(ScreenScratch)) == cudaSuccess;
  if (ok) {
    const int fwd = kP * sizeof(float), bwd = (kH * kH + kH) * sizeof(float);
    const int inf = kScoreSmem;
    ok = cudaFuncSetAttribute(mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, fwd) ==
             cudaSuccess &&
         cudaFuncSetAttribute(mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, bwd) ==
             cudaSuccess &&
         cudaFuncSetAttribute(score_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, inf) ==
             cudaSuccess &&
         cudaFuncSetAttribute(screen_score, cudaFuncAttributeMaxDynamicSharedMemorySize, inf) ==
             cudaSuccess;
  }
  if (!ok) {
    mpmi_screener_free(s);
    return fail(MPMI_E_OOM, "screener: device allocation failed");
  }
  s->bytes = bytes;
  ctx->used += bytes;
  *out = s;
  return MPMI_OK;
}

void mpmi_screener_free(mpmi_screener* s) {
  if (!s) return;
  cudaFree(s->params);
  cudaFree(s->adam_m);
  cudaFree(s->adam_v);
  cudaFree(s->grad);
  cudaFree(s->infer);
  cudaFree(s->look);
  cudaFree(s->act);
  cudaFree(s->gemm_out);
  cudaFree(s->keys);
  cudaFree(s->list);
  cudaFree(s->ss);
  for (cudaEvent_t& e : s->ev)
    if (e) cudaEventDestroy(e);
  if (s->ctx) s->ctx->used -= s->bytes;
  delete s;
}

int mpmi_screener_set_timing(mpmi_screener* s, int32_t on) {
  if (!s) return fail(MPMI_E_INVALID_ARG, "screener_set_timing: NULL screener");
  if (on && !s->ev[0])  // on the current device, like the screener's launches
    for (cudaEvent_t& e : s->ev) SCR_CUDA(cudaEventCreate(&e), "cudaEventCreate");
  s->timing = on != 0;
  return MPMI_OK;
}

int mpmi_screener_phase_times(mpmi_screener* s, float* ms_out) {
  if (!s || !ms_out) return fail(MPMI_E_INVALID_ARG, "screener_phase_times: NULL argument");
  if (!s->ev[0]) return fail(MPMI_E_NOT_READY, "screener_phase_times: timing is off");
  for (int i = 0; i < 4; ++i) {
    SCR_CUDA(cudaEventSynchronize(s->ev[i + 1]), "cudaEventSynchronize");
    SCR_CUDA(cudaEventElapsedTime(&ms_out[i], s->ev[i], s->ev[i + 1]), "cudaEventElapsedTime");
  }
  return MPMI_OK;
}

int mpmi_screener_get_weights(const mpmi_screener* s, float* out) {
  if (!s || !out) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  SCR_CUDA(cudaMemcpy(out, s->params, kP * sizeof(float), cudaMemcpyDeviceToHost), "read weights");
  return MPMI_OK;
}

int mpmi_screener_set_weights(mpmi_screener* s, const float* w) {
  if (!s || !w) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  SCR_CUDA(cudaMemcpy(s->params, w, kP * sizeof(float), cudaMemcpyHostToDevice), "write weights");
  SCR_CUDA(cudaMemset(s->adam_m, 0, kP * sizeof(float)), "reset Adam");
  SCR_CUDA(cudaMemset(s->adam_v, 0, kP * sizeof(float)), "reset Adam");
  s->step = 0;
  s->stale = true;
  return MPMI_OK;
}

int mpmi_screener_tick_features(mpmi_screener* s, const double* x_t_dev, float* out_dev,
                                void* stream) {
  if (!s || !x_t_dev || !out_dev) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  tick_features<<<1, 256, 0, (cudaStream_t)stream>>>(feature_src(s), x_t_dev, out_dev);
  SCR_CUDA(cudaGetLastError(), "tick_features launch");
  return MPMI_OK;
}

int mpmi_screener_features(mpmi_screener* s, mpmi_session* session, const double* x_t_dev,
                           const double* u_h_dev, uint64_t tick, float* out_dev, void* stream) {
  if (!s || !session || !x_t_dev || !u_h_dev || !out_dev)
    return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  if (session->model != s->model) return fail(MPMI_E_INVALID_ARG, "screener: another model");
  if (session->cfg.sampler == MPMI_SAMPLER_EXTERNAL)
    return fail(MPMI_E_UNSUPPORTED, "screener: sampled candidates only");
  TickArgs a = make_tick_args(session, tick);
  a.x_t = x_t_dev;
  a.u_h = u_h_dev;
  const int blocks = (session->n_slots + 255) / 256 < 1024 ? (session->n_slots + 255) / 256 : 1024;
  slot_features<<<blocks, 256, 0, (cudaStream_t)stream>>>(a, feature_src(s), out_dev);
  SCR_CUDA(cudaGetLastError(), "slot_features launch");
  return MPMI_OK;
}

int mpmi_screener_gradients(mpmi_screener* s, const float* feats, const float* target,
                            int32_t batch, float* grad_dev, float* loss_dev, void* stream) {
  if (!s || !feats || !target || !grad_dev || !loss_dev)
    return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  if (batch < 1 || batch > s->max_batch) return fail(MPMI_E_INVALID_ARG, "screener: batch size");
  return gradients(s, feats, target, batch, grad_dev, loss_dev, (cudaStream_t)stream);
}

int mpmi_screener_train_step(mpmi_screener* s, const float* feats, const float* target,
                             int32_t batch, float lr, float* loss_dev, void* stream) {
  if (!s || !feats || !target || !loss_dev) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  if (batch < 1 || batch > s->max_batch) return fail(MPMI_E_INVALID_ARG, "screener: batch size");
  if (!(lr > 0.f)) return fail(MPMI_E_INVALID_ARG, "screener: learning rate must be > 0");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = gradients(s, feats, target, batch, s->grad, loss_dev, st);
  if (rc != MPMI_OK) return rc;
  s->step += 1;
  const float c1 = 1.f - powf(0.9f, (float)s->step), c2 = 1.f - powf(0.999f, (float)s->step);
  adam<<<(kP + 255) / 256, 256, 0, st>>>(s->params, s->grad, s->adam_m, s->adam_v, lr, c1, c2);
  SCR_CUDA(cudaGetLastError(), "adam launch");
  s->stale = true;
  return MPMI_OK;
}

int mpmi_screener_score(mpmi_screener* s, const float* feats, int32_t batch, float* scores,
                        void* stream) {
  if (!s || !feats || !scores) return fail(MPMI_E_INVALID_ARG, "screener: NULL argument");
  if (batch < 1) return fail(MPMI_E_INVALID_ARG, "screener: batch size");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = refresh_infer(s, st);
  if (rc != MPMI_OK) return rc;
  // one 128-row tile per block and step, at most two blocks per SM (each holds
  // 128 TMEM columns)
  const int tiles = (batch + kTileRows - 1) / kTileRows;
  const int blocks = tiles < 2 * s->ctx->sm_count ? tiles : 2 * s->ctx->sm_count;
  score_rows<<<blocks, kScoreThreads, kScoreSmem, st>>>(s->infer, feats, batch, scores);
  SCR_CUDA(cudaGetLastError(), "score_rows launch");
  return MPMI_OK;
}

int mpmi_evaluate_screened(mpmi_session* session, mpmi_screener* s, const double* x_t_dev,
                           const double* u_h_dev, uint64_t tick, int32_t k, float tau,
                           int32_t m, mpmi_result* result_dev, int32_t* list_dev,
                           int32_t* n_list_dev, void* stream) {
  if (!session || !s || !x_t_dev || !u_h_dev || !result_dev)
    return fail(MPMI_E_INVALID_ARG, "evaluate_screened: NULL argument");
  int rc = screened_checks(session, s, k, tau, m);
  if (rc != MPMI_OK) return rc;
  TickArgs a = make_tick_args(session, tick);
  a.x_t = x_t_dev;
  a.u_h = u_h_dev;
  a.result = result_dev;
  return screened_chain(session, s, a, k, tau, m, list_dev, n_list_dev, (cudaStream_t)stream);
}

int mpmi_evaluate_screened_host(mpmi_session* session, mpmi_screener* s, const double* x_t,
                                const double* u_h, uint64_t tick, int32_t k, float tau,
                                int32_t m, void* stream) {
  if (!session || !s || !x_t || !u_h)
    return fail(MPMI_E_INVALID_ARG, "evaluate_screened_host: NULL argument");
  int rc = screened_checks(session, s, k, tau, m);
  if (rc != MPMI_OK) return rc;
  const mpmi_model* mdl = session->model;
  for (int j = 0; j < mdl->nx; ++j)
    if (!isfinite(x_t[j])) return fail(MPMI_E_NONFINITE, "x_t holds NaN/Inf");
  for (int j = 0; j < mdl->nu; ++j)
    if (!isfinite(u_h[j])) return fail(MPMI_E_NONFINITE, "u_h holds NaN/Inf");
  DeviceGuard guard(session->ctx->device);
  if (guard.err != cudaSuccess) return cfail(guard.err, "cudaSetDevice");
  if ((rc = host_tick_begin(session)) != MPMI_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  memcpy(session->in_host, x_t, sizeof(double) * mdl->nx);
  memcpy(session->in_host + 8, u_h, sizeof(double) * mdl->nu);
  TickArgs a = make_tick_args(session, tick);
  if (session->zero_copy) {
    // the kernels read x_t and u_h from the pinned buffer and write the result
    // into pinned memory; the launch whose result is final stores the number
    a.x_t = session->in_map;
    a.u_h = session->in_map + 8;
    a.result = session->result_map;
    a.seq_out = session->seq_map;
    a.seq = ++session->seq;  // taken even if a launch fails: a later tick never reuses it
  } else {
    SCR_CUDA(cudaMemcpyAsync(session->in_dev, session->in_host, 12 * sizeof(double),
                             cudaMemcpyHostToDevice, st), "copy x_t/u_h to the device");
    a.x_t = session->in_dev;
    a.u_h = session->in_dev + 8;
    a.result = session->result_dev;
  }
  if ((rc = screened_chain(session, s, a, k, tau, m, nullptr, nullptr, st)) != MPMI_OK) {
    // launches queued before the failing one may still run: later launches and
    // closing the session wait for them
    if (cudaEventRecord(session->done, st) == cudaSuccess) session->tail_pending = true;
    return rc;
  }
  if (!session->zero_copy)
    SCR_CUDA(cudaMemcpyAsync(session->result_host, session->result_dev, sizeof(mpmi_result),
                             cudaMemcpyDeviceToHost, st), "copy the result to the host");
  return host_tick_end(session, st);
}

}  // extern "C"
