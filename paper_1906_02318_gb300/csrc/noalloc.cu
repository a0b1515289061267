// A tick entry point that allocates nothing (mpmi_evaluate_candidates_noalloc).
//
// Who needs it: callers that must not allocate device memory while they run --
// a hard real-time control loop that forbids allocation after start-up
// (cudaMalloc/cudaFree can block and synchronise the whole device, which breaks
// a 100 Hz deadline), or a host framework that owns all device memory through
// its own allocator and only hands this library finished buffers.  Such callers
// cannot open a session, because a session allocates its reduction record,
// result and staging buffers.
//
// This entry point takes every buffer from the caller (K, x_t, u_h, the optional
// candidates and the result) and keeps the only scratch the tick needs -- one
// partial (selection key, counts) per thread block plus a block counter -- in
// the file-scope array g_noalloc_scratch below.  That array is part of the
// loaded module: every GPU that loads the library holds it (16,392 bytes) until
// the process exits.  Because the array is shared, calls whose kernels overlap
// on the GPU (different streams, or several host threads) race and corrupt each
// other's results; serialise them on one stream.  The array keeps whatever the
// last call left; the block counter, the only part that must start at zero, is
// cleared (cudaMemsetAsync, which allocates nothing) before every launch.
//
// Limits: at most kNoAllocMaxBlocks thread blocks per call, so at most
// kNoAllocMaxBlocks * (block / 32) * (32 / lanes) candidate slots; larger calls
// are rejected with MPMI_E_INVALID_ARG.  The safety set is the per-coordinate
// box only (a track needs a preprocessed grid, i.e. an allocation).
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress, with that device current, and caches it.  Make the
// first call on a device before any stream capture begins.  A cudaDeviceReset
// destroys the module and with it the cached address: do not reset a device
// while the library is in use on it.
//
// Alignment: K_dev 16 bytes (read as float4 by the register-resident shapes),
// x_t_dev, u_h_dev and result_dev 8 bytes, candidates_dev 4 bytes; a misaligned
// buffer is refused before any CUDA call.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "tick_kernel.cuh"

namespace mpmi {

constexpr int kNoAllocMaxBlocks = 1024;
constexpr int kNoAllocWords = 2 * kNoAllocMaxBlocks + 1;  // keys, counts, block counter

// The scratch of every no-allocation call (see the header comment).
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
static unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once).
static int scratch_address(int dev, unsigned long long** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(MPMI_E_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(MPMI_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MPMI_OK;
}

struct NoAllocKernel {
  void (*launch)(const TickArgs&, int, int, size_t, cudaStream_t) = nullptr;
  size_t k_smem = 0;
};

template <int KIND, int L, bool KSMEM>
static void launch_noalloc(const TickArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  tick_kernel<KIND, L, 1, KSMEM, false, true><<<grid, block, smem, st>>>(a);
}

template <int KIND, int L, bool KSMEM>
static NoAllocKernel make_noalloc() {
  NoAllocKernel k;
  k.launch = &launch_noalloc<KIND, L, KSMEM>;
  k.k_smem = KSMEM ? KSmem<BasisTraits<KIND>::N>::BYTES : 0;
  return k;
}

static NoAllocKernel pick_noalloc(int kind, int lanes) {
  switch (kind) {
    case kBot:
      if (lanes == 1) return make_noalloc<kBot, 1, false>();
      if (lanes == 2) return make_noalloc<kBot, 2, false>();
      if (lanes == 4) return make_noalloc<kBot, 4, false>();
      break;
    case kCar:
      if (lanes == 1) return make_noalloc<kCar, 1, true>();
      if (lanes == 8) return make_noalloc<kCar, 8, false>();
      if (lanes == 16) return make_noalloc<kCar, 16, false>();
      break;
    case kLin11: if (lanes == 1) return make_noalloc<kLin11, 1, false>(); break;
    case kLin22: if (lanes == 1) return make_noalloc<kLin22, 1, false>(); break;
    case kLin41: if (lanes == 1) return make_noalloc<kLin41, 1, false>(); break;
  }
  return NoAllocKernel{};
}

}  // namespace mpmi

using namespace mpmi;

extern "C" int mpmi_evaluate_candidates_noalloc(
    const mpmi_basis_desc* basis, const float* K_dev, const mpmi_safety_spec* spec,
    const mpmi_session_config* cfg, const double* x_t_dev, const double* u_h_dev,
    const float* candidates_dev, uint64_t tick, mpmi_result* result_dev, void* stream) {
  if (!basis || !K_dev || !spec || !cfg || !x_t_dev || !u_h_dev || !result_dev)
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: NULL argument");
  // The register-resident shapes read K as float4 and the kernel reads x_t, u_h
  // and writes the result as 8-byte words: a misaligned caller buffer would be a
  // misaligned-address fault on the device, so refuse it here, before any CUDA call.
  if (reinterpret_cast<uintptr_t>(K_dev) & 15)
    return fail(MPMI_E_INVALID_ARG,
                "evaluate_candidates_noalloc: K_dev must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(x_t_dev) | reinterpret_cast<uintptr_t>(u_h_dev) |
       reinterpret_cast<uintptr_t>(result_dev)) & 7)
    return fail(MPMI_E_INVALID_ARG,
                "evaluate_candidates_noalloc: x_t_dev, u_h_dev and result_dev must be 8-byte "
                "aligned");
  if (reinterpret_cast<uintptr_t>(candidates_dev) & 3)
    return fail(MPMI_E_INVALID_ARG,
                "evaluate_candidates_noalloc: candidates_dev must be 4-byte aligned");
  const int kind = basis_kind(basis->basis, basis->nx, basis->nu);
  if (kind < 0) return fail(MPMI_E_UNSUPPORTED, "evaluate_candidates_noalloc: basis not compiled");
  int n, nx, nu, np;
  kind_dims(kind, &n, &nx, &nu, &np);
  if (spec->track_xy)
    return fail(MPMI_E_UNSUPPORTED,
                "evaluate_candidates_noalloc: only box safety sets (a track needs a session)");
  if (!(spec->inflation >= 0.0) || !isfinite(spec->inflation))
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: bad inflation");
  if (cfg->n_samples < 0 || cfg->horizon < 1 || cfg->horizon > MPMI_MAX_HORIZON ||
      (cfg->include_user != 0 && cfg->include_user != 1))
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: bad N, H or include_user");
  const long long slots = (long long)cfg->n_samples + cfg->include_user;
  if (slots < 1 || slots > MPMI_MAX_SLOTS)
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: slot count out of range");
  if (cfg->sampler != MPMI_SAMPLER_UNIFORM && cfg->sampler != MPMI_SAMPLER_EXTERNAL)
    return fail(MPMI_E_UNSUPPORTED, "evaluate_candidates_noalloc: uniform or external samples");
  if ((cfg->sampler == MPMI_SAMPLER_EXTERNAL) != (candidates_dev != nullptr) && cfg->n_samples > 0)
    return fail(MPMI_E_INVALID_ARG,
                "evaluate_candidates_noalloc: candidates_dev goes with the EXTERNAL sampler");
  for (int j = 0; j < nu; ++j) {
    if (!isfinite(cfg->input_lo[j]) || !isfinite(cfg->input_hi[j]) ||
        !(cfg->input_lo[j] < cfg->input_hi[j]))
      return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: bad input box");
  }
  int lanes = cfg->lanes ? cfg->lanes : 1;
  const int block = cfg->block ? cfg->block : 128;
  if (block % 32 != 0 || block < 32 || block > kMaxBlock)
    return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: block must be 32..256, x32");
  if (cfg->cands_per_thread > 1)
    return fail(MPMI_E_UNSUPPORTED, "evaluate_candidates_noalloc: one candidate per thread");
  NoAllocKernel kn = pick_noalloc(kind, lanes);
  if (!kn.launch) return fail(MPMI_E_UNSUPPORTED, "evaluate_candidates_noalloc: lanes not compiled");
  const long long per_block = (long long)block / lanes;
  const long long grid = (slots + per_block - 1) / per_block;
  if (grid > kNoAllocMaxBlocks)
    return fail(MPMI_E_INVALID_ARG,
                "evaluate_candidates_noalloc: " + std::to_string(slots) +
                    " candidate slots need " + std::to_string(grid) + " blocks; the scratch " +
                    "holds " + std::to_string(kNoAllocMaxBlocks) + " (at most " +
                    std::to_string(kNoAllocMaxBlocks * per_block) +
                    " slots with this launch shape)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MPMI_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned long long* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != MPMI_OK) return rc;

  TickArgs a;
  memset(&a, 0, sizeof(a));
  a.K = K_dev;
  a.x_t = x_t_dev;
  a.u_h = u_h_dev;
  a.ext = candidates_dev;
  for (int j = 0; j < MPMI_MAX_NX; ++j) {
    if (j < nx) {
      if (isnan(spec->state_lo[j]) || isnan(spec->state_hi[j]))
        return fail(MPMI_E_INVALID_ARG, "evaluate_candidates_noalloc: NaN bound");
      a.safety.lo[j] = (float)(spec->state_lo[j] + spec->inflation);
      a.safety.hi[j] = (float)(spec->state_hi[j] - spec->inflation);
    } else {
      a.safety.lo[j] = -INFINITY;
      a.safety.hi[j] = INFINITY;
    }
  }
  a.safety.has_track = 0;
  a.kind = kind;
  a.n_samples = cfg->n_samples;
  a.n_slots = (int)slots;
  a.horizon = cfg->horizon;
  a.include_user = cfg->include_user;
  a.sampler = cfg->sampler;
  for (int j = 0; j < MPMI_MAX_NU; ++j) {
    a.in_lo[j] = (float)cfg->input_lo[j];
    a.in_w[j] = (float)(cfg->input_hi[j] - cfg->input_lo[j]);
    a.in_lo64[j] = cfg->input_lo[j];
    a.in_hi64[j] = cfg->input_hi[j];
  }
  a.key0 = (uint32_t)(cfg->seed & 0xFFFFFFFFull);
  a.key1 = (uint32_t)(cfg->seed >> 32);
  a.t_lo = (uint32_t)(tick & 0xFFFFFFFFull);
  a.t_hi = (uint32_t)(tick >> 32);
  a.stream = cfg->stream_id;
  a.tick = tick;
  a.result = result_dev;
  a.partials = scratch;
  a.partials_cap = kNoAllocMaxBlocks;
  cudaStream_t st = (cudaStream_t)stream;
  // the block counter must start at zero (a failed earlier call may have left it set)
  e = cudaMemsetAsync(scratch + 2 * kNoAllocMaxBlocks, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  kn.launch(a, (int)grid, block, kn.k_smem, st);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(MPMI_E_CUDA, std::string("no-allocation tick launch: ") + cudaGetErrorString(e));
  return MPMI_OK;
}
