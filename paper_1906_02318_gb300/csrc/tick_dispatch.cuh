// Launch table of the fused tick kernel: which template instance serves a
// (basis, lanes, candidates per thread, trajectories, noise) combination.  The
// noise-free instances are compiled in mpmi_api.cu, the noisy ones in
// tick_noise.cu, so the two halves build in parallel.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "tick_kernel.cuh"

namespace mpmi {

struct TickKernel {
  const void* fn = nullptr;
  void (*launch)(const TickArgs&, int, int, size_t, cudaStream_t) = nullptr;
  size_t k_smem = 0;  // bytes of K staged in shared memory
};

// A TickArgs with `chained` set is launched with programmatic stream
// serialisation (it may start before the previous kernel on the stream ends and
// waits for it in the kernel); any other launch is an ordinary one.
template <int KIND, int L, int C, bool KSMEM, bool TRAJ, bool NOISE>
static void launch_tick(const TickArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  if (!a.chained) {
    tick_kernel<KIND, L, C, KSMEM, TRAJ, false, NOISE><<<grid, block, smem, st>>>(a);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, tick_kernel<KIND, L, C, KSMEM, TRAJ, false, NOISE>, a);
}

template <int KIND, int L, int C, bool KSMEM, bool TRAJ, bool NOISE>
static TickKernel make_kernel() {
  TickKernel k;
  k.fn = reinterpret_cast<const void*>(&tick_kernel<KIND, L, C, KSMEM, TRAJ, false, NOISE>);
  k.launch = &launch_tick<KIND, L, C, KSMEM, TRAJ, NOISE>;
  k.k_smem = (size_t)ksmem_words<KIND, L, KSMEM, true>() * 16;
  return k;
}

// Compiled launch shapes: (lanes, candidates per thread).  The race car keeps K
// in shared memory with 1, 2 or 4 lanes per candidate and in registers with 8 or
// 16; the other bases keep K in registers.
template <int KIND, bool TRAJ, bool NOISE>
static TickKernel pick_shape(int lanes, int cands) {
  if constexpr (KIND == kBot) {
    if (lanes == 1 && cands == 1) return make_kernel<KIND, 1, 1, false, TRAJ, NOISE>();
    if (lanes == 1 && cands == 2) return make_kernel<KIND, 1, 2, false, TRAJ, NOISE>();
    if (lanes == 2 && cands == 1) return make_kernel<KIND, 2, 1, false, TRAJ, NOISE>();
    if (lanes == 4 && cands == 1) return make_kernel<KIND, 4, 1, false, TRAJ, NOISE>();
  } else if constexpr (KIND == kCar) {
    if (lanes == 1 && cands == 1) return make_kernel<KIND, 1, 1, true, TRAJ, NOISE>();
    if (lanes == 1 && cands == 2) return make_kernel<KIND, 1, 2, true, TRAJ, NOISE>();
    if (lanes == 2 && cands == 1) return make_kernel<KIND, 2, 1, true, TRAJ, NOISE>();
    if (lanes == 4 && cands == 1) return make_kernel<KIND, 4, 1, true, TRAJ, NOISE>();
    if (lanes == 8 && cands == 1) return make_kernel<KIND, 8, 1, false, TRAJ, NOISE>();
    if (lanes == 16 && cands == 1) return make_kernel<KIND, 16, 1, false, TRAJ, NOISE>();
  } else {
    if (lanes == 1 && cands == 1) return make_kernel<KIND, 1, 1, false, TRAJ, NOISE>();
  }
  return TickKernel{};
}

template <bool NOISE>
static TickKernel pick_variant(int kind, int lanes, int cands, bool traj) {
  switch (kind) {
#define MPMI_PICK(K) \
    case K: return traj ? pick_shape<K, true, NOISE>(lanes, cands) : pick_shape<K, false, NOISE>(lanes, cands);
    MPMI_PICK(kBot)
    MPMI_PICK(kCar)
    MPMI_PICK(kLin11)
    MPMI_PICK(kLin22)
    MPMI_PICK(kLin41)
#undef MPMI_PICK
  }
  return TickKernel{};
}

// the noisy half of the table (tick_noise.cu)
TickKernel pick_tick_noise(int kind, int lanes, int cands, bool traj);

}  // namespace mpmi
