// The noisy instances of the fused tick kernel (Alg. 2 with its per-step
// Gaussian noise z_i), compiled apart from the noise-free ones.
#include "tick_dispatch.cuh"

namespace mpmi {

TickKernel pick_tick_noise(int kind, int lanes, int cands, bool traj) {
  return pick_variant<true>(kind, lanes, cands, traj);
}

}  // namespace mpmi
