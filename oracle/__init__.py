"""FP64 CPU oracle for the MPMI-SC per-tick path (Broad, Murphey & Argall,
"Highly Parallelized Data-driven MPC for Minimal Intervention Shared Control").

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the controller computes, used to check the CUDA path.  Only
the test-suite, the package's smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA path (and imports nothing from
it); the two meet only through the seeded inputs of the ``workloads`` package.

Modules, each citing the passage it follows:

* ``philox``   counter-based generator (Salmon et al., SC'11) for Alg. 2's samples
* ``sampling`` candidate inputs xi ~ U^{M x N} (Alg. 2), the equally spaced
               grid of Sec. IV-B, and Alg. 2's per-step Gaussian noise z_i
               (Box-Muller normals from the same generator)
* ``basis``    lifted features Psi(x, u) of the learned linear model (Sec. IV-A)
* ``fit``      least-squares fit of the lifted operator K (Sec. IV-A) and the
               sparsity-promoting basis selection (Sec. IV-A, V-C.3)
* ``safety``   isSafe: geometric checks with an inflated barrier (Sec. V-C.1)
* ``mpmi``     Alg. 2 (prediction, rejection, minimal-intervention argmin)
* ``screener`` the learned candidate screener (not in the paper): features,
               network, loss, gradients, Adam

Parity unpinned (stated here and in the design notes): how well a fitted K
predicts the true plant (it is a model; only the fit residual is reported), and
every human-study result (Sec. VI-A, VI-B, Table I values).
"""
from . import philox, sampling, basis, fit, safety, mpmi  # noqa: F401
