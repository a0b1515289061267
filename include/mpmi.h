/*
 * mpmi.h - C ABI of the MPMI-SC per-tick hot path on one GPU.
 *
 * Method: Model Predictive Minimal Intervention Shared Control (Broad, Murphey &
 * Argall, "Highly Parallelized Data-driven MPC for Minimal Intervention Shared
 * Control").  Each control tick takes the plant state x_t and the user's input
 * u_h and returns the input u_r to apply (Alg. 2): sample N constant candidate
 * inputs, predict each one's lifted state over H steps with a learned linear
 * operator (z <- K z, Sec. IV-A), reject every candidate whose prediction leaves
 * the safety set at any step (Sec. IV-B, Sec. V-C.1), and choose the safe
 * candidate nearest to u_h (Alg. 2's argmin, Sec. IV-D).
 *
 * Conventions
 *   - Every call returns MPMI_OK (0) or a negative MPMI_E_* code; nothing is
 *     thrown across the ABI.  mpmi_last_error() returns the calling thread's
 *     message for the last failed call.
 *   - The library owns its handles (create/free in pairs).  The caller owns every
 *     buffer it passes; the library copies what it keeps (K, the track, configs).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory on the context's device (e.g. a torch tensor's data_ptr()).
 *   - Streams are cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work on one session must be stream-ordered: two ticks of the same session
 *     may not run concurrently (they share the session's reduction slots).
 *   - Arrays are row-major and densely packed.
 *
 * Data layout on the device
 *   - K: n x n float32, row-major (z_next[i] = sum_k K[i][k] z[k]).
 *   - candidates: N x M float32, row-major (sample i, input dim j at i*M + j).
 *   - per-candidate outputs are indexed by slot: slot 0 is u_h when the session
 *     includes it, slots 1..N are the samples (slots 0..N-1 otherwise).
 */
#ifndef MPMI_H
#define MPMI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define MPMI_OK 0
#define MPMI_E_INVALID_ARG (-1) /* bad pointer, size, enum or state         */
#define MPMI_E_OOM (-2)         /* device/host allocation failed or the
                                   context's memory budget would be exceeded */
#define MPMI_E_NONFINITE (-3)   /* NaN/Inf in a host input that must be finite */
#define MPMI_E_CUDA (-4)        /* a CUDA runtime call failed                 */
#define MPMI_E_NOT_READY (-5)   /* select_input without an evaluate in flight */
#define MPMI_E_UNSUPPORTED (-6) /* combination not compiled into the library  */
#define MPMI_E_TIMEOUT (-7)     /* a bounded wait inside a kernel ran out (the
                                   tick's result has status MPMI_TIMEOUT)      */

/* ---- enums ------------------------------------------------------------- */
/* Lifted bases (Sec. IV-A; the paper's own 6- and 26-function bases were chosen
 * by code that is not published, so these are fixed lists of the same kinds):
 *   BALANCE_BOT: n = 12, x = (theta, theta_dot, x, x_dot), one input u
 *   RACE_CAR:    n = 32, x = (px, py, psi, vx, vy, omega), u = (steer, throttle)
 *   LINEAR:      n = nx + nu, z = (x, u); compiled for (nx, nu) in
 *                {(1, 1), (2, 2), (4, 1)}
 * State coordinates come first in z, so the predicted state is z[0..nx). */
#define MPMI_BASIS_BALANCE_BOT 0
#define MPMI_BASIS_RACE_CAR 1
#define MPMI_BASIS_LINEAR 2

/* Selection status (Alg. 2 argmin; the fallback is this library's reading of
 * the case the paper leaves open: no candidate safe over the whole horizon). */
#define MPMI_SAFE 0
#define MPMI_FALLBACK 1
/* Not a selection: a block of the tick kernel gave up waiting (about a second)
 * for its shared-memory staging, skipped its candidates and flagged the tick;
 * the other fields are not meaningful.  Never expected in normal operation. */
#define MPMI_TIMEOUT 2

/* Candidate sources (Alg. 2 draws xi ~ U^{M x N}; Sec. IV-B describes an
 * equally spaced discretisation; EXTERNAL reads caller-provided samples). */
#define MPMI_SAMPLER_UNIFORM 0
#define MPMI_SAMPLER_GRID 1
#define MPMI_SAMPLER_EXTERNAL 2

#define MPMI_MAX_NX 8
#define MPMI_MAX_NU 4
#define MPMI_MAX_HORIZON 511         /* H - ttv must fit 9 bits of the key    */
#define MPMI_MAX_SLOTS 8388607       /* 2^23 - 1: slot must fit 23 bits        */
#define MPMI_MAX_TRACK_VERTICES 65535

/* ---- plain structs ------------------------------------------------------ */
typedef struct mpmi_ctx mpmi_ctx;
typedef struct mpmi_model mpmi_model;
typedef struct mpmi_session mpmi_session;

typedef struct {
  int32_t basis; /* MPMI_BASIS_* */
  int32_t nx;    /* state dimension: must be 4 (bot), 6 (car) or as compiled  */
  int32_t nu;    /* input dimension M: 1 (bot), 2 (car) or as compiled        */
} mpmi_basis_desc;

/* Safety set (Sec. V-C.1): the predicted state x = z[0..nx) is safe iff
 *   state_lo[j] + inflation < x[j] < state_hi[j] - inflation   for every j < nx
 * (use -INFINITY / +INFINITY for free coordinates) and, when track_xy != NULL,
 *   dist((x[track_x], x[track_y]), closed polyline) < track_half_width - inflation.
 * Comparisons are strict; NaN is unsafe.  inflation is the paper's inflated
 * barrier (>= 0). */
typedef struct {
  double state_lo[MPMI_MAX_NX];
  double state_hi[MPMI_MAX_NX];
  double inflation;
  const double* track_xy; /* host, n_track (x, y) pairs; NULL = no track test  */
  int32_t n_track;        /* 3..MPMI_MAX_TRACK_VERTICES; segment i joins vertex
                             i to vertex (i + 1) mod n_track                    */
  int32_t track_x;        /* state coordinate holding the position's x         */
  int32_t track_y;        /* state coordinate holding the position's y         */
  int32_t pad0;
  double track_half_width;
} mpmi_safety_spec;

typedef struct {
  int32_t n_samples;    /* N >= 0 sampled candidates per tick                  */
  int32_t horizon;      /* H in 1..MPMI_MAX_HORIZON prediction steps           */
  int32_t include_user; /* 1: slot 0 is u_h itself (a safe u_h passes through
                           unchanged); 0: the N samples only (Alg. 2 as printed) */
  int32_t sampler;      /* MPMI_SAMPLER_*                                      */
  double input_lo[MPMI_MAX_NU]; /* candidate box per input dimension           */
  double input_hi[MPMI_MAX_NU];
  uint64_t seed;        /* Philox key (UNIFORM)                                */
  uint32_t stream_id;   /* Philox counter word 3 (UNIFORM): session identity   */
  int32_t lanes;        /* 0 = library choice; else lanes per candidate        */
  int32_t block;        /* 0 = library choice; else threads per block          */
  int32_t cands_per_thread; /* 0 = library choice; else candidates per thread
                               (with one lane per candidate)                    */
} mpmi_session_config;

/* One tick's outcome (written by the device, 80 bytes). */
typedef struct {
  double u_r[MPMI_MAX_NU];  /* selected input: u_h exactly when slot 0 (the user)
                               wins, else the candidate's float32 value           */
  int32_t index;            /* selected slot                                      */
  int32_t status;           /* MPMI_SAFE, MPMI_FALLBACK (or MPMI_TIMEOUT)         */
  int32_t n_safe;           /* candidates safe over all H steps                   */
  int32_t ttv;              /* steps the selected candidate passed (H if safe)    */
  float cost;               /* ||u_r - u_h||^2 in float32                         */
  int32_t n_slots;          /* N + include_user                                   */
  uint64_t executed_steps;  /* prediction steps actually taken (early exit)       */
  uint64_t tick;            /* tick counter the call was given                    */
  uint64_t reserved;
} mpmi_result;

/* ---- context ------------------------------------------------------------ */
/* Binds the library to CUDA device `device`.  mem_budget_bytes caps the device
 * memory sessions and models may hold (0 = no cap); session_open fails with
 * MPMI_E_OOM beyond it.  *out receives the handle. */
int mpmi_create(int32_t device, uint64_t mem_budget_bytes, mpmi_ctx** out);
void mpmi_destroy(mpmi_ctx* ctx); /* close sessions and free models first */
const char* mpmi_last_error(void);
const char* mpmi_version(void);
/* Bytes of device memory currently held against the budget. */
uint64_t mpmi_memory_in_use(const mpmi_ctx* ctx);

/* ---- fit_model (Sec. IV-A) ---------------------------------------------- */
/* Least-squares fit of the lifted operator over m transitions (host, float64):
 *   K = argmin sum_m || Psi(x_next[m], u[m]) - K Psi(x[m], u[m]) ||^2
 * x, x_next: m x nx row-major; u: m x nu row-major (the input is held over the
 * step, so the target lifts x_next with the same u).  Solved by Householder QR
 * in float64 on the host (an offline step, Sec. IV-A "learned offline").
 * *residual_out (may be NULL) = ||X K^T - Y||_F / ||Y||_F.  The model's device
 * copy of K is float32 (round to nearest).  Fails with INVALID_ARG when m < n,
 * NONFINITE on NaN/Inf input, and INVALID_ARG if the lifted data is rank
 * deficient. */
int mpmi_fit_model(mpmi_ctx* ctx, const mpmi_basis_desc* basis, const double* x,
                   const double* u, const double* x_next, int64_t m,
                   mpmi_model** out, double* residual_out);
/* The same fit without a context or a device: writes K (host, n x n float64
 * row-major) to K_out.  Pure host code (usable on machines without a GPU). */
int mpmi_fit_operator(const mpmi_basis_desc* basis, const double* x, const double* u,
                      const double* x_next, int64_t m, double* K_out,
                      double* residual_out);

/* Sparsity-promoting selection of the basis (Sec. IV-A and V-C.3 select the
 * basis functions with sparsity-promoting DMD, Jovanovic et al. 2014; reading:
 * its two stages applied to feature selection).  Stage 1 solves, by ADMM with
 * penalty parameter rho for `iters` iterations,
 *   min (1/m) ||A V - B||_F^2 + gamma sum_{j candidate} ||V[j, :]||_2
 * with A, B the lifted regressors and targets scaled to unit RMS per column and
 * one group per candidate feature (every feature but the state and the held
 * input features); stage 2 refits K by least squares (Householder QR, float64)
 * on the features whose group survived.  K_out (n x n row-major): zero column
 * and zero row for every dropped feature, exact unit rows for held features, so
 * mpmi_model_from_operator accepts it and the tick reads no dropped feature.
 * support_out (n bytes, may be NULL): 1 = kept.  *residual_out (may be NULL):
 * ||X K^T - Y||_F / ||Y||_F over the kept features.  gamma finite >= 0 (0 keeps
 * every feature and equals mpmi_fit_operator up to rounding); rho finite > 0
 * (1 is a good default); iters >= 1 (400 converges on the shipped bases).
 * Pure host code.  INVALID_ARG / NONFINITE / UNSUPPORTED as mpmi_fit_operator. */
int mpmi_fit_operator_sparse(const mpmi_basis_desc* basis, const double* x, const double* u,
                             const double* x_next, int64_t m, double gamma, double rho,
                             int32_t iters, double* K_out, uint8_t* support_out,
                             double* residual_out);
/* A model from a given operator K (host, n x n float64 row-major). */
int mpmi_model_from_operator(mpmi_ctx* ctx, const mpmi_basis_desc* basis,
                             const double* K, mpmi_model** out);
/* Copies the float64 operator to K_out (host, n*n) and n to *n_out. */
int mpmi_model_get_operator(const mpmi_model* model, double* K_out, int32_t* n_out);
void mpmi_model_free(mpmi_model* model); /* sessions using it must be closed */

/* ---- set_safety_set (Sec. V-C.1) --------------------------------------- */
/* Installs the safety set on a model (copied; replaces any previous one).  The
 * track is preprocessed on the host into a uniform grid whose cells are marked
 * inside / outside / boundary (the last with the list of segments that can be
 * nearest), so the device test reads at most a few segments per step and gives
 * the same answer as the brute-force minimum over all segments.  Sessions opened
 * afterwards use the new set. */
int mpmi_set_safety_set(mpmi_model* model, const mpmi_safety_spec* spec);

/* ---- sessions ----------------------------------------------------------- */
/* A controller instance: one model, fixed N and H, its own sampler stream and
 * reduction slots.  Allocates ~200 bytes of device memory and a small pinned
 * host buffer. */
int mpmi_session_open(mpmi_ctx* ctx, const mpmi_model* model,
                      const mpmi_session_config* cfg, mpmi_session** out);
void mpmi_session_close(mpmi_session* s);
/* Lanes per candidate, candidates per thread and threads per block the session
 * launches with (any output pointer may be NULL). */
int mpmi_session_launch_shape(const mpmi_session* s, int32_t* lanes, int32_t* cands,
                              int32_t* block);

/* ---- launch-shape autotuner --------------------------------------------- */
/* Outcome of one tuning run: the fastest shape and its median tick time. */
typedef struct {
  int32_t lanes;     /* lanes per candidate                                    */
  int32_t cands;     /* candidates per thread                                  */
  int32_t block;     /* threads per block                                      */
  int32_t n_tried;   /* shapes measured                                        */
  double us;         /* median device time per tick of the winner (microseconds) */
  double default_us; /* the same for the library's default shape               */
} mpmi_tune_result;

/* Times every compiled launch shape (lanes per candidate x candidates per thread)
 * at 64, 128, 160, 192, 224 and 256 threads per block (every size the built-in
 * rule picks) for one tick configuration -- the model,
 * cfg's N, H, sampler and user slot (cfg's lanes, cands_per_thread and block are
 * ignored) -- from the host state x_t (nx doubles) and input u_h (nu doubles):
 * two warm-up ticks, then `reps` device-resident ticks (1..1000) each timed with
 * CUDA events, median per shape.  The winner is returned in *out and recorded in
 * the context: a later mpmi_session_open with lanes, cands_per_thread and block
 * all 0 and the same (basis, N + include_user, H) uses it instead of the built-in
 * rule.  Every shape computes bit-identical results, so tuning changes speed
 * only.  Opens and closes temporary sessions (device memory within the budget);
 * blocks until done.  INVALID_ARG / NONFINITE as for session_open and
 * evaluate_candidates, OOM beyond the budget. */
int mpmi_tune_launch_shape(mpmi_ctx* ctx, const mpmi_model* model,
                           const mpmi_session_config* cfg, const double* x_t,
                           const double* u_h, int32_t reps, mpmi_tune_result* out);
/* Alg. 2's per-step Gaussian noise z_i ("to account for inaccuracies in the
 * dynamics model"; the paper gives no variance).  After every prediction step t
 * the lifted state's first `count` coordinates (the state read-out, x_0 ..
 * x_{count-1}) get sigma[j] * n_j, n_j standard normal, before step t's safety
 * test; the perturbed state is carried into step t + 1.  The normals come from
 * Philox4x32-10 under the session's seed with counter (slot, tick mod 2^32,
 * (tick div 2^32 mod 2^16) + 2^16 t + 2^25 b, stream_id) for coordinates
 * 4b..4b+3, mapped by Box-Muller (u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8)
 * 2^-24, n = sqrt(-2 ln u1)(cos 2 pi u2, sin 2 pi u2); words (w2, w3) give the
 * next pair), so a tick's noise is a function of (seed, stream, tick, slot)
 * alone.  sigma: count host doubles, finite and >= 0 (rounded to float32);
 * count = 0 turns the noise off (the default).  Applies to every later tick of
 * the session (host, device, trajectory and screened evaluations); ticks must
 * then stay below 2^48.  MPMI_E_INVALID_ARG for count outside 0..nx or a tick
 * in flight, MPMI_E_NONFINITE for a NaN/Inf sigma. */
int mpmi_session_set_noise(mpmi_session* s, const double* sigma, int32_t count);

/* Rollout form of the session's ticks.  FULL (the default) predicts z <- K z as
 * Alg. 2 does.  FACTORED is an ablation that is exact in real arithmetic: with
 * the input held over the horizon (Sec. IV-A, VII-B) and the lifting affine in
 * the input monomials p_k, z_0 = a(x_t) + sum_k p_k(xi) b_k(x_t), so each
 * predicted state coordinate is e_j K^t a + sum_k p_k e_j K^t b_k.  Setting it
 * computes the rows C K^t (t = 1..H, the n_x state rows) on the device once
 * (H * n_x * n floats of device memory, counted against the budget); each tick
 * then folds them with a(x_t), b_k(x_t) and tests only the coordinates the
 * safety set bounds (and the position for a track), at (1 + P) FMAs per
 * read-out per step instead of n^2.  Results agree with FULL up to rounding.
 * Ticks of a FACTORED session return MPMI_E_UNSUPPORTED for trajectory
 * recording and with noise switched on (the noise enters after K and does not
 * factor).  MPMI_E_INVALID_ARG for an unknown mode or a tick in flight,
 * MPMI_E_OOM beyond the budget.  Blocks until the rows are computed. */
#define MPMI_ROLLOUT_FULL 0
#define MPMI_ROLLOUT_FACTORED 1
/* TENSOR (race car only): the same z <- K z as FULL, computed for tiles of 128
 * candidates as one matrix product per step on the tcgen05 tensor cores (Sec.
 * IV-A: a batch of predictions is one matrix-matrix product).  Each float32
 * operand is split into two TF32 parts and the product taken as hi*hi + lo*hi
 * (one float32 accumulator in tensor memory) plus hi*lo (a second one), the two
 * added in float32 (error of the order of float32 rounding); held features are
 * restored exactly after every step.
 * Results agree with the float64 reference under the same tolerance as FULL but
 * are not bit-identical to it.  Supports trajectories, noise and screened
 * ticks; no extra device memory.  MPMI_E_UNSUPPORTED for other bases. */
#define MPMI_ROLLOUT_TENSOR 2
int mpmi_session_set_rollout(mpmi_session* s, int32_t mode);

/* Persistent host ticks (not part of the method; the tick itself is Alg. 2
 * unchanged).  With on != 0, host ticks (mpmi_evaluate_candidates) of the FULL
 * rollout without noise and with a built-in sampler run in one kernel that stays
 * resident on the device between ticks: it stages K and the track grid once and
 * then waits on a mailbox in pinned host memory; each host tick writes x_t, u_h
 * and the tick into the mailbox and publishes its sequence number with one
 * system-scope compare-and-swap, and select_input waits for the completion word
 * as for zero-copy ticks.  No CUDA call is made per tick.  Results are
 * bit-identical to the launched tick of the same session.
 *   idle_ms: the kernel exits after this long without a command (0 = 1000 ms;
 *     at most 60000); the next host tick relaunches it.  Every wait inside the
 *     kernel is bounded by it.
 *   Other ticks of the session (device-resident, trajectories, screened ticks,
 *   ticks with noise or another rollout) first stop the resident kernel and run
 *   as launches; the next host tick restarts it.  on = 0 stops it (after any
 *   tick in flight has been published) and returns to launched host ticks.
 * The resident kernel holds at most one block per SM (cooperative launch, on a
 * stream of its own) and one polling thread per block while idle; other work on
 * the device gets the remaining resources until the idle limit or a stop.  The
 * resident grids of several persistent sessions must fit beside each other: a
 * grid that cannot start waits until another one exits.
 * MPMI_E_UNSUPPORTED where the device cannot map host memory, has no native
 * host-memory atomics or cooperative launch, or the session's launch shape has
 * no persistent form; MPMI_E_INVALID_ARG for idle_ms outside 0..60000 or NaN. */
int mpmi_session_set_persistent(mpmi_session* s, int32_t on, double idle_ms);

/* ---- evaluate_candidates + select_input (Alg. 2) ------------------------ */
/* Queues one tick on `stream`: copies x_t (nx doubles) and u_h (nu doubles) into
 * the session's pinned staging buffer, samples the candidates (counter = tick),
 * predicts, tests, scores and reduces them on the GPU, and brings the result back
 * to pinned host memory.  Where the device can map host memory the kernel reads
 * the staging buffer and writes the result over the host link directly
 * (zero-copy); otherwise two asynchronous copies do it.  Returns without waiting.
 * candidates_dev: device N x M float32 samples for MPMI_SAMPLER_EXTERNAL, else
 * must be NULL.  NONFINITE if x_t or u_h holds NaN/Inf.  If a previous tick of
 * this session is still in flight, waits for it first.  In persistent mode
 * (mpmi_session_set_persistent) the tick is handed to the resident kernel through
 * the mailbox and `stream` is not used. */
int mpmi_evaluate_candidates(mpmi_session* s, const double* x_t, const double* u_h,
                             const float* candidates_dev, uint64_t tick,
                             void* stream);
/* Waits for the tick queued by mpmi_evaluate_candidates and copies its outcome
 * to *out (host).  With zero-copy ticks it returns as soon as the kernel has
 * published the result (a completion word stored after it, polled for up to a
 * second before falling back to the tick's CUDA event); the session's next
 * launch is ordered behind the rest of that kernel on the GPU.  A tick handed to
 * a resident kernel (mpmi_session_set_persistent) is waited for on the same word
 * for the idle limit plus a second; then the kernel is stopped (it finishes the
 * tick first) and TIMEOUT is returned if still nothing was published.  NOT_READY
 * if no tick is in flight; TIMEOUT for a result with status MPMI_TIMEOUT. */
int mpmi_select_input(mpmi_session* s, mpmi_result* out);

/* Device-resident form of one tick (nothing is copied to or from the host and
 * nothing is waited for; graph-capturable): x_t_dev (nx doubles) and u_h_dev (nu
 * doubles) are device pointers, the outcome is written to result_dev (device,
 * one mpmi_result).  ttv_dev (int32, n_slots) and cost_dev (float32, n_slots)
 * are optional device outputs per slot (NULL = not written). */
int mpmi_evaluate_candidates_device(mpmi_session* s, const double* x_t_dev,
                                    const double* u_h_dev,
                                    const float* candidates_dev, uint64_t tick,
                                    mpmi_result* result_dev, int32_t* ttv_dev,
                                    float* cost_dev, void* stream);

/* ---- step-level entry points (parity checks) ---------------------------- */
/* Alg. 2 first step alone: writes the tick's n_slots x M candidate values (slot
 * order, slot 0 = u_h when included) to out_dev (device float32).  u_h_dev is
 * read only when the session includes the user's input. */
int mpmi_sample_candidates(mpmi_session* s, const double* u_h_dev,
                           const float* candidates_dev, uint64_t tick,
                           float* out_dev, void* stream);
/* The same tick as mpmi_evaluate_candidates_device that also records the lifted
 * trajectories: traj_dev (device float32, n_slots x (H + 1) x n) receives z_0 and
 * every predicted z_t the candidate reached (t <= min(ttv + 1, H)); entries past
 * a candidate's early exit are left untouched. */
/* Test hook, not part of the method: with on != 0 every later tick of the
 * session announces its shared-memory staging (K rows and the track grid) to
 * the kernel's mbarrier but issues no copy, so each block's bounded wait runs
 * out after about a second (twice), the blocks skip their candidates and the
 * result comes back with status MPMI_TIMEOUT (select_input: MPMI_E_TIMEOUT).
 * Exercises the wait limit without a fault; only shapes that stage shared
 * memory (race car with K in shared memory or a track, factorised race car)
 * are affected.  on = 0 restores normal ticks. */
int mpmi_debug_withhold_staging(mpmi_session* s, int32_t on);

/* Host mirror of the race car's track test (Sec. V-C.1: unsafe off the road),
 * for checking the grid the library builds without a GPU.  Builds the grid of
 * the closed centre line track_xy (n_track vertices, row-major x, y) for the
 * half width and answers, for each float32 point (x, y) of points (n_points x 2,
 * host), whether it lies within the half width of the centre line, with the
 * device's own cell lookup and listed-segment test in float32.  on_road: n_points
 * bytes (host).  Pure host code.  INVALID_ARG for bad sizes, NONFINITE for a
 * non-finite vertex, UNSUPPORTED if the grid does not fit shared memory. */
int mpmi_debug_track_query(const double* track_xy, int32_t n_track, double half_width,
                           const float* points, int64_t n_points, uint8_t* on_road);

/* Test hook for Alg. 2's sampling step: the generator the candidates come from is
 * Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  For each of n records of
 * six uint32 words (counter c0 c1 c2 c3, key k0 k1; records_dev, device, n x 6)
 * writes the four output words of the device's generator to words_dev (device,
 * n x 4 uint32), so the device function can be checked against the published
 * known-answer vectors.  Buffers 4-byte aligned and caller-owned.  Asynchronous
 * on `stream`.  INVALID_ARG for NULL buffers, misalignment or n outside
 * [0, 2^30]; CUDA if the launch fails. */
int mpmi_debug_philox(const uint32_t* records_dev, int64_t n, uint32_t* words_dev,
                      void* stream);

/* Measured FP32 FMA throughput of CUDA device `device` (not part of the method;
 * the denominator of the tick kernels' ALU roofline): every resident warp runs
 * eight independent FMA chains for about `seconds` (0 < seconds <= 10); the
 * flops over the launch's CUDA-event time, in TFLOP/s, go to *tflops_out (host).
 * The rate is the one at the clocks the device ran at.  Blocks until done.
 * INVALID_ARG for a NULL output or seconds out of range, CUDA/OOM on failure. */
int mpmi_measure_fp32_peak(int32_t device, double seconds, double* tflops_out);

int mpmi_debug_trajectories(mpmi_session* s, const double* x_t_dev,
                            const double* u_h_dev, const float* candidates_dev,
                            uint64_t tick, mpmi_result* result_dev,
                            int32_t* ttv_dev, float* cost_dev, float* traj_dev,
                            void* stream);

/* ---- continuous-batching server ------------------------------------------ */
/* Serves many control sessions of one model together: each admitted session has
 * its own N, H, input box, sampler seed/stream and tick counter; the requests
 * staged for a batch run in one launch (replayed from a CUDA graph) whose warps
 * stride over all requests' candidates, and every request's result is
 * bit-identical to the same tick evaluated alone (same per-candidate arithmetic,
 * exact min-reduction).  Up to four batches of the server run at once, each on a
 * stream of the server's own, while the requests of the next one are staged on
 * the host; a launch's blocks beyond its batch's candidates leave at once, so
 * batches in flight share the device.  A session has at most one request staged
 * or on the GPU at a time.  The server snapshots the model's operator and safety
 * set when it is created.  Served sessions draw uniform samples. */
typedef struct mpmi_server mpmi_server;
/* max_sessions session slots; their reduction records and five batch tables are
 * allocated here (and counted against the context's memory budget). */
int mpmi_server_create(mpmi_ctx* ctx, const mpmi_model* model, int32_t max_sessions,
                       mpmi_server** out);
void mpmi_server_free(mpmi_server* s); /* waits for the batches in flight */
/* Admission: a free slot and room in the context's memory budget for the
 * session's share, else MPMI_E_OOM.  *slot_out identifies the session. */
int mpmi_server_admit(mpmi_server* s, const mpmi_session_config* cfg, int32_t* slot_out);
/* Frees a session slot (NOT_READY while it has a staged or running request). */
int mpmi_server_release(mpmi_server* s, int32_t slot);
/* Stages n requests for the next batch (host arrays): slots[n], x_t (n x nx),
 * u_h (n x nu), ticks[n].  INVALID_ARG for a session that already has a request
 * staged or on the GPU (a controller needs its last output before its next
 * input). */
int mpmi_server_submit(mpmi_server* s, int32_t n, const int32_t* slots, const double* x_t,
                       const double* u_h, const uint64_t* ticks);
/* Requests staged so far for the next batch. */
int mpmi_server_staged(const mpmi_server* s, int32_t* n_out);
/* Launches the staged batch (one graph launch) and returns.  The batch is ordered
 * after the work queued so far on `stream` and runs on its buffer's own stream,
 * so it overlaps the batches already in flight.  NOT_READY when max_in_flight
 * batches are on the GPU.  *n_launched may be 0 (nothing staged). */
int mpmi_server_launch(mpmi_server* s, void* stream, int32_t* n_launched);
/* How many batches may be on the GPU at once: 1..4 (default 4).  1 gives one batch
 * at a time (a launch waits for the previous batch to be collected). */
int mpmi_server_set_max_in_flight(mpmi_server* s, int32_t n);
/* Batches on the GPU now (launched, not yet collected). */
int mpmi_server_in_flight(const mpmi_server* s, int32_t* n_out);
/* *done = 1 when a batch in flight has finished (0 if none has, or none flies). */
int mpmi_server_poll(mpmi_server* s, int32_t* done);
/* Collects one batch in flight: the earliest launched of those that have
 * finished, else waits for the earliest launched.  Copies its results (host, in
 * submission order) with the sessions they belong to; *n_out = number of
 * results.  NOT_READY if no batch is in flight. */
int mpmi_server_collect(mpmi_server* s, mpmi_result* out, int32_t* slots_out, int32_t* n_out);
/* Autotunes the server's launch shape for a request mix: for every compiled
 * shape of the model's basis (lanes per candidate x candidates per thread) at 64,
 * 128 and 256 threads per block, serves `reps` batches (1..100, after one
 * warm-up batch) of the n requests described by cfgs[n] (session configurations,
 * admitted on temporary slots and released again), x_t (n x nx) and u_h (n x nu)
 * through the server's own submit / launch / collect path, timing each graph
 * launch with CUDA events; the shape with the lowest median batch time is kept
 * for all later batches and returned in *out (default_us: the server's initial
 * shape).  Results are bit-identical across shapes.  NOT_READY while a batch is
 * staged or in flight, OOM without n free slots. */
int mpmi_server_tune(mpmi_server* s, int32_t n, const mpmi_session_config* cfgs,
                     const double* x_t, const double* u_h, int32_t reps,
                     mpmi_tune_result* out);

/* ---- learned candidate screener (not in the paper) ----------------------- */
/* A small network (12 -> 128 -> 128 -> 1, tanh-form GELU, sigmoid output) that
 * predicts, for the race car, each candidate's normalised time to violation
 * ttv / H from the state, the track ahead and the candidate, so that only the
 * most promising candidates go through the exact rollout.  Inputs: the signed
 * lateral offset from the nearest centre-line segment / half width, sin and cos
 * of the heading error, vx / 25, vy / 5, omega / 2, 10 x the curvature at the
 * first vertex 5, 10, 20, 40 m ahead, delta / 0.4 and the throttle.  Weights
 * are float32 (training, on the GPU with this library's own forward and
 * backward kernels) with a bfloat16 copy for tensor-core inference.  Packed
 * weight layout (float32, MPMI_SCREENER_PARAMS values): W1 (128 x 12, row-major),
 * b1 (128), W2 (128 x 128), b2 (128), w3 (128), b3 (1). */
#define MPMI_SCREENER_PARAMS 18305
#define MPMI_SCREENER_INPUTS 12
typedef struct mpmi_screener mpmi_screener;

/* A screener for a race-car model whose safety set has a track (the features
 * use the track).  weights: host, packed initial weights.  max_batch bounds the
 * training minibatch; max_slots bounds the candidate slots of screened ticks. */
int mpmi_screener_create(mpmi_ctx* ctx, const mpmi_model* model, const float* weights,
                         int32_t max_batch, int32_t max_slots, mpmi_screener** out);
void mpmi_screener_free(mpmi_screener* s);
int mpmi_screener_get_weights(const mpmi_screener* s, float* weights_out);
int mpmi_screener_set_weights(mpmi_screener* s, const float* weights);
/* The 10 per-tick inputs of a state (device x_t_dev, 6 doubles -> out_dev). */
int mpmi_screener_tick_features(mpmi_screener* s, const double* x_t_dev, float* out_dev,
                                void* stream);
/* The 12 inputs of every slot of a session's tick (slot order, slot 0 = u_h when
 * included) -> out_dev (n_slots x 12 float32). */
int mpmi_screener_features(mpmi_screener* s, mpmi_session* session, const double* x_t_dev,
                           const double* u_h_dev, uint64_t tick, float* out_dev,
                           void* stream);
/* Mean squared error and its gradient (packed like the weights) on a minibatch:
 * features (batch x 12) and targets (batch, in [0, 1]), all device float32. */
int mpmi_screener_gradients(mpmi_screener* s, const float* features_dev,
                            const float* targets_dev, int32_t batch, float* grad_dev,
                            float* loss_dev, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a minibatch; *loss_dev gets
 * the minibatch loss before the step. */
int mpmi_screener_train_step(mpmi_screener* s, const float* features_dev,
                             const float* targets_dev, int32_t batch, float lr,
                             float* loss_dev, void* stream);
/* Network output (sigmoid, predicted ttv / H) for feature rows, computed with
 * bfloat16 weights and activations on tensor cores with float32 accumulation. */
int mpmi_screener_score(mpmi_screener* s, const float* features_dev, int32_t batch,
                        float* scores_dev, void* stream);
/* A screened tick (exact): roll out a prefix of the tick's cost order (least
 * ||xi - u_h||^2 first), cut between two cost bins (the float32 exponent and the
 * top three mantissa bits of the cost), so that every slot left out costs more
 * than every slot kept.  The prefix is the shortest one holding at least k slots
 * and, with the network (tau > 0), at least m slots the network predicts safe
 * (score >= tau); tau <= 0 skips the network (the k cheapest slots, the exact
 * cost-ordered search).  The kept slots go through the exact rollout; if none of
 * them is safe and they are not every slot, the full evaluation runs on the
 * device with no host round trip.  Either the kept slots contain the least-cost
 * safe candidate of the whole tick or they are all unsafe, so the selection is
 * always the exhaustive one: the network decides only how far down the cost
 * order the tick goes.  result_dev's reserved word carries flags: bit 0 the
 * screened set was evaluated, bit 1 the full evaluation ran; executed_steps
 * counts the steps of both launches, n_slots the slots of the last.  list_dev
 * (optional, n_slots int32) receives the kept slots and n_list_dev (optional,
 * one int32) their number.  INVALID_ARG for k < 1, or m < 1 with tau > 0. */
int mpmi_evaluate_screened(mpmi_session* session, mpmi_screener* s, const double* x_t_dev,
                           const double* u_h_dev, uint64_t tick, int32_t k, float tau,
                           int32_t m, mpmi_result* result_dev, int32_t* list_dev,
                           int32_t* n_list_dev, void* stream);

/* The same screened tick from host buffers (x_t: nx doubles, u_h: nu doubles,
 * both read before the call returns), for a closed loop on the host: queued on
 * `stream` like mpmi_evaluate_candidates, and its result is collected with
 * mpmi_select_input (flags and counts as above).  On devices that can map host
 * memory the kernels read x_t and u_h from the session's pinned buffer and write
 * the result into pinned memory, and the launch whose result is final stores
 * the tick's number, which select_input polls; otherwise the inputs and the
 * result are copied.  A tick still in flight on the session is waited for
 * first.  Errors as mpmi_evaluate_screened, and NONFINITE for a NaN or
 * infinite x_t or u_h. */
int mpmi_evaluate_screened_host(mpmi_session* session, mpmi_screener* s, const double* x_t,
                                const double* u_h, uint64_t tick, int32_t k, float tau,
                                int32_t m, void* stream);

/* Phase timing of screened ticks (a measurement aid, not part of the method):
 * with on != 0 every later mpmi_evaluate_screened of this screener records CUDA
 * events on its stream around its four launches; mpmi_screener_phase_times waits
 * for the last tick's events and writes ms_out[4] (host): the screen (network or
 * cost keys and histograms), the compaction, the exact rollout of the kept slots
 * and the fallback launch (which returns at once when it is not needed).  The
 * events are created on the first switch-on.  NOT_READY if timing was never on. */
int mpmi_screener_set_timing(mpmi_screener* s, int32_t on);
int mpmi_screener_phase_times(mpmi_screener* s, float* ms_out);

/* ---- a tick that allocates nothing -------------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that may
 * not allocate device memory while they run: a hard real-time control loop that
 * forbids allocation after start-up (cudaMalloc/cudaFree can block and
 * synchronise the device, breaking the tick deadline), or a framework that owns
 * all device memory and only hands this library finished buffers.  It performs
 * the same tick as mpmi_evaluate_candidates_device without a session and calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *   basis          the lifted basis (as for mpmi_model_from_operator)
 *   K_dev          device, n x n float32 row-major operator (caller-owned),
 *                  16-byte aligned
 *   spec           host; per-coordinate box and inflation only: track_xy must be
 *                  NULL (a track needs the grid a model allocates)
 *   cfg            host; N, H, include_user, sampler (UNIFORM or EXTERNAL),
 *                  input box, seed, stream_id, lanes, block (0 = defaults)
 *   x_t_dev, u_h_dev, candidates_dev, tick, result_dev, stream: as for
 *                  mpmi_evaluate_candidates_device
 * Scratch: one partial result per thread block lives in a static device array of
 * 16,392 bytes inside the library, held by every GPU that loads the library until
 * the process exits.  A call may use at most 1024 blocks, i.e. at most
 * 1024 * (block / lanes) candidate slots; larger calls fail with
 * MPMI_E_INVALID_ARG and a message giving the limit.  All calls share that array:
 * calls whose kernels overlap on the GPU race and must not be issued (keep them on
 * one stream).  The first call on each device looks up the array's address; make
 * it before any stream capture begins, and do not cudaDeviceReset a device the
 * library is in use on (the looked-up address dies with the module).
 * Alignment: K_dev must be 16-byte aligned (the register-resident launch shapes
 * read it as float4), x_t_dev, u_h_dev and result_dev 8-byte aligned,
 * candidates_dev 4-byte aligned; otherwise MPMI_E_INVALID_ARG before any CUDA
 * call.  Returns without waiting. */
int mpmi_evaluate_candidates_noalloc(const mpmi_basis_desc* basis, const float* K_dev,
                                     const mpmi_safety_spec* spec,
                                     const mpmi_session_config* cfg, const double* x_t_dev,
                                     const double* u_h_dev, const float* candidates_dev,
                                     uint64_t tick, mpmi_result* result_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPMI_H */
