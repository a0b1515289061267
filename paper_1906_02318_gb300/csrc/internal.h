// Internal types shared by the host side of the library and the tick kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mpmi.h"
#include "basis.h"

namespace mpmi {

// Track grid cell word: bits 0-1 class, bits 2-23 list offset, bits 24-31 count.
enum CellClass : uint32_t { kCellOutside = 0, kCellInside = 1, kCellBoundary = 2 };

// Track grid staged into shared memory by every block: one blob of 16-byte
// aligned sections  cells (u32) | segment lists (u16) | segments (float4
// ax, ay, dx, dy) | 1/|d|^2 (float).
struct DevTrack {
  const uint4* blob;      // device copy of the blob
  int blob_bytes;         // multiple of 16
  int off_list, off_seg, off_inv;  // byte offsets of the sections
  float gx0, gy0, inv_h;  // grid origin and 1 / cell size
  int gnx, gny;
  float w2;               // (half width - inflation)^2
};

struct DevSafety {
  float lo[MPMI_MAX_NX];  // inflated open bounds (float32)
  float hi[MPMI_MAX_NX];
  int has_track;
  DevTrack track;
};

// Per-session reduction slots the tick kernel accumulates into.  The block that
// finishes last decodes them into the result and resets them for the next tick.
struct TickScratch {
  unsigned long long key;     // min over candidates of the selection key
  unsigned long long counts;  // (n_safe << 40) + executed prediction steps
  unsigned int done;          // blocks finished
  unsigned int error;         // set by a block whose bounded staging wait ran out
  unsigned int pad[2];
};

struct TickArgs {
  const float* K;      // n x n float32 row-major (device)
  const float* Ks;     // the same K with each row's columns in staging order
  const float* Kp;     // the free rows of K in pairs (KPair layout; race car)
                       // (free columns, then held ones; shared-memory shapes)
  const double* x_t;   // device, nx
  const double* u_h;   // device, nu
  const float* ext;    // device samples N x nu (EXTERNAL) or null
  DevSafety safety;
  int kind;            // BasisKind
  int n_samples, n_slots, horizon, include_user, sampler;
  float in_lo[MPMI_MAX_NU], in_w[MPMI_MAX_NU];        // float32 box (UNIFORM)
  double in_lo64[MPMI_MAX_NU], in_hi64[MPMI_MAX_NU];  // float64 box (GRID)
  int grid_g;          // points per dimension (GRID)
  uint32_t key0, key1, t_lo, t_hi, stream;
  unsigned long long tick;
  TickScratch* scratch;
  mpmi_result* result;
  int32_t* ttv_out;
  float* cost_out;
  float* traj_out;
  // per-block partial results (no-allocation variant only): keys [0, cap),
  // counts [cap, 2 cap), block counter at [2 cap]
  unsigned long long* partials;
  int partials_cap;
  // screened ticks: evaluate only the slots slot_list[0 .. *n_list) (device);
  // skip the whole launch when *skip_if_safe already holds a SAFE result;
  // result_flags is stored in the result's reserved word
  const int* slot_list;
  const int* n_list;
  const mpmi_result* skip_if_safe;
  unsigned long long result_flags;
  // Alg. 2's per-step noise z_i: sigma per state coordinate (zero past n_noise)
  float noise_sigma[MPMI_MAX_NX];
  int n_noise;
  // factorised rollout: rows C K^t (t = 1..H, n_x rows of n each) and the state
  // coordinates the safety test reads (position first when a track is set)
  const float* ck;
  int ro_n;
  int ro_idx[MPMI_MAX_NX];
  // test hook: stage nothing, so the bounded staging wait runs out
  int withhold_staging;
  // launched as a programmatic dependent of the previous kernel on the stream
  // (a screened tick's chain): wait for it before reading anything
  int chained;
  // zero-copy host ticks: after the result, the decoding block stores seq here
  // (pinned host memory) behind a system-scope fence
  unsigned long long* seq_out;
  unsigned long long seq;
  // a screened host tick's kept-slot rollout: store seq only when its result is
  // the tick's final one (a safe pick, or every slot kept); otherwise the
  // fallback launch, which then runs the full evaluation, stores it
  int seq_if_final;
};

// Persistent host ticks: the mailbox (pinned host memory) and its device copy
// are kCmdWords 64-bit words: [0] command number, [1] tick, [2, 10) x_t,
// [10, 14) u_h (doubles); word kCmdHalt of the device copy is block 0's halt
// flag.  Flags in the mailbox's word 0: kCmdStop (host: halt once the pending
// command is done), kCmdExit (kernel: exited after the idle limit).
constexpr int kCmdWords = 16;
constexpr int kCmdPayload = 14;  // words 0 .. 13
constexpr int kCmdHalt = 14;
constexpr unsigned long long kCmdStop = 1ull << 63;
constexpr unsigned long long kCmdExit = 1ull << 62;
constexpr unsigned long long kCmdSeqMask = kCmdExit - 1;

struct PersistArgs {
  unsigned long long* mbox;  // device alias of the pinned mailbox
  unsigned long long* cmd;   // device copy that blocks other than 0 read
  unsigned long long start_seq;  // commands numbered above this one are new
  unsigned long long idle_ns;    // exit after this long without a command
};

}  // namespace mpmi

// ---- host handles ----------------------------------------------------------
struct mpmi_ctx {
  int device = 0;
  uint64_t budget = 0;
  uint64_t used = 0;
  int sm_count = 0;
  // launch shapes chosen by the autotuner, keyed by (basis, slots, horizon)
  struct TunedShape {
    int kind, n_slots, horizon, lanes, cands, block;
  };
  std::vector<TunedShape> tuned;
};

struct mpmi_model {
  mpmi_ctx* ctx = nullptr;
  int basis = 0, kind = 0, n = 0, nx = 0, nu = 0, np = 0;
  std::vector<double> K64;
  // n x n row-major, then the same rows in staging order, then (race car) the
  // pair layout of the one-lane shared-memory shapes
  float* K32_dev = nullptr;
  bool has_safety = false;
  mpmi_safety_spec spec{};
  std::vector<double> track_host;
  mpmi::DevSafety dev_safety{};
  uint4* track_dev = nullptr;  // packed track grid (see DevTrack)
  uint64_t track_bytes = 0;
  uint64_t bytes = 0;
};

struct mpmi_session {
  mpmi_ctx* ctx = nullptr;
  const mpmi_model* model = nullptr;
  mpmi_session_config cfg{};
  int n_slots = 0, lanes = 1, cands = 1, block = 128, grid_g = 0;
  // resident blocks on the device per launch kind (plain or trajectories, all
  // slots or the few-candidate shape, with or without noise) and the dynamic
  // shared memory they assume
  // (index: trajectories + 2 few-candidate shape + 4 noise + 8 sixteen lanes in
  // the few-candidate shape)
  int max_grid[16] = {};
  size_t grid_smem[16] = {};
  mpmi::TickScratch* scratch_dev = nullptr;
  mpmi_result* result_dev = nullptr;
  double* in_dev = nullptr;        // x_t (8 doubles) then u_h (4 doubles)
  double* in_host = nullptr;       // pinned staging
  mpmi_result* result_host = nullptr;  // pinned
  // device-side aliases of the pinned buffers (zero-copy host ticks)
  double* in_map = nullptr;
  mpmi_result* result_map = nullptr;
  bool zero_copy = false;
  unsigned long long* seq_host = nullptr;  // pinned; written by the device after a result
  unsigned long long* seq_map = nullptr;
  unsigned long long seq = 0;
  // select_input returned on the completion word while the kernel may still be
  // resetting the reduction record: the next launch waits for `done` first
  bool tail_pending = false;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
  float noise_sigma[MPMI_MAX_NX] = {0, 0, 0, 0, 0, 0, 0, 0};
  int n_noise = 0;
  int rollout = MPMI_ROLLOUT_FULL;
  float* ck_dev = nullptr;         // C K^t rows (factorised rollout)
  uint64_t ck_bytes = 0;
  int fact_grid = 0;               // resident blocks of the factorised kernel
  size_t fact_smem = 0;
  int tc_grid[2] = {0, 0};         // resident CTAs of the tensor-core rollout (plain, traj)
  size_t tc_smem[2] = {0, 0};        // its shared memory need, and what a launch asks for
  size_t tc_req[2] = {0, 0};
  int withhold_staging = 0;        // test hook (mpmi_debug_withhold_staging)
  // persistent host ticks (persistent.cu)
  bool persist = false;            // requested by mpmi_session_set_persistent
  bool persist_running = false;    // a resident kernel may be waiting on the mailbox
  bool persist_posted = false;     // the tick in flight went through the mailbox
  unsigned long long persist_idle_ns = 0;
  unsigned long long* mbox_host = nullptr;  // pinned, kCmdWords words
  unsigned long long* mbox_map = nullptr;
  unsigned long long* cmd_dev = nullptr;    // kCmdWords words
  unsigned long long cmd_init[mpmi::kCmdWords] = {};  // source of the copy that resets it
  cudaStream_t persist_stream = nullptr;
  cudaEvent_t persist_done = nullptr;
  uint64_t bytes = 0;
};

namespace mpmi {
// Makes the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = err == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// tick launch helpers shared by the API and the screener (mpmi_api.cu)
TickArgs make_tick_args(const mpmi_session* s, uint64_t tick);
// list_lanes: lanes per race-car candidate of a launch over a device-side list
// (16, or 0 for the built-in 8)
int launch_tick_args(mpmi_session* s, TickArgs& a, bool traj, cudaStream_t st, int n_hint,
                     int list_lanes = 0);
// host ticks: wait for the one in flight; record the completion event after the launches
int host_tick_begin(mpmi_session* s);
int host_tick_end(mpmi_session* s, cudaStream_t st);
// factorised rollout (factored.cu)
int compute_powers(int kind, const float* K, int H, float* out, cudaStream_t st);
int launch_factored(mpmi_session* s, TickArgs& a, cudaStream_t st, int n_hint);
// persistent host ticks (persistent.cu)
bool persist_supported(int kind, int lanes, int cands);
int launch_persistent(mpmi_session* s, const TickArgs& a, const PersistArgs& p);
// tensor-core rollout (tensor.cu)
int launch_tensor(mpmi_session* s, TickArgs& a, bool traj, cudaStream_t st, int n_hint);
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
// host helpers implemented in fit.cpp / track.cpp
int fit_householder(int kind, const double* x, const double* u, const double* xn,
                    int64_t m, std::vector<double>* K, double* residual, std::string* err);
int fit_sparse(int kind, const double* x, const double* u, const double* xn, int64_t m,
               double gamma, double rho, int iters, std::vector<double>* K,
               std::vector<unsigned char>* support, double* residual, std::string* err);
struct TrackGrid {
  std::vector<uint32_t> cells;
  std::vector<uint16_t> list;
  double gx0 = 0, gy0 = 0, h = 1;
  int gnx = 0, gny = 0;
  // packed blob (16-byte aligned sections) and its section offsets
  std::vector<uint8_t> blob;
  int off_list = 0, off_seg = 0, off_inv = 0;
};
constexpr int kMaxTrackBytes = 96 * 1024;  // shared-memory budget of the grid
int build_track_grid(const double* xy, int n, double half_width, TrackGrid* g,
                     std::string* err);
int track_query_host(const double* xy, int n, double half_width, const float* pts, int64_t np,
                     uint8_t* on_road, std::string* err);
}  // namespace mpmi
