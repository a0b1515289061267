"""Thin Python binding of libmpmi.so (include/mpmi.h): argument marshalling only.

Every computation of a tick runs in the CUDA library; this module converts
numpy arrays and torch tensors to pointers, checks return codes and turns the
80-byte result record into a dict.  There is no Python or CPU fallback: if the
shared library is missing, loading raises.

Names follow the C ABI: fit_model, model_from_operator, set_safety_set,
Session (session_open/close), evaluate_candidates, select_input,
evaluate_candidates_device, sample_candidates, debug_trajectories.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmpmi.so")

BASIS = {"bot": 0, "car": 1, "linear": 2}
BASIS_DIMS = {"bot": (4, 1), "car": (6, 2)}
BASIS_SIZE = {"bot": 12, "car": 32}   # lifted dimension n; the linear basis has nx + nu
SAMPLER = {"uniform": 0, "grid": 1, "external": 2}
ROLLOUT = {"full": 0, "factored": 1, "tensor": 2}
SAFE, FALLBACK, TIMEOUT = 0, 1, 2
MAX_NX, MAX_NU = 8, 4
MAX_HORIZON, MAX_SLOTS = 511, 8388607
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "NONFINITE", -4: "CUDA", -5: "NOT_READY",
          -6: "UNSUPPORTED", -7: "TIMEOUT"}

c_i32, c_u32, c_i64, c_u64, c_dbl, c_vp = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p)
P_dbl = ctypes.POINTER(ctypes.c_double)


class BasisDesc(ctypes.Structure):
    _fields_ = [("basis", c_i32), ("nx", c_i32), ("nu", c_i32)]


class SafetySpecC(ctypes.Structure):
    _fields_ = [("state_lo", c_dbl * MAX_NX), ("state_hi", c_dbl * MAX_NX),
                ("inflation", c_dbl), ("track_xy", P_dbl), ("n_track", c_i32),
                ("track_x", c_i32), ("track_y", c_i32), ("pad0", c_i32),
                ("track_half_width", c_dbl)]


class TuneResult(ctypes.Structure):
    _fields_ = [("lanes", c_i32), ("cands", c_i32), ("block", c_i32), ("n_tried", c_i32),
                ("us", c_dbl), ("default_us", c_dbl)]


class SessionConfig(ctypes.Structure):
    _fields_ = [("n_samples", c_i32), ("horizon", c_i32), ("include_user", c_i32),
                ("sampler", c_i32), ("input_lo", c_dbl * MAX_NU), ("input_hi", c_dbl * MAX_NU),
                ("seed", c_u64), ("stream_id", c_u32), ("lanes", c_i32), ("block", c_i32),
                ("cands_per_thread", c_i32)]


class Result(ctypes.Structure):
    _fields_ = [("u_r", c_dbl * MAX_NU), ("index", c_i32), ("status", c_i32),
                ("n_safe", c_i32), ("ttv", c_i32), ("cost", ctypes.c_float),
                ("n_slots", c_i32), ("executed_steps", c_u64), ("tick", c_u64),
                ("reserved", c_u64)]


RESULT_BYTES = ctypes.sizeof(Result)
assert RESULT_BYTES == 80 and ctypes.sizeof(SafetySpecC) == 168
assert ctypes.sizeof(SessionConfig) == 104

_SIGNATURES = {
    "mpmi_create": (c_i32, [c_i32, c_u64, ctypes.POINTER(c_vp)]),
    "mpmi_destroy": (None, [c_vp]),
    "mpmi_last_error": (ctypes.c_char_p, []),
    "mpmi_version": (ctypes.c_char_p, []),
    "mpmi_memory_in_use": (c_u64, [c_vp]),
    "mpmi_fit_model": (c_i32, [c_vp, ctypes.POINTER(BasisDesc), c_vp, c_vp, c_vp, c_i64,
                               ctypes.POINTER(c_vp), P_dbl]),
    "mpmi_fit_operator": (c_i32, [ctypes.POINTER(BasisDesc), c_vp, c_vp, c_vp, c_i64, c_vp,
                                  P_dbl]),
    "mpmi_model_from_operator": (c_i32, [c_vp, ctypes.POINTER(BasisDesc), c_vp,
                                         ctypes.POINTER(c_vp)]),
    "mpmi_model_get_operator": (c_i32, [c_vp, c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_model_free": (None, [c_vp]),
    "mpmi_set_safety_set": (c_i32, [c_vp, ctypes.POINTER(SafetySpecC)]),
    "mpmi_session_open": (c_i32, [c_vp, c_vp, ctypes.POINTER(SessionConfig),
                                  ctypes.POINTER(c_vp)]),
    "mpmi_session_close": (None, [c_vp]),
    "mpmi_session_set_noise": (c_i32, [c_vp, P_dbl, c_i32]),
    "mpmi_session_set_rollout": (c_i32, [c_vp, c_i32]),
    "mpmi_session_set_persistent": (c_i32, [c_vp, c_i32, c_dbl]),
    "mpmi_measure_fp32_peak": (c_i32, [c_i32, c_dbl, P_dbl]),
    "mpmi_tune_launch_shape": (c_i32, [c_vp, c_vp, ctypes.POINTER(SessionConfig), c_vp, c_vp,
                                       c_i32, ctypes.POINTER(TuneResult)]),
    "mpmi_server_tune": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_i32,
                                 ctypes.POINTER(TuneResult)]),
    "mpmi_debug_withhold_staging": (c_i32, [c_vp, c_i32]),
    "mpmi_fit_operator_sparse": (c_i32, [ctypes.POINTER(BasisDesc), c_vp, c_vp, c_vp, c_i64,
                                          c_dbl, c_dbl, c_i32, c_vp, c_vp, P_dbl]),
    "mpmi_debug_track_query": (c_i32, [P_dbl, c_i32, c_dbl, c_vp, c_i64, c_vp]),
    "mpmi_debug_philox": (c_i32, [c_vp, c_i64, c_vp, c_vp]),
    "mpmi_session_launch_shape": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32),
                                          ctypes.POINTER(c_i32)]),
    "mpmi_evaluate_candidates": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_vp]),
    "mpmi_select_input": (c_i32, [c_vp, c_vp]),
    "mpmi_evaluate_candidates_device": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_vp, c_vp,
                                                c_vp, c_vp]),
    "mpmi_sample_candidates": (c_i32, [c_vp, c_vp, c_vp, c_u64, c_vp, c_vp]),
    "mpmi_debug_trajectories": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_vp, c_vp, c_vp,
                                        c_vp, c_vp]),
    "mpmi_server_create": (c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(c_vp)]),
    "mpmi_server_free": (None, [c_vp]),
    "mpmi_server_admit": (c_i32, [c_vp, ctypes.POINTER(SessionConfig), ctypes.POINTER(c_i32)]),
    "mpmi_server_release": (c_i32, [c_vp, c_i32]),
    "mpmi_server_submit": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "mpmi_server_staged": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_server_launch": (c_i32, [c_vp, c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_server_poll": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_server_set_max_in_flight": (c_i32, [c_vp, c_i32]),
    "mpmi_server_in_flight": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_server_collect": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(c_i32)]),
    "mpmi_screener_create": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "mpmi_screener_free": (None, [c_vp]),
    "mpmi_screener_get_weights": (c_i32, [c_vp, c_vp]),
    "mpmi_screener_set_weights": (c_i32, [c_vp, c_vp]),
    "mpmi_screener_tick_features": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "mpmi_screener_features": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_vp, c_vp]),
    "mpmi_screener_gradients": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "mpmi_screener_train_step": (c_i32, [c_vp, c_vp, c_vp, c_i32, ctypes.c_float, c_vp, c_vp]),
    "mpmi_screener_score": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "mpmi_screener_set_timing": (c_i32, [c_vp, c_i32]),
    "mpmi_screener_phase_times": (c_i32, [c_vp, c_vp]),
    "mpmi_evaluate_screened": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_i32, ctypes.c_float,
                                       c_i32, c_vp, c_vp, c_vp, c_vp]),
    "mpmi_evaluate_screened_host": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_i32,
                                            ctypes.c_float, c_i32, c_vp]),
    "mpmi_evaluate_candidates_noalloc": (c_i32, [ctypes.POINTER(BasisDesc), c_vp,
                                                 ctypes.POINTER(SafetySpecC),
                                                 ctypes.POINTER(SessionConfig), c_vp, c_vp,
                                                 c_vp, c_u64, c_vp, c_vp]),
}

_lib = None


class MpmiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libmpmi.so (built by paper_1906_02318_gb300.build); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_1906_02318_gb300.build`"
                           " (the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        raise MpmiError(rc, load().mpmi_last_error().decode())


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _require(t, name, itemsize, min_numel, dtype=None):
    """Check a caller's CUDA tensor before its address crosses the C ABI: on the
    current device, contiguous, of the element size (and dtype) the entry point
    reads, with at least min_numel elements."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: must live on the current CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if t.element_size() != itemsize:
        raise TypeError(f"{name}: expected {itemsize}-byte elements, got {t.dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: needs at least {min_numel} elements, has {t.numel()}")


def _f64(a, n=None):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def result_dict(r: Result, nu: int) -> dict:
    return dict(u_r=np.array(r.u_r[:nu]), index=r.index, status=r.status, n_safe=r.n_safe,
                ttv=r.ttv, cost=r.cost, n_slots=r.n_slots, executed_steps=r.executed_steps,
                tick=r.tick, flags=r.reserved)


def result_from_bytes(buf, nu: int) -> dict:
    """Decode an mpmi_result record (bytes / uint8 array / CPU uint8 tensor)."""
    if hasattr(buf, "numpy"):
        buf = buf.numpy()
    raw = bytes(np.asarray(buf, dtype=np.uint8).reshape(-1)[:RESULT_BYTES])
    return result_dict(Result.from_buffer_copy(raw), nu)


class Context:
    """mpmi_create / mpmi_destroy: the library bound to one CUDA device."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        self.lib = load()
        h = c_vp()
        _check(self.lib.mpmi_create(device, mem_budget, ctypes.byref(h)))
        self.handle = h
        self.device = device

    def memory_in_use(self) -> int:
        return int(self.lib.mpmi_memory_in_use(self.handle))

    def close(self):
        if self.handle:
            self.lib.mpmi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """A fitted (or given) lifted operator K with its safety set."""

    def __init__(self, ctx: Context, handle, basis: str, nx: int, nu: int):
        self.ctx, self.handle, self.basis, self.nx, self.nu = ctx, handle, basis, nx, nu
        self.safety = None  # the last set_safety_set arguments (for checkpoints)

    def get_operator(self) -> np.ndarray:
        n = c_i32()
        _check(self.ctx.lib.mpmi_model_get_operator(self.handle, None, ctypes.byref(n)))
        K = np.empty((n.value, n.value), dtype=np.float64)
        _check(self.ctx.lib.mpmi_model_get_operator(self.handle, K.ctypes.data, ctypes.byref(n)))
        return K

    def free(self):
        if self.handle:
            self.ctx.lib.mpmi_model_free(self.handle)
            self.handle = None


def _desc(basis: str, nx: int | None, nu: int | None) -> BasisDesc:
    if basis in BASIS_DIMS:
        nx, nu = BASIS_DIMS[basis]
    return BasisDesc(BASIS[basis], nx, nu)


def fit_model(ctx: Context, basis: str, x, u, x_next, nx: int | None = None,
              nu: int | None = None):
    """mpmi_fit_model: float64 least squares over transitions; returns (Model, residual)."""
    d = _desc(basis, nx, nu)
    x = _f64(x).reshape(-1, d.nx)
    u = _f64(u).reshape(-1, d.nu)
    xn = _f64(x_next).reshape(-1, d.nx)
    h = c_vp()
    res = ctypes.c_double()
    _check(ctx.lib.mpmi_fit_model(ctx.handle, ctypes.byref(d), x.ctypes.data, u.ctypes.data,
                                  xn.ctypes.data, x.shape[0], ctypes.byref(h),
                                  ctypes.byref(res)))
    return Model(ctx, h, basis, d.nx, d.nu), res.value


def fit_operator(basis: str, x, u, x_next, nx: int | None = None, nu: int | None = None):
    """mpmi_fit_operator: the host float64 fit alone (no device); returns (K, residual)."""
    lib = load()
    d = _desc(basis, nx, nu)
    x = _f64(x).reshape(-1, d.nx)
    u = _f64(u).reshape(-1, d.nu)
    xn = _f64(x_next).reshape(-1, d.nx)
    n = d.nx + d.nu if basis == "linear" else {"bot": 12, "car": 32}[basis]
    K = np.empty((n, n), dtype=np.float64)
    res = ctypes.c_double()
    _check(lib.mpmi_fit_operator(ctypes.byref(d), x.ctypes.data, u.ctypes.data, xn.ctypes.data,
                                 x.shape[0], K.ctypes.data, ctypes.byref(res)))
    return K, res.value


def fit_operator_sparse(basis: str, x, u, x_next, gamma: float, rho: float = 1.0,
                        iters: int = 400, nx: int | None = None, nu: int | None = None):
    """mpmi_fit_operator_sparse: sparsity-promoting basis selection and refit on
    the host; returns (K float64 n x n, support bool mask, residual)."""
    lib = load()
    d = _desc(basis, nx, nu)
    x = _f64(x).reshape(-1, d.nx)
    u = _f64(u).reshape(-1, d.nu)
    xn = _f64(x_next).reshape(-1, d.nx)
    n = d.nx + d.nu if basis == "linear" else {"bot": 12, "car": 32}[basis]
    K = np.empty((n, n), dtype=np.float64)
    sup = np.zeros(n, dtype=np.uint8)
    res = ctypes.c_double()
    _check(lib.mpmi_fit_operator_sparse(ctypes.byref(d), x.ctypes.data, u.ctypes.data,
                                        xn.ctypes.data, x.shape[0], float(gamma), float(rho),
                                        int(iters), K.ctypes.data, sup.ctypes.data,
                                        ctypes.byref(res)))
    return K, sup.astype(bool), res.value


def debug_track_query(track_xy, half_width: float, points) -> np.ndarray:
    """mpmi_debug_track_query: host mirror of the device's on-road test (bool per point)."""
    tr = _f64(track_xy).reshape(-1, 2)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.float32).reshape(-1, 2))
    out = np.zeros(pts.shape[0], dtype=np.uint8)
    _check(load().mpmi_debug_track_query(tr.ctypes.data_as(P_dbl), tr.shape[0], float(half_width),
                                         pts.ctypes.data, pts.shape[0], out.ctypes.data))
    return out.astype(bool)


def model_from_operator(ctx: Context, basis: str, K, nx: int | None = None,
                        nu: int | None = None) -> Model:
    """mpmi_model_from_operator: a model from a given n x n operator (float64)."""
    d = _desc(basis, nx, nu)
    K = _f64(K)
    h = c_vp()
    _check(ctx.lib.mpmi_model_from_operator(ctx.handle, ctypes.byref(d), K.ctypes.data,
                                            ctypes.byref(h)))
    return Model(ctx, h, basis, d.nx, d.nu)


def set_safety_set(model: Model, lo, hi, inflation: float = 0.0, track=None,
                   half_width: float = 0.0):
    """mpmi_set_safety_set: open per-coordinate bounds (+ optional closed track)."""
    spec = SafetySpecC()
    lo = _f64(lo)
    hi = _f64(hi)
    for j in range(MAX_NX):
        spec.state_lo[j] = lo[j] if j < lo.size else -np.inf
        spec.state_hi[j] = hi[j] if j < hi.size else np.inf
    spec.inflation = inflation
    keep = None
    if track is not None:
        keep = _f64(track).reshape(-1, 2)
        spec.track_xy = keep.ctypes.data_as(P_dbl)
        spec.n_track = keep.shape[0]
        spec.track_x, spec.track_y = 0, 1
        spec.track_half_width = half_width
    _check(model.ctx.lib.mpmi_set_safety_set(model.handle, ctypes.byref(spec)))
    model.safety = dict(lo=lo.copy(), hi=hi.copy(), inflation=float(inflation),
                        track=None if keep is None else keep.copy(),
                        half_width=float(half_width))
    del keep


def _session_config(n_samples, horizon, input_lo, input_hi, include_user=True,
                    sampler="uniform", seed=0, stream_id=0, lanes=0, block=0, cands=0):
    cfg = SessionConfig()
    cfg.n_samples, cfg.horizon = n_samples, horizon
    cfg.include_user = int(include_user)
    cfg.sampler = SAMPLER[sampler]
    lo, hi = _f64(input_lo), _f64(input_hi)
    for j in range(MAX_NU):
        cfg.input_lo[j] = lo[j] if j < lo.size else 0.0
        cfg.input_hi[j] = hi[j] if j < hi.size else 1.0
    cfg.seed, cfg.stream_id, cfg.lanes, cfg.block = seed, stream_id, lanes, block
    cfg.cands_per_thread = cands
    return cfg


def tune_launch_shape(ctx: Context, model: Model, n_samples: int, horizon: int, input_lo,
                      input_hi, x_t, u_h, reps: int = 20, include_user: bool = True,
                      sampler: str = "uniform", seed: int = 0, stream_id: int = 0) -> dict:
    """mpmi_tune_launch_shape: time every compiled launch shape for this tick
    configuration; the winner is used by later sessions opened with the library's
    choice of shape (results are bit-identical across shapes)."""
    cfg = _session_config(n_samples, horizon, input_lo, input_hi, include_user, sampler, seed,
                          stream_id)
    x = _f64(x_t, model.nx)
    u = _f64(u_h, model.nu)
    r = TuneResult()
    _check(ctx.lib.mpmi_tune_launch_shape(ctx.handle, model.handle, ctypes.byref(cfg),
                                          x.ctypes.data, u.ctypes.data, int(reps),
                                          ctypes.byref(r)))
    return dict(lanes=r.lanes, cands=r.cands, block=r.block, n_tried=r.n_tried, us=r.us,
                default_us=r.default_us)


class Session:
    """mpmi_session_open: one controller with fixed N and H."""

    def __init__(self, ctx: Context, model: Model, n_samples: int, horizon: int,
                 input_lo, input_hi, include_user: bool = True, sampler: str = "uniform",
                 seed: int = 0, stream_id: int = 0, lanes: int = 0, block: int = 0,
                 cands: int = 0):
        cfg = _session_config(n_samples, horizon, input_lo, input_hi, include_user, sampler,
                              seed, stream_id, lanes, block, cands)
        h = c_vp()
        _check(ctx.lib.mpmi_session_open(ctx.handle, model.handle, ctypes.byref(cfg),
                                         ctypes.byref(h)))
        self.ctx, self.model, self.handle = ctx, model, h
        # the opening arguments, the noise and the rollout form (for checkpoints)
        self.config = dict(n_samples=int(n_samples), horizon=int(horizon),
                           input_lo=_f64(input_lo).copy(), input_hi=_f64(input_hi).copy(),
                           include_user=bool(include_user), sampler=sampler, seed=int(seed),
                           stream_id=int(stream_id), lanes=int(lanes), block=int(block),
                           cands=int(cands))
        self.noise = np.zeros(0)
        self.rollout = "full"
        self.n_samples, self.horizon, self.include_user = n_samples, horizon, bool(include_user)
        self.n_slots = n_samples + int(include_user)
        self.nx, self.nu = model.nx, model.nu
        self.n = model.get_operator().shape[0]
        self._result = Result()   # reused by select_input
        self._result_ptr = ctypes.addressof(self._result)
        self._u_r = np.frombuffer(self._result, dtype=np.float64, count=MAX_NU)
        # x_t / u_h staging for host ticks (the library copies them during the call)
        self._in = np.zeros(MAX_NX + MAX_NU)
        self._x_ptr = self._in.ctypes.data
        self._u_ptr = self._x_ptr + 8 * MAX_NX
        self._in_x = self._in[:self.nx]
        self._in_u = self._in[MAX_NX:MAX_NX + self.nu]
        self._stream_key = self._stream_arg = None  # the last stream object and its handle

    def launch_shape(self):
        """(lanes per candidate, candidates per thread, threads per block)."""
        lanes, cands, block = c_i32(), c_i32(), c_i32()
        _check(self.ctx.lib.mpmi_session_launch_shape(self.handle, ctypes.byref(lanes),
                                                      ctypes.byref(cands), ctypes.byref(block)))
        return lanes.value, cands.value, block.value

    def set_noise(self, sigma):
        """mpmi_session_set_noise: Alg. 2's per-step Gaussian noise on the first
        len(sigma) state coordinates (an empty sigma turns it off)."""
        sig = np.ascontiguousarray(np.atleast_1d(np.asarray(sigma, dtype=np.float64)))
        _check(self.ctx.lib.mpmi_session_set_noise(
            self.handle, sig.ctypes.data_as(P_dbl), int(sig.size)))
        self.noise = sig.copy()

    def set_rollout(self, mode: str):
        """mpmi_session_set_rollout: "full" (z <- K z, Alg. 2, CUDA cores),
        "tensor" (the same on tcgen05 tensor cores, race car) or "factored"
        (read-outs from precomputed rows C K^t; an exact-in-real-arithmetic ablation)."""
        _check(self.ctx.lib.mpmi_session_set_rollout(self.handle, ROLLOUT[mode]))
        self.rollout = mode

    def set_persistent(self, on: bool = True, idle_ms: float = 0.0):
        """mpmi_session_set_persistent: host ticks run in a resident kernel fed
        through a pinned mailbox (idle_ms: exit after that long without a tick;
        0 = one second)."""
        _check(self.ctx.lib.mpmi_session_set_persistent(self.handle, int(bool(on)), float(idle_ms)))

    def withhold_staging(self, on: bool):
        """mpmi_debug_withhold_staging: test hook that makes the kernel's bounded
        staging wait run out (result status TIMEOUT)."""
        _check(self.ctx.lib.mpmi_debug_withhold_staging(self.handle, int(bool(on))))

    def close(self):
        if self.handle:
            self.ctx.lib.mpmi_session_close(self.handle)
            self.handle = None

    def __del__(self):
        # a session holds its context, so the context outlives it; closing also
        # stops a resident tick kernel instead of leaving it to its idle limit
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak(device: int = 0, seconds: float = 0.5) -> float:
    """mpmi_measure_fp32_peak: the device's FP32 FMA throughput in TFLOP/s."""
    out = c_dbl()
    _check(load().mpmi_measure_fp32_peak(device, float(seconds), ctypes.byref(out)))
    return out.value


def _stage(dst, a, n):
    """Copies a host input (x_t or u_h) into the session's staging view."""
    if isinstance(a, np.ndarray) and a.dtype == np.float64 and a.size == n:
        np.copyto(dst, a.reshape(n))
    else:
        dst[:] = _f64(a, n)


def _session_stream(s: Session, stream):
    """The stream handle for a host tick; the last stream object's handle is kept,
    so a loop on one stream converts it once."""
    if stream is not None and stream is s._stream_key:
        return s._stream_arg
    arg = _stream(stream)
    if stream is not None:
        s._stream_key, s._stream_arg = stream, arg
    return arg


def _outcome(s: Session) -> dict:
    r = s._result
    return dict(u_r=s._u_r[:s.nu].copy(), index=r.index, status=r.status, n_safe=r.n_safe,
                ttv=r.ttv, cost=r.cost, n_slots=r.n_slots, executed_steps=r.executed_steps,
                tick=r.tick, flags=r.reserved)


def evaluate_candidates(s: Session, x_t, u_h, candidates=None, tick: int = 0, stream=None):
    """mpmi_evaluate_candidates: queue one tick from host x_t / u_h (float64)."""
    _stage(s._in_x, x_t, s.nx)
    _stage(s._in_u, u_h, s.nu)
    rc = s.ctx.lib.mpmi_evaluate_candidates(s.handle, s._x_ptr, s._u_ptr,
                                            _ptr(candidates), tick, _session_stream(s, stream))
    if rc:
        _check(rc)


def select_input(s: Session) -> dict:
    """mpmi_select_input: wait for the queued tick and return its outcome."""
    rc = s.ctx.lib.mpmi_select_input(s.handle, s._result_ptr)
    if rc:
        _check(rc)
    return _outcome(s)


def evaluate_candidates_device(s: Session, x_t_dev, u_h_dev, result_dev, candidates=None,
                               tick: int = 0, ttv_dev=None, cost_dev=None, stream=None):
    """mpmi_evaluate_candidates_device: device-resident tick (torch tensors)."""
    _check(s.ctx.lib.mpmi_evaluate_candidates_device(
        s.handle, _ptr(x_t_dev), _ptr(u_h_dev), _ptr(candidates), tick, _ptr(result_dev),
        _ptr(ttv_dev), _ptr(cost_dev), _stream(stream)))


def sample_candidates(s: Session, out_dev, u_h_dev=None, candidates=None, tick: int = 0,
                      stream=None):
    """mpmi_sample_candidates: the tick's candidate values in slot order."""
    _check(s.ctx.lib.mpmi_sample_candidates(s.handle, _ptr(u_h_dev), _ptr(candidates), tick,
                                            _ptr(out_dev), _stream(stream)))


def debug_philox(records_dev, words_dev, stream=None):
    """mpmi_debug_philox: raw Philox4x32-10 words of the device generator.
    records_dev: int32/uint32 CUDA tensor (n, 6) = c0 c1 c2 c3 k0 k1;
    words_dev: (n, 4) of the same 4-byte type."""
    import torch
    n = records_dev.shape[0]
    _require(records_dev, "records_dev", 4, 6 * n)
    _require(words_dev, "words_dev", 4, 4 * n)
    _check(load().mpmi_debug_philox(_ptr(records_dev), n, _ptr(words_dev), _stream(stream)))


def debug_trajectories(s: Session, x_t_dev, u_h_dev, result_dev, traj_dev, candidates=None,
                       tick: int = 0, ttv_dev=None, cost_dev=None, stream=None):
    """mpmi_debug_trajectories: a tick that also records every predicted z_t."""
    _check(s.ctx.lib.mpmi_debug_trajectories(
        s.handle, _ptr(x_t_dev), _ptr(u_h_dev), _ptr(candidates), tick, _ptr(result_dev),
        _ptr(ttv_dev), _ptr(cost_dev), _ptr(traj_dev), _stream(stream)))


def evaluate_candidates_noalloc(basis: str, K_dev, lo, hi, n_samples: int, horizon: int,
                                input_lo, input_hi, x_t_dev, u_h_dev, result_dev,
                                inflation: float = 0.0, include_user: bool = True,
                                sampler: str = "uniform", seed: int = 0, stream_id: int = 0,
                                lanes: int = 0, block: int = 0, candidates=None, tick: int = 0,
                                nx: int | None = None, nu: int | None = None, stream=None):
    """mpmi_evaluate_candidates_noalloc: one tick from caller-owned device buffers
    only (K, x_t, u_h, result); the library allocates nothing for it."""
    lib = load()
    d = _desc(basis, nx, nu)
    spec = SafetySpecC()
    lo, hi = _f64(lo), _f64(hi)
    for j in range(MAX_NX):
        spec.state_lo[j] = lo[j] if j < lo.size else -np.inf
        spec.state_hi[j] = hi[j] if j < hi.size else np.inf
    spec.inflation = inflation
    cfg = SessionConfig()
    cfg.n_samples, cfg.horizon = n_samples, horizon
    cfg.include_user = int(include_user)
    cfg.sampler = SAMPLER[sampler]
    ilo, ihi = _f64(input_lo), _f64(input_hi)
    for j in range(MAX_NU):
        cfg.input_lo[j] = ilo[j] if j < ilo.size else 0.0
        cfg.input_hi[j] = ihi[j] if j < ihi.size else 1.0
    cfg.seed, cfg.stream_id, cfg.lanes, cfg.block = seed, stream_id, lanes, block
    import torch
    n = BASIS_SIZE[basis] if basis in BASIS_SIZE else d.nx + d.nu
    _require(K_dev, "K_dev", 4, n * n, torch.float32)
    if K_dev.numel() != n * n:
        raise ValueError(f"K_dev: expected {n} x {n} values, got {K_dev.numel()}")
    _require(x_t_dev, "x_t_dev", 8, d.nx, torch.float64)
    _require(u_h_dev, "u_h_dev", 8, d.nu, torch.float64)
    _require(result_dev, "result_dev", result_dev.element_size(),
             -(-RESULT_BYTES // result_dev.element_size()))
    if candidates is not None:
        _require(candidates, "candidates", 4, n_samples * d.nu, torch.float32)
    _check(lib.mpmi_evaluate_candidates_noalloc(
        ctypes.byref(d), _ptr(K_dev), ctypes.byref(spec), ctypes.byref(cfg), _ptr(x_t_dev),
        _ptr(u_h_dev), _ptr(candidates), tick, _ptr(result_dev), _stream(stream)))


# ---------------------------------------------------------------- learned screener
SCREENER_PARAMS = 18305
SCREENER_KEYS = (("W1", (128, 12)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
                 ("w3", (128,)), ("b3", ()))


def pack_weights(w: dict) -> np.ndarray:
    """Packed float32 weight vector (W1, b1, W2, b2, w3, b3) from a dict."""
    return np.ascontiguousarray(np.concatenate(
        [np.asarray(w[k], dtype=np.float32).reshape(-1) for k, _ in SCREENER_KEYS]))


def unpack_weights(v) -> dict:
    v = np.asarray(v, dtype=np.float64)
    out, o = {}, 0
    for k, shape in SCREENER_KEYS:
        n = int(np.prod(shape)) if shape else 1
        out[k] = v[o:o + n].reshape(shape) if shape else np.array(v[o])
        o += n
    return out


class Screener:
    """mpmi_screener_create: learned candidate screener for a race-car model."""

    def __init__(self, ctx: Context, model: Model, weights: dict, max_batch: int = 8192,
                 max_slots: int = 65537):
        self.ctx, self.model = ctx, model
        w = pack_weights(weights)
        h = c_vp()
        _check(ctx.lib.mpmi_screener_create(ctx.handle, model.handle, w.ctypes.data, max_batch,
                                            max_slots, ctypes.byref(h)))
        self.handle = h

    def get_weights(self) -> dict:
        v = np.empty(SCREENER_PARAMS, dtype=np.float32)
        _check(self.ctx.lib.mpmi_screener_get_weights(self.handle, v.ctypes.data))
        return unpack_weights(v)

    def set_weights(self, weights: dict):
        w = pack_weights(weights)
        _check(self.ctx.lib.mpmi_screener_set_weights(self.handle, w.ctypes.data))

    def tick_features(self, x_t_dev, out_dev, stream=None):
        """12 floats: the 10 per-tick inputs, the nearest segment, its distance."""
        _check(self.ctx.lib.mpmi_screener_tick_features(self.handle, _ptr(x_t_dev), _ptr(out_dev),
                                                        _stream(stream)))

    def features(self, session: Session, x_t_dev, u_h_dev, out_dev, tick: int = 0, stream=None):
        _check(self.ctx.lib.mpmi_screener_features(self.handle, session.handle, _ptr(x_t_dev),
                                                   _ptr(u_h_dev), tick, _ptr(out_dev),
                                                   _stream(stream)))

    def gradients(self, feats_dev, targets_dev, grad_dev, loss_dev, stream=None):
        _check(self.ctx.lib.mpmi_screener_gradients(self.handle, _ptr(feats_dev),
                                                    _ptr(targets_dev), feats_dev.shape[0],
                                                    _ptr(grad_dev), _ptr(loss_dev),
                                                    _stream(stream)))

    def train_step(self, feats_dev, targets_dev, loss_dev, lr: float = 1e-3, stream=None):
        _check(self.ctx.lib.mpmi_screener_train_step(self.handle, _ptr(feats_dev),
                                                     _ptr(targets_dev), feats_dev.shape[0], lr,
                                                     _ptr(loss_dev), _stream(stream)))

    def score(self, feats_dev, scores_dev, stream=None):
        _check(self.ctx.lib.mpmi_screener_score(self.handle, _ptr(feats_dev), feats_dev.shape[0],
                                                _ptr(scores_dev), _stream(stream)))

    def set_timing(self, on: bool):
        """mpmi_screener_set_timing: record CUDA events around a screened tick's launches."""
        _check(self.ctx.lib.mpmi_screener_set_timing(self.handle, int(on)))

    def phase_times(self) -> dict:
        """mpmi_screener_phase_times: the last screened tick's launch durations (ms)."""
        out = (ctypes.c_float * 4)()
        _check(self.ctx.lib.mpmi_screener_phase_times(self.handle, out))
        return dict(screen=out[0], compact=out[1], rollout=out[2], fallback=out[3])

    def free(self):
        if self.handle:
            self.ctx.lib.mpmi_screener_free(self.handle)
            self.handle = None


def evaluate_screened(s: Session, scr: Screener, x_t_dev, u_h_dev, result_dev, k: int = 4096,
                      tau: float = 0.9, m: int = 8, tick: int = 0, list_dev=None,
                      n_list_dev=None, stream=None):
    """mpmi_evaluate_screened: exact screened tick (a cost-order prefix of at least
    k slots holding at least m predicted-safe ones when tau > 0) with on-device
    fallback to the full evaluation."""
    _check(s.ctx.lib.mpmi_evaluate_screened(s.handle, scr.handle, _ptr(x_t_dev), _ptr(u_h_dev),
                                            tick, k, tau, m, _ptr(result_dev), _ptr(list_dev),
                                            _ptr(n_list_dev), _stream(stream)))


def evaluate_screened_host(s: Session, scr: Screener, x_t, u_h, k: int = 4096, tau: float = 0.9,
                           m: int = 8, tick: int = 0, stream=None):
    """mpmi_evaluate_screened_host: the screened tick from host x_t / u_h (float64),
    queued; collect it with select_input."""
    _stage(s._in_x, x_t, s.nx)
    _stage(s._in_u, u_h, s.nu)
    rc = s.ctx.lib.mpmi_evaluate_screened_host(s.handle, scr.handle, s._x_ptr, s._u_ptr, tick,
                                               k, tau, m, _session_stream(s, stream))
    if rc:
        _check(rc)


# ---------------------------------------------------------------- continuous-batching server
class Server:
    """mpmi_server_create: many sessions of one model served in batched launches."""

    def __init__(self, ctx: Context, model: Model, max_sessions: int = 256):
        self.ctx, self.model, self.max_sessions = ctx, model, max_sessions
        self.nx, self.nu = model.nx, model.nu
        h = c_vp()
        _check(ctx.lib.mpmi_server_create(ctx.handle, model.handle, max_sessions, ctypes.byref(h)))
        self.handle = h
        self._res = (Result * max_sessions)()
        self._slots = np.zeros(max_sessions, dtype=np.int32)

    def admit(self, n_samples: int, horizon: int, input_lo, input_hi, seed: int = 0,
              stream_id: int = 0, include_user: bool = True) -> int:
        cfg = SessionConfig()
        cfg.n_samples, cfg.horizon = n_samples, horizon
        cfg.include_user = int(include_user)
        cfg.sampler = SAMPLER["uniform"]
        lo, hi = _f64(input_lo), _f64(input_hi)
        for j in range(MAX_NU):
            cfg.input_lo[j] = lo[j] if j < lo.size else 0.0
            cfg.input_hi[j] = hi[j] if j < hi.size else 1.0
        cfg.seed, cfg.stream_id = seed, stream_id
        slot = c_i32()
        _check(self.ctx.lib.mpmi_server_admit(self.handle, ctypes.byref(cfg), ctypes.byref(slot)))
        return slot.value

    def release(self, slot: int):
        _check(self.ctx.lib.mpmi_server_release(self.handle, slot))

    def submit(self, slots, x_t, u_h, ticks):
        slots = np.ascontiguousarray(np.asarray(slots, dtype=np.int32))
        n = slots.size
        x = _f64(x_t).reshape(n, self.nx)
        u = _f64(u_h).reshape(n, self.nu)
        t = np.ascontiguousarray(np.asarray(ticks, dtype=np.uint64))
        _check(self.ctx.lib.mpmi_server_submit(self.handle, n, slots.ctypes.data, x.ctypes.data,
                                               u.ctypes.data, t.ctypes.data))

    def staged(self) -> int:
        n = c_i32()
        _check(self.ctx.lib.mpmi_server_staged(self.handle, ctypes.byref(n)))
        return n.value

    def launch(self, stream=None) -> int:
        n = c_i32()
        _check(self.ctx.lib.mpmi_server_launch(self.handle, _stream(stream), ctypes.byref(n)))
        return n.value

    def poll(self) -> bool:
        """True when a batch in flight has finished."""
        d = c_i32()
        _check(self.ctx.lib.mpmi_server_poll(self.handle, ctypes.byref(d)))
        return bool(d.value)

    def set_max_in_flight(self, n: int):
        """mpmi_server_set_max_in_flight: batches allowed on the GPU at once (1..4)."""
        _check(self.ctx.lib.mpmi_server_set_max_in_flight(self.handle, int(n)))

    def in_flight(self) -> int:
        n = c_i32()
        _check(self.ctx.lib.mpmi_server_in_flight(self.handle, ctypes.byref(n)))
        return n.value

    def collect(self):
        """[(slot, result dict), ...] of one batch in flight: the earliest launched
        of the finished ones, else the earliest launched (waits for it)."""
        n = c_i32()
        _check(self.ctx.lib.mpmi_server_collect(self.handle, self._res, self._slots.ctypes.data,
                                                ctypes.byref(n)))
        return [(int(self._slots[i]), result_dict(self._res[i], self.nu)) for i in range(n.value)]

    def tune(self, requests, x_t, u_h, reps: int = 10) -> dict:
        """mpmi_server_tune: pick the fastest launch shape for a request mix.
        requests: [(n_samples, horizon, input_lo, input_hi, seed, stream_id), ...];
        x_t (n x nx), u_h (n x nu)."""
        n = len(requests)
        cfgs = (SessionConfig * n)()
        for i, (ns, hz, lo, hi, seed, sid) in enumerate(requests):
            cfgs[i] = _session_config(ns, hz, lo, hi, True, "uniform", seed, sid)
        x = _f64(x_t).reshape(n, self.nx)
        u = _f64(u_h).reshape(n, self.nu)
        r = TuneResult()
        _check(self.ctx.lib.mpmi_server_tune(self.handle, n, cfgs, x.ctypes.data, u.ctypes.data,
                                             int(reps), ctypes.byref(r)))
        return dict(lanes=r.lanes, cands=r.cands, block=r.block, n_tried=r.n_tried, us=r.us,
                    default_us=r.default_us)

    def free(self):
        if self.handle:
            self.ctx.lib.mpmi_server_free(self.handle)
            self.handle = None
