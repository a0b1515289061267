"""The no-allocation tick entry point (mpmi_evaluate_candidates_noalloc).

Callers such as hard real-time loops that forbid device allocation after
start-up, or frameworks that own all device memory, pass every buffer
themselves; the library keeps the tick's only scratch in a static device array.
This test drives that entry point through the C ABI and checks that two calls in
a row return exactly what the session-based device entry point returns for the
same ticks, and that a call larger than the static scratch is refused.
"""
import numpy as np
import pytest

from workloads import data, plants

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


def _same(a, b):
    for k in ("index", "status", "n_safe", "ttv", "executed_steps", "n_slots", "tick"):
        assert a[k] == b[k], k
    assert np.array_equal(a["u_r"], b["u_r"])
    assert a["cost"] == b["cost"]


@pytest.mark.parametrize("basis,lanes", [("bot", 1), ("bot", 4), ("car", 1), ("car", 8)])
def test_noalloc_matches_session_path_twice(lib, basis, lanes):
    """The race car runs with its box bounds only (a track needs a preprocessed
    grid, which this entry point does not take); with one lane its K is staged
    in shared memory from the caller's row-major buffer."""
    import torch
    if basis == "bot":
        x, u, xn = data.transitions("bot", 1, 5000)
        safe_lo, safe_hi = data.BOT_SAFE_LO, data.BOT_SAFE_HI
        lo, hi = plants.BOT_INPUT_LO, plants.BOT_INPUT_HI
        states = [np.array([0.05, 0.0, 0.0, 0.0]), np.array([0.3, 0.8, 1.1, 0.5])]
        uhs = [np.array([0.25]), np.array([-0.75])]
        N, H = 16384, 50
    else:
        x, u, xn = data.transitions("car", 3, 20000)
        safe_lo, safe_hi = data.CAR_SAFE_LO, data.CAR_SAFE_HI
        lo, hi = plants.CAR_INPUT_LO, plants.CAR_INPUT_HI
        states = [np.array([0.0, 0.0, 0.3, 18.0, 0.5, 0.1]),
                  np.array([5.0, -3.0, 1.2, 23.0, -0.8, 0.4])]
        uhs = [np.array([0.1, 0.5]), np.array([-0.3, 0.9])]
        N, H = 16384, 60
    nu = len(uhs[0])
    K, _ = lib.fit_operator(basis, x, u, xn)
    ctx = lib.Context(0)
    model = lib.model_from_operator(ctx, basis, K)
    lib.set_safety_set(model, safe_lo, safe_hi)
    seed = 7
    sess = lib.Session(ctx, model, N, H, lo, hi, seed=seed, lanes=lanes)
    dev = torch.device("cuda")
    K_dev = torch.tensor(K, dtype=torch.float32, device=dev)   # caller-owned buffers
    for call, (x_t, u_h) in enumerate(zip(states, uhs)):
        xt = torch.tensor(x_t, dtype=torch.float64, device=dev)
        uh = torch.tensor(u_h, dtype=torch.float64, device=dev)
        ref = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
        out = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
        lib.evaluate_candidates_device(sess, xt, uh, ref, tick=call)
        # 256-thread blocks keep 8 lanes per candidate within the scratch's 1024 blocks
        lib.evaluate_candidates_noalloc(basis, K_dev, safe_lo, safe_hi, N, H,
                                        lo, hi, xt, uh, out, seed=seed, lanes=lanes,
                                        block=256 if lanes >= 8 else 0, tick=call)
        torch.cuda.synchronize()
        _same(lib.result_from_bytes(out.cpu(), nu), lib.result_from_bytes(ref.cpu(), nu))
    sess.close()
    model.free()


def test_noalloc_rejects_calls_beyond_its_scratch(lib):
    import torch
    dev = torch.device("cuda")
    K_dev = torch.eye(12, dtype=torch.float32, device=dev)
    xt = torch.zeros(4, dtype=torch.float64, device=dev)
    uh = torch.zeros(1, dtype=torch.float64, device=dev)
    out = torch.zeros(lib.RESULT_BYTES, dtype=torch.uint8, device=dev)
    # 1024 blocks of 32 threads with one candidate per thread hold 32768 slots
    with pytest.raises(lib.MpmiError) as e:
        lib.evaluate_candidates_noalloc("bot", K_dev, data.BOT_SAFE_LO, data.BOT_SAFE_HI,
                                        40000, 10, [-1.0], [1.0], xt, uh, out, lanes=1,
                                        block=32)
    assert e.value.code == -1 and "1024" in str(e.value)
    lib.evaluate_candidates_noalloc("bot", K_dev, data.BOT_SAFE_LO, data.BOT_SAFE_HI,
                                    32767, 10, [-1.0], [1.0], xt, uh, out, lanes=1, block=32)
    torch.cuda.synchronize()
    r = lib.result_from_bytes(out.cpu(), 1)
    assert r["n_slots"] == 32768 and r["status"] == lib.SAFE and r["index"] == 0
