"""The bounded wait on the bulk-copy staging of shared memory (through the C
ABI): a tick whose copies are withheld (test hook) comes back flagged
MPMI_TIMEOUT after about a second per wait instead of hanging, the context stays
usable, and the next normal tick is unaffected."""
import time

import numpy as np
import pytest

from workloads import data

from parity import car_env, gpu_model, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


@pytest.mark.parametrize("rollout", ["full", "factored"])
def test_withheld_staging_times_out_and_recovers(lib, rollout):
    ctx = lib.Context(0)
    env = car_env()
    model = gpu_model(lib, ctx, env)
    x_t = data.car_start_state(env.track, vx=14.0)
    u_h = data.to_f32_exact(data.user_input_once(5, env.lo, env.hi))
    sess = lib.Session(ctx, model, 3000, 60, env.lo, env.hi, seed=3)
    if rollout == "factored":
        sess.set_rollout("factored")
    want = run_gpu(lib, sess, x_t, u_h, tick=1)
    assert want["result"]["status"] in (lib.SAFE, lib.FALLBACK)
    sess.withhold_staging(True)
    t0 = time.perf_counter()
    got = run_gpu(lib, sess, x_t, u_h, tick=1)
    assert time.perf_counter() - t0 < 30.0
    assert got["result"]["status"] == lib.TIMEOUT
    # host path: select_input reports the timeout as an error code
    lib.evaluate_candidates(sess, x_t, u_h, tick=1)
    with pytest.raises(lib.MpmiError) as e:
        lib.select_input(sess)
    assert e.value.code == -7
    sess.withhold_staging(False)
    again = run_gpu(lib, sess, x_t, u_h, tick=1)
    assert np.array_equal(again["ttv"], want["ttv"])
    for key, v in want["result"].items():
        assert np.array_equal(again["result"][key], v), key
    sess.close()
    model.free()
