"""The C ABI used from plain C: tests/c_client/closed_loop.c, compiled with the
host C compiler against include/mpmi.h and linked with libmpmi.so, gives the same
fit (host only) and the same ticks (on a GPU) as the Python binding, bit for bit."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from workloads import data, plants

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def lib():
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


@pytest.fixture(scope="module")
def client(lib, tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    libdir = os.path.dirname(lib.LIB_PATH)
    out = str(tmp_path_factory.mktemp("c_client") / "closed_loop")
    cmd = [cc, "-std=c11", "-O2", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
           os.path.join(HERE, "c_client", "closed_loop.c"), f"-L{libdir}", "-lmpmi",
           f"-Wl,-rpath,{libdir}", "-lm", "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _inputs(path, x, u, xn, ticks=None):
    with open(path, "wb") as f:
        f.write(struct.pack("<q", len(x)))
        for a in (x, u, xn):
            f.write(np.ascontiguousarray(a, dtype="<f8").tobytes())
        if ticks is not None:
            n, H, seed, states, uhs = ticks
            f.write(struct.pack("<iiQi", n, H, seed, len(states)))
            for s, uh in zip(states, uhs):
                f.write(np.asarray(s, dtype="<f8").tobytes())
                f.write(np.asarray([uh], dtype="<f8").tobytes())


def test_c_client_fit_matches_binding(lib, client, tmp_path):
    x, u, xn = data.transitions("bot", 1, 2000)
    p = str(tmp_path / "in.bin")
    _inputs(p, x, u, xn)
    r = subprocess.run([client, "fit", p], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    K = np.zeros((12, 12))
    residual = None
    for line in r.stdout.splitlines():
        w = line.split()
        if w[0] == "K":
            K[int(w[1]), int(w[2])] = float(w[3])
        elif w[0] == "residual":
            residual = float(w[1])
    K_py, res_py = lib.fit_operator("bot", x, u, xn)
    assert np.array_equal(K, K_py) and residual == res_py


def test_c_client_reports_errors(client, tmp_path):
    p = str(tmp_path / "bad.bin")
    with open(p, "wb") as f:
        f.write(struct.pack("<q", 0))
    r = subprocess.run([client, "fit", p], capture_output=True, text=True, timeout=60)
    assert r.returncode == 1 and "transition count" in r.stderr
    r = subprocess.run([client], capture_output=True, text=True, timeout=60)
    assert r.returncode == 1 and "usage" in r.stderr


@pytest.mark.gpu
def test_c_client_ticks_match_binding(lib, client, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x, u, xn = data.transitions("bot", 1, 5000)
    N, H, seed, T = 4096, 40, 5, 20
    states = data.states_in_box(9, T, [-0.2, -0.8, -1.0, -0.8], [0.2, 0.8, 1.0, 0.8])
    uhs = data.to_f32_exact(data.ou_user_input(9, T, plants.BOT_DT, plants.BOT_INPUT_LO,
                                               plants.BOT_INPUT_HI)).reshape(T)
    p = str(tmp_path / "in.bin")
    _inputs(p, x, u, xn, (N, H, seed, states, uhs))
    r = subprocess.run([client, "ticks", p, "0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    got = [line.split() for line in r.stdout.splitlines() if line.startswith("tick ")]
    assert len(got) == T
    ctx = lib.Context(0)
    model, _ = lib.fit_model(ctx, "bot", x, u, xn)
    lib.set_safety_set(model, data.BOT_SAFE_LO, data.BOT_SAFE_HI)
    sess = lib.Session(ctx, model, N, H, plants.BOT_INPUT_LO, plants.BOT_INPUT_HI, seed=seed)
    try:
        for t in range(T):
            lib.evaluate_candidates(sess, states[t], [uhs[t]], tick=t)
            want = lib.select_input(sess)
            w = got[t]
            assert int(w[1]) == t
            assert (int(w[2]), int(w[3]), int(w[4]), int(w[5])) == \
                (want["index"], want["status"], want["n_safe"], want["ttv"]), t
            assert float(w[6]) == want["u_r"][0]
            assert int(w[7]) == int(np.float32(want["cost"]).view(np.uint32))
            assert int(w[8]) == want["executed_steps"]
    finally:
        sess.close()
        model.free()
