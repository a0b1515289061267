"""The C-ABI library builds, loads and exports every symbol include/mpmi.h
declares; its host-only fit agrees with the oracle (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import fit as ofit
from workloads import data, plants


@pytest.fixture(scope="module")
def lib(repo_root):
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


def _declared_functions(repo_root):
    text = open(os.path.join(repo_root, "include", "mpmi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpmi_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib, repo_root):
    names = _declared_functions(repo_root)
    assert len(names) >= 18
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # the binding wraps every declared entry point
    assert set(names) <= set(lib._SIGNATURES)


def test_struct_layouts_match_header(lib):
    assert ctypes.sizeof(lib.Result) == 80
    assert ctypes.sizeof(lib.SafetySpecC) == 168
    assert ctypes.sizeof(lib.SessionConfig) == 104
    assert lib.load().mpmi_version().decode().startswith("mpmi-gb300")


@pytest.mark.parametrize("kind,seed,m", [("bot", 1, 5000), ("car", 3, 20000)])
def test_host_fit_matches_oracle(lib, kind, seed, m):
    x, u, xn = data.transitions(kind, seed, m)
    K, res = lib.fit_operator(kind, x, u, xn)
    Ko, reso = ofit.fit_koopman(kind, x, u, xn)
    scale = np.abs(Ko).max()
    assert np.abs(K - Ko).max() <= 1e-9 * scale
    assert abs(res - reso) <= 1e-9
    held = (4, 11) if kind == "bot" else (6, 7, 30, 31)
    for r in held:
        assert np.array_equal(K[r], np.eye(K.shape[0])[r])


def test_host_fit_linear_closed_form(lib):
    rng = np.random.default_rng(0)
    A = np.eye(4) + 0.1 * rng.standard_normal((4, 4))
    B = rng.standard_normal((4, 1))
    x = rng.standard_normal((300, 4))
    u = rng.uniform(-1, 1, (300, 1))
    K, res = lib.fit_operator("linear", x, u, plants.linear_step(A, B, x, u), nx=4, nu=1)
    want = np.block([[A, B], [np.zeros((1, 4)), np.eye(1)]])
    assert np.abs(K - want).max() < 1e-10 and res < 1e-12


def test_host_fit_errors(lib):
    x, u, xn = data.transitions("bot", 1, 50)
    with pytest.raises(lib.MpmiError) as e:
        lib.fit_operator("bot", x[:5], u[:5], xn[:5])
    assert e.value.code == -1
    x2 = x.copy()
    x2[3, 1] = np.nan
    with pytest.raises(lib.MpmiError) as e:
        lib.fit_operator("bot", x2, u, xn)
    assert e.value.code == -3
    with pytest.raises(lib.MpmiError) as e:
        lib.fit_operator("linear", x[:, :3], u, xn[:, :3], nx=3, nu=1)
    assert e.value.code == -6
    # rank deficient: a constant state makes several features collinear
    xc = np.zeros((50, 4))
    with pytest.raises(lib.MpmiError) as e:
        lib.fit_operator("bot", xc, u, xc)
    assert e.value.code == -1


def test_context_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.MpmiError) as e:
        lib.Context(0)
    assert e.value.code in (-1, -4)


def test_missing_library_raises(lib, tmp_path):
    with pytest.raises(RuntimeError):
        lib.load(str(tmp_path / "nope.so"))


@pytest.mark.parametrize("kind,seed,m,gamma", [("bot", 1, 5000, 0.02), ("bot", 1, 5000, 1.0),
                                               ("car", 3, 20000, 1.0), ("car", 3, 20000, 0.0)])
def test_host_sparse_fit_matches_oracle(lib, kind, seed, m, gamma):
    """Sparsity-promoting basis selection: the host float64 implementation selects
    the oracle's support and refits the same K."""
    x, u, xn = data.transitions(kind, seed, m)
    K, sup, res = lib.fit_operator_sparse(kind, x, u, xn, gamma)
    Ko, supo, reso = ofit.fit_koopman_sparse(kind, x, u, xn, gamma)
    assert sup.tolist() == supo.tolist()
    assert np.abs(K - Ko).max() <= 1e-9 * np.abs(Ko).max()
    assert abs(res - reso) <= 1e-9
    if gamma > 0:
        assert 0 < sup.sum() < K.shape[0]
    assert not K[:, ~sup].any() and not K[~sup].any()


def test_host_sparse_fit_errors(lib):
    x, u, xn = data.transitions("bot", 1, 200)
    for kw, code in ((dict(gamma=-1.0), -1), (dict(gamma=np.nan), -1), (dict(gamma=0.1, rho=0.0), -1),
                     (dict(gamma=0.1, iters=0), -1)):
        with pytest.raises(lib.MpmiError) as e:
            lib.fit_operator_sparse("bot", x, u, xn, **kw)
        assert e.value.code == code


def test_noalloc_refuses_misaligned_buffers_before_any_cuda_call(lib):
    """mpmi_evaluate_candidates_noalloc reads K as float4 in its register-resident
    shapes: a K pointer that is not 16-byte aligned (a view such as buf[1:]) is
    refused on the host.  The pointers below are never dereferenced: the check
    comes before any CUDA call, so this runs without a GPU."""
    so = lib.load()
    d = lib.BasisDesc(lib.BASIS["bot"], 4, 1)
    spec = lib.SafetySpecC()
    for j in range(lib.MAX_NX):
        spec.state_lo[j], spec.state_hi[j] = -1.0, 1.0
    cfg = lib.SessionConfig()
    cfg.n_samples, cfg.horizon, cfg.include_user = 1024, 20, 1
    cfg.input_lo[0], cfg.input_hi[0] = -1.0, 1.0
    base = 0x7f0000000000
    ok8, ok16 = base + 0x100, base + 0x200

    def call(K, xt=ok8, uh=ok8, res=ok8, cand=None):
        return so.mpmi_evaluate_candidates_noalloc(
            ctypes.byref(d), ctypes.c_void_p(K), ctypes.byref(spec), ctypes.byref(cfg),
            ctypes.c_void_p(xt), ctypes.c_void_p(uh),
            None if cand is None else ctypes.c_void_p(cand), 0, ctypes.c_void_p(res), None)

    for off in (4, 8, 12):
        assert call(ok16 + off) == -1
        assert "16-byte" in so.mpmi_last_error().decode()
    assert call(ok16, xt=ok8 + 4) == -1 and "8-byte" in so.mpmi_last_error().decode()
    assert call(ok16, res=ok8 + 4) == -1 and "8-byte" in so.mpmi_last_error().decode()
    assert call(ok16, cand=ok8 + 2) == -1 and "4-byte" in so.mpmi_last_error().decode()
