"""Planted mistakes in the oracle, on the CPU: each plausible slip -- a wrong
constant, multiplier or word in the generator, a dropped factor, a swapped or
dropped feature, a transposed operand, an off-by-one count, a closed instead of
an open bound, a missing clamp, the wrong tie or fallback order, another norm
-- is written into a copy of the oracle package, and the pins (the tests of
test_oracle_pins.py and test_oracle_noise.py, run against the copy) must fail
on it; the same for the learned screener's oracle (test_oracle_screener.py) and the
sparsity-promoting basis selection (test_oracle_sparse.py).
So the pins, not the oracle's agreement with itself, stand behind the parity
tests."""
import importlib
import os
import shutil
import sys

import pytest

import test_oracle_noise
import test_oracle_pins
import test_oracle_screener
import test_oracle_sparse

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")

# (name, file, text, replacement): the text occurs exactly once in the file
MUTANTS = [
    ("philox nine rounds", "philox.py", "ROUNDS = 10", "ROUNDS = 9"),
    ("philox key schedule constant", "philox.py", "W0 = 0x9E3779B9\nW1", "W0 = 0x9E3779B1\nW1"),
    ("philox multiplier", "philox.py", "hi0, lo0 = mulhilo32(M0, c0)",
     "hi0, lo0 = mulhilo32(M1, c0)"),
    ("philox round word order", "philox.py", "(hi1 ^ c1 ^ np.uint32(k0), lo1,",
     "(hi1 ^ c3 ^ np.uint32(k0), lo1,"),
    ("uniform word shift", "sampling.py",
     "u = (words[j] >> np.uint32(8)).astype(np.float32) * TWO_M24",
     "u = (words[j] >> np.uint32(9)).astype(np.float32) * TWO_M24"),
    ("grid cell edge instead of midpoint", "sampling.py",
     "v = ((digit + 0.5) * (hi[j] - lo[j])) / g + lo[j]",
     "v = (digit * (hi[j] - lo[j])) / g + lo[j]"),
    ("Box-Muller angle without the factor 2", "sampling.py",
     "return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)",
     "return r * np.cos(np.pi * u2), r * np.sin(np.pi * u2)"),
    ("noise step in the wrong counter word", "sampling.py",
     "c2 = np.uint32(((tick >> 32) & 0xFFFF) + (int(step) << 16) + (int(block) << 25))",
     "c2 = np.uint32(((tick >> 32) & 0xFFFF) + (int(step) << 17) + (int(block) << 25))"),
    ("bot sine and cosine swapped", "basis.py", "s, c = np.sin(th), np.cos(th)",
     "s, c = np.cos(th), np.sin(th)"),
    ("car feature product", "basis.py", "om * c, om * s, vx * vy, d * d,",
     "om * c, om * s, vx * vy, d * a,"),
    ("fit returns the transposed operator", "fit.py", "K = kt.T.copy()", "K = kt.copy()"),
    ("held feature as a column", "fit.py",
     "for j in held_features(basis, nx, nu):\n        K[j] = np.eye(n)[j]",
     "for j in held_features(basis, nx, nu):\n        K[:, j] = np.eye(n)[j]"),
    ("rollout with the transposed operator", "mpmi.py", "zn = z[idx] @ K.T", "zn = z[idx] @ K"),
    ("ttv one short", "mpmi.py", "ttv[idx[ok]] = t", "ttv[idx[ok]] = t - 1"),
    ("ties to the highest slot", "mpmi.py", "order = np.lexsort((slot, cost, H - ttv))",
     "order = np.lexsort((-slot, cost, H - ttv))"),
    ("fallback to the shortest survivor", "mpmi.py",
     "order = np.lexsort((slot, cost, H - ttv))", "order = np.lexsort((slot, cost, ttv))"),
    ("cost as the 1-norm", "mpmi.py", "cost = np.sum((cands - u_h[None, :]) ** 2, axis=1)",
     "cost = np.sum(np.abs(cands - u_h[None, :]), axis=1)"),
    ("closed box bounds", "safety.py", "ok = np.all((x > lo) & (x < hi), axis=1)",
     "ok = np.all((x >= lo) & (x <= hi), axis=1)"),
    ("inflation widens the box", "safety.py",
     "    hi = np.asarray(spec.hi, dtype=np.float64) - spec.inflation\n    ok =",
     "    hi = np.asarray(spec.hi, dtype=np.float64) + spec.inflation\n    ok ="),
    ("projection onto the segment not clamped", "safety.py",
     "t = np.clip((rx * dx + ry * dy) * inv, 0.0, 1.0)  # clamped projection",
     "t = (rx * dx + ry * dy) * inv"),
    ("road without the inflation", "safety.py",
     "ok &= d < (spec.half_width - spec.inflation)", "ok &= d < spec.half_width"),
    # the learned screener's oracle (features, network, training, screening rule)
    ("curvature sign", "screener.py", "cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]",
     "cross = a[:, 1] * b[:, 0] - a[:, 0] * b[:, 1]"),
    ("look-ahead one vertex short", "screener.py", "out[i, m] = kappa[j % S]",
     "out[i, m] = kappa[(j - 1) % S]"),
    ("lateral offset sign", "screener.py", "nrm = np.array([-tau[1], tau[0]])",
     "nrm = np.array([tau[1], -tau[0]])"),
    ("heading error sign", "screener.py", "e_psi = x[2] - math.atan2(tau[1], tau[0])",
     "e_psi = math.atan2(tau[1], tau[0]) - x[2]"),
    ("GELU cubic coefficient", "screener.py", "GELU_A = 0.044715", "GELU_A = 0.04715"),
    ("GELU derivative without the factor 3", "screener.py",
     "(1.0 + 3.0 * GELU_A * z * z)", "(1.0 + GELU_A * z * z)"),
    ("loss gradient sign", "screener.py", "d3 = (2.0 / B) * (y - target) * y * (1.0 - y)",
     "d3 = (2.0 / B) * (target - y) * y * (1.0 - y)"),
    ("transposed weight gradient", "screener.py", 'g["W2"] = d2.T @ cache["h1"]',
     'g["W2"] = cache["h1"].T @ d2'),
    ("Adam without bias correction", "screener.py", "mh = m / (1 - beta1 ** step)", "mh = m"),
    ("Adam without the square root", "screener.py",
     "params[k] - lr * mh / (np.sqrt(vh) + eps)", "params[k] - lr * mh / (vh + eps)"),
    ("screen prefix one slot too long", "screener.py", "if inside.sum() >= k and",
     "if inside.sum() > k and"),
    ("predicted-safe count outside the prefix", "screener.py",
     "np.count_nonzero(inside & safe) >= m", "np.count_nonzero(safe) >= m"),
    ("screened fallback order", "screener.py",
     "return int(np.lexsort((slot, cost, H - np.asarray(ttv)))[0])",
     "return int(np.lexsort((slot, cost, np.asarray(ttv)))[0])"),
    # the sparsity-promoting basis selection (group lasso by ADMM, then polishing)
    ("group threshold halved", "fit.py", "shrink = 1.0 - (gamma / rho) / norms[j]",
     "shrink = 1.0 - (gamma / (2.0 * rho)) / norms[j]"),
    ("ADMM dual update sign", "fit.py", "U = U + V - Z", "U = U - V + Z"),
    ("data term without its factor 2", "fit.py",
     "G = 2.0 / m * (A.T @ A) + rho * np.eye(n)", "G = 1.0 / m * (A.T @ A) + rho * np.eye(n)"),
    ("no polishing refit", "fit.py", "Ws, *_ = np.linalg.lstsq(X[:, cols], Y, rcond=None)",
     "Ws = Z[cols] * rms_scale(Y)[None, :] / rms_scale(X)[cols][:, None]"),
]

PIN_MODULES = (test_oracle_pins, test_oracle_noise, test_oracle_screener, test_oracle_sparse)
PARAMS = {"test_philox_avalanche": [("counter",), ("key",)],
          "test_fit_held_input_rows_are_unit_rows": [("bot", (4, 11)),
                                                     ("car", (6, 7, 30, 31))],
          "test_brute_force_tiny": [("bot",), ("car",)],
          "test_planted_support_and_exact_polish": [(1e-3,), (1e-2,), (0.05,)],
          "test_group_lasso_optimality_conditions": [(0.02,), (0.2,)]}


def _pins(first=None):
    """Every pin; those of module `first` (the one that tests the edited file) first."""
    for mod in sorted(PIN_MODULES, key=lambda m: m is not first):
        for name, fn in list(vars(mod).items()):
            if name.startswith("test_") and callable(fn):
                for args in PARAMS.get(name, [()]):
                    yield mod, name, fn, args


def test_every_parametrised_pin_is_covered():
    for mod in PIN_MODULES:
        for name, fn in vars(mod).items():
            marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
            if name.startswith("test_") and marks:
                assert name in PARAMS, name


def _mutant_package(tmp_path, file, text, replacement):
    """A copy of the oracle package under a fresh name with one edit; returns its
    submodules by their names in the original package."""
    pkg = f"oracle_mut_{len(os.listdir(tmp_path))}"
    dst = tmp_path / pkg
    shutil.copytree(ORACLE, dst, ignore=shutil.ignore_patterns("__pycache__"))
    src = (dst / file).read_text()
    assert src.count(text) == 1, (file, text)
    (dst / file).write_text(src.replace(text, replacement))
    sys.path.insert(0, str(tmp_path))
    try:
        importlib.invalidate_caches()
        mods = {n: importlib.import_module(f"{pkg}.{n}")
                for n in ("philox", "sampling", "basis", "fit", "safety", "mpmi", "screener")}
    finally:
        sys.path.remove(str(tmp_path))
    return pkg, mods


def _failing_pins(tmp_path, monkeypatch, file, text, replacement, first_only):
    """Runs the pins against the copy with one edit; returns the failures."""
    pkg, mods = _mutant_package(tmp_path, file, text, replacement)
    try:
        for mod in PIN_MODULES:
            for attr, val in list(vars(mod).items()):
                sub = getattr(val, "__name__", "").split(".", 1)
                if len(sub) == 2 and sub[0] == "oracle" and sub[1] in mods:
                    monkeypatch.setattr(mod, attr, mods[sub[1]])
        failed = []
        first = {"screener.py": test_oracle_screener, "fit.py": test_oracle_sparse}.get(file)
        for mod, pin, fn, args in _pins(first):
            try:
                fn(*args)
            except Exception as e:  # noqa: BLE001 -- any failure of a pin counts
                failed.append(f"{pin}{args}: {type(e).__name__}")
                if first_only:
                    break
        return failed
    finally:
        for m in [m for m in sys.modules if m == pkg or m.startswith(pkg + ".")]:
            del sys.modules[m]


def test_copy_with_a_harmless_edit_passes_every_pin(tmp_path, monkeypatch):
    # the harness itself: a copy whose only change is a comment fails no pin
    assert _failing_pins(tmp_path, monkeypatch, "mpmi.py", "SAFE = 0\n",
                         "SAFE = 0  # the same value\n", first_only=False) == []


@pytest.mark.parametrize("name,file,text,replacement", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name, file, text, replacement):
    failed = _failing_pins(tmp_path, monkeypatch, file, text, replacement, first_only=True)
    assert failed, f"no pin fails with the planted mistake: {name}"
