"""Checkpoint and resume for models, screener weights and sessions.

A model file holds what a model is made of: the basis, the float64 lifted
operator K (Sec. IV-A) and the safety set (Sec. V-C.1).  A model loaded from it
ticks bit for bit like the one saved, because its device copy is K rounded to
float32 from the same float64 values.  A screener file holds the network's float32
parameters.  A session file holds the session's configuration (samples, horizon,
input box, sampler, seed, stream, launch shape, noise, rollout form) and the next
tick number.  Nothing else needs saving: the candidates come from a counter-based
generator keyed by the seed and indexed by slot, tick and stream, so a session
reopened from its file continues the tick stream exactly.

Files are numpy .npz archives of plain arrays (strings as unicode arrays, no
pickled objects), read back with allow_pickle=False.  Every file names its
format; reading checks it.
"""
from __future__ import annotations

import numpy as np

from . import mpmi

FORMAT_MODEL = "mpmi-model-1"
FORMAT_SCREENER = "mpmi-screener-1"
FORMAT_SESSION = "mpmi-session-1"


def write(path: str, record: dict) -> None:
    """Writes a record (string -> str / number / array) as an .npz archive."""
    arrays = {}
    for key, value in record.items():
        if value is None:
            continue
        arrays[key] = np.asarray(value)
        if arrays[key].dtype == object:
            raise TypeError(f"{key}: only plain arrays, numbers and strings are stored")
    with open(path, "wb") as f:
        np.savez(f, **arrays)


def read(path: str, fmt: str) -> dict:
    """Reads a record written by write(); raises ValueError for another format."""
    with np.load(path, allow_pickle=False) as z:
        record = {key: z[key] for key in z.files}
    found = str(record.get("format", ""))
    if found != fmt:
        raise ValueError(f"{path}: format {found!r}, expected {fmt!r}")
    for key, value in record.items():
        if value.ndim == 0:
            record[key] = value.item()
    return record


# ---------------------------------------------------------------- models
def model_record(basis: str, K, nx: int, nu: int, safety: dict | None = None,
                 residual: float | None = None) -> dict:
    """The contents of a model file."""
    rec = dict(format=FORMAT_MODEL, basis=basis, nx=int(nx), nu=int(nu),
               K=np.array(K, dtype=np.float64), residual=residual)
    if safety is not None:
        rec.update(safety_lo=np.asarray(safety["lo"], dtype=np.float64),
                   safety_hi=np.asarray(safety["hi"], dtype=np.float64),
                   inflation=float(safety["inflation"]),
                   half_width=float(safety["half_width"]))
        if safety["track"] is not None:
            rec["track"] = np.asarray(safety["track"], dtype=np.float64)
    return rec


def save_model(path: str, model: mpmi.Model, residual: float | None = None) -> None:
    write(path, model_record(model.basis, model.get_operator(), model.nx, model.nu,
                             model.safety, residual))


def load_model(ctx: mpmi.Context, path: str) -> mpmi.Model:
    """A model (and its safety set, if the file has one) on ctx's device."""
    rec = read(path, FORMAT_MODEL)
    model = mpmi.model_from_operator(ctx, rec["basis"], rec["K"], nx=rec["nx"], nu=rec["nu"])
    if "safety_lo" in rec:
        mpmi.set_safety_set(model, rec["safety_lo"], rec["safety_hi"], rec["inflation"],
                            rec.get("track"), rec["half_width"])
    return model


# ---------------------------------------------------------------- screener
def save_screener(path: str, screener: mpmi.Screener) -> None:
    rec = dict(format=FORMAT_SCREENER)
    rec.update({f"w_{key}": value for key, value in screener.get_weights().items()})
    write(path, rec)


def load_screener_weights(path: str) -> dict:
    """The weights dict for mpmi.Screener(...) or Screener.set_weights()."""
    rec = read(path, FORMAT_SCREENER)
    return {key[2:]: np.asarray(value, dtype=np.float32) for key, value in rec.items()
            if key.startswith("w_")}


# ---------------------------------------------------------------- sessions
def session_record(config: dict, next_tick: int, noise=None, rollout: str = "full") -> dict:
    """The contents of a session file."""
    rec = dict(format=FORMAT_SESSION, next_tick=int(next_tick), rollout=rollout,
               noise=np.asarray([] if noise is None else noise, dtype=np.float64))
    rec.update({f"cfg_{key}": value for key, value in config.items()})
    return rec


def save_session(path: str, session: mpmi.Session, next_tick: int) -> None:
    """The session's configuration and the tick it resumes at."""
    write(path, session_record(session.config, next_tick, session.noise, session.rollout))


def open_session(ctx: mpmi.Context, model: mpmi.Model, path: str):
    """(session, next tick): the saved session reopened on `model`."""
    rec = read(path, FORMAT_SESSION)
    cfg = {key[4:]: value for key, value in rec.items() if key.startswith("cfg_")}
    sess = mpmi.Session(ctx, model, cfg["n_samples"], cfg["horizon"], cfg["input_lo"],
                        cfg["input_hi"], include_user=bool(cfg["include_user"]),
                        sampler=str(cfg["sampler"]), seed=cfg["seed"],
                        stream_id=cfg["stream_id"], lanes=cfg["lanes"], block=cfg["block"],
                        cands=cfg["cands"])
    if np.size(rec["noise"]) > 0:
        sess.set_noise(rec["noise"])
    if rec["rollout"] != "full":
        sess.set_rollout(str(rec["rollout"]))
    return sess, int(rec["next_tick"])
