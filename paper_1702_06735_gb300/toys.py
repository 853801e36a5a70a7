"""Pseudo-experiment studies on the serving loop (the paper's sensitivity
study, Sec. 4 and its table of x, y resolutions: toys generated from the
model with the world-average x and y, fitted with the model fixed and x, y
floating).

Every toy is a sample the server generates on the device at admission
(tdmix_server_add_generated_sample; counter-based, so it depends only on the
seed and the toy's stream); each is fitted by its own BFGS minimiser thread
that submits NLL + gradient requests to the device-resident loop, and,
optionally, its x, y errors come from the Hessian of the NLL at the minimum
(central differences of the analytic gradient).  Host orchestration only:
every likelihood, gradient and event comes from the GPU.

Both studies can keep a checkpoint (ToyCheckpoint): every finished toy is
appended to a file as it ends, and a study started again with the same
file and the same arguments fits only the toys the file does not hold.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import hashlib
import json
import math
import os
import threading
import time
from dataclasses import dataclass

import numpy as np

from . import minimize
from .tdmix import TDMixError, TDMixServer, model_json


@dataclass
class ToyFit:
    n_events: int
    x: float
    y: float
    sx: float
    sy: float
    converged: bool
    n_eval: int


class ToyCheckpoint:
    """Checkpoint of a toy study: a JSON-lines file whose first line holds
    the study's fingerprint (model, sizes, generating parameters, seeds, MC
    sample digest, fit settings) and whose further lines are finished toys,
    {"toy": index, ...}, each appended, flushed and synced to disk when its
    fit ends.  Opening an existing file with the same fingerprint gives its
    records (`records`: index -> record) and appends to it; a different
    fingerprint raises ValueError, and so does a complete line that does not
    parse.  Text after the last newline (a line cut short when the process
    stopped) is dropped from the file.  record() may be called from several
    threads."""

    def __init__(self, path, fingerprint: dict):
        self.path = os.fspath(path)
        self.records: dict[int, dict] = {}
        self._lock = threading.Lock()
        head = json.dumps({"checkpoint": fingerprint}, sort_keys=True)
        keep, size = 0, 0
        if os.path.exists(self.path):
            with open(self.path, "rb") as f:
                raw = f.read()
            size = len(raw)
            complete = raw.split(b"\n")[:-1]  # lines that end with a newline
            if complete:
                try:
                    found = json.loads(complete[0])
                except ValueError:
                    raise ValueError(f"{self.path} is not a toy-study checkpoint") from None
                if found != json.loads(head):
                    raise ValueError(f"{self.path} is the checkpoint of a different study")
                keep = len(complete[0]) + 1
                for n, line in enumerate(complete[1:], start=2):
                    try:
                        rec = json.loads(line)
                        k = int(rec["toy"])
                    except (ValueError, KeyError, TypeError):
                        raise ValueError(f"{self.path}: line {n} is not a toy record") from None
                    self.records[k] = rec
                    keep += len(line) + 1
        if keep == 0:  # new file, or not even the fingerprint line was complete
            with open(self.path, "wb") as f:
                f.write(head.encode() + b"\n")
                f.flush()
                os.fsync(f.fileno())
        elif keep < size:
            with open(self.path, "r+b") as f:
                f.truncate(keep)
        self._f = open(self.path, "ab")

    def record(self, toy: int, **fields):
        line = json.dumps({"toy": int(toy), **fields}).encode() + b"\n"
        with self._lock:
            self._f.write(line)
            self._f.flush()
            os.fsync(self._f.fileno())

    def close(self):
        with self._lock:
            if not self._f.closed:
                self._f.close()


def _digest(a) -> str:
    """sha256 of an array's float64 values (host or device tensor, or array)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return hashlib.sha256(str(a.shape).encode() + a.tobytes()).hexdigest()


def _fingerprint(study: str, model, precision, sizes, gen_params, mc, seed, stream0, **settings) -> dict:
    out = {"study": study, "model": json.loads(model_json(model)), "precision": precision,
           "sizes": [int(n) for n in sizes], "gen_params": [float(v) for v in np.asarray(gen_params).ravel()],
           "mc_sha256": _digest(mc), "seed": int(seed), "stream0": int(stream0)}
    for k, v in settings.items():
        out[k] = None if v is None else (np.asarray(v).tolist() if isinstance(v, (np.ndarray, list, tuple)) else v)
    return out


def _objective(srv, sid):
    def fg(p):
        try:
            return srv.evaluate(sid, p, timeout_s=600.0)
        except TDMixError as e:
            if e.code in (-5, -6):
                return math.inf, np.full(len(p), np.nan)
            raise
    return fg


def run(model, precision: str, sizes, gen_params, mc, seed: int, stream0: int = 1000, clients: int = 16,
        budget_bytes: int = 4 << 30, with_errors: bool = False, start_shift: float = 1e-3, checkpoint=None):
    """Generate len(sizes) toys of the given sizes at gen_params, fit x and y
    of each (the model and the coefficients fixed) and return
    (list of ToyFit, server statistics dict).  With `checkpoint` (a path),
    finished toys are kept in a ToyCheckpoint and the toys it already holds
    are not fitted again (statistics["resumed"] counts them; the server
    statistics cover this call's fits).  A resumed toy is generated from the
    same seed and stream, but the server finds the generator's envelope again
    at its first admission, so its events are an equally valid draw of the
    model rather than the same ones."""
    gen_params = np.asarray(gen_params, dtype=np.float64)
    cp = None
    if checkpoint is not None:
        cp = ToyCheckpoint(checkpoint, _fingerprint("fixed-model toys", model, precision, sizes, gen_params, mc, seed,
                                                    stream0, with_errors=with_errors, start_shift=start_shift))
    srv = TDMixServer(model, precision, hbm_budget_bytes=budget_bytes, max_slots=256)
    try:
        srv.add_mc(mc)
        fits = [None] * len(sizes)
        if cp is not None:
            for k, rec in cp.records.items():
                if 0 <= k < len(sizes):
                    fits[k] = ToyFit(**rec["fit"])
        todo = [k for k in range(len(sizes)) if fits[k] is None]
        ids = {k: srv.add_generated_sample(gen_params, int(sizes[k]), seed, stream0 + k) for k in todo}
        mask = np.zeros(len(gen_params), dtype=bool)
        mask[-2:] = True
        scale = np.ones(len(gen_params))
        scale[-2:] = 1e-3

        def fit(k):
            fg = _objective(srv, ids[k])
            g = np.random.default_rng(seed + 7919 * k)
            x0 = gen_params.copy()
            x0[-2:] += start_shift * g.uniform(-1, 1, 2)
            r = minimize.bfgs(fg, x0, floating=mask, scale=scale, gtol=1e-3, edm_tol=1e-6, max_iter=60)
            sx = sy = float("nan")
            n_eval = r.n_eval
            if with_errors and r.converged:
                err = minimize.errors(fg, r.x, mask)
                sx, sy = float(err[-2]), float(err[-1])
                n_eval += 4
            fits[k] = ToyFit(int(sizes[k]), float(r.x[-2]), float(r.x[-1]), sx, sy, bool(r.converged), int(n_eval))
            if cp is not None:
                cp.record(k, fit=dataclasses.asdict(fits[k]))

        srv.reset_stats()
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=clients) as ex:
            list(ex.map(fit, todo))
        wall = time.perf_counter() - t0
        st = srv.stats() if todo else {}
        st.update(srv.loop_info())
        st["wall_s"] = wall
        st["resumed"] = len(sizes) - len(todo)
        return fits, st
    finally:
        srv.close()
        if cp is not None:
            cp.close()


@dataclass
class FloatingFit:
    n_events: int
    params: np.ndarray
    errors: np.ndarray
    converged: bool
    n_eval: int
    xy_fixed_model: tuple = ()  # (x, y, sx, sy) of the fixed-model fit of the same events, if asked for


def run_floating(model, precision: str, sizes, gen_params, mc, seed: int, stream0: int = 1000, floating=None,
                 start_shift: float = 1e-3, scale=None, compare_fixed: bool = False, checkpoint=None):
    """Pseudo-experiments fitted with the model floating: every parameter of
    the `floating` mask (default: every resonance mass and width with x and
    y; the chain coefficients stay at their generating values, since a
    floating DCS phase is nearly degenerate with x and y in the 2-chain
    model, whose strong phase varies little over phase space), an extension
    of the paper's fixed-model study (Sec. 4).  A floating
    model has no fixed component cache, so the fits run on one likelihood
    context (full evaluations, MC sums recomputed each time) instead of the
    serving loop; each toy is generated on the device with the same
    (seed, stream) as run() uses, so both studies fit the same events.
    Errors from the Hessian over all floating parameters.  With
    compare_fixed, the same events are also fitted with the model fixed (x, y
    floating), whose errors are the conditional ones.  Returns a list of
    FloatingFit.  With `checkpoint` (a path), finished toys are kept in a
    ToyCheckpoint with the generator's envelope, and a study started again
    takes the toys it holds from it and generates the others with the same
    envelope: the same events and fits as an uninterrupted study."""
    from .tdmix import TDMix
    gen_params = np.asarray(gen_params, dtype=np.float64)
    cp = None
    if checkpoint is not None:
        cp = ToyCheckpoint(checkpoint, _fingerprint("floating-model toys", model, precision, sizes, gen_params, mc,
                                                    seed, stream0, floating=floating, start_shift=start_shift,
                                                    scale=scale, compare_fixed=compare_fixed))
    c = TDMix(model, precision)
    try:
        if floating is None:
            mask = _model_mask(model)
            mask[:2 * len(_model_dict(model)["chains"])] = False
        else:
            mask = np.asarray(floating, dtype=bool)
        c.set_floating(mask.astype(np.int32))
        n_chains = sum(1 for _ in _model_dict(model)["chains"])
        n_res = len(_model_dict(model)["resonances"])
        sc = minimize.default_scales(gen_params, n_chains, n_res) if scale is None else scale
        fg = minimize.safe_objective(c)
        c.load_events(mc_p4=mc)
        out = []
        env = 0.0  # the generator's envelope, found by the first toy and reused (same parameters)
        done = {}
        if cp is not None:
            for k, rec in cp.records.items():
                d = dict(rec["fit"])
                done[k] = FloatingFit(int(d["n_events"]), np.asarray(d["params"], dtype=np.float64),
                                      np.asarray(d["errors"], dtype=np.float64), bool(d["converged"]),
                                      int(d["n_eval"]), tuple(d["xy_fixed_model"]))
                env = float(rec["envelope"])
        for k, n in enumerate(sizes):
            if k in done:
                out.append(done[k])
                continue
            p4, t, info = c.generate(int(n), seed=seed, stream=stream0 + k, params=gen_params, envelope=env)
            env = info["envelope"]
            c.load_events(p4, t)
            g = np.random.default_rng(seed + 7919 * k)
            x0 = gen_params.copy()
            x0[mask] += start_shift * sc[mask] * g.uniform(-1, 1, int(mask.sum()))
            r = minimize.bfgs(fg, x0, floating=mask, scale=sc, gtol=1e-3, edm_tol=1e-6, max_iter=400)
            err = minimize.errors(fg, r.x, mask) if r.converged else np.full(len(r.x), np.nan)
            fit = FloatingFit(int(n), r.x.copy(), err, bool(r.converged), int(r.n_eval) + 2 * int(mask.sum()))
            if compare_fixed:
                mxy = np.zeros(len(mask), dtype=bool)
                mxy[-2:] = True
                q0 = gen_params.copy()
                q0[-2:] = x0[-2:]
                c.set_floating(mxy.astype(np.int32))
                rf = minimize.bfgs(fg, q0, floating=mxy, scale=sc, gtol=1e-3, edm_tol=1e-6, max_iter=100)
                ef = minimize.errors(fg, rf.x, mxy) if rf.converged else np.full(len(rf.x), np.nan)
                fit.xy_fixed_model = (float(rf.x[-2]), float(rf.x[-1]), float(ef[-2]), float(ef[-1]))
                c.set_floating(mask.astype(np.int32))
            out.append(fit)
            if cp is not None:
                cp.record(k, envelope=env, fit={"n_events": fit.n_events, "params": fit.params.tolist(),
                                                "errors": np.asarray(fit.errors).tolist(), "converged": fit.converged,
                                                "n_eval": fit.n_eval, "xy_fixed_model": list(fit.xy_fixed_model)})
        return out
    finally:
        c.close()
        if cp is not None:
            cp.close()


def _model_dict(model) -> dict:
    import json
    from .tdmix import model_json
    return json.loads(model_json(model))


def _model_mask(model) -> np.ndarray:
    """The model file's floating mask (parameter order of the library)."""
    d = _model_dict(model)
    m = []
    for ch in d["chains"]:
        m += [ch.get("float", True)] * 2
    for r in d["resonances"]:
        m += [r.get("float", True)] * 2
    m += [d.get("float_xy", True)] * 2
    return np.asarray(m, dtype=bool)


def floating_pulls(fits, truth, index) -> dict:
    """Resolution and pulls of parameter `index` over converged fits."""
    ok = [f for f in fits if f.converged and np.isfinite(f.errors[index]) and f.errors[index] > 0]
    v = np.asarray([f.params[index] for f in ok])
    e = np.asarray([f.errors[index] for f in ok])
    pu = (v - truth[index]) / e
    n = len(pu)
    return {"used": n, "sigma": float(v.std(ddof=1)), "mean_error": float(e.mean()),
            "pull_mean": float(pu.mean()), "pull_mean_err": float(pu.std(ddof=1) / math.sqrt(n)),
            "pull_width": float(pu.std(ddof=1)), "pull_width_err": float(pu.std(ddof=1) / math.sqrt(2 * (n - 1)))}


def pulls(fits, x_true: float, y_true: float) -> dict:
    """Resolution and pull summary of converged toy fits with errors:
    sigma = standard deviation of the fitted values, the mean fitted error,
    pull mean and width with their statistical uncertainties."""
    ok = [f for f in fits if f.converged and np.isfinite(f.sx) and np.isfinite(f.sy)]
    out = {"toys": len(fits), "used": len(ok)}
    for name, val, err, true in (("x", [f.x for f in ok], [f.sx for f in ok], x_true),
                                 ("y", [f.y for f in ok], [f.sy for f in ok], y_true)):
        v, e = np.asarray(val), np.asarray(err)
        pu = (v - true) / e
        n = len(pu)
        out[name] = {"sigma": float(v.std(ddof=1)), "mean_error": float(e.mean()),
                     "pull_mean": float(pu.mean()), "pull_mean_err": float(pu.std(ddof=1) / math.sqrt(n)),
                     "pull_width": float(pu.std(ddof=1)), "pull_width_err": float(pu.std(ddof=1) / math.sqrt(2 * (n - 1)))}
    return out
