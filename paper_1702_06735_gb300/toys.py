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
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import time
from dataclasses import dataclass

import numpy as np

from . import minimize
from .tdmix import TDMixError, TDMixServer


@dataclass
class ToyFit:
    n_events: int
    x: float
    y: float
    sx: float
    sy: float
    converged: bool
    n_eval: int


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
        budget_bytes: int = 4 << 30, with_errors: bool = False, start_shift: float = 1e-3):
    """Generate len(sizes) toys of the given sizes at gen_params, fit x and y
    of each (the model and the coefficients fixed) and return
    (list of ToyFit, server statistics dict)."""
    gen_params = np.asarray(gen_params, dtype=np.float64)
    srv = TDMixServer(model, precision, hbm_budget_bytes=budget_bytes, max_slots=256)
    try:
        srv.add_mc(mc)
        ids = [srv.add_generated_sample(gen_params, int(n), seed, stream0 + k) for k, n in enumerate(sizes)]
        mask = np.zeros(len(gen_params), dtype=bool)
        mask[-2:] = True
        scale = np.ones(len(gen_params))
        scale[-2:] = 1e-3
        fits = [None] * len(sizes)

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

        srv.reset_stats()
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=clients) as ex:
            list(ex.map(fit, range(len(sizes))))
        wall = time.perf_counter() - t0
        st = srv.stats()
        st.update(srv.loop_info())
        st["wall_s"] = wall
        return fits, st
    finally:
        srv.close()


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
