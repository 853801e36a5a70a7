"""Quasi-Newton minimisation of the NLL (BFGS with a strong-Wolfe line search,
Nocedal & Wright, Numerical Optimization, 2nd ed., Algorithms 6.1, 3.5, 3.6)
and parameter errors from the Hessian of the NLL.

The paper fits by maximum likelihood with a MINUIT-lineage minimiser; this is
a gradient-based equivalent that uses the library's analytic gradient.  Only
the floating parameters are varied; the others stay at their start values.
Host-side orchestration only: every NLL and gradient comes from the GPU.
"""
from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass, field
from typing import Callable, Optional

import numpy as np

Objective = Callable[[np.ndarray], "tuple[float, np.ndarray]"]


@dataclass
class FitResult:
    x: np.ndarray
    fun: float
    grad: np.ndarray
    n_iter: int
    n_eval: int
    converged: bool
    message: str
    inv_hessian: np.ndarray                  # BFGS approximation, floating subspace
    history: list = field(default_factory=list)

    def to_json(self) -> str:
        d = asdict(self)
        for k in ("x", "grad", "inv_hessian"):
            d[k] = np.asarray(d[k]).tolist()
        return json.dumps(d)


def _line_search(phi, dphi, f0, g0, a1=1.0, c1=1e-4, c2=0.9, amax=50.0, maxiter=25):
    """Strong-Wolfe line search (Nocedal & Wright Alg. 3.5 with zoom, Alg. 3.6).
    phi(a) -> (f, g_vec); dphi is the directional derivative at 0.
    Returns (a, f, g) or (None, ...) on failure."""
    def zoom(alo, ahi, flo, dlo, glo, fhi, dhi):
        for _ in range(maxiter):
            if abs(ahi - alo) <= 1e-14 * max(1.0, abs(alo)):
                break
            # cubic interpolation, bisection safeguard
            d1 = dlo + dhi - 3 * (flo - fhi) / (alo - ahi)
            rad = d1 * d1 - dlo * dhi
            if rad >= 0:
                d2 = math.copysign(math.sqrt(rad), ahi - alo)
                den = dhi - dlo + 2 * d2
                a = ahi - (ahi - alo) * (dhi + d2 - d1) / den if den != 0 else 0.5 * (alo + ahi)
            else:
                a = 0.5 * (alo + ahi)
            lo, hi = min(alo, ahi), max(alo, ahi)
            if not (lo + 0.1 * (hi - lo) <= a <= hi - 0.1 * (hi - lo)):
                a = 0.5 * (alo + ahi)
            f, g, d = phi(a)
            if f > f0 + c1 * a * dphi or f >= flo:
                ahi, fhi, dhi = a, f, d
            else:
                if abs(d) <= -c2 * dphi:
                    return a, f, g
                if d * (ahi - alo) >= 0:
                    ahi, fhi, dhi = alo, flo, dlo
                alo, flo, dlo, glo = a, f, d, g
        # interval exhausted: accept the best point if it decreased f
        if alo > 0 and flo < f0:
            return alo, flo, glo
        return None, None, None

    aprev, fprev, dprev, gprev = 0.0, f0, dphi, g0
    a = a1
    for i in range(maxiter):
        f, g, d = phi(a)
        if not np.isfinite(f):
            a = 0.5 * (aprev + a)
            continue
        if f > f0 + c1 * a * dphi or (i > 0 and f >= fprev):
            return zoom(aprev, a, fprev, dprev, gprev, f, d)
        if abs(d) <= -c2 * dphi:
            return a, f, g
        if d >= 0:
            return zoom(a, aprev, f, d, g, fprev, dprev)
        aprev, fprev, dprev, gprev = a, f, d, g
        a = min(2 * a, amax)
    return None, None, None


def bfgs(fg: Objective, x0, floating=None, gtol: float = 1e-3, edm_tol: float = 1e-6, max_iter: int = 500,
         scale=None, callback=None) -> FitResult:
    """Minimise f over the floating parameters.  Convergence: estimated
    distance to minimum g^T H^{-1} g / 2 below edm_tol (the MINUIT criterion)
    or the largest scaled gradient component below gtol."""
    x0 = np.asarray(x0, dtype=np.float64)
    mask = np.ones(len(x0), dtype=bool) if floating is None else np.asarray(floating, dtype=bool)
    idx = np.flatnonzero(mask)
    s = np.ones(len(idx)) if scale is None else np.asarray(scale, dtype=np.float64)[idx]
    n_eval = 0

    def full(z):
        x = x0.copy()
        x[idx] = z * s
        return x

    def fz(z):
        nonlocal n_eval
        n_eval += 1
        f, g = fg(full(z))
        return f, np.asarray(g)[idx] * s

    z = x0[idx] / s
    f, g = fz(z)
    H = np.eye(len(idx))
    hist = []
    converged, msg, it = False, "maximum number of iterations", 0
    for it in range(1, max_iter + 1):
        p = -H @ g
        dphi = float(g @ p)
        if dphi >= 0:
            H = np.eye(len(idx))
            p = -g
            dphi = float(g @ p)

        def phi(a):
            fa, ga = fz(z + a * p)
            return fa, ga, float(ga @ p)
        a, fn, gn = _line_search(phi, dphi, f, g, a1=1.0 if it > 1 else min(1.0, 1.0 / max(1e-12, np.abs(g).max())))
        if a is None:
            msg = "line search failed"
            break
        sv = a * p
        yv = gn - g
        z, f, g = z + sv, fn, gn
        sy = float(sv @ yv)
        if sy > 1e-300:
            if it == 1:
                H = np.eye(len(idx)) * (sy / float(yv @ yv))
            rho = 1.0 / sy
            I = np.eye(len(idx))
            H = (I - rho * np.outer(sv, yv)) @ H @ (I - rho * np.outer(yv, sv)) + rho * np.outer(sv, sv)
        edm = 0.5 * float(g @ H @ g)
        hist.append({"iter": it, "f": f, "edm": edm, "max_grad": float(np.abs(g).max())})
        if callback:
            callback(it, full(z), f)
        if edm < edm_tol or np.abs(g).max() < gtol:
            converged, msg = True, "converged"
            break
    gfull = np.zeros(len(x0))
    gfull[idx] = g / s
    Hs = H * np.outer(s, s)
    return FitResult(full(z), f, gfull, it, n_eval, converged, msg, Hs, hist)


def hessian(fg: Objective, x, floating=None, rel_step: float = 1e-4, abs_step: float = 1e-7) -> np.ndarray:
    """Symmetrised central-difference Hessian of f over the floating
    parameters, from analytic gradients (2 gradient calls per parameter)."""
    x = np.asarray(x, dtype=np.float64)
    mask = np.ones(len(x), dtype=bool) if floating is None else np.asarray(floating, dtype=bool)
    idx = np.flatnonzero(mask)
    Hm = np.zeros((len(idx), len(idx)))
    for a, i in enumerate(idx):
        h = max(abs(x[i]) * rel_step, abs_step)
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        gp = np.asarray(fg(xp)[1])[idx]
        gm = np.asarray(fg(xm)[1])[idx]
        Hm[a] = (gp - gm) / (2 * h)
    return 0.5 * (Hm + Hm.T)


def errors(fg: Objective, x, floating=None) -> np.ndarray:
    """Parabolic errors sqrt(diag(H^{-1})) for the NLL (1 sigma at Delta NLL = 1/2)."""
    mask = np.ones(len(x), dtype=bool) if floating is None else np.asarray(floating, dtype=bool)
    Hm = hessian(fg, x, mask)
    cov = np.linalg.inv(Hm)
    err = np.zeros(len(x))
    err[np.flatnonzero(mask)] = np.sqrt(np.clip(np.diag(cov), 0, None))
    return err


def safe_objective(tdmix) -> Objective:
    """NLL and gradient of a TDMix context; parameter points outside the
    model's domain (|y| >= 1, non-positive widths, a rate <= 0) give
    f = +inf so that line searches step back instead of stopping."""
    from .tdmix import TDMixError

    def fg(p):
        try:
            return tdmix.nll(p, grad=True)
        except TDMixError as e:
            if e.code in (-5, -6):
                return math.inf, np.full(len(p), np.nan)
            raise
    return fg


def default_scales(p: np.ndarray, n_chains: int, n_res: int) -> np.ndarray:
    """Typical step sizes per parameter: coefficient magnitudes, 1e-3 of the
    resonance masses and 1e-2 of the widths, 1e-3 for x and y."""
    s = np.ones(len(p))
    for c in range(n_chains):
        s[2 * c:2 * c + 2] = max(abs(complex(p[2 * c], p[2 * c + 1])), 1e-3)
    for r in range(n_res):
        s[2 * n_chains + 2 * r] = 1e-3 * max(abs(p[2 * n_chains + 2 * r]), 1e-3)
        s[2 * n_chains + 2 * r + 1] = 1e-2 * max(abs(p[2 * n_chains + 2 * r + 1]), 1e-3)
    s[-2:] = 1e-3
    return s


def fit(tdmix, start, floating, n_chains: int, n_res: int, **kw) -> FitResult:
    """BFGS fit of a TDMix context from `start` over the floating mask."""
    fg = safe_objective(tdmix)
    return bfgs(fg, start, floating=floating, scale=default_scales(np.asarray(start), n_chains, n_res), **kw)
