"""Seeded synthetic event samples for the D0 -> K+ pi- pi+ pi- likelihood.

This module is shared by the CUDA path's users (bench, examples) and by the
tests that drive the oracle.  It holds no amplitude or likelihood arithmetic:
it draws flat four-body phase space (GENBOD, F. James, CERN 68-15), decay
times, and performs accept/reject selection on weights that the caller
computes with whatever model evaluator it trusts.  The paper generates its
normalisation points as flat phase space and its pseudo-events as phase-space
points weighted by the model and selected by accept/reject (Sec. 3.1).

Random numbers come from NumPy's Philox counter-based generator
(Salmon et al., SC'11); only uniform doubles are drawn from it and every
non-uniform variate is derived here, so a sample depends only on the key.

Units: GeV for energies and momenta, ps for times.  Final-state order is the
decay's name order: p0 = K+, p1 = pi-(a), p2 = pi+, p3 = pi-(b).  Events are
float64 arrays of shape (n, 4, 4) indexed [event, particle, (E, px, py, pz)].
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable

import numpy as np

# Masses (GeV) and D0 lifetime (ps) of the four-body workload.
M_D = 1.86484
M_K = 0.493677
M_PI = 0.13957
TAU_D = 0.4101
FINAL_STATE_MASSES = (M_K, M_PI, M_PI, M_PI)

# Keys: SEED_BASE + workload index; streams name what is drawn.
SEED_BASE = 1702067350
STREAM_DATA, STREAM_MC, STREAM_COEF = 0, 1, 2
STREAM_TOY0 = 1000


def rng(workload: int, stream: int) -> np.random.Generator:
    """Philox generator keyed by (SEED_BASE + workload, stream)."""
    return np.random.Generator(np.random.Philox(key=[SEED_BASE + workload, stream]))


def _breakup(m: np.ndarray, m1: np.ndarray, m2: np.ndarray) -> np.ndarray:
    """Two-body breakup momentum of mass m into m1 + m2 (zero below threshold)."""
    a = (m * m - (m1 + m2) ** 2) * (m * m - (m1 - m2) ** 2)
    return np.sqrt(np.maximum(a, 0.0)) / (2.0 * m)


def _isotropic(n: int, g: np.random.Generator) -> np.ndarray:
    u = g.random((n, 2))
    cos_t = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * math.pi * u[:, 1]
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _boost(p: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Boost four-vectors p (..., 4) by velocity beta (..., 3)."""
    b2 = np.sum(beta * beta, axis=-1)
    gamma = 1.0 / np.sqrt(1.0 - b2)
    bp = np.sum(beta * p[..., 1:], axis=-1)
    coef = np.where(b2 > 0, (gamma - 1.0) / np.where(b2 > 0, b2, 1.0), 0.0)
    e = gamma * (p[..., 0] + bp)
    vec = p[..., 1:] + (coef * bp + gamma * p[..., 0])[..., None] * beta
    return np.concatenate([e[..., None], vec], axis=-1)


@dataclass
class GenbodBatch:
    p4: np.ndarray       # (n, k, 4)
    weight: np.ndarray   # (n,) phase-space weight relative to wt_max
    wt_max: float        # GENBOD upper bound of the raw weight


def genbod(n: int, g: np.random.Generator, M: float = M_D,
           masses=FINAL_STATE_MASSES) -> GenbodBatch:
    """Weighted k-body phase space of a mass M at rest (GENBOD).

    Intermediate invariant masses M_j of particles 0..j are spaced by sorted
    uniforms; the raw weight is the product of the breakup momenta
    p(M_j -> M_{j-1} + m_j); the returned weight is raw / wt_max, where wt_max
    is GENBOD's product of breakup momenta at the extreme masses.
    """
    masses = np.asarray(masses, dtype=np.float64)
    k = len(masses)
    tecm = M - masses.sum()
    if tecm <= 0:
        raise ValueError("decay below threshold")
    r = np.sort(g.random((n, k - 2)), axis=1) if k > 2 else np.zeros((n, 0))
    cum = np.cumsum(masses)
    Mj = np.empty((n, k))
    Mj[:, 0] = masses[0]
    for j in range(1, k - 1):
        Mj[:, j] = cum[j] + r[:, j - 1] * tecm
    Mj[:, k - 1] = M
    pd = np.empty((n, k - 1))
    for j in range(1, k):
        pd[:, j - 1] = _breakup(Mj[:, j], Mj[:, j - 1], np.full(n, masses[j]))
    wt_max = 1.0
    for j in range(1, k):
        emmax = tecm + cum[j]
        emmin = cum[j - 1]
        wt_max *= float(_breakup(np.array([emmax]), np.array([emmin]), np.array([masses[j]]))[0])
    weight = np.prod(pd, axis=1) / wt_max

    # Build momenta: particles 0,1 back to back in the rest frame of M_1,
    # then each next particle against the subsystem, boosting that subsystem.
    p4 = np.zeros((n, k, 4))
    d = _isotropic(n, g)
    q = pd[:, 0]
    p4[:, 0, 1:] = q[:, None] * d
    p4[:, 0, 0] = np.sqrt(q * q + masses[0] ** 2)
    p4[:, 1, 1:] = -q[:, None] * d
    p4[:, 1, 0] = np.sqrt(q * q + masses[1] ** 2)
    for j in range(2, k):
        d = _isotropic(n, g)
        q = pd[:, j - 1]
        # subsystem 0..j-1 moves along -d with momentum q and mass M_{j-1}
        e_sub = np.sqrt(q * q + Mj[:, j - 1] ** 2)
        beta = (-q / e_sub)[:, None] * d
        p4[:, :j, :] = _boost(p4[:, :j, :], beta[:, None, :])
        p4[:, j, 1:] = q[:, None] * d
        p4[:, j, 0] = np.sqrt(q * q + masses[j] ** 2)
    return GenbodBatch(p4=p4, weight=weight, wt_max=wt_max)


def flat_phase_space(n: int, g: np.random.Generator, M: float = M_D,
                     masses=FINAL_STATE_MASSES, batch: int = 1 << 18) -> np.ndarray:
    """Exactly n unweighted (flat) phase-space events, shape (n, k, 4).

    GENBOD events are kept with probability weight / wt_max, which is exact
    because wt_max bounds the weight."""
    out = []
    have = 0
    while have < n:
        b = genbod(batch, g, M, masses)
        keep = g.random(batch) < b.weight
        sel = b.p4[keep]
        out.append(sel)
        have += len(sel)
    return np.concatenate(out, axis=0)[:n]


def exponential_times(n: int, rate: float, g: np.random.Generator) -> np.ndarray:
    """Decay times t ~ rate * exp(-rate t) by inversion."""
    u = g.random(n)
    return -np.log1p(-u) / rate


WeightFn = Callable[[np.ndarray, np.ndarray], np.ndarray]


def generate_time_dependent(n: int, g: np.random.Generator, rate_fn: WeightFn,
                            gamma: float, y: float, pilot: int = 200_000,
                            headroom: float = 1.2, batch: int = 1 << 17,
                            max_rounds: int = 4):
    """Pseudo-events distributed as rate_fn(p4, t) by accept/reject.

    Proposals are flat phase space times t ~ Exp((1-|y|) gamma).  rate_fn must
    return the unnormalised decay rate R(e) >= 0 of each proposal; the
    acceptance weight is R(e) / exp(-(1-|y|) gamma t).  The envelope is
    headroom x the largest weight of a pilot sample; if any later weight
    exceeds it, the envelope is raised to that weight times headroom and the
    sample is drawn again (at most max_rounds times).
    Returns (p4 (n,4,4), t (n,), stats dict)."""
    lam = (1.0 - abs(y)) * gamma
    pp = flat_phase_space(pilot, g)
    pt = exponential_times(pilot, lam, g)
    w = np.asarray(rate_fn(pp, pt), dtype=np.float64) / np.exp(-lam * pt)
    if not np.all(np.isfinite(w)) or np.any(w < 0):
        raise ValueError("rate_fn returned a negative or non-finite rate")
    env = headroom * float(w.max())
    for _ in range(max_rounds):
        out_p, out_t = [], []
        have = 0
        proposed = 0
        violated = 0.0
        while have < n:
            p4 = flat_phase_space(batch, g)
            t = exponential_times(batch, lam, g)
            wt = np.asarray(rate_fn(p4, t), dtype=np.float64) / np.exp(-lam * t)
            violated = max(violated, float(wt.max()))
            keep = g.random(batch) * env < wt
            out_p.append(p4[keep])
            out_t.append(t[keep])
            have += int(keep.sum())
            proposed += batch
        if violated <= env:
            p4 = np.concatenate(out_p)[:n]
            t = np.concatenate(out_t)[:n]
            return p4, t, {"envelope": env, "proposed": proposed, "efficiency": n / proposed}
        env = headroom * violated
    raise RuntimeError("accept/reject envelope kept being exceeded")


def event_planes(p4: np.ndarray) -> np.ndarray:
    """(n, 4, 4) events -> contiguous (4, 4, n) structure-of-arrays planes."""
    return np.ascontiguousarray(np.transpose(p4, (1, 2, 0)))
