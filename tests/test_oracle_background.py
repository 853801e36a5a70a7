"""Pins of the oracle's background mixture (an extension the paper leaves
out, Sec. 4): each data event's density is (1 - f) R / N + f B, B flat in the
normalised phase space and exponential in the decay time."""
import json
import math

import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples


def _model(f, tau_b=0.8, sigma=0.0):
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["background"] = {"fraction": f, "tau": tau_b}
    if sigma > 0:
        d["time_resolution"] = sigma
    return tdamp.load_model(d)


def _sample(n=60, n_mc=600):
    ev = torch.from_numpy(samples.flat_phase_space(n, samples.rng(6, samples.STREAM_DATA)))
    t = torch.linspace(0.01, 3.0, n, dtype=torch.float64)
    mc = torch.from_numpy(samples.flat_phase_space(n_mc, samples.rng(6, samples.STREAM_MC)))
    return ev, t, mc


def test_no_background_limit():
    ev, t, mc = _sample()
    m0 = tdamp.load_model(model_path("d0_k3pi_2chain"))
    m = _model(1e-13)
    p = m0.default_params()
    assert abs(float(tdamp.nll(m, ev, t, mc, p)) / float(tdamp.nll(m0, ev, t, mc, p)) - 1) <= 1e-11


def test_pure_background_closed_form():
    """f = 1: NLL = sum (t / tau_b + ln tau_b), whatever the amplitudes."""
    ev, t, mc = _sample()
    m = _model(1.0, tau_b=0.8)
    v = float(tdamp.nll(m, ev, t, mc, m.default_params()))
    ref = float((t / 0.8 + math.log(0.8)).sum())
    assert abs(v - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("sigma", [0.0, 0.045])
def test_background_density_integrates_to_one(sigma):
    """int B dt = 1 over the measured time (composite Gauss-Legendre)."""
    m = _model(0.2, tau_b=0.6, sigma=sigma)
    xg, wg = np.polynomial.legendre.leggauss(48)
    lo = -12 * sigma if sigma > 0 else 0.0
    edges = np.concatenate([np.linspace(lo, max(12 * sigma, 0.05), 9), np.geomspace(max(12 * sigma, 0.05), 100 * 0.6,
                                                                                   81)[1:]])
    nodes = np.concatenate([(b + a) / 2 + (b - a) / 2 * xg for a, b in zip(edges[:-1], edges[1:])])
    weights = np.concatenate([(b - a) / 2 * wg for a, b in zip(edges[:-1], edges[1:])])
    B = tdamp.background_density(m, torch.from_numpy(nodes)).numpy()
    assert abs((B * weights).sum() - 1) <= 1e-12


def test_background_gradient_against_central_differences():
    ev, t, mc = _sample()
    m = _model(0.3, tau_b=0.8, sigma=0.045)
    p = m.default_params().numpy()
    p[-2], p[-1] = 0.02, 0.03
    _, g = tdamp.nll_and_grad(m, ev, t, mc, p)
    for k in (2, 3, 4, 5, len(p) - 2, len(p) - 1):
        h = 1e-6 * max(1.0, abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (tdamp.nll(m, ev, t, mc, torch.from_numpy(pp)) - tdamp.nll(m, ev, t, mc, torch.from_numpy(pm))) / (2 * h)
        assert abs(float(fd) - float(g[k])) <= 1e-5 * max(1.0, abs(float(g[k])))
