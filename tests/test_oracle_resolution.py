"""Pins of the oracle's decay-time resolution (an extension the paper leaves
out, Sec. 4): the rate of Eq. (mix) folded with a Gaussian of width sigma.

The oracle folds by quadrature; these tests fix it by routes that share
nothing with that quadrature:
* the closed form of the fold of each exponential term, through the
  Faddeeva function (scipy.special.wofz):
      int_0^inf e^{-a t'} G(t - t') dt' = 1/2 e^{-t^2/(2 sigma^2)} w(i (a sigma^2 - t) / (sigma sqrt 2))
  with a = Gamma (1 -+ y) for cosh, sinh and a = Gamma (1 - i x) for cos + i sin;
* for x = y = 0 the same with the real erfcx;
* the narrow-resolution limit (the unfolded rate);
* the time integral over the real line (the unchanged normalisation)."""
import math

import numpy as np
import pytest
import torch
from scipy import special

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples


def _amps(n=40, seed=3):
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    ev = torch.from_numpy(samples.flat_phase_space(n, samples.rng(seed, samples.STREAM_MC)))
    A, Ab = tdamp.amplitudes(m, ev, m.default_params())
    return m, A, Ab


def _fold(t, a, sigma):
    """Closed form of int_0^inf e^{-a t'} G(t - t'; sigma) dt' (complex a).
    In the lower half plane w(xi) = 2 e^{-xi^2} - w(-xi), and
    1/2 e^{-t^2/(2 sigma^2)} 2 e^{-xi^2} = e^{-a t + a^2 sigma^2 / 2}."""
    t = np.asarray(t, dtype=np.float64)
    xi = 1j * (a * sigma * sigma - t) / (sigma * math.sqrt(2))
    g = np.exp(-t * t / (2 * sigma * sigma))
    up = xi.imag >= 0
    out = np.empty(t.shape, dtype=np.complex128)
    out[up] = 0.5 * g[up] * special.wofz(xi[up])
    lo = ~up
    out[lo] = np.exp(-a * t[lo] + a * a * sigma * sigma / 2) - 0.5 * g[lo] * special.wofz(-xi[lo])
    return out


def _closed_form_rate(A, Ab, t, x, y, gamma, sigma, scale=False):
    """The folded rate from the closed-form folds; with scale, also the sum of
    the four terms' magnitudes (the terms cancel where A and Abar interfere
    destructively, and rounding errors scale with this sum)."""
    A, Ab = A.numpy(), Ab.numpy()
    km, kp = _fold(t, gamma * (1 - y), sigma), _fold(t, gamma * (1 + y), sigma)
    cch, csh = (km + kp).real / 2, (km - kp).real / 2
    cc = _fold(t, gamma * (1 - 1j * x), sigma)
    A2, B2, X = np.abs(A) ** 2, np.abs(Ab) ** 2, A * np.conj(Ab)
    terms = ((A2 + B2) * cch, (A2 - B2) * cc.real, -2 * X.real * csh, -2 * X.imag * cc.imag)
    R = sum(terms)
    return (R, sum(np.abs(v) for v in terms)) if scale else R


@pytest.mark.parametrize("x,y,sigma", [(0.0049, 0.0061, 0.045), (0.3, -0.2, 0.045), (0.02, 0.05, 0.12)])
def test_fold_equals_faddeeva_closed_form(x, y, sigma):
    m, A, Ab = _amps()
    t = np.linspace(-0.3, 4.0, A.shape[0])
    R = tdamp.rate_resolved(A, Ab, torch.from_numpy(t), x, y, m.gamma, sigma).numpy()
    ref, S = _closed_form_rate(A, Ab, t, x, y, m.gamma, sigma, scale=True)
    assert np.max(np.abs(R - ref) / S) <= 1e-13


def test_no_mixing_fold_equals_erfcx():
    m, A, Ab = _amps()
    sigma = 0.045
    t = np.linspace(-0.2, 6.0, A.shape[0])
    R = tdamp.rate_resolved(A, Ab, torch.from_numpy(t), 0.0, 0.0, m.gamma, sigma).numpy()
    u = (m.gamma * sigma * sigma - t) / (sigma * math.sqrt(2))
    g = np.exp(-t * t / (2 * sigma * sigma))
    # erfcx(u) = 2 e^{u^2} - erfcx(-u) where u < 0, with e^{-t^2/(2 sigma^2) + u^2} = e^{-Gamma t + Gamma^2 sigma^2 / 2}
    fold = np.where(u >= 0, 0.5 * g * special.erfcx(np.abs(u)),
                    np.exp(-m.gamma * t + (m.gamma * sigma) ** 2 / 2) - 0.5 * g * special.erfcx(np.abs(u)))
    ref = 2 * np.abs(A.numpy()) ** 2 * fold
    assert np.max(np.abs(R - ref) / ref) <= 1e-12


def test_narrow_resolution_gives_the_unfolded_rate():
    m, A, Ab = _amps()
    t = np.linspace(0.05, 3.0, A.shape[0])
    R = tdamp.rate_resolved(A, Ab, torch.from_numpy(t), 0.3, -0.2, m.gamma, 1e-5).numpy()
    R0, _ = tdamp.rate_literal(A, Ab, torch.from_numpy(t), 0.3, -0.2, m.gamma)
    assert np.max(np.abs(R / R0.numpy() - 1)) <= 1e-8


def test_time_integral_is_the_unfolded_normalisation():
    """The integral of the folded rate over the measured time (the real line)
    equals the closed-form time integral of the unfolded rate: composite
    Gauss-Legendre over [-12 sigma, 12 sigma] and [12 sigma, 100 tau] (beyond
    100 lifetimes the rate is below e^{-80} of its start)."""
    m, A, Ab = _amps(n=3)
    x, y, sigma = 0.3, -0.2, 0.08
    ref = tdamp.norm_integrand(A, Ab, x, y, m.gamma).numpy()
    xg, wg = np.polynomial.legendre.leggauss(48)
    edges = np.concatenate([np.linspace(-12 * sigma, 12 * sigma, 17), np.geomspace(12 * sigma, 100 * m.tau, 81)[1:]])
    nodes = np.concatenate([(b + a) / 2 + (b - a) / 2 * xg for a, b in zip(edges[:-1], edges[1:])])
    weights = np.concatenate([(b - a) / 2 * wg for a, b in zip(edges[:-1], edges[1:])])
    for e in range(3):
        n = len(nodes)
        R = tdamp.rate_resolved(A[e:e + 1].expand(n), Ab[e:e + 1].expand(n), torch.from_numpy(nodes), x, y, m.gamma,
                                sigma).numpy()
        assert abs((R * weights).sum() / ref[e] - 1) <= 1e-12


def test_resolution_model_rates_and_gradient():
    """A model file with "time_resolution" uses the folded rate; the NLL
    gradient (autograd) agrees with central differences in x and y."""
    import json
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["time_resolution"] = 0.045
    m = tdamp.load_model(d)
    assert m.sigma_t == 0.045
    ev = torch.from_numpy(samples.flat_phase_space(50, samples.rng(4, samples.STREAM_DATA)))
    t = torch.linspace(-0.1, 2.0, 50, dtype=torch.float64)
    mc = torch.from_numpy(samples.flat_phase_space(500, samples.rng(4, samples.STREAM_MC)))
    p = m.default_params().numpy()
    p[-2], p[-1] = 0.03, 0.04
    v, g = tdamp.nll_and_grad(m, ev, t, mc, p)
    for k in (len(p) - 2, len(p) - 1):
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (tdamp.nll(m, ev, t, mc, torch.from_numpy(pp)) - tdamp.nll(m, ev, t, mc, torch.from_numpy(pm))) / (2 * h)
        assert abs(float(fd) - float(g[k])) <= 1e-6 * max(1.0, abs(float(g[k])))
