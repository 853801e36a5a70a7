"""Pins of the oracle's likelihood: -sum ln(R/N) with numerical
normalisation (Sec. 3.1) and its autograd gradient."""
import copy
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples

F64 = torch.float64


def _nr_model(cA, cB, x, y):
    d = {
        "parent_mass": samples.M_D,
        "final_state": [{"mass": m} for m in samples.FINAL_STATE_MASSES],
        "bose_swap": [1, 3], "tau": samples.TAU_D, "r_resonance": 1.5, "r_parent": 5.0,
        "x": x, "y": y, "resonances": [],
        "chains": [{"name": "nr A", "amp": "A", "spin": "NR", "coef": [cA.real, cA.imag]},
                   {"name": "nr Abar", "amp": "Abar", "spin": "NR", "coef": [cB.real, cB.imag]}],
    }
    return tdamp.load_model(d)


def test_nll_of_constant_amplitudes_from_time_evolution():
    """With constant amplitudes (one non-resonant chain per amplitude) the
    rate is 2|<f|D0(t)>|^2 of the two-state system and N its time integral;
    the NLL must equal -sum ln(R/N) computed that way."""
    x, y = 0.2, 0.15
    cA, cB = complex(0.3, -0.4), complex(1.0, 0.2)
    m = _nr_model(cA, cB, x, y)
    gamma = m.gamma
    ev = torch.from_numpy(samples.flat_phase_space(5, samples.rng(80, 0)))
    t = torch.tensor([0.1, 0.3, 0.7, 1.5, 2.2], dtype=F64)
    lam = np.array([1 + x * gamma / 2 - 0.5j * gamma * (1 + y), 1 - x * gamma / 2 - 0.5j * gamma * (1 - y)])
    V = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    H = V @ np.diag(lam) @ np.linalg.inv(V)
    A, Ab = 2 * cA, 2 * cB          # Bose sum of two unit spin factors

    def rate(tt):
        psi = scipy.linalg.expm(-1j * H * tt) @ np.array([1.0, 0.0])
        return 2 * abs(psi[0] * A + psi[1] * Ab) ** 2

    N, _ = scipy.integrate.quad(rate, 0, 60, epsabs=0, epsrel=1e-12, limit=500)
    expect = -sum(math.log(rate(float(tt)) / N) for tt in t)
    got = float(tdamp.nll(m, ev, t, ev, m.default_params()))
    assert abs(got - expect) <= 1e-10 * abs(expect)


def test_nll_no_mixing_limit():
    """x = y = 0: NLL = -sum ln(|A|^2/<|A|^2>) + sum (Gamma t - ln Gamma)."""
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    m.x = m.y = 0.0
    g = samples.rng(81, 0)
    data = torch.from_numpy(samples.flat_phase_space(300, g))
    t = torch.from_numpy(samples.exponential_times(300, m.gamma, g))
    mc = torch.from_numpy(samples.flat_phase_space(3000, g))
    p = m.default_params()
    A, _ = tdamp.amplitudes(m, data, p)
    Am, _ = tdamp.amplitudes(m, mc, p)
    expect = -torch.log(A.abs() ** 2 / (Am.abs() ** 2).mean()).sum() + (m.gamma * t - math.log(m.gamma)).sum()
    got = tdamp.nll(m, data, t, mc, p)
    assert abs(float(got - expect)) <= 1e-11 * abs(float(expect))


def test_weighted_normalisation_equals_replicated_sample():
    """Integer MC weights act as replicated events."""
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    mc = torch.from_numpy(samples.flat_phase_space(200, samples.rng(82, 0)))
    w = torch.from_numpy(np.random.default_rng(3).integers(1, 4, 200).astype(np.float64))
    rep = torch.repeat_interleave(mc, w.long(), dim=0)
    p = m.default_params()
    assert abs(float(tdamp.normalisation(m, mc, p, w) / tdamp.normalisation(m, rep, p)) - 1) < 1e-13


@pytest.mark.parametrize("name", ["d0_k3pi_2chain", "d0_k3pi_full"])
def test_gradient_matches_central_differences(name):
    m = tdamp.load_model(model_path(name))
    g = samples.rng(83, 0)
    data = torch.from_numpy(samples.flat_phase_space(200, g))
    t = torch.from_numpy(samples.exponential_times(200, m.gamma, g))
    mc = torch.from_numpy(samples.flat_phase_space(2000, g))
    p = m.default_params()
    v, grad = tdamp.nll_and_grad(m, data, t, mc, p)
    mask = m.floating_mask()
    for k in range(len(p)):
        if not mask[k]:
            assert grad[k] == 0
            continue
        h = 2e-5 * max(abs(float(p[k])), 0.1)

        def f(d):
            q = p.clone()
            q[k] += d
            return float(tdamp.nll(m, data, t, mc, q))
        # five-point central stencil, truncation O(h^4)
        fd = (8 * (f(h) - f(-h)) - (f(2 * h) - f(-2 * h))) / (12 * h)
        assert abs(fd - float(grad[k])) <= 2e-6 * max(abs(fd), 1.0), (k, fd, float(grad[k]))
