"""Pins of the oracle's decay rate (Eq. (mix), Sec. 2), its time integrals and
the coherent sum with Bose symmetrisation (Sec. 3)."""
import json
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg
import torch

from conftest import GOLDEN_DIR, model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples

F64 = torch.float64


def _rand_complex(n, seed):
    g = np.random.default_rng(seed)
    return torch.complex(torch.tensor(g.normal(size=n)), torch.tensor(g.normal(size=n)))


def test_paper_mixing_inputs_in_models():
    """The shipped models use the world averages quoted in the paper."""
    gold = json.load(open(f"{GOLDEN_DIR}/paper_values.json"))["mixing_inputs"]
    for name in ("d0_k3pi_2chain", "d0_k3pi_full", "d0_k3pi_full_nodedup"):
        m = tdamp.load_model(model_path(name))
        assert m.x == gold["x"] and m.y == gold["y"]


@pytest.mark.parametrize("x,y", [(0.0049, 0.0061), (0.3, -0.2), (-0.5, 0.4)])
def test_rate_equals_two_state_time_evolution(x, y):
    """2 |<f|D0(t)>|^2 from the effective Hamiltonian of the D0-D0bar system,
    with mass eigenstates D1,2 = (D0 +- D0bar)/sqrt2, x = (m1-m2)/Gamma and
    y = (Gamma1-Gamma2)/(2 Gamma), equals Eq. (mix) times e^{-Gamma t}."""
    gamma = 1 / 0.4101
    m1, m2 = 1.0 + x * gamma / 2, 1.0 - x * gamma / 2
    g1, g2 = gamma * (1 + y), gamma * (1 - y)
    lam = np.array([m1 - 0.5j * g1, m2 - 0.5j * g2])
    V = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    H = V @ np.diag(lam) @ np.linalg.inv(V)
    A = _rand_complex(4, 1)
    Ab = _rand_complex(4, 2)
    for k, t in enumerate([0.05, 0.4, 1.3, 3.0]):
        psi = scipy.linalg.expm(-1j * H * t) @ np.array([1.0, 0.0])
        amp = psi[0] * complex(A[k]) + psi[1] * complex(Ab[k])
        R, _ = tdamp.rate_literal(A[k:k + 1], Ab[k:k + 1], torch.tensor([t], dtype=F64),
                                  torch.tensor(x, dtype=F64), torch.tensor(y, dtype=F64), gamma)
        assert abs(float(R[0]) - 2 * abs(amp) ** 2) <= 1e-12 * 2 * abs(amp) ** 2


def test_literal_equals_factorised_and_nonnegative():
    A, Ab = _rand_complex(10000, 3), _rand_complex(10000, 4)
    t = torch.tensor(np.random.default_rng(5).exponential(0.4101, 10000))
    for x, y in ((0.0049, 0.0061), (0.2, -0.3)):
        x, y = torch.tensor(x, dtype=F64), torch.tensor(y, dtype=F64)
        R1, B1 = tdamp.rate_literal(A, Ab, t, x, y, 1 / 0.4101)
        R2, B2 = tdamp.rate_factorised(A, Ab, t, x, y, 1 / 0.4101)
        scale = 2 * (A.abs() + Ab.abs()) ** 2
        assert float(((B1 - B2).abs() / scale).max()) < 1e-13
        assert bool(torch.all(B2 >= 0))


def test_rate_limits():
    A, Ab = _rand_complex(100, 6), _rand_complex(100, 7)
    t = torch.linspace(0, 3, 100, dtype=F64)
    gamma = 1 / 0.4101
    z = torch.tensor(0.0, dtype=F64)
    R, _ = tdamp.rate_literal(A, Ab, t, z, z, gamma)
    assert torch.allclose(R, 2 * A.abs() ** 2 * torch.exp(-gamma * t), rtol=1e-14, atol=0)
    x, y = torch.tensor(0.0049, dtype=F64), torch.tensor(0.0061, dtype=F64)
    R, _ = tdamp.rate_literal(A, torch.zeros_like(Ab), t, x, y, gamma)
    expect = A.abs() ** 2 * (torch.cosh(y * gamma * t) + torch.cos(x * gamma * t)) * torch.exp(-gamma * t)
    assert torch.allclose(R, expect, rtol=1e-14, atol=0)


@pytest.mark.parametrize("x,y", [(0.0049, 0.0061), (0.3, -0.2), (0.0, 0.9)])
def test_time_integrals_against_quadrature(x, y):
    gamma = 1 / 0.4101
    # e^{-G t} cosh / sinh(y G t) written as half sums of exponentials to avoid overflow
    funcs = (lambda t: 0.5 * (math.exp(-(1 - y) * gamma * t) + math.exp(-(1 + y) * gamma * t)),
             lambda t: math.exp(-gamma * t) * math.cos(x * gamma * t),
             lambda t: 0.5 * (math.exp(-(1 - y) * gamma * t) - math.exp(-(1 + y) * gamma * t)),
             lambda t: math.exp(-gamma * t) * math.sin(x * gamma * t))
    closed = tdamp.time_integrals(x, y, gamma)
    for f, c in zip(funcs, closed):
        q, err = scipy.integrate.quad(f, 0, math.inf, epsabs=1e-15, epsrel=1e-13, limit=400)
        assert abs(q - c) <= 1e-11 * max(abs(c), 1e-3)


def test_norm_integrand_is_time_integral_of_rate():
    A, Ab = _rand_complex(5, 8), _rand_complex(5, 9)
    gamma, x, y = 1 / 0.4101, 0.04, 0.07
    f = tdamp.norm_integrand(A, Ab, torch.tensor(x, dtype=F64), torch.tensor(y, dtype=F64), gamma)
    for k in range(5):
        def r(t):
            R, _ = tdamp.rate_literal(A[k:k + 1], Ab[k:k + 1], torch.tensor([t], dtype=F64),
                                      torch.tensor(x, dtype=F64), torch.tensor(y, dtype=F64), gamma)
            return float(R[0])
        q, _ = scipy.integrate.quad(r, 0, math.inf, epsabs=0, epsrel=1e-12, limit=400)
        assert abs(q - float(f[k])) <= 1e-10 * abs(q)


@pytest.mark.parametrize("name", ["d0_k3pi_2chain", "d0_k3pi_full"])
def test_bose_symmetry(name):
    m = tdamp.load_model(model_path(name))
    ev = torch.from_numpy(samples.flat_phase_space(2000, samples.rng(70, 0)))
    ev_swap = ev[:, [0, 3, 2, 1], :]
    a1 = tdamp.chain_amplitudes(m, ev, m.default_params())
    a2 = tdamp.chain_amplitudes(m, ev_swap, m.default_params())
    scale = a1.abs().max(dim=0).values
    assert bool(torch.all((a1 - a2).abs().max(dim=0).values <= 1e-12 * scale))


def test_chain_factorises_into_spin_and_lineshapes():
    """A chain amplitude divided by its lineshapes is the Bose sum of spin
    factors, independent of the resonance parameters."""
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    ev = torch.from_numpy(samples.flat_phase_space(500, samples.rng(71, 0)))
    p0 = m.default_params()
    p1 = p0.clone()
    p1[4:10] = p1[4:10] * torch.tensor([1.01, 0.9, 0.99, 1.2, 1.02, 0.8], dtype=F64)
    for p in (p0, p1):
        a = tdamp.chain_amplitudes(m, ev, p)
        # CF K*rho S-wave: K*(0,1) rho(2,3) plus the swapped ordering
        tot = torch.zeros(500, dtype=torch.complex128)
        for perm in ([0, 1, 2, 3], [0, 3, 2, 1]):
            e = ev[:, perm]
            S, (s1, s2) = tdamp.spin_factor("VV_S", [e[:, i] for i in range(4)], m)
            bw1 = tdamp.breit_wigner(s1, p[4], p[5], m.resonances[0], m.r_res)
            bw2 = tdamp.breit_wigner(s2, p[6], p[7], m.resonances[1], m.r_res)
            tot = tot + S * bw1 * bw2
        assert torch.allclose(a[:, 0], tot, rtol=1e-13, atol=0)


def test_gram_hermitian_psd_and_quadratic_form():
    m = tdamp.load_model(model_path("d0_k3pi_full"))
    ev = torch.from_numpy(samples.flat_phase_space(3000, samples.rng(72, 0)))
    p = m.default_params()
    I = tdamp.component_gram(m, ev, p)
    assert torch.allclose(I, I.conj().T, rtol=0, atol=1e-14 * float(I.abs().max()))
    ev_min = float(torch.linalg.eigvalsh(I).min())
    assert ev_min >= -1e-12 * float(I.abs().max())
    coef, *_ = tdamp._unpack(m, p)
    selA = torch.tensor([c.amp == "A" for c in m.chains])
    cA = torch.where(selA, coef, torch.zeros_like(coef))
    A, _ = tdamp.amplitudes(m, ev, p)
    quad = (cA.conj() @ I @ cA).real
    assert abs(float(quad) - float((A.abs() ** 2).mean())) <= 1e-12 * float(quad)
