"""Pins of the oracle's spin factors (Sec. 3 building blocks, Fig. 2
topologies): Lorentz invariance, rest-frame closed forms on events built
from angles, kinematic zeros and parity."""
import math

import numpy as np
import pytest
import torch

from oracle import tdamp
from paper_1702_06735_gb300 import samples

F64 = torch.float64
MD, MK, MPI = samples.M_D, samples.M_K, samples.M_PI
SPINS = ["VV_S", "VV_P", "VV_D", "AP_S", "NR"]


@pytest.fixture(scope="module")
def model():
    from conftest import model_path
    return tdamp.load_model(model_path("d0_k3pi_full"))


def _boost_z(p, beta):
    """Boost four-vectors (..., 4) along +z with velocity beta."""
    g = 1.0 / math.sqrt(1 - beta * beta)
    out = p.clone()
    out[..., 0] = g * (p[..., 0] + beta * p[..., 3])
    out[..., 3] = g * (p[..., 3] + beta * p[..., 0])
    return out


def _two_body(M, ma, mb, direction):
    """Rest-frame four-momenta of a, b for M -> a b with a along `direction`."""
    q = math.sqrt((M * M - (ma + mb) ** 2) * (M * M - (ma - mb) ** 2)) / (2 * M)
    n = torch.tensor(direction, dtype=F64)
    n = n / n.norm()
    pa = torch.cat([torch.tensor([math.sqrt(q * q + ma * ma)], dtype=F64), q * n])
    pb = torch.cat([torch.tensor([math.sqrt(q * q + mb * mb)], dtype=F64), -q * n])
    return pa, pb, q


def _vv_event(m1, m2, phi1, phi2):
    """D -> R1(K pi) R2(pi pi) with R1 along +z and both decays transverse."""
    p = math.sqrt((MD ** 2 - (m1 + m2) ** 2) * (MD ** 2 - (m1 - m2) ** 2)) / (2 * MD)
    a, b, q1 = _two_body(m1, MK, MPI, [math.cos(phi1), math.sin(phi1), 0])
    c, d, q2 = _two_body(m2, MPI, MPI, [math.cos(phi2), math.sin(phi2), 0])
    e1, e2 = math.sqrt(p * p + m1 * m1), math.sqrt(p * p + m2 * m2)
    a, b = _boost_z(a, p / e1), _boost_z(b, p / e1)
    c, d = _boost_z(c, -p / e2), _boost_z(d, -p / e2)
    return [x.unsqueeze(0) for x in (a, b, c, d)], p, q1, q2


def _bw_factor(L, q2, r):
    return float(tdamp.blatt_weisskopf(L, torch.tensor([q2], dtype=F64), r)[0])


@pytest.mark.parametrize("m1,m2,phi1,phi2", [(0.9, 0.77, 0.3, 1.4), (1.1, 0.5, -2.0, 0.7), (0.7, 0.95, 2.5, -0.4)])
def test_vv_rest_frame_closed_forms(model, m1, m2, phi1, phi2):
    p4, p, q1, q2 = _vv_event(m1, m2, phi1, phi2)
    fres = _bw_factor(1, q1 * q1, model.r_res) * _bw_factor(1, q2 * q2, model.r_res)
    expect = {
        "VV_S": -4 * q1 * q2 * math.cos(phi1 - phi2) * _bw_factor(0, p * p, model.r_parent),
        "VV_P": 8 * MD * p * q1 * q2 * math.sin(phi2 - phi1) * _bw_factor(1, p * p, model.r_parent),
        "VV_D": -16.0 / 3.0 * p * p * q1 * q2 * math.cos(phi1 - phi2) * _bw_factor(2, p * p, model.r_parent),
    }
    for spin, e in expect.items():
        S, (s1, s2) = tdamp.spin_factor(spin, p4, model)
        assert abs(float(S[0]) - e * fres) <= 1e-12 * abs(e * fres), spin
        assert abs(float(s1[0]) - m1 * m1) < 1e-13 and abs(float(s2[0]) - m2 * m2) < 1e-13


@pytest.mark.parametrize("M1,M2,c_mass", [(1.25, 0.78, MPI), (1.3, 0.9, MPI), (1.3, 0.77, MK)])
def test_cascade_rest_frame_closed_form(model, M1, M2, c_mass):
    """D -> R1 d, R1 -> R2 c, R2 -> a b, all along z: S = -4 p q2 gamma1 gamma2."""
    d_mass = MPI if c_mass == MK else MK
    a_mass, b_mass = MPI, MPI
    r2, c, k = _two_body(M1, M2, c_mass, [0, 0, 1])          # in R1 frame, R2 along +z
    a, b, q2 = _two_body(M2, a_mass, b_mass, [0, 0, 1])      # in R2 frame, a along +z
    beta2 = k / float(r2[0])
    a, b = _boost_z(a, beta2), _boost_z(b, beta2)
    r1, dd, p = _two_body(MD, M1, d_mass, [0, 0, 1])         # in D frame, R1 along +z
    beta1 = p / float(r1[0])
    a, b, c = _boost_z(a, beta1), _boost_z(b, beta1), _boost_z(c, beta1)
    g1 = float(r1[0]) / M1
    g2 = float(r2[0]) / M2
    expect = -4 * p * q2 * g1 * g2 * _bw_factor(1, p * p, model.r_parent) * _bw_factor(1, q2 * q2, model.r_res)
    S, (s1, s2) = tdamp.spin_factor("AP_S", [x.unsqueeze(0) for x in (a, b, c, dd)], model)
    assert abs(float(S[0]) - expect) <= 1e-12 * abs(expect)
    assert abs(float(s1[0]) - M1 * M1) < 1e-12 and abs(float(s2[0]) - M2 * M2) < 1e-12


def _random_lorentz(seed):
    g = np.random.default_rng(seed)
    beta = g.uniform(-0.55, 0.55, 3)
    b2 = beta @ beta
    gam = 1 / math.sqrt(1 - b2)
    Lb = np.eye(4)
    Lb[0, 0] = gam
    Lb[0, 1:] = Lb[1:, 0] = gam * beta
    Lb[1:, 1:] += (gam - 1) * np.outer(beta, beta) / b2
    q, _ = np.linalg.qr(g.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    R = np.eye(4)
    R[1:, 1:] = q
    return torch.tensor(R @ Lb, dtype=F64)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_spin_factors_lorentz_invariant(model, seed):
    ev = torch.from_numpy(samples.flat_phase_space(2000, samples.rng(50 + seed, 0)))
    Lam = _random_lorentz(seed)
    ev2 = ev @ Lam.T
    for spin in SPINS:
        for parts in ([0, 1, 2, 3], [2, 1, 3, 0], [2, 1, 0, 3]):
            S1, _ = tdamp.spin_factor(spin, [ev[:, i] for i in parts], model)
            S2, _ = tdamp.spin_factor(spin, [ev2[:, i] for i in parts], model)
            scale = S1.abs().max()
            assert float((S1 - S2).abs().max()) <= 1e-11 * float(scale) + 1e-300, spin


def test_p_and_d_wave_vanish_at_zero_breakup(model):
    """m1 + m2 = m_D: both resonances at rest, L = 0 and Q parallel to P_D."""
    m1 = 1.0
    m2 = MD - m1
    a, b, _ = _two_body(m1, MK, MPI, [0.3, 0.5, 0.8])
    c, d, _ = _two_body(m2, MPI, MPI, [-0.2, 0.9, 0.1])
    p4 = [x.unsqueeze(0) for x in (a, b, c, d)]
    S0, _ = tdamp.spin_factor("VV_S", p4, model)
    for spin in ("VV_P", "VV_D"):
        S, _ = tdamp.spin_factor(spin, p4, model)
        assert abs(float(S[0])) < 1e-14 * max(1.0, abs(float(S0[0])))


def test_p_wave_vanishes_for_coplanar_momenta(model):
    ev = samples.flat_phase_space(500, samples.rng(60, 0))
    # rotate every event so that p0 and p1 lie in the xz plane, then flatten y
    ev = torch.from_numpy(ev).clone()
    ev[..., 2] = 0.0
    # restore energies so all particles stay on shell in the projected event
    m = torch.tensor(samples.FINAL_STATE_MASSES, dtype=F64)
    ev[..., 0] = torch.sqrt((ev[..., 1:] ** 2).sum(-1) + m ** 2)
    S, _ = tdamp.spin_factor("VV_P", [ev[:, i] for i in range(4)], model)
    Sref, _ = tdamp.spin_factor("VV_S", [ev[:, i] for i in range(4)], model)
    assert float(S.abs().max()) <= 1e-13 * float(Sref.abs().max())


def test_parity(model):
    """Under p -> -p the scalar spin factors are unchanged and the P-wave
    (a pseudoscalar) changes sign."""
    ev = torch.from_numpy(samples.flat_phase_space(1000, samples.rng(61, 0)))
    evp = ev.clone()
    evp[..., 1:] = -evp[..., 1:]
    for spin, sign in (("VV_S", 1), ("VV_P", -1), ("VV_D", 1), ("AP_S", 1)):
        S1, _ = tdamp.spin_factor(spin, [ev[:, i] for i in range(4)], model)
        S2, _ = tdamp.spin_factor(spin, [evp[:, i] for i in range(4)], model)
        assert torch.allclose(S2, sign * S1, rtol=1e-12, atol=1e-14 * float(S1.abs().max()))


def test_t_vector_rest_frame_magnitude():
    """In the rest frame of P, t(P; a, b) = (0, 2 q) so t.t = -4 q^2."""
    ev = torch.from_numpy(samples.flat_phase_space(1000, samples.rng(62, 0)))
    a, b = ev[:, 0], ev[:, 1]
    P = a + b
    s = tdamp.mdot(P, P)
    t = tdamp.t_vector(P, a, b)
    q2 = tdamp.breakup_q2(s, tdamp.mdot(a, a), tdamp.mdot(b, b))
    assert torch.allclose(tdamp.mdot(t, t), -4 * q2, rtol=1e-11, atol=0)
