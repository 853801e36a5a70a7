"""Pins of the oracle's lineshapes and barrier factors (building blocks of
Sec. 3) against closed forms and limits fixed by the mathematics."""
import math

import pytest
import torch

from oracle import tdamp

F64 = torch.float64
M_K, M_PI = 0.493677, 0.13957


def _res(shape, m0, g0, L=1, dm=(M_K, M_PI)):
    return tdamp.Resonance("R", m0, g0, shape, L, dm)


@pytest.mark.parametrize("shape,m0,g0,L,dm", [
    ("MDW", 0.89555, 0.0473, 1, (M_K, M_PI)),
    ("MDW", 0.77526, 0.1491, 1, (M_PI, M_PI)),
    ("MDW", 0.78266, 0.00868, 1, (M_PI, M_PI)),
    ("MDW", 1.27, 0.185, 2, (M_PI, M_PI)),
    ("CONST", 1.230, 0.420, 0, (0, 0)),
])
def test_bw_pole_modulus_and_phase(shape, m0, g0, L, dm):
    """At s = m0^2 the amplitude is i / (m0 Gamma0): modulus 1/(m0 Gamma0), phase +pi/2."""
    bw = tdamp.breit_wigner(torch.tensor([m0 * m0], dtype=F64), m0, g0, _res(shape, m0, g0, L, dm), 1.5)[0]
    assert abs(abs(bw) - 1.0 / (m0 * g0)) <= 1e-13 / (m0 * g0)
    assert abs(math.atan2(bw.imag, bw.real) - math.pi / 2) < 1e-13


def test_mdw_width_at_pole_and_threshold_power():
    """Gamma(m0^2) = Gamma0; near threshold Gamma(s) ~ q^(2L+1)."""
    for L, dm in ((1, (M_K, M_PI)), (2, (M_PI, M_PI))):
        m0, g0 = 0.9, 0.05
        assert abs(float(tdamp.mass_dependent_width(torch.tensor(m0 * m0, dtype=F64), torch.tensor(m0, dtype=F64),
                                                    torch.tensor(g0, dtype=F64), L, *dm, 1.5)) - g0) < 1e-16
        thr = (dm[0] + dm[1]) ** 2
        # q^2 is linear in (s - thr) near threshold, so Gamma ~ (s - thr)^((2L+1)/2)
        s1 = torch.tensor(thr * (1 + 1e-7), dtype=F64)
        s2 = torch.tensor(thr * (1 + 4e-7), dtype=F64)
        g1 = tdamp.mass_dependent_width(s1, torch.tensor(m0, dtype=F64), torch.tensor(g0, dtype=F64), L, *dm, 1.5)
        g2 = tdamp.mass_dependent_width(s2, torch.tensor(m0, dtype=F64), torch.tensor(g0, dtype=F64), L, *dm, 1.5)
        assert abs(float(g2 / g1) / 4 ** ((2 * L + 1) / 2) - 1) < 1e-5


def test_const_width_half_maximum_points():
    """For a constant width |BW|^2 falls to half its peak at s = m0^2 +- m0 Gamma0."""
    m0, g0 = 1.23, 0.42
    r = _res("CONST", m0, g0, 0)
    s = torch.tensor([m0 * m0, m0 * m0 - m0 * g0, m0 * m0 + m0 * g0], dtype=F64)
    bw2 = tdamp.breit_wigner(s, m0, g0, r, 1.5).abs() ** 2
    assert abs(float(bw2[1] / bw2[0]) - 0.5) < 1e-14
    assert abs(float(bw2[2] / bw2[0]) - 0.5) < 1e-14


def test_bw_far_from_pole():
    """Far from the pole |BW| -> 1/|m0^2 - s| up to O(m0 Gamma / |m0^2 - s|)."""
    m0, g0 = 0.77526, 0.1491
    r = _res("MDW", m0, g0, 1, (M_PI, M_PI))
    s = torch.tensor([0.1, 3.0], dtype=F64)
    bw = tdamp.breit_wigner(s, m0, g0, r, 1.5)
    rel = (bw.abs() * (m0 * m0 - s).abs() - 1).abs()
    gam = tdamp.mass_dependent_width(s, torch.tensor(m0, dtype=F64), torch.tensor(g0, dtype=F64), 1, M_PI, M_PI, 1.5)
    assert torch.all(rel <= (m0 * gam / (m0 * m0 - s).abs()) ** 2)


def test_blatt_weisskopf_limits():
    z0 = torch.tensor([0.0], dtype=F64)
    assert float(tdamp.blatt_weisskopf(0, z0, 1.0)) == 1.0
    assert float(tdamp.blatt_weisskopf(1, z0, 1.0)) == 1.0
    assert abs(float(tdamp.blatt_weisskopf(2, z0, 1.0)) - 1.0 / 3.0) < 1e-16
    big = torch.tensor([1e12], dtype=F64)
    assert abs(float(tdamp.blatt_weisskopf(1, big, 1.0) * big.sqrt()) - 1) < 1e-6
    assert abs(float(tdamp.blatt_weisskopf(2, big, 1.0) * big) - 1) < 1e-5


def test_blatt_weisskopf_matches_von_hippel_quigg_ratio():
    """z^(L/2) F_L(z) is proportional to the von Hippel-Quigg barrier factor
    B_1 = sqrt(2z/(1+z)), B_2 = sqrt(13 z^2 / (9 + 3z + z^2))."""
    q2 = torch.tensor([0.01, 0.1, 0.4, 2.0], dtype=F64)
    z = q2 * 1.5 ** 2
    b1 = torch.sqrt(2 * z / (1 + z))
    b2 = torch.sqrt(13 * z * z / (9 + 3 * z + z * z))
    f1 = tdamp.blatt_weisskopf(1, q2, 1.5) * z.sqrt()
    f2 = tdamp.blatt_weisskopf(2, q2, 1.5) * z
    assert torch.allclose(f1 / b1, (f1 / b1)[0].expand(4), rtol=1e-14, atol=0)
    assert torch.allclose(f2 / b2, (f2 / b2)[0].expand(4), rtol=1e-14, atol=0)


def test_breakup_momentum_two_body_closed_form():
    """q for K* -> K pi equals the momentum of either daughter in the rest frame,
    from energy conservation E_K + E_pi = sqrt(s)."""
    s = torch.tensor([0.8, 1.2], dtype=F64)
    q = tdamp.breakup_q2(s, M_K ** 2, M_PI ** 2).sqrt()
    e = torch.sqrt(q * q + M_K ** 2) + torch.sqrt(q * q + M_PI ** 2)
    assert torch.allclose(e, s.sqrt(), rtol=1e-14, atol=0)


def _phase_space_density(s, ma, mb):
    """Two-body phase-space density of a system of mass sqrt(s) decaying to
    masses ma, mb, up to a constant: in the rest frame
    Phi_2 = int d^3p / (4 E_a E_b) delta(sqrt(s) - E_a - E_b)
          = 4 pi p^2 / (4 E_a E_b |d(E_a + E_b)/dp|) at the root p = q.
    The root is found by bisection on energy conservation and the Jacobian
    by a central difference, so neither uses a closed form of q."""
    rs = math.sqrt(s)

    def etot(p):
        return math.sqrt(p * p + ma * ma) + math.sqrt(p * p + mb * mb)
    lo, hi = 0.0, rs
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if etot(mid) < rs:
            lo = mid
        else:
            hi = mid
    q = 0.5 * (lo + hi)
    h = 1e-6 * q
    jac = (etot(q + h) - etot(q - h)) / (2 * h)
    ea, eb = math.sqrt(q * q + ma * ma), math.sqrt(q * q + mb * mb)
    return math.pi * q * q / (ea * eb * jac), q


def _penetration(L, z):
    """von Hippel-Quigg centrifugal-barrier penetration factors B_L(z)^2
    (Phys. Rev. D 5 (1972) 624), including their q^(2L) behaviour."""
    return {0: 1.0, 1: 2 * z / (1 + z), 2: 13 * z * z / (9 + 3 * z + z * z)}[L]


@pytest.mark.parametrize("L,m0,g0,dm", [
    (1, 0.89555, 0.0473, (M_K, M_PI)),    # K*(892) -> K pi
    (1, 0.77526, 0.1491, (M_PI, M_PI)),   # rho(770) -> pi pi
    (2, 1.2755, 0.1867, (M_PI, M_PI)),    # a D-wave resonance -> pi pi
])
@pytest.mark.parametrize("sqrt_s_over_m0", [0.8, 0.93, 1.07, 1.4])
def test_mdw_width_off_pole_is_phase_space_times_barrier(L, m0, g0, dm, sqrt_s_over_m0):
    """Away from the pole the mass-dependent width is the pole width scaled
    by the two-body phase-space density and by the centrifugal-barrier
    penetration of the partial wave L:
        Gamma(s) / Gamma0 = [Phi_2(s) / Phi_2(m0^2)] [B_L(q r)^2 / B_L(q0 r)^2].
    Phi_2 ~ q / sqrt(s) carries the factor m0 / sqrt(s) and one power of
    q / q0; B_L^2 ~ q^(2L) F_L^2 carries the rest.  A width with sqrt(s)/m0
    in place of m0/sqrt(s), or with an unsquared barrier ratio, fails here
    (both differ by tens of percent at these points)."""
    r = 1.5
    s = (sqrt_s_over_m0 * m0) ** 2
    if math.sqrt(s) <= dm[0] + dm[1]:
        pytest.skip("below threshold")
    phi, q = _phase_space_density(s, *dm)
    phi0, q0 = _phase_space_density(m0 * m0, *dm)
    expected = g0 * (phi / phi0) * _penetration(L, (q * r) ** 2) / _penetration(L, (q0 * r) ** 2)
    got = float(tdamp.mass_dependent_width(torch.tensor(s, dtype=F64), torch.tensor(m0, dtype=F64),
                                           torch.tensor(g0, dtype=F64), L, *dm, r))
    assert abs(got / expected - 1) < 1e-8, (got, expected)
    # the two plausible mistakes are far outside the tolerance at these points
    swapped = got * s / (m0 * m0)
    unsquared = got * math.sqrt(_penetration(L, (q0 * r) ** 2) / _penetration(L, (q * r) ** 2)
                                * (q / q0) ** (2 * L))
    assert abs(swapped / expected - 1) > 1e-3 and abs(unsquared / expected - 1) > 1e-3


def test_mdw_width_values_k_star():
    """Literal values for K*(892) -> K pi (L = 1, r = 1.5 GeV^-1), worked by
    hand from energy conservation, E_K = (s + m_K^2 - m_pi^2) / (2 sqrt s),
    q^2 = E_K^2 - m_K^2: at the pole (m0 = 0.89555 GeV) q0 = 0.290823 GeV;
    at sqrt(s) = 0.80 GeV, q = 0.219187 GeV and
    Gamma = 0.0473 x (0.89555/0.80) x (q/q0)^3 x (1 + (q0 r)^2)/(1 + (q r)^2)
          = 0.0473 x 1.119437 x 0.428116 x 1.074184 = 0.0243501 GeV;
    at sqrt(s) = 1.00 GeV, q = 0.361901 GeV and
    Gamma = 0.0473 x 0.89555 x 1.927007 x 0.919373 = 0.0750457 GeV."""
    m0, g0 = 0.89555, 0.0473
    for rs, want in ((0.80, 0.0243501), (1.00, 0.0750457)):
        got = float(tdamp.mass_dependent_width(torch.tensor(rs * rs, dtype=F64), torch.tensor(m0, dtype=F64),
                                               torch.tensor(g0, dtype=F64), 1, M_K, M_PI, 1.5))
        assert abs(got / want - 1) < 5e-6, (rs, got, want)


def test_mdw_width_vanishes_below_threshold_with_finite_gradient():
    """A quasi-two-body state given a mass-dependent width to its sub-resonance
    at the nominal mass and the bachelor (the a1 to rho0 pi-): below that
    threshold Gamma(s) = 0, so BW = 1/(m0^2 - s), and the derivatives in m0
    and Gamma0 are those of that real lineshape (finite), not NaN."""
    import torch
    from oracle import tdamp
    res = tdamp.Resonance("a1", 1.23, 0.42, "MDW", 0, (0.77526, 0.13957), True)
    s = torch.tensor([0.5, 0.8, 1.2, 1.6], dtype=torch.float64)   # the first two below (0.915 GeV)^2
    m0 = torch.tensor(1.23, dtype=torch.float64, requires_grad=True)
    g0 = torch.tensor(0.42, dtype=torch.float64, requires_grad=True)
    bw = tdamp.breit_wigner(s, m0, g0, res, 1.5)
    below = s < (0.77526 + 0.13957) ** 2
    assert torch.equal(bw[below], (1.0 / (m0 * m0 - s[below])).to(torch.complex128))
    dm, dg = torch.autograd.grad(bw.real.sum() + bw.imag.sum(), (m0, g0))
    assert torch.isfinite(dm) and torch.isfinite(dg)
    # below threshold d(1/(m0^2 - s))/dm0 = -2 m0 / (m0^2 - s)^2, and nothing depends on Gamma0
    m0_, s_ = 1.23, s[below]
    ref = float((-2 * m0_ / (m0_ ** 2 - s_) ** 2).sum())
    above = s[~below]
    dm_above = torch.autograd.grad((tdamp.breit_wigner(above, m0, g0, res, 1.5).real.sum()
                                    + tdamp.breit_wigner(above, m0, g0, res, 1.5).imag.sum()), m0)[0]
    assert abs(float(dm) - (ref + float(dm_above))) <= 1e-12 * abs(float(dm))
