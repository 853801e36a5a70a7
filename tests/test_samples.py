"""Checks of the seeded phase-space generator (GENBOD) and accept/reject."""
import math

import numpy as np
import pytest

from paper_1702_06735_gb300 import samples


def test_four_momentum_conservation_and_mass_shell():
    ev = samples.flat_phase_space(20000, samples.rng(90, 0))
    tot = ev.sum(axis=1)
    assert np.abs(tot[:, 0] - samples.M_D).max() < 1e-12
    assert np.abs(tot[:, 1:]).max() < 1e-12
    m2 = ev[..., 0] ** 2 - (ev[..., 1:] ** 2).sum(-1)
    assert np.abs(m2 - np.array(samples.FINAL_STATE_MASSES) ** 2).max() < 1e-12


def test_massless_phase_space_volume():
    """<raw weight> reproduces R_n = (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!) for
    massless particles, with R_n = 2^(n-2) pi^(n-1) / M * Tecm^(n-2)/(n-2)! * <prod p>."""
    M = 2.0
    for n in (3, 4, 5):
        b = samples.genbod(400_000, samples.rng(91, n), M=M, masses=(0.0,) * n)
        raw = b.weight * b.wt_max
        est = 2 ** (n - 2) * math.pi ** (n - 1) / M * M ** (n - 2) / math.factorial(n - 2) * raw.mean()
        err = 2 ** (n - 2) * math.pi ** (n - 1) / M * M ** (n - 2) / math.factorial(n - 2) * raw.std() / math.sqrt(len(raw))
        exact = (math.pi / 2) ** (n - 1) * (M * M) ** (n - 2) / (math.factorial(n - 1) * math.factorial(n - 2))
        assert abs(est - exact) < 4 * err


def test_three_body_dalitz_plot_is_flat():
    """Flat three-body phase space is uniform in (m12^2, m23^2) inside the
    kinematic boundary: equal-area cells get equal counts."""
    M, m = 1.86484, (0.493677, 0.13957, 0.13957)
    ev = samples.flat_phase_space(200_000, samples.rng(92, 0), M=M, masses=m)
    p12 = ev[:, 0] + ev[:, 1]
    p23 = ev[:, 1] + ev[:, 2]
    s12 = p12[:, 0] ** 2 - (p12[:, 1:] ** 2).sum(-1)
    s23 = p23[:, 0] ** 2 - (p23[:, 1:] ** 2).sum(-1)
    # a square fully inside the Dalitz region, split into 4x4 cells
    x0, y0, w = 0.9, 0.6, 0.4
    sel = (s12 > x0) & (s12 < x0 + w) & (s23 > y0) & (s23 < y0 + w)
    h, _, _ = np.histogram2d(s12[sel], s23[sel], bins=4, range=[[x0, x0 + w], [y0, y0 + w]])
    exp = h.mean()
    chi2 = ((h - exp) ** 2 / exp).sum()
    assert chi2 < 40  # 15 dof; p ~ 5e-4


def test_exponential_times_mean():
    t = samples.exponential_times(400_000, 2.5, samples.rng(93, 0))
    assert abs(t.mean() - 0.4) < 4 * 0.4 / math.sqrt(len(t))


def test_accept_reject_reproduces_target_time_density():
    """A rate exp(-G t) cosh(y G t) (no phase-space dependence) yields times
    whose mean is the ratio of the moments of that density."""
    G, y = 2.0, 0.3

    def rate(p4, t):
        return np.exp(-G * t) * np.cosh(y * G * t)
    p4, t, st = samples.generate_time_dependent(100_000, samples.rng(94, 0), rate, G, y,
                                                pilot=20000, batch=1 << 16)
    m1 = 0.5 * (1 / ((1 - y) * G) ** 2 + 1 / ((1 + y) * G) ** 2)
    m0 = 0.5 * (1 / ((1 - y) * G) + 1 / ((1 + y) * G))
    mean = m1 / m0
    assert abs(t.mean() - mean) < 5 * t.std() / math.sqrt(len(t))
    assert p4.shape == (100_000, 4, 4)


def test_seeded_streams_reproducible_and_distinct():
    a = samples.flat_phase_space(100, samples.rng(1, 0))
    b = samples.flat_phase_space(100, samples.rng(1, 0))
    c = samples.flat_phase_space(100, samples.rng(1, 1))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
