"""GPU event generation (tdmix_generate) against the oracle:

* the device Philox4x32-10 equals the oracle's bit for bit (known-answer
  vectors and random counters and keys);
* flat four-body phase space: four-momentum conservation and mass shells to
  rounding, and the five projections of Sec. 3.2 indistinguishable from the
  host GENBOD generator (binned chi-square);
* time-dependent pseudo-events of the model: the five projections against
  flat phase space weighted by the oracle's time-integrated rate, and the
  decay-time distribution against the oracle's rate integrated over each
  time bin (the analogue of the paper's Fig. 3 comparison, with the oracle
  in place of the paper's second implementation); chi-square p-values and
  mean pulls are printed;
* the sample depends only on (seed, stream): repeated calls agree bitwise."""
import json
import os

import numpy as np
import pytest
import torch
from scipy import integrate, stats

from conftest import GOLDEN_DIR, model_path
from oracle import tdamp
from oracle.philox import philox4x32_10
from paper_1702_06735_gb300 import samples
from workloads import binned_chi2, projections

pytestmark = pytest.mark.gpu

M = samples.FINAL_STATE_MASSES
RANGES = [(M[0] + M[1], samples.M_D - M[2] - M[3]), (M[2] + M[3], samples.M_D - M[0] - M[1]), (-1, 1), (-1, 1),
          (-np.pi, np.pi)]
NAMES = ["m12", "m34", "cos12", "cos34", "phi"]


def test_device_philox_matches_oracle():
    from paper_1702_06735_gb300.tdmix import test_philox
    with open(os.path.join(GOLDEN_DIR, "philox4x32_10_kat.json")) as f:
        for v in json.load(f)["vectors"]:
            c, k = [int(x, 16) for x in v["counter"]], [int(x, 16) for x in v["key"]]
            assert test_philox(c, k) == tuple(int(x, 16) for x in v["out"])
    g = np.random.default_rng(1)
    for _ in range(200):
        c = [int(x) for x in g.integers(0, 2 ** 32, 4)]
        k = [int(x) for x in g.integers(0, 2 ** 32, 2)]
        assert test_philox(c, k) == philox4x32_10(c, k)


def test_flat_phase_space():
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix("d0_k3pi_2chain", "fp64")
    n = 200_000
    p4, _, info = c.generate(n, seed=11, stream=3, flat=True, with_times=False)
    p4 = p4.cpu().numpy()
    tot = p4.sum(axis=1)
    assert np.abs(tot[:, 0] - samples.M_D).max() <= 1e-12
    assert np.abs(tot[:, 1:]).max() <= 1e-12
    m2 = p4[..., 0] ** 2 - (p4[..., 1:] ** 2).sum(-1)
    assert np.abs(m2 - np.array(M) ** 2).max() <= 1e-12
    host = samples.flat_phase_space(400_000, samples.rng(5, 77))
    pg, ph = projections(p4), projections(host)
    for j, name in enumerate(NAMES):
        chi2, dof = binned_chi2(pg[:, j], ph[:, j], np.ones(len(ph)), 40, RANGES[j])
        p = stats.chi2.sf(chi2, dof)
        print(f"\nflat {name}: chi2/dof {chi2:.1f}/{dof}, p = {p:.3f}")
        assert p > 1e-4
    a, _, _ = c.generate(1000, seed=11, stream=3, flat=True, with_times=False)
    b, _, _ = c.generate(1000, seed=11, stream=4, flat=True, with_times=False)
    assert torch.equal(a, torch.from_numpy(p4[:1000]).to(a.device)) and not torch.equal(a, b)
    c.close()


@pytest.mark.parametrize("name,n_gen,n_ref", [("d0_k3pi_2chain", 300_000, 600_000), ("d0_k3pi_full", 100_000, 200_000)])
def test_model_events_against_oracle(name, n_gen, n_ref):
    from paper_1702_06735_gb300.tdmix import TDMix
    m = tdamp.load_model(model_path(name))
    par = m.default_params().numpy()
    c = TDMix(name, "fp32")
    p4, t, info = c.generate(n_gen, seed=2024, stream=1, params=par)
    p4, t = p4.cpu().numpy(), t.cpu().numpy()
    a2, t2, _ = c.generate(2000, seed=2024, stream=1, params=par)
    c.close()
    assert np.array_equal(a2.cpu().numpy(), p4[:2000]) and np.array_equal(t2.cpu().numpy(), t[:2000])
    print(f"\n{name}: envelope {info['envelope']:.4g}, {info['candidates']} candidates, "
          f"efficiency {info['efficiency']:.4f}")
    # reference: flat phase space weighted by the oracle's time-integrated rate
    flat = samples.flat_phase_space(n_ref, samples.rng(6, 88))
    pt = torch.from_numpy(par)
    with torch.no_grad():
        A, Ab = tdamp.amplitudes(m, torch.from_numpy(flat), pt)
        w = tdamp.norm_integrand(A, Ab, float(par[-2]), float(par[-1]), m.gamma).numpy()
    pg, pr = projections(p4), projections(flat)
    for j, nm in enumerate(NAMES):
        chi2, dof = binned_chi2(pg[:, j], pr[:, j], w, 40, RANGES[j])
        p = stats.chi2.sf(chi2, dof)
        mg, mr = pg[:, j].mean(), np.average(pr[:, j], weights=w)
        var_r = np.average((pr[:, j] - mr) ** 2, weights=w) * (w ** 2).sum() / w.sum() ** 2
        pull = (mg - mr) / np.sqrt(pg[:, j].var() / len(pg) + var_r)
        print(f"{name} {nm}: chi2/dof {chi2:.1f}/{dof}, p = {p:.3f}, mean pull {pull:+.2f}")
        assert p > 1e-4 and abs(pull) < 4
    # decay times: the oracle's rate averaged over phase space, integrated per bin
    with torch.no_grad():
        aa = float((A.abs() ** 2 + Ab.abs() ** 2).mean())
        bb = float((A.abs() ** 2 - Ab.abs() ** 2).mean())
        cr = float((A * Ab.conj()).real.mean())
        ci = float((A * Ab.conj()).imag.mean())
    x, y, G = float(par[-2]), float(par[-1]), m.gamma

    def f(tt):
        return np.exp(-G * tt) * (aa * np.cosh(y * G * tt) + bb * np.cos(x * G * tt)
                                  - 2 * cr * np.sinh(y * G * tt) - 2 * ci * np.sin(x * G * tt))
    edges = np.linspace(0.0, 8 * m.tau, 33)
    prob = np.array([integrate.quad(f, a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    prob /= integrate.quad(f, 0, np.inf)[0]
    obs, _ = np.histogram(t, bins=edges)
    exp = prob * len(t)
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    p = stats.chi2.sf(chi2, len(exp) - 1)
    print(f"{name} t: chi2/dof {chi2:.1f}/{len(exp) - 1}, p = {p:.3f}")
    assert p > 1e-4
    assert t.min() >= 0


def test_prescreen_gives_the_double_precision_sample():
    """Weighing candidates in single precision first (with an error band,
    the double-precision weight deciding inside it and for every candidate
    that could be the largest weight) gives exactly the sample of weighing
    every candidate in double precision."""
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix("d0_k3pi_full", "fp32")
    par = c.default_params()
    a, ta, ia = c.generate(40_000, seed=5, stream=2, params=par)
    b, tb, ib = c.generate(40_000, seed=5, stream=2, params=par, fp64_only=True)
    c.close()
    assert ia["envelope"] == ib["envelope"] and ia["candidates"] == ib["candidates"]
    assert torch.equal(a, b) and torch.equal(ta, tb)
