"""Decay-time resolution (an extension the paper leaves out, Sec. 4) through
the C ABI, against the oracle.

A model file with "time_resolution" sigma folds Eq. (mix) with a Gaussian
of width sigma in the measured time; the library evaluates it on the
runtime-table kernels in fp64 with the closed-form folds (Faddeeva
function), the oracle by quadrature.  Tolerances as for the fp64 path:
1e-12 of the cancellation-free scale of each rate and gradient component,
1e-12 relative in N and the NLL."""
import functools
import json

import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import grad_scale, oracle_rate_fn, perturbed_params

pytestmark = pytest.mark.gpu

SIGMA = 0.045  # ps


def resolution_model(sigma=SIGMA) -> dict:
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["time_resolution"] = sigma
    d["name"] = "d0_k3pi_2chain_resolution"
    return d


@functools.lru_cache(maxsize=None)
def resolution_workload(n_data: int, n_mc: int, wid: int):
    """True decay times by accept/reject on the unfolded oracle rate, then
    the measured times smeared by a seeded Gaussian of width SIGMA."""
    d = resolution_model()
    m = tdamp.load_model(d)
    base = tdamp.load_model(model_path("d0_k3pi_2chain"))
    data, t, _ = samples.generate_time_dependent(n_data, samples.rng(wid, samples.STREAM_DATA), oracle_rate_fn(base),
                                                 base.gamma, base.y, pilot=min(50_000, 20 * n_data), batch=1 << 15)
    t = t + SIGMA * np.random.default_rng(wid + 99).standard_normal(n_data)
    mc = samples.flat_phase_space(n_mc, samples.rng(wid, samples.STREAM_MC))
    return d, m, data, t, mc


def folded_rate_scale(m, data, t, p):
    """2 (sum_i |c_i a_i|)^2 K_cosh(t), K_cosh the fold of e^{-Gamma t'}
    cosh(y Gamma t'): a bound of |R| free of the cancellations between the
    terms of Eq. (mix)."""
    p = torch.as_tensor(p, dtype=torch.float64)
    coef, *_ = tdamp._unpack(m, p)
    a = tdamp.chain_amplitudes(m, torch.as_tensor(data), p)
    s = (a * coef).abs().sum(dim=1)
    n = len(t)
    one = torch.ones(n, dtype=torch.complex128)
    zero = torch.zeros(n, dtype=torch.complex128)
    tt = torch.as_tensor(t, dtype=torch.float64)
    kc = (tdamp.rate_resolved(one, zero, tt, 0.0, float(p[-1]), m.gamma, m.sigma_t)
          + tdamp.rate_resolved(zero, one, tt, 0.0, float(p[-1]), m.gamma, m.sigma_t)) / 2
    return (2 * s ** 2 * kc).numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_resolution_matches_oracle(precision):
    from paper_1702_06735_gb300.tdmix import TDMix
    d, m, data, t, mc = resolution_workload(1200, 9_001, 5)
    assert t.min() < 0  # measured times below zero occur
    c = TDMix(d, precision)
    assert c.kernel_path == "generic"
    c.load_events(data, t, mc)
    for seed, xy in ((31, None), (32, (0.3, -0.2))):
        p = perturbed_params(m, seed)
        if xy:
            p[-2], p[-1] = xy
        v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p)
        with torch.no_grad():
            R0 = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), torch.as_tensor(p)).numpy()
            N0 = float(tdamp.normalisation(m, torch.from_numpy(mc), torch.as_tensor(p)))
        R, N = c.event_rates(p)
        assert np.max(np.abs(R - R0) / folded_rate_scale(m, data, t, p)) <= 1e-12
        assert abs(N / N0 - 1) <= 1e-12
        v, g = c.nll(p)
        assert abs(v - v0) <= 1e-12 * abs(v0)
        S = grad_scale(m, data, t, mc, p)
        err = np.abs(g - g0.numpy()) / S
        print(f"\nresolution, x = {p[-2]:.4f}, y = {p[-1]:.4f}: NLL rel err {abs(v / v0 - 1):.2e}, "
              f"gradient max err / scale {err.max():.2e}")
        assert err.max() <= 1e-12, err


def test_resolution_domain_and_generation():
    """|x| Gamma sigma / sqrt 2 above 0.25 is refused; the device generator
    draws the same events as without the resolution and smears only their
    times, by a Gaussian of width sigma."""
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixError
    d, m, data, t, mc = resolution_workload(1200, 9_001, 5)
    c = TDMix(d, "fp64")
    c.load_events(data, t, mc)
    p = m.default_params().numpy()
    bad = p.copy()
    bad[-2] = 4.0
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -6
    base = TDMix("d0_k3pi_2chain", "fp64")
    n = 20_000
    p4r, tr, _ = c.generate(n, seed=11, stream=3, params=p)
    p4b, tb, _ = base.generate(n, seed=11, stream=3, params=p)
    assert torch.equal(p4r, p4b)
    dt = (tr - tb).cpu().numpy()
    assert abs(dt.mean()) <= 4 * SIGMA / np.sqrt(n)
    assert abs(dt.std() / SIGMA - 1) <= 0.03
