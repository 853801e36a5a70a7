"""Background (an extension the paper leaves out, Sec. 4) through the C ABI,
against the oracle: each data event's density is (1 - f) R / N + f B with B
flat in the normalised phase space and e^{-t/tau_b}/tau_b in the decay time
(folded with the resolution when the model has one).  The library runs the
MC pass, forms N, then the data pass of the mixture (runtime-table kernels,
fp64).  Tolerances as for the fp64 path: 1e-12 relative in the NLL, 1e-12 of
each gradient component's cancellation-free scale."""
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


def background_model(f=0.2, tau_b=0.6, sigma=0.0) -> dict:
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["background"] = {"fraction": f, "tau": tau_b}
    if sigma > 0:
        d["time_resolution"] = sigma
    d["name"] = "d0_k3pi_2chain_background"
    return d


@functools.lru_cache(maxsize=None)
def mixture_workload(n_data: int, n_mc: int, wid: int, f: float, tau_b: float, sigma: float):
    """Signal by accept/reject on the oracle's unfolded rate, background flat
    in phase space with exponential times, mixed in the proportion f; the
    measured times smeared by sigma (seeded)."""
    d = background_model(f, tau_b, sigma)
    base = tdamp.load_model(model_path("d0_k3pi_2chain"))
    g = np.random.default_rng(wid + 7)
    nb = int(g.binomial(n_data, f))
    sig, ts, _ = samples.generate_time_dependent(n_data - nb, samples.rng(wid, samples.STREAM_DATA),
                                                 oracle_rate_fn(base), base.gamma, base.y, pilot=20_000,
                                                 batch=1 << 15)
    bkg = samples.flat_phase_space(nb, samples.rng(wid, 7))
    tb = g.exponential(tau_b, nb)
    data = np.concatenate([sig, bkg])
    t = np.concatenate([ts, tb])
    if sigma > 0:
        t = t + sigma * g.standard_normal(n_data)
    mc = samples.flat_phase_space(n_mc, samples.rng(wid, samples.STREAM_MC))
    return d, tdamp.load_model(d), data, t, mc


@pytest.mark.parametrize("sigma", [0.0, 0.045])
def test_background_matches_oracle(sigma):
    from paper_1702_06735_gb300.tdmix import TDMix
    d, m, data, t, mc = mixture_workload(1300, 8_001, 6, 0.2, 0.6, sigma)
    c = TDMix(d, "fp32")
    assert c.kernel_path == "generic"
    c.load_events(data, t, mc)
    p = perturbed_params(m, 41)
    v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p)
    v, g = c.nll(p)
    assert abs(v - v0) <= 1e-12 * abs(v0)
    S = grad_scale(m, data, t, mc, p)
    err = np.abs(g - g0.numpy()) / S
    print(f"\nbackground, sigma = {sigma}: NLL rel err {abs(v / v0 - 1):.2e}, gradient max err / scale {err.max():.2e}")
    assert err.max() <= 1e-12, err
    # the signal rates and N are those of the signal model
    R, N = c.event_rates(p)
    with torch.no_grad():
        R0 = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), torch.as_tensor(p)).numpy()
        N0 = float(tdamp.normalisation(m, torch.from_numpy(mc), torch.as_tensor(p)))
    assert abs(N / N0 - 1) <= 1e-12
    assert np.max(np.abs(R - R0) / np.abs(R0).max()) <= 1e-12


def test_background_fraction_is_recovered_in_the_likelihood():
    """The NLL as a function of the model's background fraction is smallest
    near the fraction the sample was made with (a coarse scan)."""
    from paper_1702_06735_gb300.tdmix import TDMix
    _, _, data, t, mc = mixture_workload(6000, 40_001, 8, 0.3, 0.6, 0.0)
    fs = [0.1, 0.2, 0.3, 0.4, 0.5]
    vals = []
    for f in fs:
        c = TDMix(background_model(f, 0.6), "fp64")
        c.load_events(data, t, mc)
        vals.append(c.nll(c.default_params(), grad=False)[0])
        c.close()
    assert fs[int(np.argmin(vals))] in (0.2, 0.3, 0.4)
