"""Model structures without a compiled specialisation (the runtime-table
kernels) against the oracle, through the C ABI.

The model the user composes here (Sec. 3) is the 2-chain model plus a
D-wave K*0 rho0 chain in Abar_f, a structure none of the shipped model files
has.  Tolerances as for the fp64 path: 1e-12 relative (per-event rates
relative to their cancellation-free scale, gradient components relative to
theirs)."""
import copy
import functools
import json

import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import grad_scale, oracle_rate_fn, perturbed_params, rate_scale, workload

pytestmark = pytest.mark.gpu


def composed_model() -> dict:
    d = json.load(open(model_path("d0_k3pi_2chain")))
    extra = copy.deepcopy(d["chains"][0])
    extra.update(name="CF K*0 rho0 D-wave", spin="VV_D", coef=[0.3, 0.1], float=True)
    d["chains"].append(extra)
    d["name"] = "d0_k3pi_2chain_plus_dwave"
    return d


@functools.lru_cache(maxsize=None)
def composed_workload(n_data: int, n_mc: int, wid: int):
    d = composed_model()
    m = tdamp.load_model(d)
    data, t, _ = samples.generate_time_dependent(n_data, samples.rng(wid, samples.STREAM_DATA), oracle_rate_fn(m),
                                                 m.gamma, m.y, pilot=min(50_000, 20 * n_data), batch=1 << 15)
    mc = samples.flat_phase_space(n_mc, samples.rng(wid, samples.STREAM_MC))
    return d, m, data, t, mc


def _oracle(m, data, t, mc, p, w=None):
    v, g = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p,
                              None if w is None else torch.from_numpy(w))
    with torch.no_grad():
        R = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), torch.as_tensor(p)).numpy()
        N = float(tdamp.normalisation(m, torch.from_numpy(mc), torch.as_tensor(p),
                                      None if w is None else torch.from_numpy(w)))
    return v, g.numpy(), R, N


def _ctx(model, precision, data, t, mc, w=None, generic=False):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(model, precision, generic=generic)
    c.load_events(data, t, mc, w)
    return c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_composed_model_matches_oracle(precision):
    """A structure that was not compiled in runs on the generic path (also
    when fp32 is asked for: that path computes in fp64) and equals the
    oracle: rates, N, NLL and the gradient of every parameter, with masses
    and widths moved.  Sizes span several tiles with ragged tails."""
    d, m, data, t, mc = composed_workload(1500, 12_345, 3)
    c = _ctx(d, precision, data, t, mc)
    assert c.kernel_path == "generic"
    p = perturbed_params(m, 21)
    v0, g0, R0, N0 = _oracle(m, data, t, mc, p)
    R, N = c.event_rates(p)
    sc = rate_scale(m, data, t, p)
    assert np.max(np.abs(R - R0) / sc) <= 1e-12
    assert abs(N / N0 - 1) <= 1e-12
    v, g = c.nll(p)
    assert abs(v - v0) <= 1e-12 * abs(v0)
    S = grad_scale(m, data, t, mc, p)
    err = np.abs(g - g0) / S
    print(f"\ngeneric ({precision} asked): NLL rel err {abs(v / v0 - 1):.2e}, gradient max err / scale {err.max():.2e}")
    assert err.max() <= 1e-12, err


def test_composed_model_norm_matrix_and_repeatability():
    d, m, data, t, mc = composed_workload(1500, 12_345, 3)
    c = _ctx(d, "fp64", data, t, mc)
    p = perturbed_params(m, 22)
    a = c.nll(p)
    b = c.nll(p)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])  # fixed summation order
    I = c.norm_matrix()
    Ich = tdamp.component_gram(m, torch.from_numpy(mc), torch.as_tensor(p)).numpy()
    comp = [c.chain_component(i) for i in range(len(m.chains))]
    ref = np.zeros_like(I)
    for i, ci in enumerate(comp):
        for k, ck in enumerate(comp):
            ref[ci, ck] = Ich[i, k]
    assert np.max(np.abs(I - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_generic_path_weighted_mc_and_tiny_samples():
    d, m, data, t, mc = composed_workload(1500, 12_345, 3)
    w = np.random.default_rng(5).uniform(0.5, 2.0, 300)
    p = perturbed_params(m, 23)
    for nd, nm, ww in ((1, 1, None), (3, 300, w), (257, 513, None)):
        c = _ctx(d, "fp64", data[:nd], t[:nd], mc[:nm], ww)
        v, g = c.nll(p)
        v0, g0, _, _ = _oracle(m, data[:nd], t[:nd], mc[:nm], p, ww)
        assert abs(v - v0) <= 1e-12 * max(1.0, abs(v0))
        S = grad_scale(m, data[:nd], t[:nd], mc[:nm], p, ww)
        assert np.max(np.abs(g - g0) / S) <= 1e-12


@pytest.mark.parametrize("name,nd,nm,wid", [("d0_k3pi_2chain", 1000, 10_000, 0), ("d0_k3pi_full", 777, 6_001, 1),
                                            ("d0_k3pi_full_nodedup", 777, 6_001, 1)])
def test_forced_generic_equals_specialised_fp64(name, nd, nm, wid):
    """The runtime-table kernels on a shipped structure reproduce the
    specialised fp64 kernels (both against the oracle's tolerance), also on
    device parameter vectors and in a batch."""
    from paper_1702_06735_gb300.tdmix import TDMix
    m, data, t, mc = workload(name, nd, nm, wid)
    cs = _ctx(name, "fp64", data, t, mc)
    cg = _ctx(name, "fp64", data, t, mc, generic=True)
    assert cs.kernel_path == "fp64" and cg.kernel_path == "generic"
    p = perturbed_params(m, 24)
    vs, gs = cs.nll(p)
    vg, gg = cg.nll(p)
    S = grad_scale(m, data, t, mc, p)
    assert abs(vg - vs) <= 2e-12 * abs(vs)
    assert np.max(np.abs(gg - gs) / S) <= 2e-12
    dev = torch.device("cuda")
    P = torch.from_numpy(np.stack([p, perturbed_params(m, 25)])).to(dev)
    out = torch.empty(2, dtype=torch.float64, device=dev)
    grad = torch.empty(2, len(p), dtype=torch.float64, device=dev)
    cg.nll_batch(P, out, grad)
    torch.cuda.synchronize()
    assert float(out[0]) == vg and np.array_equal(grad[0].cpu().numpy(), gg)
    v1, g1 = cs.nll(P[1].cpu().numpy())
    assert abs(float(out[1]) - v1) <= 2e-12 * abs(v1)


def test_generic_path_reports_invalid_parameters_and_refuses_what_it_lacks():
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixError
    d, m, data, t, mc = composed_workload(1500, 12_345, 3)
    c = _ctx(d, "fp64", data, t, mc)
    p = perturbed_params(m, 26)
    nc = len(m.chains)
    bad = p.copy()
    bad[2 * nc + 1] = -0.1           # a negative width
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -6
    bad = p.copy()
    bad[0] = float("nan")
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -5
    # device parameters are screened in the kernel: status in the result, NaN NLL
    dev = torch.device("cuda")
    bad = p.copy()
    bad[-1] = 1.5                    # |y| >= 1
    out = torch.empty(1, dtype=torch.float64, device=dev)
    c.nll_device(torch.from_numpy(bad).to(dev), out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()
    v, _ = c.nll(p)                  # the context stays usable
    assert np.isfinite(v)
    with pytest.raises(TDMixError) as e:
        c.set_gram("tensor")
    assert e.value.code == -8
    with pytest.raises(TDMixError) as e:
        c.generate(1000, seed=1, params=p)
    assert e.value.code == -8
    from paper_1702_06735_gb300.tdmix import TDMixServer
    with pytest.raises(TDMixError) as e:
        TDMixServer(d, "fp32", hbm_budget_bytes=1 << 28)
    assert e.value.code == -8
