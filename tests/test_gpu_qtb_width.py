"""Mass-dependent widths of the quasi-two-body states (an extension; the
paper's model keeps them fixed, Sec. 4), against the oracle through the C ABI.

Reading: a quasi-two-body state R -> r c gets the mass-dependent width of a
two-body decay to the sub-resonance r at its nominal mass and the bachelor c
(the MDW shape with those daughter masses): a1 -> rho0 pi-, K1(1270) -> K*0 pi-
and K1(1400) -> K*0 pi- (S-waves; K1(1270) -> rho0 K+ is closed at the nominal
rho0 mass); below that threshold the width is 0.  The
structure differs from the shipped files (the lineshapes gain width planes),
so the runtime-table kernels evaluate it.  Tolerances as for the fp64 path."""
import functools
import json

import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import grad_scale, oracle_rate_fn, perturbed_params, rate_scale

pytestmark = pytest.mark.gpu

M_RHO, M_KSTAR, M_PI, M_K = 0.77526, 0.89555, 0.13957, 0.493677
CHANNELS = {"a1": (M_RHO, M_PI), "K1_1270": (M_KSTAR, M_PI), "K1_1400": (M_KSTAR, M_PI)}


def running_width_model(name: str) -> dict:
    d = json.load(open(model_path(name)))
    for r in d["resonances"]:
        if r["name"] in CHANNELS:
            r["shape"] = "MDW"
            r["L"] = 0
            r["daughter_masses"] = list(CHANNELS[r["name"]])
    d["name"] = name + "_running_widths"
    return d


@functools.lru_cache(maxsize=None)
def running_width_workload(name: str, n_data: int, n_mc: int, wid: int):
    d = running_width_model(name)
    m = tdamp.load_model(d)
    data, t, _ = samples.generate_time_dependent(n_data, samples.rng(wid, samples.STREAM_DATA), oracle_rate_fn(m),
                                                 m.gamma, m.y, pilot=20_000, batch=1 << 15)
    mc = samples.flat_phase_space(n_mc, samples.rng(wid, samples.STREAM_MC))
    return d, m, data, t, mc


@pytest.mark.parametrize("name,nd,nm,wid", [("d0_k3pi_2chain", 1000, 10_000, 9), ("d0_k3pi_full", 777, 6_001, 10)])
def test_running_widths_match_oracle(name, nd, nm, wid):
    from paper_1702_06735_gb300.tdmix import TDMix
    d, m, data, t, mc = running_width_workload(name, nd, nm, wid)
    c = TDMix(d, "fp64")
    assert c.kernel_path == "generic"
    c.load_events(data, t, mc)
    p = perturbed_params(m, 51)
    v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p)
    assert torch.isfinite(g0).all()
    with torch.no_grad():
        R0 = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), torch.as_tensor(p)).numpy()
    R, _ = c.event_rates(p)
    assert np.max(np.abs(R - R0) / rate_scale(m, data, t, p)) <= 1e-12
    v, g = c.nll(p)
    assert abs(v - v0) <= 1e-12 * abs(v0)
    err = np.abs(g - g0.numpy()) / grad_scale(m, data, t, mc, p)
    worst = int(np.argmax(err))
    print(f"\nrunning widths {name}: NLL rel err {abs(v / v0 - 1):.2e}, gradient max err / scale {err.max():.2e} "
          f"(parameter {worst})")
    # 1e-11 for the 16-chain model: the omega width (the narrowest lineshape) measured 3.8e-12 of its
    # scale on the runtime-table kernels, the other components below 1e-12
    assert err.max() <= (1e-12 if name == "d0_k3pi_2chain" else 1e-11), (worst, err)
