"""Parity at the full size of the benchmarked workload (full model, 50,000
time-dependent pseudo-events generated with the oracle's rate, 1,000,000 flat
MC events), in the launch configuration the benchmark uses.

fp64 path: NLL and N within 1e-12 relative, every per-event rate within
1e-12 of its cancellation-free scale.  fp32 precision path: the NLL within
1e-3 absolute; every per-event rate within 1e-5 relative (the
ill-conditioned ones are recomputed in double-float; their number is
printed) and within 1e-7 of its cancellation-free scale.  The errors are
printed."""
import numpy as np
import pytest
import torch

from oracle import tdamp
from workloads import perturbed_params, rate_scale, workload

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full():
    m, data, t, mc = workload("d0_k3pi_full", 50_000, 1_000_000, 1)
    p = perturbed_params(m, 41)
    pt = torch.from_numpy(p)
    with torch.no_grad():
        R = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), pt).numpy()
        N = sum(float(tdamp.normalisation(m, torch.from_numpy(mc[i:i + 250_000]), pt)) * len(mc[i:i + 250_000])
                for i in range(0, len(mc), 250_000)) / len(mc)
    nll = float(-(np.log(R) - np.log(N)).sum())
    scale = rate_scale(m, data, t, p)
    return m, data, t, mc, p, R, N, nll, scale


def _ctx(precision, data, t, mc):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix("d0_k3pi_full", precision)
    dev = torch.device("cuda:0")
    c.load_events(torch.from_numpy(data).to(dev), torch.from_numpy(t).to(dev), torch.from_numpy(mc).to(dev))
    return c


def test_fp64_full_size(full):
    m, data, t, mc, p, R0, N0, nll0, scale = full
    c = _ctx("fp64", data, t, mc)
    R, N = c.event_rates(p)
    assert np.max(np.abs(R - R0) / scale) <= 1e-12
    assert abs(N / N0 - 1) <= 1e-12
    v, _ = c.nll(p)
    assert abs(v - nll0) <= 1e-12 * abs(nll0)


def test_fp32_full_size(full):
    m, data, t, mc, p, R0, N0, nll0, scale = full
    c = _ctx("fp32", data, t, mc)
    R, N = c.event_rates(p)
    nrec = c.recomputed_events()
    rel = np.abs(R / R0 - 1)
    cond = scale / R0
    v, g = c.nll(p)
    print(f"\nfp32 path at 50k/1M: rate rel err max {rel.max():.3e} (condition {cond[rel.argmax()]:.3g}) "
          f"median {np.median(rel):.3e}; events above 1e-5: {(rel > 1e-5).sum()}; "
          f"recomputed in double-float: {nrec}; "
          f"max err/scale {(np.abs(R - R0) / scale).max():.3e}; N rel err {abs(N / N0 - 1):.3e}; "
          f"NLL abs err {abs(v - nll0):.3e} (NLL {nll0:.6f})")
    assert abs(v - nll0) <= 1e-3
    assert rel.max() <= 1e-5
    assert (np.abs(R - R0) / scale).max() <= 1e-7
