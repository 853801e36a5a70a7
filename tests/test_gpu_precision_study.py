"""Precision study at 10,000,000 data and 10,000,000 MC events (the precision
form of the 2-chain workload) and the 16-chain normalisation matrix over
10,000,000 MC events, both paths through the C ABI.

The fp64 path is pinned to the oracle on what the oracle computes in seconds
at this size: per-event rates of 20,000 sampled data events (1e-12 of their
cancellation-free scale) and N over all 10,000,000 MC events in chunks
(1e-12 relative).  The fp32 precision path is then measured against the fp64
path on every event and every result; the errors are printed and held to:
per-event rates 1e-5 relative on every event (ill-conditioned events, whose
amplitudes nearly cancel between chains or between the two Bose orderings
of one chain, are recomputed in double-float by the kernel; their number is
printed) and 1e-6 of the cancellation-free scale (the scale counts each
Bose ordering of each chain as a separate term), the NLL per data event
2e-8 (the 1e-3-at-50,000-events bar, scaled by the event count), N and the
normalisation matrix 1e-6 relative to their largest entry, the gradient
1e-4 of its largest component.

The data here are flat in phase space with exponential decay times (the
errors depend on the arithmetic, not on the event distribution; accept/reject
at this size would take minutes of oracle time)."""
import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import perturbed_params, rate_scale, rate_scale_terms

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_BIG = 10_000_000


@pytest.fixture(scope="module")
def big():
    g = samples.rng(3, samples.STREAM_DATA)
    data = samples.flat_phase_space(N_BIG, g)
    t = samples.exponential_times(N_BIG, 1.0 / samples.TAU_D, g)
    mc = samples.flat_phase_space(N_BIG, samples.rng(3, samples.STREAM_MC))
    return data, t, mc


def _ctx(name, precision, data, t, mc):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(name, precision)
    dev = torch.device("cuda:0")
    c.load_events(torch.from_numpy(data).to(dev), torch.from_numpy(t).to(dev), torch.from_numpy(mc).to(dev))
    return c


def test_two_chain_precision_at_ten_million(big):
    data, t, mc = big
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    p = perturbed_params(m, 77)
    c64 = _ctx("d0_k3pi_2chain", "fp64", data, t, mc)
    R64, N64 = c64.event_rates(p)
    v64, g64 = c64.nll(p)
    I64 = c64.norm_matrix()
    c64.close()
    # fp64 path pinned to the oracle
    idx = np.random.default_rng(5).choice(N_BIG, 20_000, replace=False)
    pt = torch.from_numpy(p)
    with torch.no_grad():
        R0 = tdamp.event_rates(m, torch.from_numpy(data[idx]), torch.from_numpy(t[idx]), pt).numpy()
        N0 = sum(float(tdamp.normalisation(m, torch.from_numpy(mc[i:i + 1_000_000]), pt))
                 for i in range(0, N_BIG, 1_000_000)) / (N_BIG // 1_000_000)
    sc = rate_scale(m, data[idx], t[idx], p)
    assert np.max(np.abs(R64[idx] - R0) / sc) <= 1e-12
    assert abs(N64 / N0 - 1) <= 1e-12
    # fp32 path against the fp64 path
    c32 = _ctx("d0_k3pi_2chain", "fp32", data, t, mc)
    R32, N32 = c32.event_rates(p)
    nrec = c32.recomputed_events()
    v32, g32 = c32.nll(p)
    I32 = c32.norm_matrix()
    c32.close()
    rel = np.abs(R32 / R64 - 1)
    cond = np.empty(N_BIG)
    for i in range(0, N_BIG, 1_000_000):
        sl = slice(i, i + 1_000_000)
        cond[sl] = rate_scale_terms(m, data[sl], t[sl], p) / R64[sl]
    abs_scaled = np.abs(R32 - R64) / (cond * R64)  # error over the cancellation-free scale
    dI = np.max(np.abs(I32 - I64)) / np.max(np.abs(I64))
    dg = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    print(f"\n10M/10M fp32 vs fp64: rate rel err median {np.median(rel):.3e}, max {rel.max():.3e} "
          f"(condition {cond[rel.argmax()]:.3g}); {nrec} events ({nrec / N_BIG:.2e}) recomputed in double-float; "
          f"max err over the scale {abs_scaled.max():.3e}; "
          f"NLL abs err {abs(v32 - v64):.3e} ({abs(v32 - v64) / N_BIG:.2e} per event); N rel err {abs(N32 / N64 - 1):.3e}; "
          f"I_jk max rel err {dI:.3e}; gradient max err / max |g| {dg:.3e}")
    assert rel.max() <= 1e-5
    assert abs_scaled.max() <= 1e-6
    assert abs(v32 - v64) <= 2e-8 * N_BIG
    assert abs(N32 / N64 - 1) <= 1e-6
    assert dI <= 1e-6
    assert dg <= 1e-4


def test_sixteen_chain_normalisation_matrix_at_ten_million(big):
    data, t, mc = big
    m = tdamp.load_model(model_path("d0_k3pi_full"))
    p = perturbed_params(m, 78)
    I = {}
    for prec in ("fp64", "fp32"):
        c = _ctx("d0_k3pi_full", prec, data[:1000], t[:1000], mc)
        c.nll(p)
        I[prec] = c.norm_matrix()
        c.close()
    # the oracle's Gram over the first 1,000,000 MC events pins the fp64 path
    c = _ctx("d0_k3pi_full", "fp64", data[:1000], t[:1000], mc[:1_000_000])
    c.nll(p)
    I1 = c.norm_matrix()
    comp = [c.chain_component(i) for i in range(len(m.chains))]
    c.close()
    with torch.no_grad():
        Ich = sum(tdamp.component_gram(m, torch.from_numpy(mc[i:i + 250_000]), torch.from_numpy(p)).numpy()
                  for i in range(0, 1_000_000, 250_000)) / 4
    # the oracle's Gram is over chains; the library's over the shared components
    I0 = np.zeros_like(I1)
    for i, ci in enumerate(comp):
        for k, ck in enumerate(comp):
            I0[ci, ck] = Ich[i, k]
    assert np.max(np.abs(I1 - I0)) <= 1e-12 * np.max(np.abs(I0))
    d = np.max(np.abs(I["fp32"] - I["fp64"])) / np.max(np.abs(I["fp64"]))
    print(f"\n16-chain I_jk over 10M MC: fp32 vs fp64 max rel err {d:.3e}")
    assert d <= 1e-6
