"""CUDA path (through the C ABI) against the oracle on the same seeded inputs.

Tolerances: fp64 path 1e-12 relative (per-event rates relative to their
cancellation-free scale, see workloads.rate_scale; gradient components
relative to theirs, see workloads.grad_scale); fp32 precision path 1e-5
relative per-event rate on every event and 1e-3 absolute NLL at 50,000
events."""
import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from workloads import grad_scale, perturbed_params, rate_scale, workload

pytestmark = pytest.mark.gpu

CASES = [("d0_k3pi_2chain", 1000, 10_000, 0), ("d0_k3pi_full", 777, 6_001, 1)]


def _ctx(name, precision, data, t, mc, w=None):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(name, precision)
    c.load_events(data, t, mc, w)
    return c


def _oracle(m, data, t, mc, p, w=None):
    v, g = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p,
                              None if w is None else torch.from_numpy(w))
    with torch.no_grad():
        R = tdamp.event_rates(m, torch.from_numpy(data), torch.from_numpy(t), torch.as_tensor(p)).numpy()
        N = float(tdamp.normalisation(m, torch.from_numpy(mc), torch.as_tensor(p),
                                      None if w is None else torch.from_numpy(w)))
    return v, g.numpy(), R, N


@pytest.mark.parametrize("name,nd,nm,wid", CASES)
@pytest.mark.parametrize("moved", [False, True])
def test_fp64_parity(name, nd, nm, wid, moved):
    m, data, t, mc = workload(name, nd, nm, wid)
    p = perturbed_params(m, 7 + wid) if moved else m.default_params().numpy()
    v0, g0, R0, N0 = _oracle(m, data, t, mc, p)
    c = _ctx(name, "fp64", data, t, mc)
    R, N = c.event_rates(p)
    sc = rate_scale(m, data, t, p)
    assert np.max(np.abs(R - R0) / sc) <= 1e-12
    assert abs(N / N0 - 1) <= 1e-12
    v, g = c.nll(p)
    assert abs(v - v0) <= 1e-12 * abs(v0)
    S = grad_scale(m, data, t, mc, p)
    err = np.abs(g - g0) / S
    print(f"\nfp64 gradient {name}: max |g - g_oracle| / scale {err.max():.2e}")
    assert err.max() <= 1e-12, err


@pytest.mark.parametrize("name,nd,nm,wid", CASES)
def test_norm_matrix_parity(name, nd, nm, wid):
    m, data, t, mc = workload(name, nd, nm, wid)
    p = perturbed_params(m, 11)
    c = _ctx(name, "fp64", data, t, mc)
    c.nll(p)
    I = c.norm_matrix()
    Ich = tdamp.component_gram(m, torch.from_numpy(mc), torch.as_tensor(p)).numpy()
    comp = [c.chain_component(i) for i in range(len(m.chains))]
    ref = np.zeros_like(I)
    for i, ci in enumerate(comp):
        for k, ck in enumerate(comp):
            ref[ci, ck] = Ich[i, k]
    assert np.max(np.abs(I - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("name,nd,nm,wid", CASES)
def test_cached_path_matches_full_path(name, nd, nm, wid):
    """Moving only coefficients and x, y reuses the component cache and the
    stored normalisation matrix; results still equal the oracle."""
    m, data, t, mc = workload(name, nd, nm, wid)
    c = _ctx(name, "fp64", data, t, mc)
    mask = m.floating_mask().numpy().astype(np.int32)
    nc = len(m.chains)
    mask[2 * nc:2 * nc + 2 * len(m.resonances)] = 0   # fixed model: the cache applies
    c.set_floating(mask)
    p0 = m.default_params().numpy()
    c.nll(p0)
    p1 = perturbed_params(m, 12, masses=False)
    v, g = c.nll(p1)
    v0, g0, _, _ = _oracle(m, data, t, mc, p1)
    g0 = np.where(mask.astype(bool), g0, 0.0)
    assert abs(v - v0) <= 1e-12 * abs(v0)
    S = grad_scale(m, data, t, mc, p1)
    assert np.max(np.abs(g - g0) / S) <= 1e-12


@pytest.mark.parametrize("name,nd,nm,wid", [("d0_k3pi_2chain", 1000, 10_000, 0), ("d0_k3pi_full", 3001, 60_001, 1)])
def test_fp32_cached_pass_coefficient_residues(name, nd, nm, wid):
    """The cached fp32 pass forms A and Abar with the coefficients rounded to
    fp32 and adds the rounding residues to the sum of ln B to first order in
    the finish.  (1) A coefficient step below fp32 resolution leaves every
    fp32 quantity of the pass unchanged, so the NLL moves only through the
    double-precision terms of the finish: by the gradient times the step (a
    residue term left out, of the wrong sign or on the wrong component moves
    it by the normalisation part alone, several times off).  (2) Against the
    full pass on the same component values the NLL differs by the full
    pass's fp32 rounding of A (~1e-7 per event, random) and the gradient by
    far less than the fp32 path's own error."""
    m, data, t, mc = workload(name, nd, nm, wid)
    c = _ctx(name, "fp32", data, t, mc)
    mask = m.floating_mask().numpy().astype(np.int32)
    nc, nr = len(m.chains), len(m.resonances)
    fixed = mask.copy()
    fixed[2 * nc:2 * nc + 2 * nr] = 0
    c.set_floating(fixed)
    c.nll(m.default_params().numpy())          # full pass: fills the component cache
    p1 = perturbed_params(m, 21, masses=False)
    v_c, g_c = c.nll(p1)                       # cached pass
    worst = 0.0
    for k in [q for q in range(2 * nc) if fixed[q] and p1[q] != 0][:6]:
        # two points inside the rounding interval of h = fl32(p1[k]): h + 0.05 s and
        # h + 0.2 s, s the fp32 spacing at h (the interval reaches at least s / 4 on
        # either side, also at a power of two)
        h = float(np.float32(p1[k]))
        s_k = abs(float(np.spacing(np.float32(h))))
        a, b = p1.copy(), p1.copy()
        a[k], b[k] = h + 0.05 * s_k, h + 0.2 * s_k
        assert np.float32(a[k]) == np.float32(b[k]) == np.float32(h)
        v_a, g_a = c.nll(a)
        v_b, _ = c.nll(b)
        dv, lin = v_b - v_a, g_a[k] * (b[k] - a[k])
        worst = max(worst, abs(dv - lin) / abs(lin))
        assert abs(dv - lin) <= 1e-3 * abs(lin) + 1e-10, (k, dv, lin)
    c.set_floating(mask)
    v_f, g_f = c.nll(p1)                       # full pass (masses and widths floating)
    c.close()
    S = grad_scale(m, data, t, mc, p1)
    sel = fixed.astype(bool)
    gerr = np.max(np.abs(g_c - g_f)[sel] / S[sel])
    print(f"\n{name}: sub-ulp steps {worst:.2e} of g * step; cached - full NLL {v_c - v_f:.2e}, gradient {gerr:.2e}")
    assert abs(v_c - v_f) <= 1e-4
    assert gerr <= 1e-6


def test_weighted_mc_and_ragged_tiny_samples():
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    w = np.random.default_rng(4).uniform(0.5, 2.0, 257)
    for nd, nm in ((1, 1), (3, 257), (255, 513)):
        ww = w[:nm] if nm == 257 else None
        c = _ctx("d0_k3pi_2chain", "fp64", data[:nd], t[:nd], mc[:nm], ww)
        p = perturbed_params(m, 13)
        v, g = c.nll(p)
        v0, g0, _, _ = _oracle(m, data[:nd], t[:nd], mc[:nm], p, ww)
        assert abs(v - v0) <= 1e-12 * max(1.0, abs(v0))


def test_repeatable_bitwise():
    m, data, t, mc = workload("d0_k3pi_full", 777, 6_001, 1)
    c = _ctx("d0_k3pi_full", "fp64", data, t, mc)
    p = perturbed_params(m, 14)
    a = c.nll(p)
    b = c.nll(p)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_invalid_parameters_are_reported():
    from paper_1702_06735_gb300.tdmix import TDMixError
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    c = _ctx("d0_k3pi_2chain", "fp64", data, t, mc)
    p = m.default_params().numpy()
    bad = p.copy()
    bad[2] = np.nan
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -5
    bad = p.copy()
    bad[-1] = 1.5
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -6
    bad = p.copy()
    bad[5] = -0.1   # negative width
    with pytest.raises(TDMixError) as e:
        c.nll(bad)
    assert e.value.code == -6
    v, _ = c.nll(p)       # still usable
    assert np.isfinite(v)


def test_device_pointer_path_matches_host_path():
    m, data, t, mc = workload("d0_k3pi_full", 777, 6_001, 1)
    dev = torch.device("cuda:0")
    c = _ctx("d0_k3pi_full", "fp64", torch.from_numpy(data).to(dev), torch.from_numpy(t).to(dev),
             torch.from_numpy(mc).to(dev))
    p = perturbed_params(m, 15)
    vh, gh = c.nll(p)
    pd = torch.from_numpy(p).to(dev)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    gd = torch.empty(len(p), dtype=torch.float64, device=dev)
    c.nll_device(pd, out, gd)
    torch.cuda.synchronize()
    assert float(out[0]) == vh and np.array_equal(gd.cpu().numpy(), gh)


@pytest.mark.parametrize("name,nd,nm,wid", CASES)
def test_fp32_precision_path(name, nd, nm, wid):
    m, data, t, mc = workload(name, nd, nm, wid)
    p = perturbed_params(m, 16)
    v0, g0, R0, N0 = _oracle(m, data, t, mc, p)
    c = _ctx(name, "fp32", data, t, mc)
    R, N = c.event_rates(p)
    nrec = c.recomputed_events()
    rel = np.abs(R / R0 - 1)
    print(f"\nfp32 rates {name}: max rel err {rel.max():.2e}, median {np.median(rel):.2e}, "
          f"{nrec} events recomputed in double-float")
    assert rel.max() <= 1e-5, (np.max(rel), np.median(rel))
    v, g = c.nll(p)
    assert abs(v - v0) <= 1e-3, (v, v0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_mixing_and_long_decay_times(precision):
    """x = 0.3, y = -0.2 (as in the oracle's own rate tests) with decay times
    from 1e-4 to 50 lifetimes, a third of the events log-uniform in each of
    the ranges of the three tiers of the kernels' cosh/sinh/cos/sin (series
    to z^3 for |x|, |y| Gamma t / 2 <= 0.02, series to z^5 up to 0.1, the
    math library beyond); flat phase space, 2-chain model."""
    from paper_1702_06735_gb300 import samples
    m = tdamp.load_model(model_path("d0_k3pi_2chain"))
    g = samples.rng(9, samples.STREAM_DATA)
    n = 3000
    data = samples.flat_phase_space(n, g)
    edges = [1e-4 * m.tau, 0.04 / (0.3 * m.gamma), 0.2 / (0.3 * m.gamma), 50 * m.tau]
    t = np.concatenate([np.exp(g.uniform(np.log(a * 1.001), np.log(b * 0.999), n // 3))
                        for a, b in zip(edges[:-1], edges[1:])])
    n = len(t)
    data = data[:n]
    mc = samples.flat_phase_space(20_000, samples.rng(9, samples.STREAM_MC))
    p = perturbed_params(m, 91)
    p[-2], p[-1] = 0.3, -0.2
    z = 0.3 * m.gamma * t / 2
    tiers = np.array([(z <= 0.02).mean(), ((z > 0.02) & (z <= 0.1)).mean(), (z > 0.1).mean()])
    assert np.all(tiers > 0.2), tiers
    v0, g0, R0, N0 = _oracle(m, data, t, mc, p)
    c = _ctx("d0_k3pi_2chain", precision, data, t, mc)
    R, N = c.event_rates(p)
    v, gr = c.nll(p)
    if precision == "fp64":
        sc = rate_scale(m, data, t, p)
        assert np.max(np.abs(R - R0) / sc) <= 1e-12
        assert abs(N / N0 - 1) <= 1e-12
        assert abs(v - v0) <= 1e-12 * abs(v0)
        S = grad_scale(m, data, t, mc, p)
        assert np.max(np.abs(gr - g0) / S) <= 1e-12
    else:
        rel = np.abs(R / R0 - 1)
        print(f"\nfp32, x = 0.3, y = -0.2: rate max rel err {rel.max():.2e}, NLL err {abs(v - v0):.2e}")
        assert rel.max() <= 1e-5
        assert abs(N / N0 - 1) <= 1e-6
        assert abs(v - v0) <= 1e-3
