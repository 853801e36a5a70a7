"""The MC normalisation matrix I_jk = <a_j^* a_k> (Sec. 3.1) on its three
accumulation paths, through the C ABI, against the oracle:

* tcgen05 tensor cores on exact fixed-point pieces (fp32 path; the only
  path for 16 components, selectable for 8), against the oracle's matrix
  and against the register accumulation: 1e-6 of the largest entry;
* shared-memory sums (fp64 path, 16 components): 1e-12 of the largest
  entry, NLL, N and rates at 1e-12, gradient at 1e-12 of its
  cancellation-free scale;
* the 16-component model (no shared blocks) computes the same likelihood as
  the 8-component one that shares them: equal NLL and gradient.

MC samples span many tiles and blocks, with ragged ends, a one-event sample
and weights."""
import numpy as np
import pytest
import torch

from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import grad_scale, perturbed_params, rate_scale, workload

pytestmark = pytest.mark.gpu


def _ctx(name, precision, data, t, mc, w=None, gram=None):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(name, precision)
    if gram:
        c.set_gram(gram)
    c.load_events(data, t, mc, w)
    return c


def _oracle_gram(m, comp, mc, p, w=None):
    Ich = tdamp.component_gram(m, torch.from_numpy(mc), torch.as_tensor(p),
                               None if w is None else torch.from_numpy(w)).numpy()
    U = max(comp) + 1
    ref = np.zeros((U, U), dtype=complex)
    for i, ci in enumerate(comp):
        for k, ck in enumerate(comp):
            ref[ci, ck] = Ich[i, k]
    return ref


@pytest.fixture(scope="module")
def sample():
    m, data, t, _ = workload("d0_k3pi_full", 777, 10, 1)
    mc = samples.flat_phase_space(100_003, samples.rng(21, samples.STREAM_MC))
    return m, data, t, mc


@pytest.mark.parametrize("weighted", [False, True])
def test_tensor_core_gram_eight_components(sample, weighted):
    m, data, t, mc = sample
    w = np.random.default_rng(3).uniform(0.5, 2.0, len(mc)) if weighted else None
    p = perturbed_params(m, 31)
    I = {}
    for gram in ("registers", "tensor"):
        c = _ctx("d0_k3pi_full", "fp32", data, t, mc, w, gram)
        v, g = c.nll(p)
        I[gram] = (c.norm_matrix(), v, g)
        comp = [c.chain_component(i) for i in range(len(m.chains))]
        c.close()
    ref = _oracle_gram(m, comp, mc, p, w)
    scale = np.abs(ref).max()
    e_tc = np.abs(I["tensor"][0] - ref).max() / scale
    e_rg = np.abs(I["registers"][0] - ref).max() / scale
    v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p,
                                None if w is None else torch.from_numpy(w))
    print(f"\nI_jk fp32 vs oracle (100,003 MC{', weighted' if weighted else ''}): tensor cores {e_tc:.2e}, "
          f"registers {e_rg:.2e}; NLL err tensor {abs(I['tensor'][1] - v0):.2e}, registers {abs(I['registers'][1] - v0):.2e}")
    assert e_tc <= 1e-6 and e_rg <= 1e-6
    assert np.abs(I["tensor"][0] - I["registers"][0]).max() / scale <= 1e-6
    assert abs(I["tensor"][1] - v0) <= 1e-3
    g0 = g0.numpy()
    assert np.abs(I["tensor"][2] - g0).max() <= 1e-4 * np.abs(g0).max()


def test_sixteen_components_fp64_against_oracle(sample):
    m16 = tdamp.load_model(__import__("conftest").model_path("d0_k3pi_full_nodedup"))
    m, data, t, mc = sample
    mc = mc[:20_011]
    p = perturbed_params(m16, 32)
    c = _ctx("d0_k3pi_full_nodedup", "fp64", data, t, mc)
    assert c.n_components == 16
    R, N = c.event_rates(p)
    v, g = c.nll(p)
    I = c.norm_matrix()
    comp = [c.chain_component(i) for i in range(len(m16.chains))]
    c.close()
    v0, g0 = tdamp.nll_and_grad(m16, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p)
    with torch.no_grad():
        R0 = tdamp.event_rates(m16, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(p)).numpy()
        N0 = float(tdamp.normalisation(m16, torch.from_numpy(mc), torch.from_numpy(p)))
    ref = _oracle_gram(m16, comp, mc, p)
    assert np.abs(I - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.max(np.abs(R - R0) / rate_scale(m16, data, t, p)) <= 1e-12
    assert abs(N / N0 - 1) <= 1e-12
    assert abs(v - v0) <= 1e-12 * abs(v0)
    S = grad_scale(m16, data, t, mc, p)
    assert np.max(np.abs(g - g0.numpy()) / S) <= 1e-12


def test_sixteen_components_fp32_tensor_cores(sample):
    m16 = tdamp.load_model(__import__("conftest").model_path("d0_k3pi_full_nodedup"))
    m, data, t, mc = sample
    p = perturbed_params(m16, 33)
    c = _ctx("d0_k3pi_full_nodedup", "fp32", data, t, mc)
    R, N = c.event_rates(p)
    v, g = c.nll(p)
    I = c.norm_matrix()
    comp = [c.chain_component(i) for i in range(len(m16.chains))]
    c.close()
    ref = _oracle_gram(m16, comp, mc, p)
    eI = np.abs(I - ref).max() / np.abs(ref).max()
    v0, g0 = tdamp.nll_and_grad(m16, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), p)
    with torch.no_grad():
        R0 = tdamp.event_rates(m16, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(p)).numpy()
    rel = np.abs(R / R0 - 1)
    print(f"\n16 components, fp32 (tensor cores): I_jk {eI:.2e}, NLL err {abs(v - v0):.2e}, rates max {rel.max():.2e}")
    assert eI <= 1e-6
    assert abs(v - v0) <= 1e-3
    assert rel.max() <= 1e-5
    g0 = g0.numpy()
    assert np.abs(g - g0).max() <= 1e-4 * np.abs(g0).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_shared_and_unshared_components_give_the_same_likelihood(sample, precision):
    """Sharing recurring blocks (Sec. 3) changes the layout, not the result."""
    m, data, t, mc = sample
    mc = mc[:30_001]
    p = perturbed_params(m, 34)
    out = {}
    for name in ("d0_k3pi_full", "d0_k3pi_full_nodedup"):
        c = _ctx(name, precision, data, t, mc)
        out[name] = c.nll(p)
        c.close()
    (v8, g8), (v16, g16) = out["d0_k3pi_full"], out["d0_k3pi_full_nodedup"]
    if precision == "fp64":
        assert abs(v8 - v16) <= 1e-12 * abs(v8)
        assert np.abs(g8 - g16).max() <= 1e-10 * np.abs(g8).max()
    else:
        assert abs(v8 - v16) <= 1e-3
        assert np.abs(g8 - g16).max() <= 1e-4 * np.abs(g8).max()


def test_tensor_core_gram_ragged_and_repeatable(sample):
    m, data, t, mc = sample
    p = perturbed_params(m, 35)
    for nm in (1, 255, 257, 4099):
        c = _ctx("d0_k3pi_full", "fp32", data[:50], t[:50], mc[:nm], gram="tensor")
        v, g = c.nll(p)
        I = c.norm_matrix()
        comp = [c.chain_component(i) for i in range(len(m.chains))]
        c.close()
        ref = _oracle_gram(m, comp, mc[:nm], p)
        assert np.abs(I - ref).max() <= 1e-6 * np.abs(ref).max(), nm
    c = _ctx("d0_k3pi_full_nodedup", "fp32", data, t, mc, gram="tensor")
    a, b = c.nll(p), c.nll(p)
    c.close()
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_gram_mode_validation():
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixError
    c = TDMix("d0_k3pi_full", "fp64")
    with pytest.raises(TDMixError) as e:
        c.set_gram("tensor")
    assert e.value.code == -8
    c.close()
    c = TDMix("d0_k3pi_full_nodedup", "fp32")
    with pytest.raises(TDMixError) as e:
        c.set_gram("registers")
    assert e.value.code == -8
    c.close()
