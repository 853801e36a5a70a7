"""Differentiation and fitting through the GPU library: the autograd
Function, gradient against central finite differences at the size of the
differentiation workload (1,000,000 events, 2,000,000 MC), and a maximum-
likelihood fit that recovers the generating x, y."""
import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import minimize, samples
from workloads import perturbed_params, workload

pytestmark = pytest.mark.gpu


def _ctx(name, precision, data, t, mc):
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(name, precision)
    c.load_events(data, t, mc)
    return c


def test_autograd_function_matches_library_gradient_and_gradcheck():
    from paper_1702_06735_gb300.autograd import TDMixNLL
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    c = _ctx("d0_k3pi_2chain", "fp64", data, t, mc)
    p = torch.tensor(perturbed_params(m, 31), dtype=torch.float64, requires_grad=True)
    v = TDMixNLL.apply(p, c)
    v.backward()
    v0, g0 = c.nll(p.detach().numpy())
    assert float(v.detach()) == v0
    assert np.array_equal(p.grad.numpy(), g0)
    # device tensors: same numbers, stream-ordered
    pd = p.detach().cuda().requires_grad_(True)
    vd = TDMixNLL.apply(pd, c)
    vd.backward()
    assert float(vd.detach()) == v0 and np.array_equal(pd.grad.cpu().numpy(), g0)
    # finite-difference check of the floating parameters
    mask = torch.from_numpy(m.floating_mask().numpy())
    q = p.detach().clone()

    def f(sub):
        full = q.clone()
        full[mask] = sub
        return TDMixNLL.apply(full, c)
    assert torch.autograd.gradcheck(f, (q[mask].clone().requires_grad_(True),), eps=1e-6, atol=1e-4, rtol=1e-5)


@pytest.mark.slow
def test_gradient_against_central_differences_at_differentiation_workload():
    """Full model, 1M events and 2M MC: the adjoint gradient against central
    differences with h = 1e-6 relative (five-point stencil), for one
    parameter of each kind."""
    g = samples.rng(3, 700)
    data = samples.flat_phase_space(1_000_000, g)
    t = samples.exponential_times(1_000_000, 1 / samples.TAU_D, g)
    mc = samples.flat_phase_space(2_000_000, g)
    m = tdamp.load_model(model_path("d0_k3pi_full"))
    c = _ctx("d0_k3pi_full", "fp64", data, t, mc)
    p = perturbed_params(m, 32)
    v, grad = c.nll(p)
    nc = len(m.chains)
    picks = [2, 3, 2 * nc, 2 * nc + 1, 2 * nc + 4, 2 * nc + 5, len(p) - 2, len(p) - 1]
    for k in picks:
        h = 1e-6 * max(abs(p[k]), 1e-2)

        def fk(d):
            q = p.copy()
            q[k] += d
            return c.nll(q, grad=False)[0]
        fd = (8 * (fk(h) - fk(-h)) - (fk(2 * h) - fk(-2 * h))) / (12 * h)
        # truncation O(h^4) is negligible; rounding of the NLL (~1e-15 |v|) / h dominates
        assert abs(fd - grad[k]) <= 1e-5 * abs(grad[k]) + 2e-15 * abs(v) / h, (k, fd, grad[k])


def test_fit_recovers_generated_mixing_parameters():
    """Toy fit with a fixed model and floating x, y (the paper's sensitivity
    and timing fits): the fitted x, y lie within 4 sigma of the generating
    values.  (Floating the DCS phase as well would leave x, y nearly
    degenerate with it at first order in Gamma t.)"""
    m, data, t, mc = workload("d0_k3pi_2chain", 20_000, 100_000, 5)
    c = _ctx("d0_k3pi_2chain", "fp64", data, t, mc)
    truth = m.default_params().numpy()
    mask = np.zeros(len(truth), dtype=np.int32)
    mask[[-2, -1]] = 1   # x, y
    c.set_floating(mask)
    start = truth.copy()
    start[-2] += 0.003
    start[-1] -= 0.003

    r = minimize.fit(c, start, mask.astype(bool), len(m.chains), len(m.resonances), gtol=1e-4, edm_tol=1e-8,
                     max_iter=300)
    assert r.converged, r.message
    err = minimize.errors(minimize.safe_objective(c), r.x, mask.astype(bool))
    for k in (-2, -1):
        assert err[k] > 0
        assert abs(r.x[k] - truth[k]) < 4 * err[k], (k, r.x[k], truth[k], err[k])
