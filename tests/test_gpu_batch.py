"""tdmix_nll_batch: consecutive full evaluations that overlap on the device
(each may start while the one before it finishes) give the same results as
the oracle at every parameter point, and the same as separate calls.

fp64 path: NLL within 1e-12 relative of the oracle, gradient within 1e-12
of its cancellation-free scale; fp32 path: NLL within 1e-3 absolute.  A
batch is bitwise repeatable.  The cached path after a batch (coefficients
and x, y moved) still matches the oracle."""
import numpy as np
import pytest
import torch

from oracle import tdamp
from workloads import grad_scale, perturbed_params, workload

pytestmark = pytest.mark.gpu

CASES = [("d0_k3pi_2chain", 1000, 10_000, 0), ("d0_k3pi_full", 3001, 60_001, 1)]


def _points(m, n, seed):
    return np.stack([perturbed_params(m, seed + k) for k in range(n)])


@pytest.mark.parametrize("name,nd,nm,wid", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_oracle_and_single_calls(name, nd, nm, wid, precision):
    from paper_1702_06735_gb300.tdmix import TDMix
    m, data, t, mc = workload(name, nd, nm, wid)
    c = TDMix(name, precision)
    c.load_events(data, t, mc)
    dev = torch.device("cuda:0")
    P = _points(m, 6, 300 + wid)
    Pd = torch.from_numpy(P).to(dev)
    n_p = P.shape[1]
    out = torch.empty(6, dtype=torch.float64, device=dev)
    grad = torch.empty(6, n_p, dtype=torch.float64, device=dev)
    c.nll_batch(Pd, out, grad)
    out2 = torch.empty_like(out)
    grad2 = torch.empty_like(grad)
    c.nll_batch(Pd, out2, grad2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2) and torch.equal(grad, grad2)
    # a longer batch (its constants records are reallocated) repeats the first six points bitwise
    P10 = np.concatenate([P, _points(m, 4, 400 + wid)])
    out10 = torch.empty(10, dtype=torch.float64, device=dev)
    grad10 = torch.empty(10, n_p, dtype=torch.float64, device=dev)
    c.nll_batch(torch.from_numpy(P10).to(dev), out10, grad10)
    torch.cuda.synchronize()
    assert torch.equal(out10[:6], out) and torch.equal(grad10[:6], grad)
    v_b, g_b = out.cpu().numpy(), grad.cpu().numpy()
    for k in range(6):
        v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), P[k])
        v_s, g_s = c.nll(P[k])
        if precision == "fp64":
            assert abs(v_b[k] - v0) <= 1e-12 * abs(v0)
            S = grad_scale(m, data, t, mc, P[k])
            assert np.max(np.abs(g_b[k] - g0.numpy()) / S) <= 1e-12
            assert abs(v_b[k] - v_s) <= 2e-12 * abs(v0)
        else:
            assert abs(v_b[k] - v0) <= 1e-3
            assert abs(v_b[k] - v_s) <= 1e-3
    # the cached path after a batch: coefficients and x, y moved from the last point
    mask = m.floating_mask().numpy().astype(np.int32)
    nc, nr = len(m.chains), len(m.resonances)
    mask[2 * nc:2 * nc + 2 * nr] = 0
    c.set_floating(mask)
    q = P[-1].copy()
    c.nll(q)
    q[2:2 * nc] *= 1.01
    q[-2:] *= 1.1
    v_c, _ = c.nll(q)
    v0, _ = tdamp.nll_and_grad(m, torch.from_numpy(data), torch.from_numpy(t), torch.from_numpy(mc), q)
    assert abs(v_c - v0) <= (1e-12 * abs(float(v0)) if precision == "fp64" else 1e-3)
    c.close()


def test_batch_rejects_host_pointers():
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixError
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    c = TDMix("d0_k3pi_2chain", "fp64")
    c.load_events(data, t, mc)
    P = torch.from_numpy(_points(m, 2, 5))
    with pytest.raises(TDMixError):
        c.nll_batch(P, torch.empty(2, dtype=torch.float64), None)
    c.close()
