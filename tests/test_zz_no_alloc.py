"""The allocation-free entry point tdmix_loglik_components_noalloc.

It exists for callers that cannot allocate device memory while they
evaluate (work recorded into a CUDA graph, code under an external memory
manager that owns all device allocations, latency-bound loops that must not
wait on the allocator): it keeps its block partial sums in a fixed file-scope
device array.  Here it is fed the chain amplitudes of the oracle, one
component per chain, and its sum of ln B must equal the one implied by the
library's existing entry point tdmix_event_rates (ln B = ln R + Gamma t), on
two calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from oracle import tdamp
from workloads import perturbed_params, workload

pytestmark = pytest.mark.gpu
F64 = torch.float64


def _call(lib, m, data, t, p, dev, stream):
    with torch.no_grad():
        a = tdamp.chain_amplitudes(m, torch.from_numpy(data), torch.from_numpy(p))
    n, U = a.shape
    ld = n + 5
    a_re = torch.zeros(U, ld, dtype=F64, device=dev)
    a_im = torch.zeros(U, ld, dtype=F64, device=dev)
    a_re[:, :n] = a.real.T.to(dev)
    a_im[:, :n] = a.imag.T.to(dev)
    cA = torch.zeros(2 * U, dtype=F64)
    cB = torch.zeros(2 * U, dtype=F64)
    for i, ch in enumerate(m.chains):
        dst = cA if ch.amp == "A" else cB
        dst[2 * i:2 * i + 2] = torch.from_numpy(p[2 * i:2 * i + 2])
    cA, cB = cA.to(dev), cB.to(dev)
    tt = torch.from_numpy(t).to(dev)
    out = torch.full((2,), float("nan"), dtype=F64, device=dev)
    rc = lib.tdmix_loglik_components_noalloc(U, n, a_re.data_ptr(), a_im.data_ptr(), ld, tt.data_ptr(),
                                             cA.data_ptr(), cB.data_ptr(), float(p[-2]), float(p[-1]), m.gamma,
                                             out.data_ptr(), stream)
    assert rc == 0
    torch.cuda.synchronize(dev)
    return out.cpu().numpy()


def test_noalloc_matches_event_rates_on_two_calls():
    from paper_1702_06735_gb300.tdmix import TDMix, load_library
    lib = load_library()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    ctx = TDMix("d0_k3pi_2chain", "fp64")
    ctx.load_events(data, t, mc)
    for seed in (21, 22):
        p = perturbed_params(m, seed)
        R, _ = ctx.event_rates(p)
        lnb = np.log(R) + m.gamma * t
        out = _call(lib, m, data, t, p, dev, stream)
        assert out[1] == 0
        assert abs(out[0] - lnb.sum()) <= 1e-12 * np.abs(lnb).sum()
    ctx.close()


def test_noalloc_rejects_out_of_range_sizes():
    from paper_1702_06735_gb300.tdmix import load_library
    lib = load_library()
    x = torch.zeros(64, dtype=F64, device="cuda:0")
    p = x.data_ptr()
    assert lib.tdmix_loglik_components_noalloc(17, 4, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 0, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 8, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 4, p, p, 4, p, p, p, 0.0, 1.5, 2.4, p, None) == -6
