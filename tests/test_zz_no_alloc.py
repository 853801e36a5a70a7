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


def test_noalloc_many_blocks_and_zero_rates():
    """n = 300,001 events (more blocks than the scratch array holds, so the
    grid is clamped and blocks loop over several strides; the finishing pass
    reads all 1,024 partials) with synthetic components and decay times on
    the device, against the oracle's factorised rate summed in float64 on
    the host; then the same call with one component set to zero everywhere
    and the coefficients of the others zero, so that B = 0 for every event
    and all of them are counted as bad, on two calls in a row."""
    from paper_1702_06735_gb300.tdmix import load_library
    lib = load_library()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    g = np.random.default_rng(99)
    n, U, ld = 300_001, 5, 300_016
    are = g.normal(size=(U, n))
    aim = g.normal(size=(U, n))
    t = g.exponential(0.41, n)
    cA = g.normal(size=2 * U)
    cB = g.normal(size=2 * U)
    x, y, gamma = 0.0049, 0.0061, 1.0 / 0.4101
    a = torch.complex(torch.from_numpy(are), torch.from_numpy(aim))
    A = (torch.complex(torch.from_numpy(cA[0::2]), torch.from_numpy(cA[1::2]))[:, None] * a).sum(0)
    Ab = (torch.complex(torch.from_numpy(cB[0::2]), torch.from_numpy(cB[1::2]))[:, None] * a).sum(0)
    _, B = tdamp.rate_factorised(A, Ab, torch.from_numpy(t), x, y, gamma)
    want = float(torch.log(B).sum())
    d_re = torch.zeros(U, ld, dtype=F64, device=dev)
    d_im = torch.zeros(U, ld, dtype=F64, device=dev)
    d_re[:, :n] = torch.from_numpy(are).to(dev)
    d_im[:, :n] = torch.from_numpy(aim).to(dev)
    d_t = torch.from_numpy(t).to(dev)
    d_cA = torch.from_numpy(cA).to(dev)
    d_cB = torch.from_numpy(cB).to(dev)
    out = torch.full((2,), float("nan"), dtype=F64, device=dev)
    for _ in range(2):
        rc = lib.tdmix_loglik_components_noalloc(U, n, d_re.data_ptr(), d_im.data_ptr(), ld, d_t.data_ptr(),
                                                 d_cA.data_ptr(), d_cB.data_ptr(), x, y, gamma, out.data_ptr(),
                                                 stream)
        assert rc == 0
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        assert got[1] == 0
        assert abs(got[0] - want) <= 1e-12 * float(torch.log(B).abs().sum())
    # B = 0 everywhere: component 0 is zero and only it has nonzero coefficients
    d_re[0].zero_()
    d_im[0].zero_()
    zc = torch.zeros(2 * U, dtype=F64, device=dev)
    zc[0:2] = 1.0
    for _ in range(2):
        out.fill_(float("nan"))
        rc = lib.tdmix_loglik_components_noalloc(U, n, d_re.data_ptr(), d_im.data_ptr(), ld, d_t.data_ptr(),
                                                 zc.data_ptr(), zc.data_ptr(), x, y, gamma, out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        assert got[1] == n and got[0] == 0.0


def test_noalloc_rejects_out_of_range_sizes():
    from paper_1702_06735_gb300.tdmix import load_library
    lib = load_library()
    x = torch.zeros(64, dtype=F64, device="cuda:0")
    p = x.data_ptr()
    assert lib.tdmix_loglik_components_noalloc(17, 4, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 0, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 8, p, p, 4, p, p, p, 0.0, 0.0, 2.4, p, None) == -1
    assert lib.tdmix_loglik_components_noalloc(2, 4, p, p, 4, p, p, p, 0.0, 1.5, 2.4, p, None) == -6
