"""Bounded waits on the GPU: a tile copy that is never issued makes block 0's
wait run out after one second; the evaluation must come back with
TDMIX_ERR_TIMEOUT (nothing faults or hangs), and the context must evaluate
correctly afterwards.  The copy is withheld by the library's test hook."""
import numpy as np
import pytest

from workloads import perturbed_params, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_withheld_copy_reports_timeout(precision):
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixError
    m, data, t, mc = workload("d0_k3pi_2chain", 1000, 10_000, 0)
    p = perturbed_params(m, 3)
    c = TDMix("d0_k3pi_2chain", precision)
    c.load_events(data, t, mc)
    v_ref, g_ref = c.nll(p)
    c.test_withhold_copy(True)
    with pytest.raises(TDMixError) as e:
        c.nll(p)
    assert e.value.code == -7
    # device outputs: the failure shows as NaN, the stream stays usable
    import torch
    dev = torch.device("cuda", 0)
    out = torch.full((1,), 0.0, dtype=torch.float64, device=dev)
    c.nll_device(torch.from_numpy(p).to(dev), out)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    c.test_withhold_copy(False)
    v, g = c.nll(p)
    assert v == v_ref and np.array_equal(g, g_ref)
    c.close()
