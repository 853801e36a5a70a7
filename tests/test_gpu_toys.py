"""Recovery of the generating parameters in toy fits (the check the
sensitivity study of Sec. 4 rests on): 100 pseudo-experiments of 20,000
events generated on the device from the 2-chain model at the world-average
x = 0.49 %, y = 0.61 %, each fitted on the serving loop with x, y floating
and the model fixed; errors from the Hessian of the NLL.  The pulls
(fit - true) / error must have mean 0 within 3 standard errors and width 1
within 3 standard errors (plus 0.05 for the Hessian's finite-difference
errors), and the spread of the fitted values must agree with the mean
fitted error within 20 %."""
import numpy as np
import pytest
import torch

from paper_1702_06735_gb300 import toys

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_toy_pulls_two_chain_model():
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix("d0_k3pi_2chain", "fp32")
    gen = c.default_params()
    mc, _, _ = c.generate(200_000, seed=1702067354, stream=1, flat=True, with_times=False)
    c.close()
    fits, st = toys.run("d0_k3pi_2chain", "fp32", [20_000] * 100, gen, mc, seed=1702067354, clients=16,
                        with_errors=True)
    s = toys.pulls(fits, gen[-2], gen[-1])
    print(f"\npulls: {s}\nserving: {st}")
    assert s["used"] >= 95
    for k in ("x", "y"):
        assert abs(s[k]["pull_mean"]) <= 3 * s[k]["pull_mean_err"]
        assert abs(s[k]["pull_width"] - 1) <= 3 * s[k]["pull_width_err"] + 0.05
        assert abs(s[k]["sigma"] / s[k]["mean_error"] - 1) <= 0.2
    assert st["abnormal_exits"] == 0
