"""Toy fits with the model floating (an extension of the paper's
fixed-model sensitivity study, Sec. 4): 40 pseudo-experiments of 10,000
events generated on the device from the 2-chain model, each fitted with
the model floating (the three resonance masses and widths, with x and y;
the coefficients stay fixed: a floating DCS phase is nearly degenerate with
x and y in this model) on a likelihood context of the fp64 path (the
Hessian errors come from finite differences of the gradient, which the
fp32 path's rounding would blur).  The pulls of x, y and the K* mass must
have mean 0 and width 1 within 3 standard errors (plus 0.1 for the
finite-difference Hessian and the small sample), and, fit by fit, the
error of x and y with the model floating is at least the error with the
model fixed on the same events (a marginal against a conditional variance
of one Hessian, up to the two minima differing)."""
import numpy as np
import pytest

from paper_1702_06735_gb300 import toys

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_floating_model_pulls_two_chain_model():
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix("d0_k3pi_2chain", "fp32")
    gen = c.default_params()
    mc, _, _ = c.generate(200_000, seed=1702067357, stream=1, flat=True, with_times=False)
    c.close()
    fits = toys.run_floating("d0_k3pi_2chain", "fp64", [10_000] * 40, gen, mc, seed=1702067357,
                             compare_fixed=True)
    assert sum(f.converged for f in fits) >= 38
    n_chains = 2
    kstar_mass = 2 * n_chains
    for name, idx in (("x", len(gen) - 2), ("y", len(gen) - 1), ("K* mass", kstar_mass)):
        s = toys.floating_pulls(fits, gen, idx)
        print(f"\n{name}: {s}")
        assert abs(s["pull_mean"]) <= 3 * s["pull_mean_err"] + 0.1
        assert abs(s["pull_width"] - 1) <= 3 * s["pull_width_err"] + 0.1
    ok = [f for f in fits if f.converged and f.xy_fixed_model and np.isfinite(f.xy_fixed_model[2])]
    ratio_x = np.array([f.errors[-2] / f.xy_fixed_model[2] for f in ok])
    ratio_y = np.array([f.errors[-1] / f.xy_fixed_model[3] for f in ok])
    print(f"error ratio floating / fixed model: x {np.median(ratio_x):.3f}, y {np.median(ratio_y):.3f}")
    assert ratio_x.min() >= 0.98 and ratio_y.min() >= 0.98
