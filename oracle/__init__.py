"""Oracle for the time-dependent D0 -> K+ pi- pi+ pi- likelihood.

TEST INFRASTRUCTURE ONLY.  This is a plain, slow, float64 CPU restatement of
what the GPU library computes, written from the paper (Eq. (mix) of Sec. 2,
the coherent sum of Sec. 3, numerical normalisation of Sec. 3.1) and from the
readings of its unprinted formulas listed at the top of ``tdamp``.  It shares
no code with the CUDA path and the CUDA path never calls it: only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  Gradients come from PyTorch autograd on CPU, independent of the
hand-written adjoint on the GPU.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  breit_wigner, mass_dependent_width, blatt_weisskopf ... pinned (pole closed
      form, width at the pole and off it from the two-body phase space and
      barrier ratio written out, values below threshold, barrier limits)
  spin factors ........................................... pinned (Lorentz
      invariance, rest-frame closed forms on constructed events, edge zeros)
  chain amplitudes / Bose symmetrisation ................. pinned (exchange
      symmetry, factorisation into spin x barrier x lineshape)
  decay rate, Eq. (mix) .................................. pinned (two-state
      time evolution of D0 with a matrix exponential; limits x=y=0, Abar=0)
  time integrals / normalisation ......................... pinned (quadrature)
  NLL and its gradient ................................... pinned (hand-computed
      one-chain case, central finite differences)
  rate_resolved (decay-time resolution, an extension) .... pinned (closed-form
      folds through the Faddeeva function, the erfcx case x = y = 0, the
      narrow-resolution limit, the time integral over the real line)
  background_density and the mixture NLL (an extension) .. pinned (integral
      one, pure-background closed form, the no-background limit, central
      finite differences)
  the absolute value of the NLL for the D0 -> K3pi model .. parity unpinned:
      the paper prints no worked example, model or fit values.
"""
from .tdamp import (  # noqa: F401
    Model, load_model, mdot, t_vector, kallen, breakup_q2, blatt_weisskopf,
    mass_dependent_width, breit_wigner, spin_factor, chain_amplitudes,
    amplitudes, rate_literal, rate_factorised, time_integrals, norm_integrand,
    normalisation, nll, nll_and_grad, event_rates, component_gram,
)
