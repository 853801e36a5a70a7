"""Plain float64 CPU oracle of the time-dependent four-body amplitude model.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function is a
direct transcription of a definition, vectorised over events with PyTorch CPU
tensors (float64 / complex128).  No blocking, caching, deduplication or
reordering beyond the definitions.

Where the paper prints the formula it is cited; where it only names a
building block (lineshapes, form factors, spin factors, Bose symmetrisation,
Sec. 3) the reading used here is stated in the docstring:

* lineshape: relativistic Breit-Wigner 1/(m0^2 - s - i m0 Gamma(s)); shape
  "MDW" has the mass-dependent width
      Gamma(s) = Gamma0 (m0/sqrt s) (q/q0)^(2L+1) [F_L(q r)/F_L(q0 r)]^2
  with q the breakup momentum to the resonance's nominal daughter masses;
  shape "CONST" has Gamma(s) = Gamma0; no numerator factor.
* form factors: Blatt-Weisskopf F_0 = 1, F_1 = 1/sqrt(1+z),
  F_2 = 1/sqrt(9+3z+z^2), z = (q r)^2, evaluated with the actual invariant
  masses of the vertex; the q^L part is carried by the spin factor.
* spin factors: Lorentz-covariant tensors (Zou & Bugg, EPJ A16 (2003) 537)
  built from t(P; a, b) = r - (r.P/P^2) P, r = p_a - p_b, with
  epsilon_{0123} = +1 for the P-wave.
* Bose symmetrisation: the chain amplitude is summed over the identity and
  the exchange of the two identical pi- (no 1/sqrt 2).
* normalisation: phase space by the mean over the Monte Carlo sample, decay
  time by the closed-form integrals over [0, inf).
* background (an extension; the paper's study has none, Sec. 4): when the
  model file gives "background": {"fraction": f, "tau": tau_b}, each data
  event's density is (1 - f) R / N + f B, B flat in the normalised phase
  space (volume 1: the MC mean) and e^{-t/tau_b}/tau_b in time.
* decay-time resolution (an extension; the paper's study has none, Sec. 4):
  when the model file gives "time_resolution" sigma, the rate is folded with
  a Gaussian of width sigma in the measured time, which ranges over the real
  line, so the normalisation is unchanged (rate_resolved).
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field

import torch

F64 = torch.float64
C128 = torch.complex128

SPIN_L_PARENT = {"VV_S": 0, "VV_P": 1, "VV_D": 2, "AP_S": 1, "NR": 0}


# ----------------------------------------------------------------------------
# model description (the JSON input shared with the library)
# ----------------------------------------------------------------------------
@dataclass
class Resonance:
    name: str
    mass: float
    width: float
    shape: str                  # "MDW", "CONST" or "NR"
    L: int = 0
    daughter_masses: tuple = (0.0, 0.0)
    floating: bool = True


@dataclass
class Chain:
    name: str
    amp: str                    # "A" (direct) or "Abar" (via mixing)
    spin: str                   # VV_S, VV_P, VV_D, AP_S, NR
    resonances: list
    particles: list
    coef: complex
    floating: bool = True


@dataclass
class Model:
    parent_mass: float
    masses: list
    tau: float
    r_res: float
    r_parent: float
    bose: tuple | None
    x: float
    y: float
    float_xy: bool
    sigma_t: float = 0.0   # Gaussian decay-time resolution (ps); 0: none
    bkg_fraction: float = 0.0  # fraction of background events; 0: none
    bkg_tau: float = 1.0       # background lifetime (ps)
    resonances: list = field(default_factory=list)
    chains: list = field(default_factory=list)

    @property
    def gamma(self) -> float:
        return 1.0 / self.tau

    def res_index(self, name: str) -> int:
        for i, r in enumerate(self.resonances):
            if r.name == name:
                return i
        raise KeyError(name)

    @property
    def n_params(self) -> int:
        return 2 * len(self.chains) + 2 * len(self.resonances) + 2

    def default_params(self) -> torch.Tensor:
        """Parameter vector: (Re c, Im c) per chain in model order, then
        (m0, Gamma0) per resonance in model order, then x, y."""
        v = []
        for c in self.chains:
            v += [c.coef.real, c.coef.imag]
        for r in self.resonances:
            v += [r.mass, r.width]
        v += [self.x, self.y]
        return torch.tensor(v, dtype=F64)

    def floating_mask(self) -> torch.Tensor:
        m = []
        for c in self.chains:
            m += [c.floating, c.floating]
        for r in self.resonances:
            m += [r.floating, r.floating]
        m += [self.float_xy, self.float_xy]
        return torch.tensor(m, dtype=torch.bool)


def load_model(src) -> Model:
    """Model from a JSON file path, JSON text or an already parsed dict."""
    if isinstance(src, dict):
        d = src
    elif isinstance(src, str) and src.lstrip().startswith("{"):
        d = json.loads(src)
    else:
        with open(src) as f:
            d = json.load(f)
    m = Model(parent_mass=d["parent_mass"], masses=[p["mass"] for p in d["final_state"]],
              tau=d["tau"], r_res=d["r_resonance"], r_parent=d["r_parent"],
              bose=tuple(d["bose_swap"]) if d.get("bose_swap") else None,
              x=d["x"], y=d["y"], float_xy=d.get("float_xy", True),
              sigma_t=float(d.get("time_resolution", 0.0)),
              bkg_fraction=float((d.get("background") or {}).get("fraction", 0.0)),
              bkg_tau=float((d.get("background") or {}).get("tau", 1.0)))
    for r in d["resonances"]:
        m.resonances.append(Resonance(r["name"], r["mass"], r["width"], r["shape"], r.get("L", 0),
                                      tuple(r.get("daughter_masses", (0.0, 0.0))),
                                      r.get("float", True)))
    for c in d["chains"]:
        m.chains.append(Chain(c["name"], c["amp"], c["spin"], list(c.get("resonances", [])),
                              list(c.get("particles", [0, 1, 2, 3])),
                              complex(c["coef"][0], c["coef"][1]), c.get("float", True)))
    return m


# ----------------------------------------------------------------------------
# Lorentz algebra, metric (+,-,-,-)
# ----------------------------------------------------------------------------
def mdot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def t_vector(P: torch.Tensor, pa: torch.Tensor, pb: torch.Tensor) -> torch.Tensor:
    """Relative momentum of a -> (a, b) projected orthogonal to P."""
    r = pa - pb
    return r - (mdot(r, P) / mdot(P, P)).unsqueeze(-1) * P


def levi_civita(a, b, c, d) -> torch.Tensor:
    """epsilon_{mu nu rho sigma} a^mu b^nu c^rho d^sigma with epsilon_{0123} = +1,
    i.e. the determinant of the matrix whose rows are the contravariant
    components of a, b, c, d."""
    return torch.linalg.det(torch.stack([a, b, c, d], dim=-2))


def kallen(a, b, c):
    return a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c


def breakup_q2(s, ma2, mb2):
    """Squared breakup momentum of a system of mass^2 s into masses^2 ma2, mb2,
    clamped at zero."""
    return torch.clamp(kallen(s, ma2, mb2) / (4 * s), min=0.0)


def blatt_weisskopf(L: int, q2, r: float):
    """Barrier factor without its q^L part."""
    z = q2 * r * r
    if L == 0:
        return torch.ones_like(z)
    if L == 1:
        return 1.0 / torch.sqrt(1.0 + z)
    if L == 2:
        return 1.0 / torch.sqrt(9.0 + 3.0 * z + z * z)
    raise ValueError(L)


def mass_dependent_width(s, m0, g0, L: int, ma: float, mb: float, r: float):
    """Gamma(s) = Gamma0 (m0/sqrt s) (q/q0)^(2L+1) [F_L(q r)/F_L(q0 r)]^2, and 0
    below the threshold of the nominal daughters (q = 0 there; the square
    root is taken only where q^2 > 0, so that the derivative in m0 is 0
    there rather than 0 times an infinite one)."""
    q2 = breakup_q2(s, ma * ma, mb * mb)
    q02 = breakup_q2(m0 * m0, ma * ma, mb * mb)
    above = q2 > 0
    q2s = torch.where(above, q2, torch.ones_like(q2))
    ratio = torch.where(above, torch.sqrt(q2s / q02) ** (2 * L + 1), torch.zeros_like(q2))
    ff = (blatt_weisskopf(L, q2, r) / blatt_weisskopf(L, q02, r)) ** 2
    return g0 * (m0 / torch.sqrt(s)) * ratio * ff


def breit_wigner(s, m0, g0, res: Resonance, r: float):
    """1 / (m0^2 - s - i m0 Gamma(s)) as complex128."""
    s = torch.as_tensor(s, dtype=F64)
    m0 = torch.as_tensor(m0, dtype=F64)
    g0 = torch.as_tensor(g0, dtype=F64)
    if res.shape == "NR":
        return torch.ones_like(s, dtype=C128)
    if res.shape == "MDW":
        gam = mass_dependent_width(s, m0, g0, res.L, res.daughter_masses[0], res.daughter_masses[1], r)
    elif res.shape == "CONST":
        gam = g0 * torch.ones_like(s)
    else:
        raise ValueError(res.shape)
    return 1.0 / torch.complex(m0 * m0 - s, -m0 * gam)


# ----------------------------------------------------------------------------
# spin factors and chain amplitudes (Sec. 3, Fig. 2 topologies)
# ----------------------------------------------------------------------------
def spin_factor(spin: str, p, model: Model):
    """Spin factor x barrier factors of one decay chain for momenta p given in
    the chain's particle order (a, b, c, d), each (n, 4).

    VV_*: D -> R1(a b) R2(c d).  AP_S: D -> R1 d, R1 -> R2 c, R2 -> (a b).
    Returns (spin x barrier product, (s of R1, s of R2))."""
    a, b, c, d = p
    PD = a + b + c + d
    mD2 = mdot(PD, PD)
    r, rD = model.r_res, model.r_parent
    if spin == "NR":
        return torch.ones_like(mD2), ()
    if spin.startswith("VV"):
        P1, P2 = a + b, c + d
        s1, s2 = mdot(P1, P1), mdot(P2, P2)
        t1 = t_vector(P1, a, b)
        t2 = t_vector(P2, c, d)
        L = t_vector(PD, P1, P2)
        if spin == "VV_S":
            S = mdot(t1, t2)
        elif spin == "VV_P":
            S = levi_civita(PD, P1 - P2, t1, t2)
        elif spin == "VV_D":
            S = mdot(t1, L) * mdot(t2, L) - (1.0 / 3.0) * mdot(L, L) * (
                mdot(t1, t2) - mdot(t1, PD) * mdot(t2, PD) / mD2)
        else:
            raise ValueError(spin)
        qD2 = breakup_q2(mD2, s1, s2)
        q12 = breakup_q2(s1, mdot(a, a), mdot(b, b))
        q22 = breakup_q2(s2, mdot(c, c), mdot(d, d))
        F = (blatt_weisskopf(SPIN_L_PARENT[spin], qD2, rD) * blatt_weisskopf(1, q12, r)
             * blatt_weisskopf(1, q22, r))
        return S * F, (s1, s2)
    if spin == "AP_S":
        P2 = a + b
        P1 = P2 + c
        s1, s2 = mdot(P1, P1), mdot(P2, P2)
        L = t_vector(PD, P1, d)
        t2 = t_vector(P2, a, b)
        S = mdot(L, t2) - mdot(L, P1) * mdot(t2, P1) / s1
        qD2 = breakup_q2(mD2, s1, mdot(d, d))
        q22 = breakup_q2(s2, mdot(a, a), mdot(b, b))
        F = blatt_weisskopf(1, qD2, rD) * blatt_weisskopf(1, q22, r)   # R1 -> R2 c is S-wave
        return S * F, (s1, s2)
    raise ValueError(spin)


def _unpack(model: Model, params):
    nc, nr = len(model.chains), len(model.resonances)
    cre = params[0:2 * nc:2]
    cim = params[1:2 * nc:2]
    coef = torch.complex(cre, cim)
    m0 = params[2 * nc:2 * nc + 2 * nr:2]
    g0 = params[2 * nc + 1:2 * nc + 2 * nr:2]
    x = params[2 * nc + 2 * nr]
    y = params[2 * nc + 2 * nr + 1]
    return coef, m0, g0, x, y


def _chain_one_order(model: Model, chain: Chain, ev, m0, g0):
    p = [ev[:, i, :] for i in chain.particles]
    S, svals = spin_factor(chain.spin, p, model)
    amp = S.to(C128)
    for rname, s in zip(chain.resonances, svals):
        k = model.res_index(rname)
        amp = amp * breit_wigner(s, m0[k], g0[k], model.resonances[k], model.r_res)
    return amp


def chain_amplitudes(model: Model, events, params) -> torch.Tensor:
    """Complex amplitude of every decay chain without its coefficient,
    Bose-symmetrised: a_i(e) = T_i(e) + T_i(e with the identical particles
    exchanged).  Returns (n, n_chains) complex128."""
    ev = torch.as_tensor(events, dtype=F64)
    _, m0, g0, _, _ = _unpack(model, params)
    perm = list(range(ev.shape[1]))
    if model.bose is not None:
        i, j = model.bose
        perm[i], perm[j] = perm[j], perm[i]
    ev_swap = ev[:, perm, :]
    cols = []
    for ch in model.chains:
        a = _chain_one_order(model, ch, ev, m0, g0)
        if model.bose is not None:
            a = a + _chain_one_order(model, ch, ev_swap, m0, g0)
        cols.append(a)
    return torch.stack(cols, dim=1)


def amplitudes(model: Model, events, params):
    """(A_f, Abar_f): coherent sums c_i A_i over the chains of each amplitude
    (Sec. 3, the sum over decay chains)."""
    coef, *_ = _unpack(model, params)
    a = chain_amplitudes(model, events, params)
    selA = torch.tensor([c.amp == "A" for c in model.chains])
    selB = torch.tensor([c.amp == "Abar" for c in model.chains])
    A = (a[:, selA] * coef[selA]).sum(dim=1)
    Ab = (a[:, selB] * coef[selB]).sum(dim=1)
    return A, Ab


# ----------------------------------------------------------------------------
# Eq. (mix), its time integrals, normalisation and the likelihood
# ----------------------------------------------------------------------------
def rate_literal(A, Ab, t, x, y, gamma):
    """Eq. (mix) times e^{-Gamma t}: the decay rate as printed (no CP violation)."""
    gt = gamma * torch.as_tensor(t, dtype=F64)
    A2 = A.real ** 2 + A.imag ** 2
    B2 = Ab.real ** 2 + Ab.imag ** 2
    cross = A * Ab.conj()
    Bv = ((A2 + B2) * torch.cosh(y * gt) + (A2 - B2) * torch.cos(x * gt)
          - 2 * cross.real * torch.sinh(y * gt) - 2 * cross.imag * torch.sin(x * gt))
    return torch.exp(-gt) * Bv, Bv


def rate_factorised(A, Ab, t, x, y, gamma):
    """Same rate as 2 |cosh(w) A - sinh(w) Abar|^2 e^{-Gamma t}, w = (y + i x) Gamma t / 2."""
    gt = gamma * torch.as_tensor(t, dtype=F64)
    w = torch.complex(y * gt / 2, x * gt / 2)
    Z = torch.cosh(w) * A - torch.sinh(w) * Ab
    Bv = 2 * (Z.real ** 2 + Z.imag ** 2)
    return torch.exp(-gt) * Bv, Bv


def time_integrals(x, y, gamma):
    """Integrals over t in [0, inf) of e^{-Gamma t} times cosh(y Gamma t),
    cos(x Gamma t), sinh(y Gamma t), sin(x Gamma t)."""
    return (1.0 / (gamma * (1 - y * y)), 1.0 / (gamma * (1 + x * x)),
            y / (gamma * (1 - y * y)), x / (gamma * (1 + x * x)))


def norm_integrand(A, Ab, x, y, gamma):
    """Eq. (mix) times e^{-Gamma t} integrated over t, per phase-space point."""
    ich, ic, ish, isn = time_integrals(x, y, gamma)
    A2 = A.real ** 2 + A.imag ** 2
    B2 = Ab.real ** 2 + Ab.imag ** 2
    cross = A * Ab.conj()
    return (A2 + B2) * ich + (A2 - B2) * ic - 2 * cross.real * ish - 2 * cross.imag * isn


def normalisation(model: Model, mc_events, params, mc_weights=None):
    """N = weighted mean over the phase-space sample of the time-integrated rate."""
    _, _, _, x, y = _unpack(model, params)
    A, Ab = amplitudes(model, mc_events, params)
    f = norm_integrand(A, Ab, x, y, model.gamma)
    if mc_weights is None:
        return f.mean()
    w = torch.as_tensor(mc_weights, dtype=F64)
    return (w * f).sum() / w.sum()


def event_rates(model: Model, events, t, params):
    """Unnormalised rate e^{-Gamma t} B(e) of Eq. (mix) per event (folded
    with the decay-time resolution when the model has one)."""
    _, _, _, x, y = _unpack(model, params)
    A, Ab = amplitudes(model, events, params)
    if model.sigma_t > 0:
        return rate_resolved(A, Ab, t, x, y, model.gamma, model.sigma_t)
    R, _ = rate_literal(A, Ab, t, x, y, model.gamma)
    return R


# ----------------------------------------------------------------------------
# Decay-time resolution: an extension the paper leaves out (its study has no
# resolution, Sec. 4).  Reading: the measured time is the true time plus a
# Gaussian of fixed width sigma, measured times range over the whole real
# line, so the normalisation (the time integral of the rate) is unchanged.
# ----------------------------------------------------------------------------
_GL_ORDER = 192
_GL_CACHE = {}


def _gauss_legendre(n: int):
    if n not in _GL_CACHE:
        import numpy as np
        xg, wg = np.polynomial.legendre.leggauss(n)
        _GL_CACHE[n] = (torch.tensor(xg, dtype=F64), torch.tensor(wg, dtype=F64))
    return _GL_CACHE[n]


def rate_resolved(A, Ab, t, x, y, gamma, sigma):
    """R(t) = int_0^inf dt' e^{-Gamma t'} B(t') G(t - t'; sigma), G the
    normal density of width sigma and B of Eq. (mix) (rate_literal), by
    Gauss-Legendre quadrature over t' in [max(0, t - 12 sigma), t + 12 sigma]
    (beyond 12 sigma the Gaussian is below 1e-31 of its peak)."""
    t = torch.as_tensor(t, dtype=F64)
    xg, wg = _gauss_legendre(_GL_ORDER)
    lo = torch.clamp(t - 12 * sigma, min=0.0)
    hi = torch.clamp(t + 12 * sigma, min=0.0)
    half, mid = (hi - lo) / 2, (hi + lo) / 2
    tp = mid[:, None] + half[:, None] * xg[None, :]
    R0, _ = rate_literal(A[:, None], Ab[:, None], tp, x, y, gamma)
    g = torch.exp(-(t[:, None] - tp) ** 2 / (2 * sigma * sigma)) / (sigma * math.sqrt(2 * math.pi))
    return (R0 * g * wg[None, :]).sum(dim=1) * half


def background_density(model: Model, t):
    """Density of a background event per unit of normalised phase space and
    of (measured) decay time: flat in phase space, e^{-t/tau_b} / tau_b in
    the true time (folded with the resolution when the model has one, by the
    same quadrature as rate_resolved)."""
    t = torch.as_tensor(t, dtype=F64)
    tb = model.bkg_tau
    if model.sigma_t <= 0:
        return torch.where(t >= 0, torch.exp(-torch.clamp(t, min=0.0) / tb) / tb, torch.zeros_like(t))
    sigma = model.sigma_t
    xg, wg = _gauss_legendre(_GL_ORDER)
    lo = torch.clamp(t - 12 * sigma, min=0.0)
    hi = torch.clamp(t + 12 * sigma, min=0.0)
    half, mid = (hi - lo) / 2, (hi + lo) / 2
    tp = mid[:, None] + half[:, None] * xg[None, :]
    g = torch.exp(-(t[:, None] - tp) ** 2 / (2 * sigma * sigma)) / (sigma * math.sqrt(2 * math.pi))
    return (torch.exp(-tp / tb) / tb * g * wg[None, :]).sum(dim=1) * half


def nll(model: Model, data_events, data_t, mc_events, params, mc_weights=None):
    """-sum_e ln( R(e) / N ) over the data sample; with a background
    fraction f (an extension; the paper's study has no background, Sec. 4),
    -sum_e ln( (1 - f) R(e) / N + f B(e) ), B the background density."""
    R = event_rates(model, data_events, data_t, params)
    N = normalisation(model, mc_events, params, mc_weights)
    if model.bkg_fraction > 0:
        f = model.bkg_fraction
        return -torch.log((1 - f) * R / N + f * background_density(model, data_t)).sum()
    return -(torch.log(R) - torch.log(N)).sum()


def nll_and_grad(model: Model, data_events, data_t, mc_events, params=None, mc_weights=None,
                 floating=None):
    """NLL and its gradient by reverse-mode autograd; entries of fixed
    parameters are zero."""
    if params is None:
        params = model.default_params()
    p = torch.as_tensor(params, dtype=F64).detach().clone().requires_grad_(True)
    v = nll(model, data_events, data_t, mc_events, p, mc_weights)
    (g,) = torch.autograd.grad(v, p)
    mask = model.floating_mask() if floating is None else torch.as_tensor(floating, dtype=torch.bool)
    g = torch.where(mask, g, torch.zeros_like(g))
    return float(v.detach()), g.detach()


def component_gram(model: Model, mc_events, params, mc_weights=None):
    """I_ij = <a_i^* a_j> over the phase-space sample for the chain amplitudes
    (no coefficients), as a complex (n_chains, n_chains) matrix."""
    a = chain_amplitudes(model, mc_events, params)
    if mc_weights is None:
        w = torch.ones(a.shape[0], dtype=F64)
    else:
        w = torch.as_tensor(mc_weights, dtype=F64)
    return (a.conj().T * w) @ a / w.sum()
