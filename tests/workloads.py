"""Seeded test workloads: flat phase-space MC and time-dependent pseudo-data
generated by accept/reject with the ORACLE's rate (never the CUDA path)."""
import functools

import numpy as np
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples


def oracle_rate_fn(model, params=None):
    p = model.default_params() if params is None else torch.as_tensor(params, dtype=torch.float64)

    def f(p4, t):
        with torch.no_grad():
            return tdamp.event_rates(model, torch.from_numpy(p4), torch.from_numpy(t), p).numpy()
    return f


@functools.lru_cache(maxsize=None)
def workload(name: str, n_data: int, n_mc: int, workload_id: int):
    """(model, data_p4, data_t, mc_p4) for a shipped model."""
    m = tdamp.load_model(model_path(name))
    gd = samples.rng(workload_id, samples.STREAM_DATA)
    gm = samples.rng(workload_id, samples.STREAM_MC)
    data, t, _ = samples.generate_time_dependent(n_data, gd, oracle_rate_fn(m), m.gamma, m.y,
                                                 pilot=min(50_000, 20 * n_data), batch=1 << 15)
    mc = samples.flat_phase_space(n_mc, gm)
    return m, data, t, mc


def perturbed_params(model, seed: int, scale: float = 0.05, masses: bool = True):
    """Parameters moved away from the model file's values (seeded)."""
    g = np.random.default_rng(seed)
    p = model.default_params().numpy().copy()
    nc, nr = len(model.chains), len(model.resonances)
    mask = model.floating_mask().numpy()
    for k in range(2 * nc):
        if mask[k]:
            p[k] *= 1 + scale * g.normal()
    if masses:
        for r in range(nr):
            p[2 * nc + 2 * r] *= 1 + 0.1 * scale * g.normal()
            p[2 * nc + 2 * r + 1] *= 1 + scale * g.normal()
    p[-2] += 0.002 * g.normal()
    p[-1] += 0.002 * g.normal()
    return p


def rate_scale(model, data, t, params):
    """Rounding scale of each event's rate: 2 e^{-G t} cosh(y G t) (sum |c_i A_i|)^2,
    an upper bound of |rate| obtained without cancellation."""
    p = torch.as_tensor(params, dtype=torch.float64)
    coef, *_ = tdamp._unpack(model, p)
    a = tdamp.chain_amplitudes(model, torch.as_tensor(data), p)
    s = (a * coef).abs().sum(dim=1)
    y = float(p[-1])
    gt = model.gamma * torch.as_tensor(t)
    return (2 * torch.exp(-gt) * torch.cosh(y * gt) * s ** 2).numpy()


def rate_scale_terms(model, data, t, params):
    """Like rate_scale, but the chain sum runs over every Bose ordering
    separately: 2 e^{-G t} cosh(y G t) (sum_i sum_o |c_i T_i,o|)^2.  It also
    bounds cancellations between the two orderings of one chain, which
    rate_scale (built on the Bose-summed chain amplitudes) does not see."""
    p = torch.as_tensor(params, dtype=torch.float64)
    coef, m0, g0, _, _ = tdamp._unpack(model, p)
    ev = torch.as_tensor(data, dtype=torch.float64)
    perm = list(range(ev.shape[1]))
    if model.bose is not None:
        i, j = model.bose
        perm[i], perm[j] = perm[j], perm[i]
    ev_swap = ev[:, perm, :]
    s = torch.zeros(ev.shape[0], dtype=torch.float64)
    for k, ch in enumerate(model.chains):
        s = s + coef[k].abs() * tdamp._chain_one_order(model, ch, ev, m0, g0).abs()
        if model.bose is not None:
            s = s + coef[k].abs() * tdamp._chain_one_order(model, ch, ev_swap, m0, g0).abs()
    y = float(p[-1])
    gt = model.gamma * torch.as_tensor(t)
    return (2 * torch.exp(-gt) * torch.cosh(y * gt) * s ** 2).numpy()



def grad_scale(model, data, t, mc, params, mc_weights=None):
    """Cancellation-free scale of each NLL gradient component:
    S_k = sum_e |d ln R_e / d theta_k| + N_d sum_m w_m |d f_m / d theta_k| / sum_m w_m f_m,
    with R_e the data rates and f_m the time-integrated rate of MC event m
    (NLL = -sum ln R_e + N_d ln N, N = <f>).  Rounding errors of a gradient
    formed from these terms scale with S_k, not with |g_k|, which can be
    near zero by cancellation between the data and normalisation parts.
    Forward-mode Jacobians through the oracle."""
    p = torch.as_tensor(params, dtype=torch.float64)
    d = torch.as_tensor(data, dtype=torch.float64)
    tt = torch.as_tensor(t, dtype=torch.float64)
    mm = torch.as_tensor(mc, dtype=torch.float64)
    Jd = torch.func.jacfwd(lambda q: torch.log(tdamp.event_rates(model, d, tt, q)))(p)

    def f_mc(q):
        _, _, _, x, y = tdamp._unpack(model, q)
        A, Ab = tdamp.amplitudes(model, mm, q)
        return tdamp.norm_integrand(A, Ab, x, y, model.gamma)
    with torch.no_grad():
        f = f_mc(p)
    Jm = torch.func.jacfwd(f_mc)(p)
    w = torch.ones(len(mm), dtype=torch.float64) if mc_weights is None else torch.as_tensor(mc_weights)
    S = Jd.abs().sum(0) + len(d) * (w[:, None] * Jm.abs()).sum(0) / (w * f).sum()
    return S.numpy()


def projections(p4):
    """The five variables of the four-body phase space used to display the
    fit in Sec. 3.2: m12 = m(K+ pi-), m34 = m(pi+ pi-) (particles 0 1 and
    2 3), the helicity cosines of particle 0 in the (0 1) rest frame and of
    particle 2 in the (2 3) rest frame (each against its pair's direction in
    the parent frame), and the angle phi between the two decay planes.
    p4: (n, 4, 4) parent-frame momenta.  Returns (n, 5)."""
    p4 = np.asarray(p4, dtype=np.float64)

    def mass(P):
        return np.sqrt(np.maximum(P[:, 0] ** 2 - (P[:, 1:] ** 2).sum(1), 0.0))

    def helicity_cos(pa, P):
        beta = P[:, 1:] / P[:, :1]
        b2 = (beta ** 2).sum(1)
        g = 1.0 / np.sqrt(1.0 - b2)
        bp = (beta * pa[:, 1:]).sum(1)
        k = np.where(b2 > 0, (g - 1.0) / np.where(b2 > 0, b2, 1.0) * bp, 0.0) - g * pa[:, 0]
        v = pa[:, 1:] + k[:, None] * beta        # momentum in the pair's rest frame
        d = P[:, 1:]
        return (v * d).sum(1) / np.sqrt((v ** 2).sum(1) * (d ** 2).sum(1))

    P12, P34 = p4[:, 0] + p4[:, 1], p4[:, 2] + p4[:, 3]
    n1 = np.cross(p4[:, 0, 1:], p4[:, 1, 1:])
    n2 = np.cross(p4[:, 2, 1:], p4[:, 3, 1:])
    z = P12[:, 1:] / np.linalg.norm(P12[:, 1:], axis=1, keepdims=True)
    phi = np.arctan2((np.cross(n1, n2) * z).sum(1), (n1 * n2).sum(1))
    return np.stack([mass(P12), mass(P34), helicity_cos(p4[:, 0], P12), helicity_cos(p4[:, 2], P34), phi], axis=1)


def binned_chi2(obs, ref, ref_w, bins, rng):
    """Chi-square of an unweighted sample `obs` against the distribution of a
    weighted reference sample, both histogrammed in `bins` over `rng`;
    the reference's own statistical uncertainty is included.  Returns
    (chi2, degrees of freedom)."""
    ho, _ = np.histogram(obs, bins=bins, range=rng)
    hw, _ = np.histogram(ref, bins=bins, range=rng, weights=ref_w)
    hw2, _ = np.histogram(ref, bins=bins, range=rng, weights=ref_w ** 2)
    scale = ho.sum() / hw.sum()
    exp = hw * scale
    var = exp + hw2 * scale ** 2
    keep = exp > 5
    return float((((ho - exp) ** 2)[keep] / var[keep]).sum()), int(keep.sum()) - 1
