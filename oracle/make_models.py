"""Writes the amplitude-model JSON files of the D0 -> K+ pi- pi+ pi- workloads.

TEST INFRASTRUCTURE (stored values): the chain structure is fixed below; the
complex coefficients are drawn from the seeded Philox stream STREAM_COEF
(r ~ U(0.5, 1.5), phi ~ U(-pi, pi)) and expressed relative to each chain's
size: c_i = r_i e^{i phi_i} rms_0 / rms_i, with rms_i the root mean square
of the chain amplitude over a flat phase-space sample, so that every chain
contributes comparably (the convention behind fit fractions).  The first CF
chain is the fixed reference 1 + 0i, and the DCS block (chains of A_f) is
then rescaled so that <|A_f|^2> / <|Abar_f|^2> = 0.0035.  Run:  python -m oracle.make_models
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from paper_1702_06735_gb300 import samples
from . import tdamp

OUT = os.path.join(os.path.dirname(__file__), "..", "paper_1702_06735_gb300", "amplitude_models")
M_D, M_K, M_PI = samples.M_D, samples.M_K, samples.M_PI
DCS_TO_CF = 0.0035

RES = {
    "K*0": {"name": "K*0", "mass": 0.89555, "width": 0.0473, "shape": "MDW", "L": 1,
            "daughter_masses": [M_K, M_PI]},
    "rho0": {"name": "rho0", "mass": 0.77526, "width": 0.1491, "shape": "MDW", "L": 1,
             "daughter_masses": [M_PI, M_PI]},
    "omega": {"name": "omega", "mass": 0.78266, "width": 0.00868, "shape": "MDW", "L": 1,
              "daughter_masses": [M_PI, M_PI]},
    "a1": {"name": "a1", "mass": 1.230, "width": 0.420, "shape": "CONST", "L": 0},
    "K1_1270": {"name": "K1_1270", "mass": 1.253, "width": 0.090, "shape": "CONST", "L": 0},
    "K1_1400": {"name": "K1_1400", "mass": 1.403, "width": 0.174, "shape": "CONST", "L": 0},
}

# (label, spin, resonances, particles a b c d); VV: R1=(a b), R2=(c d);
# AP_S: R2=(a b), R1=R2+c, D -> R1 d.  p0=K+, p1=pi-(a), p2=pi+, p3=pi-(b).
TOPOLOGIES = [
    ("K*0 rho0 S-wave", "VV_S", ["K*0", "rho0"], [0, 1, 2, 3]),
    ("K*0 rho0 P-wave", "VV_P", ["K*0", "rho0"], [0, 1, 2, 3]),
    ("K*0 rho0 D-wave", "VV_D", ["K*0", "rho0"], [0, 1, 2, 3]),
    ("K a1(rho0 pi) S-wave", "AP_S", ["a1", "rho0"], [2, 1, 3, 0]),
    ("K1(1270)(rho0 K) pi S-wave", "AP_S", ["K1_1270", "rho0"], [2, 1, 0, 3]),
    ("K1(1400)(K*0 pi+) pi S-wave", "AP_S", ["K1_1400", "K*0"], [0, 1, 2, 3]),
    ("K*0 omega S-wave", "VV_S", ["K*0", "omega"], [0, 1, 2, 3]),
    ("non-resonant", "NR", [], [0, 1, 2, 3]),
]


def _base(name, resonances, chains, dedup=True):
    return {
        "name": name,
        "parent_mass": M_D,
        "final_state": [{"name": "K+", "mass": M_K}, {"name": "pi-", "mass": M_PI},
                        {"name": "pi+", "mass": M_PI}, {"name": "pi-", "mass": M_PI}],
        "bose_swap": [1, 3],
        "tau": samples.TAU_D,
        "r_resonance": 1.5,
        "r_parent": 5.0,
        "dedup": dedup,
        "x": 0.0049, "y": 0.0061, "float_xy": True,
        "resonances": [dict(RES[r], float=True) for r in resonances],
        "chains": chains,
    }


def _draw_coefs(n, g):
    u = g.random((n, 2))
    mag = 0.5 + u[:, 0]
    ph = -math.pi + 2 * math.pi * u[:, 1]
    return mag * np.cos(ph), mag * np.sin(ph)


def _rescale_dcs(d, n_mc=200_000):
    m = tdamp.load_model(d)
    mc = samples.flat_phase_space(n_mc, samples.rng(99, samples.STREAM_MC))
    with torch.no_grad():
        rms = (tdamp.chain_amplitudes(m, torch.from_numpy(mc), m.default_params()).abs() ** 2).mean(0).sqrt()
    ref = float(rms[0])
    for i, c in enumerate(d["chains"]):
        if i > 0:
            k = ref / float(rms[i])
            c["coef"] = [c["coef"][0] * k, c["coef"][1] * k]
    m = tdamp.load_model(d)
    with torch.no_grad():
        A, Ab = tdamp.amplitudes(m, torch.from_numpy(mc), m.default_params())
    ratio = float((A.abs() ** 2).mean() / (Ab.abs() ** 2).mean())
    k = math.sqrt(DCS_TO_CF / ratio)
    for c in d["chains"]:
        if c["amp"] == "A":
            c["coef"] = [c["coef"][0] * k, c["coef"][1] * k]
    return d


def two_chain():
    g = samples.rng(0, samples.STREAM_COEF)
    re, im = _draw_coefs(2, g)
    chains = [
        {"name": "CF K*0 rho0 S-wave", "amp": "Abar", "spin": "VV_S", "resonances": ["K*0", "rho0"],
         "particles": [0, 1, 2, 3], "coef": [1.0, 0.0], "float": False},
        {"name": "DCS K+ a1-(rho0 pi-) S-wave", "amp": "A", "spin": "AP_S", "resonances": ["a1", "rho0"],
         "particles": [2, 1, 3, 0], "coef": [float(re[1]), float(im[1])], "float": True},
    ]
    return _rescale_dcs(_base("d0_k3pi_2chain", ["K*0", "rho0", "a1"], chains))


def full(dedup=True):
    g = samples.rng(1, samples.STREAM_COEF)
    re, im = _draw_coefs(16, g)
    chains = []
    for i, (label, spin, res, parts) in enumerate(TOPOLOGIES):
        chains.append({"name": "CF " + label, "amp": "Abar", "spin": spin, "resonances": res,
                       "particles": parts, "coef": [1.0, 0.0] if i == 0 else [float(re[i]), float(im[i])],
                       "float": i != 0})
    for i, (label, spin, res, parts) in enumerate(TOPOLOGIES):
        chains.append({"name": "DCS " + label, "amp": "A", "spin": spin, "resonances": res,
                       "particles": parts, "coef": [float(re[8 + i]), float(im[8 + i])], "float": True})
    name = "d0_k3pi_full" if dedup else "d0_k3pi_full_nodedup"
    return _rescale_dcs(_base(name, list(RES), chains, dedup=dedup))


def main():
    os.makedirs(OUT, exist_ok=True)
    for d in (two_chain(), full(True), full(False)):
        path = os.path.join(OUT, d["name"] + ".json")
        with open(path, "w") as f:
            json.dump(d, f, indent=1)
            f.write("\n")
        print("wrote", os.path.normpath(path))


if __name__ == "__main__":
    main()
