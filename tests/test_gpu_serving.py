"""Serving: batched, continuously admitted NLL + gradient requests from many
concurrent clients (fixed model, floating coefficients and x, y)."""
import threading

import numpy as np
import pytest
import torch

from conftest import model_path
from oracle import tdamp
from paper_1702_06735_gb300 import samples
from workloads import grad_scale, workload

pytestmark = pytest.mark.gpu

NAME = "d0_k3pi_2chain"


def _toys(n_toys, seed):
    """Toy samples of different sizes drawn from a pool of accept/reject
    events generated with the oracle's rate."""
    m, pool, pool_t, mc = workload(NAME, 20_000, 20_000, 0)
    g = np.random.default_rng(seed)
    sizes = (np.exp(g.uniform(np.log(300), np.log(6000), n_toys))).astype(int)
    toys = []
    for n in sizes:
        idx = g.choice(len(pool), n, replace=False)
        toys.append((pool[idx], pool_t[idx]))
    return m, toys, mc


def _params(m, g):
    p = m.default_params().numpy().copy()
    mask = m.floating_mask().numpy()
    nc = len(m.chains)
    for k in range(2 * nc):
        if mask[k]:
            p[k] *= 1 + 0.05 * g.normal()
    p[-2] += 0.002 * g.normal()
    p[-1] += 0.002 * g.normal()
    return p


def _server(precision, mc, budget=1 << 30, slots=64):
    from paper_1702_06735_gb300.tdmix import TDMixServer
    s = TDMixServer(NAME, precision, hbm_budget_bytes=budget, max_slots=slots)
    s.add_mc(mc)
    return s


def test_server_matches_oracle():
    m, toys, mc = _toys(4, 1)
    s = _server("fp64", mc)
    ids = [s.add_sample(p4, t) for p4, t in toys]
    g = np.random.default_rng(2)
    mask = m.floating_mask().numpy().copy()
    nc = len(m.chains)
    mask[2 * nc:2 * nc + 2 * len(m.resonances)] = False
    for sid, (p4, t) in zip(ids, toys):
        p = _params(m, g)
        v, grad = s.evaluate(sid, p)
        v0, g0 = tdamp.nll_and_grad(m, torch.from_numpy(p4), torch.from_numpy(t), torch.from_numpy(mc), p,
                                    floating=mask)
        assert abs(v - v0) <= 1e-12 * abs(v0)
        g0 = g0.numpy()
        S = grad_scale(m, p4, t, mc, p)
        assert np.max(np.abs(grad - g0) / S) <= 1e-12
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_result_identical_alone_and_in_a_mix(precision):
    """A request evaluated alone and inside a batch of other requests gives
    bitwise the same NLL and gradient."""
    m, toys, mc = _toys(12, 3)
    s = _server(precision, mc)
    ids = [s.add_sample(p4, t) for p4, t in toys]
    g = np.random.default_rng(4)
    probe = [(ids[k], _params(m, g)) for k in (0, 5, 11)]
    alone = [s.evaluate(sid, p) for sid, p in probe]
    # a mix: many requests submitted together, the probes among them
    tickets = []
    for rep in range(3):
        for k, sid in enumerate(ids):
            tickets.append(("x", s.submit(sid, _params(m, g))))
        for j, (sid, p) in enumerate(probe):
            tickets.append((j, s.submit(sid, p)))
    mixed = {}
    for tag, tk in tickets:
        v, gr = s.wait(tk)
        if tag != "x":
            mixed.setdefault(tag, []).append((v, gr))
    for j in range(len(probe)):
        for v, gr in mixed[j]:
            assert v == alone[j][0] and np.array_equal(gr, alone[j][1])
    s.close()


def test_admission_under_a_binding_memory_budget():
    """With room for about two samples, requests on five samples still all
    complete (least recently used samples are evicted) and the resident
    footprint never exceeds the budget."""
    m, toys, mc = _toys(5, 5)
    sizes = [len(t) for _, t in toys]
    per_event = 2 * 2 * 8 + 8      # U = 2 components (re, im, f64) + time
    budget = int(2.2 * max(sizes) * per_event) + 4096 * per_event
    s = _server("fp64", mc, budget=budget, slots=8)
    ids = [s.add_sample(p4, t) for p4, t in toys]
    g = np.random.default_rng(6)
    ref = {}
    for sid in ids:
        p = _params(m, g)
        ref[sid] = (p, s.evaluate(sid, p))
        assert s.resident_bytes() <= budget
    # again, interleaved: every sample must be re-admitted at least once
    tickets = [(sid, s.submit(sid, ref[sid][0])) for sid in ids[::-1] + ids]
    for sid, tk in tickets:
        v, gr = s.wait(tk)
        assert v == ref[sid][1][0] and np.array_equal(gr, ref[sid][1][1])
        assert s.resident_bytes() <= budget
    s.close()


def test_concurrent_minimisers_and_stats():
    """Eight client threads each run a short descent on their own sample."""
    m, toys, mc = _toys(8, 7)
    s = _server("fp32", mc)
    ids = [s.add_sample(p4, t) for p4, t in toys]
    errors = []

    def client(sid, seed):
        try:
            g = np.random.default_rng(seed)
            p = _params(m, g)
            for _ in range(15):
                v, gr = s.evaluate(sid, p)
                assert np.isfinite(v) and np.all(np.isfinite(gr))
                p[-2:] -= 1e-8 * gr[-2:]
        except Exception as e:  # noqa: BLE001
            errors.append(e)
    th = [threading.Thread(target=client, args=(sid, 100 + k)) for k, sid in enumerate(ids)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    st = s.stats()
    assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"] and st["evals_per_s"] > 0
    s.close()


def test_requests_that_move_the_model_or_leave_the_domain():
    from paper_1702_06735_gb300.tdmix import TDMixError
    m, toys, mc = _toys(1, 8)
    s = _server("fp64", mc)
    sid = s.add_sample(*toys[0])
    p = m.default_params().numpy().copy()
    bad = p.copy()
    bad[2 * len(m.chains)] += 0.01          # a resonance mass
    with pytest.raises(TDMixError) as e:
        s.submit(sid, bad)
    assert e.value.code == -1
    bad = p.copy()
    bad[-1] = 1.2                           # |y| >= 1
    with pytest.raises(TDMixError) as e:
        s.evaluate(sid, bad)
    assert e.value.code == -6
    v, _ = s.evaluate(sid, p)               # the server keeps working
    assert np.isfinite(v)
    with pytest.raises(TDMixError) as e:
        s.wait(987654321, 0.01)
    assert e.value.code == -1
    s.close()
