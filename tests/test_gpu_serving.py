"""Serving: batched, continuously admitted NLL + gradient requests from many
concurrent clients (fixed model, floating coefficients and x, y)."""
import threading
import time

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
    # the first request of each sample waited for its admission, the other
    # 14 found it resident (1 GiB holds all eight)
    assert st["admitted"]["count"] == 8 and st["resident"]["count"] == 8 * 14
    assert st["admitted"]["p50_us"] > st["resident"]["p50_us"] > 0
    # after a reset every population is empty: NaN percentiles, count 0
    import ctypes
    from paper_1702_06735_gb300.tdmix import LATENCY_ADMITTED
    s.reset_stats()
    n = ctypes.c_int64(-1)
    a, b = np.empty(1), np.empty(1)
    assert s._lib.tdmix_server_latency(s._s, LATENCY_ADMITTED, a.ctypes.data, b.ctypes.data, ctypes.byref(n)) == 0
    assert n.value == 0 and np.isnan(a[0]) and np.isnan(b[0])
    assert s._lib.tdmix_server_latency(s._s, 3, None, None, None) == -1
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


def test_request_published_mid_run_finishes_before_an_earlier_long_one():
    """Continuous batching on the device: a long request (4,000,000 events,
    256 chunks, about two rounds of the loop's blocks) is running when a
    short one (1,000 events) is published; blocks that finish a chunk take
    the newest entry's chunks in turn, so the short request completes first.
    Both samples are resident before the timing starts."""
    from paper_1702_06735_gb300.tdmix import TDMixServer
    m = tdamp.load_model(model_path("d0_k3pi_full"))
    mc = samples.flat_phase_space(20_000, samples.rng(31, samples.STREAM_MC))
    g = samples.rng(31, samples.STREAM_DATA)
    big = samples.flat_phase_space(4_000_000, g)
    big_t = samples.exponential_times(len(big), 1.0 / samples.TAU_D, g)
    small, small_t = big[:1000], big_t[:1000]
    s = TDMixServer("d0_k3pi_full", "fp64", hbm_budget_bytes=1 << 32, max_slots=16)
    s.add_mc(mc)
    id_big, id_small = s.add_sample(big, big_t), s.add_sample(small, small_t)
    p = m.default_params().numpy()
    s.evaluate(id_big, p, timeout_s=600)
    s.evaluate(id_small, p, timeout_s=600)
    order = []

    def wait(tag, tk):
        s.wait(tk, timeout_s=600)
        order.append(tag)
    t_big = s.submit(id_big, p)
    time.sleep(2e-4)
    t_small = s.submit(id_small, p)
    th = [threading.Thread(target=wait, args=("big", t_big)), threading.Thread(target=wait, args=("small", t_small))]
    for x in th:
        x.start()
    for x in th:
        x.join()
    info = s.loop_info()
    s.close()
    print(f"\nloop: {info}")
    assert order == ["small", "big"], order
    assert info["abnormal_exits"] == 0, info


def test_generated_samples_match_a_context_on_the_same_events():
    """A pseudo-experiment generated on the device at admission gives the
    same likelihood as a context loaded with the same generated events."""
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixServer
    m = tdamp.load_model(model_path(NAME))
    mc = samples.flat_phase_space(20_000, samples.rng(32, samples.STREAM_MC))
    gen = m.default_params().numpy()
    s = TDMixServer(NAME, "fp64", hbm_budget_bytes=1 << 30, max_slots=16)
    s.add_mc(mc)
    sid = s.add_generated_sample(gen, 30_000, seed=77, stream=5)
    p = _params(m, np.random.default_rng(9))
    v, gr = s.evaluate(sid, p)
    c = TDMix(NAME, "fp64")
    p4, t, _ = c.generate(30_000, seed=77, stream=5, params=gen)
    c.load_events(p4, t, mc)
    mask = m.floating_mask().numpy().astype(np.int32)
    nc = len(m.chains)
    mask[2 * nc:2 * nc + 2 * len(m.resonances)] = 0
    c.set_floating(mask)
    v0, g0 = c.nll(p)
    c.close()
    info = s.loop_info()
    s.close()
    assert abs(v - v0) <= 1e-12 * abs(v0)
    assert np.abs(gr - g0).max() <= 1e-10 * np.abs(g0).max()
    assert info["launches"] >= 1


def test_loop_stops_when_idle_and_restarts():
    m, toys, mc = _toys(2, 33)
    s = _server("fp32", mc)
    ids = [s.add_sample(p4, t) for p4, t in toys]
    p = m.default_params().numpy()
    a = s.evaluate(ids[0], p)
    time.sleep(0.2)
    assert not s.loop_info()["running"]
    b = s.evaluate(ids[0], p)
    info = s.loop_info()
    s.close()
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    assert info["launches"] >= 2 and info["abnormal_exits"] == 0
