"""Checkpoint and resume of the toy studies (host logic, no GPU).

ToyCheckpoint on its own (fingerprint check, a last line cut short, a
corrupted line, concurrent records), then both study runners with the
library replaced by fakes whose likelihood is a quadratic with a minimum
that depends on the toy's stream: a study that stops part way and is
started again with the same checkpoint fits only the missing toys and ends
with the same results as one that never stopped."""
import json
import threading

import numpy as np
import pytest

from paper_1702_06735_gb300 import toys
from paper_1702_06735_gb300.toys import FloatingFit, ToyCheckpoint, ToyFit

MODEL = "d0_k3pi_2chain"


def _fp(**kw):
    d = {"study": "t", "sizes": [10, 20, 30], "seed": 5}
    d.update(kw)
    return d


def test_checkpoint_round_trip_and_fingerprint(tmp_path):
    path = tmp_path / "cp.jsonl"
    cp = ToyCheckpoint(path, _fp())
    assert cp.records == {}
    cp.record(0, fit={"x": 0.1, "sx": float("nan")})
    cp.record(2, fit={"x": -0.2, "sx": 1e-3})
    cp.close()
    cp = ToyCheckpoint(path, _fp())
    assert sorted(cp.records) == [0, 2]
    assert cp.records[2]["fit"]["x"] == -0.2 and np.isnan(cp.records[0]["fit"]["sx"])
    cp.record(1, fit={"x": 0.3, "sx": 2e-3})
    cp.close()
    assert sorted(ToyCheckpoint(path, _fp()).records) == [0, 1, 2]
    with pytest.raises(ValueError, match="different study"):
        ToyCheckpoint(path, _fp(seed=6))


def test_checkpoint_drops_a_line_cut_short(tmp_path):
    path = tmp_path / "cp.jsonl"
    cp = ToyCheckpoint(path, _fp())
    cp.record(0, fit={"x": 1.0})
    cp.close()
    good = path.read_bytes()
    path.write_bytes(good + b'{"toy": 1, "fit": {"x": 0.')  # the process stopped mid-write
    cp = ToyCheckpoint(path, _fp())
    assert sorted(cp.records) == [0]
    assert path.read_bytes() == good
    cp.record(1, fit={"x": 2.0})
    cp.close()
    assert sorted(ToyCheckpoint(path, _fp()).records) == [0, 1]
    # a fingerprint line cut short: the file starts again
    path.write_bytes(b'{"checkpoint": {"stu')
    assert ToyCheckpoint(path, _fp()).records == {}
    assert json.loads(path.read_bytes().splitlines()[0]) == {"checkpoint": _fp()}


def test_checkpoint_refuses_a_corrupted_line(tmp_path):
    path = tmp_path / "cp.jsonl"
    cp = ToyCheckpoint(path, _fp())
    cp.record(0, fit={"x": 1.0})
    cp.close()
    path.write_bytes(path.read_bytes() + b"garbage\n" + b'{"toy": 2, "fit": {}}\n')
    with pytest.raises(ValueError, match="line 3"):
        ToyCheckpoint(path, _fp())
    path.write_bytes(b"not json\n")
    with pytest.raises(ValueError, match="not a toy-study checkpoint"):
        ToyCheckpoint(path, _fp())


def test_checkpoint_records_from_threads(tmp_path):
    path = tmp_path / "cp.jsonl"
    cp = ToyCheckpoint(path, _fp())
    th = [threading.Thread(target=lambda k=k: [cp.record(100 * k + j, fit={"v": j}) for j in range(50)])
          for k in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    cp.close()
    assert sorted(ToyCheckpoint(path, _fp()).records) == sorted(100 * k + j for k in range(8) for j in range(50))


# ---- the fixed-model study with a fake server

def _target(stream, n):
    """Minimum in (x, y) of the fake likelihood of toy `stream`, and its
    curvature 1 / sigma^2 with sigma = 0.05 / sqrt(n)."""
    g = np.random.default_rng(stream)
    return 0.004 + 1e-3 * g.normal(), 0.006 + 1e-3 * g.normal(), n / 0.05 ** 2


class _Stop(Exception):
    pass


class FakeServer:
    """Stands in for TDMixServer: a quadratic NLL in x and y per sample."""
    stop_at = None          # streams >= stop_at raise _Stop (the study is interrupted)
    evaluated = []          # streams evaluated, over all instances

    def __init__(self, model, precision, hbm_budget_bytes=0, max_slots=0):
        self.samples = {}
        self.lock = threading.Lock()

    def add_mc(self, mc):
        self.mc = mc

    def add_generated_sample(self, params, n, seed, stream):
        with self.lock:
            sid = len(self.samples)
            self.samples[sid] = (int(n), int(stream))
        return sid

    def evaluate(self, sid, p, timeout_s=0):
        n, stream = self.samples[sid]
        if FakeServer.stop_at is not None and stream >= FakeServer.stop_at:
            raise _Stop()
        with self.lock:
            FakeServer.evaluated.append(stream)
        x0, y0, c = _target(stream, n)
        dx, dy = p[-2] - x0, p[-1] - y0
        g = np.zeros(len(p))
        g[-2], g[-1] = c * dx, c * dy
        return 0.5 * c * (dx * dx + dy * dy), g

    def reset_stats(self):
        pass

    def stats(self):
        return {"p50_us": 1.0, "p99_us": 2.0, "evals_per_s": 3.0}

    def loop_info(self):
        return {"launches": 0}

    def close(self):
        pass


def _gen():
    from oracle import tdamp
    from conftest import model_path
    return tdamp.load_model(model_path(MODEL)).default_params().numpy()


def test_fixed_model_study_resumes(tmp_path, monkeypatch):
    monkeypatch.setattr(toys, "TDMixServer", FakeServer)
    gen = _gen()
    mc = np.zeros((7, 4, 4))
    sizes = [1000 + 500 * k for k in range(12)]
    kw = dict(seed=11, stream0=100, clients=4, with_errors=True)
    FakeServer.stop_at, FakeServer.evaluated = None, []
    ref, _ = toys.run(MODEL, "fp32", sizes, gen, mc, **kw)
    assert all(f.converged for f in ref)
    for k, f in enumerate(ref):  # the fake's minimum and errors come back
        x0, y0, c = _target(100 + k, sizes[k])
        assert abs(f.x - x0) < 1e-2 / np.sqrt(c) and abs(f.y - y0) < 1e-2 / np.sqrt(c)
        assert abs(f.sx * np.sqrt(c) - 1) < 1e-3

    path = tmp_path / "toys.jsonl"
    FakeServer.stop_at = 107
    with pytest.raises(_Stop):
        toys.run(MODEL, "fp32", sizes, gen, mc, checkpoint=path, **kw)
    cp = ToyCheckpoint(path, toys._fingerprint("fixed-model toys", MODEL, "fp32", sizes, gen, mc, 11, 100,
                                               with_errors=True, start_shift=1e-3))
    assert sorted(cp.records) == list(range(7))
    cp.close()

    FakeServer.stop_at, FakeServer.evaluated = None, []
    fits, st = toys.run(MODEL, "fp32", sizes, gen, mc, checkpoint=path, **kw)
    assert st["resumed"] == 7
    assert set(FakeServer.evaluated) == set(range(107, 112))   # only the missing toys were fitted
    assert fits == ref
    # a finished study is read back whole, without a fit
    FakeServer.evaluated = []
    fits, st = toys.run(MODEL, "fp32", sizes, gen, mc, checkpoint=path, **kw)
    assert fits == ref and st["resumed"] == 12 and FakeServer.evaluated == []
    # other arguments: another study
    with pytest.raises(ValueError, match="different study"):
        toys.run(MODEL, "fp32", sizes, gen, mc + 1.0, checkpoint=path, **kw)


# ---- the floating-model study with a fake likelihood context

class FakeContext:
    """Stands in for TDMix: the 'sample' generate() returns is the stream
    plus the envelope, and the NLL is a quadratic in every parameter around a
    point drawn from it.  The envelope of a generate() without one is 42 +
    the stream, so a resumed study that did not reuse the stored envelope
    would fit other samples."""
    stop_at = None
    generated = []

    def __init__(self, model, precision):
        self.stream = None

    def set_floating(self, mask):
        pass

    def load_events(self, data_p4=None, data_t=None, mc_p4=None, mc_w=None):
        if data_p4 is not None:
            self.stream = int(data_p4[0])

    def generate(self, n, seed, stream, params=None, envelope=0.0):
        if FakeContext.stop_at is not None and stream >= FakeContext.stop_at:
            raise _Stop()
        env = envelope if envelope > 0 else 42.0 + stream
        FakeContext.generated.append((stream, env))
        return np.array([stream + env]), np.zeros(1), {"envelope": env}

    def nll(self, p, grad=True):
        g = np.random.default_rng(self.stream)
        c = 1e6
        t = self.gen + 1e-4 * g.normal(size=len(p))
        d = np.asarray(p) - t
        return 0.5 * c * float(d @ d), c * d

    def close(self):
        pass


def test_floating_model_study_resumes_with_the_same_envelope(tmp_path, monkeypatch):
    import paper_1702_06735_gb300.tdmix as tdmix_mod
    monkeypatch.setattr(tdmix_mod, "TDMix", FakeContext)
    gen = _gen()
    FakeContext.gen = gen
    mc = np.zeros((5, 4, 4))
    sizes = [2000] * 6
    kw = dict(seed=3, stream0=50, compare_fixed=True)
    FakeContext.stop_at, FakeContext.generated = None, []
    ref = toys.run_floating(MODEL, "fp64", sizes, gen, mc, **kw)
    assert [e for _, e in FakeContext.generated] == [92.0] * 6  # the first toy's envelope, reused

    path = tmp_path / "floating.jsonl"
    FakeContext.stop_at, FakeContext.generated = 53, []
    with pytest.raises(_Stop):
        toys.run_floating(MODEL, "fp64", sizes, gen, mc, checkpoint=path, **kw)
    FakeContext.stop_at, FakeContext.generated = None, []
    fits = toys.run_floating(MODEL, "fp64", sizes, gen, mc, checkpoint=path, **kw)
    assert FakeContext.generated == [(53, 92.0), (54, 92.0), (55, 92.0)]
    assert len(fits) == len(ref)
    for a, b in zip(fits, ref):
        assert isinstance(a, FloatingFit) and a.converged == b.converged and a.n_eval == b.n_eval
        assert np.array_equal(a.params, b.params) and np.array_equal(a.errors, b.errors, equal_nan=True)
        assert a.xy_fixed_model == b.xy_fixed_model


def test_toyfit_fields_round_trip():
    f = ToyFit(100, 0.1, -0.2, float("nan"), 1e-3, True, 17)
    import dataclasses
    assert ToyFit(**json.loads(json.dumps(dataclasses.asdict(f)))).n_eval == 17
