"""The oracle's Philox4x32-10 (the counter-based generator the GPU event
generator draws from) against the known-answer vectors published with it
(tests/golden/philox4x32_10_kat.json, cited there), plus the properties the
generator relies on: distinct counters or keys give distinct outputs, and
the 53-bit uniform stays in [0, 1)."""
import json
import os

from conftest import GOLDEN_DIR
from oracle.philox import philox4x32_10, u01


def _kat():
    with open(os.path.join(GOLDEN_DIR, "philox4x32_10_kat.json")) as f:
        return json.load(f)["vectors"]


def test_known_answer_vectors():
    for v in _kat():
        got = philox4x32_10([int(x, 16) for x in v["counter"]], [int(x, 16) for x in v["key"]])
        assert got == tuple(int(x, 16) for x in v["out"])


def test_counters_and_keys_give_distinct_words():
    seen = set()
    for c in range(64):
        for k in range(4):
            seen.add(philox4x32_10([c, 0, 7, 1], [k, 0]))
    assert len(seen) == 64 * 4


def test_uniform_range():
    assert u01(0, 0) == 0.0
    top = u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert top < 1.0 and 1.0 - top == 2.0 ** -53
