"""The C-ABI library loads and exports every function include/tdmix.h
declares; the model compiler rejects bad descriptions (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "tdmix.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdmix_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1702_06735_gb300 import tdmix
    if not os.path.exists(tdmix.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return tdmix.load_library()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "tdmix_nll" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1702_06735_gb300 import tdmix
    assert set(_declared()) <= set(tdmix._SIGNATURES)


@pytest.mark.parametrize("bad,needle", [
    ("{", "model JSON"),
    ('{"parent_mass": 1.86}', "missing key"),
])
def test_invalid_model_text(lib, bad, needle):
    ctx = ctypes.c_void_p()
    rc = lib.tdmix_create(bad.encode(), 0, ctypes.byref(ctx))
    assert rc == -1
    assert needle in lib.tdmix_last_error(ctx).decode()
    lib.tdmix_destroy(ctx)


def test_invalid_model_semantics(lib):
    import json
    from conftest import model_path
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["chains"][0]["resonances"] = ["nope", "rho0"]
    ctx = ctypes.c_void_p()
    assert lib.tdmix_create(json.dumps(d).encode(), 0, ctypes.byref(ctx)) == -1
    assert "unknown resonance" in lib.tdmix_last_error(ctx).decode()
    lib.tdmix_destroy(ctx)
    d = json.load(open(model_path("d0_k3pi_2chain")))
    d["chains"][1]["particles"] = [0, 0, 1, 2]
    assert lib.tdmix_create(json.dumps(d).encode(), 0, ctypes.byref(ctx)) == -1
    lib.tdmix_destroy(ctx)
    assert lib.tdmix_create(b"{}", 7, ctypes.byref(ctx)) == -1


def test_null_arguments(lib):
    assert lib.tdmix_nll(None, None, None, None) == -1
    assert lib.tdmix_num_params(None) == -1
    assert lib.tdmix_last_error(None) == b"null context"


def test_model_beyond_the_compiled_specialisations_passes_the_model_checks(lib):
    """A structure none of the shipped model files has (the 2-chain model
    plus a D-wave K*0 rho0 chain) is a valid model: creation gets past the
    model compiler and the structure lookup (the runtime-table kernels take
    it) and, without a GPU, stops only at the first device call."""
    import copy
    import ctypes
    import json
    from conftest import model_path
    d = json.load(open(model_path("d0_k3pi_2chain")))
    extra = copy.deepcopy(d["chains"][0])
    extra.update(name="CF K*0 rho0 D-wave", spin="VV_D", coef=[0.3, 0.1], float=True)
    d["chains"].append(extra)
    ctx = ctypes.c_void_p()
    rc = lib.tdmix_create(json.dumps(d).encode(), 1, ctypes.byref(ctx))
    try:
        if rc == 0:   # a GPU is present
            assert lib.tdmix_kernel_path(ctx) == 2
        else:
            assert rc == -3, lib.tdmix_last_error(ctx)
    finally:
        lib.tdmix_destroy(ctx)
