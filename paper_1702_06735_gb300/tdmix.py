"""Python binding of the tdmix C ABI (include/tdmix.h) via ctypes.

Argument marshalling only: every step of the likelihood runs in the CUDA
kernels of libtdmix.so.  Importing this module does not load the library;
the first use does, and raises if it was not built (there is no CPU
fallback).  Host (NumPy) and device (torch CUDA) arrays are accepted.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdmix.so")
MODEL_DIR = os.path.join(HERE, "amplitude_models")

FP64, FP32 = 0, 1
GENERIC = 0x100      # flag: the runtime-table kernels whatever the structure
KERNEL_PATHS = {0: "fp64", 1: "fp32", 2: "generic"}
LATENCY_ALL, LATENCY_RESIDENT, LATENCY_ADMITTED = 0, 1, 2  # tdmix_latency_kind
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_NOMEM", -3: "ERR_CUDA", -4: "ERR_STATE", -5: "ERR_NONFINITE",
          -6: "ERR_DOMAIN", -7: "ERR_TIMEOUT", -8: "ERR_UNSUPPORTED"}

# Every function the header declares, with its ctypes signature.
_c_p = ctypes.c_void_p
_c_i = ctypes.c_int
_SIGNATURES = {
    "tdmix_create": (_c_i, [ctypes.c_char_p, _c_i, ctypes.POINTER(_c_p)]),
    "tdmix_set_stream": (_c_i, [_c_p, _c_p]),
    "tdmix_num_params": (_c_i, [_c_p]),
    "tdmix_kernel_path": (_c_i, [_c_p]),
    "tdmix_num_components": (_c_i, [_c_p]),
    "tdmix_chain_component": (_c_i, [_c_p, _c_i]),
    "tdmix_default_params": (_c_i, [_c_p, _c_p]),
    "tdmix_set_floating": (_c_i, [_c_p, _c_p]),
    "tdmix_test_withhold_copy": (_c_i, [_c_p, _c_i]),
    "tdmix_recomputed_events": (_c_i, [_c_p, ctypes.POINTER(ctypes.c_int64)]),
    "tdmix_set_gram": (_c_i, [_c_p, _c_i]),
    "tdmix_generate": (_c_i, [_c_p, _c_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, _c_i, _c_p, _c_p, _c_p]),
    "tdmix_test_philox": (_c_i, [_c_p, _c_p, _c_p]),
    "tdmix_test_math": (_c_i, [_c_i, ctypes.c_int64, _c_p, _c_p]),
    "tdmix_load_events": (_c_i, [_c_p, _c_p, _c_p]),
    "tdmix_nll": (_c_i, [_c_p, _c_p, _c_p, _c_p]),
    "tdmix_nll_batch": (_c_i, [_c_p, _c_p, ctypes.c_int64, _c_p, _c_p]),
    "tdmix_event_rates": (_c_i, [_c_p, _c_p, _c_p, _c_p]),
    "tdmix_norm_matrix": (_c_i, [_c_p, _c_p]),
    "tdmix_profile": (_c_i, [_c_p, _c_i]),
    "tdmix_profile_read": (_c_i, [_c_p, _c_p, _c_p, _c_i]),
    "tdmix_loglik_components_noalloc": (_c_i, [_c_i, ctypes.c_int64, _c_p, _c_p, ctypes.c_int64, _c_p, _c_p, _c_p,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _c_p, _c_p]),
    "tdmix_server_create": (_c_i, [ctypes.c_char_p, _c_i, ctypes.c_size_t, _c_i, ctypes.POINTER(_c_p)]),
    "tdmix_server_add_mc": (_c_i, [_c_p, _c_p]),
    "tdmix_server_add_sample": (_c_i, [_c_p, _c_p, ctypes.POINTER(_c_i)]),
    "tdmix_server_add_generated_sample": (_c_i, [_c_p, _c_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.POINTER(_c_i)]),
    "tdmix_server_loop_info": (_c_i, [_c_p, _c_p]),
    "tdmix_server_submit": (_c_i, [_c_p, _c_i, _c_p, ctypes.POINTER(ctypes.c_uint64)]),
    "tdmix_server_wait": (_c_i, [_c_p, ctypes.c_uint64, _c_p, _c_p, ctypes.c_double]),
    "tdmix_server_stats": (_c_i, [_c_p, _c_p, _c_p, _c_p]),
    "tdmix_server_latency": (_c_i, [_c_p, _c_i, _c_p, _c_p, ctypes.POINTER(ctypes.c_int64)]),
    "tdmix_server_reset_stats": (_c_i, [_c_p]),
    "tdmix_server_resident_bytes": (_c_i, [_c_p, ctypes.POINTER(ctypes.c_size_t)]),
    "tdmix_server_last_error": (ctypes.c_char_p, [_c_p]),
    "tdmix_server_destroy": (None, [_c_p]),
    "tdmix_trace": (_c_i, [_c_p, _c_i]),
    "tdmix_trace_read": (_c_i, [_c_p, _c_p, _c_p]),
    "tdmix_last_error": (ctypes.c_char_p, [_c_p]),
    "tdmix_destroy": (None, [_c_p]),
}

_lib = None


class TDMixError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libtdmix.so (built by ``paper_1702_06735_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1702_06735_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


MATH_CODES = {"log_table": 0, "log_cuda": 1, "rcp_f64": 2, "div_f64": 3, "rcp_f32": 4, "div_f32": 5,
              "df_rcp": 6, "mix_tier0": 7, "mix_tier1": 8, "mix_tier2": 9, "log_df": 10, "eqmix_df": 11,
              "eqmix_f64": 12, "rcp_approx_f32": 13}


def test_philox(counter, key):
    """Philox4x32-10 of the device generator (tdmix_test_philox)."""
    lib = load_library()
    c = np.asarray(counter, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    rc = lib.tdmix_test_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise TDMixError(rc, "tdmix_test_philox")
    return tuple(int(x) for x in out)


def test_math(which: str, v) -> np.ndarray:
    """Evaluates one of the kernels' math routines (or the CUDA function it
    replaces) on the device: tdmix_test_math.  Returns n values, or (n, 4)
    (cosh, sinh, cos, sin) for the mixing-series codes; the Eq. (mix) codes
    ("eqmix_df", "eqmix_f64") take (n, 8) records {Ar, Ai, Br, Bi, t, x, y,
    Gamma} and return (n, 4) {ln B, e^{-Gamma t} B, ok, 0}."""
    lib = load_library()
    a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    n = a.shape[0]
    per = 4 if which.startswith("mix") or which.startswith("eqmix") else 1
    out = np.empty(per * n)
    rc = lib.tdmix_test_math(MATH_CODES[which], n, a.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise TDMixError(rc, "tdmix_test_math")
    return out.reshape(n, 4) if per == 4 else out


class Events(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_void_p * 16), ("t", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("on_device", ctypes.c_int)]


def model_json(model) -> str:
    """JSON text of a model given as a shipped name, a path, a dict or text."""
    if isinstance(model, dict):
        return json.dumps(model)
    if isinstance(model, str):
        if model.lstrip().startswith("{"):
            return model
        path = model if os.path.exists(model) else os.path.join(MODEL_DIR, model + ".json")
        with open(path) as f:
            return f.read()
    raise TypeError("model must be a name, path, dict or JSON text")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _planes(p4, t=None, w=None):
    """Marshals (n, 4, 4) momenta (+ times, weights) into an Events struct.
    Returns (struct, keep-alive list)."""
    ev = Events()
    keep = []
    if _is_torch(p4) and p4.is_cuda:
        import torch
        planes = p4.to(torch.float64).permute(1, 2, 0).contiguous()
        n = planes.shape[-1]
        keep.append(planes)
        base = planes.data_ptr()
        for k in range(16):
            ev.p[k] = base + k * n * 8
        for name, arr in (("t", t), ("w", w)):
            if arr is not None:
                a = arr.to(device=planes.device, dtype=torch.float64).contiguous()
                keep.append(a)
                setattr(ev, name, a.data_ptr())
        ev.on_device = 1
    else:
        planes = np.ascontiguousarray(np.transpose(np.asarray(p4, dtype=np.float64), (1, 2, 0)))
        n = planes.shape[-1]
        keep.append(planes)
        base = planes.ctypes.data
        for k in range(16):
            ev.p[k] = base + k * n * 8
        for name, arr in (("t", t), ("w", w)):
            if arr is not None:
                a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64))
                keep.append(a)
                setattr(ev, name, a.ctypes.data)
        ev.on_device = 0
    ev.n = n
    return ev, keep


class TDMix:
    """One likelihood context (tdmix_ctx) on the current CUDA device."""

    def __init__(self, model, precision: str = "fp64", stream=None, generic: bool = False):
        self._lib = load_library()
        self._ctx = ctypes.c_void_p()
        prec = {"fp64": FP64, "fp32": FP32}[precision] | (GENERIC if generic else 0)
        self.precision = precision
        rc = self._lib.tdmix_create(model_json(model).encode(), prec, ctypes.byref(self._ctx))
        if rc != 0:
            msg = self._lib.tdmix_last_error(self._ctx).decode() if self._ctx else ""
            if self._ctx:
                self._lib.tdmix_destroy(self._ctx)
                self._ctx = ctypes.c_void_p()
            raise TDMixError(rc, msg)
        if stream is not None:
            self.set_stream(stream)
        self.n_params = self._lib.tdmix_num_params(self._ctx)
        self.n_components = self._lib.tdmix_num_components(self._ctx)
        # "fp64", "fp32" (structure-specialised kernels) or "generic"
        # (runtime-table kernels, float64: a structure without a compiled
        # specialisation, or generic=True)
        self.kernel_path = KERNEL_PATHS[self._lib.tdmix_kernel_path(self._ctx)]

    def _check(self, rc):
        if rc != 0:
            raise TDMixError(rc, self._lib.tdmix_last_error(self._ctx).decode())

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.tdmix_set_stream(self._ctx, handle))

    def chain_component(self, chain: int) -> int:
        c = self._lib.tdmix_chain_component(self._ctx, chain)
        if c < 0:
            self._check(c)
        return c

    def default_params(self) -> np.ndarray:
        out = np.empty(self.n_params)
        self._check(self._lib.tdmix_default_params(self._ctx, out.ctypes.data))
        return out

    def set_floating(self, mask):
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.int32))
        if m.shape != (self.n_params,):
            raise ValueError("mask length must equal the number of parameters")
        self._check(self._lib.tdmix_set_floating(self._ctx, m.ctypes.data))

    def load_events(self, data_p4=None, data_t=None, mc_p4=None, mc_w=None):
        keep = []
        d = m = None
        if data_p4 is not None:
            d, k = _planes(data_p4, t=data_t)
            keep += k
        if mc_p4 is not None:
            m, k = _planes(mc_p4, w=mc_w)
            keep += k
        self._check(self._lib.tdmix_load_events(self._ctx, ctypes.byref(d) if d else None,
                                                ctypes.byref(m) if m else None))
        if data_p4 is not None:
            self._nd = int(data_p4.shape[0])

    def nll(self, params, grad: bool = True):
        """NLL (and gradient) at host parameters; returns (float, ndarray|None)."""
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        if p.shape != (self.n_params,):
            raise ValueError("parameter vector has the wrong length")
        out = np.empty(1)
        g = np.empty(self.n_params) if grad else None
        self._check(self._lib.tdmix_nll(self._ctx, p.ctypes.data, out.ctypes.data,
                                        g.ctypes.data if grad else None))
        return float(out[0]), g

    def nll_device(self, params, nll_out, grad_out=None):
        """Enqueues an evaluation with device tensors (float64) on the context's stream."""
        self._check(self._lib.tdmix_nll(self._ctx, params.data_ptr(), nll_out.data_ptr(),
                                        grad_out.data_ptr() if grad_out is not None else None))

    def nll_batch(self, params, nll_out, grad_out=None):
        """Enqueues evaluations at every row of `params` (device float64
        [n, num_params]) into nll_out [n] and grad_out [n, num_params] on the
        context's stream; consecutive evaluations overlap on the device."""
        n = int(params.shape[0])
        self._check(self._lib.tdmix_nll_batch(self._ctx, params.data_ptr(), n, nll_out.data_ptr(),
                                              grad_out.data_ptr() if grad_out is not None else None))

    def event_rates(self, params):
        """(per-event rate e^{-Gamma t} B of every data event, normalisation N)."""
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        n = self._n_data
        rates = np.empty(n)
        norm = np.empty(1)
        self._check(self._lib.tdmix_event_rates(self._ctx, p.ctypes.data, rates.ctypes.data, norm.ctypes.data))
        return rates, float(norm[0])

    @property
    def _n_data(self):
        if not hasattr(self, "_nd"):
            raise RuntimeError("load events first")
        return self._nd

    def norm_matrix(self) -> np.ndarray:
        U = self.n_components
        out = np.empty(2 * U * U)
        self._check(self._lib.tdmix_norm_matrix(self._ctx, out.ctypes.data))
        return (out[0::2] + 1j * out[1::2]).reshape(U, U)

    def generate(self, n: int, seed: int, stream: int = 0, params=None, flat: bool = False, with_times: bool = True,
                 fp64_only: bool = False, envelope: float = 0.0):
        """n pseudo-events of the model at `params` (or flat phase space) on
        the GPU: (momenta (n, 4, 4) and times (n,) as CUDA float64 tensors,
        info dict)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        planes = torch.empty(16, n, dtype=torch.float64, device=dev)
        t = torch.empty(n, dtype=torch.float64, device=dev) if with_times else None
        p = None if flat else np.ascontiguousarray(np.asarray(params if params is not None else self.default_params(),
                                                             dtype=np.float64))
        info = np.zeros(4)
        info[0] = envelope
        flags = (1 if flat else 0) | (2 if fp64_only else 0)
        self._check(self._lib.tdmix_generate(self._ctx, None if p is None else p.ctypes.data, n, seed, stream,
                                             flags, planes.data_ptr(), t.data_ptr() if t is not None else None,
                                             info.ctypes.data))
        p4 = planes.view(4, 4, n).permute(2, 0, 1)
        return p4, t, {"envelope": float(info[0]), "candidates": int(info[1]), "efficiency": float(info[2]),
                       "restarts": int(info[3])}

    GRAM_MODES = {"auto": 0, "registers": 1, "tensor": 2}

    def set_gram(self, mode: str):
        """Accumulation of the MC normalisation matrix: "auto", "registers" or
        "tensor" (tcgen05 tensor cores, fp32 path)."""
        self._check(self._lib.tdmix_set_gram(self._ctx, self.GRAM_MODES[mode]))

    def recomputed_events(self) -> int:
        """Data events the last evaluation recomputed in double-float (fp32 path)."""
        n = ctypes.c_int64()
        self._check(self._lib.tdmix_recomputed_events(self._ctx, ctypes.byref(n)))
        return n.value

    def test_withhold_copy(self, enable: bool = True):
        """Test hook: block 0 withholds its first tile copy, so its bounded
        wait runs out and evaluations report TDMIX_ERR_TIMEOUT."""
        self._check(self._lib.tdmix_test_withhold_copy(self._ctx, int(enable)))

    PROF_CLASSES = ("eval", "precompute")

    def profile(self, enable: bool = True):
        """Times every kernel launch of this context with CUDA events."""
        self._check(self._lib.tdmix_profile(self._ctx, int(enable)))

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel class: (total ms, launches)} since the last reset."""
        ms = np.zeros(len(self.PROF_CLASSES))
        n = np.zeros(len(self.PROF_CLASSES), dtype=np.int64)
        self._check(self._lib.tdmix_profile_read(self._ctx, ms.ctypes.data, n.ctypes.data, int(reset)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PROF_CLASSES)}

    TRACE_PHASES = ("start", "constants", "mc_done", "data_done", "partials", "reduced", "nll", "end")

    def trace(self, enable: bool = True):
        """Per-block phase timestamps of the evaluation kernel."""
        self._check(self._lib.tdmix_trace(self._ctx, int(enable)))

    def trace_read(self) -> np.ndarray:
        """(blocks, phases) array of ns stamps of the last evaluation."""
        buf = np.zeros(1024 * len(self.TRACE_PHASES), dtype=np.uint64)
        nb = ctypes.c_int()
        self._check(self._lib.tdmix_trace_read(self._ctx, buf.ctypes.data, ctypes.byref(nb)))
        return buf[:nb.value * len(self.TRACE_PHASES)].reshape(nb.value, len(self.TRACE_PHASES))

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.tdmix_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TDMixServer:
    """Batched, continuously admitted NLL + gradient requests (tdmix_server)."""

    def __init__(self, model, precision: str = "fp32", hbm_budget_bytes: int = 4 << 30, max_slots: int = 256):
        self._lib = load_library()
        self._s = ctypes.c_void_p()
        prec = {"fp64": FP64, "fp32": FP32}[precision]
        rc = self._lib.tdmix_server_create(model_json(model).encode(), prec, hbm_budget_bytes, max_slots,
                                           ctypes.byref(self._s))
        if rc != 0:
            msg = self._lib.tdmix_server_last_error(self._s).decode() if self._s else ""
            self.close()
            raise TDMixError(rc, msg)
        m = json.loads(model_json(model))
        self.n_params = 2 * len(m["chains"]) + 2 * len(m["resonances"]) + 2

    def _check(self, rc):
        if rc != 0:
            raise TDMixError(rc, self._lib.tdmix_server_last_error(self._s).decode())

    def add_mc(self, mc_p4, mc_w=None):
        ev, keep = _planes(mc_p4, w=mc_w)
        self._check(self._lib.tdmix_server_add_mc(self._s, ctypes.byref(ev)))

    def add_sample(self, p4, t) -> int:
        ev, keep = _planes(p4, t=t)
        sid = ctypes.c_int()
        self._check(self._lib.tdmix_server_add_sample(self._s, ctypes.byref(ev), ctypes.byref(sid)))
        return sid.value

    def add_generated_sample(self, params, n: int, seed: int, stream: int) -> int:
        """A pseudo-experiment of n events generated on the device at each
        admission from the model at `params` (seed, stream)."""
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        sid = ctypes.c_int()
        self._check(self._lib.tdmix_server_add_generated_sample(self._s, p.ctypes.data, n, seed, stream,
                                                                ctypes.byref(sid)))
        return sid.value

    def loop_info(self) -> dict:
        v = np.zeros(6, dtype=np.int64)
        self._check(self._lib.tdmix_server_loop_info(self._s, v.ctypes.data))
        return {"launches": int(v[0]), "abnormal_exits": int(v[1]), "published": int(v[2]), "running": bool(v[3]),
                "last_exit_status": int(v[4]), "last_exit_after_us": int(v[5])}

    def submit(self, sample_id: int, params) -> int:
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        tk = ctypes.c_uint64()
        self._check(self._lib.tdmix_server_submit(self._s, sample_id, p.ctypes.data, ctypes.byref(tk)))
        return tk.value

    def wait(self, ticket: int, timeout_s: float = 60.0):
        """(nll, gradient) of a submitted request."""
        v = np.empty(1)
        g = np.empty(self.n_params)
        self._check(self._lib.tdmix_server_wait(self._s, ticket, v.ctypes.data, g.ctypes.data, timeout_s))
        return float(v[0]), g

    def evaluate(self, sample_id: int, params, timeout_s: float = 60.0):
        return self.wait(self.submit(sample_id, params), timeout_s)

    def stats(self) -> dict:
        """p50/p99 latency over all completed requests and throughput; the same
        percentiles for requests on resident samples ("resident") and for those
        that waited for their sample's admission ("admitted"), with counts."""
        a, b, c = np.empty(1), np.empty(1), np.empty(1)
        self._check(self._lib.tdmix_server_stats(self._s, a.ctypes.data, b.ctypes.data, c.ctypes.data))
        out = {"p50_us": float(a[0]), "p99_us": float(b[0]), "evals_per_s": float(c[0])}
        for kind, name in ((LATENCY_RESIDENT, "resident"), (LATENCY_ADMITTED, "admitted")):
            n = ctypes.c_int64()
            self._check(self._lib.tdmix_server_latency(self._s, kind, a.ctypes.data, b.ctypes.data, ctypes.byref(n)))
            out[name] = {"count": int(n.value), "p50_us": float(a[0]), "p99_us": float(b[0])}
        return out

    def reset_stats(self):
        self._check(self._lib.tdmix_server_reset_stats(self._s))

    def resident_bytes(self) -> int:
        b = ctypes.c_size_t()
        self._check(self._lib.tdmix_server_resident_bytes(self._s, ctypes.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "_s", None):
            self._lib.tdmix_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
