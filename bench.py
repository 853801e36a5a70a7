#!/usr/bin/env python
"""Benchmark of the time-dependent D0 -> K+ pi- pi+ pi- likelihood on GB300.

Headline: NLL + gradient evaluations per second of the full model (8 CF + 8
DCS decay chains sharing 8 components, 44 floating parameters) with 50,000
time-dependent pseudo-events (x = 0.49 %, y = 0.61 %) and 1,000,000 flat
phase-space MC events, on the fp32 precision path, with the plain fp64 path
beside it.  One step is one NLL + gradient evaluation in which every
parameter moved, so every per-evaluation step runs: lineshapes, components,
the MC normalisation matrix, Eq. (mix) per data event, the fixed-order
reductions and the adjoint.  Every sample is generated on the device
(Philox4x32-10, GENBOD phase space, accept/reject on the model's rate) and
stays resident; event ingest and the parameter-independent precompute run
once per sample (load_ms).

The same JSON line carries the other measured configurations:
  config1_latency      2-chain model, 1,000 events + 10,000 MC: one fp64 NLL
  change_classes       the headline workload per class of parameter change
  config3_precision    2-chain model at 10M + 10M events: fp32 against fp64
                       per result, timings; the 16-component normalisation
                       matrix over 10M MC per accumulation mode; the cached
                       data pass against the HBM roofline at 10M events
  config4_gradient_fit 16-chain model at 1M + 2M: gradient against central
                       finite differences, wall time of a gradient fit
  paper_fit_benchmark  the fit of the paper's timing table (Sec. 5)
  toy_study            1,000 pseudo-experiments on the serving loop
  sensitivity          sigma(x), sigma(y) and pulls at 20k / 50k / 70k events

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tdmix|reference]

With N > 1 (torchrun) every rank evaluates an independent replica problem
(its own seeded sample); the value is the sum over ranks ("replicas only":
the likelihood of one sample is not sharded).  --impl reference times the
CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "NLL+grad evals/s (50k data, 1M MC) vs FP64 path; toy-study p50/p99 eval latency"
MODEL = "d0_k3pi_full"
MODEL_2CHAIN = "d0_k3pi_2chain"
MODEL_U16 = "d0_k3pi_full_nodedup"
N_DATA, N_MC = 50_000, 1_000_000
KEY0 = 1702067350                    # Philox key of configuration k is KEY0 + k
STREAM_DATA, STREAM_MC, STREAM_TOY0 = 0, 1, 1000
REF_BUDGET_S = 150.0                 # wall time the reference arm's steps may take


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="tdmix", choices=["tdmix", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--studies", default="all", choices=["all", "none"],
                    help="'none': the headline, isolated launches and e2e only (profiling runs)")
    ap.add_argument("--toys", type=int, default=1000, help="pseudo-experiments of the fp32 toy study (0: skip)")
    ap.add_argument("--toys-fp64", type=int, default=200, help="the first toys of the study run again on fp64")
    ap.add_argument("--sensitivity", type=int, default=100, help="toys per sample size of the sensitivity study")
    ap.add_argument("--cached-only", type=int, default=0, metavar="N",
                    help="only the cached data pass of the 16-chain model at N events (profiling runs)")
    ap.add_argument("--flush-l2", action="store_true",
                    help="write 256 MB between timed steps (default: none; the inputs of one evaluation exceed L2)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_streams(replica: int):
    """Sample streams (data, MC) of replica `replica`: rank 0 takes the
    workload's own streams, every other rank a distinct pair."""
    if replica == 0:
        return STREAM_DATA, STREAM_MC
    return 10 + 2 * replica, 11 + 2 * replica


def max_over_ranks(values, world: int, device=None):
    """Element-wise maximum of per-rank timings over all ranks (every rank
    gets the result)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as tdist
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def model_path(name=MODEL):
    return os.path.join(HERE, "paper_1702_06735_gb300", "amplitude_models", name + ".json")


def model_sizes(name=MODEL):
    with open(model_path(name)) as f:
        m = json.load(f)
    return len(m["chains"]), len(m["resonances"])


def kernel_source_digest():
    """sha256 over the sources the evaluation kernel is compiled from
    (eval_inst.cu, which instantiates and launches it, and the headers that
    define it; not the generator's or the serving loop's, sorted by name)."""
    d = os.path.join(HERE, "paper_1702_06735_gb300", "csrc")
    names = ["async_copy.cuh", "device_tables.hpp", "df.cuh", "eval.cuh", "eval_inst.cu", "fused.cuh", "gram_tc.cuh",
             "kernels.hpp", "kinematics.cuh", "model.hpp", "tcgen05.cuh"]
    h = hashlib.sha256()
    for n in sorted(names):
        h.update(n.encode())
        with open(os.path.join(d, n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


# DRAM bytes read + written by one launch of the headline evaluation kernel
# (k_eval, fp32 path, all parameters moved), from one ncu capture with warm
# caches (the second of two captured launches of `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum --cache-control none -k
# regex:k_eval -s 5 -c 2 python bench.py --studies none --steps 5 --warmup 3
# --no-cpu-baseline`); valid only for the kernel sources of the digest below
# (the figure is reported as null once the sources change).  The capture ran
# on sources whose only difference from these is how the cached pass's
# finish sums the coefficient residue term (serially rather than over a
# warp); the full evaluation measured here compiles none of that code.
TRAFFIC = {"bytes_per_launch": 141791488 + 4130816, "sources_sha256": "2da986de3cd6cce09d14f6b69dac5afc424cc854e292d7a31e72fe37276bcf33"}


def step_params(p0, move, k: int):
    """Parameter vector of step k: every parameter of the mask moved by a
    seeded relative 1e-3 (so masses and widths, when moved, change)."""
    g = np.random.default_rng(1000 + k)
    p = p0.copy()
    for i in range(len(p)):
        if move[i]:
            p[i] *= 1 + 1e-3 * g.normal()
    return p


def class_masks(n_params, nc, nr):
    """(all parameters but the fixed reference coefficient; coefficients and
    x, y only; masses and widths only)"""
    every = np.ones(n_params, dtype=bool)
    every[[0, 1]] = False
    coef_xy = every.copy()
    coef_xy[2 * nc:2 * nc + 2 * nr] = False
    res = np.zeros(n_params, dtype=bool)
    res[2 * nc:2 * nc + 2 * nr] = True
    return every, coef_xy, res


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """SM clock and clock-event reasons polled every 0.2 ms through NVML's
    read-only queries while the timed region runs (nvidia-smi at 200 ms
    where NVML is not available)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, device):
        self.samples = []
        self.stop_flag = False
        self.lib = None
        self.smi = None
        self.max_mhz = None
        try:
            import torch
            props = torch.cuda.get_device_properties(device)
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            rc = -1
            u = str(getattr(props, "uuid", ""))
            if u:
                rc = lib.nvmlDeviceGetHandleByUUID((u if u.startswith("GPU-") else "GPU-" + u).encode(), ctypes.byref(h))
            if rc != 0 and hasattr(props, "pci_bus_id"):
                bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
                rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h))
            if rc != 0:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device.index or 0), ctypes.byref(h))
            if rc != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))      # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.lib, self.h = lib, h
        except (OSError, AttributeError, RuntimeError, ImportError):
            self.lib = None

    def _poll(self):
        c, r = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop_flag:
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0 and \
                    self.reasons_fn(self.h, ctypes.byref(r)) == 0:
                self.samples.append((time.perf_counter(), float(c.value), int(r.value)))
            time.sleep(0.0002)

    def _read_smi(self):
        for line in self.smi.stdout:
            f = [x.strip() for x in line.split(",")]
            try:
                mask = sum(bit for bit, v in zip((0x8, 0x40, 0x20, 0x4), f[2:6]) if v.lower() == "active")
                self.samples.append((time.perf_counter(), float(f[0]), mask))
                self.max_mhz = float(f[1])
            except (ValueError, IndexError):
                continue

    def start(self):
        if self.lib is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
        else:
            try:
                self.smi = subprocess.Popen(
                    ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                     "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                     "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                self.smi = None
                return self
            self.t = threading.Thread(target=self._read_smi, daemon=True)
        self.t.start()
        return self

    def stop(self, t_begin, t_end):
        """Summary of the samples taken between t_begin and t_end
        (perf_counter); the nearest sample on each side where none fell
        inside."""
        if self.smi is not None:
            time.sleep(0.25)
            self.smi.terminate()
            try:
                self.smi.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.smi.kill()
        self.stop_flag = True
        if getattr(self, "t", None) is not None:
            self.t.join(timeout=2)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no clock samples"], "samples": 0}
        inside = [s for s in self.samples if t_begin <= s[0] <= t_end]
        used = inside
        if not inside:
            before = [s for s in self.samples if s[0] < t_begin][-1:]
            after = [s for s in self.samples if s[0] > t_end][:1]
            used = before + after
        reasons = sorted({name for _, _, m in used for bit, name in self.REASONS.items() if m & bit})
        return {"sm_mhz": statistics.median(s[1] for s in used), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(used), "in_timed_region": len(inside),
                "source": "NVML, 0.2 ms polling" if self.lib is not None else "nvidia-smi, 200 ms"}


def measured_peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(data, t, mc, evals: int, threads: int, warmup: int = 0, name=MODEL):
    """Seconds per NLL + gradient evaluation of the oracle on the given
    events with `threads` intra-op threads (every parameter moved)."""
    import torch
    from oracle import tdamp
    old = torch.get_num_threads()
    torch.set_num_threads(threads)
    try:
        m = tdamp.load_model(model_path(name))
        d, tt, mm = (torch.from_numpy(np.ascontiguousarray(a)) for a in (data, t, mc))
        p0 = m.default_params().numpy()
        every, _, _ = class_masks(len(p0), *model_sizes(name))
        for k in range(warmup):
            tdamp.nll_and_grad(m, d, tt, mm, step_params(p0, every, k))
        t0 = time.perf_counter()
        for k in range(evals):
            tdamp.nll_and_grad(m, d, tt, mm, step_params(p0, every, warmup + k))
        return (time.perf_counter() - t0) / evals, torch.get_num_threads()
    finally:
        torch.set_num_threads(old)


def cpu_baseline(data, t, mc):
    """The oracle on this workload's own events (copied to the host): all host
    cores, then one core."""
    n = host_cores()
    s_all, used = time_oracle(data, t, mc, evals=2, threads=n)
    s_one, _ = time_oracle(data, t, mc, evals=1, threads=1)
    return {"value": 1.0 / s_all, "unit": "evals/s", "cores": used, "kind": "oracle",
            "sample": f"the full workload ({len(t)} data + {len(mc)} MC events of this run), 2 NLL + gradient "
                      f"evaluations on {used} threads ({2 * s_all:.1f} s) and 1 on one thread",
            "one_core": {"value": 1.0 / s_one, "unit": "evals/s", "cores": 1, "seconds": s_one},
            "nproc": n}


def run_reference(args):
    """The oracle as the reference arm: every step one NLL + gradient
    evaluation of the oracle on the headline workload's configuration (same
    model and sizes) on all host cores.  The data events are flat phase
    space with exponential decay times: the oracle does the same arithmetic
    for every event wherever it lies, and drawing the accept/reject sample
    with the oracle's own rate costs minutes of host time (the GPU arm's
    cpu_baseline times the oracle on that run's own accept/reject events).
    If K + W full evaluations would take longer than REF_BUDGET_S, each
    step evaluates the same fraction of the data and MC events and the rate
    is scaled to the full workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import tdamp
    from paper_1702_06735_gb300 import samples
    n = host_cores()
    m = tdamp.load_model(model_path())
    g = samples.rng(KEY0 + 2, STREAM_DATA)
    data = samples.flat_phase_space(N_DATA, g)
    t = samples.exponential_times(N_DATA, m.gamma, g)
    mc = samples.flat_phase_space(N_MC, samples.rng(KEY0 + 2, STREAM_MC))
    # one untimed calibration evaluation of the full workload
    s_full, used = time_oracle(data, t, mc, evals=1, threads=n)
    frac = min(1.0, REF_BUDGET_S / (max(args.steps + args.warmup, 1) * s_full))
    nd, nm = max(256, int(N_DATA * frac)), max(256, int(N_MC * frac))
    frac = (nd + nm) / (N_DATA + N_MC)
    s, used = time_oracle(data[:nd], t[:nd], mc[:nm], evals=max(args.steps, 1), threads=n, warmup=args.warmup)
    value = frac / s
    whole = "the full workload" if frac == 1 else "a fraction of it; rate scaled by event count"
    sample = (f"{nd} data + {nm} MC events per step ({whole}), {args.steps} timed NLL + gradient evaluations "
              f"on {used} threads; data events flat in phase space with exponential decay times")
    out = {"metric": METRIC, "impl": "reference", "value": value, "unit": "evals/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * s,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{MODEL}: 16 chains, 44 floating params, {N_DATA} data + {N_MC} MC events",
                      "parallelism": "replicas"},
           "cpu_baseline": {"value": value, "unit": "evals/s", "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "calibration_s_per_full_eval": s_full}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------
# GPU helpers
# ----------------------------------------------------------------------------
def generate(ctx, n, config, stream, params=None, flat=False, with_times=True):
    """n device events of configuration `config` (Philox key KEY0 + config)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p4, t, info = ctx.generate(n, seed=KEY0 + config, stream=stream, params=params, flat=flat, with_times=with_times)
    torch.cuda.synchronize()
    info["seconds"] = time.perf_counter() - t0
    info["events_per_s"] = n / info["seconds"]
    return p4, t, info


def load(name, precision, data, t, mc, stream=None):
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(name, precision, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c.load_events(data, t, mc)
    torch.cuda.synchronize()
    return c, (time.perf_counter() - t0) * 1e3


def device_steps(c, dev, stream, K, W, move, flush=None, sampler=None, batch=False):
    """K timed evaluations with device parameters (every evaluation a full
    one) bracketed by device synchronisations.  batch=False: one call per
    evaluation, CUDA events around each (an isolated launch each);
    batch=True: one tdmix_nll_batch call for the K evaluations (consecutive
    evaluations overlap on the device), CUDA events around it.  Returns
    (per-evaluation ms, wall s, {kernel class: (ms, launches)}, clocks)."""
    import torch
    p0 = c.default_params()
    P = torch.from_numpy(np.stack([step_params(p0, move, k) for k in range(K + W)])).to(dev)
    out = torch.empty(K + W, dtype=torch.float64, device=dev)
    grad = torch.empty(K + W, len(p0), dtype=torch.float64, device=dev)
    if batch:
        if W > 0:
            c.nll_batch(P[:W], out[:W], grad[:W])
    else:
        for k in range(W):
            c.nll_device(P[k], out[k:k + 1], grad[k])
    torch.cuda.synchronize(dev)
    c.profile(True)
    c.profile_read(reset=True)
    n_ev = 1 if batch else K
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_ev)]
    if sampler is not None:
        sampler.start()
        time.sleep(0.01)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    if batch:
        ev[0][0].record(stream)
        c.nll_batch(P[W:], out[W:], grad[W:])
        ev[0][1].record(stream)
    else:
        for k in range(K):
            if flush is not None:
                flush.zero_()
            ev[k][0].record(stream)
            c.nll_device(P[W + k], out[W + k:W + k + 1], grad[W + k])
            ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    clocks = sampler.stop(t0, t1) if sampler is not None else None
    ms = [ev[0][0].elapsed_time(ev[0][1]) / K] * K if batch else [a.elapsed_time(b) for a, b in ev]
    prof = c.profile_read(reset=True)
    c.profile(False)
    if not torch.isfinite(out).all():
        raise RuntimeError("non-finite NLL in the timed region")
    return ms, t1 - t0, prof, clocks


def host_steps(c, K, W, move, seed0=5000):
    """K evaluations through the C ABI with host parameters (H2D of the
    parameters, D2H of NLL and gradient inside each call); the library's
    CUDA-event profile gives the kernel time.  Returns (evals/s, kernel
    ms per evaluation, launches)."""
    import torch
    p0 = c.default_params()
    ps = [step_params(p0, move, seed0 + k) for k in range(K + W)]
    for k in range(W):
        c.nll(ps[k])
    torch.cuda.synchronize()
    c.profile(True)
    c.profile_read(reset=True)
    t0 = time.perf_counter()
    for k in range(K):
        c.nll(ps[W + k])
    dt = time.perf_counter() - t0
    prof = c.profile_read(reset=True)
    c.profile(False)
    ms, n = prof["eval"]
    return K / dt, ms / max(n, 1), n


def median_ms(ms):
    return statistics.median(ms)


# ----------------------------------------------------------------------------
# roofline bookkeeping
# ----------------------------------------------------------------------------
def full_eval_bytes(n_data, n_mc, NS=7, NX=4, U=8, NO=2):
    """Algorithmic bytes of one full fp32 evaluation: per event the
    invariants (hi + lo fp32), width factors and spin x barrier factors; per
    data event also its decay time (f64) and the component cache written
    back (U complex fp32)."""
    plane = NS * 8 + NX * 4 + U * NO * 4
    return n_mc * plane + n_data * (plane + 8 + 2 * U * 4)


def cached_eval_bytes(n_data, U, es):
    """Algorithmic bytes of one cached data pass: the component cache (U
    complex) and the decay time (f64) per event."""
    return n_data * (2 * U * es + 8)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------
def config1_latency(dev, reps=200):
    """2-chain model, 1,000 events + 10,000 MC: latency of one fp64 NLL +
    gradient through the C ABI (every parameter moved, so every step runs)."""
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix
    g = TDMix(MODEL_2CHAIN, "fp64")
    p0 = g.default_params()
    data, t, _ = generate(g, 1000, 1, STREAM_DATA, params=p0)
    mc, _, _ = generate(g, 10_000, 1, STREAM_MC, flat=True, with_times=False)
    g.close()
    c, load_ms = load(MODEL_2CHAIN, "fp64", data, t, mc)
    every, _, _ = class_masks(len(p0), *model_sizes(MODEL_2CHAIN))
    ps = [step_params(p0, every, k) for k in range(reps + 10)]
    for k in range(10):
        c.nll(ps[k])
    lat = []
    c.profile(True)
    c.profile_read(reset=True)
    for k in range(reps):
        t0 = time.perf_counter()
        c.nll(ps[10 + k])
        lat.append((time.perf_counter() - t0) * 1e6)
    ms, n = c.profile_read(reset=True)["eval"]
    c.close()
    lat.sort()
    return {"workload": f"{MODEL_2CHAIN}: 1000 accept/reject events, 10000 flat MC, fp64",
            "latency_us_p50": lat[len(lat) // 2], "latency_us_p99": lat[int(0.99 * (len(lat) - 1))],
            "kernel_us": 1e3 * ms / max(n, 1), "load_ms": load_ms, "evals": reps}


def change_classes(c64, c32, nc, nr, K):
    """NLL + gradient evaluations per second of the headline workload for
    (i) coefficients and x, y moved (cached components and normalisation
    matrix), (ii) masses and widths moved too (full evaluation), host
    parameters through the C ABI.  The minimiser mix is measured by the
    full-model fit (config 2's fit)."""
    out = {}
    for prec, c in (("fp32", c32), ("fp64", c64)):
        n_p = c.n_params
        every, coef_xy, _ = class_masks(n_p, nc, nr)
        fl = np.zeros(n_p, dtype=np.int32)
        fl[coef_xy] = 1
        c.set_floating(fl)
        c.nll(c.default_params())
        v_i, k_i, _ = host_steps(c, K, 5, coef_xy, seed0=7000)
        fl[:] = 0
        fl[every] = 1
        c.set_floating(fl)
        v_ii, k_ii, _ = host_steps(c, K, 5, every, seed0=8000)
        out[prec] = {"coefficients_xy": {"evals_per_s": v_i, "kernel_us": 1e3 * k_i},
                     "masses_widths": {"evals_per_s": v_ii, "kernel_us": 1e3 * k_ii}}
    return out


def full_model_fit(c32, nc, nr, label, start=None):
    """A complete amplitude fit (every coefficient, mass and width floating;
    x and y fixed: with the coefficient phases free they are nearly
    degenerate at first order in Gamma t) from a seeded start away from the
    generating values, BFGS with the library's NLL + gradient through the
    host-buffer path.  Reports the fraction of evaluations that moved a
    mass or width (the minimiser's mix of change classes)."""
    from paper_1702_06735_gb300 import minimize
    p0 = c32.default_params()
    fl = np.ones(len(p0), dtype=np.int32)
    fl[[0, 1, len(p0) - 2, len(p0) - 1]] = 0
    c32.set_floating(fl)
    if start is None:
        g = np.random.default_rng(777)
        start = p0.copy()
        start[2:2 * nc] *= 1 + 0.02 * g.normal(size=2 * nc - 2)
        start[2 * nc:2 * nc + 2 * nr:2] *= 1 + 0.001 * g.normal(size=nr)
        start[2 * nc + 1:2 * nc + 2 * nr:2] *= 1 + 0.01 * g.normal(size=nr)
    inner = minimize.safe_objective(c32)
    last = [None]
    moved = [0, 0]

    def fg(p):
        r = p[2 * nc:2 * nc + 2 * nr]
        moved[0 if last[0] is not None and np.array_equal(r, last[0]) else 1] += 1
        last[0] = r.copy()
        return inner(p)
    t0 = time.perf_counter()
    # MINUIT's default stop (tolerance 0.1: distance to minimum below 2e-4)
    fr = minimize.bfgs(fg, start, floating=fl.astype(bool), scale=minimize.default_scales(start, nc, nr),
                       gtol=1e-2, edm_tol=2e-4, max_iter=400)
    wall = time.perf_counter() - t0
    return {"fit_s": wall, "evals": int(fr.n_eval), "evals_per_s": fr.n_eval / wall, "converged": bool(fr.converged),
            "message": fr.message, "floating_params": int(fl.sum()), "nll": float(fr.fun),
            "fraction_moving_masses_widths": moved[1] / max(sum(moved), 1), "note": label, "x": fr.x.tolist()}


def config3_precision(dev, stream, peak):
    """Config 3: the 2-chain model at 10M data + 10M MC, fp32 against fp64
    for every result; the 16-chain model's normalisation matrix over 10M MC
    in each accumulation mode (U = 8 and, without cross-amplitude dedup,
    U = 16); the cached data pass of the 16-chain model at 10M events
    against the HBM roofline."""
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix
    out = {}
    # --- precision errors, 2-chain model ---
    g = TDMix(MODEL_2CHAIN, "fp64")
    p0 = g.default_params()
    data, t, gi = generate(g, 10_000_000, 3, STREAM_DATA, params=p0)
    mc, _, mi = generate(g, 10_000_000, 3, STREAM_MC, flat=True, with_times=False)
    g.close()
    nc, nr = model_sizes(MODEL_2CHAIN)
    every, coef_xy, _ = class_masks(len(p0), nc, nr)
    p = step_params(p0, every, 31)
    res = {}
    for prec in ("fp64", "fp32"):
        c, load_ms = load(MODEL_2CHAIN, prec, data, t, mc, stream)
        R, N = c.event_rates(p)
        rec = c.recomputed_events() if prec == "fp32" else 0
        v, gr = c.nll(p)
        I = c.norm_matrix()
        ms, _, prof, _ = device_steps(c, dev, stream, 5, 2, every)
        fl = np.zeros(len(p0), dtype=np.int32)
        fl[coef_xy] = 1
        c.set_floating(fl)
        c.nll(p0)
        v_c, k_c, _ = host_steps(c, 20, 3, coef_xy)
        res[prec] = (R, N, v, gr, I, rec)
        U = c.n_components
        es = 4 if prec == "fp32" else 8
        cb = cached_eval_bytes(len(t), U, es)
        out[f"2chain_{prec}"] = {"full_eval_ms": median_ms(ms), "load_ms": load_ms,
                                 "cached_pass_us": 1e3 * k_c, "cached_pass_gbs": cb / (k_c * 1e-3) / 1e9,
                                 "cached_pass_frac_hbm": cb / (k_c * 1e-3) / 1e9 / peak,
                                 "cached_pass_bytes": cb}
        c.close()
        del R
    R64, N64, v64, g64, I64, _ = res["fp64"]
    R32, N32, v32, g32, I32, rec = res["fp32"]
    rel = np.abs(R32 / R64 - 1)
    gs = np.maximum(np.abs(g64), 1e-3 * np.abs(g64).max())
    out["errors_fp32_vs_fp64"] = {
        "rate_rel_max": float(rel.max()), "rate_rel_median": float(np.median(rel)),
        "events_recomputed": int(rec), "norm_rel": abs(N32 / N64 - 1), "nll_abs": abs(v32 - v64),
        "grad_rel_max": float(np.max(np.abs(g32 - g64) / gs)),
        "norm_matrix_rel_max": float(np.abs(I32 - I64).max() / np.abs(I64).max()),
        "note": "the fp64 path is pinned to the oracle at 1e-12 by the parity tests"}
    out["generation"] = {"data": gi, "mc": mi}
    del data, t, mc, res, R64, R32
    torch.cuda.empty_cache()

    # --- 16-component normalisation matrix over 10M MC, and the cached pass ---
    g = TDMix(MODEL, "fp64")
    p0 = g.default_params()
    data, t, gi = generate(g, 10_000_000, 3, 10, params=p0)
    mc, _, _ = generate(g, 10_000_000, 3, 11, flat=True, with_times=False)
    g.close()
    nc, nr = model_sizes(MODEL)
    every, coef_xy, _ = class_masks(len(p0), nc, nr)
    gram = {}
    mats = {}
    small = slice(0, 50_000)
    for name, prec, mode in ((MODEL, "fp32", "registers"), (MODEL, "fp32", "tensor"), (MODEL, "fp64", "auto"),
                             (MODEL_U16, "fp32", "tensor"), (MODEL_U16, "fp64", "auto")):
        c, _ = load(name, prec, data[small], t[small], mc, stream)
        c.set_gram(mode)
        ms, _, _, _ = device_steps(c, dev, stream, 5, 2, every)
        c.nll(p0)
        mats[(name, prec, mode)] = c.norm_matrix()
        U = c.n_components
        gram[f"U{U}_{prec}_{mode}"] = {"full_eval_ms": median_ms(ms), "ns_per_mc_event": 1e6 * median_ms(ms) / len(mc)}
        c.close()
    for (name, prec, mode), I in mats.items():
        ref = mats[(name, "fp64", "auto")]
        gram[f"U{I.shape[0]}_{prec}_{mode}"]["rel_err_vs_fp64"] = float(np.abs(I - ref).max() / np.abs(ref).max())
    out["norm_matrix_10M_mc"] = {"workload": f"16-chain model, 50000 data + {len(mc)} MC events, full evaluations "
                                             "(all parameters moved)", **gram}
    c, load_ms = load(MODEL, "fp32", data, t, mc, stream)
    fl = np.zeros(len(p0), dtype=np.int32)
    fl[coef_xy] = 1
    c.set_floating(fl)
    c.nll(p0)
    v_c, k_c, _ = host_steps(c, 50, 5, coef_xy)
    cb = cached_eval_bytes(len(t), c.n_components, 4)
    fl[:] = 0
    fl[every] = 1
    c.set_floating(fl)
    ms, _, _, _ = device_steps(c, dev, stream, 5, 2, every)
    fb = full_eval_bytes(len(t), len(mc))
    c.close()
    out["cached_data_pass_16chain_10M"] = {
        "kernel_us": 1e3 * k_c, "algorithmic_bytes": cb, "bytes_per_event": cb / len(t),
        "achieved_gbs": cb / (k_c * 1e-3) / 1e9, "frac_hbm": cb / (k_c * 1e-3) / 1e9 / peak,
        "full_eval_ms": median_ms(ms), "full_eval_gbs": fb / (median_ms(ms) * 1e-3) / 1e9,
        "full_eval_frac_hbm": fb / (median_ms(ms) * 1e-3) / 1e9 / peak, "load_ms": load_ms,
        "generation": gi}
    del data, t, mc
    torch.cuda.empty_cache()
    return out


def cached_pass(dev, stream, n_events, peak, steps=20):
    """The cached data pass (coefficients and x, y moved; component cache
    and stored normalisation reused) of the 16-chain model at n_events
    generated events, fp32 path: kernel time per evaluation and its
    algorithmic bytes against the HBM roofline."""
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix
    g = TDMix(MODEL, "fp64")
    p0 = g.default_params()
    data, t, _ = generate(g, n_events, 3, 10, params=p0)
    mc, _, _ = generate(g, 100_000, 3, 11, flat=True, with_times=False)
    g.close()
    nc, nr = model_sizes(MODEL)
    _, coef_xy, _ = class_masks(len(p0), nc, nr)
    c, load_ms = load(MODEL, "fp32", data, t, mc, stream)
    fl = np.zeros(len(p0), dtype=np.int32)
    fl[coef_xy] = 1
    c.set_floating(fl)
    c.nll(p0)
    v, k_ms, n = host_steps(c, steps, 3, coef_xy)
    cb = cached_eval_bytes(n_events, c.n_components, 4)
    c.close()
    del data, t, mc
    torch.cuda.empty_cache()
    return {"events": n_events, "kernel_us": 1e3 * k_ms, "launches": n, "algorithmic_bytes": cb,
            "achieved_gbs": cb / (k_ms * 1e-3) / 1e9, "frac_hbm": cb / (k_ms * 1e-3) / 1e9 / peak,
            "evals_per_s_host_calls": v}


def config4_gradient_fit(dev, stream):
    """Config 4: the 16-chain model at 1M data + 2M MC: the fp64 adjoint
    gradient against central finite differences (h = 1e-6 max(|theta|,
    1e-3)) for every floating parameter, and the wall time of a gradient fit:
    the fp32 path down to its rounding-noise floor, then the fp64 path from
    there to the distance-to-minimum stop."""
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix
    g = TDMix(MODEL, "fp64")
    p0 = g.default_params()
    data, t, _ = generate(g, 1_000_000, 4, STREAM_DATA, params=p0)
    mc, _, _ = generate(g, 2_000_000, 4, STREAM_MC, flat=True, with_times=False)
    g.close()
    nc, nr = model_sizes(MODEL)
    every, _, _ = class_masks(len(p0), nc, nr)
    p = step_params(p0, every, 41)
    c64, _ = load(MODEL, "fp64", data, t, mc, stream)
    _, gr = c64.nll(p)
    fd = np.zeros(len(p))
    t0 = time.perf_counter()
    for i in np.flatnonzero(every):
        h = 1e-6 * max(abs(p[i]), 1e-3)
        a, b = p.copy(), p.copy()
        a[i] += h
        b[i] -= h
        fd[i] = (c64.nll(a, grad=False)[0] - c64.nll(b, grad=False)[0]) / (2 * h)
    fd_s = time.perf_counter() - t0
    idx = np.flatnonzero(every)
    gmax = np.abs(gr[idx]).max()
    big = idx[np.abs(gr[idx]) > 1e-2 * gmax]
    # fp32 to its noise floor, then fp64 from the fp32 optimum (the fp32
    # NLL of 1M events carries ~1e-2 of rounding noise, above the
    # distance-to-minimum target)
    c32, load_ms = load(MODEL, "fp32", data, t, mc, stream)
    fit32 = full_model_fit(c32, nc, nr, f"{len(t)} events, {len(mc)} MC, fp32 path, host-buffer evaluations")
    c32.close()
    fit64 = full_model_fit(c64, nc, nr, "fp64 path from the fp32 result", start=np.asarray(fit32.pop("x")))
    fit64.pop("x")
    c64.close()
    del data, t, mc
    torch.cuda.empty_cache()
    return {"workload": f"{MODEL}: 1,000,000 accept/reject events, 2,000,000 flat MC",
            "grad_vs_central_fd": {"max_abs_over_max_grad": float(np.abs(fd[idx] - gr[idx]).max() / gmax),
                                   "max_rel_components_above_1pct_of_max": float(
                                       np.max(np.abs(fd[big] - gr[big]) / np.abs(gr[big]))),
                                   "params": int(len(idx)), "seconds": fd_s,
                                   "note": "fp64 path; h = 1e-6 max(|theta|, 1e-3); central differences of an NLL "
                                           "of magnitude 7e5 carry ~1e-10 relative rounding noise"},
            "gradient_fit": {"fp32_stage": fit32, "fp64_stage": fit64,
                             "fit_s": fit32["fit_s"] + fit64["fit_s"], "evals": fit32["evals"] + fit64["evals"],
                             "converged": fit64["converged"]},
            "load_ms": load_ms}


def paper_fit_benchmark(dev, stream, mc_sizes=(750_000, 1_500_000, 3_000_000, 6_000_000)):
    """The fit of the paper's timing table (Sec. 5): 100,000 pseudo-events,
    fixed model, x and y floating, normalisation samples of 0.75M - 6M
    points; wall time of a complete fit (BFGS, strong-Wolfe line search,
    MINUIT-style distance-to-minimum stop) including the first evaluation
    that computes the normalisation matrix.  The paper's table reports the
    same fit on its hardware: context, not a target."""
    import torch
    from paper_1702_06735_gb300 import minimize
    from paper_1702_06735_gb300.tdmix import TDMix
    g = TDMix(MODEL, "fp64")
    p0 = g.default_params()
    data, t, _ = generate(g, 100_000, 6, STREAM_DATA, params=p0)
    mc_all, _, _ = generate(g, max(mc_sizes), 6, STREAM_MC, flat=True, with_times=False)
    g.close()
    mask = np.zeros(len(p0), dtype=bool)
    mask[-2:] = True
    scale = np.ones(len(p0))
    scale[-2:] = 1e-3
    out = []
    for n_mc in mc_sizes:
        c, _ = load(MODEL, "fp32", data, t, mc_all[:n_mc], stream)
        c.set_floating(mask.astype(np.int32))
        x0 = p0.copy()
        x0[-2] += 0.001
        x0[-1] -= 0.001
        fg = minimize.safe_objective(c)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = minimize.bfgs(fg, x0, floating=mask, scale=scale, gtol=1e-3, edm_tol=1e-6, max_iter=100)
        wall = time.perf_counter() - t0
        out.append({"mc_points": n_mc, "fit_s": wall, "evals": int(r.n_eval), "converged": bool(r.converged),
                    "x": float(r.x[-2]), "y": float(r.x[-1])})
        c.close()
    return {"data_events": len(t), "precision": "fp32", "fits": out,
            "note": "fixed model, x and y floating; includes the evaluation that computes the normalisation"}


def toy_study(precision, sizes, mc, p0, label):
    """Pseudo-experiments generated on the device at admission, each fitted
    (x, y floating) by its own BFGS minimiser submitting NLL + gradient
    requests to the device-resident serving loop; 4 GB HBM budget."""
    from paper_1702_06735_gb300 import toys
    budget = 4 << 30
    fits, st = toys.run(MODEL, precision, sizes, p0, mc, seed=KEY0 + 5, stream0=STREAM_TOY0, clients=16,
                        budget_bytes=budget)
    evals = sum(f.n_eval for f in fits)
    event_evals = sum(f.n_eval * f.n_events for f in fits)
    return {"workload": label, "toys": len(sizes), "events_total": int(sum(sizes)), "min_events": int(min(sizes)),
            "max_events": int(max(sizes)), "clients": 16, "hbm_budget_bytes": budget, "evals": evals,
            "p50_us": st["p50_us"], "p99_us": st["p99_us"], "evals_per_s": st["evals_per_s"],
            "resident": st["resident"], "admitted": st["admitted"],
            "event_evals_per_s": event_evals / st["wall_s"], "wall_s": st["wall_s"],
            "converged": sum(1 for f in fits if f.converged),
            "loop": {k: st[k] for k in ("launches", "abnormal_exits", "published", "last_exit_status")}}


def serving_throughput(mc, p0, precision="fp32", n_samples=64, n_events=100_000, rounds=160, clients=16,
                       per_client=4):
    """The device-resident serving loop at steady state: n_samples generated
    samples of n_events (model fixed) are made resident by one request each,
    then `clients` threads each keep `per_client` requests in flight (submit
    for all of their samples, then wait for all) for `rounds` rounds, at
    parameter points with the coefficients and x, y moved.  Reports evals/s,
    event-evaluations/s, p50/p99 latency from the server's statistics, and the
    single-context cached pass (one evaluation per call with device
    parameters) on one of the same samples for comparison."""
    import torch
    from paper_1702_06735_gb300.tdmix import TDMix, TDMixServer
    srv = TDMixServer(MODEL, precision, hbm_budget_bytes=8 << 30, max_slots=256)
    try:
        srv.add_mc(mc)
        ids = [srv.add_generated_sample(p0, n_events, KEY0 + 6, STREAM_TOY0 + 5000 + k) for k in range(n_samples)]
        nc = model_sizes()[0]
        move = np.zeros(len(p0), dtype=bool)
        move[2:2 * nc] = True
        move[-2:] = True
        for sid in ids:                       # admission (generation + component cache)
            srv.evaluate(sid, p0, timeout_s=600.0)
        mine = [ids[c::clients] for c in range(clients)]

        def client(c):
            for r in range(rounds):
                for q in range(0, len(mine[c]), per_client):
                    group = mine[c][q:q + per_client]
                    tickets = [srv.submit(sid, step_params(p0, move, 97 * r + sid)) for sid in group]
                    for tk in tickets:
                        srv.wait(tk, timeout_s=600.0)
        srv.reset_stats()
        t0 = time.perf_counter()
        with cf_pool(clients) as ex:
            list(ex.map(client, range(clients)))
        wall = time.perf_counter() - t0
        st = srv.stats()
    finally:
        srv.close()
    evals = n_samples * rounds
    # the single-context cached pass on one sample of the same size
    g = TDMix(MODEL, "fp64")
    d, t, _ = generate(g, n_events, 6, STREAM_TOY0 + 5000, params=p0)
    g.close()
    c, _ = load(MODEL, precision, d, t, mc)
    mask = np.zeros(len(p0), dtype=np.int32)
    mask[2:2 * nc] = 1
    mask[-2:] = 1
    c.set_floating(mask)
    c.nll(p0)                                 # component cache and MC sums at the fixed model
    dev = torch.device("cuda", torch.cuda.current_device())
    K = 200
    P = torch.from_numpy(np.stack([step_params(p0, move, k) for k in range(K)])).to(dev)
    out = torch.empty(K, dtype=torch.float64, device=dev)
    grad = torch.empty(K, len(p0), dtype=torch.float64, device=dev)
    c.nll(step_params(p0, move, 1))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for k in range(K):
        c.nll_device(P[k], out[k:k + 1], grad[k])
    torch.cuda.synchronize()
    single = K / (time.perf_counter() - t1)
    c.close()
    return {"workload": f"{MODEL}, {n_samples} resident generated samples of {n_events} events, model fixed, "
                        f"coefficients and x, y moved; {clients} clients with {per_client} requests in flight each",
            "evals": evals, "wall_s": wall, "evals_per_s": evals / wall, "event_evals_per_s": evals * n_events / wall,
            "p50_us": st["p50_us"], "p99_us": st["p99_us"],
            "single_context_cached": {"evals_per_s": single, "event_evals_per_s": single * n_events,
                                      "note": "one tdmix_nll call per evaluation, device parameters, same sample size"}}


def floating_model_toys(n_toys=100, n_events=20_000):
    """Pseudo-experiments fitted with the model floating (every resonance mass
    and width, x and y; the coefficients fixed), an extension of the paper's
    fixed-model study (Sec. 4), on the 2-chain model; the same
    events are also fitted with the model fixed.  Reports pulls and the
    growth of the x, y errors when the model floats."""
    from paper_1702_06735_gb300 import toys
    from paper_1702_06735_gb300.tdmix import TDMix
    c = TDMix(MODEL_2CHAIN, "fp64")
    gen = c.default_params()
    mc, _, _ = generate(c, 1_000_000, 7, STREAM_MC, flat=True, with_times=False)
    c.close()
    t0 = time.perf_counter()
    fits = toys.run_floating(MODEL_2CHAIN, "fp64", [n_events] * n_toys, gen, mc, seed=KEY0 + 7,
                             stream0=STREAM_TOY0, compare_fixed=True)
    wall = time.perf_counter() - t0
    nc = model_sizes(MODEL_2CHAIN)[0]
    out = {"workload": f"{MODEL_2CHAIN}: {n_toys} toys of {n_events} events generated on the device, 1,000,000 MC; "
                       "fits with the model floating and, on the same events, with the model fixed",
           "precision": "fp64 (Hessian errors from finite differences of the gradient)",
           "converged": sum(f.converged for f in fits), "wall_s": wall,
           "evals": sum(f.n_eval for f in fits)}
    for name, idx in (("x", len(gen) - 2), ("y", len(gen) - 1), ("kstar_mass", 2 * nc), ("kstar_width", 2 * nc + 1)):
        out[name] = toys.floating_pulls(fits, gen, idx)
    ok = [f for f in fits if f.converged and f.xy_fixed_model and np.isfinite(f.xy_fixed_model[2])]
    out["xy_error_ratio_floating_over_fixed"] = {
        "x": float(np.median([f.errors[-2] / f.xy_fixed_model[2] for f in ok])),
        "y": float(np.median([f.errors[-1] / f.xy_fixed_model[3] for f in ok]))}
    return out


def cf_pool(n):
    import concurrent.futures as cf
    return cf.ThreadPoolExecutor(max_workers=n)


def sensitivity(mc, p0, n_toys, sizes=(20_000, 50_000, 70_000)):
    """The sensitivity study of Sec. 4: for each sample size, n_toys
    pseudo-experiments of the fixed model at the world-average x, y, fitted
    with x, y floating, errors from the Hessian; the resolution sigma(x),
    sigma(y), the mean fitted error and the pulls; sigma x sqrt(N) tests the
    1/sqrt(N) scaling of the paper's table."""
    from paper_1702_06735_gb300 import toys
    out = {}
    for j, n in enumerate(sizes):
        fits, st = toys.run(MODEL, "fp32", [n] * n_toys, p0, mc, seed=KEY0 + 5,
                            stream0=STREAM_TOY0 + 1000 * (j + 1), clients=16, with_errors=True)
        s = toys.pulls(fits, p0[-2], p0[-1])
        s["sigma_x_sqrtN"] = s["x"]["sigma"] * math.sqrt(n)
        s["sigma_y_sqrtN"] = s["y"]["sigma"] * math.sqrt(n)
        s["wall_s"] = st["wall_s"]
        out[str(n)] = s
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_tdmix(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    from paper_1702_06735_gb300.tdmix import TDMix

    stream = torch.cuda.current_stream(dev)
    nc, nr = model_sizes(MODEL)
    if args.cached_only > 0:
        if rank == 0:
            print(json.dumps({"cached_pass": cached_pass(dev, stream, args.cached_only, measured_peaks()[0])}),
                  flush=True)
        return 0

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize(dev)

    # the headline workload (config 2), generated on this device
    g = TDMix(MODEL, "fp64")
    p0 = g.default_params()
    sd, sm = replica_streams(rank)
    data, t, gen_d = generate(g, N_DATA, 2, sd, params=p0)
    mc, _, gen_m = generate(g, N_MC, 2, sm, flat=True, with_times=False)
    g.close()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if args.flush_l2 else None
    every, coef_xy, _ = class_masks(len(p0), nc, nr)

    c32, load32 = load(MODEL, "fp32", data, t, mc, stream)
    c64, load64 = load(MODEL, "fp64", data, t, mc, stream)
    barrier()
    # the timed region: K evaluations in one batch (consecutive evaluations
    # overlap on the device), or one call each when L2 is flushed in between
    ms32, wall32, prof32, clocks = device_steps(c32, dev, stream, args.steps, args.warmup, every, flush,
                                                ClockSampler(dev), batch=flush is None)
    ms64, _, prof64, _ = device_steps(c64, dev, stream, max(3, min(args.steps, 50)), 3, every, flush,
                                      batch=flush is None)
    # isolated launches (one call and CUDA events per evaluation): the latency of one evaluation
    ms_iso, _, _, _ = device_steps(c32, dev, stream, min(args.steps, 100), 3, every)

    # end to end through the C ABI with host buffers (params in, NLL + gradient out)
    ps = [step_params(p0, every, 6000 + k) for k in range(args.steps + args.warmup)]  # made before timing
    for k in range(args.warmup):
        c32.nll(ps[k])
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        c32.nll(ps[args.warmup + k])
    e2e_s = time.perf_counter() - t0

    step_ms = sum(ms32) / len(ms32)
    step_ms, e2e_s, wall32 = max_over_ranks([step_ms, e2e_s, wall32], world, dev)

    studies = {}
    if rank == 0 and args.studies == "all":
        studies["change_classes"] = change_classes(c64, c32, nc, nr, max(args.steps, 100))
        studies["config2_fit"] = full_model_fit(c32, nc, nr, f"{N_DATA} events, {N_MC} MC, fp32 path, "
                                                             "host-buffer evaluations")
        studies["config2_fit"].pop("x")
    c32.close()
    c64.close()
    if rank != 0:
        return 0

    peak, peak_kind = measured_peaks()
    if args.studies == "all":
        studies["config1_latency"] = config1_latency(dev)
        studies["config3_precision"] = config3_precision(dev, stream, peak)
        studies["config4_gradient_fit"] = config4_gradient_fit(dev, stream)
        studies["paper_fit_benchmark"] = paper_fit_benchmark(dev, stream)
        studies["floating_model_toys"] = floating_model_toys()
        if args.toys > 0 or args.sensitivity > 0:
            gm = TDMix(MODEL, "fp64")
            mc2, _, _ = generate(gm, 2_000_000, 5, STREAM_MC, flat=True, with_times=False)
            gm.close()
            if args.toys > 0:
                sz = np.exp(np.random.default_rng(KEY0 + 5).uniform(np.log(5_000), np.log(500_000), args.toys))
                sizes = [int(s) for s in sz]
                lab = (f"{MODEL}, sizes log-uniform in [5000, 500000] (seeded), 2,000,000 shared MC, "
                       "model fixed, x and y floating")
                studies["toy_study"] = {"fp32": toy_study("fp32", sizes, mc2, p0, lab)}
                if args.toys_fp64 > 0:
                    studies["toy_study"]["fp64"] = toy_study("fp64", sizes[:args.toys_fp64], mc2, p0,
                                                             lab + f"; the first {args.toys_fp64} toys")
            studies["serving_throughput"] = {"fp32": serving_throughput(mc2, p0, "fp32"),
                                             "fp64": serving_throughput(mc2, p0, "fp64", rounds=10)}
            if args.sensitivity > 0:
                studies["sensitivity"] = sensitivity(mc2, p0, args.sensitivity)
            del mc2

    # roofline of the evaluation kernel (the only kernel of a step)
    bytes_per_launch = full_eval_bytes(N_DATA, N_MC)
    # algorithmic fp32 flops (an FMA counts 2) of the full model per event:
    # MC: lineshapes 162, components 142, Gram 256, A and Abar 128, u 20,
    # adjoint 534 (W_j 128, terms 252, lineshapes 154); data: lineshapes and
    # components 304, A and Abar with low parts 256, fp32 Eq. (mix) adjoint 82,
    # gA/gB 128, adjoint 534 (Eq. (mix) itself is fp64 and not counted)
    FLOP_MC, FLOP_DATA = 1242, 1304
    flops_per_launch = N_MC * FLOP_MC + N_DATA * FLOP_DATA
    ev_ms, ev_n = prof32["eval"]
    ev_launch_ms = ev_ms / ev_n
    achieved = bytes_per_launch / (ev_launch_ms * 1e-3) / 1e9
    alu_tflops = flops_per_launch / (ev_launch_ms * 1e-3) / 1e12
    ALU_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock (GHz) = 80.5
    l2_mb = torch.cuda.get_device_properties(dev).L2_cache_size / 1e6
    traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["sources_sha256"] == kernel_source_digest() else None
    n_p = len(p0)
    out = {
        "metric": METRIC,
        "value": world * 1000.0 / step_ms,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (f64 for Eq. (mix) terms, log sum and accumulations)",
        "data": "synthetic (generated on the device: Philox4x32-10, GENBOD, accept/reject on the model's rate)",
        "config": {"workload": f"{MODEL}: 16 chains (8 shared components), 44 floating params, "
                               f"{N_DATA} accept/reject events (x=0.49%, y=0.61%), {N_MC} flat MC events; "
                               f"every parameter moved each step",
                   "l2": ("flushed between timed steps (256 MB write, outside the step events)" if args.flush_l2 else
                          f"not flushed: one evaluation streams {bytes_per_launch / 1e6:.0f} MB of event planes, "
                          f"more than the {l2_mb:.0f} MB L2, so every step reads its inputs from HBM (ncu DRAM bytes "
                          f"per launch with warm caches in profiles/)"),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "fp64_path": {"value": 1000.0 / (sum(ms64) / len(ms64)), "unit": "evals/s",
                      "ms_per_step": sum(ms64) / len(ms64),
                      "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in prof64.items()}},
        "speedup_vs_fp64": (sum(ms64) / len(ms64)) / step_ms,
        "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in prof32.items()},
        "timed_region": ("one tdmix_nll_batch call of K evaluations (consecutive evaluations overlap on the "
                         "device), CUDA events around it" if flush is None else
                         "one tdmix_nll call per evaluation, CUDA events around each"),
        "isolated_launch": {"ms": sum(ms_iso) / len(ms_iso), "evals_per_s": 1000.0 * len(ms_iso) / sum(ms_iso),
                            "frac_hbm": full_eval_bytes(N_DATA, N_MC) / (sum(ms_iso) / len(ms_iso) * 1e-3) / 1e9
                            / measured_peaks()[0],
                            "note": "one call and CUDA events per evaluation (no overlap between evaluations)"},
        "roofline": {"kernel": "k_eval (one full evaluation, fp32 path; average launch duration of the batched "
                               "timed region)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
                     "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
                     "launch_ms": ev_launch_ms,
                     "alu": {"achieved": alu_tflops, "peak": ALU_PEAK, "unit": "TFLOP/s", "frac": alu_tflops / ALU_PEAK,
                             "algorithmic_flops_per_launch": flops_per_launch,
                             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"}},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": 8 * n_p,
                "d2h_bytes_per_step": 8 * (4 + n_p)},
        # the evaluations counted by the library's profile, plus the batch's one k_derive launch
        "gpu_launches": sum(n for _, n in prof32.values()) + (1 if flush is None and args.steps > 1 else 0),
        "clocks": clocks,
        "load_ms": {"fp32": load32, "fp64": load64},
        "generation": {"data": gen_d, "mc": gen_m},
        "wall_s_timed_region": wall32,
        **studies,
    }
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(data.cpu().numpy(), t.cpu().numpy(), mc.cpu().numpy())
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_tdmix(args)


if __name__ == "__main__":
    sys.exit(main())
