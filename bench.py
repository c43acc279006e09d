"""Benchmark of the Hermite block-timestep N-body path on GB300.

Default workload (N = 1): Plummer sphere, N = 16384, equal masses, eps = 1/1024,
mixed precision (FP32 pair arithmetic, FP64 state / predictor / corrector),
eta = 0.01, power-of-two block steps, integrated from t = 0 to t = 1.
One bench step = load the resident initial state (nb_init_dev: initial forces
with s = N and first steps), energy at t = 0, nb_run to t = 1 (one CUDA-graph
launch), energy at t = 1. The metric is force+jerk interactions per second
(sum over block steps of s*N, plus the initial s = N pass); block steps per
second and |dE/E| are reported beside it, and the same for the FP64 GPU path.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has) on a bounded sample of the same workload.
Under torchrun (N > 1) every rank integrates its own replica (the workload is
one system; ranks share no data), timing is the max over ranks, and the value
is the sum of all ranks' interactions over that time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FLOP_PER_INTERACTION = 60          # the customary count for one force + jerk pair
T_END = 1.0
WORKLOAD = {"workload": "plummer N=16384 eps=1/1024 eta=0.01 t=0->1, mixed FP32/FP64",
            "n": 16384, "eps": 1.0 / 1024, "eta": 0.01, "t_end": T_END,
            "seed": 20071108}


# ---------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend: str):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return ws, rank


def dist_max(x: float, device=None) -> float:
    ws, _, _ = dist_env()
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, device=None) -> float:
    ws, _, _ = dist_env()
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_barrier():
    ws, _, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 200):
        self.index = index
        self.period = period_ms
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 f"-lms={self.period}"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------- helpers

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def fp32_peak_tflops(num_sms: int, sm_mhz: float) -> float:
    """Non-tensor FP32 peak: SMs x 128 FMA lanes x 2 flop x clock."""
    return num_sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(snap, t_end: float, nthreads: int):
    """The FP64 CPU oracle, as it stands, on the workload from t = 0 to t_end."""
    import oracle
    t0 = time.perf_counter()
    sysr = oracle.System(snap.m, snap.x, snap.v, snap.eps2, eta=WORKLOAD["eta"], nthreads=nthreads)
    assert sysr.status == 0
    assert sysr.run(t_end) == 0
    dt = time.perf_counter() - t0
    c = sysr.counters
    inter = c["interactions"] + float(snap.n) * snap.n   # + the initial s = N pass
    return {"seconds": dt, "interactions": inter, "block_steps": c["block_steps"]}


# ---------------------------------------------------------------- reference

def run_reference(args):
    ws, rank = dist_init("gloo")
    if rank != 0:
        return 0
    import ics
    import oracle
    oracle.build()
    snap = ics.config(2)
    nthreads = oracle.default_threads()
    t_sample = args.ref_t_end
    for _ in range(args.warmup):
        oracle_sample(snap, t_sample / 4, nthreads)
    secs, inter, bsteps = 0.0, 0.0, 0
    for _ in range(args.steps):
        r = oracle_sample(snap, t_sample, nthreads)
        secs += r["seconds"]; inter += r["interactions"]; bsteps += r["block_steps"]
    value = inter / secs
    line = {
        "impl": "reference", "metric": "force+jerk interactions/s", "value": value,
        "unit": "interactions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer sphere)",
        "config": dict(WORKLOAD, sample=f"t=0->{t_sample} per step"),
        "block_steps_per_s": bsteps / secs,
        "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"init (s=N pass) + block steps to t={t_sample} of the N=16384 Plummer run, "
                                   f"per step; host {cpu_model()}"},
        "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- GPU arm

def _r(x, d=4):
    """x rounded to d significant digits (compact JSON)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not math.isfinite(x):
        return x
    return float(f"{x:.{d}g}")


def _stats3(e):
    """[max, p99, median] of an error array, rounded."""
    e = np.asarray(e, dtype=float)
    return [_r(float(e.max()), 3), _r(float(np.percentile(e, 99)), 3), _r(float(np.median(e)), 3)]


def golden_energy(cfg):
    """The oracle's stored |dE/E| and step count for a timed integration (tests/golden/c<cfg>_energy.txt,
    written by tests/golden/make_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"c{cfg}_energy.txt")
    out = {}
    try:
        with open(path) as f:
            for ln in f:
                ln = ln.split("#", 1)[0].strip()
                if ln:
                    key, val = ln.split()[:2]
                    out[key] = val
        return {"abs_dE_over_E": float.fromhex(out["abs_dE_over_E"]), "block_steps": int(out["block_steps"])}
    except (OSError, KeyError, ValueError):
        return None


def main_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    dev = torch.device("cuda", local)

    import ics
    import paper_0711_0643_gb300 as pkg
    if rank == 0 or ws == 1:
        pkg.build()
    dist_barrier()
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()

    snap = ics.config(2)
    n = snap.n
    m_d = torch.tensor(snap.m, device=dev)
    x_d = torch.tensor(snap.x, device=dev)
    v_d = torch.tensor(snap.v, device=dev)
    # a dedicated stream: the library and the CUDA events must share it (torch's legacy
    # default stream has handle 0, which the C ABI reads as "create your own")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def make_ctx(prec):
        c = nb.Context(precision=prec, device=local, stream=sptr)
        nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
        c.n = n
        nb.nb_autotune(c.ctx)
        return c

    def step(c):
        nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
        E0, _, _ = nb.nb_energy(c.ctx)
        nb.nb_run(c.ctx, T_END)
        E1, _, _ = nb.nb_energy(c.ctx)
        st = nb.nb_stats(c.ctx)
        return E0, E1, st

    def timed_steps(c, k):
        ms, last = [], None
        for _ in range(k):
            l2_flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(c)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return ms, last

    # ---- mixed precision: the headline
    c = make_ctx(nb.NB_PREC_MIXED)
    eng_smax, eng_cluster = nb.nb_get_engine(c.ctx)
    for _ in range(args.warmup):
        step(c)
    dist_barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local).start()
    ms, (E0, E1, st) = timed_steps(c, args.steps)
    torch.cuda.synchronize(dev)
    dist_barrier()
    clk = clocks.stop()
    total_ms = dist_max(sum(ms), dev)
    inter_step = st["interactions"] + float(n) * n
    inter_all = dist_sum(inter_step * args.steps, dev)
    value = inter_all / (total_ms / 1e3)
    bsteps = st["block_steps"]
    dE = abs(E1 - E0) / abs(E0)
    # kernels per step: layout (2) + pad, predict, iota, force, init_steps (5) + energy 2 x 2
    # + the run loop's first selection (1) + per step slot of the loop (counted on the
    # device): the engine (when on), selection, predictor, force, corrector
    per_slot = 5 if eng_smax > 0 else 4
    launches = 2 + 5 + 4 + 1 + per_slot * st["loop_slots"]

    # ---- roofline of the dominant kernel, same trajectory, events around each launch
    nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
    torch.cuda.synchronize(dev)
    clk_rf = ClockSampler(local).start()
    tm = nb.nb_run_timed(c.ctx, T_END, phases=True)
    clk_rf_s = clk_rf.stop()
    sm_mhz = clk["sm_mhz"] or clk_rf_s["sm_mhz"] or load_peaks().get("clocks_under_load", {}).get("sm_mhz_median")
    peak = fp32_peak_tflops(num_sms, sm_mhz) if sm_mhz else None
    nl, ne = tm["force_launches"], tm["engine_steps"]
    force_ms, eng_ms = tm["force_ms"], tm["phase_ms"]["engine"]
    achieved = FLOP_PER_INTERACTION * tm["force_interactions"] / (force_ms / 1e3) / 1e12
    eng_tflops = FLOP_PER_INTERACTION * tm["engine_interactions"] / (eng_ms / 1e3) / 1e12 if eng_ms > 0 else None
    mean_s = tm["force_interactions"] / max(nl, 1) / n
    traffic = force_traffic(mean_s)
    roofline = {"bound": "alu", "achieved": _r(achieved), "peak": _r(peak), "unit": "TFLOP/s",
                "frac": _r(achieved / peak) if peak else None, "traffic": _r(traffic),
                "kernel": "force_mixed_kernel", "launches": nl, "avg_launch_us": _r(1e3 * force_ms / max(nl, 1)),
                "mean_s": _r(mean_s),
                "peak_basis": f"{num_sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz} MHz (median SM clock "
                              f"sampled during the timed region)",
                "flop_convention": f"{FLOP_PER_INTERACTION} flop per force+jerk interaction",
                "phases_us_per_step": {k: _r(1e3 * v / max(nl if k != "engine" else ne, 1), 3)
                                       for k, v in tm["phase_ms"].items()},
                "share_of_timed_kernels": {"force": _r(force_ms / (force_ms + eng_ms), 3),
                                           "engine": _r(eng_ms / (force_ms + eng_ms), 3)}}
    engine = {"s_max": eng_smax, "cluster": eng_cluster, "steps": ne, "four_kernel_steps": nl,
              "us_per_step": _r(1e3 * eng_ms / max(ne, 1), 3), "tflops": _r(eng_tflops, 3),
              "frac_fp32_peak": _r(eng_tflops / peak, 3) if (peak and eng_tflops) else None}

    # ---- end to end through the C ABI with host buffers
    m_h = np.ascontiguousarray(snap.m); x_h = np.ascontiguousarray(snap.x); v_h = np.ascontiguousarray(snap.v)
    ce = nb.Context(precision=nb.NB_PREC_MIXED, device=local, stream=sptr)
    ce.init(snap)
    nb.nb_autotune(ce.ctx)
    e2e_ms = []
    for k in range(max(1, args.steps)):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        nb.nb_init(ce.ctx, m_h, x_h, v_h, snap.eps2)
        nb.nb_energy(ce.ctx)
        nb.nb_run(ce.ctx, T_END)
        nb.nb_energy(ce.ctx)
        out = ce.state()
        torch.cuda.synchronize(dev)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    ce.close()
    e2e_total = dist_max(sum(e2e_ms), dev)
    e2e_value = dist_sum(inter_step * len(e2e_ms), dev) / (e2e_total / 1e3)
    h2d = n * (8 + 24 + 24)
    d2h = n * (8 + 24 * 4 + 8 + 8) + 3 * 8

    # ---- FP64 GPU path on the same workload (one step, events)
    fp64 = None
    if not args.no_fp64:
        c64 = make_ctx(nb.NB_PREC_FP64)
        step(c64)   # warm
        ms64, (F0, F1, st64) = timed_steps(c64, 1)
        fp64 = {"ips": _r((st64["interactions"] + float(n) * n) / (ms64[0] / 1e3)),
                "bsps": _r(st64["block_steps"] / (ms64[0] / 1e3)), "dE": _r(abs(F1 - F0) / abs(F0)),
                "ms": _r(ms64[0]), "block_steps": st64["block_steps"],
                "mixed_over_fp64_bsps": _r((bsteps * args.steps / (total_ms / 1e3)) /
                                           (st64["block_steps"] / (ms64[0] / 1e3)), 3)}
        c64.close()

    ens = ensemble_bench(nb, torch, dev, sptr, stream) if (args.ensemble and rank == 0) else None
    salp = salpeter_bench(nb, torch, dev, sptr, stream) if (args.salpeter and rank == 0) else None
    king = king_bench(nb, torch, dev, sptr, stream) if (args.king and rank == 0) else None
    pert, pert_out = perturbers_bench(nb, torch, dev, sptr, stream) if (args.perturbers and rank == 0) else (None, None)

    # ---- full-N force sweep (King W0 = 6, N = 2^20), mixed and FP64, one evaluation per s
    sweep = None
    if args.sweep and rank == 0:
        mx = force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz)
        f64 = force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz, s_list=(1, 64, 1024, 16384), autotune=False,
                          precision=nb.NB_PREC_FP64, reps=2)
        sweep = {"workload": mx["workload"], "l2": mx["l2"],
                 "mixed": [{"s": p["s"], "ms": _r(p["ms"]), "frac_fp32": _r(p["frac_fp32_peak"], 3),
                            "roof": p.get("roof_bound"), "roof_frac": _r(p.get("roof_frac"), 3)}
                           for p in mx["points"]],
                 "fp64": [{"s": q["s"], "ms": _r(q["ms"]), "mixed_over_fp64": _r(q["ms"] / p["ms"], 3)}
                          for p, q in zip(mx["points"], f64["points"])]}

    model = timing_model(nb, torch, dev, stream) if (args.model and rank == 0) else None

    # ---- CPU oracle baseline (rank 0, N = 1 only); the force errors against the oracle on
    # sampled particles of each workload's own state are taken in the same leg
    cpu, ferr = None, None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        nth = oracle.default_threads()
        r = oracle_sample(snap, args.ref_t_end, nth)
        cpu = {"value": r["interactions"] / r["seconds"], "unit": "interactions/s", "cores": nth,
               "kind": "oracle", "sample": f"init (s=N pass) + {r['block_steps']} block steps to "
                                          f"t={args.ref_t_end} of the same N=16384 Plummer run "
                                          f"({r['seconds']:.1f} s); host {cpu_model()}"}
        ferr = force_error_report(nb, oracle, nth, sptr, local)
        if pert_out is not None:
            # the perturber lists against the oracle's on the same positions, bit for bit
            pm, px, pp, pg, pn, pl, pc = pert_out
            ol, oc = oracle.perturbers(pm, px, pp, gamma=pg, nmax=pn)
            pert["oracle_equal"] = bool(np.array_equal(pl, ol) and np.array_equal(pc, oc))

    c.close()
    if rank == 0:
        g2 = golden_energy(2)
        line = {
            "metric": "force+jerk interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair arithmetic, f64 state",
            "data": "synthetic (seeded Plummer sphere, N-body units)",
            "config": dict(WORKLOAD, l2="flushed (256 MB write) before every timed step",
                           parallelism=f"replicas x{ws}" if ws > 1 else "single GPU"),
            "gpu_launches": launches * args.steps,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "interactions/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_total / len(e2e_ms)},
            "cpu_baseline": cpu,
            "roofline": roofline,
            "block_steps": bsteps,
            "block_steps_per_s": dist_sum(bsteps * args.steps, dev) / (total_ms / 1e3),
            "abs_dE_over_E": dE,
            "oracle_abs_dE_over_E": g2["abs_dE_over_E"] if g2 else None,
            "engine": engine,
            "king": king,
            "force_sweep": sweep,
            "ensemble": ens, "salpeter": salp, "perturbers": pert, "fp64_gpu": fp64, "timing_model": model,
            "force_error": ferr,
        }
        print(json.dumps(line))
    return 0


def size_hist(st):
    """Block steps per block-size bucket, {upper bound 2^b: count} for the non-empty buckets."""
    return {str(1 << b): int(c) for b, c in enumerate(st["size_hist"]) if c}


def force_traffic(mean_s):
    """DRAM bytes per force launch at the mean block size mean_s, from the committed ncu figures
    (profiles/force_traffic.json: per-launch read + write bytes at a few block sizes of this
    workload, fitted as a + b s), or None when the kernel sources have changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "force_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for name in rec["sources"]:
            with open(os.path.join(ROOT, "paper_0711_0643_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != rec["sha256"]:
            return None
        return rec["fit"]["a_bytes"] + rec["fit"]["b_bytes_per_s"] * mean_s
    except (OSError, KeyError, ValueError):
        return None


def _condition_scales(m, xp, vp, eps2, idx, chunk=8):
    """A_i = sum m_j/(r^2+eps^2) and K_i = sum m_j(|w|/(r^2+eps^2)^1.5 + 3|r.w||r|/(r^2+eps^2)^2.5),
    j != i: the sizes the sums would have without cancellation (error normalisation)."""
    A = np.zeros(idx.size)
    K = np.zeros(idx.size)
    for q0 in range(0, idx.size, chunk):
        ii = idx[q0:q0 + chunk]
        r = xp[None, :, :] - xp[ii][:, None, :]
        w = vp[None, :, :] - vp[ii][:, None, :]
        rr = np.einsum("ijk,ijk->ij", r, r)
        d2 = rr + eps2
        wn = np.sqrt(np.einsum("ijk,ijk->ij", w, w))
        rw = np.abs(np.einsum("ijk,ijk->ij", r, w))
        mask = np.ones_like(d2, dtype=bool)
        mask[np.arange(ii.size), ii] = False
        with np.errstate(divide="ignore", invalid="ignore"):
            A[q0:q0 + chunk] = np.where(mask, m[None, :] / d2, 0.0).sum(1)
            K[q0:q0 + chunk] = np.where(mask, m[None, :] * (wn / d2 ** 1.5 + 3 * rw * np.sqrt(rr) / d2 ** 2.5),
                                        0.0).sum(1)
    return A, K


def force_error_report(nb, oracle, nth, sptr, local):
    """Force and jerk error of the mixed path against the FP64 oracle, per workload, on sampled
    active particles of the GPU's own predicted state (the oracle summing over all N j):
    condition-scaled e_a = |da|/A_i, e_k = |dk|/K_i, forward ea_f, ek_f and phi's forward error,
    each as [max, p99, median]; with the condition numbers kappa at the worst forward errors."""
    import ics
    out = {}
    cases = [("c2_t0", ics.config(2), 256, 0), ("c2_step400", ics.config(2), 256, 400),
             ("c3_t0", ics.config(3), 256, 0), ("c5_t0", ics.config(5), 256, 0)]
    for name, snap, ns, steps in cases:
        c = nb.Context(precision=nb.NB_PREC_MIXED, device=local, stream=sptr)
        c.init(snap)
        for _ in range(steps):
            nb.nb_step(c.ctx)
        if steps:
            tn, s = nb.nb_next_block(c.ctx)
            idx = nb.nb_get_active(c.ctx, s)
            nb.nb_predict(c.ctx, tn)
        else:
            nb.nb_predict(c.ctx, 0.0)
            idx = np.sort(np.argsort(ics.SplitMix64(ics.BASE_SEED + 900).uniform(snap.n))[:ns]).astype(np.int32)
        xp, vp = nb.nb_get_predicted(c.ctx, snap.n)
        a, k, phi = nb.nb_force_jerk(c.ctx, idx)
        c.close()
        pos = np.unique(np.linspace(0, idx.size - 1, min(idx.size, ns)).astype(np.int64))
        sample = idx[pos]
        ar, kr, pr = oracle.force(snap.m, xp, vp, snap.eps2, sample, nthreads=nth)
        A, K = _condition_scales(snap.m, xp, vp, snap.eps2, sample, chunk=max(1, (1 << 22) // snap.n))
        da = np.linalg.norm(a[pos] - ar, axis=1)
        dk = np.linalg.norm(k[pos] - kr, axis=1)
        na, nk = np.linalg.norm(ar, axis=1), np.linalg.norm(kr, axis=1)
        eaf, ekf = da / na, dk / nk
        out[name] = {"n": snap.n, "s": int(idx.size), "sampled": int(sample.size),
                     "ea": _stats3(da / A), "ek": _stats3(dk / K), "ep": _stats3(np.abs(phi[pos] - pr) / np.abs(pr)),
                     "ea_f": _stats3(eaf), "ek_f": _stats3(ekf),
                     "kappa_at_worst": [_r(float((A / na)[np.argmax(eaf)]), 3), _r(float((K / nk)[np.argmax(ekf)]), 3)]}
    return out


def ensemble_bench(nb, torch, dev, sptr, stream, nc=256, n_lo=256, n_hi=8192, tune=True):
    """256 independent Plummer clusters, N_c = round(exp(U[ln 256, ln 8192])) (seeded),
    eps = 4/N_c, equal masses, each with its own block schedule, advanced to t = 1 by
    one persistent launch of thread-block clusters (mixed precision). The launch shape
    (cluster size, j-split cap) is autotuned on the same ensemble before the timed
    region; the timed region is nb_ensemble_init + nb_ensemble_run."""
    import ics
    members = ics.ensemble(nc, ics.BASE_SEED + 4, n_lo=n_lo, n_hi=n_hi)
    off = np.zeros(nc + 1, dtype=np.int64)
    off[1:] = np.cumsum([c.n for c in members])
    m = np.concatenate([c.m for c in members])
    x = np.concatenate([c.x for c in members])
    v = np.concatenate([c.v for c in members])
    e2 = np.array([c.eps2 for c in members])
    c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=sptr)
    # warm-up on a small ensemble (module load, cluster-occupancy query)
    nb.nb_ensemble_init(c.ctx, off[:3], m[:off[2]], x[:off[2]], v[:off[2]], e2[:2])
    nb.nb_ensemble_run(c.ctx, 1.0 / 64)
    shape = None
    if tune:
        # launch shape (cluster size, j-split cap) tuned on this ensemble, untimed
        nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
        nb.nb_ensemble_autotune(c.ctx, 1.0 / 16)
        shape = nb.nb_ensemble_get_shape(c.ctx)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2v = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
    if shape:
        nb.nb_ensemble_set_shape(c.ctx, shape[0], shape[2])
    e1.record(stream)
    shape = nb.nb_ensemble_get_shape(c.ctx)
    E0 = nb.nb_ensemble_energy(c.ctx, nc)
    nb.nb_ensemble_run(c.ctx, T_END)
    e2v.record(stream)
    torch.cuda.synchronize(dev)
    E1 = nb.nb_ensemble_energy(c.ctx, nc)
    bs, ps, inter = nb.nb_ensemble_stats(c.ctx, nc)
    c.close()
    run_s = e1.elapsed_time(e2v) / 1e3
    init_s = e0.elapsed_time(e1) / 1e3
    dE = np.abs(E1 - E0) / np.abs(E0)
    total_inter = float(inter.sum()) + float(np.sum(np.diff(off).astype(float) ** 2))
    return {"workload": f"{nc} Plummer clusters N in [{int(np.diff(off).min())}, {int(np.diff(off).max())}] "
                        f"(total {int(off[-1])}), eps=4/N, t=0->{T_END}",
            "run_ms": _r(run_s * 1e3), "init_ms": _r(init_s * 1e3),
            "ips": _r(total_inter / (run_s + init_s)), "tflops": _r(60 * total_inter / (run_s + init_s) / 1e12, 3),
            "bsps": _r(float(bs.sum()) / run_s), "block_steps": int(bs.sum()),
            "worst_dE": _r(float(dE.max()), 5), "median_dE": _r(float(np.median(dE)), 3),
            "worst_member": [int(np.argmax(dE)), int(np.diff(off)[int(np.argmax(dE))])],
            "shape": {"cluster": shape[0], "clusters": shape[1], "split_cap": shape[2], "tuned": bool(tune)}}


def perturbers_bench(nb, torch, dev, sptr, stream, n=16384, nbin=1638, gamma=1e-7, nmax=256):
    """Perturber lists of binaries (Sect. 3.1): Plummer N = 16384 of which 2 x 1638 stars in
    primordial binaries (separations log-uniform in [1e-4, 1e-2]), gamma = 1e-7, N_pert = 256;
    one nb_perturbers_dev call (device arrays, all binaries against all stars) timed with
    events, median of 10 after 3 warm-up calls (the 0.4 MB of positions stay in L2). Returns
    the summary and the lists and counts (compared with the oracle's in the CPU leg)."""
    import ics
    snap = ics.plummer_binaries(n, nbin, ics.BASE_SEED + 49, 1.0 / 1024)
    pairs = snap.meta["pairs"]
    c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=sptr)
    c.init(snap)
    p_d = torch.tensor(pairs, device=dev)
    l_d = torch.empty((nbin, nmax), dtype=torch.int32, device=dev)
    c_d = torch.empty(nbin, dtype=torch.int32, device=dev)

    def call():
        nb.nb_perturbers_dev(c.ctx, nbin, p_d.data_ptr(), gamma, nmax, 0, -1, l_d.data_ptr(), c_d.data_ptr())

    for _ in range(3):
        call()
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    lists, counts = l_d.cpu().numpy(), c_d.cpu().numpy()
    c.close()
    tests = float(nbin) * (n - 2)
    summary = {"workload": f"plummer N={n} with {nbin} primordial binaries, gamma={gamma}, N_pert={nmax}",
               "ms": _r(ms, 4), "tests_per_s": _r(tests / (ms / 1e3)),
               "mean_count": _r(float(counts.mean()), 4), "lists_full": int((counts > nmax).sum()),
               "oracle_equal": None}
    return summary, (snap.m, snap.x, pairs, gamma, nmax, lists, counts)


def salpeter_bench(nb, torch, dev, sptr, stream, t_end=0.5):
    """Plummer N = 65536 with a Salpeter mass spectrum (slope -2.35 on [0.1, 100],
    normalised to M = 1), eps = 1/4096, mixed precision, t = 0 -> 0.5, autotuned:
    one timed run (init + energy + nb_run + energy) after a short warm-up run.
    Active-set sizes span 1 to N."""
    import ics
    snap = ics.config(3)
    n = snap.n
    m_d = torch.tensor(snap.m, device=dev)
    x_d = torch.tensor(snap.x, device=dev)
    v_d = torch.tensor(snap.v, device=dev)
    c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=sptr)
    nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
    nb.nb_autotune(c.ctx)
    nb.nb_run(c.ctx, 1.0 / 64)   # warm-up: graph instantiation, caches
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
    E0 = nb.nb_energy(c.ctx)[0]
    nb.nb_run(c.ctx, t_end)
    E1 = nb.nb_energy(c.ctx)[0]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = nb.nb_stats(c.ctx)
    c.close()
    sec = e0.elapsed_time(e1) / 1e3
    inter = st["interactions"] + float(n) * n
    g3 = golden_energy(3)
    return {"workload": f"plummer N={n} Salpeter [0.1, 100] -2.35, eps=1/4096, t=0->{t_end}, mixed",
            "ms": _r(sec * 1e3), "ips": _r(inter / sec), "block_steps": st["block_steps"],
            "bsps": _r(st["block_steps"] / sec), "mean_s": _r(st["particle_steps"] / max(st["block_steps"], 1)),
            "dE": _r(abs(E1 - E0) / abs(E0)), "oracle_dE": _r(g3["abs_dE_over_E"]) if g3 else None,
            "oracle_block_steps": g3["block_steps"] if g3 else None}


def king_bench(nb, torch, dev, sptr, stream, n=16384, t_end=0.25):
    """Centrally concentrated models: King W0 = 6 and W0 = 9, N = 16384, eps = 1/1024, equal
    masses, mixed precision, autotuned, t = 0 -> 1/4 (seeds 20071106 + 56 and + 59): one timed
    run (init + energy + nb_run + energy) each after a short warm-up run."""
    import ics
    out = []
    for w0 in (6.0, 9.0):
        snap = ics.king(n, seed=ics.BASE_SEED + 50 + int(w0), w0=w0, eps=1.0 / 1024)
        m_d = torch.tensor(snap.m, device=dev)
        x_d = torch.tensor(snap.x, device=dev)
        v_d = torch.tensor(snap.v, device=dev)
        c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=sptr)
        nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
        nb.nb_autotune(c.ctx)
        nb.nb_run(c.ctx, 1.0 / 64)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
        E0 = nb.nb_energy(c.ctx)[0]
        nb.nb_run(c.ctx, t_end)
        E1 = nb.nb_energy(c.ctx)[0]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = nb.nb_stats(c.ctx)
        c.close()
        sec = e0.elapsed_time(e1) / 1e3
        out.append({"w0": w0, "n": n, "t_end": t_end, "ms": _r(sec * 1e3),
                    "ips": _r((st["interactions"] + float(n) * n) / sec),
                    "block_steps": st["block_steps"], "bsps": _r(st["block_steps"] / sec),
                    "mean_s": _r(st["particle_steps"] / max(st["block_steps"], 1)),
                    "dE": _r(abs(E1 - E0) / abs(E0))})
    return out


def force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz, n_override=None, s_list=None, autotune=True,
                precision=None, reps=None):
    """King W0 = 6, N = 1,048,576, eps = 1e-3: one mixed force evaluation per active-set
    size s in {1, 64, 1024, 16384, N} (active = first s of a seeded permutation, ascending),
    split factor autotuned; interactions/s and FP32 roofline fraction per s. Each point is
    the median of single nb_force_jerk_dev calls (active list in, a/k/phi out, all on the
    device), each timed with L2 flushed before it and the launch queued behind a short spin
    (the events bracket the device work, not the host's launch latency)."""
    import ics
    snap = ics.config(5, n=n_override)
    n = snap.n
    m_d = torch.tensor(snap.m, device=dev)
    x_d = torch.tensor(snap.x, device=dev)
    v_d = torch.tensor(snap.v, device=dev)
    prec = nb.NB_PREC_MIXED if precision is None else precision
    c = nb.Context(precision=prec, device=0, stream=sptr)
    nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
    nb.nb_predict(c.ctx, 0.0)
    if autotune:
        nb.nb_autotune(c.ctx)
    perm = np.argsort(ics.SplitMix64(ics.BASE_SEED + 5).uniform(n))
    out = {"workload": f"king W0=6 N={n} eps=1e-3, single evaluation", "points": [],
           "precision": "fp64" if prec == nb.NB_PREC_FP64 else "mixed",
           "l2": "flushed (256 MB write) before every timed call; median of single calls, each queued "
                 "behind a short spin so the events bracket device work"}
    stream = torch.cuda.current_stream(dev)
    assert stream.cuda_stream == sptr
    l2_flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2
    for s in (s_list or (1, 64, 1024, 16384, n)):
        s = min(int(s), n)
        idx = np.sort(perm[:s]).astype(np.int32)
        idx_d = torch.tensor(idx, device=dev)
        a_d = torch.empty((s, 3), dtype=torch.float64, device=dev)
        k_d = torch.empty_like(a_d)
        p_d = torch.empty(s, dtype=torch.float64, device=dev)
        for _ in range(3 if reps is None else 1):
            nb.nb_force_jerk_dev(c.ctx, idx_d.data_ptr(), s, a_d.data_ptr(), k_d.data_ptr(), p_d.data_ptr())
        # each timed call starts with L2 flushed (the j-records, 40 MB at N = 2^20, would
        # otherwise stay in the 129 MB L2 between calls): median of single calls
        nrep = reps if reps is not None else (9 if s < n else 2)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(nrep):
            l2_flush.zero_()
            torch.cuda.synchronize(dev)
            # a short spin on the stream first: the call is queued behind it before the
            # start event is processed, so the events bracket the device work and not the
            # host's launch latency
            torch.cuda._sleep(100000)
            e0.record(stream)
            nb.nb_force_jerk_dev(c.ctx, idx_d.data_ptr(), s, a_d.data_ptr(), k_d.data_ptr(), p_d.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1) / 1e3)
        sec = float(np.median(times))
        ips = s * float(n) / sec
        tfl = FLOP_PER_INTERACTION * ips / 1e12
        peak = fp32_peak_tflops(num_sms, sm_mhz) if sm_mhz else None
        point = {"s": s, "ms": sec * 1e3, "interactions_per_s": ips, "tflops": tfl,
                 "frac_fp32_peak": tfl / peak if peak else None}
        hbm = load_peaks().get("hbm_gbs")
        if peak and hbm:
            # the roof of this point: the longer of the FP32 time (60 flop per interaction) and
            # the HBM time of its algorithmic bytes (N j-records of 40 B, s x (40 B + 56 B))
            t_fp32 = FLOP_PER_INTERACTION * s * float(n) / (peak * 1e12)
            t_hbm = (40.0 * n + 96.0 * s) / (hbm * 1e9)
            point["roof_bound"] = "fp32" if t_fp32 >= t_hbm else "hbm"
            point["roof_frac"] = max(t_fp32, t_hbm) / sec
        out["points"].append(point)
    c.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-t-end", type=float, default=1.0 / 16,
                    help="integration horizon of one oracle sample (bounded CPU work)")
    ap.add_argument("--t-end", type=float, default=1.0,
                    help="integration horizon of one step (default 1; shorter only for profiling runs)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ensemble", action=argparse.BooleanOptionalAction, default=True,
                    help="batched ensemble of 256 clusters (default on)")
    ap.add_argument("--sweep", action=argparse.BooleanOptionalAction, default=True,
                    help="full-N force sweep on King N=2^20 (default on)")
    ap.add_argument("--salpeter", action=argparse.BooleanOptionalAction, default=True,
                    help="Plummer N=65536 with Salpeter masses to t=0.5 (default on; ~15 s of input generation)")
    ap.add_argument("--king", action=argparse.BooleanOptionalAction, default=True,
                    help="King W0 = 6 and 9, N = 16384, to t = 1/4 (default on)")
    ap.add_argument("--model", action=argparse.BooleanOptionalAction, default=True,
                    help="refit the per-block-step timing model on this GPU (default on)")
    ap.add_argument("--model-only", action="store_true", help="run only the timing model and print it")
    ap.add_argument("--perturbers", action=argparse.BooleanOptionalAction, default=True,
                    help="time the perturber lists of a Plummer model with primordial binaries")
    ap.add_argument("--perturbers-only", action="store_true",
                    help="run only the perturber-list timing and print it")
    ap.add_argument("--salpeter-only", action="store_true",
                    help="run only the Salpeter workload and print it")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="run only the ensemble workload and print it (profiling)")
    ap.add_argument("--ens-nc", type=int, default=256, help="systems of --ensemble-only")
    ap.add_argument("--ens-nmax", type=int, default=8192, help="largest system of --ensemble-only")
    ap.add_argument("--sweep-only", action="store_true",
                    help="run only the force sweep and print it (profiling and kernel studies)")
    ap.add_argument("--sweep-n", type=int, default=None, help="particle count of --sweep-only")
    ap.add_argument("--sweep-s", type=str, default=None, help="comma-separated active counts of --sweep-only")
    ap.add_argument("--sweep-fp64", action="store_true", help="--sweep-only with the FP64 kernels")
    ap.add_argument("--no-autotune", action="store_true", help="--sweep-only with the default tuning table")
    args = ap.parse_args(argv)
    global T_END  # noqa: PLW0603
    T_END = args.t_end
    WORKLOAD["t_end"] = T_END
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep_only:
        return main_sweep(args)
    if args.ensemble_only:
        return main_ensemble(args)
    if args.salpeter_only:
        return main_salpeter(args)
    if args.perturbers_only:
        return main_perturbers(args)
    if args.model_only:
        return main_model(args)
    return main_gpu(args)


def main_perturbers(args):
    """Only the perturber-list timing, printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    print(json.dumps(perturbers_bench(nb, torch, dev, stream.cuda_stream, stream)[0]))
    return 0


def main_ensemble(args):
    """Only the batched ensemble, printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    out = ensemble_bench(nb, torch, dev, stream.cuda_stream, stream, nc=args.ens_nc, n_hi=args.ens_nmax)
    print(json.dumps(out))
    return 0


def timing_model(nb, torch, dev, stream):
    """The paper's timing model (Sect. 4.1: T = tau_pr N + tau_f N s / p + tau_cr s + communication)
    refitted on this GPU, per block step and phase: selection and predictor a + b N, force
    a + tau_f s N, corrector a + tau_cr s (the four-kernel step), and the small-block engine's
    whole step a + b N + c s N. Fitted by least squares to the phase totals of host-driven runs
    (nb_run_timed, each phase bracketed by events; ~3.7 us of the gate in every a) of Plummer models
    N = 1024 .. 65536 (eps = 4/N, t = 0 -> 1/16, autotuned); the graph loop's measured time (nb_run)
    is printed beside the sum of the fitted phase times of the same run."""
    import ics
    rows = []
    for n in (1024, 2048, 4096, 8192, 16384, 32768, 65536):
        snap = ics.plummer(n, seed=ics.BASE_SEED + 70 + n.bit_length(), eps=4.0 / n,
                           scale="continuum" if n > 16384 else "auto")
        c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=stream.cuda_stream)
        c.init(snap)
        nb.nb_autotune(c.ctx)
        c.init(snap)
        tm = nb.nb_run_timed(c.ctx, 1.0 / 16, phases=True)
        c.init(snap)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        nb.nb_run(c.ctx, 1.0 / 16)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = nb.nb_stats(c.ctx)
        c.close()
        rows.append({"n": n, "tm": tm, "run_us": 1e3 * e0.elapsed_time(e1), "steps": st["block_steps"]})
    fit = {}

    def lsq(cols, y):
        coef, *_ = np.linalg.lstsq(np.array(cols, dtype=float), np.array(y, dtype=float), rcond=None)
        return [float(x) for x in coef]

    k4 = [r["tm"]["force_launches"] for r in rows]
    ns = [r["n"] for r in rows]
    fI = [r["tm"]["force_interactions"] for r in rows]
    for ph in ("select", "predict"):
        fit[ph] = lsq([(k, k * n) for k, n in zip(k4, ns)], [1e3 * r["tm"]["phase_ms"][ph] for r in rows])
    fit["force"] = lsq([(k, i) for k, i in zip(k4, fI)], [1e3 * r["tm"]["phase_ms"]["force"] for r in rows])
    fit["correct"] = lsq([(k, i / n) for k, i, n in zip(k4, fI, ns)], [1e3 * r["tm"]["phase_ms"]["correct"]
                                                                       for r in rows])
    ke = [r["tm"]["engine_steps"] for r in rows]
    used = [q for q, k in enumerate(ke) if k > 0]
    if len(used) >= 3:
        fit["engine"] = lsq([(ke[q], ke[q] * ns[q], rows[q]["tm"]["engine_interactions"]) for q in used],
                            [1e3 * rows[q]["tm"]["phase_ms"]["engine"] for q in used])
    runs = []
    for r, k, n, i in zip(rows, k4, ns, fI):
        t = (fit["select"][0] + fit["predict"][0] + fit["force"][0] + fit["correct"][0]) * k
        t += (fit["select"][1] + fit["predict"][1]) * k * n + fit["force"][1] * i + fit["correct"][1] * i / n
        if "engine" in fit and r["tm"]["engine_steps"]:
            e = r["tm"]["engine_steps"]
            t += fit["engine"][0] * e + fit["engine"][1] * e * n + fit["engine"][2] * r["tm"]["engine_interactions"]
        runs.append({"n": n, "steps": r["steps"], "engine_steps": r["tm"]["engine_steps"],
                     "run_ms": _r(r["run_us"] / 1e3), "model_ms": _r(t / 1e3), "run_over_model": _r(r["run_us"] / t, 3)})
    # units: a in us per step; b in ns per particle (select, predict), tau in ps per
    # interaction (force, engine), tau_cr in ns per active particle
    out = {"select": [_r(fit["select"][0], 3), _r(1e3 * fit["select"][1], 3)],
           "predict": [_r(fit["predict"][0], 3), _r(1e3 * fit["predict"][1], 3)],
           "force": [_r(fit["force"][0], 3), _r(1e6 * fit["force"][1], 3)],
           "correct": [_r(fit["correct"][0], 3), _r(1e3 * fit["correct"][1], 3)],
           "units": "[a us/step, b ns/particle | tau_f ps/interaction | tau_cr ns/active]", "runs": runs}
    if "engine" in fit:
        out["engine"] = [_r(fit["engine"][0], 3), _r(1e3 * fit["engine"][1], 3), _r(1e6 * fit["engine"][2], 3)]
    return out


def main_model(args):
    """Only the timing model, printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    print(json.dumps(timing_model(nb, torch, dev, stream)))
    return 0


def main_salpeter(args):
    """Only the Salpeter N = 65536 workload, printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    out = salpeter_bench(nb, torch, dev, stream.cuda_stream, stream)
    print(json.dumps(out))
    return 0


def main_sweep(args):
    """Only the force sweep, printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = ClockSampler(0).start()
    s_list = [int(q) for q in args.sweep_s.split(",")] if args.sweep_s else None
    out = force_sweep(nb, torch, dev, stream.cuda_stream, num_sms, None, n_override=args.sweep_n, s_list=s_list,
                      autotune=not args.no_autotune,
                      precision=nb.NB_PREC_FP64 if args.sweep_fp64 else nb.NB_PREC_MIXED)
    clk = clocks.stop()
    if clk["sm_mhz"]:
        peak = fp32_peak_tflops(num_sms, clk["sm_mhz"])
        for p in out["points"]:
            p["frac_fp32_peak"] = p["tflops"] / peak
    out["clocks"] = clk
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
