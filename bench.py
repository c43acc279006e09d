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
            "model": "plummer", "n": 16384, "eps": 1.0 / 1024, "eta": 0.01, "t_end": T_END,
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
    # + the run loop's first selection (1) + 4 per loop step (selection, predictor, force,
    # corrector); the loop runs whole passes of 16 steps, the one that finds no block due
    # and those after it in its pass as no-ops
    loop_steps = (bsteps // 16 + 1) * 16
    launches = 2 + 5 + 4 + 1 + 4 * loop_steps

    # ---- roofline of the dominant kernel (force), same trajectory, events around each launch
    nb.nb_init_dev(c.ctx, n, m_d.data_ptr(), x_d.data_ptr(), v_d.data_ptr(), snap.eps2)
    torch.cuda.synchronize(dev)
    clk_rf = ClockSampler(local).start()
    force_ms, nlaunch, eng_steps, phase_ms = nb.nb_run_timed(c.ctx, T_END, phases=True)
    clk_rf_s = clk_rf.stop()
    st_rf = nb.nb_stats(c.ctx)
    sm_mhz = clk["sm_mhz"] or clk_rf_s["sm_mhz"] or load_peaks().get("clocks_under_load", {}).get("sm_mhz_median")
    peak = fp32_peak_tflops(num_sms, sm_mhz) if sm_mhz else None
    achieved = FLOP_PER_INTERACTION * st_rf["interactions"] / (force_ms / 1e3) / 1e12
    traffic = force_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None, "traffic": traffic,
                "traffic_basis": "mean DRAM read+write bytes per force launch, cold-cache ncu capture of this "
                                 "workload to t = 1/64 (profiles/force_traffic_plummer_n16384_t1over64.md)"
                                 if traffic else None,
                "kernel": "force_mixed_kernel", "launches": nlaunch,
                "avg_launch_us": 1e3 * force_ms / max(nlaunch, 1),
                "peak_basis": f"{num_sms} SMs x 128 FP32 lanes x 2 flop x {sm_mhz} MHz (median SM clock "
                              f"sampled during the timed region)",
                "flop_convention": f"{FLOP_PER_INTERACTION} flop per force+jerk interaction",
                "phases_us_per_block_step": {k: 1e3 * v / max(nlaunch, 1) for k, v in phase_ms.items()}}

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
        fp64 = {"interactions_per_s": (st64["interactions"] + float(n) * n) / (ms64[0] / 1e3),
                "block_steps_per_s": st64["block_steps"] / (ms64[0] / 1e3),
                "abs_dE_over_E": abs(F1 - F0) / abs(F0), "ms_per_step": ms64[0],
                "block_steps": st64["block_steps"]}
        c64.close()

    # ---- batched ensemble: 256 Plummer clusters, one persistent cluster launch to t = 1
    ens = None
    if args.ensemble and rank == 0:
        ens = ensemble_bench(nb, torch, dev, sptr, stream)

    # ---- Plummer N = 65536 with Salpeter masses to t = 0.5 (opt-in: slow input generation)
    salp = None
    if args.salpeter and rank == 0:
        salp = salpeter_bench(nb, torch, dev, sptr, stream)

    # ---- centrally concentrated models: King W0 = 6 and 9, N = 16384, to t = 1/4
    king = None
    if args.king and rank == 0:
        king = king_bench(nb, torch, dev, sptr, stream)

    # ---- full-N force sweep (King W0 = 6, N = 2^20), mixed, one evaluation per s
    sweep = None
    if args.sweep and rank == 0:
        sweep = force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz)
        # mixed vs FP64 kernels on the same model at N = 131072 (an FP64 pass over N = 2^20
        # would take a minute): interactions/s per s, both autotuned
        sl = (1, 64, 1024, 16384)
        mx = force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz, n_override=131072, s_list=sl)
        f64 = force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz, n_override=131072, s_list=sl,
                          precision=nb.NB_PREC_FP64)
        sweep["mixed_vs_fp64_n131072"] = [
            {"s": a["s"], "mixed_interactions_per_s": a["interactions_per_s"],
             "fp64_interactions_per_s": b["interactions_per_s"],
             "speedup": a["interactions_per_s"] / b["interactions_per_s"]} for a, b in zip(mx["points"], f64["points"])]

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        nth = oracle.default_threads()
        r = oracle_sample(snap, args.ref_t_end, nth)
        cpu = {"value": r["interactions"] / r["seconds"], "unit": "interactions/s", "cores": nth,
               "kind": "oracle", "sample": f"init (s=N pass) + {r['block_steps']} block steps to "
                                          f"t={args.ref_t_end} of the same N=16384 Plummer run "
                                          f"({r['seconds']:.1f} s); host {cpu_model()}"}

    c.close()
    if rank == 0:
        line = {
            "metric": "force+jerk interactions/s", "value": value, "unit": "interactions/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair arithmetic, f64 state",
            "data": "synthetic (seeded Plummer sphere, N-body units)",
            "config": dict(WORKLOAD, l2="flushed (256 MB write) before every timed step",
                           parallelism=f"replicas x{ws}" if ws > 1 else "single GPU"),
            "block_steps_per_s": dist_sum(bsteps * args.steps, dev) / (total_ms / 1e3),
            "block_steps": bsteps, "abs_dE_over_E": dE, "block_size_hist": size_hist(st),
            "gpu_launches": launches * args.steps,
            "clocks": clk,
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "interactions/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_total / len(e2e_ms)},
            "fp64_gpu": fp64,
            "ensemble": ens, "salpeter": salp, "king": king,
            "force_sweep": sweep,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    return 0


def size_hist(st):
    """Block steps per block-size bucket, {upper bound 2^b: count} for the non-empty buckets."""
    return {str(1 << b): int(c) for b, c in enumerate(st["size_hist"]) if c}


def force_traffic():
    """Per-launch DRAM traffic of the force kernel on this workload, from the committed ncu
    summary, or None when the kernel sources have changed since it was taken."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    prof = os.path.join(root, "profiles", "force_traffic_plummer_n16384_t1over64.md")
    srcs = ["nb_force.cu", "nb_pair.cuh", "nb_internal.cuh"]
    try:
        text = open(prof).read()
        h = hashlib.sha256()
        for f in srcs:
            with open(os.path.join(root, "paper_0711_0643_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() not in text:
            return None
        for line in text.splitlines():
            if line.startswith("traffic_bytes_per_launch:"):
                return float(line.split(":")[1])
    except OSError:
        return None
    return None


def ensemble_bench(nb, torch, dev, sptr, stream, nc=256, n_lo=256, n_hi=8192):
    """256 independent Plummer clusters, N_c = round(exp(U[ln 256, ln 8192])) (seeded),
    eps = 4/N_c, equal masses, each with its own block schedule, advanced to t = 1 by
    one persistent launch of thread-block clusters (mixed precision)."""
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
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2v = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nb.nb_ensemble_init(c.ctx, off, m, x, v, e2)
    e1.record(stream)
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
    return {"workload": f"{nc} Plummer clusters, N log-uniform in [{n_lo}, {n_hi}] (total {int(off[-1])}), eps=4/N, "
                        f"t=0->{T_END}, one persistent cluster launch",
            "run_ms": run_s * 1e3, "init_ms": init_s * 1e3,
            "interactions_per_s": total_inter / (run_s + init_s),
            "block_steps_per_s": float(bs.sum()) / run_s, "block_steps": int(bs.sum()),
            "worst_abs_dE_over_E": float(dE.max()), "median_abs_dE_over_E": float(np.median(dE)),
            "worst_member": {"index": int(np.argmax(dE)), "n": int(np.diff(off)[int(np.argmax(dE))])},
            "n_min": int(np.diff(off).min()), "n_max": int(np.diff(off).max())}


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
    return {"workload": f"plummer N={n} Salpeter masses [0.1, 100] slope -2.35, eps=1/4096, t=0->{t_end}, mixed",
            "ms": sec * 1e3, "interactions_per_s": inter / sec, "block_steps": st["block_steps"],
            "block_steps_per_s": st["block_steps"] / sec, "mean_active": st["particle_steps"] / max(st["block_steps"], 1),
            "abs_dE_over_E": abs(E1 - E0) / abs(E0), "block_size_hist": size_hist(st)}


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
        out.append({"workload": f"king W0={w0:g} N={n} eps=1/1024, t=0->{t_end}, mixed", "ms": sec * 1e3,
                    "interactions_per_s": (st["interactions"] + float(n) * n) / sec,
                    "block_steps": st["block_steps"], "block_steps_per_s": st["block_steps"] / sec,
                    "mean_active": st["particle_steps"] / max(st["block_steps"], 1),
                    "abs_dE_over_E": abs(E1 - E0) / abs(E0), "block_size_hist": size_hist(st)})
    return out


def force_sweep(nb, torch, dev, sptr, num_sms, sm_mhz, n_override=None, s_list=None, autotune=True,
                precision=None):
    """King W0 = 6, N = 1,048,576, eps = 1e-3: one mixed force evaluation per active-set
    size s in {1, 64, 1024, 16384, N} (active = first s of a seeded permutation, ascending),
    split factor autotuned; interactions/s and FP32 roofline fraction per s. Each point is
    the median of single nb_force_jerk_dev calls (active list in, a/k/phi out, all on the
    device), each timed with L2 flushed before it."""
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
           "l2": "flushed (256 MB write) before every timed call; median of single calls"}
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
        for _ in range(3):
            nb.nb_force_jerk_dev(c.ctx, idx_d.data_ptr(), s, a_d.data_ptr(), k_d.data_ptr(), p_d.data_ptr())
        # each timed call starts with L2 flushed (the j-records, 40 MB at N = 2^20, would
        # otherwise stay in the 129 MB L2 between calls): median of single calls
        reps = 9 if s < n else 2
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        times = []
        for _ in range(reps):
            l2_flush.zero_()
            torch.cuda.synchronize(dev)
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
    ap.add_argument("--model", action="store_true",
                    help="fit the per-block-step timing model (select, predict, force, correct) and print it")
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
    if args.model:
        return main_model(args)
    return main_gpu(args)


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


def main_model(args):
    """The paper's timing model (Sect. 4.1) refitted on this GPU: per block step
    T = [a_sel + b_sel N] + [a_pr + b_pr N] + [a_f + tau_f s N] + [a_cr + tau_cr s], fitted by
    least squares to the phase totals of host-driven runs (nb_run_timed, each phase bracketed
    by events) of Plummer models N = 1024 .. 65536 (eps = 4/N, t = 0 -> 1/16, autotuned); the
    fitted model then predicts every graph-loop run (nb_run) from its block-step count and
    sum of s, next to the measured time. Printed as one JSON line (not a bench line)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    import paper_0711_0643_gb300 as pkg
    pkg.build()
    from paper_0711_0643_gb300 import nbody as nb
    nb.load()
    import ics
    gate_us = None
    rows = []
    for n in (1024, 2048, 4096, 8192, 16384, 32768, 65536):
        snap = ics.plummer(n, seed=ics.BASE_SEED + 70 + n.bit_length(), eps=4.0 / n,
                           scale="continuum" if n > 16384 else "auto")
        c = nb.Context(precision=nb.NB_PREC_MIXED, device=0, stream=stream.cuda_stream)
        c.init(snap)
        nb.nb_autotune(c.ctx)
        c.init(snap)
        _, nl, _, ph = nb.nb_run_timed(c.ctx, 1.0 / 16, phases=True)
        st = nb.nb_stats(c.ctx)
        c.init(snap)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        nb.nb_run(c.ctx, 1.0 / 16)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st2 = nb.nb_stats(c.ctx)
        c.close()
        rows.append({"n": n, "steps": st["block_steps"], "sum_s": st["particle_steps"],
                     "phase_us": {k: 1e3 * v for k, v in ph.items()},
                     "run_steps": st2["block_steps"], "run_sum_s": st2["particle_steps"],
                     "run_us": 1e3 * e0.elapsed_time(e1)})
    # every phase total of run r: steps_r * a + (N_r * steps_r or sum(s N) or sum s) * b
    A = {"select": [], "predict": [], "force": [], "correct": []}
    y = {k: [] for k in A}
    for r in rows:
        n, k, ss = r["n"], r["steps"], r["sum_s"]
        A["select"].append((k, k * n)); A["predict"].append((k, k * n))
        A["force"].append((k, ss * n)); A["correct"].append((k, ss))
        for key in A:
            y[key].append(r["phase_us"][key])
    fit = {}
    for key in A:
        coef, *_ = np.linalg.lstsq(np.array(A[key], dtype=float), np.array(y[key]), rcond=None)
        fit[key] = {"a_us": float(coef[0]), "b_us": float(coef[1])}
    # the phases above include a gate (delay kernel + events) each; the graph loop has none:
    # predict the graph loop's time with the fixed terms less the measured gate overhead
    for r in rows:
        k, ss, n = r["run_steps"], r["run_sum_s"], r["n"]
        t = 0.0
        for key, f in fit.items():
            lin = {"select": k * n, "predict": k * n, "force": ss * n, "correct": ss}[key]
            t += f["a_us"] * k + f["b_us"] * lin
        r["model_phase_sum_us"] = t
        r["ratio_measured_to_phase_sum"] = r["run_us"] / t
    out = {"model": "per block step T = sum over phases of (a + b x work), work = N (select, predict), "
                     "s N (force), s (correct); fitted to nb_run_timed phase totals",
           "fit": fit, "runs": rows}
    print(json.dumps(out))
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
