"""Throughput of the SDPD time step (Velocity Verlet + Metropolised
Shardlow-like sweep) on GB300.

Workload (default): a single large fluid of N = 128^3 = 2,097,152 particles on
a jittered simple-cubic lattice (spacing a = 1, jitter +-0.05a, L = 128),
Lucy kernel h = 2.5a, kT = 1, K = 50, eta = 1, dt = 0.005, EMS, mixed
precision (float32 pair arithmetic, float64 internal energies).  One bench
step = one full time step of every stage on the device.

Prints one JSON line (see the keys below).  With torchrun (N > 1 ranks) every
rank runs an independent replica (different seed) on its own GPU; ``value`` is
the particle-steps of all ranks divided by the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload, see ``cpu_sample``).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1707_04232_gb300.inputs import Workload, lattice_state  # noqa: E402

METRIC = "particle-steps/s (SDPD+Metropolis SSA) at N=2M; % HBM roofline; vs FP64 form"
UNIT = "particle-steps/s"
SMS = 152
FP32_LANES_PER_SM = 128
NOMINAL_SM_MHZ = 2070.0
FALLBACK_HBM_GBS = 6800.0
# algorithmic traffic of one particle-step: state read + written once
BYTES_PER_PARTICLE_STEP = {"mixed": 64.0, "fp64": 112.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's run length, 1000 fluid, 500 ensemble, 5 adjoint)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=128, help="lattice sites per axis")
    ap.add_argument("--scheme", default="ems", choices=["ssa", "ams", "ems", "none"])
    ap.add_argument("--K", type=float, default=50.0)
    ap.add_argument("--dt", type=float, default=0.005)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 form of the same step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=32, help="lattice sites per axis of the CPU sample")
    ap.add_argument("--workload", default="fluid", choices=["fluid", "ensemble", "adjoint"],
                    help="fluid: the single large fluid; ensemble: 256 independent replicas; "
                         "adjoint: gradient of the virial pressure after 100 Velocity Verlet steps")
    ap.add_argument("--adj-n", type=int, default=32, help="adjoint workload: lattice sites per axis")
    ap.add_argument("--adj-K", type=float, default=100.0)
    ap.add_argument("--adj-steps", type=int, default=100, help="adjoint workload: Verlet steps per gradient")
    ap.add_argument("--adj-every", type=int, default=10, help="adjoint workload: checkpoint interval")
    ap.add_argument("--adj-sweep64", action="store_true",
                    help="adjoint workload: float64 pair arithmetic in the recorded sweeps (default float32)")
    ap.add_argument("--replicas", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of timing the candidates first")
    ap.add_argument("--shapes", default=None,
                    help="fixed launch shapes fd_variant/pair_threads (e.g. 2/32) instead of the autotuner")
    args = ap.parse_args()
    if args.steps is None:  # the run length of each workload's configuration
        args.steps = {"fluid": 1000, "ensemble": 500, "adjoint": 5}[args.workload]
    return args


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            return d, "measured"
        except Exception:
            pass
    return {}, "fallback"


def hbm_peak():
    d, src = measured_peaks()
    for k in ("hbm_gbs", "hbm_GBs", "hbm"):
        if k in d:
            v = d[k]
            if isinstance(v, dict):
                v = v.get("value", v.get("gbs"))
            try:
                return float(v), "of measured"
            except Exception:
                pass
    return FALLBACK_HBM_GBS, "of fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def cpu_sample(args, steps: int, n: int | None = None, K: float | None = None, kT: float = 1.0):
    """Time the FP64 oracle on a bounded sample of the workload: an n^3
    (default args.cpu_n^3) sub-lattice with the same density, temperature,
    K, dt and scheme.  Returns (particle-steps/s, threads, description)."""
    import oracle as O

    n = args.cpu_n if n is None else n
    w = Workload(n=n, K=args.K if K is None else K, kT=kT)
    q, p, e = lattice_state(w)
    scheme = {"ssa": O.SCHEME_SSA, "ams": O.SCHEME_AMS, "ems": O.SCHEME_EMS, "none": O.SCHEME_NONE}[args.scheme]
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=scheme).params()
    O.lib()
    t0 = time.perf_counter()
    st, q, p, e, stats, _ = O.run(P, q, p, e, args.dt, steps, seed=1)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    desc = ("O(N^2) brute-force FP64 oracle, %d^3 = %d-particle sub-lattice of the same fluid, %d step(s), "
            "%.1f s" % (n, w.N, steps, dt))
    return w.N * steps / dt, threads, desc


# seconds of oracle work the reference arm's timed steps may take in total;
# a larger --steps shrinks the per-step sample instead (cost ~ N^2 = n^6)
REFERENCE_BUDGET_S = 240.0


def _bounded_n(n: int, t_step: float, steps: int, n_min: int = 10) -> int:
    """Largest lattice size <= n whose steps fit REFERENCE_BUDGET_S, given
    one step's time at n (the oracle's cost grows as n^6)."""
    if steps * t_step <= REFERENCE_BUDGET_S:
        return n
    return max(n_min, int(n * (REFERENCE_BUDGET_S / (steps * t_step)) ** (1.0 / 6.0)))


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, for the workload's metric
    and config: each timed step is a bounded sample of the workload (a
    sub-lattice of the fluid, one replica-sized lattice of the ensemble, or
    one oracle gradient).  One untimed probe step (the warm-up) sizes the
    sample so that the timed steps stay within REFERENCE_BUDGET_S."""
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    if args.workload == "adjoint":
        metric, config = adjoint_metric(args.adj_steps), adjoint_config(args, Workload(n=args.adj_n, K=args.adj_K))
        ps1, _, _ = adjoint_cpu_sample(args)
        n = _bounded_n(16, 16 ** 3 / ps1 * 2, steps)
        t, threads, descs = 0.0, 1, []
        for _ in range(steps):
            ps_k, threads, d = adjoint_cpu_sample(args, n=n)
            t += n ** 3 * 2 / ps_k
            descs.append(d)
        ps, desc, per_step_units = steps * n ** 3 * 2 / t, "%d samples: %s" % (steps, descs[-1]), n ** 3 * 2
    else:
        if args.workload == "ensemble":
            ws = ensemble_members(args, 0)
            metric, config = METRIC, ensemble_config(args, ws)
            w0 = min(ws, key=lambda w: w.n)  # the smallest replica, with its K and kT
            n0, K, kT, what = w0.n, w0.K, w0.kT, "replica-sized"
        else:
            metric, config = METRIC, workload_config(args)
            n0, K, kT, what = args.cpu_n, args.K, 1.0, "sub-lattice"
        ps1, _, _ = cpu_sample(args, 1, n=n0, K=K, kT=kT)
        n = _bounded_n(n0, n0 ** 3 / ps1, steps)
        ps, threads, desc = cpu_sample(args, steps, n=n, K=K, kT=kT)
        desc = "%s sample; %s" % (what, desc)
        per_step_units = n ** 3
    line = {
        "impl": "reference", "metric": metric, "value": ps, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * per_step_units / ps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": ps, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": ps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def workload_config(args):
    N = args.n ** 3
    return {"workload": "single large fluid: %d^3 = %d particles, jittered sc lattice, L=%d, Lucy h=2.5a, "
                        "kT=1, K=%g, dt=%g, %s, %s" % (args.n, N, args.n, args.K, args.dt,
                                                      args.scheme.upper(), args.precision),
            "N": N, "K": args.K, "kT": 1.0, "dt": args.dt, "h": 2.5, "kernel": "lucy",
            "scheme": args.scheme, "precision": args.precision,
            "l2": "inputs larger than L2 (per-step working set > 129 MB)"}


# algorithmic float operations of the pair passes, per neighbour pair (r < h)
# visit (counted from each kernel's arithmetic: displacement, r^2, sqrt,
# kernel polynomial, accumulation; adj_pass_* are the reverse passes), and of
# one pair update of the sweep
FLOPS_PER_VISIT = {"density_eos": 18.0, "kick1_drift_bin": 24.0, "kick2": 24.0,
                   "adj_pass_A": 23.0, "adj_pass_B": 66.0}
FP64_NOMINAL_TFLOPS = 1.25  # GB300 float64, nominal
# DRAM traffic of one colour launch of the mixed-precision sweep, per
# particle: dram__bytes_read.sum + dram__bytes_write.sum of one launch at
# N = 96^3 (50.21 MB + 3.26 MB), divided by the particles every colour
# launch visits once; a launch's traffic scales with N
FD_COLOUR_DRAM_BYTES_PER_PARTICLE = (50.207488e6 + 3.262720e6) / 96 ** 3
FLOPS_PER_PAIR_UPDATE = {"ems": 210.0, "ams": 150.0, "ssa": 140.0}


def autotune(args, s, seed):
    """The library's autotuner on the loaded state (it restores the state):
    the chosen launch shapes and their time per step, or the defaults, or
    the shapes given on the command line."""
    if args.shapes:
        v, t = (int(x) for x in args.shapes.split("/"))
        s.set_tuning(v, t)
        return {"autotuned": False, **s.tuning}
    if args.no_autotune:
        return {"autotuned": False, **s.tuning}
    t, ms = s.autotune(args.dt, steps=2, seed=seed)
    return {"autotuned": True, **t, "trial_ms_per_step": ms}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1707_04232_gb300 import sdpd

    torch.cuda.set_device(local_rank)
    dev_index = torch.cuda.current_device()
    w = replica_workload(args, rank)
    q, p, e = lattice_state(w)
    scheme = {"ssa": sdpd.SCHEME_SSA, "ams": sdpd.SCHEME_AMS, "ems": sdpd.SCHEME_EMS, "none": sdpd.SCHEME_NONE}[args.scheme]
    prec = sdpd.MIXED if args.precision == "mixed" else sdpd.FP64
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        fma = sdpd.sdpd_fma_peak(prec, stream.cuda_stream)
        s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=prec, scheme=scheme, stream=stream)
        s.set_state(q, p, e)
        for _ in range(args.warmup):
            s.step(args.dt, 1, seed=1234 + rank)
        tuning = autotune(args, s, 1234 + rank)
        s.sync()
        o0 = s.observables()
        s.reset_counters()
        launches0 = s.kernel_launches
        s.enable_stage_timing(True)
        clocks = ClockSampler(dev_index)
        clocks.start()
        barrier(world)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        s.step(args.dt, args.steps, seed=1234 + rank)
        end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        ms = start.elapsed_time(end)
        stages = s.stage_times()
        launches = s.kernel_launches - launches0
        o1 = s.observables()
    value, ms_max = aggregate(w.N, args.steps, ms, world)
    # ---- roofline of the dominant stage ----
    top = max(stages, key=lambda k: stages[k][0])
    top_ms, top_launches = stages[top]
    per_launch_s = top_ms * 1e-3 / max(1, top_launches)
    sm_max = (clk or {}).get("sm_max_mhz") or NOMINAL_SM_MHZ
    alu_peak = (SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12 if args.precision == "mixed"
                else FP64_NOMINAL_TFLOPS)  # TFLOP/s of the arithmetic the pair passes use
    if top == "fd_colours":
        units = o1["n_pairs"] / max(1, top_launches)  # pair updates per colour launch
        flops = FLOPS_PER_PAIR_UPDATE[args.scheme] * units
    elif top in FLOPS_PER_VISIT:
        nvisits = w.N * 80.0  # neighbour visits per launch (lattice: 80 per particle)
        flops = FLOPS_PER_VISIT[top] * nvisits
    else:
        flops = None
    roof = None
    if flops is not None:
        ach = flops / per_launch_s / 1e12
        traffic = (FD_COLOUR_DRAM_BYTES_PER_PARTICLE * w.N
                   if top == "fd_colours" and args.precision == "mixed" else None)
        roof = {"kernel": top, "bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": ach / alu_peak, "traffic": traffic,
                "peak_note": ("FP32 FMA peak = 152 SMs x 128 lanes x 2 x %.0f MHz (recipe unit counts, "
                              "sampled max clock)" % sm_max if args.precision == "mixed" else
                              "float64 nominal of GB300 (recipe)")
                             + "; measured %s FMA rate %.2f TFLOP/s (sdpd_fma_peak)"
                             % ("float32" if args.precision == "mixed" else "float64", fma / 1e12),
                "per_launch_ms": per_launch_s * 1e3}
    hbm, hbm_note = hbm_peak()
    bpp = BYTES_PER_PARTICLE_STEP[args.precision]
    hbm_frac = value / world * bpp / (hbm * 1e9)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic", "config": workload_config(args),
        "hbm_roofline": {"bytes_per_particle_step": bpp, "peak_gbs": hbm, "frac": hbm_frac,
                         "note": hbm_note},
        "roofline": roof,
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
        "gpu_launches": launches,
        "clocks": clk,
        "launch_shapes": tuning,
        "physics": {"E0": o0["E"], "E1": o1["E"], "T_kin": o1["T_kin"], "T_int": o1["T_int"],
                    "eps_min": o1["eps_min"], "n_pairs": o1["n_pairs"],
                    "reject_rate": (o1["n_reject_bound"] + o1["n_reject_metropolis"]) / max(1, o1["n_pairs"]),
                    "status": o1["status"]},
    }
    # ---- end to end through the public API with host buffers ----
    if not args.no_e2e:
        e2e = run_e2e(args, s, q, p, e, stream, world, w.N)
        line["e2e"] = e2e
    del s
    # ---- the float64 form of the same step (same workload, a few steps) ----
    if args.precision == "mixed" and not args.no_fp64:
        line["vs_fp64"] = run_fp64_form(args, w, q, p, e, scheme, stream, world, value)
    if rank == 0 and not args.no_cpu and world == 1:
        ps, threads, desc = cpu_sample(args, 2)
        line["cpu_baseline"] = {"value": ps, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))


def run_fp64_form(args, w, q, p, e, scheme, stream, world, mixed_value):
    """Particle-steps/s of the float64 form of the same workload (3 steps
    after 1 warm-up step, CUDA events on the handle's stream), and the
    mixed-precision speed-up over it."""
    import torch
    from paper_1707_04232_gb300 import sdpd

    steps = 3
    with torch.cuda.stream(stream):
        s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=sdpd.FP64, scheme=scheme, stream=stream)
        s.set_state(q, p, e)
        s.step(args.dt, 1, seed=77)
        tuning = None
        if not args.no_autotune and not args.shapes:
            t, _ = s.autotune(args.dt, steps=1, seed=77)
            tuning = t
        s.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        a.record(stream)
        s.step(args.dt, steps, seed=77)
        b.record(stream)
        b.synchronize()
        ms = allreduce_max(a.elapsed_time(b), world)
        del s
    ps = w.N * steps * world / (ms * 1e-3)
    return {"value": ps, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "speedup_of_mixed": mixed_value / ps, "launch_shapes": tuning}


def ensemble_members(args, rank):
    """The batched-ensemble workload: replica sizes log-uniform in
    [2048, 65536] rounded to cubes n^3, K uniform in {5, 20, 100}, kT uniform
    in [0.1, 1.0].  A size whose 2x2x2 cell blocks would hold more than ~200
    particles on average (L/h just below an even number) moves up to the next
    size that fits the block capacity."""
    rng = np.random.default_rng(1000 + rank)
    out = []
    for r in range(args.replicas):
        N = float(np.exp(rng.uniform(np.log(2048.0), np.log(65536.0))))
        n = int(round(N ** (1.0 / 3.0)))
        n = min(max(n, 13), 40)
        while True:
            nc = int(np.floor(n / 2.5))
            nc -= nc % 2
            if (2.0 * n / nc) ** 3 <= 200.0:
                break
            n += 1
        K = float(rng.choice([5.0, 20.0, 100.0]))
        kT = float(rng.uniform(0.1, 1.0))
        out.append(Workload(n=n, K=K, kT=kT, seed=1000 * rank + r))
    return out


def ensemble_config(args, ws):
    return {"workload": "batched ensemble: %d replicas, N log-uniform in [2048, 65536] (cubes), "
                        "K in {5,20,100}, kT in [0.1,1], dt=%g, %s, %s" % (len(ws), args.dt,
                                                                          args.scheme.upper(), args.precision),
            "particles": sum(w.N for w in ws), "replicas": len(ws),
            "sizes": sorted({w.n for w in ws}),
            "l2": "inputs larger than L2"}


def run_ensemble(args, rank, world, local_rank):
    import torch
    from paper_1707_04232_gb300 import sdpd

    torch.cuda.set_device(local_rank)
    dev_index = torch.cuda.current_device()
    ws = ensemble_members(args, rank)
    prec = sdpd.MIXED if args.precision == "mixed" else sdpd.FP64
    scheme = {"ssa": sdpd.SCHEME_SSA, "ams": sdpd.SCHEME_AMS, "ems": sdpd.SCHEME_EMS, "none": sdpd.SCHEME_NONE}[args.scheme]
    members = []
    for w in ws:
        q, p, e = lattice_state(w)
        m = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=prec, scheme=scheme, stream=torch.cuda.Stream())
        m.set_state(q, p, e)
        members.append(m)
    ens = sdpd.SDPDEnsemble(members)
    seeds = [7 + k for k in range(len(members))]
    ntot = sum(w.N for w in ws)
    ens.step(args.dt, 2 * max(2, args.warmup), seeds)  # capture + warm-up
    torch.cuda.synchronize()
    tuning = {"autotuned": False}
    if not args.no_autotune and not args.shapes:
        # the default shapes first, then every member tuned alone, then the
        # graph recaptured with the chosen shapes
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(ens.stream)
        ens.step(args.dt, args.steps, seeds)
        b.record(ens.stream)
        torch.cuda.synchronize()
        untuned_ms = a.elapsed_time(b)
        tuned_trial_ms = ens.autotune(args.dt, steps=4, seeds=seeds)
        ens.step(args.dt, 2 * max(2, args.warmup), seeds)
        torch.cuda.synchronize()
        shapes = {}
        for m in members:
            t = m.tuning
            key = "%d/%d" % (t["fd_variant"], t["pair_threads"])
            shapes[key] = shapes.get(key, 0) + 1
        tuning = {"autotuned": True, "members_by_shape(fd_variant/pair_threads)": shapes,
                  "tuner_ms_per_step": tuned_trial_ms,
                  "untuned_ms_per_step": untuned_ms / args.steps,
                  "untuned_value": ntot * args.steps / (untuned_ms * 1e-3)}
    launches0 = sum(m.kernel_launches for m in members)
    clocks = ClockSampler(dev_index)
    clocks.start()
    barrier(world)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(ens.stream)
    ens.step(args.dt, args.steps, seeds)
    end.record(ens.stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    launches = sum(m.kernel_launches for m in members) - launches0
    # the same members stepped one after the other on one stream, no graph
    seq_steps = 2
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for m in members:
        m.step(args.dt, seq_steps, seed=3)
    torch.cuda.synchronize()
    seq_ps = ntot * seq_steps / (time.perf_counter() - t0)
    # temperatures against the equilibrium value fixed by the energy
    terr = []
    for w, m in zip(ws, members):
        o = m.observables()
        C_K = 1.5 * (w.K - 1.0)
        T_eq = o["E"] / (1.5 * (w.N - 1) + w.N * C_K)
        terr.append(abs(o["T_int"] - T_eq) / T_eq)
    ms_max = allreduce_max(ms, world)
    value = ntot * world * args.steps / (ms_max * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {**ensemble_config(args, ws), "graph_kernel_nodes_per_2_steps": ens.kernel_nodes},
        "unbatched_sequential": {"value": seq_ps, "unit": UNIT, "steps": seq_steps,
                                 "note": "same replicas stepped one after the other on one stream"},
        "temperature_error": {"max": max(terr), "mean": float(np.mean(terr)),
                              "definition": "|<T_int> - T_eq| / T_eq, T_eq = E / (3(N-1)/2 + N C_K)"},
        "gpu_launches": launches, "clocks": clk,
        "launch_shapes": tuning,
    }
    if rank == 0:
        print(json.dumps(line))


def adjoint_cpu_sample(args, n: int = 16):
    """The oracle's gradient on an n^3 (default 16^3) lattice of the same
    fluid, 2 steps: the full steps with their exact Metropolised sweeps
    (increments kept), the virial pressure's gradient, the reverse pass of
    the frozen map (O(N^2) pair loops, forward states kept in memory)."""
    import oracle as O

    w = Workload(n=n, K=args.adj_K, kT=1.0, seed=0)
    q, p, e = lattice_state(w)
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=O.SCHEME_EMS).params()
    O.lib()
    steps = 2
    t0 = time.perf_counter()
    dps, des, (qn, pn, en) = O.sweep_increments(P, q, p, e, args.dt, steps, 3)
    _, gq, gp, ge, _ = O.virial_vjp(P, qn, pn, en)
    O.frozen_vjp(P, q, p, e, args.dt, steps, dps, des, gq, gp, ge)
    dt = time.perf_counter() - t0
    desc = ("FP64 oracle gradient of the virial pressure with the EMS sweeps frozen (O(N^2) pair loops, "
            "single thread), %d^3 = %d-particle lattice of the same fluid, %d steps, %.1f s" % (n, w.N, steps, dt))
    return w.N * steps / dt, 1, desc


def adjoint_metric(ns):
    return "gradient particle-steps/s (virial pressure after %d steps, EMS sweeps frozen, reverse mode)" % ns


def adjoint_config(args, w):
    ns, every = args.adj_steps, args.adj_every
    return {"workload": "adjoint: %d^3 = %d particles, jittered sc lattice, L=%d, Lucy h=2.5a, kT=1, "
                        "K=%g, dt=%g, %d steps (Verlet + EMS sweep, increments frozen), "
                        "checkpoint every %d, float64 state, Verlet and reverse pass; sweep pair "
                        "arithmetic %s"
                        % (w.n, w.N, w.n, w.K, args.dt, ns, every,
                           "float64" if args.adj_sweep64 else "float32"),
            "N": w.N, "K": w.K, "steps_per_gradient": ns, "checkpoint_every": every,
            "l2": "working set below L2 (the workload is fixed at 32^3)"}


def run_adjoint(args, rank, world, local_rank):
    """One bench step = one gradient of the virial pressure after
    args.adj_steps steps (float64 Velocity Verlet, then the exact
    Metropolised sweep with its increments frozen, the sweep's pair
    arithmetic in float32 unless --adj-sweep64; checkpoint every
    args.adj_every steps) with respect to (q0, p0, eps0, h, c_rho, C_K):
    set_state from device-resident inputs, the recorded forward run, the
    virial pressure and its gradient, the reverse pass (float64)."""
    import torch
    from paper_1707_04232_gb300 import sdpd

    torch.cuda.set_device(local_rank)
    dev_index = torch.cuda.current_device()
    w = Workload(n=args.adj_n, K=args.adj_K, kT=1.0, seed=rank)
    q, p, e = lattice_state(w)
    ns, every = args.adj_steps, args.adj_every
    stream = torch.cuda.Stream()
    steps = max(1, min(args.steps, 5))
    with torch.cuda.stream(stream):
        fma64 = sdpd.sdpd_fma_peak(sdpd.FP64, stream.cuda_stream)
        s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=sdpd.FP64, scheme=sdpd.SCHEME_EMS,
                      sweep_f32=not args.adj_sweep64, stream=stream)
        qd, pd, ed = (torch.as_tensor(a, device="cuda") for a in (q, p, e))

        s.set_state(qd, pd, ed)
        tuning = autotune(args, s, 3)

        def gradient():
            s.set_state(qd, pd, ed)
            tape = s.vv_record(args.dt, ns, every, 3)
            val, gq, gp, ge, gth = s.virial(grad=True)
            return val, s.vv_adjoint(tape, gq, gp, ge), gth

        for _ in range(max(1, args.warmup)):
            gradient()
        torch.cuda.synchronize()
        s.reset_counters()
        launches0 = s.kernel_launches
        s.enable_stage_timing(True)
        clocks = ClockSampler(dev_index)
        clocks.start()
        barrier(world)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        fwd_ms = adj_ms = 0.0
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.set_state(qd, pd, ed)
            tape = s.vv_record(args.dt, ns, every, 3)
            b.record(stream)
            val, gq, gp, ge, gth = s.virial(grad=True)
            g0 = s.vv_adjoint(tape, gq, gp, ge)
            c.record(stream)
            c.synchronize()
            fwd_ms += a.elapsed_time(b)
            adj_ms += b.elapsed_time(c)
        ev[1].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop()
        ms = ev[0].elapsed_time(ev[1])
        stages = s.stage_times()
        launches = s.kernel_launches - launches0
        nbr_mean = float(s.neighbour_counts().mean())
    ms_max = allreduce_max(ms, world)
    value = w.N * ns * steps * world / (ms_max * 1e-3)
    # roofline of the dominant stage (float64 arithmetic)
    top = max((k for k in stages if k in FLOPS_PER_VISIT or k == "fd_colours"), key=lambda k: stages[k][0])
    top_ms, top_launches = stages[top]
    per_launch_s = top_ms * 1e-3 / max(1, top_launches)
    if top == "fd_colours":
        # pair updates per colour launch: every neighbour pair once per sweep,
        # over 8 colour launches
        units = w.N * nbr_mean / 2.0 / 8.0
        flops = FLOPS_PER_PAIR_UPDATE["ems"] * units
    else:
        units = w.N * nbr_mean
        flops = FLOPS_PER_VISIT[top] * units
    ach = flops / per_launch_s / 1e12
    if top == "fd_colours" and not args.adj_sweep64:  # float32 pair arithmetic
        sm_max = (clk or {}).get("sm_max_mhz") or NOMINAL_SM_MHZ
        peak = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        note = ("FP32 FMA peak = 152 SMs x 128 lanes x 2 x %.0f MHz (recipe unit counts, sampled max "
                "clock); the sweep's pair arithmetic is float32" % sm_max)
    else:
        peak = FP64_NOMINAL_TFLOPS
        note = ("float64 nominal of GB300 (recipe); measured float64 FMA rate %.3f TFLOP/s "
                "(sdpd_fma_peak), frac of measured %.3f" % (fma64 / 1e12, ach / (fma64 / 1e12)))
    roof = {"kernel": top, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None, "peak_note": note,
            "per_launch_ms": per_launch_s * 1e3,
            ("pair_updates_per_launch" if top == "fd_colours" else "visits_per_launch"): units}
    # end to end: host inputs in, host gradients out
    qh, ph, eh = (torch.from_numpy(a).pin_memory() for a in (q, p, e))
    outs = [torch.empty((w.N, 3), dtype=torch.float64).pin_memory() for _ in range(2)]
    outs.append(torch.empty(w.N, dtype=torch.float64).pin_memory())
    t0 = time.perf_counter()
    e2e_steps = 2
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            qd.copy_(qh, non_blocking=True)
            pd.copy_(ph, non_blocking=True)
            ed.copy_(eh, non_blocking=True)
            _, (gq0, gp0, ge0, _), _ = gradient()
            for o, g in zip(outs, (gq0, gp0, ge0)):
                o.copy_(g, non_blocking=True)
        stream.synchronize()
    e2e_s = allreduce_max(time.perf_counter() - t0, world)
    line = {
        "metric": adjoint_metric(ns),
        "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.adj_sweep64 else "f64 (sweep f32)", "data": "synthetic",
        "config": adjoint_config(args, w),
        "forward_ms_per_gradient": fwd_ms / steps, "reverse_ms_per_gradient": adj_ms / steps,
        "reverse_over_forward": adj_ms / max(fwd_ms, 1e-9),
        "roofline": roof,
        "stages_ms_per_gradient": {k: v[0] / steps for k, v in stages.items()},
        "gpu_launches": launches, "clocks": clk,
        "e2e": {"value": w.N * ns * e2e_steps * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 56 * w.N,
                "d2h_bytes_per_step": 56 * w.N, "steps": e2e_steps,
                "note": "per gradient: state from pinned host, forward + reverse, gradients to pinned host"},
        "launch_shapes": tuning,
        "physics": {"virial_pressure": val, "dP_dtheta(h,c_rho,C_K)": [float(x) for x in g0[3] + gth]},
    }
    if rank == 0 and not args.no_cpu and world == 1:
        ps, threads, desc = adjoint_cpu_sample(args)
        line["cpu_baseline"] = {"value": ps, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))


def run_e2e(args, s, q, p, e, stream, world, N):
    """Each e2e step: host->device copy of the state from pinned memory
    (sdpd_set_state), one time step, device->host copy of the new state
    (sdpd_get_state)."""
    import torch

    qh = torch.from_numpy(q).pin_memory()
    ph = torch.from_numpy(p).pin_memory()
    eh = torch.from_numpy(e).pin_memory()
    qo = torch.empty_like(qh).pin_memory()
    po = torch.empty_like(ph).pin_memory()
    eo = torch.empty_like(eh).pin_memory()
    from paper_1707_04232_gb300 import sdpd

    def one(k):
        sdpd._check(sdpd.sdpd_set_state(s.h, qh.data_ptr(), ph.data_ptr(), eh.data_ptr(), 0), "set_state")
        s.fd_step = k
        s.step(args.dt, 1, seed=99)
        sdpd._check(sdpd.sdpd_get_state(s.h, qo.data_ptr(), po.data_ptr(), eo.data_ptr(), 0), "get_state")

    nsteps = max(1, min(args.steps, 10))
    for k in range(2):
        one(k)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(nsteps):
        one(k)
    torch.cuda.synchronize()
    dt = allreduce_max(time.perf_counter() - t0, world)
    return {"value": N * nsteps * world / dt, "unit": UNIT, "h2d_bytes_per_step": 56 * N,
            "d2h_bytes_per_step": 56 * N, "steps": nsteps,
            "note": "per step: set_state from pinned host (q,p,eps f64), 1 time step, get_state to pinned host"}


_dist = None


def set_process_group(dist_module):
    """Use an initialised torch.distributed (NCCL on GPUs, gloo on CPU) for
    the barrier and the max-over-ranks of the timings."""
    global _dist
    _dist = dist_module


def barrier(world):
    if world > 1:
        _dist.barrier()


def allreduce_max(x, world):
    """The largest of the ranks' values of x (every rank gets it)."""
    if world == 1:
        return x
    import torch
    dev = "cuda" if _dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    _dist.all_reduce(t, op=_dist.ReduceOp.MAX)
    return float(t.item())


def replica_workload(args, rank):
    """Each rank's independent replica: the same fluid, its own seed."""
    return Workload(n=args.n, K=args.K, kT=1.0, seed=rank)


def aggregate(n_local, steps, ms_local, world):
    """Whole-job throughput of weakly scaled replicas: all ranks'
    particle-steps over the slowest rank's time.  Returns (value, ms_max)."""
    ms_max = allreduce_max(ms_local, world)
    return n_local * steps * world / (ms_max * 1e-3), ms_max


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
        set_process_group(dist)
    if args.workload == "ensemble":
        run_ensemble(args, rank, world, local_rank)
    elif args.workload == "adjoint":
        run_adjoint(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        _dist.destroy_process_group()


if __name__ == "__main__":
    main()
