"""Benchmark: noisy QAOA trajectory ensembles on GB300 through the libqnoise C ABI.

Workload (one "step"): the 20-qubit p=3 QAOA MaxCut circuit on a seeded
3-regular graph with depolarizing noise (p1=1e-3, p2=1e-2) and amplitude damping
(gamma=5e-3) after every gate, K=4096 trajectories: Philox Kraus sampling, every
gate sweep with its damping draws, and the ensemble accumulation of <C> and
sigma_approx (the one-statevector-per-trajectory mode runs 64 statevectors per
launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gq|reference] [--sharing 0|1]

Prints one JSON line (rank 0).  `value` is trajectories/s timed with CUDA events
on the library's stream (inputs -- graph, angles, noise -- resident; every step
regenerates all trajectories on the device).  The default mode shares the state
of common Kraus prefixes between trajectories (exact); the same line reports
the one-statevector-per-trajectory mode under `per_trajectory_mode`.  `e2e` times the same call through
the C ABI from host buffers to the host-side <C> and sigma_approx.
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
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

from paper_2210_15874_gb300 import workloads as W  # noqa: E402

METRIC = "noisy trajectories/s at fixed <C> error"
UNIT = "trajectories/s"
PROFILE_PERIOD = 4  # time every 4th sweep launch with a CUDA event pair


WORKLOADS = {
    # name: (factory, headline mode, comparison mode); a mode is (sharing, fusion)
    "damping20": (W.damping_n20, (True, True), (False, True)),
    "precision26": (W.precision_n26, (False, True), (False, False)),
    "precision30": (W.precision_n30, (False, True), (False, False)),
    "gradient16": (W.gradient_n16, (False, True), (False, False)),
    "plain8": (W.plain_n8, (False, True), (False, False)),
}


def workload(name="damping20"):
    return WORKLOADS[name][0]()


def config_of(w, extra=None):
    state_mib = 8 * (1 << w.n) / 2 ** 20
    cfg = {"workload": w.name, "n": w.n, "p": w.p, "graph": "seeded 3-regular", "edges": int(len(w.edges)),
           "gates": w.gate_count, "trajectories": w.trajectories, "launch_batch": w.batch,
           "noise": {"p1": w.p1, "p2": w.p2, "damping": w.damping, "twoq": "15-Pauli depolarizing"},
           "state": f"complex64 statevector, {state_mib:g} MiB per trajectory",
           "l2": f"inputs larger than L2: {state_mib * w.batch / 1024:g} GiB of statevectors per launch "
                 "(L2 129 MB)" if state_mib * w.batch > 129 else "launch fits in L2"}
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            why = "nvidia-smi unavailable" if self.proc is None else "no sample: timed region under 200 ms"
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w, budget_s: float = 15.0):
    """FP64 oracle (trajectory simulator) on the host's cores: a bounded sample
    of the same workload's trajectories (the first `count` ids)."""
    import oracle

    cores = os.cpu_count() or 1
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    # calibrate on one trajectory per core, then extend up to the budget
    t = time.perf_counter()
    oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, 0, cores, want_amps=False, want_branches=False,
                    threads=cores)
    first = time.perf_counter() - t
    count = cores
    rounds = max(0, int((budget_s - first) / max(first, 1e-3)))
    if rounds > 0:
        t = time.perf_counter()
        oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, cores, cores * rounds, want_amps=False,
                        want_branches=False, threads=cores)
        el = time.perf_counter() - t
        count, elapsed = cores * rounds, el
    else:
        elapsed = first
    # one core alone, on one trajectory of the same workload
    t = time.perf_counter()
    oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, 0, 1, want_amps=False, want_branches=False, threads=1)
    single = 1.0 / (time.perf_counter() - t)
    return {"value": count / elapsed, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{count} trajectories (ids {'0' if rounds == 0 else cores}..) of {w.name}, "
                      f"FP64 statevector oracle, OpenMP over trajectories",
            "single_thread": {"value": single, "unit": UNIT, "sample": f"trajectory 0 of {w.name}, 1 thread"},
            "cpu_model": cpu_model()}


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle as it stands, timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    w = workload()
    cores = os.cpu_count() or 1
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    per_step = cores  # one trajectory per core per step: a bounded sample of the 4096

    def step(i):
        oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, (i * per_step) % w.trajectories, per_step,
                        want_amps=False, want_branches=False, threads=cores)

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    el = time.perf_counter() - t
    value = per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, {"sample_per_step": per_step}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} trajectories per step of {w.name}"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def measure(qn, w, args, mode, stream, rank, world, local, pg, with_e2e, precision=0):
    """Time `args.steps` whole-ensemble steps (after `args.warmup`) in one mode."""
    import torch

    sharing, fusion = mode
    b = qn.Batch(w.n, w.trajectories, w.seed, launch_batch=0 if sharing else w.batch, stream=stream)
    b.set_sharing(sharing)
    b.set_fusion(fusion)
    b.set_precision(precision)
    b.set_launch_mode(getattr(args, "launch_mode", 0))
    # weak scaling: rank r evolves global trajectories [r K, (r+1) K)
    if world > 1:
        b.set_offset(rank * w.trajectories)
    kw = w.noise_kwargs()

    def step():
        b.run_qaoa(w.edges, w.gammas, w.betas, **kw)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    mean, se = b.expectation()
    b.set_profiling(PROFILE_PERIOD)
    for k in range(5):
        b.profile_read(k)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches, sweep_bytes, states = 0, 0.0, 0
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            info = b.run_info()
            launches += info["launches"]
            sweep_bytes += info["sweep_bytes"]
            states += info["states"]
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
        pg.barrier()
    res = dict(ms=ms, value=w.trajectories * args.steps * world / (ms / 1e3), mean=mean, se=se,
               launches=launches, sweep_bytes_per_step=sweep_bytes / args.steps, states_per_step=states / args.steps,
               sweeps=b.profile_read(0), inits=b.profile_read(1), accs=b.profile_read(2),
               groups=b.profile_read(3), mixers=b.profile_read(4), clocks=clocks.summary())
    b.set_profiling(0)
    if with_e2e:
        # end to end through the C ABI from host buffers: run + <C> + sigma to a page-locked host buffer
        e2e_steps = max(1, min(args.steps, 3))
        sigma = torch.empty(1 << w.n, dtype=torch.float64, pin_memory=True).numpy()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            b.run_qaoa(w.edges, w.gammas, w.betas, **kw)
            b.expectation()
            b.probs(out=sigma)
        el = time.perf_counter() - t
        if pg:
            tt = torch.tensor([el], device="cuda")
            pg.all_reduce(tt, op=pg.ReduceOp.MAX)
            el = float(tt.item())
        res["e2e_value"] = w.trajectories * e2e_steps * world / el
    b.close()
    return res


def precision_leg(qn, args, stream, local, roof_of):
    """The precision workload (n=26, p=4, depolarizing only, 64 trajectories of 512 MiB):
    fused layers (FP32 on the CUDA cores, 4 sweeps per layer at n=26, and the tensor cores
    in TF32 and BF16x3, ceil(n/5) sweeps per layer) against one sweep per gate on the same
    trajectories --
    throughput, the sweeps' HBM fraction, and each form's <C> beside the ensemble's
    statistical error (the comparison "at equal <C> error")."""
    w = W.precision_n26()
    legs = {}
    sub = argparse.Namespace(steps=max(2, min(args.steps, 3)), warmup=3)
    for name, mode, prec in (("fused", (False, True), 0), ("tensor_tf32", (False, True), 1),
                             ("tensor_bf16x3", (False, True), 2), ("per_gate", (False, False), 0)):
        res = measure(qn, w, sub, mode, stream, 0, 1, local, None, with_e2e=False, precision=prec)
        kname = ("k_tc_sweep (tensor-core windows of 5 qubits, 16 B per amplitude)" if prec else
                 "k_fused_tile12 / k_fused_win / k_fused_sweep (fused layer sweeps)") if mode[1] else \
            "k_sweep_zz / k_sweep_rx (gate sweeps)"
        r = roof_of(res, kname, "sweeps")
        legs[name] = {"value": res["value"], "unit": UNIT, "ms_per_step": res["ms"] / sub.steps,
                      "c_mean": res["mean"], "c_stderr": res["se"], "sweep_bytes_per_step": res["sweep_bytes_per_step"],
                      "roofline": {k: r[k] for k in ("kernel", "achieved", "peak", "unit", "frac", "avg_launch_ms")},
                      "clocks": res["clocks"]}
    for name in ("fused", "tensor_tf32", "tensor_bf16x3"):
        legs[name]["speedup_over_per_gate"] = legs[name]["value"] / legs["per_gate"]["value"]
        legs[name]["c_difference_to_per_gate"] = abs(legs[name]["c_mean"] - legs["per_gate"]["c_mean"])
    legs["config"] = config_of(w, {"steps": sub.steps, "warmup": sub.warmup})
    return legs


def hbm_peak_of():
    """The measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs, GB/s), else the fallback."""
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk_path)) if os.path.exists(pk_path) else {}
    return float(peaks.get("hbm_gbs", 6800.0)), ("measured" if "hbm_gbs" in peaks else "fallback")


def fused_window_count(n: int) -> int:
    """Sweeps per layer of the fused forward layers (the library's fused_windows: the window
    of qubits 0-11 where it saves a sweep, else 0-7, then windows of at most 7; five per
    window below 10 qubits)."""
    if n < 10:
        return -(-n // 5)
    return 1 + min(-(-(n - 8) // 7), -(-(n - 12) // 7) if n > 12 else n)


def adjoint_window_count(n: int) -> int:
    """Sweeps per layer of the fused adjoint (the library's adj_tile_windows for n >= 12:
    qubits 0-9, then windows of at most six, the cost diagonal in the last one's sweep;
    adj_windows below: qubits 0-3, then windows of two or three, plus the phase sweep)."""
    if n >= 12:
        return 1 + -(-(n - 10) // 6)
    rest = n - min(4, n)
    return 2 + (-(-rest // 3) if rest > 0 else 0)


def gradient_leg(qn, args, stream, local):
    """The gradient workload (n=16, p=6, depolarizing only, K=2048): one step is the noisy
    forward run of the whole ensemble plus the adjoint gradient of <C> in all 12 angles
    (qn_run_qaoa + qn_grad), timed with CUDA events on the library's stream."""
    import torch

    w = W.gradient_n16()
    steps, warmup = max(2, min(args.steps, 3)), 3
    b = qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch, stream=stream)
    kw = w.noise_kwargs()

    def step():
        b.run_qaoa(w.edges, w.gammas, w.betas, **kw)
        return b.grad()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        ev0.record(stream)
        for _ in range(steps):
            dg, db = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    mean, se = b.expectation()
    b.close()
    # bytes of one step: the fused forward sweeps (16 B per amplitude), the sigma pass (8 B), the
    # adjoint's start (read psi, write lambda: 16 B) and its sweeps (psi and lambda: 32 B), each
    # layer's mixer windows and its cost diagonal
    amps = float(w.trajectories) * (1 << w.n)
    step_bytes = amps * (16.0 * fused_window_count(w.n) * w.p + 8.0 + 16.0 +
                         32.0 * adjoint_window_count(w.n) * w.p)
    peak, peak_src = hbm_peak_of()
    achieved = step_bytes / (ms / steps / 1e3) / 1e9
    return {"value": w.trajectories * steps / (ms / 1e3), "unit": "trajectories/s (forward + adjoint gradient)",
            "ms_per_step": ms / steps, "c_mean": mean, "c_stderr": se,
            "step_roofline": {"bound": "hbm", "bytes_per_step": step_bytes, "achieved": achieved, "peak": peak,
                              "unit": "GB/s", "frac": achieved / peak,
                              "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)"},
            "dC_dgamma": [float(x) for x in dg], "dC_dbeta": [float(x) for x in db], "clocks": clocks.summary(),
            "config": config_of(w, {"steps": steps, "warmup": warmup,
                                    "step": "qn_run_qaoa (fused layers) + qn_grad (fused adjoint: a layer's mixer "
                                            "reversed in tiles of psi and lambda through shared memory, qubits 0-9 "
                                            "then windows of up to 6, the cost diagonal in the last window's sweep)"})}


def gpu_arm(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn

    w = workload(args.workload)
    hbm_peak, peak_src = hbm_peak_of()
    stream = torch.cuda.current_stream()

    _, main_mode, other_mode = WORKLOADS[args.workload]
    if not args.sharing:
        main_mode = (False, main_mode[1])
    if not args.fusion:
        main_mode = (main_mode[0], False)
    sharing = main_mode[0] and w.damping > 0
    main = measure(qn, w, args, main_mode, stream, rank, world, local, pg, with_e2e=True, precision=args.precision)
    other = None
    if not args.single_mode and other_mode != main_mode:
        other = measure(qn, w, args, other_mode, stream, rank, world, local, pg, with_e2e=False)
    # the same step with device-driven launches, and as a replayed CUDA graph
    modes = {}
    if main_mode[0] and not args.single_mode and args.launch_mode == 0:
        for lm in (1, 2):
            a2 = argparse.Namespace(**{**vars(args), "launch_mode": lm})
            modes[lm] = measure(qn, w, a2, main_mode, stream, rank, world, local, pg, with_e2e=(lm == 2))

    G, n, K = w.gate_count, w.n, w.trajectories
    h2d = int(len(w.edges) * 8 + 2 * w.p * 8 + 40 + G * 20)
    d2h = int((1 << n) * 8 + 16 + 4)
    if sharing:
        # grouping of the noisy H layer into the first slots, per-gate live-slot
        # counts, and the slot order for the final accumulation
        d2h += K * (n + 32 + 4 + 8 * n) + 4 * (G - n) + 4 + K * 12
        h2d += K * (4 + 8 + 32 + 8 * n + 12) + 16

    def roof(res, kernel, family="sweeps"):
        sw = res[family]
        avg_ms = sw["ms"] / max(sw["launches"], 1)
        achieved = (sw["bytes"] / max(sw["launches"], 1)) / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else 0.0
        traffic = None
        tr_path = os.path.join(ROOT, "profiles", "k_sweep_n20_damping_traffic.json")
        if os.path.exists(tr_path):
            try:
                tj = json.load(open(tr_path))
                entry = tj.get("kernels", {}).get(kernel.split(" ")[0])
                if entry and tj.get("kernel_source_hash") == kernel_hash():
                    states_per_launch = (sw["bytes"] / max(sw["launches"], 1)) / (16.0 * (1 << w.n))
                    traffic = entry["traffic_bytes_per_state"] * states_per_launch
            except (ValueError, OSError, KeyError):
                traffic = None
        return {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "launches_timed": sw["launches"], "avg_launch_ms": avg_ms,
                "share_of_step": sw["ms"] * PROFILE_PERIOD / res["ms"] if res["ms"] > 0 else None}

    if rank == 0:
        fused = main_mode[1] and w.damping == 0
        grouped = sharing and main_mode[1] and main["groups"]["launches"] > 0
        blocks = grouped and main["mixers"]["launches"] > 0
        kname = "k_mix_sweep (mixer blocks over live prefix states: the factors of block 0-7 with the rotations of 8-11, the rotations of 12-15 with the factors of block 8-15, then 4 qubits per sweep; 16 B per amplitude)" if blocks else \
            "k_slot_sweep (mixer gate sweeps over live prefix states)" if grouped else \
            "k_slot_sweep (gate sweeps over live prefix states)" if sharing else \
            (("k_tc_sweep (tensor-core windows of 5 qubits, %s, 16 B per amplitude)" %
              ("TF32" if args.precision == 1 else "BF16x3") if args.precision and w.n >= 11 else
              "k_fused_tile12 / k_fused_win / k_fused_sweep (fused layer sweeps, 16 B per amplitude)") if fused else
             "k_sweep_zz / k_sweep_rx (gate sweeps, 16 B per amplitude)")
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "tf32 (f32 accumulate)", 2: "bf16x3 (f32 accumulate)"}[args.precision if fused else 0],
            "data": "synthetic",
            "config": config_of(w, {
                "parallelism": f"trajectory shards x{world}" if world > 1 else "single GPU",
                "mode": ("shared-prefix: one statevector per distinct Kraus prefix, all trajectories in one "
                         "prefix tree" + ("; phase gates applied in groups on <= 10 qubits, one sweep per group, "
                                          "and each layer's mixer rotations in blocks: qubits 0-7 and 8-15 drawn as "
                                          "8-qubit blocks over two sweeps each, then 4 qubits per sweep" if grouped
                                          else "; one sweep per gate")
                         + ("; launches sized on the host from the live-slot count" if args.launch_mode == 0 else
                            "; device-driven persistent launches" + (" replayed as a CUDA graph"
                                                                      if args.launch_mode == 2 else ""))) if sharing else
                        (f"fused layers: qubits 0-11 (one shared-memory tile) or 0-7, then windows of <= 7 qubits, "
                         f"one sweep each per QAOA layer, "
                         f"{w.batch} trajectories per launch" if fused
                         else f"one statevector per trajectory, one sweep per gate, {w.batch} per launch")}),
            "amp_updates_per_s": main["value"] * G * (1 << n),
            "distinct_states_per_step": main["states_per_step"],
            "sweep_bytes_per_step": main["sweep_bytes_per_step"],
            "c_mean": main["mean"], "c_stderr": main["se"],
            "roofline": roof(main, kname, "mixers" if blocks else "sweeps"),
            "kernels": {"gate sweeps (sampled 1/%d)" % PROFILE_PERIOD: main["sweeps"],
                        "phase-group sweeps (sampled 1/%d)" % PROFILE_PERIOD: main["groups"],
                        "mixer-block sweeps (sampled 1/%d)" % PROFILE_PERIOD: main["mixers"],
                        "k_init": main["inits"], "observables (k_observe, k_probs or k_probs_mix)": main["accs"]},
            "e2e": {"value": main["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": main["launches"],
            "clocks": main["clocks"],
        }
        if grouped:
            line["roofline_phase_groups"] = roof(main, "k_group_apply + k_group_mix + k_group_hist (phase-group "
                                                       "sweeps, 16 B and 8 B per amplitude)", "groups")
        if other is not None:
            key = "per_trajectory_mode" if sharing else "per_gate_mode"
            line[key] = {
                "value": other["value"], "unit": UNIT, "ms_per_step": other["ms"] / args.steps,
                "c_mean": other["mean"], "gpu_launches": other["launches"], "clocks": other["clocks"],
                "sweep_bytes_per_step": other["sweep_bytes_per_step"],
                "roofline": roof(other, "k_sweep_zz / k_sweep_rx (gate sweeps, 16 B per amplitude)")}
        if modes:
            line["launch_modes"] = {
                {1: "device_driven", 2: "cuda_graph"}[lm]: {
                    "value": r["value"], "unit": UNIT, "ms_per_step": r["ms"] / args.steps, "c_mean": r["mean"],
                    "clocks": r["clocks"], **({"e2e": r["e2e_value"]} if "e2e_value" in r else {}),
                    "launches": ("persistent sweeps over the slots the device counts; the host reads nothing "
                                 "until the step is over" if lm == 1 else
                                 "the same launches captured once in a CUDA graph, replayed every step")}
                for lm, r in modes.items()}
        if world == 1 and not args.no_cpu_baseline and w.n <= 20:
            line["cpu_baseline"] = cpu_baseline(w)
        if world == 1 and args.workload == "damping20" and not args.no_legs:
            line["precision26"] = precision_leg(qn, args, stream, local, roof_of=roof)
            line["gradient16"] = gradient_leg(qn, args, stream, local)
            line["serving"] = serving_levels(args.requests, args.inflight, local)
            line["serving_host_launches"] = serving_levels(args.requests, args.inflight, local, policy="host",
                                                           levels=(0.8,))
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def serving_levels(requests: int, inflight: int, clock_index: int = 0, policy: str = "auto",
                   levels=(0.5, 0.8)):
    """Serving workload: closed-loop capacity, then Poisson arrivals at the given fractions
    of it; per level the request count, span, throughput and p50/p99 latency."""
    from paper_2210_15874_gb300 import serving

    reqs = serving.serving_mix(requests)
    warm = serving.serving_mix(4, seed=99)
    srv = serving.Server(max_inflight=inflight, launch_policy=policy)
    for f in [srv.submit(r) for r in warm]:
        f.result()

    def run(rate):
        rng = np.random.default_rng(7)
        t0 = time.perf_counter()
        futs = []
        for r in reqs:
            if rate:
                time.sleep(float(rng.exponential(1.0 / rate)))
            futs.append(srv.submit(r))
        res = [f.result() for f in futs]
        span = time.perf_counter() - t0
        lat = [x.latency for x in res]
        traj = sum(r.trajectories for r in reqs)
        return {"requests": len(reqs), "seconds": span, "requests_per_s": len(reqs) / span,
                "trajectories_per_s": traj / span, "p50_latency_s": serving.percentile(lat, 50),
                "p99_latency_s": serving.percentile(lat, 99), "mean_latency_s": float(np.mean(lat))}

    out = {}
    with ClockSampler(clock_index) as clocks:
        cap = run(0)
        out["capacity"] = cap
        for f in levels:
            out[f"load_{f}"] = run(f * cap["requests_per_s"])
    srv.close()
    launches = {"auto": "device-driven launches (persistent sweeps reading the live-slot count on the device); "
                        "a request that runs in several launch batches captures its first in a CUDA graph and "
                        "replays it",
                "host": "launches sized on the host from the live-slot count read after every decide",
                "device": "device-driven launches", "graph": "device-driven launches captured in CUDA graphs"}
    cfg = {"workload": "serving: n ~ U{10..24}, p ~ U{1..6}, K ~ log-uniform[256, 8192], depolarizing "
                       "1e-3/1e-2 + damping 5e-3, seeded regular graphs",
           "requests": requests, "max_inflight": inflight,
           "admission": "HBM footprint (launch batch of statevectors + tables) within 60% of free memory",
           "mode": "shared-prefix mode per request, one CUDA stream per in-flight request",
           "launch_policy": policy, "launches": launches[policy]}
    out.update({"clocks": clocks.summary(), "config": cfg})
    return out


def serving_arm(args):
    """--workload serving: the serving levels as their own JSON line."""
    import torch

    from paper_2210_15874_gb300 import build
    build.build()

    torch.cuda.set_device(0)
    sv = serving_levels(args.requests, args.inflight, policy=args.serving_policy)
    line = {"metric": "noisy trajectories/s and p50/p99 request latency under Poisson load", "value":
            sv["load_0.8"]["trajectories_per_s"], "unit": "trajectories/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "config": sv["config"],
            "capacity": sv["capacity"], "load_0.5": sv["load_0.5"], "load_0.8": sv["load_0.8"],
            "clocks": sv["clocks"]}
    print(json.dumps(line), flush=True)


def profile_case(sharing=False, depth=1, fusion=True, precision=-1, launch_mode=0, grad=False):
    """Small case of the bench's kernels for ncu (inputs larger than L2, 256 MiB of state);
    depth 2 adds a layer, so the last mixer block of the first one forms the next layer's joint.
    precision 0, 1 or 2: the precision workload's fused layers in FP32 or on the tensor cores
    (n=24, p=depth, depolarizing only, 8 states of 128 MiB; with depth 2 the first layer's last
    window also applies the second layer's phase).  grad: the gradient workload's circuit
    (n=16, p=depth, depolarizing only) for 512 trajectories in one launch batch (256 MiB of
    states and 256 MiB of adjoint states): the fused forward run and the fused adjoint."""
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn

    if grad:
        w = W.qaoa_workload(f"ncu_n16_p{depth}_grad", 16, depth, index=4, trajectories=512, batch=512)
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            dg, db = b.grad()
            print(json.dumps({"case": w.name, "c": b.expectation(), "dC_dgamma": [float(x) for x in dg],
                              "dC_dbeta": [float(x) for x in db]}))
        return
    if precision >= 0:
        w = W.qaoa_workload(f"ncu_n24_p{depth}_tc", 24, depth, index=2, trajectories=8, batch=8)
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
            b.set_fusion(True)
            b.set_precision(precision)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            print(json.dumps({"case": w.name, "precision": precision, "c": b.expectation()}))
        return
    if sharing:
        # heavy Pauli noise so that most of the 64 trajectories fork early: the
        # late gates sweep ~64 live states (512 MiB, above L2)
        w = W.qaoa_workload(f"ncu_n20_p{depth}_damp_shared", 20, depth, index=1, trajectories=64, batch=64, p1=0.1,
                            p2=0.3, damping=5e-3)
    else:
        w = W.qaoa_workload(f"ncu_n20_p{depth}_damp", 20, depth, index=1, trajectories=32, batch=32, damping=5e-3)
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
        b.set_sharing(sharing)
        b.set_fusion(fusion)
        b.set_launch_mode(launch_mode)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        print(json.dumps({"case": w.name, "c": b.expectation(), "states": b.run_info()["states"]}))


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    for fn in ("qn_kernels.cu", "qn_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2210_15874_gb300", "csrc", fn), "rb").read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gq", choices=["gq", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=40, help="serving workload: requests per load level")
    ap.add_argument("--inflight", type=int, default=4, help="serving workload: concurrent requests")
    ap.add_argument("--workload", default="damping20", choices=sorted(WORKLOADS) + ["serving"],
                    help="damping20 (default, the headline), precision26 / precision30 (Pauli-only, fused layers "
                         "vs one sweep per gate), gradient16, plain8")
    ap.add_argument("--sharing", type=int, default=1, choices=[0, 1],
                    help="1: shared-prefix mode (trajectories share common Kraus prefixes); "
                         "0: every trajectory evolved separately, 64 per launch")
    ap.add_argument("--fusion", type=int, default=1, choices=[0, 1],
                    help="1: fused sweeps (phase groups and mixer blocks with damping, fused layers without); "
                         "0: one sweep per gate")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="arithmetic of the fused layers of Pauli-only workloads: 0 FP32 (default), 1 TF32 or "
                         "2 BF16x3 tensor cores")
    ap.add_argument("--serving-policy", default="auto", choices=["auto", "host", "device", "graph"],
                    help="serving workload: launch policy of the requests")
    ap.add_argument("--launch-mode", type=int, default=0, choices=[0, 1, 2],
                    help="shared-prefix launches sized on the host (0), on the device (1), or the run as a "
                         "CUDA graph (2)")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the precision (n=26), gradient (n=16) and serving legs of the default line")
    ap.add_argument("--single-mode", action="store_true",
                    help="time only the selected mode (skip the per-trajectory comparison run)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one small ensemble for ncu captures, then exit (n=20, p=1: 32 trajectories in "
                         "one launch, or with --sharing 1 64 heavily noisy trajectories)")
    ap.add_argument("--profile-depth", type=int, default=1, choices=[1, 2], help="QAOA depth of --profile-case")
    ap.add_argument("--profile-grad", action="store_true",
                    help="--profile-case: the gradient workload's circuit, forward run and fused adjoint")
    ap.add_argument("--profile-precision", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="--profile-case of the Pauli-only fused layers (0 FP32, 1 TF32, 2 BF16x3 tensor cores) "
                         "instead of the damping case")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(bool(args.sharing), args.profile_depth, bool(args.fusion), args.profile_precision,
                     args.launch_mode, args.profile_grad)
        return
    if args.workload == "serving":
        serving_arm(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
