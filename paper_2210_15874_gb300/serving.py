"""Continuous batching of noisy-QAOA requests on one GPU.

A request is one ensemble (graph, depth, angles, noise, K trajectories, seed).
The server admits requests in arrival order as soon as (a) a worker slot is
free and (b) the request's HBM footprint -- 2^n x 8 B x its launch batch of
statevectors plus its tables -- fits in the memory budget next to the requests
already running; a request that does not fit waits while later, smaller ones
may pass it (a bounded look-ahead).  Every admitted request runs on its own
CUDA stream from its own worker thread, so requests that arrive while others
are on the GPU start at once and their kernels overlap on the device.  Device
memory comes from the PyTorch caching allocator, so finishing a request frees
nothing device-wide (no cudaFree synchronisation).

Launches (qn_batch_set_launch_mode, shared-prefix requests).  A small request
(up to AUTO_DEVICE_QUBITS qubits) is launch-bound: under the default policy
"auto" it runs device-driven -- persistent sweeps that read the live-slot count
on the device, so its worker never waits on the GPU between groups of gates --
and, when it runs in more than one launch batch (chunk), its first chunk is
captured in a CUDA graph that the later chunks replay.  A larger request is
bound by HBM, where host-sized grids sweep a few percent faster than
persistent ones, so it runs with launches sized on the host (a read of the
live count after each decide).  "host", "device" and "graph" force modes 0, 1
and 2 for every request.

All arithmetic runs in libqnoise's kernels; this module only schedules.  A
request's result does not depend on what runs beside it, nor on the launch
policy: its launch batch size is a function of the request alone, every draw
is keyed by (seed, trajectory id), and every launch mode gives bit-identical
results.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import qn

STATE_BUDGET_BYTES = 8 << 30  # statevectors per launch batch (one prefix tree) of one request
# The largest request the "auto" launch policy runs device-driven (measured on GB300: at
# 10-12 qubits device-driven runs are 3-10% faster, at 14 qubits even, beyond slower).
AUTO_DEVICE_QUBITS = 12


@dataclasses.dataclass
class Request:
    n: int
    edges: np.ndarray
    gammas: np.ndarray
    betas: np.ndarray
    trajectories: int
    seed: int
    p1: float = 1e-3
    p2: float = 1e-2
    damping: float = 0.0
    want_probs: bool = False

    def launch_batch(self) -> int:
        return int(max(1, min(self.trajectories, STATE_BUDGET_BYTES // (8 << self.n))))

    def chunks(self) -> int:
        """Launch batches (prefix trees) the request runs in, one after the other."""
        return -(-self.trajectories // self.launch_batch())

    def footprint(self) -> int:
        """HBM bytes the request holds while it runs: its launch batch of complex64
        statevectors plus per-trajectory tables and the sigma accumulator."""
        B = self.launch_batch()
        G = self.n + len(self.gammas) * (len(self.edges) + self.n)
        return B * (8 << self.n) + B * (G * 13 + 64) + (16 << self.n) + self.trajectories * 8 + (1 << 20)


@dataclasses.dataclass
class Result:
    mean: float
    std_err: float
    probs: np.ndarray | None
    submitted: float
    started: float
    finished: float
    # the request's span on the device: CUDA events on its stream at its first and after its
    # last launch, in ms after the server's reference event (None outside a Server)
    device_start: float | None = None
    device_end: float | None = None
    # the launch mode the request ran in, and its graph use (qn_graph_info)
    launch: dict | None = None

    @property
    def latency(self) -> float:
        return self.finished - self.submitted


LAUNCH_POLICIES = ("auto", "host", "device", "graph")


def launch_mode_for(req: Request, policy: str = "auto") -> int:
    """qn_batch_set_launch_mode value of a request under a launch policy."""
    if policy not in LAUNCH_POLICIES:
        raise ValueError(f"launch policy {policy!r} not in {LAUNCH_POLICIES}")
    if policy == "auto":
        if req.n > AUTO_DEVICE_QUBITS:
            return 0
        return 2 if req.chunks() > 1 else 1
    return {"host": 0, "device": 1, "graph": 2}[policy]


class Server:
    """Admit-and-run loop.  `max_inflight` worker threads (one CUDA stream each),
    a device memory budget in bytes and a launch policy (LAUNCH_POLICIES)."""

    def __init__(self, max_inflight: int = 4, mem_budget: int | None = None, lookahead: int = 8,
                 launch_policy: str = "auto"):
        import torch

        launch_mode_for(Request(1, np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), 1, 0), launch_policy)
        self.launch_policy = launch_policy
        self._torch = torch
        self.device = torch.cuda.current_device()
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info()
            mem_budget = int(free * 0.6)
        self.mem_budget = mem_budget
        self.max_inflight = max_inflight
        self.lookahead = lookahead
        self._lock = threading.Condition()
        self._pending: collections.deque = collections.deque()
        self._inflight = 0
        self._mem_used = 0
        self._stop = False
        self._streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        self._ref = torch.cuda.Event(enable_timing=True)  # origin of the requests' device spans
        self._ref.record()
        self._ref.synchronize()
        self._free_streams = list(range(max_inflight))
        self._threads = []
        # one entry per admission: (time, requests in flight, footprint bytes held), after admitting
        self.admissions: list[tuple[float, int, int]] = []
        self._dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self._dispatcher.start()

    # -- public ---------------------------------------------------------------
    def submit(self, req: Request) -> Future:
        if req.footprint() > self.mem_budget:
            raise ValueError(f"request needs {req.footprint()} bytes, above the budget {self.mem_budget}")
        fut: Future = Future()
        with self._lock:
            self._pending.append((req, fut, time.perf_counter()))
            self._lock.notify_all()
        return fut

    def close(self) -> None:
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._dispatcher.join()
        for t in self._threads:
            t.join()

    # -- scheduling -------------------------------------------------------------
    def _pick(self):
        """First pending request (within the look-ahead) that fits now."""
        for i, (req, fut, ts) in enumerate(self._pending):
            if i >= self.lookahead:
                break
            if self._mem_used + req.footprint() <= self.mem_budget:
                del self._pending[i]
                return req, fut, ts
        return None

    def _dispatch(self):
        while True:
            with self._lock:
                item = None
                while item is None:
                    if self._inflight < self.max_inflight and self._pending:
                        item = self._pick()
                        if item is not None:
                            break
                    if self._stop and not self._pending:
                        return
                    self._lock.wait(0.05)
                req, fut, ts = item
                self._inflight += 1
                self._mem_used += req.footprint()
                self.admissions.append((time.perf_counter(), self._inflight, self._mem_used))
                si = self._free_streams.pop()
            th = threading.Thread(target=self._run, args=(req, fut, ts, si), daemon=True)
            self._threads.append(th)
            th.start()

    def _run(self, req: Request, fut: Future, submitted: float, si: int):
        torch = self._torch
        try:
            torch.cuda.set_device(self.device)
            stream = self._streams[si]
            started = time.perf_counter()
            ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev_a.record(stream)
            with qn.Batch(req.n, req.trajectories, req.seed, launch_batch=req.launch_batch(), stream=stream,
                          torch_allocator=True) as b:
                b.set_sharing(req.damping > 0)
                mode = launch_mode_for(req, self.launch_policy)
                b.set_launch_mode(mode)
                b.run_qaoa(req.edges, req.gammas, req.betas, p1=req.p1, p2=req.p2, damping=req.damping)
                mean, se = b.expectation()
                probs = b.probs() if req.want_probs else None
                ev_b.record(stream)
                ev_b.synchronize()
                launch = dict(mode=mode, **b.graph_info())
            fut.set_result(Result(mean, se, probs, submitted, started, time.perf_counter(),
                                  self._ref.elapsed_time(ev_a), self._ref.elapsed_time(ev_b), launch))
        except Exception as exc:  # delivered to the caller through the future
            fut.set_exception(exc)
        finally:
            with self._lock:
                self._inflight -= 1
                self._mem_used -= req.footprint()
                self._free_streams.append(si)
                self._lock.notify_all()


def run_alone(req: Request, launch_policy: str = "host") -> Result:
    """The same request on its own (a fresh handle on the default stream)."""
    t0 = time.perf_counter()
    with qn.Batch(req.n, req.trajectories, req.seed, launch_batch=req.launch_batch()) as b:
        b.set_sharing(req.damping > 0)
        b.set_launch_mode(launch_mode_for(req, launch_policy))
        b.run_qaoa(req.edges, req.gammas, req.betas, p1=req.p1, p2=req.p2, damping=req.damping)
        mean, se = b.expectation()
        probs = b.probs() if req.want_probs else None
    t1 = time.perf_counter()
    return Result(mean, se, probs, t0, t0, t1)


def serving_mix(count: int, seed: int = 2213):
    """The serving workload: n ~ U{10..24}, p ~ U{1..6}, K ~ floor(exp(U[ln 256, ln 8192])),
    depolarizing p1=1e-3 / p2=1e-2 plus damping 5e-3, seeded regular graphs (3-regular for
    even n, 4-regular for odd n, which has no 3-regular graph), seeded angles."""
    from . import workloads as W

    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.integers(10, 25))
        p = int(rng.integers(1, 7))
        K = int(np.floor(np.exp(rng.uniform(np.log(256), np.log(8192)))))
        g, b = W.angles(p, seed * 1000 + i)
        d = 3 if n % 2 == 0 else 4
        reqs.append(Request(n, W.regular_graph(n, d, seed * 1000 + n), g, b, K,
                            W.PHILOX_SEED_BASE + 3000 + i, damping=5e-3))
    return reqs


def percentile(values, q):
    return float(np.percentile(np.asarray(values), q)) if len(values) else float("nan")
