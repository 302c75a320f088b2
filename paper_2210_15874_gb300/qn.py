"""Thin ctypes binding of libqnoise (include/qn.h): argument marshalling only.

Every entry point keeps its C name (qn_batch_create, qn_run_qaoa, ...).  The
binding does no arithmetic of the method; all of it runs in the library's CUDA
kernels.  Importing this module loads libqnoise.so and raises ImportError when
the library has not been built -- there is no CPU fallback.

``Batch`` is a small convenience wrapper over one handle.  PyTorch is used only
to hand the library a CUDA stream and, optionally, its caching allocator.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libqnoise.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with `python -m paper_2210_15874_gb300.build` "
                      "(or __graft_entry__.build()); there is no CPU fallback")
_lib = ctypes.CDLL(_LIB_PATH)

QN_OK, QN_EINVAL, QN_ENOMEM, QN_ECUDA, QN_ETIMEOUT, QN_ESTATE = range(6)
_STATUS = {0: "QN_OK", 1: "QN_EINVAL", 2: "QN_ENOMEM", 3: "QN_ECUDA", 4: "QN_ETIMEOUT", 5: "QN_ESTATE"}

P = ctypes.POINTER
c_i32, c_i64, c_u64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class qn_graph(ctypes.Structure):
    _fields_ = [("n", c_i32), ("num_edges", c_i32), ("edges", P(c_i32))]


class qn_noise(ctypes.Structure):
    _fields_ = [("p1", c_dbl), ("p2", c_dbl), ("damping", c_dbl), ("twoq_mode", c_i32), ("param", c_i32)]


ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp)

_SIGS = {
    "qn_batch_create": (c_i32, [c_i32, c_i64, c_u64, P(c_vp)]),
    "qn_batch_set_stream": (c_i32, [c_vp, c_vp]),
    "qn_batch_set_allocator": (c_i32, [c_vp, ALLOC_FN, FREE_FN, c_vp]),
    "qn_batch_set_launch_batch": (c_i32, [c_vp, c_i64]),
    "qn_batch_set_offset": (c_i32, [c_vp, c_i64]),
    "qn_batch_set_sharing": (c_i32, [c_vp, c_i32]),
    "qn_batch_set_fusion": (c_i32, [c_vp, c_i32]),
    "qn_batch_set_precision": (c_i32, [c_vp, c_i32]),
    "qn_batch_set_launch_mode": (c_i32, [c_vp, c_i32]),
    "qn_graph_info": (c_i32, [c_vp, P(c_i64), P(c_i64), P(c_i64)]),
    "qn_run_qaoa": (c_i32, [c_vp, P(qn_graph), c_i32, P(c_dbl), P(c_dbl), P(qn_noise)]),
    "qn_expectation": (c_i32, [c_vp, P(c_dbl), P(c_dbl)]),
    "qn_probs": (c_i32, [c_vp, P(c_dbl), c_i64]),
    "qn_grad": (c_i32, [c_vp, P(c_dbl), P(c_dbl)]),
    "qn_grad_traj": (c_i32, [c_vp, c_i64, c_i64, P(c_dbl), P(c_dbl)]),
    "qn_traj_debug": (c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "qn_shared_readout": (c_i32, [c_vp, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "qn_fidelity_error": (c_i32, [P(c_dbl), P(c_dbl), c_i64, P(c_dbl)]),
    "qn_run_info": (c_i32, [c_vp, P(c_i64), P(c_i64), P(c_dbl), P(c_i64)]),
    "qn_batch_set_profiling": (c_i32, [c_vp, c_i32]),
    "qn_profile_read": (c_i32, [c_vp, c_i32, P(c_i64), P(c_dbl), P(c_dbl)]),
    "qn_run_qaoa_noalloc": (c_i32, [c_i32, P(qn_graph), c_i32, P(c_dbl), P(c_dbl), P(qn_noise), c_u64, c_i64,
                                    c_i32, c_vp, c_vp, c_vp, c_vp]),
    "qn_group_plan": (c_i32, [c_i32, P(qn_graph), c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, P(c_i32)]),
    "qn_mix_tile_map": (c_i32, [c_i32, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, P(c_i32)]),
    "qn_fused_windows": (c_i32, [c_i32, c_i32, c_i32, c_vp, c_vp, P(c_i32)]),
    "qn_last_error": (ctypes.c_char_p, []),
    "qn_batch_destroy": (None, [c_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

LIBRARY_PATH = _LIB_PATH
EXPORTED = tuple(_SIGS)


class QnError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = qn_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != QN_OK:
        raise QnError(status, where)


def _dptr(a):
    return a.ctypes.data_as(P(c_dbl))


def _vp(a):
    return ctypes.c_void_p(a.ctypes.data)


class Batch:
    """One qn_batch handle: n qubits, `trajectories` ensemble members, Philox `seed`."""

    def __init__(self, n: int, trajectories: int, seed: int, *, launch_batch: int = 0, stream=None,
                 torch_allocator: bool = False):
        h = c_vp()
        check(qn_batch_create(int(n), int(trajectories), c_u64(int(seed) & (2 ** 64 - 1)), ctypes.byref(h)),
              "qn_batch_create")
        self._h = h
        self.n, self.trajectories, self.seed = int(n), int(trajectories), int(seed)
        self.p = 0
        self.generation = 0  # number of qn_run_qaoa calls made on this handle
        self._keep = []
        if launch_batch:
            check(qn_batch_set_launch_batch(h, int(launch_batch)), "qn_batch_set_launch_batch")
        self._stream = stream
        if stream is not None:
            self.set_stream(stream)
        if torch_allocator:
            self._use_torch_allocator()

    # -- configuration ------------------------------------------------------
    def set_stream(self, stream) -> None:
        """Queue work on `stream` (a torch.cuda.Stream or a raw cudaStream_t int)."""
        raw = getattr(stream, "cuda_stream", stream)
        check(qn_batch_set_stream(self._h, c_vp(int(raw) if raw else None)), "qn_batch_set_stream")

    def _use_torch_allocator(self) -> None:
        import torch

        dev = torch.cuda.current_device()

        stream = self._stream if isinstance(getattr(self, "_stream", None), torch.cuda.Stream) else None

        def _alloc(size, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(size), dev, stream)
            except Exception:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        a, f = ALLOC_FN(_alloc), FREE_FN(_free)
        self._keep += [a, f]
        check(qn_batch_set_allocator(self._h, a, f, None), "qn_batch_set_allocator")

    def set_fusion(self, on: bool) -> None:
        """Fused layers for Pauli-only noise (default on)."""
        check(qn_batch_set_fusion(self._h, int(bool(on))), "qn_batch_set_fusion")

    def set_precision(self, mode) -> None:
        """Arithmetic of the fused layers: 0 / "fp32" (CUDA cores), 1 / "tf32" or 2 / "bf16x3"
        (tensor cores, five qubits per sweep)."""
        m = {"fp32": 0, "tf32": 1, "bf16x3": 2}.get(mode, mode)
        check(qn_batch_set_precision(self._h, int(m)), "qn_batch_set_precision")

    def set_sharing(self, on: bool) -> None:
        """Shared-prefix mode: trajectories share their common Kraus prefix."""
        check(qn_batch_set_sharing(self._h, int(bool(on))), "qn_batch_set_sharing")

    def set_launch_mode(self, mode) -> None:
        """How shared-prefix launches are sized: 0 / "host" (from the live-slot count read
        after every decide), 1 / "device" (persistent launches that read it on the device),
        2 / "graph" (as 1, the run captured in a CUDA graph and replayed)."""
        m = {"host": 0, "device": 1, "graph": 2}.get(mode, mode)
        check(qn_batch_set_launch_mode(self._h, int(m)), "qn_batch_set_launch_mode")

    def graph_info(self) -> dict:
        c, r, u = c_i64(), c_i64(), c_i64()
        check(qn_graph_info(self._h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(u)), "qn_graph_info")
        return dict(captures=c.value, replays=r.value, updates=u.value)

    def set_offset(self, first_trajectory: int) -> None:
        """Global id of this handle's first trajectory (shards of one ensemble)."""
        check(qn_batch_set_offset(self._h, int(first_trajectory)), "qn_batch_set_offset")

    def set_profiling(self, period: int) -> None:
        """Time every `period`-th sweep launch with CUDA events (0 = off)."""
        check(qn_batch_set_profiling(self._h, int(period)), "qn_batch_set_profiling")

    # -- the method ---------------------------------------------------------
    def run_qaoa(self, edges, gammas, betas, *, p1=0.0, p2=0.0, damping=0.0, twoq_mode=0, param=0) -> None:
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        b = np.ascontiguousarray(betas, dtype=np.float64)
        if len(g) != len(b):
            raise ValueError("gammas and betas differ in length")
        graph = qn_graph(self.n, len(e) // 2, e.ctypes.data_as(P(c_i32)))
        noise = qn_noise(float(p1), float(p2), float(damping), int(twoq_mode), int(param))
        self.p = len(g)
        self.generation += 1
        check(qn_run_qaoa(self._h, ctypes.byref(graph), len(g), _dptr(g), _dptr(b), ctypes.byref(noise)),
              "qn_run_qaoa")

    def expectation(self) -> tuple[float, float]:
        m, s = c_dbl(), c_dbl()
        check(qn_expectation(self._h, ctypes.byref(m), ctypes.byref(s)), "qn_expectation")
        return m.value, s.value

    def probs(self, out: np.ndarray | None = None) -> np.ndarray:
        """sigma, the ensemble's output distribution (2^n float64), into `out` if given: a
        caller that reads it every step can pass the same (e.g. page-locked) buffer each time."""
        if out is None:
            out = np.empty(1 << self.n, dtype=np.float64)
        elif out.dtype != np.float64 or out.size != (1 << self.n) or not out.flags.c_contiguous or not out.flags.writeable:
            raise ValueError(f"out must be a writable contiguous float64 array of 2^n = {1 << self.n} elements")
        check(qn_probs(self._h, _dptr(out), out.size), "qn_probs")
        return out

    def grad(self) -> tuple[np.ndarray, np.ndarray]:
        dg = np.zeros(max(self.p, 1), dtype=np.float64)
        db = np.zeros(max(self.p, 1), dtype=np.float64)
        check(qn_grad(self._h, _dptr(dg), _dptr(db)), "qn_grad")
        return dg[:self.p], db[:self.p]

    def grad_traj(self, t0: int, count: int) -> tuple[np.ndarray, np.ndarray]:
        dg = np.zeros((max(count, 1), max(self.p, 1)), dtype=np.float64)
        db = np.zeros_like(dg)
        check(qn_grad_traj(self._h, int(t0), int(count), _dptr(dg), _dptr(db)), "qn_grad_traj")
        return dg[:count, :self.p], db[:count, :self.p]

    def traj_debug(self, t0: int, count: int, *, amps=True, branches=True, c=True):
        dim = 1 << self.n
        info = self.run_info()
        a = np.zeros((count, dim, 2), dtype=np.float32) if amps else None
        br = np.zeros((count, max(info["gates"], 1)), dtype=np.uint8) if branches else None
        cc = np.zeros(max(count, 1), dtype=np.float64) if c else None
        vp = lambda x: None if x is None else c_vp(x.ctypes.data)
        check(qn_traj_debug(self._h, int(t0), int(count), vp(a), vp(br), vp(cc)), "qn_traj_debug")
        return dict(amps=None if a is None else a.view(np.complex64)[..., 0],
                    branches=None if br is None else br[:, :info["gates"]],
                    c_traj=None if cc is None else cc[:count])

    def shared_readout(self, t0: int, count: int, *, amps=True, branches=True, c=True):
        """The last shared-prefix run's own per-trajectory results (no re-simulation):
        final states, the Kraus strings that run drew, and <C>_t."""
        dim = 1 << self.n
        info = self.run_info()
        a = np.zeros((count, dim, 2), dtype=np.float32) if amps else None
        br = np.zeros((count, max(info["gates"], 1)), dtype=np.uint8) if branches else None
        cc = np.zeros(max(count, 1), dtype=np.float64) if c else None
        vp = lambda x: None if x is None else c_vp(x.ctypes.data)
        check(qn_shared_readout(self._h, int(t0), int(count), vp(a), vp(br), vp(cc)), "qn_shared_readout")
        return dict(amps=None if a is None else a.view(np.complex64)[..., 0],
                    branches=None if br is None else br[:, :info["gates"]],
                    c_traj=None if cc is None else cc[:count])

    def run_info(self) -> dict:
        g, l, b, st = c_i64(), c_i64(), c_dbl(), c_i64()
        check(qn_run_info(self._h, ctypes.byref(g), ctypes.byref(l), ctypes.byref(b), ctypes.byref(st)),
              "qn_run_info")
        return dict(gates=g.value, launches=l.value, sweep_bytes=b.value, states=st.value)

    def profile_read(self, kind: int) -> dict:
        l, ms, b = c_i64(), c_dbl(), c_dbl()
        check(qn_profile_read(self._h, int(kind), ctypes.byref(l), ctypes.byref(ms), ctypes.byref(b)),
              "qn_profile_read")
        return dict(launches=l.value, ms=ms.value, bytes=b.value)

    # -- lifetime -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None):
            qn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fidelity_error(sa, se) -> float:
    """Error = 1 - (sum sqrt(sa se))^2 (Eq. 1), computed by the library's host code."""
    a = np.ascontiguousarray(sa, dtype=np.float64)
    b = np.ascontiguousarray(se, dtype=np.float64)
    out = c_dbl()
    check(qn_fidelity_error(_dptr(a), _dptr(b), len(a), ctypes.byref(out)), "qn_fidelity_error")
    return out.value


def group_plan(n: int, edges, p: int) -> list:
    """The gate groups of shared-prefix mode with damping and fusion (host only):
    a list of dicts kind (0 phase gates, 1 mixer rotations), first_gate, gates, qubits."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = qn_graph(n, len(e) // 2, e.ctypes.data_as(P(c_i32)))
    cnt = c_i32()
    check(qn_group_plan(n, ctypes.byref(g), p, 0, None, None, None, None, ctypes.byref(cnt)), "qn_group_plan")
    k = np.zeros(cnt.value, dtype=np.int32)
    f = np.zeros(cnt.value, dtype=np.int32)
    m = np.zeros(cnt.value, dtype=np.int32)
    q = np.zeros(cnt.value, dtype=np.uint32)
    if cnt.value:
        check(qn_group_plan(n, ctypes.byref(g), p, cnt.value, _vp(k), _vp(f), _vp(m), _vp(q),
                            ctypes.byref(cnt)), "qn_group_plan")
    return [dict(kind=int(k[i]), first_gate=int(f[i]), gates=int(m[i]),
                 qubits=[b for b in range(n) if (int(q[i]) >> b) & 1]) for i in range(cnt.value)]


def fused_windows(n: int, reverse: bool = False) -> list:
    """The fused layers' window schedule (host only): (first qubit, qubits) per sweep of one
    layer, forward or, with reverse, the fused adjoint's mixer windows."""
    cnt = c_i32()
    check(qn_fused_windows(n, int(reverse), 0, None, None, ctypes.byref(cnt)), "qn_fused_windows")
    lo = np.zeros(cnt.value, dtype=np.int32)
    m = np.zeros(cnt.value, dtype=np.int32)
    if cnt.value:
        check(qn_fused_windows(n, int(reverse), cnt.value, _vp(lo), _vp(m), ctypes.byref(cnt)), "qn_fused_windows")
    return [(int(lo[i]), int(m[i])) for i in range(cnt.value)]


def mix_tile_map(n: int, q_lo: int, m: int, m_next: int) -> dict:
    """Float4-index bits of a mixer-block sweep's tile (host only): lane, a, b, tile."""
    lane = np.zeros(3, dtype=np.int8)
    a = np.zeros(4, dtype=np.int8)
    b = np.zeros(4, dtype=np.int8)
    t = np.zeros(32, dtype=np.int8)
    nt = c_i32()
    check(qn_mix_tile_map(n, q_lo, m, m_next, _vp(lane), _vp(a), _vp(b), _vp(t), ctypes.byref(nt)),
          "qn_mix_tile_map")
    return dict(lane=lane.tolist(), a=a.tolist(), b=b.tolist(), tile=t[:nt.value].tolist())
