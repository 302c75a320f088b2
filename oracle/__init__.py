"""FP64 CPU oracle for stochastic noisy-QAOA ensembles -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
library never loads it, and it shares no code with the CUDA path: the C file
``qn_oracle.c`` restates the paper's definitions on its own.

Functions follow arXiv 2210.15874:
  * ``dm_run``      -- O1, exact noisy density matrix; channels as the operator
                       sum of Eq. op_sum with the depolarizing Kraus set of Sec.
                       "Modeling Noise" and the amplitude-damping Kraus pair.
  * ``traj_run``    -- O2, the stochastic ensemble of Sec. "Stochastic Noise
                       Implementation": per gate, one uniform number per channel
                       picks a Kraus operator; phi = |psi|^2, sigma = sum phi / K.
  * ``error``       -- Error = 1 - (sum sqrt(sa * se))^2 (Eq. 1).
  * ``philox4x32_10`` -- the counter-based generator both sides draw from.

Parity status of every function is pinned by tests/test_oracle_*.py; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

H, ZZ, RX = 0, 1, 2


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("angle", ctypes.c_double)]


class Noise(ctypes.Structure):
    _fields_ = [("p1", ctypes.c_double), ("p2", ctypes.c_double), ("damping", ctypes.c_double),
                ("twoq_mode", ctypes.c_int32), ("param", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile qn_oracle.c into liborc.so next to it (gcc, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_qaoa_gate_count.restype = ctypes.c_int32
        L.orc_qaoa_gate_count.argtypes = [ctypes.c_int32] * 3
        L.orc_qaoa_gates.restype = ctypes.c_int32
        L.orc_qaoa_gates.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), ctypes.c_int32,
                                     P(ctypes.c_double), P(ctypes.c_double), P(Gate)]
        L.orc_pauli_probs.restype = ctypes.c_int32
        L.orc_pauli_probs.argtypes = [P(Noise), ctypes.c_int32, P(ctypes.c_double)]
        L.orc_thresholds.argtypes = [P(ctypes.c_double), ctypes.c_int32, P(ctypes.c_uint64)]
        L.orc_traj_run.restype = ctypes.c_int32
        L.orc_traj_run.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(Gate), ctypes.c_int32,
                                   P(Noise), ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int32]
        L.orc_traj_forced.restype = ctypes.c_int32
        L.orc_traj_forced.argtypes = [ctypes.c_int32, P(Gate), ctypes.c_int32, P(Noise), ctypes.c_void_p,
                                      ctypes.c_void_p, P(ctypes.c_double)]
        L.orc_dm_apply_1q.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        L.orc_dm_depolarize_1q.restype = ctypes.c_int32
        L.orc_dm_depolarize_1q.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, P(Noise)]
        L.orc_dm_depolarize_2q.restype = ctypes.c_int32
        L.orc_dm_depolarize_2q.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           P(Noise)]
        L.orc_dm_damp.restype = ctypes.c_int32
        L.orc_dm_damp.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double]
        L.orc_dm_gate.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(Gate)]
        L.orc_dm_run.restype = ctypes.c_int32
        L.orc_dm_run.argtypes = [ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32), P(Gate), ctypes.c_int32,
                                 P(Noise), ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_double)]
        L.orc_error.restype = ctypes.c_double
        L.orc_error.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int64]
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_noise(p1=0.0, p2=0.0, damping=0.0, twoq_mode=0, param=0) -> Noise:
    return Noise(float(p1), float(p2), float(damping), int(twoq_mode), int(param))


def philox4x32_10(counter, key) -> np.ndarray:
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def qaoa_gates(n, edges, gammas, betas):
    """Gate list of the QAOA MaxCut circuit (H layer, then p x (ZZ per edge, RX per qubit))."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    b = np.ascontiguousarray(betas, dtype=np.float64)
    p = len(g)
    G = lib().orc_qaoa_gate_count(n, len(e) // 2, p)
    gates = (Gate * max(G, 1))()
    lib().orc_qaoa_gates(n, len(e) // 2, _ptr(e, ctypes.c_int32), p, _ptr(g, ctypes.c_double),
                         _ptr(b, ctypes.c_double), gates)
    return gates, G


def gate_array(gate_list):
    """Build a ctypes gate array from tuples (kind, q0, q1, angle)."""
    arr = (Gate * max(len(gate_list), 1))()
    for i, (k, a, b, ang) in enumerate(gate_list):
        arr[i] = Gate(k, a, b, ang)
    return arr, len(gate_list)


def pauli_probs(noise: Noise, two_qubit: bool) -> np.ndarray:
    out = np.zeros(16, dtype=np.float64)
    k = lib().orc_pauli_probs(ctypes.byref(noise), int(bool(two_qubit)), _ptr(out, ctypes.c_double))
    return out[:k].copy()


def thresholds(probs) -> np.ndarray:
    p = np.ascontiguousarray(probs, dtype=np.float64)
    out = np.zeros(len(p), dtype=np.uint64)
    lib().orc_thresholds(_ptr(p, ctypes.c_double), len(p), _ptr(out, ctypes.c_uint64))
    return out


def traj_run(n, edges, gates, G, noise: Noise, seed: int, t0: int, count: int, *, want_amps=True,
             want_branches=True, threads=0):
    """O2 over trajectories t0..t0+count-1.

    Returns dict(amps [count, 2^n] complex128 | None, branches [count, G] uint8 | None,
    c_traj [count], probs_sum [2^n] (sum over the trajectories of |psi|^2), s1, s2).
    """
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    dim = 1 << n
    amps = np.zeros((count, dim), dtype=np.complex128) if want_amps else None
    br = np.zeros((count, max(G, 1)), dtype=np.uint8) if want_branches else None
    ct = np.zeros(max(count, 1), dtype=np.float64)
    probs = np.zeros(dim, dtype=np.float64)
    sums = np.zeros(2, dtype=np.float64)
    rc = lib().orc_traj_run(n, len(e) // 2, _ptr(e, ctypes.c_int32), gates, G, ctypes.byref(noise),
                            ctypes.c_uint64(seed), t0, count, _vp(amps), _vp(br), _vp(ct), _vp(probs),
                            _vp(sums), threads)
    if rc != 0:
        raise MemoryError("oracle traj_run failed")
    return dict(amps=amps, branches=None if br is None else br[:, :G], c_traj=ct[:count],
                probs_sum=probs, s1=float(sums[0]), s2=float(sums[1]))


def traj_forced(n, gates, G, noise: Noise, branch_bytes):
    """One trajectory along a forced Kraus string; returns (psi, Born weight) or (None, 0.0)."""
    fb = np.ascontiguousarray(branch_bytes, dtype=np.uint8)
    psi = np.zeros(1 << n, dtype=np.complex128)
    w = ctypes.c_double(0.0)
    rc = lib().orc_traj_forced(n, gates, G, ctypes.byref(noise), _vp(fb), _vp(psi), ctypes.byref(w))
    if rc != 0:
        return None, 0.0
    return psi, float(w.value)


def dm_run(n, edges, gates, G, noise: Noise, want_rho=False):
    """O1.  Returns dict(rho [2^n,2^n] | None, diag [2^n], c)."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    dim = 1 << n
    rho = np.zeros((dim, dim), dtype=np.complex128) if want_rho else None
    diag = np.zeros(dim, dtype=np.float64)
    c = ctypes.c_double(0.0)
    rc = lib().orc_dm_run(n, len(e) // 2, _ptr(e, ctypes.c_int32), gates, G, ctypes.byref(noise), _vp(rho),
                          _vp(diag), ctypes.byref(c))
    if rc != 0:
        raise MemoryError("oracle dm_run failed")
    return dict(rho=rho, diag=diag, c=float(c.value))


def dm_apply_1q(rho, n, q, m):
    m = np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(4))
    lib().orc_dm_apply_1q(_vp(rho), n, q, _vp(m))


def dm_depolarize_1q(rho, n, q, noise):
    assert lib().orc_dm_depolarize_1q(_vp(rho), n, q, ctypes.byref(noise)) == 0


def dm_depolarize_2q(rho, n, q0, q1, noise):
    assert lib().orc_dm_depolarize_2q(_vp(rho), n, q0, q1, ctypes.byref(noise)) == 0


def dm_damp(rho, n, q, gamma):
    assert lib().orc_dm_damp(_vp(rho), n, q, float(gamma)) == 0


def dm_gate(rho, n, kind, q0, q1=-1, angle=0.0):
    g = Gate(kind, q0, q1, float(angle))
    lib().orc_dm_gate(_vp(rho), n, ctypes.byref(g))


def error(sa, se) -> float:
    """Error = 1 - F(sa, se) = 1 - (sum_x sqrt(sa_x se_x))^2  (Eq. 1)."""
    a = np.ascontiguousarray(sa, dtype=np.float64)
    b = np.ascontiguousarray(se, dtype=np.float64)
    return float(lib().orc_error(_ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), len(a)))


def cut_values(n, edges) -> np.ndarray:
    """C(x) for every basis index x (number of cut edges)."""
    x = np.arange(1 << n, dtype=np.int64)
    c = np.zeros(1 << n, dtype=np.float64)
    for i, j in np.asarray(edges, dtype=np.int64).reshape(-1, 2):
        c += ((x >> i) ^ (x >> j)) & 1
    return c
