"""CPU oracle for NI-SB multi-objective MaxCut (test infrastructure only).

Thin ctypes wrapper over ``moq_oracle.c``: plain double-precision dynamics, int64 cut
values and exact __int128 hypervolumes, written from the paper and sharing no code
with the CUDA library. Only the tests, the smoke check and the benchmark's CPU
baseline call it; the product path never does.

Parity status: every function is pinned by tests under ``tests/`` against what the
paper and the mathematics fix (see the header of ``moq_oracle.c``); the Gaussian noise
is pinned by its moments only (not bitwise), and SB trajectories beyond a few steps
are compared by distribution only, being chaotic.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmoq_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE arithmetic: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32p, i64p, u64p, dp = (np.ctypeslib.ndpointer(t, flags="C_CONTIGUOUS")
                                    for t in (np.int32, np.int64, np.uint64, np.float64))
            vp = C.c_void_p
            lib.or_philox4x32_10.argtypes = [np.ctypeslib.ndpointer(np.uint32), np.ctypeslib.ndpointer(np.uint32),
                                             np.ctypeslib.ndpointer(np.uint32)]
            lib.or_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]
            lib.or_normal.restype = C.c_double
            lib.or_normal_fill.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int64, dp]
            lib.or_initial_state.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_float,
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.or_cuts.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, i32p, i32p, C.c_int64, u64p, i64p]
            lib.or_energies.argtypes = lib.or_cuts.argtypes
            lib.or_brute_force.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, i32p, i32p, u64p, i64p]
            lib.or_dominates.argtypes = [C.c_int, i64p, i64p]
            lib.or_dominates.restype = C.c_int
            lib.or_pareto_filter.argtypes = [C.c_int, C.c_int64, i64p, i64p]
            lib.or_pareto_filter.restype = C.c_int64
            lib.or_hypervolume.argtypes = [C.c_int, C.c_int64, i64p, i64p, i64p]
            lib.or_das_dennis.argtypes = [C.c_int, C.c_int, C.c_int, vp]
            lib.or_das_dennis.restype = C.c_int64
            lib.or_dirichlet.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint64, dp]
            lib.or_sb.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, i32p, i32p, C.c_int, dp,
                                  C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_float, vp, C.c_int,
                                  C.c_uint64, C.c_uint64, vp, vp, u64p, vp, vp, vp]
            lib.or_sb.restype = C.c_int
            lib.or_reference_point.argtypes = [C.c_int, C.c_int64, i32p, i64p]
            lib.or_mlp_param_count.argtypes = [C.c_int, C.c_int, C.c_int]
            lib.or_mlp_param_count.restype = C.c_int64
            lib.or_mlp_forward.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_int64, dp, dp]
            lib.or_mlp_loss_grad.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_int64, dp, dp, dp]
            lib.or_mlp_loss_grad.restype = C.c_double
            lib.or_bf16.argtypes = [C.c_double]
            lib.or_bf16.restype = C.c_double
            lib.or_mlp_forward_bf16.argtypes = lib.or_mlp_forward.argtypes
            lib.or_mlp_loss_grad_bf16.argtypes = lib.or_mlp_loss_grad.argtypes
            lib.or_mlp_loss_grad_bf16.restype = C.c_double
            lib.or_e4m3.argtypes = [C.c_double]
            lib.or_e4m3.restype = C.c_double
            lib.or_e4m3_couplings.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, i32p, i32p, dp, dp, dp]
            lib.or_force_e4m3.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, i32p, dp, dp, C.c_int, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _inst_arrays(inst):
    return (np.ascontiguousarray(inst.ei, np.int32), np.ascontiguousarray(inst.ej, np.int32),
            np.ascontiguousarray(inst.w, np.int32))


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def normal(seed: int, round_: int, r: int, i: int, m: int) -> float:
    return _load().or_normal(seed, round_, r, i, m)


def normals(seed: int, round_: int, r: int, i: int, m0: int, count: int) -> np.ndarray:
    """The noise draws of steps m0 .. m0 + count - 1 of one spin and replica."""
    out = np.zeros(count, np.float64)
    _load().or_normal_fill(seed, round_, r, i, m0, count, out)
    return out


def initial_state(seed: int, round_: int, r: int, i: int, amp: float = 0.1):
    x, y = C.c_double(), C.c_double()
    _load().or_initial_state(seed, round_, r, i, amp, C.byref(x), C.byref(y))
    return x.value, y.value


def cuts(inst, bits: np.ndarray) -> np.ndarray:
    """Cut vectors C(s) (M, K) int64 of packed spin configurations (M, W) uint64."""
    ei, ej, w = _inst_arrays(inst)
    bits = np.ascontiguousarray(bits, np.uint64)
    M = bits.shape[0]
    out = np.zeros((M, inst.K), np.int64)
    _load().or_cuts(inst.n, inst.K, inst.E, ei, ej, w, M, bits, out)
    return out


def energies(inst, bits: np.ndarray) -> np.ndarray:
    ei, ej, w = _inst_arrays(inst)
    bits = np.ascontiguousarray(bits, np.uint64)
    out = np.zeros((bits.shape[0], inst.K), np.int64)
    _load().or_energies(inst.n, inst.K, inst.E, ei, ej, w, bits.shape[0], bits, out)
    return out


def brute_force(inst):
    """All 2^(n-1) configurations with s_0 = +1: (bits (2^(n-1), W), cuts (2^(n-1), K))."""
    if inst.n > 26:
        raise ValueError("brute force limited to n <= 26")
    ei, ej, w = _inst_arrays(inst)
    cnt = 1 << (inst.n - 1)
    W = (inst.n + 63) // 64
    bits = np.zeros((cnt, W), np.uint64)
    cut = np.zeros((cnt, inst.K), np.int64)
    _load().or_brute_force(inst.n, inst.K, inst.E, ei, ej, w, bits, cut)
    return bits, cut


def dominates(u, v) -> bool:
    u = np.ascontiguousarray(u, np.int64)
    return bool(_load().or_dominates(u.size, u, np.ascontiguousarray(v, np.int64)))


def pareto_filter(cuts_: np.ndarray) -> np.ndarray:
    """Pool indices (ascending) of the distinct non-dominated cut vectors."""
    cuts_ = np.ascontiguousarray(cuts_, np.int64)
    M, K = cuts_.shape
    keep = np.zeros(max(M, 1), np.int64)
    F = _load().or_pareto_filter(K, M, cuts_, keep)
    return keep[:F].copy()


def hypervolume(points: np.ndarray, ref) -> int:
    """Exact hypervolume (python int) of the union of boxes [ref, p]."""
    pts = np.ascontiguousarray(points, np.int64).reshape(-1, len(ref))
    ref = np.ascontiguousarray(ref, np.int64)
    out = np.zeros(2, np.int64)
    _load().or_hypervolume(ref.size, pts.shape[0], pts, ref, out)
    lo, hi = int(out[0]) & ((1 << 64) - 1), int(out[1])
    return (hi << 64) | lo


def das_dennis(K: int, H: int, interior: bool = True) -> np.ndarray:
    lib = _load()
    cnt = lib.or_das_dennis(K, H, int(interior), None)
    out = np.zeros((cnt, K), np.float64)
    lib.or_das_dennis(K, H, int(interior), out.ctypes.data_as(C.c_void_p))
    return out


def dirichlet(R: int, K: int, seed: int, round_: int = 0) -> np.ndarray:
    out = np.zeros((R, K), np.float64)
    _load().or_dirichlet(R, K, seed, round_, out)
    return out


def reference_point(inst) -> np.ndarray:
    out = np.zeros(inst.K, np.int64)
    _load().or_reference_point(inst.K, inst.E, np.ascontiguousarray(inst.w, np.int32), out)
    return out


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def sb(inst, lam, *, variant: str = "dsb", steps: int = 1000, dt: float = 0.5, a0: float = 1.0,
       alpha: float = 0.0, init_amp: float = 0.1, schedule=None, noise_sqrt_dt: bool = False,
       seed: int = 0, round_: int = 0, x_init=None, y_init=None):
    """Run R NI-SB replicas in double precision. Returns dict(bits, x, y, c0)."""
    ei, ej, w = _inst_arrays(inst)
    lam = np.ascontiguousarray(np.asarray(lam, np.float64).reshape(-1, inst.K))
    R, n = lam.shape[0], inst.n
    W = (n + 63) // 64
    bits = np.zeros((R, W), np.uint64)
    x = np.zeros((R, n), np.float64)
    y = np.zeros((R, n), np.float64)
    c0 = np.zeros(R, np.float64)
    sched = None if schedule is None else np.ascontiguousarray(schedule, np.float64)
    if sched is not None and sched.size != steps:
        raise ValueError("schedule must have one entry per step")
    xi = None if x_init is None else np.ascontiguousarray(np.asarray(x_init, np.float64).reshape(R, n))
    yi = None if y_init is None else np.ascontiguousarray(np.asarray(y_init, np.float64).reshape(R, n))
    _load().or_sb(n, inst.K, inst.E, ei, ej, w, R, lam, 0 if variant == "dsb" else 1, steps, dt, a0, alpha,
                  init_amp, _ptr(sched), int(noise_sqrt_dt), seed, round_, _ptr(xi), _ptr(yi), bits,
                  _ptr(x), _ptr(y), _ptr(c0))
    return {"bits": bits, "x": x, "y": y, "c0": c0}


def mlp_param_count(din: int, h: int, dout: int) -> int:
    return int(_load().or_mlp_param_count(din, h, dout))


def mlp_forward(params, X, din: int, h: int, dout: int) -> np.ndarray:
    """Surrogate MLP forward in double precision: (B, din) -> (B, dout)."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, din))
    Y = np.zeros((X.shape[0], dout), np.float64)
    _load().or_mlp_forward(din, h, dout, np.ascontiguousarray(params, np.float64), X.shape[0], X, Y)
    return Y


def mlp_loss_grad(params, X, T, din: int, h: int, dout: int):
    """Mean squared error and its gradient with respect to the flat parameter vector."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, din))
    T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(-1, dout))
    g = np.zeros(mlp_param_count(din, h, dout), np.float64)
    loss = _load().or_mlp_loss_grad(din, h, dout, np.ascontiguousarray(params, np.float64), X.shape[0], X, T, g)
    return loss, g


def bf16(v: float) -> float:
    """v rounded to the nearest BF16 value (ties to an even significand)."""
    return float(_load().or_bf16(float(v)))


def mlp_forward_bf16(params, X, din: int, h: int, dout: int) -> np.ndarray:
    """The network with every matrix-product operand rounded to BF16 (exact sums)."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, din))
    Y = np.zeros((X.shape[0], dout), np.float64)
    _load().or_mlp_forward_bf16(din, h, dout, np.ascontiguousarray(params, np.float64), X.shape[0], X, Y)
    return Y


def mlp_loss_grad_bf16(params, X, T, din: int, h: int, dout: int):
    """Loss and gradient with BF16 matrix-product operands (exact sums, exact bias gradients)."""
    X = np.ascontiguousarray(np.asarray(X, np.float64).reshape(-1, din))
    T = np.ascontiguousarray(np.asarray(T, np.float64).reshape(-1, dout))
    g = np.zeros(mlp_param_count(din, h, dout), np.float64)
    loss = _load().or_mlp_loss_grad_bf16(din, h, dout, np.ascontiguousarray(params, np.float64), X.shape[0], X, T, g)
    return loss, g


def e4m3(values) -> np.ndarray:
    """Nearest E4M3 value of each input (ties to an even mantissa, saturating at +-448)."""
    v = np.asarray(values, np.float64)
    lib = _load()
    return np.array([lib.or_e4m3(float(a)) for a in v.ravel()]).reshape(v.shape)


def e4m3_couplings(inst):
    """Couplings of the FP8 force: (wq_i, wq_j, scale): the value of each edge's weight as
    seen from row ei and from row ej (K x E each) and the power-of-two row scales (K x n)."""
    ei, ej, w = _inst_arrays(inst)
    K, E = w.shape
    wq_i = np.zeros((K, E)); wq_j = np.zeros((K, E)); sc = np.zeros((K, inst.n))
    _load().or_e4m3_couplings(inst.n, K, E, ei, ej, w, wq_i, wq_j, sc)
    return wq_i, wq_j, sc


def force_e4m3(inst, lam, phi, c0) -> np.ndarray:
    """One-step SB force c0 sum_j (-J(c)_ij) phi_j with the FP8 couplings (R x n)."""
    ei, ej, _ = _inst_arrays(inst)
    wq_i, wq_j, _ = e4m3_couplings(inst)
    lam = np.ascontiguousarray(np.asarray(lam, np.float64).reshape(-1, inst.K))
    phi = np.ascontiguousarray(np.asarray(phi, np.float64))
    c0 = np.ascontiguousarray(np.asarray(c0, np.float64))
    f = np.zeros_like(phi)
    _load().or_force_e4m3(inst.n, inst.K, wq_i.shape[1], ei, ej, wq_i, wq_j, lam.shape[0], lam, c0, phi, f)
    return f
