"""Python binding of the ``libmoqaia.so`` C ABI (``include/moqaia.h``).

Argument marshalling only: every function forwards to the C entry point of the same
name. Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed), host
buffers are numpy arrays, and ``stream`` defaults to torch's current CUDA stream.
Failures raise ``MoqError`` carrying the library's status code and message. Importing
this module without the built library raises ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoqaia.so")

MOQ_OK = 0
MOQ_ERR_ARG = -1
MOQ_ERR_OOM = -2
MOQ_ERR_CUDA = -3
MOQ_ERR_TIMEOUT = -4
MOQ_ERR_CAPACITY = -5
MOQ_ERR_OVERFLOW = -6
MOQ_ERR_UNSUPPORTED = -7
MOQ_DSB = 0
MOQ_BSB = 1
MOQ_LAYOUT_PLAIN = -1
MOQ_LAYOUT_DEFAULT = 0
MOQ_PREC_FP32 = 0
MOQ_PREC_FP16 = 1
MOQ_MLP_CUDA_CORES = 0
MOQ_MLP_TENSOR_CORES = 1


class MoqError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where} failed with {code}: {message}")
        self.code = code


class moq_instance_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("K", C.c_int32), ("E", C.c_int64), ("max_degree", C.c_int32),
                ("words", C.c_int32), ("weight_sum", C.c_int64 * 8), ("abs_sum", C.c_int64 * 8),
                ("ref_point", C.c_int64 * 8), ("features", C.c_float * 8)]


class moq_sample_params(C.Structure):
    _fields_ = [("variant", C.c_int32), ("steps", C.c_int32), ("dt", C.c_float), ("a0", C.c_float),
                ("alpha", C.c_float), ("init_amp", C.c_float), ("noise_sqrt_dt", C.c_int32),
                ("schedule", C.c_void_p), ("x_init", C.c_void_p), ("y_init", C.c_void_p),
                ("x_out", C.c_void_p), ("y_out", C.c_void_p), ("replica_offset", C.c_uint32), ("precision", C.c_int32)]


class moq_hv(C.Structure):
    _fields_ = [("lo", C.c_int64), ("hi", C.c_int64), ("approx", C.c_double)]

    def value(self) -> int:
        return (int(self.hi) << 64) | (int(self.lo) & ((1 << 64) - 1))


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python paper_2604_26477_b300/build.py` (needs nvcc)")
_lib = C.CDLL(LIB_PATH)

_vp, _i32, _i64, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
_sigs = {
    "moq_default_params": (None, [C.POINTER(moq_sample_params)]),
    "moq_create_instance": (C.c_int, [_i32, _i32, _i64, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "moq_create_instance_layout": (C.c_int, [_i32, _i32, _i64, _vp, _vp, _vp, _i32, _vp, C.POINTER(_vp)]),
    "moq_create_instance_dense": (C.c_int, [_i32, _i32, _vp, _vp, C.POINTER(_vp)]),
    "moq_plan_gather_layout": (C.c_int, [_i32, _i64, _vp, _vp, _vp, _vp, _vp]),
    "moq_destroy_instance": (None, [_vp]),
    "moq_instance_get_info": (C.c_int, [_vp, C.POINTER(moq_instance_info)]),
    "moq_sample": (C.c_int, [_vp, _vp, _i32, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_evaluate_cuts": (C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "moq_archive_create": (C.c_int, [_i32, _i32, _i64, _i64, C.POINTER(_vp)]),
    "moq_archive_destroy": (None, [_vp]),
    "moq_archive_reset": (C.c_int, [_vp, _vp]),
    "moq_pareto_front": (C.c_int, [_vp, _vp, _vp, _i64, _i64, C.POINTER(_i64), _vp]),
    "moq_archive_merge": (C.c_int, [_vp, _vp, _vp]),
    "moq_archive_size": (C.c_int, [_vp, C.POINTER(_i64), _vp]),
    "moq_archive_copy_out": (C.c_int, [_vp, _vp, _vp, _vp, _i64, C.POINTER(_i64), _vp]),
    "moq_archive_device_view": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
    "moq_hypervolume": (C.c_int, [_vp, _vp, C.POINTER(moq_hv), _vp]),
    "moq_hypervolume_many": (C.c_int, [C.POINTER(_vp), _vp, _i32, C.POINTER(moq_hv), _vp]),
    "moq_hypervolume_workspace_size": (_i64, [_i64, _i32]),
    "moq_hypervolume_points": (C.c_int, [_vp, _i64, _i32, _vp, _vp, C.POINTER(moq_hv), _vp]),
    "moq_hypervolume_noalloc_max_points": (_i64, []),
    "moq_hypervolume_points_noalloc": (C.c_int, [_vp, _i64, _i32, _vp, C.POINTER(moq_hv), _vp]),
    "moq_lambda_das_dennis": (C.c_int, [_i32, _i32, _i32, _vp, _i64, C.POINTER(_i64), _vp]),
    "moq_lambda_dirichlet": (C.c_int, [_i32, _i32, _u64, _u64, _vp, _vp]),
    "moq_batch_create": (C.c_int, [_vp, _i32, _vp, C.POINTER(_vp)]),
    "moq_batch_destroy": (None, [_vp]),
    "moq_batch_layout": (C.c_int, [_vp, _vp, _vp]),
    "moq_batch_set_tiles": (C.c_int, [_vp, _i32, _i32, C.POINTER(_i32)]),
    "moq_batch_set_replicas": (C.c_int, [_vp, _vp]),
    "moq_sample_batch": (C.c_int, [_vp, _vp, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_evaluate_cuts_batch": (C.c_int, [_vp, _vp, _vp, _vp]),
    "moq_dense_create": (C.c_int, [_vp, _i32, C.POINTER(_vp)]),
    "moq_dense_destroy": (None, [_vp]),
    "moq_sample_dense": (C.c_int, [_vp, _vp, _i32, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_dense_status": (C.c_int, [_vp, _vp]),
    "moq_dense_evaluate_cuts": (C.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "moq_sample_dense_fp8": (C.c_int, [_vp, _vp, _i32, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_sample_dense_split": (C.c_int, [_vp, _vp, _i32, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_dense_fp32_create": (C.c_int, [_vp, _i32, C.POINTER(_vp)]),
    "moq_dense_fp32_destroy": (None, [_vp]),
    "moq_sample_dense_fp32": (C.c_int, [_vp, _vp, _i32, C.POINTER(moq_sample_params), _u64, _u64, _vp, _vp]),
    "moq_mlp_create": (C.c_int, [_i32, _i32, _i32, _i32, _u64, C.POINTER(_vp)]),
    "moq_mlp_destroy": (None, [_vp]),
    "moq_mlp_param_count": (_i64, [_vp]),
    "moq_mlp_set_params": (C.c_int, [_vp, _vp]),
    "moq_mlp_get_params": (C.c_int, [_vp, _vp, _i32]),
    "moq_mlp_forward": (C.c_int, [_vp, _vp, _i32, _vp, _vp]),
    "moq_mlp_gradient": (C.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "moq_mlp_adam_step": (C.c_int, [_vp, C.c_float, _vp]),
    "moq_mlp_train_step": (C.c_int, [_vp, _vp, _vp, _i32, C.c_float, _vp, _vp]),
    "moq_mlp_set_engine": (C.c_int, [_vp, _i32]),
    "moq_mlp_status": (C.c_int, [_vp, _vp]),
    "moq_lambda_propose": (C.c_int, [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _u64, _u64, _vp, _i32, _vp]),
    "moq_mlp_make_rows": (C.c_int, [_i32, _i32, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "moq_release_cached_memory": (C.c_int, []),
    "moq_strerror": (C.c_char_p, [C.c_int]),
    "moq_last_error_message": (C.c_char_p, []),
    "moq_last_status": (C.c_int, []),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


def moq_last_status() -> int:
    """Code of the last failed call on this thread (MOQ_OK before any failure)."""
    return int(_lib.moq_last_status())


def _check(rc: int, where: str):
    if rc != MOQ_OK:
        raise MoqError(rc, where, _lib.moq_last_error_message().decode(errors="replace"))


def _stream(stream):
    if stream is not None:  # a torch.cuda.Stream or a raw cudaStream_t value
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, name, dtypes=None, numel=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtypes is not None and t.dtype not in dtypes:
        raise TypeError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _torch_types():
    import torch
    f32 = (torch.float32,)
    i64 = (torch.int64,)
    u64 = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
    return f32, i64, u64


# ---------------------------------------------------------------------------- C ABI
def moq_strerror(code: int) -> str:
    return _lib.moq_strerror(code).decode()


def moq_last_error_message() -> str:
    return _lib.moq_last_error_message().decode(errors="replace")


def moq_default_params(**overrides) -> moq_sample_params:
    p = moq_sample_params()
    _lib.moq_default_params(C.byref(p))
    p._tensors = {}  # keeps the tensors behind the optional device pointers alive
    for k, v in overrides.items():
        if k == "variant" and isinstance(v, str):
            v = {"dsb": MOQ_DSB, "bsb": MOQ_BSB}[v.lower()]
        if k == "precision" and isinstance(v, str):
            v = {"fp32": MOQ_PREC_FP32, "fp16": MOQ_PREC_FP16}[v.lower()]
        if k in ("schedule", "x_init", "y_init", "x_out", "y_out"):
            p._tensors[k] = v
            v = None if v is None else _dptr(v, k, _torch_types()[0])
        setattr(p, k, v)
    return p


def moq_create_instance(n, K, E, ei, ej, w, stream=None, layout=None) -> C.c_void_p:
    """``layout=None``: ``moq_create_instance`` (layout from the environment); else
    ``moq_create_instance_layout`` with MOQ_LAYOUT_PLAIN, MOQ_LAYOUT_DEFAULT or an effort m > 0."""
    ei_, pei = _hptr(ei, np.int32)
    ej_, pej = _hptr(ej, np.int32)
    w_, pw = _hptr(w, np.int32)
    if ei_.size != E or ej_.size != E or w_.size != K * E:
        raise ValueError("edge arrays must have E entries and w K*E")
    h = C.c_void_p()
    if layout is None:
        _check(_lib.moq_create_instance(n, K, E, pei, pej, pw, _stream(stream), C.byref(h)), "moq_create_instance")
    else:
        _check(_lib.moq_create_instance_layout(n, K, E, pei, pej, pw, int(layout), _stream(stream), C.byref(h)),
               "moq_create_instance_layout")
    return h


def moq_create_instance_dense(n, K, J_upper, stream=None) -> C.c_void_p:
    J_, pj = _hptr(J_upper, np.int32)
    if J_.size != K * n * (n - 1) // 2:
        raise ValueError("J_upper must hold K * n(n-1)/2 weights")
    h = C.c_void_p()
    _check(_lib.moq_create_instance_dense(n, K, pj, _stream(stream), C.byref(h)), "moq_create_instance_dense")
    return h


def moq_plan_gather_layout(n, ei, ej):
    """Host-only: (slot_spin[n], gather[2E], passes[4]) as moq_create_instance lays the graph out."""
    ei_, pei = _hptr(ei, np.int32)
    ej_, pej = _hptr(ej, np.int32)
    if ei_.size != ej_.size:
        raise ValueError("ei and ej must have the same length")
    slot = np.zeros(n, np.int32)
    gather = np.zeros(2 * ei_.size, np.int32)
    passes = np.zeros(4, np.int64)
    _check(_lib.moq_plan_gather_layout(n, ei_.size, pei, pej, slot.ctypes.data_as(_vp), gather.ctypes.data_as(_vp),
                                       passes.ctypes.data_as(_vp)), "moq_plan_gather_layout")
    return slot, gather, passes


def moq_destroy_instance(h):
    _lib.moq_destroy_instance(h)


def moq_instance_get_info(h) -> dict:
    info = moq_instance_info()
    _check(_lib.moq_instance_get_info(h, C.byref(info)), "moq_instance_get_info")
    K = info.K
    return {"n": info.n, "K": K, "E": info.E, "max_degree": info.max_degree, "words": info.words,
            "weight_sum": list(info.weight_sum[:K]), "abs_sum": list(info.abs_sum[:K]),
            "ref_point": list(info.ref_point[:K]), "features": list(info.features)}


def moq_sample(inst, lam, R, params, seed, round_, bits, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample(inst, _dptr(lam, "lambda", f32), R, C.byref(params), seed, round_,
                           _dptr(bits, "bits", u64), _stream(stream)), "moq_sample")


def moq_evaluate_cuts(inst, bits, M, cuts, stream=None):
    _, i64, u64 = _torch_types()
    _check(_lib.moq_evaluate_cuts(inst, _dptr(bits, "bits", u64), M, _dptr(cuts, "cuts", i64), _stream(stream)),
           "moq_evaluate_cuts")


def moq_archive_create(n, K, capacity, max_batch) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.moq_archive_create(n, K, capacity, max_batch, C.byref(h)), "moq_archive_create")
    return h


def moq_archive_destroy(h):
    _lib.moq_archive_destroy(h)


def moq_archive_reset(a, stream=None):
    _check(_lib.moq_archive_reset(a, _stream(stream)), "moq_archive_reset")


def moq_pareto_front(a, cuts, bits, M, index_base, want_size=False, stream=None):
    _, i64, u64 = _torch_types()
    size = C.c_int64(-1)
    _check(_lib.moq_pareto_front(a, _dptr(cuts, "cuts", i64), _dptr(bits, "bits", u64), M, index_base,
                                 C.byref(size) if want_size else None, _stream(stream)), "moq_pareto_front")
    return int(size.value) if want_size else None


def moq_archive_merge(dst, src, stream=None):
    _check(_lib.moq_archive_merge(dst, src, _stream(stream)), "moq_archive_merge")


def moq_archive_size(a, stream=None) -> int:
    s = C.c_int64()
    _check(_lib.moq_archive_size(a, C.byref(s), _stream(stream)), "moq_archive_size")
    return int(s.value)


def moq_archive_copy_out(a, K, W, stream=None):
    """Returns (cuts (F,K) int64, bits (F,W) uint64, index (F,) int64) as numpy arrays."""
    F = moq_archive_size(a, stream)
    cuts = np.zeros((max(F, 1), K), np.int64)
    bits = np.zeros((max(F, 1), W), np.uint64)
    idx = np.zeros(max(F, 1), np.int64)
    n = C.c_int64()
    _check(_lib.moq_archive_copy_out(a, cuts.ctypes.data_as(_vp), bits.ctypes.data_as(_vp), idx.ctypes.data_as(_vp),
                                     F, C.byref(n), _stream(stream)), "moq_archive_copy_out")
    F = int(n.value)
    return cuts[:F], bits[:F], idx[:F]


def moq_archive_copy_out_into(a, cuts, bits, index, stream=None) -> int:
    """Copies the front into caller-owned host arrays (cuts (cap,K) int64, bits (cap,W) uint64
    or int64, index (cap,) int64, C-contiguous; page-locked memory makes each copy one DMA) and
    returns the front's size F; only the first min(F, cap) rows are written."""
    cap = index.shape[0]
    for arr, name in ((cuts, "cuts"), (bits, "bits"), (index, "index")):
        if not arr.flags["C_CONTIGUOUS"] or arr.dtype.itemsize != 8 or arr.shape[0] != cap:
            raise ValueError(f"moq_archive_copy_out_into: {name} must be C-contiguous 8-byte rows, {cap} of them")
    n = C.c_int64()
    _check(_lib.moq_archive_copy_out(a, cuts.ctypes.data_as(_vp), bits.ctypes.data_as(_vp), index.ctypes.data_as(_vp),
                                     cap, C.byref(n), _stream(stream)), "moq_archive_copy_out")
    return int(n.value)


def moq_archive_device_view(a):
    cuts, bits, idx, size = _vp(), _vp(), _vp(), _vp()
    _check(_lib.moq_archive_device_view(a, C.byref(cuts), C.byref(bits), C.byref(idx), C.byref(size)),
           "moq_archive_device_view")
    return cuts.value, bits.value, idx.value, size.value


def moq_hypervolume(a, ref, stream=None) -> int:
    ref_, pref = _hptr(ref, np.int64)
    out = moq_hv()
    _check(_lib.moq_hypervolume(a, pref, C.byref(out), _stream(stream)), "moq_hypervolume")
    return out.value()


def moq_hypervolume_many(archives, refs, stream=None) -> list:
    """Exact hypervolumes of several archives of one K (refs: count x K), two synchronisations in all."""
    count = len(archives)
    refs_, pref = _hptr(refs, np.int64)
    if count and (refs_.size % count or refs_.size // count < 2):
        raise ValueError("refs must hold one reference point (K >= 2 entries) per archive")
    hs = (_vp * max(count, 1))(*[a.value if isinstance(a, C.c_void_p) else a for a in archives])
    out = (moq_hv * max(count, 1))()
    _check(_lib.moq_hypervolume_many(hs, pref, count, out, _stream(stream)), "moq_hypervolume_many")
    return [out[i].value() for i in range(count)]


def moq_hypervolume_workspace_size(F, K) -> int:
    return int(_lib.moq_hypervolume_workspace_size(F, K))


def moq_hypervolume_points(pts, F, K, ref, workspace, stream=None) -> int:
    _, i64, _ = _torch_types()
    ref_, pref = _hptr(ref, np.int64)
    out = moq_hv()
    _check(_lib.moq_hypervolume_points(_dptr(pts, "pts", i64), F, K, pref, _dptr(workspace, "workspace"),
                                       C.byref(out), _stream(stream)), "moq_hypervolume_points")
    return out.value()


def moq_batch_create(instances, replicas) -> C.c_void_p:
    arr = (C.c_void_p * len(instances))(*[h.value if isinstance(h, C.c_void_p) else h for h in instances])
    reps, preps = _hptr(replicas, np.int32)
    h = C.c_void_p()
    _check(_lib.moq_batch_create(arr, len(instances), preps, C.byref(h)), "moq_batch_create")
    return h


def moq_batch_destroy(h):
    _lib.moq_batch_destroy(h)


def moq_batch_layout(h, count):
    """(replica_offsets, word_offsets), each count + 1 int64 entries."""
    ro = np.zeros(count + 1, np.int64)
    wo = np.zeros(count + 1, np.int64)
    _check(_lib.moq_batch_layout(h, ro.ctypes.data_as(_vp), wo.ctypes.data_as(_vp)), "moq_batch_layout")
    return ro, wo


def moq_batch_set_tiles(h, block_threads, slots_per_thread) -> int:
    items = C.c_int32()
    _check(_lib.moq_batch_set_tiles(h, block_threads, slots_per_thread, C.byref(items)), "moq_batch_set_tiles")
    return int(items.value)


def moq_batch_set_replicas(h, replicas):
    reps, preps = _hptr(replicas, np.int32)
    _check(_lib.moq_batch_set_replicas(h, preps), "moq_batch_set_replicas")


def moq_sample_batch(h, lam_all, params, seed, round_, bits_all, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample_batch(h, _dptr(lam_all, "lambda_all", f32), C.byref(params), seed, round_,
                                 _dptr(bits_all, "bits_all", u64), _stream(stream)), "moq_sample_batch")


def moq_evaluate_cuts_batch(h, bits_all, cuts_all, stream=None):
    _, i64, u64 = _torch_types()
    _check(_lib.moq_evaluate_cuts_batch(h, _dptr(bits_all, "bits_all", u64), _dptr(cuts_all, "cuts_all", i64),
                                        _stream(stream)), "moq_evaluate_cuts_batch")


def moq_dense_create(inst, max_replicas) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.moq_dense_create(inst, max_replicas, C.byref(h)), "moq_dense_create")
    return h


def moq_dense_destroy(h):
    _lib.moq_dense_destroy(h)


def moq_sample_dense(h, lam, R, params, seed, round_, bits, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample_dense(h, _dptr(lam, "lambda", f32), R, C.byref(params), seed, round_,
                                 _dptr(bits, "bits", u64), _stream(stream)), "moq_sample_dense")


def moq_sample_dense_fp8(h, lam, R, params, seed, round_, bits, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample_dense_fp8(h, _dptr(lam, "lambda", f32), R, C.byref(params), seed, round_,
                                     _dptr(bits, "bits", u64), _stream(stream)), "moq_sample_dense_fp8")


def moq_sample_dense_split(h, lam, R, params, seed, round_, bits, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample_dense_split(h, _dptr(lam, "lambda", f32), R, C.byref(params), seed, round_,
                                       _dptr(bits, "bits", u64), _stream(stream)), "moq_sample_dense_split")


def moq_dense_status(h, stream=None):
    _check(_lib.moq_dense_status(h, _stream(stream)), "moq_sample_dense")


def moq_dense_evaluate_cuts(h, bits, M, cuts, stream=None):
    _, i64, u64 = _torch_types()
    _check(_lib.moq_dense_evaluate_cuts(h, _dptr(bits, "bits", u64), M, _dptr(cuts, "cuts", i64), _stream(stream)),
           "moq_dense_evaluate_cuts")


def moq_dense_fp32_create(inst, max_replicas) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.moq_dense_fp32_create(inst, max_replicas, C.byref(h)), "moq_dense_fp32_create")
    return h


def moq_dense_fp32_destroy(h):
    _lib.moq_dense_fp32_destroy(h)


def moq_sample_dense_fp32(h, lam, R, params, seed, round_, bits, stream=None):
    f32, _, u64 = _torch_types()
    _check(_lib.moq_sample_dense_fp32(h, _dptr(lam, "lambda", f32), R, C.byref(params), seed, round_,
                                      _dptr(bits, "bits", u64), _stream(stream)), "moq_sample_dense_fp32")


def moq_mlp_create(d_in, d_out, max_batch, max_candidates, seed) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.moq_mlp_create(d_in, d_out, max_batch, max_candidates, seed, C.byref(h)), "moq_mlp_create")
    return h


def moq_mlp_destroy(h):
    _lib.moq_mlp_destroy(h)


def moq_mlp_param_count(h) -> int:
    return int(_lib.moq_mlp_param_count(h))


def moq_mlp_set_params(h, params):
    p, pp = _hptr(params, np.float32)
    _check(_lib.moq_mlp_set_params(h, pp), "moq_mlp_set_params")


def moq_mlp_get_params(h, bf16_rounded=False) -> np.ndarray:
    out = np.zeros(moq_mlp_param_count(h), np.float32)
    _check(_lib.moq_mlp_get_params(h, out.ctypes.data_as(_vp), int(bf16_rounded)), "moq_mlp_get_params")
    return out


def moq_mlp_forward(h, X, B, Y, stream=None):
    f32, _, _ = _torch_types()
    _check(_lib.moq_mlp_forward(h, _dptr(X, "X", f32), B, _dptr(Y, "Y", f32), _stream(stream)), "moq_mlp_forward")


def moq_mlp_gradient(h, X, T, B, grad=None, loss=None, stream=None):
    f32, _, _ = _torch_types()
    _check(_lib.moq_mlp_gradient(h, _dptr(X, "X", f32), _dptr(T, "T", f32), B, _dptr(grad, "grad", f32),
                                 _dptr(loss, "loss", f32), _stream(stream)), "moq_mlp_gradient")


def moq_mlp_adam_step(h, lr, stream=None):
    _check(_lib.moq_mlp_adam_step(h, lr, _stream(stream)), "moq_mlp_adam_step")


def moq_release_cached_memory():
    _check(_lib.moq_release_cached_memory(), "moq_release_cached_memory")


def moq_mlp_train_step(h, X, T, B, lr, loss=None, stream=None):
    f32, _, _ = _torch_types()
    _check(_lib.moq_mlp_train_step(h, _dptr(X, "X", f32), _dptr(T, "T", f32), B, lr, _dptr(loss, "loss", f32), _stream(stream)),
           "moq_mlp_train_step")


def moq_mlp_set_engine(h, engine):
    if isinstance(engine, str):
        engine = {"cuda_cores": MOQ_MLP_CUDA_CORES, "tensor_cores": MOQ_MLP_TENSOR_CORES}[engine]
    _check(_lib.moq_mlp_set_engine(h, engine), "moq_mlp_set_engine")


def moq_mlp_status(h, stream=None):
    _check(_lib.moq_mlp_status(h, _stream(stream)), "moq_mlp_status")


def moq_mlp_make_rows(K, features, lam, cuts, M, offset, scale, X, T, stream=None):
    f32, i64, _ = _torch_types()
    feat, pf = _hptr(features, np.float32)
    off, po = _hptr(offset, np.int64)
    sc, ps = _hptr(scale, np.int64)
    _check(_lib.moq_mlp_make_rows(K, feat.size, _dptr(lam, "lambda", f32), _dptr(cuts, "cuts", i64), M, pf, po, ps,
                                  _dptr(X, "X", f32), _dptr(T, "T", f32), _stream(stream)), "moq_mlp_make_rows")


def moq_lambda_propose(h, archive, features, offset, scale, n_candidates, seed, round_, lam_out, R, stream=None):
    f32, _, _ = _torch_types()
    feat, pf = _hptr(features, np.float32)
    off, po = _hptr(offset, np.int64)
    sc, ps = _hptr(scale, np.int64)
    _check(_lib.moq_lambda_propose(h, archive, pf, feat.size, po, ps, n_candidates, seed, round_,
                                   _dptr(lam_out, "lambda_out", f32), R, _stream(stream)), "moq_lambda_propose")


def moq_hypervolume_noalloc_max_points() -> int:
    return int(_lib.moq_hypervolume_noalloc_max_points())


def moq_hypervolume_points_noalloc(pts, F, K, ref, stream=None) -> int:
    """Hypervolume without any device allocation, for callers that cannot allocate device
    memory at that point; the scratch is a fixed array inside the library (at most
    ``moq_hypervolume_noalloc_max_points()`` points). Overlapping calls race on it."""
    _, i64, _ = _torch_types()
    ref_, pref = _hptr(ref, np.int64)
    out = moq_hv()
    _check(_lib.moq_hypervolume_points_noalloc(_dptr(pts, "pts", i64), F, K, pref, C.byref(out), _stream(stream)),
           "moq_hypervolume_points_noalloc")
    return out.value()


def moq_lambda_das_dennis(K, H, interior, lam, capacity, stream=None) -> int:
    f32, _, _ = _torch_types()
    cnt = C.c_int64()
    _check(_lib.moq_lambda_das_dennis(K, H, int(interior), _dptr(lam, "lambda", f32), capacity, C.byref(cnt),
                                      _stream(stream)), "moq_lambda_das_dennis")
    return int(cnt.value)


def moq_lambda_dirichlet(K, R, seed, round_, lam, stream=None):
    f32, _, _ = _torch_types()
    _check(_lib.moq_lambda_dirichlet(K, R, seed, round_, _dptr(lam, "lambda", f32), _stream(stream)),
           "moq_lambda_dirichlet")
