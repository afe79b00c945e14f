"""Thin Python binding of ``libcfs.so`` (declared in ``include/cfs.h``).

Argument marshalling only: every step of the chaos game runs in the library's
CUDA kernels.  Device buffers are torch tensors; streams are torch streams.
There is no CPU fallback: if the library cannot be built or loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

MAX_MAPS = 16
MAX_OPS = 32
MAX_TARGETS = 4
OP_PARAMS = 16

MAP_KINDS = {"affine": 0, "circle": 1}
OP_KINDS = {
    "affine2": 1, "affine3": 2, "rotate2": 3, "rotate3": 4, "translate3": 5, "swirl": 6,
    "sinusoidal": 7, "sinusoidal3": 8, "stretch": 9, "torus": 10, "perspective": 11,
    "twist_z": 12, "bend": 13, "inversion": 14, "splat": 15, "reset": 16, "stars": 17,
    "hemisphere": 18, "bands": 19,
}
TARGET_KINDS = {"hist_u32": 0, "rgba_f32": 1, "depth_u64": 2}
FLAG_REUSE = 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "COMPILE", 4: "CUDA", 5: "OOM",
          6: "TIMEOUT"}


class CfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cfs {STATUS.get(status, status)}: {msg}")
        self.status = status


class cfs_map(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("params", ctypes.c_float * 12)]


class cfs_transform(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("params", ctypes.c_float * OP_PARAMS)]


class cfs_target(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("channels", ctypes.c_int32),
                ("x0", ctypes.c_float), ("x1", ctypes.c_float),
                ("y0", ctypes.c_float), ("y1", ctypes.c_float),
                ("data", ctypes.c_void_p),
                ("palette", (ctypes.c_float * 4) * MAX_MAPS),
                ("palette8", ctypes.c_uint32 * MAX_MAPS)]


class cfs_render_params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("system_id", ctypes.c_uint32),
                ("point_begin", ctypes.c_uint32), ("n_points", ctypes.c_uint32),
                ("step_begin", ctypes.c_uint32), ("iters", ctypes.c_uint32),
                ("burn_in", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("start", ctypes.c_void_p), ("discards", ctypes.c_void_p)]


class cfs_frame(ctypes.Structure):
    _fields_ = [("system", ctypes.c_void_p), ("n_points", ctypes.c_uint32),
                ("point_begin", ctypes.c_uint32), ("system_id", ctypes.c_uint32),
                ("start_count", ctypes.c_uint32), ("start", ctypes.c_void_p),
                ("targets", cfs_target * MAX_TARGETS)]


class cfs_batch_tuning(ctypes.Structure):
    _fields_ = [("ilp", ctypes.c_int), ("tile", ctypes.c_int), ("chunk", ctypes.c_uint32),
                ("trial_ms", ctypes.c_float), ("trials", ctypes.c_int),
                ("window_words", ctypes.c_uint32), ("warp_agg", ctypes.c_int),
                ("n_classes", ctypes.c_int), ("classes_windowed", ctypes.c_int),
                ("from_cache", ctypes.c_int), ("classes_used", ctypes.c_int)]


class cfs_batch_plan(ctypes.Structure):
    _fields_ = [("ilp", ctypes.c_int), ("window", ctypes.c_int),
                ("window_words", ctypes.c_uint32), ("warp_agg", ctypes.c_int),
                ("chunk", ctypes.c_uint32)]


class cfs_train_options(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("systems_per_step", ctypes.c_uint32),
                ("points_per_system", ctypes.c_uint32), ("n_proj", ctypes.c_uint32),
                ("lr", ctypes.c_float), ("lr_final", ctypes.c_float), ("seed", ctypes.c_uint64)]


class cfs_display_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_float), ("brightness", ctypes.c_float),
                ("a_max", ctypes.c_float), ("background", ctypes.c_uint32)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "cfs_system_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(cfs_map),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(_P)]),
    "cfs_system_destroy": (ctypes.c_int, [_P]),
    "cfs_compose": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(cfs_transform), ctypes.c_int,
                                   ctypes.POINTER(_P)]),
    "cfs_compose_ex": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(cfs_transform), ctypes.c_int,
                                      ctypes.c_uint32, ctypes.POINTER(_P)]),
    "cfs_chain_destroy": (ctypes.c_int, [_P]),
    "cfs_compose_scribble": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p, ctypes.c_char_p,
                                            ctypes.c_uint32, ctypes.POINTER(_P)]),
    "cfs_chain_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "cfs_chain_set_params": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "cfs_render": (ctypes.c_int, [_P, _P, ctypes.POINTER(cfs_render_params),
                                  ctypes.POINTER(cfs_target), ctypes.c_int, _P]),
    "cfs_prepare": (ctypes.c_int, [_P, _P, ctypes.POINTER(cfs_target), ctypes.c_int]),
    "cfs_trace": (ctypes.c_int, [_P, _P, ctypes.POINTER(cfs_render_params), _P,
                                 ctypes.c_uint32, _P, _P, _P, _P]),
    "cfs_codegen_check": (ctypes.c_int, [_P, _P, ctypes.POINTER(cfs_target), ctypes.c_int,
                                         ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t,
                                         ctypes.c_char_p, ctypes.c_size_t]),
    "cfs_target_clear": (ctypes.c_int, [ctypes.POINTER(cfs_target), ctypes.c_int, _P]),
    "cfs_philox": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32, _P]),
    "cfs_atomic_bench": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, _P]),
    "cfs_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(cfs_frame),
                                        ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "cfs_batch_set_system": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cfs_batch_launch": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "cfs_batch_discards": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "cfs_batch_windows": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "cfs_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(ctypes.c_uint32),
                                      ctypes.POINTER(ctypes.c_uint32)]),
    "cfs_batch_destroy": (ctypes.c_int, [_P]),
    "cfs_batch_tune": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, _P,
                                      ctypes.POINTER(cfs_batch_tuning)]),
    "cfs_batch_get_plan": (ctypes.c_int, [_P, ctypes.POINTER(cfs_batch_plan)]),
    "cfs_batch_set_plan": (ctypes.c_int, [_P, ctypes.POINTER(cfs_batch_plan)]),
    "cfs_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "cfs_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "cfs_tune_cache_clear": (ctypes.c_int, []),
    "cfs_tune_cache_size": (ctypes.c_uint32, []),
    "cfs_render_batch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(cfs_frame),
                                        ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, _P]),
    "cfs_pointcloud_generate": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P]),
    "cfs_render_points": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint32,
                                         ctypes.POINTER(cfs_target), ctypes.c_int, _P, _P]),
    "cfs_pointcloud_reorder": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_int, _P, _P,
                                              _P, _P]),
    "cfs_stream_status": (ctypes.c_int, [_P]),
    "cfs_render_arg_bytes": (ctypes.c_uint32, []),
    "cfs_debug_raise_device_error": (ctypes.c_int, [ctypes.c_uint32]),
    "cfs_sampler_param_count": (ctypes.c_uint32, []),
    "cfs_sampler_create": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "cfs_sampler_destroy": (ctypes.c_int, [_P]),
    "cfs_sampler_get_params": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint32)]),
    "cfs_sampler_set_params": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_uint32]),
    "cfs_sampler_forward": (ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P]),
    "cfs_sampler_backward": (ctypes.c_int, [_P, _P, ctypes.c_uint32, _P, _P, _P]),
    "cfs_sw_loss": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_uint32, _P,
                                   ctypes.c_uint32, _P, _P, _P]),
    "cfs_sampler_adam": (ctypes.c_int, [_P, _P, ctypes.c_uint32, ctypes.c_float, _P]),
    "cfs_sampler_train": (ctypes.c_int, [_P, ctypes.POINTER(_P), _P, ctypes.c_int,
                                         ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_float, ctypes.c_uint64, _P,
                                         _P]),
    "cfs_sampler_train_ex": (ctypes.c_int, [_P, ctypes.POINTER(_P), _P, ctypes.c_int,
                                            ctypes.POINTER(cfs_train_options), _P, _P]),
    "cfs_sampler_start_points": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_uint32,
                                                ctypes.c_uint64, _P, _P]),
    "cfs_render_batch_noalloc": (ctypes.c_int, [ctypes.POINTER(cfs_frame), ctypes.c_int,
                                                ctypes.c_uint32, ctypes.c_uint32,
                                                ctypes.c_uint64, ctypes.c_int, _P, _P]),
    "cfs_sampler_start_points_batch": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), _P,
                                                      _P, _P, ctypes.POINTER(_P), _P]),
    "cfs_tonemap": (ctypes.c_int, [ctypes.POINTER(cfs_target), ctypes.POINTER(cfs_display_params),
                                   _P, _P, _P]),
    "cfs_batch_display": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(cfs_display_params),
                                         ctypes.POINTER(_P), _P, _P]),
    "cfs_last_error": (ctypes.c_char_p, []),
    "cfs_version": (ctypes.c_char_p, []),
}

_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Builds (if needed) and loads libcfs.so; raises if that fails."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _check(status: int):
    if status != 0:
        msg = lib().cfs_last_error().decode(errors="replace")
        raise CfsError(status, msg)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class System:
    """An IFS (Section 1): maps with probabilities.  ``desc`` has ``.dim``,
    ``.maps`` (``.kind``, ``.params``) and ``.probs``."""

    def __init__(self, desc):
        n = len(desc.maps)
        maps = (cfs_map * max(n, 1))()
        for j, m in enumerate(desc.maps):
            maps[j].kind = MAP_KINDS[m.kind]
            for q, v in enumerate(m.params):
                maps[j].params[q] = float(v)
        probs = (ctypes.c_double * max(n, 1))(*[float(p) for p in desc.probs])
        h = _P()
        _check(lib().cfs_system_create(desc.dim, n, maps, probs, ctypes.byref(h)))
        self.handle = h
        self.dim = desc.dim
        self.n_maps = n

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.cfs_system_destroy(h)
            self.handle = None


def _transforms(ops) -> Tuple[ctypes.Array, int]:
    n = len(ops)
    arr = (cfs_transform * max(n, 1))()
    for j, o in enumerate(ops):
        arr[j].kind = OP_KINDS[o.kind]
        for q, v in enumerate(o.params):
            arr[j].params[q] = float(v)
    return arr, n


class Chain:
    """A composed transform chain (Section 3, Fig. 2B) for points of
    dimension ``dim_in``; ``ops`` are ``.kind`` / ``.params`` records."""

    def __init__(self, ops, dim_in: int, fast_trig: bool = False, fold_linear: bool = False):
        arr, n = _transforms(ops)
        h = _P()
        flags = (1 if fast_trig else 0) | (4 if fold_linear else 0)
        _check(lib().cfs_compose_ex(dim_in, arr, n, flags, ctypes.byref(h)))
        self.fast_trig = fast_trig
        self.handle = h
        self.ops = list(ops)
        self.dim_in = dim_in
        self.n_splat = sum(1 for o in ops if o.kind == "splat")

    @classmethod
    def from_scribble(cls, source: str, poem: str, dim_in: int, fast_trig: bool = False):
        """A chain written as a scribble poem (verses, stanzas, poems; see
        ``cfs_compose_scribble`` in include/cfs.h for the language)."""
        self = cls.__new__(cls)
        h = _P()
        _check(lib().cfs_compose_scribble(dim_in, source.encode(), poem.encode(),
                                          1 if fast_trig else 0, ctypes.byref(h)))
        self.fast_trig = fast_trig
        self.handle = h
        self.ops = []
        self.dim_in = dim_in
        ns = ctypes.c_int()
        _check(lib().cfs_chain_info(h, None, None, ctypes.byref(ns)))
        self.n_splat = ns.value
        return self

    def set_params(self, index: int, params: Sequence[float]):
        buf = (ctypes.c_float * OP_PARAMS)(*([float(v) for v in params] +
                                             [0.0] * (OP_PARAMS - len(params))))
        _check(lib().cfs_chain_set_params(self.handle, index, buf))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.cfs_chain_destroy(h)
            self.handle = None


# ---------------------------------------------------------------------------
# targets
# ---------------------------------------------------------------------------
def target_shape(desc) -> Tuple[Tuple[int, ...], str]:
    if desc.kind == "hist_u32":
        return (desc.C, desc.H, desc.W), "int32"
    if desc.kind == "rgba_f32":
        return (desc.H, desc.W, 4), "float32"
    if desc.kind == "depth_u64":
        return (desc.H, desc.W), "int64"
    raise ValueError(desc.kind)


def alloc_target(desc, device="cuda"):
    """A device tensor for ``desc`` (u32 histograms and u64 depth keys live in
    int32 / int64 tensors of the same bytes), cleared to the empty value."""
    import torch
    shape, dt = target_shape(desc)
    t = torch.empty(shape, dtype=getattr(torch, dt), device=device)
    if desc.kind == "depth_u64":
        t.fill_(-1)
    else:
        t.zero_()
    return t


def make_targets(descs, tensors=None, fake_ptr: bool = False):
    n = len(descs)
    if n > MAX_TARGETS:
        raise ValueError("at most 4 targets")
    arr = (cfs_target * max(n, 1))()
    for j, d in enumerate(descs):
        t = arr[j]
        t.kind = TARGET_KINDS[d.kind]
        t.width, t.height = d.W, d.H
        t.channels = d.C if d.kind == "hist_u32" else 1
        t.x0, t.x1, t.y0, t.y1 = [float(v) for v in d.view]
        if fake_ptr:
            t.data = 256
        else:
            tt = tensors[j]
            if not tt.is_cuda or not tt.is_contiguous():
                raise ValueError("targets must be contiguous CUDA tensors")
            shape, _ = target_shape(d)
            if tuple(tt.shape) != shape:
                raise ValueError(f"target {j}: shape {tuple(tt.shape)} != {shape}")
            t.data = tt.data_ptr()
        if getattr(d, "palette", None) is not None:
            p = np.asarray(d.palette, dtype=np.float32)
            for k in range(min(MAX_MAPS, p.shape[0])):
                for c in range(4):
                    t.palette[k][c] = float(p[k, c])
        if getattr(d, "palette8", None) is not None:
            p8 = np.asarray(d.palette8, dtype=np.uint32)
            for k in range(min(MAX_MAPS, p8.shape[0])):
                t.palette8[k] = int(p8[k])
    return arr, n


def target_clear(descs, tensors, stream=None):
    arr, n = make_targets(descs, tensors)
    _check(lib().cfs_target_clear(arr, n, _stream_handle(stream)))


# ---------------------------------------------------------------------------
# calls
# ---------------------------------------------------------------------------
def _params(*, seed, system_id, point_begin, n_points, step_begin, iters, burn_in, flags,
            start, discards):
    p = cfs_render_params()
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.system_id, p.point_begin, p.n_points = int(system_id), int(point_begin), int(n_points)
    p.step_begin, p.iters, p.burn_in, p.flags = int(step_begin), int(iters), int(burn_in), flags
    p.start = start.data_ptr() if start is not None else None
    p.discards = discards.data_ptr() if discards is not None else None
    return p


def render(system: System, chain: Chain, target_descs, target_tensors, *, n_points: int,
           iters: int, burn_in: int, seed: int = 0, system_id: int = 0, point_begin: int = 0,
           step_begin: int = 0, reuse: bool = False, start=None, discards=None, stream=None):
    """Enqueues the chaos game for points point_begin .. +n_points on
    ``stream`` (default: torch's current stream).  ``start``: optional device
    float32 [dim, n_points]; ``discards``: optional device int64
    [n_targets] to which discarded splats are added."""
    arr, n = make_targets(target_descs, target_tensors)
    if start is not None:
        assert start.is_cuda and start.is_contiguous() and start.shape == (system.dim, n_points)
    if discards is not None:
        assert discards.is_cuda and discards.numel() >= n
    p = _params(seed=seed, system_id=system_id, point_begin=point_begin, n_points=n_points,
                step_begin=step_begin, iters=iters, burn_in=burn_in,
                flags=FLAG_REUSE if reuse else 0, start=start, discards=discards)
    _check(lib().cfs_render(system.handle, chain.handle, ctypes.byref(p), arr, n,
                            _stream_handle(stream)))


def prepare(system: System, chain: Chain, target_descs, target_tensors):
    arr, n = make_targets(target_descs, target_tensors)
    _check(lib().cfs_prepare(system.handle, chain.handle, arr, n))


def trace(system: System, chain: Chain, ids, *, iters: int, seed: int = 0, system_id: int = 0,
          step_begin: int = 0, burn_in: int = 0, reuse: bool = False, start=None, stream=None):
    """Per-step map index, point and chain inputs of the points in ``ids``
    (device uint32/int32 tensor); returns device tensors k [n, steps],
    p [n, steps, 3], q [n, steps, n_splat, 4]."""
    import torch
    n = int(ids.numel())
    steps = iters - step_begin
    n_sp = max(1, chain.n_splat)
    dev = ids.device
    k = torch.empty((n, steps), dtype=torch.int32, device=dev)
    p = torch.empty((n, steps, 3), dtype=torch.float32, device=dev)
    q = torch.empty((n, steps, n_sp, 4), dtype=torch.float32, device=dev)
    prm = _params(seed=seed, system_id=system_id, point_begin=0, n_points=n,
                  step_begin=step_begin, iters=iters, burn_in=burn_in,
                  flags=FLAG_REUSE if reuse else 0, start=start, discards=None)
    _check(lib().cfs_trace(system.handle, chain.handle, ctypes.byref(prm), ids.data_ptr(), n,
                           k.data_ptr(), p.data_ptr(), q.data_ptr(), _stream_handle(stream)))
    return k, p, q


def philox(ctr, key, stream=None):
    """Philox4x32-10 on the GPU: ctr int32 [n, 4], key int32 [n, 2] device
    tensors (bit patterns of u32) -> int32 [n, 4]."""
    import torch
    n = ctr.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    _check(lib().cfs_philox(ctr.data_ptr(), key.data_ptr(), out.data_ptr(), n,
                            _stream_handle(stream)))
    return out


# ---------------------------------------------------------------------------
# stored clouds
# ---------------------------------------------------------------------------
def pointcloud_generate(system: System, n: int, iters: int, *, seed: int = 0,
                        system_id: int = 0, xyz=None, fn=None, stream=None):
    """Returns device tensors xyz float32 [dim, n] (SoA) and fn uint8 [n]."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    if xyz is None:
        xyz = torch.empty((system.dim, n), dtype=torch.float32, device=dev)
    if fn is None:
        fn = torch.empty((n,), dtype=torch.uint8, device=dev)
    _check(lib().cfs_pointcloud_generate(system.handle, int(seed) & 0xFFFFFFFFFFFFFFFF,
                                         system_id, n, iters, xyz.data_ptr(), fn.data_ptr(),
                                         _stream_handle(stream)))
    return xyz, fn


def pointcloud_reorder(xyz, fn, stream=None, want_perm: bool = False):
    """Morton-ordered copy of a stored cloud: (xyz_out, fn_out[, perm])."""
    import torch
    dim, n = xyz.shape
    xo = torch.empty_like(xyz)
    fo = torch.empty_like(fn)
    perm = torch.empty(n, dtype=torch.int32, device=xyz.device) if want_perm else None
    _check(lib().cfs_pointcloud_reorder(xyz.data_ptr(), fn.data_ptr(), n, dim, xo.data_ptr(),
                                        fo.data_ptr(),
                                        perm.data_ptr() if perm is not None else None,
                                        _stream_handle(stream)))
    return (xo, fo, perm) if want_perm else (xo, fo)


def render_points(chain: Chain, xyz, fn, target_descs, target_tensors, *, discards=None,
                  stream=None):
    """Streams the stored cloud (xyz float32 [dim, n], fn uint8 [n]) through
    ``chain`` into the targets."""
    arr, nt = make_targets(target_descs, target_tensors)
    assert xyz.is_cuda and xyz.is_contiguous() and fn.is_cuda and fn.is_contiguous()
    n = int(fn.numel())
    assert xyz.shape == (chain.dim_in, n)
    _check(lib().cfs_render_points(chain.handle, xyz.data_ptr(), fn.data_ptr(), n, arr, nt,
                                   discards.data_ptr() if discards is not None else None,
                                   _stream_handle(stream)))


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------
def _frames(frames):
    """frames: list of (System, n_points, point_begin, system_id, target_descs,
    target_tensors[, start]) -> ctypes array; ``start`` an optional device
    float32 [dim, m] tensor of start points, m <= n_points (point j starts at
    start point j mod m)."""
    arr = (cfs_frame * len(frames))()
    n_t = None
    for f, fr in enumerate(frames):
        sysh, n, pb, sid, descs, tens = fr[:6]
        start = fr[6] if len(fr) > 6 else None
        arr[f].system = sysh.handle
        arr[f].n_points, arr[f].point_begin, arr[f].system_id = int(n), int(pb), int(sid)
        if start is not None:
            assert start.is_cuda and start.is_contiguous() and start.shape[1] <= n
            arr[f].start = start.data_ptr()
            arr[f].start_count = int(start.shape[1])
        t_arr, nt = make_targets(descs, tens)
        for t in range(nt):
            arr[f].targets[t] = t_arr[t]
        n_t = nt if n_t is None else n_t
        if nt != n_t:
            raise ValueError("every frame needs the same number of targets")
    return arr, (n_t or 0)


class Batch:
    """Many frames in one persistent launch replayed as a CUDA graph.  Frames
    are (System, n_points, point_begin, system_id, target_descs,
    target_tensors) tuples; they share ``chain``, ``iters``, ``burn_in`` and
    ``seed``."""

    def __init__(self, chain: Chain, frames, *, iters: int, burn_in: int, seed: int = 0,
                 step_begin: int = 0):
        arr, nt = _frames(frames)
        h = _P()
        _check(lib().cfs_batch_create(chain.handle, nt, arr, len(frames), step_begin, iters,
                                      burn_in, int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(h)))
        self.handle = h
        self.n_frames = len(frames)
        self.n_targets = nt
        d0 = frames[0][4][0] if frames and nt else None
        self.window_channels = max(1, int(d0.C)) if d0 is not None and d0.kind == "hist_u32" \
            else 1
        self._keep = [f[0] for f in frames] + [chain]

    def launch(self, clear: bool = True, stream=None):
        _check(lib().cfs_batch_launch(self.handle, 1 if clear else 0, _stream_handle(stream)))

    def set_system(self, frame: int, system: System):
        _check(lib().cfs_batch_set_system(self.handle, frame, system.handle))
        self._keep.append(system)

    def discards(self) -> np.ndarray:
        out = np.zeros((self.n_frames, max(1, self.n_targets)), dtype=np.uint64)
        _check(lib().cfs_batch_discards(self.handle,
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return out

    def windows(self) -> np.ndarray:
        """Each frame's privatized windows in the last launch: int32
        [n_frames][channels][4] = (x0, y0, x1, y1), inclusive pixels of
        each channel of target 0; (0, 0, -1, -1) where there was none."""
        out = np.zeros((self.n_frames, self.window_channels, 4), dtype=np.int32)
        _check(lib().cfs_batch_windows(self.handle,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def info(self):
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().cfs_batch_info(self.handle, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(c)))
        return {"n_items": a.value, "chunk": b.value, "grid": c.value}

    def tune(self, trial_iters: int = 0, stream=None, retune: bool = False):
        """Times the candidate plans on these frames (program, then per shape
        class) and keeps the fastest, or takes them from the tuning cache
        (the targets hold trial output afterwards); returns the choice."""
        t = cfs_batch_tuning()
        _check(lib().cfs_batch_tune(self.handle, int(trial_iters), 1 if retune else 0,
                                    _stream_handle(stream), ctypes.byref(t)))
        return {"ilp": t.ilp, "tile": t.tile, "chunk": t.chunk, "trial_ms": t.trial_ms,
                "trials": t.trials, "window_words": t.window_words, "warp_agg": t.warp_agg,
                "n_classes": t.n_classes, "classes_windowed": t.classes_windowed,
                "from_cache": bool(t.from_cache), "classes_used": bool(t.classes_used)}

    def plan(self) -> dict:
        p = cfs_batch_plan()
        _check(lib().cfs_batch_get_plan(self.handle, ctypes.byref(p)))
        return {"ilp": p.ilp, "window": p.window, "window_words": p.window_words,
                "warp_agg": p.warp_agg, "chunk": p.chunk}

    def set_plan(self, **kw):
        """Replaces plan fields (ilp, window, window_words, warp_agg, chunk)."""
        cur = self.plan()
        unknown = set(kw) - set(cur)
        if unknown:
            raise ValueError(f"unknown plan fields {sorted(unknown)}")
        cur.update(kw)
        p = cfs_batch_plan(int(cur["ilp"]), int(cur["window"]), int(cur["window_words"]),
                           int(cur["warp_agg"]), int(cur["chunk"]))
        _check(lib().cfs_batch_set_plan(self.handle, ctypes.byref(p)))

    def display(self, outs, *, slot: int = 0, gamma: float = 2.2, brightness: float = 1.0,
                a_max: float = 0.0, background: int = 0, a_max_out=None, stream=None):
        """Displays target ``slot`` of every frame into ``outs`` (one int32
        [H, W] CUDA tensor per frame, holding packed RGBA8): one maximum and
        one mapping launch for all frames.  ``a_max_out``: optional float32
        [n_frames] CUDA tensor receiving each frame's density maximum."""
        if len(outs) != self.n_frames:
            raise ValueError("one output per frame")
        ptrs = (_P * self.n_frames)()
        for f, o in enumerate(outs):
            if not o.is_cuda or not o.is_contiguous():
                raise ValueError("outputs must be contiguous CUDA tensors")
            ptrs[f] = o.data_ptr()
        p = _display_params(gamma, brightness, a_max, background)
        _check(lib().cfs_batch_display(self.handle, slot, ctypes.byref(p), ptrs,
                                       a_max_out.data_ptr() if a_max_out is not None else None,
                                       _stream_handle(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.cfs_batch_destroy(h)
            self.handle = None


def render_batch(chain: Chain, frames, *, iters: int, burn_in: int, seed: int = 0,
                 clear: bool = True, step_begin: int = 0, stream=None):
    """One-shot batch: plans, launches and frees (returns after rendering)."""
    arr, nt = _frames(frames)
    _check(lib().cfs_render_batch(chain.handle, nt, arr, len(frames), step_begin, iters, burn_in,
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, 1 if clear else 0,
                                  _stream_handle(stream)))


# ---------------------------------------------------------------------------
# density-estimation display
# ---------------------------------------------------------------------------
def _display_params(gamma, brightness, a_max, background):
    p = cfs_display_params()
    p.gamma, p.brightness, p.a_max = float(gamma), float(brightness), float(a_max)
    p.background = int(background) & 0xFFFFFFFF
    return p


def tonemap(desc, tensor, out=None, *, gamma: float = 2.2, brightness: float = 1.0,
            a_max: float = 0.0, background: int = 0, a_max_out=None, stream=None):
    """Log-density display of one layer into packed RGBA8 (an int32 [H, W]
    CUDA tensor, allocated when ``out`` is None).  With ``a_max`` <= 0 the
    layer's own maximum is found on the device and written to ``a_max_out``
    (a float32 CUDA tensor with at least one element, allocated when None).
    Returns (out, a_max_out)."""
    import torch
    arr, _ = make_targets([desc], [tensor])
    if out is None:
        out = torch.empty((desc.H, desc.W), dtype=torch.int32, device=tensor.device)
    if a_max_out is None and a_max <= 0 and desc.kind != "depth_u64":
        a_max_out = torch.empty(1, dtype=torch.float32, device=tensor.device)
    p = _display_params(gamma, brightness, a_max, background)
    _check(lib().cfs_tonemap(arr, ctypes.byref(p), out.data_ptr(),
                             a_max_out.data_ptr() if a_max_out is not None else None,
                             _stream_handle(stream)))
    return out, a_max_out


# ---------------------------------------------------------------------------
# learned warm-start sampler
# ---------------------------------------------------------------------------
def _fptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Sampler:
    """The warm-start network (include/cfs.h): FP32 master parameters and
    Adam state on the device, BF16 tensor-core forward/backward."""

    def __init__(self, params=None, seed: int = 0):
        h = _P()
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().cfs_sampler_create(_fptr(p), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                        ctypes.byref(h)))
        self.handle = h
        self.n_params = int(lib().cfs_sampler_param_count())

    def get_params(self):
        w = np.zeros(self.n_params, np.float32)
        m = np.zeros(self.n_params, np.float32)
        v = np.zeros(self.n_params, np.float32)
        st = ctypes.c_uint32()
        _check(lib().cfs_sampler_get_params(self.handle, _fptr(w), _fptr(m), _fptr(v),
                                            ctypes.byref(st)))
        return w, m, v, st.value

    def set_params(self, w, m=None, v=None, step: int = 0):
        w = np.ascontiguousarray(w, np.float32)
        m = None if m is None else np.ascontiguousarray(m, np.float32)
        v = None if v is None else np.ascontiguousarray(v, np.float32)
        _check(lib().cfs_sampler_set_params(self.handle, _fptr(w), _fptr(m), _fptr(v), step))

    def forward(self, U, stream=None):
        """U: device bfloat16 [B, 64] -> device float32 [B, 2]."""
        import torch
        B = U.shape[0]
        Y = torch.empty((B, 2), dtype=torch.float32, device=U.device)
        _check(lib().cfs_sampler_forward(self.handle, U.data_ptr(), B, Y.data_ptr(),
                                         _stream_handle(stream)))
        return Y

    def backward(self, U, dY, grads=None, stream=None):
        import torch
        if grads is None:
            grads = torch.zeros(self.n_params, dtype=torch.float32, device=U.device)
        _check(lib().cfs_sampler_backward(self.handle, U.data_ptr(), U.shape[0], dY.data_ptr(),
                                          grads.data_ptr(), _stream_handle(stream)))
        return grads

    def adam(self, grads, t: int, lr: float = 1e-3, stream=None):
        _check(lib().cfs_sampler_adam(self.handle, grads.data_ptr(), t, lr,
                                      _stream_handle(stream)))

    def train(self, systems, t_values, steps: int, *, systems_per_step: int = 64,
              points_per_system: int = 1024, n_proj: int = 64, lr: float = 1e-3,
              lr_final: Optional[float] = None, seed: int = 0, stream=None):
        """systems: list of System handles; returns the loss per step.
        ``lr_final``: cosine decay of the step size from ``lr`` to it over
        the run (None: constant ``lr``)."""
        arr = (_P * len(systems))(*[s.handle for s in systems])
        tv = np.ascontiguousarray(t_values, np.float32)
        hist = np.zeros(max(steps, 1), np.float32)
        if lr_final is None:
            _check(lib().cfs_sampler_train(self.handle, arr, _fptr(tv), len(systems), steps,
                                           systems_per_step, points_per_system, n_proj, lr,
                                           int(seed) & 0xFFFFFFFFFFFFFFFF, _fptr(hist),
                                           _stream_handle(stream)))
        else:
            o = cfs_train_options(steps, systems_per_step, points_per_system, n_proj, lr,
                                  lr_final, int(seed) & 0xFFFFFFFFFFFFFFFF)
            _check(lib().cfs_sampler_train_ex(self.handle, arr, _fptr(tv), len(systems),
                                              ctypes.byref(o), _fptr(hist),
                                              _stream_handle(stream)))
        return hist[:steps]

    def start_points(self, system: System, t: float, n: int, seed: int = 0, out=None,
                     stream=None):
        """Device float32 [2, n] warm-start points (SoA) for ``system``."""
        import torch
        if out is None:
            out = torch.empty((2, n), dtype=torch.float32,
                              device=torch.device("cuda", torch.cuda.current_device()))
        _check(lib().cfs_sampler_start_points(self.handle, system.handle, float(t), n,
                                              int(seed) & 0xFFFFFFFFFFFFFFFF, out.data_ptr(),
                                              _stream_handle(stream)))
        return out

    def start_points_batch(self, systems, t_values, outs, seeds, stream=None):
        """One launch for many frames: outs[f] (device float32 [2, m_f]) gets
        m_f samples for systems[f] at time t_values[f] with seeds[f]."""
        n = len(systems)
        sy = (_P * n)(*[s.handle for s in systems])
        tv = np.ascontiguousarray(t_values, np.float32)
        cn = np.array([o.shape[1] for o in outs], np.uint32)
        sd = np.array([int(v) & 0xFFFFFFFFFFFFFFFF for v in seeds], np.uint64)
        op = (_P * n)(*[o.data_ptr() for o in outs])
        _check(lib().cfs_sampler_start_points_batch(self.handle, n, sy, _fptr(tv), _fptr(cn),
                                                    _fptr(sd), op, _stream_handle(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _LIB is not None:
            _LIB.cfs_sampler_destroy(h)
            self.handle = None


def sw_loss(X, T, phi, stream=None):
    """Sliced-Wasserstein loss of device point sets X, T [S, N, 2] over
    angles phi [P] -> (loss tensor [1], dX tensor)."""
    import torch
    S, N, _ = X.shape
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    dX = torch.zeros_like(X)
    _check(lib().cfs_sw_loss(X.data_ptr(), T.data_ptr(), S, N, phi.data_ptr(), phi.numel(),
                             loss.data_ptr(), dX.data_ptr(), _stream_handle(stream)))
    return loss, dX


def render_batch_noalloc(frames, *, iters: int, burn_in: int, seed: int = 0,
                         clear: bool = True, discards=None, stream=None):
    """Histogram frames (splat-only chain) rendered with the library's fixed
    device workspace instead of an allocation; ``frames`` as for ``Batch``
    (targets[0] a u32 histogram), at most 256 of them; ``discards``: optional
    device int64 [n_frames] receiving each frame's discarded splats."""
    arr, _ = _frames(frames)
    _check(lib().cfs_render_batch_noalloc(arr, len(frames), iters, burn_in,
                                          int(seed) & 0xFFFFFFFFFFFFFFFF, 1 if clear else 0,
                                          discards.data_ptr() if discards is not None else None,
                                          _stream_handle(stream)))


def atomic_bench(kind: int, buf, n_elems: int, blocks: int, iters: int, seed: int = 1,
                 stream=None):
    """Enqueues the atomic microbenchmark (see include/cfs.h) on ``stream``."""
    _check(lib().cfs_atomic_bench(kind, buf.data_ptr(), n_elems, blocks, iters, seed,
                                  _stream_handle(stream)))


def codegen_check(system: System, chain: Chain, target_descs, mode: int = 0,
                  cap: int = 1 << 20) -> Tuple[str, str]:
    """Generated source and NVRTC log (ptxas usage) of the fused program; no
    GPU needed."""
    arr, n = make_targets(target_descs, fake_ptr=True)
    src = ctypes.create_string_buffer(cap)
    log = ctypes.create_string_buffer(cap)
    st = lib().cfs_codegen_check(system.handle, chain.handle, arr, n, mode, src, cap, log, cap)
    if st != 0:
        raise CfsError(st, lib().cfs_last_error().decode(errors="replace"))
    return src.value.decode(), log.value.decode()


def tune_cache_load(path: str):
    _check(lib().cfs_tune_cache_load(os.fsencode(path)))


def tune_cache_save(path: str):
    _check(lib().cfs_tune_cache_save(os.fsencode(path)))


def tune_cache_clear():
    _check(lib().cfs_tune_cache_clear())


def tune_cache_size() -> int:
    return int(lib().cfs_tune_cache_size())


DEVICE_ERR_TC_TIMEOUT = 1


def stream_status(stream=None):
    """Waits for the stream's work; raises CfsError (CUDA or TIMEOUT) for a
    failure of that work or a device-side error flag set since the last
    report (cfs_stream_status)."""
    _check(lib().cfs_stream_status(_stream_handle(stream)))


def debug_raise_device_error(flags: int = DEVICE_ERR_TC_TIMEOUT):
    """Sets device error flags from the host, as a timed-out kernel would."""
    _check(lib().cfs_debug_raise_device_error(flags))


def render_arg_bytes() -> int:
    """Bytes of the argument block a render launch copies to the device."""
    return int(lib().cfs_render_arg_bytes())


def version() -> str:
    return lib().cfs_version().decode()
