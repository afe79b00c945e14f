"""Python access to the CPU oracle (``cfs_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, single-threaded
restatement of the chaos game the CUDA library is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this module.  It imports nothing from the library
package: systems, chains and targets arrive as plain objects with the
attributes documented in ``render``.

``build()`` compiles the C file with gcc (``-ffp-contract=off``, so the
compiler adds no fused multiply-adds of its own).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_LOCK = threading.Lock()
_LIB = None

MAX_MAPS = 16

MAP_KINDS = {"affine": 0, "circle": 1}
OP_KINDS = {
    "affine2": 1, "affine3": 2, "rotate2": 3, "rotate3": 4, "translate3": 5,
    "swirl": 6, "sinusoidal": 7, "sinusoidal3": 8, "stretch": 9, "torus": 10,
    "perspective": 11, "twist_z": 12, "bend": 13, "inversion": 14, "splat": 15,
    "reset": 16, "stars": 17, "hemisphere": 18, "bands": 19,
}
TARGET_KINDS = {"hist_u32": 0, "rgba_f32": 1, "depth_u64": 2}


class _System(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_maps", ctypes.c_int),
                ("kind", ctypes.POINTER(ctypes.c_int)),
                ("prm", ctypes.POINTER(ctypes.c_float)),
                ("prob", ctypes.POINTER(ctypes.c_double))]


class _Chain(ctypes.Structure):
    _fields_ = [("n_ops", ctypes.c_int), ("op", ctypes.POINTER(ctypes.c_int)),
                ("prm", ctypes.POINTER(ctypes.c_float)), ("band_eps", ctypes.c_float)]


class _Target(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("W", ctypes.c_int), ("H", ctypes.c_int),
                ("C", ctypes.c_int), ("x0", ctypes.c_float), ("x1", ctypes.c_float),
                ("y0", ctypes.c_float), ("y1", ctypes.c_float),
                ("buf", ctypes.c_void_p),
                ("palette", ctypes.POINTER(ctypes.c_float)),
                ("palette8", ctypes.POINTER(ctypes.c_uint32)),
                ("margin_px", ctypes.c_float),
                ("amb", ctypes.POINTER(ctypes.c_uint32)),
                ("zlo", ctypes.POINTER(ctypes.c_float)),
                ("zhi", ctypes.POINTER(ctypes.c_float)),
                ("klo", ctypes.POINTER(ctypes.c_uint64)),
                ("zalt", ctypes.POINTER(ctypes.c_float)),
                ("n_splat", ctypes.c_uint64), ("n_discard", ctypes.c_uint64),
                ("n_amb", ctypes.c_uint64)]


class _Run(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("system_id", ctypes.c_uint32),
                ("point_begin", ctypes.c_uint32), ("n_points", ctypes.c_uint32),
                ("step_begin", ctypes.c_uint32), ("iters", ctypes.c_uint32),
                ("burn_in", ctypes.c_uint32), ("reuse", ctypes.c_int),
                ("start", ctypes.POINTER(ctypes.c_float))]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so``; returns its path."""
    src = [os.path.join(_HERE, "cfs_oracle.c")]
    hdr = os.path.join(_HERE, "cfs_oracle.h")
    with _LOCK:
        newest = max(os.path.getmtime(p) for p in src + [hdr])
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp] + src + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _LIB
    if _LIB is None:
        so = build()
        L = ctypes.CDLL(so)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_thresholds.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64)]
        L.orc_choose.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
        L.orc_render.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Chain),
                                 ctypes.POINTER(_Target), ctypes.c_int, ctypes.POINTER(_Run)]
        L.orc_trace.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Chain),
                                ctypes.POINTER(_Run), ctypes.c_uint32, u32p,
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float), ctypes.c_int]
        L.orc_pointcloud_generate.argtypes = [ctypes.POINTER(_System), ctypes.c_uint64,
                                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(ctypes.c_uint8)]
        L.orc_render_points.argtypes = [ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32,
                                        ctypes.POINTER(_Chain), ctypes.POINTER(_Target),
                                        ctypes.c_int]
        L.orc_density_max.argtypes = [ctypes.POINTER(_Target)]
        L.orc_density_max.restype = ctypes.c_float
        L.orc_tonemap.argtypes = [ctypes.POINTER(_Target), ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_uint32, u32p,
                                  ctypes.POINTER(ctypes.c_uint8), ctypes.c_double]
        _LIB = L
    return _LIB


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------------------
# marshalling of plain descriptions
# ---------------------------------------------------------------------------
class _Keep:
    """Holds the numpy arrays a ctypes structure points into."""

    def __init__(self):
        self.arrays = []

    def __call__(self, a):
        self.arrays.append(a)
        return a


def _system(sys, keep):
    n = len(sys.maps)
    kind = keep(np.array([MAP_KINDS[m.kind] for m in sys.maps], dtype=np.int32))
    prm = keep(np.zeros((n, 12), dtype=np.float32))
    for j, m in enumerate(sys.maps):
        prm[j, :len(m.params)] = np.asarray(m.params, dtype=np.float32)
    prob = keep(np.asarray(sys.probs, dtype=np.float64).copy())
    return _System(sys.dim, n, _ptr(kind, ctypes.c_int), _ptr(prm, ctypes.c_float),
                   _ptr(prob, ctypes.c_double))


def _chain(chain, keep, band_eps=0.0):
    n = len(chain)
    op = keep(np.array([OP_KINDS[o.kind] for o in chain] or [0], dtype=np.int32))
    prm = keep(np.zeros((max(n, 1), 16), dtype=np.float32))
    for j, o in enumerate(chain):
        prm[j, :len(o.params)] = np.asarray(o.params, dtype=np.float32)
    return _Chain(n, _ptr(op, ctypes.c_int), _ptr(prm, ctypes.c_float), float(band_eps))


def alloc_target_buffer(t):
    """Host buffer initialised as an empty target (zeros; depth: all ones)."""
    if t.kind == "hist_u32":
        return np.zeros((t.C, t.H, t.W), dtype=np.uint32)
    if t.kind == "rgba_f32":
        return np.zeros((t.H, t.W, 4), dtype=np.float32)
    if t.kind == "depth_u64":
        return np.full((t.H, t.W), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    raise ValueError(t.kind)


class TargetResult:
    """A target's buffer, counters and (when tracked) the near-edge records:
    ``amb`` slack per pixel; for depth layers ``zlo`` (lowest depth that may
    land), ``zhi`` (lowest depth that surely lands), ``klo`` (lowest key of
    any splat that may land) and ``zalt`` (lowest depth that may land with a
    colour other than ``klo``'s)."""

    def __init__(self, buf, amb, zlo, zhi, klo=None, zalt=None):
        self.buf, self.amb, self.zlo, self.zhi = buf, amb, zlo, zhi
        self.klo, self.zalt = klo, zalt
        self.n_splat = 0
        self.n_discard = 0
        self.n_amb = 0


def _target(t, keep, buf, margin_px, track, prev=None):
    pal = keep(np.zeros((MAX_MAPS, 4), dtype=np.float32))
    if getattr(t, "palette", None) is not None:
        p = np.asarray(t.palette, dtype=np.float32)
        pal[:p.shape[0]] = p
    pal8 = keep(np.zeros(MAX_MAPS, dtype=np.uint32))
    if getattr(t, "palette8", None) is not None:
        p8 = np.asarray(t.palette8, dtype=np.uint32)
        pal8[:p8.shape[0]] = p8
    amb = zlo = zhi = klo = zalt = None
    if track and prev is not None:
        amb, zlo, zhi, klo, zalt = prev.amb, prev.zlo, prev.zhi, prev.klo, prev.zalt
    elif track:
        amb = np.zeros((t.H, t.W), dtype=np.uint32)
        if t.kind == "depth_u64":
            zlo = np.full((t.H, t.W), np.inf, dtype=np.float32)
            zhi = np.full((t.H, t.W), np.inf, dtype=np.float32)
            klo = np.full((t.H, t.W), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
            zalt = np.full((t.H, t.W), np.inf, dtype=np.float32)
    x0, x1, y0, y1 = t.view
    s = _Target(TARGET_KINDS[t.kind], t.W, t.H, getattr(t, "C", 1) or 1,
                x0, x1, y0, y1, buf.ctypes.data,
                _ptr(pal, ctypes.c_float), _ptr(pal8, ctypes.c_uint32),
                float(margin_px),
                _ptr(amb, ctypes.c_uint32) if amb is not None else None,
                _ptr(zlo, ctypes.c_float) if zlo is not None else None,
                _ptr(zhi, ctypes.c_float) if zhi is not None else None,
                _ptr(klo, ctypes.c_uint64) if klo is not None else None,
                _ptr(zalt, ctypes.c_float) if zalt is not None else None,
                *((prev.n_splat, prev.n_discard, prev.n_amb) if prev is not None else (0, 0, 0)))
    return s, TargetResult(buf, amb, zlo, zhi, klo, zalt)


def _run(seed, system_id, point_begin, n_points, step_begin, iters, burn_in, reuse, start, keep):
    sp = None
    if start is not None:
        st = np.zeros((n_points, 3), dtype=np.float32)
        a = np.asarray(start, dtype=np.float32)
        st[:, :a.shape[1]] = a
        keep(st)
        sp = _ptr(st, ctypes.c_float)
    return _Run(seed, system_id, point_begin, n_points, step_begin, iters, burn_in,
                1 if reuse else 0, sp)


# ---------------------------------------------------------------------------
# public helpers
# ---------------------------------------------------------------------------
def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def thresholds(probs):
    p = np.asarray(probs, dtype=np.float64)
    T = np.zeros(max(len(p), 1), dtype=np.uint64)
    rc = lib().orc_thresholds(len(p), _ptr(p, ctypes.c_double), _ptr(T, ctypes.c_uint64))
    if rc != 0:
        raise ValueError("invalid probabilities")
    return T[:len(p) - 1]


def choose(w, T, n_maps):
    T = np.asarray(T, dtype=np.uint64)
    return lib().orc_choose(w, n_maps, _ptr(T, ctypes.c_uint64))


def render(system, chain, targets, *, n_points, iters, burn_in, seed=0, system_id=0,
           point_begin=0, step_begin=0, reuse=False, start=None, margin_px=0.0,
           track=False, bufs=None, prev=None, band_eps=0.0):
    """Runs the chaos game for points point_begin .. point_begin + n_points - 1.

    ``system``: ``.dim``, ``.maps`` (each ``.kind``, ``.params``), ``.probs``.
    ``chain``: list of ops (``.kind``, ``.params``).  ``targets``: list with
    ``.kind``, ``.W``, ``.H``, ``.C``, ``.view`` = (x0, x1, y0, y1),
    ``.palette`` (RGBA), ``.palette8`` (depth).  ``bufs`` lets a caller
    accumulate into existing host buffers; ``prev`` (the results of an earlier
    call with ``track``) continues its near-edge records and counters;
    ``band_eps`` (with ``track``) marks splats whose band op's coordinate lies
    within that distance of a band edge as of unsure colour.  Returns one
    ``TargetResult`` per target.
    """
    keep = _Keep()
    s = _system(system, keep)
    c = _chain(chain, keep, band_eps if track else 0.0)
    results = []
    arr = (_Target * max(len(targets), 1))()
    for j, t in enumerate(targets):
        buf = prev[j].buf if prev is not None else (
            bufs[j] if bufs is not None else alloc_target_buffer(t))
        ts, tr = _target(t, keep, buf, margin_px, track, prev[j] if prev is not None else None)
        arr[j] = ts
        results.append(tr)
    r = _run(seed, system_id, point_begin, n_points, step_begin, iters, burn_in, reuse,
             start, keep)
    rc = lib().orc_render(ctypes.byref(s), ctypes.byref(c), arr, len(targets), ctypes.byref(r))
    if rc != 0:
        raise ValueError("oracle rejected the system")
    for j, tr in enumerate(results):
        tr.n_splat, tr.n_discard, tr.n_amb = arr[j].n_splat, arr[j].n_discard, arr[j].n_amb
    return results


def trace(system, chain, ids, *, iters, seed=0, system_id=0, point_begin=0, step_begin=0,
          burn_in=0, reuse=False, start=None):
    """Per-step map index k [n, steps], point p [n, steps, 3] and, per SPLAT op,
    the chain input q [n, steps, n_splat, 4] (x, y, z, alive)."""
    keep = _Keep()
    s = _system(system, keep)
    c = _chain(chain, keep)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    n_pts = int(ids.shape[0]) if start is None else int(np.asarray(start).shape[0])
    r = _run(seed, system_id, point_begin, n_pts, step_begin, iters, burn_in, reuse, start, keep)
    steps = iters - step_begin
    n_sp = max(1, sum(1 for o in chain if o.kind == "splat"))
    k = np.zeros((len(ids), steps), dtype=np.int32)
    p = np.zeros((len(ids), steps, 3), dtype=np.float32)
    q = np.zeros((len(ids), steps, n_sp, 4), dtype=np.float32)
    rc = lib().orc_trace(ctypes.byref(s), ctypes.byref(c), ctypes.byref(r), len(ids),
                         _ptr(ids, ctypes.c_uint32), _ptr(k, ctypes.c_int32),
                         _ptr(p, ctypes.c_float), _ptr(q, ctypes.c_float), n_sp)
    if rc != 0:
        raise ValueError("oracle rejected the system")
    return k, p, q


def pointcloud_generate(system, n, iters, *, seed=0, system_id=0):
    keep = _Keep()
    s = _system(system, keep)
    xyz = np.zeros((n, 3), dtype=np.float32)
    fn = np.zeros(n, dtype=np.uint8)
    rc = lib().orc_pointcloud_generate(ctypes.byref(s), seed, system_id, n, iters,
                                       _ptr(xyz, ctypes.c_float), _ptr(fn, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("oracle rejected the system")
    return xyz, fn


def render_points(xyz, fn, chain, targets, *, margin_px=0.0, track=False, bufs=None, prev=None,
                  band_eps=0.0):
    """Streams stored points (xyz [n][3], colour index fn [n]) once through the
    chain; targets, ``bufs``, ``track``, ``prev`` and ``band_eps`` as in
    ``render``."""
    keep = _Keep()
    c = _chain(chain, keep, band_eps if track else 0.0)
    xyz = keep(np.ascontiguousarray(xyz, dtype=np.float32))
    fn = keep(np.ascontiguousarray(fn, dtype=np.uint8))
    results = []
    arr = (_Target * max(len(targets), 1))()
    for j, t in enumerate(targets):
        buf = prev[j].buf if prev is not None else (
            bufs[j] if bufs is not None else alloc_target_buffer(t))
        ts, tr = _target(t, keep, buf, margin_px, track, prev[j] if prev is not None else None)
        arr[j] = ts
        results.append(tr)
    lib().orc_render_points(_ptr(xyz, ctypes.c_float), _ptr(fn, ctypes.c_uint8),
                            xyz.shape[0], ctypes.byref(c), arr, len(targets))
    for j, tr in enumerate(results):
        tr.n_splat, tr.n_discard, tr.n_amb = arr[j].n_splat, arr[j].n_discard, arr[j].n_amb
    return results


def tonemap(target, buf, *, gamma=2.2, brightness=1.0, a_max=0.0, background=0, eps=1e-3):
    """Density-estimation display of a layer: returns (rgba8 u32 [H][W],
    near-boundary component mask u8 [H][W], density maximum used)."""
    keep = _Keep()
    buf = keep(np.ascontiguousarray(buf))
    ts, _ = _target(target, keep, buf, 0.0, False)
    out = np.zeros((target.H, target.W), dtype=np.uint32)
    near = np.zeros((target.H, target.W), dtype=np.uint8)
    L = lib()
    used = float(a_max) if a_max > 0 else (
        0.0 if target.kind == "depth_u64" else float(L.orc_density_max(ctypes.byref(ts))))
    rc = L.orc_tonemap(ctypes.byref(ts), gamma, brightness, a_max, background,
                       _ptr(out, ctypes.c_uint32), _ptr(near, ctypes.c_uint8), eps)
    if rc != 0:
        raise ValueError("invalid tone-mapping parameters")
    return out, near, used
