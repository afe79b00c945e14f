"""Seeded synthetic inputs for the chaos-game hot path.

This module only *describes* inputs -- systems of maps with probabilities,
transform chains, output targets and run sizes -- and draws the random
parameters of the animated and 3D workloads from numpy's seeded generators.
It holds none of the method's arithmetic: iterating, choosing maps,
transforming and splatting live in the CUDA library and, separately, in the
oracle.  Both sides take these descriptions as their input.

Workloads (sizes as the method's evaluation uses them):
  * ``square_render`` -- the square primitive of Section 1 (four half-scale
    maps toward the corners of the unit square, probability 1/4 each),
    2^16 points, 200 steps, burn-in 20, 512x512 four-channel u32 histogram.
  * ``composed_render`` -- square primitive plus a Sierpinski triangle,
    composed with rotation 0.7 rad, swirl and sinusoidal (2D branch, FP32 RGBA
    accumulation) and a torus embedding with perspective (3D branch, packed
    64-bit depth+colour minimum), 2^22 points, 500 steps, 2048x2048.
  * ``animation_frames`` -- 256 frames of 2-8 random contractive affine maps
    interpolated between two keyframes; uneven point counts and resolutions.
  * ``cloud_system`` / ``cloud_chain`` -- a 3D IFS of 8 maps stored as a
    2^26-point cloud and streamed through an 8-transform chain per frame.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

MAX_MAPS = 16


@dataclass(frozen=True)
class Map:
    kind: str                      # "affine" | "circle"
    params: Tuple[float, ...]      # affine 2D: a b c d e f; 3D: A(9) b(3); circle: f_id


@dataclass
class System:
    dim: int
    maps: List[Map]
    probs: List[float]


@dataclass(frozen=True)
class Op:
    kind: str
    params: Tuple[float, ...] = ()


@dataclass
class Target:
    kind: str                                  # "hist_u32" | "rgba_f32" | "depth_u64"
    W: int
    H: int
    C: int = 1
    view: Tuple[float, float, float, float] = (0.0, 1.0, 0.0, 1.0)   # x0 x1 y0 y1
    palette: Optional[np.ndarray] = None       # [n,4] float32 (RGBA)
    palette8: Optional[np.ndarray] = None      # [n] uint32 packed RGBA8 (depth)


@dataclass
class RenderJob:
    """One generator system over a range of global point indices."""
    system: System
    point_begin: int
    n_points: int
    system_id: int = 0


@dataclass
class Workload:
    name: str
    jobs: List[RenderJob]
    chain: List[Op]
    targets: List[Target]
    iters: int
    burn_in: int
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def point_steps(self) -> int:
        return sum(j.n_points for j in self.jobs) * self.iters

    @property
    def splat_steps(self) -> int:
        return sum(j.n_points for j in self.jobs) * (self.iters - self.burn_in)


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
def f32(x) -> float:
    return float(np.float32(x))


def _toward(vx, vy, s=0.5):
    """Affine map p -> s p + (1 - s) v (scale s toward vertex v)."""
    return Map("affine", (f32(s), 0.0, 0.0, f32(s), f32((1 - s) * vx), f32((1 - s) * vy)))


def square_system() -> System:
    """Four half-scale maps toward the corners (0,0), (1,0), (0,1), (1,1)."""
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    return System(2, [_toward(x, y) for x, y in corners], [0.25] * 4)


def sierpinski_system(right_angle: bool = False) -> System:
    """Three half-scale maps toward the triangle's vertices, probability 1/3."""
    if right_angle:
        verts = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0)]
    else:
        verts = [(0.0, 0.0), (1.0, 0.0), (0.5, math.sqrt(3.0) / 2.0)]
    return System(2, [_toward(x, y) for x, y in verts], [1.0 / 3.0] * 3)


def circle_system() -> System:
    """The two non-affine maps of Eq. 1 (f_id = 0 and 1), probability 1/2."""
    return System(2, [Map("circle", (0.0,)), Map("circle", (1.0,))], [0.5, 0.5])


def single_affine_system(a, b, c, d, e, f) -> System:
    return System(2, [Map("affine", tuple(f32(v) for v in (a, b, c, d, e, f)))], [1.0])


def palette_rgba(n: int) -> np.ndarray:
    """Colours with components in {0, 0.5, 1} and alpha 1, so FP32 sums of
    them are exact (and independent of order) while a bin holds < 2^23."""
    base = [(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (1.0, 1.0, 0.0),
            (0.0, 1.0, 1.0), (1.0, 0.0, 1.0), (1.0, 0.5, 0.0), (0.5, 0.0, 1.0),
            (0.5, 1.0, 0.5), (1.0, 0.5, 0.5), (0.5, 0.5, 1.0), (1.0, 1.0, 1.0),
            (0.5, 0.5, 0.0), (0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.5)]
    out = np.zeros((MAX_MAPS, 4), dtype=np.float32)
    for j in range(MAX_MAPS):
        out[j, :3] = base[j % len(base)]
        out[j, 3] = 1.0
    return out[:max(n, 1)] if n < MAX_MAPS else out


def palette_rgba8(n: int) -> np.ndarray:
    """Packed R | G << 8 | B << 16 | A << 24 colours."""
    p = palette_rgba(MAX_MAPS)
    u8 = np.round(p * 255.0).astype(np.uint32)
    packed = u8[:, 0] | (u8[:, 1] << 8) | (u8[:, 2] << 16) | (u8[:, 3] << 24)
    return packed.astype(np.uint32)[:max(n, 1)] if n < MAX_MAPS else packed.astype(np.uint32)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def square_render(n_points: int = 1 << 16, iters: int = 200, burn_in: int = 20,
                  W: int = 512, seed: int = 0) -> Workload:
    t = Target("hist_u32", W, W, 4, (0.0, 1.0, 0.0, 1.0))
    return Workload("square primitive, 2^16 points x 200 steps, 512^2 x 4ch u32",
                    [RenderJob(square_system(), 0, n_points)],
                    [Op("splat", (0,))], [t], iters, burn_in, seed)


def composed_chain(focal: float = 2.0, R: float = 1.0, r: float = 0.35) -> List[Op]:
    """2D branch: rotate 0.7 -> swirl -> sinusoidal -> RGBA splat.
    3D branch (fresh copy of the generator point (u, v)): torus(R, r) ->
    rotate 1.0 rad about x -> z += 3.5 -> perspective(focal) -> depth splat."""
    return [Op("rotate2", (0.7,)), Op("swirl"), Op("sinusoidal"), Op("splat", (0,)),
            Op("reset"), Op("torus", (R, r)), Op("rotate3", (1.0, 0.0)),
            Op("translate3", (0.0, 0.0, 3.5)), Op("perspective", (focal, 1e-3)),
            Op("splat", (1,))]


def composed_targets(W: int = 2048) -> List[Target]:
    view = (-1.0, 1.0, -1.0, 1.0)
    return [Target("rgba_f32", W, W, 4, view, palette=palette_rgba(MAX_MAPS)),
            Target("depth_u64", W, W, 1, view, palette8=palette_rgba8(MAX_MAPS))]


def composed_render(n_points: int = 1 << 22, iters: int = 500, burn_in: int = 20,
                    W: int = 2048, seed: int = 0) -> Workload:
    half = n_points // 2
    jobs = [RenderJob(square_system(), 0, half),
            RenderJob(sierpinski_system(), half, n_points - half)]
    return Workload("composed square+Sierpinski, rotate/swirl/sinusoidal + torus/perspective, "
                    f"{n_points} points x {iters} steps, {W}^2 RGBA f32 + depth u64",
                    jobs, composed_chain(), composed_targets(W), iters, burn_in, seed)


def _rot2(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s], [s, c]])


def _random_affine2(rng) -> Tuple[np.ndarray, np.ndarray]:
    theta = rng.uniform(0.0, 2.0 * math.pi)
    s = rng.uniform(0.3, 0.7, size=2)
    A = _rot2(theta) @ np.diag(s)
    b = rng.uniform(-1.0, 1.0, size=2)
    return A, b


@dataclass
class Frame:
    system: System
    n_points: int
    W: int
    t: float


def animation_frames(n_frames: int = 256, seed: int = 0, min_log2: int = 16,
                     max_log2: int = 22, resolutions=(256, 512, 1024, 2048)) -> List[Frame]:
    """Frames of 2-8 affine maps (singular values U[0.3, 0.7], rotation
    U[0, 2 pi), translation U[-1, 1]^2) interpolated linearly between two
    seeded keyframes at t = f / (n_frames - 1); probabilities proportional to
    |det A| (floored at 1e-6); point counts log-uniform in
    2^min_log2..2^max_log2; resolution uniform over ``resolutions``."""
    frames = []
    for f in range(n_frames):
        rng = np.random.default_rng([seed, 7001, f])
        n_maps = int(rng.integers(2, 9))
        key0 = [_random_affine2(rng) for _ in range(n_maps)]
        key1 = [_random_affine2(rng) for _ in range(n_maps)]
        u = rng.uniform()
        n_points = int(round(2.0 ** (min_log2 + (max_log2 - min_log2) * u)))
        W = int(resolutions[int(rng.integers(0, len(resolutions)))])
        t = f / (n_frames - 1) if n_frames > 1 else 0.0
        maps, probs = [], []
        for (A0, b0), (A1, b1) in zip(key0, key1):
            A = (1 - t) * A0 + t * A1
            b = (1 - t) * b0 + t * b1
            maps.append(Map("affine", tuple(f32(v) for v in (A[0, 0], A[0, 1], A[1, 0], A[1, 1],
                                                              b[0], b[1]))))
            probs.append(max(abs(float(np.linalg.det(A))), 1e-6))
        frames.append(Frame(System(2, maps, probs), n_points, W, t))
    return frames


ANIMATION_VIEW = (-4.8, 4.8, -4.8, 4.8)


def animation_target(W: int) -> Target:
    """Four-channel u32 histogram over [-4.8, 4.8]^2; a contraction with
    ||A|| <= 0.7 and |b| <= sqrt(2) keeps every point within sqrt(2)/0.3."""
    return Target("hist_u32", W, W, 4, ANIMATION_VIEW)


def _random_rotation3(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def cloud_system(seed: int = 0) -> System:
    """3D IFS: 8 maps A = s R (s ~ U[0.35, 0.55], R a uniform random rotation),
    b ~ U[-1, 1]^3, equal probabilities."""
    rng = np.random.default_rng([seed, 7004])
    maps = []
    for _ in range(8):
        A = rng.uniform(0.35, 0.55) * _random_rotation3(rng)
        b = rng.uniform(-1.0, 1.0, size=3)
        maps.append(Map("affine", tuple(f32(v) for v in list(A.reshape(-1)) + list(b))))
    return System(3, maps, [0.125] * 8)


def cloud_chain(frame: int, n_frames: int = 64, seed: int = 0, focal: float = 3.5) -> List[Op]:
    """Twist about z (kappa = 2 pi t), bend (beta = 0.25 + 0.5 t), sphere
    inversion (centre (0, 0, 6), radius 4), sinusoidal, four random affines
    (rotation + translation U[-0.1, 0.1]^3), camera at distance 8 and a
    perspective splat into the depth target; t = frame / (n_frames - 1)."""
    t = frame / (n_frames - 1) if n_frames > 1 else 0.0
    rng = np.random.default_rng([seed, 7005])
    ops = [Op("twist_z", (f32(2 * math.pi * t),)), Op("bend", (f32(0.25 + 0.5 * t),)),
           Op("inversion", (0.0, 0.0, 6.0, 4.0)), Op("sinusoidal3")]
    for _ in range(4):
        R = _random_rotation3(rng)
        b = rng.uniform(-0.1, 0.1, size=3)
        ops.append(Op("affine3", tuple(f32(v) for v in list(R.reshape(-1)) + list(b))))
    ops += [Op("translate3", (0.0, 0.0, 8.0)), Op("perspective", (f32(focal), 1e-3)),
            Op("splat", (0,))]
    return ops


def cloud_target(W: int = 8192) -> Target:
    return Target("depth_u64", W, W, 1, (-1.0, 1.0, -1.0, 1.0), palette8=palette_rgba8(MAX_MAPS))


def uniform_points(n: int, dim: int, seed: int) -> np.ndarray:
    """Seeded uniform points in [0, 1)^dim (FP32), for chains applied to
    stored clouds in tests."""
    rng = np.random.default_rng([seed, 7006])
    return rng.uniform(0.0, 1.0, size=(n, dim)).astype(np.float32)


# ---------------------------------------------------------------------------
# synthetic accumulated layers (inputs of the display, drawn directly: heavy-
# tailed splat counts with empty pixels, as a chaos-game layer has them)
# ---------------------------------------------------------------------------
def synthetic_layer(kind: str, W: int, H: int, C: int = 4, seed: int = 0,
                    empty: float = 0.3) -> np.ndarray:
    """A seeded layer of the given kind: hist_u32 -> uint32 [C, H, W] counts
    (log-normal, a fraction `empty` of pixels zero in every channel);
    rgba_f32 -> float32 [H, W, 4] with alpha an integer count and R, G, B
    multiples of 1/2 in [0, alpha]; depth_u64 -> uint64 [H, W] keys of
    positive depths with random colours, `empty` of them all ones."""
    rng = np.random.default_rng([seed, 7011, W, H])
    zero = rng.random((H, W)) < empty
    if kind == "hist_u32":
        n = np.floor(np.exp(rng.normal(1.5, 1.8, size=(C, H, W)))).astype(np.uint32)
        n[:, zero] = 0
        return n
    if kind == "rgba_f32":
        a = np.floor(np.exp(rng.normal(2.0, 1.8, size=(H, W)))).astype(np.float64)
        a[zero] = 0
        out = np.zeros((H, W, 4), dtype=np.float32)
        for c in range(3):
            out[..., c] = np.floor(rng.random((H, W)) * (2 * a + 1)) / 2
        out[..., 3] = a
        return out
    if kind == "depth_u64":
        z = rng.uniform(0.5, 20.0, size=(H, W)).astype(np.float32)
        col = rng.integers(0, 2**32, size=(H, W), dtype=np.uint64)
        keys = (z.view(np.uint32).astype(np.uint64) << np.uint64(32)) | col
        keys[zero] = np.uint64(0xFFFFFFFFFFFFFFFF)
        return keys
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# scene of many objects from one primitive (Section 3.2): stars, a banded
# planet and its ring, all drawn from the circle IFS of Eq. 1
# ---------------------------------------------------------------------------
SPACE_ASPECT = 16.0 / 9.0
# palette indices: 0-1 the generator maps, 4-7 planet bands, 8 stars, 9 ring
SPACE_STAR_COLOUR, SPACE_RING_COLOUR, SPACE_BAND_BASE = 8, 9, 4


def space_palette8() -> np.ndarray:
    cols = np.zeros((MAX_MAPS, 4), dtype=np.float64)
    cols[:, 3] = 1.0
    cols[0, :3] = (0.5, 0.5, 0.5)
    cols[1, :3] = (0.5, 0.5, 0.5)
    cols[4, :3] = (0.86, 0.62, 0.38)        # planet bands
    cols[5, :3] = (0.72, 0.45, 0.26)
    cols[6, :3] = (0.93, 0.83, 0.66)
    cols[7, :3] = (0.60, 0.36, 0.22)
    cols[8, :3] = (1.0, 1.0, 0.94)          # stars
    cols[9, :3] = (0.78, 0.74, 0.66)        # ring
    u8 = np.round(cols * 255.0).astype(np.uint32)
    return (u8[:, 0] | (u8[:, 1] << 8) | (u8[:, 2] << 16) | (u8[:, 3] << 24)).astype(np.uint32)


def space_chain(n_stars: int = 400, focal: float = 2.0, tilt: float = 1.25) -> List[Op]:
    """Three objects from one copy of the circle primitive's point, each a
    branch into one depth+colour layer: stars (duplication by the auxiliary
    Philox stream) far behind, a planet (the disk as a hemisphere facing the
    camera, banded) at z = 6 and a tilted thin torus as its ring."""
    star = [Op("stars", (float(n_stars), -16.0, 16.0, -9.0, 9.0, 14.0, 20.0, 0.01, 0.04)),
            Op("bands", (0.0, 0.0, 0.0, 1.0, float(SPACE_STAR_COLOUR))),
            Op("perspective", (focal, 0.1)), Op("splat", (0,))]
    planet = [Op("hemisphere", (1.0,)),
              Op("bands", (1.0, 3.0, 0.5, 4.0, float(SPACE_BAND_BASE))),
              Op("rotate3", (0.25, 2.0)), Op("translate3", (0.0, 0.0, 6.0)),
              Op("perspective", (focal, 0.1)), Op("splat", (0,))]
    ring = [Op("torus", (1.8, 0.04)),
            Op("bands", (0.0, 0.0, 0.0, 1.0, float(SPACE_RING_COLOUR))),
            Op("rotate3", (tilt, 0.0)), Op("rotate3", (0.25, 2.0)),
            Op("translate3", (0.0, 0.0, 6.0)),
            Op("perspective", (focal, 0.1)), Op("splat", (0,))]
    return star + [Op("reset")] + planet + [Op("reset")] + ring


def space_target(W: int = 1920, H: int = 1080) -> Target:
    return Target("depth_u64", W, H, 1, (-SPACE_ASPECT, SPACE_ASPECT, -1.0, 1.0),
                  palette8=space_palette8())


def space_render(n_points: int = 1 << 20, iters: int = 200, burn_in: int = 20, W: int = 1920,
                 H: int = 1080, seed: int = 0, n_stars: int = 400) -> Workload:
    """The scene at 1920 x 1080 (packed RGBA8 after the display, as the
    paper's output): every point of the circle IFS draws a star, the planet
    and the ring each step after burn-in."""
    return Workload("space scene: circle IFS -> stars + banded planet + ring, depth layer",
                    [RenderJob(circle_system(), 0, n_points, 0)], space_chain(n_stars),
                    [space_target(W, H)], iters, burn_in, seed)
