"""The seeded synthetic inputs: reproducible from their seeds, and shaped as
the input recipes say (animation frames, the 3D cloud system, the space
scene, the display layers).  No method arithmetic is involved here."""
import math

import numpy as np

from paper_2606_02226_gb300 import workloads as W


def _maps(frame):
    return [np.array(m.params, dtype=np.float64) for m in frame.system.maps]


def test_animation_frames_reproducible_and_in_range():
    a = W.animation_frames(n_frames=24, seed=0)
    b = W.animation_frames(n_frames=24, seed=0)
    c = W.animation_frames(n_frames=24, seed=1)
    assert all(np.array_equal(x, y) for fa, fb in zip(a, b) for x, y in zip(_maps(fa), _maps(fb)))
    assert [f.n_points for f in a] == [f.n_points for f in b]
    assert any(f.n_points != g.n_points for f, g in zip(a, c))
    for f in a:
        assert 2 <= len(f.system.maps) <= 8
        assert 2 ** 16 - 1 <= f.n_points <= 2 ** 22 + 1
        assert f.W in (256, 512, 1024, 2048)
        assert all(p >= 1e-6 for p in f.system.probs)
        for m in _maps(f):
            A, bvec = m[:4].reshape(2, 2), m[4:6]
            # a convex combination of two keyframes with singular values in
            # [0.3, 0.7]: still a contraction with norm <= 0.7
            assert np.linalg.norm(A, 2) <= 0.7 + 1e-6
            assert np.all(np.abs(bvec) <= 1.0 + 1e-6)
    # every attractor fits the view: |x| <= |b| / (1 - ||A||) <= sqrt(2) / 0.3
    assert math.sqrt(2.0) / 0.3 < W.ANIMATION_VIEW[1]


def test_cloud_system_maps_are_scaled_rotations():
    s = W.cloud_system(seed=0)
    assert s.dim == 3 and len(s.maps) == 8 and s.probs == [0.125] * 8
    for m in s.maps:
        p = np.array(m.params, dtype=np.float64)
        A, bvec = p[:9].reshape(3, 3), p[9:12]
        sv = np.linalg.svd(A, compute_uv=False)
        assert 0.35 - 1e-6 <= sv.min() and sv.max() <= 0.55 + 1e-6
        assert sv.max() - sv.min() < 1e-5                  # s R: equal singular values
        assert np.linalg.det(A) > 0                        # a rotation, not a reflection
        assert np.all(np.abs(bvec) <= 1.0 + 1e-6)
    t = W.cloud_system(seed=0)
    assert [m.params for m in s.maps] == [m.params for m in t.maps]


def test_space_scene_recipe():
    wl = W.space_render()
    assert wl.jobs[0].n_points == 1 << 20 and wl.iters == 200 and wl.burn_in == 20
    t = wl.targets[0]
    assert (t.W, t.H, t.kind) == (1920, 1080, "depth_u64")
    stars = [op for op in wl.chain if op.kind == "stars"]
    assert len(stars) == 1 and stars[0].params[0] == 400.0
    assert sum(op.kind == "splat" for op in wl.chain) == 3
    assert sum(op.kind == "reset" for op in wl.chain) == 2


def test_synthetic_layers_reproducible_and_shaped():
    for kind in ("hist_u32", "rgba_f32", "depth_u64"):
        x = W.synthetic_layer(kind, 37, 19, C=3, seed=5)
        y = W.synthetic_layer(kind, 37, 19, C=3, seed=5)
        assert np.array_equal(x, y)
    h = W.synthetic_layer("hist_u32", 64, 32, C=4, seed=1)
    assert h.shape == (4, 32, 64) and h.dtype == np.uint32
    assert 0.2 < float((h.sum(axis=0) == 0).mean()) < 0.4     # about 30% empty pixels
    r = W.synthetic_layer("rgba_f32", 64, 32, seed=1)
    assert np.all(r[..., :3] <= r[..., 3:4]) and np.all(r[..., 3] == np.floor(r[..., 3]))
    d = W.synthetic_layer("depth_u64", 64, 32, seed=1)
    full = d != np.uint64(0xFFFFFFFFFFFFFFFF)
    z = (d[full] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.all((z >= 0.5) & (z <= 20.0))
