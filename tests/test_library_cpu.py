"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every symbol the public header declares, validates arguments, and
its code generator produces programs NVRTC compiles for sm_103a without
register spills."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_02226_gb300 import cfs
from paper_2606_02226_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cfs_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = cfs.lib()
    names = _declared_functions()
    assert "cfs_render" in names and "cfs_compose" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_version_string():
    assert "sm_103a" in cfs.version()


def test_render_arg_bytes():
    # system (848 B), chain constants (2048), four targets (1504), Philox
    # round keys (80) and the launch's pointers and counts
    assert 4400 < cfs.render_arg_bytes() <= 4 * 1024 + 1024


def test_tune_cache_files_need_no_gpu(tmp_path):
    cfs.tune_cache_clear()
    assert cfs.tune_cache_size() == 0
    cfs.tune_cache_load(str(tmp_path / "missing.txt"))       # nothing there: nothing loaded
    good = tmp_path / "cache.txt"
    good.write_text("class|dev|prog|p16.w64x64 chunk=2048,nowin=0\n"
                    "batch|dev|prog|p16.w64x64:3; ilp=2,win=1,words=53248,agg=0,chunk=4096\n")
    cfs.tune_cache_load(str(good))
    assert cfs.tune_cache_size() == 2
    out = tmp_path / "out.txt"
    cfs.tune_cache_save(str(out))
    assert sorted(out.read_text().splitlines()) == sorted(good.read_text().splitlines())
    bad = tmp_path / "bad.txt"
    bad.write_text("no-value-here\n")
    assert _err(lambda: cfs.tune_cache_load(str(bad))) == 1
    cfs.tune_cache_clear()
    assert cfs.tune_cache_size() == 0


def test_fold_linear_runs_one_affine_op():
    # the cloud chain's four affines and camera translation become one op in
    # the generated program; op indices for animation stay the user's
    ops = W.cloud_chain(3)
    t = W.cloud_target(64)
    s = cfs.System(W.cloud_system())
    plain, _ = cfs.codegen_check(s, cfs.Chain(ops, 3), [t], mode=4)
    c = cfs.Chain(ops, 3, fold_linear=True)
    folded, _ = cfs.codegen_check(s, c, [t], mode=4)
    assert plain.count("cfs_affine3(") == 4 and folded.count("cfs_affine3(") == 1
    assert "cfs_translate" not in folded or folded.count("cfs_translate") < plain.count("cfs_translate")
    c.set_params(0, ops[0].params)       # twist, still op 0
    c.set_params(5, ops[5].params)       # an affine inside the folded run
    assert _err(lambda: c.set_params(11, (0.0,))) == 1


def test_device_error_injection_rejects_unknown_bits():
    # validated before any device access
    assert _err(lambda: cfs.debug_raise_device_error(0)) == 1
    assert _err(lambda: cfs.debug_raise_device_error(1 << 7)) == 1


def _err(fn):
    with pytest.raises(cfs.CfsError) as e:
        fn()
    return e.value.status


def test_system_validation():
    ok = W.Map("affine", (0.5, 0, 0, 0.5, 0, 0))
    assert _err(lambda: cfs.System(W.System(2, [ok], [0.0]))) == 1
    assert _err(lambda: cfs.System(W.System(2, [ok, ok], [-1.0, 2.0]))) == 1
    assert _err(lambda: cfs.System(W.System(2, [ok], [float("nan")]))) == 1
    assert _err(lambda: cfs.System(W.System(4, [ok], [1.0]))) == 1
    assert _err(lambda: cfs.System(W.System(2, [ok] * 17, [1.0] * 17))) == 1
    assert _err(lambda: cfs.System(W.System(3, [W.Map("circle", (0.0,))], [1.0]))) == 1
    bad = W.Map("affine", (float("inf"), 0, 0, 0.5, 0, 0))
    assert _err(lambda: cfs.System(W.System(2, [bad], [1.0]))) == 1
    cfs.System(W.System(2, [ok, ok], [0.0, 1.0]))   # zero probabilities are fine


def test_chain_validation():
    assert _err(lambda: cfs.Chain([W.Op("perspective", (1.0, 0.1))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("torus", (1.0, 0.3)), W.Op("torus", (1, 0.3))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("bend", (0.0,))], 3)) == 1
    assert _err(lambda: cfs.Chain([W.Op("rotate3", (0.1, 5.0))], 3)) == 1
    assert _err(lambda: cfs.Chain([W.Op("splat", (7,))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("splat", (0,))] * 33, 2)) == 1
    c = cfs.Chain([W.Op("torus", (1.0, 0.3)), W.Op("perspective", (2.0, 0.1)),
                   W.Op("reset"), W.Op("swirl"), W.Op("splat", (0,))], 2)
    c.set_params(0, (1.0, 0.5))
    assert _err(lambda: c.set_params(9, (0.0,))) == 1
    assert _err(lambda: c.set_params(4, (1.0,))) == 1      # a splat's slot is fixed


def test_render_argument_errors_need_no_gpu():
    s = cfs.System(W.square_system())
    c = cfs.Chain([W.Op("splat", (1,))], 2)
    t = [W.Target("hist_u32", 8, 8, 4)]
    # slot 1 but one target: rejected before anything touches the GPU
    with pytest.raises(cfs.CfsError):
        cfs.codegen_check(s, c, t)
    c3 = cfs.Chain([W.Op("torus", (1.0, 0.3)), W.Op("splat", (0,))], 2)
    with pytest.raises(cfs.CfsError):
        cfs.codegen_check(cfs.System(W.cloud_system()), c3, t)  # 3D system, 2D chain
    cd = cfs.Chain([W.Op("splat", (0,))], 2)
    with pytest.raises(cfs.CfsError):                            # depth needs 3D
        cfs.codegen_check(s, cd, [W.Target("depth_u64", 8, 8, 1)])


def _programs():
    comp = W.composed_render(n_points=16, iters=30, W=64)
    yield "square", W.square_system(), W.square_render().chain, W.square_render().targets
    yield "composed_sq", comp.jobs[0].system, comp.chain, comp.targets
    yield "composed_si", comp.jobs[1].system, comp.chain, comp.targets
    yield "circle", W.circle_system(), [W.Op("stretch"), W.Op("splat", (0,))], \
        [W.Target("hist_u32", 64, 64, 2, (-3, 3, -3, 3))]
    sq = W.square_system()
    mixed = W.System(2, sq.maps[:3] + [W.Map("circle", (1.0,))], [0.25] * 4)
    yield "mixed", mixed, [W.Op("splat", (0,))], [W.Target("hist_u32", 64, 64, 4)]
    yield "cloud", W.cloud_system(), W.cloud_chain(10), [W.cloud_target(64)]
    frames = W.animation_frames(n_frames=3)
    yield "frame", frames[0].system, [W.Op("splat", (0,))], [W.animation_target(256)]


@pytest.mark.parametrize("prog", list(_programs()), ids=lambda p: p[0])
def test_codegen_compiles_without_spills(prog):
    name, sysd, chain, targets = prog
    s = cfs.System(sysd)
    c = cfs.Chain(chain, sysd.dim)
    modes = (0, 1, 2) if name in ("square", "frame", "circle") else (0, 1)
    for mode in modes:
        src, log = cfs.codegen_check(s, c, targets, mode=mode)
        assert "cfs_chain" in src and "cfs_kernels.cuh" in src
        assert "error" not in log.lower()
        spills = [int(m) for m in re.findall(r"(\d+) bytes spill stores", log)]
        if mode == 2:
            # the batch kernel keeps a frame's target geometry live across its
            # loops; at full occupancy a few words of it go to the (L1-cached)
            # stack, which measured faster than fewer resident warps
            assert spills and max(spills) <= 64, log
        else:
            assert spills and max(spills) == 0, log
        regs = [int(m) for m in re.findall(r"Used (\d+) registers", log)]
        assert regs and max(regs) <= 64, log


def test_codegen_is_structural():
    # two systems of the same structure share one program text
    a = cfs.codegen_check(cfs.System(W.square_system()), cfs.Chain([W.Op("splat", (0,))], 2),
                          [W.Target("hist_u32", 8, 8, 4)])[0]
    sq = W.square_system()
    sq.maps[0] = W.Map("affine", (0.1, 0.2, 0.3, 0.4, 0.5, 0.6))
    sq.probs = [0.1, 0.2, 0.3, 0.4]
    b = cfs.codegen_check(cfs.System(sq), cfs.Chain([W.Op("splat", (0,))], 2),
                          [W.Target("hist_u32", 512, 512, 4, (-1, 2, -1, 2))])[0]
    assert a == b


def test_display_argument_errors_need_no_gpu():
    L = cfs.lib()
    arr, _ = cfs.make_targets([W.Target("rgba_f32", 16, 16, 1)], fake_ptr=True)
    p = cfs._display_params(2.2, 1.0, 0.0, 0)

    def call(params, out, amax):
        return L.cfs_tonemap(arr, ctypes.byref(params), out, amax, None)

    assert call(cfs._display_params(0.0, 1.0, 0.0, 0), 1 << 20, 1 << 21) == 1   # gamma
    assert call(cfs._display_params(2.2, -1.0, 0.0, 0), 1 << 20, 1 << 21) == 1  # brightness
    assert call(cfs._display_params(2.2, 1.0, float("nan"), 0), 1 << 20, 1 << 21) == 1
    assert call(p, None, 1 << 21) == 1               # no output
    assert call(p, (1 << 20) + 4, 1 << 21) == 1      # misaligned output
    assert call(p, 256, 1 << 21) == 1                # output overlaps the layer
    assert call(p, 1 << 20, None) == 1               # maximum wanted, nowhere to put it
    assert L.cfs_tonemap(None, ctypes.byref(p), 1 << 20, 1 << 21, None) == 1
    assert L.cfs_batch_display(None, 0, ctypes.byref(p), None, None, None) == 1


def test_new_op_validation_and_codegen():
    ok = cfs.Chain([W.Op("stars", (5.0, -1, 1, -1, 1, 0, 1, 0.1, 0.2)), W.Op("splat", (0,))], 2)
    assert _err(lambda: cfs.Chain([W.Op("stars", (0.0,)), W.Op("splat", (0,))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("stars", (2.5,)), W.Op("splat", (0,))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("bands", (2.0, 1.0, 0.0, 2.0, 0.0))], 2)) == 1  # no z
    assert _err(lambda: cfs.Chain([W.Op("bands", (0.0, 1.0, 0.0, 4.0, 14.0))], 2)) == 1
    assert _err(lambda: cfs.Chain([W.Op("torus", (1.0, 0.2)), W.Op("hemisphere", (1.0,))], 2)) == 1
    c = cfs.Chain([W.Op("bands", (1.0, 1.0, 0.0, 2.0, 0.0)), W.Op("splat", (0,))], 2)
    assert _err(lambda: c.set_params(0, (0.0, 1.0, 0.0, 2.0, 0.0))) == 1      # axis is compiled in
    c.set_params(0, (1.0, 3.0, 0.5, 2.0, 1.0))
    wl = W.space_render(n_points=64, iters=24, W=64, H=36)
    src, log = cfs.codegen_check(cfs.System(wl.jobs[0].system), cfs.Chain(wl.chain, 2),
                                 wl.targets)
    assert "#define CFS_AUX 1" in src and "cfs_hemisphere(" in src
    # the first duplication op reads its per-CTA star table, with the Philox
    # block as the fallback for more stars than the table holds
    assert "#define CFS_STARS_TAB 512" in src and "cfs_chain_prologue" in src
    assert "sm.stars[j_]" in src and "cfs_star_centre(a, j_" in src
    assert "0 bytes spill stores" in log
    two = [W.Op("stars", (8.0, -1.0, 1.0, -1.0, 1.0, 2.0, 3.0, 0.1, 0.2)), W.Op("reset"),
           W.Op("stars", (4.0, -1.0, 1.0, -1.0, 1.0, 2.0, 3.0, 0.1, 0.2)), W.Op("splat", (0,))]
    src3, _ = cfs.codegen_check(cfs.System(W.square_system()), cfs.Chain(two, 2),
                                [W.Target("depth_u64", 8, 8, 1)])
    assert src3.count("sm.stars[j_]") == 1 and "cfs_stars(a, " in src3   # second op: Philox
    src2, _ = cfs.codegen_check(cfs.System(W.square_system()), ok, [W.Target("hist_u32", 8, 8, 4)])
    assert "#define CFS_AUX 1" in src2


# ---------------------------------------------------------------------------
# scribble frontend (Section 3.1): expansion and its errors, no GPU needed
# ---------------------------------------------------------------------------
def _scribble_err(src, poem="p", dim=2):
    with pytest.raises(cfs.CfsError) as e:
        cfs.Chain.from_scribble(src, poem, dim)
    return str(e.value)


def test_scribble_expansion_errors():
    assert "unknown verse" in _scribble_err("__poem p() { @VCALL nope(); }")
    assert "@VCALL" in _scribble_err("__verse v() { } __poem p() { @SCALL v() { } }")
    assert "__split_stanza" in _scribble_err("__stanza s() { qx = 1; } __poem p() { }")
    assert "positional" in _scribble_err("__verse v(a, b) { } __poem p() { @VCALL v(qx); }")
    assert "no keyword" in _scribble_err("__verse v(| float f = 1;) { } "
                                         "__poem p() { @VCALL v(| g = 2;); }")
    assert "literal slot" in _scribble_err("__poem p() { int s = 0; splat(s); }")
    assert "deeper than 32" in _scribble_err("__verse v() { @VCALL v(); } __poem p() { @VCALL v(); }")
    assert "no poem" in _scribble_err("__poem q() { }")
    assert "takes no parameters" in _scribble_err("__poem p(float a) { }")
    assert "duplicate" in _scribble_err("__verse v() { } __verse v() { } __poem p() { }")


def test_scribble_composed_chain_compiles():
    from paper_2606_02226_gb300 import scribbles
    ch = cfs.Chain.from_scribble(scribbles.COMPOSED, "composed", 2)
    assert ch.n_splat == 2
    wl = W.composed_render(n_points=64, iters=24, W=64)
    src, log = cfs.codegen_check(cfs.System(wl.jobs[0].system), ch, wl.targets)
    assert "/* verse flame */" in src and "/* stanza branch */" in src
    assert "float dist = (3.5f);" in src             # keyword default
    assert "0 bytes spill stores" in log
    # a splat slot beyond the targets is rejected before compiling
    with pytest.raises(cfs.CfsError):
        cfs.codegen_check(cfs.System(wl.jobs[0].system), ch, wl.targets[:1])
