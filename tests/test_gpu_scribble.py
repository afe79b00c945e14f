"""GPU tests of the scribble frontend (Section 3.1's verses, stanzas and
poems lowered into the fused chain), through the C ABI: a poem written for
the composed scene renders the op chain's frame bit for bit (and so meets the
op chain's oracle bars), keyword arguments and stanza splits behave as
written, and batches take scribble chains too."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2606_02226_gb300 import scribbles
from paper_2606_02226_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _render(torch, wl, chain):
    from paper_2606_02226_gb300 import cfs
    tensors = [cfs.alloc_target(t) for t in wl.targets]
    disc = torch.zeros(len(wl.targets), dtype=torch.int64, device="cuda")
    for job in wl.jobs:
        cfs.render(cfs.System(job.system), chain, wl.targets, tensors, n_points=job.n_points,
                   iters=wl.iters, burn_in=wl.burn_in, seed=wl.seed, system_id=job.system_id,
                   point_begin=job.point_begin, discards=disc)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in tensors], disc.cpu().numpy()


def test_scribble_composed_scene_equals_op_chain(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    wl = W.composed_render(n_points=5000, iters=60, W=256)
    g_ops, d_ops = _render(torch_cuda, wl, cfs.Chain(wl.chain, 2))
    g_scr, d_scr = _render(torch_cuda, wl, cfs.Chain.from_scribble(scribbles.COMPOSED,
                                                                   "composed", 2))
    assert np.array_equal(g_ops[0], g_scr[0])          # RGBA sums of exact palette values
    assert np.array_equal(g_ops[1], g_scr[1])          # depth keys
    assert np.array_equal(d_ops, d_scr)


def test_scribble_keywords_splits_and_references(torch_cuda):
    """q = ((p.x + 0.5) * 3, p.y * 2 + 0.5): the stanza's code runs around the
    injected block, a keyword overrides its default, the positional
    parameter aliases the caller's variable."""
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    src = r"""
    __verse scale(v | float f = 2.0f;) { v = v * f; }
    __stanza around(| float add = 1.0f;) { qx = qx + add; __split_stanza(); qy = qy + add; }
    __poem test() {
        @SCALL around(| add = 0.5f;) {
            @VCALL scale(qx | f = 3.0f;);
            @VCALL scale(qy);
        }
        splat(0);
    }
    """
    ch = cfs.Chain.from_scribble(src, "test", 2)
    sysd = W.square_system()
    ids = np.arange(32, dtype=np.uint32)
    k, p, q = cfs.trace(cfs.System(sysd), ch, torch.from_numpy(ids.view(np.int32)).cuda(),
                        iters=12)
    p = p.cpu().numpy()
    q = q.cpu().numpy()
    px, py = p[..., 0].astype(np.float32), p[..., 1].astype(np.float32)
    ex = (px + np.float32(0.5)) * np.float32(3.0)
    ey = py * np.float32(2.0) + np.float32(0.5)
    assert np.array_equal(q[..., 0, 0], ex) and np.array_equal(q[..., 0, 1], ey)
    # the generator's own trajectory is the oracle's (copy semantics)
    ko, po, _ = O.trace(sysd, [W.Op("splat", (0,))], ids, iters=12)
    assert np.array_equal(k.cpu().numpy(), ko) and np.array_equal(p, po)


def test_scribble_chain_in_a_batch(torch_cuda):
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    frames = W.animation_frames(n_frames=5, seed=4, min_log2=9, max_log2=11, resolutions=(64,))
    src = r"""
    __verse shear(| float s = 0.25f;) { affine2(1.0f, s, 0.0f, 1.0f, 0.0f, 0.0f); }
    __poem frame() { @VCALL shear(| s = 0.5f;); bands(1, 2.0f, 0.0f, 2, 0); splat(0); }
    """
    ops = [W.Op("affine2", (1.0, 0.5, 0.0, 1.0, 0.0, 0.0)), W.Op("bands", (1.0, 2.0, 0.0, 2.0, 0.0)),
           W.Op("splat", (0,))]
    outs = []
    for chain in (cfs.Chain(ops, 2), cfs.Chain.from_scribble(src, "frame", 2)):
        items, tens, begin = [], [], 0
        for f, fr in enumerate(frames):
            t = W.Target("hist_u32", 64, 64, 2, (-6.0, 6.0, -6.0, 6.0))
            ten = cfs.alloc_target(t)
            items.append((cfs.System(fr.system), fr.n_points, begin, f, [t], [ten]))
            tens.append(ten)
            begin += fr.n_points
        b = cfs.Batch(chain, items, iters=30, burn_in=10, seed=2)
        b.launch(clear=True)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in tens])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)
    # and the op chain's batch is the oracle's
    begin = 0
    for f, fr in enumerate(frames):
        res = O.render(fr.system, ops, [W.Target("hist_u32", 64, 64, 2, (-6.0, 6.0, -6.0, 6.0))],
                       n_points=fr.n_points, iters=30, burn_in=10, seed=2, system_id=f,
                       point_begin=begin)
        assert np.array_equal(outs[1][f].view(np.uint32), res[0].buf)
        begin += fr.n_points


FIG3_STYLE = r"""
// a verse whose default factor (8) every call below overrides
__verse mult_by(v | float factor = 8.0f;) { v = v * factor; }
// a stanza: under the index bound, sum two inputs into `out`, run the
// injected block, add one; its keyword r is passed but never used
__stanza sum_check(a_in, b_in, out | float r = 1.0f;) {
    if (k < limit) {
        out = a_in + b_in;
        __split_stanza();
        out = out + 1.0f;
    }
}
__poem fig3() {
    int stanza_num = STANZA;
    int limit = 2;
    if (stanza_num == 0) {
        @SCALL sum_check(px, py, qx | r = 5.0f;) {
            @VCALL mult_by(qx | factor = 2.0f;);
        }
        if (k < limit) {
            @VCALL mult_by(qx | factor = 0.5f;);
        }
    }
    splat(0);
}
"""


@pytest.mark.parametrize("stanza", [0, 1])
def test_scribble_fig3_semantics(torch_cuda, stanza):
    """The composition Fig. 3 shows (Section 3.1), in this library's dialect:
    a stanza that sums two inputs into an output, has a verse call injected
    at its split point and adds one afterwards, all under an index bound and
    a stanza selector, followed by a second call of the same verse.  The
    verse's default factor 8 is overridden by 2 inside the stanza and by 0.5
    after it; the stanza's keyword r = 5 is unused.  Inputs are the
    generator's point (px, py), the output the copy's x, the index the map
    k (bound 2).  Expected: qx = ((px + py) 2 + 1) 0.5 where the selector is
    0 and k < 2, else qx = px; qy = py throughout."""
    from paper_2606_02226_gb300 import cfs
    torch = torch_cuda
    ch = cfs.Chain.from_scribble(FIG3_STYLE.replace("STANZA", str(stanza)), "fig3", 2)
    sysd = W.square_system()
    ids = np.arange(256, dtype=np.uint32)
    k, p, q = cfs.trace(cfs.System(sysd), ch, torch.from_numpy(ids.view(np.int32)).cuda(),
                        iters=16)
    k, p, q = k.cpu().numpy(), p.cpu().numpy(), q.cpu().numpy()
    px, py = p[..., 0].astype(np.float32), p[..., 1].astype(np.float32)
    f32 = np.float32
    inner = ((px + py) * f32(2.0) + f32(1.0)) * f32(0.5)
    ex = np.where((k < 2) & (stanza == 0), inner, px)
    assert np.array_equal(q[..., 0, 0], ex)
    assert np.array_equal(q[..., 0, 1], py)
    assert ((k < 2).mean() > 0.3) and ((k >= 2).mean() > 0.3)   # both branches taken
    ko, po, _ = O.trace(sysd, [W.Op("splat", (0,))], ids, iters=16)
    assert np.array_equal(k, ko) and np.array_equal(p, po)
