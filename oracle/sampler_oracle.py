"""CPU oracle of the learned warm-start sampler (test infrastructure only).

Plain numpy in float64.  Only the tests, ``__graft_entry__.smoke()`` and the
timed CPU baseline may import this module; the CUDA library never does.

What it restates (the paper leaves the initial distribution of the primitive
to future work -- Section 4 suggests deriving it automatically; the sampler
is that idea made concrete):
  * input u in R^64: u[0:2] Gaussian noise, u[2:50] the affine parameters
    (a b c d e f) of up to 8 maps, zero for missing maps, u[50] the frame
    time t, u[51:64] zero;
  * MLP 64 -> 128 -> 128 -> 128 -> 2 with SiLU(x) = x / (1 + e^-x) after the
    first three layers; weights W_l [out, in], biases b_l;
  * precision of the product: weights and activations rounded to BF16
    (round to nearest even from FP32), products accumulated in FP32; the
    oracle evaluates the same rounded operands exactly (float64);
  * sliced-Wasserstein loss of predicted points X [S, N, 2] against target
    points Y [S, N, 2] over projections theta_j = (cos phi_j, sin phi_j):
    L = mean_{s, j} mean_i (sort(X_s theta_j)_i - sort(Y_s theta_j)_i)^2,
    gradient through the sorting permutation (stable sort);
  * Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

D_IN = 64
H = 128
D_OUT = 2
LAYERS = [(H, D_IN), (H, H), (H, H), (D_OUT, H)]


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as
    float32.  NaN stays NaN."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out).astype(np.float32)


def silu(x):
    return x / (1.0 + np.exp(-x))


def silu_grad(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def init_params(seed: int = 0):
    """Uniform +-1/sqrt(fan_in) weights, zero biases (float32 master copy)."""
    rng = np.random.default_rng([seed, 7007])
    params = []
    for (o, i) in LAYERS:
        bound = 1.0 / np.sqrt(i)
        W = rng.uniform(-bound, bound, size=(o, i)).astype(np.float32)
        b = np.zeros(o, dtype=np.float32)
        params.append((W, b))
    return params


def forward(params, U, bf16: bool = True):
    """Returns (Y float64 [B, 2], cache for backward).  With bf16 the
    weights, the input and every hidden activation are BF16-rounded."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = np.asarray(rnd(U), dtype=np.float64)
    cache = {"a": [a], "z": []}
    for l, (W, b) in enumerate(params):
        Wr = np.asarray(rnd(W), dtype=np.float64)
        z = a @ Wr.T + np.asarray(b, dtype=np.float64)
        cache["z"].append(z)
        if l < len(params) - 1:
            h = silu(z)
            a = np.asarray(rnd(h.astype(np.float32)), dtype=np.float64) if bf16 else h
            cache["a"].append(a)
        else:
            a = z
    return a, cache


def backward(params, cache, dY, bf16: bool = True):
    """Gradients of sum(dY * Y) w.r.t. every weight and bias (float64),
    using the forward's (rounded) activations; returns [(dW, db), ...]."""
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    grads = [None] * len(params)
    g = np.asarray(dY, dtype=np.float64)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        a_in = cache["a"][l]
        grads[l] = (g.T @ a_in, g.sum(axis=0))
        if l > 0:
            Wr = np.asarray(rnd(W), dtype=np.float64)
            g = (g @ Wr) * silu_grad(cache["z"][l - 1])
    return grads


def sw_loss_grad(X, Y, phi):
    """Sliced-Wasserstein loss and its gradient w.r.t. X.  X, Y: [S, N, 2];
    phi: [P] projection angles."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    S, N, _ = X.shape
    P = len(phi)
    th = np.stack([np.cos(phi), np.sin(phi)], axis=1)      # [P, 2]
    loss = 0.0
    dX = np.zeros_like(X)
    for s in range(S):
        px = X[s] @ th.T                                    # [N, P]
        py = Y[s] @ th.T
        for j in range(P):
            ox = np.argsort(px[:, j], kind="stable")
            sy = np.sort(py[:, j], kind="stable")
            diff = px[ox, j] - sy                           # i-th smallest vs i-th smallest
            loss += np.mean(diff * diff)
            g = np.zeros(N)
            g[ox] = 2.0 * diff / N
            dX[s] += np.outer(g, th[j])
    scale = 1.0 / (S * P)
    return loss * scale, dX * scale


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (w, m, v) as float64."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1**t)
    vh = v / (1 - b2**t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def make_inputs(noise, sys_params, t):
    """u rows from noise [B, 2], per-row map parameters [B, 48] and t [B]."""
    B = noise.shape[0]
    U = np.zeros((B, D_IN), dtype=np.float32)
    U[:, 0:2] = noise
    U[:, 2:50] = sys_params
    U[:, 50] = t
    return U


def noise(seed: int, n: int, step: int = 0):
    """Gaussian noise of rows 0..n-1: Box-Muller (Box & Muller 1958) on the
    Philox4x32-10 block (row, step, 0, 3) with key (seed lo, seed hi):
    u1 = ((w0 >> 8) + 1/2) 2^-24, u2 = (w1 >> 8) 2^-24,
    (n0, n1) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2)."""
    from oracle import oracle as O
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    out = np.zeros((n, 2))
    for r in range(n):
        w = O.philox([r, step, 0, 3], key)
        u1 = ((int(w[0]) >> 8) + 0.5) * 2.0**-24
        u2 = (int(w[1]) >> 8) * 2.0**-24
        rad = np.sqrt(-2.0 * np.log(u1))
        out[r] = rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)
    return out


def conditioning(maps, t):
    """u[2:51] of a system: a b c d e f of each map (up to 8, zero after),
    then t.  The maps go in canonical order, decreasing |det A| = |a d - b c|
    (float64 from the FP32 parameters), ties by index: an attractor does not
    depend on the order in which its maps are listed."""
    prm = [np.asarray(m, dtype=np.float32).astype(np.float64)[:6] for m in maps[:8]]
    order = sorted(range(len(prm)), key=lambda k: (-abs(prm[k][0] * prm[k][3] -
                                                        prm[k][1] * prm[k][2]), k))
    c = np.zeros(49)
    for q, k in enumerate(order):
        c[6 * q:6 * q + 6] = prm[k]
    c[48] = t
    return c


def start_points(params, maps, t, n, seed):
    """The warm-start points of a system: network(noise, conditioning)."""
    U = np.zeros((n, D_IN), dtype=np.float32)
    U[:, 0:2] = noise(seed, n)
    U[:, 2:51] = conditioning(maps, t)
    Y, _ = forward(params, U, bf16=True)
    return Y
