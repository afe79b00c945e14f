/*
 * cfs_oracle.c -- plain, slow, single-threaded CPU oracle of the chaos-game
 * hot path of "Composable function systems as a general-purpose rendering
 * framework" (Schloss).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or
 * call this file: only the tests, the smoke check and the timed CPU baseline
 * of bench.py use it.  It shares no code, header, table or constant generator
 * with the CUDA library; the two agree only because both follow the same
 * written rules, listed below with the passage of the paper each one follows.
 *
 * Precision: FP32 on the per-point path, every fused multiply-add written out
 * as fmaf(); the file is compiled with -ffp-contract=off so the compiler adds
 * no fusion of its own.  Doubles appear only where the rules below say so
 * (threshold table, rotation/derived constants).
 *
 * Rules (the paper is silent on most of these; the readings are the ones the
 * design document lists):
 *  - Chaos game (Section 1; Section 3): a point starts at a random position,
 *    every step picks one map at random, applies it, then (after burn-in)
 *    a COPY of the point goes through the transform chain and is splatted
 *    (Fig. 2B).  With `reuse` set the chain's result replaces the point
 *    (Fig. 2C).
 *  - Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *    (seed low 32 bits, seed high 32 bits).  Start point: counter
 *    (i, 0, system, 1), coordinate j = (word_j >> 8) * 2^-24.  Step n: counter
 *    (i, n >> 2, system, 0), word n & 3.
 *  - Map choice: with S_k the running sum of probabilities divided by their
 *    total (double), T_k = floor(S_k * 2^32) (k < n-1) and the chosen map is
 *    k = #{ j < n-1 : w >= T_j }  (thresholds >= 2^32 never count).
 *  - Colour (Section 1: the colour tells which function moved the point last): the index k of the
 *    last generator map applied.
 *  - Duplication (Section 3.2: the stars are generated on the fly by a PRNG
 *    scheme): STARS moves the copy onto one of n small copies of the
 *    primitive.  The star is j = floor(w_aux * n / 2^32) with w_aux word
 *    n & 3 of Philox block (i, n >> 2, system, 2); star j's centre and size
 *    come from Philox block (j, 0, 0, 7), u_c = (word_c >> 8) * 2^-24:
 *    centre (x0 + (x1 - x0) u_0, y0 + (y1 - y0) u_1, z0 + (z1 - z0) u_2),
 *    size s0 + (s1 - s0) u_3 (each a single fma); q' = centre + size * q.
 *  - Splat (Section 1: the point lands in the pixel it falls in): ix = floor((x - x0) * sx)
 *    with sx = W / (x1 - x0) in FP32, valid for x0 <= x <= x1, the last bin
 *    closed (ix = min(ix, W-1)); outside or non-finite points are counted as
 *    discarded.  Rows likewise from y.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cfs_oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon et al. 2011,
 * Section 4: multipliers 0xD2511F53, 0xCD9E8D57; key schedule Weyl constants
 * 0x9E3779B9, 0xBB67AE85; ten rounds).                                      */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                            uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------ */
/* Threshold table and map choice (each step draws a function at random,
 * Section 3; per-map probabilities as the workloads specify).              */
/* ------------------------------------------------------------------------ */
int orc_thresholds(int n_maps, const double* prob, uint64_t* T)
{
    if (n_maps < 1 || n_maps > ORC_MAX_MAPS) return -1;
    double total = 0.0;
    for (int j = 0; j < n_maps; ++j) {
        if (!(prob[j] >= 0.0) || isinf(prob[j])) return -1;
        total += prob[j];
    }
    if (!(total > 0.0) || isinf(total)) return -1;
    double running = 0.0;
    for (int k = 0; k < n_maps - 1; ++k) {
        running += prob[k];
        double s = running / total;
        double t = floor(s * 4294967296.0);
        if (t < 0.0) t = 0.0;
        T[k] = (uint64_t)t; /* may be 2^32 (or more, by rounding): never reached */
    }
    return 0;
}

int orc_choose(uint32_t w, int n_maps, const uint64_t* T)
{
    int k = 0;
    for (int j = 0; j < n_maps - 1; ++j)
        if ((uint64_t)w >= T[j]) k += 1;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Generator maps.                                                           */
/* ------------------------------------------------------------------------ */
static const float ORC_PI_F = 3.14159265358979323846f;
static const float ORC_TWO_PI_F = 6.28318530717958647692f;

/* Affine map (Section 1's square primitive: four maps f_1..f_4).
 * 2D params (a, b, c, d, e, f): x' = a x + b y + e, y' = c x + d y + f.
 * 3D params: row-major A (9) then b (3).  Evaluation order: innermost term
 * first, x' = fma(a, x, fma(b, y, e)). */
static void affine2(const float* m, float* p)
{
    float x = p[0], y = p[1];
    p[0] = fmaf(m[0], x, fmaf(m[1], y, m[4]));
    p[1] = fmaf(m[2], x, fmaf(m[3], y, m[5]));
}

static void affine3(const float* m, float* p)
{
    float x = p[0], y = p[1], z = p[2];
    p[0] = fmaf(m[0], x, fmaf(m[1], y, fmaf(m[2], z, m[9])));
    p[1] = fmaf(m[3], x, fmaf(m[4], y, fmaf(m[5], z, m[10])));
    p[2] = fmaf(m[6], x, fmaf(m[7], y, fmaf(m[8], z, m[11])));
}

/* Non-affine circle IFS, Eq. 1, read as: r = |p|, theta = atan2(y, x) taken
 * into [0, 2 pi), theta2 = pi (r + f_id), r2 = sqrt(theta / 2 pi),
 * p' = r2 (cos theta2, sin theta2).  (The printed equation uses atan(y/x) and
 * r^2 in the last two lines; the reading uses atan2 and r2, which is what
 * maps the disk onto its upper (f_id = 0) or lower (f_id = 1) half.) */
static void circle_map(float fid, float* p)
{
    float x = p[0], y = p[1];
    float r = sqrtf(fmaf(x, x, y * y));
    float th = atan2f(y, x);
    if (th < 0.0f) th = th + ORC_TWO_PI_F;
    float th2 = ORC_PI_F * (r + fid);
    float r2 = sqrtf(th / ORC_TWO_PI_F);
    p[0] = r2 * cosf(th2);
    p[1] = r2 * sinf(th2);
}

static void apply_map(const orc_system* s, int k, float* p)
{
    const float* m = s->prm + 12 * k;
    switch (s->kind[k]) {
    case ORC_MAP_AFFINE:
        if (s->dim == 2) affine2(m, p); else affine3(m, p);
        break;
    case ORC_MAP_CIRCLE:
        circle_map(m[0], p);
        break;
    default:
        break;
    }
}

/* ------------------------------------------------------------------------ */
/* Transform chain (Section 3: a human-readable spatial function applied to a
 * copy of the point, Fig. 1 and Fig. 2B; Eq. 2 stretch).  Each op reads its
 * parameters from 16 floats.  Rotation-type ops are turned into affine
 * parameters here with double-precision cos/sin rounded to float.          */
/* ------------------------------------------------------------------------ */
static void derive_affine(int op, const float* v, float* m /* 12 */)
{
    memset(m, 0, 12 * sizeof(float));
    if (op == ORC_OP_ROTATE2) {
        float c = (float)cos((double)v[0]), s = (float)sin((double)v[0]);
        m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
    } else if (op == ORC_OP_ROTATE3) {
        /* rotation about axis v[1] (0 = x, 1 = y, 2 = z) by angle v[0] */
        float c = (float)cos((double)v[0]), s = (float)sin((double)v[0]);
        int axis = (int)v[1];
        float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        if (axis == 0) { R[4] = c; R[5] = -s; R[7] = s; R[8] = c; }
        else if (axis == 1) { R[0] = c; R[2] = s; R[6] = -s; R[8] = c; }
        else { R[0] = c; R[1] = -s; R[3] = s; R[4] = c; }
        memcpy(m, R, sizeof(R));
    } else if (op == ORC_OP_TRANSLATE3) {
        m[0] = 1; m[4] = 1; m[8] = 1; m[9] = v[0]; m[10] = v[1]; m[11] = v[2];
    }
}

/* per-step context of the stochastic and recolouring ops */
typedef struct {
    uint64_t seed;   /* Philox key of the render */
    uint32_t aux;    /* word n & 3 of block (i, n >> 2, system, 2) */
    int* k;          /* colour index of the branch (BANDS changes it) */
    float band_eps;  /* tolerance of a band op's coordinate (0: not tracked) */
    int* k_unsure;   /* set when a band op's coordinate lies within band_eps
                        of a band edge: another platform may pick the other band */
} orc_opctx;

static float unit24(uint32_t w) { return (float)(w >> 8) * 0x1.0p-24f; }

/* Applies op `op` to q; returns 0 when the op discards the point. */
static int apply_op(int op, const float* v, float* q, const orc_opctx* cx)
{
    float x = q[0], y = q[1], z = q[2];
    switch (op) {
    case ORC_OP_STARS: {
        uint32_t n = (uint32_t)v[0];
        uint32_t j = (uint32_t)(((uint64_t)cx->aux * (uint64_t)n) >> 32);
        uint32_t ctr[4] = {j, 0u, 0u, 7u};
        uint32_t key[2] = {(uint32_t)cx->seed, (uint32_t)(cx->seed >> 32)};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        float cxs = fmaf(v[2] - v[1], unit24(r[0]), v[1]);
        float cys = fmaf(v[4] - v[3], unit24(r[1]), v[3]);
        float czs = fmaf(v[6] - v[5], unit24(r[2]), v[5]);
        float sz = fmaf(v[8] - v[7], unit24(r[3]), v[7]);
        q[0] = fmaf(sz, x, cxs);
        q[1] = fmaf(sz, y, cys);
        q[2] = fmaf(sz, z, czs);
        return 1;
    }
    case ORC_OP_HEMISPHERE: {
        /* the disk seen as the front (z <= 0) half of a sphere of radius R */
        float r2 = fmaf(x, x, y * y);
        float h = sqrtf(fmaxf(0.0f, 1.0f - r2));
        q[0] = v[0] * x;
        q[1] = v[0] * y;
        q[2] = -(v[0] * h);
        return 1;
    }
    case ORC_OP_BANDS: {
        /* colour = base + (floor(freq * coord + phase) mod n) */
        int axis = (int)v[0], nb = (int)v[3], base = (int)v[4];
        float t = fmaf(v[1], q[axis], v[2]);
        int m = 0;
        if (isfinite(t) && fabsf(t) < 1.0e9f) {
            long b = (long)floorf(t);
            m = (int)(((b % nb) + nb) % nb);
            if (cx->band_eps > 0.0f && v[1] != 0.0f) {
                /* the band the coordinate reaches when it moves by band_eps */
                double e = fabs((double)v[1]) * (double)cx->band_eps;
                if (floor((double)t - e) != floor((double)t + e)) *cx->k_unsure = 1;
            }
        }
        *cx->k = base + m;
        return 1;
    }
    case ORC_OP_AFFINE2: affine2(v, q); return 1;
    case ORC_OP_AFFINE3: affine3(v, q); return 1;
    case ORC_OP_ROTATE2: { float m[12]; derive_affine(op, v, m); affine2(m, q); return 1; }
    case ORC_OP_ROTATE3:
    case ORC_OP_TRANSLATE3: { float m[12]; derive_affine(op, v, m); affine3(m, q); return 1; }
    case ORC_OP_SWIRL: {
        /* swirl of the fractal-flame variations (Draves & Reckase):
         * (x sin r^2 - y cos r^2, x cos r^2 + y sin r^2) */
        float r2 = fmaf(x, x, y * y);
        float s = sinf(r2), c = cosf(r2);
        q[0] = fmaf(x, s, -(y * c));
        q[1] = fmaf(x, c, y * s);
        return 1;
    }
    case ORC_OP_SINUSOIDAL:
        q[0] = sinf(x); q[1] = sinf(y);
        return 1;
    case ORC_OP_SINUSOIDAL3:
        q[0] = sinf(x); q[1] = sinf(y); q[2] = sinf(z);
        return 1;
    case ORC_OP_STRETCH:
        /* Eq. 2: x2 = 2 x, y2 = y - cos(x) */
        q[0] = 2.0f * x;
        q[1] = y - cosf(x);
        return 1;
    case ORC_OP_TORUS: {
        /* (u, v) in [0,1]^2 -> torus with radii R = v[0], r = v[1] */
        float a = ORC_TWO_PI_F * x, b = ORC_TWO_PI_F * y;
        float ca = cosf(a), sa = sinf(a), cb = cosf(b), sb = sinf(b);
        float w = fmaf(v[1], cb, v[0]);
        q[0] = w * ca;
        q[1] = w * sa;
        q[2] = v[1] * sb;
        return 1;
    }
    case ORC_OP_PERSPECTIVE: {
        /* pinhole: (f x / z, f y / z, z); z must exceed the near plane v[1] */
        if (!(z > v[1])) return 0;
        float inv = 1.0f / z;
        q[0] = (v[0] * x) * inv;
        q[1] = (v[0] * y) * inv;
        return 1;
    }
    case ORC_OP_TWIST_Z: {
        float ang = v[0] * z;
        float c = cosf(ang), s = sinf(ang);
        q[0] = fmaf(x, c, -(y * s));
        q[1] = fmaf(x, s, y * c);
        return 1;
    }
    case ORC_OP_BEND: {
        /* bend about the y axis with curvature beta = v[0] (Barr 1984) */
        float invb = 1.0f / v[0];
        float t = v[0] * x;
        float s = sinf(t), c = cosf(t);
        float d = invb - z;
        q[0] = s * d;
        q[2] = invb - c * d;
        return 1;
    }
    case ORC_OP_INVERSION: {
        /* sphere inversion about centre (v0, v1, v2), radius v3 */
        float dx = x - v[0], dy = y - v[1], dz = z - v[2];
        float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (!(d2 >= 1e-12f)) return 0;
        float s = (v[3] * v[3]) / d2;
        q[0] = fmaf(s, dx, v[0]);
        q[1] = fmaf(s, dy, v[1]);
        q[2] = fmaf(s, dz, v[2]);
        return 1;
    }
    default:
        return 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Splatting.                                                                */
/* ------------------------------------------------------------------------ */
static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* bin of coordinate u along an axis of n bins over [lo, hi]; -1 = outside */
static int bin_of(float u, float lo, float hi, float scale, int n)
{
    if (!(u >= lo && u <= hi)) return -1;
    int b = (int)floorf((u - lo) * scale);
    if (b > n - 1) b = n - 1;
    return b;
}

/* same rule applied to a pixel-space coordinate (for the ambiguity bound) */
static int bin_of_px(double upx, int n)
{
    if (!(upx >= 0.0 && upx <= (double)n)) return -1;
    int b = (int)floor(upx);
    if (b > n - 1) b = n - 1;
    return b;
}

/* Near-edge bookkeeping of one candidate splat (depth z, packed colour col)
 * at pixel pix, for the depth-parity bounds: zlo = lowest depth of any
 * candidate (sure or near-edge), zhi = lowest depth of a sure splat, klo =
 * lowest key (depth bits << 32 | colour, the buffer's own order) of any
 * candidate, zalt = lowest depth of a candidate whose colour differs from
 * klo's or is unsure (a band edge within tolerance).  zalt follows from the
 * rule that klo's depth is the smallest depth seen: when a new lowest key of
 * another colour arrives, the old lowest depth becomes the lowest depth of
 * another colour. */
static void note_candidate(orc_target* t, size_t pix, float z, uint32_t col, int sure,
                           int unsure)
{
    if (t->zlo && z < t->zlo[pix]) t->zlo[pix] = z;
    if (sure && t->zhi && z < t->zhi[pix]) t->zhi[pix] = z;
    if (t->klo && t->zalt) {
        uint64_t key = ((uint64_t)fbits(z) << 32) | (uint64_t)col;
        uint64_t cur = t->klo[pix];
        if (key < cur) {
            if (cur != ~(uint64_t)0 && (uint32_t)cur != col) {
                uint32_t zb = (uint32_t)(cur >> 32);
                float zc;
                memcpy(&zc, &zb, 4);
                t->zalt[pix] = zc;
            }
            t->klo[pix] = key;
            if (unsure) t->zalt[pix] = z;
        } else if (((uint32_t)cur != col || unsure) && z < t->zalt[pix]) {
            t->zalt[pix] = z;
        }
    }
}

static void splat(orc_target* t, const float* q, int alive, int k, int unsure)
{
    if (!alive) { t->n_discard++; return; }
    float sx = (float)t->W / (t->x1 - t->x0);
    float sy = (float)t->H / (t->y1 - t->y0);
    int ix = bin_of(q[0], t->x0, t->x1, sx, t->W);
    int iy = bin_of(q[1], t->y0, t->y1, sy, t->H);
    uint32_t col = t->kind == ORC_TGT_DEPTH_U64 ? t->palette8[k] : 0u;

    int ambiguous = 0;
    if (t->amb && t->margin_px > 0.0f && isfinite(q[0]) && isfinite(q[1])) {
        /* Near-edge accounting for the parity bound: the bins the point could
         * reach if its pixel coordinate (computed as the bin rule computes it)
         * moved by up to margin_px (< 1 px, so at most one neighbour per
         * axis).  Every such bin inside the view gets one unit of slack and
         * the point as a possible (not sure) depth candidate. */
        double ux = (double)((q[0] - t->x0) * sx), uy = (double)((q[1] - t->y0) * sy);
        double m = t->margin_px;
        int xs[2] = {bin_of_px(ux - m, t->W), bin_of_px(ux + m, t->W)};
        int ys[2] = {bin_of_px(uy - m, t->H), bin_of_px(uy + m, t->H)};
        ambiguous = xs[0] != xs[1] || ys[0] != ys[1];
        if (ambiguous) {
            t->n_amb++;
            for (int a = 0; a < 2; ++a) {
                if (a == 1 && xs[1] == xs[0]) continue;
                for (int b = 0; b < 2; ++b) {
                    if (b == 1 && ys[1] == ys[0]) continue;
                    if (xs[a] < 0 || ys[b] < 0) continue;
                    size_t pix = (size_t)ys[b] * t->W + xs[a];
                    t->amb[pix] += 1;
                    note_candidate(t, pix, q[2], col, 0, unsure);
                }
            }
        }
    }
    if (ix < 0 || iy < 0) { t->n_discard++; return; }
    size_t pix = (size_t)iy * t->W + ix;
    if (!ambiguous) {
        note_candidate(t, pix, q[2], col, 1, unsure);
        /* a splat of unsure colour may land in another channel of its bin */
        if (unsure && t->amb) t->amb[pix] += 1;
    }
    t->n_splat++;
    if (t->kind == ORC_TGT_HIST_U32) {
        uint32_t* h = (uint32_t*)t->buf;
        int ch = k % t->C;
        h[(size_t)ch * t->W * t->H + pix] += 1;
    } else if (t->kind == ORC_TGT_RGBA_F32) {
        float* img = (float*)t->buf;
        const float* col = t->palette + 4 * k;
        for (int c = 0; c < 4; ++c) img[4 * pix + c] += col[c];
    } else if (t->kind == ORC_TGT_DEPTH_U64) {
        uint64_t* d = (uint64_t*)t->buf;
        uint64_t key = ((uint64_t)fbits(q[2]) << 32) | (uint64_t)t->palette8[k];
        if (key < d[pix]) d[pix] = key;
    }
}

/* Runs the chain on q (a copy of the iterated point, Fig. 2B) and splats at
 * every SPLAT op.  RESET starts a new branch from a fresh copy of p.  A
 * discarding op skips the rest of its branch; that branch's splats count as
 * discarded.  Records q at each SPLAT into rec (4 floats each: x, y, z,
 * alive) when rec is not NULL.  Returns the number of SPLAT ops met. */
static int run_chain(const orc_chain* ch, const float* p, float* q_out, orc_target* tg,
                     int n_tg, int k, int do_splat, float* rec, uint64_t seed, uint32_t aux)
{
    float q[3] = {p[0], p[1], p[2]};
    int alive = 1, n_rec = 0;
    int kc = k;   /* the branch's colour index */
    int unsure = 0;
    orc_opctx cx = {seed, aux, &kc, ch->band_eps, &unsure};
    for (int o = 0; o < ch->n_ops; ++o) {
        int op = ch->op[o];
        const float* v = ch->prm + 16 * o;
        if (op == ORC_OP_RESET) {
            q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
            alive = 1;
            kc = k;
            unsure = 0;
        } else if (op == ORC_OP_SPLAT) {
            int ti = (int)v[0];
            if (rec) {
                rec[4 * n_rec + 0] = q[0]; rec[4 * n_rec + 1] = q[1];
                rec[4 * n_rec + 2] = q[2]; rec[4 * n_rec + 3] = (float)alive;
            }
            n_rec++;
            if (do_splat && ti >= 0 && ti < n_tg) splat(&tg[ti], q, alive, kc, unsure);
        } else if (alive) {
            alive = apply_op(op, v, q, &cx);
        }
    }
    if (q_out) { q_out[0] = q[0]; q_out[1] = q[1]; q_out[2] = q[2]; }
    return alive;
}

static void start_point(uint64_t seed, uint32_t sys_id, uint32_t i, int dim, float* p)
{
    uint32_t ctr[4] = {i, 0u, sys_id, 1u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    p[0] = (float)(r[0] >> 8) * 0x1.0p-24f;
    p[1] = (float)(r[1] >> 8) * 0x1.0p-24f;
    p[2] = dim == 3 ? (float)(r[2] >> 8) * 0x1.0p-24f : 0.0f;
}

/* ------------------------------------------------------------------------ */
/* The chaos game (Section 1 and Section 3), one point after another.       */
/* ------------------------------------------------------------------------ */
static int chain_has_aux(const orc_chain* ch)
{
    for (int o = 0; o < ch->n_ops; ++o)
        if (ch->op[o] == ORC_OP_STARS) return 1;
    return 0;
}

int orc_render(const orc_system* sys, const orc_chain* ch, orc_target* tg, int n_tg,
               const orc_run* run)
{
    uint64_t T[ORC_MAX_MAPS];
    if (orc_thresholds(sys->n_maps, sys->prob, T) != 0) return -1;
    int has_aux = chain_has_aux(ch);
    for (uint32_t j = 0; j < run->n_points; ++j) {
        uint32_t i = run->point_begin + j;
        float p[3];
        if (run->start) {
            for (int d = 0; d < 3; ++d) p[d] = d < sys->dim ? run->start[(size_t)j * 3 + d] : 0.0f;
        } else {
            start_point(run->seed, run->system_id, i, sys->dim, p);
        }
        for (uint32_t n = run->step_begin; n < run->iters; ++n) {
            uint32_t w = philox_word(run->seed, i, n >> 2, run->system_id, 0u, (int)(n & 3u));
            int k = orc_choose(w, sys->n_maps, T);
            apply_map(sys, k, p);
            int live = n >= run->burn_in;
            uint32_t aux = has_aux ? philox_word(run->seed, i, n >> 2, run->system_id, 2u,
                                                 (int)(n & 3u)) : 0u;
            if (run->reuse) {
                /* Fig. 2C: the transformed point is the one iterated on */
                float q[3];
                if (run_chain(ch, p, q, tg, n_tg, k, live, NULL, run->seed, aux)) {
                    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
                }
            } else if (live) {
                run_chain(ch, p, NULL, tg, n_tg, k, 1, NULL, run->seed, aux);
            }
        }
    }
    return 0;
}

/* Per-step record of chosen map, iterated point and the chain's splat inputs
 * for the listed points; the same rules as orc_render. */
int orc_trace(const orc_system* sys, const orc_chain* ch, const orc_run* run,
              uint32_t n_ids, const uint32_t* ids, int32_t* k_out, float* p_out,
              float* q_out, int n_splat_ops)
{
    uint64_t T[ORC_MAX_MAPS];
    if (orc_thresholds(sys->n_maps, sys->prob, T) != 0) return -1;
    uint32_t n_steps = run->iters - run->step_begin;
    int has_aux = chain_has_aux(ch);
    for (uint32_t j = 0; j < n_ids; ++j) {
        uint32_t i = ids[j];
        float p[3];
        if (run->start) {
            uint32_t local = i - run->point_begin;
            for (int d = 0; d < 3; ++d) p[d] = d < sys->dim ? run->start[(size_t)local * 3 + d] : 0.0f;
        } else {
            start_point(run->seed, run->system_id, i, sys->dim, p);
        }
        for (uint32_t n = run->step_begin; n < run->iters; ++n) {
            size_t s = (size_t)j * n_steps + (n - run->step_begin);
            uint32_t w = philox_word(run->seed, i, n >> 2, run->system_id, 0u, (int)(n & 3u));
            int k = orc_choose(w, sys->n_maps, T);
            apply_map(sys, k, p);
            float* rec = q_out ? q_out + s * (size_t)n_splat_ops * 4 : NULL;
            float qq[3];
            uint32_t aux = has_aux ? philox_word(run->seed, i, n >> 2, run->system_id, 2u,
                                                 (int)(n & 3u)) : 0u;
            int alive = run_chain(ch, p, qq, NULL, 0, k, 0, rec, run->seed, aux);
            if (run->reuse && alive) { p[0] = qq[0]; p[1] = qq[1]; p[2] = qq[2]; }
            k_out[s] = k;
            p_out[3 * s + 0] = p[0]; p_out[3 * s + 1] = p[1]; p_out[3 * s + 2] = p[2];
        }
    }
    return 0;
}

/* Stored point cloud (Section 3: the staged alternative that keeps every point, then transforms it):
 * iterate each point `iters` steps and keep its final position and the index
 * of the last map applied. */
int orc_pointcloud_generate(const orc_system* sys, uint64_t seed, uint32_t system_id,
                            uint32_t n, uint32_t iters, float* xyz, uint8_t* fn)
{
    uint64_t T[ORC_MAX_MAPS];
    if (orc_thresholds(sys->n_maps, sys->prob, T) != 0) return -1;
    for (uint32_t i = 0; i < n; ++i) {
        float p[3];
        int k = 0;
        start_point(seed, system_id, i, sys->dim, p);
        for (uint32_t s = 0; s < iters; ++s) {
            uint32_t w = philox_word(seed, i, s >> 2, system_id, 0u, (int)(s & 3u));
            k = orc_choose(w, sys->n_maps, T);
            apply_map(sys, k, p);
        }
        xyz[3 * (size_t)i + 0] = p[0];
        xyz[3 * (size_t)i + 1] = p[1];
        xyz[3 * (size_t)i + 2] = p[2];
        fn[i] = (uint8_t)k;
    }
    return 0;
}

/* Streams a stored cloud through the chain and splats each point once. */
int orc_render_points(const float* xyz, const uint8_t* fn, uint32_t n, const orc_chain* ch,
                      orc_target* tg, int n_tg)
{
    for (uint32_t i = 0; i < n; ++i) {
        float p[3] = {xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2]};
        run_chain(ch, p, NULL, tg, n_tg, fn[i], 1, NULL, 0u, 0u);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Density-estimation display.  The paper names density estimation (fractal
 * flames, caustics) as the output that keeps atomics on the path (Section 4)
 * and leaves its display unspecified; the reading here is the log-density
 * mapping of fractal flames (Draves & Reckase 2003): per pixel
 *   A   = accumulated alpha (the number of splats for palette alpha 1),
 *   S   = accumulated colour,
 *   d   = ln(1 + A) / ln(1 + A_max),   v = brightness * d^(1/gamma),
 *   rgb = clamp(S / A * v),  alpha = clamp(v),
 * each component quantised to 8 bits as (uint)(255 x + 1/2), packed
 * r | g << 8 | b << 16 | a << 24.  Pixels with A = 0 take the background.
 * A histogram layer contributes, per channel c, n_c * palette[c] (products,
 * then sums over c = 0..C-1 in order).  A depth layer is resolved to the
 * colour in the low 32 bits of its key (background where empty).
 * All of it in FP32 (logf, powf, IEEE division), the same precision the
 * device takes the decisions in.  When `near` is given, it receives per
 * pixel a 4-bit mask of the components whose 255 x + 1/2, evaluated in
 * double from the same FP32 inputs, lies within `eps` of an integer (codes
 * another libm may round the other way). */
/* ------------------------------------------------------------------------ */
static void pixel_sums(const orc_target* t, size_t pix, float* s)
{
    if (t->kind == ORC_TGT_RGBA_F32) {
        const float* img = (const float*)t->buf;
        for (int c = 0; c < 4; ++c) s[c] = img[4 * pix + c];
        return;
    }
    const uint32_t* h = (const uint32_t*)t->buf;
    s[0] = s[1] = s[2] = s[3] = 0.0f;
    for (int ch = 0; ch < t->C; ++ch) {
        float n = (float)h[(size_t)ch * t->W * t->H + pix];
        for (int c = 0; c < 4; ++c) {
            float prod = n * t->palette[4 * ch + c];
            s[c] = s[c] + prod;
        }
    }
}

static uint32_t quant8(float x)
{
    if (!(x > 0.0f)) x = 0.0f;
    if (x > 1.0f) x = 1.0f;
    float y = 255.0f * x;
    y = y + 0.5f;
    return (uint32_t)y;
}

static int near_code(float x, double eps)
{
    if (!(x > 0.0f) || x > 1.0f) return 0;
    double y = 255.0 * (double)x + 0.5;
    double fr = y - floor(y);
    return fr < eps || fr > 1.0 - eps;
}

float orc_density_max(const orc_target* t)
{
    float m = 0.0f;
    size_t n = (size_t)t->W * t->H;
    for (size_t pix = 0; pix < n; ++pix) {
        float s[4];
        pixel_sums(t, pix, s);
        if (s[3] > m) m = s[3];
    }
    return m;
}

int orc_tonemap(const orc_target* t, float gamma, float brightness, float a_max,
                uint32_t background, uint32_t* out, uint8_t* near, double eps)
{
    size_t n = (size_t)t->W * t->H;
    if (t->kind == ORC_TGT_DEPTH_U64) {
        const uint64_t* d = (const uint64_t*)t->buf;
        for (size_t pix = 0; pix < n; ++pix) {
            out[pix] = d[pix] == ~(uint64_t)0 ? background : (uint32_t)d[pix];
            if (near) near[pix] = 0;
        }
        return 0;
    }
    if (!(gamma > 0.0f) || !(brightness > 0.0f)) return -1;
    if (!(a_max > 0.0f)) a_max = orc_density_max(t);
    float inv_gamma = 1.0f / gamma;
    float l_max = a_max > 0.0f ? logf(1.0f + a_max) : 1.0f;
    for (size_t pix = 0; pix < n; ++pix) {
        float s[4];
        pixel_sums(t, pix, s);
        if (!(s[3] > 0.0f)) {
            out[pix] = background;
            if (near) near[pix] = 0;
            continue;
        }
        float d = logf(1.0f + s[3]) / l_max;
        float v = brightness * powf(d, inv_gamma);
        float x[4];
        for (int c = 0; c < 3; ++c) {
            float mean = s[c] / s[3];
            x[c] = mean * v;
        }
        x[3] = v;
        uint32_t code = 0;
        uint8_t mask = 0;
        for (int c = 0; c < 4; ++c) {
            code |= quant8(x[c]) << (8 * c);
            if (near_code(x[c], eps)) mask |= (uint8_t)(1u << c);
        }
        out[pix] = code;
        if (near) near[pix] = mask;
    }
    return 0;
}
