/*
 * cfs_device.cuh -- device helpers of the generated chaos-game kernels.
 *
 * This text is handed to NVRTC together with the generated prelude (the
 * structural #defines and the fused map/chain functions) and cfs_kernels.cuh.
 * It is compiled for sm_103a with --fmad=false: every fused multiply-add is
 * written out with fmaf(), and no other contraction happens, so the FP32
 * results follow the written evaluation order exactly.
 */
#ifndef CFS_DEVICE_CUH
#define CFS_DEVICE_CUH

#include "cfs_args.h"

typedef unsigned int u32;
typedef unsigned long long u64;

#define CFS_TWO_PI_F 6.28318530717958647692f
#define CFS_PI_F 3.14159265358979323846f
#define CFS_INV_2_24 5.9604644775390625e-08f

/* ---- Philox4x32-10 (Salmon et al. 2011): 10 rounds of two 32x32->64
 *      multiplies; the round keys of the launch's seed are precomputed on the
 *      host (key + r * (0x9E3779B9, 0xBB67AE85)) and read from the constant
 *      bank. ------------------------------------------------------------- */
__device__ __forceinline__ uint4 cfs_philox_rk(const unsigned int (&rk)[10][2], u32 c0, u32 c1,
                                               u32 c2, u32 c3)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const u64 p0 = (u64)0xD2511F53u * (u64)c0;
        const u64 p1 = (u64)0xCD9E8D57u * (u64)c2;
        const u32 hi0 = (u32)(p0 >> 32), lo0 = (u32)p0;
        const u32 hi1 = (u32)(p1 >> 32), lo1 = (u32)p1;
        c0 = hi1 ^ c1 ^ rk[r][0];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk[r][1];
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 cfs_philox(const cfs_launch_args& a, u32 c0, u32 c1, u32 c2,
                                            u32 c3)
{
    return cfs_philox_rk(a.rk, c0, c1, c2, c3);
}

__device__ __forceinline__ u32 cfs_word(uint4 r, u32 s)
{
    return s == 0 ? r.x : (s == 1 ? r.y : (s == 2 ? r.z : r.w));
}

/* ---- shared-memory copy of the per-launch tables ---------------------- */
#ifndef CFS_STARS_TAB
#define CFS_STARS_TAB 0
#endif
struct CfsSmem {
    float4 prm4[3][CFS_A_MAX_MAPS];           /* map k's params 4j..4j+3 at [j][k] */
    float4 pal[CFS_A_MAX_TARGETS][CFS_A_MAX_MAPS];
    u32 pal8[CFS_A_MAX_TARGETS][CFS_A_MAX_MAPS];
#if CFS_STARS_TAB
    /* centre and size of the chain's first duplication op's stars (up to
     * CFS_STARS_TAB of them), filled once per CTA: the per-step lookup
     * replaces a Philox block per point-step with the same values */
    float4 stars[CFS_STARS_TAB];
#endif
};

__device__ __forceinline__ void cfs_load_smem(const cfs_launch_args& a, CfsSmem& sm)
{
    for (int t = threadIdx.x; t < 3 * CFS_A_MAX_MAPS; t += blockDim.x) {
        const int j = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
        sm.prm4[j][k] = make_float4(a.sys.prm[4 * j][k], a.sys.prm[4 * j + 1][k],
                                    a.sys.prm[4 * j + 2][k], a.sys.prm[4 * j + 3][k]);
    }
    for (int t = threadIdx.x; t < CFS_A_MAX_TARGETS * CFS_A_MAX_MAPS; t += blockDim.x) {
        const int g = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
        sm.pal[g][k] = make_float4(a.tg[g].palette[k][0], a.tg[g].palette[k][1],
                                   a.tg[g].palette[k][2], a.tg[g].palette[k][3]);
        sm.pal8[g][k] = a.tg[g].palette8[k];
    }
}

/* ---- generator maps ------------------------------------------------------ */
/* Affine 2D map k from the shared table: x' = fma(a, x, fma(b, y, e)). */
__device__ __forceinline__ void cfs_affine2_tab(int k, float& x, float& y, const CfsSmem& sm)
{
    /* (a, b, c, d) in one 16-byte load, (e, f) in one 8-byte load */
    const float4 m = sm.prm4[0][k];
    const float2 ef = *reinterpret_cast<const float2*>(&sm.prm4[1][k]);
    const float nx = fmaf(m.x, x, fmaf(m.y, y, ef.x));
    const float ny = fmaf(m.z, x, fmaf(m.w, y, ef.y));
    x = nx;
    y = ny;
}

/* Affine 3D map k: row-major A then b. */
__device__ __forceinline__ void cfs_affine3_tab(int k, float& x, float& y, float& z,
                                                const CfsSmem& sm)
{
    const float4 p0 = sm.prm4[0][k], p1 = sm.prm4[1][k], p2 = sm.prm4[2][k];
    const float nx = fmaf(p0.x, x, fmaf(p0.y, y, fmaf(p0.z, z, p2.y)));
    const float ny = fmaf(p0.w, x, fmaf(p1.x, y, fmaf(p1.y, z, p2.z)));
    const float nz = fmaf(p1.z, x, fmaf(p1.w, y, fmaf(p2.x, z, p2.w)));
    x = nx;
    y = ny;
    z = nz;
}

__device__ __forceinline__ void cfs_affine2(float a, float b, float c, float d, float e, float f,
                                            float& x, float& y)
{
    const float nx = fmaf(a, x, fmaf(b, y, e));
    const float ny = fmaf(c, x, fmaf(d, y, f));
    x = nx;
    y = ny;
}

__device__ __forceinline__ void cfs_affine3(float m0, float m1, float m2, float m3, float m4,
                                            float m5, float m6, float m7, float m8, float b0,
                                            float b1, float b2, float& x, float& y, float& z)
{
    const float nx = fmaf(m0, x, fmaf(m1, y, fmaf(m2, z, b0)));
    const float ny = fmaf(m3, x, fmaf(m4, y, fmaf(m5, z, b1)));
    const float nz = fmaf(m6, x, fmaf(m7, y, fmaf(m8, z, b2)));
    x = nx;
    y = ny;
    z = nz;
}

/* Rotations about one axis: the affine evaluation above with its zero terms
 * dropped (x' = fma(1, x, fma(0, y, fma(0, z, 0))) is x; the two rotated
 * coordinates keep their fma(a, u, fma(b, v, 0)) = fma(a, u, b v) form). */
__device__ __forceinline__ void cfs_rotate3_0(float, float, float, float, float m4, float m5,
                                              float m6, float m7, float m8, float, float, float,
                                              float& x, float& y, float& z)
{
    (void)m6; (void)x;
    const float ny = fmaf(m4, y, m5 * z);
    const float nz = fmaf(m7, y, m8 * z);
    y = ny;
    z = nz;
}

__device__ __forceinline__ void cfs_rotate3_1(float m0, float, float m2, float, float, float,
                                              float m6, float, float m8, float, float, float,
                                              float& x, float& y, float& z)
{
    (void)y;
    const float nx = fmaf(m0, x, m2 * z);
    const float nz = fmaf(m6, x, m8 * z);
    x = nx;
    z = nz;
}

__device__ __forceinline__ void cfs_rotate3_2(float m0, float m1, float, float m3, float m4,
                                              float, float, float, float, float, float, float,
                                              float& x, float& y, float& z)
{
    (void)z;
    const float nx = fmaf(m0, x, m1 * y);
    const float ny = fmaf(m3, x, m4 * y);
    x = nx;
    y = ny;
}

/* Eq. 1 (circle IFS), read with atan2 taken into [0, 2 pi) and r2 in the last
 * two lines: theta2 = pi (r + f_id), r2 = sqrt(theta / 2 pi). */
__device__ __forceinline__ void cfs_circle(float fid, float& x, float& y)
{
    const float r = sqrtf(fmaf(x, x, y * y));
    float th = atan2f(y, x);
    if (th < 0.0f) th = th + CFS_TWO_PI_F;
    const float th2 = CFS_PI_F * (r + fid);
    const float r2 = sqrtf(th / CFS_TWO_PI_F);
    float s, c;
    sincosf(th2, &s, &c);
    x = r2 * c;
    y = r2 * s;
}

/* ---- trigonometry of the chain ops ---------------------------------------
 * CFS_FAST_TRIG selects how the chain's sines and cosines are computed:
 *  0: CUDA's sinf / cosf / sincosf;
 *  1: reduced to [-pi, pi] by Cody & Waite's method (Software Manual for the
 *     Elementary Functions, 1980): k = rint(x / 2 pi), r = x - k C1 - k C2 -
 *     k C3 with 2 pi = C1 + C2 + C3 split so that k C1 is exact (C1 = 6.28125
 *     has 8 significant bits), then the hardware sine/cosine (__sinf,
 *     __cosf); absolute error about 4e-7 for |x| < 2^16. */
#ifndef CFS_FAST_TRIG
#define CFS_FAST_TRIG 0
#endif
__device__ __forceinline__ float cfs_reduce_2pi(float x)
{
    const float k = rintf(x * 0.15915494309189533577f);
    float r = fmaf(-k, 6.28125f, x);
    r = fmaf(-k, 1.9353071693331003e-3f, r);     /* float nearest 2 pi - C1 */
    r = fmaf(-k, 1.0253376606378075e-11f, r);    /* 2 pi - C1 - C2 */
    return r;
}

__device__ __forceinline__ float cfs_sin(float x)
{
#if CFS_FAST_TRIG == 1
    return __sinf(cfs_reduce_2pi(x));
#else
    return sinf(x);
#endif
}

__device__ __forceinline__ float cfs_cos(float x)
{
#if CFS_FAST_TRIG == 1
    return __cosf(cfs_reduce_2pi(x));
#else
    return cosf(x);
#endif
}

__device__ __forceinline__ void cfs_sincos(float x, float* s, float* c)
{
#if CFS_FAST_TRIG == 1
    const float r = cfs_reduce_2pi(x);
    *s = __sinf(r);
    *c = __cosf(r);
#else
    sincosf(x, s, c);
#endif
}

/* ---- transform chain ops (Section 3; Eq. 2) ------------------------------ */
__device__ __forceinline__ void cfs_swirl(float& x, float& y)
{
    const float r2 = fmaf(x, x, y * y);
    float s, c;
    cfs_sincos(r2, &s, &c);
    const float nx = fmaf(x, s, -(y * c));
    const float ny = fmaf(x, c, y * s);
    x = nx;
    y = ny;
}

__device__ __forceinline__ void cfs_sinusoidal(float& x, float& y)
{
    x = cfs_sin(x);
    y = cfs_sin(y);
}

__device__ __forceinline__ void cfs_sinusoidal3(float& x, float& y, float& z)
{
    x = cfs_sin(x);
    y = cfs_sin(y);
    z = cfs_sin(z);
}

__device__ __forceinline__ void cfs_stretch(float& x, float& y)
{
    const float ox = x;
    x = 2.0f * ox;
    y = y - cfs_cos(ox);
}

__device__ __forceinline__ void cfs_torus(float R, float r, float& x, float& y, float& z)
{
    const float a = CFS_TWO_PI_F * x, b = CFS_TWO_PI_F * y;
    float sa, ca, sb, cb;
    cfs_sincos(a, &sa, &ca);
    cfs_sincos(b, &sb, &cb);
    const float w = fmaf(r, cb, R);
    x = w * ca;
    y = w * sa;
    z = r * sb;
}

__device__ __forceinline__ bool cfs_perspective(float f, float near_z, float& x, float& y,
                                                float z)
{
    const float inv = 1.0f / z;
    x = (f * x) * inv;
    y = (f * y) * inv;
    return z > near_z;
}

__device__ __forceinline__ void cfs_twist_z(float kappa, float& x, float& y, float z)
{
    float s, c;
    cfs_sincos(kappa * z, &s, &c);
    const float nx = fmaf(x, c, -(y * s));
    const float ny = fmaf(x, s, y * c);
    x = nx;
    y = ny;
}

/* beta and 1/beta (the latter rounded once, on the host) */
__device__ __forceinline__ void cfs_bend(float beta, float invb, float& x, float& z)
{
    float s, c;
    cfs_sincos(beta * x, &s, &c);
    const float d = invb - z;
    x = s * d;
    z = invb - c * d;
}

/* centre (cx, cy, cz), rho2 = rho * rho rounded once on the host */
__device__ __forceinline__ bool cfs_inversion(float cx, float cy, float cz, float rho2,
                                              float& x, float& y, float& z)
{
    const float dx = x - cx, dy = y - cy, dz = z - cz;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float s = rho2 / d2;
    x = fmaf(s, dx, cx);
    y = fmaf(s, dy, cy);
    z = fmaf(s, dz, cz);
    return d2 >= 1e-12f;
}

/* Duplication (Section 3.2): the copy lands on star j = floor(aux n / 2^32)
 * of n, whose centre and size come from Philox block (j, 0, 0, 7):
 * q' = centre + size q.  Parameters: n (integer bits), x0, x1 - x0, y0,
 * y1 - y0, z0, z1 - z0, s0, s1 - s0. */
__device__ __forceinline__ float4 cfs_star_centre(const cfs_launch_args& a, u32 j, float x0,
                                                  float dx, float y0, float dy, float z0,
                                                  float dz, float s0, float ds)
{
    const uint4 r = cfs_philox(a, j, 0u, 0u, 7u);
    return make_float4(fmaf(dx, (float)(r.x >> 8) * CFS_INV_2_24, x0),
                       fmaf(dy, (float)(r.y >> 8) * CFS_INV_2_24, y0),
                       fmaf(dz, (float)(r.z >> 8) * CFS_INV_2_24, z0),
                       fmaf(ds, (float)(r.w >> 8) * CFS_INV_2_24, s0));
}

__device__ __forceinline__ void cfs_star_place(float4 c, float& x, float& y, float& z)
{
    x = fmaf(c.w, x, c.x);
    y = fmaf(c.w, y, c.y);
    z = fmaf(c.w, z, c.z);
}

__device__ __forceinline__ void cfs_stars(const cfs_launch_args& a, u32 n, float x0, float dx,
                                          float y0, float dy, float z0, float dz, float s0,
                                          float ds, u32 aux, float& x, float& y, float& z)
{
    const u32 j = __umulhi(aux, n);
    cfs_star_place(cfs_star_centre(a, j, x0, dx, y0, dy, z0, dz, s0, ds), x, y, z);
}

/* The unit disk as the front (z <= 0) half of a sphere of radius R. */
__device__ __forceinline__ void cfs_hemisphere(float R, float& x, float& y, float& z)
{
    const float r2 = fmaf(x, x, y * y);
    const float h = sqrtf(fmaxf(0.0f, 1.0f - r2));
    x = R * x;
    y = R * y;
    z = -(R * h);
}

/* Band texture: colour base + (floor(freq u + phase) mod n).  Inside the
 * guarded range |t| < 1e9 the floor fits a 32-bit int, so the modulo stays
 * in 32-bit integer arithmetic (64-bit conversions and divisions would run
 * on the slow double-precision path). */
__device__ __forceinline__ int cfs_bands(float u, float freq, float phase, int n, int base)
{
    const float t = fmaf(freq, u, phase);
    int m = 0;
    if (isfinite(t) && fabsf(t) < 1.0e9f) {
        const int b = __float2int_rd(t);
        m = ((b % n) + n) % n;
    }
    return base + m;
}

/* ---- splats (Section 1: the point colours the pixel it lands in) --------- */
/* Bin of one coordinate: floor((u - lo) * scale), valid for lo <= u <= hi,
 * the last bin closed.  Returns -1 when outside (NaN included). */
__device__ __forceinline__ int cfs_bin(float u, float lo, float hi, float scale, int n)
{
    const bool in = (u >= lo) && (u <= hi);
    const int b = min(__float2int_rd((u - lo) * scale), n - 1);
    return in ? b : -1;
}

/* The same bin with its validity apart: ok is lo <= u <= hi (false for NaN),
 * and then the bin lies in 0..n-1; the value is meaningless when !ok.  (The
 * splats test ok instead of a -1.) */
__device__ __forceinline__ int cfs_bin_ok(float u, float lo, float hi, float scale, int n,
                                          bool& ok)
{
    ok = (u >= lo) && (u <= hi);
    return min(__float2int_rd((u - lo) * scale), n - 1);
}

/* The splat reductions carry no "memory" clobber: nothing in a kernel reads
 * a target except the depth test, which is correct under any order (keys
 * only decrease), so the compiler may schedule them freely. */
__device__ __forceinline__ void cfs_red_add_u32(u32* p, u32 v)
{
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v));
}

__device__ __forceinline__ void cfs_red_add_v4f32(float* p, float4 v)
{
    asm volatile("red.global.v4.f32.add [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w));
}

__device__ __forceinline__ void cfs_red_min_u64(u64* p, u64 v)
{
    asm volatile("red.global.min.u64 [%0], %1;" ::"l"(p), "l"(v));
}

/* Not volatile: the compiler may issue it early (before the previous splat's
 * reduction) or reuse an earlier load of the same address -- both return a
 * value the key had at some point, and keys only decrease. */
__device__ __forceinline__ u64 cfs_ld_relaxed_u64(const u64* p)
{
    u64 v;
    asm("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

/* u32 histogram [C][H][W]: +1 in channel ch. */
__device__ __forceinline__ void cfs_splat_hist(const cfs_dev_target& t, float x, float y,
                                               bool alive, int ch, u32& disc)
{
    bool okx, oky;
    const int ix = cfs_bin_ok(x, t.x0, t.x1, t.sx, t.W, okx);
    const int iy = cfs_bin_ok(y, t.y0, t.y1, t.sy, t.H, oky);
    if (alive && okx && oky) {
        u32* base = reinterpret_cast<u32*>(t.data);
        const size_t off = ((size_t)ch * (size_t)t.H + (size_t)iy) * (size_t)t.W + (size_t)ix;
        cfs_red_add_u32(base + off, 1u);
    } else {
        disc += 1;
    }
}

/* What a windowed batch splat reads of its target: the frame's values,
 * copied to the batch kernel's locals once per frame so that they stay in
 * registers instead of being read from shared memory on every splat. */
struct CfsBinTarget {
    unsigned long long data;
    int W, H;
    float x0, x1, sx, y0, y1, sy;
};

/* The privatized window of a batch frame's u32 histogram: one pixel box
 * per channel (a channel's splats come from its own maps, whose images are
 * smaller copies of the attractor, so each channel's box sits over that
 * channel's densest region), the channels' counters packed one after the
 * other in shared memory. */
struct CfsTile {
    u32* cnt;           /* shared counters */
    const int4* win;    /* shared, per channel: (x0, y0, w | h << 16, first counter);
                           w = 0: no window */
};

/* u32 histogram splat that adds to the shared window of its channel when
 * the bin lies in it (one shared atomic per group of lanes hitting the same
 * counter with CFS_WARP_AGG) and to global memory otherwise. */
template <class T>
__device__ __forceinline__ void cfs_splat_hist_tile(const T& t, const CfsTile& tl, float x,
                                                    float y, bool alive, int ch, u32& disc)
{
    bool okx, oky;
    const int ix = cfs_bin_ok(x, t.x0, t.x1, t.sx, t.W, okx);
    const int iy = cfs_bin_ok(y, t.y0, t.y1, t.sy, t.H, oky);
    const bool ok = alive && okx && oky;
    const int4 g = tl.win[ch];
    const u32 lx = (u32)(ix - g.x), ly = (u32)(iy - g.y);
    const u32 w = (u32)g.z & 0xFFFFu, h = (u32)g.z >> 16;
    if (ok && lx < w && ly < h) {
        const u32 idx = (u32)g.w + ly * w + lx;
#if CFS_WARP_AGG
        const u32 act = __activemask();
        const u32 peers = __match_any_sync(act, idx);
        if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(tl.cnt + idx, __popc(peers));
#else
        atomicAdd(tl.cnt + idx, 1u);
#endif
    } else if (ok) {
        u32* base = reinterpret_cast<u32*>(t.data);
        const size_t off = ((size_t)ch * (size_t)t.H + (size_t)iy) * (size_t)t.W + (size_t)ix;
        cfs_red_add_u32(base + off, 1u);
    } else {
        disc += 1;
    }
}

/* Adds the windows' nonzero counters to the global histogram and zeroes
 * them; every thread of the CTA takes part. */
__device__ __forceinline__ void cfs_flush_tile(const cfs_dev_target& t, const CfsTile& tl, int C)
{
    u32* base = reinterpret_cast<u32*>(t.data);
    for (int ch = 0; ch < C; ++ch) {
        const int4 g = tl.win[ch];
        const u32 w = (u32)g.z & 0xFFFFu, h = (u32)g.z >> 16;
        u32* cc = tl.cnt + (u32)g.w;
        for (u32 e = threadIdx.x; e < w * h; e += blockDim.x) {
            const u32 v = cc[e];
            cc[e] = 0u;
            if (v) {
                const u32 ly = e / w, lx = e - ly * w;
                const size_t off = ((size_t)ch * (size_t)t.H + (size_t)(g.y + (int)ly)) *
                                       (size_t)t.W + (size_t)(g.x + (int)lx);
                cfs_red_add_u32(base + off, v);
            }
        }
    }
}

/* f32 RGBA [H][W][4]: += colour (one 16-byte vector reduction). */
__device__ __forceinline__ void cfs_splat_rgba(const cfs_dev_target& t, float x, float y,
                                               bool alive, float4 col, u32& disc)
{
    bool okx, oky;
    const int ix = cfs_bin_ok(x, t.x0, t.x1, t.sx, t.W, okx);
    const int iy = cfs_bin_ok(y, t.y0, t.y1, t.sy, t.H, oky);
    if (alive && okx && oky) {
        float* base = reinterpret_cast<float*>(t.data);
        const size_t off = ((size_t)iy * (size_t)t.W + (size_t)ix) * 4;
        cfs_red_add_v4f32(base + off, col);
    } else {
        disc += 1;
    }
}

/* u64 depth+colour [H][W]: min= (bits(z) << 32) | rgba8.  With
 * CFS_DEPTH_TEST the current value is read first (a strong relaxed load) and
 * the reduction is skipped when it could not lower it: keys only decrease,
 * so a key not below an observed value is not below the final one either. */
__device__ __forceinline__ void cfs_splat_depth(const cfs_dev_target& t, float x, float y,
                                                float z, bool alive, u32 rgba8, u32& disc)
{
    bool okx, oky;
    const int ix = cfs_bin_ok(x, t.x0, t.x1, t.sx, t.W, okx);
    const int iy = cfs_bin_ok(y, t.y0, t.y1, t.sy, t.H, oky);
    if (alive && okx && oky) {
        u64* base = reinterpret_cast<u64*>(t.data);
        u64* p = base + ((size_t)iy * (size_t)t.W + (size_t)ix);
        const u64 key = ((u64)__float_as_uint(z) << 32) | (u64)rgba8;
#if CFS_DEPTH_TEST
        if (key < cfs_ld_relaxed_u64(p)) cfs_red_min_u64(p, key);
#else
        cfs_red_min_u64(p, key);
#endif
    } else {
        disc += 1;
    }
}

/* Adds each thread's discard counts to the per-target u64 counters: one
 * atomic per warp and target. */
__device__ __forceinline__ void cfs_flush_discards(const cfs_launch_args& a, const u32* disc,
                                                   int n)
{
    if (a.discards == 0ull) return;
    u64* out = reinterpret_cast<u64*>(a.discards);
    for (int t = 0; t < n; ++t) {
        const u32 s = __reduce_add_sync(0xffffffffu, disc[t]);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(out + t, (u64)s);
    }
}

#endif /* CFS_DEVICE_CUH */
