/*
 * cfs_oracle.h -- interface of the CPU oracle (test infrastructure only; see
 * cfs_oracle.c).  Not included by, and not compatible with, the library's
 * public header: the two sides share no declarations.
 */
#ifndef CFS_ORACLE_H
#define CFS_ORACLE_H

#include <stdint.h>

#define ORC_MAX_MAPS 16

/* generator map kinds */
enum { ORC_MAP_AFFINE = 0, ORC_MAP_CIRCLE = 1 };

/* transform-chain op kinds; each op carries 16 float parameters */
enum {
    ORC_OP_AFFINE2 = 1,     /* a b c d e f                                    */
    ORC_OP_AFFINE3 = 2,     /* A (row-major 9) then b (3)                     */
    ORC_OP_ROTATE2 = 3,     /* angle                                          */
    ORC_OP_ROTATE3 = 4,     /* angle, axis (0 x, 1 y, 2 z)                    */
    ORC_OP_TRANSLATE3 = 5,  /* tx ty tz                                       */
    ORC_OP_SWIRL = 6,
    ORC_OP_SINUSOIDAL = 7,  /* x, y                                           */
    ORC_OP_SINUSOIDAL3 = 8, /* x, y, z                                        */
    ORC_OP_STRETCH = 9,     /* Eq. 2                                          */
    ORC_OP_TORUS = 10,      /* R, r                                           */
    ORC_OP_PERSPECTIVE = 11,/* focal, near                                    */
    ORC_OP_TWIST_Z = 12,    /* kappa                                          */
    ORC_OP_BEND = 13,       /* beta                                           */
    ORC_OP_INVERSION = 14,  /* cx cy cz rho                                   */
    ORC_OP_SPLAT = 15,      /* target index                                   */
    ORC_OP_RESET = 16,      /* new branch from a fresh copy of the point      */
    ORC_OP_STARS = 17,      /* n, x0 x1 y0 y1 z0 z1, s0 s1: duplication        */
    ORC_OP_HEMISPHERE = 18, /* R: unit disk -> front hemisphere of radius R   */
    ORC_OP_BANDS = 19       /* axis, freq, phase, n, base: recolour by bands   */
};

enum { ORC_TGT_HIST_U32 = 0, ORC_TGT_RGBA_F32 = 1, ORC_TGT_DEPTH_U64 = 2 };

typedef struct {
    int dim;             /* 2 or 3 */
    int n_maps;          /* 1..16 */
    const int* kind;     /* [n_maps] */
    const float* prm;    /* [n_maps][12] */
    const double* prob;  /* [n_maps] */
} orc_system;

typedef struct {
    int n_ops;
    const int* op;       /* [n_ops] */
    const float* prm;    /* [n_ops][16] */
    float band_eps;      /* parity bookkeeping: a BANDS coordinate within band_eps
                            of a band edge makes the splat's colour unsure (0 = off) */
} orc_chain;

typedef struct {
    int kind;
    int W, H, C;
    float x0, x1, y0, y1;
    void* buf;                  /* HIST: u32 [C][H][W]; RGBA: f32 [H][W][4]; DEPTH: u64 [H][W] */
    const float* palette;       /* RGBA: [16][4] */
    const uint32_t* palette8;   /* DEPTH: [16] packed RGBA8 */
    float margin_px;            /* near-edge margin for the parity bound (0 = off) */
    uint32_t* amb;              /* optional [H][W] near-edge slack */
    float* zlo;                 /* optional [H][W] lowest depth that may land here */
    float* zhi;                 /* optional [H][W] lowest depth that surely lands here */
    uint64_t* klo;              /* optional [H][W] lowest key (depth bits << 32 | colour)
                                   of any splat that may land here (init all ones) */
    float* zalt;                /* optional [H][W] lowest depth of a splat that may land
                                   here with another colour than klo's (init +inf) */
    uint64_t n_splat;           /* out */
    uint64_t n_discard;         /* out */
    uint64_t n_amb;             /* out: near-edge splats */
} orc_target;

typedef struct {
    uint64_t seed;
    uint32_t system_id;
    uint32_t point_begin;  /* global index of the first point (Philox counter word 0) */
    uint32_t n_points;
    uint32_t step_begin;   /* first step index n */
    uint32_t iters;        /* steps run: n = step_begin .. iters-1 */
    uint32_t burn_in;      /* steps n < burn_in are not splatted */
    int reuse;             /* 0: copy semantics (Fig. 2B); 1: reuse (Fig. 2C) */
    const float* start;    /* optional [n_points][3] start positions */
} orc_run;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int orc_thresholds(int n_maps, const double* prob, uint64_t* T);
int orc_choose(uint32_t w, int n_maps, const uint64_t* T);
int orc_render(const orc_system* sys, const orc_chain* ch, orc_target* tg, int n_tg,
               const orc_run* run);
int orc_trace(const orc_system* sys, const orc_chain* ch, const orc_run* run,
              uint32_t n_ids, const uint32_t* ids, int32_t* k_out, float* p_out,
              float* q_out, int n_splat_ops);
int orc_pointcloud_generate(const orc_system* sys, uint64_t seed, uint32_t system_id,
                            uint32_t n, uint32_t iters, float* xyz, uint8_t* fn);
int orc_render_points(const float* xyz, const uint8_t* fn, uint32_t n, const orc_chain* ch,
                      orc_target* tg, int n_tg);

/* Density-estimation display of a layer (log density, gamma, 8-bit RGBA);
 * a_max <= 0 takes the layer's own maximum.  near (optional, [H][W]) gets the
 * mask of components within eps of a rounding boundary. */
float orc_density_max(const orc_target* t);
int orc_tonemap(const orc_target* t, float gamma, float brightness, float a_max,
                uint32_t background, uint32_t* out, uint8_t* near, double eps);

#endif
