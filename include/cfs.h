/*
 * cfs.h -- C ABI of libcfs, the GB300 (sm_103a) chaos-game renderer for
 * composable function systems (Schloss, "Composable function systems as a
 * general-purpose rendering framework").
 *
 * The library runs the chaos game of Section 1 / Section 3 on the GPU: every
 * point starts at a random position; every step it draws one map of an
 * iterated function system with that map's probability and applies it; after
 * burn-in a copy of the point goes through a composed chain of spatial
 * transforms (Fig. 1, Fig. 2B) and is splatted into caller-owned device
 * buffers.  The generator maps and the chain are compiled together into one
 * fused kernel at run time (NVRTC), so no map or transform is called through
 * a function pointer.
 *
 * Conventions (every entry point):
 *  - Return value: CFS_OK (0) or an error code; cfs_last_error() returns a
 *    thread-local message for the last failure on the calling thread.
 *  - Argument errors are reported synchronously and nothing is launched.
 *  - Handles (cfs_system, cfs_chain) are owned by the library from create to
 *    destroy; destroying a handle while work that uses it is still queued is
 *    allowed (launch arguments are copied at launch time).
 *  - Device buffers (targets, start points, counters, clouds) are owned by
 *    the caller; the library never frees them and never allocates outputs.
 *  - All GPU work is enqueued on the caller's stream (a cudaStream_t passed
 *    as void*; NULL = the legacy default stream) and returns without waiting.
 *  - Rendering ACCUMULATES into targets; clear them with cfs_target_clear.
 *  - The current CUDA device of the calling thread is the one used.
 *
 * Randomness: Philox4x32-10 (Salmon et al., SC'11) with key (seed low 32 bits,
 * seed high 32 bits); step n of point i of system s uses word n & 3 of the
 * block for counter (i, n >> 2, s, 0); the start point uses counter
 * (i, 0, s, 1), coordinate j = (word_j >> 8) * 2^-24.  Results therefore do
 * not depend on the launch configuration.
 */
#ifndef CFS_H
#define CFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CFS_OK = 0,
    CFS_ERR_INVALID_ARG = 1,
    CFS_ERR_UNSUPPORTED = 2,
    CFS_ERR_COMPILE = 3,   /* NVRTC failed; the log is in cfs_last_error() */
    CFS_ERR_CUDA = 4,      /* a CUDA runtime/driver call failed */
    CFS_ERR_OOM = 5,
    CFS_ERR_TIMEOUT = 6
} cfs_status;

#define CFS_MAX_MAPS 16
#define CFS_MAX_OPS 32
#define CFS_MAX_TARGETS 4
#define CFS_OP_PARAMS 16

/* ---- generator maps (Section 1: f_1 .. f_n of an IFS) -------------------- */
typedef enum {
    /* Affine map.  2D params: a b c d e f with x' = a x + b y + e,
     * y' = c x + d y + f, evaluated as fma(a, x, fma(b, y, e)).  3D params:
     * row-major A (9 floats) then b (3). */
    CFS_MAP_AFFINE = 0,
    /* Non-affine circle map of Eq. 1 (2D only), params[0] = f_id (0 or 1):
     * theta = atan2(y, x) in [0, 2 pi), r = |p|, theta2 = pi (r + f_id),
     * r2 = sqrt(theta / 2 pi), p' = r2 (cos theta2, sin theta2). */
    CFS_MAP_CIRCLE = 1
} cfs_map_kind;

typedef struct {
    int32_t kind;        /* cfs_map_kind */
    float params[12];
} cfs_map;

/* ---- transform chain ops (Section 3: human-readable spatial functions
 *      applied to a copy of the iterated point, Fig. 1, Fig. 2B) ----------- */
typedef enum {
    CFS_OP_AFFINE2 = 1,      /* a b c d e f (as CFS_MAP_AFFINE)                  */
    CFS_OP_AFFINE3 = 2,      /* A (row-major 9) then b (3)                        */
    CFS_OP_ROTATE2 = 3,      /* angle: affine with (float)cos, (float)sin of the
                                angle evaluated in double                         */
    CFS_OP_ROTATE3 = 4,      /* angle, axis (0 = x, 1 = y, 2 = z)                 */
    CFS_OP_TRANSLATE3 = 5,   /* tx ty tz                                          */
    CFS_OP_SWIRL = 6,        /* (x sin r^2 - y cos r^2, x cos r^2 + y sin r^2)    */
    CFS_OP_SINUSOIDAL = 7,   /* (sin x, sin y)                                    */
    CFS_OP_SINUSOIDAL3 = 8,  /* (sin x, sin y, sin z)                             */
    CFS_OP_STRETCH = 9,      /* Eq. 2: (2 x, y - cos x)                           */
    CFS_OP_TORUS = 10,       /* R, r: (u, v) -> ((R + r cos 2pi v) cos 2pi u,
                                (R + r cos 2pi v) sin 2pi u, r sin 2pi v); lifts
                                2D to 3D                                          */
    CFS_OP_PERSPECTIVE = 11, /* focal, near: (f x / z, f y / z, z); discards the
                                point unless z > near                             */
    CFS_OP_TWIST_Z = 12,     /* kappa: rotate (x, y) by kappa z                   */
    CFS_OP_BEND = 13,        /* beta: x' = sin(beta x)(1/beta - z),
                                z' = 1/beta - cos(beta x)(1/beta - z)             */
    CFS_OP_INVERSION = 14,   /* cx cy cz rho: c + rho^2 (p - c) / |p - c|^2;
                                discards when |p - c|^2 < 1e-12                   */
    CFS_OP_SPLAT = 15,       /* params[0] = target slot: splat the current point */
    CFS_OP_RESET = 16,       /* start a new branch from a fresh copy of the
                                iterated point (and of its colour index)          */
    /* Duplication (Section 3.2: many small copies of one primitive placed by a
     * PRNG, nothing stored): n, x0 x1 y0 y1 z0 z1, s0 s1.  Star j =
     * floor(w n / 2^32), w = word (step & 3) of Philox block (point, step >> 2,
     * system, 2); star j's centre (x0 + (x1-x0) u0, y0 + (y1-y0) u1,
     * z0 + (z1-z0) u2) and size s0 + (s1-s0) u3 come from Philox block
     * (j, 0, 0, 7), u = (word >> 8) 2^-24; q' = centre + size q (3D out;
     * a 2D point has z = 0).  n in 1..2^24.  Not for stored clouds.        */
    CFS_OP_STARS = 17,
    /* R: the unit disk seen as the front half of a sphere: (R x, R y,
     * -R sqrt(max(0, 1 - x^2 - y^2))); 2D -> 3D                            */
    CFS_OP_HEMISPHERE = 18,
    /* axis, freq, phase, n, base: the branch's colour index becomes
     * base + (floor(freq coord[axis] + phase) mod n), a band texture (0 when
     * the argument is not finite or beyond 1e9); n >= 1, base + n <= 16    */
    CFS_OP_BANDS = 19
} cfs_op_kind;

typedef struct {
    int32_t kind;        /* cfs_op_kind */
    float params[CFS_OP_PARAMS];
} cfs_transform;

/* ---- output targets (Section 1: points are accumulated into an output
 *      layer; the colour tells which map moved the point last) ---------- */
typedef enum {
    /* u32 [C][H][W]; +1 in channel (k mod C), k = last generator map */
    CFS_TARGET_HIST_U32 = 0,
    /* f32 [H][W][4]; += palette[k] (vector reduction) */
    CFS_TARGET_RGBA_F32 = 1,
    /* u64 [H][W]; min= (float bits of depth z) << 32 | palette8[k]; the empty
     * value is all ones; needs a 3D point at the splat */
    CFS_TARGET_DEPTH_U64 = 2
} cfs_target_kind;

typedef struct {
    int32_t kind;                 /* cfs_target_kind */
    int32_t width, height, channels;
    /* view window: x in [x0, x1] -> columns, y in [y0, y1] -> rows; bin
     * ix = floor((x - x0) * (W / (x1 - x0))) in FP32, last bin closed; points
     * outside the window are discarded (and counted) */
    float x0, x1, y0, y1;
    void* data;                   /* device pointer, 16-byte aligned */
    float palette[CFS_MAX_MAPS][4];   /* RGBA colours per map index */
    uint32_t palette8[CFS_MAX_MAPS];  /* packed RGBA8 per map index (depth) */
} cfs_target;

/* ---- render parameters -------------------------------------------------- */
#define CFS_FLAG_REUSE 1u   /* Fig. 2C: the chain's result replaces the point */

typedef struct {
    uint64_t seed;
    uint32_t system_id;    /* Philox counter word 2 */
    uint32_t point_begin;  /* global index of the first point (counter word 0) */
    uint32_t n_points;
    uint32_t step_begin;   /* first step index n run (0 for a fresh start) */
    uint32_t iters;        /* steps n = step_begin .. iters-1 are run */
    uint32_t burn_in;      /* steps n < burn_in are not splatted */
    uint32_t flags;        /* CFS_FLAG_* */
    /* optional device SoA start points, [dim][n_points] floats (point j of
     * this call at start[d * n_points + j]); NULL = Philox start point */
    const float* start;
    /* optional device u64 [n_targets]: discarded splats per target are ADDED
     * here (splats + discards = n_points * (iters - max(step_begin, burn_in))) */
    unsigned long long* discards;
} cfs_render_params;

typedef struct cfs_system cfs_system;
typedef struct cfs_chain cfs_chain;

/* Creates an IFS (Section 1): `n_maps` maps (1..16) of dimension `dim` (2|3)
 * with probabilities `probs` (>= 0, finite, positive sum; normalised here).
 * The threshold table is T_k = floor(S_k 2^32), S_k = (sum_{j<=k} p_j)/sum p
 * in double; map k = #{j < n-1 : w >= T_j}.  All pointers are host pointers
 * and are copied. */
cfs_status cfs_system_create(int dim, int n_maps, const cfs_map* maps, const double* probs,
                             cfs_system** out);
cfs_status cfs_system_destroy(cfs_system* sys);

/* Composes a transform chain (Section 3, Fig. 2B) for points of dimension
 * `dim_in` (the generator's).  Validates dimensions (3D ops need a 3D point;
 * TORUS lifts 2D to 3D), derives the per-op constants and keeps a host copy;
 * the fused kernel is generated and compiled (NVRTC, cached by structure) at
 * the first render that uses it, or ahead of time by cfs_prepare. */
cfs_status cfs_compose(int dim_in, const cfs_transform* ops, int n_ops, cfs_chain** out);
/* As cfs_compose, with flags:
 *  CFS_COMPOSE_FAST_TRIG -- the chain's sines and cosines reduce their
 *  argument to [-pi, pi] (Cody-Waite with 2 pi split in three parts) and use
 *  the hardware sine/cosine: absolute error about 4e-7 per evaluation for
 *  |x| < 2^16 instead of about 1 ulp; several times fewer instructions.
 *  The generator maps are not affected. */
#define CFS_COMPOSE_FAST_TRIG 1u
/*  CFS_COMPOSE_FOLD_LINEAR -- a run of two or more consecutive linear ops
 *  (AFFINE2/ROTATE2 on 2D points; AFFINE3/ROTATE3/TRANSLATE3 on 3D points)
 *  runs as one affine op whose matrix and offset are the run's product,
 *  formed in double from the ops' FP32 constants and rounded once to FP32,
 *  wherever that op costs fewer multiply-adds than the run (a rotation about
 *  an axis costs 4, a translation 3, a general 3D affine 9, a 2D one 4).  Positions then differ from op-by-op FP32 evaluation by a few
 *  ulps (fewer roundings); op indices (cfs_chain_set_params, cfs_chain_info)
 *  stay those of the ops as given. */
#define CFS_COMPOSE_FOLD_LINEAR 4u
cfs_status cfs_compose_ex(int dim_in, const cfs_transform* ops, int n_ops, uint32_t flags,
                          cfs_chain** out);
cfs_status cfs_chain_destroy(cfs_chain* chain);

/* Composes a chain from a scribble program (Section 3.1: verses, stanzas and
 * poems composed at the user's request before compilation).  `source` holds
 * any number of fragments:
 *   __verse  NAME(p1, p2 | T k1 = d1; T k2 = d2;) { BODY }
 *   __stanza NAME(p1 | T k = d;) { PRE __split_stanza(); POST }
 *   __poem   NAME() { statements }
 * and `poem` names the poem that is the chain.  Its statements run once per
 * splat step on the copy of the point (float qx, qy, qz), its colour index
 * (int kc), the step's auxiliary random word (u32 aux), with the generator's
 * point (px, py, pz) and map index k readable and `alive` cleared by
 * discarding ops.  Calls: `@VCALL v(args | k = value;);` inlines verse v as a
 * block that binds each positional parameter by reference to its argument
 * and each keyword parameter to the call's value or else its default;
 * `@SCALL s(args | ...) { BLOCK }` does the same for stanza s with BLOCK
 * injected at its __split_stanza().  Bodies are CUDA C++ and may use the
 * calling context's names.  The library's ops are functions of the poem:
 * reset(), discard(), affine2(a, b, c, d, e, f), rotate2(angle) and
 * rotate3(angle, axis) (cos and sin in double), translate3(x, y, z), swirl(), sinusoidal(), sinusoidal3(),
 * stretch(), torus(R, r), perspective(f, near), twist_z(kappa), bend(beta),
 * inversion(cx, cy, cz, rho), hemisphere(R), bands(axis, freq, phase, n,
 * base), stars(n, x0, x1, y0, y1, z0, z1, s0, s1), with the op semantics
 * listed above; splat(SLOT) (a literal slot 0..3) splats into that target.
 * Expansion and argument errors are reported here (CFS_ERR_INVALID_ARG);
 * compile errors of the bodies at the first render (CFS_ERR_COMPILE, NVRTC
 * log in cfs_last_error()).  flags: CFS_COMPOSE_FAST_TRIG or 0 (a poem's ops are
 * its own code, so CFS_COMPOSE_FOLD_LINEAR does not apply). */
cfs_status cfs_compose_scribble(int dim_in, const char* source, const char* poem,
                                uint32_t flags, cfs_chain** out);
/* Input dimension, op count (0 for a scribble chain) and splat count (the
 * records per step of cfs_trace) of a chain; any output may be NULL. */
cfs_status cfs_chain_info(const cfs_chain* chain, int* dim_in, int* n_ops, int* n_splat);
/* Replaces the parameters of op `index` (same kind); for animated chains. */
cfs_status cfs_chain_set_params(cfs_chain* chain, int index, const float* params);

/* Runs the chaos game (Section 1, Section 3) for points point_begin ..
 * point_begin + n_points - 1 and splats into `targets` (device buffers of
 * the caller; at most CFS_MAX_TARGETS; the chain's SPLAT ops name slots in
 * this array).  Enqueued on `stream`. */
cfs_status cfs_render(const cfs_system* sys, const cfs_chain* chain,
                      const cfs_render_params* params, const cfs_target* targets,
                      int n_targets, void* stream);

/* Compiles (or finds in the cache) the fused kernel a cfs_render with these
 * arguments would use, without launching; lets callers keep compilation out
 * of timed or captured regions. */
cfs_status cfs_prepare(const cfs_system* sys, const cfs_chain* chain,
                       const cfs_target* targets, int n_targets);

/* ---- stored point clouds (Section 3: the staged alternative, "store all
 *      points ... then transform", used for controllable deformation of a
 *      cloud over many frames, Section 4) --------------------------------- */
/* Generates n points: point i runs steps 0 .. iters-1 of the chaos game
 * from its Philox start point (the rules of cfs_render, system id
 * `system_id`); its final position is written SoA to xyz (device, dim
 * floats per point: xyz[d * n + i]) and the index of its last map to fn[i]
 * (device u8).  Enqueued on `stream`. */
cfs_status cfs_pointcloud_generate(const cfs_system* sys, uint64_t seed, uint32_t system_id,
                                   uint32_t n, uint32_t iters, float* xyz, uint8_t* fn,
                                   void* stream);
/* Streams a stored cloud (device SoA xyz [chain dim_in][n], u8 fn [n]) once
 * through the chain and splats every point (colour index fn[i]).  n must be
 * a multiple of 4; xyz 16-byte aligned, fn 4-byte aligned.  Discarded
 * splats are added to `discards` (device u64 [n_targets]) when not NULL. */
cfs_status cfs_render_points(const cfs_chain* chain, const float* xyz, const uint8_t* fn,
                             uint32_t n, const cfs_target* targets, int n_targets,
                             unsigned long long* discards, void* stream);

/* Reorders a stored cloud into Morton (Z-curve) order of its positions so
 * that streaming it splats neighbouring points into neighbouring pixels.
 * Key: each coordinate quantized to 10 bits over the cloud's bounding box,
 * q = min(1023, (int)((v - lo) * (1024 / (hi - lo)))) in FP32 (non-finite
 * or degenerate -> 0), bits interleaved with x lowest; stable sort (equal
 * keys keep their order), so the permutation is unique.  Inputs xyz [dim][n]
 * and fn [n]; outputs xyz_out, fn_out (not in place) and, if not NULL,
 * perm_out [n] with xyz_out[d][j] = xyz[d][perm_out[j]].  Allocates its
 * scratch (about 16 bytes per point) stream-ordered on `stream`. */
cfs_status cfs_pointcloud_reorder(const float* xyz, const uint8_t* fn, uint32_t n, int dim,
                                  float* xyz_out, uint8_t* fn_out, uint32_t* perm_out,
                                  void* stream);

/* ---- batched rendering (many frames in one persistent launch) ---------- */
/* One frame of a batch: its own system, range of point indices and targets
 * (device buffers of the caller).  Frames of a batch share the chain, the
 * step counts and the seed; their systems have maps of one kind (all affine
 * or all circle) and the same dimension; their targets have the same kinds. */
typedef struct {
    const cfs_system* system;
    uint32_t n_points;
    uint32_t point_begin;
    uint32_t system_id;
    /* number of points in `start` (0: n_points); point j of the frame starts
     * at start point j mod start_count, so a few network samples can seed
     * every point (the cleanup steps decorrelate the copies) */
    uint32_t start_count;
    /* optional device SoA start points [dim][start_count] of this frame
     * (e.g. from cfs_sampler_start_points); NULL = Philox start points */
    const float* start;
    cfs_target targets[CFS_MAX_TARGETS];
} cfs_frame;

typedef struct cfs_batch cfs_batch;

/* Plans a batch (the paper's animation frames and in-betweens, Section 4):
 * copies the frames (systems by value), compiles the batch program, cuts the
 * points into work items numbered frame by frame and allocates a device
 * workspace (frame descriptors, work counter, per-frame discard counters)
 * owned by the batch.  The kernel is persistent: CTAs take items from the
 * counter with one atomicAdd each and never wait for one another.  Every
 * point runs steps step_begin .. iters-1 (splats from burn_in on), from its
 * frame's start array or its Philox start point. */
cfs_status cfs_batch_create(const cfs_chain* chain, int n_targets, const cfs_frame* frames,
                            int n_frames, uint32_t step_begin, uint32_t iters, uint32_t burn_in,
                            uint64_t seed, cfs_batch** out);
/* Replaces frame `frame`'s system (same dimension and map kind, at most as
 * many thresholds as planned); waits for the previous launch's upload. */
cfs_status cfs_batch_set_system(cfs_batch* batch, int frame, const cfs_system* sys);
/* Enqueues the batch on `stream` as one CUDA graph: upload of the frame
 * descriptors, counter reset, (clear != 0) clear of every frame's targets,
 * the persistent kernel.  The graph is captured at the first launch of each
 * clear mode. */
cfs_status cfs_batch_launch(cfs_batch* batch, int clear, void* stream);
/* Discarded splats of the last launch, host u64 [n_frames][n_targets];
 * waits for that launch. */
cfs_status cfs_batch_discards(cfs_batch* batch, uint64_t* out);
/* Work items, points per item (the plan's default), persistent grid size. */
cfs_status cfs_batch_info(const cfs_batch* batch, uint32_t* n_items, uint32_t* chunk,
                          uint32_t* grid);
/* The privatized shared-memory windows of every frame in the last launch
 * (or, after cfs_batch_tune, its last trial),
 * host int32 [n_frames][C][4] (C: the channels of target 0's histogram) =
 * (x0, y0, x1, y1): the inclusive pixel box of channel c of target 0 whose
 * splats the launch counted in shared memory (every other splat is a
 * global reduction); (0, 0, -1, -1) for none (window off in the plan or
 * for the frame's shape class, no sample of the channel landed, or a
 * channel's share of the counters below one pixel).  The channels' windows
 * together hold at most the plan's window_words pixels.
 * Measurement aid: with the frame's histogram it gives the numbers of
 * shared-memory and global splats exactly.  Waits for the launch;
 * CFS_ERR_INVALID_ARG before the first launch. */
cfs_status cfs_batch_windows(cfs_batch* batch, int32_t* out);

/* Launch plan of a batch (its tuning knobs: points per thread, privatized
 * tile size and atomic strategy, work-item size).  The first
 * four fields shape the compiled program; chunk is the default work-item
 * size of every frame.  cfs_batch_create starts from the measured default
 * plan (ilp 2, window on when the chain splats once into a histogram, 53248
 * words, warp aggregation off, 4096 points per item). */
typedef struct {
    int ilp;                /* trajectories stepped together per thread: 1 or 2 */
    int window;             /* privatized shared-memory window for the chain's histogram
                               splat: 0 off, 1 on (ignored unless the chain splats once,
                               into a histogram, and is not a scribble) */
    uint32_t window_words;  /* window capacity in u32 counters: 1024..53248, multiple of 256;
                               the histogram's channels share them in proportion to their
                               sampled splats, one window (pixel box) per channel */
    int warp_agg;           /* window adds aggregated across a warp (match.any): 0 or 1 */
    uint32_t chunk;         /* points per work item: a multiple of 32 in 32..2^20 */
} cfs_batch_plan;
cfs_status cfs_batch_get_plan(const cfs_batch* batch, cfs_batch_plan* out);
/* Replaces the plan (compiling the program if needed; waits for the batch's
 * last launch) and clears per-class choices of an earlier cfs_batch_tune:
 * every frame then uses plan->chunk and the window setting. */
cfs_status cfs_batch_set_plan(cfs_batch* batch, const cfs_batch_plan* plan);

/* Autotuner.  Two stages, each timing the batch's own frames for the first
 * `trial_iters` steps (all when 0), best of two trials per candidate:
 *  1. the program, on the whole batch, one knob at a time from the current
 *     plan: trajectories per thread (1, 2), window on/off, window size
 *     (13312, 26624, 53248 words), warp aggregation, then the item size
 *     (2048..16384 points);
 *  2. per shape class -- frames grouped by point count (log2 rounded down
 *     to even: 2^16-2^17, 2^18-2^19, ...) and target size (width x height of
 *     target 0) -- the item size and whether the frame uses the window, timed
 *     on that class's frames alone; the classes' choices are then kept only
 *     if the whole batch runs faster with them than under stage 1's plan
 *     (batches of more than 32 classes skip this stage).
 * The choices are kept in the library's tuning cache under keys made of the
 * device (name, SM count), the program's structure and the classes; a later
 * cfs_batch_tune whose keys are all cached applies them without trials
 * unless `flags` has CFS_TUNE_RETUNE.  Synchronous; the frames' targets hold
 * trial output afterwards (launch with clear = 1).  `out` (may be NULL)
 * receives the result. */
#define CFS_TUNE_RETUNE 1u
typedef struct {
    int ilp;                /* chosen program */
    int tile;               /* window on */
    uint32_t chunk;         /* default item size */
    float trial_ms;         /* whole-batch trial time of the chosen program */
    int trials;             /* candidates timed (0 when every choice came from the cache) */
    uint32_t window_words;
    int warp_agg;
    int n_classes;          /* shape classes */
    int classes_windowed;   /* classes that use the window */
    int from_cache;         /* 1 when the cache supplied every choice */
    int classes_used;       /* 1 when the per-class choices beat the program's plan
                               alone on the whole batch (else every frame uses it) */
} cfs_batch_tuning;
cfs_status cfs_batch_tune(cfs_batch* batch, uint32_t trial_iters, uint32_t flags, void* stream,
                          cfs_batch_tuning* out);

/* The tuning cache (library-wide, in memory; thread-safe).  Load merges the
 * entries of a text file written by save (one "key value" line each; a
 * missing file loads nothing and returns CFS_OK; a malformed line is
 * CFS_ERR_INVALID_ARG).  Save writes every entry.  Clear empties it. */
cfs_status cfs_tune_cache_load(const char* path);
cfs_status cfs_tune_cache_save(const char* path);
cfs_status cfs_tune_cache_clear(void);
/* Number of cached entries. */
uint32_t cfs_tune_cache_size(void);

/* Waits for the batch's last launch, then frees it. */
cfs_status cfs_batch_destroy(cfs_batch* batch);
/* One-shot: create, launch, destroy.  Returns after the frames are rendered
 * (the plan's workspace is freed on return). */
cfs_status cfs_render_batch(const cfs_chain* chain, int n_targets, const cfs_frame* frames,
                            int n_frames, uint32_t step_begin, uint32_t iters, uint32_t burn_in,
                            uint64_t seed, int clear, void* stream);

/* ---- density-estimation display -----------------------------------------
 * Section 4 names density estimation (fractal flames, caustics) as the
 * output that keeps atomics on the path; the paper does not say how such a
 * layer is shown.  The mapping here is the log-density display of fractal
 * flames (Draves & Reckase 2003), per pixel:
 *   A   = accumulated alpha (the number of splats for palette alpha 1),
 *   S   = accumulated colour (RGB),
 *   d   = ln(1 + A) / ln(1 + A_max),  v = brightness * d^(1/gamma),
 *   out = (clamp(S/A * v), clamp(v)) quantised as (uint)(255 x + 0.5) and
 *         packed r | g << 8 | b << 16 | a << 24;
 * pixels with A <= 0 take `background`.  A histogram layer (u32 [C][H][W])
 * counts as the RGBA layer sum_c n_c * palette[c] (products, then sums in
 * channel order); a depth layer resolves to the packed colour in the low 32
 * bits of its key (background where empty, no density).  FP32 throughout
 * (logf, powf, IEEE division). */
typedef struct {
    float gamma;          /* > 0 */
    float brightness;     /* > 0 */
    float a_max;          /* > 0: the density shown at full brightness;
                             <= 0: the layer's own maximum, found on the device */
    uint32_t background;  /* packed RGBA8 of pixels nothing landed on */
} cfs_display_params;

/* Displays one layer into `rgba8` (device u32 [H][W], 16-byte aligned,
 * caller-owned; may not overlap the layer).  `a_max_out` (device float, 4-byte
 * aligned) receives the density maximum used; it is required when
 * params->a_max <= 0 and the layer is not a depth layer, else may be NULL.
 * Two kernels (maximum, then mapping), no allocation, stream-ordered. */
cfs_status cfs_tonemap(const cfs_target* layer, const cfs_display_params* params,
                       uint32_t* rgba8, float* a_max_out, void* stream);

/* Displays target `slot` of every frame of a batch in one maximum launch and
 * one mapping launch: frame f into outs[f] (host array of n_frames device
 * u32 [H][W] pointers, 16-byte aligned).  `a_max_out` (device float
 * [n_frames]) receives each frame's maximum, or NULL to keep it in the
 * batch's workspace.  Usually enqueued right after cfs_batch_launch on the
 * same stream.  The out-pointer upload is staged in pinned memory: a call
 * waits for the previous display of the same batch to have been uploaded. */
cfs_status cfs_batch_display(cfs_batch* batch, int slot, const cfs_display_params* params,
                             uint32_t* const* outs, float* a_max_out, void* stream);

/* ---- learned warm-start sampler (the initial distribution the paper
 *      proposes to derive automatically, Section 4) ---------------------- */
/* Network: u (64) -> 128 -> 128 -> 128 -> 2 with SiLU after the first three
 * layers; u = [Gaussian noise (2), affine parameters a b c d e f of up to 8
 * maps (48, zero for missing maps), frame time t (1), zeros (13)].  BF16
 * weights and activations (round to nearest even), FP32 accumulation on the
 * tensor cores; FP32 master weights and Adam state on the device.
 * Parameter vector (FP32, this order): W1 [128][64], b1 [128], W2 [128][128],
 * b2, W3 [128][128], b3, W4 [2][128], b4 [2]: cfs_sampler_param_count()
 * floats. */
typedef struct cfs_sampler cfs_sampler;

uint32_t cfs_sampler_param_count(void);
/* Creates a sampler with host parameters `params` (NULL: uniform
 * +-1/sqrt(fan_in) weights from Philox with `seed`, zero biases); Adam state
 * zero, step 0. */
cfs_status cfs_sampler_create(const float* params, uint64_t seed, cfs_sampler** out);
cfs_status cfs_sampler_destroy(cfs_sampler* s);
/* Host copies of the parameters, Adam moments and step (any may be NULL):
 * a checkpoint.  Synchronizes the device.  Returns CFS_ERR_TIMEOUT (once) if
 * a tensor-core GEMM of earlier work gave up waiting on its pipeline barrier
 * (bounded waits; the affected results are then incomplete): it reads and
 * clears the device error word as cfs_stream_status does. */
cfs_status cfs_sampler_get_params(const cfs_sampler* s, float* params, float* adam_m,
                                  float* adam_v, uint32_t* step);
/* Restores a checkpoint (moments may be NULL: left as they are). */
cfs_status cfs_sampler_set_params(cfs_sampler* s, const float* params, const float* adam_m,
                                  const float* adam_v, uint32_t step);
/* Y (device f32 [B][2]) = network(U), U device BF16 [B][64], 16-byte aligned
 * (the tensor-core GEMMs read it in 16-byte vectors). */
cfs_status cfs_sampler_forward(cfs_sampler* s, const void* U, uint32_t B, float* Y, void* stream);
/* Adds to `grads` (device f32 [param_count], 16-byte aligned) the gradient
 * of sum(dY * Y) (dY device f32 [B][2]) with respect to every parameter. */
cfs_status cfs_sampler_backward(cfs_sampler* s, const void* U, uint32_t B, const float* dY,
                                float* grads, void* stream);
/* Sliced-Wasserstein loss of point sets X against T (device f32
 * [n_sys][n_per][2]; n_per a power of two in 32..1024) over projections
 * (cos phi_j, sin phi_j) (phi device f32 [n_proj]):
 * L = mean_{s,j} mean_i (sort(X_s theta_j)_i - sort(T_s theta_j)_i)^2.
 * L is added to *loss and dL/dX to dX (device).  Projected keys must be
 * finite.  A predicted key that ties another one exactly receives the
 * gradient of the first rank of the tie. */
cfs_status cfs_sw_loss(const float* X, const float* T, uint32_t n_sys, uint32_t n_per,
                       const float* phi, uint32_t n_proj, float* loss, float* dX, void* stream);
/* One Adam step (beta 0.9, 0.999, eps 1e-8, bias-corrected at step t >= 1)
 * with device gradients `grads`. */
cfs_status cfs_sampler_adam(cfs_sampler* s, const float* grads, uint32_t t, float lr,
                            void* stream);
/* Trains for `steps` Adam steps on chaos-game points of `systems` (2D,
 * affine, at most 8 maps; frame times t_values): every step picks
 * systems_per_step systems, draws points_per_system targets per system from
 * the library's own chaos game (40 steps from a uniform start), evaluates
 * the network on fresh noise and applies the sliced-Wasserstein loss over
 * n_proj projections (randomly rotated each step).  One step is captured as
 * a CUDA graph and replayed.  Writes the per-step loss to loss_history
 * (host, steps floats, may be NULL); returns when training is done. */
cfs_status cfs_sampler_train(cfs_sampler* s, const cfs_system* const* systems,
                             const float* t_values, int n_systems, uint32_t steps,
                             uint32_t systems_per_step, uint32_t points_per_system,
                             uint32_t n_proj, float lr, uint64_t seed, float* loss_history,
                             void* stream);
/* As cfs_sampler_train, with the run's settings in a struct and a
 * learning-rate schedule: step i of the run (0-based, of `steps`) uses
 * lr_final + (lr - lr_final) (1 + cos(pi i / (steps - 1))) / 2, a cosine
 * decay from lr to lr_final (lr_final == lr: constant, as cfs_sampler_train).
 * Both rates positive and finite, else CFS_ERR_INVALID_ARG. */
typedef struct {
    uint32_t steps;
    uint32_t systems_per_step;
    uint32_t points_per_system;   /* power of two in 32..1024 */
    uint32_t n_proj;
    float lr;
    float lr_final;
    uint64_t seed;
} cfs_train_options;
cfs_status cfs_sampler_train_ex(cfs_sampler* s, const cfs_system* const* systems,
                                const float* t_values, int n_systems,
                                const cfs_train_options* options, float* loss_history,
                                void* stream);
/* Warm-start points for `sys` at frame time t: n network outputs on noise
 * drawn from (seed) -- Box-Muller on Philox4x32-10 blocks (row, 0, 0, 3)
 * with key (seed lo, seed hi) -- written SoA to start (device f32 [2][n]),
 * the `start` of a cfs_render_params.  Enqueued on `stream`. */
cfs_status cfs_sampler_start_points(cfs_sampler* s, const cfs_system* sys, float t, uint32_t n,
                                    uint64_t seed, float* start, void* stream);

/* ---- batched histograms without allocation --------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory while rendering -- a real-time or embedded
 * host whose memory budget is fixed after start-up (an allocation there can
 * fail or stall a frame), a process whose GPU memory belongs to another
 * allocator that has taken the device's free memory.
 * It renders the same histograms as cfs_render_batch with a chain that only
 * splats (CFS_OP_SPLAT into slot 0), but keeps its workspace (frame
 * descriptors, work counter, discard counters) in one fixed device array
 * compiled into the library instead of calling cudaMalloc.  It calls no
 * allocating routine.
 *  - At most CFS_NOALLOC_MAX_FRAMES frames per call (else
 *    CFS_ERR_INVALID_ARG); each frame: a 2D system of affine maps, at most
 *    2^32 - 1024 points, and targets[0] a u32 histogram; other targets are
 *    ignored.
 *  - The array (about 140 KB) exists on every GPU that loads the library,
 *    until the process exits, and every call shares it: calls whose GPU
 *    work overlaps (other streams, other threads) race and corrupt each
 *    other.  The work and discard counters are reset on the stream at the
 *    start of each call.
 *  - The first call on a device looks up the array's device address and
 *    the grid size (cudaGetSymbolAddress, occupancy query); make that first
 *    call before any stream capture.
 *  - clear != 0 zeroes the histograms first (on the stream).
 *  - discards, if not NULL: device u64 [n_frames], set to the discarded
 *    splats of each frame.
 *  - Frame descriptors are copied from host memory with cudaMemcpyAsync,
 *    which has read its (pageable) source when it returns. */
#define CFS_NOALLOC_MAX_FRAMES 256
cfs_status cfs_render_batch_noalloc(const cfs_frame* frames, int n_frames, uint32_t iters,
                                    uint32_t burn_in, uint64_t seed, int clear,
                                    unsigned long long* discards, void* stream);

/* Start points for many frames in one launch: frame f gets counts[f]
 * network samples (noise from seeds[f]) for systems[f] at time t[f],
 * written SoA to starts[f] (device f32 [2][counts[f]]).  All host arrays
 * are read before the call returns (the call waits for the previous one's
 * upload on the same stream). */
cfs_status cfs_sampler_start_points_batch(cfs_sampler* s, int n_frames,
                                          const cfs_system* const* systems, const float* t,
                                          const uint32_t* counts, const uint64_t* seeds,
                                          float* const* starts, void* stream);

/* Records, for the n_ids points listed in the device array `ids` (global
 * indices), every step's map index (device i32 [n_ids][steps]), iterated
 * point (device f32 [n_ids][steps][3]) and, per SPLAT op of the chain, the
 * point reaching it (device f32 [n_ids][steps][n_splat_ops][4]: x y z alive),
 * steps = iters - step_begin.  The same generated step code as cfs_render;
 * nothing is splatted.  `params->start`, if set, holds [dim][n_ids]. */
cfs_status cfs_trace(const cfs_system* sys, const cfs_chain* chain,
                     const cfs_render_params* params, const uint32_t* ids, uint32_t n_ids,
                     int32_t* k_out, float* p_out, float* q_out, void* stream);

/* Debugging aid, needs no GPU: writes the CUDA source of the fused program
 * that cfs_render (mode 0), cfs_trace (mode 1), a batch of frames like this
 * one (mode 2), cfs_pointcloud_generate (mode 3) or cfs_render_points (mode
 * 4) would use into `src` (at most
 * src_cap bytes, NUL-terminated), compiles it with NVRTC for sm_103a and
 * writes the compiler log, including ptxas register/spill usage, into `log`.
 * Either buffer may be NULL. */
cfs_status cfs_codegen_check(const cfs_system* sys, const cfs_chain* chain,
                             const cfs_target* targets, int n_targets, int mode, char* src,
                             size_t src_cap, char* log, size_t log_cap);

/* Fills targets with their empty value (0; depth: all ones). */
cfs_status cfs_target_clear(const cfs_target* targets, int n_targets, void* stream);

/* Philox4x32-10 of n (counter, key) pairs: ctr device u32 [n][4], key device
 * u32 [n][2], out device u32 [n][4]. */
cfs_status cfs_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, uint32_t n,
                      void* stream);

/* Atomic-throughput microbenchmark of the splat operations (the roofline of
 * the splat path): `blocks` x 256 threads each issue `iters` reductions at
 * uniformly random element indices of `buf` (device, n_elems elements, a
 * power of two): kind 0 = red.add.u32 (4-byte elements), 1 =
 * red.add.v4.f32 (16-byte), 2 = red.min.u64 (8-byte), 3 = strong u64 load
 * then red.min.u64 when it lowers the value seen (the depth test), 4 = u32
 * add into each CTA's shared memory over n_elems <= 8192 words (the
 * privatized windows of batches; each CTA adds its counts to buf at the
 * end).  The caller times it on `stream`; contents of buf are overwritten
 * (kind 4: accumulated into). */
cfs_status cfs_atomic_bench(int kind, void* buf, uint64_t n_elems, uint32_t blocks,
                            uint32_t iters, uint32_t seed, void* stream);

/* ---- device-side errors (the asynchronous half of the error reporting:
 *      argument errors return at the call, kernel-side failures here) ----- */
/* Bits of the current device's error word, set by kernels of this library:
 * a tensor-core GEMM of the sampler whose bounded mbarrier wait (a TMA
 * arrival, an MMA commit, an epilogue hand-off) ran out skips its output,
 * frees its tensor memory and sets CFS_DEVICE_ERR_TC_TIMEOUT. */
#define CFS_DEVICE_ERR_TC_TIMEOUT 1u
#define CFS_DEVICE_ERR_ALL 1u
/* Waits for the work enqueued on `stream` (NULL: the legacy default stream),
 * then reports, in this order: CFS_ERR_CUDA if that work failed (the CUDA
 * error in cfs_last_error(); a sticky error leaves the context unusable),
 * CFS_ERR_TIMEOUT if a kernel set CFS_DEVICE_ERR_TC_TIMEOUT since the last
 * report, else CFS_OK.  The device's error word is read and cleared, so each
 * device-side error is reported once (by this call or by
 * cfs_sampler_get_params, which reads the same word).  The word is per
 * device, not per stream: a flag set by work on another stream of the same
 * device is reported here too. */
cfs_status cfs_stream_status(void* stream);
/* Testing aid for the reporting path: ORs `flags` (CFS_DEVICE_ERR_* bits)
 * into the current device's error word from the host, as a kernel would,
 * without launching anything.  CFS_ERR_INVALID_ARG for other bits. */
cfs_status cfs_debug_raise_device_error(uint32_t flags);

/* Message of the last failed call on this thread ("" if none). */
const char* cfs_last_error(void);

/* Bytes of the argument block each cfs_render launch copies from the host to
 * the device: the system, the chain's constants, the targets and the Philox
 * round keys travel there, not in device buffers. */
uint32_t cfs_render_arg_bytes(void);

/* Library version string. */
const char* cfs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CFS_H */
