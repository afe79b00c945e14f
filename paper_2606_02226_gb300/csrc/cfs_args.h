/*
 * cfs_args.h -- the by-value kernel argument block of the generated kernels.
 * Compiled twice: by the host library (to fill it) and, as text handed to
 * NVRTC, by every generated kernel (to read it as a __grid_constant__).
 * Plain C, no includes, fixed-width layout.
 */
#ifndef CFS_ARGS_H
#define CFS_ARGS_H

#define CFS_A_MAX_MAPS 16
#define CFS_A_MAX_OPS 32
#define CFS_A_MAX_TARGETS 4
#define CFS_A_OP_PARAMS 16

typedef struct {
    unsigned long long data;            /* device pointer */
    int W, H, C, kind;
    float x0, x1, y0, y1;
    float sx, sy;                       /* W / (x1 - x0), H / (y1 - y0) in FP32 */
    int pad0, pad1;
    float palette[CFS_A_MAX_MAPS][4];
    unsigned int palette8[CFS_A_MAX_MAPS];
} cfs_dev_target;

typedef struct {
    unsigned int T[CFS_A_MAX_MAPS];     /* thresholds < 2^32, ascending; n_cmp used */
    int n_maps, n_cmp, dim, pad;
    float prm[12][CFS_A_MAX_MAPS];      /* map parameters, SoA: prm[j][k] */
} cfs_dev_system;

/* one frame of a batch (device copy, read by the persistent batch kernel) */
#define CFS_FRAME_NO_WINDOW 1   /* flags: the frame's splats skip the privatized window */
typedef struct {
    unsigned int T[CFS_A_MAX_MAPS];
    int n_maps, n_cmp, dim, flags;
    float prm[12][CFS_A_MAX_MAPS];
    unsigned int n_points, point_begin, system_id, item_begin;   /* first work item */
    unsigned int chunk, start_count;                             /* points per item */
    unsigned long long start;           /* device f32 SoA [dim][n_points] or 0 */
    cfs_dev_target tg[CFS_A_MAX_TARGETS];
} cfs_dev_frame;

typedef struct {
    cfs_dev_system sys;
    float op[CFS_A_MAX_OPS][CFS_A_OP_PARAMS];   /* derived per-op constants */
    cfs_dev_target tg[CFS_A_MAX_TARGETS];
    unsigned int rk[10][2];             /* Philox round keys for this seed */
    unsigned long long discards;        /* device u64 [n_targets] or 0 */
    unsigned long long start;           /* device f32 SoA [dim][n_points] or 0 */
    unsigned long long ids;             /* trace: device u32 [n_ids] */
    unsigned long long k_out, p_out, q_out;   /* trace outputs */
    unsigned int system_id, point_begin, n_points, step_begin;
    unsigned int iters, burn_in, flags, pad2;
    /* stored clouds: SoA positions [dim][n_points] and map index [n_points] */
    unsigned long long cloud_xyz, cloud_fn;
    /* batch: frames, work counter, per-frame discard counters */
    unsigned long long frames, work_counter, frame_discards;
    unsigned long long frame_bbox;      /* int4 [n_frames]: sampled pixel box of target 0 */
    unsigned int n_frames, n_items, chunk, tile_cap;    /* tile_cap: shared u32 counters */
} cfs_launch_args;

#endif
