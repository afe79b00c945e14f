/*
 * cfs_kernels.cuh -- kernel bodies of the generated chaos-game programs.
 *
 * Included by NVRTC after the generated prelude, which defines
 *   CFS_DIM, CFS_NCMP (thresholds compared), CFS_NT (targets), CFS_REUSE,
 *   CFS_BATCH, CFS_BLOCK, CFS_MINB,
 *   cfs_gen_map(a, k, x, y, z, sm)        -- the fused generator switch
 *   cfs_chain(a, tg, sm, px, py, pz, k, disc, splat, rec, qx, qy, qz)
 *                                         -- the fused transform chain
 * Every point lives in registers for its whole trajectory (SoA state: x, y,
 * z); only the splats touch global memory.
 */
#ifndef CFS_KERNELS_CUH
#define CFS_KERNELS_CUH

#define CFS_NT_ARR (CFS_NT > 0 ? CFS_NT : 1)

/* map choice k = #{ j < n_cmp : w >= T_j }: thresholds of a single render
 * come from the constant bank, those of a batch frame from shared memory */
struct CfsChooseConst {
    const cfs_launch_args& a;
    __device__ __forceinline__ int operator()(u32 w) const
    {
        int k = 0;
#pragma unroll
        for (int j = 0; j < CFS_NCMP; ++j) k += (w >= a.sys.T[j]) ? 1 : 0;
        return k;
    }
};

struct CfsChooseTab {
    const u32* T;   /* shared memory */
    int n_cmp;
    __device__ __forceinline__ int operator()(u32 w) const
    {
        int k = 0;
#pragma unroll
        for (int j = 0; j < CFS_NCMP; ++j) k += (j < n_cmp && w >= T[j]) ? 1 : 0;
        return k;
    }
};

/* start point: Philox block (i, 0, s, 1), coordinates (word >> 8) * 2^-24,
 * or the caller's SoA start array (index j of this launch) */
__device__ __forceinline__ void cfs_start(const cfs_launch_args& a, u32 i, u32 sid, u32 j,
                                          u32 n_start, float& x, float& y, float& z)
{
    if (a.start) {
        const float* s = reinterpret_cast<const float*>(a.start);
        x = s[j];
        y = s[(size_t)n_start + j];
        z = CFS_DIM == 3 ? s[2 * (size_t)n_start + j] : 0.0f;
    } else {
        const uint4 r = cfs_philox(a, i, 0u, sid, 1u);
        x = (float)(r.x >> 8) * CFS_INV_2_24;
        y = (float)(r.y >> 8) * CFS_INV_2_24;
        z = CFS_DIM == 3 ? (float)(r.z >> 8) * CFS_INV_2_24 : 0.0f;
    }
}

/* One chaos-game step n with random word w (Section 1): choose, apply, and
 * after burn-in send a copy through the chain (Fig. 2B) -- or, with
 * CFS_REUSE, let the chain's result replace the point (Fig. 2C). */
template <class CH, class TG>
__device__ __forceinline__ void cfs_step(const cfs_launch_args& a, const CH& choose, const TG& tg,
                                         const CfsSmem& sm, u32 n, u32 w, float& x, float& y,
                                         float& z, u32* disc)
{
    const int k = choose(w);
    cfs_gen_map(a, k, x, y, z, sm);
#if CFS_REUSE
    {
        float qx, qy, qz;
        if (cfs_chain(a, tg, sm, x, y, z, k, disc, n >= a.burn_in, (float*)0, qx, qy, qz)) {
            x = qx; y = qy; z = qz;
        }
    }
#else
    if (n >= a.burn_in) {
        float qx, qy, qz;
        cfs_chain(a, tg, sm, x, y, z, k, disc, true, (float*)0, qx, qy, qz);
    }
#endif
}

/* Runs steps step_begin .. iters-1 of point i of system sid: one Philox
 * block per four steps.  Blocks cut by step_begin or iters run their steps
 * under warp-uniform guards, so the step code appears four times, not more
 * (the generated chain can be long; instruction-cache pressure matters). */
template <class CH, class TG>
__device__ __forceinline__ void cfs_run_point(const cfs_launch_args& a, const CH& choose,
                                              const TG& tg, const CfsSmem& sm, u32 i, u32 sid,
                                              float& x, float& y, float& z, u32* disc)
{
    const u32 b0 = a.step_begin, b1 = a.iters;
    const bool whole = ((b0 | b1) & 3u) == 0u;
#pragma unroll 1
    for (u32 nb = b0 >> 2; (nb << 2) < b1; ++nb) {
        const uint4 r = cfs_philox(a, i, nb, sid, 0u);
        const u32 n = nb << 2;
        if (whole || (n >= b0 && n < b1)) cfs_step(a, choose, tg, sm, n, r.x, x, y, z, disc);
        if (whole || (n + 1 >= b0 && n + 1 < b1))
            cfs_step(a, choose, tg, sm, n + 1, r.y, x, y, z, disc);
        if (whole || (n + 2 >= b0 && n + 2 < b1))
            cfs_step(a, choose, tg, sm, n + 2, r.z, x, y, z, disc);
        if (whole || (n + 3 >= b0 && n + 3 < b1))
            cfs_step(a, choose, tg, sm, n + 3, r.w, x, y, z, disc);
    }
}

#if !CFS_BATCH
/* The render kernel: a persistent grid (a multiple of the SM count) strides
 * over the points of this launch. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_render_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_load_smem(a, sm);
    __syncthreads();
    u32 disc[CFS_NT_ARR];
#pragma unroll
    for (int t = 0; t < CFS_NT_ARR; ++t) disc[t] = 0;
    const CfsChooseConst choose{a};
    const u32 stride = gridDim.x * blockDim.x;
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n_points; j += stride) {
        const u32 i = a.point_begin + j;
        float x, y, z;
        cfs_start(a, i, a.system_id, j, a.n_points, x, y, z);
        cfs_run_point(a, choose, a.tg, sm, i, a.system_id, x, y, z, disc);
    }
    cfs_flush_discards(a, disc, CFS_NT);
}

/* The trace kernel: the same step code, recording instead of splatting. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK)
cfs_trace_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_load_smem(a, sm);
    __syncthreads();
    const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n_points) return;
    const u32 i = reinterpret_cast<const u32*>(a.ids)[j];
    float x, y, z;
    cfs_start(a, i, a.system_id, j, a.n_points, x, y, z);
    const u32 steps = a.iters - a.step_begin;
    int* kout = reinterpret_cast<int*>(a.k_out);
    float* pout = reinterpret_cast<float*>(a.p_out);
    float* qout = reinterpret_cast<float*>(a.q_out);
    const CfsChooseConst choose{a};
    u32 disc[CFS_NT_ARR];
    for (u32 n = a.step_begin; n < a.iters; ++n) {
        const size_t s = (size_t)j * steps + (n - a.step_begin);
        const uint4 r = cfs_philox(a, i, n >> 2, a.system_id, 0u);
        const int k = choose(cfs_word(r, n & 3u));
        cfs_gen_map(a, k, x, y, z, sm);
        float qx, qy, qz;
        const bool alive = cfs_chain(a, a.tg, sm, x, y, z, k, disc, false,
                                     qout + s * (size_t)CFS_NSPLAT_ARR * 4, qx, qy, qz);
#if CFS_REUSE
        if (alive) { x = qx; y = qy; z = qz; }
#else
        (void)alive;
#endif
        kout[s] = k;
        pout[3 * s + 0] = x;
        pout[3 * s + 1] = y;
        pout[3 * s + 2] = z;
    }
}
#else  /* CFS_BATCH */

/* Adds this CTA's discard counts of frame f to the per-frame counters. */
__device__ __forceinline__ void cfs_flush_frame_discards(const cfs_launch_args& a, int f,
                                                         u32* disc)
{
    u64* out = reinterpret_cast<u64*>(a.frame_discards) + (size_t)f * CFS_NT_ARR;
    for (int t = 0; t < CFS_NT; ++t) {
        const u32 s = __reduce_add_sync(0xffffffffu, disc[t]);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(out + t, (u64)s);
        disc[t] = 0;
    }
}

/* The batched renderer (many frames of different systems, one launch): a
 * persistent grid whose CTAs take work items -- a chunk of one frame's
 * points -- from a global counter (one atomicAdd per item; no CTA ever waits
 * for another).  Items are numbered frame by frame and every frame has at
 * least as many items as the grid has CTAs (small frames get small items),
 * so the whole grid works on one or two frames at a time and their layers
 * stay in L2.  A CTA loads a
 * frame's thresholds, maps, palettes and target geometry into shared memory
 * when its next item belongs to another frame. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_batch_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    __shared__ u32 s_T[CFS_A_MAX_MAPS];
    __shared__ cfs_dev_target s_tg[CFS_NT_ARR];
    __shared__ u32 s_item, s_frame, s_npts, s_pbeg, s_sid, s_ibeg, s_chunk;
    __shared__ int s_ncmp;
    const cfs_dev_frame* frames = reinterpret_cast<const cfs_dev_frame*>(a.frames);
    u32* counter = reinterpret_cast<u32*>(a.work_counter);
    int cur = -1;
    u32 disc[CFS_NT_ARR];
#pragma unroll
    for (int t = 0; t < CFS_NT_ARR; ++t) disc[t] = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const u32 item = atomicAdd(counter, 1u);
            u32 lo = 0;
            if (item < a.n_items) {
                /* the frame whose items start at or before `item` */
                u32 hi = a.n_frames;
                while (hi - lo > 1) {
                    const u32 mid = (lo + hi) >> 1;
                    if (frames[mid].item_begin <= item) lo = mid; else hi = mid;
                }
            }
            s_item = item;
            s_frame = lo;
        }
        __syncthreads();
        const u32 item = s_item;
        if (item >= a.n_items) break;
        const int f = (int)s_frame;
        if (f != cur) {
            if (cur >= 0) cfs_flush_frame_discards(a, cur, disc);
            const cfs_dev_frame& fr = frames[f];
            for (int t = threadIdx.x; t < 6 * CFS_A_MAX_MAPS; t += blockDim.x) {
                const int jj = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
                sm.prm2[jj][k] = make_float2(fr.prm[2 * jj][k], fr.prm[2 * jj + 1][k]);
            }
            for (int t = threadIdx.x; t < CFS_NT_ARR * CFS_A_MAX_MAPS; t += blockDim.x) {
                const int g = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
                sm.pal[g][k] = make_float4(fr.tg[g].palette[k][0], fr.tg[g].palette[k][1],
                                           fr.tg[g].palette[k][2], fr.tg[g].palette[k][3]);
                sm.pal8[g][k] = fr.tg[g].palette8[k];
            }
            if (threadIdx.x < CFS_A_MAX_MAPS) s_T[threadIdx.x] = fr.T[threadIdx.x];
            if (threadIdx.x < CFS_NT_ARR) s_tg[threadIdx.x] = fr.tg[threadIdx.x];
            if (threadIdx.x == 0) {
                s_npts = fr.n_points;
                s_pbeg = fr.point_begin;
                s_sid = fr.system_id;
                s_ibeg = fr.item_begin;
                s_chunk = fr.chunk;
                s_ncmp = fr.n_cmp;
            }
            __syncthreads();
            cur = f;
        }
        const CfsChooseTab choose{s_T, s_ncmp};
        const u32 sid = s_sid, pbeg = s_pbeg;
        const u32 j0 = (item - s_ibeg) * s_chunk;
        const u32 j1 = min(j0 + s_chunk, s_npts);
        for (u32 j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const u32 i = pbeg + j;
            const uint4 r = cfs_philox(a, i, 0u, sid, 1u);
            float x = (float)(r.x >> 8) * CFS_INV_2_24;
            float y = (float)(r.y >> 8) * CFS_INV_2_24;
            float z = CFS_DIM == 3 ? (float)(r.z >> 8) * CFS_INV_2_24 : 0.0f;
            cfs_run_point(a, choose, s_tg, sm, i, sid, x, y, z, disc);
        }
        __syncthreads();
    }
    if (cur >= 0) cfs_flush_frame_discards(a, cur, disc);
}
#endif /* CFS_BATCH */

#endif /* CFS_KERNELS_CUH */
