/*
 * cfs_kernels.cuh -- kernel bodies of the generated chaos-game programs.
 *
 * Included by NVRTC after the generated prelude, which defines
 *   CFS_DIM, CFS_NCMP (thresholds compared), CFS_NT (targets), CFS_REUSE,
 *   CFS_BATCH, CFS_BLOCK, CFS_MINB,
 *   cfs_gen_map(a, k, x, y, z, sm)        -- the fused generator switch
 *   cfs_chain(a, tg, sm, px, py, pz, k, aux, disc, splat, rec, qx, qy, qz)
 *                                         -- the fused transform chain
 * Every point lives in registers for its whole trajectory (SoA state: x, y,
 * z); only the splats touch global memory.
 */
#ifndef CFS_KERNELS_CUH
#define CFS_KERNELS_CUH

#define CFS_NT_ARR (CFS_NT > 0 ? CFS_NT : 1)
#ifndef CFS_AUX
#define CFS_AUX 0
#endif

/* auxiliary random block of steps 4 nb .. 4 nb + 3 of point i (stochastic
 * chain ops): Philox (i, nb, s, 2); zeros when the chain has none */
__device__ __forceinline__ uint4 cfs_aux_block(const cfs_launch_args& a, u32 i, u32 nb, u32 sid)
{
#if CFS_AUX
    return cfs_philox(a, i, nb, sid, 2u);
#else
    (void)a; (void)i; (void)nb; (void)sid;
    return make_uint4(0u, 0u, 0u, 0u);
#endif
}

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

#if CFS_BATCH
/* Map choice of a batch frame through a bucket table: the top 12 bits of the
 * word pick one of 4096 buckets of 2^20 words; a bucket without a threshold
 * inside gives every word in it the same k (the table holds it), the at most
 * n_cmp buckets with one fall back to the comparisons.  Same k as
 * CfsChooseTab for every word. */
#define CFS_KTAB_BITS 12
struct CfsChooseKtab {
    const u32* T;               /* shared memory */
    const unsigned char* kt;    /* shared memory, 2^CFS_KTAB_BITS entries; 0xFF: compare */
    int n_cmp;
    __device__ __forceinline__ int operator()(u32 w) const
    {
        const u32 e = kt[w >> (32 - CFS_KTAB_BITS)];
        if (e != 0xFFu) return (int)e;
        int k = 0;
#pragma unroll
        for (int j = 0; j < CFS_NCMP; ++j) k += (j < n_cmp && w >= T[j]) ? 1 : 0;
        return k;
    }
};

/* the frame's bucket table from its thresholds (all threads; the caller
 * synchronizes before and after) */
__device__ __forceinline__ void cfs_build_ktab(const u32* T, int n_cmp, unsigned char* kt)
{
    for (u32 b = threadIdx.x; b < (1u << CFS_KTAB_BITS); b += blockDim.x) {
        const u32 w0 = b << (32 - CFS_KTAB_BITS), w1 = w0 | ((1u << (32 - CFS_KTAB_BITS)) - 1u);
        int k0 = 0, k1 = 0;
        for (int j = 0; j < n_cmp; ++j) {
            k0 += w0 >= T[j] ? 1 : 0;
            k1 += w1 >= T[j] ? 1 : 0;
        }
        kt[b] = k0 == k1 ? (unsigned char)k0 : (unsigned char)0xFFu;
    }
}
#endif

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
                                         const CfsSmem& sm, u32 n, u32 w, u32 aux, float& x,
                                         float& y, float& z, u32* disc, const CfsTile& tile)
{
    const int k = choose(w);
    cfs_gen_map(a, k, x, y, z, sm);
#if CFS_REUSE
    {
        float qx, qy, qz;
        if (cfs_chain(a, tg, sm, x, y, z, k, aux, disc, n >= a.burn_in, (float*)0, qx, qy, qz,
                      tile)) {
            x = qx; y = qy; z = qz;
        }
    }
#else
    if (n >= a.burn_in) {
        float qx, qy, qz;
        cfs_chain(a, tg, sm, x, y, z, k, aux, disc, true, (float*)0, qx, qy, qz, tile);
    }
#endif
}

/* One step past the burn-in with copy semantics: choose, apply, splat the
 * copy through the chain. */
template <class CH, class TG>
__device__ __forceinline__ void cfs_step_splat(const cfs_launch_args& a, const CH& choose,
                                               const TG& tg, const CfsSmem& sm, u32 w, u32 aux,
                                               float& x, float& y, float& z, u32* disc,
                                               const CfsTile& tile)
{
    const int k = choose(w);
    cfs_gen_map(a, k, x, y, z, sm);
    float qx, qy, qz;
    cfs_chain(a, tg, sm, x, y, z, k, aux, disc, true, (float*)0, qx, qy, qz, tile);
}

/* Runs steps step_begin .. iters-1 of point i of system sid: one Philox
 * block per four steps.  Blocks cut by step_begin or iters run their steps
 * under warp-uniform guards (when none is cut and the burn-in ends on a
 * block boundary, a guard-free loop runs instead).  CFS_UNROLL (4, 2 or 1) is how many copies of
 * the step code the loop holds: the generated chain can be long, and
 * instruction-cache pressure trades against the scheduler's freedom to
 * overlap consecutive steps. */
#ifndef CFS_UNROLL
#define CFS_UNROLL 4
#endif
template <class CH, class TG>
__device__ __forceinline__ void cfs_run_point(const cfs_launch_args& a, const CH& choose,
                                              const TG& tg, const CfsSmem& sm, u32 i, u32 sid,
                                              float& x, float& y, float& z, u32* disc,
                                              const CfsTile& tile)
{
    const u32 b0 = a.step_begin, b1 = a.iters;
    const bool whole = ((b0 | b1) & 3u) == 0u;
#if !CFS_REUSE && !(CFS_BATCH && CFS_ILP == 2)
    /* (the two-trajectory batch program calls this only for a frame's odd
     * last point: the general loop keeps its code small) */
    if (whole && (a.burn_in & 3u) == 0u) {
        /* every block whole and the burn-in ending on a block boundary: the
         * burn-in blocks move the point without the chain, the rest splat
         * every step, and no step needs a guard (the same steps, in the same
         * order, as the general loop below) */
        const u32 nb1 = b1 >> 2, nbs = min(max(b0, a.burn_in) >> 2, nb1);
        u32 nb = b0 >> 2;
#pragma unroll 1
        for (; nb < nbs; ++nb) {
            const uint4 r = cfs_philox(a, i, nb, sid, 0u);
            cfs_gen_map(a, choose(r.x), x, y, z, sm);
            cfs_gen_map(a, choose(r.y), x, y, z, sm);
            cfs_gen_map(a, choose(r.z), x, y, z, sm);
            cfs_gen_map(a, choose(r.w), x, y, z, sm);
        }
#pragma unroll 1
        for (; nb < nb1; ++nb) {
            const uint4 r = cfs_philox(a, i, nb, sid, 0u);
            const uint4 ra = cfs_aux_block(a, i, nb, sid);
#if CFS_UNROLL == 4
            cfs_step_splat(a, choose, tg, sm, r.x, ra.x, x, y, z, disc, tile);
            cfs_step_splat(a, choose, tg, sm, r.y, ra.y, x, y, z, disc, tile);
            cfs_step_splat(a, choose, tg, sm, r.z, ra.z, x, y, z, disc, tile);
            cfs_step_splat(a, choose, tg, sm, r.w, ra.w, x, y, z, disc, tile);
#elif CFS_UNROLL == 2
#pragma unroll 1
            for (u32 h = 0; h < 4; h += 2) {
                cfs_step_splat(a, choose, tg, sm, h ? r.z : r.x, h ? ra.z : ra.x, x, y, z, disc,
                               tile);
                cfs_step_splat(a, choose, tg, sm, h ? r.w : r.y, h ? ra.w : ra.y, x, y, z, disc,
                               tile);
            }
#else
            u32 w[4] = {r.x, r.y, r.z, r.w};
            u32 v[4] = {ra.x, ra.y, ra.z, ra.w};
#pragma unroll 1
            for (u32 h = 0; h < 4; ++h) {
                cfs_step_splat(a, choose, tg, sm, w[0], v[0], x, y, z, disc, tile);
                w[0] = w[1]; w[1] = w[2]; w[2] = w[3];
                v[0] = v[1]; v[1] = v[2]; v[2] = v[3];
            }
#endif
        }
        return;
    }
#endif
#pragma unroll 1
    for (u32 nb = b0 >> 2; (nb << 2) < b1; ++nb) {
        const uint4 r = cfs_philox(a, i, nb, sid, 0u);
        const uint4 ra = cfs_aux_block(a, i, nb, sid);
        const u32 n = nb << 2;
#if CFS_UNROLL == 4
        if (whole || (n >= b0 && n < b1))
            cfs_step(a, choose, tg, sm, n, r.x, ra.x, x, y, z, disc, tile);
        if (whole || (n + 1 >= b0 && n + 1 < b1))
            cfs_step(a, choose, tg, sm, n + 1, r.y, ra.y, x, y, z, disc, tile);
        if (whole || (n + 2 >= b0 && n + 2 < b1))
            cfs_step(a, choose, tg, sm, n + 2, r.z, ra.z, x, y, z, disc, tile);
        if (whole || (n + 3 >= b0 && n + 3 < b1))
            cfs_step(a, choose, tg, sm, n + 3, r.w, ra.w, x, y, z, disc, tile);
#elif CFS_UNROLL == 2
#pragma unroll 1
        for (u32 h = 0; h < 4; h += 2) {
            const u32 w0 = h ? r.z : r.x, w1 = h ? r.w : r.y;
            const u32 a0 = h ? ra.z : ra.x, a1 = h ? ra.w : ra.y;
            if (whole || (n + h >= b0 && n + h < b1))
                cfs_step(a, choose, tg, sm, n + h, w0, a0, x, y, z, disc, tile);
            if (whole || (n + h + 1 >= b0 && n + h + 1 < b1))
                cfs_step(a, choose, tg, sm, n + h + 1, w1, a1, x, y, z, disc, tile);
        }
#else
        u32 w[4] = {r.x, r.y, r.z, r.w};
        u32 v[4] = {ra.x, ra.y, ra.z, ra.w};
#pragma unroll 1
        for (u32 h = 0; h < 4; ++h) {
            if (whole || (n + h >= b0 && n + h < b1))
                cfs_step(a, choose, tg, sm, n + h, w[0], v[0], x, y, z, disc, tile);
            w[0] = w[1]; w[1] = w[2]; w[2] = w[3];
            v[0] = v[1]; v[1] = v[2]; v[2] = v[3];
        }
#endif
    }
}

#if CFS_BATCH && CFS_ILP == 2
/* cfs_run_point for two points i0, i1 at once: step n of both before step
 * n + 1 of either.  Each point still follows exactly its own Philox stream,
 * so the results equal two cfs_run_point calls. */
template <class CH, class TG>
__device__ __forceinline__ void cfs_run_point2(const cfs_launch_args& a, const CH& choose,
                                               const TG& tg, const CfsSmem& sm, u32 i0, u32 i1,
                                               u32 sid, float& x0, float& y0, float& z0,
                                               float& x1, float& y1, float& z1, u32* disc,
                                               const CfsTile& tile)
{
    const u32 b0 = a.step_begin, b1 = a.iters;
    const bool whole = ((b0 | b1) & 3u) == 0u;
#if !CFS_REUSE
    if (whole && (a.burn_in & 3u) == 0u) {
        /* every block whole and the burn-in ending on a block boundary: the
         * burn-in blocks move the points without the chain, the rest splat
         * every step, and no step needs a guard (the same steps, in the same
         * order, as the general loop below) */
        const u32 nb1 = b1 >> 2, nbs = min(max(b0, a.burn_in) >> 2, nb1);
        u32 nb = b0 >> 2;
#pragma unroll 1
        for (; nb < nbs; ++nb) {
            const uint4 r0 = cfs_philox(a, i0, nb, sid, 0u);
            const uint4 r1 = cfs_philox(a, i1, nb, sid, 0u);
            const u32 w0[4] = {r0.x, r0.y, r0.z, r0.w};
            const u32 w1[4] = {r1.x, r1.y, r1.z, r1.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cfs_gen_map(a, choose(w0[q]), x0, y0, z0, sm);
                cfs_gen_map(a, choose(w1[q]), x1, y1, z1, sm);
            }
        }
#pragma unroll 1
        for (; nb < nb1; ++nb) {
            const uint4 r0 = cfs_philox(a, i0, nb, sid, 0u);
            const uint4 r1 = cfs_philox(a, i1, nb, sid, 0u);
            const uint4 a0 = cfs_aux_block(a, i0, nb, sid);
            const uint4 a1 = cfs_aux_block(a, i1, nb, sid);
            const u32 w0[4] = {r0.x, r0.y, r0.z, r0.w};
            const u32 w1[4] = {r1.x, r1.y, r1.z, r1.w};
            const u32 v0[4] = {a0.x, a0.y, a0.z, a0.w};
            const u32 v1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cfs_step_splat(a, choose, tg, sm, w0[q], v0[q], x0, y0, z0, disc, tile);
                cfs_step_splat(a, choose, tg, sm, w1[q], v1[q], x1, y1, z1, disc, tile);
            }
        }
        return;
    }
#endif
#pragma unroll 1
    for (u32 nb = b0 >> 2; (nb << 2) < b1; ++nb) {
        const uint4 r0 = cfs_philox(a, i0, nb, sid, 0u);
        const uint4 r1 = cfs_philox(a, i1, nb, sid, 0u);
        const uint4 a0 = cfs_aux_block(a, i0, nb, sid);
        const uint4 a1 = cfs_aux_block(a, i1, nb, sid);
        const u32 n = nb << 2;
        const u32 w0[4] = {r0.x, r0.y, r0.z, r0.w};
        const u32 w1[4] = {r1.x, r1.y, r1.z, r1.w};
        const u32 v0[4] = {a0.x, a0.y, a0.z, a0.w};
        const u32 v1[4] = {a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (whole || (n + q >= b0 && n + q < b1)) {
                cfs_step(a, choose, tg, sm, n + q, w0[q], v0[q], x0, y0, z0, disc, tile);
                cfs_step(a, choose, tg, sm, n + q, w1[q], v1[q], x1, y1, z1, disc, tile);
            }
        }
    }
}
#endif

#if CFS_CLOUD
/* Stored point cloud (Section 3: the staged alternative that keeps every point, then transforms it):
 * point i runs steps 0 .. iters-1 from its Philox start point; its final
 * position goes to SoA xyz[d][i] (coalesced) and the index of its last map
 * to fn[i]. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_cloud_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
    cfs_load_smem(a, sm);
    __syncthreads();
    const CfsChooseConst choose{a};
    float* xyz = reinterpret_cast<float*>(a.cloud_xyz);
    unsigned char* fn = reinterpret_cast<unsigned char*>(a.cloud_fn);
    const u32 n_pts = a.n_points, sid = a.system_id;
    const u32 stride = gridDim.x * blockDim.x;
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pts; j += stride) {
        const u32 i = a.point_begin + j;
        float x, y, z;
        cfs_start(a, i, sid, j, n_pts, x, y, z);
        int k = 0;
#pragma unroll 1
        for (u32 nb = 0; (nb << 2) < a.iters; ++nb) {
            const uint4 r = cfs_philox(a, i, nb, sid, 0u);
            const u32 w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((nb << 2) + q < a.iters) {
                    k = choose(w[q]);
                    cfs_gen_map(a, k, x, y, z, sm);
                }
            }
        }
        xyz[j] = x;
        xyz[(size_t)n_pts + j] = y;
        if (CFS_DIM == 3) xyz[2 * (size_t)n_pts + j] = z;
        fn[j] = (unsigned char)k;
    }
}
#endif

#if CFS_POINTS
/* 16-byte streaming load that neither allocates in L1 nor lingers in L2
 * (the cloud is read once per frame; L2 is kept for the layer). */
__device__ __forceinline__ float4 cfs_ld_stream_f4(const float* p, u64 policy)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(policy));
    return v;
}

__device__ __forceinline__ u32 cfs_ld_stream_u32(const void* p, u64 policy)
{
    u32 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
                 : "=r"(v)
                 : "l"(p), "l"(policy));
    return v;
}

/* Streams a stored cloud through the chain: each thread takes four
 * consecutive points (three 16-byte loads of x, y, z and one 4-byte load of
 * the map indices), runs the fused chain on each and splats it.  n_points is
 * a multiple of 4 and the arrays are 16-byte aligned (checked on the host). */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_points_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
    cfs_load_smem(a, sm);
    __syncthreads();
    u32 disc[CFS_NT_ARR];
#pragma unroll
    for (int t = 0; t < CFS_NT_ARR; ++t) disc[t] = 0;
    u64 policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    const float* xs = reinterpret_cast<const float*>(a.cloud_xyz);
    const unsigned char* fn = reinterpret_cast<const unsigned char*>(a.cloud_fn);
    const u32 n_pts = a.n_points;
    const u32 groups = n_pts >> 2;
    const u32 stride = gridDim.x * blockDim.x;
    for (u32 g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += stride) {
        const size_t o = (size_t)g * 4;
        const float4 X = cfs_ld_stream_f4(xs + o, policy);
        const float4 Y = cfs_ld_stream_f4(xs + (size_t)n_pts + o, policy);
        float4 Z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (CFS_DIM == 3) Z = cfs_ld_stream_f4(xs + 2 * (size_t)n_pts + o, policy);
        const u32 K = cfs_ld_stream_u32(fn + o, policy);
        const CfsTile nt{0, 0};
        float qx, qy, qz;
        cfs_chain(a, a.tg, sm, X.x, Y.x, Z.x, (int)(K & 0xFFu), 0u, disc, true, (float*)0, qx, qy, qz,
                  nt);
        cfs_chain(a, a.tg, sm, X.y, Y.y, Z.y, (int)((K >> 8) & 0xFFu), 0u, disc, true, (float*)0, qx,
                  qy, qz, nt);
        cfs_chain(a, a.tg, sm, X.z, Y.z, Z.z, (int)((K >> 16) & 0xFFu), 0u, disc, true, (float*)0, qx,
                  qy, qz, nt);
        cfs_chain(a, a.tg, sm, X.w, Y.w, Z.w, (int)(K >> 24), 0u, disc, true, (float*)0, qx, qy, qz,
                  nt);
    }
    cfs_flush_discards(a, disc, CFS_NT);
}
#endif

#if !CFS_BATCH && !CFS_CLOUD && !CFS_POINTS
/* The render kernel: a persistent grid (a multiple of the SM count) strides
 * over the points of this launch. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_render_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
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
        cfs_run_point(a, choose, a.tg, sm, i, a.system_id, x, y, z, disc,
                      CfsTile{0, 0});
    }
    cfs_flush_discards(a, disc, CFS_NT);
}

/* The trace kernel: the same step code, recording instead of splatting. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK)
cfs_trace_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
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
        const u32 aux = cfs_word(cfs_aux_block(a, i, n >> 2, a.system_id), n & 3u);
        float qx, qy, qz;
        const bool alive = cfs_chain(a, a.tg, sm, x, y, z, k, aux, disc, false,
                                     qout + s * (size_t)CFS_NSPLAT_ARR * 4, qx, qy, qz,
                                     CfsTile{0, 0});
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
#endif

#if CFS_BATCH

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

/* Frame descriptor -> shared tables (all threads; the caller syncs). */
__device__ __forceinline__ void cfs_load_frame(const cfs_dev_frame& fr, CfsSmem& sm, u32* s_T,
                                               cfs_dev_target* s_tg)
{
    for (int t = threadIdx.x; t < 3 * CFS_A_MAX_MAPS; t += blockDim.x) {
        const int jj = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
        sm.prm4[jj][k] = make_float4(fr.prm[4 * jj][k], fr.prm[4 * jj + 1][k],
                                     fr.prm[4 * jj + 2][k], fr.prm[4 * jj + 3][k]);
    }
    for (int t = threadIdx.x; t < CFS_NT_ARR * CFS_A_MAX_MAPS; t += blockDim.x) {
        const int g = t / CFS_A_MAX_MAPS, k = t % CFS_A_MAX_MAPS;
        sm.pal[g][k] = make_float4(fr.tg[g].palette[k][0], fr.tg[g].palette[k][1],
                                   fr.tg[g].palette[k][2], fr.tg[g].palette[k][3]);
        sm.pal8[g][k] = fr.tg[g].palette8[k];
    }
    if (threadIdx.x < CFS_A_MAX_MAPS) s_T[threadIdx.x] = fr.T[threadIdx.x];
    if (threadIdx.x < CFS_NT_ARR) s_tg[threadIdx.x] = fr.tg[threadIdx.x];
}

#if CFS_TILE
/* The first blockDim points of a frame, run for up to 32 splat steps past
 * the burn-in: calls visit(ix, iy, k) for every sample that lands in target
 * 0 (k: the generator map of the step). */
template <class Visit>
__device__ __forceinline__ void cfs_window_samples(const cfs_launch_args& a,
                                                   const cfs_dev_frame& fr,
                                                   const CfsChooseTab& choose,
                                                   const cfs_dev_target* s_tg, const CfsSmem& sm,
                                                   Visit visit)
{
    const u32 j = threadIdx.x;
    if (j >= fr.n_points) return;
    const u32 i = fr.point_begin + j, sid = fr.system_id;
    const uint4 r0 = cfs_philox(a, i, 0u, sid, 1u);
    float x = (float)(r0.x >> 8) * CFS_INV_2_24;
    float y = (float)(r0.y >> 8) * CFS_INV_2_24;
    float z = CFS_DIM == 3 ? (float)(r0.z >> 8) * CFS_INV_2_24 : 0.0f;
    const u32 n1 = min(a.iters, a.burn_in + 32u);
    const cfs_dev_target& t0 = s_tg[0];
    u32 disc[CFS_NT_ARR];
    for (u32 n = 0; n < n1; ++n) {
        const uint4 r = cfs_philox(a, i, n >> 2, sid, 0u);
        const int k = choose(cfs_word(r, n & 3u));
        cfs_gen_map(a, k, x, y, z, sm);
        if (n < a.burn_in) continue;
        const u32 aux = cfs_word(cfs_aux_block(a, i, n >> 2, sid), n & 3u);
        float rec[4 * CFS_NSPLAT_ARR];
        float qx, qy, qz;
        cfs_chain(a, s_tg, sm, x, y, z, k, aux, disc, false, rec, qx, qy, qz,
                  CfsTile{0, 0});
        const int ix = cfs_bin(rec[0], t0.x0, t0.x1, t0.sx, t0.W);
        const int iy = cfs_bin(rec[1], t0.y0, t0.y1, t0.sy, t0.H);
        if (rec[3] != 0.0f && ix >= 0 && iy >= 0) visit(ix, iy, k);
    }
}

#define CFS_WG 64                        /* coarse density grid: CFS_WG x CFS_WG cells */
#define CFS_WIN_SHAPES 5                 /* window aspect ratios 1/4, 1/2, 1, 2, 4 */

/* Window shape q of the pre-pass (width / height = 2^(q - 2), q = 0..4):
 * at most cap pixels, inside a bw x bh box, widened to the cap once the
 * height is clamped. */
__device__ __forceinline__ void cfs_window_shape(int q, int cap, int bw, int bh, int& ww, int& wh)
{
    ww = (int)sqrtf((float)cap * ldexpf(1.0f, q - 2));
    ww = max(1, min(ww, bw));
    wh = max(1, min(bh, cap / ww));
    ww = max(1, min(bw, cap / wh));
}

/* Pre-pass of the privatized windows: one CTA per frame samples the frame's
 * first blockDim trajectories (see cfs_window_samples) and writes, for each
 * channel c of target 0, the pixel box its window covers to
 * frame_bbox[f * CFS_A_MAX_MAPS + c] (empty when no sample of the channel
 * landed).  The channels share the tile_cap counters in proportion to
 * their sampled splats (a channel's capacity, in pixels, is its share,
 * rounded down, so the windows together never pass tile_cap).  A sample's
 * channel is its map index mod CFS_TILE_C (a chain that recolours moves
 * splats to other channels; they then miss the window more often, nothing
 * else).
 * When the channel's sampled box fits its window, the window is that box.
 * Otherwise the channel's samples are binned into a coarse grid over the
 * box, and of the windows of the channel's capacity (five aspect ratios,
 * positions on the grid's cell boundaries) the one holding the most
 * samples wins: attractors are far from uniform, and the densest region is
 * where privatizing the counters saves the most L2 reductions.  Splats
 * outside the windows still go to global memory, so the choice changes the
 * speed only, never the histogram.  The trajectories are run again for
 * every pass (one for the channels' splat counts, then two per channel at
 * most): that is cheaper than storing the samples. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK)
cfs_bbox_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
    __shared__ u32 s_T[CFS_A_MAX_MAPS];
    __shared__ cfs_dev_target s_tg[CFS_NT_ARR];
    __shared__ int s_box[4];
    __shared__ u32 s_grid[CFS_WG * CFS_WG];
    __shared__ unsigned long long s_best;
    __shared__ u32 s_mass[CFS_TILE_C];
    const int f = blockIdx.x;
    const cfs_dev_frame& fr = reinterpret_cast<const cfs_dev_frame*>(a.frames)[f];
    cfs_load_frame(fr, sm, s_T, s_tg);
    const CfsChooseTab choose{s_T, fr.n_cmp};
    if (threadIdx.x < CFS_TILE_C) s_mass[threadIdx.x] = 0u;
    __syncthreads();
    {
        /* the channels' sampled splats */
        u32 m[CFS_TILE_C];
#pragma unroll
        for (int c = 0; c < CFS_TILE_C; ++c) m[c] = 0u;
        cfs_window_samples(a, fr, choose, s_tg, sm, [&](int ix, int iy, int k) {
            (void)ix; (void)iy;
            const int ch = k % CFS_TILE_C;
#pragma unroll
            for (int c = 0; c < CFS_TILE_C; ++c) m[c] += ch == c ? 1u : 0u;
        });
#pragma unroll
        for (int c = 0; c < CFS_TILE_C; ++c)
            if (m[c]) atomicAdd(&s_mass[c], m[c]);
    }
    __syncthreads();
    u32 total = 0;
    for (int c = 0; c < CFS_TILE_C; ++c) total += s_mass[c];
    int4* out = reinterpret_cast<int4*>(a.frame_bbox) + (size_t)f * CFS_A_MAX_MAPS;
    for (int c = 0; c < CFS_TILE_C; ++c) {
        /* window pixels of this channel */
        const int cap = total ? (int)(((unsigned long long)a.tile_cap * s_mass[c]) / total) : 0;
        if (threadIdx.x == 0) {
            s_box[0] = 0x7fffffff; s_box[1] = 0x7fffffff; s_box[2] = -1; s_box[3] = -1;
            s_best = 0ull;
        }
        for (int e = threadIdx.x; e < CFS_WG * CFS_WG; e += blockDim.x) s_grid[e] = 0u;
        __syncthreads();
        int bx0 = 0x7fffffff, by0 = 0x7fffffff, bx1 = -1, by1 = -1;
        cfs_window_samples(a, fr, choose, s_tg, sm, [&](int ix, int iy, int k) {
            if (k % CFS_TILE_C != c) return;
            bx0 = min(bx0, ix); by0 = min(by0, iy);
            bx1 = max(bx1, ix); by1 = max(by1, iy);
        });
        atomicMin(&s_box[0], bx0); atomicMin(&s_box[1], by0);
        atomicMax(&s_box[2], bx1); atomicMax(&s_box[3], by1);
        __syncthreads();
        int4 box = make_int4(s_box[0], s_box[1], s_box[2], s_box[3]);
        const int bw = box.z - box.x + 1, bh = box.w - box.y + 1;
        if (box.z >= box.x && box.w >= box.y && cap >= 1 && (long long)bw * bh > cap) {
            /* the grid: cells of cw x ch pixels over the box, gx x gy of them */
            const int cw = (bw + CFS_WG - 1) / CFS_WG, ch = (bh + CFS_WG - 1) / CFS_WG;
            const int gx = (bw + cw - 1) / cw, gy = (bh + ch - 1) / ch;
            cfs_window_samples(a, fr, choose, s_tg, sm, [&](int ix, int iy, int k) {
                if (k % CFS_TILE_C == c && ix >= box.x && ix <= box.z && iy >= box.y &&
                    iy <= box.w)
                    atomicAdd(&s_grid[((iy - box.y) / ch) * CFS_WG + (ix - box.x) / cw], 1u);
            });
            __syncthreads();
            /* summed-area table: rows, then columns */
            for (int r = threadIdx.x; r < gy; r += blockDim.x) {
                u32 s = 0u;
                for (int q = 0; q < gx; ++q) s_grid[r * CFS_WG + q] = (s += s_grid[r * CFS_WG + q]);
            }
            __syncthreads();
            for (int q = threadIdx.x; q < gx; q += blockDim.x) {
                u32 s = 0u;
                for (int r = 0; r < gy; ++r) s_grid[r * CFS_WG + q] = (s += s_grid[r * CFS_WG + q]);
            }
            __syncthreads();
            /* candidates: shape q, cell position (i0, j0); the window's whole
             * cells nw x nh are counted */
            const int per = CFS_WG * CFS_WG;
            for (int cand = threadIdx.x; cand < CFS_WIN_SHAPES * per; cand += blockDim.x) {
                const int q = cand / per, pos = cand - q * per;
                const int j0 = pos / CFS_WG, i0 = pos - j0 * CFS_WG;
                int ww, wh;
                cfs_window_shape(q, cap, bw, bh, ww, wh);
                const int nw = max(1, ww / cw), nh = max(1, wh / ch);
                if (i0 + nw > gx || j0 + nh > gy) continue;
                auto at = [&](int r, int col) -> u32 {
                    return (r < 0 || col < 0) ? 0u : s_grid[r * CFS_WG + col];
                };
                const int r1 = j0 + nh - 1, c1 = i0 + nw - 1;
                const u32 mass = at(r1, c1) - at(j0 - 1, c1) - at(r1, i0 - 1) + at(j0 - 1, i0 - 1);
                /* most samples; ties to the lowest candidate number */
                const unsigned long long key =
                    ((unsigned long long)mass << 32) | (unsigned long long)(0xffffffffu - (u32)cand);
                atomicMax(&s_best, key);
            }
            __syncthreads();
            int ww, wh, x0, y0;
            if (s_best != 0ull) {
                const u32 cand = 0xffffffffu - (u32)(s_best & 0xffffffffull);
                const int q = (int)(cand / (u32)per), pos = (int)(cand % (u32)per);
                const int j0 = pos / CFS_WG, i0 = pos - j0 * CFS_WG;
                cfs_window_shape(q, cap, bw, bh, ww, wh);
                const int nw = max(1, ww / cw), nh = max(1, wh / ch);
                /* centre the window on the counted cells */
                x0 = box.x + i0 * cw + (nw * cw - ww) / 2;
                y0 = box.y + j0 * ch + (nh * ch - wh) / 2;
            } else {                   /* (no candidate) the square shape, centred */
                cfs_window_shape(2, cap, bw, bh, ww, wh);
                x0 = box.x + (bw - ww) / 2;
                y0 = box.y + (bh - wh) / 2;
            }
            /* inside the box */
            x0 = max(box.x, min(x0, box.z - ww + 1));
            y0 = max(box.y, min(y0, box.w - wh + 1));
            box = make_int4(x0, y0, x0 + ww - 1, y0 + wh - 1);
        } else if (cap < 1) {
            box = make_int4(0, 0, -1, -1);
        }
        if (threadIdx.x == 0) out[c] = box;
        __syncthreads();                /* s_box, s_grid and s_best are reused */
    }
}

/* Windows of frame f into s_win (thread 0 writes them): the pre-pass's
 * boxes, their counters packed one channel after the other; none when the
 * frame's shape class runs without a window (and, as a guard, for a box
 * that would pass the counters' end). */
__device__ __forceinline__ void cfs_frame_window(const cfs_launch_args& a, int f, int4* s_win)
{
    if (threadIdx.x != 0) return;
    const bool off = (reinterpret_cast<const cfs_dev_frame*>(a.frames)[f].flags &
                      CFS_FRAME_NO_WINDOW) != 0;
    const int4* box = reinterpret_cast<const int4*>(a.frame_bbox) + (size_t)f * CFS_A_MAX_MAPS;
    u32 used = 0;
    for (int c = 0; c < CFS_TILE_C; ++c) {
        const int4 b = box[c];
        const long long w = (long long)b.z - b.x + 1, h = (long long)b.w - b.y + 1;
        if (off || w < 1 || h < 1 || w > 0xFFFF || h > 0x7FFF ||
            (long long)used + w * h > (long long)a.tile_cap) {
            s_win[c] = make_int4(0, 0, 0, 0);
            continue;
        }
        s_win[c] = make_int4(b.x, b.y, (int)((u32)w | ((u32)h << 16)), (int)used);
        used += (u32)(w * h);
    }
}
#endif

/* The batched renderer (many frames of different systems, one launch): a
 * persistent grid whose CTAs take work items -- a chunk of one frame's
 * points -- from a global counter (one atomicAdd per item; no CTA ever waits
 * for another).  Items are numbered frame by frame and every frame has at
 * least as many items as the grid has CTAs (small frames get small items),
 * so the whole grid works on one or two frames at a time and their layers
 * stay in L2.  A CTA loads a frame's thresholds, maps, palettes and target
 * geometry into shared memory when its next item belongs to another frame.
 * With CFS_TILE the first splat goes to a privatized shared-memory window
 * of the frame's histogram, one per channel, placed by the pre-pass
 * (attractors are small and dense: many splats hit the same bins), flushed
 * to global memory when the CTA leaves the frame. */
extern "C" __global__ void __launch_bounds__(CFS_BLOCK, CFS_MINB)
cfs_batch_kernel(const __grid_constant__ cfs_launch_args a)
{
    __shared__ CfsSmem sm;
    cfs_chain_prologue(a, sm);   /* per-CTA tables of the chain (before the first barrier) */
    __shared__ u32 s_T[CFS_A_MAX_MAPS];
    __shared__ cfs_dev_target s_tg[CFS_NT_ARR];
    __shared__ u32 s_item, s_frame, s_npts, s_pbeg, s_sid, s_ibeg, s_chunk;
    __shared__ const float* s_start;
    __shared__ u32 s_scount;
    __shared__ int s_ncmp;
    __shared__ unsigned char s_kt[1u << CFS_KTAB_BITS];   /* the frame's bucket table */
#if CFS_TILE
    extern __shared__ u32 s_cnt[];
    __shared__ int4 s_win[CFS_TILE_C];
    for (u32 e = threadIdx.x; e < a.tile_cap; e += blockDim.x) s_cnt[e] = 0u;
    if (threadIdx.x < CFS_TILE_C) s_win[threadIdx.x] = make_int4(0, 0, 0, 0);
    const CfsTile tile{s_cnt, s_win};
#else
    const CfsTile tile{0, 0};
#endif
    const cfs_dev_frame* frames = reinterpret_cast<const cfs_dev_frame*>(a.frames);
    u32* counter = reinterpret_cast<u32*>(a.work_counter);
    int cur = -1;
#if CFS_TILE
    /* the windowed chain splats once, into target 0: its bin values in
     * registers (the flush still reads s_tg) */
    CfsBinTarget bt[1] = {};
#define CFS_BATCH_TG bt
#else
#define CFS_BATCH_TG s_tg
#endif
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
            if (cur >= 0) {
                cfs_flush_frame_discards(a, cur, disc);
#if CFS_TILE
                cfs_flush_tile(s_tg[0], tile, CFS_TILE_C);
#endif
            }
            __syncthreads();
            const cfs_dev_frame& fr = frames[f];
            cfs_load_frame(fr, sm, s_T, s_tg);
            if (threadIdx.x == 0) {
                s_npts = fr.n_points;
                s_pbeg = fr.point_begin;
                s_sid = fr.system_id;
                s_ibeg = fr.item_begin;
                s_chunk = fr.chunk;
                s_ncmp = fr.n_cmp;
                s_start = reinterpret_cast<const float*>(fr.start);
                s_scount = fr.start_count;
            }
#if CFS_TILE
            cfs_frame_window(a, f, s_win);
#endif
            __syncthreads();
            cfs_build_ktab(s_T, s_ncmp, s_kt);
            __syncthreads();
#if CFS_TILE
            bt[0] = CfsBinTarget{s_tg[0].data, s_tg[0].W, s_tg[0].H, s_tg[0].x0, s_tg[0].x1,
                                 s_tg[0].sx, s_tg[0].y0, s_tg[0].y1, s_tg[0].sy};
#endif
            cur = f;
        }
        const CfsChooseKtab choose{s_T, s_kt, s_ncmp};
        const u32 sid = s_sid, pbeg = s_pbeg;
        const u32 j0 = (item - s_ibeg) * s_chunk;
        const u32 j1 = min(j0 + s_chunk, s_npts);
        const float* st = s_start;
        const u32 sc = s_scount;
        const u32 npts = s_npts;
        /* start of point j of the frame: the frame's own start points (e.g.
         * a learned warm start), reused cyclically when there are fewer than
         * points, or the Philox start block */
        auto start_of = [&](u32 j, float& x, float& y, float& z) {
            if (st) {
                const u32 js = sc < npts ? j % sc : j;
                x = st[js];
                y = st[(size_t)sc + js];
                z = CFS_DIM == 3 ? st[2 * (size_t)sc + js] : 0.0f;
            } else {
                const uint4 r = cfs_philox(a, pbeg + j, 0u, sid, 1u);
                x = (float)(r.x >> 8) * CFS_INV_2_24;
                y = (float)(r.y >> 8) * CFS_INV_2_24;
                z = CFS_DIM == 3 ? (float)(r.z >> 8) * CFS_INV_2_24 : 0.0f;
            }
        };
#if CFS_ILP == 2
        /* two trajectories per thread, stepped in lockstep: their
         * independent dependency chains hide each other's latency */
        for (u32 j = j0 + threadIdx.x; j < j1; j += 2 * blockDim.x) {
            const u32 j2 = j + blockDim.x;
            float x, y, z;
            start_of(j, x, y, z);
            if (j2 < j1) {
                float x2, y2, z2;
                start_of(j2, x2, y2, z2);
                cfs_run_point2(a, choose, CFS_BATCH_TG, sm, pbeg + j, pbeg + j2, sid, x, y, z, x2, y2,
                               z2, disc, tile);
            } else {
                cfs_run_point(a, choose, CFS_BATCH_TG, sm, pbeg + j, sid, x, y, z, disc, tile);
            }
        }
#else
        for (u32 j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            float x, y, z;
            start_of(j, x, y, z);
            cfs_run_point(a, choose, CFS_BATCH_TG, sm, pbeg + j, sid, x, y, z, disc, tile);
        }
#endif
        __syncthreads();
    }
    if (cur >= 0) {
        cfs_flush_frame_discards(a, cur, disc);
#if CFS_TILE
        cfs_flush_tile(s_tg[0], tile, CFS_TILE_C);
#endif
    }
}
#endif /* CFS_BATCH */

#endif /* CFS_KERNELS_CUH */
