/*
 * cfs_kernels.cuh -- kernel bodies of the generated chaos-game programs.
 *
 * Included by NVRTC after the generated prelude, which defines
 *   CFS_DIM, CFS_NCMP, CFS_NT (targets), CFS_REUSE, CFS_BLOCK, CFS_MINB,
 *   cfs_gen_map(a, k, x, y, z, sm)              -- the fused generator switch
 *   cfs_chain(a, sm, px, py, pz, k, disc, splat, rec, qx, qy, qz)
 *                                               -- the fused transform chain
 * Every point lives in registers for its whole trajectory (SoA state: x, y,
 * z); only the splats touch global memory.
 */
#ifndef CFS_KERNELS_CUH
#define CFS_KERNELS_CUH

#define CFS_NT_ARR (CFS_NT > 0 ? CFS_NT : 1)

/* map choice: k = #{ j < n_cmp : w >= T_j } (thresholds in the constant bank) */
__device__ __forceinline__ int cfs_choose(const cfs_launch_args& a, u32 w)
{
    int k = 0;
#pragma unroll
    for (int j = 0; j < CFS_NCMP; ++j) k += (w >= a.sys.T[j]) ? 1 : 0;
    return k;
}

/* start point: Philox block (i, 0, s, 1), coordinates (word >> 8) * 2^-24,
 * or the caller's SoA start array (index j of this launch) */
__device__ __forceinline__ void cfs_start(const cfs_launch_args& a, u32 i, u32 j, u32 n_start,
                                          float& x, float& y, float& z)
{
    if (a.start) {
        const float* s = reinterpret_cast<const float*>(a.start);
        x = s[j];
        y = s[(size_t)n_start + j];
        z = CFS_DIM == 3 ? s[2 * (size_t)n_start + j] : 0.0f;
    } else {
        const uint4 r = cfs_philox(a, i, 0u, a.system_id, 1u);
        x = (float)(r.x >> 8) * CFS_INV_2_24;
        y = (float)(r.y >> 8) * CFS_INV_2_24;
        z = CFS_DIM == 3 ? (float)(r.z >> 8) * CFS_INV_2_24 : 0.0f;
    }
}

/* One chaos-game step n with random word w (Section 1): choose, apply, and
 * after burn-in send a copy through the chain (Fig. 2B) -- or, with
 * CFS_REUSE, let the chain's result replace the point (Fig. 2C). */
__device__ __forceinline__ void cfs_step(const cfs_launch_args& a, const CfsSmem& sm, u32 n,
                                         u32 w, float& x, float& y, float& z, int& k, u32* disc)
{
    k = cfs_choose(a, w);
    cfs_gen_map(a, k, x, y, z, sm);
#if CFS_REUSE
    {
        float qx, qy, qz;
        if (cfs_chain(a, sm, x, y, z, k, disc, n >= a.burn_in, (float*)0, qx, qy, qz)) {
            x = qx; y = qy; z = qz;
        }
    }
#else
    if (n >= a.burn_in) {
        float qx, qy, qz;
        cfs_chain(a, sm, x, y, z, k, disc, true, (float*)0, qx, qy, qz);
    }
#endif
}

/* Runs steps step_begin .. iters-1 of point i: one Philox block per four
 * steps in the main loop, a single-step loop for an unaligned head and the
 * tail. */
__device__ __forceinline__ void cfs_run_point(const cfs_launch_args& a, const CfsSmem& sm, u32 i,
                                              float& x, float& y, float& z, u32* disc)
{
    u32 n = a.step_begin;
    const u32 iters = a.iters;
    int k = 0;
#pragma unroll 1
    while (n < iters && (n & 3u)) {
        const uint4 r = cfs_philox(a, i, n >> 2, a.system_id, 0u);
        cfs_step(a, sm, n, cfs_word(r, n & 3u), x, y, z, k, disc);
        ++n;
    }
#pragma unroll 1
    for (; n + 4 <= iters; n += 4) {
        const uint4 r = cfs_philox(a, i, n >> 2, a.system_id, 0u);
        cfs_step(a, sm, n, r.x, x, y, z, k, disc);
        cfs_step(a, sm, n + 1, r.y, x, y, z, k, disc);
        cfs_step(a, sm, n + 2, r.z, x, y, z, k, disc);
        cfs_step(a, sm, n + 3, r.w, x, y, z, k, disc);
    }
#pragma unroll 1
    while (n < iters) {
        const uint4 r = cfs_philox(a, i, n >> 2, a.system_id, 0u);
        cfs_step(a, sm, n, cfs_word(r, n & 3u), x, y, z, k, disc);
        ++n;
    }
}

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
    const u32 stride = gridDim.x * blockDim.x;
    for (u32 j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n_points; j += stride) {
        const u32 i = a.point_begin + j;
        float x, y, z;
        cfs_start(a, i, j, a.n_points, x, y, z);
        cfs_run_point(a, sm, i, x, y, z, disc);
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
    cfs_start(a, i, j, a.n_points, x, y, z);
    const u32 steps = a.iters - a.step_begin;
    int* kout = reinterpret_cast<int*>(a.k_out);
    float* pout = reinterpret_cast<float*>(a.p_out);
    float* qout = reinterpret_cast<float*>(a.q_out);
    u32 disc[CFS_NT_ARR];
    for (u32 n = a.step_begin; n < a.iters; ++n) {
        const size_t s = (size_t)j * steps + (n - a.step_begin);
        const uint4 r = cfs_philox(a, i, n >> 2, a.system_id, 0u);
        const int k = cfs_choose(a, cfs_word(r, n & 3u));
        cfs_gen_map(a, k, x, y, z, sm);
        float qx, qy, qz;
        const bool alive = cfs_chain(a, sm, x, y, z, k, disc, false,
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

#endif /* CFS_KERNELS_CUH */
