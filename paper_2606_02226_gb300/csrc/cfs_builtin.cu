// cfs_builtin.cu -- kernels compiled ahead of time with nvcc (not generated):
// the stand-alone Philox4x32-10 check.  They use the same device helpers
// (cfs_device.cuh) as the generated programs.
#include <cuda_runtime.h>

#include "cfs_device.cuh"
#include "cfs_internal.h"

namespace {

__global__ void __launch_bounds__(256) philox_kernel(const u32* __restrict__ ctr,
                                                     const u32* __restrict__ key,
                                                     u32* __restrict__ out, u32 n)
{
    const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint4 c = reinterpret_cast<const uint4*>(ctr)[j];
    unsigned int rk[10][2];
    u32 k0 = key[2 * j], k1 = key[2 * j + 1];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0;
        rk[r][1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    reinterpret_cast<uint4*>(out)[j] = cfs_philox_rk(rk, c.x, c.y, c.z, c.w);
}

/* Uniformly random reductions over a power-of-two footprint: kind 0 u32
 * add, 1 v4.f32 add (16-byte elements), 2 u64 min, 3 strong u64 load + u64
 * min only when it lowers the value seen (the depth test of the splat path),
 * 4 u32 add into the CTA's shared memory (the privatized windows; footprint
 * at most kSmemBenchWords, the sums land in buf once per CTA).  Addresses
 * come from a per-thread xorshift32 stream, so the kernel spends little
 * besides the memory operation. */
constexpr u32 kSmemBenchWords = 8192;

// kind 4, a kernel of its own: the global kinds keep zero shared memory (and
// so their full occupancy)
__global__ void __launch_bounds__(256) smem_atomic_bench_kernel(void* buf, u32 mask, u32 iters,
                                                                u32 seed)
{
    __shared__ u32 s_cnt[kSmemBenchWords];
    u32 h = (blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B1u + seed;
    h |= 1u;
    for (u32 e = threadIdx.x; e < kSmemBenchWords; e += blockDim.x) s_cnt[e] = 0u;
    __syncthreads();
    for (u32 j = 0; j < iters; ++j) {
        h ^= h << 13;
        h ^= h >> 17;
        h ^= h << 5;
        atomicAdd(&s_cnt[h & mask], 1u);
    }
    __syncthreads();
    for (u32 e = threadIdx.x; e <= mask; e += blockDim.x)
        if (s_cnt[e]) atomicAdd(reinterpret_cast<u32*>(buf) + e, s_cnt[e]);
}

__global__ void __launch_bounds__(256) atomic_bench_kernel(int kind, void* buf, u32 mask,
                                                           u32 iters, u32 seed)
{
    u32 h = (blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B1u + seed;
    h |= 1u;
    u32 acc = 0;
    for (u32 j = 0; j < iters; ++j) {
        h ^= h << 13;
        h ^= h >> 17;
        h ^= h << 5;
        const u32 idx = h & mask;
        if (kind == 0) {
            cfs_red_add_u32(reinterpret_cast<u32*>(buf) + idx, 1u);
        } else if (kind == 1) {
            cfs_red_add_v4f32(reinterpret_cast<float*>(buf) + 4 * (size_t)idx,
                              make_float4(1.0f, 0.5f, 0.0f, 1.0f));
        } else if (kind == 2) {
            cfs_red_min_u64(reinterpret_cast<u64*>(buf) + idx, ((u64)h << 32) | j);
        } else {
            u64* p = reinterpret_cast<u64*>(buf) + idx;
            const u64 key = ((u64)h << 32) | j;
            const u64 cur = cfs_ld_relaxed_u64(p);
            if (key < cur) cfs_red_min_u64(p, key);
            acc += (u32)cur;
        }
    }
    if (acc == 0xFFFFFFFFu && kind == 3) reinterpret_cast<u32*>(buf)[0] = acc;
}

}  // namespace

extern "C" cfs_status cfs_atomic_bench(int kind, void* buf, uint64_t n_elems, uint32_t blocks,
                                       uint32_t iters, uint32_t seed, void* stream)
{
    cfs::clear_error();
    if (kind < 0 || kind > 4) return cfs::fail(CFS_ERR_INVALID_ARG, "kind must be 0..4");
    if (!buf || n_elems == 0 || (n_elems & (n_elems - 1)) != 0 || n_elems > (1ull << 32))
        return cfs::fail(CFS_ERR_INVALID_ARG, "n_elems must be a power of two <= 2^32");
    if (kind == 4 && n_elems > kSmemBenchWords)
        return cfs::fail(CFS_ERR_INVALID_ARG, "shared-memory footprint is at most 8192 words");
    if (((uintptr_t)buf) % 16 != 0) return cfs::fail(CFS_ERR_INVALID_ARG, "buf not aligned");
    if (blocks == 0) return CFS_OK;
    if (kind == 4)
        smem_atomic_bench_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
            buf, (u32)(n_elems - 1), iters, seed);
    else
        atomic_bench_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(
            kind, buf, (u32)(n_elems - 1), iters, seed);
    return cfs::check_cuda(cudaGetLastError(), "atomic_bench_kernel launch");
}

extern "C" cfs_status cfs_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                 uint32_t n, void* stream)
{
    cfs::clear_error();
    if (n == 0) return CFS_OK;
    if (!ctr || !key || !out) return cfs::fail(CFS_ERR_INVALID_ARG, "NULL pointer");
    if (((uintptr_t)ctr | (uintptr_t)out) % 16 != 0)
        return cfs::fail(CFS_ERR_INVALID_ARG, "ctr and out must be 16-byte aligned");
    philox_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(ctr, key, out, n);
    return cfs::check_cuda(cudaGetLastError(), "philox_kernel launch");
}
