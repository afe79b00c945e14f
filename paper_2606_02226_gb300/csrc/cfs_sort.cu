// cfs_sort.cu -- spatial reordering of a stored point cloud.
//
// Streaming a stored cloud through a smooth deformation keeps neighbours
// together (Section 3's staged alternative; the deformation use of Section
// 4): if the cloud is stored in Morton (Z-curve) order of its positions,
// consecutive points splat into neighbouring pixels and the depth layer's
// sectors are reused in L1/L2 instead of being fetched at random.  This file
// sorts a cloud by a 30-bit Morton key with a stable LSD radix sort (four
// 8-bit passes: digit histograms per tile, one exclusive scan, a stable
// scatter that ranks equal digits in index order) and gathers it.  Stable
// sorting makes the permutation unique: ties keep their original order.
#include <cuda_runtime.h>

#include <cstdint>

#include "cfs_device.cuh"
#include "cfs_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                    // keys per thread per tile
constexpr int kTile = kThreads * kItems;      // 4096 keys per tile
constexpr int kRadix = 256;

// float <-> order-preserving unsigned
__device__ __forceinline__ u32 f2o(float f)
{
    const u32 u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(u32 o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

// box[0..2] = min (ordered), box[3..5] = max (ordered); NaNs are skipped
__global__ void __launch_bounds__(kThreads) bbox_kernel(const float* __restrict__ xyz, u32 n,
                                                        int dim, u32* box)
{
    u32 lo[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, hi[3] = {0u, 0u, 0u};
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int d = 0; d < dim; ++d) {
            const float v = xyz[(size_t)d * n + i];
            if (v == v) {
                lo[d] = min(lo[d], f2o(v));
                hi[d] = max(hi[d], f2o(v));
            }
        }
    for (int d = 0; d < dim; ++d) {
        const u32 a = __reduce_min_sync(0xffffffffu, lo[d]);
        const u32 b = __reduce_max_sync(0xffffffffu, hi[d]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(box + d, a);
            atomicMax(box + 3 + d, b);
        }
    }
}

__device__ __forceinline__ u32 spread10(u32 v)
{
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ u32 spread10_2(u32 v)
{
    v &= 0x3FFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Morton key: each coordinate quantized to 10 bits over the box,
// q = min(1023, (int)((v - lo) * (1024 / (hi - lo)))) in FP32 (no
// contraction), bits interleaved x lowest.  Non-finite coordinates map to 0.
__global__ void __launch_bounds__(kThreads) key_kernel(const float* __restrict__ xyz, u32 n,
                                                       int dim, const u32* box, u32* keys,
                                                       u32* vals)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u32 key = 0;
    for (int d = 0; d < dim; ++d) {
        const float lo = o2f(box[d]), hi = o2f(box[3 + d]);
        const float ext = hi - lo;
        const float scale = ext > 0.0f ? 1024.0f / ext : 0.0f;
        const float v = xyz[(size_t)d * n + i];
        const float u = __fmul_rn(__fsub_rn(v, lo), scale);
        u32 q = (u >= 0.0f) ? (u32)min((int)u, 1023) : 0u;   // NaN fails the test
        key |= (dim == 3 ? spread10(q) : spread10_2(q)) << d;
    }
    keys[i] = key;
    vals[i] = i;
}

// digit counts per tile, stored digit-major: hist[digit * n_tiles + tile]
__global__ void __launch_bounds__(kThreads) hist_kernel(const u32* __restrict__ keys, u32 n,
                                                        int shift, u32 n_tiles, u32* hist)
{
    __shared__ u32 cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * kTile;
    for (int q = 0; q < kItems; ++q) {
        const size_t i = base + (size_t)q * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan in three launches: per-chunk sums, a scan of the sums
// (one block), per-chunk scans with their offsets
constexpr int kScanChunk = 2048;

__global__ void __launch_bounds__(kThreads) scan_sums_kernel(const u32* __restrict__ a, size_t m,
                                                             u32* sums)
{
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    u32 s = 0;
    for (int q = threadIdx.x; q < kScanChunk; q += kThreads)
        if (base + q < m) s += a[base + q];
    s = __reduce_add_sync(0xffffffffu, s);
    __shared__ u32 w[kThreads / 32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int k = 0; k < kThreads / 32; ++k) t += w[k];
        sums[blockIdx.x] = t;
    }
}

// block-wide exclusive scan of one value per thread; returns the total
__device__ __forceinline__ u32 block_exclusive_scan(u32 v, u32* s_w, u32& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 t = 0;
        for (int k = 0; k < kThreads / 32; ++k) {
            const u32 c = s_w[k];
            s_w[k] = t;
            t += c;
        }
        s_w[kThreads / 32] = t;
    }
    __syncthreads();
    const u32 excl = s_w[warp] + x - v;
    total = s_w[kThreads / 32];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(kThreads) scan_top_kernel(u32* sums, u32 n_sums)
{
    __shared__ u32 s_w[kThreads / 32 + 1];
    u32 carry = 0;
    for (u32 base = 0; base < n_sums; base += kThreads) {
        const u32 i = base + threadIdx.x;
        const u32 v = i < n_sums ? sums[i] : 0u;
        u32 total;
        const u32 e = block_exclusive_scan(v, s_w, total);
        if (i < n_sums) sums[i] = carry + e;
        carry += total;
    }
}

__global__ void __launch_bounds__(kThreads) scan_apply_kernel(u32* a, size_t m, const u32* sums)
{
    __shared__ u32 s_w[kThreads / 32 + 1];
    const size_t base = (size_t)blockIdx.x * kScanChunk;
    u32 carry = sums[blockIdx.x];
    for (int q = 0; q < kScanChunk; q += kThreads) {
        const size_t i = base + q + threadIdx.x;
        const u32 v = i < m ? a[i] : 0u;
        u32 total;
        const u32 e = block_exclusive_scan(v, s_w, total);
        if (i < m) a[i] = carry + e;
        carry += total;
    }
}

// Stable scatter: the tile's keys are ranked in index order, 256 at a time
// (one per thread): rank = keys of the same digit in earlier rounds + in
// earlier warps of this round + in lower lanes of this warp.
__global__ void __launch_bounds__(kThreads) scatter_kernel(const u32* __restrict__ kin,
                                                           const u32* __restrict__ vin, u32 n,
                                                           int shift, u32 n_tiles,
                                                           const u32* __restrict__ offs,
                                                           u32* kout, u32* vout)
{
    __shared__ u32 run[kRadix];                       // per digit: placed so far
    __shared__ u32 wcnt[kThreads / 32][kRadix];       // this round, per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(size_t)threadIdx.x * n_tiles + blockIdx.x];
    const size_t base = (size_t)blockIdx.x * kTile;
    const u32 lt = (1u << lane) - 1u;
    for (int q = 0; q < kItems; ++q) {
        for (int w = 0; w < kThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const size_t i = base + (size_t)q * kThreads + threadIdx.x;
        const bool ok = i < n;
        const u32 k = ok ? kin[i] : 0u;
        const u32 v = ok ? vin[i] : 0u;
        const u32 d = ok ? ((k >> shift) & 0xFFu) : 0x100u;   // past-the-end: no digit
        const u32 peers = __match_any_sync(0xffffffffu, d);
        const u32 before = __popc(peers & lt);
        if (ok && before == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // exclusive prefix over warps for digit threadIdx.x; advance run
        u32 acc = 0;
        const u32 mydig = threadIdx.x;
        u32 pre[kThreads / 32];
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            pre[w] = acc;
            acc += wcnt[w][mydig];
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) wcnt[w][mydig] = pre[w];
        __syncthreads();
        if (ok) {
            const u32 dst = run[d] + wcnt[warp][d] + before;
            kout[dst] = k;
            vout[dst] = v;
        }
        __syncthreads();
        run[mydig] += acc;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) gather_kernel(const float* __restrict__ xyz,
                                                          const unsigned char* __restrict__ fn,
                                                          const u32* __restrict__ perm, u32 n,
                                                          int dim, float* xyz_out,
                                                          unsigned char* fn_out)
{
    const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const u32 i = perm[j];
    for (int d = 0; d < dim; ++d) xyz_out[(size_t)d * n + j] = xyz[(size_t)d * n + i];
    fn_out[j] = fn[i];
}

}  // namespace

extern "C" cfs_status cfs_pointcloud_reorder(const float* xyz, const uint8_t* fn, uint32_t n,
                                             int dim, float* xyz_out, uint8_t* fn_out,
                                             uint32_t* perm_out, void* stream_)
{
    using cfs::check_cuda;
    using cfs::fail;
    cfs::clear_error();
    if (n == 0) return CFS_OK;
    if (dim != 2 && dim != 3) return fail(CFS_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (!xyz || !fn || !xyz_out || !fn_out)
        return fail(CFS_ERR_INVALID_ARG, "NULL cloud pointer");
    if (xyz_out == xyz || fn_out == fn)
        return fail(CFS_ERR_INVALID_ARG, "the reorder cannot run in place");
    cudaStream_t s = (cudaStream_t)stream_;
    const u32 n_tiles = (n + kTile - 1) / kTile;
    const size_t m = (size_t)kRadix * n_tiles;
    const u32 n_chunks = (u32)((m + kScanChunk - 1) / kScanChunk);
    // scratch: box | keys x2 | vals x2 | hist | chunk sums
    const size_t bytes = 256 + 4 * (size_t)n * 4 + 4 * m + 4 * (size_t)n_chunks + 256;
    unsigned char* ws = nullptr;
    cfs_status st = check_cuda(cudaMallocAsync((void**)&ws, bytes, s), "cudaMallocAsync");
    if (st != CFS_OK) return st;
    u32* box = reinterpret_cast<u32*>(ws);
    u32* k0 = reinterpret_cast<u32*>(ws + 256);
    u32* k1 = k0 + n;
    u32* v0 = k1 + n;
    u32* v1 = v0 + n;
    u32* hist = v1 + n;
    u32* sums = hist + m;
    cudaError_t e = cudaMemsetAsync(box, 0xFF, 12, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(box + 3, 0x00, 12, s);
    if (e == cudaSuccess) {
        const u32 g = min((n + kThreads - 1) / kThreads, 152u * 8u);
        bbox_kernel<<<g, kThreads, 0, s>>>(xyz, n, dim, box);
        key_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(xyz, n, dim, box, k0, v0);
        const int passes = dim == 3 ? 4 : 3;   // 30 or 20 key bits, 8 per pass
        for (int p = 0; p < passes; ++p) {
            const int shift = 8 * p;
            hist_kernel<<<n_tiles, kThreads, 0, s>>>(k0, n, shift, n_tiles, hist);
            scan_sums_kernel<<<n_chunks, kThreads, 0, s>>>(hist, m, sums);
            scan_top_kernel<<<1, kThreads, 0, s>>>(sums, n_chunks);
            scan_apply_kernel<<<n_chunks, kThreads, 0, s>>>(hist, m, sums);
            scatter_kernel<<<n_tiles, kThreads, 0, s>>>(k0, v0, n, shift, n_tiles, hist, k1, v1);
            u32* t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
        gather_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(xyz, fn, v0, n, dim,
                                                                         xyz_out, fn_out);
        if (perm_out)
            e = cudaMemcpyAsync(perm_out, v0, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return check_cuda(e, "cloud reorder");
    return check_cuda(e2, "cudaFreeAsync");
}
