// cfs_sampler.cu -- the learned warm-start sampler.
//
// The paper leaves the initial distribution of the primitive to future work
// (Section 4: generate it automatically from the function systems).  The
// sampler is that idea made concrete: an MLP maps Gaussian noise, the affine
// parameters of a system (up to 8 maps) and the frame time t to a point near
// the system's attractor, so a render can start its points there and skip
// most of the burn-in.  It is trained on chaos-game points the library
// itself generates, with a sliced-Wasserstein loss.
//
// Network: u (64) -> 128 -> 128 -> 128 -> 2, SiLU after the first three
// layers; BF16 weights and activations, FP32 accumulation on the tensor
// cores, FP32 master weights and Adam state.  Training runs its GEMMs on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory); the fused inference kernel keeps its small per-point products in
// registers (mma.sync m16n8k16 bf16).
//
// Parameter vector (FP32, this order): W1 [128][64], b1 [128], W2 [128][128],
// b2, W3 [128][128], b3, W4 [2][128], b4 [2] -- 41602 floats.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "cfs_device.cuh"
#include "cfs_internal.h"

namespace {

typedef unsigned short bf16r;

constexpr int D_IN = 64, HID = 128, D_OUT = 2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * D_IN;
constexpr int OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * HID;
constexpr int OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + D_OUT * HID;
constexpr int N_PARAMS = OFF_B4 + D_OUT;   // 41602
constexpr int MAX_SYS_MAPS = 8;
constexpr int COND = 6 * MAX_SYS_MAPS;     // 48 conditioning parameters

__device__ __forceinline__ bf16r to_bf16(float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const bf16r*>(&h);
}

__device__ __forceinline__ float from_bf16(bf16r v)
{
    return __uint_as_float(((u32)v) << 16);
}

// SiLU and its derivative in training: sigma(z) = 1 / (1 + e^-z) with the
// hardware exponential and reciprocal (relative error a few ulps, far below
// the BF16 rounding of the activations and gradients they feed)
__device__ __forceinline__ float sigmoid_f(float z)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + __expf(-z)));
    return r;
}

__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = sigmoid_f(z);
    return s * (1.0f + z * (1.0f - s));
}

// ---------------------------------------------------------------------------
// GEMM on the fifth-generation tensor cores:
//   D[M][N] = A[M][K] B[N][K]^T,  A and B BF16 and K-major in global memory,
//   D accumulated in FP32 in tensor memory (TMEM).
// CTA tile: 128 rows x the whole width N (64 or 128).  K runs in chunks of
// 64, staged by the CTA's 128 threads into shared memory in the no-swizzle
// K-major layout of 8-row x 16-byte core matrices (K-adjacent cores 128 B
// apart, 8-row groups 1024 B apart).  Two stages: while the tensor core
// multiplies chunk c, the threads stage chunk c + 1.  Thread 0 issues the
// four tcgen05.mma of a chunk (M = 128, N, K = 16 each) and commits them to
// the stage's mbarrier; the stage is refilled only after that barrier
// completes.  The epilogue reads the accumulator with tcgen05.ld: warp w
// owns TMEM lanes 32w..32w+31, so every thread holds one output row.
// Every wait is bounded: on a time-out the CTA records it in g_tc_error,
// skips its epilogue, frees its TMEM and returns.
// ---------------------------------------------------------------------------
enum Epi { EPI_SILU = 1, EPI_SILU_GRAD = 2, EPI_ATOMIC = 3 };

constexpr int TC_M = 128, TC_K = 64, TC_THREADS = 256;
constexpr int TC_NV = 128 * 8 / TC_THREADS;   // 16-byte vectors per thread per operand tile
constexpr int TC_TILE_BYTES = 128 * TC_K * 2;             // 16 KB: 128 rows x 64 K
// dynamic shared memory of the kernel with ST stages of (A, B) chunks, plus
// barriers and alignment; one stage is padded to 50 KB so that at most four
// CTAs share an SM (four times 128 TMEM columns fill its 512)
template <int ST>
constexpr int tc_smem_bytes()
{
    return ST == 1 ? 50 * 1024 : 2 * ST * TC_TILE_BYTES + 1024 + 1024;
}
constexpr u32 TC_WAIT_LIMIT = 1u << 24;
constexpr int TC_COPIES = 16;   // copies of the bias-gradient sums (spread the atomics)

__device__ unsigned int g_tc_error = 0;
// chunk stages of the register-staged GEMM kernel: by the chunks a CTA runs
// (one stage for at most two: four CTAs per SM then take all row tiles of a
// GEMM in one wave; two stages for K-split weight gradients, whose CTAs run
// four chunks).

struct TcArgs {
    int M, N, K;                 // N in {64, 128}
    const bf16r* A; int lda;     // [M][lda], K contiguous
    const bf16r* B; int ldb;     // [N][ldb], K contiguous
    int k_split;                 // K per blockIdx.z, a multiple of TC_K
    int mode;
    const float* bias;           // SILU: [N]
    float* C; int ldc;           // SILU: pre-activation Z out; ATOMIC: C += D
    bf16r* H; int ldh;           // SILU: activation out; SILU_GRAD: dZ out
    bf16r* HT; int ldt;          // SILU, SILU_GRAD: transposed copy [N][ldt] (or null)
    const float* Zin; int ldz;   // SILU_GRAD: pre-activation of the layer
    float* colsum;               // SILU_GRAD: bias gradient partials, [TC_COPIES][N]; CTA b
                                 // adds its column sums into copy b % TC_COPIES
    int K2;                      // tc_rows_kernel<true>: K of the recomputed pre-activation
};

__device__ __forceinline__ u32 smem_addr(const void* p)
{
    return (u32)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading (K) byte offset
// 128, stride (8-row group) byte offset 1024, descriptor version 1 (bit 46),
// base offset 0, no swizzle
__device__ __forceinline__ u64 tc_desc(u32 saddr)
{
    return (u64)((saddr >> 4) & 0x3FFFu) | ((u64)(128u >> 4) << 16) |
           ((u64)(1024u >> 4) << 32) | ((u64)1 << 46);
}

// instruction descriptor of kind::f16: D F32 (bit 4), A and B BF16 (bits 7,
// 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ u32 tc_idesc(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((u32)(N >> 3) << 17) |
           ((u32)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(u32 d_tmem, u64 adesc, u64 bdesc, u32 idesc, u32 acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(u32 bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(u32 bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity)
{
    for (u32 it = 0; it < TC_WAIT_LIMIT; ++it) {
        u32 done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane, without the wait
// (the caller issues tcgen05.wait::ld before using them)
__device__ __forceinline__ void tc_ld16_nowait(u32 taddr, u32 (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(u32 taddr, float (&v)[16])
{
    u32 r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Staging of rows row0 .. row0 + n_rows - 1 (those < rows_valid), K columns
// k0 .. k0 + 63 (those < k_end) of a K-major BF16 matrix into the core-matrix
// layout, zeros elsewhere.  Vector v -> row (v / 64) * 8 + v % 8, K group
// (v / 8) % 8, so each 8-lane phase of a warp writes one contiguous 128-byte
// core matrix.  Two phases -- every load of the tile first, then the shared
// stores -- keep TC_NV loads per thread in flight.
__device__ __forceinline__ void tc_stage_load(uint4 (&val)[TC_NV], const bf16r* src, int ld,
                                              int rows_valid, int row0, int n_rows, int k0,
                                              int k_end)
{
#pragma unroll
    for (int i = 0; i < TC_NV; ++i) {
        const int v = (int)threadIdx.x + i * TC_THREADS;
        const int r = ((v >> 6) << 3) | (v & 7), k8 = (v >> 3) & 7;
        const int gr = row0 + r, gk = k0 + 8 * k8;
        val[i] = make_uint4(0u, 0u, 0u, 0u);
        if (v < n_rows * 8 && gr < rows_valid && gk < k_end) {
            const bf16r* p = src + (size_t)gr * ld + gk;
            if (gk + 8 <= k_end) {
                val[i] = __ldg(reinterpret_cast<const uint4*>(p));
            } else {
                u32 w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (gk + e < k_end) w[e >> 1] |= (u32)p[e] << (16 * (e & 1));
                val[i] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

__device__ __forceinline__ void tc_stage_store(u32 dst, const uint4 (&val)[TC_NV], int n_rows)
{
#pragma unroll
    for (int i = 0; i < TC_NV; ++i) {
        const int v = (int)threadIdx.x + i * TC_THREADS;
        if (v < n_rows * 8) {
            const int r = ((v >> 6) << 3) | (v & 7), k8 = (v >> 3) & 7;
            const u32 a = dst + (u32)((r >> 3) * 1024 + k8 * 128 + (r & 7) * 16);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};"
                         :
                         : "r"(a), "r"(val[i].x), "r"(val[i].y), "r"(val[i].z), "r"(val[i].w)
                         : "memory");
        }
    }
}

__device__ __forceinline__ u32 pack_bf16x2(float a, float b)
{
    return (u32)to_bf16(a) | ((u32)to_bf16(b) << 16);
}

// pre-activations of columns c0 .. c0 + 15 of this thread's row (SILU_GRAD)
__device__ __forceinline__ void tc_load_z(const TcArgs& g, int row, int c0, float (&z)[16])
{
    if (g.mode != EPI_SILU_GRAD || row >= g.M) return;
    const float4* zp = reinterpret_cast<const float4*>(g.Zin + (size_t)row * g.ldz + c0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = __ldg(zp + q);
        z[4 * q] = t.x; z[4 * q + 1] = t.y; z[4 * q + 2] = t.z; z[4 * q + 3] = t.w;
    }
}

// sums of 16 values over the warp's 32 lanes by halving exchanges (16
// shuffles instead of 80): on return lanes 2c and 2c + 1 hold the sum of
// value c
__device__ __forceinline__ float warp_colsum16(float (&h)[16])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1) {
        // this lane keeps values [0, w) or [w, 2w) of the current 2w and
        // adds the partner's copy of the same ones; the bit that decides is
        // lane bit log2(w) + 1 (16, 8, 4, 2 for w = 8, 4, 2, 1)
        const bool upper = (lane & (2 * w)) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const float send = upper ? h[k] : h[k + w];
            const float keep = upper ? h[k + w] : h[k];
            h[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * w);
        }
    }
    return h[0] + __shfl_xor_sync(0xffffffffu, h[0], 1);
}

__device__ __forceinline__ void tc_epilogue(const TcArgs& g, int row, int c0, const float (&v)[16],
                                            const float (&zi)[16], float* s_col,
                                            const float* bias)
{
    const bool in = row < g.M;
    if (g.mode == EPI_ATOMIC) {
        if (in) {
            float* c = g.C + (size_t)row * g.ldc + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cfs_red_add_v4f32(c + 4 * q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2],
                                                         v[4 * q + 3]));
        }
        return;
    }
    float h[16];
    if (g.mode == EPI_SILU) {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            z[j] = v[j] + bias[c0 + j];
            h[j] = silu_f(z[j]);
        }
        if (in && g.C) {
            float4* zc = reinterpret_cast<float4*>(g.C + (size_t)row * g.ldc + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) zc[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
        }
    } else {   // EPI_SILU_GRAD
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = in ? v[j] * silu_grad_f(zi[j]) : 0.0f;
        // bias gradient: column sums over the warp's 32 rows, one atomic per column
        float hs[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hs[j] = h[j];
        const float s = warp_colsum16(hs);
        const int lane = threadIdx.x & 31;
        if (!(lane & 1) && s != 0.0f) atomicAdd(s_col + c0 + (lane >> 1), s);
    }
    if (in && g.H) {
        uint4* hp = reinterpret_cast<uint4*>(g.H + (size_t)row * g.ldh + c0);
        hp[0] = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                           pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
        hp[1] = make_uint4(pack_bf16x2(h[8], h[9]), pack_bf16x2(h[10], h[11]),
                           pack_bf16x2(h[12], h[13]), pack_bf16x2(h[14], h[15]));
    }
    if (in && g.HT) {
        // consecutive lanes hold consecutive rows: each column's stores coalesce
#pragma unroll
        for (int j = 0; j < 16; ++j) g.HT[(size_t)(c0 + j) * g.ldt + row] = to_bf16(h[j]);
    }
}

template <int ST>
__global__ void __launch_bounds__(TC_THREADS) tc_gemm_kernel(const __grid_constant__ TcArgs g)
{
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
    // stage s: A at sm + 2 s TILE, B right after it
    u64* bars = reinterpret_cast<u64*>(sm + 2 * ST * TC_TILE_BYTES);
    u32* s_tmem = reinterpret_cast<u32*>(sm + 2 * ST * TC_TILE_BYTES + 64);
    float* s_col = reinterpret_cast<float*>(sm + 2 * ST * TC_TILE_BYTES + 128);   // [128]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * TC_M;
    const int kb = blockIdx.z * g.k_split;
    const int ke = min(g.K, kb + g.k_split);
    const int n_chunks = ke > kb ? (ke - kb + TC_K - 1) / TC_K : 0;
    const u32 ncols = g.N <= 64 ? 64u : 128u;
    // stage s's barrier completes once per chunk c = s, s + ST, ...: chunk c
    // is its (c / ST)-th phase
    auto bar = [&](int c) { return smem_addr(&bars[c % ST]); };
    auto phase = [](int c) { return (u32)(c / ST) & 1u; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(s_tmem)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid < 128) s_col[tid] = 0.0f;
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < ST; ++q) mbar_init(smem_addr(&bars[q]), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tmem = *s_tmem;
    const u32 idesc = tc_idesc(g.N);

    bool ok = true;
    for (int c = 0; c < n_chunks; ++c) {
        const int s = c % ST;
        // the stage's previous chunk (c - ST) must have left the tensor core
        if (c >= ST) ok = mbar_wait(bar(c - ST), phase(c - ST));
        if (!__syncthreads_and(ok)) { ok = false; break; }
        const int k0 = kb + c * TC_K;
        const u32 sA = smem_addr(sm + 2 * s * TC_TILE_BYTES), sB = sA + TC_TILE_BYTES;
        {
            uint4 va[TC_NV], vb[TC_NV];
            tc_stage_load(va, g.A, g.lda, g.M, m0, TC_M, k0, ke);
            tc_stage_load(vb, g.B, g.ldb, g.N, 0, g.N, k0, ke);
            tc_stage_store(sA, va, TC_M);
            tc_stage_store(sB, vb, g.N);
        }
        // generic-proxy stores -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk)
                tc_mma(tmem, tc_desc(sA + kk * 256), tc_desc(sB + kk * 256), idesc,
                       (c > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar(c));
        }
    }
    // epilogue split: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows)
    // and the columns of half w / 4
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + (tid & 31);
    const int c_begin = half * (g.N / 2), c_end = c_begin + g.N / 2;
    float z_next[16];
    tc_load_z(g, row, c_begin, z_next);   // independent of the MMAs: overlaps them
    if (ok && n_chunks > 0) {
        const int last = n_chunks - 1;
        ok = mbar_wait(bar(last), phase(last));
    }
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (ok && n_chunks > 0) {
        const u32 lane_base = tmem + ((u32)(quad * 32) << 16);
        for (int c0 = c_begin; c0 < c_end; c0 += 16) {
            float z[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = z_next[j];
            if (c0 + 16 < c_end) tc_load_z(g, row, c0 + 16, z_next);
            float v[16];
            tc_ld16(lane_base + (u32)c0, v);
            tc_epilogue(g, row, c0, v, z, s_col, g.bias);
        }
    } else if (!ok && tid == 0) {
        atomicOr(&g_tc_error, (unsigned)CFS_DEVICE_ERR_TC_TIMEOUT);
        // give in-flight MMAs a bounded chance to drain before TMEM is freed
        if (n_chunks > 0) {
            const int last = n_chunks - 1;
            mbar_wait(bar(last), phase(last));
        }
    }
    tc_fence_before();
    __syncthreads();
    // the CTA's bias-gradient column sums: one atomic per column into copy
    // blockIdx.x % TC_COPIES
    if (g.mode == EPI_SILU_GRAD && ok && tid < g.N && s_col[tid] != 0.0f)
        atomicAdd(g.colsum + (blockIdx.x % TC_COPIES) * g.N + tid, s_col[tid]);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :
                     : "r"(tmem), "r"(ncols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// The row GEMMs of training and inference, D[rows][128] = A[rows][K] W^T
// (K = 64 or 128) with the SILU / SILU_GRAD epilogues, as one persistent
// warp-specialized kernel per GEMM (one CTA per SM, row tiles of 128 strided
// over the CTAs):
//   warp 0  -- TMA: the weights once, then each tile's A into a ring of
//              TrCfg::STAGES shared-memory slots (2D tensor maps, boxes of 128
//              rows x 8 K elements, i.e. one 16-byte column of core
//              matrices: K-adjacent cores 2048 B apart, 8-row groups 128 B);
//   warp 1  -- TMEM owner; one thread issues the tile's tcgen05.mma into one
//              of two accumulator buffers and commits it to the slot's
//              "empty" barrier and the accumulator's "full" barrier;
//   warps 2..17 -- the epilogue of tile i (warp w reads TMEM lanes
//              32 (w % 4) .. + 31 and a quarter of the columns) while tile
//              i + 1 is loaded and multiplied; each warp arrives on the
//              accumulator's "empty" barrier as soon as its columns are in
//              registers.
// tc_rows_kernel<true> (SILU_GRAD of the input gradients) also loads the
// layer below's activations A2 and weights W2 and multiplies them into a
// second accumulator: its pre-activation Z = A2 W2^T + b, the same MMAs the
// forward ran, so the SiLU derivative needs no stored Z.
// Every wait is bounded; a time-out sets g_tc_error and the role stops.
// ---------------------------------------------------------------------------
constexpr int TR_EPI_WARPS = 16;
constexpr int TR_THREADS = 32 * (2 + TR_EPI_WARPS);
constexpr int TR_TILE = 128 * 128 * 2;   // one A tile or the weights at K = 128

// shapes of the two variants: RC also recomputes the pre-activation Z of
// the layer below (second operand pair, second accumulator)
template <bool RC>
struct TrCfg {
    static constexpr int STAGES = RC ? 2 : 3;
    static constexpr int SLOT = RC ? 2 * TR_TILE : TR_TILE;      // A (and A2) of a tile
    static constexpr int WEIGHTS = RC ? 2 * TR_TILE : TR_TILE;   // W (and W2)
    static constexpr int SMEM = 1024 + WEIGHTS + STAGES * SLOT + 256 + 4 * 128;
    static constexpr int ACC = RC ? 256 : 128;                   // TMEM columns per buffer
};

__device__ __forceinline__ u64 tc_desc_kn(u32 saddr, u32 lbo, u32 sbo)
{
    return (u64)((saddr >> 4) & 0x3FFFu) | ((u64)((lbo >> 4) & 0x3FFFu) << 16) |
           ((u64)((sbo >> 4) & 0x3FFFu) << 32) | ((u64)1 << 46);
}

__device__ __forceinline__ void mbar_expect_tx(u32 bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(u32 bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// one box of a 2D tensor map at element coordinates (x = K, y = row)
__device__ __forceinline__ void tma_load_2d(u32 dst, const CUtensorMap* map, int x, int y, u32 bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<u64>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

template <bool RC>
__global__ void __launch_bounds__(TR_THREADS, 1) tc_rows_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
    const __grid_constant__ TcArgs g)
{
    using Cf = TrCfg<RC>;
    constexpr int ST = Cf::STAGES;
    extern __shared__ unsigned char tr_smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tr_smem_raw) + 1023) & ~(uintptr_t)1023);
    // W at sm (W2 after it), then ST slots of A (A2 after it in the slot)
    const u32 sB = smem_addr(sm), sB2 = sB + TR_TILE, sA = sB + Cf::WEIGHTS;
    u64* bars = reinterpret_cast<u64*>(sm + Cf::WEIGHTS + ST * Cf::SLOT);
    // barriers: full[s], empty[s] (s < ST), wfull, tfull[2], tempty[2]
    auto full = [&](int s) { return smem_addr(&bars[s]); };
    auto empty = [&](int s) { return smem_addr(&bars[ST + s]); };
    const u32 wfull = smem_addr(&bars[2 * ST]);
    auto tfull = [&](int b) { return smem_addr(&bars[2 * ST + 1 + b]); };
    auto tempty = [&](int b) { return smem_addr(&bars[2 * ST + 3 + b]); };
    u32* s_tmem = reinterpret_cast<u32*>(bars + 16);
    __shared__ int s_err;
    float* s_col = reinterpret_cast<float*>(bars + 32);   // [128]
    // SILU: the layer's bias; RC: the bias of the recomputed pre-activation
    __shared__ float s_bias[128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (g.M + TC_M - 1) / TC_M;
    const int kch = g.K / 8, kch2 = RC ? g.K2 / 8 : 0;   // 16-byte K columns
    const u32 tile_bytes = (u32)(TC_M * (g.K + (RC ? g.K2 : 0)) * 2);
    const u32 w_bytes = tile_bytes;                     // W rows = tile rows = 128

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(s_tmem)), "r"(2u * (u32)Cf::ACC)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x < 128) {
        s_col[threadIdx.x] = 0.0f;
        s_bias[threadIdx.x] = (g.mode == EPI_SILU || RC) ? g.bias[threadIdx.x] : 0.0f;
    }
    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < ST; ++s) {
            mbar_init(full(s), 1u);
            mbar_init(empty(s), 1u);
        }
        mbar_init(wfull, 1u);
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1u);
            mbar_init(tempty(b), (u32)TR_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tmem = *s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(wfull, w_bytes);
            for (int kc = 0; kc < kch; ++kc) tma_load_2d(sB + kc * 2048, &tmB, kc * 8, 0, wfull);
            for (int kc = 0; kc < kch2; ++kc) tma_load_2d(sB2 + kc * 2048, &tmB2, kc * 8, 0, wfull);
            int i = 0, issued = 0;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
                const int s = i % ST;
                if (i >= ST && !mbar_wait(empty(s), (u32)(i / ST - 1) & 1u)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                mbar_expect_tx(full(s), tile_bytes);
                const u32 a = sA + (u32)(s * Cf::SLOT);
                for (int kc = 0; kc < kch; ++kc)
                    tma_load_2d(a + kc * 2048, &tmA, kc * 8, tile * TC_M, full(s));
                for (int kc = 0; kc < kch2; ++kc)
                    tma_load_2d(a + TR_TILE + kc * 2048, &tmA2, kc * 8, tile * TC_M, full(s));
                issued = i + 1;
            }
            // every load issued has landed before the CTA may leave
            for (int j = (issued > ST ? issued - ST : 0); j < issued; ++j)
                mbar_wait(full(j % ST), (u32)(j / ST) & 1u);
            mbar_wait(wfull, 0u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const u32 idesc = tc_idesc(128);
            bool ok = mbar_wait(wfull, 0u);
            int i = 0, committed = 0;
            for (int tile = blockIdx.x; ok && tile < n_tiles; tile += gridDim.x, ++i) {
                const int s = i % ST, b = i & 1;
                if (!mbar_wait(full(s), (u32)(i / ST) & 1u)) { ok = false; break; }
                if (i >= 2 && !mbar_wait(tempty(b), (u32)(i / 2 - 1) & 1u)) { ok = false; break; }
                tc_fence_after();
                const u32 a = sA + (u32)(s * Cf::SLOT), d = tmem + (u32)(b * Cf::ACC);
                for (int kk = 0; kk < g.K / 16; ++kk)
                    tc_mma(d, tc_desc_kn(a + kk * 4096, 2048u, 128u),
                           tc_desc_kn(sB + kk * 4096, 2048u, 128u), idesc, kk > 0 ? 1u : 0u);
                // the layer below's pre-activation: the forward's MMAs on the
                // same operands in the same order, so the same bits
                for (int kk = 0; kk < kch2 / 2; ++kk)
                    tc_mma(d + 128u, tc_desc_kn(a + TR_TILE + kk * 4096, 2048u, 128u),
                           tc_desc_kn(sB2 + kk * 4096, 2048u, 128u), idesc, kk > 0 ? 1u : 0u);
                tc_commit(empty(s));
                tc_commit(tfull(b));
                committed = i + 1;
            }
            if (!ok) atomicExch(&s_err, 1);
            // the last accumulator's MMAs complete before TMEM is freed
            if (committed > 0) {
                const int j = committed - 1;
                mbar_wait(tfull(j & 1), (u32)(j / 2) & 1u);
            }
        }
    } else {
        const int ew = warp - 2, quad = warp & 3;
        const int c_begin = (ew >> 2) * 32;
        int i = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            const int row = tile * TC_M + quad * 32 + lane;
            float z_next[16];
            if (!RC) tc_load_z(g, row, c_begin, z_next);   // overlaps the wait
            if (!mbar_wait(tfull(b), (u32)(i / 2) & 1u)) {
                atomicExch(&s_err, 1);
                break;
            }
            tc_fence_after();
            const u32 base = tmem + ((u32)(quad * 32) << 16) + (u32)(b * Cf::ACC);
            if constexpr (RC) {
                // per 16 columns: the product and the recomputed pre-activation
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = c_begin + 16 * h;
                    u32 r[16], q[16];
                    tc_ld16_nowait(base + (u32)c0, r);
                    tc_ld16_nowait(base + 128u + (u32)c0, q);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (h == 1) {   // the accumulators are read: release them
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(tempty(b));
                    }
                    float v[16], z[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] = __uint_as_float(r[j]);
                        z[j] = __uint_as_float(q[j]) + s_bias[c0 + j];
                    }
                    tc_epilogue(g, row, c0, v, z, s_col, s_bias);
                }
            } else {
                // both 16-column loads in flight before the one wait
                u32 r0[16], r1[16];
                tc_ld16_nowait(base + (u32)c_begin, r0);
                tc_ld16_nowait(base + (u32)(c_begin + 16), r1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the accumulator is read: release it to the MMA thread before
                // the arithmetic and the stores
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty(b));
                {
                    float v[16], z[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        v[j] = __uint_as_float(r0[j]);
                        z[j] = z_next[j];
                    }
                    tc_load_z(g, row, c_begin + 16, z_next);
                    tc_epilogue(g, row, c_begin, v, z, s_col, s_bias);
                }
                {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r1[j]);
                    tc_epilogue(g, row, c_begin + 16, v, z_next, s_col, s_bias);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (g.mode == EPI_SILU_GRAD && !s_err && threadIdx.x < 128 && s_col[threadIdx.x] != 0.0f)
        atomicAdd(g.colsum + (blockIdx.x % TC_COPIES) * 128 + threadIdx.x, s_col[threadIdx.x]);
    if (threadIdx.x == 0 && s_err) atomicOr(&g_tc_error, (unsigned)CFS_DEVICE_ERR_TC_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2u * (u32)Cf::ACC)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradients dW[M = 128][N] += A[128][K] B[N][K]^T (A = dZ^T, B = H^T or
// U^T, both K-major over the rows, N = 128 or 64) split over K: CTA b takes
// a run of 64-row K chunks.  Warp 0 loads each chunk's A and B with TMA into
// a ring of SK_STAGES slots, one thread of warp 1 accumulates the chunks into
// one TMEM accumulator, and warps 2..5 add it to dW with vector reductions at
// the end.  Every wait is bounded, as in tc_rows_kernel.
// ---------------------------------------------------------------------------
constexpr int SK_STAGES = 4;
constexpr int SK_THREADS = 32 * 6;
constexpr int SK_SLOT = 2 * 128 * TC_K * 2;   // A and B chunk (64 K) of 128 rows each
constexpr int SK_SMEM = 1024 + SK_STAGES * SK_SLOT + 256;

__global__ void __launch_bounds__(SK_THREADS, 1) tc_splitk_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ TcArgs g)
{
    extern __shared__ unsigned char sk_smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sk_smem_raw) + 1023) & ~(uintptr_t)1023);
    const u32 s0 = smem_addr(sm);
    u64* bars = reinterpret_cast<u64*>(sm + SK_STAGES * SK_SLOT);
    auto full = [&](int s) { return smem_addr(&bars[s]); };
    auto empty = [&](int s) { return smem_addr(&bars[SK_STAGES + s]); };
    const u32 tdone = smem_addr(&bars[2 * SK_STAGES]);
    u32* s_tmem = reinterpret_cast<u32*>(bars + 16);
    __shared__ int s_err;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_chunks = (g.K + TC_K - 1) / TC_K;
    const int per = (n_chunks + gridDim.x - 1) / gridDim.x;
    const int c_first = blockIdx.x * per, c_last = min(n_chunks, c_first + per);
    const u32 chunk_bytes = (u32)((128 + g.N) * TC_K * 2);
    const u32 ncols = g.N <= 64 ? 64u : 128u;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(s_tmem)), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < SK_STAGES; ++s) {
            mbar_init(full(s), 1u);
            mbar_init(empty(s), 1u);
        }
        mbar_init(tdone, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tmem = *s_tmem;
    // slot s: A at s0 + s SLOT ([8 K columns][128 rows][16 B]), B after 16 KB
    if (warp == 0) {
        if (lane == 0) {
            int i = 0, issued = 0;
            for (int c = c_first; c < c_last; ++c, ++i) {
                const int s = i % SK_STAGES;
                if (i >= SK_STAGES && !mbar_wait(empty(s), (u32)(i / SK_STAGES - 1) & 1u)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                mbar_expect_tx(full(s), chunk_bytes);
                const u32 a = s0 + (u32)(s * SK_SLOT), b = a + 128 * TC_K * 2;
                for (int kc = 0; kc < TC_K / 8; ++kc) {
                    tma_load_2d(a + kc * 2048, &tmA, c * TC_K + kc * 8, 0, full(s));
                    tma_load_2d(b + kc * (u32)(g.N * 16), &tmB, c * TC_K + kc * 8, 0, full(s));
                }
                issued = i + 1;
            }
            for (int j = (issued > SK_STAGES ? issued - SK_STAGES : 0); j < issued; ++j)
                mbar_wait(full(j % SK_STAGES), (u32)(j / SK_STAGES) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const u32 idesc = tc_idesc(g.N);
            bool ok = true;
            int i = 0;
            for (int c = c_first; c < c_last; ++c, ++i) {
                const int s = i % SK_STAGES;
                if (!mbar_wait(full(s), (u32)(i / SK_STAGES) & 1u)) { ok = false; break; }
                tc_fence_after();
                const u32 a = s0 + (u32)(s * SK_SLOT), b = a + 128 * TC_K * 2;
#pragma unroll
                for (int kk = 0; kk < TC_K / 16; ++kk)
                    tc_mma(tmem, tc_desc_kn(a + kk * 4096, 2048u, 128u),
                           tc_desc_kn(b + kk * (u32)(g.N * 32), (u32)(g.N * 16), 128u), idesc,
                           (i > 0 || kk > 0) ? 1u : 0u);
                tc_commit(empty(s));
            }
            if (!ok) atomicExch(&s_err, 1);
            tc_commit(tdone);   // every MMA issued above (none: arrives at once)
        }
    } else {
        const int quad = warp & 3;
        const bool any = c_last > c_first;
        if (!mbar_wait(tdone, 0u)) {
            atomicExch(&s_err, 1);
        } else if (any && !s_err) {
            tc_fence_after();
            const int row = quad * 32 + lane;
            const u32 base = tmem + ((u32)(quad * 32) << 16);
            const float zi[16] = {};
            for (int c0 = 0; c0 < g.N; c0 += 16) {
                float v[16];
                tc_ld16(base + (u32)c0, v);
                tc_epilogue(g, row, c0, v, zi, nullptr, nullptr);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_err) atomicOr(&g_tc_error, (unsigned)CFS_DEVICE_ERR_TC_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ncols)
                     : "memory");
    }
}

// output layer forward Y = H3 W4^T + b4 (N = 2: a dot product per output,
// not a tensor-core shape): one thread per row
__global__ void __launch_bounds__(256) out_forward_kernel(const bf16r* __restrict__ H3,
                                                          const bf16r* __restrict__ wb,
                                                          const float* __restrict__ w, int B,
                                                          float* Y)
{
    __shared__ float w4[D_OUT][HID];
    for (int e = threadIdx.x; e < D_OUT * HID; e += blockDim.x)
        w4[e / HID][e % HID] = from_bf16(wb[OFF_W4 + e]);
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B) return;
    const uint4* h = reinterpret_cast<const uint4*>(H3 + (size_t)r * HID);
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll 4
    for (int q = 0; q < HID / 8; ++q) {
        const uint4 p = h[q];
        const u32 pw[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float x = from_bf16((bf16r)(pw[e >> 1] >> (16 * (e & 1))));
            y0 = fmaf(x, w4[0][8 * q + e], y0);
            y1 = fmaf(x, w4[1][8 * q + e], y1);
        }
    }
    Y[2 * r] = y0 + w[OFF_B4];
    Y[2 * r + 1] = y1 + w[OFF_B4 + 1];
}

// gradient partial sums gathered in TC_COPIES copies to spread the atomics:
// [2][TC_COPIES][HID] bias gradients b2 and b1 (GEMM epilogues), then
// [TC_COPIES][OB_PART] of the output layer's backward: W4 rows 0 and 1
// (2 x HID), b3 (HID), b4 (2), padding
constexpr int OB_PART = 3 * HID + 4;
constexpr int PART_FLOATS = TC_COPIES * (2 * HID + OB_PART);

// sums the copies and adds them to grads
__global__ void __launch_bounds__(512) part_reduce_kernel(const float* __restrict__ part,
                                                          float* grads)
{
    for (int e = threadIdx.x; e < 2 * HID + 3 * HID + 2; e += blockDim.x) {
        float s = 0.0f;
        if (e < 2 * HID) {
            const int l = e / HID, c = e % HID;
            for (int k = 0; k < TC_COPIES; ++k) s += part[((size_t)l * TC_COPIES + k) * HID + c];
            grads[(l == 0 ? OFF_B2 : OFF_B1) + c] += s;
        } else {
            const int q = e - 2 * HID;
            const float* ob = part + (size_t)2 * TC_COPIES * HID;
            for (int k = 0; k < TC_COPIES; ++k) s += ob[(size_t)k * OB_PART + q];
            grads[q < 2 * HID ? OFF_W4 + q : (q < 3 * HID ? OFF_B3 + q - 2 * HID
                                                          : OFF_B4 + q - 3 * HID)] += s;
        }
    }
}

// U [rows][D_IN] -> UT [D_IN][ldt] (the K-major operand of dW1)
__global__ void __launch_bounds__(256) transpose_in_kernel(const bf16r* __restrict__ U, int rows,
                                                           bf16r* UT, int ldt)
{
    __shared__ bf16r tile[32][D_IN + 2];
    const int r0 = blockIdx.x * 32;
    for (int e = threadIdx.x; e < 32 * D_IN; e += blockDim.x) {
        const int r = e / D_IN, c = e % D_IN;
        tile[r][c] = r0 + r < rows ? U[(size_t)(r0 + r) * D_IN + c] : (bf16r)0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * D_IN; e += blockDim.x) {
        const int c = e / 32, r = e % 32;
        if (r0 + r < rows) UT[(size_t)c * ldt + r0 + r] = tile[r][c];
    }
}

// output layer backward: dH3 = dY W4 (N = 2, not a tensor-core shape), dZ3 =
// dH3 * silu'(Z3) written as dZ3 and its transpose dZ3^T; dW4 = dY^T H3,
// db3 = sum dZ3, db4 = sum dY.  A block takes OB_ROWS rows, a warp one row
// at a time, lane l the four units 4l .. 4l+3 (16-byte loads of Z3, 8-byte
// loads of H3); the block's dZ3 tile is transposed in shared memory, and its
// sums combine across warps there before one atomic per value into copy
// blockIdx.x % TC_COPIES of `part`.
constexpr int OB_ROWS = 64;
constexpr int OB_THREADS = 256;

__global__ void __launch_bounds__(OB_THREADS) out_backward_kernel(const float* __restrict__ dY,
                                                                  const bf16r* __restrict__ wb,
                                                                  const bf16r* __restrict__ H3,
                                                                  const float* __restrict__ Z3,
                                                                  int B, bf16r* dZ3, bf16r* dZ3T,
                                                                  int ldt, float* part)
{
    __shared__ bf16r tT[HID][OB_ROWS + 1];   // the block's dZ3 tile, transposed
    __shared__ float s_sum[3 * HID + 2];     // W4 rows 0 and 1, b3, b4
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = 4 * lane;
    float w0[4], w1[4], a0[4], a1[4], ab[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        w0[j] = from_bf16(wb[OFF_W4 + c + j]);
        w1[j] = from_bf16(wb[OFF_W4 + HID + c + j]);
        a0[j] = a1[j] = ab[j] = 0.0f;
    }
    float b40 = 0.0f, b41 = 0.0f;
    for (int e = threadIdx.x; e < 3 * HID + 2; e += OB_THREADS) s_sum[e] = 0.0f;
    const int r0 = blockIdx.x * OB_ROWS;
#pragma unroll 2
    for (int k = warp; k < OB_ROWS; k += OB_THREADS / 32) {
        const int r = r0 + k;
        if (r >= B) break;
        const float y0 = dY[2 * r], y1 = dY[2 * r + 1];
        const float4 z = *reinterpret_cast<const float4*>(Z3 + (size_t)r * HID + c);
        const uint2 hv = *reinterpret_cast<const uint2*>(H3 + (size_t)r * HID + c);
        const float zz[4] = {z.x, z.y, z.z, z.w};
        const float h[4] = {__uint_as_float(hv.x << 16), __uint_as_float(hv.x & 0xFFFF0000u),
                            __uint_as_float(hv.y << 16), __uint_as_float(hv.y & 0xFFFF0000u)};
        bf16r db[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float dh = fmaf(y0, w0[j], y1 * w1[j]);
            const float d = dh * silu_grad_f(zz[j]);
            db[j] = to_bf16(d);
            tT[c + j][k] = db[j];
            ab[j] += d;
            a0[j] = fmaf(y0, h[j], a0[j]);
            a1[j] = fmaf(y1, h[j], a1[j]);
        }
        *reinterpret_cast<uint2*>(dZ3 + (size_t)r * HID + c) =
            make_uint2((u32)db[0] | ((u32)db[1] << 16), (u32)db[2] | ((u32)db[3] << 16));
        b40 += y0;
        b41 += y1;
    }
    __syncthreads();   // tT complete, s_sum zeroed
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        atomicAdd(&s_sum[c + j], a0[j]);
        atomicAdd(&s_sum[HID + c + j], a1[j]);
        atomicAdd(&s_sum[2 * HID + c + j], ab[j]);
    }
    if (lane == 0) {
        atomicAdd(&s_sum[3 * HID], b40);
        atomicAdd(&s_sum[3 * HID + 1], b41);
    }
    // dZ3^T rows: a warp writes 64 consecutive rows of one unit as 32 words
    for (int e = threadIdx.x; e < HID * (OB_ROWS / 2); e += OB_THREADS) {
        const int u = e / (OB_ROWS / 2), jp = 2 * (e % (OB_ROWS / 2));
        const int r = r0 + jp;
        if (r + 1 < B) {
            *reinterpret_cast<u32*>(dZ3T + (size_t)u * ldt + r) =
                (u32)tT[u][jp] | ((u32)tT[u][jp + 1] << 16);
        } else if (r < B) {
            dZ3T[(size_t)u * ldt + r] = tT[u][jp];
        }
    }
    __syncthreads();   // s_sum complete
    float* cp = part + (size_t)(blockIdx.x % TC_COPIES) * OB_PART;
    for (int e = threadIdx.x; e < 3 * HID + 2; e += OB_THREADS)
        if (s_sum[e] != 0.0f) atomicAdd(cp + e, s_sum[e]);
}

// ---------------------------------------------------------------------------
// sliced-Wasserstein loss and gradient.  A CTA takes one system and a run of
// its projections; a group of G = N / 8 threads sorts one projection at a
// time, each thread holding 8 projected predicted keys (x) and 8 projected
// target keys (y).
//
// Sorting network: bitonic.  Merge k (blocks of 2^k positions) runs
// compare-exchange stages on position bits k-1, ..., 0.  A position's bits
// are split into a window of 3 register bits [a, a + 3) -- the key's slot
// in its thread -- and the others, which number the thread in the group; a
// stage on a bit of the window is a min/max of two slots of one thread.
// When the next stage's bit lies outside the window, the group moves its
// keys through shared memory into the window that holds it (19 moves for
// N = 1024, each one barrier of the group's threads; two buffers alternate).  Blocks that a merge
// sorts descending hold their keys negated, so every stage puts the smaller
// key at the lower position and a merge boundary only flips signs.  The
// shared-memory slots are XOR-swizzled so that the 16 lanes of a half-warp
// hit distinct banks in every window.
//
// After the sort, thread t holds ranks 8t .. 8t+7.  A point's rank is then
// found by binary search of its own key (recomputed bit for bit) among the
// sorted predicted keys, stored in the search's breadth-first order, so the
// network carries no indices.  Gradients of the
// group's projections are summed per point in shared memory (each point
// belongs to one thread of the group), then over the groups, then added to
// dX with one atomic per coordinate and CTA.  Keys must be finite.
// ---------------------------------------------------------------------------
constexpr int SW_E = 8;            // keys per thread and set
constexpr int SW_THREADS = 256;    // threads per CTA at most

__device__ __forceinline__ float sw_key(float u0, float u1, float c, float sn)
{
    return fmaf(u0, c, u1 * sn);
}

// bank swizzle of a float2 slot: bits 4, 5, 6 fold into the low bits
__host__ __device__ constexpr int sw_swz(int p)
{
    return p ^ (((p >> 4) & 1) << 1) ^ (((p >> 5) & 1) << 2) ^ (((p >> 6) & 1) * 9);
}

// position bits of thread t in window a (slot bits left zero)
__device__ __forceinline__ int sw_tpos(int a, int t)
{
    return (t & ((1 << a) - 1)) | ((t >> a) << (a + 3));
}

// compare-exchange of the slot pairs that differ in register bit M
template <int M>
__device__ __forceinline__ void sw_reg_stage(float (&x)[SW_E], float (&y)[SW_E])
{
#pragma unroll
    for (int e = 0; e < SW_E; ++e) {
        if (e & (1 << M)) continue;
        const int f = e | (1 << M);
        const float xl = fminf(x[e], x[f]), xh = fmaxf(x[e], x[f]);
        const float yl = fminf(y[e], y[f]), yh = fmaxf(y[e], y[f]);
        x[e] = xl; x[f] = xh;
        y[e] = yl; y[f] = yh;
    }
}

// barrier of the G threads of group g: a named barrier (ids 1 ..) for whole
// warps, the group's lanes of its warp below that
template <int G>
__device__ __forceinline__ void sw_group_sync(int g)
{
    if constexpr (G >= 64) {
        asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(G) : "memory");
    } else if constexpr (G == 32) {
        __syncwarp();
    } else {
        __syncwarp(((1u << G) - 1u) << ((threadIdx.x & 31u) & ~(unsigned)(G - 1)));
    }
}

// moves the group's keys from window A to window NA through buffer `par`
template <int N, int A, int NA>
__device__ __forceinline__ void sw_move(float (&x)[SW_E], float (&y)[SW_E], int t, int g,
                                        float2* base, int& par)
{
    float2* buf = base + (par ? N : 0);
    par ^= 1;
    // t passes through an opaque move so that each move computes its own
    // addresses here instead of all of them staying live from the start
    int tv;
    asm volatile("mov.b32 %0, %1;" : "=r"(tv) : "r"(t));
    t = tv;
    const int pw = sw_swz(sw_tpos(A, t));
#pragma unroll
    for (int e = 0; e < SW_E; ++e) buf[pw ^ sw_swz(e << A)] = make_float2(x[e], y[e]);
    sw_group_sync<N / SW_E>(g);
    const int pr = sw_swz(sw_tpos(NA, t));
#pragma unroll
    for (int e = 0; e < SW_E; ++e) {
        const float2 v = buf[pr ^ sw_swz(e << NA)];
        x[e] = v.x;
        y[e] = v.y;
    }
}

// the windows of merge K from the one whose top stage bit is HI down; the
// keys are in window CUR on entry and in window 0 on return
template <int N, int K, int HI, int CUR>
__device__ __forceinline__ void sw_windows(float (&x)[SW_E], float (&y)[SW_E], int t, int g,
                                           float2* base, int& par)
{
    constexpr int A = HI >= 2 ? HI - 2 : 0;
    if constexpr (A != CUR) sw_move<N, CUR, A>(x, y, t, g, base, par);
    if constexpr (HI - A >= 2) sw_reg_stage<2>(x, y);
    if constexpr (HI - A >= 1) sw_reg_stage<1>(x, y);
    sw_reg_stage<0>(x, y);
    if constexpr (A > 0) sw_windows<N, K, A - 1, A>(x, y, t, g, base, par);
}

// sign of a key in merge K: negative where position bit K is set (the
// descending blocks); the last merge (2^K = N) is ascending everywhere
template <int N, int K>
__device__ __forceinline__ bool sw_neg(int p)
{
    return (1 << K) < N && ((p >> K) & 1);
}

template <int N, int K>
__device__ __forceinline__ void sw_merges(float (&x)[SW_E], float (&y)[SW_E], int t, int g,
                                          float2* base, int& par)
{
    sw_windows<N, K, K - 1, 0>(x, y, t, g, base, par);
    if constexpr ((1 << K) < N) {
        // window 0 holds position (t << 3) | e: flip where merge K and K + 1
        // disagree on the sign (t opaque again, as in the moves)
        int tv;
        asm volatile("mov.b32 %0, %1;" : "=r"(tv) : "r"(t));
#pragma unroll
        for (int e = 0; e < SW_E; ++e) {
            const int p = (tv << 3) | e;
            const bool f = sw_neg<N, K>(p) != sw_neg<N, K + 1>(p);
            const float sg = f ? -1.0f : 1.0f;
            x[e] *= sg;
            y[e] *= sg;
        }
        sw_merges<N, K + 1>(x, y, t, g, base, par);
    }
}

template <int N>
__global__ void __launch_bounds__(SW_THREADS, 3) sw_kernel(const float* __restrict__ X,
                                                          const float* __restrict__ T,
                                                          const float* __restrict__ phi, int P,
                                                          int pc, float scale, float* loss,
                                                          float* dX)
{
    constexpr int G = N / SW_E;
    extern __shared__ float4 sw_smem[];
    const int groups = blockDim.x / G;
    float4* pts = sw_smem;                             // [8][G] (x0, x1, t0, t1), point 8t+e at e*G+t
    float2* gacc = reinterpret_cast<float2*>(pts + N); // [groups][N] gradient sums
    float2* bufs = gacc + (size_t)groups * N;          // [groups][2][N]
    __shared__ float red[SW_THREADS / 32];
    const int g = threadIdx.x / G, t = threadIdx.x % G;
    const int cps = (P + pc - 1) / pc;
    const int s = blockIdx.x / cps, j0 = (blockIdx.x % cps) * pc, j1 = min(P, j0 + pc);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const size_t r = ((size_t)s * N + i) * 2;
        pts[(i & (SW_E - 1)) * G + (i >> 3)] = make_float4(X[r], X[r + 1], T[r], T[r + 1]);
    }
    for (int i = threadIdx.x; i < groups * N; i += blockDim.x) gacc[i] = make_float2(0.0f, 0.0f);
    __syncthreads();
    float lacc = 0.0f;
    // each group takes every groups-th projection of the CTA's run; from here
    // to the final sums a group synchronizes only its own threads
    for (int j = j0 + g; j < j1; j += groups) {
        float sn, c;
        sincosf(phi[j], &sn, &c);
        // every address below derives from t and g: recomputing them per
        // projection costs a few integer operations, keeping all of them live
        // across the loop would cost registers
        int tt, gg;
        asm volatile("mov.b32 %0, %1;" : "=r"(tt) : "r"(t));
        asm volatile("mov.b32 %0, %1;" : "=r"(gg) : "r"(g));
        float x[SW_E], y[SW_E];
#pragma unroll
        for (int e = 0; e < SW_E; ++e) {
            const float4 q = pts[e * G + tt];
            // merge 1 starts with the blocks where position bit 1 is set negated
            const float sg = sw_neg<N, 1>(e) ? -1.0f : 1.0f;
            x[e] = sg * sw_key(q.x, q.y, c, sn);
            y[e] = sg * sw_key(q.z, q.w, c, sn);
        }
        // the moves alternate between the group's two buffers, starting from
        // the first in every projection (the barrier after the previous
        // projection's search makes that safe), so every choice is static
        int par = 0;
        sw_merges<N, 1>(x, y, tt, gg, bufs + (size_t)gg * 2 * N, par);
        // ranks 8t .. 8t+7: squared differences; each rank's gradient
        // (linear order) and the sorted keys go to the buffer the last move
        // did not read.  The keys are stored as the binary search visits
        // them (breadth-first, Eytzinger order: the pivot of rank r = (2m +
        // 1) h - 1 at node N / 2h + m, node 1 the root), so the first six
        // levels of every search read at most 32 consecutive words: no bank
        // conflicts there, where the sorted order put every pivot of a level
        // in one bank
        float* sk = reinterpret_cast<float*>(bufs + ((size_t)gg * 2 + par) * N);
        float* sgr = sk + N;
        float d[SW_E];
#pragma unroll
        for (int e = 0; e < SW_E; ++e) {
            d[e] = x[e] - y[e];
            lacc = fmaf(d[e], d[e], lacc);
            d[e] = 2.0f * d[e] / (float)N;
            const int q = tt * SW_E + e + 1;            // rank + 1
            if (q < N) {
                const int tz = __ffs(q) - 1;             // h = 2^tz
                sk[((N / 2) >> tz) + ((q >> tz) >> 1)] = x[e];
            }
        }
        reinterpret_cast<float4*>(sgr)[2 * tt] = make_float4(d[0], d[1], d[2], d[3]);
        reinterpret_cast<float4*>(sgr)[2 * tt + 1] = make_float4(d[4], d[5], d[6], d[7]);
        sw_group_sync<G>(gg);
#pragma unroll 2
        for (int e = 0; e < SW_E; ++e) {
            const int i = tt * SW_E + e;
            const float4 q = pts[e * G + tt];
            const float kx = sw_key(q.x, q.y, c, sn);
            int k = 1;
#pragma unroll
            for (int h = N / 2; h >= 1; h >>= 1) k = 2 * k + (sk[k] < kx ? 1 : 0);
            const float gv = sgr[k - N];
            float2 a = gacc[(size_t)gg * N + sw_swz(i)];
            a.x = fmaf(gv, c, a.x);
            a.y = fmaf(gv, sn, a.y);
            gacc[(size_t)gg * N + sw_swz(i)] = a;
        }
        sw_group_sync<G>(gg);
    }
    float v = lacc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        float ax = 0.0f, ay = 0.0f;
        for (int q = 0; q < groups; ++q) {
            const float2 a = gacc[(size_t)q * N + sw_swz(i)];
            ax += a.x;
            ay += a.y;
        }
        atomicAdd(dX + ((size_t)s * N + i) * 2, ax * scale);
        atomicAdd(dX + ((size_t)s * N + i) * 2 + 1, ay * scale);
    }
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        atomicAdd(loss, tot * scale / (float)N);
    }
}

// dynamic shared memory of sw_kernel<N> with `groups` groups
size_t sw_smem_bytes(int N, int groups)
{
    return sizeof(float4) * N + sizeof(float2) * 3 * (size_t)N * groups;
}

template <int N>
const void* sw_func()
{
    return reinterpret_cast<const void*>(&sw_kernel<N>);
}

const void* sw_kernel_of(int N)
{
    switch (N) {
    case 32: return sw_func<32>();
    case 64: return sw_func<64>();
    case 128: return sw_func<128>();
    case 256: return sw_func<256>();
    case 512: return sw_func<512>();
    default: return sw_func<1024>();
    }
}

// per device: the shared-memory opt-in of every sw_kernel instance and how
// many full-size CTAs of each fit on an SM (set outside stream capture)
struct SwDevInfo {
    bool ready = false;
    int sms = 0;
    int ctas[6] = {0, 0, 0, 0, 0, 0};
};
SwDevInfo g_sw_info[64];

int sw_log2(int N)
{
    int l = 0;
    while ((1 << l) < N) ++l;
    return l;
}

cfs_status sw_init()
{
    int dev = 0;
    cfs_status st = cfs::check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != CFS_OK) return st;
    if (dev < 0 || dev >= 64) return cfs::fail(CFS_ERR_UNSUPPORTED, "device index out of range");
    SwDevInfo& d = g_sw_info[dev];
    if (d.ready) return CFS_OK;
    st = cfs::check_cuda(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev), "SMs");
    for (int N = 32; N <= 1024 && st == CFS_OK; N *= 2) {
        const int groups = SW_THREADS / (N / SW_E);
        const size_t bytes = sw_smem_bytes(N, groups);
        const void* f = sw_kernel_of(N);
        st = cfs::check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes),
                        "cudaFuncSetAttribute(sw_kernel)");
        int n = 0;
        if (st == CFS_OK)
            st = cfs::check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, SW_THREADS,
                                                                          bytes),
                            "occupancy(sw_kernel)");
        d.ctas[sw_log2(N) - 5] = std::max(1, n);
    }
    if (st == CFS_OK) d.ready = true;
    return st;
}

// launches the SW kernel for N points per system (a power of two, 32..1024);
// sw_init() must have run on this device
void sw_launch(const float* X, const float* T, const float* phi, int P, int N, int n_sys,
               float scale, float* loss, float* dX, cudaStream_t st)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const SwDevInfo& d = g_sw_info[dev >= 0 && dev < 64 ? dev : 0];
    const int G = N / SW_E;
    // groups per CTA: enough for the projections, whole warps
    int groups = std::min(SW_THREADS / G, P);
    const int per_warp = std::max(1, 32 / G);
    groups = std::min(SW_THREADS / G, (groups + per_warp - 1) / per_warp * per_warp);
    // sorts per group: shortest makespan over the resident CTAs, a CTA
    // costing its sorts plus about 0.3 of a sort for staging the points and
    // adding its gradient sums to dX
    const long slots = (long)std::max(1, d.sms) * std::max(1, d.ctas[sw_log2(N) - 5]);
    int best_pg = 1;
    double best = -1.0;
    for (int pg = 1; pg <= 16; ++pg) {
        const long ctas = (long)n_sys * ((P + groups * pg - 1) / (groups * pg));
        const double span = (double)((ctas + slots - 1) / slots) * (pg + 0.3);
        if (best < 0.0 || span < best) { best = span; best_pg = pg; }
        if (groups * pg >= P) break;
    }
    const int pc = groups * best_pg;
    const unsigned grid = (unsigned)n_sys * (unsigned)((P + pc - 1) / pc);
    const unsigned threads = (unsigned)(groups * G);
    const size_t bytes = sw_smem_bytes(N, groups);
    switch (N) {
    case 32: sw_kernel<32><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    case 64: sw_kernel<64><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    case 128: sw_kernel<128><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    case 256: sw_kernel<256><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    case 512: sw_kernel<512><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    default: sw_kernel<1024><<<grid, threads, bytes, st>>>(X, T, phi, P, pc, scale, loss, dX); break;
    }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) with bias correction on the FP32 master weights; writes
// the BF16 copies the GEMMs read.  t (1-based) is *step + 1.
// ---------------------------------------------------------------------------
// BF16 copy of parameter i; W2 and W3 also go transposed into wbT
// ([2][in][out]): the K-major operands of the backward GEMMs
__device__ __forceinline__ void store_bf16_weight(bf16r* wb, bf16r* wbT, int i, float wi)
{
    const bf16r b = to_bf16(wi);
    wb[i] = b;
    if (i >= OFF_W2 && i < OFF_W2 + HID * HID) {
        const int e = i - OFF_W2;
        wbT[(e % HID) * HID + e / HID] = b;
    } else if (i >= OFF_W3 && i < OFF_W3 + HID * HID) {
        const int e = i - OFF_W3;
        wbT[HID * HID + (e % HID) * HID + e / HID] = b;
    }
}

// Step size of a training run of `total` steps that started at step `first`:
// cosine decay from lr to lr_final (Loshchilov & Hutter's schedule without
// restarts); lr_final == lr keeps it constant.
__device__ __forceinline__ float lr_at(u32 step, u32 first, u32 total, float lr, float lr_final)
{
    if (lr_final == lr || total < 2) return lr;
    const float x = fminf(1.0f, (float)(step - first) / (float)(total - 1));
    return lr_final + 0.5f * (lr - lr_final) * (1.0f + cosf(3.14159265358979f * x));
}

__global__ void __launch_bounds__(256) adam_kernel(float* w, float* m, float* v,
                                                   const float* g, bf16r* wb, bf16r* wbT, int n,
                                                   const u32* step, u32 t_explicit, float lr0,
                                                   float lr_final, u32 first, u32 total,
                                                   float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32 t = step ? (*step + 1u) : t_explicit;
    const float lr = step ? lr_at(*step, first, total, lr0, lr_final) : lr0;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    store_bf16_weight(wb, wbT, i, wi);
}

__global__ void to_bf16_kernel(const float* w, bf16r* wb, bf16r* wbT, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) store_bf16_weight(wb, wbT, i, w[i]);
}

// ---------------------------------------------------------------------------
// training data, inputs, per-step randomness
// ---------------------------------------------------------------------------
// one system of the training family: threshold table + maps (chaos game)
// and the conditioning vector of the network
struct SysRec {
    u32 T[16];
    int n_cmp, n_maps, pad0, pad1;
    float prm[MAX_SYS_MAPS][6];
    float cond[COND];
    float t;
    float pad[3];
};

__device__ __forceinline__ uint4 philox_key(u64 seed, u32 c0, u32 c1, u32 c2, u32 c3)
{
    unsigned int rk[10][2];
    u32 k0 = (u32)seed, k1 = (u32)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0; rk[r][1] = k1;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return cfs_philox_rk(rk, c0, c1, c2, c3);
}

constexpr u32 TAG_NOISE = 3, TAG_PROJ = 4, TAG_DATA = 8, TAG_DATA_INIT = 9, TAG_PICK = 10;

// per step: pick the systems of the batch and the projection angles
__global__ void prep_kernel(const u32* step, u64 seed, int n_sys, int S, u32* sel, float* phi,
                            int P)
{
    const int j = threadIdx.x;
    const u32 st = *step;
    if (j < S) sel[j] = philox_key(seed, (u32)j, st, 0u, TAG_PICK).x % (u32)n_sys;
    const float u = (float)(philox_key(seed, 0u, st, 0u, TAG_PROJ).x >> 8) * CFS_INV_2_24;
    if (j < P) phi[j] = ((float)j + u) * (6.28318530717958647692f / (float)P);
}

// network inputs of row r: Gaussian noise (Box-Muller on a Philox block),
// the conditioning vector of its system and t, written as eight 16-byte
// vectors
__device__ __forceinline__ void write_inputs_row(const SysRec& q, int r, u32 st, u64 seed,
                                                 bf16r* U)
{
    const uint4 w = philox_key(seed, (u32)r, st, 0u, TAG_NOISE);
    const float u1 = ((float)(w.x >> 8) + 0.5f) * CFS_INV_2_24;
    const float u2 = (float)(w.y >> 8) * CFS_INV_2_24;
    const float rad = sqrtf(-2.0f * logf(u1));
    float sn, c;
    sincosf(6.28318530717958647692f * u2, &sn, &c);
    u32 w32[D_IN / 2];
    w32[0] = (u32)to_bf16(rad * c) | ((u32)to_bf16(rad * sn) << 16);
#pragma unroll
    for (int j = 0; j < COND / 2; ++j)
        w32[1 + j] = (u32)to_bf16(q.cond[2 * j]) | ((u32)to_bf16(q.cond[2 * j + 1]) << 16);
    w32[1 + COND / 2] = (u32)to_bf16(q.t);
#pragma unroll
    for (int j = 2 + COND / 2; j < D_IN / 2; ++j) w32[j] = 0u;
    uint4* row = reinterpret_cast<uint4*>(U + (size_t)r * D_IN);
#pragma unroll
    for (int v = 0; v < D_IN / 8; ++v)
        row[v] = make_uint4(w32[4 * v], w32[4 * v + 1], w32[4 * v + 2], w32[4 * v + 3]);
}

// the records of the systems that rows r0 .. r0 + blockDim.x - 1 belong to
// (row r: system sel[r / N]; at most 8 with N >= 32) into shared memory
__device__ __forceinline__ int stage_systems(const SysRec* __restrict__ sys,
                                            const u32* __restrict__ sel, int N, int rows,
                                            SysRec* s_sys)
{
    const int r0 = blockIdx.x * blockDim.x;
    const int first = r0 / N;
    const int last = min(r0 + (int)blockDim.x - 1, rows - 1) / N;
    constexpr int W = (int)(sizeof(SysRec) / 4);
    for (int e = threadIdx.x; e < (last - first + 1) * W; e += blockDim.x) {
        const int q = e / W, w = e % W;
        reinterpret_cast<u32*>(&s_sys[q])[w] =
            reinterpret_cast<const u32*>(&sys[sel ? sel[first + q] : 0])[w];
    }
    __syncthreads();
    return first;
}

// training rows of one step: row r = s * N + j gets the chaos-game point of
// its system after `steps` steps from a uniform start (the target) and, when
// U is given, its network inputs
__global__ void __launch_bounds__(256) data_kernel(const SysRec* __restrict__ sys,
                                                   const u32* __restrict__ sel, const u32* step,
                                                   u64 seed, int N, int rows, int steps,
                                                   float* out, bf16r* U)
{
    __shared__ SysRec s_sys[256 / 32];
    const int first = stage_systems(sys, sel, N, rows, s_sys);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const SysRec& q = s_sys[r / N - first];
    const u32 st = *step;
    if (U) write_inputs_row(q, r, st, seed, U);
    const uint4 s0 = philox_key(seed, (u32)r, st, 0u, TAG_DATA_INIT);
    float x = (float)(s0.x >> 8) * CFS_INV_2_24, y = (float)(s0.y >> 8) * CFS_INV_2_24;
    for (int n = 0; n < steps; n += 4) {
        const uint4 w = philox_key(seed, (u32)r, st, (u32)(n >> 2), TAG_DATA);
        const u32 ws[4] = {w.x, w.y, w.z, w.w};
        for (int h = 0; h < 4 && n + h < steps; ++h) {
            int k = 0;
            for (int j = 0; j < q.n_cmp; ++j) k += ws[h] >= q.T[j] ? 1 : 0;
            const float* m = q.prm[k];
            const float nx = fmaf(m[0], x, fmaf(m[1], y, m[4]));
            const float ny = fmaf(m[2], x, fmaf(m[3], y, m[5]));
            x = nx;
            y = ny;
        }
    }
    out[2 * r] = x;
    out[2 * r + 1] = y;
}

__global__ void step_inc_kernel(u32* step) { *step += 1u; }

// loss of the current step into the run's history (index: step - first)
__global__ void gather_loss_kernel(const float* loss, const u32* step, u32 first, float* hist,
                                   u32 cap)
{
    const u32 s = *step - first;
    if (s < cap) hist[s] = *loss;
}


// ---------------------------------------------------------------------------
// fused inference on the tensor cores: start points of many frames straight
// from noise, 128 rows (points) per tile.
// Layer 1 is a rank-2 update: only the noise varies from row to row, so
// z1 = c1 + W1[:, 0] n0 + W1[:, 1] n1 with c1 = W1[:, 2:51] u_cond + b1 (one
// vector per frame, cond_kernel); each thread computes its row's 128
// activations and writes them, BF16, as the A operand of layer 2 in shared
// memory (no-swizzle K-major core matrices: 8-column K groups 2048 B apart,
// 8-row groups 128 B apart).  Layers 2 and 3 (128 x 128) and the output
// layer (padded to N = 16) are one tcgen05.mma chain each (M = 128, K = 16
// per instruction) into the group's 128 TMEM columns; the epilogue reads
// each thread's row back (tcgen05.ld, TMEM lane = row), adds the bias,
// applies SiLU and writes the next layer's A tile in place.
// A CTA holds the weights once and runs IT_GROUPS independent warpgroups,
// each on its own tiles with its own A tile, TMEM columns and mbarrier, so
// one group's MMAs overlap the other groups' SiLU epilogues.  Every wait is
// bounded (a time-out sets the device error flag and the group stops).
// ---------------------------------------------------------------------------
// SiLU for inference: z sigma(z) = z (1 + tanh(z / 2)) / 2 with the hardware
// tanh (one special-function operation instead of an exponential and a
// reciprocal; relative error about 2^-11, below the BF16 rounding of the
// activation that follows)
__device__ __forceinline__ float silu_fast(float z)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    const float h = 0.5f * z;
    return fmaf(h, t, h);
}

// c1 = W1[:, 2:51] u_cond + b1 with the BF16-rounded operands (one block
// per frame)
__global__ void cond_kernel(const bf16r* __restrict__ wb, const float* __restrict__ w,
                            const SysRec* __restrict__ recs, float* c1_all)
{
    const int j = threadIdx.x;
    if (j >= HID) return;
    const SysRec* rec = recs + blockIdx.x;
    float* c1 = c1_all + (size_t)blockIdx.x * HID;
    float acc = w[OFF_B1 + j];
    for (int q = 0; q < COND; ++q)
        acc = fmaf(from_bf16(wb[OFF_W1 + j * D_IN + 2 + q]), from_bf16(to_bf16(rec->cond[q])), acc);
    acc = fmaf(from_bf16(wb[OFF_W1 + j * D_IN + 2 + COND]), from_bf16(to_bf16(rec->t)), acc);
    c1[j] = acc;
}

constexpr int IT_GROUPS = 4;
constexpr int IT_THREADS = 128 * IT_GROUPS;
constexpr int IT_W = HID * HID * 2;            // W2 or W3 in shared memory (bytes)
constexpr int IT_N4 = 16;                      // output layer rows, padded
constexpr int IT_W4 = IT_N4 * HID * 2;
constexpr int IT_A = 128 * HID * 2;            // one group's activation tile
constexpr int IT_SMEM = 1024 + 2 * IT_W + IT_W4 + IT_GROUPS * IT_A + 256;

// byte offset of element (row r, column k) of a K-major tile whose 8-row
// groups are 128 B apart and whose 8-column K groups are `kstride` apart
__device__ __forceinline__ u32 it_off(int r, int k, u32 kstride)
{
    return (u32)(k >> 3) * kstride + (u32)r * 16u + (u32)(k & 7) * 2u;
}

// two floats to packed BF16 (round to nearest even), lo in the low half
__device__ __forceinline__ u32 it_bf16x2(float lo, float hi)
{
    u32 r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void it_st16(u32 addr, u32 a, u32 b, u32 c, u32 d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ void it_fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void it_group_sync(int g)
{
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}

// group barrier that also ANDs a flag over the group's 128 threads: every
// thread leaves with the same answer, so a time-out seen by one thread
// stops the whole group together
__device__ __forceinline__ bool it_group_all(int g, bool v)
{
    u32 r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((u32)v), "r"(g + 1)
        : "memory");
    return r != 0;
}

// frames of one inference launch: tile_begin[f] = first 128-row tile of
// frame f (tile_begin[n_sys] = all tiles), its c1 vector, row count, seed
// and output (SoA [2][count])
struct InferFrames {
    const float* c1;          // [n_sys][HID]
    const u32* tile_begin;    // [n_sys + 1]
    const u32* count;         // [n_sys]
    const u64* seed;          // [n_sys]
    float* const* out;        // [n_sys]
    int n_sys;
};

__global__ void __launch_bounds__(IT_THREADS, 1) infer_tc_kernel(const bf16r* __restrict__ wb,
                                                                 const float* __restrict__ w,
                                                                 const InferFrames fs)
{
    extern __shared__ unsigned char it_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(it_raw) + 1023) & ~(uintptr_t)1023);
    const u32 sW2 = smem_addr(sm), sW3 = sW2 + IT_W, sW4 = sW3 + IT_W;
    const u32 sA0 = sW4 + IT_W4;
    u64* bars = reinterpret_cast<u64*>(sm + 2 * IT_W + IT_W4 + IT_GROUPS * IT_A);
    u32* s_tmem = reinterpret_cast<u32*>(bars + IT_GROUPS);
    __shared__ __align__(16) float s_w10[HID], s_w11[HID], s_b2[HID], s_b3[HID], s_b4[4];
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights into the B-operand layout (rows = output features n, K = inputs)
    for (int e = tid; e < HID * HID; e += IT_THREADS) {
        const int n = e / HID, k = e % HID;
        const u32 o = it_off(n, k, 2048u);
        *reinterpret_cast<bf16r*>(sm + o) = wb[OFF_W2 + e];
        *reinterpret_cast<bf16r*>(sm + IT_W + o) = wb[OFF_W3 + e];
    }
    for (int e = tid; e < IT_N4 * HID; e += IT_THREADS) {
        const int n = e / HID, k = e % HID;
        *reinterpret_cast<bf16r*>(sm + 2 * IT_W + it_off(n, k, (u32)IT_N4 * 16u)) =
            n < D_OUT ? wb[OFF_W4 + e] : (bf16r)0;
    }
    for (int j = tid; j < HID; j += IT_THREADS) {
        s_w10[j] = from_bf16(wb[OFF_W1 + j * D_IN]);
        s_w11[j] = from_bf16(wb[OFF_W1 + j * D_IN + 1]);
        s_b2[j] = w[OFF_B2 + j];
        s_b3[j] = w[OFF_B3 + j];
    }
    if (tid < 2) s_b4[tid] = w[OFF_B4 + tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(s_tmem)), "r"(128u * IT_GROUPS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_err = 0;
        for (int g = 0; g < IT_GROUPS; ++g) mbar_init(smem_addr(&bars[g]), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    it_fence_async_smem();          // the weights, written by st.shared, feed the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int g = warp >> 2, wq = warp & 3, r = wq * 32 + lane;   // r: row in the tile
    const u32 sA = sA0 + (u32)(g * IT_A);
    const u32 bar = smem_addr(&bars[g]);
    const u32 tcol = *s_tmem + (u32)(g * 128);                    // the group's columns
    const u32 tlane = tcol + ((u32)(wq * 32) << 16);              // this warp's lanes
    const bool issuer = wq == 0 && lane == 0;
    const u32 idesc128 = tc_idesc(128), idesc16 = tc_idesc(IT_N4);
    u32 phase = 0;
    int pending = 0;               // commits issued and not yet waited for (issuer)
    bool ok = true;

    // layer k's MMAs on the A tile into the group's columns, committed to bar
    auto mma_layer = [&](u32 sW, u32 lbo_w, u32 idesc) {
        it_fence_async_smem();
        tc_fence_before();
        it_group_sync(g);
        if (issuer) {
            tc_fence_after();
            for (int kk = 0; kk < HID / 16; ++kk)
                tc_mma(tcol, tc_desc_kn(sA + (u32)kk * 4096u, 2048u, 128u),
                       tc_desc_kn(sW + (u32)kk * 2u * lbo_w, lbo_w, 128u), idesc,
                       kk > 0 ? 1u : 0u);
            tc_commit(bar);
            pending = 1;
        }
    };
    auto wait_layer = [&]() -> bool {
        const bool done = it_group_all(g, mbar_wait(bar, phase));
        if (done) {
            phase ^= 1u;
            if (issuer) pending = 0;
        }
        tc_fence_after();
        return done;
    };
    // epilogue of a hidden layer: bias, SiLU, BF16, written as the next A tile
    auto hidden_epilogue = [&](const float* bias) {
        const float4* b4 = reinterpret_cast<const float4*>(bias);
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 16) {
            float v[16];
            tc_ld16(tlane + (u32)c0, v);
            u32 q[8];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 bb = b4[c0 / 4 + j];
                q[2 * j] = it_bf16x2(silu_fast(v[4 * j] + bb.x), silu_fast(v[4 * j + 1] + bb.y));
                q[2 * j + 1] = it_bf16x2(silu_fast(v[4 * j + 2] + bb.z),
                                         silu_fast(v[4 * j + 3] + bb.w));
            }
            it_st16(sA + it_off(r, c0, 2048u), q[0], q[1], q[2], q[3]);
            it_st16(sA + it_off(r, c0 + 8, 2048u), q[4], q[5], q[6], q[7]);
        }
    };

    const u32 tiles = fs.tile_begin[fs.n_sys];
    for (u32 tile = blockIdx.x * IT_GROUPS + (u32)g; tile < tiles;
         tile += gridDim.x * IT_GROUPS) {
        // the frame of this tile: last f with tile_begin[f] <= tile
        int lo = 0, hi = fs.n_sys;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (fs.tile_begin[mid] <= tile) lo = mid; else hi = mid;
        }
        const int f = lo;
        const u32 row = (tile - fs.tile_begin[f]) * 128u + (u32)r;
        const u32 n = fs.count[f];
        const float* c1 = fs.c1 + (size_t)f * HID;
        // noise of this row (Box-Muller on Philox (row, 0, 0, 3))
        float n0, n1;
        {
            const uint4 q = philox_key(fs.seed[f], row, 0u, 0u, TAG_NOISE);
            const float u1 = ((float)(q.x >> 8) + 0.5f) * CFS_INV_2_24;
            const float u2 = (float)(q.y >> 8) * CFS_INV_2_24;
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincosf(6.28318530717958647692f * u2, &sn, &cs);
            n0 = from_bf16(to_bf16(rad * cs));
            n1 = from_bf16(to_bf16(rad * sn));
        }
        // layer 1 (rank-2 update) into the A tile (16-byte loads of c1 and
        // of the two noise columns of W1, shared by the whole group)
        const float4* c14 = reinterpret_cast<const float4*>(c1);
        const float4* w04 = reinterpret_cast<const float4*>(s_w10);
        const float4* w14 = reinterpret_cast<const float4*>(s_w11);
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 8) {
            u32 q[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 cc = __ldg(c14 + c0 / 4 + h);
                const float4 a0 = w04[c0 / 4 + h], a1 = w14[c0 / 4 + h];
                q[2 * h] = it_bf16x2(silu_fast(fmaf(a1.x, n1, fmaf(a0.x, n0, cc.x))),
                                     silu_fast(fmaf(a1.y, n1, fmaf(a0.y, n0, cc.y))));
                q[2 * h + 1] = it_bf16x2(silu_fast(fmaf(a1.z, n1, fmaf(a0.z, n0, cc.z))),
                                         silu_fast(fmaf(a1.w, n1, fmaf(a0.w, n0, cc.w))));
            }
            it_st16(sA + it_off(r, c0, 2048u), q[0], q[1], q[2], q[3]);
        }
        mma_layer(sW2, 2048u, idesc128);
        if (!(ok = wait_layer())) break;
        hidden_epilogue(s_b2);
        mma_layer(sW3, 2048u, idesc128);
        if (!(ok = wait_layer())) break;
        hidden_epilogue(s_b3);
        mma_layer(sW4, (u32)IT_N4 * 16u, idesc16);
        if (!(ok = wait_layer())) break;
        float y[16];
        tc_ld16(tlane, y);
        tc_fence_before();          // TMEM read: the next tile's MMAs may overwrite it
        if (row < n) {
            float* out = fs.out[f];
            out[row] = y[0] + s_b4[0];
            out[(size_t)n + row] = y[1] + s_b4[1];
        }
    }
    if (!ok) {
        atomicExch(&s_err, 1);
        // the MMAs of an unfinished commit complete before TMEM is freed
        if (issuer && pending) mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(&g_tc_error, (unsigned)CFS_DEVICE_ERR_TC_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tmem),
                     "r"(128u * IT_GROUPS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// The training forward pass fused per 128-row tile (the same structure as
// infer_tc_kernel): the tile of inputs U goes from global memory into the
// group's A tile; layer 1 (K = 64), layer 2 and layer 3 run as tcgen05.mma
// chains into the group's TMEM columns, each epilogue adding the bias,
// applying SiLU and writing the next A tile in place.  What the backward
// pass reads is written on the way: H1 (row-major: the input of the
// recomputed Z2) and its transpose, H2's transpose, H3 and Z3 (the output
// layer's backward); the output layer itself (N = 2) runs on the CUDA cores
// in the layer-3 epilogue.  H2 in row-major form, which only the next
// layer's GEMM read, never leaves the chip.
// ---------------------------------------------------------------------------
constexpr int TF_GROUPS = 4;
constexpr int TF_THREADS = 128 * TF_GROUPS;
constexpr int TF_W1 = HID * D_IN * 2;          // 16 KB
constexpr int TF_SMEM = 1024 + TF_W1 + 2 * IT_W + TF_GROUPS * IT_A + 256;

struct TrainFwdArgs {
    const bf16r* U;                // [B][D_IN]
    int B;
    bf16r *H1, *H1T, *H2T, *H3;    // H1, H3 [B][HID]; transposes [HID][ldt]
    int ldt;
    float *Z3, *Y;                 // Z3 [B][HID], Y [B][2]
};

__global__ void __launch_bounds__(TF_THREADS, 1) train_fwd_kernel(const bf16r* __restrict__ wb,
                                                                  const float* __restrict__ w,
                                                                  const TrainFwdArgs g)
{
    extern __shared__ unsigned char tf_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tf_raw) + 1023) & ~(uintptr_t)1023);
    const u32 sW1 = smem_addr(sm), sW2 = sW1 + TF_W1, sW3 = sW2 + IT_W;
    const u32 sA0 = sW3 + IT_W;
    u64* bars = reinterpret_cast<u64*>(sm + TF_W1 + 2 * IT_W + TF_GROUPS * IT_A);
    u32* s_tmem = reinterpret_cast<u32*>(bars + TF_GROUPS);
    __shared__ __align__(16) float s_b1[HID], s_b2[HID], s_b3[HID], s_w4[D_OUT][HID];
    __shared__ float s_b4[2];
    __shared__ int s_err;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights into the B-operand layout (rows = output features, K = inputs)
    for (int e = tid; e < HID * D_IN; e += TF_THREADS) {
        const int n = e / D_IN, k = e % D_IN;
        *reinterpret_cast<bf16r*>(sm + it_off(n, k, 2048u)) = wb[OFF_W1 + e];
    }
    for (int e = tid; e < HID * HID; e += TF_THREADS) {
        const int n = e / HID, k = e % HID;
        const u32 o = it_off(n, k, 2048u);
        *reinterpret_cast<bf16r*>(sm + TF_W1 + o) = wb[OFF_W2 + e];
        *reinterpret_cast<bf16r*>(sm + TF_W1 + IT_W + o) = wb[OFF_W3 + e];
    }
    for (int j = tid; j < HID; j += TF_THREADS) {
        s_b1[j] = w[OFF_B1 + j];
        s_b2[j] = w[OFF_B2 + j];
        s_b3[j] = w[OFF_B3 + j];
        s_w4[0][j] = from_bf16(wb[OFF_W4 + j]);
        s_w4[1][j] = from_bf16(wb[OFF_W4 + HID + j]);
    }
    if (tid < 2) s_b4[tid] = w[OFF_B4 + tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_addr(s_tmem)), "r"(128u * TF_GROUPS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        s_err = 0;
        for (int q = 0; q < TF_GROUPS; ++q) mbar_init(smem_addr(&bars[q]), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    it_fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int gi = warp >> 2, wq = warp & 3, r = wq * 32 + lane;
    const u32 sA = sA0 + (u32)(gi * IT_A);
    const u32 bar = smem_addr(&bars[gi]);
    const u32 tcol = *s_tmem + (u32)(gi * 128);
    const u32 tlane = tcol + ((u32)(wq * 32) << 16);
    const bool issuer = wq == 0 && lane == 0;
    const u32 idesc = tc_idesc(128);
    u32 phase = 0;
    int pending = 0;
    bool ok = true;

    auto mma_layer = [&](u32 sW, int K) {
        it_fence_async_smem();
        tc_fence_before();
        it_group_sync(gi);
        if (issuer) {
            tc_fence_after();
            for (int kk = 0; kk < K / 16; ++kk)
                tc_mma(tcol, tc_desc_kn(sA + (u32)kk * 4096u, 2048u, 128u),
                       tc_desc_kn(sW + (u32)kk * 4096u, 2048u, 128u), idesc, kk > 0 ? 1u : 0u);
            tc_commit(bar);
            pending = 1;
        }
    };
    auto wait_layer = [&]() -> bool {
        const bool done = it_group_all(gi, mbar_wait(bar, phase));
        if (done) {
            phase ^= 1u;
            if (issuer) pending = 0;
        }
        tc_fence_after();
        return done;
    };
    // epilogue of layers 1 and 2: H = SiLU(acc + b) as BF16 into the next A
    // tile, and into global memory (row-major and / or transposed)
    auto hidden_epilogue = [&](const float* bias, int row, bool in, bf16r* H, bf16r* HT) {
        const float4* b4 = reinterpret_cast<const float4*>(bias);
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 16) {
            float v[16];
            tc_ld16(tlane + (u32)c0, v);
            float h[16];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 bb = b4[c0 / 4 + j];
                h[4 * j] = silu_f(v[4 * j] + bb.x);
                h[4 * j + 1] = silu_f(v[4 * j + 1] + bb.y);
                h[4 * j + 2] = silu_f(v[4 * j + 2] + bb.z);
                h[4 * j + 3] = silu_f(v[4 * j + 3] + bb.w);
            }
            u32 q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) q[j] = pack_bf16x2(h[2 * j], h[2 * j + 1]);
            it_st16(sA + it_off(r, c0, 2048u), q[0], q[1], q[2], q[3]);
            it_st16(sA + it_off(r, c0 + 8, 2048u), q[4], q[5], q[6], q[7]);
            if (in && H) {
                uint4* hp = reinterpret_cast<uint4*>(H + (size_t)row * HID + c0);
                hp[0] = make_uint4(q[0], q[1], q[2], q[3]);
                hp[1] = make_uint4(q[4], q[5], q[6], q[7]);
            }
            if (in && HT) {
                // consecutive lanes hold consecutive rows: each column's stores coalesce
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    HT[(size_t)(c0 + j) * g.ldt + row] = (bf16r)(q[j >> 1] >> (16 * (j & 1)));
            }
        }
    };

    const int n_tiles = (g.B + 127) / 128;
    for (int tile = blockIdx.x * TF_GROUPS + gi; tile < n_tiles; tile += gridDim.x * TF_GROUPS) {
        const int row = tile * 128 + r;
        const bool in = row < g.B;
        // the tile's inputs: row r's 64 BF16 values into K groups 0..7
        {
            const uint4* src = reinterpret_cast<const uint4*>(g.U + (size_t)row * D_IN);
#pragma unroll
            for (int kq = 0; kq < D_IN / 8; ++kq) {
                const uint4 v = in ? __ldg(src + kq) : make_uint4(0u, 0u, 0u, 0u);
                it_st16(sA + it_off(r, 8 * kq, 2048u), v.x, v.y, v.z, v.w);
            }
        }
        mma_layer(sW1, D_IN);
        if (!(ok = wait_layer())) break;
        hidden_epilogue(s_b1, row, in, g.H1, g.H1T);
        mma_layer(sW2, HID);
        if (!(ok = wait_layer())) break;
        hidden_epilogue(s_b2, row, in, nullptr, g.H2T);
        mma_layer(sW3, HID);
        if (!(ok = wait_layer())) break;
        // layer 3: Z3 (FP32) and H3 (BF16) out, then the output layer on
        // the BF16 activations, columns in order
        float y0 = 0.0f, y1 = 0.0f;
#pragma unroll 1
        for (int c0 = 0; c0 < HID; c0 += 16) {
            float v[16];
            tc_ld16(tlane + (u32)c0, v);
            float z[16];
            u32 q[8];
#pragma unroll
            for (int j = 0; j < 16; ++j) z[j] = v[j] + s_b3[c0 + j];
#pragma unroll
            for (int j = 0; j < 8; ++j) q[j] = pack_bf16x2(silu_f(z[2 * j]), silu_f(z[2 * j + 1]));
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float x = __uint_as_float((q[j >> 1] >> (16 * (j & 1))) << 16);
                y0 = fmaf(x, s_w4[0][c0 + j], y0);
                y1 = fmaf(x, s_w4[1][c0 + j], y1);
            }
            if (in) {
                float4* zp = reinterpret_cast<float4*>(g.Z3 + (size_t)row * HID + c0);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    zp[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
                uint4* hp = reinterpret_cast<uint4*>(g.H3 + (size_t)row * HID + c0);
                hp[0] = make_uint4(q[0], q[1], q[2], q[3]);
                hp[1] = make_uint4(q[4], q[5], q[6], q[7]);
            }
        }
        tc_fence_before();          // TMEM read: the next tile's MMAs may overwrite it
        if (in) {
            g.Y[2 * (size_t)row] = y0 + s_b4[0];
            g.Y[2 * (size_t)row + 1] = y1 + s_b4[1];
        }
    }
    if (!ok) {
        atomicExch(&s_err, 1);
        if (issuer && pending) mbar_wait(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_err) atomicOr(&g_tc_error, (unsigned)CFS_DEVICE_ERR_TC_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*s_tmem),
                     "r"(128u * TF_GROUPS)
                     : "memory");
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host object
// ---------------------------------------------------------------------------
struct cfs_sampler {
    int device = 0;
    float* w = nullptr;      // master params [N_PARAMS]
    float* m = nullptr;
    float* v = nullptr;
    bf16r* wb = nullptr;     // bf16 copies
    bf16r* wbT = nullptr;    // bf16 W2^T, W3^T ([2][in][out]) for the backward GEMMs
    float* bias_part = nullptr;   // PART_FLOATS gradient partial sums (part_reduce_kernel)
    u32* d_step = nullptr;   // Adam step counter (device)
    u32 step = 0;            // host mirror (checkpoints)
    // inference workspace for n frames (grown on demand): records, c1,
    // tile offsets, counts, seeds, output pointers
    int cap_frames = 0;
    unsigned char* inf = nullptr;
    unsigned char* inf_host = nullptr;   // pinned staging of the same layout
    cudaEvent_t uploaded = nullptr;      // the staging buffer's last upload
    bool upload_pending = false;
    // activations for B rows (grown on demand)
    int cap_rows = 0;
    int ldt = 0;             // row stride of the transposed copies (>= cap_rows)
    unsigned char* act = nullptr;
    float *Z1, *Z2, *Z3, *Y;
    bf16r *H1, *H2, *H3, *dZ1, *dZ2, *dZ3;
    // transposed copies [features][ldt]: the K-major operands of dW = dZ^T A
    bf16r *UT, *H1T, *H2T, *dZ1T, *dZ2T, *dZ3T;
};

namespace {
using namespace cfs;

cfs_status ensure_rows(cfs_sampler* s, int B)
{
    if (B <= s->cap_rows) return CFS_OK;
    if (s->act) cudaFree(s->act);
    s->act = nullptr;
    s->cap_rows = 0;
    const size_t fz = (size_t)B * HID * 4, fh = (size_t)B * HID * 2;
    const int ldt = (B + 63) / 64 * 64;
    const size_t ft = (size_t)ldt * HID * 2, fu = (size_t)ldt * D_IN * 2;
    const size_t bytes = 3 * fz + (size_t)B * 2 * 4 + 6 * fh + 5 * ft + fu + 13 * 256;
    cfs_status st = check_cuda(cudaMalloc(&s->act, bytes), "cudaMalloc(sampler activations)");
    if (st != CFS_OK) return st;
    unsigned char* p = s->act;
    auto take = [&](size_t n) {
        unsigned char* r = p;
        p += (n + 255) & ~(size_t)255;
        return r;
    };
    s->Z1 = (float*)take(fz); s->Z2 = (float*)take(fz); s->Z3 = (float*)take(fz);
    s->Y = (float*)take((size_t)B * 2 * 4);
    s->H1 = (bf16r*)take(fh); s->H2 = (bf16r*)take(fh); s->H3 = (bf16r*)take(fh);
    s->dZ1 = (bf16r*)take(fh); s->dZ2 = (bf16r*)take(fh); s->dZ3 = (bf16r*)take(fh);
    s->UT = (bf16r*)take(fu);
    s->H1T = (bf16r*)take(ft); s->H2T = (bf16r*)take(ft);
    s->dZ1T = (bf16r*)take(ft); s->dZ2T = (bf16r*)take(ft); s->dZ3T = (bf16r*)take(ft);
    s->ldt = ldt;
    s->cap_rows = B;
    return CFS_OK;
}

// D = A B^T on the tensor cores (both operands K-major), split over K into
// `splits` CTA ranges (ATOMIC adds the partial products)
cfs_status tc_gemm(cudaStream_t st, int M, int N, int K, const bf16r* A, int lda, const bf16r* B,
             int ldb, int mode, const float* bias, float* C, int ldc, bf16r* H, int ldh,
             bf16r* HT, int ldt, const float* Zin, int ldz, float* colsum, int splits = 1)
{
    // the staging reads 16-byte vectors, the epilogue writes them: every
    // operand and output of this library is laid out for that; anything
    // else is a bug here, so stop before a misaligned launch
    const bool aligned =
        ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && lda % 8 == 0 && ldb % 8 == 0 &&
        (!C || ((uintptr_t)C % 16 == 0 && ldc % 4 == 0)) &&
        (!H || ((uintptr_t)H % 16 == 0 && ldh % 8 == 0)) &&
        (!Zin || ((uintptr_t)Zin % 16 == 0 && ldz % 4 == 0)) && (N == 64 || N == 128);
    if (!aligned)
        return fail(CFS_ERR_INVALID_ARG, "tensor-core GEMM operands not 16-byte aligned");
    TcArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda;
    g.B = B; g.ldb = ldb;
    const int per = (K + splits - 1) / splits;
    g.k_split = (per + TC_K - 1) / TC_K * TC_K;
    g.mode = mode; g.bias = bias; g.C = C; g.ldc = ldc; g.H = H; g.ldh = ldh;
    g.HT = HT; g.ldt = ldt; g.Zin = Zin; g.ldz = ldz; g.colsum = colsum;
    dim3 grid((M + TC_M - 1) / TC_M, 1, (K + g.k_split - 1) / g.k_split);
    const int stages = g.k_split / TC_K <= 2 ? 1 : 2;
    if (stages == 1)
        tc_gemm_kernel<1><<<grid, TC_THREADS, tc_smem_bytes<1>(), st>>>(g);
    else
        tc_gemm_kernel<2><<<grid, TC_THREADS, tc_smem_bytes<2>(), st>>>(g);
    return CFS_OK;
}

// row GEMM D[M][128] = A[M][K] W^T (K = 64 or 128) with the SILU or
// SILU_GRAD epilogue on the persistent TMA kernel (tc_gemm_kernel for
// fewer rows than one tile)

// whether row GEMMs of M rows run on tc_rows_kernel: then the backward
// recomputes the pre-activations Z1 and Z2 and the forward need not store them
bool rows_on_tma(int M) { return M >= TC_M; }

// A2, W2 (K2 = 64 or 128), bias2: SILU_GRAD with the pre-activation of the
// layer below recomputed as A2 W2^T + bias2 instead of read from Zin (only
// where rows_on_tma(M); elsewhere Zin is read)
cfs_status tc_rows(cudaStream_t st, int M, int K, const bf16r* A, int lda, const bf16r* W, int ldw,
                   int mode, const float* bias, float* C, int ldc, bf16r* H, int ldh, bf16r* HT,
                   int ldt, const float* Zin, int ldz, float* colsum,
                   const bf16r* A2 = nullptr, int lda2 = 0, const bf16r* W2 = nullptr,
                   int ldw2 = 0, int K2 = 0, const float* bias2 = nullptr)
{
    // fewer rows than one tile: the register-staged kernel (no tensor map with
    // an extent below its box)
    if (!rows_on_tma(M))
        return tc_gemm(st, M, HID, K, A, lda, W, ldw, mode, bias, C, ldc, H, ldh, HT, ldt, Zin,
                       ldz, colsum);
    const bool rc = A2 != nullptr;
    const bool aligned =
        (K == 64 || K == 128) && lda % 8 == 0 && ldw % 8 == 0 &&
        (!C || ((uintptr_t)C % 16 == 0 && ldc % 4 == 0)) &&
        (!H || ((uintptr_t)H % 16 == 0 && ldh % 8 == 0)) &&
        (!Zin || ((uintptr_t)Zin % 16 == 0 && ldz % 4 == 0)) &&
        (!rc || ((K2 == 64 || K2 == 128) && lda2 % 8 == 0 && ldw2 % 8 == 0 && W2 && bias2 &&
                 mode == EPI_SILU_GRAD));
    if (!aligned) return fail(CFS_ERR_INVALID_ARG, "row GEMM operands not aligned");
    CUtensorMap ta, tb, ta2, tb2;
    cfs_status r = make_tmap_2d_bf16(&ta, A, (uint64_t)K, (uint64_t)M, (uint64_t)lda, 8u, 128u);
    if (r == CFS_OK) r = make_tmap_2d_bf16(&tb, W, (uint64_t)K, 128u, (uint64_t)ldw, 8u, 128u);
    if (r == CFS_OK && rc)
        r = make_tmap_2d_bf16(&ta2, A2, (uint64_t)K2, (uint64_t)M, (uint64_t)lda2, 8u, 128u);
    if (r == CFS_OK && rc)
        r = make_tmap_2d_bf16(&tb2, W2, (uint64_t)K2, 128u, (uint64_t)ldw2, 8u, 128u);
    if (r != CFS_OK) return r;
    if (!rc) { ta2 = ta; tb2 = tb; }   // unused
    TcArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = M; g.N = HID; g.K = K;
    g.A = A; g.lda = lda; g.B = W; g.ldb = ldw;
    g.k_split = K;
    g.mode = mode; g.bias = rc ? bias2 : bias; g.C = C; g.ldc = ldc; g.H = H; g.ldh = ldh;
    g.HT = HT; g.ldt = ldt; g.Zin = rc ? nullptr : Zin; g.ldz = ldz; g.colsum = colsum;
    g.K2 = rc ? K2 : 0;
    const int tiles = (M + TC_M - 1) / TC_M;
    const int grid = std::min(tiles, std::max(1, device_sm_count()));
    if (rc)
        tc_rows_kernel<true><<<grid, TR_THREADS, TrCfg<true>::SMEM, st>>>(ta, tb, ta2, tb2, g);
    else
        tc_rows_kernel<false><<<grid, TR_THREADS, TrCfg<false>::SMEM, st>>>(ta, tb, ta2, tb2, g);
    return CFS_OK;
}

// weight gradient C[128][N] += A[128][K] B[N][K]^T on the split-K TMA kernel
// (N = 128 or 64)
cfs_status tc_splitk(cudaStream_t st, int N, int K, const bf16r* A, int lda, const bf16r* Bm,
                     int ldb, float* C, int ldc)
{
    // fewer rows than one chunk: the register-staged kernel (as in tc_rows)
    if (K > 0 && K < TC_K) {
        const int splits = std::max(1, std::min(256, K / 256));
        return tc_gemm(st, HID, N, K, A, lda, Bm, ldb, EPI_ATOMIC, nullptr, C, ldc, nullptr, 0,
                       nullptr, 0, nullptr, 0, nullptr, splits);
    }
    if (K < 1) return CFS_OK;
    if (!(N == 64 || N == 128) || lda % 8 || ldb % 8 || (uintptr_t)C % 16 || ldc % 4)
        return fail(CFS_ERR_INVALID_ARG, "weight-gradient GEMM operands not aligned");
    CUtensorMap ta, tb;
    cfs_status r = make_tmap_2d_bf16(&ta, A, (uint64_t)K, 128u, (uint64_t)lda, 8u, 128u);
    if (r == CFS_OK)
        r = make_tmap_2d_bf16(&tb, Bm, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, 8u, (uint32_t)N);
    if (r != CFS_OK) return r;
    TcArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = HID; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.B = Bm; g.ldb = ldb;
    g.k_split = K;
    g.mode = EPI_ATOMIC; g.C = C; g.ldc = ldc;
    const int chunks = (K + TC_K - 1) / TC_K;
    const int sms = std::max(1, device_sm_count());
    tc_splitk_kernel<<<std::min(chunks, sms), SK_THREADS, SK_SMEM, st>>>(ta, tb, g);
    return CFS_OK;
}

// forward of B rows of U: Z1..Z3 (fp32), H1..H3 (bf16), H1^T, H2^T, Y (fp32 [B][2])
cfs_status forward(cfs_sampler* s, const bf16r* U, int B, cudaStream_t st)
{
    const bf16r* wb = s->wb;
    if (rows_on_tma(B) && (uintptr_t)U % 16 == 0) {
        // the fused pass (one launch): what the backward reads, and Y
        static int smem_dev = -1;
        if (smem_dev != s->device) {
            cfs_status r = check_cuda(cudaFuncSetAttribute(train_fwd_kernel,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           TF_SMEM),
                                      "cudaFuncSetAttribute(train_fwd_kernel)");
            if (r != CFS_OK) return r;
            smem_dev = s->device;
        }
        TrainFwdArgs a;
        a.U = U; a.B = B;
        a.H1 = s->H1; a.H1T = s->H1T; a.H2T = s->H2T; a.H3 = s->H3;
        a.ldt = s->ldt; a.Z3 = s->Z3; a.Y = s->Y;
        const int tiles = (B + 127) / 128;
        const int grid = std::max(1, std::min(device_sm_count(), (tiles + TF_GROUPS - 1) / TF_GROUPS));
        train_fwd_kernel<<<grid, TF_THREADS, TF_SMEM, st>>>(wb, s->w, a);
        return check_cuda(cudaGetLastError(), "train_fwd_kernel launch");
    }
    // Z1 and Z2 only where the backward reads them (it recomputes them on
    // tc_rows_kernel); Z3 always (the output layer's backward reads it)
    const bool keep_z = !rows_on_tma(B);
    cfs_status r = tc_rows(st, B, D_IN, U, D_IN, wb + OFF_W1, D_IN, EPI_SILU, s->w + OFF_B1,
                           keep_z ? s->Z1 : nullptr, HID, s->H1, HID, s->H1T, s->ldt, nullptr, 0,
                           nullptr);
    if (r == CFS_OK)
        r = tc_rows(st, B, HID, s->H1, HID, wb + OFF_W2, HID, EPI_SILU, s->w + OFF_B2,
                    keep_z ? s->Z2 : nullptr, HID, s->H2, HID, s->H2T, s->ldt, nullptr, 0,
                    nullptr);
    if (r == CFS_OK)
        r = tc_rows(st, B, HID, s->H2, HID, wb + OFF_W3, HID, EPI_SILU, s->w + OFF_B3, s->Z3, HID,
                    s->H3, HID, nullptr, 0, nullptr, 0, nullptr);
    if (r != CFS_OK) return r;
    out_forward_kernel<<<(B + 255) / 256, 256, 0, st>>>(s->H3, wb, s->w, B, s->Y);
    return CFS_OK;
}

// backward of sum(dY * Y) after forward(): adds into grads [N_PARAMS]
cfs_status backward(cfs_sampler* s, const bf16r* U, int B, const float* dY, float* grads,
                    cudaStream_t st)
{
    const bf16r* wb = s->wb;
    // gradient sums of the output layer and of the biases gather in copies
    // (bias_part) first: fewer atomics on the same address
    cudaMemsetAsync(s->bias_part, 0, sizeof(float) * PART_FLOATS, st);
    out_backward_kernel<<<(B + OB_ROWS - 1) / OB_ROWS, OB_THREADS, 0, st>>>(
        dY, wb, s->H3, s->Z3, B, s->dZ3, s->dZ3T, s->ldt, s->bias_part + 2 * TC_COPIES * HID);
    // dZ2 = (dZ3 W3) * silu'(Z2): the K-major B operand is W3^T
    // (on tc_rows_kernel the pre-activations Z2 = H1 W2^T + b2 and Z1 = U W1^T
    // + b1 are recomputed, bit for bit, instead of read)
    cfs_status r = tc_rows(st, B, HID, s->dZ3, HID, s->wbT + HID * HID, HID, EPI_SILU_GRAD,
                           nullptr, nullptr, 0, s->dZ2, HID, s->dZ2T, s->ldt, s->Z2, HID,
                           s->bias_part, s->H1, HID, wb + OFF_W2, HID, HID, s->w + OFF_B2);
    if (r == CFS_OK)
        r = tc_rows(st, B, HID, s->dZ2, HID, s->wbT, HID, EPI_SILU_GRAD, nullptr, nullptr, 0,
                    nullptr, 0, s->dZ1T, s->ldt, s->Z1, HID, s->bias_part + TC_COPIES * HID, U,
                    D_IN, wb + OFF_W1, D_IN, D_IN, s->w + OFF_B1);
    if (r != CFS_OK) return r;
    part_reduce_kernel<<<1, 512, 0, st>>>(s->bias_part, grads);
    transpose_in_kernel<<<(B + 31) / 32, 256, 0, st>>>(U, B, s->UT, s->ldt);
    // weight gradients dW = dZ^T A: K = the rows, split over CTAs, atomic
    r = tc_splitk(st, HID, B, s->dZ3T, s->ldt, s->H2T, s->ldt, grads + OFF_W3, HID);
    if (r == CFS_OK)
        r = tc_splitk(st, HID, B, s->dZ2T, s->ldt, s->H1T, s->ldt, grads + OFF_W2, HID);
    if (r == CFS_OK)
        r = tc_splitk(st, D_IN, B, s->dZ1T, s->ldt, s->UT, s->ldt, grads + OFF_W1, D_IN);
    return r;
}

void init_params_host(uint64_t seed, std::vector<float>& p)
{
    // uniform +-1/sqrt(fan_in) from Philox (host), zero biases
    p.assign(N_PARAMS, 0.0f);
    const int offs[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
    const int outs[4] = {HID, HID, HID, D_OUT}, ins[4] = {D_IN, HID, HID, HID};
    for (int l = 0; l < 4; ++l) {
        const float bound = 1.0f / std::sqrt((float)ins[l]);
        for (int e = 0; e < outs[l] * ins[l]; ++e) {
            uint32_t c[4] = {(uint32_t)e, (uint32_t)l, 0u, 6u};
            // Philox on the host for the initial weights (Salmon et al.)
            uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
            uint32_t c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
            for (int r = 0; r < 10; ++r) {
                const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
                const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
                c1 = (uint32_t)p1; c3 = (uint32_t)p0; c0 = n0; c2 = n2;
                k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
            }
            const float u = (float)(c0 >> 8) * (1.0f / 16777216.0f);
            p[offs[l] + e] = (2.0f * u - 1.0f) * bound;
        }
    }
}

cfs_status upload_params(cfs_sampler* s, const float* host)
{
    cfs_status st = check_cuda(cudaMemcpy(s->w, host, sizeof(float) * N_PARAMS,
                                          cudaMemcpyHostToDevice), "cudaMemcpy(params)");
    if (st != CFS_OK) return st;
    to_bf16_kernel<<<(N_PARAMS + 255) / 256, 256>>>(s->w, s->wb, s->wbT, N_PARAMS);
    return check_cuda(cudaDeviceSynchronize(), "sampler params");
}

// The system's record: thresholds and maps in their own order (the chaos
// game that makes training targets), and the conditioning vector with the
// maps in canonical order -- decreasing |det A| = |a d - b c| (in double
// from the FP32 parameters), ties by index -- because the attractor does
// not depend on the order in which the maps are listed.
void pack_system(const cfs_system* sys, float t, SysRec* r)
{
    std::memset(r, 0, sizeof(*r));
    for (int j = 0; j < sys->n_cmp; ++j) r->T[j] = sys->T[j];
    r->n_cmp = sys->n_cmp;
    r->n_maps = sys->n_maps;
    const int n = std::min(sys->n_maps, MAX_SYS_MAPS);
    int order[MAX_SYS_MAPS];
    double adet[MAX_SYS_MAPS];
    for (int k = 0; k < n; ++k) {
        const float* v = sys->maps[k].params;
        order[k] = k;
        adet[k] = std::fabs((double)v[0] * (double)v[3] - (double)v[1] * (double)v[2]);
        for (int j = 0; j < 6; ++j) r->prm[k][j] = v[j];
    }
    std::stable_sort(order, order + n, [&](int a, int b) { return adet[a] > adet[b]; });
    for (int q = 0; q < n; ++q)
        for (int j = 0; j < 6; ++j) r->cond[6 * q + j] = sys->maps[order[q]].params[j];
    r->t = t;
}

}  // namespace

namespace cfs {
cfs_status take_device_flags(unsigned int* flags)
{
    unsigned int v = 0;
    cfs_status st = check_cuda(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(v)), "error flags");
    if (st == CFS_OK && v) {
        const unsigned int zero = 0;
        st = check_cuda(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(zero)), "error flags");
    }
    *flags = v;
    return st;
}

cfs_status raise_device_flags(unsigned int flags)
{
    unsigned int v = 0;
    cfs_status st = check_cuda(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(v)), "error flags");
    v |= flags;
    if (st == CFS_OK)
        st = check_cuda(cudaMemcpyToSymbol(g_tc_error, &v, sizeof(v)), "error flags");
    return st;
}
}  // namespace cfs

namespace {
cfs_status check_sampler_system(const cfs_system* sys)
{
    if (!sys) return fail(CFS_ERR_INVALID_ARG, "NULL system");
    if (sys->dim != 2 || sys->n_maps > MAX_SYS_MAPS)
        return fail(CFS_ERR_UNSUPPORTED, "the sampler conditions on 2D systems of up to 8 maps");
    for (int k = 0; k < sys->n_maps; ++k)
        if (sys->maps[k].kind != CFS_MAP_AFFINE)
            return fail(CFS_ERR_UNSUPPORTED, "the sampler conditions on affine maps");
    return CFS_OK;
}
}  // namespace

extern "C" {

cfs_status cfs_sampler_create(const float* params, uint64_t seed, cfs_sampler** out)
{
    clear_error();
    if (!out) return fail(CFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    cfs_sampler* s = new (std::nothrow) cfs_sampler();
    if (!s) return fail(CFS_ERR_OOM, "host allocation failed");
    cudaGetDevice(&s->device);
    // w | m | v (FP32), then the BF16 copies on 256-byte boundaries: the
    // tensor-core GEMMs read the weights with 16-byte loads
    const size_t off_wb = (sizeof(float) * N_PARAMS * 3 + 255) & ~(size_t)255;
    const size_t off_wbT = off_wb + ((sizeof(bf16r) * N_PARAMS + 255) & ~(size_t)255);
    const size_t off_part = off_wbT + sizeof(bf16r) * 2 * HID * HID;
    cfs_status st = check_cuda(cudaMalloc(&s->w, off_part + sizeof(float) * PART_FLOATS),
                               "cudaMalloc(sampler params)");
    if (st != CFS_OK) { delete s; return st; }
    s->m = s->w + N_PARAMS;
    s->v = s->m + N_PARAMS;
    s->wb = reinterpret_cast<bf16r*>(reinterpret_cast<unsigned char*>(s->w) + off_wb);
    s->wbT = reinterpret_cast<bf16r*>(reinterpret_cast<unsigned char*>(s->w) + off_wbT);
    s->bias_part = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(s->w) + off_part);
    // the tensor-core GEMM stages its chunk pairs in dynamic shared memory
    if (st == CFS_OK)
        st = check_cuda(cudaFuncSetAttribute(tc_gemm_kernel<1>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc_smem_bytes<1>()),
                        "cudaFuncSetAttribute(tc_gemm_kernel)");
    if (st == CFS_OK)
        st = check_cuda(cudaFuncSetAttribute(tc_gemm_kernel<2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc_smem_bytes<2>()),
                        "cudaFuncSetAttribute(tc_gemm_kernel)");
    if (st == CFS_OK)
        st = check_cuda(cudaFuncSetAttribute(tc_rows_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TrCfg<false>::SMEM),
                        "cudaFuncSetAttribute(tc_rows_kernel)");
    if (st == CFS_OK)
        st = check_cuda(cudaFuncSetAttribute(tc_rows_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             TrCfg<true>::SMEM),
                        "cudaFuncSetAttribute(tc_rows_kernel)");
    if (st == CFS_OK)
        st = check_cuda(cudaFuncSetAttribute(tc_splitk_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, SK_SMEM),
                        "cudaFuncSetAttribute(tc_splitk_kernel)");
    if (st == CFS_OK) st = sw_init();
    if (st == CFS_OK) st = check_cuda(cudaMalloc(&s->d_step, 256), "cudaMalloc(step)");
    if (st == CFS_OK) st = check_cuda(cudaMemset(s->m, 0, sizeof(float) * N_PARAMS * 2), "memset");
    if (st == CFS_OK) st = check_cuda(cudaMemset(s->d_step, 0, 256), "memset");
    std::vector<float> init;
    if (!params) { init_params_host(seed, init); params = init.data(); }
    if (st == CFS_OK) st = upload_params(s, params);
    if (st != CFS_OK) { cfs_sampler_destroy(s); return st; }
    *out = s;
    return CFS_OK;
}

cfs_status cfs_sampler_destroy(cfs_sampler* s)
{
    if (!s) return CFS_OK;
    cudaDeviceSynchronize();
    if (s->act) cudaFree(s->act);
    if (s->inf) cudaFree(s->inf);
    if (s->inf_host) cudaFreeHost(s->inf_host);
    if (s->uploaded) cudaEventDestroy(s->uploaded);
    if (s->w) cudaFree(s->w);
    if (s->d_step) cudaFree(s->d_step);
    delete s;
    return CFS_OK;
}

uint32_t cfs_sampler_param_count(void) { return N_PARAMS; }

cfs_status cfs_sampler_get_params(const cfs_sampler* s, float* params, float* adam_m,
                                  float* adam_v, uint32_t* step)
{
    clear_error();
    if (!s) return fail(CFS_ERR_INVALID_ARG, "NULL sampler");
    cfs_status st = check_cuda(cudaDeviceSynchronize(), "sampler sync");
    const float* src[3] = {s->w, s->m, s->v};
    float* dst[3] = {params, adam_m, adam_v};
    for (int j = 0; j < 3 && st == CFS_OK; ++j)
        if (dst[j])
            st = check_cuda(cudaMemcpy(dst[j], src[j], sizeof(float) * N_PARAMS,
                                       cudaMemcpyDeviceToHost), "cudaMemcpy(params)");
    if (st == CFS_OK && step)
        st = check_cuda(cudaMemcpy(step, s->d_step, 4, cudaMemcpyDeviceToHost), "step");
    // a tensor-core GEMM whose barrier wait ran out of time skipped its
    // output: report it once
    unsigned int flags = 0;
    if (st == CFS_OK) st = take_device_flags(&flags);
    if (st == CFS_OK && (flags & CFS_DEVICE_ERR_TC_TIMEOUT))
        return fail(CFS_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting for its mbarrier");
    return st;
}

cfs_status cfs_sampler_set_params(cfs_sampler* s, const float* params, const float* adam_m,
                                  const float* adam_v, uint32_t step)
{
    clear_error();
    if (!s || !params) return fail(CFS_ERR_INVALID_ARG, "NULL sampler or params");
    cfs_status st = check_cuda(cudaDeviceSynchronize(), "sampler sync");
    if (st == CFS_OK) st = upload_params(s, params);
    if (st == CFS_OK && adam_m)
        st = check_cuda(cudaMemcpy(s->m, adam_m, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice), "m");
    if (st == CFS_OK && adam_v)
        st = check_cuda(cudaMemcpy(s->v, adam_v, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice), "v");
    if (st == CFS_OK)
        st = check_cuda(cudaMemcpy(s->d_step, &step, 4, cudaMemcpyHostToDevice), "step");
    return st;
}

cfs_status cfs_sampler_forward(cfs_sampler* s, const void* U, uint32_t B, float* Y, void* stream)
{
    clear_error();
    if (!s || !U || !Y) return fail(CFS_ERR_INVALID_ARG, "NULL argument");
    if (B == 0) return CFS_OK;
    if (B > (1u << 24)) return fail(CFS_ERR_INVALID_ARG, "B too large");
    cfs_status st = ensure_rows(s, (int)B);
    if (st != CFS_OK) return st;
    cudaStream_t sm = (cudaStream_t)stream;
    st = forward(s, (const bf16r*)U, (int)B, sm);
    if (st != CFS_OK) return st;
    st = check_cuda(cudaMemcpyAsync(Y, s->Y, sizeof(float) * 2 * B, cudaMemcpyDeviceToDevice, sm),
                    "copy Y");
    if (st != CFS_OK) return st;
    return check_cuda(cudaGetLastError(), "sampler forward");
}

cfs_status cfs_sampler_backward(cfs_sampler* s, const void* U, uint32_t B, const float* dY,
                                float* grads, void* stream)
{
    clear_error();
    if (!s || !U || !dY || !grads) return fail(CFS_ERR_INVALID_ARG, "NULL argument");
    if (B == 0) return CFS_OK;
    if (B > (1u << 24)) return fail(CFS_ERR_INVALID_ARG, "B too large");
    cfs_status st = ensure_rows(s, (int)B);
    if (st != CFS_OK) return st;
    cudaStream_t sm = (cudaStream_t)stream;
    st = forward(s, (const bf16r*)U, (int)B, sm);
    if (st == CFS_OK) st = backward(s, (const bf16r*)U, (int)B, dY, grads, sm);
    if (st != CFS_OK) return st;
    return check_cuda(cudaGetLastError(), "sampler backward");
}

cfs_status cfs_sw_loss(const float* X, const float* T, uint32_t n_sys, uint32_t n_per,
                       const float* phi, uint32_t n_proj, float* loss, float* dX, void* stream)
{
    clear_error();
    if (!X || !T || !phi || !loss || !dX) return fail(CFS_ERR_INVALID_ARG, "NULL argument");
    if (n_per < 32 || n_per > 1024 || (n_per & (n_per - 1)))
        return fail(CFS_ERR_INVALID_ARG, "points per system must be a power of two in 32..1024");
    if (n_sys == 0 || n_proj == 0) return CFS_OK;
    const float scale = 1.0f / ((float)n_sys * (float)n_proj);
    cfs_status st = sw_init();
    if (st != CFS_OK) return st;
    sw_launch(X, T, phi, (int)n_proj, (int)n_per, (int)n_sys, scale, loss, dX,
              (cudaStream_t)stream);
    return check_cuda(cudaGetLastError(), "sw_kernel launch");
}

cfs_status cfs_sampler_adam(cfs_sampler* s, const float* grads, uint32_t t, float lr,
                            void* stream)
{
    clear_error();
    if (!s || !grads || t == 0) return fail(CFS_ERR_INVALID_ARG, "bad arguments");
    adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        s->w, s->m, s->v, grads, s->wb, s->wbT, N_PARAMS, nullptr, t, lr, lr, 0u, 0u, 0.9f,
        0.999f, 1e-8f);
    return check_cuda(cudaGetLastError(), "adam launch");
}

cfs_status cfs_sampler_train(cfs_sampler* s, const cfs_system* const* systems,
                             const float* t_values, int n_systems, uint32_t steps,
                             uint32_t systems_per_step, uint32_t points_per_system,
                             uint32_t n_proj, float lr, uint64_t seed, float* loss_history,
                             void* stream)
{
    cfs_train_options o;
    o.steps = steps;
    o.systems_per_step = systems_per_step;
    o.points_per_system = points_per_system;
    o.n_proj = n_proj;
    o.lr = lr;
    o.lr_final = lr;
    o.seed = seed;
    return cfs_sampler_train_ex(s, systems, t_values, n_systems, &o, loss_history, stream);
}

cfs_status cfs_sampler_train_ex(cfs_sampler* s, const cfs_system* const* systems,
                                const float* t_values, int n_systems,
                                const cfs_train_options* opt, float* loss_history, void* stream)
{
    clear_error();
    if (!s || !systems || !t_values || n_systems <= 0 || !opt)
        return fail(CFS_ERR_INVALID_ARG, "NULL sampler, systems or options");
    const uint32_t steps = opt->steps, systems_per_step = opt->systems_per_step;
    const uint32_t points_per_system = opt->points_per_system, n_proj = opt->n_proj;
    const float lr = opt->lr, lr_final = opt->lr_final;
    const uint64_t seed = opt->seed;
    if (!(lr > 0.0f) || !(lr_final > 0.0f) || !std::isfinite(lr) || !std::isfinite(lr_final))
        return fail(CFS_ERR_INVALID_ARG, "learning rates must be positive and finite");
    if (points_per_system < 32 || points_per_system > 1024 ||
        (points_per_system & (points_per_system - 1)))
        return fail(CFS_ERR_INVALID_ARG, "points per system must be a power of two in 32..1024");
    if (systems_per_step == 0 || systems_per_step > 1024 || n_proj == 0 || n_proj > 1024)
        return fail(CFS_ERR_INVALID_ARG, "systems per step and projections must be in 1..1024");
    for (int i = 0; i < n_systems; ++i) {
        cfs_status st = check_sampler_system(systems[i]);
        if (st != CFS_OK) return st;
    }
    cudaStream_t sm = (cudaStream_t)stream;
    const int S = (int)systems_per_step, N = (int)points_per_system, B = S * N;
    cfs_status st = ensure_rows(s, B);
    if (st != CFS_OK) return st;
    // device workspace of the run
    std::vector<SysRec> recs(n_systems);
    for (int i = 0; i < n_systems; ++i) pack_system(systems[i], t_values[i], &recs[i]);
    const size_t bytes = sizeof(SysRec) * n_systems + 4 * 1024 + 4 * 1024 +
                         sizeof(float) * (size_t)B * 2 * 2 + sizeof(bf16r) * (size_t)B * D_IN +
                         sizeof(float) * N_PARAMS + 256 + sizeof(float) * (steps + 1) + 8 * 256;
    unsigned char* ws = nullptr;
    st = check_cuda(cudaMalloc(&ws, bytes), "cudaMalloc(training workspace)");
    if (st != CFS_OK) return st;
    unsigned char* p = ws;
    auto take = [&](size_t n) {
        unsigned char* r = p;
        p += (n + 255) & ~(size_t)255;
        return r;
    };
    SysRec* d_sys = (SysRec*)take(sizeof(SysRec) * n_systems);
    u32* d_sel = (u32*)take(4 * 1024);
    float* d_phi = (float*)take(4 * 1024);
    float* d_T = (float*)take(sizeof(float) * (size_t)B * 2);
    float* d_dY = (float*)take(sizeof(float) * (size_t)B * 2);
    bf16r* d_U = (bf16r*)take(sizeof(bf16r) * (size_t)B * D_IN);
    float* d_g = (float*)take(sizeof(float) * N_PARAMS);
    float* d_loss = (float*)take(256);
    float* d_hist = (float*)take(sizeof(float) * (steps + 1));
    u32 step0 = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    st = check_cuda(cudaMemcpy(d_sys, recs.data(), sizeof(SysRec) * n_systems,
                               cudaMemcpyHostToDevice), "upload systems");
    if (st == CFS_OK) st = check_cuda(cudaMemcpy(&step0, s->d_step, 4, cudaMemcpyDeviceToHost), "step");
    if (st == CFS_OK) st = check_cuda(cudaMemset(d_hist, 0, sizeof(float) * (steps + 1)), "memset");
    if (st == CFS_OK) st = check_cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream");
    // one training step, captured once and replayed
    if (st == CFS_OK) st = check_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "capture");
    if (st == CFS_OK) {
        cudaMemsetAsync(d_g, 0, sizeof(float) * N_PARAMS, cap);
        cudaMemsetAsync(d_dY, 0, sizeof(float) * (size_t)B * 2, cap);
        cudaMemsetAsync(d_loss, 0, 4, cap);
        prep_kernel<<<1, 1024, 0, cap>>>(s->d_step, seed, n_systems, S, d_sel, d_phi, (int)n_proj);
        data_kernel<<<(B + 255) / 256, 256, 0, cap>>>(d_sys, d_sel, s->d_step, seed, N, B, 40, d_T,
                                                      d_U);
        cfs_status fst = forward(s, d_U, B, cap);
        sw_launch(s->Y, d_T, d_phi, (int)n_proj, N, S, 1.0f / ((float)S * (float)n_proj),
                  d_loss, d_dY, cap);
        gather_loss_kernel<<<1, 1, 0, cap>>>(d_loss, s->d_step, step0, d_hist, steps);
        if (fst == CFS_OK) fst = backward(s, d_U, B, d_dY, d_g, cap);
        adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, cap>>>(s->w, s->m, s->v, d_g, s->wb, s->wbT,
                                                             N_PARAMS, s->d_step, 0u, lr,
                                                             lr_final, step0, steps, 0.9f,
                                                             0.999f, 1e-8f);
        step_inc_kernel<<<1, 1, 0, cap>>>(s->d_step);
        cudaError_t e = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        st = check_cuda(e != cudaSuccess ? e : e2, "training step capture");
        if (st == CFS_OK && fst != CFS_OK) st = fst;
    }
    if (st == CFS_OK) st = check_cuda(cudaGraphInstantiate(&exec, graph, 0), "instantiate");
    for (uint32_t i = 0; i < steps && st == CFS_OK; ++i)
        st = check_cuda(cudaGraphLaunch(exec, sm), "cudaGraphLaunch");
    if (st == CFS_OK) st = check_cuda(cudaStreamSynchronize(sm), "training");
    if (st == CFS_OK && loss_history && steps > 0)
        st = check_cuda(cudaMemcpy(loss_history, d_hist, sizeof(float) * steps,
                                   cudaMemcpyDeviceToHost), "loss history");
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(ws);
    return st;
}

namespace {
struct InferLayout {
    size_t rec, c1, tiles, count, seed, out, total;
};

InferLayout infer_layout(int n)
{
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    InferLayout l;
    l.rec = 0;
    l.c1 = up(l.rec + sizeof(SysRec) * (size_t)n);
    l.tiles = up(l.c1 + sizeof(float) * HID * (size_t)n);
    l.count = up(l.tiles + sizeof(u32) * ((size_t)n + 1));
    l.seed = up(l.count + sizeof(u32) * (size_t)n);
    l.out = up(l.seed + sizeof(u64) * (size_t)n);
    l.total = up(l.out + sizeof(float*) * (size_t)n);
    return l;
}
}  // namespace

cfs_status cfs_sampler_start_points_batch(cfs_sampler* s, int n_frames,
                                          const cfs_system* const* systems, const float* t,
                                          const uint32_t* counts, const uint64_t* seeds,
                                          float* const* starts, void* stream)
{
    clear_error();
    if (!s || !systems || !t || !counts || !seeds || !starts || n_frames <= 0)
        return fail(CFS_ERR_INVALID_ARG, "NULL argument or no frames");
    uint64_t tiles = 0;
    for (int f = 0; f < n_frames; ++f) {
        cfs_status st = check_sampler_system(systems[f]);
        if (st != CFS_OK) return st;
        if (counts[f] > (1u << 30)) return fail(CFS_ERR_INVALID_ARG, "count too large");
        if (counts[f] && !starts[f]) return fail(CFS_ERR_INVALID_ARG, "NULL output");
        tiles += (counts[f] + 127) / 128;
    }
    if (tiles >= (1ull << 31)) return fail(CFS_ERR_INVALID_ARG, "too many rows");
    cudaStream_t sm = (cudaStream_t)stream;
    const InferLayout L = infer_layout(n_frames);
    if (n_frames > s->cap_frames) {
        // the previous staging buffer may still feed an upload
        cfs_status st = check_cuda(cudaDeviceSynchronize(), "sampler sync");
        if (st != CFS_OK) return st;
        if (s->inf) cudaFree(s->inf);
        if (s->inf_host) cudaFreeHost(s->inf_host);
        s->inf = nullptr;
        s->inf_host = nullptr;
        s->cap_frames = 0;
        st = check_cuda(cudaMalloc(&s->inf, L.total), "cudaMalloc(inference workspace)");
        if (st == CFS_OK)
            st = check_cuda(cudaMallocHost(&s->inf_host, L.total), "cudaMallocHost(inference)");
        if (st != CFS_OK) return st;
        s->cap_frames = n_frames;
    } else if (s->upload_pending) {
        // the staging buffer is rewritten: wait for its last upload only
        cfs_status st = check_cuda(cudaEventSynchronize(s->uploaded), "sampler upload sync");
        if (st != CFS_OK) return st;
    }
    if (!s->uploaded) {
        cfs_status st = check_cuda(cudaEventCreateWithFlags(&s->uploaded, cudaEventDisableTiming),
                                   "cudaEventCreate");
        if (st != CFS_OK) return st;
    }
    unsigned char* h = s->inf_host;
    u32* h_tiles = reinterpret_cast<u32*>(h + L.tiles);
    u32 acc = 0;
    for (int f = 0; f < n_frames; ++f) {
        pack_system(systems[f], t[f], reinterpret_cast<SysRec*>(h + L.rec) + f);
        h_tiles[f] = acc;
        acc += (counts[f] + 127) / 128;
        reinterpret_cast<u32*>(h + L.count)[f] = counts[f];
        reinterpret_cast<u64*>(h + L.seed)[f] = seeds[f];
        reinterpret_cast<float**>(h + L.out)[f] = starts[f];
    }
    h_tiles[n_frames] = acc;
    cfs_status st = check_cuda(cudaMemcpyAsync(s->inf, h, L.total, cudaMemcpyHostToDevice, sm),
                               "cudaMemcpyAsync(inference frames)");
    if (st == CFS_OK) st = check_cuda(cudaEventRecord(s->uploaded, sm), "cudaEventRecord");
    if (st != CFS_OK) return st;
    s->upload_pending = true;
    unsigned char* d = s->inf;
    cond_kernel<<<n_frames, HID, 0, sm>>>(s->wb, s->w, reinterpret_cast<const SysRec*>(d + L.rec),
                                         reinterpret_cast<float*>(d + L.c1));
    if (acc == 0) return check_cuda(cudaGetLastError(), "sampler conditioning");
    static int smem_set = -1;
    if (smem_set != s->device) {
        st = check_cuda(cudaFuncSetAttribute(infer_tc_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             IT_SMEM),
                        "cudaFuncSetAttribute");
        if (st != CFS_OK) return st;
        smem_set = s->device;
    }
    // persistent: one CTA per SM (its shared memory and 512 TMEM columns),
    // IT_GROUPS tiles in flight per CTA
    const int sms = std::max(1, device_sm_count());
    const int grid = (int)std::min<uint64_t>((uint64_t)sms, (acc + IT_GROUPS - 1) / IT_GROUPS);
    InferFrames fs;
    fs.c1 = reinterpret_cast<const float*>(d + L.c1);
    fs.tile_begin = reinterpret_cast<const u32*>(d + L.tiles);
    fs.count = reinterpret_cast<const u32*>(d + L.count);
    fs.seed = reinterpret_cast<const u64*>(d + L.seed);
    fs.out = reinterpret_cast<float* const*>(d + L.out);
    fs.n_sys = n_frames;
    infer_tc_kernel<<<grid, IT_THREADS, IT_SMEM, sm>>>(s->wb, s->w, fs);
    return check_cuda(cudaGetLastError(), "sampler start points");
}

cfs_status cfs_sampler_start_points(cfs_sampler* s, const cfs_system* sys, float t, uint32_t n,
                                    uint64_t seed, float* start, void* stream)
{
    if (n == 0) {
        clear_error();
        if (!s || !start) return fail(CFS_ERR_INVALID_ARG, "NULL sampler or output");
        return check_sampler_system(sys);
    }
    return cfs_sampler_start_points_batch(s, 1, &sys, &t, &n, &seed, &start, stream);
}

}  // extern "C"
