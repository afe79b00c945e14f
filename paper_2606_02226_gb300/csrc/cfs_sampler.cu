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
// cores (mma.sync m16n8k16 bf16), FP32 master weights and Adam state.
//
// Parameter vector (FP32, this order): W1 [128][64], b1 [128], W2 [128][128],
// b2, W3 [128][128], b3, W4 [2][128], b4 [2] -- 41602 floats.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
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

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// ---------------------------------------------------------------------------
// GEMM: C[M][N] = op(A)[M][K] op(B)[K][N], BF16 in, FP32 accumulate.
//   op(A)(m, k) = transA ? A[k * lda + m] : A[m * lda + k]
//   op(B)(k, n) = transB ? B[n * ldb + k] : B[k * ldb + n]
// Tiles of 64 x 128 (8 warps, each 16 x 64), K in steps of 32 staged in
// shared memory as [m][k] and [n][k] (rows padded to 80 bytes: ldmatrix
// reads are conflict-free), fragments by ldmatrix, mma.sync m16n8k16.
// ---------------------------------------------------------------------------
enum Epi { EPI_STORE = 0, EPI_SILU = 1, EPI_SILU_GRAD = 2, EPI_ATOMIC = 3 };

struct GemmArgs {
    int M, N, K;
    const bf16r* A;
    int lda, transA;
    const bf16r* B;
    int ldb, transB;
    int k_split;          // K range per blockIdx.z
    int mode;
    const float* bias;    // [N] or null
    float* C;             // fp32 out (STORE, ATOMIC) or pre-activation out (SILU)
    int ldc;
    bf16r* H;             // bf16 out (SILU: activation, SILU_GRAD: dZ)
    int ldh;
    const float* Zin;     // SILU_GRAD: pre-activation
    int ldz;
    float* colsum;        // SILU_GRAD: bias gradient (atomic)
};

constexpr int BM = 64, BN = 128, BK = 32, SPAD = 8;

__device__ __forceinline__ void ldsm_x4(u32 (&r)[4], const void* p)
{
    const u32 a = (u32)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const u32 (&a)[4], u32 b0, u32 b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) gemm_kernel(const GemmArgs g)
{
    __shared__ __align__(16) bf16r sA[BM][BK + SPAD];
    __shared__ __align__(16) bf16r sB[BN][BK + SPAD];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * g.k_split;
    const int ke = min(g.K, kb + g.k_split);
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

    for (int k0 = kb; k0 < ke; k0 += BK) {
        // stage op(A) tile as [m][k]; consecutive threads walk the
        // contiguous dimension of the source
        for (int e = threadIdx.x; e < BM * BK; e += blockDim.x) {
            int r, c;
            if (g.transA) { r = e % BM; c = e / BM; } else { r = e / BK; c = e % BK; }
            const int m = m0 + r, k = k0 + c;
            bf16r v = 0;
            if (m < g.M && k < ke)
                v = g.transA ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
            sA[r][c] = v;
        }
        for (int e = threadIdx.x; e < BN * BK; e += blockDim.x) {
            int r, c;
            if (g.transB) { r = e / BK; c = e % BK; } else { r = e % BN; c = e / BN; }
            const int n = n0 + r, k = k0 + c;
            bf16r v = 0;
            if (n < g.N && k < ke)
                v = g.transB ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
            sB[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            u32 a[4];
            ldsm_x4(a, &sA[wm * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int nt = 0; nt < 8; nt += 2) {
                u32 b[4];
                const int nrow = wn * 64 + nt * 8 + (lane & 7) + ((lane >> 4) << 3);
                const int kcol = kk + ((lane >> 3) & 1) * 8;
                ldsm_x4(b, &sB[nrow][kcol]);
                mma_bf16(acc[nt], a, b[0], b[1]);
                mma_bf16(acc[nt + 1], a, b[2], b[3]);
            }
        }
        __syncthreads();
    }

    // epilogue: thread (g, t) holds rows g, g + 8 and columns 2t, 2t + 1 of
    // each 16 x 8 tile
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float cs[2] = {0.0f, 0.0f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = m0 + wm * 16 + gq + 8 * h;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int col = n0 + wn * 64 + nt * 8 + 2 * tq + q;
                const float v = acc[nt][2 * h + q];
                const bool in = row < g.M && col < g.N;
                if (g.mode == EPI_STORE) {
                    if (in) g.C[(size_t)row * g.ldc + col] = v + (g.bias ? g.bias[col] : 0.0f);
                } else if (g.mode == EPI_SILU) {
                    if (in) {
                        const float z = v + g.bias[col];
                        g.C[(size_t)row * g.ldc + col] = z;
                        g.H[(size_t)row * g.ldh + col] = to_bf16(silu_f(z));
                    }
                } else if (g.mode == EPI_SILU_GRAD) {
                    float d = 0.0f;
                    if (in) {
                        d = v * silu_grad_f(g.Zin[(size_t)row * g.ldz + col]);
                        g.H[(size_t)row * g.ldh + col] = to_bf16(d);
                    }
                    cs[q] += d;
                } else {
                    if (in) atomicAdd(g.C + (size_t)row * g.ldc + col, v);
                }
            }
        }
        if (g.mode == EPI_SILU_GRAD) {
            // column sums over the warp's 16 rows: reduce across gq
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float s = cs[q];
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 8);
                s += __shfl_xor_sync(0xffffffffu, s, 16);
                const int col = n0 + wn * 64 + nt * 8 + 2 * tq + q;
                if (gq == 0 && col < g.N && s != 0.0f) atomicAdd(g.colsum + col, s);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// output layer backward: dH3 = dY W4, dZ3 = dH3 * silu'(Z3) (bf16 out),
// db3 += sum dZ3, dW4 += dY^T H3, db4 += sum dY.  One thread per hidden
// unit, 64 rows per block.
// ---------------------------------------------------------------------------
constexpr int OB_ROWS = 64;

__global__ void __launch_bounds__(HID) out_backward_kernel(const float* __restrict__ dY,
                                                           const bf16r* __restrict__ wb,
                                                           const bf16r* __restrict__ H3,
                                                           const float* __restrict__ Z3, int B,
                                                           bf16r* dZ3, float* grads)
{
    const int n = threadIdx.x;
    const float w0 = from_bf16(wb[OFF_W4 + n]), w1 = from_bf16(wb[OFF_W4 + HID + n]);
    float db3 = 0.0f, dw0 = 0.0f, dw1 = 0.0f, db40 = 0.0f, db41 = 0.0f;
    const int r0 = blockIdx.x * OB_ROWS;
    for (int r = r0; r < min(B, r0 + OB_ROWS); ++r) {
        const float y0 = dY[2 * r], y1 = dY[2 * r + 1];
        const float dh = fmaf(y0, w0, y1 * w1);
        const float d = dh * silu_grad_f(Z3[(size_t)r * HID + n]);
        dZ3[(size_t)r * HID + n] = to_bf16(d);
        db3 += d;
        const float h = from_bf16(H3[(size_t)r * HID + n]);
        dw0 = fmaf(y0, h, dw0);
        dw1 = fmaf(y1, h, dw1);
        db40 += y0;
        db41 += y1;
    }
    atomicAdd(grads + OFF_B3 + n, db3);
    atomicAdd(grads + OFF_W4 + n, dw0);
    atomicAdd(grads + OFF_W4 + HID + n, dw1);
    if (n == 0) {
        atomicAdd(grads + OFF_B4, db40);
        atomicAdd(grads + OFF_B4 + 1, db41);
    }
}

// ---------------------------------------------------------------------------
// sliced-Wasserstein loss and gradient: one CTA of N threads (N a power of
// two in 32..1024) per system; per projection both point sets are projected,
// bitonic-sorted in shared memory (predicted points with their indices) and
// matched rank by rank.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) sw_kernel(const float* __restrict__ X,
                                                  const float* __restrict__ T,
                                                  const float* __restrict__ phi, int P, int N,
                                                  float scale, float* loss, float* dX)
{
    __shared__ float kx[1024], ky[1024], gxs[1024], gys[1024];
    __shared__ int ix[1024];
    __shared__ float red[32];
    const int s = blockIdx.x, i = threadIdx.x;
    const float xi0 = X[((size_t)s * N + i) * 2], xi1 = X[((size_t)s * N + i) * 2 + 1];
    const float ti0 = T[((size_t)s * N + i) * 2], ti1 = T[((size_t)s * N + i) * 2 + 1];
    gxs[i] = 0.0f;
    gys[i] = 0.0f;
    float lacc = 0.0f;
    for (int j = 0; j < P; ++j) {
        float sn, c;
        sincosf(phi[j], &sn, &c);
        kx[i] = fmaf(xi0, c, xi1 * sn);
        ky[i] = fmaf(ti0, c, ti1 * sn);
        ix[i] = i;
        __syncthreads();
        for (int k = 2; k <= N; k <<= 1) {
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                const int p = i ^ jj;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const float a = kx[i], b = kx[p];
                    if ((a > b) == up) {
                        kx[i] = b; kx[p] = a;
                        const int t = ix[i]; ix[i] = ix[p]; ix[p] = t;
                    }
                    const float u = ky[i], v = ky[p];
                    if ((u > v) == up) { ky[i] = v; ky[p] = u; }
                }
                __syncthreads();
            }
        }
        const float diff = kx[i] - ky[i];
        lacc = fmaf(diff, diff, lacc);
        const float gv = 2.0f * diff / (float)N;
        const int idx = ix[i];
        gxs[idx] = fmaf(gv, c, gxs[idx]);
        gys[idx] = fmaf(gv, sn, gys[idx]);
        __syncthreads();
    }
    dX[((size_t)s * N + i) * 2] += gxs[i] * scale;
    dX[((size_t)s * N + i) * 2 + 1] += gys[i] * scale;
    float v = lacc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((i & 31) == 0) red[i >> 5] = v;
    __syncthreads();
    if (i == 0) {
        float t = 0.0f;
        for (int w = 0; w < (N + 31) / 32; ++w) t += red[w];
        atomicAdd(loss, t * scale / (float)N);
    }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) with bias correction on the FP32 master weights; writes
// the BF16 copies the GEMMs read.  t (1-based) is *step + 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) adam_kernel(float* w, float* m, float* v,
                                                   const float* g, bf16r* wb, int n,
                                                   const u32* step, u32 t_explicit, float lr,
                                                   float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32 t = step ? (*step + 1u) : t_explicit;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = to_bf16(wi);
}

__global__ void to_bf16_kernel(const float* w, bf16r* wb, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = to_bf16(w[i]);
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

// chaos-game points of the batch's systems: row r = s * N + j starts
// uniform and runs `steps` steps (enough to reach the attractor)
__global__ void __launch_bounds__(256) data_kernel(const SysRec* __restrict__ sys,
                                                   const u32* __restrict__ sel, const u32* step,
                                                   u64 seed, int N, int rows, int steps,
                                                   float* out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const SysRec& q = sys[sel[r / N]];
    const u32 st = *step;
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

// network inputs: row r = s * N + j gets Gaussian noise (Box-Muller on a
// Philox block), the conditioning vector of its system and t
__global__ void __launch_bounds__(256) inputs_kernel(const SysRec* __restrict__ sys,
                                                     const u32* __restrict__ sel,
                                                     const u32* step, u32 step_explicit,
                                                     u64 seed, int N, int rows, bf16r* U)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const SysRec& q = sys[sel ? sel[r / N] : 0];
    const u32 st = step ? *step : step_explicit;
    const uint4 w = philox_key(seed, (u32)r, st, 0u, TAG_NOISE);
    const float u1 = ((float)(w.x >> 8) + 0.5f) * CFS_INV_2_24;
    const float u2 = (float)(w.y >> 8) * CFS_INV_2_24;
    const float rad = sqrtf(-2.0f * logf(u1));
    float sn, c;
    sincosf(6.28318530717958647692f * u2, &sn, &c);
    bf16r* row = U + (size_t)r * D_IN;
    row[0] = to_bf16(rad * c);
    row[1] = to_bf16(rad * sn);
    for (int j = 0; j < COND; ++j) row[2 + j] = to_bf16(q.cond[j]);
    row[2 + COND] = to_bf16(q.t);
    for (int j = 3 + COND; j < D_IN; ++j) row[j] = 0;
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
// fused inference: start points of one system straight from noise.
// Layer 1 is a rank-2 update: only the noise varies from row to row, so
// z1 = c1 + W1[:, 0] n0 + W1[:, 1] n1 with c1 = W1[:, 2:51] u_cond + b1 (one
// vector per call).  Layers 2-4 run on the tensor cores (mma.sync m16n8k16
// bf16); each warp keeps its 16 rows' activations in registers: the FP32
// accumulator fragments of one layer, rounded to BF16, are exactly the A
// fragments of the next.  Weights live in shared memory with rows padded to
// 272 bytes (conflict-free ldmatrix).
// ---------------------------------------------------------------------------
constexpr int IP = 136;                       // padded row length (bf16)
constexpr int IW = 4;                         // warps per CTA
struct InferSmem {
    bf16r w2[HID][IP];
    bf16r w3[HID][IP];
    bf16r w4[8][IP];
    float c1[HID], w10[HID], w11[HID], b2[HID], b3[HID], b4[2];
};

__device__ __forceinline__ u32 pack2(float lo, float hi)
{
    return (u32)to_bf16(lo) | ((u32)to_bf16(hi) << 16);
}

__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

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

__device__ __forceinline__ void hidden_layer(const bf16r (*W)[IP], const float* bias, u32 (&a)[8][4],
                                             int lane)
{
    float acc[16][4];
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
#pragma unroll
        for (int nt = 0; nt < 16; nt += 2) {
            u32 b[4];
            ldsm_x4(b, &W[nt * 8 + (lane & 7) + ((lane >> 4) << 3)][kt * 16 + ((lane >> 3) & 1) * 8]);
            mma_bf16(acc[nt], a[kt], b[0], b[1]);
            mma_bf16(acc[nt + 1], a[kt], b[2], b[3]);
        }
    }
    const int tq = lane & 3;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const int c0 = (2 * kt) * 8 + 2 * tq, c1 = (2 * kt + 1) * 8 + 2 * tq;
        a[kt][0] = pack2(silu_fast(acc[2 * kt][0] + bias[c0]), silu_fast(acc[2 * kt][1] + bias[c0 + 1]));
        a[kt][1] = pack2(silu_fast(acc[2 * kt][2] + bias[c0]), silu_fast(acc[2 * kt][3] + bias[c0 + 1]));
        a[kt][2] = pack2(silu_fast(acc[2 * kt + 1][0] + bias[c1]),
                         silu_fast(acc[2 * kt + 1][1] + bias[c1 + 1]));
        a[kt][3] = pack2(silu_fast(acc[2 * kt + 1][2] + bias[c1]),
                         silu_fast(acc[2 * kt + 1][3] + bias[c1 + 1]));
    }
}

// frames of one inference launch: tile_begin[f] = first 16-row tile of
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

__global__ void __launch_bounds__(IW * 32) infer_kernel(const bf16r* __restrict__ wb,
                                                        const float* __restrict__ w,
                                                        const InferFrames fs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem& sm = *reinterpret_cast<InferSmem*>(smem_raw);
    for (int e = threadIdx.x; e < HID * HID; e += blockDim.x) {
        const int r = e / HID, c = e % HID;
        sm.w2[r][c] = wb[OFF_W2 + e];
        sm.w3[r][c] = wb[OFF_W3 + e];
    }
    for (int e = threadIdx.x; e < 8 * HID; e += blockDim.x) {
        const int r = e / HID, c = e % HID;
        sm.w4[r][c] = r < D_OUT ? wb[OFF_W4 + e] : (bf16r)0;
    }
    for (int j = threadIdx.x; j < HID; j += blockDim.x) {
        sm.w10[j] = from_bf16(wb[OFF_W1 + j * D_IN]);
        sm.w11[j] = from_bf16(wb[OFF_W1 + j * D_IN + 1]);
        sm.b2[j] = w[OFF_B2 + j];
        sm.b3[j] = w[OFF_B3 + j];
    }
    if (threadIdx.x < 2) sm.b4[threadIdx.x] = w[OFF_B4 + threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const u32 tiles = fs.tile_begin[fs.n_sys];
    for (u32 tile = blockIdx.x * IW + warp; tile < tiles; tile += gridDim.x * IW) {
        // the frame of this tile: last f with tile_begin[f] <= tile
        int lo = 0, hi = fs.n_sys;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (fs.tile_begin[mid] <= tile) lo = mid; else hi = mid;
        }
        const int f = lo;
        const u32 lt = tile - fs.tile_begin[f];
        const int n = (int)fs.count[f];
        const u64 seed = fs.seed[f];
        const float* c1 = fs.c1 + (size_t)f * HID;
        float* start = fs.out[f];
        // noise of rows gq and gq + 8 (Box-Muller on Philox (row, 0, 0, 3))
        float nz[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const u32 row = lt * 16 + (u32)(gq + 8 * h);
            const uint4 r = philox_key(seed, row, 0u, 0u, TAG_NOISE);
            const float u1 = ((float)(r.x >> 8) + 0.5f) * CFS_INV_2_24;
            const float u2 = (float)(r.y >> 8) * CFS_INV_2_24;
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincosf(6.28318530717958647692f * u2, &sn, &cs);
            nz[h][0] = from_bf16(to_bf16(rad * cs));
            nz[h][1] = from_bf16(to_bf16(rad * sn));
        }
        // layer 1 (rank-2 update), straight into the A fragments of layer 2
        u32 a[8][4];
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int c = (2 * kt + half) * 8 + 2 * tq;
                float v[2][2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float cc = c1[c + q];
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        v[h][q] = silu_fast(fmaf(sm.w11[c + q], nz[h][1],
                                                 fmaf(sm.w10[c + q], nz[h][0], cc)));
                }
                a[kt][2 * half + 0] = pack2(v[0][0], v[0][1]);
                a[kt][2 * half + 1] = pack2(v[1][0], v[1][1]);
            }
        }
        hidden_layer(sm.w2, sm.b2, a, lane);
        hidden_layer(sm.w3, sm.b3, a, lane);
        // output layer: one 16 x 8 tile, columns 0 and 1 are the point
        float y[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kt = 0; kt < 8; ++kt) {
            u32 b[4];
            ldsm_x4(b, &sm.w4[(lane & 7)][kt * 16 + ((lane >> 3) & 1) * 8]);
            mma_bf16(y, a[kt], b[0], b[1]);
        }
        if (tq == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = (int)lt * 16 + gq + 8 * h;
                if (row < n) {
                    start[row] = y[2 * h] + sm.b4[0];
                    start[(size_t)n + row] = y[2 * h + 1] + sm.b4[1];
                }
            }
        }
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
    unsigned char* act = nullptr;
    float *Z1, *Z2, *Z3, *Y;
    bf16r *H1, *H2, *H3, *dZ1, *dZ2, *dZ3;
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
    const size_t bytes = 3 * fz + (size_t)B * 2 * 4 + 6 * fh + 6 * 256;
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
    s->cap_rows = B;
    return CFS_OK;
}

void gemm(cudaStream_t st, int M, int N, int K, const bf16r* A, int lda, int tA, const bf16r* B,
          int ldb, int tB, int mode, const float* bias, float* C, int ldc, bf16r* H, int ldh,
          const float* Zin, int ldz, float* colsum, int splits = 1)
{
    GemmArgs g;
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.transA = tA;
    g.B = B; g.ldb = ldb; g.transB = tB;
    const int kc = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    g.k_split = kc;
    g.mode = mode; g.bias = bias; g.C = C; g.ldc = ldc; g.H = H; g.ldh = ldh;
    g.Zin = Zin; g.ldz = ldz; g.colsum = colsum;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, (K + kc - 1) / kc);
    gemm_kernel<<<grid, 256, 0, st>>>(g);
}

// forward of B rows of U: Z1..Z3 (fp32), H1..H3 (bf16), Y (fp32 [B][2])
void forward(cfs_sampler* s, const bf16r* U, int B, cudaStream_t st)
{
    const bf16r* wb = s->wb;
    gemm(st, B, HID, D_IN, U, D_IN, 0, wb + OFF_W1, D_IN, 1, EPI_SILU, s->w + OFF_B1, s->Z1, HID,
         s->H1, HID, nullptr, 0, nullptr);
    gemm(st, B, HID, HID, s->H1, HID, 0, wb + OFF_W2, HID, 1, EPI_SILU, s->w + OFF_B2, s->Z2,
         HID, s->H2, HID, nullptr, 0, nullptr);
    gemm(st, B, HID, HID, s->H2, HID, 0, wb + OFF_W3, HID, 1, EPI_SILU, s->w + OFF_B3, s->Z3,
         HID, s->H3, HID, nullptr, 0, nullptr);
    gemm(st, B, D_OUT, HID, s->H3, HID, 0, wb + OFF_W4, HID, 1, EPI_STORE, s->w + OFF_B4, s->Y,
         D_OUT, nullptr, 0, nullptr, 0, nullptr);
}

// backward of sum(dY * Y) after forward(): adds into grads [N_PARAMS]
void backward(cfs_sampler* s, const bf16r* U, int B, const float* dY, float* grads,
              cudaStream_t st)
{
    const bf16r* wb = s->wb;
    out_backward_kernel<<<(B + OB_ROWS - 1) / OB_ROWS, HID, 0, st>>>(dY, wb, s->H3, s->Z3, B,
                                                                      s->dZ3, grads);
    // dZ2 = (dZ3 W3) * silu'(Z2): op(B)(k = o, n = i) = W3[o][i]
    gemm(st, B, HID, HID, s->dZ3, HID, 0, wb + OFF_W3, HID, 0, EPI_SILU_GRAD, nullptr, nullptr,
         0, s->dZ2, HID, s->Z2, HID, grads + OFF_B2);
    gemm(st, B, HID, HID, s->dZ2, HID, 0, wb + OFF_W2, HID, 0, EPI_SILU_GRAD, nullptr, nullptr,
         0, s->dZ1, HID, s->Z1, HID, grads + OFF_B1);
    // weight gradients dW = dZ^T A over the rows (split-K, atomic)
    const int splits = B >= 8192 ? 32 : (B >= 1024 ? 8 : 1);
    gemm(st, HID, HID, B, s->dZ3, HID, 1, s->H2, HID, 0, EPI_ATOMIC, nullptr, grads + OFF_W3, HID,
         nullptr, 0, nullptr, 0, nullptr, splits);
    gemm(st, HID, HID, B, s->dZ2, HID, 1, s->H1, HID, 0, EPI_ATOMIC, nullptr, grads + OFF_W2, HID,
         nullptr, 0, nullptr, 0, nullptr, splits);
    gemm(st, HID, D_IN, B, s->dZ1, HID, 1, U, D_IN, 0, EPI_ATOMIC, nullptr, grads + OFF_W1, D_IN,
         nullptr, 0, nullptr, 0, nullptr, splits);
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
    to_bf16_kernel<<<(N_PARAMS + 255) / 256, 256>>>(s->w, s->wb, N_PARAMS);
    return check_cuda(cudaDeviceSynchronize(), "sampler params");
}

void pack_system(const cfs_system* sys, float t, SysRec* r)
{
    std::memset(r, 0, sizeof(*r));
    for (int j = 0; j < sys->n_cmp; ++j) r->T[j] = sys->T[j];
    r->n_cmp = sys->n_cmp;
    r->n_maps = sys->n_maps;
    for (int k = 0; k < sys->n_maps && k < MAX_SYS_MAPS; ++k)
        for (int j = 0; j < 6; ++j) {
            r->prm[k][j] = sys->maps[k].params[j];
            r->cond[6 * k + j] = sys->maps[k].params[j];
        }
    r->t = t;
}

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
    cfs_status st = check_cuda(cudaMalloc(&s->w, sizeof(float) * N_PARAMS * 3 +
                                                     sizeof(bf16r) * N_PARAMS + 256),
                               "cudaMalloc(sampler params)");
    if (st != CFS_OK) { delete s; return st; }
    s->m = s->w + N_PARAMS;
    s->v = s->m + N_PARAMS;
    s->wb = reinterpret_cast<bf16r*>(s->v + N_PARAMS);
    st = check_cuda(cudaMalloc(&s->d_step, 256), "cudaMalloc(step)");
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
    forward(s, (const bf16r*)U, (int)B, sm);
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
    forward(s, (const bf16r*)U, (int)B, sm);
    backward(s, (const bf16r*)U, (int)B, dY, grads, sm);
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
    sw_kernel<<<n_sys, n_per, 0, (cudaStream_t)stream>>>(X, T, phi, (int)n_proj, (int)n_per,
                                                         scale, loss, dX);
    return check_cuda(cudaGetLastError(), "sw_kernel launch");
}

cfs_status cfs_sampler_adam(cfs_sampler* s, const float* grads, uint32_t t, float lr,
                            void* stream)
{
    clear_error();
    if (!s || !grads || t == 0) return fail(CFS_ERR_INVALID_ARG, "bad arguments");
    adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        s->w, s->m, s->v, grads, s->wb, N_PARAMS, nullptr, t, lr, 0.9f, 0.999f, 1e-8f);
    return check_cuda(cudaGetLastError(), "adam launch");
}

cfs_status cfs_sampler_train(cfs_sampler* s, const cfs_system* const* systems,
                             const float* t_values, int n_systems, uint32_t steps,
                             uint32_t systems_per_step, uint32_t points_per_system,
                             uint32_t n_proj, float lr, uint64_t seed, float* loss_history,
                             void* stream)
{
    clear_error();
    if (!s || !systems || !t_values || n_systems <= 0)
        return fail(CFS_ERR_INVALID_ARG, "NULL sampler or systems");
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
        data_kernel<<<(B + 255) / 256, 256, 0, cap>>>(d_sys, d_sel, s->d_step, seed, N, B, 40, d_T);
        inputs_kernel<<<(B + 255) / 256, 256, 0, cap>>>(d_sys, d_sel, s->d_step, 0u, seed, N, B, d_U);
        forward(s, d_U, B, cap);
        sw_kernel<<<S, N, 0, cap>>>(s->Y, d_T, d_phi, (int)n_proj, N,
                                    1.0f / ((float)S * (float)n_proj), d_loss, d_dY);
        gather_loss_kernel<<<1, 1, 0, cap>>>(d_loss, s->d_step, step0, d_hist, steps);
        backward(s, d_U, B, d_dY, d_g, cap);
        adam_kernel<<<(N_PARAMS + 255) / 256, 256, 0, cap>>>(s->w, s->m, s->v, d_g, s->wb,
                                                             N_PARAMS, s->d_step, 0u, lr, 0.9f,
                                                             0.999f, 1e-8f);
        step_inc_kernel<<<1, 1, 0, cap>>>(s->d_step);
        cudaError_t e = cudaGetLastError();
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        st = check_cuda(e != cudaSuccess ? e : e2, "training step capture");
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
        tiles += (counts[f] + 15) / 16;
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
        acc += (counts[f] + 15) / 16;
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
    const int smem = (int)sizeof(InferSmem);
    static int smem_set = -1;
    if (smem_set != s->device) {
        st = check_cuda(cudaFuncSetAttribute(infer_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                        "cudaFuncSetAttribute");
        if (st != CFS_OK) return st;
        smem_set = s->device;
    }
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, infer_kernel, IW * 32, smem);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    int grid = std::max(1, per_sm) * std::max(1, sms);
    grid = (int)std::min<uint64_t>((uint64_t)grid, (acc + IW - 1) / IW);
    InferFrames fs;
    fs.c1 = reinterpret_cast<const float*>(d + L.c1);
    fs.tile_begin = reinterpret_cast<const u32*>(d + L.tiles);
    fs.count = reinterpret_cast<const u32*>(d + L.count);
    fs.seed = reinterpret_cast<const u64*>(d + L.seed);
    fs.out = reinterpret_cast<float* const*>(d + L.out);
    fs.n_sys = n_frames;
    infer_kernel<<<grid, IW * 32, smem, sm>>>(s->wb, s->w, fs);
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
