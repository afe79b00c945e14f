// cfs_display.cu -- density-estimation display: accumulated layers to packed
// 8-bit RGBA (log density with a gamma, the fractal-flame display of Draves &
// Reckase 2003; the paper names density estimation as the output that keeps
// atomics on the path, Section 4).
//
// Two kernels over work items of kDisplayPxPerItem pixels, numbered layer by
// layer, so one launch covers one layer or every frame of a batch:
//   density_max_kernel -- per-layer maximum of the accumulated alpha
//                         (block reduction, then one atomicMax on the float
//                         bits, which order like the values for A >= 0);
//   display_map_kernel -- per pixel d = ln(1 + A) / ln(1 + A_max),
//                         v = brightness d^(1/gamma), colour S/A v, 8 bits.
// Both are streaming passes (16 B per RGBA pixel or 4 C B per histogram
// pixel read by each, 4 B written by the second): 4 pixels per thread with
// 16-byte loads and stores.
#include <cmath>
#include <cstring>
#include <sstream>

#include <cuda_runtime.h>

#include "cfs_internal.h"

namespace {
using cfs::DisplayLayer;
using cfs::kDisplayPxPerItem;
typedef unsigned int u32;
typedef unsigned long long u64;

constexpr int kThreads = 256;

struct DispArgs {
    DisplayLayer one;             // the layer when `layers` is null
    const DisplayLayer* layers;   // device [n_layers] or null
    float* a_max;                 // device [n_layers]
    int n_layers;
    u32 n_items;
    float inv_gamma, brightness, a_max_fixed;
    u32 background;
};

__device__ __forceinline__ int layer_of(const DispArgs& a, u32 item)
{
    if (!a.layers) return 0;
    int lo = 0, hi = a.n_layers - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.layers[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// copies the item's layer description into shared memory (all threads)
__device__ __forceinline__ int load_layer(const DispArgs& a, u32 item, DisplayLayer& sL)
{
    const int li = layer_of(a, item);
    const DisplayLayer* src = a.layers ? a.layers + li : &a.one;
    constexpr int kWords = (int)(sizeof(DisplayLayer) / 4);
    static_assert(sizeof(DisplayLayer) % 4 == 0 && kWords <= kThreads, "layer copy");
    if ((int)threadIdx.x < kWords)
        reinterpret_cast<u32*>(&sL)[threadIdx.x] = reinterpret_cast<const u32*>(src)[threadIdx.x];
    __syncthreads();
    return li;
}

// accumulated (R, G, B, A) of pixels p .. p+3; `vec`: all four exist and the
// layer's planes allow 16-byte loads
__device__ __forceinline__ void sums4(const DisplayLayer& L, u32 p, bool vec, bool last_read,
                                      float4 (&s)[4])
{
    if (L.kind == CFS_TARGET_RGBA_F32) {
        const float4* src = reinterpret_cast<const float4*>(L.data) + p;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (vec || p + j < L.n_px) s[j] = last_read ? __ldcs(src + j) : __ldg(src + j);
            else s[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        return;
    }
    // histogram: s = s + n_c * palette[c], channel by channel (no fusion)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const u32* h = reinterpret_cast<const u32*>(L.data);
    for (int c = 0; c < L.C; ++c) {
        const u32* plane = h + (size_t)c * L.n_px;
        u32 n[4];
        if (vec) {
            const uint4* q = reinterpret_cast<const uint4*>(plane + p);
            const uint4 v = last_read ? __ldcs(q) : __ldg(q);
            n[0] = v.x; n[1] = v.y; n[2] = v.z; n[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) n[j] = p + j < L.n_px ? plane[p + j] : 0u;
        }
        const float* pc = L.pal[c];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float f = (float)n[j];
            s[j].x = __fadd_rn(s[j].x, __fmul_rn(f, pc[0]));
            s[j].y = __fadd_rn(s[j].y, __fmul_rn(f, pc[1]));
            s[j].z = __fadd_rn(s[j].z, __fmul_rn(f, pc[2]));
            s[j].w = __fadd_rn(s[j].w, __fmul_rn(f, pc[3]));
        }
    }
}

__device__ __forceinline__ float block_max(float m, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (int)threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    return m;
}

__global__ void __launch_bounds__(kThreads) density_max_kernel(const __grid_constant__ DispArgs a)
{
    __shared__ __align__(16) DisplayLayer sL;
    __shared__ float red[kThreads / 32];
    for (u32 item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int li = load_layer(a, item, sL);
        float m = 0.0f;
        if (sL.kind != CFS_TARGET_DEPTH_U64) {
            const u32 p0 = (item - sL.item_begin) * kDisplayPxPerItem;
            const u32 p1 = min(sL.n_px, p0 + kDisplayPxPerItem);
            const bool planes_ok = sL.kind != CFS_TARGET_HIST_U32 || (sL.n_px & 3u) == 0;
            for (u32 p = p0 + 4 * threadIdx.x; p < p1; p += 4 * kThreads) {
                float4 s[4];
                sums4(sL, p, planes_ok && p + 4 <= sL.n_px, false, s);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (s[j].w > m) m = s[j].w;   // NaN and negatives never count
            }
        }
        m = block_max(m, red);
        if (threadIdx.x == 0 && m > 0.0f)
            atomicMax(reinterpret_cast<u32*>(a.a_max + li), __float_as_uint(m));
        __syncthreads();   // sL and red are reused by the next item
    }
}

__device__ __forceinline__ u32 quant8(float x)
{
    if (!(x > 0.0f)) x = 0.0f;
    if (x > 1.0f) x = 1.0f;
    const float y = __fadd_rn(__fmul_rn(255.0f, x), 0.5f);
    return (u32)y;
}

__device__ __forceinline__ u32 map_pixel(const float4 s, float l_max, const DispArgs& a)
{
    if (!(s.w > 0.0f)) return a.background;
    const float d = __fdiv_rn(logf(__fadd_rn(1.0f, s.w)), l_max);
    const float v = __fmul_rn(a.brightness, powf(d, a.inv_gamma));
    const float r = __fmul_rn(__fdiv_rn(s.x, s.w), v);
    const float g = __fmul_rn(__fdiv_rn(s.y, s.w), v);
    const float b = __fmul_rn(__fdiv_rn(s.z, s.w), v);
    return quant8(r) | (quant8(g) << 8) | (quant8(b) << 16) | (quant8(v) << 24);
}

__global__ void __launch_bounds__(kThreads, 4) display_map_kernel(const __grid_constant__ DispArgs a)
{
    __shared__ __align__(16) DisplayLayer sL;
    for (u32 item = blockIdx.x; item < a.n_items; item += gridDim.x) {
        const int li = load_layer(a, item, sL);
        const u32 p0 = (item - sL.item_begin) * kDisplayPxPerItem;
        const u32 p1 = min(sL.n_px, p0 + kDisplayPxPerItem);
        u32* out = reinterpret_cast<u32*>(sL.out);
        if (sL.kind == CFS_TARGET_DEPTH_U64) {
            const u64* keys = reinterpret_cast<const u64*>(sL.data);
            for (u32 p = p0 + 4 * threadIdx.x; p < p1; p += 4 * kThreads) {
                u32 c[4];
                if (p + 4 <= sL.n_px) {
                    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(keys + p);
                    const ulonglong2 k0 = __ldcs(q), k1 = __ldcs(q + 1);
                    const u64 k[4] = {k0.x, k0.y, k1.x, k1.y};
#pragma unroll
                    for (int j = 0; j < 4; ++j) c[j] = k[j] == ~0ull ? a.background : (u32)k[j];
                    __stcs(reinterpret_cast<uint4*>(out + p), make_uint4(c[0], c[1], c[2], c[3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (p + j < sL.n_px) {
                            const u64 k = keys[p + j];
                            out[p + j] = k == ~0ull ? a.background : (u32)k;
                        }
                    }
                }
            }
        } else {
            const float am = a.a_max_fixed > 0.0f ? a.a_max_fixed : a.a_max[li];
            const float l_max = am > 0.0f ? logf(__fadd_rn(1.0f, am)) : 1.0f;
            const bool planes_ok = sL.kind != CFS_TARGET_HIST_U32 || (sL.n_px & 3u) == 0;
            if (sL.kind == CFS_TARGET_HIST_U32 && sL.C <= 4 && planes_ok) {
                // histograms of up to 4 channels (whole quads: n_px % 4 == 0):
                // the next quad's planes are in flight while this quad maps
                const u32* h = reinterpret_cast<const u32*>(sL.data);
                const int C = sL.C;
                auto load = [&](u32 q, uint4 (&v)[4]) {
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        v[c] = c < C ? __ldcs(reinterpret_cast<const uint4*>(
                                           h + (size_t)c * sL.n_px + q))
                                     : make_uint4(0u, 0u, 0u, 0u);
                };
                uint4 cur[4], nxt[4];
                u32 p = p0 + 4 * threadIdx.x;
                if (p < p1) load(p, cur);
                for (; p < p1; p += 4 * kThreads) {
                    if (p + 4 * kThreads < p1) load(p + 4 * kThreads, nxt);
                    // s = s + n_c * palette[c], channel by channel (as sums4)
                    float4 sq[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) sq[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (c >= C) break;
                        const u32 n[4] = {cur[c].x, cur[c].y, cur[c].z, cur[c].w};
                        const float* pc = sL.pal[c];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float f = (float)n[j];
                            sq[j].x = __fadd_rn(sq[j].x, __fmul_rn(f, pc[0]));
                            sq[j].y = __fadd_rn(sq[j].y, __fmul_rn(f, pc[1]));
                            sq[j].z = __fadd_rn(sq[j].z, __fmul_rn(f, pc[2]));
                            sq[j].w = __fadd_rn(sq[j].w, __fmul_rn(f, pc[3]));
                        }
                    }
                    u32 cq[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) cq[j] = map_pixel(sq[j], l_max, a);
                    __stcs(reinterpret_cast<uint4*>(out + p), make_uint4(cq[0], cq[1], cq[2], cq[3]));
#pragma unroll
                    for (int c = 0; c < 4; ++c) cur[c] = nxt[c];
                }
            } else
            for (u32 p = p0 + 4 * threadIdx.x; p < p1; p += 4 * kThreads) {
                const bool full = p + 4 <= sL.n_px;
                float4 s[4];
                sums4(sL, p, planes_ok && full, true, s);
                u32 c[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) c[j] = map_pixel(s[j], l_max, a);
                if (full) {
                    __stcs(reinterpret_cast<uint4*>(out + p), make_uint4(c[0], c[1], c[2], c[3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (p + j < sL.n_px) out[p + j] = c[j];
                }
            }
        }
        __syncthreads();   // sL is reused by the next item
    }
}

size_t layer_bytes(const cfs_target& t)
{
    const size_t n = (size_t)t.width * (size_t)t.height;
    if (t.kind == CFS_TARGET_HIST_U32) return n * 4 * (size_t)t.channels;
    if (t.kind == CFS_TARGET_RGBA_F32) return n * 16;
    return n * 8;
}
}  // namespace

namespace cfs {

cfs_status display_check(const cfs_target& t, const void* out, const char* what)
{
    std::ostringstream m;
    m << what << ": ";
    if (t.kind < CFS_TARGET_HIST_U32 || t.kind > CFS_TARGET_DEPTH_U64)
        return fail(CFS_ERR_INVALID_ARG, m.str() + "unknown layer kind");
    if (t.width <= 0 || t.height <= 0 || t.width > 65536 || t.height > 65536 ||
        (uint64_t)t.width * (uint64_t)t.height > 0xFFFFFFFFull - kDisplayPxPerItem)
        return fail(CFS_ERR_INVALID_ARG, m.str() + "width/height out of range");
    if (t.kind == CFS_TARGET_HIST_U32 && (t.channels < 1 || t.channels > CFS_MAX_MAPS))
        return fail(CFS_ERR_INVALID_ARG, m.str() + "histogram channels must be in 1..16");
    if (!t.data || ((uintptr_t)t.data) % 16 != 0)
        return fail(CFS_ERR_INVALID_ARG, m.str() + "layer data must be non-NULL, 16-byte aligned");
    if (!out || ((uintptr_t)out) % 16 != 0)
        return fail(CFS_ERR_INVALID_ARG, m.str() + "output must be non-NULL, 16-byte aligned");
    const uintptr_t d0 = (uintptr_t)t.data, d1 = d0 + layer_bytes(t);
    const uintptr_t o0 = (uintptr_t)out, o1 = o0 + 4 * (size_t)t.width * (size_t)t.height;
    if (o0 < d1 && d0 < o1) return fail(CFS_ERR_INVALID_ARG, m.str() + "output overlaps the layer");
    return CFS_OK;
}

uint32_t display_fill(const cfs_target& t, uint32_t* out, uint32_t item_begin, DisplayLayer* d)
{
    std::memset(d, 0, sizeof(*d));
    d->data = (unsigned long long)(uintptr_t)t.data;
    d->out = (unsigned long long)(uintptr_t)out;
    d->n_px = (uint32_t)t.width * (uint32_t)t.height;
    d->kind = t.kind;
    d->C = t.kind == CFS_TARGET_HIST_U32 ? t.channels : 1;
    d->item_begin = item_begin;
    std::memcpy(d->pal, t.palette, sizeof(d->pal));
    return (d->n_px + kDisplayPxPerItem - 1) / kDisplayPxPerItem;
}

cfs_status display_enqueue(const DisplayLayer* one, const DisplayLayer* layers, int n_layers,
                           uint32_t n_items, bool any_density, float* a_max,
                           const cfs_display_params& p, cudaStream_t stream)
{
    if (n_items == 0) return CFS_OK;
    DispArgs a;
    std::memset(&a, 0, sizeof(a));
    if (one) a.one = *one;
    a.layers = layers;
    a.a_max = a_max;
    a.n_layers = n_layers;
    a.n_items = n_items;
    a.inv_gamma = 1.0f / p.gamma;
    a.brightness = p.brightness;
    a.a_max_fixed = p.a_max > 0.0f ? p.a_max : 0.0f;
    a.background = p.background;
    const int sms = device_sm_count();
    const unsigned grid = (unsigned)std::min<uint64_t>(n_items, (uint64_t)std::max(1, sms) * 8);
    if (any_density && !(p.a_max > 0.0f)) {
        cfs_status st = check_cuda(cudaMemsetAsync(a_max, 0, sizeof(float) * (size_t)n_layers,
                                                   stream), "cudaMemsetAsync(a_max)");
        if (st != CFS_OK) return st;
        density_max_kernel<<<grid, kThreads, 0, stream>>>(a);
        st = check_cuda(cudaGetLastError(), "density_max_kernel launch");
        if (st != CFS_OK) return st;
    }
    display_map_kernel<<<grid, kThreads, 0, stream>>>(a);
    return check_cuda(cudaGetLastError(), "display_map_kernel launch");
}

cfs_status display_params_check(const cfs_display_params* p)
{
    if (!p) return fail(CFS_ERR_INVALID_ARG, "params is NULL");
    if (!(std::isfinite(p->gamma) && p->gamma > 0.0f))
        return fail(CFS_ERR_INVALID_ARG, "gamma must be finite and > 0");
    if (!(std::isfinite(p->brightness) && p->brightness > 0.0f))
        return fail(CFS_ERR_INVALID_ARG, "brightness must be finite and > 0");
    if (!std::isfinite(p->a_max)) return fail(CFS_ERR_INVALID_ARG, "a_max must be finite");
    return CFS_OK;
}

}  // namespace cfs

extern "C" cfs_status cfs_tonemap(const cfs_target* layer, const cfs_display_params* params,
                                  uint32_t* rgba8, float* a_max_out, void* stream)
{
    using namespace cfs;
    clear_error();
    if (!layer) return fail(CFS_ERR_INVALID_ARG, "layer is NULL");
    cfs_status st = display_params_check(params);
    if (st != CFS_OK) return st;
    st = display_check(*layer, rgba8, "layer");
    if (st != CFS_OK) return st;
    const bool density = layer->kind != CFS_TARGET_DEPTH_U64;
    if (density && !(params->a_max > 0.0f) &&
        (!a_max_out || ((uintptr_t)a_max_out) % 4 != 0))
        return fail(CFS_ERR_INVALID_ARG, "a_max_out (4-byte aligned) is needed to find the "
                                         "layer's maximum");
    DisplayLayer one;
    const uint32_t items = display_fill(*layer, rgba8, 0, &one);
    return display_enqueue(&one, nullptr, 1, items, density, a_max_out, *params,
                           (cudaStream_t)stream);
}
