// cfs_noalloc.cu -- batched histogram rendering that allocates nothing.
//
// Some callers cannot allocate device memory while they render: a
// real-time or embedded host whose memory budget is fixed after start-up
// (an allocation can fail or stall a frame), or a process whose GPU memory
// is handed out by another allocator that owns the device's free memory.
// cfs_render_batch needs a per-batch workspace (frame descriptors, a work
// counter, discard counters) and gets it with cudaMalloc; this variant keeps
// that workspace in one file-scope device array instead, sized for at most
// CFS_NOALLOC_MAX_FRAMES frames.  The caller still passes every input and
// output (systems, targets).
//
// The array lives as long as the library is loaded, on every GPU that
// loads it, and all calls share it: calls whose GPU work overlaps (two
// streams, or two host threads) race on it.  Everything that must start
// at zero (work counter, discard counters) is cleared on the stream at the
// start of every call.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <mutex>

#include "cfs_device.cuh"
#include "cfs_internal.h"

namespace {

constexpr int kMaxFrames = CFS_NOALLOC_MAX_FRAMES;
constexpr int kBlock = 256;
constexpr uint32_t kChunk = 1024;   // points per work item

struct NaTarget {
    unsigned long long data;
    int W, H, C, pad;
    float x0, x1, y0, y1, sx, sy;
};

struct NaFrame {
    u32 T[16];
    int n_cmp;
    u32 n_points, point_begin, system_id;
    u32 item_begin, pad0, pad1, pad2;
    float prm[6][16];               // a b c d e f of every map, SoA
    NaTarget tg;
};

struct NaScratch {
    NaFrame frames[kMaxFrames];
    unsigned int counter;
    unsigned int pad[63];
    unsigned long long discards[kMaxFrames];
};

// the workspace: one per GPU that loads the library, shared by every call
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

struct NaArgs {
    unsigned int rk[10][2];
    u32 iters, burn_in, n_frames, n_items;
    NaScratch* ws;
};

__global__ void __launch_bounds__(kBlock) noalloc_batch_kernel(const NaArgs a)
{
    __shared__ NaFrame fr;
    __shared__ u32 s_item, s_frame;
    NaScratch* ws = a.ws;
    int cur = -1;
    u32 disc = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const u32 item = atomicAdd(&ws->counter, 1u);
            u32 lo = 0;
            if (item < a.n_items) {
                u32 hi = a.n_frames;
                while (hi - lo > 1) {
                    const u32 mid = (lo + hi) >> 1;
                    if (ws->frames[mid].item_begin <= item) lo = mid; else hi = mid;
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
                const u32 s = __reduce_add_sync(0xffffffffu, disc);
                if ((threadIdx.x & 31) == 0 && s) atomicAdd(&ws->discards[cur], (u64)s);
                disc = 0;
            }
            // whole-struct copy into shared memory, 4 bytes per thread step
            const u32* src = reinterpret_cast<const u32*>(&ws->frames[f]);
            u32* dst = reinterpret_cast<u32*>(&fr);
            for (int e = threadIdx.x; e < (int)(sizeof(NaFrame) / 4); e += blockDim.x)
                dst[e] = src[e];
            __syncthreads();
            cur = f;
        }
        // n_points <= 2^32 - kChunk (checked on the host): no wrap here
        const u32 j0 = (item - fr.item_begin) * kChunk;
        const u32 j1 = min(j0 + kChunk, fr.n_points);
        for (u32 j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const u32 i = fr.point_begin + j, sid = fr.system_id;
            const uint4 r0 = cfs_philox_rk(a.rk, i, 0u, sid, 1u);
            float x = (float)(r0.x >> 8) * CFS_INV_2_24;
            float y = (float)(r0.y >> 8) * CFS_INV_2_24;
            for (u32 nb = 0; (nb << 2) < a.iters; ++nb) {
                const uint4 r = cfs_philox_rk(a.rk, i, nb, sid, 0u);
                const u32 w4[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const u32 n = (nb << 2) + q;
                    if (n >= a.iters) break;
                    int k = 0;
                    for (int t = 0; t < fr.n_cmp; ++t) k += w4[q] >= fr.T[t] ? 1 : 0;
                    const float nx = fmaf(fr.prm[0][k], x, fmaf(fr.prm[1][k], y, fr.prm[4][k]));
                    const float ny = fmaf(fr.prm[2][k], x, fmaf(fr.prm[3][k], y, fr.prm[5][k]));
                    x = nx;
                    y = ny;
                    if (n < a.burn_in) continue;
                    const int ix = cfs_bin(x, fr.tg.x0, fr.tg.x1, fr.tg.sx, fr.tg.W);
                    const int iy = cfs_bin(y, fr.tg.y0, fr.tg.y1, fr.tg.sy, fr.tg.H);
                    if (ix >= 0 && iy >= 0) {
                        u32* base = reinterpret_cast<u32*>(fr.tg.data);
                        const size_t off = ((size_t)(k % fr.tg.C) * (size_t)fr.tg.H + (size_t)iy) *
                                               (size_t)fr.tg.W + (size_t)ix;
                        cfs_red_add_u32(base + off, 1u);
                    } else {
                        disc += 1;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (cur >= 0) {
        const u32 s = __reduce_add_sync(0xffffffffu, disc);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(&ws->discards[cur], (u64)s);
    }
}

// per-device set-up: the device address of the array and the grid size
struct DeviceSetup {
    bool ready = false;
    NaScratch* ws = nullptr;
    int grid = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

cfs_status setup_device(int dev, DeviceSetup** out)
{
    using cfs::check_cuda;
    if (dev < 0 || dev >= kMaxDevices) return cfs::fail(CFS_ERR_UNSUPPORTED, "device index");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        // host code must not use g_noalloc_scratch directly: it is a host
        // stand-in; the device address comes from the runtime
        void* p = nullptr;
        cfs_status st = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                                   "cudaGetSymbolAddress(no-alloc scratch)");
        if (st != CFS_OK) return st;
        int per_sm = 0, sms = 0;
        st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm,
                                                                      noalloc_batch_kernel,
                                                                      kBlock, 0),
                        "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (st != CFS_OK) return st;
        st = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                        "cudaDeviceGetAttribute");
        if (st != CFS_OK) return st;
        s.ws = static_cast<NaScratch*>(p);
        s.grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        s.ready = true;
    }
    *out = &s;
    return CFS_OK;
}

}  // namespace

extern "C" cfs_status cfs_render_batch_noalloc(const cfs_frame* frames, int n_frames,
                                               uint32_t iters, uint32_t burn_in, uint64_t seed,
                                               int clear, unsigned long long* discards,
                                               void* stream_)
{
    using cfs::check_cuda;
    using cfs::fail;
    cfs::clear_error();
    if (!frames || n_frames <= 0) return fail(CFS_ERR_INVALID_ARG, "need at least one frame");
    if (n_frames > kMaxFrames)
        return fail(CFS_ERR_INVALID_ARG,
                    "cfs_render_batch_noalloc takes at most CFS_NOALLOC_MAX_FRAMES (256) frames");
    for (int f = 0; f < n_frames; ++f) {
        const cfs_frame& fr = frames[f];
        const cfs_system* s = fr.system;
        const cfs_target& t = fr.targets[0];
        if (!s || s->dim != 2) return fail(CFS_ERR_INVALID_ARG, "every frame needs a 2D system");
        for (int k = 0; k < s->n_maps; ++k)
            if (s->maps[k].kind != CFS_MAP_AFFINE)
                return fail(CFS_ERR_UNSUPPORTED, "the no-allocation batch renders affine maps");
        if (t.kind != CFS_TARGET_HIST_U32 || !t.data || t.width <= 0 || t.height <= 0 ||
            t.channels < 1 || t.channels > CFS_MAX_MAPS || !(t.x1 > t.x0) || !(t.y1 > t.y0) ||
            t.width > 65536 || t.height > 65536)
            return fail(CFS_ERR_INVALID_ARG, "every frame needs one u32 histogram target");
        if ((uint64_t)fr.point_begin + fr.n_points > (1ull << 32))
            return fail(CFS_ERR_INVALID_ARG, "point indices exceed 2^32");
        if ((uint64_t)fr.n_points > (1ull << 32) - kChunk)
            return fail(CFS_ERR_INVALID_ARG, "a frame may hold at most 2^32 - 1024 points");
        if (fr.start)
            return fail(CFS_ERR_UNSUPPORTED,
                        "the no-allocation batch starts every point from Philox");
    }
    int dev = 0;
    cfs_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != CFS_OK) return st;
    DeviceSetup* ds = nullptr;
    st = setup_device(dev, &ds);
    if (st != CFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream_;
    if (burn_in > iters) burn_in = iters;

    // work items, counted in 64 bits: the persistent CTAs draw item numbers
    // from a 32-bit counter that runs up to n_items + grid
    uint64_t n_items = 0;
    for (int f = 0; f < n_frames; ++f) n_items += ((uint64_t)frames[f].n_points + kChunk - 1) / kChunk;
    if (n_items + (uint64_t)ds->grid >= (1ull << 32))
        return fail(CFS_ERR_INVALID_ARG, "too many points in one call");

    // frame descriptors go up one at a time from a stack buffer: a copy
    // from pageable memory has read its source when cudaMemcpyAsync returns
    uint32_t item = 0;
    for (int f = 0; f < n_frames; ++f) {
        const cfs_frame& fr = frames[f];
        const cfs_system& sy = *fr.system;
        const cfs_target& t = fr.targets[0];
        NaFrame d;
        std::memset(&d, 0, sizeof(d));
        for (int j = 0; j < sy.n_cmp; ++j) d.T[j] = sy.T[j];
        d.n_cmp = sy.n_cmp;
        d.n_points = fr.n_points;
        d.point_begin = fr.point_begin;
        d.system_id = fr.system_id;
        d.item_begin = item;
        for (int k = 0; k < sy.n_maps; ++k)
            for (int j = 0; j < 6; ++j) d.prm[j][k] = sy.maps[k].params[j];
        d.tg.data = (unsigned long long)(uintptr_t)t.data;
        d.tg.W = t.width;
        d.tg.H = t.height;
        d.tg.C = t.channels;
        d.tg.x0 = t.x0; d.tg.x1 = t.x1; d.tg.y0 = t.y0; d.tg.y1 = t.y1;
        d.tg.sx = (float)t.width / (t.x1 - t.x0);
        d.tg.sy = (float)t.height / (t.y1 - t.y0);
        st = check_cuda(cudaMemcpyAsync(&ds->ws->frames[f], &d, sizeof(d),
                                        cudaMemcpyHostToDevice, s),
                        "cudaMemcpyAsync(frame)");
        if (st != CFS_OK) return st;
        item += (uint32_t)(((uint64_t)fr.n_points + kChunk - 1) / kChunk);
        if (clear) {
            st = check_cuda(cudaMemsetAsync(t.data, 0,
                                            (size_t)t.width * t.height * 4 * (size_t)t.channels,
                                            s),
                            "cudaMemsetAsync(target)");
            if (st != CFS_OK) return st;
        }
    }
    // the work counter and the discard counters start at zero every call
    st = check_cuda(cudaMemsetAsync(&ds->ws->counter, 0,
                                    sizeof(NaScratch) - offsetof(NaScratch, counter), s),
                    "cudaMemsetAsync(counters)");
    if (st != CFS_OK) return st;
    if (item > 0) {
        NaArgs a;
        cfs::philox_round_keys(seed, a.rk);
        a.iters = iters;
        a.burn_in = burn_in;
        a.n_frames = (u32)n_frames;
        a.n_items = item;
        a.ws = ds->ws;
        const unsigned grid = (unsigned)(ds->grid < (int)item ? ds->grid : (int)item);
        noalloc_batch_kernel<<<grid, kBlock, 0, s>>>(a);
        st = check_cuda(cudaGetLastError(), "noalloc_batch_kernel launch");
        if (st != CFS_OK) return st;
    }
    if (discards)
        st = check_cuda(cudaMemcpyAsync(discards, ds->ws->discards,
                                        sizeof(unsigned long long) * (size_t)n_frames,
                                        cudaMemcpyDeviceToDevice, s),
                        "cudaMemcpyAsync(discards)");
    return st;
}
