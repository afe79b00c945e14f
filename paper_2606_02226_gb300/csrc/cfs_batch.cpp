// cfs_batch.cpp -- batched rendering of many frames in one persistent launch
// (animation frames and in-betweens of different systems; the paper's
// smear-frame / in-between application, Section 4).
//
// A batch is planned once on the host: frame descriptors (thresholds, map
// tables, target geometry, point ranges) are packed into a pinned staging
// buffer, the work is cut into items of `chunk` points numbered frame by
// frame, and the whole frame -- descriptor upload, counter reset, optional
// clears of every frame's targets, the persistent kernel -- is captured into
// a CUDA graph that each cfs_batch_launch replays on the caller's stream.
#include <algorithm>
#include <cstring>
#include <new>
#include <sstream>
#include <vector>

#include "cfs_internal.h"

namespace cfs {
void fill_args_common(cfs_launch_args* a, const cfs_chain* ch, uint64_t seed, uint32_t iters,
                      uint32_t burn_in);
cfs_status validate_targets_ext(const cfs_chain* ch, const cfs_target* tg, int n_tg);
}  // namespace cfs

struct cfs_batch {
    int device = 0;
    int n_frames = 0;
    int n_targets = 0;
    cfs_chain chain;
    uint32_t iters = 0, burn_in = 0;
    uint64_t seed = 0;
    std::vector<cfs_frame> frames;        // host copy (targets by value)
    std::vector<cfs_system> systems;      // host copies
    std::vector<uint32_t> chunks;         // points per item, per frame
    cfs::ProgramSpec spec;
    cfs::Kernel kernel;
    cfs::Kernel bbox_kernel;              // pre-pass of the privatized window
    uint32_t tile_cap = 0;
    cfs_launch_args args;
    uint32_t chunk = 0, n_items = 0, grid = 0;
    cfs_dev_frame* h_frames = nullptr;    // pinned staging
    unsigned char* d_work = nullptr;      // frames | counter | discards
    cfs_dev_frame* d_frames = nullptr;
    unsigned int* d_counter = nullptr;
    unsigned long long* d_disc = nullptr;
    int* d_bbox = nullptr;
    size_t work_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // [clear]
    cudaEvent_t done = nullptr;
    bool launched = false;
    // display (cfs_batch_display): layer descriptions staged in pinned memory
    cfs::DisplayLayer* h_disp = nullptr;
    unsigned char* d_disp = nullptr;      // DisplayLayer [n_frames] | float a_max [n_frames]
    cudaEvent_t disp_done = nullptr;
    bool disp_launched = false;
};

namespace {
using namespace cfs;

void pack_frame(cfs_dev_frame* d, const cfs_system& s, const cfs_frame& f, int n_targets,
                uint32_t item_begin, uint32_t chunk)
{
    std::memset(d, 0, sizeof(*d));
    for (int j = 0; j < s.n_cmp; ++j) d->T[j] = s.T[j];
    d->n_maps = s.n_maps;
    d->n_cmp = s.n_cmp;
    d->dim = s.dim;
    for (int k = 0; k < s.n_maps; ++k)
        for (int j = 0; j < 12; ++j) d->prm[j][k] = s.maps[k].params[j];
    d->n_points = f.n_points;
    d->point_begin = f.point_begin;
    d->system_id = f.system_id;
    d->item_begin = item_begin;
    d->chunk = chunk;
    d->start = (unsigned long long)(uintptr_t)f.start;
    d->start_count = f.start_count ? f.start_count : f.n_points;
    for (int t = 0; t < n_targets; ++t) {
        const cfs_target& g = f.targets[t];
        cfs_dev_target& o = d->tg[t];
        o.data = (unsigned long long)(uintptr_t)g.data;
        o.W = g.width;
        o.H = g.height;
        o.C = g.channels < 1 ? 1 : g.channels;
        o.kind = g.kind;
        o.x0 = g.x0; o.x1 = g.x1; o.y0 = g.y0; o.y1 = g.y1;
        o.sx = (float)g.width / (g.x1 - g.x0);
        o.sy = (float)g.height / (g.y1 - g.y0);
        std::memcpy(o.palette, g.palette, sizeof(o.palette));
        std::memcpy(o.palette8, g.palette8, sizeof(o.palette8));
    }
}

size_t target_bytes(const cfs_target& g)
{
    size_t n = (size_t)g.width * (size_t)g.height;
    if (g.kind == CFS_TARGET_HIST_U32) return n * 4 * (size_t)(g.channels < 1 ? 1 : g.channels);
    if (g.kind == CFS_TARGET_RGBA_F32) return n * 16;
    return n * 8;
}

void release(cfs_batch* b)
{
    for (auto& e : b->exec)
        if (e) cudaGraphExecDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->d_work) cudaFree(b->d_work);
    if (b->h_frames) cudaFreeHost(b->h_frames);
    if (b->disp_done) cudaEventDestroy(b->disp_done);
    if (b->d_disp) cudaFree(b->d_disp);
    if (b->h_disp) cudaFreeHost(b->h_disp);
}

cfs_status capture(cfs_batch* b, int clear)
{
    cudaStream_t s = b->cap_stream;
    cfs_status st = check_cuda(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal),
                               "cudaStreamBeginCapture");
    if (st != CFS_OK) return st;
    cudaError_t e = cudaMemcpyAsync(b->d_frames, b->h_frames,
                                    sizeof(cfs_dev_frame) * (size_t)b->n_frames,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_counter, 0,
                            b->work_bytes - ((unsigned char*)b->d_counter - b->d_work), s);
    if (e == cudaSuccess && clear) {
        for (int f = 0; f < b->n_frames && e == cudaSuccess; ++f)
            for (int t = 0; t < b->n_targets && e == cudaSuccess; ++t) {
                const cfs_target& g = b->frames[f].targets[t];
                e = cudaMemsetAsync(g.data, g.kind == CFS_TARGET_DEPTH_U64 ? 0xFF : 0,
                                    target_bytes(g), s);
            }
    }
    cfs_status lst = CFS_OK;
    if (e == cudaSuccess && b->n_items > 0 && b->spec.tile)
        lst = launch(b->bbox_kernel, (unsigned)b->n_frames, &b->args, sizeof(b->args), s);
    if (e == cudaSuccess && lst == CFS_OK && b->n_items > 0)
        lst = launch(b->kernel, b->grid, &b->args, sizeof(b->args), s);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return check_cuda(e, "batch capture");
    }
    if (lst != CFS_OK) {
        if (g) cudaGraphDestroy(g);
        return lst;
    }
    st = check_cuda(e2, "cudaStreamEndCapture");
    if (st != CFS_OK) return st;
    st = check_cuda(cudaGraphInstantiate(&b->exec[clear], g, 0), "cudaGraphInstantiate");
    cudaGraphDestroy(g);
    return st;
}
}  // namespace

namespace cfs {
// Launch shape of the persistent batch program (also used by the compile-only
// check); returns the privatized window's capacity in u32 counters.
uint32_t batch_spec_defaults(ProgramSpec& sp)
{
    // measured on GB300: one 1024-thread CTA per SM sharing a ~208 KB
    // privatized window beats smaller CTAs with smaller windows (the flush
    // volume and the global-atomic share both shrink)
    sp.block = 1024;
    if (const char* e = std::getenv("CFS_BATCH_BLOCK")) {
        const int v = std::atoi(e);
        if (v == 128 || v == 256 || v == 512 || v == 1024) sp.block = v;
    }
    sp.min_blocks = std::max(1, 2048 / sp.block);
    sp.spill_allowance = 64;
    sp.depth_test = 1;
    // privatized window: when the chain splats once, into a histogram
    sp.tile = (sp.splats.size() == 1 && sp.splats[0].kind == CFS_TARGET_HIST_U32) ? 1 : 0;
    // warp-level aggregation of equal window addresses (match.any) measured
    // slower than plain shared atomics on the animation batch: off
    sp.warp_agg = 0;
    uint32_t tile_cap = sp.block >= 1024 ? 53248 : 8192;
    if (const char* e = std::getenv("CFS_TILE")) sp.tile = sp.tile && std::atoi(e) != 0;
    if (const char* e = std::getenv("CFS_WARP_AGG")) sp.warp_agg = std::atoi(e) != 0;
    // copies of small windows (one per warp) measured slower on the animation
    // batch (the flush grows with the copies); kept as a knob
    sp.tile_reps = 1;
    if (const char* e = std::getenv("CFS_TILE_REPS")) sp.tile_reps = std::max(1, std::atoi(e));
    // two trajectories per thread: 755 vs 764 ms for the 256-frame batch
    sp.ilp = 2;
    if (const char* e = std::getenv("CFS_BATCH_ILP")) sp.ilp = std::atoi(e) == 2 ? 2 : 1;
    if (const char* e = std::getenv("CFS_TILE_CAP")) {
        const int c = std::atoi(e);
        if (c >= 256 && c <= 53248) tile_cap = (uint32_t)c;
    }
    if (!sp.tile) { sp.warp_agg = 0; tile_cap = 0; }
    sp.dyn_smem = (int)(tile_cap * sizeof(uint32_t));
    // a window above half of the SM's shared memory leaves room for one CTA
    // per SM: asking for two would only cap the registers (and spill)
    if (sp.dyn_smem > 112 * 1024) sp.min_blocks = 1;
    if (const char* e = std::getenv("CFS_BATCH_MINB")) sp.min_blocks = std::max(1, std::atoi(e));
    return tile_cap;
}
}  // namespace cfs

namespace {
// Cuts every frame into items of `chunk` points (whole warps), numbers the
// items frame by frame, repacks the staged frame descriptors and sets the
// persistent grid (resident CTAs, at most one per item).
cfs_status plan_items(cfs_batch* b, uint32_t chunk)
{
    b->chunk = chunk;
    b->grid = (uint32_t)std::max(1, b->kernel.max_blocks_per_sm * std::max(1, b->kernel.num_sms));
    uint64_t total = 0;
    b->chunks.assign(b->n_frames, chunk);
    for (int f = 0; f < b->n_frames; ++f)
        total += ((uint64_t)b->frames[f].n_points + chunk - 1) / chunk;
    if (total >= (1ull << 31)) return fail(CFS_ERR_INVALID_ARG, "too many work items");
    b->n_items = (uint32_t)total;
    if (b->grid > b->n_items && b->n_items > 0) b->grid = b->n_items;
    if (b->h_frames) {
        uint32_t item = 0;
        for (int f = 0; f < b->n_frames; ++f) {
            pack_frame(&b->h_frames[f], b->systems[f], b->frames[f], b->n_targets, item, chunk);
            item += (b->frames[f].n_points + chunk - 1) / chunk;
        }
    }
    b->args.n_items = b->n_items;
    b->args.chunk = chunk;
    return CFS_OK;
}

// Compiles the batch program (and the window pre-pass when tiled) for the
// spec's current knobs.
cfs_status build_program(cfs_batch* b)
{
    cfs_status st = get_kernel(b->spec, "cfs_batch_kernel", &b->kernel);
    if (st != CFS_OK) return st;
    if (b->spec.tile) {
        ProgramSpec bs = b->spec;
        bs.dyn_smem = 0;
        st = get_kernel(bs, "cfs_bbox_kernel", &b->bbox_kernel);
    }
    b->args.tile_cap = b->tile_cap;
    return st;
}

void drop_graphs(cfs_batch* b)
{
    for (auto& e : b->exec)
        if (e) { cudaGraphExecDestroy(e); e = nullptr; }
}

// the launch sequence of a batch without a graph (the autotuner's trials)
cfs_status run_direct(cfs_batch* b, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    cudaError_t e = cudaMemcpyAsync(b->d_frames, b->h_frames,
                                    sizeof(cfs_dev_frame) * (size_t)b->n_frames,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_counter, 0,
                            b->work_bytes - ((unsigned char*)b->d_counter - b->d_work), s);
    for (int f = 0; f < b->n_frames && e == cudaSuccess; ++f)
        for (int t = 0; t < b->n_targets && e == cudaSuccess; ++t) {
            const cfs_target& g = b->frames[f].targets[t];
            e = cudaMemsetAsync(g.data, g.kind == CFS_TARGET_DEPTH_U64 ? 0xFF : 0,
                                target_bytes(g), s);
        }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    cfs_status st = check_cuda(e, "batch trial set-up");
    if (st == CFS_OK && b->n_items > 0 && b->spec.tile)
        st = launch(b->bbox_kernel, (unsigned)b->n_frames, &b->args, sizeof(b->args), s);
    if (st == CFS_OK && b->n_items > 0)
        st = launch(b->kernel, b->grid, &b->args, sizeof(b->args), s);
    if (st == CFS_OK) st = check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
    return st;
}
}  // namespace

extern "C" {

cfs_status cfs_batch_create(const cfs_chain* chain, int n_targets, const cfs_frame* frames,
                            int n_frames, uint32_t step_begin, uint32_t iters, uint32_t burn_in,
                            uint64_t seed, cfs_batch** out)
{
    clear_error();
    if (!out) return fail(CFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!chain || !frames || n_frames <= 0)
        return fail(CFS_ERR_INVALID_ARG, "need a chain and at least one frame");
    if (n_targets < 0 || n_targets > CFS_MAX_TARGETS)
        return fail(CFS_ERR_INVALID_ARG, "n_targets must be in 0..4");
    const cfs_system* s0 = frames[0].system;
    if (!s0) return fail(CFS_ERR_INVALID_ARG, "frame 0 has no system");
    int max_cmp = 0;
    for (int f = 0; f < n_frames; ++f) {
        const cfs_frame& fr = frames[f];
        std::ostringstream m;
        m << "frame " << f << ": ";
        if (!fr.system) return fail(CFS_ERR_INVALID_ARG, m.str() + "no system");
        if (fr.system->dim != chain->dim_in)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "system dimension differs from the chain's");
        for (int k = 0; k < fr.system->n_maps; ++k)
            if (fr.system->maps[k].kind != s0->maps[0].kind)
                return fail(CFS_ERR_UNSUPPORTED,
                            m.str() + "a batch needs maps of one kind in every frame");
        if ((uint64_t)fr.point_begin + fr.n_points > (1ull << 32))
            return fail(CFS_ERR_INVALID_ARG, m.str() + "point indices exceed 2^32");
        cfs_status st = validate_targets_ext(chain, fr.targets, n_targets);
        if (st != CFS_OK) return fail(st, m.str() + cfs_last_error());
        if (fr.start && fr.start_count > fr.n_points)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "start_count exceeds n_points");
        for (int t = 0; t < n_targets; ++t)
            if (fr.targets[t].kind != frames[0].targets[t].kind ||
                (fr.targets[t].kind == CFS_TARGET_HIST_U32 &&
                 fr.targets[t].channels != frames[0].targets[t].channels))
                return fail(CFS_ERR_INVALID_ARG, m.str() + "target kinds differ between frames");
        max_cmp = std::max(max_cmp, fr.system->n_cmp);
    }
    if (burn_in > iters) burn_in = iters;
    if (step_begin > iters) return fail(CFS_ERR_INVALID_ARG, "step_begin > iters");

    cfs_batch* b = new (std::nothrow) cfs_batch();
    if (!b) return fail(CFS_ERR_OOM, "host allocation failed");
    cfs_status st = check_cuda(cudaGetDevice(&b->device), "cudaGetDevice");
    if (st != CFS_OK) { delete b; return st; }
    b->n_frames = n_frames;
    b->n_targets = n_targets;
    b->chain = *chain;
    b->iters = iters;
    b->burn_in = burn_in;
    b->seed = seed;
    b->frames.assign(frames, frames + n_frames);
    b->systems.resize(n_frames);
    for (int f = 0; f < n_frames; ++f) b->systems[f] = *frames[f].system;

    // program: table-driven generator, thresholds from shared memory
    ProgramSpec& sp = b->spec;
    sp.mode = Mode::Batch;
    sp.dim = s0->dim;
    sp.n_maps = CFS_MAX_MAPS;
    for (int j = 0; j < CFS_MAX_MAPS; ++j) sp.map_kind[j] = s0->maps[0].kind;
    sp.n_cmp = max_cmp;
    sp.n_ops = chain->n_ops;
    sp.n_targets = n_targets;
    sp.fast_trig = trig_mode(chain->flags);
    for (int o = 0; o < chain->n_ops; ++o) {
        sp.op_kind[o] = chain->ops[o].kind;
        if (chain->ops[o].kind == CFS_OP_ROTATE3) sp.op_axis[o] = (int)chain->ops[o].params[1];
        if (chain->ops[o].kind == CFS_OP_BANDS) sp.op_axis[o] = (int)chain->ops[o].params[0];
        if (chain->ops[o].kind == CFS_OP_SPLAT) {
            const int slot = (int)chain->ops[o].params[0];
            SplatSpec ss;
            ss.slot = slot;
            ss.kind = frames[0].targets[slot].kind;
            ss.channels = ss.kind == CFS_TARGET_HIST_U32 ? frames[0].targets[slot].channels : 1;
            sp.splats.push_back(ss);
        }
    }
    sp.scribble = chain->scribble;
    for (int slot : chain->scribble_slots) {
        SplatSpec ss;
        ss.slot = slot;
        ss.kind = frames[0].targets[slot].kind;
        ss.channels = ss.kind == CFS_TARGET_HIST_U32 ? frames[0].targets[slot].channels : 1;
        sp.splats.push_back(ss);
    }
    b->tile_cap = batch_spec_defaults(sp);
    if (!sp.scribble.empty() && sp.tile) {
        // the privatized window needs the splat's code shape of an op chain
        sp.tile = 0;
        sp.warp_agg = 0;
        b->tile_cap = 0;
        sp.dyn_smem = 0;
    }
    st = build_program(b);
    if (st != CFS_OK) { delete b; return st; }

    // Items: every frame is cut into items of `chunk` points (whole warps);
    // all CTAs work on one or two frames at a time, so the live layers stay
    // in L2.  cfs_batch_tune picks the chunk (and the program's knobs) by
    // measurement.
    uint32_t chunk = 4096;
    if (const char* e = std::getenv("CFS_BATCH_CHUNK")) {
        const int c = std::atoi(e);
        if (c >= 32 && c % 32 == 0) chunk = (uint32_t)c;
    }
    st = plan_items(b, chunk);
    if (st != CFS_OK) { delete b; return st; }

    // workspace: frames | bbox (int4 per frame) | counter (u32, padded to
    // 256 B) | discards (the counter and discards are reset every launch)
    const size_t fbytes = sizeof(cfs_dev_frame) * (size_t)n_frames;
    const size_t off_bbox = (fbytes + 255) & ~(size_t)255;
    const size_t off_counter = (off_bbox + 16 * (size_t)n_frames + 255) & ~(size_t)255;
    const size_t off_disc = off_counter + 256;
    b->work_bytes = off_disc + sizeof(unsigned long long) * (size_t)n_frames *
                                   (size_t)std::max(1, n_targets);
    st = check_cuda(cudaMalloc(&b->d_work, b->work_bytes), "cudaMalloc(batch workspace)");
    if (st == CFS_OK)
        st = check_cuda(cudaMallocHost(&b->h_frames, fbytes), "cudaMallocHost(batch frames)");
    if (st == CFS_OK)
        st = check_cuda(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking),
                        "cudaStreamCreate");
    if (st == CFS_OK)
        st = check_cuda(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming),
                        "cudaEventCreate");
    if (st != CFS_OK) { release(b); delete b; return st; }
    b->d_frames = reinterpret_cast<cfs_dev_frame*>(b->d_work);
    b->d_bbox = reinterpret_cast<int*>(b->d_work + off_bbox);
    b->d_counter = reinterpret_cast<unsigned int*>(b->d_work + off_counter);
    b->d_disc = reinterpret_cast<unsigned long long*>(b->d_work + off_disc);

    fill_args_common(&b->args, chain, seed, iters, burn_in);
    st = plan_items(b, b->chunk);        // now that the staging buffer exists
    if (st != CFS_OK) { release(b); delete b; return st; }
    b->args.step_begin = step_begin;
    b->args.frames = (unsigned long long)(uintptr_t)b->d_frames;
    b->args.work_counter = (unsigned long long)(uintptr_t)b->d_counter;
    b->args.frame_discards = (unsigned long long)(uintptr_t)b->d_disc;
    b->args.n_frames = (unsigned)n_frames;
    b->args.frame_bbox = (unsigned long long)(uintptr_t)b->d_bbox;
    b->args.tile_cap = b->tile_cap;
    *out = b;
    return CFS_OK;
}

cfs_status cfs_batch_set_system(cfs_batch* b, int frame, const cfs_system* sys)
{
    clear_error();
    if (!b || !sys) return fail(CFS_ERR_INVALID_ARG, "NULL batch or system");
    if (frame < 0 || frame >= b->n_frames) return fail(CFS_ERR_INVALID_ARG, "frame out of range");
    if (sys->dim != b->chain.dim_in || sys->n_cmp > b->spec.n_cmp)
        return fail(CFS_ERR_INVALID_ARG, "system does not fit the batch's program "
                                         "(dimension or more maps than planned)");
    for (int k = 0; k < sys->n_maps; ++k)
        if (sys->maps[k].kind != b->spec.map_kind[0])
            return fail(CFS_ERR_UNSUPPORTED, "a batch needs maps of one kind");
    // the staging buffer is read by the previous launch's upload: wait for it
    if (b->launched) {
        cfs_status st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
        if (st != CFS_OK) return st;
    }
    b->systems[frame] = *sys;
    const uint32_t item_begin = b->h_frames[frame].item_begin;
    pack_frame(&b->h_frames[frame], b->systems[frame], b->frames[frame], b->n_targets, item_begin,
               b->chunks[frame]);
    return CFS_OK;
}

cfs_status cfs_batch_launch(cfs_batch* b, int clear, void* stream)
{
    clear_error();
    if (!b) return fail(CFS_ERR_INVALID_ARG, "NULL batch");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(CFS_ERR_INVALID_ARG, "batch belongs to another device");
    clear = clear ? 1 : 0;
    if (!b->exec[clear]) {
        cfs_status st = capture(b, clear);
        if (st != CFS_OK) return st;
    }
    cfs_status st = check_cuda(cudaGraphLaunch(b->exec[clear], (cudaStream_t)stream),
                               "cudaGraphLaunch");
    if (st != CFS_OK) return st;
    b->launched = true;
    return check_cuda(cudaEventRecord(b->done, (cudaStream_t)stream), "cudaEventRecord");
}

cfs_status cfs_batch_discards(cfs_batch* b, uint64_t* out)
{
    clear_error();
    if (!b || !out) return fail(CFS_ERR_INVALID_ARG, "NULL batch or out");
    if (b->launched) {
        cfs_status st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
        if (st != CFS_OK) return st;
    }
    return check_cuda(cudaMemcpy(out, b->d_disc,
                                 sizeof(uint64_t) * (size_t)b->n_frames *
                                     (size_t)std::max(1, b->n_targets),
                                 cudaMemcpyDeviceToHost),
                      "cudaMemcpy(discards)");
}

cfs_status cfs_batch_info(const cfs_batch* b, uint32_t* n_items, uint32_t* chunk, uint32_t* grid)
{
    clear_error();
    if (!b) return fail(CFS_ERR_INVALID_ARG, "NULL batch");
    if (n_items) *n_items = b->n_items;
    if (chunk) *chunk = b->chunk;
    if (grid) *grid = b->grid;
    return CFS_OK;
}

cfs_status cfs_batch_display(cfs_batch* b, int slot, const cfs_display_params* params,
                             uint32_t* const* outs, float* a_max_out, void* stream)
{
    clear_error();
    if (!b || !outs) return fail(CFS_ERR_INVALID_ARG, "NULL batch or outs");
    cfs_status st = display_params_check(params);
    if (st != CFS_OK) return st;
    if (slot < 0 || slot >= b->n_targets)
        return fail(CFS_ERR_INVALID_ARG, "slot names no target of the batch");
    if (a_max_out && ((uintptr_t)a_max_out) % 4 != 0)
        return fail(CFS_ERR_INVALID_ARG, "a_max_out must be 4-byte aligned");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(CFS_ERR_INVALID_ARG, "batch belongs to another device");
    for (int f = 0; f < b->n_frames; ++f) {
        std::ostringstream m;
        m << "frame " << f;
        st = display_check(b->frames[f].targets[slot], outs[f], m.str().c_str());
        if (st != CFS_OK) return st;
    }
    const size_t lbytes = sizeof(DisplayLayer) * (size_t)b->n_frames;
    const size_t off_amax = (lbytes + 255) & ~(size_t)255;
    if (!b->d_disp) {
        st = check_cuda(cudaMalloc(&b->d_disp, off_amax + sizeof(float) * (size_t)b->n_frames),
                        "cudaMalloc(display workspace)");
        if (st == CFS_OK)
            st = check_cuda(cudaMallocHost(&b->h_disp, lbytes), "cudaMallocHost(display)");
        if (st == CFS_OK)
            st = check_cuda(cudaEventCreateWithFlags(&b->disp_done, cudaEventDisableTiming),
                            "cudaEventCreate");
        if (st != CFS_OK) return st;
    }
    // the staging buffer is read by the previous display's upload: wait for it
    if (b->disp_launched) {
        st = check_cuda(cudaEventSynchronize(b->disp_done), "cudaEventSynchronize");
        if (st != CFS_OK) return st;
    }
    uint64_t items = 0;
    bool density = false;
    for (int f = 0; f < b->n_frames; ++f) {
        const cfs_target& t = b->frames[f].targets[slot];
        items += display_fill(t, outs[f], (uint32_t)items, &b->h_disp[f]);
        if (items >= (1ull << 31)) return fail(CFS_ERR_INVALID_ARG, "too many pixels");
        density = density || t.kind != CFS_TARGET_DEPTH_U64;
    }
    DisplayLayer* d_layers = reinterpret_cast<DisplayLayer*>(b->d_disp);
    float* amax = a_max_out ? a_max_out : reinterpret_cast<float*>(b->d_disp + off_amax);
    st = check_cuda(cudaMemcpyAsync(d_layers, b->h_disp, lbytes, cudaMemcpyHostToDevice,
                                    (cudaStream_t)stream),
                    "cudaMemcpyAsync(display layers)");
    if (st != CFS_OK) return st;
    st = display_enqueue(nullptr, d_layers, b->n_frames, (uint32_t)items, density, amax, *params,
                         (cudaStream_t)stream);
    if (st != CFS_OK) return st;
    b->disp_launched = true;
    return check_cuda(cudaEventRecord(b->disp_done, (cudaStream_t)stream), "cudaEventRecord");
}

cfs_status cfs_batch_tune(cfs_batch* b, uint32_t trial_iters, void* stream,
                          cfs_batch_tuning* out)
{
    clear_error();
    if (!b) return fail(CFS_ERR_INVALID_ARG, "NULL batch");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(CFS_ERR_INVALID_ARG, "batch belongs to another device");
    cudaStream_t s = (cudaStream_t)stream;
    cfs_status st = CFS_OK;
    if (b->launched) st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    if (b->disp_launched && st == CFS_OK)
        st = check_cuda(cudaEventSynchronize(b->disp_done), "cudaEventSynchronize");
    if (st != CFS_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    st = check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    if (st == CFS_OK) st = check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    if (st != CFS_OK) {
        if (e0) cudaEventDestroy(e0);
        return st;
    }
    // trials run the first trial_iters steps (the whole run when 0)
    const uint32_t full_iters = b->args.iters;
    if (trial_iters > 0)
        b->args.iters = std::min(full_iters, b->args.step_begin + std::max(trial_iters, 1u));
    const ProgramSpec base = b->spec;
    const bool tile_ok = base.scribble.empty() && base.splats.size() == 1 &&
                         base.splats[0].kind == CFS_TARGET_HIST_U32;
    const uint32_t base_cap = b->tile_cap ? b->tile_cap : (base.block >= 1024 ? 53248u : 8192u);
    struct Cand { int ilp, tile; uint32_t chunk; float ms; };
    std::vector<Cand> tried;
    Cand best{base.ilp, base.tile, b->chunk, 1e30f};
    const uint32_t chunks[] = {2048, 4096, 8192, 16384};
    for (int tile = tile_ok ? 1 : 0; tile >= 0 && st == CFS_OK; --tile) {
        for (int ilp = 1; ilp <= 2 && st == CFS_OK; ++ilp) {
            b->spec = base;
            b->spec.ilp = ilp;
            b->spec.tile = tile;
            b->spec.warp_agg = 0;
            b->tile_cap = tile ? base_cap : 0;
            b->spec.dyn_smem = (int)(b->tile_cap * sizeof(uint32_t));
            st = build_program(b);
            for (uint32_t c : chunks) {
                if (st != CFS_OK) break;
                st = plan_items(b, c);
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && st == CFS_OK; ++rep) {
                    st = run_direct(b, s, e0, e1);
                    if (st == CFS_OK) st = check_cuda(cudaEventSynchronize(e1), "trial");
                    float t = 0.0f;
                    if (st == CFS_OK) st = check_cuda(cudaEventElapsedTime(&t, e0, e1), "time");
                    ms = std::min(ms, t);
                }
                if (st != CFS_OK) break;
                tried.push_back({ilp, tile, c, ms});
                if (ms < best.ms) best = {ilp, tile, c, ms};
            }
        }
    }
    // keep the winner (or restore the starting point after an error)
    b->spec = base;
    if (st == CFS_OK) {
        b->spec.ilp = best.ilp;
        b->spec.tile = best.tile;
        b->spec.warp_agg = 0;
        b->tile_cap = best.tile ? base_cap : 0;
        b->spec.dyn_smem = (int)(b->tile_cap * sizeof(uint32_t));
    } else {
        b->tile_cap = base.tile ? base_cap : 0;
    }
    cfs_status st2 = build_program(b);
    if (st2 == CFS_OK) st2 = plan_items(b, st == CFS_OK ? best.chunk : 4096u);
    b->args.iters = full_iters;
    drop_graphs(b);                     // the next launch captures the new plan
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CFS_OK) return st;
    if (st2 != CFS_OK) return st2;
    if (out) {
        out->ilp = best.ilp;
        out->tile = best.tile;
        out->chunk = best.chunk;
        out->trial_ms = best.ms;
        out->trials = (int)tried.size();
    }
    return CFS_OK;
}

cfs_status cfs_batch_destroy(cfs_batch* b)
{
    if (!b) return CFS_OK;
    if (b->launched) cudaEventSynchronize(b->done);
    if (b->disp_launched) cudaEventSynchronize(b->disp_done);
    release(b);
    delete b;
    return CFS_OK;
}

cfs_status cfs_render_batch(const cfs_chain* chain, int n_targets, const cfs_frame* frames,
                            int n_frames, uint32_t step_begin, uint32_t iters, uint32_t burn_in,
                            uint64_t seed, int clear, void* stream)
{
    cfs_batch* b = nullptr;
    cfs_status st = cfs_batch_create(chain, n_targets, frames, n_frames, step_begin, iters,
                                     burn_in, seed, &b);
    if (st != CFS_OK) return st;
    st = cfs_batch_launch(b, clear, stream);
    cfs_batch_destroy(b);   // waits for the launch: the workspace must outlive it
    return st;
}

}  // extern "C"
