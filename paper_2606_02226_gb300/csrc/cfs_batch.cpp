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
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
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
    std::vector<uint8_t> nowin;           // per frame: skip the privatized window
    cfs_batch_plan plan;                  // program knobs and default item size
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
    // the window set-up of the last launch or trial (cfs_batch_windows)
    bool last_tile = false;
    uint32_t last_tile_cap = 0;
    std::vector<uint8_t> last_nowin;
    // display (cfs_batch_display): layer descriptions staged in pinned memory
    cfs::DisplayLayer* h_disp = nullptr;
    unsigned char* d_disp = nullptr;      // DisplayLayer [n_frames] | float a_max [n_frames]
    cudaEvent_t disp_done = nullptr;
    bool disp_launched = false;
};

namespace {
using namespace cfs;

void pack_frame(cfs_dev_frame* d, const cfs_system& s, const cfs_frame& f, int n_targets,
                uint32_t item_begin, uint32_t chunk, bool nowin)
{
    std::memset(d, 0, sizeof(*d));
    for (int j = 0; j < s.n_cmp; ++j) d->T[j] = s.T[j];
    d->n_maps = s.n_maps;
    d->n_cmp = s.n_cmp;
    d->dim = s.dim;
    d->flags = nowin ? CFS_FRAME_NO_WINDOW : 0;
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
// check): the default plan's program knobs; returns the privatized window's
// capacity in u32 counters (0 when the chain cannot use one).
uint32_t batch_spec_defaults(ProgramSpec& sp)
{
    // measured on GB300: one 1024-thread CTA per SM sharing a ~208 KB
    // privatized window beats smaller CTAs with smaller windows (the flush
    // volume and the global-atomic share both shrink)
    sp.block = 1024;
    sp.min_blocks = 2;
    sp.spill_allowance = 64;
    sp.depth_test = 1;
    // privatized window: when the chain splats once, into a histogram
    sp.tile = (sp.splats.size() == 1 && sp.splats[0].kind == CFS_TARGET_HIST_U32 &&
               sp.scribble.empty()) ? 1 : 0;
    // warp-level aggregation of equal window addresses (match.any) measured
    // slower than plain shared atomics on the animation batch: off
    sp.warp_agg = 0;
    // two trajectories per thread: 755 vs 764 ms for the 256-frame batch
    sp.ilp = 2;
    const uint32_t tile_cap = sp.tile ? 53248u : 0u;
    sp.dyn_smem = (int)(tile_cap * sizeof(uint32_t));
    // a window above half of the SM's shared memory leaves room for one CTA
    // per SM: asking for two would only cap the registers (and spill)
    if (sp.dyn_smem > 112 * 1024) sp.min_blocks = 1;
    return tile_cap;
}
}  // namespace cfs

namespace {
// Cuts every frame into items of its own chunk of points (whole warps),
// numbers the items frame by frame, repacks the staged frame descriptors and
// sets the persistent grid (resident CTAs, at most one per item).  Frames
// outside `active` (when given) get no items: an autotuner trial of one
// shape class.
cfs_status plan_items(cfs_batch* b, const std::vector<uint8_t>* active = nullptr)
{
    b->grid = (uint32_t)std::max(1, b->kernel.max_blocks_per_sm * std::max(1, b->kernel.num_sms));
    uint64_t total = 0;
    std::vector<uint32_t> begin(b->n_frames);
    for (int f = 0; f < b->n_frames; ++f) {
        begin[f] = (uint32_t)total;
        if (active && !(*active)[f]) continue;
        total += ((uint64_t)b->frames[f].n_points + b->chunks[f] - 1) / b->chunks[f];
        if (total >= (1ull << 31)) return fail(CFS_ERR_INVALID_ARG, "too many work items");
    }
    b->n_items = (uint32_t)total;
    if (b->grid > b->n_items && b->n_items > 0) b->grid = b->n_items;
    if (b->h_frames) {
        for (int f = 0; f < b->n_frames; ++f) {
            const uint32_t np = (active && !(*active)[f]) ? 0u : b->frames[f].n_points;
            cfs_frame fr = b->frames[f];
            fr.n_points = np;
            pack_frame(&b->h_frames[f], b->systems[f], fr, b->n_targets, begin[f], b->chunks[f],
                       b->nowin[f] != 0);
        }
    }
    b->chunk = b->plan.chunk;
    b->args.n_items = b->n_items;
    b->args.chunk = b->plan.chunk;
    return CFS_OK;
}

bool window_allowed(const ProgramSpec& sp)
{
    return sp.scribble.empty() && sp.splats.size() == 1 &&
           sp.splats[0].kind == CFS_TARGET_HIST_U32;
}

cfs_status check_plan(const cfs_batch_plan& p)
{
    if (p.ilp != 1 && p.ilp != 2) return fail(CFS_ERR_INVALID_ARG, "plan: ilp must be 1 or 2");
    if (p.window != 0 && p.window != 1) return fail(CFS_ERR_INVALID_ARG, "plan: window 0 or 1");
    if (p.window_words < 1024 || p.window_words > 53248 || p.window_words % 256)
        return fail(CFS_ERR_INVALID_ARG,
                    "plan: window_words must be a multiple of 256 in 1024..53248");
    if (p.warp_agg != 0 && p.warp_agg != 1)
        return fail(CFS_ERR_INVALID_ARG, "plan: warp_agg 0 or 1");
    if (p.chunk < 32 || p.chunk > (1u << 20) || p.chunk % 32)
        return fail(CFS_ERR_INVALID_ARG, "plan: chunk must be a multiple of 32 in 32..2^20");
    return CFS_OK;
}

// Sets the program knobs of the spec from the plan (window only where the
// chain allows one) and the window capacity of the launch.
void spec_from_plan(cfs_batch* b)
{
    ProgramSpec& sp = b->spec;
    sp.ilp = b->plan.ilp;
    sp.tile = (b->plan.window && window_allowed(sp)) ? 1 : 0;
    sp.warp_agg = sp.tile ? b->plan.warp_agg : 0;
    b->tile_cap = sp.tile ? b->plan.window_words : 0u;
    sp.dyn_smem = (int)(b->tile_cap * sizeof(uint32_t));
    // a window above half of the SM's shared memory leaves room for one CTA
    // per SM: asking for two would only cap the registers (and spill)
    sp.min_blocks = sp.dyn_smem > 112 * 1024 ? 1 : 2;
}

// Compiles the batch program (and the window pre-pass when tiled) for the
// plan's knobs.
cfs_status build_program(cfs_batch* b)
{
    spec_from_plan(b);
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
// remembers the window set-up a launch runs with
void note_windows(cfs_batch* b)
{
    b->last_tile = b->spec.tile != 0;
    b->last_tile_cap = b->tile_cap;
    b->last_nowin = b->nowin;
}

cfs_status run_direct(cfs_batch* b, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    note_windows(b);
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
// the autotuner's per-class stage runs for batches of at most this many shape
// classes
constexpr int kMaxTunedClasses = 32;

// ---- the tuning cache ------------------------------------------------------
// Keys hold no spaces (the file format is "key value" per line).
std::map<std::string, std::string> g_cache;
std::mutex g_cache_mu;

bool cache_get(const std::string& k, std::string* v)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = g_cache.find(k);
    if (it == g_cache.end()) return false;
    *v = it->second;
    return true;
}

void cache_put(const std::string& k, const std::string& v)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_cache[k] = v;
}

std::string no_spaces(std::string t)
{
    for (char& c : t)
        if (c == ' ' || c == '\t' || c == '\n' || c == '\r') c = '_';
    return t;
}

cfs_status device_key(int dev, std::string* out)
{
    cudaDeviceProp p;
    cfs_status st = check_cuda(cudaGetDeviceProperties(&p, dev), "cudaGetDeviceProperties");
    if (st != CFS_OK) return st;
    std::ostringstream o;
    o << no_spaces(p.name) << ".sm" << p.multiProcessorCount << ".cc" << p.major << p.minor;
    *out = o.str();
    return CFS_OK;
}

// the program's structure without the knobs the tuner sets
std::string structure_key(const ProgramSpec& sp)
{
    ProgramSpec k = sp;
    k.ilp = 0;
    k.tile = 0;
    k.warp_agg = 0;
    k.min_blocks = 0;
    k.dyn_smem = 0;
    return no_spaces(k.key());
}

// point-count bucket (log2 rounded down to even) and target 0's size
std::string frame_class(const cfs_frame& f, int n_targets)
{
    int lg = 0;
    while (lg < 32 && (1ull << (lg + 1)) <= (uint64_t)std::max(1u, f.n_points)) ++lg;
    std::ostringstream o;
    o << "p" << (lg & ~1);
    if (n_targets > 0) o << ".w" << f.targets[0].width << "x" << f.targets[0].height;
    return o.str();
}

std::string format_plan(const cfs_batch_plan& p)
{
    std::ostringstream o;
    o << "ilp=" << p.ilp << ",win=" << p.window << ",words=" << p.window_words
      << ",agg=" << p.warp_agg << ",chunk=" << p.chunk;
    return o.str();
}

bool parse_plan(const std::string& v, cfs_batch_plan* p)
{
    unsigned words = 0, chunk = 0;
    int ilp = 0, win = 0, agg = 0;
    if (std::sscanf(v.c_str(), "ilp=%d,win=%d,words=%u,agg=%d,chunk=%u", &ilp, &win, &words,
                    &agg, &chunk) != 5)
        return false;
    p->ilp = ilp;
    p->window = win;
    p->window_words = words;
    p->warp_agg = agg;
    p->chunk = chunk;
    return true;
}

std::string format_class(uint32_t chunk, uint8_t nowin)
{
    std::ostringstream o;
    o << "chunk=" << chunk << ",nowin=" << (int)nowin;
    return o.str();
}

bool parse_class(const std::string& v, uint32_t* chunk, uint8_t* nowin)
{
    unsigned c = 0;
    int nw = 0;
    if (std::sscanf(v.c_str(), "chunk=%u,nowin=%d", &c, &nw) != 2) return false;
    if (c < 32 || c > (1u << 20) || c % 32 || (nw != 0 && nw != 1)) return false;
    *chunk = c;
    *nowin = (uint8_t)nw;
    return true;
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
    sp.n_ops = chain->n_xops;
    sp.n_targets = n_targets;
    sp.fast_trig = trig_mode(chain->flags);
    for (int o = 0; o < chain->n_xops; ++o) {
        sp.op_kind[o] = chain->xops[o].kind;
        if (chain->xops[o].kind == CFS_OP_ROTATE3) sp.op_axis[o] = (int)chain->xops[o].params[1];
        if (chain->xops[o].kind == CFS_OP_BANDS) sp.op_axis[o] = (int)chain->xops[o].params[0];
        if (chain->xops[o].kind == CFS_OP_SPLAT) {
            const int slot = (int)chain->xops[o].params[0];
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
    batch_spec_defaults(sp);
    // the default plan; cfs_batch_set_plan and cfs_batch_tune change it
    b->plan.ilp = sp.ilp;
    b->plan.window = 1;
    b->plan.window_words = 53248;
    b->plan.warp_agg = 0;
    b->plan.chunk = 4096;
    st = build_program(b);
    if (st != CFS_OK) { delete b; return st; }

    // Items: every frame is cut into items of its chunk of points (whole
    // warps); all CTAs work on one or two frames at a time, so the live
    // layers stay in L2.  cfs_batch_tune picks the chunks (and the program's
    // knobs) by measurement.
    b->chunks.assign(n_frames, b->plan.chunk);
    b->nowin.assign(n_frames, 0);
    st = plan_items(b);
    if (st != CFS_OK) { delete b; return st; }

    // workspace: frames | window boxes (an int4 per frame and histogram
    // channel, CFS_A_MAX_MAPS slots per frame) | counter (u32, padded to
    // 256 B) | discards (the counter and discards are reset every launch)
    const size_t fbytes = sizeof(cfs_dev_frame) * (size_t)n_frames;
    const size_t off_bbox = (fbytes + 255) & ~(size_t)255;
    const size_t off_counter =
        (off_bbox + 16 * (size_t)CFS_A_MAX_MAPS * (size_t)n_frames + 255) & ~(size_t)255;
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
    st = plan_items(b);                  // now that the staging buffer exists
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
               b->chunks[frame], b->nowin[frame] != 0);
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
    note_windows(b);
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

// histogram channels of the batch's target 0 (the windowed splat's)
static int window_channels(const cfs_batch* b)
{
    if (b->n_frames < 1 || b->n_targets < 1) return 1;
    const cfs_target& g = b->frames[0].targets[0];
    return g.kind == CFS_TARGET_HIST_U32 ? std::max(1, g.channels) : 1;
}

cfs_status cfs_batch_windows(cfs_batch* b, int32_t* out)
{
    clear_error();
    if (!b || !out) return fail(CFS_ERR_INVALID_ARG, "NULL batch or out");
    if (!b->launched) return fail(CFS_ERR_INVALID_ARG, "the batch has not been launched");
    cfs_status st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    if (st != CFS_OK) return st;
    const int C = window_channels(b);
    const size_t n = 4 * (size_t)CFS_A_MAX_MAPS * (size_t)b->n_frames;
    std::vector<int32_t> box(n, 0);
    if (b->last_tile) {
        st = check_cuda(cudaMemcpy(box.data(), b->d_bbox, sizeof(int32_t) * n,
                                   cudaMemcpyDeviceToHost),
                        "cudaMemcpy(windows)");
        if (st != CFS_OK) return st;
    }
    for (int f = 0; f < b->n_frames; ++f) {
        // the kernel's rule: the channels' windows take consecutive counters;
        // none for a frame without one, an empty box, or a box that would
        // pass the last counter
        long long used = 0;
        for (int c = 0; c < C; ++c) {
            int32_t* o = out + 4 * ((size_t)f * (size_t)C + (size_t)c);
            const int32_t* w = box.data() + 4 * ((size_t)f * CFS_A_MAX_MAPS + (size_t)c);
            const long long ww = (long long)w[2] - w[0] + 1, wh = (long long)w[3] - w[1] + 1;
            const bool none = !b->last_tile || b->last_nowin[f] || ww < 1 || wh < 1 ||
                              ww > 0xFFFF || wh > 0x7FFF ||
                              used + ww * wh > (long long)b->last_tile_cap;
            if (!none) used += ww * wh;
            o[0] = none ? 0 : w[0];
            o[1] = none ? 0 : w[1];
            o[2] = none ? -1 : w[2];
            o[3] = none ? -1 : w[3];
        }
    }
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

cfs_status cfs_batch_get_plan(const cfs_batch* b, cfs_batch_plan* out)
{
    clear_error();
    if (!b || !out) return fail(CFS_ERR_INVALID_ARG, "NULL batch or out");
    *out = b->plan;
    return CFS_OK;
}

cfs_status cfs_batch_set_plan(cfs_batch* b, const cfs_batch_plan* plan)
{
    clear_error();
    if (!b || !plan) return fail(CFS_ERR_INVALID_ARG, "NULL batch or plan");
    cfs_status st = check_plan(*plan);
    if (st != CFS_OK) return st;
    if (b->launched) st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    if (st != CFS_OK) return st;
    const cfs_batch_plan old = b->plan;
    b->plan = *plan;
    st = build_program(b);
    if (st != CFS_OK) {
        b->plan = old;
        build_program(b);
        return st;
    }
    std::fill(b->chunks.begin(), b->chunks.end(), b->plan.chunk);
    std::fill(b->nowin.begin(), b->nowin.end(), (uint8_t)0);
    st = plan_items(b);
    drop_graphs(b);                     // the next launch captures the new plan
    return st;
}

cfs_status cfs_batch_tune(cfs_batch* b, uint32_t trial_iters, uint32_t flags, void* stream,
                          cfs_batch_tuning* out)
{
    clear_error();
    if (!b) return fail(CFS_ERR_INVALID_ARG, "NULL batch");
    if (flags & ~CFS_TUNE_RETUNE) return fail(CFS_ERR_INVALID_ARG, "unknown tuning flags");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(CFS_ERR_INVALID_ARG, "batch belongs to another device");
    cudaStream_t s = (cudaStream_t)stream;
    cfs_status st = CFS_OK;
    if (b->launched) st = check_cuda(cudaEventSynchronize(b->done), "cudaEventSynchronize");
    if (b->disp_launched && st == CFS_OK)
        st = check_cuda(cudaEventSynchronize(b->disp_done), "cudaEventSynchronize");
    if (st != CFS_OK) return st;
    std::string devkey;
    st = device_key(b->device, &devkey);
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
    const bool retune = (flags & CFS_TUNE_RETUNE) != 0;
    const bool win_ok = window_allowed(b->spec);
    int trials = 0;
    bool all_cached = true;

    // shape classes: point-count bucket and target size
    std::vector<std::string> cls(b->n_frames);
    std::map<std::string, int> counts;
    for (int f = 0; f < b->n_frames; ++f) {
        cls[f] = frame_class(b->frames[f], b->n_targets);
        counts[cls[f]]++;
    }
    std::ostringstream mix;
    for (const auto& kv : counts) mix << kv.first << ":" << kv.second << ";";
    const std::string skey = structure_key(b->spec);

    // one timed trial of the current program and item plan (best of two)
    auto trial = [&](const std::vector<uint8_t>* active, float* ms) -> cfs_status {
        cfs_status r = plan_items(b, active);
        float best = 1e30f;
        for (int rep = 0; rep < 2 && r == CFS_OK; ++rep) {
            r = run_direct(b, s, e0, e1);
            if (r == CFS_OK) r = check_cuda(cudaEventSynchronize(e1), "trial");
            float t = 0.0f;
            if (r == CFS_OK) r = check_cuda(cudaEventElapsedTime(&t, e0, e1), "time");
            best = std::min(best, t);
        }
        ++trials;
        *ms = best;
        return r;
    };
    auto set_all = [&](uint32_t chunk, uint8_t nowin) {
        std::fill(b->chunks.begin(), b->chunks.end(), chunk);
        std::fill(b->nowin.begin(), b->nowin.end(), nowin);
    };

    // ---- stage 1: the program, on the whole batch ------------------------
    const std::string gkey = "batch|" + devkey + "|" + skey + "|" + mix.str();
    cfs_batch_plan best = b->plan;
    float best_ms = 0.0f;
    std::string cached;
    if (!retune && cache_get(gkey, &cached) && parse_plan(cached, &best) &&
        check_plan(best) == CFS_OK) {
        b->plan = best;
        st = build_program(b);
        set_all(best.chunk, 0);
    } else {
        all_cached = false;
        set_all(best.chunk, 0);
        st = build_program(b);
        if (st == CFS_OK) st = trial(nullptr, &best_ms);
        // one knob at a time, keeping each improvement
        auto consider = [&](cfs_batch_plan cand) {
            if (st != CFS_OK) return;
            b->plan = cand;
            st = build_program(b);
            set_all(cand.chunk, 0);
            float ms = 0.0f;
            if (st == CFS_OK) st = trial(nullptr, &ms);
            if (st == CFS_OK && ms < best_ms) { best = cand; best_ms = ms; }
        };
        for (int ilp = 1; ilp <= 2; ++ilp)
            if (ilp != best.ilp) { cfs_batch_plan c = best; c.ilp = ilp; consider(c); }
        if (win_ok) {
            { cfs_batch_plan c = best; c.window = 1 - best.window; consider(c); }
            if (best.window) {
                for (uint32_t w : {13312u, 26624u, 53248u})
                    if (w != best.window_words) {
                        cfs_batch_plan c = best; c.window_words = w; consider(c);
                    }
                { cfs_batch_plan c = best; c.warp_agg = 1 - best.warp_agg; consider(c); }
            }
        }
        for (uint32_t c0 : {2048u, 4096u, 8192u, 16384u})
            if (c0 != best.chunk) { cfs_batch_plan c = best; c.chunk = c0; consider(c); }
        if (st == CFS_OK) {
            cache_put(gkey, format_plan(best));
            b->plan = best;
            st = build_program(b);
            set_all(best.chunk, 0);
        }
    }

    // ---- stage 2: item size and window per shape class -------------------
    // (only for a batch of at most kMaxTunedClasses classes: each class costs
    // up to eight trials)
    int n_win = b->spec.tile ? (int)counts.size() : 0;
    bool use_classes = false;
    if (st == CFS_OK && (int)counts.size() <= kMaxTunedClasses) {
        n_win = 0;
        cfs_batch_plan prog = b->plan;
        prog.chunk = 0;                 // the program's knobs only
        const std::string pkey = format_plan(prog);
        std::vector<uint8_t> active(b->n_frames);
        for (const auto& kv : counts) {
            if (st != CFS_OK) break;
            const std::string ckey = "class|" + devkey + "|" + skey + "|" + pkey + "|" + kv.first;
            uint32_t c_best = b->plan.chunk;
            uint8_t nw_best = 0;
            std::string v;
            if (!retune && cache_get(ckey, &v) && parse_class(v, &c_best, &nw_best)) {
                // cached
            } else {
                all_cached = false;
                for (int f = 0; f < b->n_frames; ++f) active[f] = cls[f] == kv.first;
                float cls_best = 1e30f;
                const int n_nw = (win_ok && b->plan.window) ? 2 : 1;
                for (int nw = 0; nw < n_nw && st == CFS_OK; ++nw)
                    for (uint32_t c0 : {2048u, 4096u, 8192u, 16384u}) {
                        for (int f = 0; f < b->n_frames; ++f)
                            if (active[f]) { b->chunks[f] = c0; b->nowin[f] = (uint8_t)nw; }
                        float ms = 0.0f;
                        st = trial(&active, &ms);
                        if (st != CFS_OK) break;
                        if (ms < cls_best) { cls_best = ms; c_best = c0; nw_best = (uint8_t)nw; }
                    }
                if (st == CFS_OK) cache_put(ckey, format_class(c_best, nw_best));
            }
            for (int f = 0; f < b->n_frames; ++f)
                if (cls[f] == kv.first) { b->chunks[f] = c_best; b->nowin[f] = nw_best; }
            if (!nw_best && b->spec.tile) ++n_win;
        }
        // a class timed alone is not the class inside the batch (frames of
        // other classes share the CTAs and the L2): the classes' choices are
        // kept only when the whole batch runs faster with them than with the
        // program's plan alone
        if (st == CFS_OK) {
            const std::string ukey = "classes|" + devkey + "|" + skey + "|" + pkey + "|" +
                                     mix.str();
            std::string v;
            if (!retune && cache_get(ukey, &v) && (v == "1" || v == "0")) {
                use_classes = v == "1";
            } else {
                all_cached = false;
                const std::vector<uint32_t> ch = b->chunks;
                const std::vector<uint8_t> nw = b->nowin;
                float with_ms = 0.0f, without_ms = 0.0f;
                st = trial(nullptr, &with_ms);
                set_all(b->plan.chunk, 0);
                if (st == CFS_OK) st = trial(nullptr, &without_ms);
                use_classes = with_ms < without_ms;
                b->chunks = ch;
                b->nowin = nw;
                if (st == CFS_OK) cache_put(ukey, use_classes ? "1" : "0");
            }
            if (!use_classes) {
                set_all(b->plan.chunk, 0);
                n_win = b->spec.tile ? (int)counts.size() : 0;
            }
        }
    }

    // keep the result (or restore a consistent plan after an error)
    if (st != CFS_OK) {
        b->plan = best;
        build_program(b);
        set_all(b->plan.chunk, 0);
    }
    cfs_status st2 = plan_items(b);
    b->args.iters = full_iters;
    drop_graphs(b);                     // the next launch captures the new plan
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CFS_OK) return st;
    if (st2 != CFS_OK) return st2;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        out->ilp = b->plan.ilp;
        out->tile = b->spec.tile;
        out->chunk = b->plan.chunk;
        out->trial_ms = best_ms;
        out->trials = trials;
        out->window_words = b->spec.tile ? b->plan.window_words : 0u;
        out->warp_agg = b->spec.warp_agg;
        out->n_classes = (int)counts.size();
        out->classes_windowed = n_win;
        out->from_cache = all_cached ? 1 : 0;
        out->classes_used = use_classes ? 1 : 0;
    }
    return CFS_OK;
}

cfs_status cfs_tune_cache_load(const char* path)
{
    clear_error();
    if (!path) return fail(CFS_ERR_INVALID_ARG, "NULL path");
    std::ifstream in(path);
    if (!in) return CFS_OK;
    std::map<std::string, std::string> got;
    std::string line;
    while (std::getline(in, line)) {
        if (line.empty()) continue;
        const size_t sp = line.rfind(' ');
        if (sp == std::string::npos || sp == 0 || sp + 1 >= line.size())
            return fail(CFS_ERR_INVALID_ARG, "malformed tuning-cache line: " + line);
        got[line.substr(0, sp)] = line.substr(sp + 1);
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (auto& kv : got) g_cache[kv.first] = kv.second;
    return CFS_OK;
}

cfs_status cfs_tune_cache_save(const char* path)
{
    clear_error();
    if (!path) return fail(CFS_ERR_INVALID_ARG, "NULL path");
    std::ofstream o(path, std::ios::trunc);
    if (!o) return fail(CFS_ERR_INVALID_ARG, std::string("cannot write ") + path);
    std::lock_guard<std::mutex> lock(g_cache_mu);
    for (const auto& kv : g_cache) o << kv.first << " " << kv.second << "\n";
    o.flush();
    if (!o) return fail(CFS_ERR_INVALID_ARG, std::string("cannot write ") + path);
    return CFS_OK;
}

cfs_status cfs_tune_cache_clear(void)
{
    clear_error();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    g_cache.clear();
    return CFS_OK;
}

uint32_t cfs_tune_cache_size(void)
{
    std::lock_guard<std::mutex> lock(g_cache_mu);
    return (uint32_t)g_cache.size();
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
