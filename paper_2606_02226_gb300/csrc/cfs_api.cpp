// cfs_api.cpp -- the extern "C" entry points of libcfs (include/cfs.h).
//
// Host work only: argument validation, the threshold table, per-op
// constants, the kernel argument block, and launches of the generated
// programs on the caller's stream.  Every step of the chaos game itself runs
// in the generated CUDA kernels.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <sstream>

#include "cfs_internal.h"

namespace cfs {
const char* last_error();

void philox_round_keys(uint64_t seed, unsigned int rk[10][2])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[r][0] = k0;
        rk[r][1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

void derive_op_params(const cfs_transform& op, float out[CFS_OP_PARAMS])
{
    std::memset(out, 0, sizeof(float) * CFS_OP_PARAMS);
    const float* v = op.params;
    switch (op.kind) {
    case CFS_OP_ROTATE2: {
        const float c = (float)std::cos((double)v[0]), s = (float)std::sin((double)v[0]);
        out[0] = c; out[1] = -s; out[2] = s; out[3] = c;
        break;
    }
    case CFS_OP_ROTATE3: {
        const float c = (float)std::cos((double)v[0]), s = (float)std::sin((double)v[0]);
        float R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        const int axis = (int)v[1];
        if (axis == 0) { R[4] = c; R[5] = -s; R[7] = s; R[8] = c; }
        else if (axis == 1) { R[0] = c; R[2] = s; R[6] = -s; R[8] = c; }
        else { R[0] = c; R[1] = -s; R[3] = s; R[4] = c; }
        std::memcpy(out, R, sizeof(R));
        break;
    }
    case CFS_OP_TRANSLATE3:
        out[0] = 1; out[4] = 1; out[8] = 1;
        out[9] = v[0]; out[10] = v[1]; out[11] = v[2];
        break;
    case CFS_OP_BEND:
        out[0] = v[0];
        out[1] = 1.0f / v[0];
        break;
    case CFS_OP_INVERSION:
        out[0] = v[0]; out[1] = v[1]; out[2] = v[2];
        out[3] = v[3] * v[3];
        break;
    case CFS_OP_STARS:
        // n as an integer's bits; box origins and extents (FP32 differences,
        // as the oracle forms them)
        {
            const uint32_t n = (uint32_t)v[0];
            std::memcpy(&out[0], &n, 4);
        }
        out[1] = v[1]; out[2] = v[2] - v[1];
        out[3] = v[3]; out[4] = v[4] - v[3];
        out[5] = v[5]; out[6] = v[6] - v[5];
        out[7] = v[7]; out[8] = v[8] - v[7];
        break;
    default:
        std::memcpy(out, v, sizeof(float) * CFS_OP_PARAMS);
        break;
    }
}

namespace {
bool linear2(int k) { return k == CFS_OP_AFFINE2 || k == CFS_OP_ROTATE2; }

// multiply-adds a linear op costs in the generated code (rotations about an
// axis and translations have specialised forms)
int linear_cost(int k)
{
    switch (k) {
    case CFS_OP_AFFINE2: case CFS_OP_ROTATE2: return 4;
    case CFS_OP_AFFINE3: return 9;
    case CFS_OP_ROTATE3: return 4;
    case CFS_OP_TRANSLATE3: return 3;
    default: return 0;
    }
}
bool linear3(int k)
{
    return k == CFS_OP_AFFINE3 || k == CFS_OP_ROTATE3 || k == CFS_OP_TRANSLATE3;
}

// x -> M x + t of a linear op (3D form; 2D ops act on x, y and keep z), from
// the FP32 constants the kernels would use
void op_matrix(const cfs_transform& op, double M[9], double t[3])
{
    float d[CFS_OP_PARAMS];
    derive_op_params(op, d);
    for (int j = 0; j < 9; ++j) M[j] = 0.0;
    t[0] = t[1] = t[2] = 0.0;
    if (linear2(op.kind)) {
        const float* v = op.kind == CFS_OP_AFFINE2 ? op.params : d;
        M[0] = v[0]; M[1] = v[1]; M[3] = v[2]; M[4] = v[3]; M[8] = 1.0;
        if (op.kind == CFS_OP_AFFINE2) { t[0] = v[4]; t[1] = v[5]; }
    } else {
        const float* v = op.kind == CFS_OP_AFFINE3 ? op.params : d;
        for (int j = 0; j < 9; ++j) M[j] = v[j];
        for (int j = 0; j < 3; ++j) t[j] = v[9 + j];
    }
}
}  // namespace

void refresh_exec_ops(cfs_chain* c)
{
    c->n_xops = 0;
    for (int o = 0; o < c->n_ops;) {
        const int k = c->ops[o].kind;
        int e = o + 1;
        if (c->flags & CFS_COMPOSE_FOLD_LINEAR) {
            while (e < c->n_ops && ((linear2(k) && linear2(c->ops[e].kind)) ||
                                    (linear3(k) && linear3(c->ops[e].kind))))
                ++e;
        }
        // fold only where one affine op is cheaper than the run as written
        int run_cost = 0;
        for (int j = o; j < e; ++j) run_cost += linear_cost(c->ops[j].kind);
        const int folded_cost = linear2(k) ? linear_cost(CFS_OP_AFFINE2)
                                           : linear_cost(CFS_OP_AFFINE3);
        if (e - o < 2 || folded_cost >= run_cost) {
            for (int j = o; j < e; ++j) c->xops[c->n_xops++] = c->ops[j];
            o = e;
            continue;
        }
        // compose in double: after op j, x -> M_j (...) + t_j
        double M[9], t[3];
        op_matrix(c->ops[o], M, t);
        for (int j = o + 1; j < e; ++j) {
            double N[9], u[3], P[9], w[3];
            op_matrix(c->ops[j], N, u);
            for (int r = 0; r < 3; ++r) {
                for (int q = 0; q < 3; ++q)
                    P[3 * r + q] = N[3 * r] * M[q] + N[3 * r + 1] * M[3 + q] + N[3 * r + 2] * M[6 + q];
                w[r] = N[3 * r] * t[0] + N[3 * r + 1] * t[1] + N[3 * r + 2] * t[2] + u[r];
            }
            std::memcpy(M, P, sizeof(M));
            std::memcpy(t, w, sizeof(t));
        }
        cfs_transform f;
        std::memset(&f, 0, sizeof(f));
        if (linear2(k)) {
            f.kind = CFS_OP_AFFINE2;
            const double v[6] = {M[0], M[1], M[3], M[4], t[0], t[1]};
            for (int j = 0; j < 6; ++j) f.params[j] = (float)v[j];
        } else {
            f.kind = CFS_OP_AFFINE3;
            for (int j = 0; j < 9; ++j) f.params[j] = (float)M[j];
            for (int j = 0; j < 3; ++j) f.params[9 + j] = (float)t[j];
        }
        c->xops[c->n_xops++] = f;
        o = e;
    }
}

namespace {

bool finite_all(const float* v, int n)
{
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(v[j])) return false;
    return true;
}

int op_out_dim(int kind, int dim_in)
{
    switch (kind) {
    case CFS_OP_TORUS: case CFS_OP_STARS: case CFS_OP_HEMISPHERE: return 3;
    default: return dim_in;
    }
}

// parameter rules of the ops whose parameters carry structure
bool op_params_ok(const cfs_transform& op, int dim, std::string* why)
{
    const float* v = op.params;
    if (op.kind == CFS_OP_STARS) {
        if (!(v[0] >= 1.0f && v[0] <= 16777216.0f && v[0] == std::floor(v[0]))) {
            *why = "stars: n must be an integer in 1..2^24";
            return false;
        }
    } else if (op.kind == CFS_OP_BANDS) {
        const int axis = (int)v[0], n = (int)v[3], base = (int)v[4];
        if (!(v[0] == (float)axis && axis >= 0 && axis < dim)) {
            *why = "bands: axis must name a coordinate of the point";
            return false;
        }
        if (!(v[3] == (float)n && v[4] == (float)base && n >= 1 && base >= 0 &&
              base + n <= CFS_MAX_MAPS)) {
            *why = "bands: n >= 1, base >= 0 (integers), base + n <= 16";
            return false;
        }
    }
    return true;
}

bool op_needs_3d(int kind)
{
    switch (kind) {
    case CFS_OP_AFFINE3: case CFS_OP_ROTATE3: case CFS_OP_TRANSLATE3: case CFS_OP_SINUSOIDAL3:
    case CFS_OP_PERSPECTIVE: case CFS_OP_TWIST_Z: case CFS_OP_BEND: case CFS_OP_INVERSION:
        return true;
    default:
        return false;
    }
}

cfs_status validate_targets(const cfs_chain* ch, const cfs_target* tg, int n_tg)
{
    if (n_tg < 0 || n_tg > CFS_MAX_TARGETS)
        return fail(CFS_ERR_INVALID_ARG, "n_targets must be in 0..4");
    if (n_tg > 0 && !tg) return fail(CFS_ERR_INVALID_ARG, "targets is NULL");
    for (int t = 0; t < n_tg; ++t) {
        const cfs_target& g = tg[t];
        std::ostringstream m;
        m << "target " << t << ": ";
        if (g.kind < CFS_TARGET_HIST_U32 || g.kind > CFS_TARGET_DEPTH_U64)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "unknown kind");
        if (g.width <= 0 || g.height <= 0 || g.width > 65536 || g.height > 65536)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "width/height must be in 1..65536");
        if (g.kind == CFS_TARGET_HIST_U32 && (g.channels < 1 || g.channels > CFS_MAX_MAPS))
            return fail(CFS_ERR_INVALID_ARG, m.str() + "histogram channels must be in 1..16");
        if (!g.data) return fail(CFS_ERR_INVALID_ARG, m.str() + "data is NULL");
        if (((uintptr_t)g.data) % 16 != 0)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "data must be 16-byte aligned");
        if (!(std::isfinite(g.x0) && std::isfinite(g.x1) && std::isfinite(g.y0) &&
              std::isfinite(g.y1) && g.x1 > g.x0 && g.y1 > g.y0))
            return fail(CFS_ERR_INVALID_ARG, m.str() + "view needs finite x0 < x1, y0 < y1");
    }
    for (int slot : ch->scribble_slots)
        if (slot >= n_tg) {
            std::ostringstream m;
            m << "scribble splat names target slot " << slot << " but only " << n_tg
              << " targets were given";
            return fail(CFS_ERR_INVALID_ARG, m.str());
        }
    // every SPLAT names an existing slot, and depth splats see a 3D point
    int dim = ch->dim_in;
    for (int o = 0; o < ch->n_ops; ++o) {
        const cfs_transform& op = ch->ops[o];
        if (op.kind == CFS_OP_RESET) dim = ch->dim_in;
        if (op.kind == CFS_OP_SPLAT) {
            const int slot = (int)op.params[0];
            if (slot < 0 || slot >= n_tg) {
                std::ostringstream m;
                m << "op " << o << ": SPLAT names target slot " << slot << " but only " << n_tg
                  << " targets were given";
                return fail(CFS_ERR_INVALID_ARG, m.str());
            }
            if (tg[slot].kind == CFS_TARGET_DEPTH_U64 && dim != 3)
                return fail(CFS_ERR_INVALID_ARG, "depth targets need a 3D point at the splat");
        }
        dim = op_out_dim(op.kind, dim);
    }
    return CFS_OK;
}

ProgramSpec make_spec(Mode mode, const cfs_system* sys, const cfs_chain* ch,
                      const cfs_target* tg, int n_tg, bool reuse)
{
    ProgramSpec sp;
    sp.mode = mode;
    sp.dim = sys->dim;
    sp.n_maps = sys->n_maps;
    for (int j = 0; j < sys->n_maps; ++j) sp.map_kind[j] = sys->maps[j].kind;
    sp.n_cmp = sys->n_cmp;
    sp.reuse = reuse;
    sp.n_ops = ch->n_xops;
    sp.n_targets = n_tg;
    sp.fast_trig = trig_mode(ch->flags);
    for (int o = 0; o < ch->n_xops; ++o) {
        sp.op_kind[o] = ch->xops[o].kind;
        if (ch->xops[o].kind == CFS_OP_ROTATE3) sp.op_axis[o] = (int)ch->xops[o].params[1];
        if (ch->xops[o].kind == CFS_OP_BANDS) sp.op_axis[o] = (int)ch->xops[o].params[0];
        if (ch->xops[o].kind == CFS_OP_SPLAT) {
            const int slot = (int)ch->xops[o].params[0];
            SplatSpec s;
            s.slot = slot;
            s.kind = tg ? tg[slot].kind : CFS_TARGET_HIST_U32;
            s.channels = (tg && tg[slot].kind == CFS_TARGET_HIST_U32) ? tg[slot].channels : 1;
            sp.splats.push_back(s);
        }
    }
    sp.scribble = ch->scribble;
    for (int slot : ch->scribble_slots) {
        SplatSpec s;
        s.slot = slot;
        s.kind = tg ? tg[slot].kind : CFS_TARGET_HIST_U32;
        s.channels = (tg && tg[slot].kind == CFS_TARGET_HIST_U32) ? tg[slot].channels : 1;
        sp.splats.push_back(s);
    }
    // register budget: 256 threads x 8 blocks (full occupancy) leaves 32
    // registers per thread; the generated programs fit without spills
    sp.block = 256;
    sp.min_blocks = 8;
    sp.depth_test = 1;
    // long chains (three objects from one point, 19 ops) ran 5% faster with two
    // copies of the step code than with four (instruction-cache misses); the
    // composed scene's 10 ops ran 2.5% faster with four
    sp.unroll = ch->n_xops > 12 ? 2 : 4;
    return sp;
}

void fill_args(cfs_launch_args* a, const cfs_system* sys, const cfs_chain* ch,
               const cfs_target* tg, int n_tg, const cfs_render_params* p)
{
    std::memset(a, 0, sizeof(*a));
    for (int j = 0; j < sys->n_cmp; ++j) a->sys.T[j] = sys->T[j];
    a->sys.n_maps = sys->n_maps;
    a->sys.n_cmp = sys->n_cmp;
    a->sys.dim = sys->dim;
    for (int k = 0; k < sys->n_maps; ++k)
        for (int j = 0; j < 12; ++j) a->sys.prm[j][k] = sys->maps[k].params[j];
    for (int o = 0; o < ch->n_xops; ++o) derive_op_params(ch->xops[o], a->op[o]);
    for (int t = 0; t < n_tg; ++t) {
        const cfs_target& g = tg[t];
        cfs_dev_target& d = a->tg[t];
        d.data = (unsigned long long)(uintptr_t)g.data;
        d.W = g.width;
        d.H = g.height;
        d.C = g.channels < 1 ? 1 : g.channels;
        d.kind = g.kind;
        d.x0 = g.x0; d.x1 = g.x1; d.y0 = g.y0; d.y1 = g.y1;
        d.sx = (float)g.width / (g.x1 - g.x0);
        d.sy = (float)g.height / (g.y1 - g.y0);
        std::memcpy(d.palette, g.palette, sizeof(d.palette));
        std::memcpy(d.palette8, g.palette8, sizeof(d.palette8));
    }
    philox_round_keys(p->seed, a->rk);
    a->discards = (unsigned long long)(uintptr_t)p->discards;
    a->start = (unsigned long long)(uintptr_t)p->start;
    a->system_id = p->system_id;
    a->point_begin = p->point_begin;
    a->n_points = p->n_points;
    a->step_begin = p->step_begin;
    a->iters = p->iters;
    a->burn_in = p->burn_in;
    a->flags = p->flags;
}

cfs_status validate_run(const cfs_system* sys, const cfs_chain* ch, const cfs_render_params* p)
{
    if (!sys || !ch || !p) return fail(CFS_ERR_INVALID_ARG, "NULL system, chain or params");
    if (ch->dim_in != sys->dim)
        return fail(CFS_ERR_INVALID_ARG, "chain was composed for another dimension");
    if (p->step_begin > p->iters) return fail(CFS_ERR_INVALID_ARG, "step_begin > iters");
    if ((uint64_t)p->point_begin + p->n_points > (1ull << 32))
        return fail(CFS_ERR_INVALID_ARG, "point indices exceed 2^32");
    if (p->flags & ~CFS_FLAG_REUSE) return fail(CFS_ERR_INVALID_ARG, "unknown flags");
    if (p->flags & CFS_FLAG_REUSE) {
        int dim = ch->dim_in;
        for (int o = 0; o < ch->n_ops; ++o) {
            if (ch->ops[o].kind == CFS_OP_RESET) dim = ch->dim_in;
            dim = op_out_dim(ch->ops[o].kind, dim);
        }
        if (dim != ch->dim_in)
            return fail(CFS_ERR_INVALID_ARG, "reuse needs a chain that keeps the dimension");
    }
    return CFS_OK;
}

}  // namespace

cfs_status validate_targets_ext(const cfs_chain* ch, const cfs_target* tg, int n_tg)
{
    return validate_targets(ch, tg, n_tg);
}

// chain constants, Philox round keys and step range of a launch
void fill_args_common(cfs_launch_args* a, const cfs_chain* ch, uint64_t seed, uint32_t iters,
                      uint32_t burn_in)
{
    std::memset(a, 0, sizeof(*a));
    for (int o = 0; o < ch->n_xops; ++o) derive_op_params(ch->xops[o], a->op[o]);
    philox_round_keys(seed, a->rk);
    a->iters = iters;
    a->burn_in = burn_in;
}
}  // namespace cfs

using namespace cfs;

extern "C" {

const char* cfs_last_error(void) { return cfs::last_error(); }

const char* cfs_version(void) { return "cfs-gb300 0.1 (sm_103a)"; }

uint32_t cfs_render_arg_bytes(void) { return (uint32_t)sizeof(cfs_launch_args); }

cfs_status cfs_stream_status(void* stream)
{
    clear_error();
    cfs_status st = check_cuda(cudaStreamSynchronize((cudaStream_t)stream),
                               "work on the stream failed");
    if (st != CFS_OK) return st;
    unsigned int flags = 0;
    st = take_device_flags(&flags);
    if (st != CFS_OK) return st;
    if (flags & CFS_DEVICE_ERR_TC_TIMEOUT)
        return fail(CFS_ERR_TIMEOUT, "a tensor-core GEMM timed out waiting for its mbarrier; "
                                     "its output is incomplete");
    if (flags) return fail(CFS_ERR_CUDA, "unknown device error flags");
    return CFS_OK;
}

cfs_status cfs_debug_raise_device_error(uint32_t flags)
{
    clear_error();
    if (flags == 0 || (flags & ~(uint32_t)CFS_DEVICE_ERR_ALL))
        return fail(CFS_ERR_INVALID_ARG, "flags must name CFS_DEVICE_ERR_* bits");
    return raise_device_flags(flags);
}

cfs_status cfs_system_create(int dim, int n_maps, const cfs_map* maps, const double* probs,
                             cfs_system** out)
{
    clear_error();
    if (!out) return fail(CFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(CFS_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (n_maps < 1 || n_maps > CFS_MAX_MAPS)
        return fail(CFS_ERR_INVALID_ARG, "n_maps must be in 1..16");
    if (!maps || !probs) return fail(CFS_ERR_INVALID_ARG, "maps or probs is NULL");
    double total = 0.0;
    for (int j = 0; j < n_maps; ++j) {
        if (!(probs[j] >= 0.0) || std::isinf(probs[j]))
            return fail(CFS_ERR_INVALID_ARG, "probabilities must be finite and >= 0");
        total += probs[j];
    }
    if (!(total > 0.0) || std::isinf(total))
        return fail(CFS_ERR_INVALID_ARG, "probabilities must have a positive finite sum");
    for (int j = 0; j < n_maps; ++j) {
        if (maps[j].kind != CFS_MAP_AFFINE && maps[j].kind != CFS_MAP_CIRCLE)
            return fail(CFS_ERR_INVALID_ARG, "unknown map kind");
        if (maps[j].kind == CFS_MAP_CIRCLE && dim != 2)
            return fail(CFS_ERR_INVALID_ARG, "the circle map (Eq. 1) is 2D");
        if (!finite_all(maps[j].params, 12))
            return fail(CFS_ERR_INVALID_ARG, "map parameters must be finite");
    }
    cfs_system* s = new (std::nothrow) cfs_system();
    if (!s) return fail(CFS_ERR_OOM, "host allocation failed");
    s->dim = dim;
    s->n_maps = n_maps;
    for (int j = 0; j < n_maps; ++j) {
        s->maps[j] = maps[j];
        if (maps[j].kind == CFS_MAP_AFFINE && dim == 2)
            for (int q = 6; q < 12; ++q) s->maps[j].params[q] = 0.0f;
        s->probs[j] = probs[j];
    }
    // T_k = floor(S_k 2^32) for k < n-1; those >= 2^32 never count (they can
    // only trail, the sums being non-decreasing)
    double running = 0.0;
    s->n_cmp = 0;
    for (int k = 0; k < n_maps - 1; ++k) {
        running += probs[k];
        const double t = std::floor((running / total) * 4294967296.0);
        if (t >= 4294967296.0) break;
        s->T[s->n_cmp++] = (uint32_t)(t < 0.0 ? 0.0 : t);
    }
    *out = s;
    return CFS_OK;
}

cfs_status cfs_system_destroy(cfs_system* sys)
{
    delete sys;
    return CFS_OK;
}

cfs_status cfs_compose(int dim_in, const cfs_transform* ops, int n_ops, cfs_chain** out)
{
    return cfs_compose_ex(dim_in, ops, n_ops, 0u, out);
}

cfs_status cfs_compose_ex(int dim_in, const cfs_transform* ops, int n_ops, uint32_t flags,
                          cfs_chain** out)
{
    clear_error();
    if (flags & ~(uint32_t)(CFS_COMPOSE_FAST_TRIG | CFS_COMPOSE_FOLD_LINEAR)) {
        if (out) *out = nullptr;
        return fail(CFS_ERR_INVALID_ARG, "unknown compose flags");
    }
    if (!out) return fail(CFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dim_in != 2 && dim_in != 3) return fail(CFS_ERR_INVALID_ARG, "dim_in must be 2 or 3");
    if (n_ops < 0 || n_ops > CFS_MAX_OPS)
        return fail(CFS_ERR_INVALID_ARG, "n_ops must be in 0..32");
    if (n_ops > 0 && !ops) return fail(CFS_ERR_INVALID_ARG, "ops is NULL");
    int dim = dim_in, n_splat = 0;
    for (int o = 0; o < n_ops; ++o) {
        const cfs_transform& op = ops[o];
        std::ostringstream m;
        m << "op " << o << ": ";
        if (op.kind < CFS_OP_AFFINE2 || op.kind > CFS_OP_BANDS)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "unknown kind");
        if (!finite_all(op.params, CFS_OP_PARAMS))
            return fail(CFS_ERR_INVALID_ARG, m.str() + "parameters must be finite");
        if (op.kind == CFS_OP_RESET) dim = dim_in;
        if (op_needs_3d(op.kind) && dim != 3)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "needs a 3D point");
        if (op.kind == CFS_OP_TORUS && dim != 2)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "torus embeds a 2D point");
        if (op.kind == CFS_OP_HEMISPHERE && dim != 2)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "hemisphere lifts a 2D point");
        {
            std::string why;
            if (!op_params_ok(op, dim, &why)) return fail(CFS_ERR_INVALID_ARG, m.str() + why);
        }
        if (op.kind == CFS_OP_BEND && op.params[0] == 0.0f)
            return fail(CFS_ERR_INVALID_ARG, m.str() + "bend needs a nonzero curvature");
        if (op.kind == CFS_OP_ROTATE3 && (op.params[1] != 0.0f && op.params[1] != 1.0f &&
                                          op.params[1] != 2.0f))
            return fail(CFS_ERR_INVALID_ARG, m.str() + "rotate3 axis must be 0, 1 or 2");
        if (op.kind == CFS_OP_SPLAT) {
            const float s = op.params[0];
            if (!(s >= 0.0f && s < CFS_MAX_TARGETS && s == std::floor(s)))
                return fail(CFS_ERR_INVALID_ARG, m.str() + "splat slot must be 0..3");
            ++n_splat;
        }
        dim = op_out_dim(op.kind, dim);
    }
    cfs_chain* c = new (std::nothrow) cfs_chain();
    if (!c) return fail(CFS_ERR_OOM, "host allocation failed");
    c->dim_in = dim_in;
    c->n_ops = n_ops;
    c->flags = flags;
    for (int o = 0; o < n_ops; ++o) c->ops[o] = ops[o];
    c->n_splat = n_splat;
    refresh_exec_ops(c);
    *out = c;
    return CFS_OK;
}

cfs_status cfs_chain_destroy(cfs_chain* chain)
{
    delete chain;
    return CFS_OK;
}

cfs_status cfs_chain_info(const cfs_chain* chain, int* dim_in, int* n_ops, int* n_splat)
{
    clear_error();
    if (!chain) return fail(CFS_ERR_INVALID_ARG, "NULL chain");
    if (dim_in) *dim_in = chain->dim_in;
    if (n_ops) *n_ops = chain->n_ops;
    if (n_splat) *n_splat = chain->n_splat;
    return CFS_OK;
}

cfs_status cfs_compose_scribble(int dim_in, const char* source, const char* poem, uint32_t flags,
                                cfs_chain** out)
{
    clear_error();
    if (!out) return fail(CFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dim_in != 2 && dim_in != 3) return fail(CFS_ERR_INVALID_ARG, "dim_in must be 2 or 3");
    if (!source || !poem) return fail(CFS_ERR_INVALID_ARG, "NULL source or poem name");
    if ((flags & ~(uint32_t)CFS_COMPOSE_FAST_TRIG) != 0)
        return fail(CFS_ERR_INVALID_ARG, "unknown flags");
    std::string body;
    std::vector<int> slots;
    cfs_status st = scribble_expand(source, poem, &body, &slots);
    if (st != CFS_OK) return st;
    cfs_chain* c = new (std::nothrow) cfs_chain();
    if (!c) return fail(CFS_ERR_OOM, "host allocation failed");
    c->dim_in = dim_in;
    c->n_ops = 0;
    c->flags = flags;
    c->n_splat = (int)slots.size();
    c->scribble = body;
    c->scribble_slots = slots;
    *out = c;
    return CFS_OK;
}

cfs_status cfs_chain_set_params(cfs_chain* chain, int index, const float* params)
{
    clear_error();
    if (!chain || !params) return fail(CFS_ERR_INVALID_ARG, "NULL chain or params");
    if (index < 0 || index >= chain->n_ops) return fail(CFS_ERR_INVALID_ARG, "index out of range");
    if (!finite_all(params, CFS_OP_PARAMS))
        return fail(CFS_ERR_INVALID_ARG, "parameters must be finite");
    cfs_transform t = chain->ops[index];
    std::memcpy(t.params, params, sizeof(t.params));
    if (t.kind == CFS_OP_SPLAT && t.params[0] != chain->ops[index].params[0])
        return fail(CFS_ERR_INVALID_ARG, "a SPLAT's slot cannot change");
    if ((t.kind == CFS_OP_BANDS && t.params[0] != chain->ops[index].params[0]) ||
        (t.kind == CFS_OP_ROTATE3 && t.params[1] != chain->ops[index].params[1]))
        return fail(CFS_ERR_INVALID_ARG, "an op's axis is part of the compiled program");
    if (t.kind == CFS_OP_BEND && t.params[0] == 0.0f)
        return fail(CFS_ERR_INVALID_ARG, "bend needs a nonzero curvature");
    {
        // the op's input dimension is that of the chain up to it
        int dim = chain->dim_in;
        for (int o = 0; o < index; ++o)
            dim = chain->ops[o].kind == CFS_OP_RESET ? chain->dim_in
                                                      : op_out_dim(chain->ops[o].kind, dim);
        std::string why;
        if (!op_params_ok(t, dim, &why)) return fail(CFS_ERR_INVALID_ARG, why);
    }
    chain->ops[index] = t;
    refresh_exec_ops(chain);
    return CFS_OK;
}

cfs_status cfs_prepare(const cfs_system* sys, const cfs_chain* chain, const cfs_target* targets,
                       int n_targets)
{
    clear_error();
    if (!sys || !chain) return fail(CFS_ERR_INVALID_ARG, "NULL system or chain");
    if (chain->dim_in != sys->dim)
        return fail(CFS_ERR_INVALID_ARG, "chain was composed for another dimension");
    cfs_status st = validate_targets(chain, targets, n_targets);
    if (st != CFS_OK) return st;
    ProgramSpec sp = make_spec(Mode::Render, sys, chain, targets, n_targets, false);
    Kernel k;
    return get_kernel(sp, "cfs_render_kernel", &k);
}

cfs_status cfs_render(const cfs_system* sys, const cfs_chain* chain,
                      const cfs_render_params* params, const cfs_target* targets, int n_targets,
                      void* stream)
{
    clear_error();
    cfs_status st = validate_run(sys, chain, params);
    if (st != CFS_OK) return st;
    st = validate_targets(chain, targets, n_targets);
    if (st != CFS_OK) return st;
    if (params->n_points == 0 || params->step_begin >= params->iters) return CFS_OK;
    ProgramSpec sp = make_spec(Mode::Render, sys, chain, targets, n_targets,
                               (params->flags & CFS_FLAG_REUSE) != 0);
    Kernel k;
    st = get_kernel(sp, "cfs_render_kernel", &k);
    if (st != CFS_OK) return st;
    cfs_launch_args a;
    fill_args(&a, sys, chain, targets, n_targets, params);
    const uint64_t blocks_needed = ((uint64_t)params->n_points + k.block - 1) / k.block;
    uint64_t grid = (uint64_t)k.max_blocks_per_sm * (uint64_t)(k.num_sms > 0 ? k.num_sms : 1);
    if (grid == 0) grid = 1;
    if (grid > blocks_needed) grid = blocks_needed;
    return launch(k, (unsigned)grid, &a, sizeof(a), (cudaStream_t)stream);
}

cfs_status cfs_trace(const cfs_system* sys, const cfs_chain* chain,
                     const cfs_render_params* params, const uint32_t* ids, uint32_t n_ids,
                     int32_t* k_out, float* p_out, float* q_out, void* stream)
{
    clear_error();
    cfs_status st = validate_run(sys, chain, params);
    if (st != CFS_OK) return st;
    if (n_ids == 0 || params->step_begin >= params->iters) return CFS_OK;
    if (!ids || !k_out || !p_out || !q_out)
        return fail(CFS_ERR_INVALID_ARG, "NULL ids or trace output");
    // the trace splats nothing: targets are only needed for their kinds
    ProgramSpec sp = make_spec(Mode::Trace, sys, chain, nullptr, 0,
                               (params->flags & CFS_FLAG_REUSE) != 0);
    Kernel k;
    st = get_kernel(sp, "cfs_trace_kernel", &k);
    if (st != CFS_OK) return st;
    cfs_launch_args a;
    cfs_render_params p = *params;
    p.n_points = n_ids;
    p.discards = nullptr;
    fill_args(&a, sys, chain, nullptr, 0, &p);
    a.ids = (unsigned long long)(uintptr_t)ids;
    a.k_out = (unsigned long long)(uintptr_t)k_out;
    a.p_out = (unsigned long long)(uintptr_t)p_out;
    a.q_out = (unsigned long long)(uintptr_t)q_out;
    const unsigned grid = (n_ids + k.block - 1) / k.block;
    return launch(k, grid, &a, sizeof(a), (cudaStream_t)stream);
}

cfs_status cfs_pointcloud_generate(const cfs_system* sys, uint64_t seed, uint32_t system_id,
                                   uint32_t n, uint32_t iters, float* xyz, uint8_t* fn,
                                   void* stream)
{
    clear_error();
    if (!sys) return fail(CFS_ERR_INVALID_ARG, "NULL system");
    if (n == 0) return CFS_OK;
    if (!xyz || !fn) return fail(CFS_ERR_INVALID_ARG, "NULL xyz or fn");
    if (iters == 0) return fail(CFS_ERR_INVALID_ARG, "iters must be >= 1");
    cfs_chain empty;
    empty.dim_in = sys->dim;
    empty.n_ops = 0;
    ProgramSpec sp = make_spec(Mode::Cloud, sys, &empty, nullptr, 0, false);
    Kernel k;
    cfs_status st = get_kernel(sp, "cfs_cloud_kernel", &k);
    if (st != CFS_OK) return st;
    cfs_render_params p{};
    p.seed = seed;
    p.system_id = system_id;
    p.n_points = n;
    p.iters = iters;
    cfs_launch_args a;
    fill_args(&a, sys, &empty, nullptr, 0, &p);
    a.cloud_xyz = (unsigned long long)(uintptr_t)xyz;
    a.cloud_fn = (unsigned long long)(uintptr_t)fn;
    const uint64_t need = ((uint64_t)n + k.block - 1) / k.block;
    uint64_t grid = (uint64_t)k.max_blocks_per_sm * (uint64_t)(k.num_sms > 0 ? k.num_sms : 1);
    if (grid == 0) grid = 1;
    if (grid > need) grid = need;
    return launch(k, (unsigned)grid, &a, sizeof(a), (cudaStream_t)stream);
}

cfs_status cfs_render_points(const cfs_chain* chain, const float* xyz, const uint8_t* fn,
                             uint32_t n, const cfs_target* targets, int n_targets,
                             unsigned long long* discards, void* stream)
{
    clear_error();
    if (!chain) return fail(CFS_ERR_INVALID_ARG, "NULL chain");
    if (n == 0) return CFS_OK;
    if (!xyz || !fn) return fail(CFS_ERR_INVALID_ARG, "NULL xyz or fn");
    if (n % 4 != 0) return fail(CFS_ERR_INVALID_ARG, "n must be a multiple of 4");
    if ((uintptr_t)xyz % 16 != 0 || (uintptr_t)fn % 4 != 0)
        return fail(CFS_ERR_INVALID_ARG, "xyz must be 16-byte and fn 4-byte aligned");
    cfs_status st = validate_targets(chain, targets, n_targets);
    if (st != CFS_OK) return st;
    bool aux = chain->scribble.find("stars") != std::string::npos ||
               chain->scribble.find("aux") != std::string::npos;
    for (int o = 0; o < chain->n_ops; ++o) aux = aux || chain->ops[o].kind == CFS_OP_STARS;
    if (aux)
        return fail(CFS_ERR_UNSUPPORTED, "stars draw from the per-step random stream, which "
                                         "a stored cloud does not have");
    // the generator plays no part: a one-map stand-in of the chain's dimension
    cfs_system stand_in;
    stand_in.dim = chain->dim_in;
    stand_in.n_maps = 1;
    stand_in.maps[0].kind = CFS_MAP_AFFINE;
    std::memset(stand_in.maps[0].params, 0, sizeof(stand_in.maps[0].params));
    stand_in.n_cmp = 0;
    ProgramSpec sp = make_spec(Mode::Points, &stand_in, chain, targets, n_targets, false);
    Kernel k;
    st = get_kernel(sp, "cfs_points_kernel", &k);
    if (st != CFS_OK) return st;
    cfs_render_params p{};
    p.n_points = n;
    p.iters = 1;
    p.discards = discards;
    cfs_launch_args a;
    fill_args(&a, &stand_in, chain, targets, n_targets, &p);
    a.cloud_xyz = (unsigned long long)(uintptr_t)xyz;
    a.cloud_fn = (unsigned long long)(uintptr_t)fn;
    const uint64_t need = ((uint64_t)(n / 4) + k.block - 1) / k.block;
    uint64_t grid = (uint64_t)k.max_blocks_per_sm * (uint64_t)(k.num_sms > 0 ? k.num_sms : 1);
    if (grid == 0) grid = 1;
    if (grid > need) grid = need;
    return launch(k, (unsigned)grid, &a, sizeof(a), (cudaStream_t)stream);
}

cfs_status cfs_codegen_check(const cfs_system* sys, const cfs_chain* chain,
                             const cfs_target* targets, int n_targets, int mode, char* src,
                             size_t src_cap, char* log, size_t log_cap)
{
    clear_error();
    if (!sys || !chain) return fail(CFS_ERR_INVALID_ARG, "NULL system or chain");
    if (chain->dim_in != sys->dim)
        return fail(CFS_ERR_INVALID_ARG, "chain was composed for another dimension");
    if (mode < 0 || mode > 4) return fail(CFS_ERR_INVALID_ARG, "mode must be in 0..4");
    cfs_status st = CFS_OK;
    const bool tg = mode != 1 && mode != 3;
    if (tg) {
        st = validate_targets(chain, targets, n_targets);
        if (st != CFS_OK) return st;
    }
    const Mode modes[] = {Mode::Render, Mode::Trace, Mode::Batch, Mode::Cloud, Mode::Points};
    ProgramSpec sp = make_spec(modes[mode], sys, chain, tg ? targets : nullptr,
                               tg ? n_targets : 0, false);
    if (mode == 2) {
        for (int k = 0; k < sys->n_maps; ++k)
            if (sys->maps[k].kind != sys->maps[0].kind)
                return fail(CFS_ERR_UNSUPPORTED, "a batch needs maps of one kind");
        sp.n_maps = CFS_MAX_MAPS;
        for (int j = 0; j < CFS_MAX_MAPS; ++j) sp.map_kind[j] = sys->maps[0].kind;
        batch_spec_defaults(sp);
    }
    std::string s, l;
    st = compile_only(sp, &s, &l);
    auto copy = [](const std::string& from, char* to, size_t cap) {
        if (!to || cap == 0) return;
        const size_t n = from.size() < cap - 1 ? from.size() : cap - 1;
        std::memcpy(to, from.data(), n);
        to[n] = '\0';
    };
    copy(s, src, src_cap);
    copy(l, log, log_cap);
    return st;
}

cfs_status cfs_target_clear(const cfs_target* targets, int n_targets, void* stream)
{
    clear_error();
    if (n_targets < 0 || n_targets > CFS_MAX_TARGETS || (n_targets > 0 && !targets))
        return fail(CFS_ERR_INVALID_ARG, "bad targets");
    for (int t = 0; t < n_targets; ++t) {
        const cfs_target& g = targets[t];
        if (!g.data || g.width <= 0 || g.height <= 0)
            return fail(CFS_ERR_INVALID_ARG, "bad target");
        size_t n = (size_t)g.width * (size_t)g.height;
        int fill = 0;
        if (g.kind == CFS_TARGET_HIST_U32) n *= 4 * (size_t)(g.channels < 1 ? 1 : g.channels);
        else if (g.kind == CFS_TARGET_RGBA_F32) n *= 16;
        else if (g.kind == CFS_TARGET_DEPTH_U64) { n *= 8; fill = 0xFF; }
        else return fail(CFS_ERR_INVALID_ARG, "unknown target kind");
        cfs_status st = check_cuda(cudaMemsetAsync(g.data, fill, n, (cudaStream_t)stream),
                                   "cudaMemsetAsync");
        if (st != CFS_OK) return st;
    }
    return CFS_OK;
}

}  // extern "C"
