// cfs_codegen.cpp -- emits the fused generator + transform-chain program.
//
// The paper's renderer composes user functions into one large kernel so that
// no map or transform is called through a function pointer (Section 1,
// Section 2; Fig. 3 shows its verse/stanza injection).  Here the same idea is
// applied to CUDA: from the structure of a render -- generator map kinds,
// the chain's op sequence, the kinds of the targets it splats into -- this
// file writes straight-line device code (a switch only where maps of
// different kinds meet) that NVRTC compiles for sm_103a.  Every numeric
// parameter stays in the kernel's argument block, so one compiled program
// serves every system and chain of the same structure.
#include <cstdlib>
#include <sstream>

#include "cfs_internal.h"

namespace cfs {

int trig_mode(uint32_t flags) { return (flags & CFS_COMPOSE_FAST_TRIG) ? 1 : 0; }

std::string ProgramSpec::key() const
{
    std::ostringstream s;
    s << "m" << int(mode) << ".d" << dim << ".n" << n_maps << ".c" << n_cmp << ".r" << reuse
      << ".t" << n_targets << ".z" << depth_test << ".b" << block << "." << min_blocks << "."
      << spill_allowance << ".p" << tile << warp_agg << ".f" << fast_trig
      << ".u" << unroll << ".i" << ilp << ".k";
    for (int j = 0; j < n_maps; ++j) s << map_kind[j];
    s << ".o";
    for (int j = 0; j < n_ops; ++j) {
        const bool ax = op_kind[j] == CFS_OP_ROTATE3 || op_kind[j] == CFS_OP_BANDS;
        s << op_kind[j] << (ax ? "r" : "") << (ax ? op_axis[j] : 0) << ",";
    }
    s << ".s";
    for (const auto& sp : splats) s << sp.slot << ":" << sp.kind << ":" << sp.channels << ",";
    if (!scribble.empty()) {
        // FNV-1a of the expanded poem: one program per distinct text
        uint64_t h = 1469598103934665603ull;
        for (unsigned char c : scribble) h = (h ^ c) * 1099511628211ull;
        s << ".q" << std::hex << h << std::dec << "." << scribble.size();
    }
    return s.str();
}

static std::string P(int o, int j)
{
    std::ostringstream s;
    s << "a.op[" << o << "][" << j << "]";
    return s.str();
}

static std::string Plist(int o, int n)
{
    std::ostringstream s;
    for (int j = 0; j < n; ++j) s << P(o, j) << ", ";
    return s.str();
}

// Generator: one map evaluation for map index k.
static void emit_gen_map(std::ostringstream& s, const ProgramSpec& sp)
{
    s << "__device__ __forceinline__ void cfs_gen_map(const cfs_launch_args& a, int k, float& x,"
         " float& y, float& z, const CfsSmem& sm)\n{\n    (void)a; (void)sm;\n";
    bool all_affine = true, all_circle = true;
    for (int j = 0; j < sp.n_maps; ++j) {
        all_affine = all_affine && sp.map_kind[j] == CFS_MAP_AFFINE;
        all_circle = all_circle && sp.map_kind[j] == CFS_MAP_CIRCLE;
    }
    if (all_affine) {
        // one code path for every map: parameters gathered from shared memory
        if (sp.dim == 2)
            s << "    cfs_affine2_tab(k, x, y, sm);\n    (void)z;\n";
        else
            s << "    cfs_affine3_tab(k, x, y, z, sm);\n";
    } else if (all_circle) {
        s << "    cfs_circle(sm.prm4[0][k].x, x, y);\n    (void)z;\n";
    } else {
        // maps of different kinds: the fused switch
        s << "    switch (k) {\n";
        for (int j = 0; j < sp.n_maps; ++j) {
            s << "    case " << j << ": ";
            if (sp.map_kind[j] == CFS_MAP_AFFINE) {
                if (sp.dim == 2)
                    s << "cfs_affine2(a_sys_prm(0, " << j << "), a_sys_prm(1, " << j
                      << "), a_sys_prm(2, " << j << "), a_sys_prm(3, " << j
                      << "), a_sys_prm(4, " << j << "), a_sys_prm(5, " << j << "), x, y);";
                else {
                    s << "cfs_affine3(";
                    for (int q = 0; q < 12; ++q) s << "a_sys_prm(" << q << ", " << j << "), ";
                    s << "x, y, z);";
                }
            } else {
                s << "cfs_circle(a_sys_prm(0, " << j << "), x, y);";
            }
            s << " break;\n";
        }
        s << "    default: break;\n    }\n";
    }
    s << "}\n\n";
}

// Chain: the copy of the point through every op, splats where the chain says.
// splat of the current point into target t (record index si for traces)
static void emit_splat(std::ostringstream& s, const ProgramSpec& sp, size_t si)
{
    const SplatSpec& t = sp.splats[si];
    s << "if (rec) { rec[" << 4 * si << "] = qx; rec[" << 4 * si + 1 << "] = qy; rec["
      << 4 * si + 2 << "] = qz; rec[" << 4 * si + 3 << "] = alive ? 1.0f : 0.0f; } ";
    s << "if (do_splat) ";
    if (t.kind == CFS_TARGET_HIST_U32 && sp.tile && si == 0)
        s << "cfs_splat_hist_tile(tg[" << t.slot << "], tile, qx, qy, alive, kc % " << t.channels
          << ", disc[" << t.slot << "]);";
    else if (t.kind == CFS_TARGET_HIST_U32)
        s << "cfs_splat_hist(tg[" << t.slot << "], qx, qy, alive, kc % " << t.channels
          << ", disc[" << t.slot << "]);";
    else if (t.kind == CFS_TARGET_RGBA_F32)
        s << "cfs_splat_rgba(tg[" << t.slot << "], qx, qy, alive, sm.pal[" << t.slot
          << "][kc], disc[" << t.slot << "]);";
    else
        s << "cfs_splat_depth(tg[" << t.slot << "], qx, qy, qz, alive, sm.pal8[" << t.slot
          << "][kc], disc[" << t.slot << "]);";
}

// A chain written as a scribble poem: the expanded text between the same
// prologue and epilogue, with the library's ops as local functions.
static void emit_scribble_chain(std::ostringstream& s, const ProgramSpec& sp)
{
    s << "template <class TG>\n__device__ __forceinline__ bool cfs_chain(const cfs_launch_args& a,"
         " const TG& tg, const CfsSmem& sm, float px, float py, float pz, int k, u32 aux,"
         " u32* disc, bool do_splat, float* rec, float& ox, float& oy, float& oz,"
         " const CfsTile& tile)\n{\n";
    s << "    (void)tile; (void)aux; (void)a; (void)tg; (void)sm; (void)disc; (void)do_splat;"
         " (void)rec;\n";
    s << "    float qx = px, qy = py, qz = pz;\n    bool alive = true;\n    int kc = k;\n";
    s << R"(    auto reset = [&]() { qx = px; qy = py; qz = pz; alive = true; kc = k; };
    auto discard = [&]() { alive = false; };
    auto affine2 = [&](float a0, float b0, float c0, float d0, float e0, float f0) {
        cfs_affine2(a0, b0, c0, d0, e0, f0, qx, qy); };
    auto rotate2 = [&](float ang) {
        const float c = (float)cos((double)ang), sn = (float)sin((double)ang);
        cfs_affine2(c, -sn, sn, c, 0.0f, 0.0f, qx, qy); };
    auto rotate3 = [&](float ang, int axis) {
        const float c = (float)cos((double)ang), sn = (float)sin((double)ang);
        if (axis == 0) cfs_rotate3_0(1.0f, 0.0f, 0.0f, 0.0f, c, -sn, 0.0f, sn, c, 0.0f, 0.0f, 0.0f, qx, qy, qz);
        else if (axis == 1) cfs_rotate3_1(c, 0.0f, sn, 0.0f, 1.0f, 0.0f, -sn, 0.0f, c, 0.0f, 0.0f, 0.0f, qx, qy, qz);
        else cfs_rotate3_2(c, -sn, 0.0f, sn, c, 0.0f, 0.0f, 0.0f, 1.0f, 0.0f, 0.0f, 0.0f, qx, qy, qz); };
    auto translate3 = [&](float x0, float y0, float z0) {
        qx = qx + x0; qy = qy + y0; qz = qz + z0; };
    auto swirl = [&]() { cfs_swirl(qx, qy); };
    auto sinusoidal = [&]() { cfs_sinusoidal(qx, qy); };
    auto sinusoidal3 = [&]() { cfs_sinusoidal3(qx, qy, qz); };
    auto stretch = [&]() { cfs_stretch(qx, qy); };
    auto torus = [&](float R, float r) { cfs_torus(R, r, qx, qy, qz); };
    auto perspective = [&](float f, float nz) {
        alive = cfs_perspective(f, nz, qx, qy, qz) && alive; };
    auto twist_z = [&](float kap) { cfs_twist_z(kap, qx, qy, qz); };
    auto bend = [&](float beta) { cfs_bend(beta, 1.0f / beta, qx, qz); };
    auto inversion = [&](float cx, float cy, float cz, float rho) {
        alive = cfs_inversion(cx, cy, cz, rho * rho, qx, qy, qz) && alive; };
    auto hemisphere = [&](float R) { cfs_hemisphere(R, qx, qy, qz); };
    auto bands = [&](int axis, float freq, float phase, int n, int base) {
        kc = cfs_bands(axis == 0 ? qx : (axis == 1 ? qy : qz), freq, phase, n, base); };
    auto stars = [&](unsigned n, float x0, float x1, float y0, float y1, float z0, float z1,
                     float s0, float s1) {
        cfs_stars(a, n, x0, x1 - x0, y0, y1 - y0, z0, z1 - z0, s0, s1 - s0, aux, qx, qy, qz); };
    (void)reset; (void)discard; (void)affine2; (void)rotate2; (void)rotate3; (void)translate3;
    (void)swirl;
    (void)sinusoidal; (void)sinusoidal3; (void)stretch; (void)torus; (void)perspective;
    (void)twist_z; (void)bend; (void)inversion; (void)hemisphere; (void)bands; (void)stars;
)";
    for (size_t si = 0; si < sp.splats.size(); ++si) {
        s << "#define CFS_SCRIBBLE_SPLAT_" << si << "() { ";
        emit_splat(s, sp, si);
        s << " }\n";
    }
    s << "    {\n" << sp.scribble << "\n    }\n";
    for (size_t si = 0; si < sp.splats.size(); ++si) s << "#undef CFS_SCRIBBLE_SPLAT_" << si << "\n";
    s << "    ox = qx; oy = qy; oz = qz;\n    return alive;\n}\n\n";
}

// index of the op chain's first duplication op (-1: none or a scribble chain)
static int first_stars_op(const ProgramSpec& sp)
{
    if (!sp.scribble.empty()) return -1;
    for (int o = 0; o < sp.n_ops; ++o)
        if (sp.op_kind[o] == CFS_OP_STARS) return o;
    return -1;
}

// per-CTA setup of the chain, run by every kernel before its first barrier:
// the first duplication op's star table
static void emit_chain_prologue(std::ostringstream& s, const ProgramSpec& sp)
{
    s << "__device__ __forceinline__ void cfs_chain_prologue(const cfs_launch_args& a, CfsSmem& sm)"
         "\n{\n    (void)a; (void)sm;\n";
    const int o = first_stars_op(sp);
    if (o >= 0) {
        s << "    const u32 n_ = min(__float_as_uint(" << P(o, 0) << "), (u32)CFS_STARS_TAB);\n"
          << "    for (u32 j = threadIdx.x; j < n_; j += blockDim.x)\n"
          << "        sm.stars[j] = cfs_star_centre(a, j, " << P(o, 1) << ", " << P(o, 2) << ", "
          << P(o, 3) << ", " << P(o, 4) << ", " << P(o, 5) << ", " << P(o, 6) << ", "
          << P(o, 7) << ", " << P(o, 8) << ");\n";
    }
    s << "}\n\n";
}

static void emit_chain(std::ostringstream& s, const ProgramSpec& sp)
{
    if (!sp.scribble.empty()) {
        emit_scribble_chain(s, sp);
        return;
    }
    s << "template <class TG>\n__device__ __forceinline__ bool cfs_chain(const cfs_launch_args& a,"
         " const TG& tg, const CfsSmem& sm, float px, float py, float pz, int k, u32 aux,"
         " u32* disc, bool do_splat, float* rec, float& ox, float& oy, float& oz,"
         " const CfsTile& tile)\n{\n";
    s << "    (void)tile; (void)aux;\n";
    s << "    float qx = px, qy = py, qz = pz;\n    bool alive = true;\n";
    s << "    int kc = k;   /* the branch's colour index */\n";
    s << "    (void)a; (void)tg; (void)sm; (void)disc; (void)do_splat; (void)rec; (void)kc;\n";
    size_t si = 0;
    for (int o = 0; o < sp.n_ops; ++o) {
        s << "    /* op " << o << " */ ";
        switch (sp.op_kind[o]) {
        case CFS_OP_AFFINE2:
        case CFS_OP_ROTATE2:
            s << "cfs_affine2(" << Plist(o, 6) << "qx, qy);\n";
            break;
        case CFS_OP_AFFINE3:
            s << "cfs_affine3(" << Plist(o, 12) << "qx, qy, qz);\n";
            break;
        case CFS_OP_ROTATE3:
            // the affine evaluation with the zero entries dropped: the same
            // roundings (only the sign of an exact zero can differ)
            s << "cfs_rotate3_" << sp.op_axis[o] << "(" << Plist(o, 12) << "qx, qy, qz);\n";
            break;
        case CFS_OP_TRANSLATE3:
            s << "qx = qx + " << P(o, 9) << "; qy = qy + " << P(o, 10) << "; qz = qz + "
              << P(o, 11) << ";\n";
            break;
        case CFS_OP_SWIRL: s << "cfs_swirl(qx, qy);\n"; break;
        case CFS_OP_SINUSOIDAL: s << "cfs_sinusoidal(qx, qy);\n"; break;
        case CFS_OP_SINUSOIDAL3: s << "cfs_sinusoidal3(qx, qy, qz);\n"; break;
        case CFS_OP_STRETCH: s << "cfs_stretch(qx, qy);\n"; break;
        case CFS_OP_TORUS: s << "cfs_torus(" << Plist(o, 2) << "qx, qy, qz);\n"; break;
        case CFS_OP_PERSPECTIVE:
            s << "alive = cfs_perspective(" << Plist(o, 2) << "qx, qy, qz) && alive;\n";
            break;
        case CFS_OP_TWIST_Z: s << "cfs_twist_z(" << P(o, 0) << ", qx, qy, qz);\n"; break;
        case CFS_OP_BEND: s << "cfs_bend(" << Plist(o, 2) << "qx, qz);\n"; break;
        case CFS_OP_INVERSION:
            s << "alive = cfs_inversion(" << Plist(o, 4) << "qx, qy, qz) && alive;\n";
            break;
        case CFS_OP_STARS:
            if (o == first_stars_op(sp)) {
                // the table of cfs_chain_prologue when it holds every star
                s << "{ const u32 n_ = __float_as_uint(" << P(o, 0) << "); const u32 j_ = "
                  << "__umulhi(aux, n_); cfs_star_place(n_ <= CFS_STARS_TAB ? sm.stars[j_] : "
                  << "cfs_star_centre(a, j_, " << P(o, 1) << ", " << P(o, 2)
                  << ", " << P(o, 3) << ", " << P(o, 4) << ", " << P(o, 5) << ", " << P(o, 6)
                  << ", " << P(o, 7) << ", " << P(o, 8) << "), qx, qy, qz); }\n";
            } else {
                s << "cfs_stars(a, __float_as_uint(" << P(o, 0) << "), " << P(o, 1) << ", "
                  << P(o, 2) << ", " << P(o, 3) << ", " << P(o, 4) << ", " << P(o, 5) << ", "
                  << P(o, 6) << ", " << P(o, 7) << ", " << P(o, 8) << ", aux, qx, qy, qz);\n";
            }
            break;
        case CFS_OP_HEMISPHERE:
            s << "cfs_hemisphere(" << P(o, 0) << ", qx, qy, qz);\n";
            break;
        case CFS_OP_BANDS: {
            const char* coord = sp.op_axis[o] == 0 ? "qx" : (sp.op_axis[o] == 1 ? "qy" : "qz");
            s << "kc = cfs_bands(" << coord << ", " << P(o, 1) << ", " << P(o, 2) << ", (int)"
              << P(o, 3) << ", (int)" << P(o, 4) << ");\n";
            break;
        }
        case CFS_OP_RESET:
            s << "qx = px; qy = py; qz = pz; alive = true; kc = k;\n";
            break;
        case CFS_OP_SPLAT: {
            const SplatSpec& t = sp.splats[si];
            s << "\n    if (rec) { rec[" << 4 * si << "] = qx; rec[" << 4 * si + 1
              << "] = qy; rec[" << 4 * si + 2 << "] = qz; rec[" << 4 * si + 3
              << "] = alive ? 1.0f : 0.0f; }\n";
            s << "    if (do_splat) ";
            if (t.kind == CFS_TARGET_HIST_U32 && sp.tile && si == 0)
                s << "cfs_splat_hist_tile(tg[" << t.slot << "], tile, qx, qy, alive, kc % "
                  << t.channels << ", disc[" << t.slot << "]);\n";
            else if (t.kind == CFS_TARGET_HIST_U32)
                s << "cfs_splat_hist(tg[" << t.slot << "], qx, qy, alive, kc % " << t.channels
                  << ", disc[" << t.slot << "]);\n";
            else if (t.kind == CFS_TARGET_RGBA_F32)
                s << "cfs_splat_rgba(tg[" << t.slot << "], qx, qy, alive, sm.pal[" << t.slot
                  << "][kc], disc[" << t.slot << "]);\n";
            else
                s << "cfs_splat_depth(tg[" << t.slot << "], qx, qy, qz, alive, sm.pal8["
                  << t.slot << "][kc], disc[" << t.slot << "]);\n";
            ++si;
            break;
        }
        default: s << "\n"; break;
        }
    }
    s << "    ox = qx; oy = qy; oz = qz;\n    return alive;\n}\n\n";
}

std::string generate_source(const ProgramSpec& sp)
{
    std::ostringstream s;
    s << "// generated: " << sp.key() << "\n";
    s << "#define CFS_DIM " << sp.dim << "\n";
    s << "#define CFS_NCMP " << sp.n_cmp << "\n";
    s << "#define CFS_NT " << sp.n_targets << "\n";
    s << "#define CFS_NSPLAT_ARR " << (sp.splats.empty() ? 1 : sp.splats.size()) << "\n";
    s << "#define CFS_REUSE " << (sp.reuse ? 1 : 0) << "\n";
    s << "#define CFS_FAST_TRIG " << sp.fast_trig << "\n";
    s << "#define CFS_UNROLL " << sp.unroll << "\n";
    s << "#define CFS_ILP " << (sp.ilp == 2 ? 2 : 1) << "\n";
    {
        bool aux = false;
        for (int o = 0; o < sp.n_ops; ++o) aux = aux || sp.op_kind[o] == CFS_OP_STARS;
        aux = aux || sp.scribble.find("stars") != std::string::npos ||
              sp.scribble.find("aux") != std::string::npos;
        s << "#define CFS_AUX " << (aux ? 1 : 0) << "\n";
    }
    s << "#define CFS_BATCH " << (sp.mode == Mode::Batch ? 1 : 0) << "\n";
    s << "#define CFS_CLOUD " << (sp.mode == Mode::Cloud ? 1 : 0) << "\n";
    s << "#define CFS_TILE " << (sp.tile ? 1 : 0) << "\n";
    s << "#define CFS_WARP_AGG " << (sp.warp_agg ? 1 : 0) << "\n";
    s << "#define CFS_TILE_C " << (sp.splats.empty() ? 1 : sp.splats[0].channels) << "\n";
    s << "#define CFS_POINTS " << (sp.mode == Mode::Points ? 1 : 0) << "\n";
    s << "#define CFS_DEPTH_TEST " << sp.depth_test << "\n";
    s << "#define CFS_BLOCK " << sp.block << "\n";
    s << "#define CFS_MINB " << sp.min_blocks << "\n";
    s << "#define CFS_STARS_TAB " << (first_stars_op(sp) >= 0 ? 512 : 0) << "\n";
    s << "#include \"cfs_device.cuh\"\n";
    // generator parameters with constant indices come straight from the
    // argument block (the constant bank); only the table path uses smem
    s << "#define a_sys_prm(j, k) (a.sys.prm[j][k])\n\n";
    emit_gen_map(s, sp);
    emit_chain_prologue(s, sp);
    emit_chain(s, sp);
    s << "#include \"cfs_kernels.cuh\"\n";
    return s.str();
}

}  // namespace cfs
