// cfs_internal.h -- host-side internals of libcfs (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "cfs.h"
#include "cfs_args.h"

struct cfs_system {
    int dim = 2;
    int n_maps = 0;
    cfs_map maps[CFS_MAX_MAPS];
    double probs[CFS_MAX_MAPS];
    uint32_t T[CFS_MAX_MAPS];   // thresholds below 2^32
    int n_cmp = 0;              // how many of them count
};

struct cfs_chain {
    int dim_in = 2;
    int n_ops = 0;
    uint32_t flags = 0;         // CFS_COMPOSE_*
    cfs_transform ops[CFS_MAX_OPS];
    // the ops the kernels run: `ops`, or with CFS_COMPOSE_FOLD_LINEAR every
    // run of consecutive linear ops folded into one affine op
    int n_xops = 0;
    cfs_transform xops[CFS_MAX_OPS];
    int n_splat = 0;
    // a chain written as a scribble poem (cfs_compose_scribble): the expanded
    // body with CFS_SCRIBBLE_SPLAT_i() for the i-th splat call, and its slots
    std::string scribble;
    std::vector<int> scribble_slots;
};

namespace cfs {

// ---- error reporting (thread-local message) -------------------------------
cfs_status fail(cfs_status s, const std::string& msg);
void clear_error();

// ---- structural description of one generated program ----------------------
enum class Mode { Render = 0, Trace = 1, Cloud = 2, Points = 3, Batch = 4 };

struct SplatSpec {
    int slot;        // target slot
    int kind;        // cfs_target_kind
    int channels;    // histogram channel count
};

struct ProgramSpec {
    Mode mode = Mode::Render;
    int dim = 2;
    int n_maps = 1;
    int map_kind[CFS_MAX_MAPS] = {};
    int n_cmp = 0;
    bool reuse = false;
    int n_ops = 0;
    int op_kind[CFS_MAX_OPS] = {};
    int op_axis[CFS_MAX_OPS] = {};   // rotate3: 0 x, 1 y, 2 z
    std::vector<SplatSpec> splats;   // in op order
    int n_targets = 0;
    int depth_test = 1;
    int block = 256;
    int min_blocks = 8;        // upper bound; lowered while ptxas spills
    int spill_allowance = 0;   // bytes of spill stores accepted at min_blocks
    int tile = 0;              // batch: privatized shared window for the first splat
    int warp_agg = 0;          // warp-aggregated shared atomics in that window
    int fast_trig = 0;         // chain trigonometry: 0 libm, 1 reduced argument + hardware
    int unroll = 4;            // copies of the step code in the step loop (4, 2, 1)
    int ilp = 1;               // batch: trajectories stepped together per thread (1, 2)
    int dyn_smem = 0;          // dynamic shared memory per CTA (bytes)
    std::string scribble;      // expanded poem body (empty: the op list)

    std::string key() const;
};

std::string generate_source(const ProgramSpec& spec);
// chain trigonometry of compose flags: 0 CUDA libm, 1 reduced argument + hardware
int trig_mode(uint32_t flags);

// ---- runtime: driver entry points, NVRTC, module cache ---------------------
struct Kernel {
    void* fn = nullptr;         // CUfunction
    int max_blocks_per_sm = 0;
    int block = 256;
    int num_sms = 0;
    int dyn_smem = 0;     // dynamic shared memory per CTA at launch (bytes)
};

// Compiles (or fetches from the cache) the program and returns the named
// kernel.  Thread-safe.
cfs_status get_kernel(const ProgramSpec& spec, const char* name, Kernel* out);
// NVRTC only (no GPU needed): generated source and compiler log with the
// ptxas resource usage.
cfs_status compile_only(const ProgramSpec& spec, std::string* src, std::string* log);
cfs_status launch(const Kernel& k, unsigned grid, const void* args, size_t args_size,
                  cudaStream_t stream);
cfs_status check_cuda(cudaError_t e, const char* what);
int device_sm_count();
// 2D tensor map (TMA) of a BF16 matrix [rows][cols], row stride ld elements,
// box_rows x box_cols boxes, no swizzle, zeros outside (cfs_runtime.cpp)
cfs_status make_tmap_2d_bf16(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                             uint64_t ld, uint32_t box_cols, uint32_t box_rows);

// Expands poem `poem` of a scribble program into a chain body; splat(N)
// calls become CFS_SCRIBBLE_SPLAT_i() with their slots in splat_slots.
cfs_status scribble_expand(const std::string& source, const std::string& poem, std::string* body,
                           std::vector<int>* splat_slots);

// Launch shape of the persistent batch program under the default plan
// (block, occupancy, privatized window, warp aggregation, ILP); returns the
// window's capacity in u32 counters and sets dyn_smem.
uint32_t batch_spec_defaults(ProgramSpec& sp);

// ---- density-estimation display (cfs_display.cu) ---------------------------
// One layer as the display kernels read it.  Work is cut into items of
// kDisplayPxPerItem pixels numbered layer by layer from item_begin.
constexpr uint32_t kDisplayPxPerItem = 8192;
struct DisplayLayer {
    unsigned long long data;   // device pointer of the layer
    unsigned long long out;    // device u32 [H][W]
    uint32_t n_px;             // W * H
    int32_t kind, C;           // cfs_target_kind, histogram channels
    uint32_t item_begin;
    float pal[CFS_MAX_MAPS][4];
};
// Checks display parameters (gamma, brightness > 0, finite a_max).
cfs_status display_params_check(const cfs_display_params* p);
// Checks a layer description and its output for the display calls.
cfs_status display_check(const cfs_target& t, const void* out, const char* what);
// Fills d from a target; returns the layer's work items.
uint32_t display_fill(const cfs_target& t, uint32_t* out, uint32_t item_begin, DisplayLayer* d);
// Enqueues the maximum (when params.a_max <= 0 and some layer is not a depth
// layer; a_max is zeroed first) and mapping kernels over n_items items.
// Either `one` (a single layer, by value) or `layers` (device array) is used.
cfs_status display_enqueue(const DisplayLayer* one, const DisplayLayer* layers, int n_layers,
                           uint32_t n_items, bool any_density, float* a_max,
                           const cfs_display_params& p, cudaStream_t stream);

// ---- device-side error flags (cfs_sampler.cu) ----------------------------
// Bits of the current device's error word, set by kernels whose bounded
// waits ran out (CFS_DEVICE_ERR_* in cfs.h).  take_: reads and clears it;
// raise_: ORs bits into it (tests of the reporting path).
cfs_status take_device_flags(unsigned int* flags);
cfs_status raise_device_flags(unsigned int flags);

// Recomputes chain->xops from chain->ops (after compose and set_params).
void refresh_exec_ops(cfs_chain* chain);

// ---- host-side tables ---------------------------------------------------
void philox_round_keys(uint64_t seed, unsigned int rk[10][2]);
// per-op constants the kernels read (rotations turned into affine params, ...)
void derive_op_params(const cfs_transform& op, float out[CFS_OP_PARAMS]);

}  // namespace cfs
