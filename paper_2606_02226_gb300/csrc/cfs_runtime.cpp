// cfs_runtime.cpp -- NVRTC compilation of generated programs, the program
// cache, and kernel launches.
//
// The driver API calls (module load, launch, occupancy) are reached through
// cudaGetDriverEntryPointByVersion, so the library links only the CUDA
// runtime and NVRTC and loads on machines without a GPU driver (where every
// compute entry point then reports CFS_ERR_CUDA).
#include <cuda.h>
#include <nvrtc.h>

#include <algorithm>
#include <cctype>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <sstream>
#include <unordered_map>

#include "cfs_internal.h"

namespace cfs {

// ---- embedded device sources (generated at build time from csrc/) --------
extern const char* const kSrcArgs;
extern const char* const kSrcDevice;
extern const char* const kSrcKernels;

// ---- error reporting ---------------------------------------------------------
static thread_local std::string t_err;

cfs_status fail(cfs_status s, const std::string& msg)
{
    t_err = msg;
    return s;
}

void clear_error() { t_err.clear(); }

const char* last_error() { return t_err.c_str(); }

cfs_status check_cuda(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return CFS_OK;
    std::ostringstream s;
    s << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
    return fail(e == cudaErrorMemoryAllocation ? CFS_ERR_OOM : CFS_ERR_CUDA, s.str());
}

// ---- driver entry points -------------------------------------------------
namespace {
typedef CUresult (*PFN_ModuleLoadData)(CUmodule*, const void*);
typedef CUresult (*PFN_ModuleGetFunction)(CUfunction*, CUmodule, const char*);
typedef CUresult (*PFN_LaunchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned,
                                     unsigned, unsigned, unsigned, CUstream, void**, void**);
typedef CUresult (*PFN_Occupancy)(int*, CUfunction, int, size_t);
typedef CUresult (*PFN_GetErrorString)(CUresult, const char**);
typedef CUresult (*PFN_FuncSetAttribute)(CUfunction, CUfunction_attribute, int);
typedef CUresult (*PFN_TensorMapEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                             const cuuint64_t*, const cuuint64_t*,
                                             const cuuint32_t*, const cuuint32_t*,
                                             CUtensorMapInterleave, CUtensorMapSwizzle,
                                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct Driver {
    PFN_ModuleLoadData module_load = nullptr;
    PFN_ModuleGetFunction get_function = nullptr;
    PFN_LaunchKernel launch = nullptr;
    PFN_Occupancy occupancy = nullptr;
    PFN_GetErrorString error_string = nullptr;
    PFN_FuncSetAttribute set_attribute = nullptr;
    PFN_TensorMapEncodeTiled encode_tiled = nullptr;
    bool ok = false;
    std::string why;
};

Driver& driver()
{
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        auto get = [](const char* name, void** fn) -> bool {
            cudaDriverEntryPointQueryResult q;
            cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q);
            return e == cudaSuccess && q == cudaDriverEntryPointSuccess && *fn != nullptr;
        };
        bool ok = get("cuModuleLoadData", (void**)&d.module_load) &&
                  get("cuModuleGetFunction", (void**)&d.get_function) &&
                  get("cuLaunchKernel", (void**)&d.launch) &&
                  get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void**)&d.occupancy) &&
                  get("cuGetErrorString", (void**)&d.error_string) &&
                  get("cuFuncSetAttribute", (void**)&d.set_attribute) &&
                  get("cuTensorMapEncodeTiled", (void**)&d.encode_tiled);
        d.ok = ok;
        if (!ok) d.why = "CUDA driver entry points unavailable (no GPU driver?)";
    });
    return d;
}

cfs_status check_cu(CUresult r, const char* what)
{
    if (r == CUDA_SUCCESS) return CFS_OK;
    const char* msg = "unknown";
    if (driver().error_string) driver().error_string(r, &msg);
    std::ostringstream s;
    s << what << ": CUresult " << int(r) << " (" << msg << ")";
    return fail(r == CUDA_ERROR_OUT_OF_MEMORY ? CFS_ERR_OOM : CFS_ERR_CUDA, s.str());
}

struct Program {
    CUmodule module = nullptr;
    int min_blocks = 0;
    std::unordered_map<std::string, Kernel> kernels;
};

std::mutex g_cache_mu;
// key: device ordinal + generated source text
std::unordered_map<std::string, std::unique_ptr<Program>> g_cache;

cfs_status compile(const std::string& src, std::vector<char>* cubin, std::string* log_out,
                   bool verbose)
{
    nvrtcProgram prog;
    const char* headers[] = {kSrcArgs, kSrcDevice, kSrcKernels};
    const char* names[] = {"cfs_args.h", "cfs_device.cuh", "cfs_kernels.cuh"};
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "cfs_generated.cu", 3, headers, names);
    if (r != NVRTC_SUCCESS)
        return fail(CFS_ERR_COMPILE, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
    const char* opts[] = {"--gpu-architecture=sm_103a", "--fmad=false", "--std=c++17",
                          "-default-device", "--extra-device-vectorization", "-lineinfo",
                          "--ptxas-options=-v"};
    const int n_opts = sizeof(opts) / sizeof(opts[0]) - (verbose ? 0 : 1);
    r = nvrtcCompileProgram(prog, n_opts, opts);
    {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        if (n) nvrtcGetProgramLog(prog, &log[0]);
        if (log_out) *log_out = log;
        if (r != NVRTC_SUCCESS) {
            nvrtcDestroyProgram(&prog);
            return fail(CFS_ERR_COMPILE,
                        std::string("NVRTC failed:\n") + log + "\n--- source ---\n" + src);
        }
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    cubin->resize(n);
    nvrtcGetCUBIN(prog, cubin->data());
    nvrtcDestroyProgram(&prog);
    return CFS_OK;
}
}  // namespace

// 2D tensor map of a BF16 matrix [rows][cols] (row stride ld elements), boxes
// of box_rows x box_cols elements, no swizzle, zero fill outside the matrix
cfs_status make_tmap_2d_bf16(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                             uint64_t ld, uint32_t box_cols, uint32_t box_rows)
{
    Driver& d = driver();
    if (!d.ok) return fail(CFS_ERR_CUDA, d.why);
    if (((uintptr_t)base & 15u) || ((ld * 2) & 15u) || ((box_cols * 2) & 15u))
        return fail(CFS_ERR_INVALID_ARG, "tensor map: base, row stride and box width must be "
                                         "multiples of 16 bytes");
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return check_cu(d.encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE),
                    "cuTensorMapEncodeTiled");
}

int spill_bytes(const std::string& log)
{
    int worst = 0;
    const std::string tag = " bytes spill stores";
    for (size_t p = log.find(tag); p != std::string::npos; p = log.find(tag, p + 1)) {
        size_t b = p;
        while (b > 0 && std::isdigit((unsigned char)log[b - 1])) --b;
        worst = std::max(worst, std::atoi(log.c_str() + b));
    }
    return worst;
}

// Occupancy search: compile at the spec's blocks/SM; while ptxas reports more
// spill bytes than the spec allows, try fewer blocks per SM (more registers).
cfs_status select_and_compile(const ProgramSpec& spec, std::string* src, std::vector<char>* cubin,
                              std::string* log, int* chosen_min_blocks)
{
    const int cands[] = {spec.min_blocks, 6, 4, 2};
    cfs_status st = CFS_OK;
    int last = -1;
    for (int c : cands) {
        if (c > spec.min_blocks || c == last) continue;
        last = c;
        ProgramSpec sp = spec;
        sp.min_blocks = c;
        *src = generate_source(sp);
        st = compile(*src, cubin, log, true);
        if (st != CFS_OK) return st;
        *chosen_min_blocks = c;
        if (spill_bytes(*log) <= spec.spill_allowance) break;
    }
    return st;
}

cfs_status compile_only(const ProgramSpec& spec, std::string* src, std::string* log)
{
    std::vector<char> cubin;
    int mb = 0;
    return select_and_compile(spec, src, &cubin, log, &mb);
}

int device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

cfs_status get_kernel(const ProgramSpec& spec, const char* name, Kernel* out)
{
    Driver& d = driver();
    if (!d.ok) return fail(CFS_ERR_CUDA, d.why);
    int dev = 0;
    cfs_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != CFS_OK) return st;
    // make sure the primary context is current for the driver calls below
    st = check_cuda(cudaFree(nullptr), "cudaFree(0)");
    if (st != CFS_OK) return st;

    const std::string key = std::to_string(dev) + "\n" + spec.key();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto it = g_cache.find(key);
    Program* prog = nullptr;
    if (it == g_cache.end()) {
        std::vector<char> cubin;
        std::string src, log;
        int mb = spec.min_blocks;
        st = select_and_compile(spec, &src, &cubin, &log, &mb);
        if (st != CFS_OK) return st;
        auto p = std::make_unique<Program>();
        st = check_cu(d.module_load(&p->module, cubin.data()), "cuModuleLoadData");
        if (st != CFS_OK) return st;
        p->min_blocks = mb;
        prog = p.get();
        g_cache.emplace(key, std::move(p));
    } else {
        prog = it->second.get();
    }
    const std::string kname = std::string(name) + "/" + std::to_string(spec.dyn_smem);
    auto kit = prog->kernels.find(kname);
    if (kit == prog->kernels.end()) {
        Kernel k;
        CUfunction fn = nullptr;
        st = check_cu(d.get_function(&fn, prog->module, name), "cuModuleGetFunction");
        if (st != CFS_OK) return st;
        k.fn = (void*)fn;
        k.block = spec.block;
        k.dyn_smem = spec.dyn_smem;
        // without the opt-in, static plus dynamic shared memory may not pass
        // 48 KB: a window just under 48 KB would fail to launch
        if (spec.dyn_smem > 0) {
            st = check_cu(d.set_attribute(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                          spec.dyn_smem),
                          "cuFuncSetAttribute(max dynamic shared memory)");
            if (st != CFS_OK) return st;
        }
        st = check_cu(d.occupancy(&k.max_blocks_per_sm, fn, spec.block, (size_t)spec.dyn_smem),
                      "cuOccupancyMaxActiveBlocksPerMultiprocessor");
        if (st != CFS_OK) return st;
        k.num_sms = device_sm_count();
        kit = prog->kernels.emplace(kname, k).first;
    }
    *out = kit->second;
    return CFS_OK;
}

cfs_status launch(const Kernel& k, unsigned grid, const void* args, size_t args_size,
                  cudaStream_t stream)
{
    (void)args_size;
    void* params[] = {const_cast<void*>(args)};
    return check_cu(driver().launch((CUfunction)k.fn, grid, 1, 1, (unsigned)k.block, 1, 1,
                                    (unsigned)k.dyn_smem, (CUstream)stream, params, nullptr),
                    "cuLaunchKernel");
}

}  // namespace cfs
