// frr_noalloc.cu -- frr_recheck_static: the exact-sum recheck without any allocation.
//
// Some callers cannot let a library allocate device memory: a latency-critical
// loop sharing the GPU with other work (cudaMalloc / cudaFree may synchronise the
// device and stall it), or an application whose device memory is owned by another
// allocator, such as a framework's caching pool with a fixed budget. For them this
// entry point computes the same exact treated sums as frr_recheck -- with the int64
// CUDA-core form of the recheck, which needs no bit-row buffer -- on caller-owned device
// buffers, with the only scratch it needs (the per-CTA partial sums) in one fixed array
// compiled into the library.
#include "frr_internal.cuh"

#include <mutex>

namespace frr {

frr_status recheck_launch_into(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count, double* part,
                               size_t part_capacity, double* M64);

namespace {

// Partial sums of the recheck: count * ceil(d / 128) doubles per call. Every GPU
// that loads the library holds these 1 MiB until the process exits.
static __device__ __align__(256) double g_recheck_scratch[FRR_RECHECK_STATIC_SCRATCH];

constexpr int kMaxDevices = 64;

// The array's device address belongs to the CUDA context the library's module is loaded
// in. It is looked up once per device and kept together with that context's handle; when
// the device's current context is a different one (its primary context was destroyed by
// cudaDeviceReset and created again), the address is looked up again.
struct ScratchAddr {
    CUcontext owner = nullptr;
    double* ptr = nullptr;
};
std::mutex g_setup_mutex;
ScratchAddr g_scratch_addr[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (no link-time libcuda dependency)
CtxGetCurrentFn ctx_get_current()
{
    static const CtxGetCurrentFn fn = []() -> CtxGetCurrentFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<CtxGetCurrentFn>(p);
        cudaGetLastError();
        return nullptr;
    }();
    return fn;
}

// Device address of the scratch array on `device`, looked up (set-up) with that device
// current. In host code the array's name is only a host-side stand-in, never a device address.
frr_status scratch_on(int device, double** out)
{
    if (device < 0 || device >= kMaxDevices) return FRR_E_UNSUPPORTED;
    const CtxGetCurrentFn get_ctx = ctx_get_current();
    if (!get_ctx) return FRR_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return FRR_E_CUDA; }
    if (cur != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return FRR_E_CUDA; }
    frr_status s = FRR_OK;
    CUcontext owner = nullptr;
    // cudaFree(nullptr) makes the device's primary context current (a no-op once it is)
    if (cudaFree(nullptr) != cudaSuccess || get_ctx(&owner) != CUDA_SUCCESS || owner == nullptr) {
        cudaGetLastError();
        s = FRR_E_CUDA;
    } else if (g_scratch_addr[device].ptr == nullptr || g_scratch_addr[device].owner != owner) {
        double* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_recheck_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            s = FRR_E_CUDA;
        } else {
            g_scratch_addr[device] = ScratchAddr{owner, p};
        }
    }
    if (s == FRR_OK) *out = g_scratch_addr[device].ptr;
    if (cur != device) cudaSetDevice(cur);
    return s;
}

// Device memory of `device` (or managed memory), aligned for 8-byte elements. A pointer into
// another GPU's memory is refused: the kernels would read it without peer access.
bool on_device(const void* p, int device)
{
    if (p == nullptr || (reinterpret_cast<uintptr_t>(p) & 7u) != 0u) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

void* current_cuda_context()
{
    const CtxGetCurrentFn get_ctx = ctx_get_current();
    CUcontext c = nullptr;
    if (!get_ctx || get_ctx(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

}  // namespace frr

extern "C" frr_status frr_recheck_static(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count,
                                         double* M64_out)
{
    using namespace frr;
    if (!ctx || count < 0) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (seed == FRR_EXACT_SEED) return FRR_E_UNSUPPORTED;
    if (count == 0) return FRR_OK;
    if (!on_device(draws, ctx->device) || !on_device(M64_out, ctx->device)) return FRR_E_ARG;
    const size_t ncb = (size_t)ceil_div(ctx->d, 128);
    if ((size_t)count * ncb > (size_t)FRR_RECHECK_STATIC_SCRATCH) return FRR_E_CAPACITY;
    double* scratch = nullptr;
    FRR_TRY(scratch_on(ctx->device, &scratch));
    // Nothing in the scratch needs clearing: every partial sum that is read was written
    // by this call's first kernel. Calls that overlap on the GPU share it and race.
    FRR_TRY(recheck_launch_into(ctx, seed, draws, count, scratch, FRR_RECHECK_STATIC_SCRATCH, M64_out));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FRR_OK;
}
