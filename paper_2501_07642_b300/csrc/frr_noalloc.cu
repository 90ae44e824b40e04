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
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (looked up once per device, with
// that device current). In host code the array's name is only a host-side stand-in.
frr_status scratch_on(int device, double** out)
{
    if (device < 0 || device >= kMaxDevices) return FRR_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[device] == nullptr) {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) { cudaGetLastError(); return FRR_E_CUDA; }
        if (cur != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return FRR_E_CUDA; }
        double* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_recheck_scratch);
        if (cur != device) cudaSetDevice(cur);
        if (e != cudaSuccess || p == nullptr) { cudaGetLastError(); return FRR_E_CUDA; }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return FRR_OK;
}

}  // namespace
}  // namespace frr

extern "C" frr_status frr_recheck_static(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count,
                                         double* M64_out)
{
    using namespace frr;
    if (!ctx || count < 0) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (seed == FRR_EXACT_SEED) return FRR_E_UNSUPPORTED;
    if (count == 0) return FRR_OK;
    if (!draws || !M64_out || !is_device_ptr(draws) || !is_device_ptr(M64_out)) return FRR_E_ARG;
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
