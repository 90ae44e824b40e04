// frr_capi.cu -- the extern "C" entry points of include/frr.h: argument checks,
// context ownership, host/device marshalling. All arithmetic runs in the
// kernels of the other translation units.
#include "frr_internal.cuh"

#include <mutex>
#include <string>
#include <unordered_map>

#include <cstdio>

#include <chrono>
#include <immintrin.h>
#include <new>
#include <vector>

namespace frr {

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t set_smem_limit(const void* fn, int bytes, int device)
{
    static std::mutex mu;
    static std::unordered_map<std::string, int> done;
    char key[64];
    snprintf(key, sizeof(key), "%p/%d", fn, device);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = done.find(key);
        if (it != done.end() && it->second >= bytes) return cudaSuccess;
    }
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(mu);
        int& v = done[key];
        if (v < bytes) v = bytes;
    }
    return e;
}

static bool is_lent(const frr_ctx* ctx, const void* p)
{
    const char* c = static_cast<const char*>(p);
    return ctx->lend != nullptr && c >= ctx->lend && c < ctx->lend + ctx->lend_cap;
}

frr_status ensure_device(frr_ctx* ctx, void** buf, size_t* cap_bytes, size_t bytes)
{
    // stream-ordered allocations from the library pool: no device-wide synchronisation
    if (bytes == 0) bytes = 16;
    if (*buf != nullptr && *cap_bytes >= bytes) return FRR_OK;
    const size_t carve = (bytes + 255) & ~size_t(255);
    if (ctx->lend != nullptr && ctx->lend_cap - ctx->lend_off >= carve) {
        // from the lent slice: no allocation call (each costs the issuing thread ~25 us while
        // the device is busy, and a batch makes ~1500 of them)
        if (*buf != nullptr && !is_lent(ctx, *buf)) cudaFreeAsync(*buf, ctx->stream);
        *buf = ctx->lend + ctx->lend_off;
        ctx->lend_off += carve;
        *cap_bytes = carve;
        return FRR_OK;
    }
    if (*buf != nullptr) {
        if (!is_lent(ctx, *buf)) cudaFreeAsync(*buf, ctx->stream);
        *buf = nullptr;
        *cap_bytes = 0;
    }
    cudaMemPool_t pool = temp_pool(ctx->device);
    if (pool == nullptr) return FRR_E_CUDA;
    const size_t grown = bytes + bytes / 4;
    cudaError_t e = cudaMallocFromPoolAsync(buf, grown, pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return FRR_E_NOMEM;
    }
    *cap_bytes = grown;
    return FRR_OK;
}

// Pinned host blocks are kept by the library between contexts and calls (size classes
// below): cudaMallocHost is slow and cudaFreeHost synchronises the device, which a batch of
// many short-lived contexts would otherwise pay once per context.
namespace {
std::mutex g_pinned_mu;
std::unordered_map<size_t, std::vector<void*>> g_pinned_free;

// size classes: powers of two from 4 KiB to 16 MiB, then multiples of 16 MiB
size_t pinned_class(size_t bytes)
{
    const size_t big = size_t(16) << 20;
    if (bytes > big) return (bytes + big - 1) / big * big;
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    return c;
}
}  // namespace

void pinned_put(void* p, size_t cap)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free[cap].push_back(p);
}

void* pinned_get(size_t bytes, size_t* cap_out)
{
    const size_t cap = pinned_class(bytes);
    *cap_out = cap;
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        auto it = g_pinned_free.find(cap);
        if (it != g_pinned_free.end() && !it->second.empty()) {
            void* p = it->second.back();
            it->second.pop_back();
            return p;
        }
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

frr_status ensure_host_pinned(frr_ctx* ctx, size_t bytes)
{
    if (ctx->host_pinned != nullptr && ctx->host_pinned_bytes >= bytes) return FRR_OK;
    // the old block may still be the target of a copy in flight on this stream
    if (ctx->host_pinned) {
        FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        pinned_put(ctx->host_pinned, ctx->host_pinned_bytes);
    }
    ctx->host_pinned = nullptr;
    ctx->host_pinned_bytes = 0;
    const size_t cap = pinned_class(bytes);
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        auto it = g_pinned_free.find(cap);
        if (it != g_pinned_free.end() && !it->second.empty()) {
            ctx->host_pinned = it->second.back();
            it->second.pop_back();
        }
    }
    if (ctx->host_pinned == nullptr && cudaMallocHost(&ctx->host_pinned, cap) != cudaSuccess) {
        cudaGetLastError();
        ctx->host_pinned = nullptr;
        return FRR_E_NOMEM;
    }
    ctx->host_pinned_bytes = cap;
    return FRR_OK;
}

frr_status copy_in(frr_ctx* ctx, void* dst_dev, const void* src_any, size_t bytes)
{
    if (bytes == 0) return FRR_OK;
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(dst_dev, src_any, bytes, cudaMemcpyDefault, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FRR_OK;
}

frr_status copy_out(frr_ctx* ctx, void* dst_any, const void* src_dev, size_t bytes)
{
    if (bytes == 0) return FRR_OK;
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(dst_any, src_dev, bytes, cudaMemcpyDefault, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FRR_OK;
}

frr_status take_device_error(frr_ctx* ctx)
{
    int err = 0;
    FRR_CUDA_TRY(ctx, cudaMemcpyAsync(&err, ctx->dev_counters + 12, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (err == 0) return FRR_OK;
    FRR_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dev_counters + 12, 0, sizeof(int), ctx->stream));
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FRR_E_TIMEOUT;
}

static frr_status check_range(const frr_ctx* ctx, uint64_t seed, uint64_t first, uint64_t B)
{
    if (first + B < first) return FRR_E_RANGE;
    if (seed == FRR_EXACT_SEED) {
        if (ctx->n > kExactMaxN) return FRR_E_UNSUPPORTED;
        if (first + B > binom_host((int)ctx->n, (int)ctx->n1)) return FRR_E_RANGE;
    }
    return FRR_OK;
}

cudaMemPool_t temp_pool(int device)
{
    static std::mutex mu;
    static std::unordered_map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // Memory freed to the pool stays mapped up to this much across synchronisations. A batch
    // of 256 experiments peaks near 2 GiB (contexts and preparation temporaries); below its
    // peak the pool was trimmed and mapped again on later calls (5-10 ms per batch).
    uint64_t keep = 8ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[device] = pool;
    return pool;
}

static void release(frr_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    // the fixed arrays (Zc64 ... dev_counters) live in ctx->arena; all of these come from the
    // library pool and go back to it in stream order
    void* bufs[] = {ctx->arena, ctx->Mhat, ctx->ret_idx[0], ctx->ret_idx[1], ctx->ret_m[0], ctx->ret_m[1], ctx->M64,
                    ctx->ukeys, ctx->misc, ctx->misc2, ctx->rt, ctx->sel};
    for (void* b : bufs)
        if (b && !is_lent(ctx, b)) cudaFreeAsync(b, ctx->stream ? ctx->stream : 0);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    pinned_put(ctx->host_pinned, ctx->host_pinned_bytes);
    for (cudaEvent_t e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

// Argument checks of frr_init (also applied to every experiment of frr_batch_run).
// Copies n*d values from X to dst (pinned staging) and checks that they are finite, in one pass.
namespace {
// Copy with the non-finite check (exponent field all ones), one word at a time.
uint64_t stage_words(const uint64_t* bits, int64_t count, uint64_t* out)
{
    const uint64_t em = 0x7ff0000000000000ull;
    uint64_t bad = 0;
    for (int64_t k = 0; k < count; ++k) {
        const uint64_t b = bits[k];
        out[k] = b;
        bad |= (uint64_t)((b & em) == em);
    }
    return bad;
}

// The same with 32-byte loads and non-temporal stores: the staging block is written once and
// read only by the DMA engine, so the stores bypass the caches (no read for ownership).
__attribute__((target("avx2"))) uint64_t stage_words_avx2(const uint64_t* bits, int64_t count, uint64_t* out)
{
    int64_t k = 0;
    uint64_t bad = 0;
    const int64_t head = (int64_t)(((32 - (reinterpret_cast<uintptr_t>(out) & 31)) & 31) / 8);
    if ((reinterpret_cast<uintptr_t>(out) & 7) != 0 || head >= count) return stage_words(bits, count, out);
    bad |= stage_words(bits, head, out);
    k = head;
    const __m256i em = _mm256_set1_epi64x(0x7ff0000000000000ll);
    __m256i acc = _mm256_setzero_si256();
    for (; k + 4 <= count; k += 4) {
        const __m256i v = _mm256_loadu_si256(reinterpret_cast<const __m256i*>(bits + k));
        _mm256_stream_si256(reinterpret_cast<__m256i*>(out + k), v);
        acc = _mm256_or_si256(acc, _mm256_cmpeq_epi64(_mm256_and_si256(v, em), em));
    }
    _mm_sfence();
    if (!_mm256_testz_si256(acc, acc)) bad = 1;
    return bad | stage_words(bits + k, count - k, out + k);
}

const bool g_has_avx2 = __builtin_cpu_supports("avx2");
}  // namespace

frr_status stage_finite(const double* X, int64_t count, double* dst)
{
    const uint64_t* bits = reinterpret_cast<const uint64_t*>(X);
    uint64_t* out = reinterpret_cast<uint64_t*>(dst);
    const uint64_t bad = g_has_avx2 ? stage_words_avx2(bits, count, out) : stage_words(bits, count, out);
    return bad ? FRR_E_ARG : FRR_OK;
}

frr_status check_init_args(const double* X, int64_t n, int64_t d, int64_t n1, const frr_opts& o, bool scan_x)
{
    if (!X) return FRR_E_ARG;
    if (n < 2 || d < 1 || n1 < 1 || n1 > n - 1) return FRR_E_ARG;
    if (n > kMaxN) return FRR_E_UNSUPPORTED;
    if (o.precision != FRR_SPLIT_BF16 && o.precision != FRR_F32) return FRR_E_ARG;
    if (o.whiten != FRR_CHOL && o.whiten != FRR_RIDGE && o.whiten != FRR_DIAG) return FRR_E_ARG;
    if (o.whiten == FRR_RIDGE && !(o.ridge > 0.0 && isfinite(o.ridge))) return FRR_E_ARG;
    if (!(o.band_safety >= 1.0 && isfinite(o.band_safety))) return FRR_E_ARG;
    if (o.prep != FRR_PREP_TENSOR && o.prep != FRR_PREP_FP64_CHAIN) return FRR_E_ARG;
    if (scan_x && !all_finite(X, n * d)) return FRR_E_ARG;
    if (o.whiten == FRR_CHOL && d >= n - 1) return FRR_E_DEGENERATE;
    return FRR_OK;
}

bool all_finite(const double* X, int64_t count)
{
    // non-finite entries have an all-ones exponent field; branch-free so that it vectorises
    const uint64_t* bits = reinterpret_cast<const uint64_t*>(X);
    const uint64_t em = 0x7ff0000000000000ull;
    uint64_t bad = 0;
    for (int64_t k = 0; k < count; ++k) bad |= (uint64_t)((bits[k] & em) == em);
    return bad == 0;
}

// A context for an (n, d, n1) experiment with checked options: streams, events and the fixed
// arrays allocated, nothing prepared yet. with_aux: also the second stream of the preparation
// (the batched driver prepares on streams of its own).
// The per-phase timing events are created when first recorded: a context that never records
// them (the batched driver turns the timing off) makes no event calls, which contend in the
// driver when many contexts are created on several threads.
void record_ev(frr_ctx* ctx, int i)
{
    if (!ctx->ev[i] && cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
        cudaGetLastError();
        ctx->ev[i] = nullptr;
        ctx->st.timing = false;  // no event: the phase times of this call are not reported
        ctx->st.times_pending = false;
        return;
    }
    cudaEventRecord(ctx->ev[i], ctx->stream);
}

frr_status ctx_create(frr_ctx** out, int64_t n, int64_t d, int64_t n1, const frr_opts& o, bool with_aux)
{
    *out = nullptr;
    frr_ctx* ctx = new (std::nothrow) frr_ctx();
    if (!ctx) return FRR_E_NOMEM;
    ctx->n = n; ctx->d = d; ctx->n1 = n1; ctx->n0 = n - n1;
    ctx->opts = o;
    ctx->c_M = (double)n / ((double)n1 * (double)(n - n1));
    const int blocks = ceil_div(n, 128);
    int kb = 1;
    while (kb < blocks) kb <<= 1;
    ctx->kb = kb;
    ctx->kused = 128 * blocks;
    ctx->kpad = 128 * kb;
    ctx->dpad32 = 128 * ceil_div(d, 128);
    ctx->stats.boundary_gap_rel = NAN;

    auto bail = [&](frr_status s) { release(ctx); return s; };
#define INIT_CUDA(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { cudaGetLastError(); \
        return bail(_e == cudaErrorMemoryAllocation ? FRR_E_NOMEM : FRR_E_CUDA); } } while (0)
    INIT_CUDA(cudaGetDevice(&ctx->device));
    INIT_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
    if (o.cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        INIT_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    if (with_aux) INIT_CUDA(cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    {
        // the fixed per-context arrays in one allocation (each part 256-byte aligned)
        const size_t nd = (size_t)n * d;
        const size_t sizes[10] = {nd * sizeof(double),
                                  (size_t)ctx->kpad * ctx->dpad32 * sizeof(float),
                                  (size_t)d * ctx->kpad * sizeof(__nv_bfloat16),
                                  (size_t)d * ctx->kpad * sizeof(__nv_bfloat16),
                                  (size_t)ctx->kpad * d * sizeof(long long),
                                  (size_t)d * sizeof(long long),
                                  (size_t)d * sizeof(int),
                                  64 * 64 * sizeof(uint64_t),
                                  (size_t)kDigitPlanes * d * ctx->kpad * sizeof(__half),
                                  16 * sizeof(int)};
        size_t offs[10], total = 0;
        for (int i = 0; i < 10; ++i) {
            offs[i] = total;
            total += (sizes[i] + 255) & ~size_t(255);
        }
        cudaMemPool_t pool = temp_pool(ctx->device);
        if (pool == nullptr) return bail(FRR_E_CUDA);
        INIT_CUDA(cudaMallocFromPoolAsync(&ctx->arena, total, pool, ctx->stream));
        char* a = static_cast<char*>(ctx->arena);
        ctx->Zc64 = reinterpret_cast<double*>(a + offs[0]);
        ctx->Z32 = reinterpret_cast<float*>(a + offs[1]);
        ctx->Zhi = reinterpret_cast<__nv_bfloat16*>(a + offs[2]);
        ctx->Zlo = reinterpret_cast<__nv_bfloat16*>(a + offs[3]);
        ctx->Q = reinterpret_cast<long long*>(a + offs[4]);
        ctx->Qsum = reinterpret_cast<long long*>(a + offs[5]);
        ctx->qexp = reinterpret_cast<int*>(a + offs[6]);
        ctx->binom = reinterpret_cast<uint64_t*>(a + offs[7]);
        ctx->Zq = reinterpret_cast<__half*>(a + offs[8]);
        ctx->dev_counters = reinterpret_cast<int*>(a + offs[9]);
        INIT_CUDA(cudaMemsetAsync(ctx->dev_counters, 0, 16 * sizeof(int), ctx->stream));
    }
#undef INIT_CUDA
    *out = ctx;
    return FRR_OK;
}

void ctx_release(frr_ctx* ctx) { release(ctx); }

}  // namespace frr

using namespace frr;

extern "C" {

void frr_default_opts(frr_opts* o)
{
    if (!o) return;
    o->precision = FRR_SPLIT_BF16;
    o->whiten = FRR_CHOL;
    o->ridge = 0.1;
    o->band_safety = 2.0;
    o->cuda_stream = nullptr;
    o->autotune = 0;
    o->prep = FRR_PREP_TENSOR;
}

const char* frr_strerror(frr_status s)
{
    switch (s) {
        case FRR_OK: return "ok";
        case FRR_E_ARG: return "invalid argument";
        case FRR_E_DEGENERATE: return "degenerate covariance (d >= n-1 under Cholesky whitening, or a pivot below tolerance)";
        case FRR_E_CUDA: return "CUDA error (context unusable)";
        case FRR_E_NOMEM: return "out of memory";
        case FRR_E_TIMEOUT: return "bounded device wait expired";
        case FRR_E_CAPACITY: return "output array too small (K_out holds the size needed)";
        case FRR_E_RANGE: return "draw range out of bounds";
        case FRR_E_STATE: return "call out of sequence";
        case FRR_E_UNSUPPORTED: return "shape not covered by the compiled kernels";
        case FRR_E_MISMATCH: return "internal consistency check failed";
    }
    return "unknown status";
}

frr_status frr_init(frr_ctx** out, const double* X, int64_t n, int64_t d, int64_t n1, const frr_opts* opts)
{
    if (!out || !X) return FRR_E_ARG;
    *out = nullptr;
    frr_opts o;
    frr_default_opts(&o);
    if (opts) o = *opts;
    // X is checked for non-finite entries on the device, where the preparation centres it
    // (FRR_E_ARG from its status word); the host scans X only where the device cannot tell (no
    // context, a failed preparation), so that a non-finite X is reported before any other error,
    // GPU or not.
    {
        const frr_status c = check_init_args(X, n, d, n1, o, false);
        if (c == FRR_E_DEGENERATE) return check_init_args(X, n, d, n1, o, true);
        if (c != FRR_OK) return c;
    }
    const auto t0 = std::chrono::steady_clock::now();
    frr_ctx* ctx = nullptr;
    {
        const frr_status c = ctx_create(&ctx, n, d, n1, o, true);
        if (c != FRR_OK) return all_finite(X, n * d) ? c : FRR_E_ARG;
    }
    // (A host scan on its own thread beside the preparation, the earlier design, read the 8 MB
    // of an n = d = 1000 X at host memory speed: its join added 0.1-2.3 ms to the call.)
    const frr_status s = prep_run(ctx, X);
    if (s != FRR_OK) {
        release(ctx);
        if (s == FRR_E_ARG) return s;  // a non-finite covariate, found on the device
        return all_finite(X, n * d) ? s : FRR_E_ARG;
    }
    ctx->stats.ms_init = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = ctx;
    return FRR_OK;
}

void frr_destroy(frr_ctx* ctx) { release(ctx); }

frr_status frr_balance(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t B, float* M_out)
{
    if (!ctx || (!M_out && B > 0)) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    FRR_TRY(check_range(ctx, seed, first_draw, B));
    if (B == 0) return FRR_OK;
    const bool exact = (seed == FRR_EXACT_SEED);
    if (is_device_ptr(M_out)) {
        FRR_TRY(balance_launch(ctx, seed, exact, first_draw, B, M_out));
        FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        return take_device_error(ctx);
    }
    const uint64_t chunk = 1ull << 22;
    for (uint64_t off = 0; off < B; off += chunk) {
        const uint64_t bc = (B - off < chunk) ? (B - off) : chunk;
        FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->Mhat), &ctx->Mhat_bytes, bc * sizeof(float)));
        FRR_TRY(balance_launch(ctx, seed, exact, first_draw + off, bc, ctx->Mhat));
        FRR_TRY(copy_out(ctx, M_out + off, ctx->Mhat, bc * sizeof(float)));
        FRR_TRY(take_device_error(ctx));
    }
    return FRR_OK;
}

frr_status frr_balance_exact(frr_ctx* ctx, uint64_t first_rank, uint64_t B, float* M_out)
{
    return frr_balance(ctx, FRR_EXACT_SEED, first_rank, B, M_out);
}

static frr_status check_mode(double q, double threshold)
{
    const bool hq = !isnan(q), ht = !isnan(threshold);
    if (hq == ht) return FRR_E_ARG;
    if (hq && !(q > 0.0 && q <= 1.0)) return FRR_E_ARG;
    if (ht && !(threshold >= 0.0)) return FRR_E_ARG;
    return FRR_OK;
}

frr_status frr_stream_begin(frr_ctx* ctx, uint64_t seed, double q, double threshold, uint64_t B_total)
{
    if (!ctx) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    FRR_TRY(check_mode(q, threshold));
    if (B_total == 0) return FRR_E_ARG;
    if (seed == FRR_EXACT_SEED) {
        if (ctx->n > kExactMaxN) return FRR_E_UNSUPPORTED;
        if (B_total > binom_host((int)ctx->n, (int)ctx->n1)) return FRR_E_RANGE;
    }
    return stream_begin(ctx, seed, q, threshold, B_total);
}

frr_status frr_stream_chunk(frr_ctx* ctx, uint64_t first_draw, uint64_t B_chunk)
{
    if (!ctx) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (!ctx->st.active) return FRR_E_STATE;
    FRR_TRY(check_range(ctx, ctx->st.seed, first_draw, B_chunk));
    return stream_chunk(ctx, first_draw, B_chunk);
}

frr_status frr_stream_end(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out)
{
    if (!ctx || !K_out || cap < 0 || (!keys_out && cap > 0)) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    return stream_end(ctx, keys_out, M64_out, cap, K_out);
}

frr_status frr_stream_save(frr_ctx* ctx, void* blob, size_t cap, size_t* size_out)
{
    if (!ctx || !size_out) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    return stream_save(ctx, blob, cap, size_out);
}

frr_status frr_stream_load(frr_ctx* ctx, const void* blob, size_t size)
{
    if (!ctx || !blob) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    return stream_load(ctx, blob, size);
}

frr_status frr_stream_blob_info(const void* blob, size_t size, frr_stream_info* out)
{
    if (!blob || !out) return FRR_E_ARG;
    return stream_blob_check(blob, size, out);
}

frr_status frr_select(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t B, double q, double threshold,
                      uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out)
{
    if (!ctx || !K_out || cap < 0 || (!keys_out && cap > 0) || B == 0) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    FRR_TRY(check_mode(q, threshold));
    FRR_TRY(check_range(ctx, seed, first_draw, B));
    for (int attempt = 0; attempt < 2; ++attempt) {
        FRR_TRY(stream_begin(ctx, seed, q, threshold, B));
        // one call: the recheck may read the candidate count on the device (first attempt)
        ctx->st.defer_count = attempt == 0;
        frr_status s = stream_chunk(ctx, first_draw, B);
        if (s != FRR_OK) { ctx->st.active = false; return s; }
        s = stream_end(ctx, keys_out, M64_out, cap, K_out);
        if (!(s == FRR_E_CAPACITY && ctx->st.overflowed)) return s;
    }
    return FRR_E_CAPACITY;
}

frr_status frr_assignments(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t count, uint8_t* w_out)
{
    if (!ctx || (!w_out && count > 0)) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    FRR_TRY(check_range(ctx, seed, first_draw, count));
    const bool exact = (seed == FRR_EXACT_SEED);
    const bool dev = count > 0 && is_device_ptr(w_out);
    const uint64_t chunk = 1ull << 16;
    const size_t words = 4 * (size_t)ctx->kb;
    for (uint64_t off = 0; off < count; off += chunk) {
        const uint64_t c = (count - off < chunk) ? (count - off) : chunk;
        const size_t rows_bytes = (size_t)c * words * sizeof(uint32_t);
        FRR_TRY(ensure_device(ctx, &ctx->misc2, &ctx->misc2_bytes, rows_bytes + (dev ? 0 : (size_t)c * ctx->n)));
        uint32_t* rows = static_cast<uint32_t*>(ctx->misc2);
        uint8_t* wdst = dev ? w_out + off * ctx->n : reinterpret_cast<uint8_t*>(static_cast<char*>(ctx->misc2) + rows_bytes);
        FRR_TRY(bits_launch(ctx, seed, exact, first_draw + off, c, nullptr, rows));
        FRR_TRY(unpack_launch(ctx, rows, c, wdst));
        if (!dev) FRR_TRY(copy_out(ctx, w_out + off * ctx->n, wdst, (size_t)c * ctx->n));
    }
    FRR_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return FRR_OK;
}

frr_status frr_assignment(frr_ctx* ctx, uint64_t seed, uint64_t key, uint8_t* w_out)
{
    return frr_assignments(ctx, seed, key, 1, w_out);
}

frr_status frr_assignment_from_words(frr_ctx* ctx, const uint32_t* words, uint8_t* w_out)
{
    if (!ctx || !words || !w_out) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    const size_t wbytes = (size_t)ctx->n * sizeof(uint32_t), rbytes = (size_t)4 * ctx->kb * sizeof(uint32_t);
    FRR_TRY(ensure_device(ctx, &ctx->misc2, &ctx->misc2_bytes, wbytes + rbytes + (size_t)ctx->n + 64));
    uint32_t* dwords = static_cast<uint32_t*>(ctx->misc2);
    uint32_t* row = dwords + ctx->n;
    uint8_t* dw = reinterpret_cast<uint8_t*>(row + 4 * ctx->kb);
    FRR_TRY(copy_in(ctx, dwords, words, wbytes));
    FRR_TRY(words_select_launch(ctx, dwords, row));
    FRR_TRY(unpack_launch(ctx, row, 1, dw));
    FRR_TRY(copy_out(ctx, w_out, dw, (size_t)ctx->n));
    return FRR_OK;
}

frr_status frr_recheck(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count, double* M64_out)
{
    if (!ctx || count < 0 || (count > 0 && (!draws || !M64_out))) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (count == 0) return FRR_OK;
    const bool exact = (seed == FRR_EXACT_SEED);
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->ukeys), &ctx->ukeys_bytes, (size_t)count * 8));
    FRR_TRY(copy_in(ctx, ctx->ukeys, draws, (size_t)count * 8));
    if (exact) {
        if (ctx->n > kExactMaxN) return FRR_E_UNSUPPORTED;
        std::vector<uint64_t> h((size_t)count);
        FRR_TRY(copy_out(ctx, h.data(), ctx->ukeys, (size_t)count * 8));
        const uint64_t tot = binom_host((int)ctx->n, (int)ctx->n1);
        for (uint64_t v : h)
            if (v >= tot) return FRR_E_RANGE;
    }
    FRR_TRY(ensure_device(ctx, reinterpret_cast<void**>(&ctx->M64), &ctx->M64_bytes, (size_t)count * 8));
    FRR_TRY(recheck_launch(ctx, seed, exact, ctx->ukeys, count, ctx->M64));
    FRR_TRY(copy_out(ctx, M64_out, ctx->M64, (size_t)count * 8));
    return FRR_OK;
}

frr_status frr_randtest(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, int64_t K, uint64_t obs_key,
                        const double* Y, const double* tau, int64_t T, double alpha, double* p_out,
                        int64_t* count_out, double* ci_lo, double* ci_hi)
{
    if (!ctx || !keys || K < 1 || !Y || !tau || T < 1 || !p_out || !(alpha >= 0.0 && alpha <= 1.0)) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (seed == FRR_EXACT_SEED && ctx->n > kExactMaxN) return FRR_E_UNSUPPORTED;
    return randtest_run(ctx, seed, keys, K, obs_key, Y, tau, T, alpha, p_out, count_out, ci_lo, ci_hi);
}

frr_status frr_whitened(const frr_ctx* ctx, double* Zc_out)
{
    if (!ctx || !Zc_out) return FRR_E_ARG;
    if (ctx->failed) return FRR_E_CUDA;
    if (cudaMemcpy(Zc_out, ctx->Zc64, (size_t)ctx->n * ctx->d * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        return FRR_E_CUDA;
    }
    return FRR_OK;
}

frr_status frr_last_stats(const frr_ctx* ctx, frr_stats* out)
{
    if (!ctx || !out) return FRR_E_ARG;
    *out = ctx->stats;
    return FRR_OK;
}

}  // extern "C"
