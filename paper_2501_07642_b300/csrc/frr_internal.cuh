// frr_internal.cuh -- context layout and helpers shared by the CUDA sources of libfrr.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <math.h>

#include "../../include/frr.h"

namespace frr {

// Largest n the generation kernels cover: 16 Philox blocks (64 unit words) per lane.
constexpr int kMaxN = 2048;
constexpr int kExactMaxN = 63;

// Fixed-point scale for the exact-sum recheck: |Q_ij| <= 2^kQBits (the rounding of Zc to Q
// then moves a column sum by at most n 2^-kQBits times the column's largest magnitude),
// and sums over at most 2^12 units stay below 2^58.
constexpr int kQBits = 46;

// The fixed-point covariates of the exact recheck are written in kDigitPlanes balanced digits
// of kDigitBits bits, Q = sum_k D_k 2^(kDigitBits k) with D_k in [-2^(kDigitBits-1),
// 2^(kDigitBits-1)), each plane stored in FP16 (every integer of magnitude <= 2^11 is exact in
// FP16, so 12-bit balanced digits are). Four 12-bit digits cover |Q| <= 2^kQBits; a plane's
// sum over <= 2047 treated units stays below 2047 * 2^11 < 2^22 in magnitude, so FP32
// accumulation of it is exact in any order. Four planes of a 64-column chunk make one
// 256-row B tile: one N = 256 MMA per K step.
constexpr int kDigitPlanes = 4;
constexpr int kDigitBits = 12;
static_assert(kDigitPlanes * kDigitBits >= kQBits + 2, "digit planes cover the fixed-point range");

// Fluctuation multiplier of the accumulation term of the error band (number of
// standard deviations of a partial sum under complete randomization).
constexpr double kBandLambda = 6.0;

struct BandConsts {
    // band(M) = safety * (lin * sqrt(M) + quad + rel * M), M in T^2 units
    double lin = 0.0, quad = 0.0, rel = 0.0;
};

struct StreamState {
    bool active = false;
    bool exact = false;
    uint64_t seed = 0;
    bool q_mode = true;
    double q = NAN, threshold = NAN;
    uint64_t total = 0, seen = 0;
    int64_t K = 0;            // target accepted count (q mode)
    int64_t retained = 0;     // entries in the retained (candidate) set; -1: only on the device
    int64_t retained_bound = 0;  // upper bound of the retained count when it is only on the device
    bool defer_count = false; // the last chunk leaves the retained count on the device (no read-back)
    bool times_pending = false;  // that chunk's event times are read after the final synchronisation
    bool timing = true;       // record the per-phase events of frr_stats (off in the batched driver)
    bool overflowed = false;  // stream_end found the deferred retained set larger than its buffer
    float cut = INFINITY;     // current cut on the approximate M (keep M_hat <= cut)
    int parity = 0;           // histogram set of the next chunk's selection
    // stream_end_enqueue -> stream_end_finish: where the outputs go
    bool end_enqueued = false, end_direct = false, end_host_keys = false, end_host_m = false, end_stage = false;
    bool end_dev_count = false;
    int64_t end_rb = 0, end_stage_n = 0;
    size_t end_pinned = 0;    // pinned bytes used by the summary and the staged outputs
};

}  // namespace frr

struct frr_ctx {
    int64_t n = 0, d = 0, n1 = 0, n0 = 0;
    frr_opts opts{};
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;  // second stream of the prep (forward substitution beside Cholesky)
    int kb = 0;                // Philox blocks per lane, power of two: n <= 128 * kb
    int kused = 0;             // K positions holding units: 128 * ceil(n / 128)
    int kpad = 0;              // 128 * kb
    int dpad32 = 0;            // d rounded up to 128 (FP32 SIMT column tiles)
    double c_M = 0.0;          // n / (n1 n0)

    // device copies (K-order = the order in which the generator emits unit bits)
    double* Zc64 = nullptr;    // n x d, natural unit order
    float* Z32 = nullptr;      // kpad x dpad32, K-order rows, zero padding
    __nv_bfloat16* Zhi = nullptr;  // d x kpad (K-major), K-order columns
    __nv_bfloat16* Zlo = nullptr;
    long long* Q = nullptr;    // kpad x d fixed-point Zc, K-order rows
    long long* Qsum = nullptr; // d
    int* qexp = nullptr;       // d: Q_ij = Zc_ij * 2^qexp_j (rounded)
    uint64_t* binom = nullptr; // 64 x 64 binomial table (exact mode)
    __half* Zq = nullptr;          // kDigitPlanes x d x kpad: balanced digit planes of Q (exact recheck)
    CUtensorMap qmap{};            // tensor map over Zq (rows kDigitPlanes d, columns kpad)
    bool qmap_ready = false;
    CUtensorMap map_hi{}, map_lo{};  // tensor maps over Zhi / Zlo (balance kernel B operand)
    bool maps_ready = false;

    frr::BandConsts band32{}, band_tc{};

    void* arena = nullptr;     // one allocation holding the fixed per-context arrays above

    // scratch
    float* Mhat = nullptr;  size_t Mhat_bytes = 0;       // approximate M of a chunk
    uint64_t* ret_idx[2] = {nullptr, nullptr};           // retained candidates (ping-pong)
    float* ret_m[2] = {nullptr, nullptr};
    size_t ret_bytes_idx[2] = {0, 0}, ret_bytes_m[2] = {0, 0};
    int ret_cur = 0;
    int* dev_counters = nullptr;  // small device scalars
    double* M64 = nullptr; size_t M64_bytes = 0;
    uint64_t* ukeys = nullptr; size_t ukeys_bytes = 0;   // key staging
    void* misc = nullptr; size_t misc_bytes = 0;          // replay / randtest scratch
    void* misc2 = nullptr; size_t misc2_bytes = 0;
    void* rt = nullptr; size_t rt_bytes = 0;             // randomization-test scratch
    // a slice of a block owned by frr_batch_run, lent for the batch's duration: ensure_device
    // carves scratch from it before it asks the pool, and release() does not free what it carved
    char* lend = nullptr; size_t lend_off = 0, lend_cap = 0;
    void* sel = nullptr; size_t sel_bytes = 0;           // device state of the running selection
    void* host_pinned = nullptr; size_t host_pinned_bytes = 0;
    cudaEvent_t ev[8] = {};

    frr::StreamState st;
    frr_stats stats{};
    bool failed = false;
};

namespace frr {

// ---- programmatic dependent launch ------------------------------------------
// The selection and recheck kernels of one frr_select follow each other on one stream. Launched
// with launch_pdl, a kernel's blocks may be scheduled while the previous kernel finishes; each
// such kernel calls pdl_wait() before it touches memory, which returns once the previous
// kernel has completed and its writes are visible, and pdl_launch_dependents() to let the next
// kernel be scheduled early. Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream, A... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// ---- status helpers ------------------------------------------------------
#define FRR_CUDA_TRY(ctx, expr)                                                   \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess) {                                                  \
            if ((ctx) != nullptr) (ctx)->failed = true;                           \
            return (_e == cudaErrorMemoryAllocation) ? FRR_E_NOMEM : FRR_E_CUDA;  \
        }                                                                         \
    } while (0)

#define FRR_TRY(expr)                        \
    do {                                     \
        frr_status _s = (expr);              \
        if (_s != FRR_OK) return _s;         \
    } while (0)

// true if p is device-accessible memory (device or managed); false for pageable / pinned host
bool is_device_ptr(const void* p);

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) once per (kernel, device, size):
// the attribute belongs to the function, so repeating it at every launch only costs host time
cudaError_t set_smem_limit(const void* fn, int bytes, int device);
template <typename... P>
inline cudaError_t set_smem_limit(void (*kernel)(P...), int bytes, int device)
{
    return set_smem_limit(reinterpret_cast<const void*>(kernel), bytes, device);
}

// handle of the CUDA context current on the calling thread (null if there is none): it
// changes when a device's primary context is destroyed (cudaDeviceReset) and created again,
// which invalidates every device address and graph made in the old one
void* current_cuda_context();

// stream-ordered memory pool of the library for short-lived temporaries on `device`; it keeps
// up to 8 GiB reserved between calls instead of returning it at every synchronisation (a
// 256-experiment batch peaks near 2 GiB)
cudaMemPool_t temp_pool(int device);

// grow a device buffer to at least `bytes` (old contents are not kept)
frr_status ensure_device(frr_ctx* ctx, void** buf, size_t* cap_bytes, size_t bytes);

// pinned host staging of at least `bytes`
frr_status ensure_host_pinned(frr_ctx* ctx, size_t bytes);

// FRR_E_TIMEOUT if a kernel of the context recorded an expired bounded wait (the word is cleared)
frr_status take_device_error(frr_ctx* ctx);

// copies between a caller buffer (host or device) and a device buffer of the context
frr_status copy_in(frr_ctx* ctx, void* dst_dev, const void* src_any, size_t bytes);
frr_status copy_out(frr_ctx* ctx, void* dst_any, const void* src_dev, size_t bytes);

// kernel families (defined in their own translation units)
// scan_x: also reject non-finite entries of X (else the caller checks them, e.g. stage_finite)
frr_status check_init_args(const double* X, int64_t n, int64_t d, int64_t n1, const frr_opts& o, bool scan_x);
bool all_finite(const double* X, int64_t count);
frr_status stage_finite(const double* X, int64_t count, double* dst);
// pinned host blocks pooled by the library (size classes: powers of two up to 16 MiB, then multiples of 16 MiB)
void* pinned_get(size_t bytes, size_t* cap_out);
void pinned_put(void* p, size_t cap);
// records per-phase timing event i on the context's stream (created on first use)
void record_ev(frr_ctx* ctx, int i);
frr_status ctx_create(frr_ctx** out, int64_t n, int64_t d, int64_t n1, const frr_opts& o, bool with_aux);
void ctx_release(frr_ctx* ctx);
// prepares one context (its arrays allocated) from host covariates X_host, with one
// synchronisation at the end
frr_status prep_run(frr_ctx* ctx, const double* X_host);
// prepares E contexts (created, arrays allocated) together on streams s and aux; st_out[e]
// receives each one's status (FRR_E_DEGENERATE for a failed pivot, FRR_E_TIMEOUT for an
// expired bounded wait); the return value is a CUDA failure common to all, else FRR_OK
frr_status prep_run_batch(frr_ctx* const* ctxs, const double* const* X_host, int E, cudaStream_t s, cudaStream_t aux,
                          frr_status* st_out);
// One experiment's covariance from digit products on the tensor cores (frr_prep_tc.cu).
struct CovJob {
    int n, d, npad, dpad;       // npad = 64 ceil(n / 64), dpad = 128 ceil(d / 128)
    const double* Xc;           // centred covariates, n x d row-major
    int* cexp;                  // d column exponents
    __nv_bfloat16* G;           // 8 digit planes, dpad x npad each
    const CUtensorMap* gmap;    // over G (8 dpad rows x npad columns), in device memory
    long long* acc;             // d x d int64 sums (elements on or above the diagonal)
    double* S;                  // d x d covariance (output)
    int* status;                // the preparation's status word (bit 2: a bounded wait expired)
    double rinv;                // RN(1 / (n - 1))
};
// Columns per block of the forward substitution's tensor-core updates (a multiple of the
// panel width, 32, and of the digit kernel's K block, 64).
constexpr int kFwdBlock = 256;
// One experiment's forward-substitution updates across 256-column blocks from digit products
// on the tensor cores (frr_prep_tc.cu): after block b, rows i of the working Zc and rows
// 256 (b + 1) + j of L, both over the block's columns, give ZT_i,256(b+1)+j -= their product.
struct FwdJob {
    int n, d, npadA, dpadB;     // plane rows: 128 ceil(n / 128), 128 ceil((d - 256) / 128)
    double* ZT;                 // working Zc, n x d row-major
    const double* L;            // Cholesky factor, d x d row-major (lower part)
    int* expA;                  // n row exponents of the Zc block
    int* expB;                  // d - 256 row exponents of the L rows
    __nv_bfloat16* GA;          // 8 planes, npadA x 256 each
    __nv_bfloat16* GB;          // 8 planes, dpadB x 256 each
    const CUtensorMap* mapA;    // over GA (8 npadA rows x 256 columns), in device memory
    const CUtensorMap* mapB;    // over GB
    long long* acc;             // n x d int64 sums, zero between blocks
    int* status;
};
int fwd_tc_npadA(int n);
int fwd_tc_dpadB(int d);
size_t fwd_tc_plane_bytes_a(int n);
size_t fwd_tc_plane_bytes_b(int d);
// blocks (or work units) per experiment of the three launches after block b (0 when no
// column follows the block)
unsigned fwd_tc_digit_blocks(int n, int d, int b);
unsigned fwd_tc_units(int n, int d, int b);
unsigned fwd_tc_apply_blocks(int n, int d, int b);
bool fwd_tc_maps(CUtensorMap* ma, CUtensorMap* mb, const FwdJob& j);
cudaError_t fwd_tc_launch(const FwdJob* jobs, const unsigned* const prefix[3], const unsigned total[3], int E, int b,
                          int device, int num_sms, cudaStream_t s);
int cov_tc_npad(int n);
int cov_tc_dpad(int d);
size_t cov_tc_plane_bytes(int n, int d);
// blocks (or work units) per experiment of the four launches of cov_tc_launch
unsigned cov_tc_exp_blocks(int n, int d);
unsigned cov_tc_digit_blocks(int n, int d);
unsigned cov_tc_units(int n, int d);
unsigned cov_tc_finish_blocks(int n, int d);
// the tensor map over an experiment's digit planes G (device address)
bool cov_tc_map(CUtensorMap* m, const __nv_bfloat16* G, int n, int d);
// column exponents, digit planes, tensor-core sums and S for the experiments of the device
// table `jobs`; prefix[l] / total[l]: the prefix sums of launch l's blocks over the jobs
cudaError_t cov_tc_launch(const CovJob* jobs, const unsigned* const prefix[4], const unsigned total[4], int E,
                          int device, int num_sms, cudaStream_t s);
// the tensor-core sums' shared-memory limits on `device`, set before a launch sequence is
// captured into a graph (cov_tc_launch and fwd_tc_launch then make no attribute call)
cudaError_t prep_tc_setup(int device);
frr_status balance_f32_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout_dev);
// hist0 (split BF16 only, may be NULL): 4096 counters that also receive the level-0 histogram
// of the scored M_hat (bits [31:20] of each value) for the streaming selection
frr_status balance_tc_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout_dev,
                             unsigned* hist0 = nullptr);
frr_status balance_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout_dev,
                          unsigned* hist0 = nullptr);
// count_dev: when given, the count is read on the device and `count` only bounds it; the
// kernel also zeroes zero[0, nzero) (counters of the kernel launched after it)
frr_status bits_launch(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t count,
                       const uint64_t* draws_dev, uint32_t* rows_dev, const long long* count_dev = nullptr,
                       int* zero = nullptr, int nzero = 0);
frr_status words_select_launch(frr_ctx* ctx, const uint32_t* words_dev, uint32_t* row_dev);
frr_status unpack_launch(frr_ctx* ctx, const uint32_t* rows_dev, uint64_t count, uint8_t* w_dev);
frr_status recheck_launch(frr_ctx* ctx, uint64_t seed, bool exact, const uint64_t* draws_dev, int64_t count,
                          double* M64_dev, const long long* count_dev = nullptr);
frr_status recheck_tc_launch(frr_ctx* ctx, uint64_t seed, bool exact, const uint64_t* draws_dev, int64_t count,
                             double* M64_dev, const long long* count_dev = nullptr);
// M64 = scale * (sum over the ncb column-block partial sums of each draw) / denom
frr_status recheck_sum_launch(frr_ctx* ctx, const double* part, int ncb, int64_t count, double* M64_dev, double scale,
                              double denom, const long long* count_dev = nullptr);
frr_status stream_begin(frr_ctx* ctx, uint64_t seed, double q, double threshold, uint64_t total);
frr_status stream_chunk(frr_ctx* ctx, uint64_t first, uint64_t B);
frr_status stream_end(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out);
// checkpoint of a running stream between chunks (layout in include/frr.h, frr_stream_save)
frr_status stream_save(frr_ctx* ctx, void* blob, size_t cap, size_t* size_out);
frr_status stream_load(frr_ctx* ctx, const void* blob, size_t size);
// checks a blob's magic, version, size and checksum; fills *info when given
frr_status stream_blob_check(const void* blob, size_t size, frr_stream_info* info);
// stream_end in two halves: the first enqueues the recheck, ordering, placement and read-back
// copies (reserving extra_pinned bytes of pinned memory after its own for the caller); the
// second synchronises the stream, reads the summary and writes the outputs
frr_status stream_end_enqueue(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, size_t extra_pinned);
frr_status stream_end_finish(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out);
// after stream_end_enqueue: the device array the accepted keys are placed in (ascending draw
// index; q mode: exactly K of them), and the first pinned byte free for the caller
const uint64_t* stream_end_keys_dev(const frr_ctx* ctx, const uint64_t* keys_out);
size_t stream_end_pinned_used(const frr_ctx* ctx);
// after stream_begin: an upper bound of the pinned bytes stream_end_enqueue takes for its own
// use, when the stream is one deferred chunk into a fresh context (so that the caller can
// reserve the block before anything is in flight: growing it later synchronises the stream)
size_t stream_end_pinned_bound(const frr_ctx* ctx, int64_t cap);
frr_status stream_chunk_precomputed(frr_ctx* ctx, uint64_t first, uint64_t B, const float* Mhat_dev);
// the test's kernels on ctx->stream for K checked keys (host, or device when keys_on_device; obs = index of the
// observed assignment) and checked Y (n), tau (T) (host or device); the results stay on the
// device: p (T), count (T), ci (2)
frr_status randtest_enqueue(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, bool keys_on_device, int64_t K,
                            int64_t obs, const double* Y, const double* tau, int64_t T, double alpha,
                            const double** dp, const long long** dcount, const double** dci);
frr_status randtest_run(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, int64_t K, uint64_t obs_key,
                        const double* Y, const double* tau, int64_t T, double alpha, double* p_out,
                        int64_t* count_out, double* ci_lo, double* ci_hi);

inline uint64_t binom_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) r = r * (unsigned)(n - k + i) / (unsigned)i;
    return (r > (unsigned __int128)UINT64_MAX) ? UINT64_MAX : (uint64_t)r;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// band of the approximate M of the chosen bulk path
inline const BandConsts& band_of(const frr_ctx* ctx)
{
    return ctx->opts.precision == FRR_F32 ? ctx->band32 : ctx->band_tc;
}

__host__ __device__ inline double band_value(double lin, double quad, double rel, double safety, double m)
{
    return safety * (lin * sqrt(m > 0.0 ? m : 0.0) + quad + rel * m);
}

}  // namespace frr
