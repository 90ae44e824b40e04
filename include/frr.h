/*
 * frr.h -- C ABI of the B300-native rerandomization balance-check library.
 *
 * The method is the batched balance check of FastRerandomize (Goldstein,
 * Jerzak, Kamat, Zhu; arXiv 2501.07642):
 *   1. regenerate each candidate assignment of n1 treated out of n units from
 *      its counter-based key (Sec. 2.1, "Key-only storage");
 *   2. score it by Hotelling's T^2 / the Mahalanobis balance M of the whitened
 *      covariates (Sec. 2.2, Sec. 2.3 generate_randomizations);
 *   3. keep the keys whose M lies in the accepted q-quantile, or below a fixed
 *      threshold (Sec. 2.2 "Choosing stringency");
 *   4. replay the accepted keys for the randomization test conditional on
 *      acceptance and its fiducial interval by test inversion (Sec. 2.3
 *      randomization_test, Sec. 4 "Design-based inference").
 *
 * Units of M. Every M crossing this ABI is in T^2 units:
 *   M = (n1 n0 / n) * sum_j (m1_j - m0_j)^2 = n / (n1 n0) * ||w^T Zc||^2,
 * where m1, m0 are the treated / control means of the whitened covariates Zc.
 * The paper's M = Delta^T Delta of Sec. 2.2 equals this value times
 * (1/n1 + 1/n0); a threshold a_paper converts to a_paper * n1 n0 / n.
 *
 * Keys. A key is a 64-bit draw index b under a 64-bit pool seed (two 32-bit
 * words each, the paper's "two integers" of Sec. 4). Unit i of draw b gets the
 * 32-bit word r_i = word (i mod 4) of Philox4x32-10 (Salmon et al., SC'11) with
 * counter (floor(i/4), 0, lo32(b), hi32(b)) and key (lo32(seed), hi32(seed));
 * the n1 units with the smallest pairs (r_i, i) are treated. With
 * seed == FRR_EXACT_SEED the draw index is instead a colex rank in
 * [0, C(n, n1)), i.e. the position of the n-bit mask in increasing integer
 * order (Sec. 2.3, randomization_type = "exact"); this needs n <= 63.
 *
 * Conventions (all entry points):
 *   - Every call returns frr_status; nothing aborts or throws across the ABI.
 *   - The caller owns every input and output buffer. Buffers marked "host or
 *     device" may live in either memory space: the library asks the CUDA
 *     runtime which one it is and copies as needed. All others are host.
 *   - frr_init copies X; the context owns its device copies, its scratch and,
 *     unless the caller passes one, its CUDA stream.
 *   - A context is not thread-safe: use one per host thread.
 *   - After FRR_E_CUDA the context is unusable; destroy it.
 *   - Calls are synchronous with respect to the host: when a call returns,
 *     its outputs are written.
 */
#ifndef FRR_H
#define FRR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct frr_ctx frr_ctx;

typedef enum {
    FRR_OK = 0,
    FRR_E_ARG = -1,        /* invalid argument: n < 2, n1 not in [1, n-1], d < 1, NULL pointer,
                              non-finite value in X or Y, q not in (0, 1], both or neither of
                              q / threshold given, unknown option value */
    FRR_E_DEGENERATE = -2, /* d >= n-1 with whiten = FRR_CHOL, or a Cholesky pivot <= 1e-12 max S_jj */
    FRR_E_CUDA = -3,       /* a CUDA runtime / driver call failed; the context is unusable */
    FRR_E_NOMEM = -4,      /* device or pinned-host allocation failed */
    FRR_E_TIMEOUT = -5,    /* a bounded device-side wait expired */
    FRR_E_CAPACITY = -6,   /* an output array is smaller than the result (*K_out holds the size needed) */
    FRR_E_RANGE = -7,      /* first_draw + B overflows 64 bits, or an exact rank >= C(n, n1) */
    FRR_E_STATE = -8,      /* call out of sequence (e.g. frr_stream_chunk before frr_stream_begin) */
    FRR_E_UNSUPPORTED = -9, /* shape outside what the compiled kernels cover (n > 2048, exact mode n > 63) */
    FRR_E_MISMATCH = -10    /* internal consistency check failed: two configurations of a kernel disagreed on
                              the same input, or a q-mode selection did not keep exactly K draws */
} frr_status;

/* precision of the bulk balance evaluation (the accepted set is always decided in FP64 accuracy) */
enum { FRR_SPLIT_BF16 = 0, /* tcgen05 tensor cores: Zc = hi + lo (two BF16 parts), FP32 accumulate */
       FRR_F32 = 1 };      /* CUDA-core FP32 SIMT path */

/* whitening rule (Sec. 2.2; App. A "general Sigma_X" remark) */
enum { FRR_CHOL = 0,  /* S = L L^T, Zc = Xc L^{-T}: Hotelling T^2 (needs d <= n - 2) */
       FRR_RIDGE = 1, /* S + ridge * (tr S / d) I = L L^T (any d; needs ridge > 0) */
       FRR_DIAG = 2 };/* L = diag(sqrt(S_jj)): sum of squared standardised mean differences */

/* how frr_init rounds the sums of its FP64 preparation (Sec. 2.2 defines the covariance
 * S = Xc^T Xc / (n - 1), its Cholesky factor S = L L^T and Zc = Xc L^{-T}, not their rounding) */
enum { FRR_PREP_TENSOR = 0,    /* the covariance, and the forward substitution's updates of every column
                                  from the 256-column blocks before it, as exact integer sums on the tensor
                                  cores: each vector (a centred column; a row of Zc or of L over one block)
                                  rounded to a 56-bit integer relative to its largest entry and cut into
                                  eight balanced 7-bit digits, the products of digit pairs summed exactly
                                  (integer-valued FP32 accumulators) and the sum rounded once to FP64 (the
                                  pairs whose weight lies below 2^-56 of the leading one are left out); the
                                  Cholesky factor and the updates inside a block keep FP64 chains, with each
                                  pivot and its column from a reciprocal square root (L_ww = a y, L_rw = t y
                                  with y ~ 1/sqrt(a) within about half an ulp) and the row divisions as
                                  products with the pivot's reciprocal (each within ~1.5 ulp of the
                                  correctly rounded value),
                                  and the column means and the trace as blocked sums.
                                  Each sum is within about (terms) 2^-53 max|a| max|b| of the exact one, the
                                  order of an FP64 dot product's own error; Zc agrees with the FP64 chain to
                                  ~1e-14 of each column's largest entry on the workloads tested. Default. */
       FRR_PREP_FP64_CHAIN = 1 }; /* every dot-product term added by one FP64 fused multiply-add, terms in
                                  ascending order: the operation sequence of the FP64 reference, so that Zc
                                  is bit-identical to it; B300's FP64 rate makes frr_init ~3.8 ms at
                                  n = d = 1000 (~2.0 ms in FRR_PREP_TENSOR) */

#define FRR_EXACT_SEED UINT64_MAX

typedef struct {
    int precision;      /* FRR_SPLIT_BF16 (default) or FRR_F32 */
    int whiten;         /* FRR_CHOL (default), FRR_RIDGE or FRR_DIAG */
    double ridge;       /* ridge weight for FRR_RIDGE, relative to tr(S)/d; default 0.1 */
    double band_safety; /* multiplier on the error band of the approximate M; default 2.0, must be >= 1 */
    void* cuda_stream;  /* cudaStream_t to run on; NULL = the context creates its own */
    int autotune;       /* frr_batch_run only: 1 = time the split-BF16 kernel configurations on a
                           probe of the batch before its launch (see frr_autotune); default 0 */
    int prep;           /* FRR_PREP_TENSOR (default) or FRR_PREP_FP64_CHAIN */
} frr_opts;

typedef struct {
    int64_t draws;              /* draws scored by the last frr_select / stream */
    int64_t candidates;         /* draws re-checked with the FP64-accurate exact-sum recheck */
    int64_t accepted;           /* accepted draws */
    double threshold_m64;       /* largest accepted M (T^2 units) */
    double band_at_threshold;   /* error band of the approximate M at that threshold */
    double max_rel_err;         /* max |M_approx - M64| / M64 over re-checked draws */
    double max_err_over_band;   /* max |M_approx - M64| / band over re-checked draws (must stay < 1) */
    double boundary_gap_rel;    /* (M64[K+1] - M64[K]) / M64[K] among re-checked draws (q mode; NaN if none) */
    int parity_at_risk;         /* 1 if boundary_gap_rel < 1e-11: the K-th / (K+1)-th order rests on rounding */
    int band_violations;        /* re-checked draws with |M_approx - M64| > band (must be 0) */
    double ms_init;             /* wall time of frr_init */
    double ms_balance;          /* device time of the balance kernels in the last call */
    double ms_select;           /* device time of the running selection */
    double ms_recheck;          /* device time of the exact-sum recheck and final ordering */
} frr_stats;

/* Fills *o with the defaults listed above. */
void frr_default_opts(frr_opts* o);

/* Prepares an experiment (Sec. 2.2: centre, covariance with the n-1 denominator,
 * optional ridge, Cholesky factor, whitening Zc = Xc L^{-T}; FP64 on the GPU, its sums
 * rounded as opts.prep says).
 * X: host, n x d row-major FP64 (rows are units). n1: number of treated units.
 * opts: NULL for defaults. On success *out owns device memory; release it with
 * frr_destroy. Supports n <= 2048.
 * The first call of a shape (n, d, n1, whitening, opts.prep) on a device records the
 * preparation's launches as a CUDA graph that keeps its own temporary device block (at most
 * 512 MiB, four shapes per device, least recently used dropped first); later calls of that
 * shape replay it (~200 dependent launches then follow each other sooner on the device, and
 * the host enqueues one graph instead of each launch). A call that finds its shape's graph in
 * use by another thread enqueues the launches itself. */
frr_status frr_init(frr_ctx** out, const double* X, int64_t n, int64_t d, int64_t n1, const frr_opts* opts);

/* Balance of draws [first_draw, first_draw + B) (Sec. 2.1 batched processing,
 * Sec. 2.3 Hotelling T^2). M_out: host or device, B floats, approximate M in
 * T^2 units from the bulk path chosen by opts.precision. */
frr_status frr_balance(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t B, float* M_out);

/* Same as frr_balance with seed = FRR_EXACT_SEED: ranks [first_rank, first_rank + B). */
frr_status frr_balance_exact(frr_ctx* ctx, uint64_t first_rank, uint64_t B, float* M_out);

/* ---- kernel autotuning --------------------------------------------------------------
 * The split-BF16 balance kernel (Sec. 2.1 batched processing) is compiled in several
 * configurations for each number of Philox blocks per lane kb (n <= 128 kb): the number of
 * generating warps per CTA, which sets how many per-draw selections run concurrently on an
 * SM, and the depth of the covariate-tile pipeline in shared memory. All produce
 * bit-identical M_hat. Without tuning a built-in choice per kb is used. */
#define FRR_TUNE_MAX 8
typedef struct {
    int kb;                  /* Philox blocks per lane of the shape class */
    int chunks;              /* covariate chunks of 256 columns, ceil(d / 256) */
    int candidates;          /* configurations timed (entries used below) */
    int chosen;              /* index of the fastest, now used for this shape class */
    int ng[FRR_TUNE_MAX];    /* generating warps per CTA */
    int sb[FRR_TUNE_MAX];    /* covariate-tile stages in shared memory */
    float ms[FRR_TUNE_MAX];  /* fastest timed launch of each on the probe (device ms) */
} frr_tune_result;

/* Times every configuration compiled for this context's kb on B_probe draws of a fixed
 * probe seed (0: 8 tiles of 128 draws per SM; at most 2^24), checks that each reproduces
 * the first one's M_hat bit for bit (else FRR_E_MISMATCH), and makes the fastest the
 * configuration of every later split-BF16 launch of this shape class (device, kb,
 * ceil(d / 256)) in this process, for any context. The context's scratch buffer for
 * M_hat is reused; no other state changes. FRR_E_UNSUPPORTED for an FP32 context. */
frr_status frr_autotune(frr_ctx* ctx, uint64_t B_probe, frr_tune_result* out);

/* Test of the failure path (the paper has no counterpart; for tests only). Runs one
 * split-BF16 balance launch of this context (128 draws per SM) in which the producer of the
 * covariate tiles issues nothing, so the first wait for a tile is never satisfied. Every
 * bounded wait of that launch gives up after wait_cycles SM clock cycles (clamped to
 * [1e4, 2^31]; 2^31, about one second, is the limit of every normal launch): the kernel
 * records which wait expired, releases its tensor memory and returns, and the call returns
 * FRR_E_TIMEOUT with the recorded error cleared and the context still usable. No other call
 * is affected. FRR_E_UNSUPPORTED for an FP32 context. */
frr_status frr_test_wait_expiry(frr_ctx* ctx, uint64_t wait_cycles);

/* Accepted pool of draws [first_draw, first_draw + B) (Sec. 2.2, 2.3). Exactly one of
 * q (0 < q <= 1: keep the K = ceil(qB - 1e-9 qB) draws with the smallest
 * (M, draw index)) and threshold (>= 0: keep every draw with M <= threshold, T^2 units)
 * is used; pass NAN for the other. keys_out (host or device, cap entries): accepted
 * draw indices in ascending order; M64_out (host or device, cap entries, may be NULL):
 * their M in FP64 accuracy. *K_out: number accepted. If K > cap, nothing is written
 * and FRR_E_CAPACITY is returned with *K_out = K. */
frr_status frr_select(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t B, double q,
                      double threshold, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out);

/* Streaming form of frr_select over B_total draws fed in chunks (Sec. 2.1 batched
 * processing; bounded memory). The accepted set after frr_stream_end is identical
 * to one frr_select over the union of the chunks. Chunks may come in any order but
 * must not overlap; their lengths must add up to B_total before frr_stream_end. */
frr_status frr_stream_begin(frr_ctx* ctx, uint64_t seed, double q, double threshold, uint64_t B_total);
frr_status frr_stream_chunk(frr_ctx* ctx, uint64_t first_draw, uint64_t B_chunk);
frr_status frr_stream_end(frr_ctx* ctx, uint64_t* keys_out, double* M64_out, int64_t cap, int64_t* K_out);

/* ---- stream checkpoints (Sec. 2.1 key-only storage) -----------------------------------
 * Between two frr_stream_chunk calls a stream is described by its parameters, its current
 * cut on the approximate M and the retained (draw index, approximate M) pairs -- about K
 * plus the draws inside the error band, 12 bytes each. frr_stream_save writes that state to
 * a caller-owned host blob; frr_stream_load restores it into a context prepared from the
 * same covariates with the same options (in this or another process), after which the
 * remaining chunks and frr_stream_end give exactly the accepted set of the uninterrupted
 * stream.
 *
 * Blob layout, version 1, little-endian: a 256-byte header -- bytes 0-7 "FRRSTRM\0",
 * 8-11 version (uint32), 12-15 header size 256 (uint32), 16-39 n, d, n1 (int64), 40-47
 * precision, whiten (int32), 48-63 ridge, band_safety (double), 64-87 the three error-band
 * constants of the context (double), 88-111 seed, B_total, draws seen so far (uint64),
 * 112-119 exact, q_mode (int32), 120-135 q, threshold (double), 136-151 K, retained count r
 * (int64), 152-155 cut (float), 160-183 the draws / balance / selection statistics (int64,
 * double, double), 184-247 zero, 248-255 FNV-1a 64-bit checksum of the whole blob with these
 * 8 bytes taken as zero -- then r draw indices (uint64) and their r approximate M (float).
 * The blob is 256 + 12 r bytes. */
typedef struct {
    int32_t version;
    int64_t n, d, n1;
    int32_t precision;
    uint64_t seed, total, seen;  /* pool seed, B_total, draws streamed so far */
    double q, threshold;         /* the one not used is NaN */
    int64_t K;                   /* target accepted count (q mode), 0 in threshold mode */
    int64_t retained;            /* retained (candidate) pairs stored in the blob */
} frr_stream_info;

/* Saves the running stream (after frr_stream_begin and any number of chunks). blob: host,
 * cap bytes; *size_out receives the blob's size. blob == NULL or cap too small: nothing is
 * written and FRR_E_CAPACITY is returned with *size_out set. FRR_E_STATE when no stream is
 * running. The stream continues unchanged. */
frr_status frr_stream_save(frr_ctx* ctx, void* blob, size_t cap, size_t* size_out);

/* Replaces the context's stream state with a saved one (any running stream is dropped).
 * FRR_E_ARG for a corrupted blob or one saved by a context of another shape, options or
 * covariates (band constants differ); FRR_E_UNSUPPORTED for an unknown version. */
frr_status frr_stream_load(frr_ctx* ctx, const void* blob, size_t size);

/* Checks a blob (magic, version, size, checksum) without a context or GPU and describes it.
 * FRR_E_ARG for a corrupted blob, FRR_E_UNSUPPORTED for an unknown version. */
frr_status frr_stream_blob_info(const void* blob, size_t size, frr_stream_info* out);

/* Regenerates the assignment of one key (Sec. 2.1 key-only storage).
 * w_out: host or device, n bytes, 1 = treated, in unit order. */
frr_status frr_assignment(frr_ctx* ctx, uint64_t seed, uint64_t key, uint8_t* w_out);

/* Regenerates draws [first_draw, first_draw + count). w_out: host or device, count x n bytes. */
frr_status frr_assignments(frr_ctx* ctx, uint64_t seed, uint64_t first_draw, uint64_t count, uint8_t* w_out);

/* The second half of the key -> assignment mapping on caller-supplied unit words:
 * units whose (word, index) pairs are the n1 smallest are treated, ties in the word
 * broken by the lower unit index (the same warp selection the draws use; this entry
 * point exists to verify it, e.g. on words with ties). words: host or device, n
 * 32-bit words in unit order; w_out: host or device, n bytes. */
frr_status frr_assignment_from_words(frr_ctx* ctx, const uint32_t* words, uint8_t* w_out);

/* M in FP64 accuracy for an explicit list of draws (the same exact-sum recheck that
 * decides acceptance). draws, M64_out: host or device, count entries. */
frr_status frr_recheck(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count, double* M64_out);

/* Allocation-free form of frr_recheck (the paper has no counterpart: this is a property
 * of this library's interface). For callers that must not have the library allocate
 * device memory: a latency-critical loop that shares the GPU with other work, where a
 * cudaMalloc / cudaFree could synchronise the device and stall it, or an application
 * whose device memory belongs to another allocator (for example a framework's caching
 * pool with a fixed budget). draws (count entries) and M64_out (count doubles) must be
 * device memory of the context's GPU (or managed memory), owned by the caller and 8-byte
 * aligned; anything else -- host memory, another GPU's memory -- returns FRR_E_ARG and runs
 * nothing. Pool seeds only (FRR_EXACT_SEED gives FRR_E_UNSUPPORTED); count == 0 returns
 * FRR_OK without touching the buffers. The kernels' scratch -- count * ceil(d / 128)
 * partial sums -- lives in one fixed device array of FRR_RECHECK_STATIC_SCRATCH doubles
 * (1 MiB) compiled into the library, which every GPU that loads the library holds until the
 * process exits; larger requests return FRR_E_CAPACITY and run nothing. The first call on a
 * device looks up that array's device address (set-up), and so does the first call after
 * the device's primary context was destroyed and created again (cudaDeviceReset); make
 * such a first call before any stream capture. Every call on a device shares the array:
 * calls that overlap on the GPU (from other host threads or other contexts on the same
 * device) race, and the caller must serialise them. The call waits for the context's
 * stream before it returns, like the other entry points; it allocates no device or host
 * memory. */
#define FRR_RECHECK_STATIC_SCRATCH 131072
frr_status frr_recheck_static(frr_ctx* ctx, uint64_t seed, const uint64_t* draws, int64_t count, double* M64_out);

/* Randomization test conditional on acceptance and its inversion (Sec. 2.3
 * randomization_test; Sec. 4). Sharp null Y(1) = Y(0) + tau; statistic: the two-sided
 * difference in means. For each tau_g: count_out[g] = #{k : |t_k(tau_g)| >= |t_obs(tau_g)|}
 * over the K accepted assignments (the observed one included, so p >= 1/K), with
 * t_k(tau) = a_k - tau b_k, a_k = DiM_{w_k}(Y), b_k = DiM_{w_k}(w_obs);
 * p_out[g] = count_out[g] / K. The interval is [min, max] of the grid points with
 * p > alpha (NAN, NAN when none). keys: host or device, K entries; obs_key must be
 * one of them. Y: host or device, n. tau: host or device, T. p_out, count_out: host or
 * device, T entries (count_out may be NULL). ci_lo, ci_hi: host, may be NULL. */
frr_status frr_randtest(frr_ctx* ctx, uint64_t seed, const uint64_t* keys, int64_t K, uint64_t obs_key,
                        const double* Y, const double* tau, int64_t T, double alpha,
                        double* p_out, int64_t* count_out, double* ci_lo, double* ci_hi);

/* One experiment of a batched run (Sec. 2.1 "Batched processing": many independent
 * rerandomizations evaluated together). Inputs are read; outputs and results are written
 * by frr_batch_run. Exactly one of q / threshold is used (the other NAN), as in frr_select.
 * Y == NULL skips the randomization test; otherwise w_obs is the accepted key with the
 * smallest draw index, as in the paper's usage example, and the test follows frr_randtest. */
typedef struct {
    const double* X;           /* host, n x d row-major */
    int64_t n, d, n1;
    int whiten;                /* FRR_CHOL, FRR_RIDGE or FRR_DIAG */
    double ridge;
    uint64_t seed, first_draw, B;
    double q, threshold;
    uint64_t* keys_out;        /* host or device, cap entries (ascending draw index) */
    double* M64_out;           /* host or device, cap entries, may be NULL */
    int64_t cap;
    const double* Y;           /* host or device, n, or NULL */
    const double* tau;         /* host or device, T */
    int64_t T;
    double alpha;
    double* p_out;             /* host or device, T */
    int64_t* count_out;        /* host or device, T, may be NULL */
    double ci_lo, ci_hi;       /* out: interval (NAN if empty) */
    int64_t K_out;             /* out: accepted count */
    frr_status status;         /* out: status of this experiment */
} frr_experiment;

typedef struct {
    int64_t experiments, draws, failed;
    double ms_init;            /* wall time of the preparation of all experiments */
    double ms_balance;         /* device time of the balance evaluation of all experiments */
    double ms_select;          /* wall time after the preparation beyond ms_balance: selection, recheck
                                  and tests (issued while the balance runs) */
} frr_batch_stats;

/* Runs E independent experiments (Sec. 2.1 batched processing). All experiments are
 * prepared together (each preparation kernel covers every experiment). With
 * opts->precision = FRR_SPLIT_BF16 the balance of every draw of every experiment is
 * evaluated by one persistent tensor-core launch per class of n (Philox blocks per lane),
 * each over all experiments of its class (shapes may differ), the launches replayed as one
 * CUDA graph; opts->autotune = 1 first times the kernel configurations of each class
 * not yet timed in this process (the choices are kept process-wide).
 * Selection, recheck and tests follow per experiment. Results equal those of frr_init +
 * frr_select (+ frr_randtest) per experiment. opts: NULL for defaults (its whiten and ridge
 * are ignored; each experiment carries its own). Returns FRR_OK if every experiment
 * succeeded, else the first failing status; ex[e].status holds each one. stats may be NULL. */
frr_status frr_batch_run(frr_experiment* ex, int64_t E, const frr_opts* opts, frr_batch_stats* stats);

/* ---- planning diagnostics (Sec. 2.2 "Choosing stringency"; App. A-D) -------------------
 * Host-only scalar math; needs no context and no GPU. k = 1/n_T + 1/n_C and
 * sigma_prog^2 = R2 / (1 - R2) sigma^2. Inputs set to NaN switch their group of outputs off;
 * outputs that were not computed are NaN. */
typedef struct {
    int64_t n_T, n_C;    /* group sizes, >= 1 */
    int64_t d;           /* covariates, >= 1 */
    double R2;           /* share of outcome variance explained by the covariates, [0, 1) */
    double sigma;        /* residual standard deviation, > 0 */
    double q;            /* acceptance probability (0, 1] for the ex-ante outputs, or NaN */
    double M_obs;        /* an observed imbalance M >= 0 for the realised outputs, or NaN */
    double tau;          /* effect size of interest for power and q*, or NaN */
    double alpha;        /* two-sided size, (0, 1); read only when tau is given */
    double power;        /* target power, (0, 1); read only when tau is given */
} frr_diag_in;

typedef struct {
    double k;                /* 1/n_T + 1/n_C */
    double sigma2_prog;      /* R2 / (1 - R2) sigma^2 */
    double rmse_complete;    /* ex-ante RMSE under complete randomization, sqrt(k (sigma^2 + sigma2_prog)) (App. B) */
    /* from M_obs (App. A) */
    double rmse_realised;    /* typical orientation: sqrt(sigma^2 k + sigma2_prog M / d) */
    double rmse_cs_bound;    /* Cauchy-Schwarz upper bound: sqrt(sigma^2 k + sigma2_prog M) */
    /* at q (Sec. 2.2, App. C) */
    double c_q;              /* chi2_d quantile at q (inf at q = 1) */
    double a_q;              /* implied threshold on M, k c_q */
    double v_a;              /* shrinkage factor P(chi2_{d+2} <= c_q) / q */
    double rmse_accept;      /* ex-ante RMSE given acceptance, sqrt(k (sigma^2 + v_a sigma2_prog)) */
    double rmse_reduction;   /* 1 - rmse_accept / rmse_complete */
    double expected_M;       /* E[M | accept] = k d v_a */
    double power_at_q;       /* two-sided normal-approximation power at tau (needs tau) */
    /* inversion for tau, alpha, power (App. D) */
    double snr_needed;       /* z_{1-alpha/2} + z_{power} */
    double q_star;           /* largest q with rmse_accept(q) <= |tau| / snr_needed; 0 below the double range */
    double log10_q_star;     /* log10 of q_star, finite even where q_star underflows */
    double c_star;           /* chi-square cut at q_star */
    double v_star;           /* v_a at q_star */
    double draws_per_accept; /* 1 / q_star */
    int32_t q_star_status;   /* 0 found by the line search, 1 q = 1 already meets the target,
                                2 unreachable (sigma^2 k alone exceeds the target), -1 not asked */
} frr_diag_out;

/* Fills *out from *in. FRR_E_ARG for a NULL pointer or an input outside the ranges above. */
frr_status frr_diagnose(const frr_diag_in* in, frr_diag_out* out);

/* ---- pairwise distances (Sec. 4 "Compatibility and ecosystem", fast_distance) ---------
 * D[i * m + j] = ||X_i - Y_j||_2 for the rows of X (n x d) and Y (m x d), row-major FP32,
 * or its square when squared != 0. Y == NULL means Y = X (m is then ignored). X, Y and
 * D_out may each be host or device memory; the call returns when D_out is written. Work
 * runs on cuda_stream (NULL = the default stream). Every temporary -- the split operands
 * ((n + m) * 6 dp bytes), the norms, and for host buffers the device copies of X, Y and D_out
 * -- comes from a memory pool the library keeps per device, which retains its largest
 * footprint for later calls until the process exits.
 * The cross term runs on the tensor cores with each value split into two BF16 parts and
 * FP32 accumulation; the squared norms are compensated sums rounded once to FP32.
 * |D^2 - exact| <= (3 * 2^-18 + (3 dp + 4) * 2^-24) (||X_i||^2 + ||Y_j||^2) with dp = d
 * rounded up to 64 (a worst-case bound; typical errors are far smaller).
 * FRR_E_ARG for NULL X / D_out or n, m, d < 1; FRR_E_UNSUPPORTED for n or m > 2^30 or
 * d > 2^20; FRR_E_NOMEM if the temporaries do not fit. */
frr_status frr_fast_distance(const float* X, int64_t n, const float* Y, int64_t m, int64_t d, int squared,
                             float* D_out, void* cuda_stream);

/* Copies the whitened covariates Zc (host, n x d row-major FP64) out of the context. */
frr_status frr_whitened(const frr_ctx* ctx, double* Zc_out);

/* Statistics of the last call (see frr_stats). */
frr_status frr_last_stats(const frr_ctx* ctx, frr_stats* out);

/* Static description of a status code. */
const char* frr_strerror(frr_status status);

/* Releases everything the context owns. NULL is ignored. */
void frr_destroy(frr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FRR_H */
