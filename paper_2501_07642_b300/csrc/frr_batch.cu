// frr_batch.cu -- frr_batch_run: many independent experiments, one balance launch.
//
// Sec. 2.1 evaluates candidates in batches to amortise launches and saturate the
// device. Here the batch is a set of whole experiments of uneven n and d: each is
// prepared (FP64 init) on its own, then the approximate balance of every draw of every
// experiment comes from ONE persistent tcgen05 launch whose global tile index space
// concatenates the experiments' draw tiles (experiment tables in device memory), so
// small and large experiments share all SMs. Selection, exact recheck and the
// randomization test then run per experiment on the resulting M_hat arrays. Preparation
// and the per-experiment stages run on several host threads, one stream each, so that the
// small kernels of different experiments run concurrently.
#include "frr_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cuda.h>
#include <thread>
#include <vector>

#include "frr_tcexp.cuh"

namespace frr {

frr_status tc_describe(frr_ctx* ctx, uint64_t seed, bool exact, uint64_t first, uint64_t B, float* Mout, TcExp* x);
frr_status balance_tc_batch_launch(frr_ctx* owner, cudaStream_t stream, const TcExp* table,
                                   const unsigned long long* prefix, int E, unsigned long long tiles, int kbmax,
                                   int nchmax, int* err);
frr_status balance_tc_batch_tune(frr_ctx* owner, cudaStream_t stream, const TcExp* table,
                                 const unsigned long long* prefix, int E, unsigned long long tiles, int kbmax,
                                 int nchmax, int* err);

}  // namespace frr

using namespace frr;

namespace {

// host worker threads of the batched driver (each owns one stream)
constexpr int kWorkers = 8;

template <typename F>
void run_workers(int nw, F&& f)
{
    std::vector<std::thread> th;
    th.reserve((size_t)nw);
    for (int w = 1; w < nw; ++w) th.emplace_back(f, w);
    f(0);
    for (auto& t : th) t.join();
}

}  // namespace

extern "C" frr_status frr_batch_run(frr_experiment* ex, int64_t E, const frr_opts* opts, frr_batch_stats* stats)
{
    if (!ex || E < 1) return FRR_E_ARG;
    frr_opts base;
    frr_default_opts(&base);
    if (opts) base = *opts;
    if (base.precision != FRR_SPLIT_BF16 && base.precision != FRR_F32) return FRR_E_ARG;
    if (base.autotune != 0 && base.autotune != 1) return FRR_E_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<frr_ctx*> ctx((size_t)E, nullptr);
    frr_status first_err = FRR_OK;
    auto note = [&](int64_t e, frr_status s) {
        ex[e].status = s;
        if (s != FRR_OK && first_err == FRR_OK) first_err = s;
    };
    cudaStream_t stream = static_cast<cudaStream_t>(base.cuda_stream);
    bool own_stream = false;
    if (!stream) {
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); return FRR_E_CUDA; }
        own_stream = true;
    }
    int64_t draws = 0;
    // Preparation (FP64, latency-bound on B300) of several experiments at once: worker
    // threads, each with its own stream, so that their small kernels share the SMs (the
    // contexts allocate stream-ordered from a pool, so the threads do not synchronise the
    // device through allocations).
    const int nw = (int)std::min<int64_t>(kWorkers, E);
    std::vector<cudaStream_t> ws((size_t)nw, nullptr);
    for (int w = 0; w < nw; ++w)
        if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ws[w] = stream;
        }
    std::vector<frr_status> st_init((size_t)E, FRR_OK);
    // argument checks and context creation on the worker threads (each context later runs
    // its selection on the stream of the worker that created it)
    auto create = [&](int w) {
        for (int64_t e = w; e < E; e += nw) {
            ex[e].K_out = 0;
            ex[e].ci_lo = ex[e].ci_hi = NAN;
            const bool hq = !isnan(ex[e].q), ht = !isnan(ex[e].threshold);
            if (hq == ht || (hq && !(ex[e].q > 0.0 && ex[e].q <= 1.0)) || (ht && !(ex[e].threshold >= 0.0)) ||
                ex[e].B == 0 || ex[e].first_draw + ex[e].B < ex[e].first_draw) {
                st_init[e] = FRR_E_ARG;
                continue;
            }
            frr_opts o = base;
            o.whiten = ex[e].whiten;
            o.ridge = ex[e].ridge;
            o.cuda_stream = ws[w];
            frr_status s = check_init_args(ex[e].X, ex[e].n, ex[e].d, ex[e].n1, o);
            if (s == FRR_OK && ex[e].seed == FRR_EXACT_SEED) {
                if (ex[e].n > kExactMaxN) s = FRR_E_UNSUPPORTED;
                else if (ex[e].first_draw + ex[e].B > binom_host((int)ex[e].n, (int)ex[e].n1)) s = FRR_E_RANGE;
            }
            if (s == FRR_OK) s = ctx_create(&ctx[e], ex[e].n, ex[e].d, ex[e].n1, o, false);
            st_init[e] = s;
        }
        // the contexts' arrays come from stream-ordered allocations on this worker's stream
        if (cudaStreamSynchronize(ws[w]) != cudaSuccess) cudaGetLastError();
    };
    run_workers(nw, create);
    {
        // one preparation of every created context: each launch covers all of them
        std::vector<frr_ctx*> pc;
        std::vector<const double*> px;
        std::vector<int64_t> pe;
        for (int64_t e = 0; e < E; ++e)
            if (ctx[e]) {
                pc.push_back(ctx[e]);
                px.push_back(ex[e].X);
                pe.push_back(e);
            }
        if (!pc.empty()) {
            cudaStream_t paux = nullptr;
            std::vector<frr_status> pst(pc.size(), FRR_E_CUDA);
            if (cudaStreamCreateWithFlags(&paux, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
            } else {
                prep_run_batch(pc.data(), px.data(), (int)pc.size(), stream, paux, pst.data());
                cudaStreamDestroy(paux);
            }
            for (size_t k = 0; k < pc.size(); ++k) {
                st_init[(size_t)pe[k]] = pst[k];
                if (pst[k] != FRR_OK) {
                    ctx_release(ctx[(size_t)pe[k]]);
                    ctx[(size_t)pe[k]] = nullptr;
                }
            }
        }
    }
    for (int64_t e = 0; e < E; ++e) note(e, st_init[e]);
    const auto t1 = std::chrono::steady_clock::now();

    // approximate M of every draw of every prepared experiment
    std::vector<int64_t> live;
    for (int64_t e = 0; e < E; ++e)
        if (ctx[e]) live.push_back(e);
    float* mhat = nullptr;
    TcExp* d_table = nullptr;
    unsigned long long* d_prefix = nullptr;
    int* d_err = nullptr;
    float ms_balance = 0.f;
    frr_status rc = FRR_OK;
    if (!live.empty()) {
        std::vector<size_t> off(live.size() + 1, 0);
        for (size_t k = 0; k < live.size(); ++k) off[k + 1] = off[k] + ex[live[k]].B;
        frr_ctx* owner = ctx[live[0]];
        cudaEvent_t ea, eb;
        cudaEventCreate(&ea);
        cudaEventCreate(&eb);
        if (cudaMalloc(&mhat, off.back() * sizeof(float)) != cudaSuccess) { cudaGetLastError(); rc = FRR_E_NOMEM; }
        if (rc == FRR_OK && base.precision == FRR_SPLIT_BF16) {
            std::vector<TcExp> table(live.size());
            std::vector<unsigned long long> prefix(live.size() + 1, 0);
            int kbmax = 1, nchmax = 1;
            for (size_t k = 0; k < live.size() && rc == FRR_OK; ++k) {
                const frr_experiment& x = ex[live[k]];
                rc = tc_describe(ctx[live[k]], x.seed, x.seed == FRR_EXACT_SEED, x.first_draw, x.B, mhat + off[k],
                                 &table[k]);
                prefix[k + 1] = prefix[k] + (x.B + 127) / 128;
                if (ctx[live[k]]->kb > kbmax) kbmax = ctx[live[k]]->kb;
                if (table[k].nchunks > nchmax) nchmax = table[k].nchunks;
            }
            // probe batch for the tuner: every experiment with about 1/16 of its draws
            std::vector<TcExp> probe;
            std::vector<unsigned long long> probe_prefix;
            if (rc == FRR_OK && base.autotune) {
                probe = table;
                probe_prefix.assign(live.size() + 1, 0);
                for (size_t k = 0; k < live.size(); ++k) {
                    const uint64_t tiles_k = (probe[k].B + 127) / 128;
                    const uint64_t pt = std::max<uint64_t>(1, tiles_k / 16);
                    probe[k].B = std::min<uint64_t>(probe[k].B, pt * 128);
                    probe_prefix[k + 1] = probe_prefix[k] + pt;
                }
            }
            if (rc == FRR_OK &&
                (cudaMalloc(&d_table, table.size() * sizeof(TcExp)) != cudaSuccess ||
                 cudaMalloc(&d_prefix, prefix.size() * sizeof(unsigned long long)) != cudaSuccess ||
                 cudaMalloc(&d_err, sizeof(int)) != cudaSuccess)) {
                cudaGetLastError();
                rc = FRR_E_NOMEM;
            }
            if (rc == FRR_OK && base.autotune) {
                cudaMemcpyAsync(d_table, probe.data(), probe.size() * sizeof(TcExp), cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(d_prefix, probe_prefix.data(), probe_prefix.size() * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, stream);
                cudaMemsetAsync(d_err, 0, sizeof(int), stream);
                rc = balance_tc_batch_tune(owner, stream, d_table, d_prefix, (int)live.size(), probe_prefix.back(),
                                           kbmax, nchmax, d_err);
                int herr = 0;
                if (rc == FRR_OK && (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                                     cudaStreamSynchronize(stream) != cudaSuccess)) {
                    cudaGetLastError();
                    rc = FRR_E_CUDA;
                } else if (rc == FRR_OK && herr != 0) {
                    rc = FRR_E_TIMEOUT;
                }
            }
            if (rc == FRR_OK) {
                cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(TcExp), cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(d_prefix, prefix.data(), prefix.size() * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, stream);
                cudaMemsetAsync(d_err, 0, sizeof(int), stream);
                cudaEventRecord(ea, stream);
                rc = balance_tc_batch_launch(owner, stream, d_table, d_prefix, (int)live.size(), prefix.back(), kbmax,
                                             nchmax, d_err);
                cudaEventRecord(eb, stream);
                int herr = 0;
                if (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                    cudaStreamSynchronize(stream) != cudaSuccess) {
                    cudaGetLastError();
                    rc = FRR_E_CUDA;
                } else if (herr != 0) {
                    rc = FRR_E_TIMEOUT;
                }
            }
        } else if (rc == FRR_OK) {
            cudaEventRecord(ea, stream);
            // FP32: one launch per experiment, on its context's stream
            for (size_t k = 0; k < live.size() && rc == FRR_OK; ++k) {
                const frr_experiment& x = ex[live[k]];
                rc = balance_f32_launch(ctx[live[k]], x.seed, x.seed == FRR_EXACT_SEED, x.first_draw, x.B, mhat + off[k]);
            }
            for (cudaStream_t w : ws)
                if (cudaStreamSynchronize(w) != cudaSuccess) { cudaGetLastError(); rc = FRR_E_CUDA; }
            cudaEventRecord(eb, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) { cudaGetLastError(); rc = FRR_E_CUDA; }
        }
        cudaEventElapsedTime(&ms_balance, ea, eb);
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        // selection, recheck and tests per experiment, on the workers' streams (each context
        // is used by one thread only)
        std::vector<frr_status> st_sel(live.size(), FRR_OK);
        auto finish = [&](int w) {
            for (size_t k = (size_t)w; k < live.size(); k += (size_t)nw) {
                const int64_t e = live[k];
                frr_experiment& x = ex[e];
                if (rc != FRR_OK) { st_sel[k] = rc; continue; }
                frr_status s = stream_begin(ctx[e], x.seed, x.q, x.threshold, x.B);
                if (s == FRR_OK) s = stream_chunk_precomputed(ctx[e], x.first_draw, x.B, mhat + off[k]);
                int64_t K = 0;
                if (s == FRR_OK) s = stream_end(ctx[e], x.keys_out, x.M64_out, x.cap, &K);
                x.K_out = K;
                if (s == FRR_OK && x.Y != nullptr && K > 0) {
                    uint64_t obs = 0;
                    s = copy_out(ctx[e], &obs, x.keys_out, sizeof(uint64_t));
                    if (s == FRR_OK) {
                        if (!x.tau || x.T < 1 || !x.p_out || !(x.alpha >= 0.0 && x.alpha <= 1.0)) s = FRR_E_ARG;
                        else s = randtest_run(ctx[e], x.seed, x.keys_out, K, obs, x.Y, x.tau, x.T, x.alpha, x.p_out,
                                              x.count_out, &x.ci_lo, &x.ci_hi);
                    }
                }
                st_sel[k] = s;
            }
        };
        run_workers(nw, finish);
        for (size_t k = 0; k < live.size(); ++k) {
            note(live[k], st_sel[k]);
            draws += (int64_t)ex[live[k]].B;
        }
    }
    const auto t2 = std::chrono::steady_clock::now();
    cudaFree(mhat);
    cudaFree(d_table);
    cudaFree(d_prefix);
    cudaFree(d_err);
    for (frr_ctx* c : ctx) frr_destroy(c);
    for (cudaStream_t w : ws)
        if (w != stream) cudaStreamDestroy(w);
    if (own_stream) cudaStreamDestroy(stream);
    if (stats) {
        stats->experiments = E;
        stats->draws = draws;
        int64_t failed = 0;
        for (int64_t e = 0; e < E; ++e) failed += ex[e].status != FRR_OK ? 1 : 0;
        stats->failed = failed;
        stats->ms_init = std::chrono::duration<double, std::milli>(t1 - t0).count();
        stats->ms_balance = ms_balance;
        stats->ms_select = std::chrono::duration<double, std::milli>(t2 - t1).count() - ms_balance;
    }
    return first_err;
}
