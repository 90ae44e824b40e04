// frr_batch.cu -- frr_batch_run: many independent experiments, few launches.
//
// Sec. 2.1 evaluates candidates in batches to amortise launches and saturate the
// device. Here the batch is a set of whole experiments of uneven n and d:
//   1. contexts are created (argument checks, fixed arrays) on a few host threads;
//   2. all experiments are prepared together (FP64 init): every preparation kernel covers
//      the blocks of every experiment (frr_prep.cu), one synchronisation at the end;
//   3. the approximate balance of every draw of every experiment comes from one persistent
//      tcgen05 launch per class of Philox blocks per lane (experiment tables in device
//      memory, so small and large experiments share all SMs), the launches captured as
//      parallel branches of one CUDA graph; the kernel configuration of each class is the
//      built-in or autotuned one;
//   4. selection, exact recheck and the randomization test run per experiment on the
//      resulting M_hat arrays, on the host threads, one stream each, so that the small
//      kernels of different experiments run concurrently.
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

// host threads that check arguments, copy the covariates into the pinned staging block (with
// the scan for non-finite values) and create contexts: one per hardware thread, at most 16;
// with the 256-experiment workload (226 MB of covariates) on 16 host threads, 16 of them
// prepare ~2 ms sooner than 8, and 8 about 6 ms sooner than 4. The selection chains are
// enqueued from one thread: from several, the driver's calls contended (4 threads were
// 40-60 % slower for that phase)
constexpr int kMaxWorkers = 16;
constexpr size_t kLendBytes = size_t(4) << 20;  // lent scratch per experiment
int worker_count()
{
    const unsigned hw = std::thread::hardware_concurrency();
    return hw == 0 ? 8 : (int)std::min<unsigned>(hw, kMaxWorkers);
}
// streams of the contexts: the selection and test chains of different experiments overlap
constexpr int kStreams = 8;

template <typename F>
void run_workers(int nw, F&& f)
{
    // the workers use the calling thread's device (a new thread starts on device 0)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    std::vector<std::thread> th;
    th.reserve((size_t)nw);
    for (int w = 1; w < nw; ++w)
        th.emplace_back([&f, dev, w] {
            cudaSetDevice(dev);
            f(w);
        });
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
    const int nw = (int)std::min<int64_t>(worker_count(), E);
    // the contexts' streams, assigned round-robin (experiment e runs on ws[e % ns])
    const int ns = (int)std::min<int64_t>(kStreams, E);
    std::vector<cudaStream_t> ws((size_t)ns, nullptr);
    for (int w = 0; w < ns; ++w)
        if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            ws[w] = stream;
        }
    std::vector<frr_status> st_init((size_t)E, FRR_OK);
    // The covariates go to the device through one pinned staging block (the copy into it is
    // also the check for non-finite values), so that their upload is DMA from pinned memory
    // rather than the driver staging pageable memory on the calling thread.
    std::vector<size_t> xoff((size_t)E + 1, 0);
    for (int64_t e = 0; e < E; ++e) {
        const bool sized = ex[e].X && ex[e].n >= 2 && ex[e].n <= kMaxN && ex[e].d >= 1 && ex[e].d <= (1 << 20);
        xoff[(size_t)e + 1] = xoff[(size_t)e] + (sized ? (size_t)ex[e].n * (size_t)ex[e].d : 0);
    }
    size_t stage_cap = 0;
    double* stage = xoff[(size_t)E] > 0
                        ? static_cast<double*>(pinned_get(xoff[(size_t)E] * sizeof(double), &stage_cap))
                        : nullptr;
    // argument checks and context creation on the worker threads
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
            o.cuda_stream = ws[(size_t)(e % ns)];
            frr_status s = check_init_args(ex[e].X, ex[e].n, ex[e].d, ex[e].n1, o, stage == nullptr);
            if (s == FRR_OK && stage) s = stage_finite(ex[e].X, ex[e].n * ex[e].d, stage + xoff[(size_t)e]);
            if (s == FRR_OK && ex[e].seed == FRR_EXACT_SEED) {
                if (ex[e].n > kExactMaxN) s = FRR_E_UNSUPPORTED;
                else if (ex[e].first_draw + ex[e].B > binom_host((int)ex[e].n, (int)ex[e].n1)) s = FRR_E_RANGE;
            }
            if (s == FRR_OK) s = ctx_create(&ctx[e], ex[e].n, ex[e].d, ex[e].n1, o, false);
            st_init[e] = s;
        }
    };
    run_workers(nw, create);
    // the contexts' arrays come from stream-ordered allocations on their streams
    for (cudaStream_t w : ws)
        if (cudaStreamSynchronize(w) != cudaSuccess) cudaGetLastError();
    {
        // one preparation of every created context: each launch covers all of them
        std::vector<frr_ctx*> pc;
        std::vector<const double*> px;
        std::vector<int64_t> pe;
        for (int64_t e = 0; e < E; ++e)
            if (ctx[e]) {
                pc.push_back(ctx[e]);
                px.push_back(stage ? stage + xoff[(size_t)e] : ex[e].X);
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
            // (the uploads from the staging block have finished even if the preparation failed)
            if (cudaStreamSynchronize(stream) != cudaSuccess) cudaGetLastError();
            pinned_put(stage, stage_cap);
            stage = nullptr;
            for (size_t k = 0; k < pc.size(); ++k) {
                st_init[(size_t)pe[k]] = pst[k];
                if (pst[k] != FRR_OK) {
                    ctx_release(ctx[(size_t)pe[k]]);
                    ctx[(size_t)pe[k]] = nullptr;
                }
            }
        }
    }
    pinned_put(stage, stage_cap);  // (when nothing was prepared)
    for (int64_t e = 0; e < E; ++e) note(e, st_init[e]);
    const auto t1 = std::chrono::steady_clock::now();

    // approximate M of every draw of every prepared experiment
    std::vector<int64_t> live;
    for (int64_t e = 0; e < E; ++e)
        if (ctx[e]) live.push_back(e);
    float* mhat = nullptr;
    char* lend_block = nullptr;  // the experiments' lent scratch (ensure_device)
    TcExp* d_table = nullptr;
    unsigned long long* d_prefix = nullptr;
    int* d_err = nullptr;
    float ms_balance = 0.f;
    frr_status rc = FRR_OK;
    // the balance graph and what it uses, kept until the end of the batch (the selection is
    // issued while the graph runs); bal_err: its error word, read once the selection is issued
    cudaGraph_t bal_graph = nullptr;
    cudaGraphExec_t bal_exec = nullptr;
    std::vector<cudaEvent_t> bal_gev;
    std::vector<cudaStream_t> bal_gs;
    const int* bal_err = nullptr;
    if (!live.empty()) {
        std::vector<size_t> off(live.size() + 1, 0);
        for (size_t k = 0; k < live.size(); ++k) off[k + 1] = off[k] + ex[live[k]].B;
        frr_ctx* owner = ctx[live[0]];
        cudaEvent_t ea, eb;
        cudaEventCreate(&ea);
        cudaEventCreate(&eb);
        if (cudaMalloc(&mhat, off.back() * sizeof(float)) != cudaSuccess) { cudaGetLastError(); rc = FRR_E_NOMEM; }
        if (rc == FRR_OK) {
            // Each experiment's selection chain draws its scratch (retained sets, recheck rows,
            // test buffers) from a slice of one block instead of ~6 stream-ordered allocations,
            // which cost the issuing thread ~25 us each while the balance runs (~1500 per
            // 256-experiment batch: longer than the balance itself on a slower host). A chain
            // that needs more than its slice takes the rest from the pool.
            cudaMemPool_t pool = temp_pool(owner->device);
            if (pool != nullptr &&
                cudaMallocFromPoolAsync(reinterpret_cast<void**>(&lend_block), live.size() * kLendBytes, pool, stream) ==
                    cudaSuccess &&
                cudaStreamSynchronize(stream) == cudaSuccess) {
                for (size_t k = 0; k < live.size(); ++k) {
                    frr_ctx* c = ctx[live[k]];
                    c->lend = lend_block + k * kLendBytes;
                    c->lend_off = 0;
                    c->lend_cap = kLendBytes;
                }
            } else {
                cudaGetLastError();
                lend_block = nullptr;
            }
        }
        if (rc == FRR_OK && base.precision == FRR_SPLIT_BF16) {
            // Experiments are grouped by Philox blocks per lane (kb): each group runs in a
            // persistent launch of the kernel configuration compiled (and tuned) for its kb, so
            // short experiments get many generating warps instead of the register budget of the
            // longest one. The group launches are captured as parallel branches of one CUDA
            // graph; a group's CTAs start on the SMs that the previous group's tail frees.
            std::vector<TcExp> desc(live.size());
            for (size_t k = 0; k < live.size() && rc == FRR_OK; ++k) {
                const frr_experiment& x = ex[live[k]];
                rc = tc_describe(ctx[live[k]], x.seed, x.seed == FRR_EXACT_SEED, x.first_draw, x.B, mhat + off[k],
                                 &desc[k]);
            }
            struct Group {
                int kb = 0, nch = 1;
                size_t t0 = 0, cnt = 0;          // slice of the concatenated tables
                size_t p0 = 0, pp0 = 0;          // slices of the concatenated prefix arrays
                unsigned long long tiles = 0, probe_tiles = 0;
            };
            std::vector<Group> groups;
            std::vector<TcExp> table, probe;
            std::vector<unsigned long long> prefix, probe_prefix;
            for (int kb = 16; kb >= 1 && rc == FRR_OK; kb >>= 1) {
                Group g;
                g.kb = kb;
                g.t0 = table.size();
                g.p0 = prefix.size();
                g.pp0 = probe_prefix.size();
                prefix.push_back(0);
                probe_prefix.push_back(0);
                for (size_t k = 0; k < live.size(); ++k) {
                    if (ctx[live[k]]->kb != kb) continue;
                    table.push_back(desc[k]);
                    const uint64_t tk = (desc[k].B + 127) / 128;
                    g.tiles += tk;
                    prefix.push_back(g.tiles);
                    g.nch = std::max(g.nch, desc[k].nchunks);
                    // probe for the tuner: about 1/16 of each experiment's tiles
                    TcExp pr = desc[k];
                    const uint64_t pt = std::max<uint64_t>(1, tk / 16);
                    pr.B = std::min<uint64_t>(pr.B, pt * 128);
                    probe.push_back(pr);
                    g.probe_tiles += pt;
                    probe_prefix.push_back(g.probe_tiles);
                }
                g.cnt = table.size() - g.t0;
                if (g.cnt == 0) {
                    prefix.resize(g.p0);
                    probe_prefix.resize(g.pp0);
                    continue;
                }
                groups.push_back(g);
            }
            // one device block: tables, probe tables, prefixes, probe prefixes, error word
            const size_t tb = table.size() * sizeof(TcExp);
            const size_t pb = prefix.size() * sizeof(unsigned long long);
            const size_t ppb = probe_prefix.size() * sizeof(unsigned long long);
            char* dbuf = nullptr;
            if (rc == FRR_OK && cudaMalloc(&dbuf, 2 * tb + pb + ppb + 256) != cudaSuccess) {
                cudaGetLastError();
                rc = FRR_E_NOMEM;
            }
            if (rc == FRR_OK) {
                d_table = reinterpret_cast<TcExp*>(dbuf);
                TcExp* d_probe = reinterpret_cast<TcExp*>(dbuf + tb);
                d_prefix = reinterpret_cast<unsigned long long*>(dbuf + 2 * tb);
                unsigned long long* d_pprefix = reinterpret_cast<unsigned long long*>(dbuf + 2 * tb + pb);
                d_err = reinterpret_cast<int*>(dbuf + 2 * tb + pb + ppb);
                cudaMemcpyAsync(d_table, table.data(), tb, cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(d_probe, probe.data(), tb, cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(d_prefix, prefix.data(), pb, cudaMemcpyHostToDevice, stream);
                cudaMemcpyAsync(d_pprefix, probe_prefix.data(), ppb, cudaMemcpyHostToDevice, stream);
                cudaMemsetAsync(d_err, 0, sizeof(int), stream);
                for (const Group& g : groups) {
                    if (!base.autotune || rc != FRR_OK) break;
                    rc = balance_tc_batch_tune(owner, stream, d_probe + g.t0, d_pprefix + g.pp0, (int)g.cnt,
                                               g.probe_tiles, g.kb, g.nch, d_err);
                }
                // the launches of all groups as one graph: a fork from `stream`, one branch per
                // group on its own capture stream, joined back into `stream`
                std::vector<cudaStream_t> gs(groups.size(), nullptr);
                std::vector<cudaEvent_t> gev(groups.size() + 1, nullptr);
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                bool ok = rc == FRR_OK;
                for (size_t i = 0; i < groups.size() && ok; ++i)
                    ok = cudaStreamCreateWithFlags(&gs[i], cudaStreamNonBlocking) == cudaSuccess;
                for (size_t i = 0; i < gev.size() && ok; ++i)
                    ok = cudaEventCreateWithFlags(&gev[i], cudaEventDisableTiming) == cudaSuccess;
                if (ok && cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                    bool cap = cudaEventRecord(gev[0], stream) == cudaSuccess;
                    for (size_t i = 0; i < groups.size() && cap; ++i) {
                        const Group& g = groups[i];
                        cap = cudaStreamWaitEvent(gs[i], gev[0], 0) == cudaSuccess &&
                              balance_tc_batch_launch(owner, gs[i], d_table + g.t0, d_prefix + g.p0, (int)g.cnt,
                                                      g.tiles, g.kb, g.nch, d_err) == FRR_OK &&
                              cudaEventRecord(gev[i + 1], gs[i]) == cudaSuccess &&
                              cudaStreamWaitEvent(stream, gev[i + 1], 0) == cudaSuccess;
                    }
                    const bool ended = cudaStreamEndCapture(stream, &graph) == cudaSuccess;
                    ok = cap && ended && graph != nullptr &&
                         cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
                } else {
                    ok = false;
                }
                if (ok) {
                    cudaEventRecord(ea, stream);
                    ok = cudaGraphLaunch(exec, stream) == cudaSuccess;
                    cudaEventRecord(eb, stream);
                }
                if (rc == FRR_OK && !ok) {
                    cudaGetLastError();
                    rc = FRR_E_CUDA;
                }
                if (rc == FRR_OK) {
                    // The experiments' streams wait for the balance on the device, so that this
                    // thread issues their selection chains while the graph runs.
                    for (cudaStream_t w : ws)
                        if (cudaStreamWaitEvent(w, eb, 0) != cudaSuccess) { cudaGetLastError(); rc = FRR_E_CUDA; }
                    bal_err = d_err;
                }
                bal_exec = exec;
                bal_graph = graph;
                bal_gev = gev;
                bal_gs = gs;
                cudaGetLastError();
            }
            d_prefix = nullptr;  // parts of dbuf
            d_err = nullptr;
            d_table = reinterpret_cast<TcExp*>(dbuf);
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
        // Selection, recheck and tests, issued from this thread. q-mode experiments whose test
        // inputs are in host memory are pipelined: each one's whole chain is enqueued on its
        // context's stream without a read-back (q mode accepts exactly K draws, so the test
        // reads the placed keys on the device), and the results are collected after every
        // chain is enqueued. The others (threshold mode, device test inputs) run one by one.
        std::vector<frr_status> st_sel(live.size(), FRR_OK);
        auto one_by_one = [&](size_t k, bool defer) -> frr_status {
            const int64_t e = live[k];
            frr_experiment& x = ex[e];
            frr_status s = stream_begin(ctx[e], x.seed, x.q, x.threshold, x.B);
            // one chunk: the recheck may read the candidate count on the device
            ctx[e]->st.defer_count = defer;
            if (s == FRR_OK) s = stream_chunk_precomputed(ctx[e], x.first_draw, x.B, mhat + off[k]);
            int64_t K = 0;
            if (s == FRR_OK) s = stream_end(ctx[e], x.keys_out, x.M64_out, x.cap, &K);
            x.K_out = K;
            if (s == FRR_OK && x.Y != nullptr && K > 0) {
                uint64_t obs = 0;
                if (is_device_ptr(x.keys_out)) s = copy_out(ctx[e], &obs, x.keys_out, sizeof(uint64_t));
                else obs = x.keys_out[0];
                if (s == FRR_OK) {
                    if (!x.tau || x.T < 1 || !x.p_out || !(x.alpha >= 0.0 && x.alpha <= 1.0)) s = FRR_E_ARG;
                    else s = randtest_run(ctx[e], x.seed, x.keys_out, K, obs, x.Y, x.tau, x.T, x.alpha, x.p_out,
                                          x.count_out, &x.ci_lo, &x.ci_hi);
                }
            }
            return s;
        };
        struct Pending {
            bool piped = false, test = false, p_dev = false, c_dev = false;
            size_t off = 0;
        };
        std::vector<Pending> pend(live.size());
        for (size_t k = 0; k < live.size() && rc == FRR_OK; ++k) {
            const int64_t e = live[k];
            frr_experiment& x = ex[e];
            frr_ctx* c = ctx[e];
            const bool host_test = x.Y == nullptr || (!is_device_ptr(x.Y) && x.tau != nullptr && !is_device_ptr(x.tau));
            if (isnan(x.q) || !host_test) continue;
            Pending& P = pend[k];
            P.piped = true;
            frr_status s = stream_begin(c, x.seed, x.q, x.threshold, x.B);
            c->st.defer_count = true;
            c->st.timing = false;  // per-experiment phase times are not reported by the batch
            if (s == FRR_OK) {
                // the context's pinned block, sized once before anything is in flight on its
                // (shared) stream: growing it later would wait for the stream
                const size_t need = stream_end_pinned_bound(c, x.cap) + (x.Y ? (size_t)std::max<int64_t>(x.T, 0) * 16 + 16 : 0);
                if (need <= (size_t(1) << 20)) s = ensure_host_pinned(c, need);
            }
            if (s == FRR_OK) s = stream_chunk_precomputed(c, x.first_draw, x.B, mhat + off[k]);
            size_t extra = 0;
            if (s == FRR_OK && x.Y != nullptr) {
                if (!x.tau || x.T < 1 || !x.p_out || !(x.alpha >= 0.0 && x.alpha <= 1.0)) s = FRR_E_ARG;
                for (int64_t i = 0; i < x.n && s == FRR_OK; ++i)
                    if (!isfinite(x.Y[i])) s = FRR_E_ARG;
                for (int64_t g = 0; g < x.T && s == FRR_OK; ++g)
                    if (!isfinite(x.tau[g])) s = FRR_E_ARG;
                P.test = s == FRR_OK && c->st.K <= x.cap;  // else FRR_E_CAPACITY from the selection
                if (P.test) extra = (size_t)x.T * 16 + 16;
            }
            if (s == FRR_OK) s = stream_end_enqueue(c, x.keys_out, x.M64_out, x.cap, extra);
            if (s == FRR_OK && P.test) {
                const double* dp = nullptr;
                const long long* dc = nullptr;
                const double* dci = nullptr;
                s = randtest_enqueue(c, x.seed, stream_end_keys_dev(c, x.keys_out), true, c->st.K, 0, x.Y, x.tau,
                                     x.T, x.alpha, &dp, &dc, &dci);
                if (s == FRR_OK) {
                    P.off = stream_end_pinned_used(c);
                    char* hp = static_cast<char*>(c->host_pinned) + P.off;
                    P.p_dev = is_device_ptr(x.p_out);
                    P.c_dev = x.count_out != nullptr && is_device_ptr(x.count_out);
                    const size_t tb = (size_t)x.T * 8;
                    if (cudaMemcpyAsync(P.p_dev ? (void*)x.p_out : (void*)hp, dp, tb,
                                        P.p_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                        (x.count_out && cudaMemcpyAsync(P.c_dev ? (void*)x.count_out : (void*)(hp + tb), dc, tb,
                                                        P.c_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                                        c->stream) != cudaSuccess) ||
                        cudaMemcpyAsync(hp + 2 * tb, dci, 16, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
                        cudaGetLastError();
                        s = FRR_E_CUDA;
                    }
                }
            }
            st_sel[k] = s;
        }
        if (bal_err != nullptr && rc == FRR_OK) {
            int herr = 0;
            if (cudaMemcpyAsync(&herr, bal_err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                cudaGetLastError();
                rc = FRR_E_CUDA;
            } else if (herr != 0) {
                rc = FRR_E_TIMEOUT;  // the selection issued on its output is discarded
            }
        }
        for (size_t k = 0; k < live.size(); ++k) {
            if (rc != FRR_OK) { st_sel[k] = rc; continue; }
            if (!pend[k].piped) {
                st_sel[k] = one_by_one(k, true);
                if (st_sel[k] == FRR_E_CAPACITY && ctx[live[k]]->st.overflowed) st_sel[k] = one_by_one(k, false);
                continue;
            }
            if (st_sel[k] != FRR_OK) continue;
            const int64_t e = live[k];
            frr_experiment& x = ex[e];
            frr_ctx* c = ctx[e];
            int64_t K = 0;
            frr_status s = stream_end_finish(c, x.keys_out, x.M64_out, x.cap, &K);  // synchronises the stream
            x.K_out = K;
            if (s == FRR_E_CAPACITY && c->st.overflowed) {
                // the retained set outgrew its deferred buffer: this experiment again, undeferred
                st_sel[k] = one_by_one(k, false);
                continue;
            }
            if (s == FRR_OK && pend[k].test) {
                const char* hp = static_cast<const char*>(c->host_pinned) + pend[k].off;
                const size_t tb = (size_t)x.T * 8;
                if (!pend[k].p_dev) memcpy(x.p_out, hp, tb);
                if (x.count_out && !pend[k].c_dev) memcpy(x.count_out, hp + tb, tb);
                double ci[2];
                memcpy(ci, hp + 2 * tb, sizeof(ci));
                x.ci_lo = ci[0];
                x.ci_hi = ci[1];
            }
            st_sel[k] = s;
        }
        if (cudaStreamSynchronize(stream) != cudaSuccess) cudaGetLastError();
        if (cudaEventElapsedTime(&ms_balance, ea, eb) != cudaSuccess) { cudaGetLastError(); ms_balance = 0.f; }
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        if (bal_exec) cudaGraphExecDestroy(bal_exec);
        if (bal_graph) cudaGraphDestroy(bal_graph);
        for (cudaEvent_t ev : bal_gev)
            if (ev) cudaEventDestroy(ev);
        for (cudaStream_t st : bal_gs)
            if (st) cudaStreamDestroy(st);
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
    for (frr_ctx* c : ctx) frr_destroy(c);  // (each synchronises its stream first)
    if (lend_block) cudaFreeAsync(lend_block, stream);
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
        stats->ms_select = std::max(0.0, std::chrono::duration<double, std::milli>(t2 - t1).count() - ms_balance);
    }
    return first_err;
}
