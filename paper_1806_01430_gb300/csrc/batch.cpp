// Batched gene evaluation over a suite of programs.
//
// The GA scores a gene by the processing time of the program it places (Sec. 3.3,
// Sec. 5.1.2).  For a suite of many programs of uneven sizes (e.g. 64 six-loop
// programs with n from 128 to 2048), launching every small program's kernels one by
// one leaves the GPU idle between tiny launches.  A batch runs a gene over the whole
// suite phase by phase instead: for loop i, every program's loop i runs at once -- on
// the GPU when gene bit i is 1, on the host when it is 0 -- so each GPU phase is a
// single CUDA graph launch.  The graphs are captured when the batch (or a replica of its
// suite) is made: each phase forks the programs' kernels over several side streams
// (small kernels of different programs run concurrently); the INIT loop of all programs
// is one grouped launch; for the GEMM loop of a tensor-core precision the phase graph
// holds the operand splits and every program's GEMM then runs in one grouped persistent
// tcgen05 launch over all of the programs' tiles.  With fused chains, a gene that puts
// the GEMM -> scale-add -> transpose [-> row sums] [-> norm] chain on the GPU runs it in
// the grouped launch's epilogue (the problems carry the chain; one finalize graph per
// chain shape reduces the norms and row sums).
//
// Generations.  With replicas (batch_set_replicas), the batch holds R copies of the
// suite, and up to R genes of a generation run together: the copies' phases go one
// after another on one stream, and the GEMMs of every gene that offloads the GEMM loop
// -- all genes x all programs -- go into ONE grouped launch.  A gene's time is then
// attributed (it shares the launch with other genes): the device time of its own phase
// graphs and copies (CUDA events around them), the span of its own problems inside the
// grouped launch (global-timer stamps the kernel writes), and the host time of its CPU
// loops.  Without replicas a gene's time is the wall time of the whole suite under it.
// A gene measured before is served from the batch's cache (Sec. 4).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "ga_engine.h"
#include "gao_internal.h"
#include "gemm_tc.h"
#include "prog_internal.h"

using namespace gao;

namespace {
constexpr int kSide = 8;
constexpr int kEv = 6;  // events per replica and loop: copies 0-1, phase graph 2-3, chain finalize 4-5
}  // namespace

struct gao_batch {
    // The GEMM phase with one chain shape in the grouped launch's epilogue.
    struct ChainVar {
        bool ok = false;                // every program of the suite has this chain
        Chain ch;
        std::vector<TcProblem> probs;   // problem table (gemm order) with the chain's epilogue
        cudaGraph_t g = nullptr;        // finalize: each program's norm and row sums
        cudaGraphExec_t fin = nullptr;
        int kernels = 0;
    };
    // One copy of the suite and everything captured for it.
    struct Replica {
        std::vector<gao_prog*> progs;
        std::vector<cudaGraph_t> graph;       // per loop (the grouped GEMM loop: its operand splits)
        std::vector<cudaGraphExec_t> exec;
        std::vector<int> kernels;             // kernels in each phase graph
        std::vector<TcProblem> probs;         // grouped GEMM problems (plain epilogue), gemm order
        std::unordered_map<int, ChainVar> chains;
        InitEntry* d_init = nullptr;          // grouped INIT table of this copy
    };
    std::vector<Replica> reps;      // reps[0]: the caller's programs
    std::vector<gao_prog*> owned;   // programs of reps[1..], made (and destroyed) by the batch
    int n_progs = 0, n_loops = 0;
    int n_genes = 0;  // offloadable loops (gene length)
    int prec = 0;
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, g0 = nullptr, g1 = nullptr, tab_ev = nullptr;
    std::vector<cudaEvent_t> ev;    // [replica][loop][kEv], then [replica][2] for the final copies
    int gemm_loop = -1;
    bool grouped_gemm = false;
    bool chunked = false;           // some program restarts its accumulators every K chunk
    int init_loop = -1;             // INIT loop run as one grouped launch over all programs
    int n_init = 0;
    int64_t init_total4 = 0;
    std::vector<size_t> gemm_order;  // programs in problem-table order (largest GEMM first)
    int tiles_per_suite = 0;
    double flops_per_suite = 0.0;
    TcProblem* d_probs = nullptr;    // the grouped launch's table (capacity table_cap)
    TcProblem* h_table = nullptr;    // pinned staging of it
    unsigned long long* d_span = nullptr;  // span starts [table_cap], then ends [table_cap]
    unsigned long long* h_span = nullptr;  // pinned copy after a launch
    int table_cap = 0;
    int* d_err = nullptr;
    int* h_err = nullptr;
    std::unordered_map<uint64_t, double> cache;
    gao_batch_stat stat{};
    double timeout_s = 0.0;
    bool fuse = false;
};

namespace {

using Replica = gao_batch::Replica;
using ChainVar = gao_batch::ChainVar;

void free_replica_graphs(Replica& R) {
    for (auto& kv : R.chains) {
        if (kv.second.fin) cudaGraphExecDestroy(kv.second.fin);
        if (kv.second.g) cudaGraphDestroy(kv.second.g);
    }
    R.chains.clear();
    for (auto e : R.exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto g : R.graph)
        if (g) cudaGraphDestroy(g);
    R.exec.clear();
    R.graph.clear();
    if (R.d_init) cudaFree(R.d_init);
    R.d_init = nullptr;
}

void free_tables(gao_batch* b) {
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->d_span) cudaFree(b->d_span);
    if (b->h_span) cudaFreeHost(b->h_span);
    b->d_probs = nullptr;
    b->h_table = nullptr;
    b->d_span = nullptr;
    b->h_span = nullptr;
    b->table_cap = 0;
    for (auto e : b->ev)
        if (e) cudaEventDestroy(e);
    b->ev.clear();
}

void free_batch(gao_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    for (auto& R : b->reps) free_replica_graphs(R);
    for (auto* p : b->owned) prog_destroy(p);
    free_tables(b);
    for (auto e : b->join)
        if (e) cudaEventDestroy(e);
    for (auto s : b->side)
        if (s) cudaStreamDestroy(s);
    for (auto e : {b->fork, b->g0, b->g1, b->tab_ev})
        if (e) cudaEventDestroy(e);
    if (b->d_err) cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

cudaError_t fork_side(gao_batch* b) {
    cudaError_t e = cudaEventRecord(b->fork, b->st);
    for (int k = 0; k < kSide && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[(size_t)k], b->fork, 0);
    return e;
}

cudaError_t join_side(gao_batch* b) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kSide && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[(size_t)k], b->side[(size_t)k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->join[(size_t)k], 0);
    }
    return e;
}

void gemm_shape(const gao_prog* p, int gl, int64_t* m, int64_t* nn, int64_t* k) {
    const gao_loop& L = p->loops[(size_t)gl];
    *m = p->bufs[(size_t)L.ins[0]].d.rows;
    *k = p->bufs[(size_t)L.ins[0]].d.cols;
    *nn = p->bufs[(size_t)L.ins[1]].d.cols;
}

// Capture the GPU work of loop li for every program of replica R into one graph.  For the
// grouped GEMM loop the graph holds the operand splits only, and R.probs describes the
// problems for the grouped launch made at run time.
gao_status capture_phase(gao_batch* b, Replica& R, int li) {
    cudaStream_t st = b->st;
    GAO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gao_status status = GAO_OK;
    cudaError_t e = fork_side(b);
    const bool tc_gemm = li == b->gemm_loop && b->grouped_gemm;
    const bool group_init = li == b->init_loop;  // one launch after the (empty) branches
    std::vector<size_t> order(R.progs.size());
    std::iota(order.begin(), order.end(), 0);
    int kernels = 0;
    if (tc_gemm) {
        order = b->gemm_order;
        R.probs.assign(R.progs.size(), TcProblem{});
    }
    for (size_t j = 0; j < order.size() && e == cudaSuccess && status == GAO_OK && !group_init; ++j) {
        gao_prog* p = R.progs[order[j]];
        cudaStream_t s = b->side[j % kSide];
        if (tc_gemm) {
            const gao_loop& L = p->loops[(size_t)li];
            int64_t M, N, K;
            gemm_shape(p, li, &M, &N, &K);
            float* c0 = L.ins[2] >= 0 ? (float*)p->bufs[(size_t)L.ins[2]].dev : (float*)p->bufs[(size_t)L.outs[0]].dev;
            std::string why;
            int nl = 0;
            e = tc_prepare(b->prec, (float*)p->bufs[(size_t)L.outs[0]].dev, (const float*)p->bufs[(size_t)L.ins[0]].dev,
                           (const float*)p->bufs[(size_t)L.ins[1]].dev, c0, M, N, K, (float)L.alpha,
                           L.ins[2] >= 0 ? (float)L.beta : 0.0f, p->opts.kchunk, p->opts.tile_cfg,
                           p->arena + p->lay.tc_off, p->lay.tc_bytes, s, &R.probs[j], &nl, &why);
            if (e != cudaSuccess && !why.empty()) status = fail(GAO_EINVAL, "batch GEMM: " + why);
            kernels += nl;
        } else {
            RunCtx rc{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, s, false};
            const int before = p->stats[(size_t)li].launches;
            status = run_gpu_loop(rc, li);
            kernels += p->stats[(size_t)li].launches - before;
            p->stats[(size_t)li].launches = before;
        }
    }
    if (e == cudaSuccess) e = join_side(b);
    if (group_init && e == cudaSuccess) {
        e = launch_init_group(R.d_init, b->n_init, b->init_total4, st);
        kernels += 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (status != GAO_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (status != GAO_OK) return status;
        return cuda_fail(e != cudaSuccess ? e : e2, "batch capture");
    }
    R.graph[(size_t)li] = g;
    R.kernels[(size_t)li] = kernels;
    GAO_CUDA_TRY(cudaGraphInstantiate(&R.exec[(size_t)li], g, 0));
    return GAO_OK;
}

int chain_key(const Chain& ch) { return (ch.rowsum + 1) * 1024 + (ch.frob + 1); }

// The chain variant `ch` of replica R's GEMM phase: its problems with the chain in the
// epilogue (the splits are shared with the plain problems) and the finalize graph.
gao_status make_chain(gao_batch* b, Replica& R, uint64_t mask, const Chain& ch, ChainVar* cv) {
    const size_t n = R.progs.size();
    cv->ch = ch;
    cv->ok = true;
    for (auto* p : R.progs) {  // the same chain in every program, or no fusion for this shape
        Chain c;
        if (!find_chain(p, b->gemm_loop, mask, true, &c) || c.axpy != ch.axpy || c.transpose != ch.transpose ||
            c.rowsum != ch.rowsum || c.frob != ch.frob)
            cv->ok = false;
    }
    if (!cv->ok) return GAO_OK;
    auto dev = [](gao_prog* p, int bi) { return (float*)p->bufs[(size_t)bi].dev; };
    cv->probs = R.probs;
    std::vector<TcFuse> fz(n);
    for (size_t j = 0; j < n; ++j) {
        gao_prog* p = R.progs[b->gemm_order[j]];
        const gao_loop &X = p->loops[(size_t)ch.axpy], &T = p->loops[(size_t)ch.transpose];
        fz[j] = TcFuse{dev(p, X.ins[1]), dev(p, X.outs[0]), dev(p, T.outs[0]),
                       ch.frob >= 0 ? (double*)p->bufs[(size_t)p->loops[(size_t)ch.frob].outs[0]].dev : nullptr,
                       (float)X.alpha, 0, ch.rowsum >= 0 ? dev(p, p->loops[(size_t)ch.rowsum].outs[0]) : nullptr};
        int64_t M, N, K;
        gemm_shape(p, b->gemm_loop, &M, &N, &K);
        tc_attach_chain(b->prec, M, N, K, p->arena + p->lay.tc_off, fz[j], &cv->probs[j]);
    }
    GAO_CUDA_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = fork_side(b);
    for (size_t j = 0; j < n && e == cudaSuccess; ++j) {
        gao_prog* p = R.progs[b->gemm_order[j]];
        int64_t M, N, K;
        gemm_shape(p, b->gemm_loop, &M, &N, &K);
        int nl = 0;
        e = tc_finalize_chain(b->prec, M, N, K, p->arena + p->lay.tc_off, fz[j], b->side[j % kSide], &nl);
        cv->kernels += nl;
    }
    if (e == cudaSuccess) e = join_side(b);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cv->ok = false;
        return cuda_fail(e != cudaSuccess ? e : e2, "batch chain capture");
    }
    cv->g = g;
    cudaError_t e3 = cudaGraphInstantiate(&cv->fin, g, 0);
    if (e3 != cudaSuccess) {
        cv->ok = false;
        return cuda_fail(e3, "cudaGraphInstantiate(chain)");
    }
    return GAO_OK;
}

// Every chain shape a gene can give (the GEMM, scale-add and transpose on the GPU; each
// later reduction of E on the GPU or not), made up front so that no gene's time holds a
// capture.
gao_status make_chains(gao_batch* b, Replica& R) {
    if (!b->fuse) return GAO_OK;
    const gao_prog* p0 = R.progs[0];
    const uint64_t all = loop_mask_of(p0, all_genes(b->n_genes));
    Chain full;
    if (!find_chain(p0, b->gemm_loop, all, true, &full)) return GAO_OK;
    std::vector<int> opt;
    for (int j : {full.rowsum, full.frob})
        if (j >= 0) opt.push_back(j);
    for (int sub = 0; sub < (1 << opt.size()); ++sub) {
        uint64_t m = all;
        for (size_t k = 0; k < opt.size(); ++k)
            if (!((sub >> k) & 1)) m &= ~(1ULL << opt[k]);
        Chain c;
        if (!find_chain(p0, b->gemm_loop, m, true, &c) || R.chains.count(chain_key(c))) continue;
        ChainVar& cv = R.chains[chain_key(c)];
        gao_status s = make_chain(b, R, m, c, &cv);
        if (s != GAO_OK) return s;
    }
    return GAO_OK;
}

// INIT table of a replica: every program's INIT outputs (no row scaling).
gao_status make_init_table(gao_batch* b, Replica& R) {
    if (b->init_loop < 0) return GAO_OK;
    std::vector<InitEntry> tab;
    int64_t start = 0;
    for (auto* p : R.progs) {
        const gao_loop& L = p->loops[(size_t)b->init_loop];
        for (int t = 0; t < GAO_MAX_IO; ++t) {
            const int bi = L.outs[t];
            if (bi < 0) continue;
            const gao_buffer& d = p->bufs[(size_t)bi].d;
            const int64_t n4 = (d.rows * d.cols + 3) / 4;
            if (n4 <= 0) continue;
            tab.push_back(InitEntry{(float*)p->bufs[(size_t)bi].dev, d.rows, d.cols, p->opts.seed, (uint32_t)bi, start});
            start += n4;
        }
    }
    if ((int)tab.size() != b->n_init || start != b->init_total4) return fail(GAO_EINVAL, "batch INIT tables differ");
    GAO_CUDA_TRY(cudaMalloc((void**)&R.d_init, sizeof(InitEntry) * tab.size()));
    GAO_CUDA_TRY(cudaMemcpy(R.d_init, tab.data(), sizeof(InitEntry) * tab.size(), cudaMemcpyHostToDevice));
    return GAO_OK;
}

// Capture everything of a replica (its programs already in R.progs).
gao_status make_replica(gao_batch* b, Replica& R) {
    R.graph.assign((size_t)b->n_loops, nullptr);
    R.exec.assign((size_t)b->n_loops, nullptr);
    R.kernels.assign((size_t)b->n_loops, 0);
    for (auto* p : R.progs) GAO_CUDA_TRY(cudaStreamSynchronize(p->st));
    gao_status s = make_init_table(b, R);
    if (s != GAO_OK) return s;
    const gao_prog* p0 = R.progs[0];
    for (int li = 0; li < b->n_loops; ++li) {
        if (p0->verdict[(size_t)li] != GAO_OFFLOAD_OK) continue;  // host-only loop: no graph
        if ((s = capture_phase(b, R, li)) != GAO_OK) return s;
    }
    if (b->grouped_gemm) {
        int tiles = 0;
        for (auto& pr : R.probs) tiles += pr.tiles_m * pr.tiles_n;
        if (tiles != b->tiles_per_suite) return fail(GAO_EINVAL, "batch tile count mismatch");
    }
    return make_chains(b, R);
}

// Room for the grouped launch's table and spans, and the timing events, for `reps` replicas.
gao_status size_tables(gao_batch* b, int reps) {
    free_tables(b);
    const int cap = std::max(1, reps * b->n_progs);
    GAO_CUDA_TRY(cudaMalloc((void**)&b->d_probs, sizeof(TcProblem) * (size_t)cap));
    GAO_CUDA_TRY(cudaMallocHost((void**)&b->h_table, sizeof(TcProblem) * (size_t)cap));
    GAO_CUDA_TRY(cudaMalloc((void**)&b->d_span, sizeof(unsigned long long) * 2 * (size_t)cap));
    GAO_CUDA_TRY(cudaMallocHost((void**)&b->h_span, sizeof(unsigned long long) * 2 * (size_t)cap));
    b->table_cap = cap;
    b->ev.assign((size_t)reps * ((size_t)b->n_loops * kEv + 2), nullptr);
    for (auto& e : b->ev) GAO_CUDA_TRY(cudaEventCreate(&e));
    return GAO_OK;
}

// One grouped launch over the GEMM problems of the replicas in `parts` (their plain
// problems, or a chain variant's where cv[r] is set), in that order; with `spans` every
// problem's time span is recorded and copied to h_span (stream order).
gao_status grouped_launch(gao_batch* b, const std::vector<int>& parts, const std::vector<ChainVar*>& cv, bool spans) {
    GAO_CUDA_TRY(cudaEventSynchronize(b->tab_ev));  // the previous table copy has read h_table
    int k = 0, start = 0;
    for (int r : parts) {
        const std::vector<TcProblem>& src = cv[(size_t)r] ? cv[(size_t)r]->probs : b->reps[(size_t)r].probs;
        for (const TcProblem& pr : src) {
            if (k >= b->table_cap) return fail(GAO_EINVAL, "batch problem table overflow");
            TcProblem t = pr;
            t.tile_start = start;
            start += t.tiles_m * t.tiles_n;
            t.span_start = spans ? b->d_span + k : nullptr;
            t.span_end = spans ? b->d_span + b->table_cap + k : nullptr;
            b->h_table[k++] = t;
        }
    }
    GAO_CUDA_TRY(cudaMemcpyAsync(b->d_probs, b->h_table, sizeof(TcProblem) * (size_t)k, cudaMemcpyHostToDevice, b->st));
    GAO_CUDA_TRY(cudaEventRecord(b->tab_ev, b->st));
    if (spans) {
        GAO_CUDA_TRY(cudaMemsetAsync(b->d_span, 0xFF, sizeof(unsigned long long) * (size_t)k, b->st));
        GAO_CUDA_TRY(cudaMemsetAsync(b->d_span + b->table_cap, 0, sizeof(unsigned long long) * (size_t)k, b->st));
    }
    GAO_CUDA_TRY(cudaEventRecord(b->g0, b->st));
    GAO_CUDA_TRY(tc_launch_grouped(b->prec, b->chunked, b->d_probs, k, start, b->d_err, b->st));
    GAO_CUDA_TRY(cudaEventRecord(b->g1, b->st));
    if (spans) {
        GAO_CUDA_TRY(cudaMemcpyAsync(b->h_span, b->d_span, sizeof(unsigned long long) * (size_t)k,
                                     cudaMemcpyDeviceToHost, b->st));
        GAO_CUDA_TRY(cudaMemcpyAsync(b->h_span + b->table_cap, b->d_span + b->table_cap,
                                     sizeof(unsigned long long) * (size_t)k, cudaMemcpyDeviceToHost, b->st));
    }
    b->stat.kernel_launches += 1;
    b->stat.grouped_launches += 1;
    b->stat.grouped_genes += (int64_t)parts.size();
    b->stat.gemm_tiles = start;
    b->stat.gemm_flops = b->flops_per_suite * (double)parts.size();
    return GAO_OK;
}

double ev_ms(cudaEvent_t a, cudaEvent_t c) {
    float ms = 0.0f;
    return cudaEventElapsedTime(&ms, a, c) == cudaSuccess ? (double)ms : 0.0;
}

// Genes genes[0..u) over replicas 0..u-1, loop by loop.  attributed = false (u == 1): the
// gene's time is the wall time of the whole suite.  attributed = true: each gene's time is
// its own device phases and copies (events), its problems' span in the shared grouped GEMM
// launch, and its host loops.  A gene over the budget is cut off at it.  seconds[r] = -1
// marks a gene that failed.
gao_status run_genes(gao_batch* b, const uint64_t* genes, int u, double* seconds, bool attributed) {
    const int L = b->n_loops;
    if (u < 1 || u > (int)b->reps.size()) return fail(GAO_EINVAL, "more genes than replicas");
    std::vector<uint64_t> mask((size_t)u);
    for (int r = 0; r < u; ++r) {
        if (b->n_genes < 64 && (genes[r] >> b->n_genes) != 0)
            return fail(GAO_EINVAL, "gene has bits above the gene length");
        mask[(size_t)r] = loop_mask_of(b->reps[0].progs[0], genes[r]);  // bit li: loop li on the GPU
    }
    const double budget = b->timeout_s;
    const double t0 = now_s();
    std::vector<std::vector<RunCtx>> rc((size_t)u);
    for (int r = 0; r < u; ++r)
        for (auto* p : b->reps[(size_t)r].progs) {
            for (auto& B : p->bufs) {
                B.vh = (B.d.role == GAO_BUF_INPUT);
                B.vd = false;
            }
            rc[(size_t)r].push_back(RunCtx{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, b->st, false});
        }
    // the chain in the grouped launch's epilogue for genes that put all of it on the GPU
    std::vector<ChainVar*> cv((size_t)u, nullptr);
    for (int r = 0; r < u; ++r) {
        Chain ch;
        if (b->fuse && ((mask[(size_t)r] >> b->gemm_loop) & 1) &&
            find_chain(b->reps[(size_t)r].progs[0], b->gemm_loop, mask[(size_t)r], true, &ch)) {
            auto it = b->reps[(size_t)r].chains.find(chain_key(ch));
            if (it != b->reps[(size_t)r].chains.end() && it->second.ok) cv[(size_t)r] = &it->second;
        }
    }
    std::vector<uint64_t> in_epi((size_t)u, 0);  // loops a replica ran in the GEMM's epilogue
    std::vector<char> dead((size_t)u, 0);         // cut off at the budget
    std::vector<double> cpu_ms((size_t)u, 0.0);
    std::vector<uint8_t> used((size_t)u * L, 0);  // events recorded: bit 0 copies, 1 phase, 2 finalize
    std::vector<char> out_used((size_t)u, 0);
    std::vector<int> parts;
    std::vector<int> part_index((size_t)u, -1);  // position of a replica's problems in the launch
    bool spans_ready = false;                     // h_span holds this run's grouped launch's stamps
    bool launched = false;                        // this run made a grouped launch
    auto evp = [&](int r, int li, int k) { return b->ev[((size_t)r * L + li) * kEv + k]; };
    auto eout = [&](int r, int k) { return b->ev[b->reps.size() * (size_t)L * kEv + (size_t)r * 2 + k]; };
    auto rec = [&](cudaEvent_t e) { return attributed ? cudaEventRecord(e, b->st) : cudaSuccess; };
    // attributed milliseconds of replica r so far (every event it recorded has completed)
    auto attributed_ms = [&](int r) {
        double t = cpu_ms[(size_t)r];
        for (int li = 0; li < L; ++li) {
            const uint8_t m = used[(size_t)r * L + li];
            if (m & 1) t += ev_ms(evp(r, li, 0), evp(r, li, 1));
            if (m & 2) t += ev_ms(evp(r, li, 2), evp(r, li, 3));
            if (m & 4) t += ev_ms(evp(r, li, 4), evp(r, li, 5));
        }
        if (spans_ready && part_index[(size_t)r] >= 0) {
            unsigned long long lo = ~0ULL, hi = 0;
            const int k0 = part_index[(size_t)r] * b->n_progs;
            for (int k = k0; k < k0 + b->n_progs; ++k) {
                lo = std::min(lo, b->h_span[k]);
                hi = std::max(hi, b->h_span[b->table_cap + k]);
            }
            if (hi > lo) t += (double)(hi - lo) * 1e-6;
        }
        if (out_used[(size_t)r]) t += ev_ms(eout(r, 0), eout(r, 1));
        return t;
    };
    GAO_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st));
    gao_loop_stat scratch{};
    for (int li = 0; li < L; ++li) {
        const bool gemm_phase = li == b->gemm_loop && b->grouped_gemm;
        parts.clear();
        bool any_cpu = false;
        for (int r = 0; r < u; ++r) {
            if (dead[(size_t)r] || ((in_epi[(size_t)r] >> li) & 1)) continue;
            const bool gpu = (mask[(size_t)r] >> li) & 1;
            any_cpu |= !gpu;
            GAO_CUDA_TRY(rec(evp(r, li, 0)));
            for (auto& c : rc[(size_t)r])
                for (int bi : loop_inputs(c.p->loops[(size_t)li])) {
                    gao_status s = make_valid(c, bi, gpu, scratch);
                    if (s != GAO_OK) return s;
                }
            if (gpu && gemm_phase && cv[(size_t)r])
                for (auto& c : rc[(size_t)r]) {  // the AXPY's second operand is read in the epilogue
                    gao_status s = make_valid(c, c.p->loops[(size_t)cv[(size_t)r]->ch.axpy].ins[1], true, scratch);
                    if (s != GAO_OK) return s;
                }
            GAO_CUDA_TRY(rec(evp(r, li, 1)));
            if (attributed) used[(size_t)r * L + li] |= 1;
            if (gpu) {
                GAO_CUDA_TRY(rec(evp(r, li, 2)));
                GAO_CUDA_TRY(cudaGraphLaunch(b->reps[(size_t)r].exec[(size_t)li], b->st));
                GAO_CUDA_TRY(rec(evp(r, li, 3)));
                if (attributed) used[(size_t)r * L + li] |= 2;
                b->stat.kernel_launches += b->reps[(size_t)r].kernels[(size_t)li];
                if (gemm_phase) parts.push_back(r);
            }
        }
        if (!parts.empty()) {
            // every offloaded GEMM of these genes' suites in one grouped launch
            for (size_t k = 0; k < parts.size(); ++k) part_index[(size_t)parts[k]] = (int)k;
            gao_status s = grouped_launch(b, parts, cv, attributed);
            if (s != GAO_OK) return s;
            launched = true;
            for (int r : parts) {
                ChainVar* c = cv[(size_t)r];
                if (!c) continue;
                GAO_CUDA_TRY(rec(evp(r, li, 4)));
                GAO_CUDA_TRY(cudaGraphLaunch(c->fin, b->st));
                GAO_CUDA_TRY(rec(evp(r, li, 5)));
                if (attributed) used[(size_t)r * L + li] |= 4;
                b->stat.kernel_launches += c->kernels;
                b->stat.fused_phases += 1;
                for (int j : {li, c->ch.axpy, c->ch.transpose, c->ch.rowsum, c->ch.frob}) {
                    if (j < 0) continue;
                    in_epi[(size_t)r] |= 1ULL << j;
                    for (auto& x : rc[(size_t)r])
                        for (int bo : loop_outputs(x.p->loops[(size_t)j])) {
                            x.p->bufs[(size_t)bo].vh = false;
                            x.p->bufs[(size_t)bo].vd = true;
                        }
                }
            }
        }
        if (any_cpu) {
            // host loops read mirrors that queued copies fill: drain the stream first
            bool to = false;
            gao_status s = stream_wait(b->st, 0.0, &to);
            if (s != GAO_OK) return s;
            if (attributed && launched) spans_ready = true;
            for (int r = 0; r < u; ++r) {
                if (dead[(size_t)r] || ((in_epi[(size_t)r] >> li) & 1) || ((mask[(size_t)r] >> li) & 1)) continue;
                double deadline = 0.0;
                if (budget > 0.0) {
                    const double so_far = attributed ? attributed_ms(r) * 1e-3 : now_s() - t0;
                    if (so_far >= budget) {
                        dead[(size_t)r] = 1;
                        continue;
                    }
                    deadline = now_s() + (budget - so_far);
                }
                const double c0 = now_s();
                for (auto& c : rc[(size_t)r]) {
                    c.cpu.deadline = deadline;
                    c.cpu.timed_out = false;
                    if ((s = run_cpu_loop(c, li)) != GAO_OK) return s;
                    if (c.cpu.timed_out) {
                        dead[(size_t)r] = 1;
                        break;
                    }
                }
                cpu_ms[(size_t)r] += (now_s() - c0) * 1e3;
            }
        }
        for (int r = 0; r < u; ++r) {  // residency after loop li (chain loops were set above)
            if (dead[(size_t)r] || ((in_epi[(size_t)r] >> li) & 1)) continue;
            const bool gpu = (mask[(size_t)r] >> li) & 1;
            for (auto& c : rc[(size_t)r])
                for (int bo : loop_outputs(c.p->loops[(size_t)li])) {
                    c.p->bufs[(size_t)bo].vh = !gpu;
                    c.p->bufs[(size_t)bo].vd = gpu;
                }
        }
        if (!attributed && budget > 0.0 && now_s() - t0 > budget) dead[0] = 1;
    }
    for (int r = 0; r < u; ++r) {
        if (dead[(size_t)r]) continue;
        GAO_CUDA_TRY(rec(eout(r, 0)));
        for (auto& c : rc[(size_t)r])
            for (size_t bi = 0; bi < c.p->bufs.size(); ++bi)
                if (c.p->bufs[bi].d.role == GAO_BUF_OUTPUT && !c.p->bufs[bi].vh) {
                    gao_status s = make_valid(c, (int)bi, false, scratch);
                    if (s != GAO_OK) return s;
                }
        GAO_CUDA_TRY(rec(eout(r, 1)));
        if (attributed) out_used[(size_t)r] = 1;
    }
    GAO_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    bool to = false;
    gao_status s = stream_wait(b->st, 0.0, &to);
    if (s != GAO_OK) return s;
    const double t1 = now_s();
    spans_ready = attributed && launched;
    if (*b->h_err != 0) {
        for (int r = 0; r < u; ++r) seconds[r] = -1.0;
        return fail(GAO_EDEVICE, "a batch kernel raised device error " + std::to_string(*b->h_err));
    }
    if (launched) b->stat.gemm_phase_ms = ev_ms(b->g0, b->g1);
    for (int r = 0; r < u; ++r) {
        if (dead[(size_t)r]) {
            seconds[r] = budget;
        } else if (!attributed) {
            seconds[r] = t1 - t0;
        } else {
            const double t = attributed_ms(r) * 1e-3;
            seconds[r] = budget > 0.0 ? std::min(t, budget) : t;
        }
    }
    return GAO_OK;
}

// Times of distinct genes not in the cache: up to `replicas` of them per run; failures
// score -1 (fitness 0).
gao_status measure(gao_batch* b, const std::vector<uint64_t>& genes, std::vector<double>* secs) {
    secs->assign(genes.size(), -1.0);
    const int R = (int)b->reps.size();
    const bool attributed = R > 1;
    for (size_t i = 0; i < genes.size(); i += (size_t)R) {
        const int u = (int)std::min<size_t>((size_t)R, genes.size() - i);
        const double w0 = now_s();
        gao_status st = run_genes(b, genes.data() + i, u, secs->data() + i, attributed);
        b->stat.exec_seconds += now_s() - w0;
        if (st == GAO_EDEVICE || st == GAO_ECPU) {
            for (int r = 0; r < u; ++r) (*secs)[i + (size_t)r] = -1.0;
        } else if (st != GAO_OK) {
            return st;
        }
        for (int r = 0; r < u; ++r) b->cache.emplace(genes[i + (size_t)r], (*secs)[i + (size_t)r]);
        b->stat.executed += u;
    }
    return GAO_OK;
}

// Times of genes (any order, repeats allowed): from the cache, the rest measured together.
gao_status times_of(gao_batch* b, const std::vector<uint64_t>& genes, std::vector<double>* out, int* hits) {
    std::vector<uint64_t> fresh;
    for (uint64_t g : genes)
        if (!b->cache.count(g) && std::find(fresh.begin(), fresh.end(), g) == fresh.end()) fresh.push_back(g);
    std::vector<double> s;
    gao_status st = measure(b, fresh, &s);
    if (st != GAO_OK) return st;
    out->resize(genes.size());
    int h = 0;
    std::vector<uint64_t> left = fresh;
    for (size_t i = 0; i < genes.size(); ++i) {
        (*out)[i] = b->cache.find(genes[i])->second;
        auto pos = std::find(left.begin(), left.end(), genes[i]);
        if (pos != left.end()) left.erase(pos);  // the first individual carrying a fresh gene measured it
        else ++h;
    }
    b->stat.served += h;
    if (hits) *hits = h;
    return GAO_OK;
}

}  // namespace

extern "C" gao_status batch_create(gao_prog* const* progs, int n_progs, gao_batch** out) {
    if (!out) return fail(GAO_EINVAL, "out is null");
    *out = nullptr;
    if (!progs || n_progs < 1) return fail(GAO_EINVAL, "a batch needs at least one program");
    const gao_prog* p0 = progs[0];
    for (int i = 0; i < n_progs; ++i) {
        const gao_prog* p = progs[i];
        if (!p) return fail(GAO_EINVAL, "null program");
        if (p->loops.size() != p0->loops.size()) return fail(GAO_EINVAL, "batch programs differ in loop count");
        for (size_t l = 0; l < p->loops.size(); ++l)
            if (p->loops[l].kind != p0->loops[l].kind || p->verdict[l] != p0->verdict[l])
                return fail(GAO_EINVAL, "batch programs differ in loop kinds or in which loops are offloadable");
        if (p->opts.gemm_prec != p0->opts.gemm_prec) return fail(GAO_EINVAL, "batch programs differ in GEMM precision");
        if (p->opts.transfer_mode != GAO_TRANSFER_RESIDENT)
            return fail(GAO_EINVAL, "batches keep buffers resident (transfer_mode RESIDENT only)");
        if (p->opts.fuse_chains == GAO_FUSE_GENE)
            return fail(GAO_EINVAL, "batch genes are loop placements only (fuse_chains GAO_FUSE_GENE is not supported)");
        if (p->opts.fuse_chains != p0->opts.fuse_chains) return fail(GAO_EINVAL, "batch programs differ in fuse_chains");
        for (auto& B : p->bufs)
            if (B.d.role == GAO_BUF_INPUT && !B.input_set) return fail(GAO_EINVAL, "INPUT buffers must be set first");
        for (int j = 0; j < i; ++j)
            if (progs[j] == p) return fail(GAO_EINVAL, "a program appears twice in the batch");
    }
    gao_status s = check_device(nullptr);
    if (s != GAO_OK) return s;
    gao_batch* b = new gao_batch();
    auto bail = [&](gao_status st) {
        free_batch(b);
        return st;
    };
    b->n_progs = n_progs;
    b->n_loops = (int)p0->loops.size();
    b->n_genes = gene_length(p0);
    b->prec = p0->opts.gemm_prec;
    for (int l = 0; l < b->n_loops; ++l)
        if (p0->loops[(size_t)l].kind == GAO_LOOP_GEMM && p0->verdict[(size_t)l] == GAO_OFFLOAD_OK) {
            if (b->gemm_loop >= 0) return bail(fail(GAO_EINVAL, "a batch supports one GEMM loop per program"));
            b->gemm_loop = l;
        }
    b->grouped_gemm = b->gemm_loop >= 0 && b->prec != GAO_GEMM_FP32_SIMT;
    b->fuse = b->grouped_gemm && p0->opts.fuse_chains == GAO_FUSE_ON && b->prec != GAO_GEMM_FP8;
    for (int i = 0; i < n_progs; ++i) b->chunked |= progs[i]->opts.kchunk > 0;
    cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    b->side.assign(kSide, nullptr);
    b->join.assign(kSide, nullptr);
    for (int k = 0; k < kSide; ++k) {
        if ((e = cudaStreamCreateWithFlags(&b->side[(size_t)k], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->join[(size_t)k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(cuda_fail(e, "side stream"));
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->tab_ev, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreate(&b->g0)) != cudaSuccess || (e = cudaEventCreate(&b->g1)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaMalloc((void**)&b->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&b->h_err, sizeof(int))) != cudaSuccess)
        return bail(cuda_fail(e, "batch error word"));
    *b->h_err = 0;
    if (b->grouped_gemm) {
        std::string why;
        if (!tc_available(&why)) return bail(fail(GAO_ENODEV, why));
        if ((e = tc_launch_grouped(b->prec, b->chunked, nullptr, 0, 0, nullptr, b->st)) != cudaSuccess)
            return bail(cuda_fail(e, "grouped GEMM set-up"));
        int64_t start = 0;
        for (int i = 0; i < n_progs; ++i) {
            int64_t m, nn, k;
            gemm_shape(progs[i], b->gemm_loop, &m, &nn, &k);
            if (m <= 0 || nn <= 0 || k <= 0)
                return bail(fail(GAO_EINVAL, "batch GEMM needs positive sizes on the tensor-core path"));
            b->flops_per_suite += 2.0 * m * nn * k;
            start += ((m + 127) / 128) * ((nn + 127) / 128);
        }
        if (start > 0x7fffffff / 256) return bail(fail(GAO_EINVAL, "batch GEMM has too many tiles"));
        b->tiles_per_suite = (int)start;
        // problem table order: largest GEMM first, so that the launch's tail is made of
        // small tiles
        b->gemm_order.resize((size_t)n_progs);
        std::iota(b->gemm_order.begin(), b->gemm_order.end(), 0);
        std::stable_sort(b->gemm_order.begin(), b->gemm_order.end(), [&](size_t x, size_t y) {
            int64_t mx, nx, kx, my, ny, ky;
            gemm_shape(progs[x], b->gemm_loop, &mx, &nx, &kx);
            gemm_shape(progs[y], b->gemm_loop, &my, &ny, &ky);
            return (double)mx * nx * kx > (double)my * ny * ky;
        });
    }
    // the first INIT loop without row scaling: one grouped launch over every program's
    // outputs instead of a launch per program (many small launches in a row cost more than
    // their writes)
    for (int li = 0; li < b->n_loops && b->init_loop < 0; ++li) {
        const gao_loop& L0 = p0->loops[(size_t)li];
        if (L0.kind != GAO_LOOP_INIT || p0->verdict[(size_t)li] != GAO_OFFLOAD_OK) continue;
        bool plain = true;
        for (int i = 0; i < n_progs; ++i) plain &= (progs[i]->loops[(size_t)li].flags & ((1u << GAO_MAX_IO) - 1)) == 0;
        if (!plain) break;
        int cnt = 0;
        int64_t start = 0;
        for (int i = 0; i < n_progs; ++i) {
            const gao_loop& L = progs[i]->loops[(size_t)li];
            for (int t = 0; t < GAO_MAX_IO; ++t) {
                if (L.outs[t] < 0) continue;
                const gao_buffer& d = progs[i]->bufs[(size_t)L.outs[t]].d;
                const int64_t n4 = (d.rows * d.cols + 3) / 4;
                if (n4 <= 0) continue;
                ++cnt;
                start += n4;
            }
        }
        if (cnt == 0) break;
        b->init_loop = li;
        b->n_init = cnt;
        b->init_total4 = start;
    }
    b->reps.resize(1);
    b->reps[0].progs.assign(progs, progs + n_progs);
    if ((s = size_tables(b, 1)) != GAO_OK) return bail(s);
    if ((s = make_replica(b, b->reps[0])) != GAO_OK) return bail(s);
    // kernels of the all-GPU gene: every offloaded loop's phase, the grouped GEMM launch and,
    // with fusion, the full chain's finalize in place of the chain's phases
    const Replica& R0 = b->reps[0];
    const uint64_t all = loop_mask_of(p0, all_genes(b->n_genes));
    Chain full;
    const bool fused = b->fuse && find_chain(p0, b->gemm_loop, all, true, &full);
    int k = 0;
    for (int li = 0; li < b->n_loops; ++li) {
        if (!((all >> li) & 1)) continue;
        if (fused && (li == full.axpy || li == full.transpose || li == full.rowsum || li == full.frob)) continue;
        k += R0.kernels[(size_t)li];
    }
    if (b->grouped_gemm) k += 1;
    if (fused) {
        auto it = R0.chains.find(chain_key(full));
        if (it != R0.chains.end() && it->second.ok) k += it->second.kernels;
    }
    b->stat.launches_per_gene = k;
    b->stat.graphs = 0;
    for (auto g : R0.exec) b->stat.graphs += g != nullptr;
    b->stat.replicas = 1;
    *out = b;
    return GAO_OK;
}

namespace {
// Drop replicas from index `keep` on (their graphs and the programs the batch made).
void drop_replicas(gao_batch* b, size_t keep) {
    for (size_t r = keep; r < b->reps.size(); ++r) {
        free_replica_graphs(b->reps[r]);
        for (auto* p : b->reps[r].progs) {
            b->owned.erase(std::remove(b->owned.begin(), b->owned.end(), p), b->owned.end());
            prog_destroy(p);
        }
    }
    if (b->reps.size() > keep) b->reps.resize(keep);
}
}  // namespace

extern "C" gao_status batch_set_replicas(gao_batch* b, int replicas) {
    if (!b) return fail(GAO_EINVAL, "batch is null");
    if (replicas < 1 || replicas > 256) return fail(GAO_EINVAL, "replicas must be in [1, 256]");
    GAO_CUDA_TRY(cudaStreamSynchronize(b->st));
    const size_t have = b->reps.size();
    gao_status s = GAO_OK;
    if ((size_t)replicas < have) drop_replicas(b, (size_t)replicas);
    for (size_t r = have; r < (size_t)replicas && s == GAO_OK; ++r) {
        b->reps.emplace_back();
        Replica& R = b->reps.back();
        for (gao_prog* p : b->reps[0].progs) {
            // a copy of the program: same loops, buffers and options, its own memory
            std::vector<gao_buffer> bufs;
            for (auto& B : p->bufs) bufs.push_back(B.d);
            gao_opts o = p->opts;
            o.stream = nullptr;
            o.dev_arena = nullptr;
            o.dev_arena_bytes = 0;
            gao_prog* q = nullptr;
            if ((s = prog_create(p->loops.data(), (int)p->loops.size(), bufs.data(), (int)bufs.size(), &o, &q)) !=
                GAO_OK)
                break;
            b->owned.push_back(q);
            R.progs.push_back(q);
            for (size_t bi = 0; bi < p->bufs.size() && s == GAO_OK; ++bi)
                if (p->bufs[bi].d.role == GAO_BUF_INPUT && p->bufs[bi].input_set)
                    s = prog_set_input(q, (int)bi, p->bufs[bi].host, p->bufs[bi].bytes);
            if (s != GAO_OK) break;
        }
        if (s == GAO_OK) s = make_replica(b, R);
    }
    if (s != GAO_OK) drop_replicas(b, have);  // back to the replicas there were
    const gao_status s2 = size_tables(b, (int)b->reps.size());
    b->stat.replicas = (int32_t)b->reps.size();
    b->cache.clear();  // the time definition changes with generations (attributed vs wall)
    return s != GAO_OK ? s : s2;
}

extern "C" gao_status batch_replica_prog(gao_batch* b, int replica, int index, gao_prog** out) {
    if (!b || !out) return fail(GAO_EINVAL, "null argument");
    if (replica < 0 || replica >= (int)b->reps.size()) return fail(GAO_EINVAL, "no such replica");
    if (index < 0 || index >= b->n_progs) return fail(GAO_EINVAL, "no such program");
    *out = b->reps[(size_t)replica].progs[(size_t)index];
    return GAO_OK;
}

extern "C" gao_status batch_evaluate(gao_batch* b, const uint64_t* population, int pop, double* fitness_out,
                                     double* seconds_out, int* cache_hits_out) {
    if (!b || !population || pop < 0) return fail(GAO_EINVAL, "bad batch or population");
    std::vector<uint64_t> genes(population, population + pop);
    std::vector<double> t;
    int hits = 0;
    gao_status s = times_of(b, genes, &t, &hits);
    if (s != GAO_OK) return s;
    for (int i = 0; i < pop; ++i) {
        if (seconds_out) seconds_out[i] = t[(size_t)i];
        if (fitness_out) fitness_out[i] = ga_fitness(t[(size_t)i]);
    }
    if (cache_hits_out) *cache_hits_out = hits;
    return GAO_OK;
}

extern "C" gao_status batch_ga_run(gao_batch* b, const gao_ga_params* params, gao_ga_result* result) {
    if (!b || !params || !result) return fail(GAO_EINVAL, "null argument");
    if (b->n_genes < 1) return fail(GAO_EINVAL, "no loop of the batch is offloadable (gene length 0)");
    const double saved = b->timeout_s;
    double budget = params->timeout_s;
    if (budget < 0.0) {  // automatic: 10 x the all-GPU time of the suite, capped at 60 s
        std::vector<double> t;
        b->timeout_s = 0.0;
        gao_status s = times_of(b, {all_genes(b->n_genes)}, &t, nullptr);
        if (s != GAO_OK) return s;
        budget = std::min(60.0, 10.0 * t[0]);
    }
    if (budget > 0.0) b->timeout_s = budget;
    // each generation's new genes measured together (up to the replica count per run)
    PopFn fn = [&](const std::vector<uint64_t>& genes, std::vector<double>* secs) {
        return times_of(b, genes, secs, nullptr);
    };
    gao_status s = ga_core_pop(b->n_genes, *params, fn, result);
    b->timeout_s = saved;
    return s;
}

extern "C" gao_status batch_stats(gao_batch* b, gao_batch_stat* out) {
    if (!b || !out) return fail(GAO_EINVAL, "null argument");
    *out = b->stat;
    if (b->stat.grouped_launches == 0) {
        out->gemm_flops = b->flops_per_suite;
        out->gemm_tiles = b->tiles_per_suite;
    }
    return GAO_OK;
}

extern "C" gao_status batch_autotune(gao_batch* b, const gao_ga_params* params, gao_autotune_result* out) {
    if (!b || !params || !out) return fail(GAO_EINVAL, "null argument");
    if (!b->grouped_gemm) return fail(GAO_EINVAL, "batch has no tensor-core GEMM loop");
    const uint64_t all = all_genes(b->n_genes);
    const gao_batch_stat saved_stat = b->stat;  // the tuning's launches are not genes'
    struct Restore {
        gao_batch* b;
        gao_batch_stat s;
        ~Restore() { b->stat = s; }
    } restore{b, saved_stat};
    double s0 = 0.0;
    gao_status st = run_genes(b, &all, 1, &s0, false);  // the GEMM's inputs on the device
    if (st != GAO_OK) return st;
    Replica& R0 = b->reps[0];
    const std::vector<TcProblem> base = R0.probs;
    auto set_cfg = [&](std::vector<TcProblem>& tab, int kchunk, int tile_cfg) {
        for (auto& pr : tab) {
            pr.group = tc_group_of(tile_cfg);
            pr.pf_kb = tc_prefetch_of(tile_cfg);
            if (b->chunked && kchunk > 0) pr.chunk_kb = std::max(1, std::min(pr.num_kb, kchunk / 64));
        }
    };
    const std::vector<ChainVar*> none((size_t)1, nullptr);
    auto time_cfg = [&](int kchunk, int tile_cfg, double* ms) -> gao_status {
        R0.probs = base;
        set_cfg(R0.probs, kchunk, tile_cfg);
        // a configuration whose launch raised the error word fails the tuning (GAO_EDEVICE)
        GAO_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st));
        std::vector<double> v;
        cudaEvent_t e0 = b->ev[0], e1 = b->ev[1];  // around the splits and the grouped launch
        for (int r = 0; r < 4; ++r) {
            GAO_CUDA_TRY(cudaEventRecord(e0, b->st));
            GAO_CUDA_TRY(cudaGraphLaunch(R0.exec[(size_t)b->gemm_loop], b->st));
            gao_status s = grouped_launch(b, {0}, none, false);
            if (s != GAO_OK) return s;
            GAO_CUDA_TRY(cudaEventRecord(e1, b->st));
            GAO_CUDA_TRY(cudaEventSynchronize(e1));
            if (r > 0) v.push_back(ev_ms(e0, e1));
        }
        GAO_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
        GAO_CUDA_TRY(cudaStreamSynchronize(b->st));
        if (*b->h_err != 0)
            return fail(GAO_EDEVICE, "batch autotune: the grouped GEMM raised device error " +
                                         std::to_string(*b->h_err) + " under tile configuration " +
                                         std::to_string(tile_cfg));
        std::sort(v.begin(), v.end());
        *ms = v[v.size() / 2];
        return GAO_OK;
    };
    const int kc0 = R0.progs[0]->opts.kchunk, tc0 = R0.progs[0]->opts.tile_cfg;
    double def_ms = 0.0;
    if ((st = time_cfg(kc0, tc0, &def_ms)) != GAO_OK) {
        R0.probs = base;
        return st;
    }
    int evals = 0;
    TimeFn fn = [&](uint64_t g, double* t) {
        int kc = 0, tc = 0;
        autotune_decode(b->prec, g, &kc, &tc);
        double ms = 0.0;
        gao_status s2 = time_cfg(kc, tc, &ms);
        *t = ms * 1e-3;
        ++evals;
        return s2;
    };
    gao_ga_result res{};
    st = ga_core(kAutotuneBits, *params, fn, &res);
    R0.probs = base;
    if (st != GAO_OK) return st;
    // the configuration in place stays unless the GA found a faster one
    int kc = kc0, tc = tc0;
    double best_ms = def_ms;
    if (res.best_s * 1e3 < def_ms) {
        autotune_decode(b->prec, res.best_mask, &kc, &tc);
        best_ms = res.best_s * 1e3;
    }
    // every replica's problem tables (plain and each chain shape) take the configuration
    for (auto& R : b->reps) {
        set_cfg(R.probs, kc, tc);
        for (auto& kv : R.chains) set_cfg(kv.second.probs, kc, tc);
        for (auto* p : R.progs) {
            if (b->chunked) p->opts.kchunk = kc;
            p->opts.tile_cfg = tc;
            drop_graphs(p);
        }
    }
    b->cache.clear();  // genes measured under the old configuration
    out->kchunk = b->chunked ? kc : 0;
    out->tile_cfg = tc;
    out->best_ms = best_ms;
    out->default_ms = def_ms;
    out->evaluations = evals;
    return GAO_OK;
}

extern "C" void batch_destroy(gao_batch* b) { free_batch(b); }
