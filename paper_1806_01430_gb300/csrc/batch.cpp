// Batched gene evaluation over a suite of programs.
//
// The GA scores a gene by the processing time of the program it places (Sec. 3.3,
// Sec. 5.1.2).  For a suite of many programs of uneven sizes (e.g. 64 six-loop
// programs with n from 128 to 2048), launching every small program's kernels one by
// one leaves the GPU idle between tiny launches.  A batch runs one gene over the whole
// suite phase by phase instead: for loop i, every program's loop i runs at once --
// on the GPU when gene bit i is 1, on the host when it is 0 -- so each GPU phase is a
// single CUDA graph launch.  The graphs are captured once, when the batch is created:
// each phase forks the programs' kernels over several side streams (small kernels of
// different programs run concurrently) and, for the GEMM loop of a tensor-core
// precision, joins into one grouped tcgen05 launch over every program's tiles; the INIT
// loop of all programs is one grouped launch too.  With fused chains, a gene that puts
// the GEMM -> scale-add -> transpose [-> row sums] [-> norm] chain on the GPU runs it in
// the grouped launch's epilogue (one captured GEMM phase per chain shape).  A gene
// then costs its boundary copies, its graph launches and its host loops.  The gene's
// time is the wall time of the whole suite under that gene; a gene measured before is
// served from the batch's cache (Sec. 4).
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

struct gao_batch {
    std::vector<gao_prog*> progs;
    int n_loops = 0;
    int n_genes = 0;  // offloadable loops (gene length)
    int prec = 0;
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, g0 = nullptr, g1 = nullptr;
    std::vector<cudaGraph_t> graph;
    std::vector<cudaGraphExec_t> exec;
    std::vector<int> phase_kernels;  // kernels in each loop's phase graph
    int gemm_loop = -1;
    bool grouped_gemm = false;
    int init_loop = -1;             // INIT loop run as one grouped launch over all programs
    InitEntry* d_init = nullptr;    // its table: every program's outputs
    int n_init = 0;
    int64_t init_total4 = 0;
    TcProblem* d_probs = nullptr;
    int n_probs = 0, total_tiles = 0;
    std::vector<size_t> gemm_order;  // programs in problem-table order (largest GEMM first)
    std::vector<TcProblem> h_probs;  // host copy of the problem table
    double gemm_flops = 0.0;
    int* d_err = nullptr;
    int* h_err = nullptr;
    std::unordered_map<uint64_t, double> cache;
    gao_batch_stat stat{};
    double timeout_s = 0.0;
    // fused chains (programs created with GAO_FUSE_ON): a gene whose chain GEMM -> AXPY ->
    // TRANSPOSE [-> ROWSUM] [-> FROBENIUS] is on the GPU runs it in the grouped GEMM's
    // epilogue; one captured GEMM phase per chain shape, made on first use
    bool fuse = false;
    struct FusedPhase {
        bool ok = false;  // every program has this chain
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        TcProblem* d_probs = nullptr;
        int kernels = 0;  // kernels in the graph
    };
    std::unordered_map<int, FusedPhase> fused;
};

namespace {

constexpr int kSide = 8;

void drop_fused(gao_batch* b) {
    for (auto& kv : b->fused) {
        if (kv.second.x) cudaGraphExecDestroy(kv.second.x);
        if (kv.second.g) cudaGraphDestroy(kv.second.g);
        if (kv.second.d_probs) cudaFree(kv.second.d_probs);
    }
    b->fused.clear();
}

void free_batch(gao_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    drop_fused(b);
    for (auto e : b->exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto g : b->graph)
        if (g) cudaGraphDestroy(g);
    for (auto e : b->join)
        if (e) cudaEventDestroy(e);
    for (auto s : b->side)
        if (s) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->g0) cudaEventDestroy(b->g0);
    if (b->g1) cudaEventDestroy(b->g1);
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->d_init) cudaFree(b->d_init);
    if (b->d_err) cudaFree(b->d_err);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->st) cudaStreamDestroy(b->st);
    delete b;
}

// Capture the GPU work of loop li for every program into one graph.
gao_status capture_phase(gao_batch* b, int li, std::vector<TcProblem>* probs) {
    cudaStream_t st = b->st;
    GAO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gao_status status = GAO_OK;
    cudaError_t e = cudaEventRecord(b->fork, st);
    for (int k = 0; k < kSide && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[(size_t)k], b->fork, 0);
    const bool tc_gemm = li == b->gemm_loop && b->grouped_gemm;
    const bool group_init = li == b->init_loop;  // one launch after the (empty) branches
    std::vector<size_t> order(b->progs.size());
    std::iota(order.begin(), order.end(), 0);
    const int32_t kernels0 = b->stat.launches_per_gene;
    if (tc_gemm) {
        order = b->gemm_order;
        probs->assign(b->progs.size(), TcProblem{});
    }
    for (size_t j = 0; j < order.size() && e == cudaSuccess && status == GAO_OK && !group_init; ++j) {
        gao_prog* p = b->progs[order[j]];
        cudaStream_t s = b->side[j % kSide];
        if (tc_gemm) {
            const gao_loop& L = p->loops[(size_t)li];
            const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
            float* c0 = L.ins[2] >= 0 ? (float*)p->bufs[(size_t)L.ins[2]].dev : (float*)p->bufs[(size_t)L.outs[0]].dev;
            std::string why;
            int nl = 0;
            e = tc_prepare(b->prec, (float*)p->bufs[(size_t)L.outs[0]].dev, (const float*)p->bufs[(size_t)L.ins[0]].dev,
                           (const float*)p->bufs[(size_t)L.ins[1]].dev, c0, A.rows, B.cols, A.cols, (float)L.alpha,
                           L.ins[2] >= 0 ? (float)L.beta : 0.0f, p->opts.kchunk, p->opts.tile_cfg,
                           p->arena + p->lay.tc_off, p->lay.tc_bytes, s, &(*probs)[j], &nl, &why);
            if (e != cudaSuccess && !why.empty()) status = fail(GAO_EINVAL, "batch GEMM: " + why);
            b->stat.launches_per_gene += nl;
        } else {
            RunCtx R{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, s, false};
            const int before = p->stats[(size_t)li].launches;
            status = run_gpu_loop(R, li);
            b->stat.launches_per_gene += p->stats[(size_t)li].launches - before;
            p->stats[(size_t)li].launches = before;
        }
    }
    for (int k = 0; k < kSide && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[(size_t)k], b->side[(size_t)k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[(size_t)k], 0);
    }
    if (group_init && e == cudaSuccess) {
        e = launch_init_group(b->d_init, b->n_init, b->init_total4, st);
        b->stat.launches_per_gene += 1;
    }
    if (tc_gemm && e == cudaSuccess && status == GAO_OK) {
        bool chunked = false;
        for (auto* p : b->progs) chunked |= p->opts.kchunk > 0;
        e = tc_launch_grouped(b->prec, chunked, b->d_probs, b->n_probs, b->total_tiles, b->d_err, st);
        b->stat.launches_per_gene += 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (status != GAO_OK) {
        if (g) cudaGraphDestroy(g);
        return status;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "batch capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    b->graph[(size_t)li] = g;
    b->phase_kernels[(size_t)li] = b->stat.launches_per_gene - kernels0;
    GAO_CUDA_TRY(cudaGraphInstantiate(&b->exec[(size_t)li], g, 0));
    return GAO_OK;
}

int chain_key(const Chain& ch) { return (ch.rowsum + 1) * 1024 + (ch.frob + 1); }

// The GEMM phase with chain `ch` fused, for every program: splits on the side streams, one
// grouped launch whose problems carry the chain's epilogue, then each program's norm and
// row sums from its partials on the side streams again.
gao_status capture_fused(gao_batch* b, uint64_t mask, const Chain& ch, gao_batch::FusedPhase* fp) {
    const size_t n = b->progs.size();
    fp->ok = true;
    for (auto* p : b->progs) {  // the same chain in every program, or no fusion for this shape
        Chain c;
        if (!find_chain(p, b->gemm_loop, mask, true, &c) || c.axpy != ch.axpy || c.transpose != ch.transpose ||
            c.rowsum != ch.rowsum || c.frob != ch.frob)
            fp->ok = false;
    }
    if (!fp->ok) return GAO_OK;
    GAO_CUDA_TRY(cudaMalloc((void**)&fp->d_probs, sizeof(TcProblem) * n));
    std::vector<TcProblem> probs(n);
    std::vector<TcFuse> fz(n);
    auto dev = [](gao_prog* p, int bi) { return (float*)p->bufs[(size_t)bi].dev; };
    cudaStream_t st = b->st;
    bool chunked = false;
    for (auto* p : b->progs) chunked |= p->opts.kchunk > 0;
    GAO_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gao_status status = GAO_OK;
    auto fork = [&]() {
        cudaError_t e = cudaEventRecord(b->fork, st);
        for (int k = 0; k < kSide && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[(size_t)k], b->fork, 0);
        return e;
    };
    auto join = [&]() {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kSide && e == cudaSuccess; ++k) {
            e = cudaEventRecord(b->join[(size_t)k], b->side[(size_t)k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[(size_t)k], 0);
        }
        return e;
    };
    cudaError_t e = fork();
    for (size_t j = 0; j < n && e == cudaSuccess && status == GAO_OK; ++j) {
        gao_prog* p = b->progs[b->gemm_order[j]];
        const gao_loop &L = p->loops[(size_t)b->gemm_loop], &X = p->loops[(size_t)ch.axpy],
                       &T = p->loops[(size_t)ch.transpose];
        const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
        fz[j] = TcFuse{dev(p, X.ins[1]), dev(p, X.outs[0]), dev(p, T.outs[0]),
                       ch.frob >= 0 ? (double*)p->bufs[(size_t)p->loops[(size_t)ch.frob].outs[0]].dev : nullptr,
                       (float)X.alpha, 0, ch.rowsum >= 0 ? dev(p, p->loops[(size_t)ch.rowsum].outs[0]) : nullptr};
        float* c0 = L.ins[2] >= 0 ? dev(p, L.ins[2]) : dev(p, L.outs[0]);
        std::string why;
        int nl = 0;
        e = tc_prepare(b->prec, dev(p, L.outs[0]), dev(p, L.ins[0]), dev(p, L.ins[1]), c0, A.rows, B.cols, A.cols,
                       (float)L.alpha, L.ins[2] >= 0 ? (float)L.beta : 0.0f, p->opts.kchunk, p->opts.tile_cfg,
                       p->arena + p->lay.tc_off, p->lay.tc_bytes, b->side[j % kSide], &probs[j], &nl, &why, &fz[j]);
        if (e != cudaSuccess && !why.empty()) status = fail(GAO_EINVAL, "batch fused GEMM: " + why);
        fp->kernels += nl;
    }
    if (e == cudaSuccess) e = join();
    if (e == cudaSuccess && status == GAO_OK) {
        e = tc_launch_grouped(b->prec, chunked, fp->d_probs, (int)n, b->total_tiles, b->d_err, st);
        fp->kernels += 1;
    }
    if (e == cudaSuccess && status == GAO_OK) e = fork();
    for (size_t j = 0; j < n && e == cudaSuccess && status == GAO_OK; ++j) {
        gao_prog* p = b->progs[b->gemm_order[j]];
        const gao_loop& L = p->loops[(size_t)b->gemm_loop];
        const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
        int nl = 0;
        e = tc_finalize_chain(b->prec, A.rows, B.cols, A.cols, p->arena + p->lay.tc_off, fz[j], b->side[j % kSide], &nl);
        fp->kernels += nl;
    }
    if (e == cudaSuccess && status == GAO_OK) e = join();
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (status != GAO_OK || e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (status != GAO_OK) return status;
        return cuda_fail(e != cudaSuccess ? e : e2, "batch fused capture");
    }
    fp->g = g;
    GAO_CUDA_TRY(cudaGraphInstantiate(&fp->x, g, 0));
    int start = 0;
    for (auto& pr : probs) {
        pr.tile_start = start;
        start += pr.tiles_m * pr.tiles_n;
    }
    if (start != b->total_tiles) return fail(GAO_EINVAL, "batch tile count mismatch");
    GAO_CUDA_TRY(cudaMemcpy(fp->d_probs, probs.data(), sizeof(TcProblem) * n, cudaMemcpyHostToDevice));
    return GAO_OK;
}

// Every chain shape a gene can give (the GEMM, scale-add and transpose on the GPU; each
// later reduction of E on the GPU or not), captured up front so that no gene's time holds
// a capture.
gao_status capture_all_fused(gao_batch* b) {
    if (!b->fuse) return GAO_OK;
    const gao_prog* p0 = b->progs[0];
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
        if (!find_chain(p0, b->gemm_loop, m, true, &c) || b->fused.count(chain_key(c))) continue;
        gao_batch::FusedPhase& slot = b->fused[chain_key(c)];
        gao_status s = capture_fused(b, m, c, &slot);
        if (s != GAO_OK || !slot.x) slot.ok = false;
        if (s != GAO_OK) return s;
    }
    return GAO_OK;
}

// One gene over the whole suite; *seconds = wall time (budget on timeout, -1 on failure).
gao_status run_gene(gao_batch* b, uint64_t gene, double* seconds) {
    const int n = b->n_loops;
    if (b->n_genes < 64 && (gene >> b->n_genes) != 0) return fail(GAO_EINVAL, "gene has bits above the gene length");
    const uint64_t mask = loop_mask_of(b->progs[0], gene);  // bit li: loop li on the GPU
    const double t0 = now_s();
    const double deadline = b->timeout_s > 0.0 ? t0 + b->timeout_s : 0.0;
    std::vector<RunCtx> R;
    R.reserve(b->progs.size());
    for (auto* p : b->progs) {
        for (auto& B : p->bufs) {
            B.vh = (B.d.role == GAO_BUF_INPUT);
            B.vd = false;
        }
        R.push_back(RunCtx{p, deadline, false, CpuCtx{p->opts.cpu_threads, deadline, false}, b->st, false});
    }
    // the chain in the GEMM's epilogue when this gene puts all of it on the GPU
    Chain ch;
    gao_batch::FusedPhase* fp = nullptr;
    if (b->fuse && ((mask >> b->gemm_loop) & 1) && find_chain(b->progs[0], b->gemm_loop, mask, true, &ch)) {
        auto it = b->fused.find(chain_key(ch));
        if (it == b->fused.end()) {
            gao_batch::FusedPhase& slot = b->fused[chain_key(ch)];
            gao_status s = capture_fused(b, mask, ch, &slot);
            if (s != GAO_OK || !slot.x) slot.ok = false;  // never launched half-made
            if (s != GAO_OK) return s;
            it = b->fused.find(chain_key(ch));
        }
        if (it->second.ok) fp = &it->second;
    }
    uint64_t in_epilogue = 0;  // loops that ran in the GEMM's epilogue
    GAO_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st));
    bool timed_out = false;
    gao_loop_stat scratch{};
    for (int li = 0; li < n && !timed_out; ++li) {
        if ((in_epilogue >> li) & 1) continue;
        const bool gpu = (mask >> li) & 1;
        for (auto& r : R)
            for (int bi : loop_inputs(r.p->loops[(size_t)li])) {
                gao_status s = make_valid(r, bi, gpu, scratch);
                if (s != GAO_OK) return s;
            }
        if (gpu && fp && li == b->gemm_loop) {
            for (auto& r : R) {  // the AXPY's second operand is read in the epilogue
                gao_status s = make_valid(r, r.p->loops[(size_t)ch.axpy].ins[1], true, scratch);
                if (s != GAO_OK) return s;
            }
            GAO_CUDA_TRY(cudaEventRecord(b->g0, b->st));
            GAO_CUDA_TRY(cudaGraphLaunch(fp->x, b->st));
            GAO_CUDA_TRY(cudaEventRecord(b->g1, b->st));
            b->stat.fused_phases += 1;
            b->stat.kernel_launches += fp->kernels;
            for (int j : {li, ch.axpy, ch.transpose, ch.rowsum, ch.frob}) {
                if (j < 0) continue;
                in_epilogue |= 1ULL << j;
                for (auto& r : R)
                    for (int bo : loop_outputs(r.p->loops[(size_t)j])) {
                        r.p->bufs[(size_t)bo].vh = false;
                        r.p->bufs[(size_t)bo].vd = true;
                    }
            }
            if (deadline > 0.0 && now_s() > deadline) timed_out = true;
            continue;
        }
        if (gpu) {
            if (li == b->gemm_loop) GAO_CUDA_TRY(cudaEventRecord(b->g0, b->st));
            GAO_CUDA_TRY(cudaGraphLaunch(b->exec[(size_t)li], b->st));
            b->stat.kernel_launches += b->phase_kernels[(size_t)li];
            if (li == b->gemm_loop) GAO_CUDA_TRY(cudaEventRecord(b->g1, b->st));
        } else {
            gao_status s = stream_wait(b->st, deadline, &timed_out);
            if (s != GAO_OK) return s;
            for (auto& r : R) {
                if (timed_out) break;
                if ((s = run_cpu_loop(r, li)) != GAO_OK) return s;
                if (r.cpu.timed_out) timed_out = true;
            }
        }
        for (auto& r : R)
            for (int bo : loop_outputs(r.p->loops[(size_t)li])) {
                r.p->bufs[(size_t)bo].vh = !gpu;
                r.p->bufs[(size_t)bo].vd = gpu;
            }
        if (deadline > 0.0 && now_s() > deadline) timed_out = true;
    }
    if (!timed_out)
        for (auto& r : R)
            for (size_t bi = 0; bi < r.p->bufs.size(); ++bi)
                if (r.p->bufs[bi].d.role == GAO_BUF_OUTPUT && !r.p->bufs[bi].vh) {
                    gao_status s = make_valid(r, (int)bi, false, scratch);
                    if (s != GAO_OK) return s;
                }
    GAO_CUDA_TRY(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    gao_status s = stream_wait(b->st, deadline, &timed_out);
    if (s != GAO_OK) return s;
    const double t1 = now_s();
    if (*b->h_err != 0) {
        *seconds = -1.0;
        return fail(GAO_EDEVICE, "a batch kernel raised device error " + std::to_string(*b->h_err));
    }
    if ((mask >> b->gemm_loop) & 1) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, b->g0, b->g1) == cudaSuccess) b->stat.gemm_phase_ms = ms;
    }
    *seconds = timed_out ? b->timeout_s : (t1 - t0);
    return GAO_OK;
}

// Time of a gene: cached, or measured now.  Failures score -1 (fitness 0).
gao_status gene_seconds(gao_batch* b, uint64_t mask, double* t, bool* cached) {
    auto it = b->cache.find(mask);
    if (it != b->cache.end()) {
        *t = it->second;
        *cached = true;
        b->stat.served += 1;
        return GAO_OK;
    }
    *cached = false;
    const double w0 = now_s();
    double s = 0.0;
    gao_status st = run_gene(b, mask, &s);
    b->stat.exec_seconds += now_s() - w0;
    if (st == GAO_EDEVICE || st == GAO_ECPU) {
        s = -1.0;
    } else if (st != GAO_OK) {
        return st;
    }
    b->cache.emplace(mask, s);
    b->stat.executed += 1;
    *t = s;
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
    b->progs.assign(progs, progs + n_progs);
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
        (e = cudaEventCreate(&b->g0)) != cudaSuccess || (e = cudaEventCreate(&b->g1)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaMalloc((void**)&b->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&b->h_err, sizeof(int))) != cudaSuccess)
        return bail(cuda_fail(e, "batch error word"));
    *b->h_err = 0;
    b->graph.assign((size_t)b->n_loops, nullptr);
    b->phase_kernels.assign((size_t)b->n_loops, 0);
    b->exec.assign((size_t)b->n_loops, nullptr);
    // everything the captures touch that is not a stream operation happens first
    for (auto* p : b->progs) {
        if ((e = cudaStreamSynchronize(p->st)) != cudaSuccess) return bail(cuda_fail(e, "program stream"));
    }
    std::vector<TcProblem> probs;
    if (b->grouped_gemm) {
        bool chunked = false;
        for (auto* p : b->progs) chunked |= p->opts.kchunk > 0;
        std::string why;
        if (!tc_available(&why)) return bail(fail(GAO_ENODEV, why));
        if ((e = tc_launch_grouped(b->prec, chunked, nullptr, 0, 0, nullptr, b->st)) != cudaSuccess)
            return bail(cuda_fail(e, "grouped GEMM set-up"));
        b->n_probs = n_progs;
        if ((e = cudaMalloc((void**)&b->d_probs, sizeof(TcProblem) * (size_t)n_progs)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc(problem table)"));
        for (auto* p : b->progs) {
            const gao_loop& L = p->loops[(size_t)b->gemm_loop];
            const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
            if (A.rows <= 0 || B.cols <= 0 || A.cols <= 0)
                return bail(fail(GAO_EINVAL, "batch GEMM needs positive sizes on the tensor-core path"));
            b->gemm_flops += 2.0 * A.rows * B.cols * A.cols;
        }
    }
    if (b->grouped_gemm) {
        // problem table order: largest GEMM first, so that the launch's tail is made of
        // small tiles; tile counts follow from the shapes (128 x 128 tiles)
        auto gemm_shape = [&](size_t x, int64_t* m, int64_t* nn, int64_t* k) {
            const gao_loop& L = b->progs[x]->loops[(size_t)b->gemm_loop];
            *m = b->progs[x]->bufs[(size_t)L.ins[0]].d.rows;
            *k = b->progs[x]->bufs[(size_t)L.ins[0]].d.cols;
            *nn = b->progs[x]->bufs[(size_t)L.ins[1]].d.cols;
        };
        b->gemm_order.resize(b->progs.size());
        std::iota(b->gemm_order.begin(), b->gemm_order.end(), 0);
        std::stable_sort(b->gemm_order.begin(), b->gemm_order.end(), [&](size_t x, size_t y) {
            int64_t mx, nx, kx, my, ny, ky;
            gemm_shape(x, &mx, &nx, &kx);
            gemm_shape(y, &my, &ny, &ky);
            return (double)mx * nx * kx > (double)my * ny * ky;
        });
        int64_t start = 0;
        for (size_t j : b->gemm_order) {
            int64_t m, nn, k;
            gemm_shape(j, &m, &nn, &k);
            start += ((m + 127) / 128) * ((nn + 127) / 128);
        }
        if (start > 0x7fffffff) return bail(fail(GAO_EINVAL, "batch GEMM has too many tiles"));
        b->total_tiles = (int)start;
    }
    // the first INIT loop without row scaling: one grouped launch over every program's
    // outputs instead of a launch per program (many small launches in a row cost more than
    // their writes)
    for (int li = 0; li < b->n_loops && b->init_loop < 0; ++li) {
        const gao_loop& L0 = p0->loops[(size_t)li];
        if (L0.kind != GAO_LOOP_INIT || p0->verdict[(size_t)li] != GAO_OFFLOAD_OK) continue;
        bool plain = true;
        for (auto* p : b->progs) plain &= (p->loops[(size_t)li].flags & ((1u << GAO_MAX_IO) - 1)) == 0;
        if (!plain) break;
        std::vector<InitEntry> tab;
        int64_t start = 0;
        for (auto* p : b->progs) {
            const gao_loop& L = p->loops[(size_t)li];
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
        if (tab.empty()) break;
        if ((e = cudaMalloc((void**)&b->d_init, sizeof(InitEntry) * tab.size())) != cudaSuccess ||
            (e = cudaMemcpy(b->d_init, tab.data(), sizeof(InitEntry) * tab.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return bail(cuda_fail(e, "INIT table"));
        b->init_loop = li;
        b->n_init = (int)tab.size();
        b->init_total4 = start;
    }
    b->stat.launches_per_gene = 0;
    for (int li = 0; li < b->n_loops; ++li) {
        if (p0->verdict[(size_t)li] != GAO_OFFLOAD_OK) continue;  // host-only loop: no graph
        if ((s = capture_phase(b, li, &probs)) != GAO_OK) return bail(s);
        if (li == b->gemm_loop && b->grouped_gemm) {
            int start = 0;
            for (auto& pr : probs) {
                pr.tile_start = start;
                start += pr.tiles_m * pr.tiles_n;
            }
            if (start != b->total_tiles) return bail(fail(GAO_EINVAL, "batch tile count mismatch"));
            if ((e = cudaMemcpy(b->d_probs, probs.data(), sizeof(TcProblem) * probs.size(),
                                cudaMemcpyHostToDevice)) != cudaSuccess)
                return bail(cuda_fail(e, "problem table upload"));
            b->h_probs = probs;
        }
    }
    b->stat.graphs = b->n_genes;
    if ((s = capture_all_fused(b)) != GAO_OK) return bail(s);
    *out = b;
    return GAO_OK;
}

extern "C" gao_status batch_evaluate(gao_batch* b, const uint64_t* population, int pop, double* fitness_out,
                                     double* seconds_out, int* cache_hits_out) {
    if (!b || !population || pop < 0) return fail(GAO_EINVAL, "bad batch or population");
    int hits = 0;
    for (int i = 0; i < pop; ++i) {
        double t = 0.0;
        bool cached = false;
        gao_status s = gene_seconds(b, population[i], &t, &cached);
        if (s != GAO_OK) return s;
        hits += cached;
        if (seconds_out) seconds_out[i] = t;
        if (fitness_out) fitness_out[i] = ga_fitness(t);
    }
    if (cache_hits_out) *cache_hits_out = hits;
    return GAO_OK;
}

extern "C" gao_status batch_ga_run(gao_batch* b, const gao_ga_params* params, gao_ga_result* result) {
    if (!b || !params || !result) return fail(GAO_EINVAL, "null argument");
    const double saved = b->timeout_s;
    double budget = params->timeout_s;
    if (budget < 0.0) {  // automatic: 10 x the all-GPU time of the suite, capped at 60 s
        const uint64_t all = all_genes(b->n_genes);
        double t = 0.0;
        bool cached = false;
        b->timeout_s = 0.0;
        gao_status s = gene_seconds(b, all, &t, &cached);
        if (s != GAO_OK) return s;
        budget = std::min(60.0, 10.0 * t);
    }
    if (budget > 0.0) b->timeout_s = budget;
    TimeFn fn = [&](uint64_t m, double* t) {
        bool cached = false;
        return gene_seconds(b, m, t, &cached);
    };
    if (b->n_genes < 1) return fail(GAO_EINVAL, "no loop of the batch is offloadable (gene length 0)");
    gao_status s = ga_core(b->n_genes, *params, fn, result);
    b->timeout_s = saved;
    return s;
}

extern "C" gao_status batch_stats(gao_batch* b, gao_batch_stat* out) {
    if (!b || !out) return fail(GAO_EINVAL, "null argument");
    *out = b->stat;
    out->gemm_flops = b->gemm_flops;
    out->gemm_tiles = b->total_tiles;
    return GAO_OK;
}

extern "C" gao_status batch_autotune(gao_batch* b, const gao_ga_params* params, gao_autotune_result* out) {
    if (!b || !params || !out) return fail(GAO_EINVAL, "null argument");
    if (!b->grouped_gemm) return fail(GAO_EINVAL, "batch has no tensor-core GEMM loop");
    const uint64_t all = all_genes(b->n_genes);
    double s0 = 0.0;
    gao_status st = run_gene(b, all, &s0);  // the GEMM's inputs on the device
    if (st != GAO_OK) return st;
    bool chunked_variant = false;
    for (auto* p : b->progs) chunked_variant |= p->opts.kchunk > 0;
    std::vector<TcProblem> table = b->h_probs;
    auto apply = [&](int kchunk, int tile_cfg) -> gao_status {
        table = b->h_probs;  // the configuration in place, then this one's changes
        for (auto& pr : table) {
            pr.group = tc_group_of(tile_cfg);
            pr.pf_kb = tc_prefetch_of(tile_cfg);
            if (chunked_variant && kchunk > 0) pr.chunk_kb = std::max(1, std::min(pr.num_kb, kchunk / 64));
        }
        GAO_CUDA_TRY(cudaMemcpyAsync(b->d_probs, table.data(), sizeof(TcProblem) * table.size(),
                                     cudaMemcpyHostToDevice, b->st));
        return GAO_OK;
    };
    auto time_cfg = [&](int kchunk, int tile_cfg, double* ms) -> gao_status {
        gao_status s = apply(kchunk, tile_cfg);
        if (s != GAO_OK) return s;
        // a configuration whose launch raised the error word fails the tuning (GAO_EDEVICE)
        GAO_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), b->st));
        std::vector<double> v;
        for (int r = 0; r < 4; ++r) {
            GAO_CUDA_TRY(cudaEventRecord(b->g0, b->st));
            GAO_CUDA_TRY(cudaGraphLaunch(b->exec[(size_t)b->gemm_loop], b->st));
            GAO_CUDA_TRY(cudaEventRecord(b->g1, b->st));
            GAO_CUDA_TRY(cudaEventSynchronize(b->g1));
            float t = 0.0f;
            cudaEventElapsedTime(&t, b->g0, b->g1);
            if (r > 0) v.push_back(t);
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
    int kc0 = b->progs[0]->opts.kchunk, tc0 = b->progs[0]->opts.tile_cfg;
    double def_ms = 0.0;
    if ((st = time_cfg(kc0, tc0, &def_ms)) != GAO_OK) return st;
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
    if ((st = ga_core(kAutotuneBits, *params, fn, &res)) != GAO_OK) return st;
    // the configuration in place stays unless the GA found a faster one
    int kc = kc0, tc = tc0;
    double best_ms = def_ms;
    if (res.best_s * 1e3 < def_ms) {
        autotune_decode(b->prec, res.best_mask, &kc, &tc);
        best_ms = res.best_s * 1e3;
    }
    if ((st = apply(kc, tc)) != GAO_OK) return st;
    b->h_probs = table;
    for (auto* p : b->progs) {
        if (chunked_variant) p->opts.kchunk = kc;
        p->opts.tile_cfg = tc;
        drop_graphs(p);
    }
    b->cache.clear();  // genes measured under the old configuration
    GAO_CUDA_TRY(cudaStreamSynchronize(b->st));
    drop_fused(b);  // fused GEMM phases are captured again with the new configuration
    if ((st = capture_all_fused(b)) != GAO_OK) return st;
    out->kchunk = chunked_variant ? kc : 0;
    out->tile_cfg = tc;
    out->best_ms = best_ms;
    out->default_ms = def_ms;
    out->evaluations = evals;
    return GAO_OK;
}

extern "C" void batch_destroy(gao_batch* b) { free_batch(b); }
