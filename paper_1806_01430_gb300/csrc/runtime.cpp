// Loop-program runtime and the C ABI (include/gao.h).
//
// A program is a list of buffers and loops (Sec. 4: the application's loops; those that
// pass the parallelisability check are numbered 0..a-1 and make up the gene).
// prog_run executes the loops in order, offloadable loop k on the GPU when gene bit k
// is 1 and every other loop on the host, and moves a buffer between host and device
// only when a loop needs it on the other side
// (Sec. 3.3: transfers between CPU and GPU memory are what make some loop
// combinations slower than others).  Residency is tracked per buffer with two bits
// (valid on host, valid on device).  The time of a run is the wall time from the
// first loop until every OUTPUT buffer is on the host; that is the benchmark time
// the GA turns into fitness (Sec. 5.1.2).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ga_engine.h"
#include "gao_internal.h"
#include "gemm_tc.h"
#include "prog_internal.h"

namespace gao {

// ---- errors -------------------------------------------------------------------------

namespace {
thread_local std::string t_err;
}

void set_error(const std::string& msg) { t_err = msg; }

gao_status fail(gao_status st, const std::string& msg) {
    t_err = msg;
    return st;
}

gao_status cuda_fail(cudaError_t e, const char* what) {
    t_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return GAO_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorNoKernelImageForDevice)
        return GAO_ENODEV;
    return GAO_ECUDA;
}

// ---- device ---------------------------------------------------------------------------

namespace {
std::mutex g_dev_mu;
int g_sm_count = 0;
}  // namespace

gao_status check_device(int* dev_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(GAO_ENODEV, "device " + std::string(prop.name) + " is sm_" + std::to_string(prop.major) +
                                    std::to_string(prop.minor) + "; this library is built for sm_103a only");
    {
        std::lock_guard<std::mutex> g(g_dev_mu);
        g_sm_count = prop.multiProcessorCount;
    }
    if (dev_out) *dev_out = dev;
    return GAO_OK;
}

int sm_count() {
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (g_sm_count == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            g_sm_count = n;
        else
            g_sm_count = 152;
    }
    return g_sm_count;
}

}  // namespace gao

using namespace gao;

// ---- program ------------------------------------------------------------------------------

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
size_t elem_size(int32_t dtype) { return dtype == GAO_F64 ? 8 : 4; }

}  // namespace

namespace {

// K elements per binary32 partial sum when the caller passes 0: the FP32 SIMT path and
// the split tensor-core paths restart their accumulators so that rounding error does
// not grow with K; plain bfloat16 is far above that error level and runs unchunked.
int default_kchunk(int prec) {
    switch (prec) {
        case GAO_GEMM_FP32_SIMT: return 256;
        case GAO_GEMM_BF16X6: return 256;
        case GAO_GEMM_BF16X3: return 1024;  // error set by the two-term split (3.4e-6 at 256 and 1024)
        default: return 0;
    }
}

gao_status validate(const gao_loop* loops, int n_loops, const gao_buffer* bufs, int n_bufs, const gao_opts* opts) {
    if (!loops || !bufs) return fail(GAO_EINVAL, "loops and buffers must be non-null");
    if (n_loops < 1 || n_loops > 64) return fail(GAO_EINVAL, "loop count must be in [1, 64]");
    if (n_bufs < 1 || n_bufs > 4096) return fail(GAO_EINVAL, "buffer count must be in [1, 4096]");
    if (opts && (opts->gemm_prec < GAO_GEMM_FP32_SIMT || opts->gemm_prec > GAO_GEMM_FP8))
        return fail(GAO_EINVAL, "unknown gemm_prec");
    if (opts && opts->transfer_mode != GAO_TRANSFER_RESIDENT && opts->transfer_mode != GAO_TRANSFER_PER_LOOP)
        return fail(GAO_EINVAL, "unknown transfer_mode");
    if (opts && (opts->fuse_chains < GAO_FUSE_OFF || opts->fuse_chains > GAO_FUSE_GENE))
        return fail(GAO_EINVAL, "fuse_chains must be GAO_FUSE_OFF, GAO_FUSE_ON or GAO_FUSE_GENE");
    for (int b = 0; b < n_bufs; ++b) {
        const gao_buffer& d = bufs[b];
        if (d.rows < 0 || d.cols < 0) return fail(GAO_EINVAL, "buffer " + std::to_string(b) + ": negative shape");
        if (d.dtype != GAO_F32 && d.dtype != GAO_F64)
            return fail(GAO_EINVAL, "buffer " + std::to_string(b) + ": unknown dtype");
        if (d.role < GAO_BUF_TEMP || d.role > GAO_BUF_OUTPUT)
            return fail(GAO_EINVAL, "buffer " + std::to_string(b) + ": unknown role");
        if (d.rows > (int64_t)1 << 31 || d.cols > (int64_t)1 << 31)
            return fail(GAO_EINVAL, "buffer " + std::to_string(b) + ": dimension above 2^31");
    }
    std::vector<char> defined((size_t)n_bufs, 0);
    for (int b = 0; b < n_bufs; ++b) defined[(size_t)b] = bufs[b].role == GAO_BUF_INPUT;
    auto okbuf = [&](int i) { return i >= 0 && i < n_bufs; };
    for (int li = 0; li < n_loops; ++li) {
        const gao_loop& L = loops[li];
        const std::string where = "loop " + std::to_string(li) + ": ";
        auto need_in = [&](int slot) -> gao_status {
            const int b = L.ins[slot];
            if (!okbuf(b)) return fail(GAO_EINVAL, where + "input slot " + std::to_string(slot) + " is not a buffer");
            if (!defined[(size_t)b])
                return fail(GAO_EINVAL, where + "reads buffer " + std::to_string(b) + " before any loop writes it");
            if (bufs[b].dtype != GAO_F32) return fail(GAO_EINVAL, where + "inputs must be binary32 matrices");
            return GAO_OK;
        };
        auto need_out = [&](int slot, int64_t r, int64_t c, int32_t dt) -> gao_status {
            const int b = L.outs[slot];
            if (!okbuf(b)) return fail(GAO_EINVAL, where + "output slot " + std::to_string(slot) + " is not a buffer");
            if (bufs[b].rows != r || bufs[b].cols != c || bufs[b].dtype != dt)
                return fail(GAO_EINVAL, where + "output buffer " + std::to_string(b) + " has shape " +
                                            std::to_string(bufs[b].rows) + "x" + std::to_string(bufs[b].cols) +
                                            ", expected " + std::to_string(r) + "x" + std::to_string(c));
            if (bufs[b].role == GAO_BUF_INPUT) return fail(GAO_EINVAL, where + "writes an INPUT buffer");
            return GAO_OK;
        };
        gao_status s = GAO_OK;
        switch (L.kind) {
            case GAO_LOOP_INIT: {
                int nout = 0;
                for (int t = 0; t < GAO_MAX_IO; ++t) {
                    if (L.outs[t] < 0) continue;
                    const int b = L.outs[t];
                    if (!okbuf(b)) return fail(GAO_EINVAL, where + "output is not a buffer");
                    if (b > 14) return fail(GAO_EINVAL, where + "INIT writes buffer ids 0..14 only");
                    if ((s = need_out(t, bufs[b].rows, bufs[b].cols, GAO_F32)) != GAO_OK) return s;
                    defined[(size_t)b] = 1;
                    ++nout;
                }
                if (nout == 0) return fail(GAO_EINVAL, where + "INIT has no output");
                continue;
            }
            case GAO_LOOP_GEMM: {
                if ((s = need_in(0)) || (s = need_in(1))) return s;
                const gao_buffer &A = bufs[L.ins[0]], &B = bufs[L.ins[1]];
                if (A.cols != B.rows) return fail(GAO_EINVAL, where + "inner dimensions of A and B differ");
                if (L.ins[2] >= 0) {
                    if ((s = need_in(2))) return s;
                    const gao_buffer& C0 = bufs[L.ins[2]];
                    if (C0.rows != A.rows || C0.cols != B.cols) return fail(GAO_EINVAL, where + "C0 shape mismatch");
                } else if (L.beta != 0.0) {
                    return fail(GAO_EINVAL, where + "beta != 0 needs a C0 input");
                }
                if ((s = need_out(0, A.rows, B.cols, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0] || L.outs[0] == L.ins[1])
                    return fail(GAO_EINVAL, where + "GEMM output may alias C0 only");
                break;
            }
            case GAO_LOOP_AXPY: {
                if ((s = need_in(0)) || (s = need_in(1))) return s;
                const gao_buffer &X = bufs[L.ins[0]], &Y = bufs[L.ins[1]];
                if (X.rows != Y.rows || X.cols != Y.cols) return fail(GAO_EINVAL, where + "AXPY operand shapes differ");
                if ((s = need_out(0, X.rows, X.cols, GAO_F32))) return s;
                break;
            }
            case GAO_LOOP_TRANSPOSE: {
                if ((s = need_in(0))) return s;
                const gao_buffer& X = bufs[L.ins[0]];
                if ((s = need_out(0, X.cols, X.rows, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0]) return fail(GAO_EINVAL, where + "TRANSPOSE cannot run in place");
                break;
            }
            case GAO_LOOP_ROWSUM: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, bufs[L.ins[0]].rows, 1, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0]) return fail(GAO_EINVAL, where + "ROWSUM cannot run in place");
                break;
            }
            case GAO_LOOP_FROBENIUS:
            case GAO_LOOP_SUM: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, 1, 1, GAO_F64))) return s;
                break;
            }
            case GAO_LOOP_RELU:
            case GAO_LOOP_SQUARE: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, bufs[L.ins[0]].rows, bufs[L.ins[0]].cols, GAO_F32))) return s;
                break;
            }
            case GAO_LOOP_COLMAX: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, 1, bufs[L.ins[0]].cols, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0]) return fail(GAO_EINVAL, where + "COLMAX cannot run in place");
                break;
            }
            case GAO_LOOP_STENCIL3: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, bufs[L.ins[0]].rows, bufs[L.ins[0]].cols, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0]) return fail(GAO_EINVAL, where + "STENCIL3 cannot run in place");
                if ((L.flags & ~GAO_LOOP_EXTERNAL_CALL) > 3)
                    return fail(GAO_EINVAL, where + "unknown STENCIL3 preset " +
                                                std::to_string(L.flags & ~GAO_LOOP_EXTERNAL_CALL));
                break;
            }
            case GAO_LOOP_RECURRENCE: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, bufs[L.ins[0]].rows, bufs[L.ins[0]].cols, GAO_F32))) return s;
                if (L.outs[0] == L.ins[0]) return fail(GAO_EINVAL, where + "RECURRENCE cannot run in place");
                break;
            }
            case GAO_LOOP_FIND: {
                if ((s = need_in(0))) return s;
                if ((s = need_out(0, bufs[L.ins[0]].rows, 1, GAO_F64))) return s;
                break;
            }
            default:
                return fail(GAO_EINVAL, where + "unknown loop kind " + std::to_string(L.kind));
        }
        defined[(size_t)L.outs[0]] = 1;
    }
    for (int b = 0; b < n_bufs; ++b)
        if (bufs[b].role == GAO_BUF_OUTPUT && !defined[(size_t)b])
            return fail(GAO_EINVAL, "OUTPUT buffer " + std::to_string(b) + " is never written");
    return GAO_OK;
}

Layout plan(const gao_loop* loops, int n_loops, const gao_buffer* bufs, int n_bufs, const gao_opts& o) {
    Layout L;
    size_t off = 0;
    L.buf_off.resize((size_t)n_bufs);
    for (int b = 0; b < n_bufs; ++b) {
        L.buf_off[(size_t)b] = off;
        off += align_up(std::max<size_t>(1, (size_t)bufs[b].rows * (size_t)bufs[b].cols * elem_size(bufs[b].dtype)));
    }
    L.err_off = off;
    off += kAlign;
    L.partial_off = off;
    off += align_up((size_t)reduce_blocks() * sizeof(double));
    L.counter_off = off;
    off += kAlign;
    size_t keys = 1, rows = 1, tc = 0, resid = 0, chainpart = 0;
    for (int i = 0; i < n_loops; ++i) {
        const gao_loop& lp = loops[i];
        if (lp.kind == GAO_LOOP_COLMAX) keys = std::max(keys, (size_t)bufs[lp.ins[0]].cols * 4);
        if (lp.kind == GAO_LOOP_STENCIL3) {  // a gradient chain's fused sum: one partial per block,
            // over one launch or over the row strips of a frame copied in from the host, of the
            // chain alone or with the blur before it
            const int64_t r = bufs[lp.ins[0]].rows, c = bufs[lp.ins[0]].cols;
            const int64_t blocks = std::max({grad_chain_blocks(r, c), kMaxRowBlocks * grad_chain_blocks_max(c),
                                             edge_chain_blocks(r, c), kMaxRowBlocks * edge_chain_blocks_max(c)});
            chainpart = std::max(chainpart, (size_t)blocks * 8);
        }
        if (lp.kind == GAO_LOOP_INIT)
            for (int t = 0; t < GAO_MAX_IO; ++t)
                if (lp.outs[t] >= 0 && ((lp.flags >> t) & 1)) rows = std::max(rows, (size_t)bufs[lp.outs[t]].rows);
        if (lp.kind == GAO_LOOP_GEMM && o.gemm_prec != GAO_GEMM_FP32_SIMT) {
            const gao_buffer &A = bufs[lp.ins[0]], &B = bufs[lp.ins[1]];
            tc = std::max(tc, tc_scratch_bytes(o.gemm_prec, A.rows, B.cols, A.cols));
        }
        if (lp.kind == GAO_LOOP_GEMM && lp.ins[2] != lp.outs[0]) {  // a GEMM prog_gemm_residual can check
            const gao_buffer &A = bufs[lp.ins[0]], &B = bufs[lp.ins[1]];
            resid = std::max(resid, align_up((size_t)B.cols * 8) + align_up((size_t)A.rows * 8) +
                                        gemm_residual_scratch_bytes(A.rows, B.cols, A.cols));
        }
    }
    L.keys_off = off;
    L.keys_bytes = keys;
    off += align_up(keys);
    L.rowexp_off = off;
    L.rowexp_bytes = rows;
    off += align_up(rows);
    off = align_up(off, 1024);
    L.tc_off = off;
    L.tc_bytes = tc;
    off += align_up(tc, 1024);
    L.resid_off = off;
    L.resid_bytes = resid;
    off += align_up(resid);
    L.chainpart_off = off;
    L.chainpart_bytes = chainpart;
    off += align_up(chainpart);
    L.total = off;
    return L;
}

}  // namespace

// Wait for the stream; with a deadline, poll and report expiry.  Work already queued
// always completes before returning (kernels bound their own waits), so the program
// is reusable afterwards; hard_cap_s bounds the wait for a GPU that stopped answering.
gao_status gao::stream_wait(cudaStream_t st, double deadline, bool* timed_out, double hard_cap_s) {
    if (deadline <= 0.0) {
        cudaError_t e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? GAO_OK : cuda_fail(e, "cudaStreamSynchronize");
    }
    const double cap = now_s() + hard_cap_s;
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return GAO_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
        const double t = now_s();
        if (t > deadline) *timed_out = true;
        if (t > cap) return fail(GAO_ETIMEOUT, "stream did not drain within the hard cap");
        std::this_thread::yield();
    }
}

namespace {

void free_prog(gao_prog* p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    for (auto& b : p->bufs) {
        if (b.registered) cudaHostUnregister(b.host);
        if (b.own_host) cudaFreeHost(b.own_host);
    }
    if (p->h_err) cudaFreeHost(p->h_err);
    if (p->cst) cudaStreamSynchronize(p->cst);
    if (p->ost) cudaStreamSynchronize(p->ost);
    if (p->st2) cudaStreamSynchronize(p->st2);
    drop_graphs(p);
    for (auto e : p->ev)
        if (e) cudaEventDestroy(e);
    for (auto e : p->pipe_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : p->out_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : p->cmp_ev)
        if (e) cudaEventDestroy(e);
    if (p->cst) cudaStreamDestroy(p->cst);
    if (p->ost) cudaStreamDestroy(p->ost);
    if (p->st2) cudaStreamDestroy(p->st2);
    if (p->own_arena && p->arena_raw) cudaFree(p->arena_raw);
    if (p->own_stream && p->st) cudaStreamDestroy(p->st);
    delete p;
}

}  // namespace

// ---- C ABI: programs -------------------------------------------------------------------

extern "C" gao_status prog_device_bytes(const gao_loop* loops, int n_loops, const gao_buffer* bufs, int n_bufs,
                                        const gao_opts* opts, uint64_t* bytes_out) {
    gao_status s = validate(loops, n_loops, bufs, n_bufs, opts);
    if (s != GAO_OK) return s;
    if (!bytes_out) return fail(GAO_EINVAL, "bytes_out is null");
    if ((s = check_device(nullptr)) != GAO_OK) return s;
    gao_opts o{};
    if (opts) o = *opts;
    *bytes_out = plan(loops, n_loops, bufs, n_bufs, o).total;
    return GAO_OK;
}

extern "C" gao_status prog_create(const gao_loop* loops, int n_loops, const gao_buffer* bufs, int n_bufs,
                                  const gao_opts* opts, gao_prog** out) {
    if (!out) return fail(GAO_EINVAL, "out is null");
    *out = nullptr;
    gao_status s = validate(loops, n_loops, bufs, n_bufs, opts);
    if (s != GAO_OK) return s;
    int dev = 0;
    if ((s = check_device(&dev)) != GAO_OK) return s;
    gao_prog* p = new gao_prog();
    p->device = dev;
    if (opts) p->opts = *opts;
    if (p->opts.kchunk <= 0) p->opts.kchunk = default_kchunk(p->opts.gemm_prec);
    p->loops.assign(loops, loops + n_loops);
    for (int i = 0; i < n_loops; ++i) {
        p->verdict.push_back((int8_t)offload_verdict(loops[i]));
        if (p->verdict.back() == GAO_OFFLOAD_OK) p->gene_loop.push_back(i);
    }
    if (p->opts.fuse_chains == GAO_FUSE_GENE && p->gene_loop.size() >= 64) {
        delete p;
        return fail(GAO_EINVAL, "64 offloadable loops leave no gene bit for GAO_FUSE_GENE");
    }
    p->lay = plan(loops, n_loops, bufs, n_bufs, p->opts);
    auto bail = [&](gao_status st) {
        free_prog(p);
        return st;
    };
    if (p->opts.stream) {
        p->st = (cudaStream_t)p->opts.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
        p->own_stream = true;
    }
    if (p->opts.dev_arena) {
        if (p->opts.dev_arena_bytes < p->lay.total)
            return bail(fail(GAO_ENOMEM, "dev_arena holds " + std::to_string(p->opts.dev_arena_bytes) +
                                             " bytes; the program needs " + std::to_string(p->lay.total)));
        if (((uintptr_t)p->opts.dev_arena) & 1023u) return bail(fail(GAO_EINVAL, "dev_arena must be 1024-byte aligned"));
        p->arena = (char*)p->opts.dev_arena;
    } else {
        // cudaMalloc guarantees 256-byte alignment only; the layout's offsets assume 1024
        cudaError_t e = cudaMalloc((void**)&p->arena_raw, p->lay.total + 1024);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(arena)"));
        p->own_arena = true;
        p->arena = p->arena_raw + ((1024u - ((uintptr_t)p->arena_raw & 1023u)) & 1023u);
    }
    p->bufs.resize((size_t)n_bufs);
    for (int b = 0; b < n_bufs; ++b) {
        BufState& B = p->bufs[(size_t)b];
        B.d = bufs[b];
        B.bytes = (size_t)bufs[b].rows * (size_t)bufs[b].cols * elem_size(bufs[b].dtype);
        B.dev = p->arena + p->lay.buf_off[(size_t)b];
        cudaError_t e = cudaMallocHost(&B.own_host, std::max<size_t>(B.bytes, 16));
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocHost(buffer mirror)"));
        memset(B.own_host, 0, std::max<size_t>(B.bytes, 16));
        B.host = B.own_host;
    }
    cudaError_t e = cudaMallocHost((void**)&p->h_err, 16);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocHost(err)"));
    *p->h_err = 0;
    // zero the scratch words the kernels expect zeroed (error word, reduction counter)
    e = cudaMemsetAsync(p->arena + p->lay.err_off, 0, p->lay.rowexp_off - p->lay.err_off, p->st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemsetAsync(scratch)"));
    e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamSynchronize"));
    p->ev.assign((size_t)n_loops * 6, nullptr);
    for (auto& ev : p->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    e = cudaStreamCreateWithFlags(&p->cst, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate(copy stream)"));
    p->pipe_ev.assign(1 + 2 * kMaxRowBlocks + kMaxColParts, nullptr);
    for (auto& ev : p->pipe_ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    e = cudaStreamCreateWithFlags(&p->ost, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate(device-to-host stream)"));
    p->out_ev.assign(1 + kMaxRowBlocks, nullptr);
    for (auto& ev : p->out_ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    e = cudaStreamCreateWithFlags(&p->st2, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate(second compute stream)"));
    p->cmp_ev.assign(3, nullptr);
    for (auto& ev : p->cmp_ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    }
    p->ev_used.assign((size_t)n_loops, 0);
    p->stats.assign((size_t)n_loops, gao_loop_stat{});
    *out = p;
    return GAO_OK;
}

extern "C" gao_status prog_set_input(gao_prog* p, int buf, const void* host_src, uint64_t bytes) {
    if (!p || !host_src) return fail(GAO_EINVAL, "null argument");
    if (buf < 0 || buf >= (int)p->bufs.size()) return fail(GAO_EINVAL, "no such buffer");
    BufState& B = p->bufs[(size_t)buf];
    if (B.d.role != GAO_BUF_INPUT) return fail(GAO_EINVAL, "buffer is not an INPUT buffer");
    if (bytes != B.bytes)
        return fail(GAO_EINVAL, "buffer holds " + std::to_string(B.bytes) + " bytes, got " + std::to_string(bytes));
    cudaError_t e = cudaStreamSynchronize(p->st);  // no copy may still be reading the mirror
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    memcpy(B.host, host_src, B.bytes);
    B.input_set = true;
    p->cache.clear();  // new data: earlier times no longer describe this program
    return GAO_OK;
}

extern "C" gao_status prog_bind_host(gao_prog* p, int buf, void* host, uint64_t bytes) {
    if (!p) return fail(GAO_EINVAL, "program is null");
    if (buf < 0 || buf >= (int)p->bufs.size()) return fail(GAO_EINVAL, "no such buffer");
    BufState& B = p->bufs[(size_t)buf];
    if (host && bytes != B.bytes)
        return fail(GAO_EINVAL, "buffer holds " + std::to_string(B.bytes) + " bytes, got " + std::to_string(bytes));
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // no queued copy may still use the memory being replaced
    if ((e = cudaStreamSynchronize(p->st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (p->cst && (e = cudaStreamSynchronize(p->cst)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (p->ost && (e = cudaStreamSynchronize(p->ost)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (B.registered) {
        cudaHostUnregister(B.host);
        B.registered = false;
    }
    if (!host) {
        B.host = B.own_host;  // back to the library's mirror (its contents are stale)
        B.vh = false;
        if (B.d.role == GAO_BUF_INPUT) B.input_set = false;
    } else {
        cudaPointerAttributes a{};
        e = cudaPointerGetAttributes(&a, host);
        if (e != cudaSuccess) cudaGetLastError();
        bool pinned = e == cudaSuccess && a.type == cudaMemoryTypeHost;
        if (!pinned && B.bytes) {
            e = cudaHostRegister(host, B.bytes, cudaHostRegisterDefault);
            if (e != cudaSuccess) {
                B.host = B.own_host;
                return cuda_fail(e, "cudaHostRegister(bound buffer)");
            }
            B.registered = true;
        }
        B.host = host;
        if (B.d.role == GAO_BUF_INPUT) B.input_set = true;
        B.vh = B.d.role == GAO_BUF_INPUT;
    }
    drop_graphs(p);   // captured copies name the old host address
    p->cache.clear(); // new input data: earlier times no longer describe this program
    return GAO_OK;
}

namespace gao {

thread_local bool g_capturing = false;
thread_local bool g_no_times = false;

void drop_graphs(gao_prog* p) {
    for (auto& kv : p->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    p->graphs.clear();
}

int offload_verdict(const gao_loop& L) {
    if (L.flags & GAO_LOOP_EXTERNAL_CALL) return GAO_OFFLOAD_EXTERNAL_CALL;
    if (L.kind == GAO_LOOP_RECURRENCE) return GAO_OFFLOAD_DEPENDENCE;
    if (L.kind == GAO_LOOP_FIND) return GAO_OFFLOAD_EARLY_EXIT;
    return GAO_OFFLOAD_OK;
}

uint64_t loop_mask_of(const gao_prog* p, uint64_t gene) {
    uint64_t m = 0;
    for (size_t k = 0; k < p->gene_loop.size(); ++k)
        if ((gene >> k) & 1) m |= 1ULL << p->gene_loop[k];
    return m;
}


// A buffer an INIT loop formed only as a GEMM's bfloat16 planes: its binary32 values, formed
// now on the device by that INIT slot alone (the same counter hash, the same row exponents).
gao_status materialize(RunCtx& R, int b) {
    gao_prog* p = R.p;
    BufState& B = p->bufs[(size_t)b];
    const gao_loop& L = p->loops[(size_t)B.gen_loop];
    const int rs = (int)((L.flags >> B.gen_slot) & 1);
    InitSet set{};
    set.o[0] = InitOut{(float*)B.dev, B.d.rows, B.d.cols, (uint32_t)b, rs};
    set.n = 1;
    set.seed = p->opts.seed;
    set.rowexp = rs ? (const int8_t*)(p->arena + p->lay.rowexp_off) : nullptr;
    if (rs) GAO_CUDA_TRY(launch_row_exponents((int8_t*)set.rowexp, B.d.rows, p->opts.seed, R.st));
    if (B.d.rows * B.d.cols > 0) GAO_CUDA_TRY(launch_init_set(set, R.st));
    B.vd = true;
    B.gen_loop = B.gen_slot = B.gen_for = -1;
    return GAO_OK;
}

// Make buffer b valid on the requested side, issuing a copy on the stream if needed.
gao_status make_valid(RunCtx& R, int b, bool on_gpu, gao_loop_stat& stat) {
    BufState& B = R.p->bufs[(size_t)b];
    if (!B.vd && !B.vh && B.gen_loop >= 0) {
        gao_status s = materialize(R, b);
        if (s != GAO_OK) return s;
    }
    if (on_gpu) {
        if (B.vd) return GAO_OK;
        if (!B.vh) return fail(GAO_EINVAL, "buffer " + std::to_string(b) + " holds no data");
        if (B.bytes) GAO_CUDA_TRY(cudaMemcpyAsync(B.dev, B.host, B.bytes, cudaMemcpyHostToDevice, R.st));
        stat.h2d_bytes += B.bytes;
        B.vd = true;
    } else {
        if (B.vh) return GAO_OK;
        if (!B.vd) return fail(GAO_EINVAL, "buffer " + std::to_string(b) + " holds no data");
        if (B.bytes) GAO_CUDA_TRY(cudaMemcpyAsync(B.host, B.dev, B.bytes, cudaMemcpyDeviceToHost, R.st));
        stat.d2h_bytes += B.bytes;
        B.vh = true;
    }
    return GAO_OK;
}

std::vector<int> loop_inputs(const gao_loop& L) {
    std::vector<int> v;
    if (L.kind == GAO_LOOP_INIT) return v;
    for (int t = 0; t < GAO_MAX_IO; ++t)
        if (L.ins[t] >= 0) {
            if (L.kind == GAO_LOOP_GEMM && t == 2 && L.beta == 0.0) continue;
            v.push_back(L.ins[t]);
        }
    return v;
}

std::vector<int> loop_outputs(const gao_loop& L) {
    std::vector<int> v;
    const int n = L.kind == GAO_LOOP_INIT ? GAO_MAX_IO : 1;
    for (int t = 0; t < n; ++t)
        if (L.outs[t] >= 0) v.push_back(L.outs[t]);
    return v;
}

gao_status run_gpu_loop(RunCtx& R, int li) {
    gao_prog* p = R.p;
    const gao_loop& L = p->loops[(size_t)li];
    cudaStream_t st = R.st;
    auto dptr = [&](int b) { return (float*)p->bufs[(size_t)b].dev; };
    auto shp = [&](int b) -> const gao_buffer& { return p->bufs[(size_t)b].d; };
    char* a = p->arena;
    int* d_err = (int*)(a + p->lay.err_off);
    ReduceScratch rs{(double*)(a + p->lay.partial_off), (unsigned*)(a + p->lay.counter_off)};
    cudaError_t e = cudaSuccess;
    int& nl = p->stats[(size_t)li].launches;
    switch (L.kind) {
        case GAO_LOOP_INIT: {
            // all outputs in one launch; the row exponents (a function of the row) once, for
            // the largest row-scaled output
            InitSet set{};
            int64_t rx_rows = 0, total = 0;
            for (int t = 0; t < GAO_MAX_IO; ++t) {
                const int b = L.outs[t];
                if (b < 0) continue;
                const int rs = (int)((L.flags >> t) & 1);
                set.o[set.n++] = InitOut{dptr(b), shp(b).rows, shp(b).cols, (uint32_t)b, rs};
                if (rs) rx_rows = std::max(rx_rows, shp(b).rows);
                total += shp(b).rows * shp(b).cols;
            }
            set.seed = p->opts.seed;
            set.rowexp = rx_rows > 0 ? (const int8_t*)(a + p->lay.rowexp_off) : nullptr;
            if (rx_rows > 0) {
                e = launch_row_exponents((int8_t*)set.rowexp, rx_rows, p->opts.seed, st);
                nl += 1;
            }
            if (e == cudaSuccess && total > 0) {
                e = launch_init_set(set, st);
                nl += 1;
            }
            break;
        }
        case GAO_LOOP_GEMM: {
            const gao_buffer &A = shp(L.ins[0]), &B = shp(L.ins[1]);
            const float* c0 = L.ins[2] >= 0 ? dptr(L.ins[2]) : nullptr;
            const float beta = c0 ? (float)L.beta : 0.0f;
            const int prec = p->opts.gemm_prec;
            cudaEvent_t k0 = R.events ? p->ev[(size_t)li * 6 + 4] : nullptr;
            cudaEvent_t k1 = R.events ? p->ev[(size_t)li * 6 + 5] : nullptr;
            if (prec == GAO_GEMM_FP32_SIMT) {
                if (k0) GAO_CUDA_TRY(record_timing(k0, st));
                e = launch_gemm_simt(dptr(L.outs[0]), dptr(L.ins[0]), dptr(L.ins[1]), c0 ? c0 : dptr(L.outs[0]),
                                     A.rows, B.cols, A.cols, (float)L.alpha, beta, p->opts.kchunk, st);
                nl += A.rows * B.cols > 0;
                if (e == cudaSuccess && k1) GAO_CUDA_TRY(record_timing(k1, st));
            } else {
                std::string why;
                TcEvents tev{k0, k1, 0};
                // operands an INIT loop formed straight into this GEMM's planes
                const unsigned ready = (p->bufs[(size_t)L.ins[0]].gen_for == li ? 1u : 0u) |
                                       (p->bufs[(size_t)L.ins[1]].gen_for == li ? 2u : 0u);
                e = launch_gemm_tc(prec, dptr(L.outs[0]), dptr(L.ins[0]), dptr(L.ins[1]), c0 ? c0 : dptr(L.outs[0]),
                                   A.rows, B.cols, A.cols, (float)L.alpha, beta, p->opts.kchunk, p->opts.tile_cfg,
                                   a + p->lay.tc_off, p->lay.tc_bytes, d_err, st, tev, &why, nullptr, nullptr,
                                   ready);
                if (e != cudaSuccess && !why.empty()) return fail(GAO_EINVAL, "tensor-core GEMM: " + why);
                nl += tev.launches;
            }
            p->ev_used[(size_t)li] |= 4;
            break;
        }
        case GAO_LOOP_AXPY: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_axpy(dptr(L.outs[0]), dptr(L.ins[0]), (float)L.alpha, dptr(L.ins[1]), X.rows * X.cols, st);
            nl += X.rows * X.cols > 0;
            break;
        }
        case GAO_LOOP_TRANSPOSE: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_transpose(dptr(L.outs[0]), dptr(L.ins[0]), X.rows, X.cols, st);
            nl += X.rows * X.cols > 0;
            break;
        }
        case GAO_LOOP_ROWSUM: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_rowsum(dptr(L.outs[0]), dptr(L.ins[0]), X.rows, X.cols, st);
            nl += X.rows > 0 && X.cols > 0;
            break;
        }
        case GAO_LOOP_FROBENIUS: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_frobenius((double*)p->bufs[(size_t)L.outs[0]].dev, dptr(L.ins[0]), X.rows * X.cols, rs, st);
            nl += 1;
            break;
        }
        case GAO_LOOP_SUM: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_sum((double*)p->bufs[(size_t)L.outs[0]].dev, dptr(L.ins[0]), X.rows * X.cols, rs, st);
            nl += 1;
            break;
        }
        case GAO_LOOP_RELU: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_relu(dptr(L.outs[0]), dptr(L.ins[0]), X.rows * X.cols, st);
            nl += X.rows * X.cols > 0;
            break;
        }
        case GAO_LOOP_SQUARE: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_square(dptr(L.outs[0]), dptr(L.ins[0]), X.rows * X.cols, st);
            nl += X.rows * X.cols > 0;
            break;
        }
        case GAO_LOOP_COLMAX: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_colmax(dptr(L.outs[0]), dptr(L.ins[0]), X.rows, X.cols, (uint32_t*)(a + p->lay.keys_off), st);
            nl += (X.cols > 0) * (1 + (X.rows > 0));
            break;
        }
        case GAO_LOOP_STENCIL3: {
            const gao_buffer& X = shp(L.ins[0]);
            e = launch_stencil3(dptr(L.outs[0]), dptr(L.ins[0]), X.rows, X.cols,
                                (int)(L.flags & ~GAO_LOOP_EXTERNAL_CALL), st);
            nl += X.rows * X.cols > 0;
            break;
        }
        case GAO_LOOP_RECURRENCE:
        case GAO_LOOP_FIND:
            return fail(GAO_EINVAL, "loop " + std::to_string(li) + " is not offloadable");
        default:
            return fail(GAO_EINVAL, "unknown loop kind");
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return GAO_OK;
}

gao_status run_cpu_loop(RunCtx& R, int li) {
    gao_prog* p = R.p;
    const gao_loop& L = p->loops[(size_t)li];
    auto hptr = [&](int b) { return (float*)p->bufs[(size_t)b].host; };
    auto shp = [&](int b) -> const gao_buffer& { return p->bufs[(size_t)b].d; };
    CpuCtx& c = R.cpu;
    switch (L.kind) {
        case GAO_LOOP_INIT:
            for (int t = 0; t < GAO_MAX_IO; ++t) {
                const int b = L.outs[t];
                if (b < 0) continue;
                cpu_init(hptr(b), shp(b).rows, shp(b).cols, p->opts.seed, (uint32_t)b, ((L.flags >> t) & 1) != 0, c);
            }
            break;
        case GAO_LOOP_GEMM: {
            const gao_buffer &A = shp(L.ins[0]), &B = shp(L.ins[1]);
            const float* c0 = L.ins[2] >= 0 ? hptr(L.ins[2]) : nullptr;
            const int kc = p->opts.gemm_prec == GAO_GEMM_FP32_SIMT ? p->opts.kchunk : 256;
            cpu_gemm(hptr(L.outs[0]), hptr(L.ins[0]), hptr(L.ins[1]), c0 ? c0 : hptr(L.outs[0]), A.rows, B.cols,
                     A.cols, (float)L.alpha, c0 ? (float)L.beta : 0.0f, kc, c);
            break;
        }
        case GAO_LOOP_AXPY: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_axpy(hptr(L.outs[0]), hptr(L.ins[0]), (float)L.alpha, hptr(L.ins[1]), X.rows * X.cols, c);
            break;
        }
        case GAO_LOOP_TRANSPOSE: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_transpose(hptr(L.outs[0]), hptr(L.ins[0]), X.rows, X.cols, c);
            break;
        }
        case GAO_LOOP_ROWSUM: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_rowsum(hptr(L.outs[0]), hptr(L.ins[0]), X.rows, X.cols, c);
            break;
        }
        case GAO_LOOP_FROBENIUS: {
            const gao_buffer& X = shp(L.ins[0]);
            *(double*)p->bufs[(size_t)L.outs[0]].host = cpu_frobenius(hptr(L.ins[0]), X.rows * X.cols, c);
            break;
        }
        case GAO_LOOP_SUM: {
            const gao_buffer& X = shp(L.ins[0]);
            *(double*)p->bufs[(size_t)L.outs[0]].host = cpu_sum(hptr(L.ins[0]), X.rows * X.cols, c);
            break;
        }
        case GAO_LOOP_RELU: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_relu(hptr(L.outs[0]), hptr(L.ins[0]), X.rows * X.cols, c);
            break;
        }
        case GAO_LOOP_SQUARE: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_square(hptr(L.outs[0]), hptr(L.ins[0]), X.rows * X.cols, c);
            break;
        }
        case GAO_LOOP_COLMAX: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_colmax(hptr(L.outs[0]), hptr(L.ins[0]), X.rows, X.cols, c);
            break;
        }
        case GAO_LOOP_STENCIL3: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_stencil3(hptr(L.outs[0]), hptr(L.ins[0]), X.rows, X.cols, (int)(L.flags & ~GAO_LOOP_EXTERNAL_CALL), c);
            break;
        }
        case GAO_LOOP_RECURRENCE: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_recurrence(hptr(L.outs[0]), hptr(L.ins[0]), X.rows, X.cols, (float)L.alpha, c);
            break;
        }
        case GAO_LOOP_FIND: {
            const gao_buffer& X = shp(L.ins[0]);
            cpu_find((double*)p->bufs[(size_t)L.outs[0]].host, hptr(L.ins[0]), X.rows, X.cols, (float)L.alpha, c);
            break;
        }
        default:
            return fail(GAO_EINVAL, "unknown loop kind");
    }
    return GAO_OK;
}

}  // namespace gao

namespace {

// A gradient chain the stencil loop li can run as one pass when the gene puts it all on
// the GPU: STENCIL3 (X -> g1), STENCIL3 (X -> g2), SQUARE of g1 and of g2 (either order),
// AXPY of the two squares (either order) in loops li..li+4.  The image is read once; an
// intermediate that is neither an OUTPUT buffer nor read by a later loop is not written.
struct GradChain {
    int x = -1, g1 = -1, g2 = -1, s1 = -1, s2 = -1, m = -1;
    int p1 = 0, p2 = 0;
    float alpha = 1.0f;
    bool swap = false;
    bool live[4] = {true, true, true, true};  // g1, g2, s1, s2
    // with `reductions`: a SUM and / or a COLMAX loop of m right after the chain (li + 5 ..
    // li + 6, on the GPU), formed in the same pass
    int sum_loop = -1, colmax_loop = -1;
    bool m_live = true;  // m itself is written: an OUTPUT, or read after the pass
    // a stencil loop `pre` (preset p0) that forms x from the raw image `raw`, in the same pass
    // (find_edge_chain); x is then written only when x_live
    int pre = -1, raw = -1, p0 = 0;
    bool x_live = true;
};

bool find_grad_chain(const gao_prog* p, int li, uint64_t mask, bool fuse, GradChain* gc, bool reductions = false) {
    if (!fuse || p->opts.transfer_mode != GAO_TRANSFER_RESIDENT) return false;
    const int n = (int)p->loops.size();
    if (li + 4 >= n) return false;
    for (int k = li; k <= li + 4; ++k)
        if (!((mask >> k) & 1)) return false;
    const gao_loop* L = &p->loops[(size_t)li];
    if (L[0].kind != GAO_LOOP_STENCIL3 || L[1].kind != GAO_LOOP_STENCIL3 || L[2].kind != GAO_LOOP_SQUARE ||
        L[3].kind != GAO_LOOP_SQUARE || L[4].kind != GAO_LOOP_AXPY)
        return false;
    GradChain c;
    c.x = L[0].ins[0];
    if (L[1].ins[0] != c.x) return false;
    c.g1 = L[0].outs[0];
    c.g2 = L[1].outs[0];
    c.p1 = (int)(L[0].flags & ~GAO_LOOP_EXTERNAL_CALL);
    c.p2 = (int)(L[1].flags & ~GAO_LOOP_EXTERNAL_CALL);
    if (L[2].ins[0] == c.g1 && L[3].ins[0] == c.g2) {
        c.s1 = L[2].outs[0];
        c.s2 = L[3].outs[0];
    } else if (L[2].ins[0] == c.g2 && L[3].ins[0] == c.g1) {
        c.s1 = L[3].outs[0];
        c.s2 = L[2].outs[0];
    } else {
        return false;
    }
    if (L[4].ins[0] == c.s1 && L[4].ins[1] == c.s2) c.swap = false;
    else if (L[4].ins[0] == c.s2 && L[4].ins[1] == c.s1) c.swap = true;
    else return false;
    c.m = L[4].outs[0];
    c.alpha = (float)L[4].alpha;
    const int bufs[6] = {c.x, c.g1, c.g2, c.s1, c.s2, c.m};
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j)
            if (bufs[i] == bufs[j]) return false;
    const int inter[4] = {c.g1, c.g2, c.s1, c.s2};
    for (int t = 0; t < 4; ++t) {
        bool live = p->bufs[(size_t)inter[t]].d.role == GAO_BUF_OUTPUT;
        for (int j = li + 5; j < n && !live; ++j)
            for (int b : loop_inputs(p->loops[(size_t)j]))
                if (b == inter[t]) live = true;
        c.live[t] = live;
    }
    if (reductions) {
        for (int j = li + 5; j <= li + 6 && j < n && ((mask >> j) & 1); ++j) {
            const gao_loop& R = p->loops[(size_t)j];
            if (R.ins[0] != c.m || R.outs[0] < 0 || R.outs[0] == c.m) break;
            if (R.kind == GAO_LOOP_SUM && c.sum_loop < 0) c.sum_loop = j;
            else if (R.kind == GAO_LOOP_COLMAX && c.colmax_loop < 0) c.colmax_loop = j;
            else break;
        }
    }
    // m is written only if it is an OUTPUT or a loop after the pass (its fused reductions
    // included in the pass) reads it
    const int last = std::max(li + 4, std::max(c.sum_loop, c.colmax_loop));
    c.m_live = p->bufs[(size_t)c.m].d.role == GAO_BUF_OUTPUT;
    for (int j = last + 1; j < n && !c.m_live; ++j)
        for (int b : loop_inputs(p->loops[(size_t)j]))
            if (b == c.m) c.m_live = true;
    if (c.sum_loop < 0 && c.colmax_loop < 0) c.m_live = true;  // the pass writes at least m
    *gc = c;
    return true;
}

// A GPU STENCIL3 loop li (the blur) whose output x starts a gradient chain (with its
// reductions): the blur joins the chain's pass, which then reads the raw image instead of x.
// x is written only when it is an OUTPUT or a loop after the chain's two stencils reads it.
bool find_edge_chain(const gao_prog* p, int li, uint64_t mask, bool fuse, GradChain* gc) {
    const int n = (int)p->loops.size();
    if (li + 1 >= n || !((mask >> li) & 1)) return false;
    const gao_loop& L = p->loops[(size_t)li];
    if (L.kind != GAO_LOOP_STENCIL3 || L.ins[0] == L.outs[0]) return false;
    GradChain c;
    if (!find_grad_chain(p, li + 1, mask, fuse, &c, true) || c.x != L.outs[0]) return false;
    const int raw = L.ins[0];
    const int made[6] = {c.x, c.g1, c.g2, c.s1, c.s2, c.m};
    for (int b : made)
        if (b == raw) return false;
    for (int j : {c.sum_loop, c.colmax_loop})
        if (j >= 0 && p->loops[(size_t)j].outs[0] == raw) return false;
    c.pre = li;
    c.raw = raw;
    c.p0 = (int)(L.flags & ~GAO_LOOP_EXTERNAL_CALL);
    c.x_live = p->bufs[(size_t)c.x].d.role == GAO_BUF_OUTPUT;
    for (int j = li + 3; j < n && !c.x_live; ++j)
        for (int b : loop_inputs(p->loops[(size_t)j]))
            if (b == c.x) c.x_live = true;
    *gc = c;
    return true;
}

// Where the chain's fused sum and column maxima go: the SUM loop's and COLMAX loop's outputs,
// the block partials and the column keys in the arena.
GradReduce grad_reduce_for(const gao_prog* p, const GradChain& gch) {
    GradReduce red{};
    if (gch.sum_loop >= 0) {
        red.sum_out = (double*)p->bufs[(size_t)p->loops[(size_t)gch.sum_loop].outs[0]].dev;
        red.part = (double*)(p->arena + p->lay.chainpart_off);
        red.part_cap = (int64_t)(p->lay.chainpart_bytes / 8);
    }
    if (gch.colmax_loop >= 0) {
        red.colmax_out = (float*)p->bufs[(size_t)p->loops[(size_t)gch.colmax_loop].outs[0]].dev;
        red.keys = (uint32_t*)(p->arena + p->lay.keys_off);
    }
    return red;
}

// Residency after the chain starting at loop first ran as one pass (with its reductions, and
// with the blur before it when gch.pre >= 0): what it wrote is valid on the device only, an
// unwritten intermediate holds nothing, and its loops are marked as run.
void grad_chain_done(gao_prog* p, const GradChain& gch, int first, uint64_t* fused) {
    const int outs[5] = {gch.g1, gch.g2, gch.s1, gch.s2, gch.m};
    for (int t = 0; t < 5; ++t) {
        BufState& B = p->bufs[(size_t)outs[t]];
        B.vh = false;
        B.vd = t == 4 ? gch.m_live : gch.live[t];
    }
    for (int j = first + 1; j <= first + 4; ++j) *fused |= 1ULL << j;
    if (gch.pre >= 0) {  // the blur ran in the pass too: the chain's first loop with it
        *fused |= 1ULL << first;
        BufState& X = p->bufs[(size_t)gch.x];
        X.vh = false;
        X.vd = gch.x_live;
    }
    for (int j : {gch.sum_loop, gch.colmax_loop}) {
        if (j < 0) continue;
        *fused |= 1ULL << j;
        BufState& B = p->bufs[(size_t)p->loops[(size_t)j].outs[0]];
        B.vh = false;
        B.vd = true;
    }
}

// A linear chain of element-wise loops starting at loop li that the gene puts on the GPU:
// RELU, SQUARE or AXPY loops over one shape, each after the first reading the previous
// loop's output and at most one buffer the chain did not produce.  Run as one pass, the
// intermediates stay in registers; an output is written only when it is an OUTPUT buffer
// or a later loop reads it.
struct EwPlan {
    int n = 0;
    int loops[kMaxChainOps];
};

bool is_elementwise(int kind) { return kind == GAO_LOOP_RELU || kind == GAO_LOOP_SQUARE || kind == GAO_LOOP_AXPY; }

bool find_ew_chain(const gao_prog* p, int li, uint64_t mask, bool fuse, EwPlan* plan) {
    if (!fuse || p->opts.transfer_mode != GAO_TRANSFER_RESIDENT) return false;
    const int n = (int)p->loops.size();
    const gao_loop& L0 = p->loops[(size_t)li];
    if (!is_elementwise(L0.kind) || !((mask >> li) & 1)) return false;
    const gao_buffer& shape = p->bufs[(size_t)L0.outs[0]].d;
    EwPlan e;
    e.loops[e.n++] = li;
    int cur = L0.outs[0];
    std::vector<int> produced{cur};
    for (int j = li + 1; j < n && e.n < kMaxChainOps; ++j) {
        const gao_loop& L = p->loops[(size_t)j];
        if (!((mask >> j) & 1) || !is_elementwise(L.kind)) break;
        const gao_buffer& o = p->bufs[(size_t)L.outs[0]].d;
        if (o.rows != shape.rows || o.cols != shape.cols) break;
        const std::vector<int> ins = loop_inputs(L);
        bool uses_cur = false, nonlinear = false;
        for (int b : ins) {
            if (b == cur) uses_cur = true;
            else if (std::find(produced.begin(), produced.end(), b) != produced.end()) nonlinear = true;
        }
        if (!uses_cur || nonlinear) break;
        e.loops[e.n++] = j;
        cur = L.outs[0];
        produced.push_back(cur);
    }
    if (e.n < 2) return false;
    *plan = e;
    return true;
}

// A chain the GEMM loop li can run as one pass when the gene puts it all on the GPU:
// GEMM (C) -> AXPY (D = C + a X) -> TRANSPOSE (E = D^T) [-> FROBENIUS of E, later, with no
// loop in between writing E].  The buffers must be distinct so that the epilogue's
// writes cannot race with its reads.
}  // namespace

bool gao::find_chain(const gao_prog* p, int li, uint64_t mask, bool fuse, Chain* ch) {
    if (!fuse || p->opts.transfer_mode != GAO_TRANSFER_RESIDENT) return false;
    const int prec = p->opts.gemm_prec;
    if (prec != GAO_GEMM_BF16 && prec != GAO_GEMM_BF16X3 && prec != GAO_GEMM_BF16X6) return false;
    const int n = (int)p->loops.size();
    if (li + 2 >= n) return false;
    for (int k = li; k <= li + 2; ++k)
        if (!((mask >> k) & 1)) return false;
    const gao_loop &G = p->loops[(size_t)li], &X = p->loops[(size_t)li + 1], &T = p->loops[(size_t)li + 2];
    if (G.kind != GAO_LOOP_GEMM || X.kind != GAO_LOOP_AXPY || T.kind != GAO_LOOP_TRANSPOSE) return false;
    const int Cb = G.outs[0], Xb = X.ins[1], Db = X.outs[0], Eb = T.outs[0];
    if (X.ins[0] != Cb || T.ins[0] != Db) return false;
    if (p->bufs[(size_t)G.ins[0]].d.cols <= 0) return false;  // K = 0
    const int gin[3] = {G.ins[0], G.ins[1], G.ins[2]};
    if (Xb == Cb || Db == Cb || Db == Xb || Eb == Cb || Eb == Xb || Eb == Db) return false;
    for (int g : gin)
        if (g >= 0 && (g == Db || g == Eb)) return false;
    ch->axpy = li + 1;
    ch->transpose = li + 2;
    ch->rowsum = ch->frob = -1;
    // later GPU loops that only reduce E (row sums, norm) join the chain when nothing between
    // rewrites E or touches their outputs: their results are formed at the GEMM's place
    const int chain_bufs[] = {gin[0], gin[1], gin[2], Cb, Xb, Db, Eb};
    auto joins = [&](int j) {
        const gao_loop& L = p->loops[(size_t)j];
        const int out = L.outs[0];
        for (int b : chain_bufs)
            if (b == out) return false;
        for (int k = li + 3; k < j; ++k) {
            const gao_loop& Q = p->loops[(size_t)k];
            for (int b : loop_inputs(Q))
                if (b == out) return false;
            for (int b : loop_outputs(Q))
                if (b == out) return false;
        }
        return true;
    };
    for (int j = li + 3; j < n; ++j) {
        const gao_loop& L = p->loops[(size_t)j];
        if (L.ins[0] == Eb && ((mask >> j) & 1)) {
            if (L.kind == GAO_LOOP_ROWSUM && ch->rowsum < 0 && joins(j)) ch->rowsum = j;
            if (L.kind == GAO_LOOP_FROBENIUS && ch->frob < 0 && joins(j)) ch->frob = j;
        }
        bool writes_e = false;
        for (int o : loop_outputs(L)) writes_e |= (o == Eb);
        if (writes_e || (ch->rowsum >= 0 && ch->frob >= 0)) break;
    }
    return true;
}

namespace {

gao_status run_gpu_chain(RunCtx& R, int li, const Chain& ch) {
    gao_prog* p = R.p;
    const gao_loop &G = p->loops[(size_t)li], &X = p->loops[(size_t)ch.axpy], &T = p->loops[(size_t)ch.transpose];
    auto dptr = [&](int b) { return (float*)p->bufs[(size_t)b].dev; };
    const gao_buffer &A = p->bufs[(size_t)G.ins[0]].d, &B = p->bufs[(size_t)G.ins[1]].d;
    const float* c0 = G.ins[2] >= 0 ? dptr(G.ins[2]) : dptr(G.outs[0]);
    const TcFuse fz{dptr(X.ins[1]), dptr(X.outs[0]), dptr(T.outs[0]),
                    ch.frob >= 0 ? (double*)p->bufs[(size_t)p->loops[(size_t)ch.frob].outs[0]].dev : nullptr,
                    (float)X.alpha, 0, ch.rowsum >= 0 ? dptr(p->loops[(size_t)ch.rowsum].outs[0]) : nullptr};
    TcEvents tev{R.events ? p->ev[(size_t)li * 6 + 4] : nullptr, R.events ? p->ev[(size_t)li * 6 + 5] : nullptr, 0};
    std::string why;
    cudaError_t e = launch_gemm_tc(p->opts.gemm_prec, dptr(G.outs[0]), dptr(G.ins[0]), dptr(G.ins[1]), c0, A.rows,
                                   B.cols, A.cols, (float)G.alpha, G.ins[2] >= 0 ? (float)G.beta : 0.0f,
                                   p->opts.kchunk, p->opts.tile_cfg, p->arena + p->lay.tc_off, p->lay.tc_bytes,
                                   (int*)(p->arena + p->lay.err_off), R.st, tev, &why, &fz);
    if (e != cudaSuccess) return why.empty() ? cuda_fail(e, "fused chain launch") : fail(GAO_EINVAL, why);
    p->stats[(size_t)li].launches += tev.launches;
    p->ev_used[(size_t)li] |= 4;
    return GAO_OK;
}

// Copy/compute overlap for a GPU GEMM loop whose A has to come from the host (the
// host-to-device link, measured at ~210 GB/s, is 30x slower than HBM): B (without a fused
// chain: its first column range, then A's first rows, then its other columns), then A and
// C0 in row blocks travel on a copy stream, and each row block's split and tensor-core GEMM
// start as soon as its rows have landed, while the next block is still on the link.  Row
// blocks and column ranges give the same bits as one launch (every output is formed the
// same way); only the split precisions take this path.
int64_t pipeline_blocks(const gao_prog* p, const gao_loop& L) {
    const int prec = p->opts.gemm_prec;
    if (L.kind != GAO_LOOP_GEMM) return 0;
    if (prec != GAO_GEMM_BF16 && prec != GAO_GEMM_BF16X3 && prec != GAO_GEMM_BF16X6) return 0;
    if (L.ins[0] == L.ins[1] || L.ins[2] == L.ins[0] || L.ins[2] == L.ins[1]) return 0;
    const BufState& A = p->bufs[(size_t)L.ins[0]];
    const gao_buffer& B = p->bufs[(size_t)L.ins[1]].d;
    if (A.vd || A.gen_for >= 0 || A.bytes < kPipelineMinBytes || A.d.cols <= 0 || B.cols <= 0) return 0;
    const int64_t blocks = std::min<int64_t>(kMaxRowBlocks, A.d.rows / 256);
    return blocks >= 2 ? blocks : 0;
}

// With early_out (C an OUTPUT the run copies back at its end), each block's rows of C go back
// to the host on a third stream as soon as the block's GEMM is done, on the link's other
// direction while later blocks are still coming in; *c_on_host tells the caller that C's host
// copy is then valid.
gao_status run_gpu_gemm_pipelined(RunCtx& R, int li, int64_t blocks, const Chain* ch, bool early_out,
                                  bool* c_on_host) {
    gao_prog* p = R.p;
    const gao_loop& L = p->loops[(size_t)li];
    gao_loop_stat& S = p->stats[(size_t)li];
    BufState &A = p->bufs[(size_t)L.ins[0]], &B = p->bufs[(size_t)L.ins[1]];
    const bool use_c0 = L.ins[2] >= 0 && L.beta != 0.0;
    BufState* C0 = use_c0 ? &p->bufs[(size_t)L.ins[2]] : nullptr;
    BufState& C = p->bufs[(size_t)L.outs[0]];
    if (!A.vh || !(B.vd || B.vh) || (C0 && !(C0->vd || C0->vh)))
        return fail(GAO_EINVAL, "a GEMM input holds no data");
    const int64_t M = A.d.rows, K = A.d.cols, N = B.d.cols;
    const int64_t rows = ((M + blocks - 1) / blocks + 255) / 256 * 256;  // whole CTA-pair tiles
    cudaStream_t st = R.st, cs = p->cst;
    cudaEvent_t* ev = &p->ev[(size_t)li * 6];
    cudaEvent_t fork = p->pipe_ev[0], b_done = p->pipe_ev[1];
    GAO_CUDA_TRY(cudaEventRecord(fork, st));  // the copies overwrite device buffers: after earlier work
    GAO_CUDA_TRY(cudaStreamWaitEvent(cs, fork, 0));
    GAO_CUDA_TRY(record_timing(ev[0], cs));
    // Without a fused chain, the first row block runs as column ranges [cut[j], cut[j + 1]) of
    // whole 256-column tiles: the first starts once B's first columns and A's first rows have
    // landed, and each next one as its columns of B land behind them (range j > 0 on
    // pipe_ev[1 + 2 kMaxRowBlocks + j]).  Each output is formed as in one launch, so the bits
    // are the same.
    int nparts = 1;
    int64_t cut[kMaxColParts + 1] = {0, N};
    if (!ch && !B.vd && N >= 512) {
        nparts = 2;  // four ranges at n = 8192 measured no faster (5.75 against 5.64-5.72 ms per step)
        for (int j = 0; j <= nparts; ++j) cut[j] = j == nparts ? N : (j * N / nparts + 255) / 256 * 256;
        for (int j = 1; j <= nparts; ++j)
            if (cut[j] <= cut[j - 1]) return fail(GAO_EINVAL, "column ranges of the first row block");
    }
    auto part_ev = [&](int j) { return j == 0 ? b_done : p->pipe_ev[1 + 2 * (size_t)kMaxRowBlocks + (size_t)j]; };
    auto copy_b_cols = [&](int64_t c0, int64_t c1) -> gao_status {  // B's columns [c0, c1), every row
        GAO_CUDA_TRY(cudaMemcpy2DAsync(B.dev + (size_t)c0 * 4, (size_t)N * 4, (const char*)B.host + (size_t)c0 * 4,
                                       (size_t)N * 4, (size_t)(c1 - c0) * 4, (size_t)K, cudaMemcpyHostToDevice, cs));
        S.h2d_bytes += (uint64_t)(c1 - c0) * K * 4;
        return GAO_OK;
    };
    gao_status cst = GAO_OK;
    if (nparts > 1) {
        if ((cst = copy_b_cols(0, cut[1])) != GAO_OK) return cst;
    } else if (!B.vd) {
        GAO_CUDA_TRY(cudaMemcpyAsync(B.dev, B.host, B.bytes, cudaMemcpyHostToDevice, cs));
        S.h2d_bytes += B.bytes;
    }
    GAO_CUDA_TRY(cudaEventRecord(b_done, cs));
    const bool copy_c0 = C0 && !C0->vd;
    // Without a fused chain, beta C0 joins each block's rows after its GEMM: the GEMM forms
    // alpha AB as its epilogue rounds it and a pass adds fma(beta, C0, .), the epilogue's own
    // last step, so the bits are the same; C0's rows then travel after the next block's A rows
    // and no GEMM waits for them (C0's block k lands on pipe_ev[2 + kMaxRowBlocks + k]).  Not
    // when C0 is C itself (the GEMM would overwrite C0 before the pass reads it).
    const int nblocks = (int)((M + rows - 1) / rows);
    const bool late_c0 = C0 && !ch && (float)L.beta != 0.0f && nblocks >= 2 && L.ins[2] != L.outs[0];
    auto copy_c0_block = [&](int k) -> gao_status {
        const int64_t r0 = k * rows, r1 = std::min(M, r0 + rows);
        const size_t off_c = (size_t)r0 * N * 4, len_c = (size_t)(r1 - r0) * N * 4;
        GAO_CUDA_TRY(cudaMemcpyAsync(C0->dev + off_c, (char*)C0->host + off_c, len_c, cudaMemcpyHostToDevice, cs));
        S.h2d_bytes += len_c;
        return GAO_OK;
    };
    int nb = 0;
    for (int64_t r0 = 0; r0 < M; r0 += rows, ++nb) {
        const int64_t r1 = std::min(M, r0 + rows);
        const size_t off_a = (size_t)r0 * K * 4, len_a = (size_t)(r1 - r0) * K * 4;
        GAO_CUDA_TRY(cudaMemcpyAsync(A.dev + off_a, (char*)A.host + off_a, len_a, cudaMemcpyHostToDevice, cs));
        S.h2d_bytes += len_a;
        if (copy_c0 && !late_c0 && (cst = copy_c0_block(nb)) != GAO_OK) return cst;
        // the copy-time stamp goes before the copy stream's last event, so that everything on
        // it is joined back into the program's stream (a captured graph needs that)
        const bool last_copy = r1 == M && !(copy_c0 && late_c0) && !(nparts > 1 && nb == 0);
        if (last_copy) GAO_CUDA_TRY(record_timing(ev[1], cs));
        GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[2 + (size_t)nb], cs));
        if (nparts > 1 && nb == 0) {  // B's other columns, range by range, right behind A's first rows
            for (int j = 1; j < nparts; ++j) {
                if ((cst = copy_b_cols(cut[j], cut[j + 1])) != GAO_OK) return cst;
                if (j == nparts - 1 && r1 == M && !(copy_c0 && late_c0)) GAO_CUDA_TRY(record_timing(ev[1], cs));
                GAO_CUDA_TRY(cudaEventRecord(part_ev(j), cs));
            }
        }
        if (copy_c0 && late_c0 && nb >= 1) {  // the previous block's C0 rows, behind this block's A rows
            if ((cst = copy_c0_block(nb - 1)) != GAO_OK) return cst;
            if (nb == nblocks - 1) {
                if ((cst = copy_c0_block(nb)) != GAO_OK) return cst;
                GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[2 + kMaxRowBlocks + (size_t)nb - 1], cs));
                GAO_CUDA_TRY(record_timing(ev[1], cs));
                GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[2 + kMaxRowBlocks + (size_t)nb], cs));
            } else {
                GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[2 + kMaxRowBlocks + (size_t)nb - 1], cs));
            }
        }
    }
    GAO_CUDA_TRY(record_timing(ev[2], st));
    GAO_CUDA_TRY(cudaStreamWaitEvent(st, b_done, 0));
    const float beta = C0 ? (float)L.beta : 0.0f;
    // a fused chain: each block's epilogue also writes its rows of D = C + alpha2 X, its
    // columns of E = D^T and its norm partials; X is the GEMM's A (copied in the blocks) or
    // already on the device
    const gao_loop* XL = ch ? &p->loops[(size_t)ch->axpy] : nullptr;
    auto fdev = [&](int b) { return (float*)p->bufs[(size_t)b].dev; };
    // Without a fused chain the blocks are independent once B's planes are formed: odd blocks
    // run on a second stream, so that a block's GEMM takes up the SMs its predecessor's last
    // tiles leave idle and its A split runs beside that GEMM (each block's A planes have a
    // region of their own).  A fused chain's blocks share the norm's and row sums' partials
    // and stay on one stream.
    const bool alt = !ch && nb >= 2;
    cudaEvent_t fork2 = p->cmp_ev[0], planes = p->cmp_ev[1], join2 = p->cmp_ev[2];
    if (alt) {
        GAO_CUDA_TRY(cudaEventRecord(fork2, st));
        GAO_CUDA_TRY(cudaStreamWaitEvent(p->st2, fork2, 0));
    }
    int i = 0;
    for (int64_t r0 = 0; r0 < M; r0 += rows, ++i) {
        const int64_t r1 = std::min(M, r0 + rows);
        cudaStream_t sx = alt && (i & 1) ? p->st2 : st;
        GAO_CUDA_TRY(cudaStreamWaitEvent(sx, p->pipe_ev[2 + (size_t)i], 0));
        if (alt && i > 0) GAO_CUDA_TRY(cudaStreamWaitEvent(sx, planes, 0));
        TcPart part{M, i > 0, r0 / 128, i == nb - 1};
        TcEvents tev{i == 0 ? ev[4] : nullptr, i == nb - 1 ? ev[5] : nullptr, 0};
        if (alt && i == 0) tev.planes = planes;
        std::string why;
        if (i == 0 && nparts > 1) {  // the first block's column ranges but the last, as B's columns land
            for (int j = 0; j + 1 < nparts; ++j) {
                TcPart pj = part;
                pj.n_begin = cut[j];
                pj.n_end = cut[j + 1];
                pj.a_ready = j > 0;  // A's planes formed by the first range
                TcEvents lev{j == 0 ? ev[4] : nullptr, nullptr, 0};
                if (j > 0) GAO_CUDA_TRY(cudaStreamWaitEvent(st, part_ev(j), 0));
                const float* c0l = C0 && !late_c0 ? (const float*)C0->dev : (const float*)C.dev;
                cudaError_t e = launch_gemm_tc(p->opts.gemm_prec, (float*)C.dev, (const float*)A.dev,
                                               (const float*)B.dev, c0l, r1 - r0, N, K, (float)L.alpha,
                                               late_c0 ? 0.0f : beta, p->opts.kchunk, p->opts.tile_cfg,
                                               p->arena + p->lay.tc_off, p->lay.tc_bytes,
                                               (int*)(p->arena + p->lay.err_off), st, lev, &why, nullptr, &pj);
                if (e != cudaSuccess) return why.empty() ? cuda_fail(e, "row-block GEMM") : fail(GAO_EINVAL, why);
                S.launches += lev.launches;
            }
            GAO_CUDA_TRY(cudaStreamWaitEvent(st, part_ev(nparts - 1), 0));
            part.n_begin = cut[nparts - 1];
            part.a_ready = true;
            tev.k0 = nullptr;
        }
        float* c = (float*)C.dev + (size_t)r0 * N;
        const float* c0 = C0 && !late_c0 ? (const float*)C0->dev + (size_t)r0 * N : c;
        TcFuse fz{};
        if (ch) {
            const gao_loop& T = p->loops[(size_t)ch->transpose];
            fz.X = fdev(XL->ins[1]) + (size_t)r0 * N;
            fz.D = fdev(XL->outs[0]) + (size_t)r0 * N;
            fz.E = fdev(T.outs[0]) + r0;
            fz.frob_out = ch->frob >= 0 ? (double*)p->bufs[(size_t)p->loops[(size_t)ch->frob].outs[0]].dev : nullptr;
            fz.alpha2 = (float)XL->alpha;
            fz.ldE = M;
            fz.rowsum_out = ch->rowsum >= 0 ? fdev(p->loops[(size_t)ch->rowsum].outs[0]) : nullptr;
        }
        cudaError_t e = launch_gemm_tc(p->opts.gemm_prec, c, (const float*)A.dev + (size_t)r0 * K,
                                       (const float*)B.dev, c0, r1 - r0, N, K, (float)L.alpha, late_c0 ? 0.0f : beta,
                                       p->opts.kchunk, p->opts.tile_cfg, p->arena + p->lay.tc_off, p->lay.tc_bytes,
                                       (int*)(p->arena + p->lay.err_off), sx, tev, &why, ch ? &fz : nullptr, &part);
        if (e != cudaSuccess) return why.empty() ? cuda_fail(e, "row-block GEMM") : fail(GAO_EINVAL, why);
        S.launches += tev.launches;
        if (late_c0) {  // C = fma(beta, C0, alpha AB) over the block's rows
            if (copy_c0) GAO_CUDA_TRY(cudaStreamWaitEvent(sx, p->pipe_ev[2 + kMaxRowBlocks + (size_t)i], 0));
            e = launch_axpy(c, c, beta, (const float*)C0->dev + (size_t)r0 * N, (r1 - r0) * N, sx);
            if (e != cudaSuccess) return cuda_fail(e, "row-block beta C0");
            S.launches += 1;
        }
        if (early_out) {
            GAO_CUDA_TRY(cudaEventRecord(p->out_ev[(size_t)i], sx));
            GAO_CUDA_TRY(cudaStreamWaitEvent(p->ost, p->out_ev[(size_t)i], 0));
            const size_t off = (size_t)r0 * N * 4, len = (size_t)(r1 - r0) * N * 4;
            GAO_CUDA_TRY(cudaMemcpyAsync((char*)C.host + off, C.dev + off, len, cudaMemcpyDeviceToHost, p->ost));
            S.d2h_bytes += len;
        }
    }
    if (alt) {  // the second stream joined back into the program's stream (a captured graph needs that)
        GAO_CUDA_TRY(cudaEventRecord(join2, p->st2));
        GAO_CUDA_TRY(cudaStreamWaitEvent(st, join2, 0));
    }
    GAO_CUDA_TRY(record_timing(ev[3], st));
    if (early_out) {  // joined back into the program's stream (a captured graph needs that)
        GAO_CUDA_TRY(cudaEventRecord(p->out_ev[(size_t)kMaxRowBlocks], p->ost));
        GAO_CUDA_TRY(cudaStreamWaitEvent(st, p->out_ev[(size_t)kMaxRowBlocks], 0));
    }
    *c_on_host = early_out;
    A.vd = B.vd = true;
    if (C0) C0->vd = true;
    p->ev_used[(size_t)li] |= 1 | 2 | 4;
    return GAO_OK;
}

// Copy/compute overlap for a GPU STENCIL3 loop whose image comes from the host (a camera
// frame, 30x slower to copy than to read from HBM): the frame is copied in row strips on
// the copy stream, and as each strip lands the stencil forms the rows whose three input rows
// are all in -- or, when the gene fuses the gradient chain on the stencil's output (gch,
// from find_edge_chain), the blur and the chain in one pass form the rows whose five raw rows
// are in.  A pixel is formed the same way whatever the row ranges, so the bits are those of
// one launch.
bool stencil_pipelined(const gao_prog* p, const gao_loop& L) {
    if (L.kind != GAO_LOOP_STENCIL3 || p->opts.transfer_mode != GAO_TRANSFER_RESIDENT) return false;
    const BufState& X = p->bufs[(size_t)L.ins[0]];
    return !X.vd && X.vh && X.bytes >= kPipelineMinBytes && X.d.rows >= 4 * kMaxRowBlocks &&
           L.ins[0] != L.outs[0];
}

gao_status run_gpu_stencil_pipelined(RunCtx& R, int li, const GradChain* gch) {
    gao_prog* p = R.p;
    const gao_loop& L = p->loops[(size_t)li];
    gao_loop_stat& S = p->stats[(size_t)li];
    BufState& X = p->bufs[(size_t)L.ins[0]];
    float* out = (float*)p->bufs[(size_t)L.outs[0]].dev;
    const int64_t rows = X.d.rows, cols = X.d.cols;
    const int nb = kMaxRowBlocks;
    cudaStream_t st = R.st, cs = p->cst;
    cudaEvent_t* ev = &p->ev[(size_t)li * 6];
    GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[0], st));  // the copy overwrites X on the device: after earlier work
    GAO_CUDA_TRY(cudaStreamWaitEvent(cs, p->pipe_ev[0], 0));
    GAO_CUDA_TRY(record_timing(ev[0], cs));
    int64_t at[kMaxRowBlocks + 1];
    for (int k = 0; k <= nb; ++k) at[k] = rows * k / nb;
    for (int k = 0; k < nb; ++k) {
        const size_t off = (size_t)at[k] * cols * 4, len = (size_t)(at[k + 1] - at[k]) * cols * 4;
        GAO_CUDA_TRY(cudaMemcpyAsync(X.dev + off, (char*)X.host + off, len, cudaMemcpyHostToDevice, cs));
        S.h2d_bytes += len;
        // the copy-time stamp goes before the last strip's event, so that everything on the
        // copy stream is joined back into the program's stream (a captured graph needs that)
        if (k == nb - 1) GAO_CUDA_TRY(record_timing(ev[1], cs));
        GAO_CUDA_TRY(cudaEventRecord(p->pipe_ev[2 + (size_t)k], cs));
    }
    GAO_CUDA_TRY(record_timing(ev[2], st));
    const int preset = (int)(L.flags & ~GAO_LOOP_EXTERNAL_CALL);
    auto chain_ptr = [&](int b, bool live) { return live ? (float*)p->bufs[(size_t)b].dev : nullptr; };
    // the chain's sum and column maxima across the strips: keys cleared by the first strip,
    // partials laid out strip after strip, added and decoded after the last
    GradReduce red{};
    if (gch) red = grad_reduce_for(p, *gch);
    const bool reduce = gch && (gch->sum_loop >= 0 || gch->colmax_loop >= 0);
    int64_t formed = 0;  // output rows done
    for (int k = 0; k < nb; ++k) {
        GAO_CUDA_TRY(cudaStreamWaitEvent(st, p->pipe_ev[2 + (size_t)k], 0));
        if (!gch) {
            const int64_t f1 = k == nb - 1 ? rows : at[k + 1] - 1;  // row r needs input row r + 1
            if (f1 > formed) {
                cudaError_t e = launch_stencil3(out, (const float*)X.dev, rows, cols, preset, st, formed, f1);
                if (e != cudaSuccess) return cuda_fail(e, "stencil strip launch");
                S.launches += 1;
                formed = f1;
            }
            continue;
        }
        // the blur and the chain in one pass: output row r needs raw rows up to r + 2
        const int64_t f1 = k == nb - 1 ? rows : at[k + 1] - 2;
        if (f1 > formed) {
            red.first = formed == 0;
            red.last = f1 == rows;
            int nl = 0;
            cudaError_t e = launch_edge_chain((const float*)X.dev, chain_ptr(gch->x, gch->x_live), rows, cols, gch->p0,
                                              gch->p1, gch->p2, gch->alpha, gch->swap,
                                              chain_ptr(gch->g1, gch->live[0]), chain_ptr(gch->g2, gch->live[1]),
                                              chain_ptr(gch->s1, gch->live[2]), chain_ptr(gch->s2, gch->live[3]),
                                              chain_ptr(gch->m, gch->m_live), st, formed, f1,
                                              reduce ? &red : nullptr, &nl);
            if (e != cudaSuccess) return cuda_fail(e, "blur and gradient chain strip launch");
            S.launches += nl;
            red.part_at += edge_chain_blocks(f1 - formed, cols);
            formed = f1;
        }
    }
    GAO_CUDA_TRY(record_timing(ev[3], st));
    X.vd = true;
    p->ev_used[(size_t)li] |= 1 | 2;
    return GAO_OK;
}

double ev_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return 0.0;
    return (double)ms;
}
}  // namespace

// Everything a run under a gene puts on the program's stream, in program order, with the
// host loops run in between: residency reset, the error word, each loop's copies and
// kernels (or its host loop), the outputs' copies back and the error word's read-back.
// When every loop is on the GPU this is also what a CUDA graph of the run captures.
// The GEMM loop that alone reads INIT loop li's output b, as its A (*which = 0) or its B
// (*which = 1), when that GEMM runs on the GPU in split bfloat16 without a fused chain: b is
// then formed straight into the GEMM's bfloat16 planes, never as binary32.  -1 otherwise (b
// is not a TEMP buffer, is read by anything else or written by another loop, the GEMM reads
// it twice or also as C0, transfers are per loop).
int planes_consumer(const gao_prog* p, int li, int b, uint64_t gene_mask, bool fuse, int* which) {
    const BufState& B = p->bufs[(size_t)b];
    if (B.d.role != GAO_BUF_TEMP || p->opts.transfer_mode != GAO_TRANSFER_RESIDENT || p->lay.tc_bytes == 0) return -1;
    const int prec = p->opts.gemm_prec;
    if (prec != GAO_GEMM_BF16 && prec != GAO_GEMM_BF16X3 && prec != GAO_GEMM_BF16X6) return -1;
    int reader = -1;
    for (int j = 0; j < (int)p->loops.size(); ++j) {
        const gao_loop& Lj = p->loops[(size_t)j];
        if (j != li)
            for (int o : loop_outputs(Lj))
                if (o == b) return -1;
        for (int i : loop_inputs(Lj))
            if (i == b) {
                if (reader >= 0 && reader != j) return -1;
                reader = j;
            }
    }
    if (reader <= li) return -1;
    const gao_loop& G = p->loops[(size_t)reader];
    if (G.kind != GAO_LOOP_GEMM || !((gene_mask >> reader) & 1)) return -1;
    if (G.outs[0] == b || G.ins[2] == b || (G.ins[0] == b) == (G.ins[1] == b)) return -1;
    Chain c;
    if (find_chain(p, reader, gene_mask, fuse, &c)) return -1;
    const gao_buffer &A = p->bufs[(size_t)G.ins[0]].d, &Bm = p->bufs[(size_t)G.ins[1]].d;
    if (A.rows <= 0 || A.cols <= 0 || Bm.cols <= 0) return -1;
    *which = G.ins[0] == b ? 0 : 1;
    return reader;
}

// INIT loop li on the GPU with the outputs whose cons[t] >= 0 formed as the planes of GEMM
// loop cons[t] (operand wh[t]) and the others written as binary32, row exponents once.
gao_status run_gpu_init_planes(RunCtx& R, int li, const int* cons, const int* wh) {
    gao_prog* p = R.p;
    const gao_loop& L = p->loops[(size_t)li];
    cudaStream_t st = R.st;
    int& nl = p->stats[(size_t)li].launches;
    char* a = p->arena;
    InitSet set{};
    int64_t rx_rows = 0, total = 0;
    for (int t = 0; t < GAO_MAX_IO; ++t) {
        const int b = L.outs[t];
        if (b < 0) continue;
        const BufState& B = p->bufs[(size_t)b];
        const int rs = (int)((L.flags >> t) & 1);
        if (rs) rx_rows = std::max(rx_rows, B.d.rows);
        if (cons[t] >= 0) continue;
        set.o[set.n++] = InitOut{(float*)B.dev, B.d.rows, B.d.cols, (uint32_t)b, rs};
        total += B.d.rows * B.d.cols;
    }
    set.seed = p->opts.seed;
    set.rowexp = rx_rows > 0 ? (const int8_t*)(a + p->lay.rowexp_off) : nullptr;
    if (rx_rows > 0) {
        GAO_CUDA_TRY(launch_row_exponents((int8_t*)set.rowexp, rx_rows, p->opts.seed, st));
        nl += 1;
    }
    if (total > 0) {
        GAO_CUDA_TRY(launch_init_set(set, st));
        nl += 1;
    }
    for (int t = 0; t < GAO_MAX_IO; ++t) {
        if (L.outs[t] < 0 || cons[t] < 0) continue;
        const gao_loop& G = p->loops[(size_t)cons[t]];
        const gao_buffer &A = p->bufs[(size_t)G.ins[0]].d, &Bm = p->bufs[(size_t)G.ins[1]].d;
        const int rs = (int)((L.flags >> t) & 1);
        int l = 0;
        GAO_CUDA_TRY(tc_init_planes(p->opts.gemm_prec, wh[t], A.rows, Bm.cols, A.cols, p->opts.kchunk,
                                    p->opts.tile_cfg, p->opts.seed, (uint32_t)L.outs[t], rs ? set.rowexp : nullptr,
                                    a + p->lay.tc_off, p->lay.tc_bytes, st, &l));
        nl += l;
    }
    return GAO_OK;
}

gao_status enqueue_run(RunCtx& R, uint64_t gene_mask, bool fuse, uint32_t flags) {
    gao_prog* p = R.p;
    const int n = (int)p->loops.size();
    for (auto& B : p->bufs) {
        B.vh = (B.d.role == GAO_BUF_INPUT);
        B.vd = false;
        B.gen_loop = B.gen_slot = B.gen_for = -1;
    }
    std::fill(p->ev_used.begin(), p->ev_used.end(), 0);
    for (auto& s : p->stats) s = gao_loop_stat{};
    const bool uses_gpu = gene_mask != 0;
    char* d_err = p->arena + p->lay.err_off;
    if (uses_gpu) GAO_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), p->st));
    gao_status status = GAO_OK;
    uint64_t fused = 0;  // loops already run inside a fused pass
    for (int li = 0; li < n && status == GAO_OK; ++li) {
        const gao_loop& L = p->loops[(size_t)li];
        const bool gpu = (gene_mask >> li) & 1;
        gao_loop_stat& S = p->stats[(size_t)li];
        S.placement = gpu ? 1 : 0;
        if ((fused >> li) & 1) {
            S.placement = 2;
            continue;
        }
        cudaEvent_t* ev = &p->ev[(size_t)li * 6];
        Chain chain;
        GradChain gch;
        if (gpu && stencil_pipelined(p, L)) {
            // the image comes from the host: strips overlapped with its copy, with the
            // gradient chain on this stencil's output in the same strips when the gene fuses it
            const bool chained = find_edge_chain(p, li, gene_mask, fuse, &gch);
            if ((status = run_gpu_stencil_pipelined(R, li, chained ? &gch : nullptr)) != GAO_OK) break;
            BufState& Bo = p->bufs[(size_t)L.outs[0]];
            Bo.vh = false;
            Bo.vd = true;
            if (chained) grad_chain_done(p, gch, li + 1, &fused);
            if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
            if (R.timed_out) break;
            continue;
        }
        // a blur whose output starts a gradient chain: both in one pass over the raw image
        // (edge); else a gradient chain starting here, in one pass over the blurred image
        const bool edge = gpu && L.kind == GAO_LOOP_STENCIL3 && find_edge_chain(p, li, gene_mask, fuse, &gch);
        if (edge || (gpu && L.kind == GAO_LOOP_STENCIL3 && find_grad_chain(p, li, gene_mask, fuse, &gch, true))) {
            const int src = edge ? gch.raw : gch.x;  // the image the pass reads
            BufState& X = p->bufs[(size_t)src];
            const bool copies = !X.vd;
            if (copies) GAO_CUDA_TRY(record_timing(ev[0], p->st));
            if ((status = make_valid(R, src, true, S)) != GAO_OK) break;
            if (copies) {
                GAO_CUDA_TRY(record_timing(ev[1], p->st));
                p->ev_used[(size_t)li] |= 1;
            }
            auto dptr = [&](int b, bool live) { return live ? (float*)p->bufs[(size_t)b].dev : nullptr; };
            GAO_CUDA_TRY(record_timing(ev[2], p->st));
            // the sum and the column maxima of m that follow the chain, in the same pass
            const GradReduce red = grad_reduce_for(p, gch);
            const bool reduce = gch.sum_loop >= 0 || gch.colmax_loop >= 0;
            int nl = 0;
            const cudaError_t e =
                edge ? launch_edge_chain((const float*)X.dev, dptr(gch.x, gch.x_live), X.d.rows, X.d.cols, gch.p0,
                                         gch.p1, gch.p2, gch.alpha, gch.swap, dptr(gch.g1, gch.live[0]),
                                         dptr(gch.g2, gch.live[1]), dptr(gch.s1, gch.live[2]),
                                         dptr(gch.s2, gch.live[3]), dptr(gch.m, gch.m_live), p->st, 0, -1,
                                         reduce ? &red : nullptr, &nl)
                     : launch_grad_chain((const float*)X.dev, X.d.rows, X.d.cols, gch.p1, gch.p2, gch.alpha,
                                         gch.swap, dptr(gch.g1, gch.live[0]), dptr(gch.g2, gch.live[1]),
                                         dptr(gch.s1, gch.live[2]), dptr(gch.s2, gch.live[3]),
                                         dptr(gch.m, gch.m_live), p->st, 0, -1, reduce ? &red : nullptr, &nl);
            if (e != cudaSuccess) {
                status = cuda_fail(e, edge ? "blur and gradient chain launch" : "gradient chain launch");
                break;
            }
            GAO_CUDA_TRY(record_timing(ev[3], p->st));
            p->ev_used[(size_t)li] |= 2;
            S.launches += nl;
            grad_chain_done(p, gch, edge ? li + 1 : li, &fused);
            if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
            if (R.timed_out) break;
            continue;
        }
        EwPlan ewp;
        if (gpu && is_elementwise(L.kind) && find_ew_chain(p, li, gene_mask, fuse, &ewp)) {
            const int last = ewp.loops[ewp.n - 1];
            // buffers the chain reads from memory: every input of its first loop, and each
            // later loop's input other than the previous loop's output
            std::vector<int> ext;
            int prev = -1;
            for (int k = 0; k < ewp.n; ++k) {
                const gao_loop& Lk = p->loops[(size_t)ewp.loops[k]];
                for (int b : loop_inputs(Lk))
                    if ((k == 0 || b != prev) && std::find(ext.begin(), ext.end(), b) == ext.end()) ext.push_back(b);
                prev = Lk.outs[0];
            }
            bool copies = false;
            for (int b : ext) copies |= !p->bufs[(size_t)b].vd;
            if (copies) GAO_CUDA_TRY(record_timing(ev[0], p->st));
            for (int b : ext)
                if ((status = make_valid(R, b, true, S)) != GAO_OK) break;
            if (status != GAO_OK) break;
            if (copies) {
                GAO_CUDA_TRY(record_timing(ev[1], p->st));
                p->ev_used[(size_t)li] |= 1;
            }
            EwChain c{};
            c.nops = ewp.n;
            c.n = (int64_t)p->bufs[(size_t)L.outs[0]].d.rows * p->bufs[(size_t)L.outs[0]].d.cols;
            std::vector<char> live((size_t)ewp.n, 0);
            prev = -1;
            for (int k = 0; k < ewp.n; ++k) {
                const gao_loop& Lk = p->loops[(size_t)ewp.loops[k]];
                EwChainOp& op = c.op[k];
                op.kind = Lk.kind == GAO_LOOP_RELU ? 0 : Lk.kind == GAO_LOOP_SQUARE ? 1 : 2;
                op.alpha = (float)Lk.alpha;
                auto src = [&](int b) -> const float* {
                    return (k > 0 && b == prev) ? nullptr : (const float*)p->bufs[(size_t)b].dev;
                };
                op.xa = src(Lk.ins[0]);
                op.yb = op.kind == 2 ? src(Lk.ins[1]) : nullptr;
                const int ob = Lk.outs[0];
                bool lv = p->bufs[(size_t)ob].d.role == GAO_BUF_OUTPUT;
                for (int j = last + 1; j < n && !lv; ++j)
                    for (int b : loop_inputs(p->loops[(size_t)j]))
                        if (b == ob) lv = true;
                live[(size_t)k] = lv;
                op.out = lv ? (float*)p->bufs[(size_t)ob].dev : nullptr;
                prev = ob;
            }
            GAO_CUDA_TRY(record_timing(ev[2], p->st));
            const cudaError_t e = launch_ew_chain(c, p->st);
            if (e != cudaSuccess) {
                status = cuda_fail(e, "element-wise chain launch");
                break;
            }
            GAO_CUDA_TRY(record_timing(ev[3], p->st));
            p->ev_used[(size_t)li] |= 2;
            S.launches += c.n > 0;
            for (int k = 0; k < ewp.n; ++k) {  // in loop order: a buffer written twice ends as the last
                BufState& B = p->bufs[(size_t)p->loops[(size_t)ewp.loops[k]].outs[0]];
                B.vh = false;
                B.vd = live[(size_t)k] != 0;  // an unwritten intermediate holds nothing
            }
            for (int k = 1; k < ewp.n; ++k) fused |= 1ULL << ewp.loops[k];
            if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
            if (R.timed_out) break;
            continue;
        }
        if (gpu && L.kind == GAO_LOOP_INIT) {
            // outputs that only a split-precision GEMM reads go straight into its planes
            int cons[GAO_MAX_IO], wh[GAO_MAX_IO], ndefer = 0;
            for (int t = 0; t < GAO_MAX_IO; ++t) {
                cons[t] = L.outs[t] >= 0 ? planes_consumer(p, li, L.outs[t], gene_mask, fuse, &wh[t]) : -1;
                ndefer += cons[t] >= 0;
            }
            if (ndefer > 0) {
                GAO_CUDA_TRY(record_timing(ev[2], p->st));
                if ((status = run_gpu_init_planes(R, li, cons, wh)) != GAO_OK) break;
                GAO_CUDA_TRY(record_timing(ev[3], p->st));
                p->ev_used[(size_t)li] |= 2;
                for (int t = 0; t < GAO_MAX_IO; ++t) {
                    if (L.outs[t] < 0) continue;
                    BufState& B = p->bufs[(size_t)L.outs[t]];
                    B.vh = false;
                    B.vd = cons[t] < 0;
                    if (cons[t] >= 0) {
                        B.gen_loop = li;
                        B.gen_slot = t;
                        B.gen_for = cons[t];
                    }
                }
                if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
                if (R.timed_out) break;
                continue;
            }
        }
        // a GEMM whose A comes from the host overlaps the copy (row blocks) rather than fusing
        const int64_t blocks = gpu ? pipeline_blocks(p, L) : 0;
        bool c_on_host = false;  // the pipelined GEMM copied C back block by block
        if (gpu && blocks == 0 && L.kind == GAO_LOOP_GEMM && find_chain(p, li, gene_mask, fuse, &chain)) {
            // inputs of the whole chain: the GEMM's and the AXPY's second operand
            std::vector<int> cin = loop_inputs(L);
            cin.push_back(p->loops[(size_t)chain.axpy].ins[1]);
            bool copies = false;
            for (int b : cin) copies |= !p->bufs[(size_t)b].vd;
            if (copies) GAO_CUDA_TRY(record_timing(ev[0], p->st));
            for (int b : cin)
                if ((status = make_valid(R, b, true, S)) != GAO_OK) break;
            if (status != GAO_OK) break;
            if (copies) {
                GAO_CUDA_TRY(record_timing(ev[1], p->st));
                p->ev_used[(size_t)li] |= 1;
            }
            GAO_CUDA_TRY(record_timing(ev[2], p->st));
            if ((status = run_gpu_chain(R, li, chain)) != GAO_OK) break;
            GAO_CUDA_TRY(record_timing(ev[3], p->st));
            p->ev_used[(size_t)li] |= 2;
            for (int j : {li, chain.axpy, chain.transpose, chain.rowsum, chain.frob}) {
                if (j < 0) continue;
                for (int b : loop_outputs(p->loops[(size_t)j])) {
                    p->bufs[(size_t)b].vh = false;
                    p->bufs[(size_t)b].vd = true;
                }
                if (j != li) fused |= 1ULL << j;
            }
            if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
            if (R.timed_out) break;
            continue;
        }
        const std::vector<int> ins = loop_inputs(L);
        const bool per_loop = p->opts.transfer_mode == GAO_TRANSFER_PER_LOOP;
        if (gpu && per_loop)  // directive offload without a data region: inputs always copied in
            for (int b : ins) p->bufs[(size_t)b].vd = false;
        if (blocks > 0) {
            // fused too when the chain qualifies and its X is the GEMM's A (copied in the
            // blocks) or already on the device
            Chain pch;
            bool pf = find_chain(p, li, gene_mask, fuse, &pch);
            if (pf) {
                const int xb = p->loops[(size_t)pch.axpy].ins[1];
                pf = xb == L.ins[0] || p->bufs[(size_t)xb].vd;
            }
            // C's rows go back to the host as their blocks finish when the run copies C back
            // anyway (an OUTPUT, device buffers not kept, resident transfers)
            const BufState& Cb = p->bufs[(size_t)L.outs[0]];
            const bool early_out = !per_loop && !(flags & GAO_RUN_KEEP_DEVICE) && Cb.d.role == GAO_BUF_OUTPUT &&
                                   Cb.host != nullptr && L.outs[0] != L.ins[0] && L.outs[0] != L.ins[1];
            c_on_host = false;
            if ((status = run_gpu_gemm_pipelined(R, li, blocks, pf ? &pch : nullptr, early_out, &c_on_host)) !=
                GAO_OK)
                break;
            if (pf) {
                for (int j : {li, pch.axpy, pch.transpose, pch.rowsum, pch.frob}) {
                    if (j < 0) continue;
                    for (int b : loop_outputs(p->loops[(size_t)j])) {
                        p->bufs[(size_t)b].vh = false;
                        p->bufs[(size_t)b].vd = true;
                    }
                    if (j != li) fused |= 1ULL << j;
                }
                if (c_on_host) p->bufs[(size_t)L.outs[0]].vh = true;
                if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
                if (R.timed_out) break;
                continue;
            }
        } else if (gpu) {
            bool copies = false;
            auto planes_only = [&](int b) { return p->bufs[(size_t)b].gen_for == li; };  // read as planes
            for (int b : ins) copies |= !p->bufs[(size_t)b].vd && !planes_only(b);
            if (copies) GAO_CUDA_TRY(record_timing(ev[0], p->st));
            for (int b : ins)
                if (!planes_only(b) && (status = make_valid(R, b, true, S)) != GAO_OK) break;
            if (status != GAO_OK) break;
            if (copies) {
                GAO_CUDA_TRY(record_timing(ev[1], p->st));
                p->ev_used[(size_t)li] |= 1;
            }
            GAO_CUDA_TRY(record_timing(ev[2], p->st));
            if ((status = run_gpu_loop(R, li)) != GAO_OK) break;
            GAO_CUDA_TRY(record_timing(ev[3], p->st));
            p->ev_used[(size_t)li] |= 2;
        } else {
            const double c0 = now_s();
            for (int b : ins)
                if ((status = make_valid(R, b, false, S)) != GAO_OK) break;
            if (status != GAO_OK) break;
            // the host loop may overwrite mirrors that queued copies still read, and
            // reads mirrors that queued copies fill: drain the stream first
            if (uses_gpu && (status = stream_wait(p->st, R.deadline, &R.timed_out)) != GAO_OK) break;
            const double c1 = now_s();
            S.copy_ms = (c1 - c0) * 1e3;
            if (R.timed_out) break;
            status = run_cpu_loop(R, li);
            S.cpu_ms = (now_s() - c1) * 1e3;
            if (R.cpu.timed_out) R.timed_out = true;
            if (status != GAO_OK || R.timed_out) break;
        }
        for (int b : loop_outputs(L)) {
            p->bufs[(size_t)b].vh = !gpu;
            p->bufs[(size_t)b].vd = gpu;
        }
        if (blocks > 0 && c_on_host) p->bufs[(size_t)L.outs[0]].vh = true;  // copied back block by block
        if (gpu && per_loop) {  // ... and outputs always copied back out; the device copy is dropped
            for (int b : loop_outputs(L))
                if ((status = make_valid(R, b, false, S)) != GAO_OK) break;
            if (status != GAO_OK) break;
            for (int b : loop_outputs(L)) p->bufs[(size_t)b].vd = false;
        }
        if (R.deadline > 0.0 && now_s() > R.deadline) R.timed_out = true;
        if (R.timed_out) break;
    }
    if (status == GAO_OK && !R.timed_out && !(flags & GAO_RUN_KEEP_DEVICE)) {
        gao_loop_stat dummy{};
        for (size_t b = 0; b < p->bufs.size(); ++b)
            if (p->bufs[b].d.role == GAO_BUF_OUTPUT && !p->bufs[b].vh)
                if ((status = make_valid(R, (int)b, false, dummy)) != GAO_OK) break;
        if (!p->stats.empty()) p->stats.back().d2h_bytes += dummy.d2h_bytes;
    }
    if (uses_gpu) {
        cudaError_t e = cudaMemcpyAsync(p->h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st);
        if (e != cudaSuccess && status == GAO_OK) status = cuda_fail(e, "cudaMemcpyAsync(err)");
    }
    return status;
}

// Capture one run of an all-GPU gene as a graph (nothing executes during the capture)
// and keep what the run leaves on the host side: residency flags and per-loop statistics.
void capture_run(RunCtx& R, uint64_t gene_mask, bool fuse, uint32_t flags, GraphEntry* ge) {
    gao_prog* p = R.p;
    if (cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        ge->failed = true;
        return;
    }
    g_capturing = true;
    const gao_status st = enqueue_run(R, gene_mask, fuse, flags);
    g_capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->st, &g);
    cudaGraphExec_t exec = nullptr;
    if (st == GAO_OK && e == cudaSuccess && g && !R.timed_out &&
        cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
        ge->exec = exec;
        ge->vh.resize(p->bufs.size());
        ge->vd.resize(p->bufs.size());
        for (size_t b = 0; b < p->bufs.size(); ++b) {
            ge->vh[b] = p->bufs[b].vh;
            ge->vd[b] = p->bufs[b].vd;
        }
        ge->stats = p->stats;
        ge->ev_used = p->ev_used;
    } else {
        cudaGetLastError();  // the run falls back to plain launches; the gene is not captured again
        ge->failed = true;
    }
    if (g) cudaGraphDestroy(g);
    R.timed_out = false;
}

extern "C" gao_status prog_run(gao_prog* p, uint64_t gene, uint32_t flags, double* seconds_out) {
    if (!p) return fail(GAO_EINVAL, "program is null");
    const int n = (int)p->loops.size();
    const int a = gene_length(p);
    if (a < 64 && (gene >> a) != 0)
        return fail(GAO_EINVAL, "gene has bits set at or above the gene length (" + std::to_string(a) + ")");
    const uint64_t gene_mask = loop_mask_of(p, gene);  // bit li: loop li runs on the GPU
    const bool fuse = gene_fuses(p, gene);
    for (auto& B : p->bufs)
        if (B.d.role == GAO_BUF_INPUT && !B.input_set)
            return fail(GAO_EINVAL, "INPUT buffers must be set with prog_set_input before a run");
    if (p->dirty_stream) {
        bool to = false;
        gao_status s = stream_wait(p->st, 0.0, &to);
        if (s != GAO_OK) return s;
        p->dirty_stream = false;
    }
    cudaError_t ce = cudaSetDevice(p->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    RunCtx R{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, p->st, true};
    const bool no_times = (flags & GAO_RUN_NO_LOOP_TIMES) != 0;
    struct TimesOff {  // record_timing is a no-op for this run only
        explicit TimesOff(bool on) { g_no_times = on; }
        ~TimesOff() { g_no_times = false; }
    } times_off(no_times);
    const double t0 = now_s();
    if (p->opts.timeout_s > 0.0) R.deadline = R.cpu.deadline = t0 + p->opts.timeout_s;
    const bool uses_gpu = gene_mask != 0;
    gao_status status = GAO_OK;
    p->stats_pending = false;
    // a gene that keeps every loop on the GPU is captured as a CUDA graph on its second
    // run and replayed from then on (one launch per run; the host work of the run is done once)
    const bool all_gpu = gene_mask == all_genes(n) && gene_length(p) > 0;
    GraphEntry* ge = nullptr;
    if (all_gpu && !(flags & GAO_RUN_NO_GRAPH)) {
        ge = &p->graphs[gene * 8 + (flags & (GAO_RUN_KEEP_DEVICE | GAO_RUN_NO_LOOP_TIMES))];
        ge->runs += 1;
    }
    if (ge && !ge->exec && !ge->failed && ge->runs >= 2) capture_run(R, gene_mask, fuse, flags, ge);
    if (ge && ge->exec) {
        cudaError_t e = cudaGraphLaunch(ge->exec, p->st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        for (size_t b = 0; b < p->bufs.size(); ++b) {
            p->bufs[b].vh = ge->vh[b] != 0;
            p->bufs[b].vd = ge->vd[b] != 0;
        }
        p->stats = ge->stats;
        p->ev_used = ge->ev_used;
    } else {
        status = enqueue_run(R, gene_mask, fuse, flags);
    }
    if (uses_gpu) {
        gao_status ws = stream_wait(p->st, R.deadline, &R.timed_out);
        if (ws != GAO_OK) {
            p->dirty_stream = true;
            return ws;
        }
    }
    const double t1 = now_s();
    if (seconds_out) *seconds_out = t1 - t0;
    if (status != GAO_OK) return status;
    if (uses_gpu && *p->h_err != 0)
        return fail(GAO_EDEVICE, "a kernel raised device error " + std::to_string(*p->h_err) +
                                     (*p->h_err == DEV_WAIT_TIMEOUT ? " (bounded wait expired)" : ""));
    if (R.timed_out) {
        if (seconds_out) *seconds_out = p->opts.timeout_s;
        return fail(GAO_ETIMEOUT, "run exceeded its budget of " + std::to_string(p->opts.timeout_s) + " s");
    }
    if (no_times) std::fill(p->ev_used.begin(), p->ev_used.end(), 0);  // no event of this run to read
    p->stats_pending = true;  // the event times are read when prog_stats asks for them
    return GAO_OK;
}

extern "C" gao_status prog_output(gao_prog* p, int buf, const void** host_ptr, gao_buffer* shape_out) {
    if (!p || !host_ptr) return fail(GAO_EINVAL, "null argument");
    if (buf < 0 || buf >= (int)p->bufs.size()) return fail(GAO_EINVAL, "no such buffer");
    BufState& B = p->bufs[(size_t)buf];
    if (!B.vh) return fail(GAO_EINVAL, "buffer " + std::to_string(buf) + " is not valid on the host after the last run");
    *host_ptr = B.host;
    if (shape_out) *shape_out = B.d;
    return GAO_OK;
}

extern "C" gao_status prog_device_ptr(gao_prog* p, int buf, void** dev_ptr) {
    if (!p || !dev_ptr) return fail(GAO_EINVAL, "null argument");
    if (buf < 0 || buf >= (int)p->bufs.size()) return fail(GAO_EINVAL, "no such buffer");
    BufState& B = p->bufs[(size_t)buf];
    if (!B.vd && !B.vh && B.gen_loop >= 0) {  // formed only as a GEMM's planes: form it now
        cudaError_t ce = cudaSetDevice(p->device);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
        RunCtx R{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, p->st, false};
        gao_status s = materialize(R, buf);
        if (s != GAO_OK) return s;
        if ((ce = cudaStreamSynchronize(p->st)) != cudaSuccess) return cuda_fail(ce, "cudaStreamSynchronize");
    }
    *dev_ptr = B.dev;
    return GAO_OK;
}

extern "C" gao_status prog_planes_for(const gao_prog* p, int buf, int* gemm_loop) {
    if (!p || !gemm_loop) return fail(GAO_EINVAL, "null argument");
    if (buf < 0 || buf >= (int)p->bufs.size()) return fail(GAO_EINVAL, "no such buffer");
    *gemm_loop = p->bufs[(size_t)buf].gen_for;
    return GAO_OK;
}

extern "C" gao_status prog_gemm_residual(gao_prog* p, int loop, const double* x, const double* y,
                                         gao_residual* out) {
    if (!p || !x || !y || !out) return fail(GAO_EINVAL, "null argument");
    if (loop < 0 || loop >= (int)p->loops.size() || p->loops[(size_t)loop].kind != GAO_LOOP_GEMM)
        return fail(GAO_EINVAL, "loop " + std::to_string(loop) + " is not a GEMM loop");
    const gao_loop& L = p->loops[(size_t)loop];
    if (L.ins[2] == L.outs[0])
        return fail(GAO_EINVAL, "the GEMM writes C over C0, so C0 is gone: give C0 a buffer of its own to check it");
    if (p->lay.resid_bytes == 0) return fail(GAO_EINVAL, "program has no residual scratch for this loop");
    const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
    const int64_t M = A.rows, K = A.cols, N = B.cols;
    if (M < 1 || N < 1) return fail(GAO_EINVAL, "empty GEMM");
    cudaError_t ce = cudaSetDevice(p->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    gao_status s = stream_wait(p->st, 0.0, nullptr);  // nothing of an earlier run still in flight
    if (s != GAO_OK) return s;
    p->dirty_stream = false;
    RunCtx R{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, p->st, false};
    gao_loop_stat dummy{};
    for (int b : {L.ins[0], L.ins[1], L.ins[2], L.outs[0]})
        if (b >= 0 && (s = make_valid(R, b, true, dummy)) != GAO_OK) return s;
    char* base = p->arena + p->lay.resid_off;
    const size_t xo = 0, yo = ((size_t)N * 8 + 255) / 256 * 256, so = yo + ((size_t)M * 8 + 255) / 256 * 256;
    GAO_CUDA_TRY(cudaMemcpyAsync(base + xo, x, (size_t)N * 8, cudaMemcpyHostToDevice, p->st));
    GAO_CUDA_TRY(cudaMemcpyAsync(base + yo, y, (size_t)M * 8, cudaMemcpyHostToDevice, p->st));
    const float* c0 = L.ins[2] >= 0 ? (const float*)p->bufs[(size_t)L.ins[2]].dev : nullptr;
    const double* nd = nullptr;
    int launches = 0;
    GAO_CUDA_TRY(launch_gemm_residual((const float*)p->bufs[(size_t)L.ins[0]].dev,
                                      (const float*)p->bufs[(size_t)L.ins[1]].dev, c0,
                                      (const float*)p->bufs[(size_t)L.outs[0]].dev, M, N, K, L.alpha,
                                      c0 ? L.beta : 0.0, (const double*)(base + xo), (const double*)(base + yo),
                                      base + so, nullptr, nullptr, p->st, &launches, &nd));
    double h[16];
    GAO_CUDA_TRY(cudaMemcpyAsync(h, nd, sizeof(h), cudaMemcpyDeviceToHost, p->st));
    GAO_CUDA_TRY(cudaStreamSynchronize(p->st));
    residual_from_norms(h, out);
    return GAO_OK;
}

extern "C" gao_status prog_gene_length(const gao_prog* p, int* length) {
    if (!p || !length) return fail(GAO_EINVAL, "null argument");
    *length = gene_length(p);
    return GAO_OK;
}

extern "C" gao_status prog_loop_offload(const gao_prog* p, int loop, int* verdict, int* gene_bit) {
    if (!p) return fail(GAO_EINVAL, "program is null");
    if (loop < 0 || loop >= (int)p->loops.size()) return fail(GAO_EINVAL, "no such loop");
    if (verdict) *verdict = p->verdict[(size_t)loop];
    if (gene_bit) {
        *gene_bit = -1;
        for (size_t k = 0; k < p->gene_loop.size(); ++k)
            if (p->gene_loop[k] == loop) *gene_bit = (int)k;
    }
    return GAO_OK;
}

extern "C" gao_status prog_stats(gao_prog* p, gao_loop_stat* out, int n) {
    if (!p || !out) return fail(GAO_EINVAL, "null argument");
    if (n < (int)p->stats.size()) return fail(GAO_EINVAL, "stats array too short");
    if (p->stats_pending) {  // the last run's CUDA-event times (its stream has drained)
        for (size_t li = 0; li < p->stats.size(); ++li) {
            gao_loop_stat& S = p->stats[li];
            cudaEvent_t* ev = &p->ev[li * 6];
            const uint8_t u = p->ev_used[li];
            if (u & 1) S.copy_ms = ev_ms(ev[0], ev[1]);
            if (u & 2) S.device_ms = ev_ms(ev[2], ev[3]);
            if (u & 4) S.kernel_ms = ev_ms(ev[4], ev[5]);
            else if (u & 2) S.kernel_ms = S.device_ms;
        }
        p->stats_pending = false;
    }
    std::copy(p->stats.begin(), p->stats.end(), out);
    return GAO_OK;
}

extern "C" gao_status prog_cache_clear(gao_prog* p) {
    if (!p) return fail(GAO_EINVAL, "program is null");
    p->cache.clear();
    drop_graphs(p);
    return GAO_OK;
}

extern "C" gao_status prog_graphs(const gao_prog* p, int* captured, int* failed) {
    if (!p) return fail(GAO_EINVAL, "program is null");
    int c = 0, f = 0;
    for (const auto& kv : p->graphs) {
        c += kv.second.exec != nullptr;
        f += kv.second.failed;
    }
    if (captured) *captured = c;
    if (failed) *failed = f;
    return GAO_OK;
}

extern "C" gao_status prog_cache_export(const gao_prog* p, uint64_t* genes, double* seconds, int cap, int* n_out) {
    if (!p || !n_out || cap < 0 || (cap > 0 && (!genes || !seconds))) return fail(GAO_EINVAL, "bad argument");
    // in gene order, so that a checkpoint does not depend on the hash table's layout
    std::vector<std::pair<uint64_t, double>> v;
    v.reserve(p->cache.size());
    for (const auto& kv : p->cache) v.emplace_back(kv.first, kv.second.seconds);
    std::sort(v.begin(), v.end());
    *n_out = (int)v.size();
    for (int i = 0; i < cap && i < (int)v.size(); ++i) {
        genes[i] = v[(size_t)i].first;
        seconds[i] = v[(size_t)i].second;
    }
    return GAO_OK;
}

extern "C" gao_status prog_cache_import(gao_prog* p, const uint64_t* genes, const double* seconds, int n) {
    if (!p || n < 0 || (n > 0 && (!genes || !seconds))) return fail(GAO_EINVAL, "bad argument");
    const int a = gene_length(p);
    for (int i = 0; i < n; ++i) {
        if (a < 64 && (genes[i] >> a) != 0) return fail(GAO_EINVAL, "imported gene longer than the gene length");
        if (!(seconds[i] == seconds[i])) return fail(GAO_EINVAL, "imported time is not a number");
    }
    for (int i = 0; i < n; ++i) {
        CacheEntry ce;
        ce.seconds = seconds[i];
        ce.status = seconds[i] >= 0.0 ? GAO_OK : GAO_EDEVICE;
        p->cache.emplace(genes[i], ce);
    }
    return GAO_OK;
}

extern "C" void prog_destroy(gao_prog* p) { free_prog(p); }

// ---- C ABI: GA ----------------------------------------------------------------------------

namespace {

// Time of one gene over all programs, measured once per program and then cached.
gao_status gene_time(gao_prog* const* progs, int n_progs, uint64_t mask, double* seconds, bool* all_cached) {
    double total = 0.0;
    bool failed = false, cached = true;
    for (int i = 0; i < n_progs; ++i) {
        gao_prog* p = progs[i];
        auto it = p->cache.find(mask);
        CacheEntry ce;
        if (it != p->cache.end()) {
            ce = it->second;
        } else {
            cached = false;
            double s = 0.0;
            gao_status st = prog_run(p, mask, 0, &s);
            if (st == GAO_EINVAL || st == GAO_ENODEV || st == GAO_ENOMEM || st == GAO_ECUDA) return st;
            ce.status = st;
            ce.seconds = st == GAO_OK ? s : (st == GAO_ETIMEOUT ? p->opts.timeout_s : -1.0);
            p->cache.emplace(mask, ce);
        }
        if (ce.seconds < 0.0) failed = true;
        total += ce.seconds;
    }
    *seconds = failed ? -1.0 : total;
    if (all_cached) *all_cached = cached;
    return GAO_OK;
}

gao_status check_progs(gao_prog* const* progs, int n_progs, int* n_genes) {
    if (!progs || n_progs < 1) return fail(GAO_EINVAL, "need at least one program");
    for (int i = 0; i < n_progs; ++i)
        if (!progs[i]) return fail(GAO_EINVAL, "null program");
    const int a = gene_length(progs[0]);
    for (int i = 0; i < n_progs; ++i)
        if (gene_length(progs[i]) != a) return fail(GAO_EINVAL, "programs differ in gene length");
    *n_genes = a;
    return GAO_OK;
}

}  // namespace

extern "C" gao_status ga_evaluate(gao_prog* const* progs, int n_progs, const uint64_t* population, int pop,
                                  double* fitness_out, double* seconds_out, int* cache_hits_out) {
    int a = 0;
    gao_status s = check_progs(progs, n_progs, &a);
    if (s != GAO_OK) return s;
    if (!population || pop < 0) return fail(GAO_EINVAL, "bad population");
    int hits = 0;
    for (int i = 0; i < pop; ++i) {
        double t = 0.0;
        bool cached = false;
        if ((s = gene_time(progs, n_progs, population[i], &t, &cached)) != GAO_OK) return s;
        hits += cached ? 1 : 0;
        if (seconds_out) seconds_out[i] = t;
        if (fitness_out) fitness_out[i] = ga_fitness(t);
    }
    if (cache_hits_out) *cache_hits_out = hits;
    return GAO_OK;
}

extern "C" gao_status ga_run(gao_prog* const* progs, int n_progs, const gao_ga_params* params,
                             gao_ga_result* result) {
    int a = 0;
    gao_status s = check_progs(progs, n_progs, &a);
    if (s != GAO_OK) return s;
    if (!params || !result) return fail(GAO_EINVAL, "null params or result");
    if (a < 1) return fail(GAO_EINVAL, "no loop of the program is offloadable (gene length 0)");
    std::vector<double> saved((size_t)n_progs);
    for (int i = 0; i < n_progs; ++i) saved[(size_t)i] = progs[i]->opts.timeout_s;
    double budget = params->timeout_s;
    if (budget < 0.0) {  // automatic: 10 x the all-GPU time, capped at 60 s
        const uint64_t all = all_genes(a);
        double t = 0.0;
        for (int i = 0; i < n_progs; ++i) {
            double ti = 0.0;
            progs[i]->opts.timeout_s = 0.0;
            if ((s = prog_run(progs[i], all, 0, &ti)) != GAO_OK) return s;
            t += ti;
        }
        budget = std::min(60.0, 10.0 * t / n_progs);
    }
    if (budget > 0.0)
        for (int i = 0; i < n_progs; ++i) progs[i]->opts.timeout_s = budget;
    TimeFn fn = [&](uint64_t m, double* t) { return gene_time(progs, n_progs, m, t, nullptr); };
    s = ga_core(a, *params, fn, result);
    for (int i = 0; i < n_progs; ++i) progs[i]->opts.timeout_s = saved[(size_t)i];
    return s;
}

extern "C" gao_status ga_run_table(const double* times, int n_genes, const gao_ga_params* params,
                                   gao_ga_result* result) {
    if (!times || !params || !result) return fail(GAO_EINVAL, "null argument");
    if (n_genes < 1 || n_genes > 24) return fail(GAO_EINVAL, "table GA supports 1..24 genes");
    TimeFn fn = [&](uint64_t m, double* t) {
        *t = times[m];
        return GAO_OK;
    };
    return ga_core(n_genes, *params, fn, result);
}

extern "C" gao_status ga_run_callback(int n_genes, const gao_ga_params* params, gao_gene_eval_fn eval, void* ctx,
                                      gao_ga_result* result) {
    if (!params || !eval || !result) return fail(GAO_EINVAL, "null argument");
    PopFn fn = [&](const std::vector<uint64_t>& genes, std::vector<double>* secs) {
        secs->assign(genes.size(), -1.0);
        const int st = eval(genes.data(), (int)genes.size(), secs->data(), ctx);
        if (st != GAO_OK) return fail((gao_status)(st > 0 && st <= GAO_ECPU ? st : GAO_ECPU), "gene evaluation callback failed");
        return GAO_OK;
    };
    return ga_core_pop(n_genes, *params, fn, result);
}

// ---- C ABI: autotuning -------------------------------------------------------------------------

extern "C" gao_status prog_autotune(gao_prog* p, const gao_ga_params* params, gao_autotune_result* out) {
    if (!p || !params || !out) return fail(GAO_EINVAL, "null argument");
    const int prec = p->opts.gemm_prec;
    if (prec == GAO_GEMM_FP32_SIMT) return fail(GAO_EINVAL, "autotuning covers the tensor-core GEMM only");
    int li = -1;
    for (size_t i = 0; i < p->loops.size(); ++i)
        if (p->loops[i].kind == GAO_LOOP_GEMM) {
            li = (int)i;
            break;
        }
    if (li < 0) return fail(GAO_EINVAL, "program has no GEMM loop");
    if (p->verdict[(size_t)li] != GAO_OFFLOAD_OK) return fail(GAO_EINVAL, "the program's GEMM loop is not offloadable");
    const uint64_t all = all_genes(gene_length(p));
    double s0 = 0.0;
    gao_status st = prog_run(p, all, GAO_RUN_KEEP_DEVICE, &s0);  // puts the GEMM's inputs on the device
    if (st != GAO_OK) return st;
    const gao_loop& L = p->loops[(size_t)li];
    {  // ... as binary32 also where the run formed them only as the GEMM's planes
        RunCtx R{p, 0.0, false, CpuCtx{p->opts.cpu_threads, 0.0, false}, p->st, false};
        gao_loop_stat dummy{};
        for (int b : {L.ins[0], L.ins[1]})
            if ((st = make_valid(R, b, true, dummy)) != GAO_OK) return st;
    }
    const gao_buffer &A = p->bufs[(size_t)L.ins[0]].d, &B = p->bufs[(size_t)L.ins[1]].d;
    float* C = (float*)p->bufs[(size_t)L.outs[0]].dev;
    const float* C0 = L.ins[2] >= 0 ? (const float*)p->bufs[(size_t)L.ins[2]].dev : C;
    const float beta = L.ins[2] >= 0 ? (float)L.beta : 0.0f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GAO_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    int* d_err = (int*)(p->arena + p->lay.err_off);
    // with fused chains the kernel that runs under the all-GPU gene carries the chain in its
    // epilogue, so that is the one timed (its D, E, row sums and norm are formed again by
    // the next run)
    Chain ch;
    TcFuse fz{};
    const bool fused = find_chain(p, li, loop_mask_of(p, all), gene_fuses(p, all), &ch);
    if (fused) {
        auto dptr = [&](int bi) { return (float*)p->bufs[(size_t)bi].dev; };
        const gao_loop &X = p->loops[(size_t)ch.axpy], &T = p->loops[(size_t)ch.transpose];
        fz = TcFuse{dptr(X.ins[1]), dptr(X.outs[0]), dptr(T.outs[0]),
                    ch.frob >= 0 ? (double*)p->bufs[(size_t)p->loops[(size_t)ch.frob].outs[0]].dev : nullptr,
                    (float)X.alpha, 0, ch.rowsum >= 0 ? dptr(p->loops[(size_t)ch.rowsum].outs[0]) : nullptr};
    }
    auto time_cfg = [&](int kchunk, int tile_cfg, double* ms) -> gao_status {
        std::vector<double> v;
        // a configuration whose kernel raised the error word (a bounded wait expired) fails
        // the tuning with GAO_EDEVICE instead of being scored by its cut-off time
        cudaError_t ze = cudaMemsetAsync(d_err, 0, sizeof(int), p->st);
        if (ze != cudaSuccess) return cuda_fail(ze, "cudaMemsetAsync(err)");
        for (int r = 0; r < 6; ++r) {
            TcEvents ev{e0, e1, 0};
            std::string why;
            cudaError_t e = launch_gemm_tc(prec, C, (const float*)p->bufs[(size_t)L.ins[0]].dev,
                                           (const float*)p->bufs[(size_t)L.ins[1]].dev, C0, A.rows, B.cols, A.cols,
                                           (float)L.alpha, beta, kchunk, tile_cfg, p->arena + p->lay.tc_off,
                                           p->lay.tc_bytes, d_err, p->st, ev, &why, fused ? &fz : nullptr);
            if (e != cudaSuccess) return why.empty() ? cuda_fail(e, "autotune launch") : fail(GAO_EINVAL, why);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return cuda_fail(e, "autotune sync");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r > 0) v.push_back(t);  // first launch warms up
        }
        cudaError_t ce2 = cudaMemcpyAsync(p->h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, p->st);
        if (ce2 == cudaSuccess) ce2 = cudaStreamSynchronize(p->st);
        if (ce2 != cudaSuccess) return cuda_fail(ce2, "autotune error word");
        if (*p->h_err != 0)
            return fail(GAO_EDEVICE, "autotune: the GEMM raised device error " + std::to_string(*p->h_err) +
                                         " under K chunk " + std::to_string(kchunk) + ", tile configuration " +
                                         std::to_string(tile_cfg));
        std::sort(v.begin(), v.end());
        *ms = v[v.size() / 2];
        return GAO_OK;
    };
    double def_ms = 0.0;
    st = time_cfg(p->opts.kchunk, p->opts.tile_cfg, &def_ms);
    int evals = 0;
    if (st == GAO_OK) {
        TimeFn fn = [&](uint64_t g, double* t) {
            int kc = 0, tc = 0;
            autotune_decode(prec, g, &kc, &tc);
            double ms = 0.0;
            gao_status s2 = time_cfg(kc, tc, &ms);
            *t = ms * 1e-3;
            ++evals;
            return s2;
        };
        gao_ga_result res{};
        st = ga_core(kAutotuneBits, *params, fn, &res);
        if (st == GAO_OK) {
            // the configuration in place stays unless the GA found a faster one
            int kc = p->opts.kchunk, tc = p->opts.tile_cfg;
            double best_ms = def_ms;
            if (res.best_s * 1e3 < def_ms) {
                autotune_decode(prec, res.best_mask, &kc, &tc);
                best_ms = res.best_s * 1e3;
            }
            p->opts.kchunk = kc;
            p->opts.tile_cfg = tc;
            drop_graphs(p);
            p->cache.clear();  // times measured under the old configuration
            out->kchunk = kc;
            out->tile_cfg = tc;
            out->best_ms = best_ms;
            out->default_ms = def_ms;
            out->evaluations = evals;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// ---- C ABI: misc ------------------------------------------------------------------------------

extern "C" const char* gao_last_error(void) { return t_err.c_str(); }

extern "C" const char* gao_version(void) { return "gaoffload 0.1 (sm_103a)"; }

extern "C" gao_status gao_selftest_device_wait(double limit_s, void* stream) {
    gao_status s = check_device(nullptr);
    if (s != GAO_OK) return s;
    if (!(limit_s > 0.0 && limit_s <= 10.0)) return fail(GAO_EINVAL, "limit_s must be in (0, 10]");
    cudaStream_t st = (cudaStream_t)stream;
    int* d = nullptr;
    GAO_CUDA_TRY(cudaMalloc((void**)&d, 2 * sizeof(int)));
    int h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = launch_wait_selftest(d, d + 1, limit_s, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    if (h[1] == DEV_WAIT_TIMEOUT) return fail(GAO_ETIMEOUT, "device wait expired after the limit (expected)");
    return fail(GAO_EDEVICE, "device wait returned without expiring");
}
