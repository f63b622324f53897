// Program state shared by the runtime's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <unordered_map>
#include <vector>

#include "gao_internal.h"

namespace gao {

struct BufState {
    gao_buffer d;
    size_t bytes = 0;
    char* dev = nullptr;
    void* host = nullptr;  // pinned host copy: the library's mirror, or caller memory bound to it
    void* own_host = nullptr;  // the library's mirror (freed with the program)
    bool registered = false;   // host is caller memory the library page-locked (cudaHostRegister)
    bool vh = false, vd = false;
    bool input_set = false;
    // Formed by an INIT loop straight into the bfloat16 planes of the one GEMM that reads it
    // (gen_for): the binary32 array holds nothing (vd and vh false) until something else
    // needs it, which then runs slot gen_slot of INIT loop gen_loop for it alone.
    int gen_loop = -1, gen_slot = -1, gen_for = -1;
};

struct CacheEntry {
    double seconds;
    gao_status status;
};

struct Layout {
    std::vector<size_t> buf_off;
    size_t err_off = 0, partial_off = 0, counter_off = 0, keys_off = 0, rowexp_off = 0, tc_off = 0;
    size_t tc_bytes = 0, keys_bytes = 0, rowexp_bytes = 0;
    size_t resid_off = 0, resid_bytes = 0;  // GEMM residual check: x, y, then its scratch
    size_t chainpart_off = 0, chainpart_bytes = 0;  // gradient chain's fused sum: block partials
    size_t total = 0;
};

}  // namespace gao

// A run of one all-GPU gene captured as a CUDA graph, and the host-side state it leaves.
struct GraphEntry {
    int runs = 0;
    bool failed = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint8_t> vh, vd;
    std::vector<gao_loop_stat> stats;
    std::vector<uint8_t> ev_used;
};

struct gao_prog {
    std::vector<gao_loop> loops;
    std::vector<gao::BufState> bufs;
    gao_opts opts{};
    int device = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    char* arena = nullptr;      // 1024-byte aligned (tensor-core scratch, TMA maps)
    char* arena_raw = nullptr;  // the library's own allocation (freed with the program)
    bool own_arena = false;
    gao::Layout lay;
    int* h_err = nullptr;  // pinned
    std::vector<gao_loop_stat> stats;
    std::vector<cudaEvent_t> ev;   // 6 per loop: copy0, copy1, loop0, loop1, kern0, kern1
    std::vector<uint8_t> ev_used;  // bit 0 copies, bit 1 loop, bit 2 kernel
    std::unordered_map<uint64_t, gao::CacheEntry> cache;
    bool dirty_stream = false;  // a previous run left work in flight
    bool stats_pending = false; // the last run's event times are not read yet
    cudaStream_t cst = nullptr;           // copy stream of the copy/compute overlap
    std::vector<cudaEvent_t> pipe_ev;     // its events: fork, B landed, one per row block
    cudaStream_t ost = nullptr;           // device-to-host stream: a GEMM's C rows as blocks finish
    std::vector<cudaEvent_t> out_ev;      // one per row block (block done), then the join
    cudaStream_t st2 = nullptr;           // second compute stream: every other row block's GEMM
    std::vector<cudaEvent_t> cmp_ev;      // its fork, B's planes formed, its join
    std::vector<int8_t> verdict;  // gao_offload of every loop
    std::vector<int> gene_loop;   // gene bit k -> index of the k-th offloadable loop
    std::unordered_map<uint64_t, GraphEntry> graphs;  // key: gene * 8 + run flags (KEEP_DEVICE, NO_LOOP_TIMES)
};

namespace gao {

constexpr int kMaxRowBlocks = 4;                 // row blocks of an overlapped GEMM loop
constexpr int kMaxColParts = 2;                  // column ranges of its first row block
constexpr size_t kPipelineMinBytes = 16u << 20;  // smallest A worth overlapping

// One execution of a program (or of a batch of programs sharing a stream).
struct RunCtx {
    gao_prog* p;
    double deadline;
    bool timed_out;
    CpuCtx cpu;
    cudaStream_t st;    // stream the GPU work and copies go to
    bool events;        // record per-loop CUDA events (not while capturing a graph)
};

gao_status make_valid(RunCtx& R, int b, bool on_gpu, gao_loop_stat& stat);
std::vector<int> loop_inputs(const gao_loop& L);
std::vector<int> loop_outputs(const gao_loop& L);
gao_status run_gpu_loop(RunCtx& R, int li);
gao_status run_cpu_loop(RunCtx& R, int li);
gao_status stream_wait(cudaStream_t st, double deadline, bool* timed_out, double hard_cap_s = 300.0);
gao_status check_device(int* dev_out);
// Parallelisability of one loop (gao_offload), and the loop placement of a gene.
int offload_verdict(const gao_loop& L);
uint64_t loop_mask_of(const gao_prog* p, uint64_t gene);
inline int gene_length(const gao_prog* p) {
    return (int)p->gene_loop.size() + (p->opts.fuse_chains == GAO_FUSE_GENE ? 1 : 0);
}
// Whether a run under `gene` fuses loop chains.
inline bool gene_fuses(const gao_prog* p, uint64_t gene) {
    if (p->opts.fuse_chains == GAO_FUSE_ON) return true;
    return p->opts.fuse_chains == GAO_FUSE_GENE && ((gene >> p->gene_loop.size()) & 1);
}
inline uint64_t all_genes(int a) { return a >= 64 ? ~0ULL : ((1ULL << a) - 1); }
void drop_graphs(gao_prog* p);

// Loops that run in the GEMM's epilogue: GEMM (loop li) -> AXPY -> TRANSPOSE [-> ROWSUM of E]
// [-> FROBENIUS of E], indices of the later loops (-1: not in the chain).
struct Chain {
    int axpy = -1, transpose = -1, rowsum = -1, frob = -1;
};
// The chain that starts at GEMM loop li under the loop mask (bit i: loop i on the GPU),
// false when there is none (fusion off, a loop of it on the host, a precision without it).
bool find_chain(const gao_prog* p, int li, uint64_t mask, bool fuse, Chain* ch);

}  // namespace gao
