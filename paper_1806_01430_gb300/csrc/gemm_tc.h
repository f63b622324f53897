// Tensor-core GEMM interface shared by the runtime and the batch executor.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace gao {

// Epilogue of one GEMM: C = alpha * acc + beta * C0 (FP8: the MMAs apply the block scales).
struct EpiArgs {
    float* C;
    const float* C0;
    int M, N;
    float alpha, beta;
    int vec;           // C, C0 16-byte aligned and N % 4 == 0
    const float* sa;   // FP8: A's scale-factor blocks [Mp / 128][kbs][512 bytes] (read as bytes)
    const float* sb;   // FP8: B's scale-factor blocks [Np / 128][kbs][512 bytes] (read as bytes)
    int kbs, sb_ld;
    // Fused loop chain (fuse != 0): D = C + alpha2 * X written row-major like C, E = D^T
    // written with row stride M, and per-warp binary64 partials of sum(D^2) (8 per tile,
    // at frob_part[tile * 8 + epilogue warp]).  D, E, X must not alias C, C0 or each other.
    const float* X;
    float* D;
    float* E;
    double* frob_part;
    float alpha2;
    int fuse;
    int64_t ldE;       // row stride of E (0: M); a row block writes columns of a larger E
    // Fused row sums of E (= column sums of D): each warp writes, for each of its columns j,
    // the value of its 32-row block in the fixed row-sum order at
    // rsum_part[(row0 / 32) * ldR + j]; null when the chain has no row-sum loop.
    float* rsum_part;
    int64_t ldR;
    int64_t ldc;  // row stride of C, C0, X and D (0: N); a column range of a wider C
};

// Loops of a chain GEMM -> AXPY (D = C + alpha2 X) -> TRANSPOSE (E = D^T) [-> ROWSUM of E]
// [-> FROBENIUS of E] done inside the GEMM's epilogue.
struct TcFuse {
    const float* X;
    float* D;
    float* E;
    double* frob_out;  // nullptr: no Frobenius loop in the chain
    float alpha2;
    int64_t ldE;       // row stride of E (0: the launch's M)
    float* rowsum_out;  // nullptr: no row-sum loop in the chain; else the N row sums of E
};

// One problem of a grouped launch: its operand planes' TMA descriptors and epilogue.
// tile_start is the index of its first CTA in the launch (prefix sum of tiles).
struct alignas(128) TcProblem {
    CUtensorMap ta, tb;
    EpiArgs ep;
    int Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, tile_start, group, pf_kb;
    // Optional time span of the problem inside the launch (global timer, ns): the producer
    // lowers *span_start to the time it starts loading each of the problem's tiles, every
    // epilogue warp raises *span_end to the time it has stored its part of a tile.  Null:
    // not recorded.  The caller sets *span_start = ~0 and *span_end = 0 before the launch.
    unsigned long long* span_start;
    unsigned long long* span_end;
};

// Raster group (row tiles per CTA group) encoded in bits 4-7 of a tile configuration
// id as a power of two; 0 selects the default of 16.
inline int tc_group_of(int tile_cfg) {
    const int g = (tile_cfg >> 4) & 15;
    return g == 0 ? 16 : (1 << g);
}

// Bit 2 of a tile configuration id: the producer also pulls each operand tile into L2
// kL2PrefetchKb K blocks before its load (a hint: it changes no value).  It pays where the
// operand re-reads of one wave of tiles fit in L2 but miss it (BF16x6 at n = 4096 on
// GB300: 5% off the GEMM) and costs where they do not, so the autotuner decides it.
constexpr int kL2PrefetchKb = 4;
inline int tc_prefetch_of(int tile_cfg) { return (tile_cfg & 4) ? kL2PrefetchKb : 0; }

// Looks up the driver's tensor-map encoder (once); false with a reason if unavailable.
bool tc_available(std::string* why);

// Split/quantise the operands of one GEMM into `scratch` (kernels on st) and describe it
// in *prob for a grouped launch (tile_start left 0).  *launches counts kernels issued.
// With `fuse`, the problem's epilogue also runs the chain (D, E, norm partials and row-sum
// block values in the problem's scratch); tc_finalize_chain then reduces the partials.
cudaError_t tc_prepare(int prec, float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                       int64_t K, float alpha, float beta, int kchunk, int tile_cfg, void* scratch,
                       size_t scratch_bytes, cudaStream_t st, TcProblem* prob, int* launches, std::string* why,
                       const TcFuse* fuse = nullptr);

// Turns a problem made by tc_prepare (same prec, shapes and scratch, BF16 variants) into
// one whose epilogue runs the chain `fuse`, on the host: the operand planes are shared, so
// the same split serves the plain problem and every chain shape.
void tc_attach_chain(int prec, int64_t M, int64_t N, int64_t K, void* scratch, const TcFuse& fuse, TcProblem* prob);

// After a grouped launch with a fused chain: the norm from the per-warp partials and the
// row sums from the block values of one problem (kernels on st).
cudaError_t tc_finalize_chain(int prec, int64_t M, int64_t N, int64_t K, void* scratch, const TcFuse& fuse,
                              cudaStream_t st, int* launches);

// One launch over nprob problems whose table (tile_start set, in order) is at d_probs
// in device memory; every problem must come from tc_prepare with the same prec and
// the same chunked-ness.  total_tiles = sum of tiles_m * tiles_n.  With total_tiles
// = 0 it only prepares the kernel (shared-memory attribute), launching nothing.
cudaError_t tc_launch_grouped(int prec, bool chunked, const TcProblem* d_probs, int nprob, int total_tiles, int* err,
                              cudaStream_t st);

}  // namespace gao
