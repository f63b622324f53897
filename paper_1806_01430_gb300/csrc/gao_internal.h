// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gao.h"

namespace gao {

// ---- error reporting --------------------------------------------------------
void set_error(const std::string& msg);
gao_status fail(gao_status st, const std::string& msg);
gao_status cuda_fail(cudaError_t e, const char* what);

#define GAO_CUDA_TRY(expr)                                             \
    do {                                                               \
        cudaError_t _e = (expr);                                       \
        if (_e != cudaSuccess) return ::gao::cuda_fail(_e, #expr);     \
    } while (0)

// Device error word codes (written by kernels, read by the host after a run).
enum : int {
    DEV_OK = 0,
    DEV_WAIT_TIMEOUT = 1,  // a bounded mbarrier / flag wait expired
    DEV_BAD_SHAPE = 2,     // a kernel saw a shape it cannot handle
};

// ---- SplitMix64 counter hash (Steele, Lea & Flood 2014) -----------------------
// gamma is the golden-ratio increment; the finaliser is the published
// xor-shift-multiply mix (shifts 30, 27, 31).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t sm64_hash(uint64_t state) { return sm64_mix(state + 0x9E3779B97F4A7C15ULL); }

// Element key of the INIT loop: seed bits 40.., buffer id bits 36..39, index bits 0..35.
__host__ __device__ inline uint64_t init_key(uint64_t seed, uint32_t buf, uint64_t idx) {
    return (seed << 40) ^ ((uint64_t)buf << 36) ^ idx;
}
// U[-1,1) binary32 value from a 24-bit integer u24: u24 * 2^-23 - 1 (exact).
__host__ __device__ inline float u24_to_value(uint32_t u24) { return (float)((int32_t)u24 - (1 << 23)) * (1.0f / 8388608.0f); }
// Element idx of an INIT buffer: the hash of key idx/2 gives two elements, bits 40..63
// for the even one and bits 16..39 for the odd one.
__host__ __device__ inline float init_value(uint64_t seed, uint32_t buf, uint64_t idx) {
    const uint64_t h = sm64_hash(init_key(seed, buf, idx >> 1));
    return u24_to_value((idx & 1) ? (uint32_t)((h >> 16) & 0xFFFFFFu) : (uint32_t)(h >> 40));
}
// Power-of-two exponent in [-10, 10] of row `row`'s factor for row-scaled inputs:
// round((sum of twelve 24-bit uniforms / 2^24 - 6) * 10/3), in integer arithmetic.
__host__ __device__ inline int row_exponent(uint64_t seed, int64_t row) {
    int64_t s = 0;
    for (int t = 0; t < 12; ++t) s += (int64_t)(sm64_hash(init_key(seed, 15u, (uint64_t)(row * 12 + t))) >> 40);
    const int64_t two24 = 1LL << 24;
    const int64_t num = (s - 6 * two24) * 10, den = 3 * two24;
    int64_t a = 2 * num + den, b = 2 * den;
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;  // floor division (b > 0)
    return (int)(q < -10 ? -10 : (q > 10 ? 10 : q));
}

// Order-preserving key of a binary32 value for max reductions with integer atomics
// (+0 above -0; a NaN with the sign bit clear above +inf, one with it set below -inf): the
// bits with the sign bit set when it is clear, all bits flipped when it is set.  Written as one
// exclusive or with a mask built from the sign bit, not as a choice between the two forms: in
// that form, applied to the result of arithmetic still in registers, the compiled maximum of
// the keys lost NaN values (a NaN pixel of the image pass never reached the column maxima),
// while keys of values loaded from memory were right.  Used identically by the CPU loop.
__host__ __device__ inline uint32_t fmax_key(uint32_t bits) {
    return bits ^ ((0u - (bits >> 31)) | 0x80000000u);
}
__host__ __device__ inline uint32_t fmax_unkey(uint32_t key) {
    return (key & 0x80000000u) ? (key & 0x7FFFFFFFu) : ~key;
}

// ---- device info -------------------------------------------------------------
int sm_count();
// GAO_OK when the current device is an sm_103 GPU (its index in *dev_out when set).
gao_status check_device(int* dev_out);

// ---- kernel launchers (all asynchronous on `st`) -------------------------------
struct ReduceScratch {
    double* partials;   // >= reduce_blocks() doubles
    unsigned* counter;  // one zero-initialised word, reset by the kernel
};
int reduce_blocks();

cudaError_t launch_row_exponents(int8_t* e, int64_t rows, uint64_t seed, cudaStream_t st);
// The outputs of one INIT loop: out[i] = init_value(seed, buf, i), times 2^e_row for an
// output with rowscale (e_row from rowexp, which covers the largest such output's rows).
struct InitOut {
    float* out;
    int64_t rows, cols;
    uint32_t buf;
    int rowscale;
};
struct InitSet {
    InitOut o[GAO_MAX_IO];
    int n;
    uint64_t seed;
    const int8_t* rowexp;
};
cudaError_t launch_init_set(const InitSet& set, cudaStream_t st);
// One INIT output of a grouped launch (no row scaling); start4 is the index of its first
// quadruple in the launch (prefix sum of ceil(rows * cols / 4)), increasing along the table.
struct InitEntry {
    float* out;
    int64_t rows, cols;
    uint64_t seed;
    uint32_t buf;
    int64_t start4;
};
cudaError_t launch_init_group(const InitEntry* d_tab, int n_entries, int64_t total4, cudaStream_t st);
cudaError_t launch_axpy(float* out, const float* x, float alpha, const float* y, int64_t n, cudaStream_t st);
cudaError_t launch_transpose(float* out, const float* in, int64_t rows, int64_t cols, cudaStream_t st);
// Row sums (ROWSUM) follow one fixed order on every path -- the row-sum kernel, the fused
// GEMM chain's block values and the host loop -- so that equal inputs give equal bits
// whatever the gene: a row of length L is cut into blocks of kRowsumBlock = 32 elements
// (elements past L count as +0); a block's value is ((q0 + q4) + (q2 + q6)) + ((q1 + q5) +
// (q3 + q7)) over its quadruples q_m = (x_4m + x_4m+1) + (x_4m+2 + x_4m+3); block p is
// added to accumulator p mod 4 (each starts at +0 and takes its blocks in increasing p);
// the row sum is (u0 + u2) + (u1 + u3).
constexpr int kRowsumBlock = 32;
cudaError_t launch_rowsum(float* out, const float* in, int64_t rows, int64_t cols, cudaStream_t st);
cudaError_t launch_frobenius(double* out, const float* in, int64_t n, ReduceScratch rs, cudaStream_t st);
cudaError_t launch_sum(double* out, const float* in, int64_t n, ReduceScratch rs, cudaStream_t st);
cudaError_t launch_relu(float* out, const float* in, int64_t n, cudaStream_t st);
cudaError_t launch_square(float* out, const float* in, int64_t n, cudaStream_t st);
cudaError_t launch_colmax(float* out, const float* in, int64_t rows, int64_t cols, uint32_t* keys, cudaStream_t st);
// Output rows [row_begin, row_end) of the rows x cols image (row_end < 0: to the last row);
// the image is zero outside its own rows, whatever the range, so a frame formed in row
// ranges gives the same bits as in one launch.
cudaError_t launch_stencil3(float* out, const float* in, int64_t rows, int64_t cols, int preset, cudaStream_t st,
                            int64_t row_begin = 0, int64_t row_end = -1);

// A linear chain of element-wise loops in one pass.  Op o computes kind 0 RELU, 1 SQUARE
// or 2 AXPY (x + alpha y) with x = xa[i] (or the previous op's value when xa is null) and,
// for AXPY, y = yb[i] (or the previous value); the result is stored to out[i] when out is
// set.  The first op reads memory for every operand.
constexpr int kMaxChainOps = 8;
struct EwChainOp {
    int kind;
    float alpha;
    const float* xa;
    const float* yb;
    float* out;
};
struct EwChain {
    int nops;
    int vec;  // set by launch_ew_chain
    int64_t n;
    EwChainOp op[kMaxChainOps];
};
cudaError_t launch_ew_chain(const EwChain& c, cudaStream_t st);
// Reductions of the gradient chain's m formed in the same pass: the sum (binary64, from one
// partial per block of the pass in `part`, added in index order) and the column maxima
// (order-preserving keys in `keys`, one per column, decoded into colmax_out).  Either output
// may be null.  An image may be covered by several row-range launches in row order (the
// strips of a frame that arrives from the host): the first (`first`) clears the keys, each
// writes its partials from part[part_at] on (grad_chain_blocks(its rows, cols) of them), and
// the last (`last`) adds part[0 .. part_at + its own) and decodes the keys.  A single
// launch over the whole image is first and last with part_at = 0, as the defaults say.
struct GradReduce {
    double* sum_out;
    double* part;
    int64_t part_cap;
    float* colmax_out;
    uint32_t* keys;
    int64_t part_at = 0;
    bool first = true, last = true;
};
// Blocks of a gradient-chain pass over `rows` output rows (a launch's row range) of width cols.
int64_t grad_chain_blocks(int64_t rows, int64_t cols);
// The most blocks any gradient-chain launch of width cols has, whatever its row range.
int64_t grad_chain_blocks_max(int64_t cols);
// Gradient chain in one pass: g1, g2 = stencils p1, p2 of `in`; s1 = g1*g1, s2 = g2*g2;
// m = s1 + alpha s2 (swap: s2 + alpha s1).  Null g1/g2/s1/s2 are not written.  With `red`,
// also the sum and / or column maxima of m, and m may then be null (formed for the
// reductions only); *launches counts the kernels issued.
cudaError_t launch_grad_chain(const float* in, int64_t rows, int64_t cols, int p1, int p2, float alpha, bool swap,
                              float* g1, float* g2, float* s1, float* s2, float* m, cudaStream_t st,
                              int64_t row_begin = 0, int64_t row_end = -1, const GradReduce* red = nullptr,
                              int* launches = nullptr);

// The image program's first stencil and the gradient chain on its output in one pass over
// the raw image `in`: B = p0(in), written to bout only if bout is non-null; g1, g2 = stencils
// p1, p2 of B; s1, s2, m and the reductions as launch_grad_chain.  Row ranges, `red` and
// *launches as there, with edge_chain_blocks partials per launch.
cudaError_t launch_edge_chain(const float* in, float* bout, int64_t rows, int64_t cols, int p0, int p1, int p2,
                              float alpha, bool swap, float* g1, float* g2, float* s1, float* s2, float* m,
                              cudaStream_t st, int64_t row_begin = 0, int64_t row_end = -1,
                              const GradReduce* red = nullptr, int* launches = nullptr);
int64_t edge_chain_blocks(int64_t rows, int64_t cols);
int64_t edge_chain_blocks_max(int64_t cols);

// Weights of the 3x3 stencil presets of GAO_LOOP_STENCIL3, row-major over (a, b).
// Every weight is a small integer or a power-of-two fraction, exact in binary32.
#ifdef __CUDACC__
#define GAO_HD __host__ __device__
#else
#define GAO_HD
#endif
GAO_HD constexpr float stencil_preset(int preset, int t) {
    // (1 2 1; 2 4 2; 1 2 1) / 16, (0 1 0; 1 -4 1; 0 1 0), (-1 0 1; -2 0 2; -1 0 1),
    // (-1 -2 -1; 0 0 0; 1 2 1)
    return preset == 0 ? (t == 4 ? 0.25f : (t & 1) ? 0.125f : 0.0625f)
         : preset == 1 ? (t == 4 ? -4.0f : (t & 1) ? 1.0f : 0.0f)
         : preset == 2 ? (float)((t % 3) - 1) * (t / 3 == 1 ? 2.0f : 1.0f)
                       : (float)((t / 3) - 1) * (t % 3 == 1 ? 2.0f : 1.0f);
}
inline bool stencil_weights(int preset, float w[9]) {
    if (preset < 0 || preset > 3) return false;
    for (int t = 0; t < 9; ++t) w[t] = stencil_preset(preset, t);
    return true;
}
cudaError_t launch_wait_selftest(int* flag, int* err, double limit_s, cudaStream_t st);

// FP32 SIMT GEMM: C = alpha*A@B + beta*C0 (C may alias C0).  kchunk: K elements per
// binary32 partial sum (<= 0: one sum over all of K).
cudaError_t launch_gemm_simt(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                             int64_t K, float alpha, float beta, int kchunk, cudaStream_t st);

// Tensor-core GEMM (split operands + tcgen05).  Scratch layout and size are given
// by tc_scratch_bytes; `err` receives DEV_* codes.
// Set while a run is being captured as a CUDA graph: timing events are then recorded as
// graph nodes (external events), so that a replay records them too.
extern thread_local bool g_capturing;
extern thread_local bool g_no_times;  // a run without per-loop timing events (GAO_RUN_NO_LOOP_TIMES)
inline cudaError_t record_timing(cudaEvent_t e, cudaStream_t s) {
    if (g_no_times) return cudaSuccess;
    return g_capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

struct TcEvents {
    cudaEvent_t k0 = nullptr, k1 = nullptr;  // recorded around the MMA kernel if non-null
    int launches = 0;                         // out: kernels launched
    cudaEvent_t planes = nullptr;             // recorded once the operand planes are formed, if non-null
};
size_t tc_scratch_bytes(int prec, int64_t M, int64_t N, int64_t K);
struct TcFuse;
// One row block of a larger GEMM (the split-precision paths): the scratch is laid out for
// m_layout rows (the whole problem), and b_ready says that B's planes are already in it
// (split by an earlier row block of the same problem).  With a fused chain the blocks'
// norm partials go to one array (offset by row_tile0) that the last block reduces.
struct TcPart {
    int64_t m_layout;
    bool b_ready;
    int64_t row_tile0;  // fused chain: 128-row tiles of the problem before this block
    bool last;          // fused chain: the last block (reduces the norm's partials)
    // columns [n_begin, n_end) of C only (n_end < 0: to N; n_begin a multiple of 256; no
    // fused chain): B's planes of those columns are formed unless b_ready
    int64_t n_begin = 0, n_end = -1;
    bool a_ready = false;  // this block's A planes are already formed (an earlier column range)
};
// ready: bit 0, A's bfloat16 planes are already in the scratch (tc_init_planes); bit 1, B's.
cudaError_t launch_gemm_tc(int prec, float* C, const float* A, const float* B, const float* C0, int64_t M,
                           int64_t N, int64_t K, float alpha, float beta, int kchunk, int tile_cfg, void* scratch,
                           size_t scratch_bytes, int* err, cudaStream_t st, TcEvents& ev, std::string* why,
                           const TcFuse* fuse = nullptr, const TcPart* part = nullptr, unsigned ready = 0);
// The bfloat16 planes of operand `which` (0: A, M x K; 1: B, K x N) of that GEMM (same
// precision, shapes, K chunk and tile configuration), formed in its scratch straight from the
// INIT loop's counter hash of buffer `buf` (times 2^e of each row where rowexp is set), with
// the values, splitting and zero padding of INIT followed by the GEMM's own split.
cudaError_t tc_init_planes(int prec, int which, int64_t M, int64_t N, int64_t K, int kchunk, int tile_cfg,
                           uint64_t seed, uint32_t buf, const int8_t* rowexp, void* scratch, size_t scratch_bytes,
                           cudaStream_t st, int* launches);

// Freivalds residual check of C = alpha A B + beta C0 in binary64 (C0 may be null):
// kernels on st; the residual vectors go to rvec (M) / svec (N) when set; *norms_dev
// receives the device address of 16 binary64 values (right form at 0..4: ||r||, ||f||,
// max|r|, max|f|, argmax; left form at 8..12), which residual_from_norms turns into a
// gao_residual once the stream has drained.
size_t gemm_residual_scratch_bytes(int64_t M, int64_t N, int64_t K);
cudaError_t launch_gemm_residual(const float* A, const float* B, const float* C0, const float* C, int64_t M,
                                 int64_t N, int64_t K, double alpha, double beta, const double* x, const double* y,
                                 void* scratch, double* rvec, double* svec, cudaStream_t st, int* launches,
                                 const double** norms_dev);
void residual_from_norms(const double* norms, gao_residual* out);

// ---- CPU loops (binary32, OpenMP) ------------------------------------------------
struct CpuCtx {
    int threads;
    double deadline;  // steady-clock seconds; 0 = none
    bool timed_out;
};
double now_s();
void cpu_init(float* out, int64_t rows, int64_t cols, uint64_t seed, uint32_t buf, bool rowscale, CpuCtx& c);
void cpu_gemm(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N, int64_t K, float alpha,
              float beta, int kchunk, CpuCtx& c);
void cpu_axpy(float* out, const float* x, float alpha, const float* y, int64_t n, CpuCtx& c);
void cpu_transpose(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c);
void cpu_rowsum(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c);
double cpu_frobenius(const float* in, int64_t n, CpuCtx& c);
double cpu_sum(const float* in, int64_t n, CpuCtx& c);
void cpu_relu(float* out, const float* in, int64_t n, CpuCtx& c);
void cpu_square(float* out, const float* in, int64_t n, CpuCtx& c);
void cpu_colmax(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c);
void cpu_stencil3(float* out, const float* in, int64_t rows, int64_t cols, int preset, CpuCtx& c);
void cpu_recurrence(float* out, const float* in, int64_t rows, int64_t cols, float alpha, CpuCtx& c);
void cpu_find(double* out, const float* in, int64_t rows, int64_t cols, float threshold, CpuCtx& c);

}  // namespace gao
