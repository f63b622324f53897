// Memory-bound loops of the program on the GPU: INIT, AXPY (scale-add), TRANSPOSE,
// ROWSUM, FROBENIUS, SUM, RELU, SQUARE, COLMAX, STENCIL3.
//
// All kernels read and write row-major binary32 with 128-bit accesses where the
// shape allows (element count or row length a multiple of 4), grid-stride over a
// grid sized in multiples of the SM count, and keep every reduction in a fixed
// order so that results are identical from run to run (no floating-point atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "gao_internal.h"

namespace gao {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

int grid_for(int64_t work_items) {
    const int64_t cap = (int64_t)sm_count() * kBlocksPerSm;
    int64_t g = (work_items + kThreads - 1) / kThreads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ---- INIT ---------------------------------------------------------------------------

__global__ void row_exponents_kernel(int8_t* e, int64_t rows, uint64_t seed) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        e[r] = (int8_t)row_exponent(seed, r);
}

constexpr int kInitQuads = 4;  // quadruples per thread and trip in the plain INIT loop

// Elements 4q .. 4q + 3 of an INIT buffer whose element keys are khi ^ index (the hashes of
// keys 2q and 2q + 1 give them).
__device__ __forceinline__ float4 init_quad(uint64_t khi, uint64_t q) {
    const uint64_t h0 = sm64_hash(khi ^ (2 * q));
    const uint64_t h1 = sm64_hash(khi ^ (2 * q + 1));
    return make_float4(u24_to_value((uint32_t)(h0 >> 40)), u24_to_value((uint32_t)((h0 >> 16) & 0xFFFFFFu)),
                       u24_to_value((uint32_t)(h1 >> 40)), u24_to_value((uint32_t)((h1 >> 16) & 0xFFFFFFu)));
}

// out[i] = init_value(seed, buf, i) (times 2^e_row).  Four consecutive elements per
// thread and iteration, stored as one float4 (a ragged last quadruple element by element).
__device__ __forceinline__ void init_body(float* __restrict__ out, int64_t rows, int64_t cols, uint64_t seed,
                                          uint32_t buf, const int8_t* __restrict__ rowexp) {
    const int64_t n = rows * cols;
    if (!rowexp && aligned16(out)) {
        // no row factors: kInitQuads independent quadruples per trip (their hashes in flight
        // together), then the ragged tail element by element
        const uint64_t khi = init_key(seed, buf, 0);
        const int64_t nq = n / 4, nth = (int64_t)gridDim.x * blockDim.x;
        float4* o4 = reinterpret_cast<float4*>(out);
        int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        for (; q + (kInitQuads - 1) * nth < nq; q += kInitQuads * nth) {
            float4 v[kInitQuads];
#pragma unroll
            for (int u = 0; u < kInitQuads; ++u) v[u] = init_quad(khi, (uint64_t)(q + u * nth));
#pragma unroll
            for (int u = 0; u < kInitQuads; ++u) o4[q + u * nth] = v[u];
        }
        for (; q < nq; q += nth) o4[q] = init_quad(khi, (uint64_t)q);
        const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (t < n - 4 * nq) out[4 * nq + t] = init_value(seed, buf, (uint64_t)(4 * nq + t));
        return;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    // a full quadruple is one float4 store; with row scaling only when no row ends inside it
    const bool vec = aligned16(out) && (!rowexp || cols % 4 == 0);
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i < n; i += stride) {
        if (vec && i + 3 < n) {
            // i is a multiple of 4: two hashes give the four elements
            const uint64_t h0 = sm64_hash(init_key(seed, buf, (uint64_t)i >> 1));
            const uint64_t h1 = sm64_hash(init_key(seed, buf, ((uint64_t)i >> 1) + 1));
            float4 v;
            v.x = u24_to_value((uint32_t)(h0 >> 40));
            v.y = u24_to_value((uint32_t)((h0 >> 16) & 0xFFFFFFu));
            v.z = u24_to_value((uint32_t)(h1 >> 40));
            v.w = u24_to_value((uint32_t)((h1 >> 16) & 0xFFFFFFu));
            if (rowexp) {
                const int e = rowexp[i / cols];
                v.x = ldexpf(v.x, e);
                v.y = ldexpf(v.y, e);
                v.z = ldexpf(v.z, e);
                v.w = ldexpf(v.w, e);
            }
            *reinterpret_cast<float4*>(out + i) = v;
        } else {
            for (int q = 0; q < 4 && i + q < n; ++q) {
                float v = init_value(seed, buf, (uint64_t)(i + q));
                if (rowexp) v = ldexpf(v, rowexp[(i + q) / cols]);
                out[i + q] = v;
            }
        }
    }
}

// INIT of many programs in one launch (a batch's INIT phase): the quadruples of all
// entries form one index space, entry e owning [start4[e], start4[e+1]); a thread finds its
// first entry by binary search and then moves forward with its index.  Each element is
// formed exactly as init_body forms it.
__global__ void init_group_kernel(const InitEntry* __restrict__ tab, int n_entries, int64_t total4) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= total4) return;
    int lo = 0, hi = n_entries - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].start4 <= g) lo = mid;
        else hi = mid - 1;
    }
    // the current entry's fields stay in registers until the index passes its end
    int e = lo;
    float* out = nullptr;
    int64_t cols = 0, n = 0, first = 0, next = 0;
    uint64_t seed = 0;
    uint32_t buf = 0;
    bool vec = false;
    auto load = [&](int k) {
        out = tab[k].out;
        cols = tab[k].cols;
        n = tab[k].rows * cols;
        seed = tab[k].seed;
        buf = tab[k].buf;
        first = tab[k].start4;
        next = k + 1 < n_entries ? tab[k + 1].start4 : total4;
        vec = aligned16(out);  // no row scaling: any full quadruple is one float4
    };
    load(e);
    for (; g < total4; g += stride) {
        while (g >= next) load(++e);
        const int64_t i = (g - first) * 4;
        if (vec && i + 3 < n) {
            const uint64_t h0 = sm64_hash(init_key(seed, buf, (uint64_t)i >> 1));
            const uint64_t h1 = sm64_hash(init_key(seed, buf, ((uint64_t)i >> 1) + 1));
            float4 v;
            v.x = u24_to_value((uint32_t)(h0 >> 40));
            v.y = u24_to_value((uint32_t)((h0 >> 16) & 0xFFFFFFu));
            v.z = u24_to_value((uint32_t)(h1 >> 40));
            v.w = u24_to_value((uint32_t)((h1 >> 16) & 0xFFFFFFu));
            *reinterpret_cast<float4*>(out + i) = v;
        } else {
            for (int q = 0; q < 4 && i + q < n; ++q) out[i + q] = init_value(seed, buf, (uint64_t)(i + q));
        }
    }
}

// Every output of one INIT loop in one launch, one after the other (the output index is
// a compile-time constant after unrolling, so the set stays in parameter space).
__global__ void init_set_kernel(const __grid_constant__ InitSet set) {
#pragma unroll
    for (int k = 0; k < GAO_MAX_IO; ++k)
        if (k < set.n)
            init_body(set.o[k].out, set.o[k].rows, set.o[k].cols, set.seed, set.o[k].buf,
                      set.o[k].rowscale ? set.rowexp : nullptr);
}

// ---- element-wise -------------------------------------------------------------------

enum class Ew { Axpy, Relu, Square };

template <Ew OP>
__device__ __forceinline__ float ew_apply(float x, float y, float alpha) {
    if constexpr (OP == Ew::Axpy) return fmaf(alpha, y, x);  // x + alpha*y, one rounding
    else if constexpr (OP == Ew::Relu) return x > 0.0f ? x : 0.0f;
    else return x * x;
}

template <Ew OP>
__global__ void ew_kernel(float* __restrict__ out, const float* __restrict__ x, const float* __restrict__ y,
                          float alpha, int64_t n) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const bool vec = aligned16(out) && aligned16(x) && (y == nullptr || aligned16(y));
    int64_t nvec = vec ? n / 4 : 0;
    if (vec) {
        const float4* x4 = reinterpret_cast<const float4*>(x);
        const float4* y4 = reinterpret_cast<const float4*>(y);
        float4* o4 = reinterpret_cast<float4*>(out);
        // two independent 16-byte loads per operand in flight per thread
        int64_t i = tid;
        for (; i + nthreads < nvec; i += 2 * nthreads) {
            float4 a0 = x4[i], a1 = x4[i + nthreads];
            float4 b0 = make_float4(0, 0, 0, 0), b1 = b0;
            if (OP == Ew::Axpy) {
                b0 = y4[i];
                b1 = y4[i + nthreads];
            }
            float4 r0, r1;
            r0.x = ew_apply<OP>(a0.x, b0.x, alpha);
            r0.y = ew_apply<OP>(a0.y, b0.y, alpha);
            r0.z = ew_apply<OP>(a0.z, b0.z, alpha);
            r0.w = ew_apply<OP>(a0.w, b0.w, alpha);
            r1.x = ew_apply<OP>(a1.x, b1.x, alpha);
            r1.y = ew_apply<OP>(a1.y, b1.y, alpha);
            r1.z = ew_apply<OP>(a1.z, b1.z, alpha);
            r1.w = ew_apply<OP>(a1.w, b1.w, alpha);
            o4[i] = r0;
            o4[i + nthreads] = r1;
        }
        for (; i < nvec; i += nthreads) {
            float4 a0 = x4[i];
            float4 b0 = make_float4(0, 0, 0, 0);
            if (OP == Ew::Axpy) b0 = y4[i];
            float4 r0;
            r0.x = ew_apply<OP>(a0.x, b0.x, alpha);
            r0.y = ew_apply<OP>(a0.y, b0.y, alpha);
            r0.z = ew_apply<OP>(a0.z, b0.z, alpha);
            r0.w = ew_apply<OP>(a0.w, b0.w, alpha);
            o4[i] = r0;
        }
    }
    for (int64_t i = nvec * 4 + tid; i < n; i += nthreads)
        out[i] = ew_apply<OP>(x[i], OP == Ew::Axpy ? y[i] : 0.0f, alpha);
}

// ---- element-wise chains ---------------------------------------------------------------

// Consecutive element-wise loops (RELU, SQUARE, AXPY) over the same shape in one pass.
// The chain is linear: every loop after the first reads the previous loop's value (held
// in registers) and at most one other buffer from memory; each value is formed with the
// separate loop's operation, and written only where `out` is set.
__global__ void ew_chain_kernel(EwChain c) {
    const int64_t n = c.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i < n; i += stride) {
        float cur[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const bool vec = c.vec != 0 && i + 4 <= n;  // a ragged last quadruple element by element
        const int w = vec ? 4 : (int)(n - i < 4 ? n - i : 4);
#pragma unroll
        for (int o = 0; o < kMaxChainOps; ++o) {
            if (o >= c.nops) break;
            const EwChainOp& op = c.op[o];
            float x[4], y[4];
            auto fetch = [&](const float* src, float* dst) {
                if (vec) {
                    const float4 v = *reinterpret_cast<const float4*>(src + i);
                    dst[0] = v.x, dst[1] = v.y, dst[2] = v.z, dst[3] = v.w;
                } else {
                    for (int q = 0; q < 4; ++q) dst[q] = q < w ? src[i + q] : 0.0f;
                }
            };
            if (op.xa) fetch(op.xa, x);
            else for (int q = 0; q < 4; ++q) x[q] = cur[q];
            if (op.kind == 2) {  // AXPY: x + alpha y
                if (op.yb) fetch(op.yb, y);
                else for (int q = 0; q < 4; ++q) y[q] = cur[q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cur[q] = op.kind == 0 ? ew_apply<Ew::Relu>(x[q], 0.0f, 0.0f)
                       : op.kind == 1 ? ew_apply<Ew::Square>(x[q], 0.0f, 0.0f)
                                      : ew_apply<Ew::Axpy>(x[q], y[q], op.alpha);
            if (op.out) {
                if (vec) {
                    *reinterpret_cast<float4*>(op.out + i) = make_float4(cur[0], cur[1], cur[2], cur[3]);
                } else {
                    for (int q = 0; q < w; ++q) op.out[i + q] = cur[q];
                }
            }
        }
    }
}

// ---- TRANSPOSE -------------------------------------------------------------------------

// 64x64 tile through shared memory; 16-byte loads along input rows and 16-byte
// stores along output rows.  Needs rows % 4 == 0 and cols % 4 == 0.
__global__ void __launch_bounds__(256) transpose_vec_kernel(float* __restrict__ out, const float* __restrict__ in,
                                                            int64_t rows, int64_t cols) {
    __shared__ float tile[64][65];
    const int t = threadIdx.x;
    const int c4 = t & 15, r = t >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t gr = r0 + r + 16 * k, gc = c0 + 4 * c4;
        float4 v = make_float4(0, 0, 0, 0);
        if (gr < rows && gc < cols) v = *reinterpret_cast<const float4*>(in + gr * cols + gc);
        tile[r + 16 * k][4 * c4 + 0] = v.x;
        tile[r + 16 * k][4 * c4 + 1] = v.y;
        tile[r + 16 * k][4 * c4 + 2] = v.z;
        tile[r + 16 * k][4 * c4 + 3] = v.w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int orow = r + 16 * k;  // output row = input column c0 + orow
        const int64_t gr = c0 + orow, gc = r0 + 4 * c4;
        if (gr < cols && gc < rows) {
            float4 v;
            v.x = tile[4 * c4 + 0][orow];
            v.y = tile[4 * c4 + 1][orow];
            v.z = tile[4 * c4 + 2][orow];
            v.w = tile[4 * c4 + 3][orow];
            *reinterpret_cast<float4*>(out + gr * rows + gc) = v;
        }
    }
}

// 32x32 tile, scalar accesses, any shape.
__global__ void __launch_bounds__(256) transpose_scalar_kernel(float* __restrict__ out, const float* __restrict__ in,
                                                               int64_t rows, int64_t cols) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = ty; k < 32; k += 8) {
        const int64_t gr = r0 + k, gc = c0 + tx;
        if (gr < rows && gc < cols) tile[k][tx] = in[gr * cols + gc];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t gr = c0 + k, gc = r0 + tx;  // output (cols x rows)
        if (gr < cols && gc < rows) out[gr * rows + gc] = tile[tx][k];
    }
}

// ---- ROWSUM ------------------------------------------------------------------------------

// Quadruple value of elements [i0, i0 + 4) of a row of length cols (+0 past the end).
__device__ __forceinline__ float row_quad(const float* row, int64_t i0, int64_t cols, bool vec) {
    if (vec) {  // cols % 4 == 0: a quadruple is wholly inside or wholly past the row
        if (i0 >= cols) return 0.0f;
        const float4 a = *reinterpret_cast<const float4*>(row + i0);
        return (a.x + a.y) + (a.z + a.w);
    }
    float x[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) x[t] = i0 + t < cols ? row[i0 + t] : 0.0f;
    return (x[0] + x[1]) + (x[2] + x[3]);
}

// One warp per row, in the fixed row-sum order: a 128-element chunk holds four 32-element
// blocks; lane l takes quadruple l of the chunk, so lanes 8b..8b+7 hold block b's eight
// quadruples and a three-step butterfly leaves the block's value in lane 8b, which adds it
// to its accumulator (lane 8b keeps accumulator b).  Eight chunks' loads are in flight.
__global__ void rowsum_kernel(float* __restrict__ out, const float* __restrict__ in, int64_t rows, int64_t cols) {
    constexpr int kAhead = 8;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool vec = (cols % 4 == 0) && aligned16(in);
    const int64_t nblk = (cols + kRowsumBlock - 1) / kRowsumBlock;
    const int64_t nchunks = (cols + 127) / 128;
    for (int64_t r = warp; r < rows; r += nwarps) {
        const float* row = in + r * cols;
        float u = 0.0f;
        for (int64_t c0 = 0; c0 < nchunks; c0 += kAhead) {
            float q[kAhead];
#pragma unroll
            for (int k = 0; k < kAhead; ++k) q[k] = row_quad(row, (c0 + k) * 128 + 4 * lane, cols, vec);
#pragma unroll
            for (int k = 0; k < kAhead; ++k) {
                float s = q[k];
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                if ((c0 + k) * 4 + (lane >> 3) < nblk) u += s;  // blocks past the row are not added
            }
        }
        u += __shfl_xor_sync(0xffffffffu, u, 16);
        u += __shfl_xor_sync(0xffffffffu, u, 8);
        if (lane == 0) out[r] = u;
    }
}

// ---- FROBENIUS / SUM -------------------------------------------------------------------------

// Neumaier-compensated binary32 accumulation: s + c carries the running sum with an
// error of about 2u times the sum of magnitudes, independent of the term count.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
}

template <bool SQUARES>
__device__ __forceinline__ float part4(const float4 a) {
    // squares: each rounded once, then a pairwise tree: at most 3u relative (positive terms)
    return SQUARES ? (a.x * a.x + a.y * a.y) + (a.z * a.z + a.w * a.w) : (a.x + a.y) + (a.z + a.w);
}

// Each thread adds binary32 partials of one float4 into a compensated binary32 sum
// (four independent 16-byte loads in flight per iteration); threads are combined in
// binary64 by a fixed tree per block, and the last block to finish adds the block
// partials in index order.  Binary64 arithmetic stays out of the streaming loop: its
// rate on this part is far below what HBM bandwidth needs.
template <bool SQUARES>
__global__ void __launch_bounds__(256) reduce64_kernel(double* __restrict__ out, const float* __restrict__ in,
                                                       int64_t n, double* __restrict__ partials,
                                                       unsigned* __restrict__ counter) {
    __shared__ double wsum[8];
    __shared__ bool last;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    float s = 0.0f, c = 0.0f;
    const bool vec = aligned16(in);
    const int64_t nvec = vec ? n / 4 : 0;
    if (vec) {
        const float4* in4 = reinterpret_cast<const float4*>(in);
        int64_t i = tid;
        for (; i + 3 * nthreads < nvec; i += 4 * nthreads) {
            const float4 a = in4[i], b = in4[i + nthreads], d = in4[i + 2 * nthreads], e = in4[i + 3 * nthreads];
            comp_add(s, c, part4<SQUARES>(a));
            comp_add(s, c, part4<SQUARES>(b));
            comp_add(s, c, part4<SQUARES>(d));
            comp_add(s, c, part4<SQUARES>(e));
        }
        for (; i < nvec; i += nthreads) comp_add(s, c, part4<SQUARES>(in4[i]));
    }
    for (int64_t i = nvec * 4 + tid; i < n; i += nthreads) {
        const float v = in[i];
        comp_add(s, c, SQUARES ? v * v : v);
    }
    double acc = (double)s + (double)c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w];
        partials[blockIdx.x] = b;
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {  // block-uniform: the whole last block adds the partials in a fixed order
        __threadfence();
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += ((volatile double*)partials)[b];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        __syncthreads();  // wsum is reused
        if (lane == 0) wsum[warp] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += wsum[w];
            *out = SQUARES ? sqrt(u) : u;
            *counter = 0u;  // ready for the next launch on this stream
        }
    }
}

// ---- COLMAX ------------------------------------------------------------------------------------

// Column maxima via order-preserving integer keys and atomicMax (max is exact and
// order-free, so the result is deterministic).  Thread = 4 consecutive columns of
// a chunk of rows.
__global__ void colmax_keys_kernel(uint32_t* __restrict__ keys, const float* __restrict__ in, int64_t rows,
                                   int64_t cols, int64_t rows_per_chunk) {
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4;
    if (c >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = r0 + rows_per_chunk < rows ? r0 + rows_per_chunk : rows;
    uint32_t m[4] = {0u, 0u, 0u, 0u};
    const bool vec = (cols % 4 == 0) && aligned16(in);
    for (int64_t r = r0; r < r1; ++r) {
        if (vec) {
            const float4 v = *reinterpret_cast<const float4*>(in + r * cols + c);
            m[0] = max(m[0], fmax_key(__float_as_uint(v.x)));
            m[1] = max(m[1], fmax_key(__float_as_uint(v.y)));
            m[2] = max(m[2], fmax_key(__float_as_uint(v.z)));
            m[3] = max(m[3], fmax_key(__float_as_uint(v.w)));
        } else {
            for (int q = 0; q < 4 && c + q < cols; ++q) m[q] = max(m[q], fmax_key(__float_as_uint(in[r * cols + c + q])));
        }
    }
    for (int q = 0; q < 4 && c + q < cols; ++q)
        if (r1 > r0) atomicMax(keys + c + q, m[q]);
}

__global__ void colmax_decode_kernel(float* __restrict__ out, const uint32_t* __restrict__ keys, int64_t cols,
                                     int64_t rows) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols; c += (int64_t)gridDim.x * blockDim.x)
        out[c] = rows > 0 ? __uint_as_float(fmax_unkey(keys[c])) : -INFINITY;
}

// ---- STENCIL3 --------------------------------------------------------------------------

struct StencilW {
    float w[9];
};

constexpr int kStencilThreads = 128;  // one block: 4 warps x 32 lanes x 4 columns = 512 columns

// One image row as a thread sees it: its four columns c0..c0+3 (one 128-bit load when
// rows are 16-byte aligned) and the two edge columns c0-1 and c0+4, which lanes
// exchange with shuffles; only the first and last lane of a warp read them.
template <bool VEC>
struct StencilRow {
    float4 m;
    float l, r;
    __device__ __forceinline__ void load(const float* __restrict__ in, int64_t y, int64_t rows, int64_t cols, int64_t c0,
                                         int lane) {
        m = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        l = 0.0f;
        r = 0.0f;
        if (y < 0 || y >= rows) return;
        const float* p = in + y * cols;
        if (VEC) {
            if (c0 < cols) m = __ldg(reinterpret_cast<const float4*>(p + c0));
        } else {
            if (c0 < cols) m.x = __ldg(p + c0);
            if (c0 + 1 < cols) m.y = __ldg(p + c0 + 1);
            if (c0 + 2 < cols) m.z = __ldg(p + c0 + 2);
            if (c0 + 3 < cols) m.w = __ldg(p + c0 + 3);
        }
        if (lane == 0 && c0 >= 1 && c0 - 1 < cols) l = __ldg(p + c0 - 1);
        if (lane == 31 && c0 + 4 < cols) r = __ldg(p + c0 + 4);
    }
    // the six values c0-1 .. c0+4 of this row
    __device__ __forceinline__ void spread(float v[6], int lane) const {
        const float fl = __shfl_up_sync(0xffffffffu, m.w, 1);
        const float fr = __shfl_down_sync(0xffffffffu, m.x, 1);
        v[0] = lane == 0 ? l : fl;
        v[1] = m.x;
        v[2] = m.y;
        v[3] = m.z;
        v[4] = m.w;
        v[5] = lane == 31 ? r : fr;
    }
};

// out[i][j] = sum_{a,b} w_ab in[i+a][j+b], zero outside the image.  Each thread owns
// four adjacent columns of a strip of `strip` rows and walks down it with a three-row
// register window, so every input row is read once per strip (plus two halo rows at
// the strip's ends).  The loads of the next kStencilAhead rows are in flight while a
// row is formed (a ring of raw rows, indexed statically under the unrolled inner
// loop); no row past the strip's lower halo is fetched.  The nine terms of an output
// are fmaf'd in row-major order, zero terms included.  Every lane of a warp runs the
// same iterations (the strip is per block), so the shuffles always see a full warp.
constexpr int kStencilAhead = 3;

// Outputs of one pass: a single stencil writes out[0]; the gradient chain (two stencils of
// the same image g1, g2, their squares s1 = g1*g1, s2 = g2*g2 and m = s_x + alpha s_y with
// (x, y) = (1, 2), or (2, 1) when `swap`) writes m and whichever of g1, g2, s1, s2 is
// non-null.  Every value is formed with the operations of the separate loops.
struct StencilOut {
    float* g1;
    float* g2;
    float* s1;
    float* s2;
    float* m;
    float alpha;
    int swap;
    // the sum and the column maxima of m in the same pass (either may be null): one binary64
    // partial per block (a compensated binary32 sum of each thread's four-column partials,
    // threads combined in binary64 by a fixed tree), and order-preserving keys per column
    double* part;
    uint32_t* keys;
};

template <bool VEC>
__device__ __forceinline__ void store4(float* row, int64_t c0, int64_t cols, const float o[4]) {
    if (VEC) {
        if (c0 < cols) *reinterpret_cast<float4*>(row + c0) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + q < cols) row[c0 + q] = o[q];
    }
}

// One output: the terms with nonzero weight in row-major order, fused multiply-adds from
// +0.  With a preset known at compile time (P >= 0) the zero terms are not even emitted;
// with run-time weights (P < 0) they are skipped by a warp-uniform test.  Starting from +0
// the partial sum is never -0, so a zero-weight term would not have changed it for finite
// data: both forms give the bits of the nine-term sum.
template <int P>
__device__ __forceinline__ float stencil9(const StencilW& w, const float* up, const float* md, const float* dn, int q) {
    const float* rowp[3] = {up, md, dn};
    float s = 0.0f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const float wt = P >= 0 ? stencil_preset(P, t) : w.w[t];
        if (wt != 0.0f) s = __fmaf_rn(wt, rowp[t / 3][q + t % 3], s);
    }
    return s;
}

constexpr int kChainAhead = 2;   // rows of loads in flight in the chain variant
constexpr int kChainBlocks = 8;  // resident blocks per SM the chain variant is built for

template <bool VEC, bool CHAIN, int P1, int P2, bool RED = false>
__global__ void __launch_bounds__(kStencilThreads, CHAIN ? kChainBlocks : 8)
    stencil3_kernel(StencilOut out, const float* __restrict__ in, int64_t rows, int64_t cols, StencilW w,
                    StencilW w2, int strip, int64_t row_begin, int64_t row_end) {
    float rs = 0.0f, rc = 0.0f;                   // RED: this thread's compensated sum of m
    uint32_t mk[4] = {0u, 0u, 0u, 0u};            // RED: its columns' maxima (keys)
    constexpr int AHEAD = CHAIN ? kChainAhead : kStencilAhead;
    const int lane = threadIdx.x & 31;
    const int64_t c0 = ((int64_t)blockIdx.x * kStencilThreads + threadIdx.x) * 4;
    // output rows [row_begin, row_end) of a rows-high image (zero outside the image only)
    const int64_t r0 = row_begin + (int64_t)blockIdx.y * strip;
    const int64_t r1 = r0 + strip < row_end ? r0 + strip : row_end;
    const int64_t ylim = r1 + 1 < rows ? r1 + 1 : rows;  // rows >= ylim are never needed
    StencilRow<VEC> ring[AHEAD];
    float up[6], md[6], dn[6];
    {
        StencilRow<VEC> a;
        a.load(in, r0 - 1, rows, cols, c0, lane);
        a.spread(up, lane);
        a.load(in, r0, rows, cols, c0, lane);
        a.spread(md, lane);
    }
#pragma unroll
    for (int k = 0; k < AHEAD; ++k) ring[k].load(in, r0 + 1 + k, ylim, cols, c0, lane);
    for (int64_t i = r0; i < r1; i += AHEAD) {
#pragma unroll
        for (int k = 0; k < AHEAD; ++k) {
            const int64_t row = i + k;
            if (row >= r1) break;  // block-uniform
            ring[k].spread(dn, lane);                                            // row + 1
            ring[k].load(in, row + 1 + AHEAD, ylim, cols, c0, lane);  // in flight for the next rows
            const int64_t off = row * cols;
            float o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = stencil9<P1>(w, up, md, dn, q);
            if constexpr (!CHAIN) {
                store4<VEC>(out.g1 + off, c0, cols, o);
            } else {
                float o2[4], a[4], b[4], m[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    o2[q] = stencil9<P2>(w2, up, md, dn, q);
                    a[q] = __fmul_rn(o[q], o[q]);
                    b[q] = __fmul_rn(o2[q], o2[q]);
                    m[q] = out.swap ? __fmaf_rn(out.alpha, a[q], b[q]) : __fmaf_rn(out.alpha, b[q], a[q]);
                }
                if (out.g1) store4<VEC>(out.g1 + off, c0, cols, o);
                if (out.g2) store4<VEC>(out.g2 + off, c0, cols, o2);
                if (out.s1) store4<VEC>(out.s1 + off, c0, cols, a);
                if (out.s2) store4<VEC>(out.s2 + off, c0, cols, b);
                if (!RED || out.m) store4<VEC>(out.m + off, c0, cols, m);  // m consumed in the pass only: not written
                if constexpr (RED) {
                    float v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        v[q] = c0 + q < cols ? m[q] : 0.0f;
                        if (c0 + q < cols) mk[q] = max(mk[q], fmax_key(__float_as_uint(m[q])));
                    }
                    if (out.part) comp_add(rs, rc, (v[0] + v[1]) + (v[2] + v[3]));
                }
            }
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                up[t] = md[t];
                md[t] = dn[t];
            }
        }
    }
    if constexpr (RED) {
        if (out.keys && r1 > r0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + q < cols) atomicMax(out.keys + c0 + q, mk[q]);  // max: exact and order-free
        }
        if (out.part) {
            __shared__ double wsum[kStencilThreads / 32];
            double acc = (double)rs + (double)rc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) wsum[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double b = 0.0;
#pragma unroll
                for (int k = 0; k < kStencilThreads / 32; ++k) b += wsum[k];
                out.part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = b;
            }
        }
    }
}

// ---- the blur and the gradient chain in one pass ----------------------------------------
//
// The image program's first stencil P0 (the blur, B = P0(X)) and the gradient chain on its
// output (g1 = P1(B), g2 = P2(B), their squares, m = s1 + alpha s2, and with RED the sum and
// column maxima of m), formed in one pass over the raw image X.  Each thread walks down a
// strip of rows holding two raw rows and three rows of B in registers: at output row r it
// forms B's row r + 1 from raw rows r .. r + 2 and the chain's row r from B's rows r - 1 ..
// r + 1, so neither B nor the chain's intermediates go through memory (B is written only when
// something else reads it).  B is zero outside the image, as the separate loops pad it, and
// every value is formed with the separate loops' operations, so the bits are theirs.
// Lanes hold kEdgeNC (eight) columns each; lanes 1 .. 30 of a warp produce its 240 output
// columns, and lanes 0 and 31 hold the eight columns either side, whose raw values and B
// values their neighbours take by shuffle, so no lane loads an edge column of its own.
constexpr int kEdgeNC = 8;          // columns a lane holds (a multiple of 4)
constexpr int kEdgeCols = 30 * kEdgeNC;  // output columns of a warp (lanes 1 .. 30)
constexpr int kEdgeBlocks = 5;      // resident 128-thread blocks per SM the kernel is built for
constexpr int kEdgeAhead = 1;       // raw rows of loads in flight
constexpr int kEdgeBlockCols = kEdgeCols * (kStencilThreads / 32);  // output columns of a block

// A lane's columns c0 .. c0 + kEdgeNC - 1 of one raw row (zero outside the image): with 16-byte
// rows, groups of four that are each wholly inside or outside the image.
struct EdgeRow {
    float4 g[kEdgeNC / 4];
};

template <bool VEC>
__device__ __forceinline__ void edge_load(EdgeRow& r, const float* __restrict__ in, int64_t y, int64_t ylim,
                                          int64_t cols, int64_t c0, const bool inc[kEdgeNC]) {
#pragma unroll
    for (int k = 0; k < kEdgeNC / 4; ++k) r.g[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (y < 0 || y >= ylim) return;
    const float* p = in + y * cols + c0;
#pragma unroll
    for (int k = 0; k < kEdgeNC / 4; ++k) {
        if (VEC) {
            if (inc[4 * k]) r.g[k] = __ldg(reinterpret_cast<const float4*>(p + 4 * k));
        } else {
            if (inc[4 * k]) r.g[k].x = __ldg(p + 4 * k);
            if (inc[4 * k + 1]) r.g[k].y = __ldg(p + 4 * k + 1);
            if (inc[4 * k + 2]) r.g[k].z = __ldg(p + 4 * k + 2);
            if (inc[4 * k + 3]) r.g[k].w = __ldg(p + 4 * k + 3);
        }
    }
}

// The values c0 - 1 .. c0 + kEdgeNC of a row whose columns c0 .. c0 + kEdgeNC - 1 this lane
// holds in b (the first and last lane's outer values are not used).
__device__ __forceinline__ void edge_spread(float v[kEdgeNC + 2], const float b[kEdgeNC]) {
    v[0] = __shfl_up_sync(0xffffffffu, b[kEdgeNC - 1], 1);
#pragma unroll
    for (int q = 0; q < kEdgeNC; ++q) v[q + 1] = b[q];
    v[kEdgeNC + 1] = __shfl_down_sync(0xffffffffu, b[0], 1);
}

__device__ __forceinline__ void edge_flat(float b[kEdgeNC], const EdgeRow& r) {
#pragma unroll
    for (int k = 0; k < kEdgeNC / 4; ++k) {
        b[4 * k] = r.g[k].x;
        b[4 * k + 1] = r.g[k].y;
        b[4 * k + 2] = r.g[k].z;
        b[4 * k + 3] = r.g[k].w;
    }
}

template <bool VEC>
__device__ __forceinline__ void edge_store(float* row, int64_t c0, const bool outc[kEdgeNC], const float v[kEdgeNC]) {
#pragma unroll
    for (int k = 0; k < kEdgeNC / 4; ++k) {
        if (VEC) {
            if (outc[4 * k])
                *reinterpret_cast<float4*>(row + c0 + 4 * k) = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        } else {
#pragma unroll
            for (int q = 4 * k; q < 4 * k + 4; ++q)
                if (outc[q]) row[c0 + q] = v[q];
        }
    }
}

template <bool VEC, int P0, int P1, int P2, bool RED, bool STORE>
__global__ void __launch_bounds__(kStencilThreads, kEdgeBlocks)
    edge_chain_kernel(StencilOut out, float* __restrict__ bout, const float* __restrict__ in, int64_t rows,
                      int64_t cols, StencilW w0, StencilW w1, StencilW w2, int strip, int64_t row_begin,
                      int64_t row_end) {
    constexpr int NC = kEdgeNC;
    float rs = 0.0f, rc = 0.0f;  // RED: this thread's compensated sum of m
    uint32_t mk[NC];             // RED: its columns' maxima (keys)
#pragma unroll
    for (int q = 0; q < NC; ++q) mk[q] = 0u;
    const int lane = threadIdx.x & 31;
    const int64_t c0 = ((int64_t)blockIdx.x * (kStencilThreads / 32) + (threadIdx.x >> 5)) * kEdgeCols - NC + NC * lane;
    bool inc[NC], outc[NC];  // column c0 + q inside the image; and produced by this lane
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int64_t c = VEC ? c0 + (q & ~3) : c0 + q;  // with 16-byte rows, by groups of four
        inc[q] = c >= 0 && c < cols;
        outc[q] = inc[q] && lane >= 1 && lane <= 30;
    }
    // output rows [r0, r1) of this block's strip; raw rows r0 - 2 .. r1 + 1 are read
    const int64_t r0 = row_begin + (int64_t)blockIdx.y * strip;
    const int64_t r1 = r0 + strip < row_end ? r0 + strip : row_end;
    const int64_t ylim = r1 + 2 < rows ? r1 + 2 : rows;
    // B's row from the raw rows above, at and below it (zero outside the image)
    // a lane whose columns are all inside the image zeroes none of its B values but in the
    // rows above and below it, so it skips the per-value choice elsewhere
    bool all_in = true;
#pragma unroll
    for (int q = 0; q < NC; ++q) all_in = all_in && inc[q];
    auto blur = [&](float b[NC], const float* xu, const float* xm, const float* xd, bool row_in) {
#pragma unroll
        for (int q = 0; q < NC; ++q) b[q] = stencil9<P0>(w0, xu, xm, xd, q);
        if (!(row_in && all_in)) {
#pragma unroll
            for (int q = 0; q < NC; ++q) b[q] = (row_in && inc[q]) ? b[q] : 0.0f;
        }
    };
    auto store_b = [&](int64_t y, const float b[NC]) {
        if (STORE && bout && y >= r0 && y < r1) edge_store<VEC>(bout + y * cols, c0, outc, b);
    };
    float xa[NC + 2], xb[NC + 2];  // raw rows r, r + 1
    float ba[NC + 2], bb[NC + 2];  // B's rows r - 1, r
    {
        EdgeRow v;
        float x0[NC + 2], f[NC], t[NC];
        edge_load<VEC>(v, in, r0 - 2, ylim, cols, c0, inc);
        edge_flat(f, v);
        edge_spread(x0, f);
        edge_load<VEC>(v, in, r0 - 1, ylim, cols, c0, inc);
        edge_flat(f, v);
        edge_spread(xa, f);
        edge_load<VEC>(v, in, r0, ylim, cols, c0, inc);
        edge_flat(f, v);
        edge_spread(xb, f);
        blur(t, x0, xa, xb, r0 >= 1);  // B's row r0 - 1
        edge_spread(ba, t);
        edge_load<VEC>(v, in, r0 + 1, ylim, cols, c0, inc);
        edge_flat(f, v);
        edge_spread(x0, f);
        blur(t, xa, xb, x0, r0 < rows);  // B's row r0
        store_b(r0, t);
        edge_spread(bb, t);
#pragma unroll
        for (int k = 0; k < NC + 2; ++k) {
            xa[k] = xb[k];
            xb[k] = x0[k];
        }
    }
    EdgeRow ring[kEdgeAhead];  // raw rows r + 2 .. r + 1 + kEdgeAhead, in flight
#pragma unroll
    for (int k = 0; k < kEdgeAhead; ++k) edge_load<VEC>(ring[k], in, r0 + 2 + k, ylim, cols, c0, inc);
    for (int64_t i = r0; i < r1; i += kEdgeAhead) {
#pragma unroll
        for (int k = 0; k < kEdgeAhead; ++k) {
            const int64_t row = i + k;
            if (row >= r1) break;  // block-uniform
            float xn[NC + 2], bn[NC], bc[NC + 2], f[NC];
            edge_flat(f, ring[k]);
            edge_spread(xn, f);  // raw row + 2
            edge_load<VEC>(ring[k], in, row + 2 + kEdgeAhead, ylim, cols, c0, inc);
            blur(bn, xa, xb, xn, row + 1 < rows);  // B's row + 1
            store_b(row + 1, bn);
            edge_spread(bc, bn);
            float o[NC], o2[NC], a[NC], b[NC], m[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                o[q] = stencil9<P1>(w1, ba, bb, bc, q);
                o2[q] = stencil9<P2>(w2, ba, bb, bc, q);
                a[q] = __fmul_rn(o[q], o[q]);
                b[q] = __fmul_rn(o2[q], o2[q]);
                m[q] = out.swap ? __fmaf_rn(out.alpha, a[q], b[q]) : __fmaf_rn(out.alpha, b[q], a[q]);
            }
            if constexpr (STORE) {
                const int64_t off = row * cols;
                if (out.g1) edge_store<VEC>(out.g1 + off, c0, outc, o);
                if (out.g2) edge_store<VEC>(out.g2 + off, c0, outc, o2);
                if (out.s1) edge_store<VEC>(out.s1 + off, c0, outc, a);
                if (out.s2) edge_store<VEC>(out.s2 + off, c0, outc, b);
                if (out.m) edge_store<VEC>(out.m + off, c0, outc, m);  // null when only the reductions read m
            }
            if constexpr (RED) {
                // the keys of every column are kept and only those of produced columns are
                // raised at the end; the sum takes produced values only: with 16-byte rows a
                // lane that produces none (the warp's outer lanes, lanes right of the image)
                // sums values that are dropped at the end, and only the groups of four right
                // of the image in a lane that produces some are zeroed here
#pragma unroll
                for (int q = 0; q < NC; ++q) mk[q] = max(mk[q], fmax_key(__float_as_uint(m[q])));
                if (out.part) {
                    float v[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) v[q] = (VEC ? (q < 4 || inc[q]) : outc[q]) ? m[q] : 0.0f;
                    float t = 0.0f;
#pragma unroll
                    for (int k = 0; k < NC / 4; ++k) {
                        const float g = (v[4 * k] + v[4 * k + 1]) + (v[4 * k + 2] + v[4 * k + 3]);
                        t = k == 0 ? g : t + g;
                    }
                    comp_add(rs, rc, t);
                }
            }
#pragma unroll
            for (int t = 0; t < NC + 2; ++t) {
                xa[t] = xb[t];
                xb[t] = xn[t];
                ba[t] = bb[t];
                bb[t] = bc[t];
            }
        }
    }
    if constexpr (RED) {
        if (out.keys && r1 > r0) {
#pragma unroll
            for (int q = 0; q < NC; ++q)
                if (outc[q]) atomicMax(out.keys + c0 + q, mk[q]);  // max: exact and order-free
        }
        if (out.part) {
            __shared__ double wsum[kStencilThreads / 32];
            double acc = (!VEC || outc[0]) ? (double)rs + (double)rc : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) wsum[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                double b = 0.0;
#pragma unroll
                for (int k = 0; k < kStencilThreads / 32; ++k) b += wsum[k];
                out.part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = b;
            }
        }
    }
}

// The block partials of a fused sum, added in index order by one block (fixed partition and
// tree).
__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ part, int64_t n,
                                                           double* __restrict__ out) {
    __shared__ double w[8];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < 8; ++k) u += w[k];
        *out = u;
    }
}

// ---- device-wait self test --------------------------------------------------------------------

__global__ void wait_selftest_kernel(volatile int* flag, int* err, unsigned long long limit_ns) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (*flag != 0) return;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            atomicExch(err, DEV_WAIT_TIMEOUT);
            return;
        }
        __nanosleep(1000);
    }
}

}  // namespace

int reduce_blocks() { return sm_count() * 8; }  // a full wave of 256-thread blocks

// Blocks of a reduction over n elements: the full wave for large arrays, fewer for small
// ones (at least kReduceMinPerBlock elements a block), so that a small array does not pay
// for a wave of empty blocks and their partials.  The grid, and with it the summation
// order, depends on n only.
constexpr int64_t kReduceMinPerBlock = 4096;
unsigned reduce_grid(int64_t n) {
    const int64_t want = (n + kReduceMinPerBlock - 1) / kReduceMinPerBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(reduce_blocks(), want));
}

cudaError_t launch_row_exponents(int8_t* e, int64_t rows, uint64_t seed, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    row_exponents_kernel<<<grid_for(rows), kThreads, 0, st>>>(e, rows, seed);
    return cudaGetLastError();
}

cudaError_t launch_init_group(const InitEntry* d_tab, int n_entries, int64_t total4, cudaStream_t st) {
    if (n_entries < 1 || total4 <= 0) return cudaSuccess;
    init_group_kernel<<<grid_for(total4), kThreads, 0, st>>>(d_tab, n_entries, total4);
    return cudaGetLastError();
}

cudaError_t launch_init_set(const InitSet& set, cudaStream_t st) {
    if (set.n < 1 || set.n > GAO_MAX_IO) return cudaErrorInvalidValue;
    int64_t total = 0;
    for (int k = 0; k < set.n; ++k) total += set.o[k].rows * set.o[k].cols;
    if (total <= 0) return cudaSuccess;
    init_set_kernel<<<grid_for((total + 3) / 4), kThreads, 0, st>>>(set);
    return cudaGetLastError();
}

cudaError_t launch_ew_chain(const EwChain& c, cudaStream_t st) {
    if (c.nops < 1 || c.nops > kMaxChainOps) return cudaErrorInvalidValue;
    if (c.n <= 0) return cudaSuccess;
    EwChain k = c;
    uintptr_t ptrs = 0;
    for (int o = 0; o < c.nops; ++o)
        ptrs |= (uintptr_t)c.op[o].xa | (uintptr_t)c.op[o].yb | (uintptr_t)c.op[o].out;
    k.vec = (ptrs & 15u) == 0;
    ew_chain_kernel<<<grid_for((c.n + 3) / 4), kThreads, 0, st>>>(k);
    return cudaGetLastError();
}

cudaError_t launch_axpy(float* out, const float* x, float alpha, const float* y, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ew_kernel<Ew::Axpy><<<grid_for((n + 7) / 8), kThreads, 0, st>>>(out, x, y, alpha, n);
    return cudaGetLastError();
}

cudaError_t launch_relu(float* out, const float* in, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ew_kernel<Ew::Relu><<<grid_for((n + 7) / 8), kThreads, 0, st>>>(out, in, nullptr, 0.0f, n);
    return cudaGetLastError();
}

cudaError_t launch_square(float* out, const float* in, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ew_kernel<Ew::Square><<<grid_for((n + 7) / 8), kThreads, 0, st>>>(out, in, nullptr, 0.0f, n);
    return cudaGetLastError();
}

cudaError_t launch_transpose(float* out, const float* in, int64_t rows, int64_t cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const bool vec = (rows % 4 == 0) && (cols % 4 == 0) && (((uintptr_t)in | (uintptr_t)out) & 15u) == 0;
    if (vec) {
        dim3 grid((unsigned)((cols + 63) / 64), (unsigned)((rows + 63) / 64));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        transpose_vec_kernel<<<grid, 256, 0, st>>>(out, in, rows, cols);
    } else {
        dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        transpose_scalar_kernel<<<grid, 256, 0, st>>>(out, in, rows, cols);
    }
    return cudaGetLastError();
}

cudaError_t launch_rowsum(float* out, const float* in, int64_t rows, int64_t cols, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (cols <= 0) return cudaMemsetAsync(out, 0, (size_t)rows * sizeof(float), st);
    const int64_t threads = rows * 32;
    int64_t g = (threads + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * kBlocksPerSm;
    if (g > cap) g = cap;
    rowsum_kernel<<<(unsigned)g, kThreads, 0, st>>>(out, in, rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_frobenius(double* out, const float* in, int64_t n, ReduceScratch rs, cudaStream_t st) {
    reduce64_kernel<true><<<reduce_grid(n), 256, 0, st>>>(out, in, n < 0 ? 0 : n, rs.partials, rs.counter);
    return cudaGetLastError();
}

cudaError_t launch_sum(double* out, const float* in, int64_t n, ReduceScratch rs, cudaStream_t st) {
    reduce64_kernel<false><<<reduce_grid(n), 256, 0, st>>>(out, in, n < 0 ? 0 : n, rs.partials, rs.counter);
    return cudaGetLastError();
}

cudaError_t launch_colmax(float* out, const float* in, int64_t rows, int64_t cols, uint32_t* keys, cudaStream_t st) {
    if (cols <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)cols * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (rows > 0) {
        const int64_t col_threads = (cols + 3) / 4;
        const unsigned gx = (unsigned)((col_threads + 255) / 256);
        // enough row chunks to put ~8 blocks on every SM
        int64_t want = ((int64_t)sm_count() * kBlocksPerSm + gx - 1) / gx;
        if (want > rows) want = rows;
        if (want > 65535) want = 65535;
        if (want < 1) want = 1;
        const int64_t per = (rows + want - 1) / want;
        const unsigned gy = (unsigned)((rows + per - 1) / per);
        colmax_keys_kernel<<<dim3(gx, gy), 256, 0, st>>>(keys, in, rows, cols, per);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    colmax_decode_kernel<<<grid_for(cols), kThreads, 0, st>>>(out, keys, cols, rows);
    return cudaGetLastError();
}

namespace {
// Grid of a stencil pass over `span` output rows: column blocks of 512 columns, and strips of
// rows for two waves of the resident 128-thread blocks (8 per SM), at least 16 rows per
// strip so that the two halo rows stay a small share.
void stencil_grid(int64_t span, int64_t cols, bool chain, int64_t* gx, int64_t* strip, int64_t* gy) {
    *gx = ((cols + 3) / 4 + kStencilThreads - 1) / kStencilThreads;
    const int64_t want_blocks = (int64_t)sm_count() * 2 * (chain ? kChainBlocks : 8);
    const int64_t strips = (want_blocks + *gx - 1) / *gx;
    int64_t s = (span + strips - 1) / strips;
    if (s < 16) s = 16;
    if ((span + s - 1) / s > 65535) s = (span + 65534) / 65535;
    *strip = s;
    *gy = (span + s - 1) / s;
}

cudaError_t launch_stencil_pass(const StencilOut& o, const float* in, int64_t rows, int64_t cols, int p1, int p2,
                                bool chain, int64_t row_begin, int64_t row_end, cudaStream_t st) {
    StencilW w, w2;
    if (!stencil_weights(p1, w.w) || (chain && !stencil_weights(p2, w2.w))) return cudaErrorInvalidValue;
    if (!chain) w2 = w;
    if (row_begin < 0 || row_end > rows || row_begin > row_end) return cudaErrorInvalidValue;
    const int64_t span = row_end - row_begin;  // output rows of this launch
    if (span <= 0 || cols <= 0) return cudaSuccess;
    int64_t gx, strip, gy;
    stencil_grid(span, cols, chain, &gx, &strip, &gy);
    if (gx > 0x7fffffff || strip > 0x7fffffff) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    uintptr_t ptrs = (uintptr_t)in | (uintptr_t)o.m | (uintptr_t)o.g1 | (uintptr_t)o.g2 | (uintptr_t)o.s1 |
                     (uintptr_t)o.s2;
    const bool vec = (cols % 4 == 0) && (ptrs & 15u) == 0;
    const int sp = (int)strip;
#define GAO_STENCIL_LAUNCH(V, C, A, B) \
    stencil3_kernel<V, C, A, B><<<grid, kStencilThreads, 0, st>>>(o, in, rows, cols, w, w2, sp, row_begin, row_end)
#define GAO_STENCIL_LAUNCH_RED(V, A, B)                                                                     \
    stencil3_kernel<V, true, A, B, true><<<grid, kStencilThreads, 0, st>>>(o, in, rows, cols, w, w2, sp, row_begin, \
                                                                          row_end)
    if (chain && (o.part || o.keys)) {
        // the sum and column maxima of m in the same pass (the image program's pair only)
        if (p1 == 2 && p2 == 3) {
            if (vec) GAO_STENCIL_LAUNCH_RED(true, 2, 3);
            else GAO_STENCIL_LAUNCH_RED(false, 2, 3);
        } else if (p1 == 3 && p2 == 2) {
            if (vec) GAO_STENCIL_LAUNCH_RED(true, 3, 2);
            else GAO_STENCIL_LAUNCH_RED(false, 3, 2);
        } else {
            if (vec) GAO_STENCIL_LAUNCH_RED(true, -1, -1);
            else GAO_STENCIL_LAUNCH_RED(false, -1, -1);
        }
    } else if (chain) {
        // the image program's pair (Sobel x, Sobel y) with compile-time weights; any
        // other pair with run-time weights
        if (p1 == 2 && p2 == 3) {
            if (vec) GAO_STENCIL_LAUNCH(true, true, 2, 3);
            else GAO_STENCIL_LAUNCH(false, true, 2, 3);
        } else if (p1 == 3 && p2 == 2) {
            if (vec) GAO_STENCIL_LAUNCH(true, true, 3, 2);
            else GAO_STENCIL_LAUNCH(false, true, 3, 2);
        } else {
            if (vec) GAO_STENCIL_LAUNCH(true, true, -1, -1);
            else GAO_STENCIL_LAUNCH(false, true, -1, -1);
        }
    } else {
        switch (p1) {
            case 0: if (vec) GAO_STENCIL_LAUNCH(true, false, 0, 0); else GAO_STENCIL_LAUNCH(false, false, 0, 0); break;
            case 1: if (vec) GAO_STENCIL_LAUNCH(true, false, 1, 1); else GAO_STENCIL_LAUNCH(false, false, 1, 1); break;
            case 2: if (vec) GAO_STENCIL_LAUNCH(true, false, 2, 2); else GAO_STENCIL_LAUNCH(false, false, 2, 2); break;
            default: if (vec) GAO_STENCIL_LAUNCH(true, false, 3, 3); else GAO_STENCIL_LAUNCH(false, false, 3, 3); break;
        }
    }
#undef GAO_STENCIL_LAUNCH
#undef GAO_STENCIL_LAUNCH_RED
    return cudaGetLastError();
}
}  // namespace

namespace {
// Grid of a blur + gradient-chain pass over `span` output rows: blocks of 480 output columns,
// and strips of rows for two waves of the resident blocks, at least 16 rows per strip (each
// strip reads four raw rows beyond its own).
void edge_grid(int64_t span, int64_t cols, int64_t* gx, int64_t* strip, int64_t* gy) {
    *gx = (cols + kEdgeBlockCols - 1) / kEdgeBlockCols;
    const int64_t want_blocks = (int64_t)sm_count() * 2 * kEdgeBlocks;
    const int64_t strips = (want_blocks + *gx - 1) / *gx;
    int64_t s = (span + strips - 1) / strips;
    if (s < 16) s = 16;
    if ((span + s - 1) / s > 65535) s = (span + 65534) / 65535;
    *strip = s;
    *gy = (span + s - 1) / s;
}
}  // namespace

int64_t edge_chain_blocks(int64_t rows, int64_t cols) {
    if (rows <= 0 || cols <= 0) return 0;
    int64_t gx, strip, gy;
    edge_grid(rows, cols, &gx, &strip, &gy);
    return gx * gy;
}

// At most this many blocks in any blur + gradient-chain launch of width cols (as for the
// chain alone: a launch has at most `strips` strips).
int64_t edge_chain_blocks_max(int64_t cols) {
    if (cols <= 0) return 0;
    const int64_t gx = (cols + kEdgeBlockCols - 1) / kEdgeBlockCols;
    const int64_t want_blocks = (int64_t)sm_count() * 2 * kEdgeBlocks;
    return gx * ((want_blocks + gx - 1) / gx);
}

cudaError_t launch_edge_chain(const float* in, float* bout, int64_t rows, int64_t cols, int p0, int p1, int p2,
                              float alpha, bool swap, float* g1, float* g2, float* s1, float* s2, float* m,
                              cudaStream_t st, int64_t row_begin, int64_t row_end, const GradReduce* red,
                              int* launches) {
    if (!m && !(red && (red->sum_out || red->colmax_out))) return cudaErrorInvalidValue;
    if (launches) *launches = 0;
    if (row_end < 0) row_end = rows;
    if (row_begin < 0 || row_end > rows || row_begin > row_end) return cudaErrorInvalidValue;
    StencilW w0, w1, w2;
    if (!stencil_weights(p0, w0.w) || !stencil_weights(p1, w1.w) || !stencil_weights(p2, w2.w))
        return cudaErrorInvalidValue;
    const bool want_sum = red && red->sum_out, want_max = red && red->colmax_out;
    const int64_t span = row_end - row_begin;
    const int64_t nblk = edge_chain_blocks(span, cols);  // this launch's partials
    if (want_sum && (!red->part || red->part_at < 0 || red->part_cap < red->part_at + nblk)) return cudaErrorInvalidValue;
    if (want_max && !red->keys) return cudaErrorInvalidValue;
    const StencilOut o{g1, g2, s1, s2, m, alpha, swap ? 1 : 0, want_sum ? red->part + red->part_at : nullptr,
                       want_max ? red->keys : nullptr};
    cudaError_t e;
    if (want_max && red->first && cols > 0) {
        if ((e = cudaMemsetAsync(red->keys, 0, (size_t)cols * sizeof(uint32_t), st)) != cudaSuccess) return e;
    }
    if (span > 0 && cols > 0) {
        int64_t gx, strip, gy;
        edge_grid(span, cols, &gx, &strip, &gy);
        if (gx > 0x7fffffff || strip > 0x7fffffff) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)gx, (unsigned)gy);
        const uintptr_t ptrs = (uintptr_t)in | (uintptr_t)bout | (uintptr_t)m | (uintptr_t)g1 | (uintptr_t)g2 |
                               (uintptr_t)s1 | (uintptr_t)s2;
        const bool vec = (cols % 4 == 0) && (ptrs & 15u) == 0;
        const bool reduce = want_sum || want_max;
        const bool stores = bout || m || g1 || g2 || s1 || s2;  // per-pixel outputs (else reductions only)
        const int sp = (int)strip;
#define GAO_EDGE_LAUNCH(V, A, B, C, R, S)                                                                \
    edge_chain_kernel<V, A, B, C, R, S><<<grid, kStencilThreads, 0, st>>>(o, bout, in, rows, cols, w0, w1, w2, \
                                                                         sp, row_begin, row_end)
#define GAO_EDGE_PAIR(A, B, C)                                          \
    do {                                                                \
        if (reduce && !stores) {                                        \
            if (vec) GAO_EDGE_LAUNCH(true, A, B, C, true, false);       \
            else GAO_EDGE_LAUNCH(false, A, B, C, true, false);          \
        } else if (reduce) {                                            \
            if (vec) GAO_EDGE_LAUNCH(true, A, B, C, true, true);        \
            else GAO_EDGE_LAUNCH(false, A, B, C, true, true);           \
        } else {                                                        \
            if (vec) GAO_EDGE_LAUNCH(true, A, B, C, false, true);       \
            else GAO_EDGE_LAUNCH(false, A, B, C, false, true);          \
        }                                                               \
    } while (0)
        // the image program's stencils (binomial blur, then Sobel x and Sobel y) with
        // compile-time weights; any other triple with run-time weights
        if (p0 == 0 && p1 == 2 && p2 == 3) GAO_EDGE_PAIR(0, 2, 3);
        else if (p0 == 0 && p1 == 3 && p2 == 2) GAO_EDGE_PAIR(0, 3, 2);
        else GAO_EDGE_PAIR(-1, -1, -1);
#undef GAO_EDGE_PAIR
#undef GAO_EDGE_LAUNCH
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    if (want_sum && red->last) {
        sum_partials_kernel<<<1, 256, 0, st>>>(red->part, red->part_at + nblk, red->sum_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    if (want_max && red->last && cols > 0) {
        colmax_decode_kernel<<<grid_for(cols), kThreads, 0, st>>>(red->colmax_out, red->keys, cols, rows);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    return cudaSuccess;
}

int64_t grad_chain_blocks(int64_t rows, int64_t cols) {
    if (rows <= 0 || cols <= 0) return 0;
    int64_t gx, strip, gy;
    stencil_grid(rows, cols, true, &gx, &strip, &gy);
    return gx * gy;
}

// At most this many blocks in any gradient-chain launch of width cols: stencil_grid makes
// strips of at least ceil(span / strips) rows, so a launch has at most `strips` of them.
int64_t grad_chain_blocks_max(int64_t cols) {
    if (cols <= 0) return 0;
    int64_t gx, strip, gy;
    stencil_grid(1, cols, true, &gx, &strip, &gy);
    const int64_t want_blocks = (int64_t)sm_count() * 2 * kChainBlocks;
    return gx * ((want_blocks + gx - 1) / gx);
}

cudaError_t launch_stencil3(float* out, const float* in, int64_t rows, int64_t cols, int preset, cudaStream_t st,
                            int64_t row_begin, int64_t row_end) {
    const StencilOut o{out, nullptr, nullptr, nullptr, nullptr, 0.0f, 0, nullptr, nullptr};
    return launch_stencil_pass(o, in, rows, cols, preset, preset, false, row_begin, row_end < 0 ? rows : row_end, st);
}

cudaError_t launch_grad_chain(const float* in, int64_t rows, int64_t cols, int p1, int p2, float alpha, bool swap,
                              float* g1, float* g2, float* s1, float* s2, float* m, cudaStream_t st,
                              int64_t row_begin, int64_t row_end, const GradReduce* red, int* launches) {
    if (!m && !(red && (red->sum_out || red->colmax_out))) return cudaErrorInvalidValue;
    if (launches) *launches = 0;
    if (row_end < 0) row_end = rows;
    if (row_begin < 0 || row_end > rows || row_begin > row_end) return cudaErrorInvalidValue;
    const bool want_sum = red && red->sum_out, want_max = red && red->colmax_out;
    const int64_t nblk = grad_chain_blocks(row_end - row_begin, cols);  // this launch's partials
    if (want_sum && (!red->part || red->part_at < 0 || red->part_cap < red->part_at + nblk)) return cudaErrorInvalidValue;
    if (want_max && !red->keys) return cudaErrorInvalidValue;
    const StencilOut o{g1, g2, s1, s2, m, alpha, swap ? 1 : 0, want_sum ? red->part + red->part_at : nullptr,
                       want_max ? red->keys : nullptr};
    cudaError_t e;
    if (want_max && red->first && cols > 0) {
        if ((e = cudaMemsetAsync(red->keys, 0, (size_t)cols * sizeof(uint32_t), st)) != cudaSuccess) return e;
    }
    if ((e = launch_stencil_pass(o, in, rows, cols, p1, p2, true, row_begin, row_end, st)) != cudaSuccess) return e;
    if (launches) *launches += nblk > 0;
    if (want_sum && red->last) {
        sum_partials_kernel<<<1, 256, 0, st>>>(red->part, red->part_at + nblk, red->sum_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    if (want_max && red->last && cols > 0) {
        colmax_decode_kernel<<<grid_for(cols), kThreads, 0, st>>>(red->colmax_out, red->keys, cols, rows);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) *launches += 1;
    }
    return cudaSuccess;
}

cudaError_t launch_wait_selftest(int* flag, int* err, double limit_s, cudaStream_t st) {
    wait_selftest_kernel<<<1, 1, 0, st>>>(flag, err, (unsigned long long)(limit_s * 1e9));
    return cudaGetLastError();
}

// ---- column maxima without any allocation ------------------------------------------------------
//
// Some callers cannot allocate device memory at the point where they need a result:
// a host framework whose pool allocator owns the device memory and forbids other
// allocations, or a latency-critical loop that cannot afford cudaMalloc/cudaFree
// (they may synchronise the device and can fail with out-of-memory mid-run).  For
// them the column-maxima loop has a variant whose scratch (one 32-bit key per
// column) lives in the file-scope array below, loaded with the library and held by
// every device that loads it until the process exits.  Host code must not use the
// array's name as a device address: it is a host-side stand-in.  The device address
// is looked up with cudaGetSymbolAddress once per device, on the first call made
// while that device is current.

namespace {

constexpr int64_t kColmaxNoallocMaxCols = 65536;  // 256 KiB of keys
static __device__ __align__(256) uint32_t g_colmax_noalloc_keys[kColmaxNoallocMaxCols];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_keys_dev[kMaxDevices] = {};  // device address of the array, per device

cudaError_t colmax_noalloc_keys(uint32_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (g_noalloc_keys_dev[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_colmax_noalloc_keys);
        if (e != cudaSuccess) return e;
        g_noalloc_keys_dev[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_keys_dev[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace gao

extern "C" gao_status gao_colmax_noalloc(const float* dev_in, int64_t rows, int64_t cols, float* dev_out,
                                         void* stream) {
    using namespace gao;
    if (rows < 0 || cols < 0) return fail(GAO_EINVAL, "gao_colmax_noalloc: negative shape");
    if (cols > kColmaxNoallocMaxCols)
        return fail(GAO_EINVAL, "gao_colmax_noalloc: cols exceeds the fixed maximum of 65536 columns");
    if (cols == 0) return GAO_OK;
    if (dev_out == nullptr || (rows > 0 && dev_in == nullptr))
        return fail(GAO_EINVAL, "gao_colmax_noalloc: null device pointer");
    uint32_t* keys = nullptr;
    cudaError_t e = colmax_noalloc_keys(&keys);
    if (e != cudaSuccess) return cuda_fail(e, "gao_colmax_noalloc: cudaGetSymbolAddress");
    // clears keys[0, cols) on the stream, then reduces and decodes into dev_out
    e = launch_colmax(dev_out, dev_in, rows, cols, keys, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gao_colmax_noalloc: launch");
    return GAO_OK;
}

