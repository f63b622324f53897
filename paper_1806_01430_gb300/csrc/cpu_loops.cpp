// CPU side of every loop (gene bit 0): binary32, OpenMP over the host cores.
//
// These are the loops as a CPU program would run them when the gene leaves them on
// the host.  Loops whose GPU version is exact (INIT, AXPY, TRANSPOSE, RELU, SQUARE,
// COLMAX) or fixes its rounding order (STENCIL3) produce bit-identical results here;
// the others agree within rounding.
// Every loop polls a deadline between blocks of work so that a run over its time
// budget stops early (the run then reports a timeout).
#include <math.h>
#include <omp.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <vector>

#include "gao_internal.h"

namespace gao {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

namespace {

inline bool expired(CpuCtx& c) {
    if (c.deadline > 0.0 && now_s() > c.deadline) {
        __atomic_store_n(&c.timed_out, true, __ATOMIC_RELAXED);
        return true;
    }
    return false;
}

inline int nthreads(const CpuCtx& c) { return c.threads > 0 ? c.threads : omp_get_max_threads(); }

}  // namespace

void cpu_init(float* out, int64_t rows, int64_t cols, uint64_t seed, uint32_t buf, bool rowscale, CpuCtx& c) {
    std::atomic<bool> stop{false};
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < rows; ++i) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if ((i & 255) == 0 && expired(c)) stop = true;
        const int e = rowscale ? row_exponent(seed, i) : 0;
        float* o = out + i * cols;
        for (int64_t j = 0; j < cols; ++j) {
            float v = init_value(seed, buf, (uint64_t)(i * cols + j));
            o[j] = rowscale ? ldexpf(v, e) : v;
        }
    }
}

namespace {

// Register-blocked piece of a K chunk: out[i][j] += sum over k of a[i][k] * b[k][j] for an
// MR x NR block, the sum formed in k order with fmaf into zero-initialised registers (the
// chunk sum) and then added to out.  bp is B packed for this block: bp[k * NR + j].
template <int MR, int NR>
inline void gemm_micro(const float* a, int64_t lda, const float* bp, int64_t kn, float* out, int64_t ldo) {
    float acc[MR][NR];
#pragma GCC unroll 16
    for (int i = 0; i < MR; ++i)
#pragma GCC unroll 16
        for (int j = 0; j < NR; ++j) acc[i][j] = 0.0f;
    for (int64_t k = 0; k < kn; ++k) {
        const float* b = bp + k * NR;
#pragma GCC unroll 16
        for (int i = 0; i < MR; ++i) {
            const float av = a[i * lda + k];
#pragma GCC unroll 16
            for (int j = 0; j < NR; ++j) acc[i][j] = fmaf(av, b[j], acc[i][j]);
        }
    }
#pragma GCC unroll 16
    for (int i = 0; i < MR; ++i)
#pragma GCC unroll 16
        for (int j = 0; j < NR; ++j) out[i * ldo + j] += acc[i][j];
}

// The same for a ragged edge block (rn <= MR rows, jn <= NR columns).
template <int MR, int NR>
inline void gemm_edge(const float* a, int64_t lda, const float* bp, int64_t kn, float* out, int64_t ldo, int64_t rn,
                      int64_t jn) {
    for (int64_t i = 0; i < rn; ++i)
        for (int64_t j = 0; j < jn; ++j) {
            float s = 0.0f;
            for (int64_t k = 0; k < kn; ++k) s = fmaf(a[i * lda + k], bp[k * NR + j], s);
            out[i * ldo + j] += s;
        }
}

}  // namespace

// C = alpha*A@B + beta*C0.  Work is split into tasks of (up to 512 rows) x (up to 256
// columns); each task walks K in chunks of `kchunk`: the chunk's B panel is packed in
// 16-column slabs, and 6 x 16 register blocks form the chunk sums (k in order, fmaf),
// which are added into the task's binary32 outer sums chunk by chunk.
void cpu_gemm(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N, int64_t K, float alpha,
              float beta, int kchunk, CpuCtx& c) {
    constexpr int64_t JT = 256, RS = 512;
    constexpr int MR = 6, NR = 16;
    const int64_t kc = kchunk > 0 ? kchunk : 256;
    const int64_t ntj = (N + JT - 1) / JT, nts = (M + RS - 1) / RS;
    std::atomic<bool> stop{false};
#pragma omp parallel num_threads(nthreads(c))
    {
        std::vector<float> outer((size_t)RS * JT), pack((size_t)std::min(kc, std::max<int64_t>(K, 1)) * JT);
#pragma omp for schedule(dynamic, 1)
        for (int64_t task = 0; task < ntj * nts; ++task) {
            if (stop.load(std::memory_order_relaxed)) continue;
            const int64_t j0 = (task % ntj) * JT, i0 = (task / ntj) * RS;
            const int64_t jn = std::min(JT, N - j0), in = std::min(RS, M - i0);
            std::fill(outer.begin(), outer.begin() + in * JT, 0.0f);
            for (int64_t k0 = 0; k0 < K; k0 += kc) {
                if (expired(c)) {
                    stop = true;
                    break;
                }
                const int64_t kn = std::min(kc, K - k0);
                // pack B[k0 .. k0+kn) x [j0 .. j0+jn) as slabs [jn / NR][kn][NR] (zero-filled)
                for (int64_t jb = 0; jb < jn; jb += NR) {
                    float* slab = pack.data() + jb * kn;
                    const int64_t w = std::min<int64_t>(NR, jn - jb);
                    for (int64_t k = 0; k < kn; ++k) {
                        const float* brow = B + (k0 + k) * N + j0 + jb;
                        for (int64_t j = 0; j < NR; ++j) slab[k * NR + j] = j < w ? brow[j] : 0.0f;
                    }
                }
                for (int64_t jb = 0; jb < jn; jb += NR) {
                    const float* slab = pack.data() + jb * kn;
                    const int64_t w = std::min<int64_t>(NR, jn - jb);
                    for (int64_t r0 = 0; r0 < in; r0 += MR) {
                        const float* a = A + (i0 + r0) * K + k0;
                        float* out = outer.data() + r0 * JT + jb;
                        const int64_t rn = std::min<int64_t>(MR, in - r0);
                        if (rn == MR && w == NR)
                            gemm_micro<MR, NR>(a, K, slab, kn, out, JT);
                        else
                            gemm_edge<MR, NR>(a, K, slab, kn, out, JT, rn, w);
                    }
                }
            }
            if (stop.load(std::memory_order_relaxed)) continue;
            for (int64_t r = 0; r < in; ++r) {
                const float* orow = outer.data() + r * JT;
                const float* c0 = C0 + (i0 + r) * N + j0;
                float* crow = C + (i0 + r) * N + j0;
                for (int64_t j = 0; j < jn; ++j) {
                    float v = alpha * orow[j];
                    if (beta != 0.0f) v = fmaf(beta, c0[j], v);
                    crow[j] = v;
                }
            }
        }
    }
}

void cpu_axpy(float* out, const float* x, float alpha, const float* y, int64_t n, CpuCtx& c) {
    const int64_t blk = 1 << 20;
    std::atomic<bool> stop{false};
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t b = 0; b < (n + blk - 1) / blk; ++b) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if (expired(c)) {
            stop = true;
            continue;
        }
        const int64_t e = std::min(n, (b + 1) * blk);
        for (int64_t i = b * blk; i < e; ++i) out[i] = fmaf(alpha, y[i], x[i]);
    }
}

void cpu_transpose(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c) {
    constexpr int64_t T = 64;
    std::atomic<bool> stop{false};
    const int64_t tr = (rows + T - 1) / T, tc = (cols + T - 1) / T;
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t t = 0; t < tr * tc; ++t) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if ((t & 63) == 0 && expired(c)) {
            stop = true;
            continue;
        }
        const int64_t r0 = (t / tc) * T, c0 = (t % tc) * T;
        const int64_t r1 = std::min(rows, r0 + T), c1 = std::min(cols, c0 + T);
        for (int64_t i = r0; i < r1; ++i)
            for (int64_t j = c0; j < c1; ++j) out[j * rows + i] = in[i * cols + j];
    }
}

void cpu_rowsum(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c) {
    std::atomic<bool> stop{false};
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < rows; ++i) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if ((i & 255) == 0 && expired(c)) {
            stop = true;
            continue;
        }
        // the fixed row-sum order shared with the GPU paths (kRowsumBlock blocks, quadruple
        // tree per block, four interleaved block accumulators)
        const float* r = in + i * cols;
        float u[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int64_t nblk = (cols + kRowsumBlock - 1) / kRowsumBlock;
        for (int64_t p = 0; p < nblk; ++p) {
            const int64_t j0 = p * kRowsumBlock;
            float x[kRowsumBlock];
            if (j0 + kRowsumBlock <= cols) {
                for (int t = 0; t < kRowsumBlock; ++t) x[t] = r[j0 + t];
            } else {
                for (int t = 0; t < kRowsumBlock; ++t) x[t] = j0 + t < cols ? r[j0 + t] : 0.0f;
            }
            float q[8];
            for (int m = 0; m < 8; ++m) q[m] = (x[4 * m] + x[4 * m + 1]) + (x[4 * m + 2] + x[4 * m + 3]);
            u[p & 3] += ((q[0] + q[4]) + (q[2] + q[6])) + ((q[1] + q[5]) + (q[3] + q[7]));
        }
        out[i] = (u[0] + u[2]) + (u[1] + u[3]);
    }
}

namespace {
template <bool SQUARES>
double cpu_reduce64(const float* in, int64_t n, CpuCtx& c) {
    const int nt = nthreads(c);
    std::vector<double> part((size_t)nt, 0.0);
    std::atomic<bool> stop{false};
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        const int64_t b = n * t / T, e = n * (t + 1) / T;
        double s = 0.0;
        for (int64_t i0 = b; i0 < e && !stop.load(std::memory_order_relaxed); i0 += (1 << 20)) {
            if (expired(c)) {
                stop = true;
                break;
            }
            const int64_t i1 = std::min(e, i0 + (int64_t)(1 << 20));
            for (int64_t i = i0; i < i1; ++i) s += SQUARES ? (double)in[i] * (double)in[i] : (double)in[i];
        }
        part[(size_t)t] = s;
    }
    double s = 0.0;
    for (double p : part) s += p;
    return SQUARES ? sqrt(s) : s;
}
}  // namespace

double cpu_frobenius(const float* in, int64_t n, CpuCtx& c) { return cpu_reduce64<true>(in, n, c); }
double cpu_sum(const float* in, int64_t n, CpuCtx& c) { return cpu_reduce64<false>(in, n, c); }

void cpu_relu(float* out, const float* in, int64_t n, CpuCtx& c) {
    (void)c;
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < n; ++i) out[i] = in[i] > 0.0f ? in[i] : 0.0f;
}

void cpu_square(float* out, const float* in, int64_t n, CpuCtx& c) {
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < n; ++i) out[i] = in[i] * in[i];
}

void cpu_colmax(float* out, const float* in, int64_t rows, int64_t cols, CpuCtx& c) {
    const int nt = nthreads(c);
    std::vector<uint32_t> keys((size_t)nt * (size_t)cols, 0u);
#pragma omp parallel num_threads(nt)
    {
        const int t = omp_get_thread_num(), T = omp_get_num_threads();
        uint32_t* k = keys.data() + (size_t)t * cols;
        const int64_t b = rows * t / T, e = rows * (t + 1) / T;
        for (int64_t i = b; i < e; ++i) {
            const uint32_t* r = reinterpret_cast<const uint32_t*>(in + i * cols);
            for (int64_t j = 0; j < cols; ++j) k[j] = std::max(k[j], fmax_key(r[j]));
        }
    }
    for (int64_t j = 0; j < cols; ++j) {
        uint32_t m = 0u;
        for (int t = 0; t < nt; ++t) m = std::max(m, keys[(size_t)t * cols + j]);
        uint32_t bits = fmax_unkey(m);
        float v;
        memcpy(&v, &bits, 4);
        out[j] = rows > 0 ? v : -INFINITY;
    }
}

// 3x3 stencil with zero padding.  Each output adds its terms in row-major (a, b) order
// with fmaf, out-of-image terms included and zero-weight terms skipped, exactly as the
// GPU kernel does, so both give the same bits.
void cpu_stencil3(float* out, const float* in, int64_t rows, int64_t cols, int preset, CpuCtx& c) {
    float w[9];
    if (!stencil_weights(preset, w)) return;
    std::atomic<bool> stop{false};
#pragma omp parallel num_threads(nthreads(c))
    {
        std::vector<float> pad[3];
        for (auto& v : pad) v.assign((size_t)cols + 2, 0.0f);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < rows; ++i) {
            if (stop.load(std::memory_order_relaxed)) continue;
            if ((i & 63) == 0 && expired(c)) {
                stop = true;
                continue;
            }
            // rows i-1, i, i+1 with one zero column on each side
            for (int a = 0; a < 3; ++a) {
                const int64_t y = i + a - 1;
                float* d = pad[a].data();
                if (y >= 0 && y < rows)
                    memcpy(d + 1, in + y * cols, sizeof(float) * (size_t)cols);
                else
                    memset(d + 1, 0, sizeof(float) * (size_t)cols);
            }
            const float *u = pad[0].data(), *m = pad[1].data(), *d = pad[2].data();
            float* o = out + i * cols;
            const float* rowp[3] = {u, m, d};
            for (int64_t j = 0; j < cols; ++j) {
                float s = 0.0f;
                for (int t = 0; t < 9; ++t)
                    if (w[t] != 0.0f) s = fmaf(w[t], rowp[t / 3][j + t % 3], s);
                o[j] = s;
            }
        }
    }
}

// First-order recurrence along each row: out[i][0] = in[i][0], then
// out[i][j] = fmaf(alpha, out[i][j-1], in[i][j]).  Rows are independent, elements of a
// row are not (the loop-carried dependence that keeps this loop on the CPU).
void cpu_recurrence(float* out, const float* in, int64_t rows, int64_t cols, float alpha, CpuCtx& c) {
    std::atomic<bool> stop{false};
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < rows; ++i) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if ((i & 255) == 0 && expired(c)) {
            stop = true;
            continue;
        }
        const float* x = in + i * cols;
        float* y = out + i * cols;
        if (cols <= 0) continue;
        float prev = x[0];
        y[0] = prev;
        for (int64_t j = 1; j < cols; ++j) {
            prev = fmaf(alpha, prev, x[j]);
            y[j] = prev;
        }
    }
}

// out[i] = the first column j with in[i][j] > threshold, cols if there is none; the
// scan of a row stops at the first hit (the early exit that keeps this loop on the CPU).
void cpu_find(double* out, const float* in, int64_t rows, int64_t cols, float threshold, CpuCtx& c) {
    std::atomic<bool> stop{false};
#pragma omp parallel for schedule(static) num_threads(nthreads(c))
    for (int64_t i = 0; i < rows; ++i) {
        if (stop.load(std::memory_order_relaxed)) continue;
        if ((i & 255) == 0 && expired(c)) {
            stop = true;
            continue;
        }
        const float* x = in + i * cols;
        int64_t j = 0;
        for (; j < cols; ++j)
            if (x[j] > threshold) break;
        out[i] = (double)j;
    }
}

}  // namespace gao
