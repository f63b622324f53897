// Residual check of a GEMM on the GPU in binary64 (Freivalds 1977).
//
// For C = alpha A B + beta C0 (A M x K, B K x N, C0 and C M x N, all row-major
// binary32) and vectors x (N) and y (M), the two identities
//   C x   = alpha A (B x)   + beta C0 x        (right form)
//   y^T C = alpha (y^T A) B + beta y^T C0      (left form)
// hold exactly for the exact product.  Every entry of C enters both sides, so a wrong
// tile, row block or single entry changes the residual vectors
//   r = C x - beta C0 x - alpha A (B x),  s = y^T C - beta y^T C0 - alpha (y^T A) B
// by exactly that entry's error times x_j (row i of r) and y_i (column j of s), while
// the check reads each matrix once instead of forming the O(MNK) product.  Every
// product and sum here is binary64 (the binary32 inputs are exact in binary64), so the
// check adds ~1e-16 relative noise to what it measures.
//
// Kernels (all deterministic: fixed partition, fixed summation order, no atomics):
//   rowdot  out[i] = sum_j X[i][j] v[j] (and the same for a second matrix), one warp per
//           row, lanes stride the row in float4 steps, a fixed butterfly at the end;
//   coldot  out[j] = sum_i w[i] X[i][j] (and a second matrix), column strips of 512 x
//           row chunks, binary64 partials per chunk, then the chunks summed in order;
//   norms   the residual vector, its 2-norm and max-norm against the reference side's.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "gao_internal.h"

namespace gao {
namespace {

constexpr int kRowdotThreads = 256;  // 8 rows per block
constexpr int kColThreads = 128;     // 4 columns per thread: 512-column strips
constexpr int kColStrip = 4 * kColThreads;
constexpr int kMaxColChunks = 64;    // row chunks of a column reduction
constexpr int kNormThreads = 1024;

// out[i] = sum_j X[i][j] v[j], and out2[i] = sum_j X2[i][j] v[j] when X2 is set.
template <bool TWO>
__global__ void __launch_bounds__(kRowdotThreads) rowdot_kernel(const float* __restrict__ X,
                                                                const float* __restrict__ X2, int64_t rows,
                                                                int64_t cols, const double* __restrict__ v,
                                                                double* __restrict__ out, double* __restrict__ out2,
                                                                int vec) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (kRowdotThreads / 32) + (threadIdx.x >> 5);
    if (i >= rows) return;
    const float* xr = X + i * cols;
    const float* xr2 = TWO ? X2 + i * cols : nullptr;
    double a = 0.0, b = 0.0;
    int64_t j0 = 0;
    if (vec) {
        const int64_t n4 = cols / 4;
        for (int64_t q = lane; q < n4; q += 32) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(xr) + q);
            const double2 v01 = __ldg(reinterpret_cast<const double2*>(v) + 2 * q);
            const double2 v23 = __ldg(reinterpret_cast<const double2*>(v) + 2 * q + 1);
            a = fma((double)u.x, v01.x, a);
            a = fma((double)u.y, v01.y, a);
            a = fma((double)u.z, v23.x, a);
            a = fma((double)u.w, v23.y, a);
            if constexpr (TWO) {
                const float4 w = __ldg(reinterpret_cast<const float4*>(xr2) + q);
                b = fma((double)w.x, v01.x, b);
                b = fma((double)w.y, v01.y, b);
                b = fma((double)w.z, v23.x, b);
                b = fma((double)w.w, v23.y, b);
            }
        }
        j0 = n4 * 4;
    }
    for (int64_t j = j0 + lane; j < cols; j += 32) {
        const double vj = v[j];
        a = fma((double)xr[j], vj, a);
        if constexpr (TWO) b = fma((double)xr2[j], vj, b);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        if constexpr (TWO) b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
        out[i] = a;
        if constexpr (TWO) out2[i] = b;
    }
}

// Partial column sums over the rows of chunk blockIdx.y:
// part[chunk][j] = sum_{i in chunk} w[i] X[i][j] (part2 likewise for X2).
template <bool TWO>
__global__ void __launch_bounds__(kColThreads) coldot_partial_kernel(const float* __restrict__ X,
                                                                     const float* __restrict__ X2, int64_t rows,
                                                                     int64_t cols, const double* __restrict__ w,
                                                                     int64_t rows_per_chunk,
                                                                     double* __restrict__ part,
                                                                     double* __restrict__ part2, int vec) {
    const int64_t j0 = (int64_t)blockIdx.x * kColStrip + 4 * threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = std::min(rows, r0 + rows_per_chunk);
    double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0};
    if (j0 < cols) {
        const bool full = vec && j0 + 3 < cols;
#pragma unroll 4
        for (int64_t i = r0; i < r1; ++i) {
            const double wi = w[i];
            const float* xr = X + i * cols + j0;
            float u[4], t[4];
            if (full) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(xr));
                u[0] = q.x, u[1] = q.y, u[2] = q.z, u[3] = q.w;
                if constexpr (TWO) {
                    const float4 q2 = __ldg(reinterpret_cast<const float4*>(X2 + i * cols + j0));
                    t[0] = q2.x, t[1] = q2.y, t[2] = q2.z, t[3] = q2.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    u[c] = j0 + c < cols ? xr[c] : 0.0f;
                    if constexpr (TWO) t[c] = j0 + c < cols ? X2[i * cols + j0 + c] : 0.0f;
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                a[c] = fma(wi, (double)u[c], a[c]);
                if constexpr (TWO) b[c] = fma(wi, (double)t[c], b[c]);
            }
        }
    }
    double* pr = part + (int64_t)blockIdx.y * cols;
    double* pr2 = TWO ? part2 + (int64_t)blockIdx.y * cols : nullptr;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (j0 + c < cols) {
            pr[j0 + c] = a[c];
            if constexpr (TWO) pr2[j0 + c] = b[c];
        }
    }
}

// out[j] = sum over chunks, in chunk order, of part[chunk][j].
__global__ void coldot_finish_kernel(const double* __restrict__ part, const double* __restrict__ part2,
                                     int64_t cols, int chunks, double* __restrict__ out, double* __restrict__ out2) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < chunks; ++c) {
        a += part[(int64_t)c * cols + j];
        if (part2) b += part2[(int64_t)c * cols + j];
    }
    out[j] = a;
    if (out2) out2[j] = b;
}

// For n entries: ref = alpha p + beta q0, res = c - beta q0 - alpha p (c = C's side);
// res written to rvec when set; norms[0] = ||res||_2, norms[1] = ||ref||_2,
// norms[2] = max |res|, norms[3] = max |ref|, norms[4] = the first index of max |res|.
__global__ void __launch_bounds__(kNormThreads) residual_norms_kernel(const double* __restrict__ c,
                                                                      const double* __restrict__ q0,
                                                                      const double* __restrict__ p, int64_t n,
                                                                      double alpha, double beta,
                                                                      double* __restrict__ rvec,
                                                                      double* __restrict__ norms) {
    __shared__ double s_rr[kNormThreads / 32], s_ff[kNormThreads / 32], s_rm[kNormThreads / 32],
        s_fm[kNormThreads / 32];
    __shared__ int64_t s_ri[kNormThreads / 32];
    double rr = 0.0, ff = 0.0, rm = -1.0, fm = 0.0;
    int64_t ri = -1;
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads) {
        const double ref = fma(alpha, p[i], beta * q0[i]);
        const double res = (c[i] - beta * q0[i]) - alpha * p[i];
        if (rvec) rvec[i] = res;
        rr = fma(res, res, rr);
        ff = fma(ref, ref, ff);
        if (fabs(res) > rm) rm = fabs(res), ri = i;  // first index of the maximum in this thread's order
        fm = fmax(fm, fabs(ref));
    }
    // fixed butterfly within the warp, then warps in order; the maximum keeps the lowest index
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, off);
        ff += __shfl_xor_sync(0xffffffffu, ff, off);
        fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, off));
        const double orm = __shfl_xor_sync(0xffffffffu, rm, off);
        const long long ori = __shfl_xor_sync(0xffffffffu, (long long)ri, off);
        if (orm > rm || (orm == rm && ori >= 0 && (ri < 0 || ori < ri))) rm = orm, ri = ori;
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s_rr[w] = rr, s_ff[w] = ff, s_rm[w] = rm, s_fm[w] = fm, s_ri[w] = ri;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, f = 0.0, m = -1.0, mf = 0.0;
        int64_t mi = -1;
        for (int k = 0; k < kNormThreads / 32; ++k) {
            a += s_rr[k];
            f += s_ff[k];
            mf = fmax(mf, s_fm[k]);
            if (s_rm[k] > m || (s_rm[k] == m && s_ri[k] >= 0 && (mi < 0 || s_ri[k] < mi))) m = s_rm[k], mi = s_ri[k];
        }
        norms[0] = sqrt(a);
        norms[1] = sqrt(f);
        norms[2] = m < 0.0 ? 0.0 : m;
        norms[3] = mf;
        norms[4] = (double)mi;
    }
}

inline size_t a256(size_t x) { return (x + 255) / 256 * 256; }

int col_chunks(int64_t rows, int64_t cols) {
    // about four blocks per SM over the whole reduction, at most kMaxColChunks chunks
    const int64_t strips = (cols + kColStrip - 1) / kColStrip;
    int64_t c = (4 * (int64_t)sm_count() + strips - 1) / std::max<int64_t>(1, strips);
    c = std::max<int64_t>(1, std::min<int64_t>({c, (int64_t)kMaxColChunks, std::max<int64_t>(1, rows)}));
    return (int)c;
}

struct ResidLayout {
    size_t bx, abx, cx, c0x, ya, yab, yc, yc0, part, part2, norms, total;
};

ResidLayout resid_layout(int64_t M, int64_t N, int64_t K) {
    ResidLayout L{};
    const size_t d = sizeof(double);
    // partial sums of the three column reductions: y^T A (K columns), (y^T A) B and y^T C (N)
    const size_t part = std::max({(size_t)col_chunks(M, K) * (size_t)K, (size_t)col_chunks(K, N) * (size_t)N,
                                  (size_t)col_chunks(M, N) * (size_t)N});
    const size_t part2 = (size_t)col_chunks(M, N) * (size_t)N;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += a256(std::max<size_t>(bytes, d));
        return o;
    };
    L.bx = take((size_t)K * d);
    L.abx = take((size_t)M * d);
    L.cx = take((size_t)M * d);
    L.c0x = take((size_t)M * d);
    L.ya = take((size_t)K * d);
    L.yab = take((size_t)N * d);
    L.yc = take((size_t)N * d);
    L.yc0 = take((size_t)N * d);
    L.part = take(part * d);
    L.part2 = take(part2 * d);
    L.norms = take(16 * d);
    L.total = off;
    return L;
}

cudaError_t launch_rowdot(const float* X, const float* X2, int64_t rows, int64_t cols, const double* v, double* out,
                          double* out2, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int vec = (cols % 4 == 0) && ((((uintptr_t)X) | ((uintptr_t)X2) | ((uintptr_t)v)) & 15u) == 0;
    const int64_t blocks = (rows + kRowdotThreads / 32 - 1) / (kRowdotThreads / 32);
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (X2) rowdot_kernel<true><<<(unsigned)blocks, kRowdotThreads, 0, st>>>(X, X2, rows, cols, v, out, out2, vec);
    else rowdot_kernel<false><<<(unsigned)blocks, kRowdotThreads, 0, st>>>(X, nullptr, rows, cols, v, out, nullptr, vec);
    return cudaGetLastError();
}

cudaError_t launch_coldot(const float* X, const float* X2, int64_t rows, int64_t cols, const double* w, double* part,
                          double* part2, double* out, double* out2, cudaStream_t st) {
    if (cols <= 0) return cudaSuccess;
    const int chunks = col_chunks(rows, cols);
    const int64_t rpc = (std::max<int64_t>(rows, 1) + chunks - 1) / chunks;
    const int vec = (cols % 4 == 0) && ((((uintptr_t)X) | ((uintptr_t)X2)) & 15u) == 0;
    const dim3 grid((unsigned)((cols + kColStrip - 1) / kColStrip), (unsigned)chunks);
    if (X2) coldot_partial_kernel<true><<<grid, kColThreads, 0, st>>>(X, X2, rows, cols, w, rpc, part, part2, vec);
    else coldot_partial_kernel<false><<<grid, kColThreads, 0, st>>>(X, nullptr, rows, cols, w, rpc, part, nullptr, vec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    coldot_finish_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(part, X2 ? part2 : nullptr, cols, chunks, out,
                                                                         X2 ? out2 : nullptr);
    return cudaGetLastError();
}

}  // namespace

size_t gemm_residual_scratch_bytes(int64_t M, int64_t N, int64_t K) { return resid_layout(M, N, K).total; }

cudaError_t launch_gemm_residual(const float* A, const float* B, const float* C0, const float* C, int64_t M,
                                 int64_t N, int64_t K, double alpha, double beta, const double* x, const double* y,
                                 void* scratch, double* rvec, double* svec, cudaStream_t st, int* launches,
                                 const double** norms_dev) {
    const ResidLayout L = resid_layout(M, N, K);
    char* s = static_cast<char*>(scratch);
    auto D = [&](size_t off) { return reinterpret_cast<double*>(s + off); };
    double *bx = D(L.bx), *abx = D(L.abx), *cx = D(L.cx), *c0x = D(L.c0x), *ya = D(L.ya), *yab = D(L.yab),
           *yc = D(L.yc), *yc0 = D(L.yc0), *part = D(L.part), *part2 = D(L.part2), *norms = D(L.norms);
    *launches = 0;
    const bool has_c0 = C0 != nullptr && beta != 0.0;
    const float* c0 = has_c0 ? C0 : nullptr;
    cudaError_t e;
    // right form: B x, A (B x), C x and C0 x
    if (K > 0) {
        if ((e = launch_rowdot(B, nullptr, K, N, x, bx, nullptr, st)) != cudaSuccess) return e;
        if ((e = launch_rowdot(A, nullptr, M, K, bx, abx, nullptr, st)) != cudaSuccess) return e;
        *launches += 2;
    } else {
        if ((e = cudaMemsetAsync(abx, 0, (size_t)std::max<int64_t>(M, 1) * sizeof(double), st)) != cudaSuccess)
            return e;
    }
    if ((e = launch_rowdot(C, c0, M, N, x, cx, c0x, st)) != cudaSuccess) return e;
    if (!has_c0 && (e = cudaMemsetAsync(c0x, 0, (size_t)std::max<int64_t>(M, 1) * sizeof(double), st)) != cudaSuccess)
        return e;
    residual_norms_kernel<<<1, kNormThreads, 0, st>>>(cx, c0x, abx, M, alpha, has_c0 ? beta : 0.0, rvec, norms);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 2;
    // left form: y^T A, (y^T A) B, y^T C and y^T C0
    if (K > 0) {
        if ((e = launch_coldot(A, nullptr, M, K, y, part, nullptr, ya, nullptr, st)) != cudaSuccess) return e;
        if ((e = launch_coldot(B, nullptr, K, N, ya, part, nullptr, yab, nullptr, st)) != cudaSuccess) return e;
        *launches += 4;
    } else {
        if ((e = cudaMemsetAsync(yab, 0, (size_t)std::max<int64_t>(N, 1) * sizeof(double), st)) != cudaSuccess)
            return e;
    }
    if ((e = launch_coldot(C, c0, M, N, y, part, part2, yc, yc0, st)) != cudaSuccess) return e;
    if (!has_c0 && (e = cudaMemsetAsync(yc0, 0, (size_t)std::max<int64_t>(N, 1) * sizeof(double), st)) != cudaSuccess)
        return e;
    residual_norms_kernel<<<1, kNormThreads, 0, st>>>(yc, yc0, yab, N, alpha, has_c0 ? beta : 0.0, svec, norms + 8);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *launches += 3;
    if (norms_dev) *norms_dev = norms;
    return cudaSuccess;
}

void residual_from_norms(const double* nr, gao_residual* out) {
    out->right = nr[1] > 0.0 ? nr[0] / nr[1] : nr[0];
    out->right_inf = nr[3] > 0.0 ? nr[2] / nr[3] : nr[2];
    out->right_argmax = (int64_t)nr[4];
    out->left = nr[9] > 0.0 ? nr[8] / nr[9] : nr[8];
    out->left_inf = nr[11] > 0.0 ? nr[10] / nr[11] : nr[10];
    out->left_argmax = (int64_t)nr[12];
}

}  // namespace gao

extern "C" gao_status gao_gemm_residual_scratch(int64_t M, int64_t N, int64_t K, uint64_t* bytes) {
    using namespace gao;
    if (!bytes) return fail(GAO_EINVAL, "bytes is null");
    if (M < 1 || N < 1 || K < 0) return fail(GAO_EINVAL, "gao_gemm_residual_scratch: M, N >= 1 and K >= 0");
    *bytes = gemm_residual_scratch_bytes(M, N, K);
    return GAO_OK;
}

extern "C" gao_status gao_gemm_residual(const float* A, const float* B, const float* C0, const float* C, int64_t M,
                                        int64_t N, int64_t K, double alpha, double beta, const double* x,
                                        const double* y, void* scratch, uint64_t scratch_bytes, double* r_out,
                                        double* s_out, gao_residual* out, void* stream) {
    using namespace gao;
    if (!out) return fail(GAO_EINVAL, "gao_gemm_residual: out is null");
    if (M < 1 || N < 1 || K < 0) return fail(GAO_EINVAL, "gao_gemm_residual: M, N >= 1 and K >= 0");
    if (!C || !x || !y || !scratch || (K > 0 && (!A || !B)))
        return fail(GAO_EINVAL, "gao_gemm_residual: null device pointer");
    if (scratch_bytes < gemm_residual_scratch_bytes(M, N, K) || ((uintptr_t)scratch & 255u))
        return fail(GAO_EINVAL, "gao_gemm_residual: scratch too small or not 256-byte aligned");
    if (M > (1LL << 40) || N > (1LL << 40) || K > (1LL << 40))
        return fail(GAO_EINVAL, "gao_gemm_residual: dimension too large");
    gao_status s = check_device(nullptr);
    if (s != GAO_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double h[16];
    const double* nd = nullptr;
    int launches = 0;
    cudaError_t e = launch_gemm_residual(A, B, C0, C, M, N, K, alpha, beta, x, y, scratch, r_out, s_out, st,
                                         &launches, &nd);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, nd, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "gao_gemm_residual");
    residual_from_norms(h, out);
    return GAO_OK;
}
