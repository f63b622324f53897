// FP32 SIMT GEMM on the CUDA cores: C = alpha * A @ B + beta * C0.
//
// The "plain FP32" comparison path.  128 x 128 block tile, K step 8, 256 threads,
// each thread an 8 x 8 register tile (two 4-row by two 4-column quadrants so that
// shared-memory reads are 16-byte and conflict-free), shared memory double buffered
// with one barrier per K step.  Accuracy: a single binary32 accumulator over a long
// K grows its rounding error with K, so the K loop is split into chunks of `kchunk`
// elements; each chunk is summed from zero and then added into a second register
// tile.  A and B are row-major (A: M x K, B: K x N).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gao_internal.h"

namespace gao {
namespace {

constexpr int BM = 128, BN = 128, BK = 8;

template <bool VEC>
__global__ void __launch_bounds__(256, 1)
    sgemm_kernel(float* C, const float* __restrict__ A, const float* __restrict__ B,
                 const float* C0, int64_t M, int64_t N, int64_t K, float alpha, float beta, int64_t kc) {
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    // global -> register staging: A row am, k offset ak..ak+3; B row bk, columns bn..bn+3
    const int am = t >> 1, ak = (t & 1) * 4;
    const int bk = t >> 5, bn = (t & 31) * 4;
    float ra[4], rb[4];

    auto load = [&](int64_t k0) {
        const int64_t gm = m0 + am, gk = k0 + ak;
        if (VEC) {
            float4 v = make_float4(0, 0, 0, 0);
            if (gm < M && gk < K) v = *reinterpret_cast<const float4*>(A + gm * K + gk);
            ra[0] = v.x, ra[1] = v.y, ra[2] = v.z, ra[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) ra[q] = (gm < M && gk + q < K) ? A[gm * K + gk + q] : 0.0f;
        }
        const int64_t gkb = k0 + bk, gn = n0 + bn;
        if (VEC) {
            float4 v = make_float4(0, 0, 0, 0);
            if (gkb < K && gn < N) v = *reinterpret_cast<const float4*>(B + gkb * N + gn);
            rb[0] = v.x, rb[1] = v.y, rb[2] = v.z, rb[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) rb[q] = (gkb < K && gn + q < N) ? B[gkb * N + gn + q] : 0.0f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) As[buf][ak + q][am] = ra[q];
        *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    };

    float acc[8][8], sum[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f, sum[i][j] = 0.0f;

    const int64_t nk = (K + BK - 1) / BK;
    if (nk > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) store(buf ^ 1);
        __syncthreads();
        if (((kt + 1) * BK) % kc == 0 || kt + 1 == nk) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) sum[i][j] += acc[i][j], acc[i][j] = 0.0f;
        }
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (gm >= M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gn = n0 + h * 64 + tx * 4;
            float r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = alpha * sum[i][h * 4 + q];
            if (VEC && gn + 3 < N) {
                if (beta != 0.0f) {
                    const float4 c = *reinterpret_cast<const float4*>(C0 + gm * N + gn);
                    r[0] = fmaf(beta, c.x, r[0]);
                    r[1] = fmaf(beta, c.y, r[1]);
                    r[2] = fmaf(beta, c.z, r[2]);
                    r[3] = fmaf(beta, c.w, r[3]);
                }
                *reinterpret_cast<float4*>(C + gm * N + gn) = make_float4(r[0], r[1], r[2], r[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (gn + q < N) {
                        float v = r[q];
                        if (beta != 0.0f) v = fmaf(beta, C0[gm * N + gn + q], v);
                        C[gm * N + gn + q] = v;
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_gemm_simt(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                             int64_t K, float alpha, float beta, int kchunk, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    int64_t kc = kchunk > 0 ? ((kchunk + BK - 1) / BK) * BK : (int64_t)1 << 62;
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    const bool vec = (K % 4 == 0) && (N % 4 == 0) &&
                     ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)C) | ((uintptr_t)C0)) & 15u) == 0;
    if (vec)
        sgemm_kernel<true><<<grid, 256, 0, st>>>(C, A, B, C0, M, N, K, alpha, beta, kc);
    else
        sgemm_kernel<false><<<grid, 256, 0, st>>>(C, A, B, C0, M, N, K, alpha, beta, kc);
    return cudaGetLastError();
}

}  // namespace gao
