// FP32 SIMT GEMM on the CUDA cores: C = alpha * A @ B + beta * C0.
//
// The "plain FP32" comparison path.  128 x 128 block tile, K step 16, 256 threads,
// each thread an 8 x 8 register tile (two 4-row by two 4-column quadrants so that
// shared-memory reads are 16-byte and conflict-free), shared memory double buffered
// with one barrier per K step.  Accuracy: a single binary32 accumulator over a long
// K grows its rounding error with K, so the K loop is split into chunks of `kchunk`
// elements; each chunk is summed from zero in registers and then added into a
// shared-memory tile of running sums (element-major, so every access is conflict-free),
// which keeps the registers under 128 for two blocks per SM.  A and B are row-major
// (A: M x K, B: K x N).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gao_internal.h"

namespace gao {
namespace {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int kThreads = 256;
constexpr size_t kTileFloats = 2 * (size_t)BK * (BM + BN);       // double-buffered A and B tiles
constexpr size_t kSmemBytes = (kTileFloats + 64 * kThreads) * 4;  // + the chunk-sum tile

template <bool VEC>
__global__ void __launch_bounds__(kThreads, 2)
    sgemm_kernel(float* C, const float* __restrict__ A, const float* __restrict__ B,
                 const float* C0, int64_t M, int64_t N, int64_t K, float alpha, float beta, int64_t kc) {
    extern __shared__ __align__(16) float smem[];
    float* As = smem;                       // [2][BK][BM]
    float* Bs = smem + 2 * BK * BM;         // [2][BK][BN]
    float* sum = smem + kTileFloats;        // [64][kThreads]: element-major, conflict-free
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    // global -> register staging: A row am, k offsets ak..ak+7; B rows bk and bk+8,
    // columns bn..bn+3
    const int am = t >> 1, ak = (t & 1) * 8;
    const int bk = t >> 5, bn = (t & 31) * 4;
    float ra[8], rb[8];

    auto load = [&](int64_t k0) {
        const int64_t gm = m0 + am;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t gk = k0 + ak + 4 * h;
            if (VEC) {
                float4 v = make_float4(0, 0, 0, 0);
                if (gm < M && gk < K) v = *reinterpret_cast<const float4*>(A + gm * K + gk);
                ra[4 * h] = v.x, ra[4 * h + 1] = v.y, ra[4 * h + 2] = v.z, ra[4 * h + 3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) ra[4 * h + q] = (gm < M && gk + q < K) ? A[gm * K + gk + q] : 0.0f;
            }
            const int64_t gkb = k0 + bk + 8 * h, gn = n0 + bn;
            if (VEC) {
                float4 v = make_float4(0, 0, 0, 0);
                if (gkb < K && gn < N) v = *reinterpret_cast<const float4*>(B + gkb * N + gn);
                rb[4 * h] = v.x, rb[4 * h + 1] = v.y, rb[4 * h + 2] = v.z, rb[4 * h + 3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) rb[4 * h + q] = (gkb < K && gn + q < N) ? B[gkb * N + gn + q] : 0.0f;
            }
        }
    };
    auto store = [&](int buf) {
        float* as = As + buf * BK * BM;
        float* bs = Bs + buf * BK * BN;
#pragma unroll
        for (int q = 0; q < 8; ++q) as[(ak + q) * BM + am] = ra[q];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<float4*>(bs + (bk + 8 * h) * BN + bn) =
                make_float4(rb[4 * h], rb[4 * h + 1], rb[4 * h + 2], rb[4 * h + 3]);
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll
    for (int e = 0; e < 64; ++e) sum[e * kThreads + t] = 0.0f;

    const int64_t nk = (K + BK - 1) / BK;
    if (nk > 0) {
        load(0);
        store(0);
    }
    __syncthreads();
    for (int64_t kt = 0; kt < nk; ++kt) {
        const int buf = (int)(kt & 1);
        if (kt + 1 < nk) load((kt + 1) * BK);
        const float* as = As + buf * BK * BM;
        const float* bs = Bs + buf * BK * BN;
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(as + k * BM + ty * 4);
            const float4 a1 = *reinterpret_cast<const float4*>(as + k * BM + 64 + ty * 4);
            const float4 b0 = *reinterpret_cast<const float4*>(bs + k * BN + tx * 4);
            const float4 b1 = *reinterpret_cast<const float4*>(bs + k * BN + 64 + tx * 4);
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
                for (int j = 0; j < 8; ++j) sum[(i * 8 + j) * kThreads + t] += acc[i][j], acc[i][j] = 0.0f;
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
            for (int q = 0; q < 4; ++q) r[q] = alpha * sum[(i * 8 + h * 4 + q) * kThreads + t];
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
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sgemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sgemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (vec)
        sgemm_kernel<true><<<grid, kThreads, kSmemBytes, st>>>(C, A, B, C0, M, N, K, alpha, beta, kc);
    else
        sgemm_kernel<false><<<grid, kThreads, kSmemBytes, st>>>(C, A, B, C0, M, N, K, alpha, beta, kc);
    return cudaGetLastError();
}

}  // namespace gao
