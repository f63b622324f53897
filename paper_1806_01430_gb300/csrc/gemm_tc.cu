// Tensor-core GEMM on sm_103a: C = alpha * A @ B + beta * C0 with binary32 A, B, C.
//
// Precision (split bfloat16).  Each binary32 operand x is written as a sum of
// bfloat16 terms, hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid) (every
// subtraction is exact).  The product is the sum of the term products whose
// magnitude matters at binary32 resolution:
//   BF16    1 product : hi.hi
//   BF16X3  3 products: hi.hi + hi.lo + lo.hi          (two-term split, ~2^-16 relative)
//   BF16X6  6 products: hi.hi + hi.mid + mid.hi + mid.mid + hi.lo + lo.hi
//                                                       (three-term split, ~2^-24)
// Each bfloat16 product is exact in binary32; the tensor core accumulates in binary32.
// An optional K chunk restarts the tensor-memory accumulator every `kchunk`
// elements and adds the chunk sums in registers, which bounds the growth of the
// accumulation error with K.
//
// Data flow.  Two memory-bound split kernels write the bfloat16 planes of A
// (M x K, K contiguous) and of B transposed (N x K, K contiguous), zero-padded to
// the tile grid.  The MMA kernel is warp-specialised, one 128 x BN output tile per
// CTA (cta_group::1), 320 threads:
//   warp 0     TMA producer: cp.async.bulk.tensor 2-D loads of every plane's
//              128 x 64 (A) and BN x 64 (B) tile into a STAGES-deep ring of
//              128-byte-swizzled shared-memory stages, completion on mbarriers;
//   warp 1     allocates tensor memory; one lane issues tcgen05.mma (kind::f16,
//              M = 128, N = BN, K = 16) for every product and 16-element K step,
//              and tcgen05.commit releases each stage and each finished accumulator;
//   warps 2-9  epilogue: tcgen05.ld 32 lanes x 32 columns per warp, alpha/beta
//              and the store to C (rows of TMEM lane quadrant warp%4, columns split
//              in two halves).
// Every mbarrier wait is bounded by the global timer; on expiry the kernel writes
// its error word, lets in-flight copies and MMAs finish (bounded), frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "gao_internal.h"

namespace gao {
namespace {

constexpr int BM = 128;  // UMMA M (one TMEM lane per output row)
constexpr int BK = 64;   // 64 bfloat16 = 128 bytes = one swizzle row
constexpr int kEpiWarps = 8;
constexpr int kThreadsTc = 64 + 32 * kEpiWarps;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr unsigned long long kDrainLimitNs = 200000000ull;  // 0.2 s

// ---- PTX wrappers -----------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the mbarrier at `a`; false if the kernel aborted or the
// wait expired (then the error word is set and every role is told to stop).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(a, parity)) return true;
        if ((i & 63u) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > kWaitLimitNs) {
                *abort_flag = 1;
                atomicExch(err, DEV_WAIT_TIMEOUT);
                return false;
            }
        }
    }
}

// Bounded wait used only while draining after an abort.
__device__ __forceinline__ void mbar_drain(uint32_t a, uint32_t parity) {
    const unsigned long long t0 = gtimer();
    while (!mbar_try(a, parity))
        if (gtimer() - t0 > kDrainLimitNs) return;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte
// offset), leading byte offset unused for this layout (encoded 1), descriptor
// version 1 (bit 46), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor for kind::f16: D binary32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
template <int N_>
__host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// Products (plane of A, plane of B); planes: 0 = hi, 1 = mid (x6) or lo (x3), 2 = lo.
//   x1: hi.hi;  x3: hi.hi, hi.lo, lo.hi;  x6: hi.hi, hi.mid, mid.hi, mid.mid, hi.lo, lo.hi
__host__ __device__ constexpr int prod_a(int nprod, int i) {
    return nprod == 6 ? (i == 2 || i == 3 ? 1 : (i == 5 ? 2 : 0)) : (nprod == 3 ? (i == 2 ? 1 : 0) : 0);
}
__host__ __device__ constexpr int prod_b(int nprod, int i) {
    return nprod == 6 ? (i == 1 || i == 3 ? 1 : (i == 4 ? 2 : 0)) : (nprod == 3 ? (i == 1 ? 1 : 0) : 0);
}
static_assert(prod_a(6, 0) == 0 && prod_b(6, 0) == 0 && prod_a(6, 1) == 0 && prod_b(6, 1) == 1 && prod_a(6, 2) == 1 &&
                  prod_b(6, 2) == 0 && prod_a(6, 3) == 1 && prod_b(6, 3) == 1 && prod_a(6, 4) == 0 &&
                  prod_b(6, 4) == 2 && prod_a(6, 5) == 2 && prod_b(6, 5) == 0,
              "x6 product table");
static_assert(prod_a(3, 0) == 0 && prod_b(3, 0) == 0 && prod_a(3, 1) == 0 && prod_b(3, 1) == 1 && prod_a(3, 2) == 1 &&
                  prod_b(3, 2) == 0,
              "x3 product table");

struct EpiArgs {
    float* C;
    const float* C0;
    int M, N;
    float alpha, beta;
    int vec;  // C, C0 16-byte aligned and N % 4 == 0
};

// Write 32 consecutive columns [gcol, gcol+32) of row grow from binary32 values v.
__device__ __forceinline__ void store_row32(const EpiArgs& e, int64_t grow, int64_t gcol, const float* v) {
    if (grow >= e.M) return;
    float* crow = e.C + grow * (int64_t)e.N;
    const float* c0row = e.C0 + grow * (int64_t)e.N;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t c = gcol + 4 * j;
        if (e.vec && c + 3 < e.N) {
            float4 o = make_float4(e.alpha * v[4 * j], e.alpha * v[4 * j + 1], e.alpha * v[4 * j + 2],
                                   e.alpha * v[4 * j + 3]);
            if (e.beta != 0.0f) {
                const float4 c0 = *reinterpret_cast<const float4*>(c0row + c);
                o.x = fmaf(e.beta, c0.x, o.x);
                o.y = fmaf(e.beta, c0.y, o.y);
                o.z = fmaf(e.beta, c0.z, o.z);
                o.w = fmaf(e.beta, c0.w, o.w);
            }
            *reinterpret_cast<float4*>(crow + c) = o;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (c + q < e.N) {
                    float o = e.alpha * v[4 * j + q];
                    if (e.beta != 0.0f) o = fmaf(e.beta, c0row[c + q], o);
                    crow[c + q] = o;
                }
            }
        }
    }
}

template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED>
struct TcCfg {
    static constexpr uint32_t A_TILE = BM * BK * 2;
    static constexpr uint32_t B_TILE = BN * BK * 2;
    static constexpr uint32_t STAGE = PA * A_TILE + PB * B_TILE;
    static constexpr int ACC = CHUNKED ? 2 : 1;  // accumulator buffers (double-buffered when chunked)
    // With more than one product, hi.hi accumulates in its own tensor-memory block and
    // the smaller products in a second one, so the large accumulator takes one rounded
    // addition per K step instead of NPROD.
    static constexpr bool SPLIT = NPROD > 1;
    static constexpr int BUF_COLS = (SPLIT ? 2 : 1) * BN;  // columns of one accumulator buffer
    static constexpr int COLS = ACC * BUF_COLS;
    static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256
                                                                                                              : 512;
    static constexpr uint32_t NBARS = 2 * STAGES + 2 * ACC + 1;
    static constexpr size_t SMEM = 1024 /*align slack*/ + (size_t)STAGES * STAGE + 8 * NBARS + 16;
    static_assert(COLS <= 512, "accumulators exceed tensor memory");
    static_assert(BN % 64 == 0 && BN >= 64 && BN <= 256, "BN");
    static_assert(!CHUNKED || BN <= 128, "chunked sums live in registers: BN <= 128");
};

template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED>
__global__ void __launch_bounds__(kThreadsTc, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiArgs ep,
                   int Mp, int Np, int num_kb, int chunk_kb, int tiles_m, int tiles_n, int* err) {
    using Cfg = TcCfg<BN, PA, PB, NPROD, STAGES, CHUNKED>;
    constexpr uint32_t IDESC = idesc_bf16<BN>();
    constexpr int ACC = Cfg::ACC;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t tiles = smem_u32(smem);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)STAGES * Cfg::STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Cfg::NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * STAGES + ACC + b); };
    const uint32_t tail_bar = bar0 + 8u * (uint32_t)(2 * STAGES + 2 * ACC);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // tile of this CTA: groups of 16 row-tiles, row-tile fastest inside a group, so the
    // CTAs of one wave share A row panels and B column panels in L2
    const int bid = blockIdx.x;
    constexpr int GROUP = 16;
    const int group_tiles = GROUP * tiles_n;
    const int first_m = (bid / group_tiles) * GROUP;
    const int gm = min(tiles_m - first_m, GROUP);
    const int tm = first_m + (bid % group_tiles) % gm;
    const int tn = (bid % group_tiles) / gm;
    const int m0 = tm * BM, n0 = tn * BN;
    const int nchunks = (num_kb + chunk_kb - 1) / chunk_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < ACC; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), kEpiWarps);
        }
        mbar_init(tail_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), Cfg::TMEM_COLS);
        tmem_relinquish();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int issued = 0;
            bool ok = true;
            for (int kb = 0; kb < num_kb; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, err)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(full_bar(s), Cfg::STAGE);
                const uint32_t st = tiles + (uint32_t)s * Cfg::STAGE;
#pragma unroll
                for (int p = 0; p < PA; ++p)
                    tma_load_2d(st + (uint32_t)p * Cfg::A_TILE, &tmA, kb * BK, p * Mp + m0, full_bar(s));
#pragma unroll
                for (int p = 0; p < PB; ++p)
                    tma_load_2d(st + PA * Cfg::A_TILE + (uint32_t)p * Cfg::B_TILE, &tmB, kb * BK, p * Np + n0,
                                full_bar(s));
                issued = kb + 1;
            }
            const int first = issued > STAGES ? issued - STAGES : 0;
            for (int kb = first; kb < issued; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (ok) {
                    // the MMA's release of the last uses of each stage
                    if (!mbar_wait(empty_bar(s), ph, abort_flag, err)) ok = false;
                }
                if (!ok) mbar_drain(full_bar(s), ph);  // let our own copies land
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                const int ab = CHUNKED ? (c & 1) : 0;
                const uint32_t aph = CHUNKED ? ((uint32_t)(c >> 1) & 1u) : ((uint32_t)c & 1u);
                if (!mbar_wait(acce_bar(ab), aph ^ 1u, abort_flag, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * Cfg::BUF_COLS);
                const int kb0 = c * chunk_kb;
                const int kb1 = min(num_kb, kb0 + chunk_kb);
                for (int kb = kb0; kb < kb1; ++kb) {
                    const int s = kb % STAGES;
                    const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                    if (!mbar_wait(full_bar(s), ph, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = tiles + (uint32_t)s * Cfg::STAGE;
                    const uint32_t b_base = a_base + PA * Cfg::A_TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                        for (int pr = 0; pr < NPROD; ++pr) {
                            const uint64_t ad =
                                sw128_kmajor_desc(a_base + (uint32_t)prod_a(NPROD, pr) * Cfg::A_TILE + kk * 32);
                            const uint64_t bd =
                                sw128_kmajor_desc(b_base + (uint32_t)prod_b(NPROD, pr) * Cfg::B_TILE + kk * 32);
                            // first product into each accumulator block of a chunk overwrites it
                            const bool first = kb == kb0 && kk == 0 && (pr == 0 || (Cfg::SPLIT && pr == 1));
                            const uint32_t dd = d + ((Cfg::SPLIT && pr > 0) ? (uint32_t)BN : 0u);
                            mma_bf16(dd, ad, bd, IDESC, first ? 0u : 1u);
                        }
                    }
                    mma_commit(empty_bar(s));
                }
                if (!ok) break;
                mma_commit(accf_bar(ab));
            }
            if (!ok) {  // no MMA may still be running when tensor memory is freed
                mma_commit(tail_bar);
                mbar_drain(tail_bar, 0);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue ----
        const int ew = warp - 2;
        const int q = warp & 3;  // TMEM lane quadrant this warp may access
        const int half = ew >> 2;
        const int colbase = half * (BN / 2);
        const int64_t grow = (int64_t)m0 + q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        constexpr int G = BN / 2 / 32;  // 32-column groups per thread
        float sum[CHUNKED ? BN / 2 : 1];
        if (CHUNKED) {
#pragma unroll
            for (int i = 0; i < (CHUNKED ? BN / 2 : 1); ++i) sum[i] = 0.0f;
        }
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int ab = CHUNKED ? (c & 1) : 0;
            const uint32_t aph = CHUNKED ? ((uint32_t)(c >> 1) & 1u) : ((uint32_t)c & 1u);
            if (!mbar_wait(accf_bar(ab), aph, abort_flag, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tb = tmem + lane_addr + (uint32_t)(ab * Cfg::BUF_COLS + colbase);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint32_t r[32];
                float v[32];
                tmem_ld32(tb + (uint32_t)(g * 32), r);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
                if constexpr (Cfg::SPLIT) {  // small products: same columns, second block
                    tmem_ld32(tb + (uint32_t)(BN + g * 32), r);
                    tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] += __uint_as_float(r[i]);
                }
                if constexpr (CHUNKED) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) sum[g * 32 + i] += v[i];
                } else {
                    store_row32(ep, grow, (int64_t)n0 + colbase + g * 32, v);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(ab));
        }
        if constexpr (CHUNKED) {
            if (ok) {
#pragma unroll
                for (int g = 0; g < G; ++g) store_row32(ep, grow, (int64_t)n0 + colbase + g * 32, sum + g * 32);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, Cfg::TMEM_COLS);
    }
}

// ---- split kernels ------------------------------------------------------------------------------

template <int P>
__device__ __forceinline__ void split8_store(const float (&x)[8], __nv_bfloat16* dst, int64_t plane_stride) {
    __align__(16) __nv_bfloat16 h[P][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float r = x[q];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const __nv_bfloat16 b = __float2bfloat16_rn(r);
            h[p][q] = b;
            r = r - __bfloat162float(b);  // exact: the rounding error of a bfloat16 rounding
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        *reinterpret_cast<uint4*>(dst + p * plane_stride) = *reinterpret_cast<const uint4*>(h[p]);
}

// A (M x K, row-major) -> P planes of Mp x Kp bfloat16, zero padded; 8 k per thread.
template <int P>
__global__ void split_rows_kernel(const float* __restrict__ A, int64_t M, int64_t K, int64_t Mp, int64_t Kp,
                                  __nv_bfloat16* __restrict__ out) {
    const int64_t gpr = Kp / 8;
    const int64_t total = Mp * gpr;
    const bool vec = (K % 4 == 0) && (((uintptr_t)A & 15u) == 0);
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / gpr, k0 = (g % gpr) * 8;
        float x[8];
        if (i < M && vec && k0 + 8 <= K) {
            const float4 u = *reinterpret_cast<const float4*>(A + i * K + k0);
            const float4 w = *reinterpret_cast<const float4*>(A + i * K + k0 + 4);
            x[0] = u.x, x[1] = u.y, x[2] = u.z, x[3] = u.w, x[4] = w.x, x[5] = w.y, x[6] = w.z, x[7] = w.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = (i < M && k0 + q < K) ? A[i * K + k0 + q] : 0.0f;
        }
        split8_store<P>(x, out + i * Kp + k0, Mp * Kp);
    }
}

// B (K x N, row-major) -> P planes of B^T, Np x Kp bfloat16, zero padded; 64 x 64 tiles
// through shared memory (coalesced reads along N, 16-byte writes along K).
template <int P>
__global__ void __launch_bounds__(256) split_cols_kernel(const float* __restrict__ B, int64_t K, int64_t N,
                                                         int64_t Np, int64_t Kp, __nv_bfloat16* __restrict__ out) {
    __shared__ float tile[64][65];
    const int t = threadIdx.x;
    const int c4 = t & 15, r = t >> 4;
    const int64_t k0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    const bool vec = (N % 4 == 0) && (((uintptr_t)B & 15u) == 0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t gk = k0 + r + 16 * j, gn = n0 + 4 * c4;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (gk < K) {
            if (vec && gn + 3 < N) {
                const float4 u = *reinterpret_cast<const float4*>(B + gk * N + gn);
                v[0] = u.x, v[1] = u.y, v[2] = u.z, v[3] = u.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = (gn + q < N) ? B[gk * N + gn + q] : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) tile[r + 16 * j][4 * c4 + q] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int idx = t + 256 * h;
        const int n = idx >> 3, kc = idx & 7;
        float x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = tile[kc * 8 + q][n];
        split8_store<P>(x, out + (n0 + n) * Kp + k0 + kc * 8, Np * Kp);
    }
}

// ---- host side ------------------------------------------------------------------------------------

inline int64_t ru(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int planes_of(int prec) { return prec == GAO_GEMM_BF16X6 ? 3 : prec == GAO_GEMM_BF16X3 ? 2 : 1; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

bool get_encode(std::string* why) {
    std::lock_guard<std::mutex> g(g_encode_mu);
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr) {
        if (why) *why = "cuTensorMapEncodeTiled is not available from the driver";
        return false;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return true;
}

bool make_map(CUtensorMap* map, void* base, int64_t inner, int64_t rows, int box_rows, std::string* why) {
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

template <int BN, int P, int NPROD, int STAGES, bool CHUNKED>
cudaError_t launch_mma(const CUtensorMap& ta, const CUtensorMap& tb, const EpiArgs& ep, int Mp, int Np, int num_kb,
                       int chunk_kb, int* err, cudaStream_t st) {
    // Np is the plane stride (a multiple of 256); only ceil(N / BN) column tiles hold data
    using Cfg = TcCfg<BN, P, P, NPROD, STAGES, CHUNKED>;
    auto kern = gemm_tc_kernel<BN, P, P, NPROD, STAGES, CHUNKED>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles_m = Mp / BM, tiles_n = (ep.N + BN - 1) / BN;
    const int64_t grid = (int64_t)tiles_m * tiles_n;
    if (grid > 0x7fffffff) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, kThreadsTc, Cfg::SMEM, st>>>(ta, tb, ep, Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, err);
    return cudaGetLastError();
}

}  // namespace

size_t tc_scratch_bytes(int prec, int64_t M, int64_t N, int64_t K) {
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_BF16X6) return 0;
    const int64_t P = planes_of(prec);
    const int64_t Mp = ru(std::max<int64_t>(M, 1), BM), Np = ru(std::max<int64_t>(N, 1), 256),
                  Kp = ru(std::max<int64_t>(K, 1), BK);
    return (size_t)(P * (Mp + Np) * Kp * 2);
}

cudaError_t launch_gemm_tc(int prec, float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                           int64_t K, float alpha, float beta, int kchunk, int tile_cfg, void* scratch,
                           size_t scratch_bytes, int* err, cudaStream_t st, TcEvents& ev, std::string* why) {
    ev.launches = 0;
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_BF16X6) {
        if (why) *why = "precision not available on the tensor-core path";
        return cudaErrorNotSupported;
    }
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (K <= 0) {  // empty inner dimension: C = beta * C0, no tensor-core work
        if (ev.k0) cudaEventRecord(ev.k0, st);
        cudaError_t e = launch_gemm_simt(C, A, B, C0, M, N, 0, alpha, beta, 0, st);
        if (ev.k1) cudaEventRecord(ev.k1, st);
        ev.launches = 1;
        return e;
    }
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) {
        if (why) *why = "dimension too large";
        return cudaErrorInvalidValue;
    }
    if (!get_encode(why)) return cudaErrorNotSupported;
    const int P = planes_of(prec);
    const int64_t Mp = ru(M, BM), Np = ru(N, 256), Kp = ru(K, BK);
    if (tc_scratch_bytes(prec, M, N, K) > scratch_bytes || ((uintptr_t)scratch & 1023u)) {
        if (why) *why = "tensor-core scratch too small or misaligned";
        return cudaErrorInvalidValue;
    }
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(scratch);
    __nv_bfloat16* pb = pa + (size_t)P * Mp * Kp;
    const int sms = sm_count();
    {
        const int64_t work = Mp * (Kp / 8);
        int64_t g = (work + 255) / 256;
        if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
        if (P == 3) split_rows_kernel<3><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else if (P == 2) split_rows_kernel<2><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else split_rows_kernel<1><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(Np / 64), (unsigned)(Kp / 64));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        if (P == 3) split_cols_kernel<3><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb);
        else if (P == 2) split_cols_kernel<2><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb);
        else split_cols_kernel<1><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ev.launches += 2;
    }
    const int num_kb = (int)(Kp / BK);
    int chunk_kb = num_kb;
    if (kchunk > 0) chunk_kb = std::max(1, (int)((kchunk + BK - 1) / BK));
    const bool chunked = chunk_kb < num_kb;
    // tile_cfg: 0 = default (128 x 256 for the unchunked single product, else 128 x 128),
    // 1 = 128 x 128, 2 = 128 x 256 (single product, unchunked only)
    int bn = 128;
    if (!chunked && P == 1 && (tile_cfg == 2 || tile_cfg == 0)) bn = 256;
    CUtensorMap ta, tb;
    if (!make_map(&ta, pa, Kp, (int64_t)P * Mp, BM, why)) return cudaErrorInvalidValue;
    if (!make_map(&tb, pb, Kp, (int64_t)P * Np, bn, why)) return cudaErrorInvalidValue;
    EpiArgs ep{C, C0, (int)M, (int)N, alpha, beta,
               (N % 4 == 0) && ((((uintptr_t)C) | ((uintptr_t)C0)) & 15u) == 0 ? 1 : 0};
    if (ev.k0) cudaEventRecord(ev.k0, st);
    cudaError_t e;
    const int mp = (int)Mp, np = (int)Np;
    if (P == 3)
        e = chunked ? launch_mma<128, 3, 6, 2, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st)
                    : launch_mma<128, 3, 6, 2, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st);
    else if (P == 2)
        e = chunked ? launch_mma<128, 2, 3, 3, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st)
                    : launch_mma<128, 2, 3, 3, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st);
    else if (chunked)
        e = launch_mma<128, 1, 1, 6, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st);
    else if (bn == 256)
        e = launch_mma<256, 1, 1, 4, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st);
    else
        e = launch_mma<128, 1, 1, 6, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, err, st);
    if (e != cudaSuccess) return e;
    ev.launches += 1;
    if (ev.k1) cudaEventRecord(ev.k1, st);
    return cudaSuccess;
}

}  // namespace gao
