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
//   FP8     e4m3 operands with one power-of-two scale per (row of A, 128-element K block)
//           and per (128-element K block, column of B): 2^e with e the smallest exponent
//           that brings the block's max |x| to <= 448.  The scales travel with the operand
//           tiles (TMA) into tensor memory (tcgen05.cp), and block-scaled MMAs (kind::
//           mxf8f6f4, UE8M0 scales, one per 32-element K step, the 128-block's scale
//           repeated over its four steps) apply them inside the tensor core, so the binary32
//           accumulator runs over all of K as for the bfloat16 products.
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
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gao_internal.h"
#include "gemm_tc.h"

namespace gao {
namespace {

constexpr int BM = 128;  // UMMA M (one TMEM lane per output row)
constexpr int BK = 64;   // 64 bfloat16 = 128 bytes = one swizzle row
constexpr int BK8 = 128; // 128 e4m3 = 128 bytes = one swizzle row
constexpr int kEpiWarps = 8;
constexpr int kMaxSmemProblems = 512;  // grouped launch: problem starts kept in shared memory
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

// Pull one tile of a tensor into L2 (no shared memory, no barrier: a hint only).
__device__ __forceinline__ void tma_prefetch_l2_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)map), "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---- CTA pairs (a cluster of two CTAs on neighbouring SMs sharing one 256-row tile) ----------

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Address in CTA `rank` of the cluster of the shared-memory location `a` of this CTA.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Arrive on an mbarrier of another CTA of the cluster (release at cluster scope).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an mbarrier of
// either CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t cluster_bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(cluster_bar)
        : "memory");
}
// 3-D tile (the scale-factor blocks of one K block) into this CTA's shared memory, counted on
// an mbarrier of either CTA of the pair.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                                 uint32_t cluster_bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
        "%3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(cluster_bar)
        : "memory");
}
// Issued by the pair's first CTA: each CTA's shared memory at this offset into its own tensor
// memory at taddr (tcgen05.cp .32x128b.warpx4, cta_group::2).
__device__ __forceinline__ void tmem_cp_pair_32x128b_x4(uint32_t taddr, uint64_t sdesc) {
    asm volatile("tcgen05.cp.cta_group::2.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}
// Block-scaled e4m3 MMA of a pair: M = 256, each CTA's rows scaled by the A factors in its own
// tensor memory, and every column by the B factors that each CTA holds for all N columns.
__device__ __forceinline__ void mma_mxf8_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}
// Completion of the pair's MMAs signalled on the mbarrier at the same offset in both CTAs.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((uint16_t)3)
        : "memory");
}
// ... on this CTA's mbarrier only.
__device__ __forceinline__ void mma_commit_pair_local(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// With PAIR, one warp of each CTA of the pair allocates (and frees) together: both get the
// same tensor-memory address, the pair's MMAs write each CTA's rows into its own.
template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    if constexpr (PAIR)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                     : "memory");
    else
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                     : "memory");
}
template <bool PAIR>
__device__ __forceinline__ void tmem_relinquish() {
    if constexpr (PAIR) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    else asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    if constexpr (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// The same MMA with the A collector buffer (coll as in prod_coll; a constant after unrolling),
// on one CTA or (PAIR) on a CTA pair.
#define GAO_MMA_F16(CG, COLL)                                                                               \
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"                                        \
                 "tcgen05.mma.cta_group::" CG ".kind::f16" COLL " [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem), \
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)                                        \
                 : "memory")
template <bool PAIR>
__device__ __forceinline__ void mma_bf16_coll(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate, int coll) {
    if constexpr (PAIR) {
        switch (coll) {
            case 1: GAO_MMA_F16("2", ".collector::a::fill"); break;
            case 2: GAO_MMA_F16("2", ".collector::a::use"); break;
            case 3: GAO_MMA_F16("2", ".collector::a::lastuse"); break;
            default: GAO_MMA_F16("2", "");
        }
    } else {
        switch (coll) {
            case 1: GAO_MMA_F16("1", ".collector::a::fill"); break;
            case 2: GAO_MMA_F16("1", ".collector::a::use"); break;
            case 3: GAO_MMA_F16("1", ".collector::a::lastuse"); break;
            default: GAO_MMA_F16("1", "");
        }
    }
}
#undef GAO_MMA_F16

// Block-scaled e4m3 MMA: A's and B's UE8M0 scale factors are read from tensor memory at
// sfa / sfb (the byte of each 32-bit word chosen by the instruction descriptor's scale ids).
__device__ __forceinline__ void mma_mxf8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t sfa,
                                         uint32_t sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// 32 lanes x 128 bits from shared memory into tensor memory, the same rows into each of
// the four lane quadrants (tcgen05.cp .32x128b.warpx4).
__device__ __forceinline__ void tmem_cp_32x128b_x4(uint32_t taddr, uint64_t sdesc) {
    asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

// Contiguous bytes (16-byte aligned, a multiple of 16) global -> shared, completion on an mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(bar)
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
// (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
// (M = 256 for a CTA pair: 128 rows of A from each CTA).
template <int N_, int M_ = BM>
__host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(M_ >> 4) << 24);
}

// Instruction descriptor for kind::mxf8f6f4 with e4m3 A and B (format code 0 at bits 7-9
// and 10-12), both K-major, UE8M0 scale factors (bit 23), N >> 3 at bits 17-22, M >> 4 at
// 24-28; the byte of the scale words used by this MMA (its 32-element K step within the
// 128-element block) is B's scale id at bits 4-5 and A's at bits 29-30.
template <int N_, int M_ = BM>
__host__ __device__ constexpr uint32_t idesc_mxf8(int kk) {
    return ((uint32_t)kk << 4) | (1u << 23) | ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(M_ >> 4) << 24) |
           ((uint32_t)kk << 29);
}

// Shared-memory descriptor of a 32 x 16-byte block without swizzle (8-row core matrices of
// 128 contiguous bytes, 128 bytes apart): the scale-factor block of a tcgen05.cp.
__device__ __forceinline__ uint64_t plain_32x16_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Scale factors of one 128-row (or 128-column) tile and one 128-element K block: 512 bytes
// laid out as tcgen05.cp .32x128b.warpx4 puts them in tensor memory for the block-scaled
// MMA: row r's scale for the K step kk at byte 16 (r % 32) + 4 (r / 32) + kk.
constexpr int kSfBlock = 512;

// Products (plane of A, plane of B); planes: 0 = hi, 1 = mid (x6) or lo (x3), 2 = lo.
//   x1: hi.hi;  x3: hi.hi, hi.lo, lo.hi;  x6: hi.hi, hi.mid, hi.lo, mid.hi, mid.mid, lo.hi
// Products that share A's plane follow one another, so that the tensor core's A collector
// buffer holds the plane across them (read from shared memory once, not once per product).
__host__ __device__ constexpr int prod_a(int nprod, int i) {
    return nprod == 6 ? (i < 3 ? 0 : (i < 5 ? 1 : 2)) : (nprod == 3 ? (i == 2 ? 1 : 0) : 0);
}
__host__ __device__ constexpr int prod_b(int nprod, int i) {
    return nprod == 6 ? (i == 1 || i == 4 ? 1 : (i == 2 ? 2 : 0)) : (nprod == 3 ? (i == 1 ? 1 : 0) : 0);
}
// A collector use of product i: 0 none, 1 fill (read A, keep it), 2 use, 3 last use.
__host__ __device__ constexpr int prod_coll(int nprod, int i) {
    return nprod == 6 ? (i == 0 || i == 3 ? 1 : (i == 1 ? 2 : (i == 2 || i == 4 ? 3 : 0)))
                      : (nprod == 3 ? (i == 0 ? 1 : (i == 1 ? 3 : 0)) : 0);
}
static_assert(prod_a(6, 0) == 0 && prod_b(6, 0) == 0 && prod_a(6, 1) == 0 && prod_b(6, 1) == 1 && prod_a(6, 2) == 0 &&
                  prod_b(6, 2) == 2 && prod_a(6, 3) == 1 && prod_b(6, 3) == 0 && prod_a(6, 4) == 1 &&
                  prod_b(6, 4) == 1 && prod_a(6, 5) == 2 && prod_b(6, 5) == 0,
              "x6 product table");
static_assert(prod_a(3, 0) == 0 && prod_b(3, 0) == 0 && prod_a(3, 1) == 0 && prod_b(3, 1) == 1 && prod_a(3, 2) == 1 &&
                  prod_b(3, 2) == 0,
              "x3 product table");
// every collector run: a fill, then uses of the same A plane, ended by a last use
static_assert(prod_coll(6, 0) == 1 && prod_coll(6, 1) == 2 && prod_coll(6, 2) == 3 && prod_coll(6, 3) == 1 &&
                  prod_coll(6, 4) == 3 && prod_coll(6, 5) == 0 && prod_coll(3, 0) == 1 && prod_coll(3, 1) == 3 &&
                  prod_coll(3, 2) == 0 && prod_coll(1, 0) == 0,
              "collector table");



// Write 32 consecutive columns [gcol, gcol+32) of row grow from binary32 values v.
// With a fused chain, also D = C + alpha2 X (same single rounding as the AXPY loop),
// E = D^T (for each column the warp's 32 rows are 32 consecutive floats of an E row: a
// coalesced 128-byte store), and the thread's sum of D^2 into *sq.
// C0 and X are read through the non-coherent read-only path: within the kernel every
// element of C0 is read once, by the thread that later overwrites it when C aliases C0,
// and X is never written, so these loads need not wait behind earlier stores.
// Shared-memory staging of the epilogue: one 32 x 16 binary32 block per warp, rows 80
// bytes apart, so that both the row-per-lane writes and the row-major reads are free of
// bank conflicts (one two-way conflict on the reads).
constexpr int kStgStride = 20;                       // floats per staged row
constexpr uint32_t kStgBytes = 32 * kStgStride * 4;  // per epilogue warp

// Final values of 32 columns [gcol, gcol + 32) of the warp's 32 rows (row0 + lane holds
// v[0..31], a row per lane as tensor memory delivers them): alpha v + beta C0 stored to C,
// and for a fused chain D = C + alpha2 X, E = D^T and the running sum of D^2.  Each 32 x 16
// half goes through the warp's staging block and is then handled row-major -- four
// consecutive columns per lane in 16-byte accesses where rows are 16-byte aligned, one
// column per lane (16 lanes per row) elsewhere -- so that C0, X, C and D move in 64-byte
// row segments; every element is formed with the same operations as in the separate loops.
template <bool MAYFUSE = true>  // false: the chain code is left out (FP8 never carries one)
__device__ __forceinline__ void store_staged32(const EpiArgs& e, int64_t row0, int64_t gcol, const float* v,
                                               float* stg, int lane, double* sq) {
    const bool fuse = MAYFUSE && e.fuse != 0;
    float s2 = 0.0f, s3 = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        __syncwarp();  // the previous half's reads are done
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(stg + lane * kStgStride + 4 * j) =
                make_float4(v[16 * h + 4 * j], v[16 * h + 4 * j + 1], v[16 * h + 4 * j + 2], v[16 * h + 4 * j + 3]);
        __syncwarp();
        if (e.vec) {
            // rows of a multiple of four floats, 16-byte aligned: lane (row group lane / 4,
            // quadruple lane % 4) moves four consecutive columns of rows lane / 4 + 8 it in
            // 16-byte accesses (a quadruple is wholly inside or outside the N columns)
            const int cq = lane & 3;
            const int64_t c = gcol + 16 * h + 4 * cq;
            const bool cin = c < e.N;
            // all of this half's C0 (and X) loads in flight before any is used
            float4 c0p[4], xp[4];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int64_t grow = row0 + it * 8 + (lane >> 2);
                c0p[it] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                xp[it] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (cin && grow < e.M) {
                    const int64_t base = grow * (e.ldc > 0 ? e.ldc : (int64_t)e.N) + c;
                    if (e.beta != 0.0f) c0p[it] = __ldg(reinterpret_cast<const float4*>(e.C0 + base));
                    if (fuse) xp[it] = __ldg(reinterpret_cast<const float4*>(e.X + base));
                }
            }
            float dd[4][4];  // fused chain: this lane's D values, staged back for the transposed store
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int r = it * 8 + (lane >> 2);
                const int64_t grow = row0 + r;
#pragma unroll
                for (int q = 0; q < 4; ++q) dd[it][q] = 0.0f;
                if (!cin || grow >= e.M) continue;
                const float4 a = *reinterpret_cast<const float4*>(stg + r * kStgStride + 4 * cq);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float c0v[4] = {c0p[it].x, c0p[it].y, c0p[it].z, c0p[it].w};
                const float xv[4] = {xp[it].x, xp[it].y, xp[it].z, xp[it].w};
                const int64_t base = grow * (e.ldc > 0 ? e.ldc : (int64_t)e.N) + c;
                float cv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    cv[q] = e.alpha * av[q];
                    if (e.beta != 0.0f) cv[q] = fmaf(e.beta, c0v[q], cv[q]);
                }
                *reinterpret_cast<float4*>(e.C + base) = make_float4(cv[0], cv[1], cv[2], cv[3]);
                if (fuse) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) dd[it][q] = fmaf(e.alpha2, xv[q], cv[q]);  // D = C + alpha2 X, one rounding
                    *reinterpret_cast<float4*>(e.D + base) = make_float4(dd[it][0], dd[it][1], dd[it][2], dd[it][3]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (q & 1) s3 = fmaf(dd[it][q], dd[it][q], s3);
                        else s2 = fmaf(dd[it][q], dd[it][q], s2);
                    }
                }
            }
            if (fuse) {
                __syncwarp();
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int r = it * 8 + (lane >> 2);
                    *reinterpret_cast<float4*>(stg + r * kStgStride + 4 * cq) =
                        make_float4(dd[it][0], dd[it][1], dd[it][2], dd[it][3]);
                }
            }
        } else {
            // rows of any length: lane (j = lane % 16, rh = lane / 16) takes column j of this
            // half in rows rh, rh + 2, ..., rh + 30, so that every access of the warp covers two
            // 64-byte row segments whatever the rows' alignment; the loads of eight rows go out
            // before any is used; D goes back into the element's own staging slot (its lane
            // owns it)
            const int j = lane & 15, rh = lane >> 4;
            const int64_t col = gcol + 16 * h + j;
            const bool cin = col < e.N;
#pragma unroll 1
            for (int b8 = 0; b8 < 2; ++b8) {
                float t[8], u[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int64_t grow = row0 + rh + 2 * (8 * b8 + k);
                    t[k] = 0.0f;
                    u[k] = 0.0f;
                    if (cin && grow < e.M) {
                        const int64_t base = grow * (e.ldc > 0 ? e.ldc : (int64_t)e.N) + col;
                        if (e.beta != 0.0f) t[k] = __ldg(e.C0 + base);
                        if (fuse) u[k] = __ldg(e.X + base);
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int r = rh + 2 * (8 * b8 + k);
                    const int64_t grow = row0 + r;
                    float dv = 0.0f;
                    if (cin && grow < e.M) {
                        const int64_t base = grow * (e.ldc > 0 ? e.ldc : (int64_t)e.N) + col;
                        float o = e.alpha * stg[r * kStgStride + j];
                        if (e.beta != 0.0f) o = fmaf(e.beta, t[k], o);
                        e.C[base] = o;
                        if (fuse) {
                            dv = fmaf(e.alpha2, u[k], o);  // D = C + alpha2 X, one rounding
                            e.D[base] = dv;
                            if (k & 1) s3 = fmaf(dv, dv, s3);
                            else s2 = fmaf(dv, dv, s2);
                        }
                    }
                    if (fuse) stg[r * kStgStride + j] = dv;  // rows >= M and columns >= N staged as +0
                }
            }
        }
        if (fuse) {
            // E = D^T: D is back in the staging block; each lane writes its own row's 16 values
            // down 16 columns of E, so that every store covers 32 rows of E in one 128-byte
            // segment
            __syncwarp();
            if (e.rsum_part) {
                // these 32 rows are block row0 / 32 of the E rows gcol + 16h + 0..15: two lanes
                // per column form the block's quadruples (rows >= M were staged as +0) and
                // combine them in the fixed row-sum order
                const int cc = lane & 15, hb = lane >> 4;
                float x[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float* col = stg + (4 * (4 * hb + k)) * kStgStride + cc;
                    x[k] = (col[0] + col[kStgStride]) + (col[2 * kStgStride] + col[3 * kStgStride]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) x[k] += __shfl_xor_sync(0xffffffffu, x[k], 16);  // q_k + q_k+4
                const float blk = (x[0] + x[2]) + (x[1] + x[3]);
                const int64_t col = gcol + 16 * h + cc;
                if (hb == 0 && col < e.N) e.rsum_part[(row0 / kRowsumBlock) * e.ldR + col] = blk;
            }
            const int64_t grow = row0 + lane;
            if (grow < e.M) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 d = *reinterpret_cast<const float4*>(stg + lane * kStgStride + 4 * j);
                    const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t col = gcol + 16 * h + 4 * j + q;
                        if (col < e.N) e.E[col * e.ldE + grow] = dv[q];
                    }
                }
            }
        }
    }
    __syncwarp();  // the staging block is free for the caller's next group
    if (fuse) *sq += (double)s2 + (double)s3;
}

// PAIR: a cluster of two CTAs computes a 256 x BN tile with M = 256 MMAs issued by the first
// CTA; each CTA holds 128 rows of A and BN / 2 rows of B^T per stage (the pair's B tile is
// split by columns), and 128 rows of the accumulator in its own tensor memory.
template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED, bool FP8 = false, bool PAIR = false>
struct TcCfg {
    static constexpr uint32_t A_TILE = BM * 128;  // 128 rows x 128 bytes
    static constexpr uint32_t B_TILE = (PAIR ? BN / 2 : BN) * 128;
    static constexpr int TILE_M = PAIR ? 2 * BM : BM;  // rows of a tile
    static constexpr uint32_t STAGE = PA * A_TILE + PB * B_TILE;
    // With more than one product, hi.hi accumulates in its own tensor-memory block and
    // the smaller products in a second one, so the large accumulator takes one rounded
    // addition per K step instead of NPROD.
    static constexpr bool SPLIT = NPROD > 1;
    static constexpr int BUF_COLS = (SPLIT ? 2 : 1) * BN;  // columns of one accumulator buffer
    // FP8: each stage's scale factors in tensor memory after the accumulators, 4 columns
    // for A's 128 rows and BN / 32 for B's BN columns
    static constexpr int SF_COLS = FP8 ? 4 + BN / 32 : 0;
    // accumulator buffers: with two, a tile's epilogue overlaps the next tile's MMAs; one
    // where two do not fit in tensor memory next to the scale factors (FP8, 256 columns)
    static constexpr int ACC = 2 * BUF_COLS + STAGES * SF_COLS <= 512 ? 2 : 1;
    static constexpr int SF_COL0 = ACC * BUF_COLS;
    static constexpr int COLS = ACC * BUF_COLS + STAGES * SF_COLS;
    static constexpr uint32_t TMEM_COLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256
                                                                                                              : 512;
    static constexpr uint32_t NBARS = 2 * STAGES + 2 * ACC + 1;
    static constexpr int EPI_ARRIVALS = (PAIR ? 2 : 1) * kEpiWarps;  // per drained accumulator
    static constexpr uint32_t STG = kEpiWarps * kStgBytes;  // epilogue staging blocks
    // FP8: scale-factor blocks of every stage (A's, then BN / 128 of B's), after the tiles
    static constexpr uint32_t SF_STAGE = FP8 ? (uint32_t)kSfBlock * (1 + BN / 128) : 0;
    static constexpr size_t SMEM = 1024 /*align slack*/ + (size_t)STAGES * (STAGE + SF_STAGE) + STG + 8 * NBARS + 16;
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert(COLS <= 512, "accumulators exceed tensor memory");
    static_assert(BN % 64 == 0 && BN >= 64 && BN <= 256, "BN");
    static_assert(!CHUNKED || BN <= 128, "chunked sums live in registers: BN <= 128");
    static_assert(!FP8 || (!CHUNKED && NPROD == 1 && PA == 1 && PB == 1), "FP8 runs one plane, scaled in the MMA");
    static_assert(!CHUNKED || ACC == 2, "K chunks drain the accumulator while the next chunk runs");
};

// One 128 x BN output tile (row tile tm, column tile tn) of one problem.
// Row tile tm and column tile tn of tile `bid` in a tiles_m x tiles_n grid: groups of
// `group` row tiles (16 by default), row tile fastest inside a group, so the tiles
// processed at the same time share A row panels and B column panels in L2.
__device__ __forceinline__ void raster(int bid, int tiles_m, int tiles_n, int group, int& tm, int& tn) {
    const int GROUP = group > 0 ? group : 16;
    const int group_tiles = GROUP * tiles_n;
    const int first_m = (bid / group_tiles) * GROUP;
    const int gm = min(tiles_m - first_m, GROUP);
    tm = first_m + (bid % group_tiles) % gm;
    tn = (bid % group_tiles) / gm;
}

// Everything one output tile needs.
struct TileInfo {
    const CUtensorMap* ta;
    const CUtensorMap* tb;
    const CUtensorMap* tsa;  // FP8 on CTA pairs: scale-factor blocks of A and B (3-D maps)
    const CUtensorMap* tsb;
    EpiArgs ep;
    int Mp, Np, num_kb, chunk_kb, m0, n0;
    int pf_kb;  // operand tiles are pulled into L2 this many K blocks ahead of their loads (0: off)
    int tiles_n;  // column tiles of the problem (row-major index of the norm partials)
    unsigned long long *span_start, *span_end;  // the problem's time span in the launch (null: none)
};

// Tiles of one problem (kernel arguments).
struct OneProblem {
    const CUtensorMap* ta;
    const CUtensorMap* tb;
    EpiArgs ep;
    int Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, group, bn, pf_kb, bm;  // bm: rows of a tile
    const CUtensorMap* tsa = nullptr;
    const CUtensorMap* tsb = nullptr;
    __device__ __forceinline__ void get(int t, TileInfo& ti) const {
        int tm, tn;
        raster(t, tiles_m, tiles_n, group, tm, tn);
        ti.ta = ta;
        ti.tb = tb;
        ti.tsa = tsa;
        ti.tsb = tsb;
        ti.ep = ep;
        ti.Mp = Mp;
        ti.Np = Np;
        ti.num_kb = num_kb;
        ti.chunk_kb = chunk_kb;
        ti.m0 = tm * bm;
        ti.n0 = tn * bn;
        ti.pf_kb = pf_kb;
        ti.tiles_n = tiles_n;
        ti.span_start = ti.span_end = nullptr;
    }
};

// Tiles of a grouped launch: tile t belongs to the problem whose range holds t
// (binary search over tile_start, which increases along the table).
struct ProblemTable {
    const TcProblem* probs;
    int nprob, bn;
    const int* starts;  // shared-memory copy of every problem's tile_start (null: read probs)
    __device__ __forceinline__ void get(int t, TileInfo& ti) const {
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((starts ? starts[mid] : probs[mid].tile_start) <= t) lo = mid;
            else hi = mid - 1;
        }
        const TcProblem* P = probs + lo;
        int tm, tn;
        raster(t - P->tile_start, P->tiles_m, P->tiles_n, P->group, tm, tn);
        ti.ta = &P->ta;
        ti.tb = &P->tb;
        ti.tsa = ti.tsb = nullptr;
        ti.ep = P->ep;
        ti.Mp = P->Mp;
        ti.Np = P->Np;
        ti.num_kb = P->num_kb;
        ti.chunk_kb = P->chunk_kb;
        ti.m0 = tm * BM;
        ti.n0 = tn * bn;
        ti.pf_kb = P->pf_kb;
        ti.tiles_n = P->tiles_n;
        ti.span_start = P->span_start;
        ti.span_end = P->span_end;
    }
};

// Persistent body: the CTA serves tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The
// shared-memory stage ring and the two tensor-memory accumulator buffers carry on
// from tile to tile, so the producer runs ahead into the next tile and the MMAs of a
// tile overlap the epilogue of the previous one.
template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED, bool FP8, bool PAIR, class Src>
__device__ __forceinline__ void gemm_tc_persistent(const Src& src, int total_tiles, int* err) {
    using Cfg = TcCfg<BN, PA, PB, NPROD, STAGES, CHUNKED, FP8, PAIR>;
    constexpr uint32_t IDESC = idesc_bf16<BN, Cfg::TILE_M>();
    // a CTA pair serves tile c, c + clusters, ... (c = its cluster); its second CTA (rank 1)
    // holds rows 128..255 of each tile and columns BN / 2.. of each B tile
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const int first_tile = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int tile_step = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
    constexpr int KBE = FP8 ? BK8 : BK;  // elements per K block
    constexpr int ACC = Cfg::ACC;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t tiles = smem_u32(smem);
    const uint32_t sf_smem = tiles + (uint32_t)STAGES * Cfg::STAGE;  // FP8 scale-factor blocks
    float* stg_all = reinterpret_cast<float*>(smem + (size_t)STAGES * (Cfg::STAGE + Cfg::SF_STAGE));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)STAGES * (Cfg::STAGE + Cfg::SF_STAGE) + Cfg::STG);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Cfg::NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * STAGES + ACC + b); };
    const uint32_t tail_bar = bar0 + 8u * (uint32_t)(2 * STAGES + 2 * ACC);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < ACC; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), Cfg::EPI_ARRIVALS);  // a pair: both CTAs' epilogue warps
        }
        mbar_init(tail_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc<PAIR>(smem_u32(tmem_slot), Cfg::TMEM_COLS);
        tmem_relinquish<PAIR>();
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();  // the peer's barriers exist before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int it = 0;  // k blocks issued so far (all tiles)
            bool ok = true;
            for (int t = first_tile; t < total_tiles && ok; t += tile_step) {
                TileInfo ti;
                src.get(t, ti);
                const int a_row = ti.m0 + (int)rank * BM;             // this CTA's 128 rows of A
                const int b_row = ti.n0 + (int)rank * (BN / 2);       // a pair: this CTA's half of B
                tma_prefetch_desc(ti.ta);
                tma_prefetch_desc(ti.tb);
                if (ti.span_start) atomicMin(ti.span_start, gtimer());
                for (int kb = 0; kb < ti.num_kb; ++kb, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (ti.pf_kb > 0) {
                        // K blocks 0..pf_kb at a tile's start, then block kb + pf_kb
                        const int k_last = min(kb + ti.pf_kb, ti.num_kb - 1);
                        for (int k2 = kb == 0 ? 0 : kb + ti.pf_kb; k2 <= k_last; ++k2) {
#pragma unroll
                            for (int p = 0; p < PA; ++p) tma_prefetch_l2_2d(ti.ta, k2 * KBE, p * ti.Mp + a_row);
#pragma unroll
                            for (int p = 0; p < PB; ++p)
                                tma_prefetch_l2_2d(ti.tb, k2 * KBE, p * ti.Np + (PAIR ? b_row : ti.n0));
                        }
                    }
                    if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = tiles + (uint32_t)s * Cfg::STAGE;
                    if constexpr (PAIR) {
                        // both CTAs' loads complete on the first CTA's full barrier, which
                        // the first CTA's producer arms with the pair's bytes
                        const uint32_t fb = cluster_addr(full_bar(s), 0);
                        if (rank == 0) mbar_expect_tx(full_bar(s), 2 * (Cfg::STAGE + Cfg::SF_STAGE));
                        if constexpr (FP8) {
                            // this CTA's rows' scale block, and the blocks of all BN columns (the
                            // pair's MMA scales each CTA's rows by the B factors in its own memory)
                            const uint32_t sd = sf_smem + (uint32_t)s * Cfg::SF_STAGE;
                            tma_load_3d_pair(sd, ti.tsa, 0, kb, a_row / BM, fb);
                            tma_load_3d_pair(sd + (uint32_t)kSfBlock, ti.tsb, 0, kb, ti.n0 / 128, fb);
                        }
#pragma unroll
                        for (int p = 0; p < PA; ++p)
                            tma_load_2d_pair(st + (uint32_t)p * Cfg::A_TILE, ti.ta, kb * KBE, p * ti.Mp + a_row, fb);
#pragma unroll
                        for (int p = 0; p < PB; ++p)
                            tma_load_2d_pair(st + PA * Cfg::A_TILE + (uint32_t)p * Cfg::B_TILE, ti.tb, kb * KBE,
                                             p * ti.Np + b_row, fb);
                        continue;
                    }
                    mbar_expect_tx(full_bar(s), Cfg::STAGE + Cfg::SF_STAGE);
                    if constexpr (FP8) {  // this K block's scale factors of the A and B tiles
                        const uint8_t* sfa = reinterpret_cast<const uint8_t*>(ti.ep.sa);
                        const uint8_t* sfb = reinterpret_cast<const uint8_t*>(ti.ep.sb);
                        const uint32_t sd = sf_smem + (uint32_t)s * Cfg::SF_STAGE;
                        bulk_load(sd, sfa + ((int64_t)(ti.m0 / BM) * ti.num_kb + kb) * kSfBlock, kSfBlock, full_bar(s));
#pragma unroll
                        for (int h = 0; h < BN / 128; ++h)
                            bulk_load(sd + (uint32_t)(1 + h) * kSfBlock,
                                      sfb + ((int64_t)(ti.n0 / 128 + h) * ti.num_kb + kb) * kSfBlock, kSfBlock,
                                      full_bar(s));
                    }
#pragma unroll
                    for (int p = 0; p < PA; ++p)
                        tma_load_2d(st + (uint32_t)p * Cfg::A_TILE, ti.ta, kb * KBE, p * ti.Mp + ti.m0, full_bar(s));
#pragma unroll
                    for (int p = 0; p < PB; ++p)
                        tma_load_2d(st + PA * Cfg::A_TILE + (uint32_t)p * Cfg::B_TILE, ti.tb, kb * KBE,
                                    p * ti.Np + ti.n0, full_bar(s));
                }
            }
            const int first = it > STAGES ? it - STAGES : 0;
            for (int u = first; u < it; ++u) {
                const int s = u % STAGES;
                const uint32_t ph = (uint32_t)(u / STAGES) & 1u;
                if (ok) {
                    // the MMA's release of the last uses of each stage
                    if (!mbar_wait(empty_bar(s), ph, abort_flag, err)) ok = false;
                }
                // let our own copies land (a pair: the first CTA's full barriers count both CTAs'
                // copies; the second CTA's land before the pair's final cluster barrier)
                if (!ok && (!PAIR || rank == 0)) mbar_drain(full_bar(s), ph);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {  // a pair's MMAs are issued by its first CTA
            // ---- MMA issuer ----
            int it = 0, gc = 0;  // k blocks consumed, accumulator chunks used (all tiles)
            bool ok = true;
            for (int t = first_tile; t < total_tiles && ok; t += tile_step) {
                TileInfo ti;
                src.get(t, ti);
                const int nchunks = (ti.num_kb + ti.chunk_kb - 1) / ti.chunk_kb;
                for (int c = 0; c < nchunks; ++c, ++gc) {
                    const int ab = ACC == 1 ? 0 : gc & 1;
                    const uint32_t aph = (uint32_t)(ACC == 1 ? gc : gc >> 1) & 1u;
                    if (!mbar_wait(acce_bar(ab), aph ^ 1u, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(ab * Cfg::BUF_COLS);
                    const int kb0 = c * ti.chunk_kb;
                    const int kb1 = min(ti.num_kb, kb0 + ti.chunk_kb);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % STAGES;
                        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                        if (!mbar_wait(full_bar(s), ph, abort_flag, err)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_base = tiles + (uint32_t)s * Cfg::STAGE;
                        const uint32_t b_base = a_base + PA * Cfg::A_TILE;
                        // FP8: this stage's scale factors into its own tensor-memory columns
                        // (free again: the MMAs that read them last released the stage)
                        const uint32_t sfa_t = tmem + (uint32_t)(Cfg::SF_COL0 + s * Cfg::SF_COLS);
                        const uint32_t sfb_t = sfa_t + 4u;
                        if constexpr (FP8 && PAIR) {  // both CTAs' blocks, each into its own memory
                            const uint32_t sd = sf_smem + (uint32_t)s * Cfg::SF_STAGE;
                            tmem_cp_pair_32x128b_x4(sfa_t, plain_32x16_desc(sd));
#pragma unroll
                            for (int h = 0; h < BN / 128; ++h)
                                tmem_cp_pair_32x128b_x4(sfb_t + 4u * (uint32_t)h,
                                                        plain_32x16_desc(sd + (uint32_t)(1 + h) * kSfBlock));
                        } else if constexpr (FP8) {
                            const uint32_t sd = sf_smem + (uint32_t)s * Cfg::SF_STAGE;
                            tmem_cp_32x128b_x4(sfa_t, plain_32x16_desc(sd));
#pragma unroll
                            for (int h = 0; h < BN / 128; ++h)
                                tmem_cp_32x128b_x4(sfb_t + 4u * (uint32_t)h,
                                                   plain_32x16_desc(sd + (uint32_t)(1 + h) * kSfBlock));
                        }
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {  // 4 MMA K steps of 32 bytes per 128-byte block
#pragma unroll
                            for (int pr = 0; pr < NPROD; ++pr) {
                                const uint64_t ad =
                                    sw128_kmajor_desc(a_base + (uint32_t)prod_a(NPROD, pr) * Cfg::A_TILE + kk * 32);
                                const uint64_t bd =
                                    sw128_kmajor_desc(b_base + (uint32_t)prod_b(NPROD, pr) * Cfg::B_TILE + kk * 32);
                                // first product into each accumulator block of a chunk overwrites it
                                const bool first = kb == kb0 && kk == 0 && (pr == 0 || (Cfg::SPLIT && pr == 1));
                                const uint32_t dd = d + ((Cfg::SPLIT && pr > 0) ? (uint32_t)BN : 0u);
                                if constexpr (FP8 && PAIR)
                                    mma_mxf8_pair(dd, ad, bd, idesc_mxf8<BN, Cfg::TILE_M>(kk), sfa_t, sfb_t,
                                                  first ? 0u : 1u);
                                else if constexpr (FP8)
                                    mma_mxf8(dd, ad, bd, idesc_mxf8<BN>(kk), sfa_t, sfb_t, first ? 0u : 1u);
                                else
                                    mma_bf16_coll<PAIR>(dd, ad, bd, IDESC, first ? 0u : 1u, prod_coll(NPROD, pr));
                            }
                        }
                        if constexpr (PAIR) mma_commit_pair(empty_bar(s));  // frees the stage in both CTAs
                        else mma_commit(empty_bar(s));
                    }
                    if (!ok) break;
                    if constexpr (PAIR) mma_commit_pair(accf_bar(ab));
                    else mma_commit(accf_bar(ab));
                }
            }
            if (!ok) {  // no MMA may still be running when tensor memory is freed
                if constexpr (PAIR) mma_commit_pair_local(tail_bar);
                else mma_commit(tail_bar);
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
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        float* stg = stg_all + ew * (kStgBytes / 4);
        constexpr int G = BN / 2 / 32;  // 32-column groups per thread
        int gc = 0;
        bool ok = true;
        for (int t = first_tile; t < total_tiles && ok; t += tile_step) {
            TileInfo ti;
            src.get(t, ti);
            const EpiArgs& ep = ti.ep;
            const int nchunks = (ti.num_kb + ti.chunk_kb - 1) / ti.chunk_kb;
            const int64_t row0 = (int64_t)ti.m0 + (int64_t)rank * BM + q * 32;
            const int64_t grow = row0 + lane;
            const int n0 = ti.n0;
            double sq = 0.0;  // fused chain: this thread's sum of D^2 over the tile
            // K chunks sum in registers; a single accumulator buffer is copied to registers
            // and released before the stores, so that the next tile's MMAs start at once
            constexpr bool HOLD = CHUNKED || ACC == 1;
            float sum[HOLD ? BN / 2 : 1];
#pragma unroll
            for (int i = 0; i < (HOLD ? BN / 2 : 1); ++i) sum[i] = 0.0f;
            for (int c = 0; c < nchunks; ++c, ++gc) {
                const int ab = ACC == 1 ? 0 : gc & 1;
                const uint32_t aph = (uint32_t)(ACC == 1 ? gc : gc >> 1) & 1u;
                if (c == (nchunks > 2 ? nchunks - 2 : 0) && grow < ep.M) {
                    // the final store reads this thread's C0 (and X) row segment: start
                    // bringing it into L2 a chunk or two ahead
                    const int64_t off = grow * (ep.ldc > 0 ? ep.ldc : (int64_t)ep.N) + n0 + colbase;
#pragma unroll
                    for (int k = 0; k < BN / 2; k += 32) {
                        if (ep.beta != 0.0f) prefetch_l2(ep.C0 + off + k);
                        if (ep.fuse) prefetch_l2(ep.X + off + k);
                    }
                }
                // warp-uniform outcome: the stores below synchronise the warp
                if (!__all_sync(0xffffffffu, mbar_wait(accf_bar(ab), aph, abort_flag, err))) {
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
                    } else if constexpr (HOLD) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) sum[g * 32 + i] = v[i];
                    } else {
                        store_staged32<!FP8>(ep, row0, (int64_t)n0 + colbase + g * 32, v, stg, lane, &sq);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (PAIR) mbar_arrive_remote(cluster_addr(acce_bar(ab), 0));  // the MMA CTA's
                    else mbar_arrive(acce_bar(ab));
                }
            }
            if constexpr (HOLD) {
                if (ok) {
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        store_staged32<!FP8>(ep, row0, (int64_t)n0 + colbase + g * 32, sum + g * 32, stg, lane, &sq);
                }
            }
            if (ep.fuse && ok) {  // fixed butterfly over the warp's rows, one partial per warp
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
                // one slot per (128-row tile, column tile, warp) in row-major tile order, so that
                // CTA pairs and single CTAs sum the same partials in the same order
                const int64_t tile128 = (int64_t)((ti.m0 + (int)rank * BM) / BM) * ti.tiles_n + ti.n0 / BN;
                if (lane == 0 && ep.frob_part) ep.frob_part[tile128 * kEpiWarps + ew] = sq;
            }
            if (ti.span_end && ok && lane == 0) {
                __threadfence();  // the warp's stores of this tile come first
                atomicMax(ti.span_end, gtimer());
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    // a pair: neither CTA leaves while the other may still arrive on its barriers, read its
    // shared memory (the MMAs) or land copies there
    if constexpr (PAIR) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<PAIR>(tmem, Cfg::TMEM_COLS);
    }
}

template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED, bool FP8>
__global__ void __launch_bounds__(kThreadsTc, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EpiArgs ep,
                   int Mp, int Np, int num_kb, int chunk_kb, int tiles_m, int tiles_n, int group, int pf_kb,
                   int* err) {
    const OneProblem src{&tmA, &tmB, ep, Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, group, BN, pf_kb, BM};
    gemm_tc_persistent<BN, PA, PB, NPROD, STAGES, CHUNKED, FP8, false>(src, tiles_m * tiles_n, err);
}

// The same GEMM on CTA pairs: tiles of 256 x BN rows (tiles_m counts 256-row tiles).
// FP8: tmSA / tmSB are the scale-factor blocks of A and B (unused otherwise).
template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED, bool FP8>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreadsTc, 1)
    gemm_tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmSA, const __grid_constant__ CUtensorMap tmSB, EpiArgs ep,
                        int Mp, int Np, int num_kb, int chunk_kb, int tiles_m, int tiles_n, int group, int pf_kb,
                        int* err) {
    const OneProblem src{&tmA,  &tmB, ep, Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, group, BN, pf_kb, 2 * BM,
                         &tmSA, &tmSB};
    gemm_tc_persistent<BN, PA, PB, NPROD, STAGES, CHUNKED, FP8, true>(src, tiles_m * tiles_n, err);
}

template <int BN, int PA, int PB, int NPROD, int STAGES, bool CHUNKED, bool FP8>
__global__ void __launch_bounds__(kThreadsTc, 1)
    gemm_tc_grouped_kernel(const TcProblem* __restrict__ probs, int nprob, int total_tiles, int* err) {
    // every role looks up its tile's problem by binary search over the problems' first
    // tiles: keep them in shared memory (the persistent body synchronises the block
    // before any lookup)
    __shared__ int s_starts[kMaxSmemProblems];
    const bool in_smem = nprob <= kMaxSmemProblems;
    if (in_smem)
        for (int i = threadIdx.x; i < nprob; i += blockDim.x) s_starts[i] = probs[i].tile_start;
    const ProblemTable src{probs, nprob, BN, in_smem ? s_starts : nullptr};
    gemm_tc_persistent<BN, PA, PB, NPROD, STAGES, CHUNKED, FP8, false>(src, total_tiles, err);
}

// Frobenius norm of a fused chain: the per-warp partials summed in index order by one
// block (fixed partition and tree), then the square root.
__global__ void __launch_bounds__(256) frob_partials_kernel(const double* __restrict__ part, int64_t n,
                                                            double* __restrict__ out) {
    __shared__ double w[8];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int i = 0; i < 8; ++i) u += w[i];
        *out = sqrt(u);
    }
}

// Row sums of E from a fused chain's block values (column j of D is row j of E): four
// threads per column, thread b keeping accumulator b of the fixed row-sum order (blocks b,
// b + 4, ... in increasing order), then (u0 + u2) + (u1 + u3) across the four.
__global__ void __launch_bounds__(256) rowsum_blocks_kernel(const float* __restrict__ part, int64_t nblk, int64_t ld,
                                                            int64_t n, float* __restrict__ out) {
    constexpr int kAhead = 8;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j = t >> 2;
    const int b = (int)(t & 3);
    float u = 0.0f;
    if (j < n) {
        int64_t p = b;
        for (; p + 4 * (kAhead - 1) < nblk; p += 4 * kAhead) {
            float v[kAhead];
#pragma unroll
            for (int k = 0; k < kAhead; ++k) v[k] = part[(p + 4 * k) * ld + j];
#pragma unroll
            for (int k = 0; k < kAhead; ++k) u += v[k];
        }
        for (; p < nblk; p += 4) u += part[p * ld + j];
    }
    u += __shfl_xor_sync(0xffffffffu, u, 2);
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    if (j < n && b == 0) out[j] = u;
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
                                                         int64_t Np, int64_t Kp, __nv_bfloat16* __restrict__ out,
                                                         int64_t cb0) {
    __shared__ float tile[64][65];
    const int t = threadIdx.x;
    const int c4 = t & 15, r = t >> 4;
    const int64_t k0 = (int64_t)blockIdx.y * 64, n0 = ((int64_t)blockIdx.x + cb0) * 64;  // columns from 64 cb0 on
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

// The same planes formed straight from the INIT loop's counter hash (element idx of buffer
// `buf` is init_value(seed, buf, idx), times 2^e of its row where rowexp is set), for an
// operand that nothing but this GEMM reads: the binary32 array is never written.  Values,
// splitting and zero padding are those of INIT followed by split_rows / split_cols.
// Eight consecutive elements idx0 .. idx0 + 7 from the hashes of idx0 / 2 .. (idx0 + 7) / 2.
__device__ __forceinline__ void init_gen8(uint64_t seed, uint32_t buf, uint64_t idx0, float (&x)[8]) {
    const uint64_t h0 = idx0 >> 1;
    const bool odd = (idx0 & 1) != 0;
    uint64_t h[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) h[j] = (j < 4 || odd) ? sm64_hash(init_key(seed, buf, h0 + j)) : 0;
    // element idx takes the high 24 bits of hash idx / 2 when idx is even, bits 16..39 when odd
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint64_t he = h[q >> 1], ho = h[(q + 1) >> 1];
        x[q] = odd ? ((q & 1) ? u24_to_value((uint32_t)(ho >> 40)) : u24_to_value((uint32_t)((h[q >> 1] >> 16) & 0xFFFFFFu)))
                   : ((q & 1) ? u24_to_value((uint32_t)((he >> 16) & 0xFFFFFFu)) : u24_to_value((uint32_t)(he >> 40)));
    }
}

template <int P>
__global__ void init_split_rows_kernel(uint64_t seed, uint32_t buf, const int8_t* __restrict__ rowexp, int64_t M,
                                       int64_t K, int64_t Mp, int64_t Kp, __nv_bfloat16* __restrict__ out) {
    const int64_t gpr = Kp / 8;
    const int64_t total = Mp * gpr;
    // (row, group) of the grid-stride index advanced by the stride's quotient and remainder
    // (no 64-bit division in the loop)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t di = stride / gpr, dq = stride % gpr;
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i = g / gpr, q8 = g % gpr;
    for (; g < total; g += stride, i += di, q8 += dq) {
        if (q8 >= gpr) {
            q8 -= gpr;
            ++i;
        }
        const int64_t k0 = q8 * 8;
        float x[8];
        if (i < M && k0 + 8 <= K) {
            init_gen8(seed, buf, (uint64_t)(i * K + k0), x);
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = (i < M && k0 + q < K) ? init_value(seed, buf, (uint64_t)(i * K + k0 + q)) : 0.0f;
        }
        if (rowexp && i < M) {
            const int e = rowexp[i];
#pragma unroll
            for (int q = 0; q < 8; ++q) x[q] = ldexpf(x[q], e);
        }
        split8_store<P>(x, out + i * Kp + k0, Mp * Kp);
    }
}

template <int P>
__global__ void __launch_bounds__(256) init_split_cols_kernel(uint64_t seed, uint32_t buf,
                                                              const int8_t* __restrict__ rowexp, int64_t K, int64_t N,
                                                              int64_t Np, int64_t Kp, __nv_bfloat16* __restrict__ out) {
    __shared__ float tile[64][65];
    const int t = threadIdx.x;
    const int c4 = t & 15, r = t >> 4;
    const int64_t k0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t gk = k0 + r + 16 * j, gn = n0 + 4 * c4;
        float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (gk < K) {
            const uint64_t idx = (uint64_t)(gk * N + gn);
            if (gn + 3 < N && (idx & 1) == 0) {  // two hashes give the four elements
                const uint64_t h0 = sm64_hash(init_key(seed, buf, idx >> 1));
                const uint64_t h1 = sm64_hash(init_key(seed, buf, (idx >> 1) + 1));
                v[0] = u24_to_value((uint32_t)(h0 >> 40));
                v[1] = u24_to_value((uint32_t)((h0 >> 16) & 0xFFFFFFu));
                v[2] = u24_to_value((uint32_t)(h1 >> 40));
                v[3] = u24_to_value((uint32_t)((h1 >> 16) & 0xFFFFFFu));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (gn + q < N) v[q] = init_value(seed, buf, idx + q);
            }
            if (rowexp) {
                const int e = rowexp[gk];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = ldexpf(v[q], e);
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

// ---- FP8 quantise kernels -----------------------------------------------------------------------

// Exponent e of the power-of-two scale of a block whose largest magnitude is amax: the
// smallest e with amax / 2^e <= 448 (e4m3's largest finite value, 1.75 * 2^8), clamped to
// the UE8M0 range; 0 for an all-zero block.
__device__ __forceinline__ int fp8_block_exp(float amax) {
    if (!(amax > 0.0f)) return 0;
    const uint32_t bits = __float_as_uint(amax);
    int e = ilogbf(amax) - 8;
    if (((bits >> 23) & 0xFFu) != 0 && (bits & 0x7FFFFFu) > 0x600000u) e += 1;  // significand above 1.75
    return max(-127, min(127, e));
}

// e4m3 of x * 2^-e (the scaling is exact), rounded to nearest, saturating.
__device__ __forceinline__ uint32_t fp8_pack4(float a, float b, float c, float d, int e) {
    const uint32_t q0 = __nv_cvt_float_to_fp8(ldexpf(a, -e), __NV_SATFINITE, __NV_E4M3);
    const uint32_t q1 = __nv_cvt_float_to_fp8(ldexpf(b, -e), __NV_SATFINITE, __NV_E4M3);
    const uint32_t q2 = __nv_cvt_float_to_fp8(ldexpf(c, -e), __NV_SATFINITE, __NV_E4M3);
    const uint32_t q3 = __nv_cvt_float_to_fp8(ldexpf(d, -e), __NV_SATFINITE, __NV_E4M3);
    return q0 | (q1 << 8) | (q2 << 16) | (q3 << 24);
}

// The 32-bit word of row (or column) r of a 128-row tile in its scale-factor block: the UE8M0
// code e + 127 in all four bytes (the 128-element block's scale for each of its 32-element
// K steps).
__device__ __forceinline__ void put_sf(uint8_t* blk, int r, int e) {
    *reinterpret_cast<uint32_t*>(blk + 16 * (r & 31) + 4 * (r >> 5)) = (uint32_t)(e + 127) * 0x01010101u;
}

// A (M x K) -> q [Mp][Kp] e4m3 and scale-factor blocks sfa [Mp / 128][Kp / 128][512 bytes];
// one warp per (row, K block), lane = 4 k.
__global__ void quant_rows_fp8_kernel(const float* __restrict__ A, int64_t M, int64_t K, int64_t Mp, int64_t Kp,
                                      uint8_t* __restrict__ q, uint8_t* __restrict__ sfa) {
    const int lane = threadIdx.x & 31;
    const int64_t kbs = Kp / 128;
    const int64_t nwork = Mp * kbs;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nwork;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t i = w / kbs, kb = w % kbs, k0 = kb * 128 + lane * 4;
        float x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = (i < M && k0 + t < K) ? A[i * K + k0 + t] : 0.0f;
        float amax = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fmaxf(fabsf(x[2]), fabsf(x[3])));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        const int e = fp8_block_exp(amax);
        *reinterpret_cast<uint32_t*>(q + i * Kp + k0) = fp8_pack4(x[0], x[1], x[2], x[3], e);
        if (lane == 0) put_sf(sfa + ((i / 128) * kbs + kb) * kSfBlock, (int)(i % 128), e);
    }
}

// B (K x N) -> q^T [Np][Kp] e4m3 and scale-factor blocks sfb [Np / 128][Kp / 128][512
// bytes]; CTA = (K block, 32 columns).
__global__ void __launch_bounds__(256) quant_cols_fp8_kernel(const float* __restrict__ B, int64_t K, int64_t N,
                                                             int64_t Np, int64_t Kp, uint8_t* __restrict__ q,
                                                             uint8_t* __restrict__ sfb) {
    __shared__ float tile[128][33];
    __shared__ float red[8][32];
    __shared__ int ex[32];
    const int t = threadIdx.x, c = t & 31, g = t >> 5;
    const int64_t kb = blockIdx.y, n0 = (int64_t)blockIdx.x * 32;
    const int64_t kbs = Kp / 128;
    float m = 0.0f;
    for (int r = g; r < 128; r += 8) {
        const int64_t k = kb * 128 + r, n = n0 + c;
        const float v = (k < K && n < N) ? B[k * N + n] : 0.0f;
        tile[r][c] = v;
        m = fmaxf(m, fabsf(v));
    }
    red[g][c] = m;
    __syncthreads();
    if (g == 0) {
        float a = red[0][c];
        for (int j = 1; j < 8; ++j) a = fmaxf(a, red[j][c]);
        const int e = fp8_block_exp(a);
        ex[c] = e;
        const int64_t n = n0 + c;
        put_sf(sfb + ((n / 128) * kbs + kb) * kSfBlock, (int)(n % 128), e);
    }
    __syncthreads();
    // column n = t / 8 of the tile becomes row n0 + n of q^T; 16 k per thread
    const int n = t >> 3, k16 = (t & 7) * 16;
    const int e = ex[n];
    uint4 o;
    o.x = fp8_pack4(tile[k16 + 0][n], tile[k16 + 1][n], tile[k16 + 2][n], tile[k16 + 3][n], e);
    o.y = fp8_pack4(tile[k16 + 4][n], tile[k16 + 5][n], tile[k16 + 6][n], tile[k16 + 7][n], e);
    o.z = fp8_pack4(tile[k16 + 8][n], tile[k16 + 9][n], tile[k16 + 10][n], tile[k16 + 11][n], e);
    o.w = fp8_pack4(tile[k16 + 12][n], tile[k16 + 13][n], tile[k16 + 14][n], tile[k16 + 15][n], e);
    *reinterpret_cast<uint4*>(q + (n0 + n) * Kp + kb * 128 + k16) = o;
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

// 2-D map over a row-major plane stack: `inner` elements per row (bf16, or e4m3 as
// bytes), box = one 128-byte row segment x box_rows rows, 128-byte swizzle.
// Scale-factor blocks [blocks][kbs][512 bytes] as a 3-D tensor of 32-bit words: a box is one
// K block's 512-byte block of box_blocks consecutive row (or column) blocks.
bool make_sf_map(CUtensorMap* map, void* base, int64_t kbs, int64_t blocks, int box_blocks, std::string* why) {
    cuuint64_t gdim[3] = {(cuuint64_t)(kSfBlock / 4), (cuuint64_t)kbs, (cuuint64_t)blocks};
    cuuint64_t gstride[2] = {(cuuint64_t)kSfBlock, (cuuint64_t)(kbs * kSfBlock)};
    cuuint32_t box[3] = {(cuuint32_t)(kSfBlock / 4), 1, (cuuint32_t)box_blocks};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, base, gdim, gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled (scale factors) failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

bool make_map(CUtensorMap* map, void* base, int64_t inner, int64_t rows, int box_rows, bool fp8, std::string* why) {
    const int esz = fp8 ? 1 : 2;
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)inner * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, gdim,
                          gstride, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return false;
    }
    return true;
}

template <int BN, int P, int NPROD, int STAGES, bool CHUNKED, bool FP8 = false>
cudaError_t launch_mma(const CUtensorMap& ta, const CUtensorMap& tb, const EpiArgs& ep, int Mp, int Np, int num_kb,
                       int chunk_kb, int group, int pf_kb, int* err, cudaStream_t st) {
    // Np is the plane stride (a multiple of 256); only ceil(N / BN) column tiles hold data
    using Cfg = TcCfg<BN, P, P, NPROD, STAGES, CHUNKED, FP8>;
    auto kern = gemm_tc_kernel<BN, P, P, NPROD, STAGES, CHUNKED, FP8>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int tiles_m = Mp / BM, tiles_n = (ep.N + BN - 1) / BN;
    const int64_t total = (int64_t)tiles_m * tiles_n;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    const int64_t grid = std::min<int64_t>(total, (int64_t)sm_count());  // persistent: one CTA per SM
    kern<<<(unsigned)grid, kThreadsTc, Cfg::SMEM, st>>>(ta, tb, ep, Mp, Np, num_kb, chunk_kb, tiles_m, tiles_n, group,
                                                        pf_kb, err);
    return cudaGetLastError();
}


// The pair kernel: Mp a multiple of 256; one cluster of two CTAs per two SMs.
template <int BN, int P, int NPROD, int STAGES, bool CHUNKED, bool FP8 = false>
cudaError_t launch_mma_pair(const CUtensorMap& ta, const CUtensorMap& tb, const EpiArgs& ep, int Mp, int Np,
                            int num_kb, int chunk_kb, int group, int pf_kb, int* err, cudaStream_t st,
                            const CUtensorMap* tsa = nullptr, const CUtensorMap* tsb = nullptr) {
    using Cfg = TcCfg<BN, P, P, NPROD, STAGES, CHUNKED, FP8, true>;
    auto kern = gemm_tc_pair_kernel<BN, P, P, NPROD, STAGES, CHUNKED, FP8>;
    if (FP8 && !(tsa && tsb)) return cudaErrorInvalidValue;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (Mp % (2 * BM) != 0) return cudaErrorInvalidValue;
    const int tiles_m = Mp / (2 * BM), tiles_n = (ep.N + BN - 1) / BN;
    const int64_t total = (int64_t)tiles_m * tiles_n;
    if (total > 0x7fffffff) return cudaErrorInvalidValue;
    // persistent: as many pairs as can be resident at once (a cluster needs two SMs of one
    // GPC, so this can be fewer than half the SMs)
    static int max_clusters = 0;
    if (max_clusters == 0) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(sm_count() & ~1));
        lc.blockDim = dim3(kThreadsTc);
        lc.dynamicSmemBytes = Cfg::SMEM;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &lc) != cudaSuccess || n <= 0) {
            (void)cudaGetLastError();
            n = sm_count() / 2;
        }
        max_clusters = std::min(n, sm_count() / 2);
    }
    const int64_t clusters = std::min<int64_t>(total, (int64_t)max_clusters);
    kern<<<(unsigned)(2 * clusters), kThreadsTc, Cfg::SMEM, st>>>(ta, tb, FP8 ? *tsa : ta, FP8 ? *tsb : tb, ep, Mp,
                                                                  Np, num_kb, chunk_kb, tiles_m, tiles_n, group,
                                                                  pf_kb, err);
    return cudaGetLastError();
}

cudaError_t launch_gemm_fp8(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N, int64_t K,
                            float alpha, float beta, int tile_cfg, void* scratch, size_t scratch_bytes, int* err,
                            cudaStream_t st, TcEvents& ev, std::string* why);

}  // namespace

// FP8 scratch: q(A) [Mp][Kp], q(B^T) [Np][Kp], then the scale-factor blocks of A
// [Mp / 128][Kp / 128][512 bytes] and of B [Np / 128][Kp / 128][512 bytes]
struct Fp8Layout {
    int64_t Mp, Mt, Np, Kp, kbs;  // Mp: stored rows (whole CTA-pair tiles); Mt: rows of 128-row tiles
    size_t qa, qb, sa, sb, total;
};
Fp8Layout fp8_layout(int64_t M, int64_t N, int64_t K) {
    Fp8Layout L;
    L.Mp = ru(std::max<int64_t>(M, 1), 2 * BM);
    L.Mt = ru(std::max<int64_t>(M, 1), BM);
    L.Np = ru(std::max<int64_t>(N, 1), 256);
    L.Kp = ru(std::max<int64_t>(K, 1), BK8);
    L.kbs = L.Kp / BK8;
    L.qa = 0;
    L.qb = ru((int64_t)(L.Mp * L.Kp), 1024);
    L.sa = L.qb + ru(L.Np * L.Kp, 1024);
    L.sb = L.sa + ru((L.Mp / 128) * L.kbs * kSfBlock, 1024);
    L.total = L.sb + ru((L.Np / 128) * L.kbs * kSfBlock, 1024);
    return L;
}

// Planes (or FP8 arrays) first, then binary64 partials for a fused chain's norm
// (8 per 128 x 128 tile), then its row sums' 32-row block values (binary32, [Mp / 32][N]).
size_t tc_planes_bytes(int prec, int64_t M, int64_t N, int64_t K) {
    if (prec == GAO_GEMM_FP8) return fp8_layout(M, N, K).total;
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_BF16X6) return 0;
    const int64_t P = planes_of(prec);
    // A's rows rounded to 256: the tile of a CTA pair
    const int64_t Mp = ru(std::max<int64_t>(M, 1), 2 * BM), Np = ru(std::max<int64_t>(N, 1), 256),
                  Kp = ru(std::max<int64_t>(K, 1), BK);
    return (size_t)ru(P * (Mp + Np) * Kp * 2, 1024);
}

size_t tc_frob_partials_bytes(int64_t M, int64_t N) {
    const int64_t tiles = (ru(std::max<int64_t>(M, 1), 2 * BM) / BM) * ((std::max<int64_t>(N, 1) + 127) / 128);
    return (size_t)ru(tiles * kEpiWarps * (int64_t)sizeof(double), 1024);
}

size_t tc_partials_bytes(int64_t M, int64_t N) {
    const int64_t blocks = ru(std::max<int64_t>(M, 1), 2 * BM) / kRowsumBlock;
    return tc_frob_partials_bytes(M, N) + (size_t)ru(blocks * std::max<int64_t>(N, 1) * 4, 1024);
}

size_t tc_scratch_bytes(int prec, int64_t M, int64_t N, int64_t K) {
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_FP8) return 0;
    return tc_planes_bytes(prec, M, N, K) + tc_partials_bytes(M, N);
}

namespace {
// Tile shape of a split-precision GEMM (see the tile configuration bits in launch_gemm_tc)
// and where its bfloat16 planes live in the scratch.
struct TcShape {
    int P, bn, num_kb, chunk_kb;
    bool chunked, pair;
    int64_t Mp, Np, Kp;
    size_t pb_elems;  // B's planes start this many bfloat16 after A's (room for Mlay rows)
};
TcShape tc_shape(int prec, int64_t M, int64_t Mlay, int64_t N, int64_t K, int kchunk, int tile_cfg,
                 const TcPart* part) {
    TcShape g{};
    g.P = planes_of(prec);
    g.Np = ru(N, 256);
    g.Kp = ru(K, BK);
    g.num_kb = (int)(g.Kp / BK);
    g.chunk_kb = g.num_kb;
    if (kchunk > 0) g.chunk_kb = std::max(1, (int)((kchunk + BK - 1) / BK));
    g.chunked = g.chunk_kb < g.num_kb;
    // tile_cfg bits 0-1: 0 = default, 1 = 128 x 128 tiles, 2 = 128 x 256 (single product,
    // unchunked only); bit 2: L2 prefetch of the operand tiles; bit 3: CTA pairs (256-row
    // tiles on two SMs, each SM loading half of every B tile); bits 4-7: raster group =
    // 2^value row tiles (0: default 16).  The default is the fastest measured shape:
    // 256 x 256 on CTA pairs for the unchunked single product (which the pair's halved B
    // traffic per SM speeds up by 14% at n = 8192), 128 x 128 on one CTA for the split
    // precisions (a pair gains nothing there).
    const int bn_sel = tile_cfg & 3;
    g.bn = 128;
    if (!g.chunked && g.P == 1 && (bn_sel == 2 || bn_sel == 0)) g.bn = 256;
    // a row block must start on a 256-row boundary to run on pairs
    g.pair = ((tile_cfg & 8) != 0 || (bn_sel == 0 && g.P == 1 && !g.chunked)) && !(part && part->row_tile0 % 2 != 0);
    g.Mp = ru(M, g.pair ? 2 * BM : BM);
    // A's planes ([P][Mp][Kp], this call's rows) at the start; B's ([P][Np][Kp]) after room
    // for the whole problem's A planes, so that row blocks can share them
    g.pb_elems = (size_t)g.P * ru(Mlay, 2 * BM) * g.Kp;
    return g;
}
}  // namespace

cudaError_t tc_init_planes(int prec, int which, int64_t M, int64_t N, int64_t K, int kchunk, int tile_cfg,
                           uint64_t seed, uint32_t buf, const int8_t* rowexp, void* scratch, size_t scratch_bytes,
                           cudaStream_t st, int* launches) {
    *launches = 0;
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_BF16X6 || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if (tc_scratch_bytes(prec, M, N, K) > scratch_bytes || ((uintptr_t)scratch & 1023u)) return cudaErrorInvalidValue;
    const TcShape g = tc_shape(prec, M, M, N, K, kchunk, tile_cfg, nullptr);
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(scratch);
    if (which == 0) {  // A (M x K) -> [P][Mp][Kp]
        int64_t blocks = (g.Mp * (g.Kp / 8) + 255) / 256;
        if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
        if (g.P == 3) init_split_rows_kernel<3><<<(unsigned)blocks, 256, 0, st>>>(seed, buf, rowexp, M, K, g.Mp, g.Kp, pa);
        else if (g.P == 2) init_split_rows_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(seed, buf, rowexp, M, K, g.Mp, g.Kp, pa);
        else init_split_rows_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(seed, buf, rowexp, M, K, g.Mp, g.Kp, pa);
    } else {  // B (K x N) -> B^T planes [P][Np][Kp]
        dim3 grid((unsigned)(g.Np / 64), (unsigned)(g.Kp / 64));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        __nv_bfloat16* pb = pa + g.pb_elems;
        if (g.P == 3) init_split_cols_kernel<3><<<grid, 256, 0, st>>>(seed, buf, rowexp, K, N, g.Np, g.Kp, pb);
        else if (g.P == 2) init_split_cols_kernel<2><<<grid, 256, 0, st>>>(seed, buf, rowexp, K, N, g.Np, g.Kp, pb);
        else init_split_cols_kernel<1><<<grid, 256, 0, st>>>(seed, buf, rowexp, K, N, g.Np, g.Kp, pb);
    }
    *launches = 1;
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(int prec, float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                           int64_t K, float alpha, float beta, int kchunk, int tile_cfg, void* scratch,
                           size_t scratch_bytes, int* err, cudaStream_t st, TcEvents& ev, std::string* why,
                           const TcFuse* fuse, const TcPart* part, unsigned ready) {
    ev.launches = 0;
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_FP8) {
        if (why) *why = "precision not available on the tensor-core path";
        return cudaErrorNotSupported;
    }
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (fuse && K <= 0) {
        if (why) *why = "a fused chain needs K > 0";
        return cudaErrorInvalidValue;
    }
    if (K <= 0) {  // empty inner dimension: C = beta * C0, no tensor-core work
        if (ev.k0) record_timing(ev.k0, st);
        cudaError_t e = launch_gemm_simt(C, A, B, C0, M, N, 0, alpha, beta, 0, st);
        if (ev.k1) record_timing(ev.k1, st);
        ev.launches = 1;
        return e;
    }
    if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) {
        if (why) *why = "dimension too large";
        return cudaErrorInvalidValue;
    }
    if (!get_encode(why)) return cudaErrorNotSupported;
    if (prec == GAO_GEMM_FP8) {
        if (fuse || part) {
            if (why) *why = "chains and row blocks are not supported on the FP8 path";
            return cudaErrorInvalidValue;
        }
        return launch_gemm_fp8(C, A, B, C0, M, N, K, alpha, beta, tile_cfg, scratch, scratch_bytes, err, st, ev,
                               why);
    }
    const int64_t Mlay = part ? part->m_layout : M;
    if (Mlay < M || (part && ready)) {
        if (why) *why = "bad row-block arguments";
        return cudaErrorInvalidValue;
    }
    // columns [ncol0, ncol1) of C (all of them unless a row block names a range)
    const int64_t ncol0 = part ? part->n_begin : 0, ncol1 = part && part->n_end >= 0 ? part->n_end : N;
    if (ncol0 < 0 || ncol0 % 256 != 0 || ncol1 > N || ncol1 <= ncol0 || (fuse && (ncol0 != 0 || ncol1 != N))) {
        if (why) *why = "bad column range";
        return cudaErrorInvalidValue;
    }
    const TcShape g = tc_shape(prec, M, Mlay, N, K, kchunk, tile_cfg, part);
    const int P = g.P, num_kb = g.num_kb, chunk_kb = g.chunk_kb, bn = g.bn;
    const bool chunked = g.chunked, pair = g.pair;
    const int64_t Mp = g.Mp, Np = g.Np, Kp = g.Kp;
    const int group = tc_group_of(tile_cfg);
    const int pf_kb = tc_prefetch_of(tile_cfg);
    if (tc_scratch_bytes(prec, Mlay, N, K) > scratch_bytes || ((uintptr_t)scratch & 1023u)) {
        if (why) *why = "tensor-core scratch too small or misaligned";
        return cudaErrorInvalidValue;
    }
    // A's planes: a row block's own region of the room kept for the whole problem's (so that
    // blocks in flight at the same time do not share one), B's after that room
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(scratch) + (part ? (size_t)P * part->row_tile0 * BM * Kp : 0);
    __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(scratch) + g.pb_elems;
    const int sms = sm_count();
    if (!(ready & 1) && !(part && part->a_ready)) {
        const int64_t work = Mp * (Kp / 8);
        int64_t blocks = (work + 255) / 256;
        if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
        if (P == 3) split_rows_kernel<3><<<(unsigned)blocks, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else if (P == 2) split_rows_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else split_rows_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ev.launches += 1;
    }
    if (!(part && part->b_ready) && !(ready & 2)) {
        // B's columns [nb0, nb1) (the column range; to the padded width at the right end)
        const int64_t nb0 = ncol0, nb1 = ncol1 == N ? Np : ncol1;
        dim3 grid((unsigned)((nb1 - nb0 + 63) / 64), (unsigned)(Kp / 64));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        const int64_t cb0 = nb0 / 64;
        if (P == 3) split_cols_kernel<3><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, cb0);
        else if (P == 2) split_cols_kernel<2><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, cb0);
        else split_cols_kernel<1><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, cb0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ev.launches += 1;
    }
    if (ev.planes) {
        cudaError_t e = cudaEventRecord(ev.planes, st);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap ta, tb;
    if (!make_map(&ta, pa, Kp, (int64_t)P * Mp, BM, false, why)) return cudaErrorInvalidValue;
    // a column range reads B's planes from row ncol0 of each plane on: the map starts there and
    // the kernel's plane offsets (multiples of Np) are unchanged
    if (!make_map(&tb, pb + (size_t)ncol0 * Kp, Kp, (int64_t)P * Np - ncol0, pair ? bn / 2 : bn, false, why))
        return cudaErrorInvalidValue;
    float* Cr = C + ncol0;
    const float* C0r = C0 + ncol0;
    const int64_t ncols = ncol1 - ncol0;
    EpiArgs ep{Cr, C0r, (int)M, (int)ncols, alpha, beta,
               (ncols % 4 == 0) && (N % 4 == 0) && ((((uintptr_t)Cr) | ((uintptr_t)C0r)) & 15u) == 0 ? 1 : 0,
               nullptr, nullptr, 0, 0};
    ep.ldc = N;
    double* fpart = reinterpret_cast<double*>(static_cast<char*>(scratch) + tc_planes_bytes(prec, Mlay, N, K));
    float* rpart = reinterpret_cast<float*>(reinterpret_cast<char*>(fpart) + tc_frob_partials_bytes(Mlay, N));
    const int64_t tiles_n = (N + bn - 1) / bn;
    ep.ldE = M;
    if (fuse) {
        ep.X = fuse->X;
        ep.D = fuse->D;
        ep.E = fuse->E;
        ep.ldE = fuse->ldE > 0 ? fuse->ldE : M;
        ep.alpha2 = fuse->alpha2;
        ep.frob_part = fuse->frob_out ? fpart + (part ? part->row_tile0 : 0) * tiles_n * kEpiWarps : nullptr;
        ep.rsum_part = fuse->rowsum_out ? rpart + (part ? part->row_tile0 : 0) * (BM / kRowsumBlock) * N : nullptr;
        ep.ldR = N;
        ep.fuse = 1;
    }
    if (ev.k0) record_timing(ev.k0, st);
    cudaError_t e;
    const int mp = (int)Mp, np = (int)Np;
    if (pair) {
        // stages per variant: as many as fit next to the epilogue's staging blocks
        if (P == 3)
            e = chunked ? launch_mma_pair<128, 3, 6, 2, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st)
                        : launch_mma_pair<128, 3, 6, 2, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err,
                                                               st);
        else if (P == 2)
            e = chunked ? launch_mma_pair<128, 2, 3, 4, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st)
                        : launch_mma_pair<128, 2, 3, 4, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err,
                                                               st);
        else if (chunked)
            e = launch_mma_pair<128, 1, 1, 8, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
        else if (bn == 256)
            e = launch_mma_pair<256, 1, 1, 6, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
        else
            e = launch_mma_pair<128, 1, 1, 8, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    } else if (P == 3)
        e = chunked ? launch_mma<128, 3, 6, 2, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st)
                    : launch_mma<128, 3, 6, 2, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    else if (P == 2)
        e = chunked ? launch_mma<128, 2, 3, 3, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st)
                    : launch_mma<128, 2, 3, 3, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    else if (chunked)
        e = launch_mma<128, 1, 1, 6, true>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    else if (bn == 256)
        e = launch_mma<256, 1, 1, 4, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    else
        e = launch_mma<128, 1, 1, 6, false>(ta, tb, ep, mp, np, num_kb, chunk_kb, group, pf_kb, err, st);
    if (e != cudaSuccess) return e;
    ev.launches += 1;
    if (ev.k1) record_timing(ev.k1, st);
    if (fuse && fuse->frob_out && (!part || part->last)) {
        const int64_t tiles = (ru(Mlay, BM) / BM) * tiles_n;  // every block's tiles
        frob_partials_kernel<<<1, 256, 0, st>>>(fpart, tiles * kEpiWarps, fuse->frob_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ev.launches += 1;
    }
    if (fuse && fuse->rowsum_out && (!part || part->last)) {
        const int64_t nblk = (Mlay + kRowsumBlock - 1) / kRowsumBlock;  // blocks of the whole E row
        rowsum_blocks_kernel<<<(unsigned)((4 * N + 255) / 256), 256, 0, st>>>(rpart, nblk, N, N, fuse->rowsum_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ev.launches += 1;
    }
    return cudaSuccess;
}


namespace {
cudaError_t launch_gemm_fp8(float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N, int64_t K,
                            float alpha, float beta, int tile_cfg, void* scratch, size_t scratch_bytes, int* err,
                            cudaStream_t st, TcEvents& ev, std::string* why) {
    const int group = tc_group_of(tile_cfg);
    // bits 0-1: 1 = 128, 2 = 256 columns per tile; bit 3: CTA pairs (256 rows); default (0):
    // 256 x 256 tiles on CTA pairs
    const int bn_sel = tile_cfg & 3;
    const bool pair = (tile_cfg & 8) != 0 || bn_sel == 0;
    const int bn = bn_sel == 1 ? 128 : 256;
    const Fp8Layout L = fp8_layout(M, N, K);
    if (L.total > scratch_bytes || ((uintptr_t)scratch & 1023u)) {
        if (why) *why = "FP8 scratch too small or misaligned";
        return cudaErrorInvalidValue;
    }
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint8_t *qa = base + L.qa, *qb = base + L.qb;
    uint8_t *sa = base + L.sa, *sb = base + L.sb;
    {
        const int64_t warps = L.Mp * L.kbs;
        int64_t g = (warps * 32 + 255) / 256;
        if (g > (int64_t)sm_count() * 8) g = (int64_t)sm_count() * 8;
        quant_rows_fp8_kernel<<<(unsigned)g, 256, 0, st>>>(A, M, K, L.Mp, L.Kp, qa, sa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(L.Np / 32), (unsigned)L.kbs);
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        quant_cols_fp8_kernel<<<grid, 256, 0, st>>>(B, K, N, L.Np, L.Kp, qb, sb);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ev.launches += 2;
    }
    CUtensorMap ta, tb;
    if (!make_map(&ta, qa, L.Kp, L.Mp, BM, true, why)) return cudaErrorInvalidValue;
    if (!make_map(&tb, qb, L.Kp, L.Np, pair ? bn / 2 : bn, true, why)) return cudaErrorInvalidValue;
    // the epilogue's sa / sb carry the scale-factor blocks (read by the producer's bulk copies
    // on one CTA; CTA pairs load them through the 3-D maps)
    EpiArgs ep{C, C0, (int)M, (int)N, alpha, beta,
               (N % 4 == 0) && ((((uintptr_t)C) | ((uintptr_t)C0)) & 15u) == 0 ? 1 : 0,
               reinterpret_cast<const float*>(sa), reinterpret_cast<const float*>(sb), (int)L.kbs, (int)L.Np};
    if (ev.k0) record_timing(ev.k0, st);
    const int kbs = (int)L.kbs;
    cudaError_t e;
    if (pair) {
        CUtensorMap tsa, tsb;
        if (!make_sf_map(&tsa, sa, L.kbs, L.Mp / 128, 1, why)) return cudaErrorInvalidValue;
        if (!make_sf_map(&tsb, sb, L.kbs, L.Np / 128, bn / 128, why)) return cudaErrorInvalidValue;
        e = bn == 256 ? launch_mma_pair<256, 1, 1, 6, false, true>(ta, tb, ep, (int)L.Mp, (int)L.Np, kbs, kbs, group, 0,
                                                                   err, st, &tsa, &tsb)
                      : launch_mma_pair<128, 1, 1, 8, false, true>(ta, tb, ep, (int)L.Mp, (int)L.Np, kbs, kbs, group, 0,
                                                                   err, st, &tsa, &tsb);
    } else {
        e = bn == 256 ? launch_mma<256, 1, 1, 4, false, true>(ta, tb, ep, (int)L.Mt, (int)L.Np, kbs, kbs, group, 0, err,
                                                              st)
                      : launch_mma<128, 1, 1, 6, false, true>(ta, tb, ep, (int)L.Mt, (int)L.Np, kbs, kbs, group, 0, err,
                                                              st);
    }
    if (e != cudaSuccess) return e;
    ev.launches += 1;
    if (ev.k1) record_timing(ev.k1, st);
    return cudaSuccess;
}
}  // namespace


// ---- grouped launches ------------------------------------------------------------------------------

namespace {

template <int BN, int P, int NPROD, int STAGES, bool CHUNKED, bool FP8 = false>
cudaError_t launch_grouped_t(const TcProblem* d_probs, int nprob, int total_tiles, int* err, cudaStream_t st) {
    using Cfg = TcCfg<BN, P, P, NPROD, STAGES, CHUNKED, FP8>;
    auto kern = gemm_tc_grouped_kernel<BN, P, P, NPROD, STAGES, CHUNKED, FP8>;
    static bool attr_set = false;  // per instantiation
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (total_tiles <= 0) return cudaSuccess;
    const int grid = std::min(total_tiles, sm_count());  // persistent: one CTA per SM
    kern<<<(unsigned)grid, kThreadsTc, Cfg::SMEM, st>>>(d_probs, nprob, total_tiles, err);
    return cudaGetLastError();
}

}  // namespace

bool tc_available(std::string* why) { return get_encode(why); }

cudaError_t tc_prepare(int prec, float* C, const float* A, const float* B, const float* C0, int64_t M, int64_t N,
                       int64_t K, float alpha, float beta, int kchunk, int tile_cfg, void* scratch,
                       size_t scratch_bytes, cudaStream_t st, TcProblem* prob, int* launches, std::string* why,
                       const TcFuse* fuse) {
    *launches = 0;
    memset(prob, 0, sizeof(*prob));
    if (prec < GAO_GEMM_BF16 || prec > GAO_GEMM_FP8 || M <= 0 || N <= 0 || K <= 0 || M > (1 << 30) ||
        N > (1 << 30) || K > (1 << 30)) {
        if (why) *why = "grouped tensor-core GEMM needs a tensor-core precision and positive sizes";
        return cudaErrorInvalidValue;
    }
    if (!get_encode(why)) return cudaErrorNotSupported;
    if (tc_scratch_bytes(prec, M, N, K) > scratch_bytes || ((uintptr_t)scratch & 1023u)) {
        if (why) *why = "tensor-core scratch too small or misaligned";
        return cudaErrorInvalidValue;
    }
    const int vec = (N % 4 == 0) && ((((uintptr_t)C) | ((uintptr_t)C0)) & 15u) == 0 ? 1 : 0;
    if (fuse && prec == GAO_GEMM_FP8) {
        if (why) *why = "chains are not supported on the FP8 path";
        return cudaErrorInvalidValue;
    }
    if (prec == GAO_GEMM_FP8) {
        const Fp8Layout L = fp8_layout(M, N, K);
        uint8_t* base = static_cast<uint8_t*>(scratch);
        uint8_t *qa = base + L.qa, *qb = base + L.qb;
        uint8_t *sa = base + L.sa, *sb = base + L.sb;
        const int64_t warps = L.Mp * L.kbs;
        int64_t g = (warps * 32 + 255) / 256;
        if (g > (int64_t)sm_count() * 8) g = (int64_t)sm_count() * 8;
        quant_rows_fp8_kernel<<<(unsigned)g, 256, 0, st>>>(A, M, K, L.Mp, L.Kp, qa, sa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(L.Np / 32), (unsigned)L.kbs);
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        quant_cols_fp8_kernel<<<grid, 256, 0, st>>>(B, K, N, L.Np, L.Kp, qb, sb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches = 2;
        if (!make_map(&prob->ta, qa, L.Kp, L.Mp, BM, true, why)) return cudaErrorInvalidValue;
        if (!make_map(&prob->tb, qb, L.Kp, L.Np, 128, true, why)) return cudaErrorInvalidValue;
        prob->ep = EpiArgs{C, C0, (int)M, (int)N, alpha, beta, vec, reinterpret_cast<const float*>(sa),
                           reinterpret_cast<const float*>(sb), (int)L.kbs, (int)L.Np};
        prob->Mp = (int)L.Mt;  // one plane: Mp only sets the 128-row tiles
        prob->Np = (int)L.Np;
        prob->num_kb = (int)L.kbs;
        prob->chunk_kb = prob->num_kb;  // one accumulation over K: the scales act inside the MMA
    } else {
        const int P = planes_of(prec);
        const int64_t Mp = ru(M, BM), Np = ru(N, 256), Kp = ru(K, BK);
        __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(scratch);
        __nv_bfloat16* pb = pa + (size_t)P * Mp * Kp;
        const int64_t work = Mp * (Kp / 8);
        int64_t g = (work + 255) / 256;
        if (g > (int64_t)sm_count() * 8) g = (int64_t)sm_count() * 8;
        if (P == 3) split_rows_kernel<3><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else if (P == 2) split_rows_kernel<2><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        else split_rows_kernel<1><<<(unsigned)g, 256, 0, st>>>(A, M, K, Mp, Kp, pa);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(Np / 64), (unsigned)(Kp / 64));
        if (grid.y > 65535u) return cudaErrorInvalidValue;
        if (P == 3) split_cols_kernel<3><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, 0);
        else if (P == 2) split_cols_kernel<2><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, 0);
        else split_cols_kernel<1><<<grid, 256, 0, st>>>(B, K, N, Np, Kp, pb, 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *launches = 2;
        if (!make_map(&prob->ta, pa, Kp, (int64_t)P * Mp, BM, false, why)) return cudaErrorInvalidValue;
        if (!make_map(&prob->tb, pb, Kp, (int64_t)P * Np, 128, false, why)) return cudaErrorInvalidValue;
        prob->ep = EpiArgs{C, C0, (int)M, (int)N, alpha, beta, vec, nullptr, nullptr, 0, 0};
        if (fuse) tc_attach_chain(prec, M, N, K, scratch, *fuse, prob);
        prob->Mp = (int)Mp;
        prob->Np = (int)Np;
        prob->num_kb = (int)(Kp / BK);
        prob->chunk_kb = kchunk > 0 ? std::max(1, (int)((kchunk + BK - 1) / BK)) : prob->num_kb;
    }
    prob->tiles_m = prob->Mp / BM;
    prob->tiles_n = (int)((N + 127) / 128);
    prob->group = tc_group_of(tile_cfg);
    prob->pf_kb = tc_prefetch_of(tile_cfg);
    return cudaSuccess;
}

void tc_attach_chain(int prec, int64_t M, int64_t N, int64_t K, void* scratch, const TcFuse& fuse, TcProblem* prob) {
    // the chain's epilogue, partials in this problem's scratch (tile-local)
    double* fpart = reinterpret_cast<double*>(static_cast<char*>(scratch) + tc_planes_bytes(prec, M, N, K));
    float* rpart = reinterpret_cast<float*>(reinterpret_cast<char*>(fpart) + tc_frob_partials_bytes(M, N));
    prob->ep.X = fuse.X;
    prob->ep.D = fuse.D;
    prob->ep.E = fuse.E;
    prob->ep.ldE = fuse.ldE > 0 ? fuse.ldE : M;
    prob->ep.alpha2 = fuse.alpha2;
    prob->ep.frob_part = fuse.frob_out ? fpart : nullptr;
    prob->ep.rsum_part = fuse.rowsum_out ? rpart : nullptr;
    prob->ep.ldR = N;
    prob->ep.fuse = 1;
}

cudaError_t tc_finalize_chain(int prec, int64_t M, int64_t N, int64_t K, void* scratch, const TcFuse& fuse,
                              cudaStream_t st, int* launches) {
    *launches = 0;
    if (M <= 0 || N <= 0) return cudaSuccess;
    double* fpart = reinterpret_cast<double*>(static_cast<char*>(scratch) + tc_planes_bytes(prec, M, N, K));
    float* rpart = reinterpret_cast<float*>(reinterpret_cast<char*>(fpart) + tc_frob_partials_bytes(M, N));
    if (fuse.frob_out) {
        const int64_t tiles = (ru(M, BM) / BM) * ((N + 127) / 128);  // 128 x 128 tiles of the grouped launch
        frob_partials_kernel<<<1, 256, 0, st>>>(fpart, tiles * kEpiWarps, fuse.frob_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 1;
    }
    if (fuse.rowsum_out) {
        rowsum_blocks_kernel<<<(unsigned)((4 * N + 255) / 256), 256, 0, st>>>(rpart, (M + kRowsumBlock - 1) / kRowsumBlock,
                                                                            N, N, fuse.rowsum_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches += 1;
    }
    return cudaSuccess;
}

cudaError_t tc_launch_grouped(int prec, bool chunked, const TcProblem* d_probs, int nprob, int total_tiles, int* err,
                              cudaStream_t st) {
    // nprob == 0 / total_tiles == 0: only sets the kernel's shared-memory attribute
    switch (prec) {
        case GAO_GEMM_BF16X6:
            return chunked ? launch_grouped_t<128, 3, 6, 2, true>(d_probs, nprob, total_tiles, err, st)
                           : launch_grouped_t<128, 3, 6, 2, false>(d_probs, nprob, total_tiles, err, st);
        case GAO_GEMM_BF16X3:
            return chunked ? launch_grouped_t<128, 2, 3, 3, true>(d_probs, nprob, total_tiles, err, st)
                           : launch_grouped_t<128, 2, 3, 3, false>(d_probs, nprob, total_tiles, err, st);
        case GAO_GEMM_BF16:
            return chunked ? launch_grouped_t<128, 1, 1, 6, true>(d_probs, nprob, total_tiles, err, st)
                           : launch_grouped_t<128, 1, 1, 6, false>(d_probs, nprob, total_tiles, err, st);
        case GAO_GEMM_FP8:
            return launch_grouped_t<128, 1, 1, 6, false, true>(d_probs, nprob, total_tiles, err, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace gao
