// Simple-GA core shared by ga_run, ga_run_table and the tile autotuner.
#pragma once
#include <functional>
#include <vector>

#include "../../include/gao.h"

namespace gao {

// Measures one gene.  Returns GAO_OK and sets *seconds (negative or non-finite for a
// failed gene), or another status to abort the whole search.
using TimeFn = std::function<gao_status(uint64_t gene, double* seconds)>;

// fitness = seconds^(-1/2), computed as 1/sqrt(seconds); 0 for a failed gene.
double ga_fitness(double seconds);

gao_status ga_core(int n_genes, const gao_ga_params& p, const TimeFn& time_of, gao_ga_result* res);

// Measures several genes at once (the distinct genes of a generation that are not in
// the cache yet, in population order).  Returns GAO_OK and fills seconds (same length).
using PopFn = std::function<gao_status(const std::vector<uint64_t>& genes, std::vector<double>* seconds)>;

// The same GA with per-generation evaluation: identical draws, cache and results as
// ga_core when the times agree.
gao_status ga_core_pop(int n_genes, const gao_ga_params& p, const PopFn& eval, gao_ga_result* res);

// Tile configuration of a 5-bit autotuning gene for GEMM precision `prec`:
// bits 0-1 raster group 4/8/16/32 (log2 2..5, stored in tile_cfg bits 4-7); bits 2-3
// K chunk 64 << v for split precisions, for plain bfloat16 and FP8 tile width 128/256
// (bit 2) and CTA pairs (bit 3, tile_cfg bit 3); bit 4 L2 prefetch of the operand tiles
// (tile_cfg bit 2, BF16 variants).
constexpr int kAutotuneBits = 5;
inline void autotune_decode(int prec, uint64_t gene, int* kchunk, int* tile_cfg) {
    const int glog = 2 + (int)(gene & 3);
    const int v = (int)((gene >> 2) & 3);
    int bn_sel = 0;
    if (prec == GAO_GEMM_BF16X6) {
        *kchunk = 64 << v;  // 64 .. 512: the six-product error stays under 1e-6
        bn_sel = 1;
    } else if (prec == GAO_GEMM_BF16X3) {
        *kchunk = 128 << v;  // 128 .. 1024: the two-term split, not the chunk, sets the error
        bn_sel = 1;
    } else if (prec == GAO_GEMM_BF16 || prec == GAO_GEMM_FP8) {
        *kchunk = 0;
        bn_sel = ((v & 1) ? 2 : 1) | ((v & 2) ? 8 : 0);
    } else {
        *kchunk = 0;
        bn_sel = 1;
    }
    *tile_cfg = bn_sel | (((gene >> 4) & 1) ? 4 : 0) | (glog << 4);
}

}  // namespace gao
