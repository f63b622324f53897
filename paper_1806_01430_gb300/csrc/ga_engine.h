// Simple-GA core shared by ga_run, ga_run_table and the tile autotuner.
#pragma once
#include <functional>

#include "../../include/gao.h"

namespace gao {

// Measures one gene.  Returns GAO_OK and sets *seconds (negative or non-finite for a
// failed gene), or another status to abort the whole search.
using TimeFn = std::function<gao_status(uint64_t gene, double* seconds)>;

// fitness = seconds^(-1/2), computed as 1/sqrt(seconds); 0 for a failed gene.
double ga_fitness(double seconds);

gao_status ga_core(int n_genes, const gao_ga_params& p, const TimeFn& time_of, gao_ga_result* res);

}  // namespace gao
