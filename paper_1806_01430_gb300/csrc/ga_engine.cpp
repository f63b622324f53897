// Simple GA of the offload search (Sec. 3.3, Sec. 4; parameters Sec. 5.1.2).
//
// Initialisation -> evaluation -> roulette selection with elite preservation ->
// one-point crossover (rate Pc) -> mutation (rate Pm) -> repeat for T evaluated
// generations; the answer is the lowest-time gene found.  A gene measured before is
// not measured again (Sec. 4): its first time is reused.
//
// All random draws come from one SplitMix64 stream in a fixed order (one draw per
// initial gene; per child pair: roulette, roulette, crossover test, [cut point],
// one mutation draw per bit of each child), so a seeded run is reproducible and
// any implementation that draws in the same order gives the same trajectory.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <unordered_map>
#include <vector>

#include "gao_internal.h"
#include "ga_engine.h"

namespace gao {

namespace {

struct Sm64 {
    uint64_t s;
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ULL;
        return sm64_mix(s);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
    uint64_t below(uint64_t n) { return ((next() >> 32) * n) >> 32; }
};

double fitness_of(double t) {
    if (!isfinite(t) || t <= 0.0) return 0.0;
    return 1.0 / sqrt(t);
}

size_t roulette(Sm64& r, const std::vector<double>& fit) {
    double total = 0.0;
    for (double f : fit) total += f;
    if (total <= 0.0) return (size_t)r.below(fit.size());
    const double x = r.uniform() * total;
    double acc = 0.0;
    for (size_t i = 0; i < fit.size(); ++i) {
        acc += fit[i];
        if (x < acc) return i;
    }
    for (size_t i = fit.size(); i-- > 0;)
        if (fit[i] > 0.0) return i;
    return fit.size() - 1;
}

uint64_t mutate(Sm64& r, uint64_t c, int n_genes, double pm, int mode) {
    if (mode == 0) {
        for (int b = 0; b < n_genes; ++b)
            if (r.uniform() < pm) c ^= 1ULL << b;
    } else {
        if (r.uniform() < pm) c ^= 1ULL << r.below((uint64_t)n_genes);
    }
    return c;
}

}  // namespace

double ga_fitness(double seconds) { return fitness_of(seconds); }

gao_status ga_core(int n_genes, const gao_ga_params& p, const TimeFn& time_of, gao_ga_result* res) {
    PopFn each = [&](const std::vector<uint64_t>& genes, std::vector<double>* secs) {
        secs->assign(genes.size(), -1.0);
        for (size_t i = 0; i < genes.size(); ++i) {
            const gao_status st = time_of(genes[i], &(*secs)[i]);
            if (st != GAO_OK) return st;
        }
        return GAO_OK;
    };
    return ga_core_pop(n_genes, p, each, res);
}

gao_status ga_core_pop(int n_genes, const gao_ga_params& p, const PopFn& eval, gao_ga_result* res) {
    if (n_genes < 1 || n_genes > 64) return fail(GAO_EINVAL, "gene length must be in [1, 64]");
    if (p.pop < 1 || p.generations < 1) return fail(GAO_EINVAL, "pop and generations must be >= 1");
    if (!(p.pc >= 0.0 && p.pc <= 1.0) || !(p.pm >= 0.0 && p.pm <= 1.0))
        return fail(GAO_EINVAL, "pc and pm must be in [0, 1]");
    if (!res) return fail(GAO_EINVAL, "result is null");
    Sm64 rng{p.seed};
    const int M = p.pop;
    std::vector<uint64_t> popu((size_t)M);
    for (int i = 0; i < M; ++i) popu[(size_t)i] = rng.next() >> (64 - n_genes);
    std::unordered_map<uint64_t, double> cache;
    bool have_best = false;
    res->best_mask = popu[0];
    res->best_s = INFINITY;
    res->evaluations = 0;
    res->cache_hits = 0;
    std::vector<double> times((size_t)M), fit((size_t)M);
    for (int g = 0; g < p.generations; ++g) {
        const auto g_start = std::chrono::steady_clock::now();
        int ev = 0, hits = 0;
        // distinct genes not measured yet, in population order
        std::vector<uint64_t> fresh;
        for (int i = 0; i < M; ++i) {
            const uint64_t m = popu[(size_t)i];
            if (cache.find(m) == cache.end() && std::find(fresh.begin(), fresh.end(), m) == fresh.end())
                fresh.push_back(m);
        }
        if (!fresh.empty()) {
            std::vector<double> secs;
            const gao_status st = eval(fresh, &secs);
            if (st != GAO_OK) return st;  // systemic failure: stop the search
            if (secs.size() != fresh.size()) return fail(GAO_EINVAL, "gene evaluation returned the wrong count");
            for (size_t j = 0; j < fresh.size(); ++j) cache.emplace(fresh[j], secs[j]);
        }
        for (int i = 0; i < M; ++i) {
            const uint64_t m = popu[(size_t)i];
            times[(size_t)i] = cache.find(m)->second;
            // the first individual carrying a fresh gene measured it; every other one is served
            const auto pos = std::find(fresh.begin(), fresh.end(), m);
            if (pos != fresh.end()) {
                ++ev;
                fresh.erase(pos);
            } else {
                ++hits;
            }
        }
        for (int i = 0; i < M; ++i) fit[(size_t)i] = fitness_of(times[(size_t)i]);
        res->evaluations += ev;
        res->cache_hits += hits;
        if (res->populations) memcpy(res->populations + (size_t)g * M, popu.data(), sizeof(uint64_t) * M);
        int gbest = -1;
        double okn = 0.0, oksum = 0.0;
        for (int i = 0; i < M; ++i) {
            const double t = times[(size_t)i];
            if (fit[(size_t)i] > 0.0) {
                oksum += t;
                okn += 1.0;
                if (gbest < 0 || t < times[(size_t)gbest]) gbest = i;
                if (!have_best || t < res->best_s) {
                    res->best_mask = popu[(size_t)i];
                    res->best_s = t;
                    have_best = true;
                }
            }
        }
        if (res->history) {
            gao_ga_gen& h = res->history[g];
            h.best_mask = gbest >= 0 ? popu[(size_t)gbest] : popu[0];
            h.best_s = gbest >= 0 ? times[(size_t)gbest] : INFINITY;
            h.mean_s = okn > 0.0 ? oksum / okn : INFINITY;
            h.evaluated = ev;
            h.cache_hits = hits;
            h.wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - g_start).count();
        }
        if (g == p.generations - 1) break;
        std::vector<uint64_t> nxt;
        nxt.reserve((size_t)M);
        if (p.elite) {
            int e = 0;
            for (int i = 1; i < M; ++i)
                if (fit[(size_t)i] > fit[(size_t)e]) e = i;
            nxt.push_back(popu[(size_t)e]);
        }
        while ((int)nxt.size() < M) {
            uint64_t c1 = popu[roulette(rng, fit)];
            uint64_t c2 = popu[roulette(rng, fit)];
            if (rng.uniform() < p.pc && n_genes >= 2) {
                const uint64_t cut = 1 + rng.below((uint64_t)(n_genes - 1));
                const uint64_t low = (1ULL << cut) - 1;
                const uint64_t a = (c1 & low) | (c2 & ~low), b = (c2 & low) | (c1 & ~low);
                c1 = a;
                c2 = b;
            }
            c1 = mutate(rng, c1, n_genes, p.pm, p.mutation);
            c2 = mutate(rng, c2, n_genes, p.pm, p.mutation);
            nxt.push_back(c1);
            if ((int)nxt.size() < M) nxt.push_back(c2);
        }
        popu.swap(nxt);
    }
    return GAO_OK;
}

}  // namespace gao
