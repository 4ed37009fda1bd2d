// Generation loop: selection, crossover and incremental evaluation.
#pragma once
#include "common.cuh"

struct gp_pop;

struct GenBufs {
    bool evaluated;
};

template <typename Alloc>
int gen_alloc(GenBufs& g, const DevPop& d, Alloc alloc) {
    (void)d; (void)alloc;
    g.evaluated = false;
    return 0;
}

inline void gen_mark_evaluated(GenBufs& g) { g.evaluated = true; }

int gen_crossover(gp_pop* pop, uint32_t generation);
int gen_incremental(gp_pop* pop);
