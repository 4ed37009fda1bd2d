/*
 * CPU ORACLE for the GP population hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct restatement of what the paper's method
 * computes.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load it; the product library never does.  It shares no
 * source with the CUDA library.  Build: gcc -O2 -ffp-contract=off (no
 * fast-math), so every FP32 operation is one IEEE single-precision
 * operation rounded to nearest, with no fused multiply-add.
 *
 * Paper: W. B. Langdon, "A Trillion Genetic Programming Instructions per
 * Second" (arXiv 2205.03251).  Each function cites the passage it follows.
 *
 * Encoding (Sec. 3.1, Sec. 5: flattened linear prefix trees, one byte per
 * node): 0 '+', 1 '-', 2 '*', 3 protected '/', 4 x, 5..255 constant
 * k[op-5]; Boolean: 0 AND, 1 OR, 2 NAND, 3 NOR, 4..9 a0 a1 d0 d1 d2 d3
 * (6-multiplexer), or 4..14 a0 a1 a2 d0..d7 (11-multiplexer, input j =
 * bit j of the case index); integer: the arithmetic opcodes over int32
 * with wrap-around.  Binary functions take the first child in prefix
 * order as the left operand.  Protected division returns 1.0 when the
 * divisor compares equal to zero (+0 or -0); otherwise it is the IEEE
 * quotient (integer: 1 for a zero divisor, INT32_MIN for INT32_MIN / -1,
 * else the quotient truncated toward zero).
 *
 * Pins: tests/test_oracle_pins.py (closed-form trees, brute force on every
 * tree of up to 7 nodes against exact rational arithmetic rounded once per
 * operation, the 6-multiplexer solved by a known tree, published
 * SplitMix64 vectors, selection frequencies against their closed forms),
 * tests/test_oracle_wide.py (the 11-multiplexer's known solution and
 * closed-form error counts, the integer set against Python integers by
 * brute force) and tests/test_oracle_disruption.py (hand-worked
 * disruption records).
 */
#include <stdint.h>
#include <string.h>
#include <math.h>
#include <stdlib.h>

/* ---------------- tree structure ---------------- */

static int is_func(uint8_t o) { return o < 4; }

/* Size of the subtree rooted at i: 1 for a leaf, else 1 + left + right,
 * the right child starting where the left one ends (prefix order, Sec. 3.1).
 * Returns 0 if the subtree runs past n (malformed input). */
static uint64_t size_rec(const uint8_t* ops, uint64_t n, uint64_t i) {
    if (i >= n) return 0;
    if (!is_func(ops[i])) return 1;
    uint64_t l = size_rec(ops, n, i + 1);
    if (!l) return 0;
    uint64_t r = size_rec(ops, n, i + 1 + l);
    if (!r) return 0;
    return 1 + l + r;
}

uint64_t or_subtree_size(const uint8_t* ops, uint64_t n, uint64_t i) {
    return size_rec(ops, n, i);
}

/* End (one past the last node) of every subtree: end(i) = i+1 for a leaf,
 * end(end(i+1)) for a function (its right child starts where its left
 * child ends).  Returns the end of the subtree at `i`, 0 if malformed. */
static uint64_t ends_rec(const uint8_t* ops, uint64_t n, uint64_t i, uint64_t* ends) {
    if (i >= n) return 0;
    uint64_t e;
    if (!is_func(ops[i])) e = i + 1;
    else {
        uint64_t l = ends_rec(ops, n, i + 1, ends);
        if (!l) return 0;
        e = ends_rec(ops, n, l, ends);
        if (!e) return 0;
    }
    ends[i] = e;
    return e;
}

int or_tree_ends(const uint8_t* ops, uint64_t n, uint64_t* ends) {
    return ends_rec(ops, n, 0, ends) == n ? 0 : -1;
}

/* Parent of node q: the nearest function node p < q whose subtree contains
 * q (end(p) > q).  Returns -1 for the root. */
static int64_t parent_of(const uint8_t* ops, const uint64_t* ends, uint64_t q) {
    for (int64_t p = (int64_t)q - 1; p >= 0; --p)
        if (is_func(ops[p]) && ends[p] > q) return p;
    return -1;
}

int64_t or_parent(const uint8_t* ops, uint64_t n, uint64_t q) {
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
    int64_t p = -2;
    if (or_tree_ends(ops, n, ends) == 0) p = parent_of(ops, ends, q);
    free(ends);
    return p;
}

/* ---------------- FP32 / FP64 interpreters (Sec. 4.2) ---------------- */

/* Depth-first recursive evaluation of one test case, as the paper's first
 * AVX interpreter does it (Sec. 4.2): each function node evaluates its left
 * then its right subtree, then applies its operation. */
static float ev32(const uint8_t* ops, uint64_t* pos, const float* k, float x) {
    uint8_t o = ops[(*pos)++];
    if (o == 4) return x;
    if (o >= 5) return k[o - 5];
    float a = ev32(ops, pos, k, x);
    float b = ev32(ops, pos, k, x);
    switch (o) {
    case 0: return a + b;
    case 1: return a - b;
    case 2: return a * b;
    default: return (b == 0.0f) ? 1.0f : a / b;
    }
}

static double ev64(const uint8_t* ops, uint64_t* pos, const float* k, double x) {
    uint8_t o = ops[(*pos)++];
    if (o == 4) return x;
    if (o >= 5) return (double)k[o - 5];
    double a = ev64(ops, pos, k, x);
    double b = ev64(ops, pos, k, x);
    switch (o) {
    case 0: return a + b;
    case 1: return a - b;
    case 2: return a * b;
    default: return (b == 0.0) ? 1.0 : a / b;
    }
}

/* Value vector of the subtree rooted at node i over all C test cases.
 * One pass per case; returns 0, or -1 on malformed input. */
int or_eval_node_f32(const uint8_t* ops, uint64_t n, uint64_t i, const float* k,
                     const float* x, uint32_t C, float* out) {
    uint64_t s = size_rec(ops, n, i);
    if (!s) return -1;
    for (uint32_t c = 0; c < C; ++c) {
        uint64_t pos = i;
        out[c] = ev32(ops, &pos, k, x[c]);
    }
    return 0;
}

int or_eval_node_f64(const uint8_t* ops, uint64_t n, uint64_t i, const float* k,
                     const float* x, uint32_t C, double* out) {
    uint64_t s = size_rec(ops, n, i);
    if (!s) return -1;
    for (uint32_t c = 0; c < C; ++c) {
        uint64_t pos = i;
        out[c] = ev64(ops, &pos, k, (double)x[c]);
    }
    return 0;
}

/* Fitness: sum over test cases, in case order, of |value - target| in FP32
 * (the error against the sextic target; lower is better). */
float or_fitness_f32(const float* v, const float* t, uint32_t C) {
    float f = 0.0f;
    for (uint32_t c = 0; c < C; ++c) f += fabsf(v[c] - t[c]);
    return f;
}

double or_fitness_f64(const double* v, const float* t, uint32_t C) {
    double f = 0.0;
    for (uint32_t c = 0; c < C; ++c) f += fabs(v[c] - (double)t[c]);
    return f;
}

/* Whole population: root value vectors (P*C, may be NULL) and fitness. */
int or_eval_pop_f32(const uint8_t* ops, const uint64_t* off, uint32_t P, const float* k,
                    const float* x, const float* t, uint32_t C, float* rootvals, float* fit) {
    float* v = (float*)malloc(sizeof(float) * C);
    for (uint32_t i = 0; i < P; ++i) {
        if (or_eval_node_f32(ops + off[i], off[i + 1] - off[i], 0, k, x, C, v)) { free(v); return -1; }
        if (rootvals) memcpy(rootvals + (uint64_t)i * C, v, sizeof(float) * C);
        fit[i] = or_fitness_f32(v, t, C);
    }
    free(v);
    return 0;
}

int or_eval_pop_f64(const uint8_t* ops, const uint64_t* off, uint32_t P, const float* k,
                    const float* x, const float* t, uint32_t C, double* fit) {
    double* v = (double*)malloc(sizeof(double) * C);
    for (uint32_t i = 0; i < P; ++i) {
        if (or_eval_node_f64(ops + off[i], off[i + 1] - off[i], 0, k, x, C, v)) { free(v); return -1; }
        fit[i] = or_fitness_f64(v, t, C);
    }
    free(v);
    return 0;
}

/* ---------------- Boolean 6-multiplexer (Sec. 4.2, bit-parallel) ---------------- */

/* All 64 cases packed in one 64-bit word, one bit per case (Sec. 4.2,
 * bit-parallel Boolean evaluation).  Case i sets a0 = bit 0, a1 = bit 1, d0..d3 = bits 2..5 of i;
 * input word j has bit i set iff bit j of i is set. */
void or_mux6_inputs(uint64_t in[6]) {
    for (int j = 0; j < 6; ++j) {
        uint64_t w = 0;
        for (int i = 0; i < 64; ++i)
            if ((i >> j) & 1) w |= (uint64_t)1 << i;
        in[j] = w;
    }
}

/* 6-multiplexer target: output bit i = data line d[a0 + 2*a1] of case i. */
uint64_t or_mux6_target(void) {
    uint64_t w = 0;
    for (int i = 0; i < 64; ++i) {
        int a = (i & 1) + 2 * ((i >> 1) & 1);
        if ((i >> (2 + a)) & 1) w |= (uint64_t)1 << i;
    }
    return w;
}

static uint64_t evb(const uint8_t* ops, uint64_t* pos, const uint64_t* in) {
    uint8_t o = ops[(*pos)++];
    if (o >= 4) return in[o - 4];
    uint64_t a = evb(ops, pos, in);
    uint64_t b = evb(ops, pos, in);
    switch (o) {
    case 0: return a & b;
    case 1: return a | b;
    case 2: return ~(a & b);
    default: return ~(a | b);
    }
}

int or_eval_node_bool(const uint8_t* ops, uint64_t n, uint64_t i, uint64_t* out) {
    uint64_t in[6];
    if (!size_rec(ops, n, i)) return -1;
    for (uint64_t p = i; p < i + size_rec(ops, n, i); ++p) if (ops[p] > 9) return -1;
    or_mux6_inputs(in);
    uint64_t pos = i;
    *out = evb(ops, &pos, in);
    return 0;
}

/* Boolean fitness: number of the 64 cases the tree gets wrong. */
uint32_t or_fitness_bool(uint64_t out) {
    uint64_t e = out ^ or_mux6_target();
    uint32_t c = 0;
    for (int i = 0; i < 64; ++i) c += (uint32_t)((e >> i) & 1);
    return c;
}

/* ---------------- wide Boolean: the k-multiplexer (Sec. 4.2) ----------------
 *
 * k address lines a0..a(k-1) and 2^k data lines d0..d(2^k - 1) are the
 * inputs 0 .. k + 2^k - 1 (opcodes 4 ..); case i (0 <= i < 2^(k + 2^k))
 * gives input j the value of bit j of i, and the target is the data line
 * the address selects: bit k + a of i, a = sum over j < k of a_j 2^j.  The
 * 6-multiplexer is k = 2 (64 cases), the 11-multiplexer k = 3 (2,048
 * cases).  Cases are packed 64 to a word: word w holds cases 64w .. 64w+63,
 * case 64w + b in bit b.  The Boolean functions act on whole words at once,
 * the bit-parallel evaluation of Sec. 4.2 widened to any number of words. */

uint32_t or_mux_inputs_count(uint32_t k) { return k + (1u << k); }

uint64_t or_mux_words(uint32_t k) { return ((uint64_t)1 << (k + (1u << k))) / 64; }

/* word w of input j */
uint64_t or_mux_input_word(uint32_t j, uint64_t w) {
    uint64_t x = 0;
    for (uint32_t b = 0; b < 64; ++b)
        if (((64 * w + b) >> j) & 1) x |= (uint64_t)1 << b;
    return x;
}

/* word w of the target */
uint64_t or_mux_target_word(uint32_t k, uint64_t w) {
    uint64_t x = 0;
    for (uint32_t b = 0; b < 64; ++b) {
        uint64_t i = 64 * w + b, a = 0;
        for (uint32_t j = 0; j < k; ++j) a |= ((i >> j) & 1) << j;
        if ((i >> (k + a)) & 1) x |= (uint64_t)1 << b;
    }
    return x;
}

static uint64_t evmux(const uint8_t* ops, uint64_t* pos, const uint64_t* in) {
    uint8_t o = ops[(*pos)++];
    if (o >= 4) return in[o - 4];
    uint64_t a = evmux(ops, pos, in);
    uint64_t b = evmux(ops, pos, in);
    switch (o) {
    case 0: return a & b;
    case 1: return a | b;
    case 2: return ~(a & b);
    default: return ~(a | b);
    }
}

/* Value words of the subtree at node i: one pass per word (64 cases). */
int or_eval_node_mux(const uint8_t* ops, uint64_t n, uint64_t i, uint32_t k, uint64_t* out) {
    uint64_t s = size_rec(ops, n, i);
    uint32_t ni = or_mux_inputs_count(k);
    uint64_t in[64];
    if (!s || ni > 64) return -1;
    for (uint64_t p = i; p < i + s; ++p) if (ops[p] >= 4 + ni) return -1;
    for (uint64_t w = 0; w < or_mux_words(k); ++w) {
        for (uint32_t j = 0; j < ni; ++j) in[j] = or_mux_input_word(j, w);
        uint64_t pos = i;
        out[w] = evmux(ops, &pos, in);
    }
    return 0;
}

/* Errors: number of cases the words get wrong. */
uint64_t or_fitness_mux(const uint64_t* out, uint32_t k) {
    uint64_t c = 0;
    for (uint64_t w = 0; w < or_mux_words(k); ++w) {
        uint64_t e = out[w] ^ or_mux_target_word(k, w);
        for (int b = 0; b < 64; ++b) c += (e >> b) & 1;
    }
    return c;
}

/* ---------------- integer GP ----------------
 *
 * The same prefix trees over 32-bit signed integers: + - * wrap around
 * modulo 2^32 (two's complement); protected division returns 1 for a zero
 * divisor, the wrapped quotient INT32_MIN for INT32_MIN / -1, and otherwise
 * the quotient truncated toward zero.  Opcodes 5..255 index a table of 251
 * integer constants.  Fitness = sum over cases of |value - target|, exact in
 * 64-bit integers, then rounded once to binary32 (the population's fitness
 * type; equal sums give equal fitness). */

static int32_t wrap32(uint32_t u) { return (int32_t)u; }   /* gcc: modulo 2^32 */

static int32_t evi(const uint8_t* ops, uint64_t* pos, const int32_t* k, int32_t x) {
    uint8_t o = ops[(*pos)++];
    if (o == 4) return x;
    if (o >= 5) return k[o - 5];
    int32_t a = evi(ops, pos, k, x);
    int32_t b = evi(ops, pos, k, x);
    switch (o) {
    case 0: return wrap32((uint32_t)a + (uint32_t)b);
    case 1: return wrap32((uint32_t)a - (uint32_t)b);
    case 2: return wrap32((uint32_t)a * (uint32_t)b);
    default:
        if (b == 0) return 1;
        if (a == INT32_MIN && b == -1) return INT32_MIN;
        return a / b;
    }
}

int or_eval_node_i32(const uint8_t* ops, uint64_t n, uint64_t i, const int32_t* k,
                     const int32_t* x, uint32_t C, int32_t* out) {
    uint64_t s = size_rec(ops, n, i);
    if (!s) return -1;
    for (uint32_t c = 0; c < C; ++c) {
        uint64_t pos = i;
        out[c] = evi(ops, &pos, k, x[c]);
    }
    return 0;
}

float or_fitness_i32(const int32_t* v, const int32_t* t, uint32_t C) {
    int64_t f = 0;
    for (uint32_t c = 0; c < C; ++c) {
        int64_t e = (int64_t)v[c] - (int64_t)t[c];
        f += e < 0 ? -e : e;
    }
    return (float)f;
}

/* ---------------- random numbers ---------------- */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output for element
 * `ctr` of the stream whose state starts at `seed`. */
uint64_t or_splitmix64(uint64_t seed, uint64_t ctr) {
    uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw k of child `child` in generation `gen`: every stochastic choice is a
 * pure function of (seed, gen, child, k), so results do not depend on
 * thread timing (Sec. 2.4, Sec. 5: choices made before the parallel phase). */
uint64_t or_draw(uint64_t seed, uint32_t gen, uint32_t child, uint32_t k) {
    uint64_t ctr = ((uint64_t)gen << 40) | ((uint64_t)child << 8) | (uint64_t)(k & 0xFF);
    return or_splitmix64(seed, ctr);
}

/* Uniform index in [0, n) from the top 32 bits of a draw. */
static uint64_t below(uint64_t r, uint64_t n) { return ((r >> 32) * n) >> 32; }

/* ---------------- selection and crossover plan (Sec. 5, Sec. 6.3) ---------------- */

/* Tournament of size T with replacement: the lowest error wins, a NaN
 * error ranks as +infinity, ties go to the earliest draw. */
uint32_t or_tournament(const float* fit, uint32_t P, uint32_t T, uint64_t seed, uint32_t gen,
                       uint32_t child, uint32_t kbase) {
    uint32_t best = 0;
    float bf = 0.0f;
    for (uint32_t j = 0; j < T; ++j) {
        uint32_t idx = (uint32_t)below(or_draw(seed, gen, child, kbase + j), P);
        float f = fit[idx];
        if (isnan(f)) f = INFINITY;
        if (j == 0 || f < bf) { best = idx; bf = f; }
    }
    return best;
}

/* One generation's plan, 100% subtree crossover, one child per crossover
 * (Sec. 3, Sec. 6.3).  Child i: mother by tournament (draws 0..T-1), father
 * by tournament (draws T..2T-1), then up to 8 attempts of crossover points
 * uniform over all nodes (mother: draw 2T+2a, father: 2T+2a+1); an attempt
 * whose child would exceed max_nodes is rejected.  If all 8 fail the child
 * is a copy of its mother (c = 0, r = s = mother size, father = mother).
 * last[i] = 1 when no later child has the same mother (that child may reuse
 * its mother's buffer in place, Fig. 2). */
void or_plan(uint32_t P, const uint8_t* ops, const uint64_t* off, const float* fit,
             uint32_t T, uint64_t seed, uint32_t gen, uint64_t max_nodes,
             uint32_t* mother, uint32_t* father, uint64_t* c, uint64_t* r,
             uint64_t* d, uint64_t* s, uint8_t* last) {
    for (uint32_t i = 0; i < P; ++i) {
        uint32_t m = or_tournament(fit, P, T, seed, gen, i, 0);
        uint32_t f = or_tournament(fit, P, T, seed, gen, i, T);
        uint64_t sm = off[m + 1] - off[m], sf = off[f + 1] - off[f];
        int ok = 0;
        for (uint32_t a = 0; a < 8 && !ok; ++a) {
            uint64_t cc = below(or_draw(seed, gen, i, 2 * T + 2 * a), sm);
            uint64_t dd = below(or_draw(seed, gen, i, 2 * T + 2 * a + 1), sf);
            uint64_t rr = size_rec(ops + off[m], sm, cc);
            uint64_t ss = size_rec(ops + off[f], sf, dd);
            if (sm - rr + ss <= max_nodes) {
                mother[i] = m; father[i] = f; c[i] = cc; r[i] = rr; d[i] = dd; s[i] = ss;
                ok = 1;
            }
        }
        if (!ok) { mother[i] = m; father[i] = m; c[i] = 0; r[i] = sm; d[i] = 0; s[i] = sm; }
    }
    for (uint32_t i = 0; i < P; ++i) {
        last[i] = 1;
        for (uint32_t j = i + 1; j < P; ++j) if (mother[j] == mother[i]) { last[i] = 0; break; }
    }
}

/* Subtree crossover by splicing (Fig. 1): mother[0,c) ++ father[d,d+s) ++
 * mother[c+r, n_m).  Returns the child's size. */
uint64_t or_splice(const uint8_t* mom, uint64_t n_m, uint64_t c, uint64_t r,
                   const uint8_t* dad, uint64_t d, uint64_t s, uint8_t* out) {
    memcpy(out, mom, c);
    memcpy(out + c, dad + d, s);
    memcpy(out + c + s, mom + c + r, n_m - c - r);
    return n_m - r + s;
}

/* ---------------- incremental evaluation with FDP (Sec. 6.2, Fig. 3) ---------------- */

static int same_bits(const float* a, const float* b, uint32_t C) {
    return memcmp(a, b, sizeof(float) * C) == 0;
}

/* Failed disruption propagation walk for one child (Sec. 6.2).  Level j is
 * the j-th node on the chain from the crossover point c (level 0) to the
 * root; at each level the mother's and the child's values at that node are
 * compared on all test cases.  The walk stops at the first level where the
 * two value vectors are identical (bit for bit); from there up the two
 * evaluations are locked together, so the child's fitness is the mother's.
 * Outputs: *stop = that level, or -1 if even the root differs; *depth =
 * number of ancestors of c.  Each level is evaluated in full from the two
 * trees, which is the definition the incremental method must reproduce. */
int or_fdp_walk(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                const float* k, const float* x, uint32_t C, int64_t* stop, int64_t* depth) {
    float* a = (float*)malloc(sizeof(float) * C);
    float* b = (float*)malloc(sizeof(float) * C);
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * n_m);
    int64_t lvl = 0, found = -1;
    int64_t q = (int64_t)c;
    if (or_tree_ends(mom, n_m, ends)) { free(a); free(b); free(ends); return -1; }
    while (q >= 0) {
        if (found < 0) {
            if (or_eval_node_f32(mom, n_m, (uint64_t)q, k, x, C, a) ||
                or_eval_node_f32(kid, n_k, (uint64_t)q, k, x, C, b)) { free(a); free(b); free(ends); return -1; }
            if (same_bits(a, b, C)) found = lvl;
        }
        int64_t p = parent_of(mom, ends, (uint64_t)q);
        if (p < 0) break;
        q = p;
        ++lvl;
    }
    *stop = found;
    *depth = lvl;
    free(a); free(b); free(ends);
    return 0;
}

/* The same walk for Boolean trees (one 64-bit word per node). */
int or_fdp_walk_bool(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k,
                     uint64_t c, int64_t* stop, int64_t* depth) {
    int64_t lvl = 0, found = -1;
    int64_t q = (int64_t)c;
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * n_m);
    if (or_tree_ends(mom, n_m, ends)) { free(ends); return -1; }
    while (q >= 0) {
        if (found < 0) {
            uint64_t a, b;
            if (or_eval_node_bool(mom, n_m, (uint64_t)q, &a) || or_eval_node_bool(kid, n_k, (uint64_t)q, &b)) {
                free(ends);
                return -1;
            }
            if (a == b) found = lvl;
        }
        int64_t p = parent_of(mom, ends, (uint64_t)q);
        if (p < 0) break;
        q = p;
        ++lvl;
    }
    *stop = found;
    *depth = lvl;
    free(ends);
    return 0;
}

/* ---------------- disruption along the walk (Fig. 4) ---------------- */

/* How a crossover's change of the test-case values fades along the chain of
 * ancestors of the crossover point (Fig. 4: the number of disrupted cases
 * and the RMS difference at each node of the chain).  For each level the
 * FDP walk compares (level 0 = c, then each ancestor, up to and including
 * the first level where the mother and the child agree on every case, or up
 * to the root), with both nodes evaluated in full from the two trees:
 *   disrupted[j] = cases whose child and mother values differ bit for bit;
 *   finite[j]    = those of them where both values are finite;
 *   sum_sq[j]    = sum over those finite cases, in case order, of
 *                  ((double)child - (double)mother)^2 in binary64.
 * Levels j < max_levels are written; *n = number of levels compared. */
int or_fdp_disruption(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                      const float* k, const float* x, uint32_t C, uint32_t max_levels,
                      uint32_t* disrupted, uint32_t* finite, double* sum_sq, int64_t* n) {
    float* a = (float*)malloc(sizeof(float) * C);
    float* b = (float*)malloc(sizeof(float) * C);
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * n_m);
    int64_t lvl = 0;
    int64_t q = (int64_t)c;
    if (or_tree_ends(mom, n_m, ends)) { free(a); free(b); free(ends); return -1; }
    for (;;) {
        if (or_eval_node_f32(mom, n_m, (uint64_t)q, k, x, C, a) ||
            or_eval_node_f32(kid, n_k, (uint64_t)q, k, x, C, b)) { free(a); free(b); free(ends); return -1; }
        uint32_t nd = 0, nf = 0;
        double sq = 0.0;
        for (uint32_t j = 0; j < C; ++j) {
            uint32_t ua, ub;
            memcpy(&ua, &a[j], 4);
            memcpy(&ub, &b[j], 4);
            if (ua == ub) continue;
            ++nd;
            if (isfinite(a[j]) && isfinite(b[j])) {
                double df = (double)b[j] - (double)a[j];
                ++nf;
                sq += df * df;
            }
        }
        if ((uint64_t)lvl < max_levels) { disrupted[lvl] = nd; finite[lvl] = nf; sum_sq[lvl] = sq; }
        ++lvl;
        if (nd == 0) break;                       /* the walk stops here */
        int64_t p = parent_of(mom, ends, (uint64_t)q);
        if (p < 0) break;                         /* the root differed */
        q = p;
    }
    *n = lvl;
    free(a); free(b); free(ends);
    return 0;
}

/* The same for Boolean trees: each of the 64 cases is one bit of the node's
 * word, a disrupted case is a differing bit and its difference is 1. */
int or_fdp_disruption_bool(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                           uint32_t max_levels, uint32_t* disrupted, uint32_t* finite, double* sum_sq,
                           int64_t* n) {
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * n_m);
    int64_t lvl = 0;
    int64_t q = (int64_t)c;
    if (or_tree_ends(mom, n_m, ends)) { free(ends); return -1; }
    for (;;) {
        uint64_t a, b;
        if (or_eval_node_bool(mom, n_m, (uint64_t)q, &a) || or_eval_node_bool(kid, n_k, (uint64_t)q, &b)) {
            free(ends);
            return -1;
        }
        uint32_t nd = 0;
        for (int t = 0; t < 64; ++t) nd += (uint32_t)(((a ^ b) >> t) & 1u);
        if ((uint64_t)lvl < max_levels) { disrupted[lvl] = nd; finite[lvl] = nd; sum_sq[lvl] = (double)nd; }
        ++lvl;
        if (nd == 0) break;
        int64_t p = parent_of(mom, ends, (uint64_t)q);
        if (p < 0) break;
        q = p;
    }
    *n = lvl;
    free(ends);
    return 0;
}

/* ---------------- the walk for the wide Boolean and integer sets ---------------- */

/* Value vector of node i for one function set: `ctx` carries the set's
 * parameters, `out` receives vbytes bytes. */
typedef int (*node_fn)(const uint8_t* ops, uint64_t n, uint64_t i, const void* ctx, void* out);

typedef struct { uint32_t k; } mux_ctx;
typedef struct { const int32_t* k; const int32_t* x; uint32_t C; } i32_ctx;

static int mux_node(const uint8_t* ops, uint64_t n, uint64_t i, const void* ctx, void* out) {
    return or_eval_node_mux(ops, n, i, ((const mux_ctx*)ctx)->k, (uint64_t*)out);
}

static int i32_node(const uint8_t* ops, uint64_t n, uint64_t i, const void* ctx, void* out) {
    const i32_ctx* c = (const i32_ctx*)ctx;
    return or_eval_node_i32(ops, n, i, c->k, c->x, c->C, (int32_t*)out);
}

/* The FDP walk of Sec. 6.2 for any set (see or_fdp_walk), comparing whole
 * value vectors bit for bit; with `profile` set, also the disruption record
 * (see or_fdp_disruption): kind 1 = Boolean words (a differing bit is a
 * disrupted case with difference 1), kind 2 = int32 cases (difference
 * child - mother exact in 64-bit integers, squared in binary64). */
static int fdp_walk_any(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                        node_fn fn, const void* ctx, size_t vbytes, int kind, uint32_t max_levels,
                        uint32_t* disrupted, uint32_t* finite, double* sum_sq, int64_t* stop, int64_t* depth,
                        int64_t* nlev) {
    uint8_t* a = (uint8_t*)malloc(vbytes);
    uint8_t* b = (uint8_t*)malloc(vbytes);
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * n_m);
    int64_t lvl = 0, found = -1, rec = 0;
    int64_t q = (int64_t)c;
    if (or_tree_ends(mom, n_m, ends)) { free(a); free(b); free(ends); return -1; }
    while (q >= 0) {
        if (found < 0) {
            if (fn(mom, n_m, (uint64_t)q, ctx, a) || fn(kid, n_k, (uint64_t)q, ctx, b)) {
                free(a); free(b); free(ends);
                return -1;
            }
            uint32_t nd = 0, nf = 0;
            double sq = 0.0;
            if (kind == 1) {
                for (size_t w = 0; w < vbytes / 8; ++w) {
                    uint64_t x, y;
                    memcpy(&x, a + 8 * w, 8);
                    memcpy(&y, b + 8 * w, 8);
                    for (int t = 0; t < 64; ++t) nd += (uint32_t)(((x ^ y) >> t) & 1u);
                }
                nf = nd;
                sq = (double)nd;
            } else {
                for (size_t j = 0; j < vbytes / 4; ++j) {
                    int32_t x, y;
                    memcpy(&x, a + 4 * j, 4);
                    memcpy(&y, b + 4 * j, 4);
                    if (x == y) continue;
                    double df = (double)((int64_t)y - (int64_t)x);
                    ++nd;
                    ++nf;
                    sq += df * df;
                }
            }
            if (disrupted && (uint64_t)lvl < max_levels) { disrupted[lvl] = nd; finite[lvl] = nf; sum_sq[lvl] = sq; }
            rec = lvl + 1;
            if (nd == 0) found = lvl;
        }
        int64_t p = parent_of(mom, ends, (uint64_t)q);
        if (p < 0) break;
        q = p;
        ++lvl;
    }
    *stop = found;
    *depth = lvl;
    if (nlev) *nlev = rec;
    free(a); free(b); free(ends);
    return 0;
}

int or_fdp_walk_mux(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                    uint32_t k, uint32_t max_levels, uint32_t* disrupted, uint32_t* finite, double* sum_sq,
                    int64_t* stop, int64_t* depth, int64_t* nlev) {
    mux_ctx ctx = {k};
    return fdp_walk_any(mom, n_m, kid, n_k, c, mux_node, &ctx, 8 * or_mux_words(k), 1, max_levels,
                        disrupted, finite, sum_sq, stop, depth, nlev);
}

int or_fdp_walk_i32(const uint8_t* mom, uint64_t n_m, const uint8_t* kid, uint64_t n_k, uint64_t c,
                    const int32_t* kt, const int32_t* x, uint32_t C, uint32_t max_levels, uint32_t* disrupted,
                    uint32_t* finite, double* sum_sq, int64_t* stop, int64_t* depth, int64_t* nlev) {
    i32_ctx ctx = {kt, x, C};
    return fdp_walk_any(mom, n_m, kid, n_k, c, i32_node, &ctx, 4 * (size_t)C, 2, max_levels,
                        disrupted, finite, sum_sq, stop, depth, nlev);
}
