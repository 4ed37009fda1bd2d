/*
 * Seeded synthetic input generators for the GP population workloads.
 *
 * This module only makes inputs: test-case x values and targets, the
 * ephemeral-constant table, and populations of prefix-encoded trees.  It
 * holds none of the evaluation, selection, crossover or incremental
 * arithmetic of the method; both the CPU oracle and the CUDA path consume
 * what it writes.
 *
 * Encoding (one byte per node, depth-first prefix order; Sec. 3.1 and
 * Sec. 5 of the paper):
 *   arithmetic set: 0 '+', 1 '-', 2 '*', 3 protected '/', 4 x,
 *                   5..255 ephemeral constant k[op-5] (table of 251 FP32)
 *   Boolean 6-mux:  0 AND, 1 OR, 2 NAND, 3 NOR, 4..9 inputs a0 a1 d0 d1 d2 d3
 * Opcodes 0..3 have two children (left child first), all others are leaves.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), element ctr of the stream
 * started at `seed`.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_draw(uint64_t seed, uint64_t ctr) {
    return sm_mix(seed + (ctr + 1) * GOLDEN);
}

typedef struct { uint64_t s; } rng_t;
static inline uint64_t rng_next(rng_t* r) { r->s += GOLDEN; return sm_mix(r->s); }
static inline uint32_t rng_below(rng_t* r, uint32_t n) {
    return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32);
}

/* 24 random bits -> exact float in [-1, 1) */
static inline float u24_pm1(uint64_t r) {
    return (float)(r >> 40) * (1.0f / 8388608.0f) - 1.0f;
}

/* Test cases x ~ U[-1,1) and sextic targets x^6 - 2x^4 + x^2 = x^2 (x^2-1)^2,
 * computed in double and rounded once to float. */
void synth_cases(uint64_t seed, uint32_t C, float* x, float* t) {
    for (uint32_t c = 0; c < C; ++c) {
        float xv = u24_pm1(synth_draw(seed ^ 0x5A5A000000000001ULL, c));
        double xd = (double)xv, x2 = xd * xd;
        x[c] = xv;
        t[c] = (float)(x2 * (x2 - 1.0) * (x2 - 1.0));
    }
}

/* 251 ephemeral constants uniform in [-1, 1). */
void synth_consts(uint64_t seed, float* k) {
    for (uint32_t i = 0; i < 251; ++i) k[i] = u24_pm1(synth_draw(seed ^ 0xC0C0000000000002ULL, i));
}

/* ---------------- ramped half-and-half ---------------- */

/* boolean: 0 for the arithmetic sets, else the number of Boolean inputs
 * (1 is read as the 6-multiplexer's 6) */
static uint64_t leaf_op(rng_t* r, int boolean) {
    if (boolean) return 4 + rng_below(r, boolean == 1 ? 6u : (uint64_t)boolean);
    if (rng_next(r) >> 63) return 4;                 /* x with p = 0.5 */
    return 5 + rng_below(r, 251);                   /* constant with p = 0.5 */
}

/* Iterative generator (explicit stack of remaining depth).  depth = edges
 * from the root to the deepest leaf allowed; the root is always a function
 * when depth >= 1; grow makes a non-root node a function with p = 0.5. */
static int64_t gen_rhh(rng_t* r, uint32_t depth, int full, int boolean, uint8_t* buf, uint64_t cap) {
    uint32_t stack[64];
    int sp = 0;
    uint64_t n = 0;
    stack[sp++] = 0;                                /* node depth */
    while (sp) {
        uint32_t d = stack[--sp];
        if (n >= cap) return -1;
        int func;
        if (d >= depth) func = 0;
        else if (d == 0 || full) func = 1;
        else func = (int)(rng_next(r) >> 63);
        if (func) {
            buf[n++] = (uint8_t)rng_below(r, 4);
            stack[sp++] = d + 1;                    /* right child (popped second) */
            stack[sp++] = d + 1;                    /* left child (popped first) */
        } else {
            buf[n++] = (uint8_t)leaf_op(r, boolean);
        }
    }
    return (int64_t)n;
}

/* Tree `idx` of a ramped half-and-half population over depths 2..12:
 * depth = 2 + (idx/2) % 11, full when idx is even, grow otherwise. */
int64_t synth_rhh(uint64_t seed, uint64_t idx, int boolean, uint8_t* buf, uint64_t cap) {
    rng_t r = { synth_draw(seed ^ 0x7011000000000003ULL, idx) };
    uint32_t depth = 2 + (uint32_t)((idx / 2) % 11);
    return gen_rhh(&r, depth, (idx % 2) == 0, boolean, buf, cap);
}

/* A donor drawn like a random member of the ramped half-and-half population. */
static int64_t gen_donor(rng_t* r, int boolean, uint8_t* buf, uint64_t cap) {
    uint32_t depth = 2 + rng_below(r, 11);
    int full = (int)(rng_next(r) >> 63);
    return gen_rhh(r, depth, full, boolean, buf, cap);
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : x > y;
}

/* Large tree: start from a ramped half-and-half tree and repeatedly graft a
 * fresh ramped half-and-half donor onto a uniformly chosen leaf until the
 * size reaches `target`.  Grafts are applied in rounds (several leaves per
 * pass) so the cost stays linear in the final size. */
int64_t synth_big(uint64_t seed, uint64_t idx, uint64_t target, int boolean, uint8_t* buf, uint64_t cap) {
    rng_t r = { synth_draw(seed ^ 0xB16B000000000004ULL, idx) };
    uint8_t* tmp = (uint8_t*)malloc(cap);
    uint8_t donor[16384];
    if (!tmp) return -1;
    int64_t n = gen_donor(&r, boolean, buf, cap);
    while (n > 0 && (uint64_t)n < target) {
        uint64_t leaves = 0;
        for (int64_t i = 0; i < n; ++i) leaves += buf[i] >= 4;
        uint64_t m = (uint64_t)n / 1024;
        uint64_t need = (target - (uint64_t)n) / 1500;   /* close about half the gap per round */
        if (m > need) m = need;
        if (m < 1) m = 1;
        uint64_t* pick = (uint64_t*)malloc(m * sizeof(uint64_t));
        for (uint64_t j = 0; j < m; ++j) pick[j] = ((rng_next(&r) >> 32) * leaves) >> 32;
        qsort(pick, m, sizeof(uint64_t), cmp_u64);
        uint64_t out = 0, leaf_rank = 0, j = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (buf[i] >= 4) {
                int grafted = 0;
                while (j < m && pick[j] == leaf_rank) {
                    if (!grafted) {
                        int64_t ds = gen_donor(&r, boolean, donor, sizeof(donor));
                        if (ds < 0 || out + (uint64_t)ds > cap) { free(pick); free(tmp); return -1; }
                        memcpy(tmp + out, donor, (size_t)ds);
                        out += (uint64_t)ds;
                        grafted = 1;
                    }
                    ++j;                              /* duplicate picks collapse */
                }
                ++leaf_rank;
                if (grafted) continue;
            }
            if (out >= cap) { free(pick); free(tmp); return -1; }
            tmp[out++] = buf[i];
        }
        free(pick);
        memcpy(buf, tmp, out);
        n = (int64_t)out;
    }
    free(tmp);
    return n;
}

/* Uniform random binary tree with `n_internal` internal nodes (Remy, 1985):
 * grow by picking a uniform node and a uniform side, inserting a new
 * internal node above it with a new leaf on the other side.  Then label:
 * internal nodes uniform over the four functions, leaves as leaf_op. */
int64_t synth_remy(uint64_t seed, uint64_t idx, uint64_t n_internal, int boolean, uint8_t* buf, uint64_t cap) {
    uint64_t total = 2 * n_internal + 1;
    if (total > cap) return -1;
    rng_t r = { synth_draw(seed ^ 0x4E3D000000000005ULL, idx) };
    /* node k: child[2k], child[2k+1] (UINT32_MAX for leaves); up[k] = slot
     * index (2*parent + side) or UINT32_MAX for the root. */
    uint32_t* child = (uint32_t*)malloc(sizeof(uint32_t) * 2 * total);
    uint32_t* up = (uint32_t*)malloc(sizeof(uint32_t) * total);
    uint32_t* stk = (uint32_t*)malloc(sizeof(uint32_t) * (total + 1));
    if (!child || !up || !stk) { free(child); free(up); free(stk); return -1; }
    uint32_t root = 0, cnt = 1;
    child[0] = child[1] = UINT32_MAX;
    up[0] = UINT32_MAX;
    for (uint64_t k = 0; k < n_internal; ++k) {
        uint32_t v = (uint32_t)(((rng_next(&r) >> 32) * (uint64_t)cnt) >> 32);
        uint32_t side = (uint32_t)(rng_next(&r) >> 63);
        uint32_t u = cnt++, l = cnt++;
        child[2 * l] = child[2 * l + 1] = UINT32_MAX;
        uint32_t slot = up[v];
        up[u] = slot;
        if (slot == UINT32_MAX) root = u; else child[slot] = u;
        child[2 * u + side] = v;       up[v] = 2 * u + side;
        child[2 * u + 1 - side] = l;   up[l] = 2 * u + 1 - side;
    }
    uint64_t n = 0; uint32_t sp = 0;
    stk[sp++] = root;
    while (sp) {
        uint32_t v = stk[--sp];
        if (child[2 * v] == UINT32_MAX) {
            buf[n++] = (uint8_t)leaf_op(&r, boolean);
        } else {
            buf[n++] = (uint8_t)rng_below(&r, 4);
            stk[sp++] = child[2 * v + 1];
            stk[sp++] = child[2 * v];
        }
    }
    free(child); free(up); free(stk);
    return (int64_t)n;
}

/* ---------------- population builders (threaded over trees) ---------------- */

enum { KIND_RHH = 0, KIND_BIG = 1, KIND_REMY = 2 };

typedef struct {
    int kind, boolean;
    uint64_t seed, param, cap;
    const uint64_t* nint;       /* per-tree internal-node count (remy) */
    const uint64_t* boff;       /* optional per-tree buffer offsets (P+1) */
    uint8_t* scratch;           /* P * cap, or boff[P] bytes */
    int64_t* sizes;
    uint32_t P, next;
    pthread_mutex_t mu;
} job_t;

static void* worker(void* arg) {
    job_t* j = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        uint32_t i = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (i >= j->P) break;
        uint64_t cap = j->boff ? j->boff[i + 1] - j->boff[i] : j->cap;
        uint8_t* b = j->scratch + (j->boff ? j->boff[i] : (uint64_t)i * j->cap);
        int64_t n;
        if (j->kind == KIND_RHH) n = synth_rhh(j->seed, i, j->boolean, b, cap);
        else if (j->kind == KIND_BIG) n = synth_big(j->seed, i, j->param, j->boolean, b, cap);
        else n = synth_remy(j->seed, i, j->nint[i], j->boolean, b, cap);
        j->sizes[i] = n;
    }
    return NULL;
}

/* Generate P trees into scratch and their sizes: tree i at i*cap, or at
 * boff[i] with room boff[i+1]-boff[i] when boff is given.  Returns 0, or
 * -1 if any tree overflowed its room. */
int synth_population(int kind, int boolean, uint64_t seed, uint32_t P, uint64_t param,
                     const uint64_t* nint, const uint64_t* boff, uint64_t cap, uint8_t* scratch,
                     int64_t* sizes, int threads) {
    job_t j;
    j.kind = kind; j.boolean = boolean; j.seed = seed; j.param = param; j.cap = cap;
    j.nint = nint; j.boff = boff; j.scratch = scratch; j.sizes = sizes; j.P = P; j.next = 0;
    pthread_mutex_init(&j.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    for (int k = 0; k < threads; ++k) pthread_create(&th[k], NULL, worker, &j);
    for (int k = 0; k < threads; ++k) pthread_join(th[k], NULL);
    pthread_mutex_destroy(&j.mu);
    for (uint32_t i = 0; i < P; ++i) if (sizes[i] < 0) return -1;
    return 0;
}
