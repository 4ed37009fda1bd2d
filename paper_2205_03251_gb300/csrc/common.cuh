// Shared device definitions for the gpfdp library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define GP_B 1024            // structure block: positions per warp pass (32 per lane)
#define GP_NCONST 251        // ephemeral constant table
#define GP_WARPS 8           // warps per CTA in the persistent kernels
#define FREE_TILE 4096       // slots per CTA in the free-slot scan
#define SLOT_NEW 0xFFFFFFFFu // cache entry whose value slot is assigned later in the generation
#define FULL 0xFFFFFFFFu

// status word bits (device side)
enum : uint32_t {
    ST_STACK = 1u << 0,      // interpreter stack deeper than the configured bound
    ST_ENTRIES = 1u << 1,    // cache-entry capacity exceeded
    ST_STRUCT = 1u << 2,     // structure pass inconsistent (malformed tree)
    ST_CAPACITY = 1u << 3,   // child larger than its buffer
    ST_SLOTS = 1u << 4,      // value-slot pool exhausted (cache budget)
    ST_TIMEOUT = 1u << 5,    // a bounded wait gave up
    ST_PATH = 1u << 6,       // incremental walk scratch exceeded
};

// queue counters
enum { Q_ITEMS = 0, Q_SKEL = 1, Q_WALK = 2, Q_MISC = 3, Q_ALLOC = 4, Q_PATHV = 5, Q_WALK_LONG = 6, NQ = 16 };

// Value kinds of the function sets.  Every value travels as 32 bits in a
// float register or slot: a binary32 number (VF), a word of 32 Boolean
// cases (VB), or a two's-complement integer (VI).
enum : int { VF = 0, VB = 1, VI = 2 };

struct DevPop {
    // sizes
    uint32_t P, C, Cpad, K, ncb, T, cap, funcset;
    uint32_t Ecap, Scap, maxdepth, W;      // entries, slots, interpreter stack bound, smem stack depth
    uint32_t ovf_warps;                    // warps with an overflow stack region
    uint32_t strict_cap;                   // 1: a cache larger than Ecap is an error (no host regrow)
    uint32_t vkind;                        // VF, VB or VI
    uint32_t mux_k;                        // Boolean: address lines of the multiplexer (C = 2^(k + 2^k) / 32 words)
    uint32_t wait_polls;                   // bound on the polls of one wait inside a walk team (>= 1)
    // population
    uint8_t* arena;      // nbuf * cap bytes
    uint32_t* buf;       // [P] buffer holding individual i
    uint32_t* size;      // [P]
    float* x;            // [Cpad] (padded cases are 0; integer set: int32 bits; Boolean: unused)
    float* t;            // [C] targets (integer set: int32 bits; Boolean: the target's case words)
    float* consts;       // [251] (integer set: int32 bits)
    float* fit;          // [P]
    // structure / cache (current population)
    uint32_t* blk_off;   // [P+1]
    uint32_t* e_cnt;     // [P]
    uint32_t* e_off;     // [P+1]
    uint32_t* e_pos;     // [Ecap]
    uint32_t* e_end;     // [Ecap]
    int32_t* e_par;      // [Ecap]
    int32_t* e_c0;       // [Ecap] large left child entry or -1
    int32_t* e_c1;       // [Ecap] large right child entry or -1
    uint32_t* e_slot;    // [Ecap] value slot
    uint32_t* e_tree;    // [Ecap] tree of the entry
    // items (small subtrees hanging off the cached skeleton)
    uint4* it_desc;      // [Ecap] (start, length, slot, buffer) of the entry's small-subtree item
    uint4* sk_desc;      // [Ecap] (slot, operand slot, op | child flags, right child entry) for the skeleton pass
    uint32_t* order;     // [Ecap] work order
    // values: one pool of slots shared by the parents' and the children's caches
    float* slots;        // [Scap][Cpad]
    uint32_t* live;      // [Scap] generation stamp of the last cache that referenced the slot
    uint32_t* freeslot;  // [Scap] free slots in slot order (first ones used for new values)
    uint32_t* ftile;     // [Scap / FREE_TILE + 1] free slots per tile, then their exclusive prefix
    float* ovf;          // interpreter stack overflow, per warp
    uint32_t* status;    // [1]
    uint32_t* errinfo;   // [4] first failure: site, individual, position, detail
    uint32_t* e_total;   // [1] cache entries found by the structure pass
    uint32_t* q;         // [NQ] queue counters
    unsigned long long* acc_ops;   // [4] actual-op counters
};

__device__ __forceinline__ uint32_t warp_bcast(uint32_t v, int src) { return __shfl_sync(FULL, v, src); }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// In graph mode the cache arrays are never regrown: a kernel that finds the
// entry count above Ecap raises ST_ENTRIES, and every later kernel of the
// (captured) sequence that indexes a cache or a plan returns at once.  The
// same holds in every mode once a generation found no free tree buffer
// (ST_CAPACITY): its selected children have no buffer to be read from.
__device__ __forceinline__ bool halted(const DevPop& d) {
    const uint32_t st = *reinterpret_cast<const volatile uint32_t*>(d.status);
    return (st & ST_CAPACITY) || (d.strict_cap && (st & ST_ENTRIES));
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bit) { atomicOr(st, bit); }

// Record the first failure site (kept until the host reads and clears it).
__device__ __forceinline__ void set_error(const DevPop& d, uint32_t bit, uint32_t site, uint32_t who,
                                          uint32_t pos, uint32_t detail) {
    atomicOr(d.status, bit);
    if (atomicCAS(d.errinfo, 0u, site) == 0u) { d.errinfo[1] = who; d.errinfo[2] = pos; d.errinfo[3] = detail; }
}

// individual i's buffer
__device__ __forceinline__ const uint8_t* tree_ptr(const DevPop& d, uint32_t i) {
    return d.arena + (size_t)d.buf[i] * d.cap;
}

// upper_bound over an exclusive prefix array off[0..n] (off[0] = 0): largest i with off[i] <= u
__device__ __forceinline__ uint32_t find_segment(const uint32_t* off, uint32_t n, uint32_t u) {
    uint32_t lo = 0, hi = n;          // off[lo] <= u < off[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// Fitness of one value vector, whose case (Boolean: word) j is at(j):
//   binary32: sum over the cases, in case order, of |v - t|, each step
//             rounded to binary32;
//   Boolean:  the number of wrong cases, popcount(v ^ target) summed over
//             the words;
//   integer:  sum of |v - t| exact in 64-bit integers, rounded once to
//             binary32.
template <typename F>
__device__ __forceinline__ float fitness_of(const DevPop& d, F at) {
    if (d.vkind == VB) {
        uint32_t e = 0;
        for (uint32_t j = 0; j < d.C; ++j) e += __popc(__float_as_uint(at(j)) ^ __float_as_uint(d.t[j]));
        return (float)e;
    }
    if (d.vkind == VI) {
        long long s = 0;
        for (uint32_t j = 0; j < d.C; ++j) {
            const long long e = (long long)__float_as_int(at(j)) - (long long)__float_as_int(d.t[j]);
            s += e < 0 ? -e : e;
        }
        return __ll2float_rn(s);
    }
    float f = 0.0f;
    for (uint32_t j = 0; j < d.C; ++j) f = __fadd_rn(f, fabsf(__fsub_rn(at(j), d.t[j])));
    return f;
}

// fitness_of with the whole warp (all 32 lanes call it; every lane returns
// the fitness): the lanes fetch and form the terms of 32 cases at a time in
// parallel, and every lane adds them in case order from shuffles, so the
// binary32 sum is rounded in the same order and has the same bits; the
// Boolean and integer sums are exact, so their order does not matter.
template <typename F>
__device__ __forceinline__ float fitness_warp(const DevPop& d, F at) {
    const uint32_t lane = threadIdx.x & 31u;
    if (d.vkind == VB) {
        uint32_t e = 0;
        for (uint32_t j = lane; j < d.C; j += 32) e += __popc(__float_as_uint(at(j)) ^ __float_as_uint(d.t[j]));
        return (float)__reduce_add_sync(FULL, e);
    }
    if (d.vkind == VI) {
        long long s = 0;
        for (uint32_t j = lane; j < d.C; j += 32) {
            const long long e = (long long)__float_as_int(at(j)) - (long long)__float_as_int(d.t[j]);
            s += e < 0 ? -e : e;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        return __ll2float_rn(s);
    }
    float f = 0.0f;
    for (uint32_t b = 0; b < d.C; b += 32) {
        const uint32_t j = b + lane;
        const float term = (j < d.C) ? fabsf(__fsub_rn(at(j), d.t[j])) : 0.0f;
        const uint32_t n = min(32u, d.C - b);
        for (uint32_t q = 0; q < n; ++q) f = __fadd_rn(f, __shfl_sync(FULL, term, q));
    }
    return f;
}
