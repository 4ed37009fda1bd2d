// One generation: selection, crossover (copy or in place), and the
// incremental evaluation of the children with failed disruption
// propagation (Sec. 5, Sec. 6.2, Sec. 6.3, Fig. 1-3).
#pragma once
#include "interp.cuh"
#include "structure.cuh"
#include "mlp.cuh"

#define SHIFT_BS 16384         // bytes of tail per block of the in-place move
#define EAGER_HALO_MAX 1024    // eager order: largest |size change| built in place (else copied)
#define COPY_CH 32768          // bytes of a copied child per work unit
#define PV_PER_CHILD 256       // walk records (new path values) reserved per child on average
#define WALK_MAXLVL 520        // small-ancestor levels held in shared memory (T <= 1024)

enum : uint32_t { F_LAST = 1u, F_CLONE = 2u, F_INPLACE = 4u };
enum { M_NCOPY = 0, M_NINPLACE, M_NSHIFT, M_PV, M_FRAG, M_STASH, NMISC = 8 };
enum { G_INTERP = 0, G_LEVELS, G_STOPPED, G_XOBYTES, G_PATHOPS, G_CHILDREN, G_EQUIV, NGSTAT = 8 };

// Read-only view of the parents' cache during a generation.
struct CacheView {
    const uint32_t* e_off;
    const uint32_t* e_pos;
    const uint32_t* e_end;
    const int32_t* e_par;
    const int32_t* e_c0;
    const int32_t* e_c1;
    const uint32_t* e_slot;
    const float* slots;
};

// one walk level of the disruption record: cases whose bits differ, those
// with both values finite, and the sum of their squared differences (binary64)
struct DisLevel {
    uint32_t nd, nf;
    double sq;
};

struct GenBufs {
    uint32_t *pbuf, *psize;          // parents (swapped with DevPop buf/size each generation)
    float* pfit;
    uint32_t *mother, *father, *cpos, *rsz, *dpos, *ssz, *flags;
    int32_t* lastidx;                // [P] highest child index of each mother, -1 if none
    uint32_t* free_buf;              // [P] buffers holding no individual
    uint32_t* free_next;             // [P]
    uint32_t* hasip;                 // [P] parent keeps its buffer (in-place child)
    uint32_t* misc;                  // [NMISC]
    uint64_t* frag_off;              // [P+1] donated subtrees (16-aligned)
    uint8_t* frag;
    uint64_t frag_cap;
    uint64_t* stash_off;             // [P+1] removed subtrees below the threshold (16-aligned)
    uint8_t* stash;
    uint64_t stash_cap;
    uint32_t* shift_off;             // [P+1] in-place move blocks per child (prefix)
    uint64_t* halo_off;              // [P+1] halo bytes per in-place child (prefix; min(|delta|, SHIFT_BS) per block)
    uint64_t halo_cap;               // bytes of the halo pool
    int32_t* lastsel;                // [P] highest index of a child selected as a parent, per mother (-1: none)
    uint32_t* npend;                 // [1] children built in place at the next crossover (fitness-first order)
    uint32_t* copy_off;              // [P+1] COPY_CH-byte chunks of the copied children (prefix)
    uint8_t* halo;                   // [halo_cap] bytes of in-place move blocks that other blocks overwrite
    uint32_t shift_cap;
    int32_t* stop;                   // [P] FDP stop level, -1 if the root differs
    uint32_t* plen;                  // [P] levels evaluated above the crossover point
    uint4* pv_rec;                   // [pvcap] (child, k, pos, slot | insert<<31)
    float* pv_val;                   // [pvcap][Cpad] the walk's new values
    int32_t* walkA;                  // [P] deepest cached ancestor (mother entry) of the crossover point
    uint32_t* nins;                  // [P] child-cached nodes the mother does not cache (inserted entries)
    uint4* mb;                       // [P] merge bounds: first mother entry >= c, >= c+r, father >= d, >= d+s
    uint32_t* mcnt;                  // [P+1] children's entry counts, then offsets
    uint32_t* src;                   // [Ecap] value source of each child entry (bit 31: walk record)
    uint32_t* pv_cnt;                // [P]
    uint32_t* pv_off;                // [P+1]
    uint4* pv_sorted;                // [pvcap] (pos, slot | insert<<31, child end, 0), per child in walk order
    uint32_t* pv_end;                // [pvcap] child end of the recorded node
    uint32_t pvcap;
    uint32_t* order;                 // [P] walk order
    uint32_t* small_cnt;             // [P] case blocks of a one-pass child evaluated so far
    float* small_val;                // [P][Cpad] root values of the one-pass children
    uint32_t* onepass;               // [P] 1: the child is evaluated in one pass (k_onepass_*), not walked
    uint32_t onepass_max;            // children of at most this many nodes are evaluated in one pass (0: none)
    float* ovf_op;                   // interpreter overflow stacks of the one-pass warps (ONEPASS_DEPTH deep)
    uint32_t* op_base;               // [P] first walk record of a one-pass child
    uint32_t* op_cnt;                // [OP_BUCKETS] one-pass children per size bucket, then [OP_BUCKETS] units taken
    uint32_t* op_bucket;             // [OP_BUCKETS][P] one-pass children by size bucket (log2 of the size)
    unsigned long long* gstat;       // [NGSTAT]
    uint32_t max_nodes, tsize;
    uint64_t seed;
    uint32_t gen;
    const uint32_t* gen_add;         // device word added to gen (generations replayed by a captured graph)
    uint32_t* stamp;                 // [1] generation stamp of the slot pool's live marks
    uint32_t* rec_entry;             // [pvcap] child cache entry that takes each walk record's value, or ~0
    // fitness-first materialisation: the next generation's plan is drawn right
    // after the walk, and only the children it selects as parents get a tree
    // buffer and a cache
    uint32_t lazy;                   // 1: the walk reads children through their mother and father
    uint32_t lazy_inplace;           // 1 (with lazy): a mother's last selected child takes her buffer
    uint32_t *nmother, *nfather, *ncpos, *nrsz, *ndpos, *nssz, *nflags;   // [P] next generation's plan
    uint32_t* sel;                   // [P] 1 for a child that is a parent of the next generation
    uint32_t* nfree;                 // [1] entries of the free-buffer stack (lazy mode: up to 2P)
    uint32_t* pref;                  // [P] parent read by a child of this generation (mother or father)
    // disruption diagnostics (Fig. 4): per child and walk level, the cases
    // where the child's value differs from the mother's
    DisLevel* dis;                   // [P][dis_L], null when not recording
    uint32_t* dis_n;                 // [P] levels recorded
    uint32_t dis_L;
    bool evaluated;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t ctr) {
    // SplitMix64 (Steele, Lea and Flood 2014): element ctr of the stream started at seed
    uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t draw(uint64_t seed, uint32_t gen, uint32_t child, uint32_t k) {
    return sm64(seed, ((uint64_t)gen << 40) | ((uint64_t)child << 8) | (uint64_t)(k & 0xFFu));
}
__device__ __forceinline__ uint64_t below(uint64_t r, uint64_t n) { return ((r >> 32) * n) >> 32; }

// Index of the entry at position x in [lo, hi) (sorted by position), or -1.
__device__ __forceinline__ int32_t find_exact(const uint32_t* e_pos, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        uint32_t v = e_pos[mid];
        if (v == x) return (int32_t)mid;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return -1;
}
// Last entry with position < x in [lo, hi), or -1.
__device__ __forceinline__ int32_t find_last_lt(const uint32_t* e_pos, uint32_t lo, uint32_t hi, uint32_t x) {
    uint32_t a = lo, b = hi;            // first index with pos >= x
    while (a < b) {
        uint32_t mid = (a + b) >> 1;
        if (e_pos[mid] < x) a = mid + 1; else b = mid;
    }
    return (a > lo) ? (int32_t)(a - 1) : -1;
}

// 16 bytes starting at any address (two aligned loads and a funnel shift);
// may read up to 31 bytes past p.
__device__ __forceinline__ uint4 load16u(const uint8_t* p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t m = (uint32_t)(a & 15u);
    const uint4* A = reinterpret_cast<const uint4*>(a - m);
    const uint4 lo = A[0];
    if (!m) return lo;
    const uint4 hi = A[1];
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    const uint32_t mw = m >> 2, sh = (m & 3u) * 8u;
    uint32_t r[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        uint32_t x = 0, y = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if ((uint32_t)c == mw) { x = w[t + c]; y = w[t + c + 1]; }
        r[t] = __funnelshift_r(x, y, sh);
    }
    return make_uint4(r[0], r[1], r[2], r[3]);
}

// Size of the subtree at x of a parent tree: a cached entry gives it
// directly; otherwise it is below the threshold and a forward balance scan
// of fewer than T bytes finds its end, here by a whole warp: 512 bytes per
// step, each lane summing (arity - 1) over 16 of them; the first lane whose
// running balance reaches zero finds the end.  All lanes return the size.
__device__ uint32_t warp_subtree_size_at(const CacheView& par, uint32_t t, const uint8_t* ops, uint32_t n,
                                         uint32_t x) {
    const int lane = lane_id();
    const int32_t e = find_exact(par.e_pos, par.e_off[t], par.e_off[t + 1], x);
    if (e >= 0) return par.e_end[e] - x;
    int bal = 1;                                      // nodes still needed at the window start
    for (uint32_t w0 = x; w0 < n; w0 += 512) {
        const uint32_t p0 = w0 + 16u * lane;
        uint32_t wd[4] = {0, 0, 0, 0};
        if (p0 < n) {
            const uint4 v = load16u(ops + p0);
            wd[0] = v.x; wd[1] = v.y; wd[2] = v.z; wd[3] = v.w;
        }
        int tot = 0, mn = 1 << 30;
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            if (p0 + b < n) {
                const uint32_t op = (wd[b >> 2] >> (8 * (b & 3))) & 0xFFu;
                tot += (op < 4) ? 1 : -1;
                mn = min(mn, tot);
            }
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int start = bal + incl - tot;
        const uint32_t hit = __ballot_sync(FULL, mn != (1 << 30) && start + mn <= 0);
        if (hit) {
            const int src = __ffs(hit) - 1;
            uint32_t end = 0;
            if (lane == src) {
                int sv = start;
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    if (end == 0 && p0 + b < n) {
                        const uint32_t op = (wd[b >> 2] >> (8 * (b & 3))) & 0xFFu;
                        sv += (op < 4) ? 1 : -1;
                        if (sv == 0) end = p0 + b + 1;
                    }
                }
            }
            end = __shfl_sync(FULL, end, src);
            return end - x;
        }
        bal += __shfl_sync(FULL, incl, 31);
    }
    return n - x;     // unreachable for well-formed trees
}

__device__ __forceinline__ uint32_t tournament(const float* fit, uint32_t P, uint32_t T, uint64_t seed,
                                               uint32_t gen, uint32_t child, uint32_t kbase) {
    uint32_t best = 0;
    float bf = 0.f;
    for (uint32_t j = 0; j < T; ++j) {
        uint32_t idx = (uint32_t)below(draw(seed, gen, child, kbase + j), P);
        float f = fit[idx];
        if (isnan(f)) f = __int_as_float(0x7F800000);
        if (j == 0 || f < bf) { best = idx; bf = f; }
    }
    return best;
}


// ------------------------------------------------------------------ A5 plan

// Child i: mother and father by tournament (draws 0..T-1 and T..2T-1), then
// up to 8 attempts of crossover points uniform over the nodes of each
// parent (draws 2T+2a, 2T+2a+1) whose child fits max_nodes; otherwise the
// child is a copy of its mother.
__global__ void k_plan(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < d.P; i += nwp) {       // one warp per child
        const uint32_t T = g.tsize;
        const uint32_t gen = g.gen + *g.gen_add;
        const uint32_t m = tournament(g.pfit, d.P, T, g.seed, gen, i, 0);
        const uint32_t f = tournament(g.pfit, d.P, T, g.seed, gen, i, T);
        const uint32_t sm = g.psize[m], sf = g.psize[f];
        const uint8_t* om = d.arena + (size_t)g.pbuf[m] * d.cap;
        const uint8_t* of = d.arena + (size_t)g.pbuf[f] * d.cap;
        uint32_t fl = F_CLONE, cc = 0, rr = sm, dd = 0, ss = sm, ff = m;
        for (uint32_t a = 0; a < 8; ++a) {
            const uint32_t c1 = (uint32_t)below(draw(g.seed, gen, i, 2 * T + 2 * a), sm);
            const uint32_t d1 = (uint32_t)below(draw(g.seed, gen, i, 2 * T + 2 * a + 1), sf);
            const uint32_t r1 = warp_subtree_size_at(par, m, om, sm, c1);
            const uint32_t s1 = warp_subtree_size_at(par, f, of, sf, d1);
            if ((uint64_t)sm - r1 + s1 <= g.max_nodes) { fl = 0; cc = c1; rr = r1; dd = d1; ss = s1; ff = f; break; }
        }
        if (lane_id() == 0) {
            g.mother[i] = m; g.father[i] = ff; g.cpos[i] = cc; g.rsz[i] = rr; g.dpos[i] = dd; g.ssz[i] = ss;
            g.flags[i] = fl;
            atomicMax(&g.lastidx[m], (int32_t)i);
        }
    }
}

// ------------------------------------------------------------------ fitness-first materialisation
//
// The paper observes that most children never become parents (Sec. 6.3) and
// that only those needed later must be built.  In this mode the walk reads a
// child through its mother's buffer and the father's donated subtree, the
// next generation's plan is drawn right after the walk, and only the
// children it selects get a tree buffer and a cache.  The draws are the same
// as in the eager order, so every result is identical.

#define BUF_NONE 0xFFFFFFFFu

// Subtree size at x of child t of the current generation (not built yet):
// from its plan and its parents' caches and bytes.
__device__ uint32_t virtual_subtree_size(const DevPop& d, const GenBufs& g, const CacheView& par, uint32_t t,
                                         uint32_t x) {
    const uint32_t m = g.mother[t];
    const uint8_t* mb = d.arena + (size_t)g.pbuf[m] * d.cap;
    const uint32_t sm = g.psize[m];
    if (g.flags[t] & F_CLONE) return warp_subtree_size_at(par, m, mb, sm, x);
    const uint32_t c = g.cpos[t], r = g.rsz[t], s = g.ssz[t];
    if (x >= c && x < c + s) {
        const uint32_t f = g.father[t];
        return warp_subtree_size_at(par, f, d.arena + (size_t)g.pbuf[f] * d.cap, g.psize[f], g.dpos[t] + (x - c));
    }
    if (x >= c + s) return warp_subtree_size_at(par, m, mb, sm, x - s + r);
    const uint32_t ms = warp_subtree_size_at(par, m, mb, sm, x);
    return (x + ms > c) ? ms + s - r : ms;          // an ancestor of c changes by the size change
}

// The next generation's plan from the current children's fitness, drawn
// exactly as k_plan draws it (generation gen + 1), one warp per child.
__global__ void k_plan_next(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < d.P; i += nwp) {
        const uint32_t T = g.tsize;
        const uint32_t gen = g.gen + 1 + *g.gen_add;
        const uint32_t m = tournament(d.fit, d.P, T, g.seed, gen, i, 0);
        const uint32_t f = tournament(d.fit, d.P, T, g.seed, gen, i, T);
        const uint32_t sm = d.size[m], sf = d.size[f];
        uint32_t fl = F_CLONE, cc = 0, rr = sm, dd = 0, ss = sm, ff = m;
        for (uint32_t a = 0; a < 8; ++a) {
            const uint32_t c1 = (uint32_t)below(draw(g.seed, gen, i, 2 * T + 2 * a), sm);
            const uint32_t d1 = (uint32_t)below(draw(g.seed, gen, i, 2 * T + 2 * a + 1), sf);
            const uint32_t r1 = virtual_subtree_size(d, g, par, m, c1);
            const uint32_t s1 = virtual_subtree_size(d, g, par, f, d1);
            if ((uint64_t)sm - r1 + s1 <= g.max_nodes) { fl = 0; cc = c1; rr = r1; dd = d1; ss = s1; ff = f; break; }
        }
        if (lane_id() == 0) {
            g.nmother[i] = m; g.nfather[i] = ff; g.ncpos[i] = cc; g.nrsz[i] = rr; g.ndpos[i] = dd; g.nssz[i] = ss;
            g.nflags[i] = fl;
            g.sel[m] = 1u;
            g.sel[ff] = 1u;
        }
    }
}

// The plan drawn after the last walk becomes this generation's.
__global__ void k_plan_take(DevPop d, GenBufs g) {
    if (halted(d)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x) {
        g.mother[i] = g.nmother[i]; g.father[i] = g.nfather[i]; g.cpos[i] = g.ncpos[i];
        g.rsz[i] = g.nrsz[i]; g.dpos[i] = g.ndpos[i]; g.ssz[i] = g.nssz[i]; g.flags[i] = g.nflags[i];
    }
}

// Block-wide exclusive scan of v (1024 threads); returns the exclusive
// prefix and adds the block total to *carry (shared).
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* ws, uint64_t* carry) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) { uint64_t t = __shfl_up_sync(FULL, s, o); if (lane >= o) s += t; }
    if (lane == 31) ws[w] = s;
    __syncthreads();
    if (w == 0) {
        uint64_t x = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { uint64_t t = __shfl_up_sync(FULL, x, o); if (lane >= o) x += t; }
        ws[lane] = x;
    }
    __syncthreads();
    const uint64_t incl = s + (w > 0 ? ws[w - 1] : 0);
    const uint64_t res = *carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) *carry += incl;
    __syncthreads();
    return res;
}

// Halo bytes reserved per block of an in-place move with size change delta:
// at most min(|delta|, SHIFT_BS) bytes of a block's source are overwritten
// by the other blocks' destinations.
__host__ __device__ __forceinline__ uint32_t halo_stride(int32_t delta) {
    const uint32_t a = (uint32_t)(delta < 0 ? -delta : delta);
    return a < (uint32_t)SHIFT_BS ? a : (uint32_t)SHIFT_BS;
}

// Buffer assignment and offsets (one CTA of 1024 threads).  The last child
// of a mother is built in place in her buffer (Fig. 2) when its size change
// is at most EAGER_HALO_MAX bytes (and the halo pool has room); every other
// child is copied into a free buffer (Fig. 1), which the eager order always
// has.  A larger size change would route most of the tail through the halo
// (about min(|delta|, SHIFT_BS) of every SHIFT_BS bytes), costing more than
// the copy.  Buffers of parents without an in-place child are freed.
__global__ void __launch_bounds__(1024) k_assign(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry[7];
    if (threadIdx.x < 7) carry[threadIdx.x] = 0;
    for (uint32_t j = threadIdx.x; j < d.P; j += blockDim.x) g.hasip[j] = 0;
    __syncthreads();
    const uint32_t P = d.P;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t copy = 0, nblk = 0, nch = 0;
        uint64_t fragb = 0, stashb = 0, xob = 0, hb = 0;
        bool last = false, clone = false;
        uint32_t m = 0, fl = 0, r = 0, s = 0, c = 0, sm = 0;
        int64_t delta = 0;
        uint64_t tail = 0;
        if (i < P) {
            m = g.mother[i];
            fl = g.flags[i];
            last = g.lastidx[m] == (int32_t)i;
            clone = (fl & F_CLONE) != 0;
            r = g.rsz[i]; s = g.ssz[i]; c = g.cpos[i];
            sm = g.psize[m];
            delta = (int64_t)s - (int64_t)r;
            tail = (uint64_t)sm - c - r;
            if (last && !clone && delta != 0 && tail > 0 && delta >= -EAGER_HALO_MAX && delta <= EAGER_HALO_MAX) {
                nblk = (uint32_t)((tail + SHIFT_BS - 1) / SHIFT_BS);
                hb = (uint64_t)nblk * halo_stride((int32_t)delta);
            }
        }
        const uint64_t ho = block_excl_scan(hb, ws, &carry[6]);
        if (i < P) {
            const bool inplace = last && (clone || (delta >= -EAGER_HALO_MAX && delta <= EAGER_HALO_MAX &&
                                                    ho + hb <= g.halo_cap));
            if (!inplace) nblk = 0;
            if (last) fl |= F_LAST;
            if (inplace) { fl |= F_INPLACE; g.hasip[m] = 1; }
            g.flags[i] = fl;
            copy = inplace ? 0 : 1;
            d.size[i] = (uint32_t)((int64_t)sm + delta);
            if (copy) nch = (uint32_t)(((int64_t)sm + delta + COPY_CH - 1) / COPY_CH);
            if (!clone) {
                fragb = (s + 15u) & ~15u;
                if (r < d.T) stashb = (r + 15u) & ~15u;
                xob = 2ull * s + (r < d.T ? 2ull * r : 0) +
                      (inplace ? (delta != 0 ? 2ull * tail : 0) + s : 2ull * ((uint64_t)sm - r + s));
            } else if (!inplace) {
                xob = 2ull * sm;
            }
            g.halo_off[i] = ho;
            const uint32_t nk = (uint32_t)((int64_t)sm + delta);
            g.onepass[i] = (!clone && nk <= g.onepass_max && !g.dis) ? 1u : 0u;
        }
        const uint64_t rank = block_excl_scan(copy, ws, &carry[0]);
        const uint64_t fo = block_excl_scan(fragb, ws, &carry[1]);
        const uint64_t so = block_excl_scan(stashb, ws, &carry[2]);
        const uint64_t bo = block_excl_scan(nblk, ws, &carry[3]);
        const uint64_t xo = block_excl_scan(xob, ws, &carry[4]);
        const uint64_t co = block_excl_scan(nch, ws, &carry[5]);
        (void)xo;
        if (i < P) {
            d.buf[i] = copy ? g.free_buf[rank] : g.pbuf[m];
            g.frag_off[i] = fo;
            g.stash_off[i] = so;
            g.shift_off[i] = (uint32_t)bo;
            g.copy_off[i] = (uint32_t)co;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        g.frag_off[P] = carry[1];
        g.stash_off[P] = carry[2];
        g.shift_off[P] = (uint32_t)carry[3];
        g.copy_off[P] = (uint32_t)carry[5];
        g.halo_off[P] = carry[6];
        g.misc[M_NCOPY] = (uint32_t)carry[0];
        g.misc[M_NSHIFT] = (uint32_t)carry[3];
        g.gstat[G_XOBYTES] = carry[4];
        if (carry[1] > g.frag_cap || carry[2] > g.stash_cap || carry[3] > g.shift_cap) set_status(d.status, ST_CAPACITY);
    }
    __syncthreads();
    // next free list: unused free buffers, then buffers of parents with no in-place child
    const uint32_t ncopy = (uint32_t)carry[0];
    __shared__ uint64_t carry2;
    if (threadIdx.x == 0) carry2 = 0;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < P - ncopy; k += blockDim.x) g.free_next[k] = g.free_buf[ncopy + k];
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        const uint32_t fr = (j < P && !g.hasip[j]) ? 1u : 0u;
        const uint64_t pos = block_excl_scan(fr, ws, &carry2);
        if (fr && (P - ncopy) + pos < P) g.free_next[(P - ncopy) + pos] = g.pbuf[j];
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < P; k += blockDim.x) g.free_buf[k] = g.free_next[k];
}

// Fitness-first order, at crossover: child sizes, fragment and stash
// offsets; no child is built yet (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_assign_lazy(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry[3];
    if (threadIdx.x < 3) carry[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t P = d.P;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint64_t fragb = 0, stashb = 0, xob = 0;
        if (i < P) {
            const uint32_t m = g.mother[i];
            const bool clone = g.flags[i] & F_CLONE;
            const uint32_t r = g.rsz[i], s = g.ssz[i];
            d.size[i] = (uint32_t)((int64_t)g.psize[m] + (int64_t)s - (int64_t)r);
            d.buf[i] = BUF_NONE;
            g.onepass[i] = (!clone && d.size[i] <= g.onepass_max && !g.dis) ? 1u : 0u;
            if (!clone) {
                fragb = (s + 15u) & ~15u;
                if (r < d.T) stashb = (r + 15u) & ~15u;
                xob = 2ull * s + (r < d.T ? 2ull * r : 0);
            }
        }
        const uint64_t fo = block_excl_scan(fragb, ws, &carry[0]);
        const uint64_t so = block_excl_scan(stashb, ws, &carry[1]);
        const uint64_t xo = block_excl_scan(xob, ws, &carry[2]);
        (void)xo;
        if (i < P) {
            g.frag_off[i] = fo;
            g.stash_off[i] = so;
            g.shift_off[i] = 0;
            g.copy_off[i] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        g.frag_off[P] = carry[0];
        g.stash_off[P] = carry[1];
        g.shift_off[P] = 0;
        g.copy_off[P] = 0;
        g.gstat[G_XOBYTES] = carry[2];
        if (carry[0] > g.frag_cap || carry[1] > g.stash_cap) set_status(d.status, ST_CAPACITY);
    }
}

// Fitness-first order, after the walk: the children selected as parents
// get their buffers.  In the memory-lean form (lazy_inplace) the last
// selected child of each mother takes her buffer and is built there in
// place at the start of the next crossover
// (Fig. 2: no sibling reads the mother after this generation's copies, and
// the children that are not built are readable through their parents only
// until then), while the halo pool of the move has room; a cloned child
// needs no move at all.  The other selected children take buffers from the
// free stack and get copy chunks; the previous parents' buffers not taken
// in place return to the stack (they are read by the copies, and by
// gp_get_tree of unselected children, until the next materialisation).
__global__ void __launch_bounds__(1024) k_materialise_assign(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry[7];
    __shared__ uint32_t nfree0;
    if (threadIdx.x < 7) carry[threadIdx.x] = 0;
    if (threadIdx.x == 0) nfree0 = *g.nfree;
    const uint32_t P = d.P;
    // parents that a child of this generation reads (its mother's tree, or
    // its father's, for the trees of the children that are not built), and
    // each mother's last selected child
    for (uint32_t j = threadIdx.x; j < P; j += blockDim.x) { g.pref[j] = 0u; g.lastsel[j] = -1; g.hasip[j] = 0u; }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
        g.pref[g.mother[i]] = 1u;
        g.pref[g.father[i]] = 1u;
        if (g.sel[i]) atomicMax(&g.lastsel[g.mother[i]], (int32_t)i);
    }
    __syncthreads();
    // parents no child reads give their buffers back first (the initial
    // population's unselected trees); the selected children then take the
    // top of the stack
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        const uint32_t b = (j < P) ? g.pbuf[j] : BUF_NONE;
        const uint32_t dead = (b != BUF_NONE && !g.pref[j]) ? 1u : 0u;
        const uint64_t pos = block_excl_scan(dead, ws, &carry[3]);
        if (dead) g.free_buf[nfree0 + pos] = b;
    }
    // which selected children are built in place (halo pool permitting)
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool ip = false, clone = false;
        uint64_t hb = 0;
        uint32_t nblk = 0;
        if (i < P && g.sel[i]) {
            const uint32_t m = g.mother[i];
            ip = g.lazy_inplace && g.lastsel[m] == (int32_t)i && g.pbuf[m] != BUF_NONE;
            clone = (g.flags[i] & F_CLONE) != 0;
            if (ip && !clone) {
                const int32_t delta = (int32_t)g.ssz[i] - (int32_t)g.rsz[i];
                const uint32_t tail = (uint32_t)((int64_t)d.size[i] - delta) - g.cpos[i] - g.rsz[i];
                if (delta != 0 && tail > 0) {
                    nblk = (tail + SHIFT_BS - 1) / SHIFT_BS;
                    hb = (uint64_t)nblk * halo_stride(delta);
                }
            }
        }
        const uint64_t ho = block_excl_scan(hb, ws, &carry[5]);
        if (i < P) {
            if (ip && !clone && ho + hb > g.halo_cap) { ip = false; nblk = 0; }
            uint32_t fl = g.flags[i] & ~F_INPLACE;
            if (ip) { fl |= F_INPLACE; g.hasip[g.mother[i]] = 1u; }
            g.flags[i] = fl;
            g.halo_off[i] = ho;
        }
        const uint64_t bo = block_excl_scan(nblk, ws, &carry[6]);
        if (i < P) g.shift_off[i] = (uint32_t)bo;
    }
    __syncthreads();
    // the children selected and not built in place need buffers
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t selc = (i < P && g.sel[i] && !(g.flags[i] & F_INPLACE)) ? 1u : 0u;
        block_excl_scan(selc, ws, &carry[2]);
    }
    const uint32_t nsel = (uint32_t)carry[2];
    const uint32_t nfree1 = nfree0 + (uint32_t)carry[3];
    if (nsel > nfree1) {
        if (threadIdx.x == 0) set_status(d.status, ST_CAPACITY);
        return;
    }
    const uint32_t take0 = nfree1 - nsel;
    __shared__ uint32_t npend;
    if (threadIdx.x == 0) npend = 0;
    __syncthreads();
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t selc = 0, nch = 0;
        uint64_t xob = 0;
        const bool ip = i < P && (g.flags[i] & F_INPLACE);
        if (i < P && g.sel[i] && !ip) {
            selc = 1;
            const uint32_t nk = d.size[i];
            nch = (nk + COPY_CH - 1) / COPY_CH;
            xob = 2ull * nk;
        } else if (ip && !(g.flags[i] & F_CLONE)) {
            const int32_t delta = (int32_t)g.ssz[i] - (int32_t)g.rsz[i];
            const uint64_t tail = (uint64_t)((int64_t)d.size[i] - delta) - g.cpos[i] - g.rsz[i];
            xob = (delta != 0 ? 2ull * tail : 0ull) + g.ssz[i];
            atomicAdd(&npend, 1u);
        }
        const uint64_t rank = block_excl_scan(selc, ws, &carry[0]);
        const uint64_t co = block_excl_scan(nch, ws, &carry[1]);
        if (i < P) {
            d.buf[i] = selc ? g.free_buf[take0 + rank] : ip ? g.pbuf[g.mother[i]] : BUF_NONE;
            g.copy_off[i] = (uint32_t)co;
            if (xob) atomicAdd(&g.gstat[G_XOBYTES], xob);
        }
    }
    __syncthreads();
    // the parents that children read go back on the stack after the targets
    // (unless a child took the buffer in place): they are overwritten no
    // earlier than the next generation's copies
    __shared__ uint64_t cfree;
    if (threadIdx.x == 0) cfree = 0;
    __syncthreads();
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t j = base + threadIdx.x;
        const uint32_t b = (j < P) ? g.pbuf[j] : BUF_NONE;
        const uint32_t has = (b != BUF_NONE && g.pref[j] && !g.hasip[j]) ? 1u : 0u;
        const uint64_t pos = block_excl_scan(has, ws, &cfree);
        if (has) g.free_buf[take0 + pos] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        g.copy_off[P] = (uint32_t)carry[1];
        g.halo_off[P] = carry[5];
        g.shift_off[P] = (uint32_t)carry[6];
        g.misc[M_NCOPY] = nsel;
        *g.nfree = take0 + (uint32_t)cfree;
        *g.npend = npend;
    }
}

// ------------------------------------------------------------------ A6 gather

// Donated subtrees (all children) and removed subtrees below the threshold
// copied out before any buffer is written (Sec. 5: fatherless crossover).
__global__ void k_gather(DevPop d, GenBufs g) {
    if (halted(d)) return;
    if (g.frag_off[d.P] > g.frag_cap || g.stash_off[d.P] > g.stash_cap) return;
    for (uint32_t i = blockIdx.x; i < d.P; i += gridDim.x) {
        if (g.flags[i] & F_CLONE) continue;
        const uint8_t* of = d.arena + (size_t)g.pbuf[g.father[i]] * d.cap + g.dpos[i];
        uint8_t* dst = g.frag + g.frag_off[i];
        const uint32_t s = g.ssz[i];
        for (uint32_t q = threadIdx.x; q < (s + 15) / 16; q += blockDim.x)
            reinterpret_cast<uint4*>(dst)[q] = load16u(of + 16 * q);
        const uint32_t r = g.rsz[i];
        if (r < d.T) {
            const uint8_t* om = d.arena + (size_t)g.pbuf[g.mother[i]] * d.cap + g.cpos[i];
            uint8_t* st = g.stash + g.stash_off[i];
            for (uint32_t q = threadIdx.x; q < (r + 15) / 16; q += blockDim.x)
                reinterpret_cast<uint4*>(st)[q] = load16u(om + 16 * q);
        }
    }
}

// ------------------------------------------------------------------ A8 materialise

// Children built in a free buffer: mother head, donated subtree, mother
// tail (Fig. 1).  The copies are cut into COPY_CH-byte chunks spread over
// the whole grid; each thread moves 16 destination bytes at a time, four
// loads in flight before the stores.
__device__ __forceinline__ uint4 child_quad(const uint8_t* __restrict__ om, const uint8_t* __restrict__ fr,
                                            uint32_t o, uint32_t c, uint32_t r, uint32_t s, uint32_t nk) {
    if (o + 16 <= c) return *reinterpret_cast<const uint4*>(om + o);
    if (o >= c + s) return load16u(om + (o - s + r));
    if (o >= c && o + 16 <= c + s) return load16u(fr + (o - c));
    uint8_t b[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const uint32_t x = o + t;
        b[t] = (x < c) ? om[x] : (x < c + s) ? fr[x - c] : (x < nk ? om[x - s + r] : 0);
    }
    return *reinterpret_cast<uint4*>(b);
}

__global__ void __launch_bounds__(256) k_copy_children(DevPop d, GenBufs g) {
    if (halted(d)) return;
    if (g.frag_off[d.P] > g.frag_cap) return;
    const uint32_t nu = g.copy_off[d.P];
    constexpr uint32_t QCH = COPY_CH / 16;
    for (uint32_t u = blockIdx.x; u < nu; u += gridDim.x) {
        const uint32_t i = find_segment(g.copy_off, d.P, u);
        const uint32_t j = u - g.copy_off[i];
        const uint32_t fl = g.flags[i];
        const uint8_t* om = d.arena + (size_t)g.pbuf[g.mother[i]] * d.cap;
        uint4* dst = reinterpret_cast<uint4*>(d.arena + (size_t)d.buf[i] * d.cap);
        const uint32_t nk = d.size[i];
        const uint32_t q0 = j * QCH, q1 = min((nk + 15) / 16, q0 + QCH);
        const bool clone = (fl & F_CLONE) != 0;
        const uint32_t c = clone ? nk : g.cpos[i], r = clone ? 0 : g.rsz[i], s = clone ? 0 : g.ssz[i];
        const uint8_t* fr = g.frag + (clone ? 0 : g.frag_off[i]);
        for (uint32_t q = q0 + threadIdx.x; q < q1; q += 4 * 256) {
            uint4 v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t qq = q + t * 256;
                if (qq < q1) v[t] = clone ? reinterpret_cast<const uint4*>(om)[qq] : child_quad(om, fr, 16 * qq, c, r, s, nk);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t qq = q + t * 256;
                if (qq < q1) dst[qq] = v[t];
            }
        }
    }
}

// In-place children (Fig. 2): the tail [c+r, n) of the mother moves by
// delta = s - r within her buffer, then the donated subtree is written at
// c.  Blocks of SHIFT_BS source bytes move concurrently.  The bytes of a
// block's source that another block's destination covers are saved first
// (k_save_halo) and read from there: for delta > 0 they are the block's
// bytes at or after c + s that the earlier blocks' destinations [c + s,
// a_j + delta) reach, for delta < 0 the bytes from a_j + L_j + delta on that
// the later blocks' destinations reach -- at most min(|delta|, SHIFT_BS)
// bytes per block, whatever the size change.  A block's own source and
// destination may overlap: it stages its source in shared memory first.
//
// Eager order builds a mother's last child at crossover (its buffer is
// d.buf[i], the mother's size psize[mother]).  Fitness-first order defers
// it to the start of the next crossover, after every sibling has been
// copied from the mother and before the buffers are read again: the
// generations have then been swapped, so the child's buffer is pbuf[i] and
// its size psize[i] (deferred = true).
struct InPlace {
    uint8_t* buf;
    uint32_t c, r, s, tail;
    int32_t delta;
};

__device__ __forceinline__ InPlace inplace_of(const DevPop& d, const GenBufs& g, uint32_t i, bool deferred) {
    InPlace q;
    q.c = g.cpos[i];
    q.r = g.rsz[i];
    q.s = g.ssz[i];
    q.delta = (int32_t)q.s - (int32_t)q.r;
    uint32_t b, nm;
    if (deferred) { b = g.pbuf[i]; nm = (uint32_t)((int64_t)g.psize[i] - q.delta); }
    else { b = d.buf[i]; nm = g.psize[g.mother[i]]; }
    q.buf = d.arena + (size_t)b * d.cap;
    q.tail = nm - q.c - q.r;
    return q;
}

// Block b of the moves: child i, its block j, source [src0, src0 + len),
// the halo range [h0, h1) of that source and where its bytes are kept.
struct ShiftBlock {
    uint32_t i, j, src0, len, h0, h1;
    InPlace q;
    uint8_t* halo;
};

__device__ __forceinline__ ShiftBlock shift_block(const DevPop& d, const GenBufs& g, uint32_t b, bool deferred) {
    ShiftBlock k;
    k.i = find_segment(g.shift_off, d.P, b);
    k.j = b - g.shift_off[k.i];
    k.q = inplace_of(d, g, k.i, deferred);
    k.src0 = k.q.c + k.q.r + k.j * SHIFT_BS;
    k.len = min((uint32_t)SHIFT_BS, k.q.tail - k.j * SHIFT_BS);
    const int64_t a = k.src0, e = (int64_t)k.src0 + k.len, dl = k.q.delta;
    int64_t h0, h1;
    if (dl > 0) { h0 = max(a, (int64_t)k.q.c + k.q.s); h1 = min(e, a + dl); }
    else { h0 = max(a, e + dl); h1 = min(e, (int64_t)k.q.c + k.q.r + k.q.tail + dl); }
    if (h1 < h0) h1 = h0;
    k.h0 = (uint32_t)h0;
    k.h1 = (uint32_t)h1;
    k.halo = g.halo + g.halo_off[k.i] + (uint64_t)k.j * halo_stride(k.q.delta);
    return k;
}

// the halo bytes of every block, before any block moves (a CTA per block)
__global__ void k_save_halo(DevPop d, GenBufs g, int deferred) {
    if (halted(d)) return;
    if (deferred && *g.npend == 0) return;          // nothing deferred (or a stale plan)
    const uint32_t nb = g.shift_off[d.P];
    if (nb > g.shift_cap || g.halo_off[d.P] > g.halo_cap) return;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const ShiftBlock k = shift_block(d, g, b, deferred != 0);
        for (uint32_t x = k.h0 + threadIdx.x; x < k.h1; x += blockDim.x) k.halo[x - k.h0] = k.q.buf[x];
    }
}

__global__ void __launch_bounds__(512) k_shift(DevPop d, GenBufs g, int deferred) {
    if (halted(d)) return;
    if (deferred && *g.npend == 0) return;          // nothing deferred (or a stale plan)
    // the block's source bytes from its 16-byte-aligned start, plus slack for the shifted reads
    __shared__ __align__(16) uint8_t sb[SHIFT_BS + 48];
    const uint32_t nb = g.shift_off[d.P];
    if (nb > g.shift_cap || g.halo_off[d.P] > g.halo_cap) return;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const ShiftBlock k = shift_block(d, g, b, deferred != 0);
        uint8_t* buf = k.q.buf;
        const uint32_t src0 = k.src0, len = k.len;
        const int32_t delta = k.q.delta;
        const uint32_t a0 = src0 & ~15u, m0 = src0 & 15u;
        // stage the source quads (the halo range, which other blocks may be writing, from the halo)
        const uint32_t nq = (m0 + len + 15u) / 16u;
        for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x)
            reinterpret_cast<uint4*>(sb)[q] = reinterpret_cast<const uint4*>(buf + a0)[q];
        __syncthreads();
        for (uint32_t x = k.h0 + threadIdx.x; x < k.h1; x += blockDim.x) sb[m0 + (x - src0)] = k.halo[x - k.h0];
        __syncthreads();
        // destination [dst0, dst0 + len): whole aligned quads in the middle, single bytes at the ends
        const uint32_t dst0 = (uint32_t)((int64_t)src0 + delta);
        const uint32_t dq0 = (dst0 + 15u) / 16u, dq1 = (dst0 + len) / 16u;
        const uint32_t head_end = min(16u * dq0, dst0 + len);
        const uint32_t tail_begin = max(16u * dq1, head_end);
        for (uint32_t x = dst0 + threadIdx.x; x < head_end; x += blockDim.x) buf[x] = sb[m0 + (x - dst0)];
        for (uint32_t x = tail_begin + threadIdx.x; x < dst0 + len; x += blockDim.x) buf[x] = sb[m0 + (x - dst0)];
        if (dq1 > dq0) {
            // sb byte of destination byte 16 dq: m0 + 16 dq - dst0 (same misalignment for every quad)
            const uint32_t u0 = m0 + 16u * dq0 - dst0;
            const uint32_t mu = u0 & 15u, mw = mu >> 2, sh = (mu & 3u) * 8u;
            uint4* dst = reinterpret_cast<uint4*>(buf);
            for (uint32_t q = dq0 + threadIdx.x; q < dq1; q += blockDim.x) {
                const uint32_t u = (u0 >> 4) + (q - dq0);
                const uint4 lo = reinterpret_cast<const uint4*>(sb)[u];
                uint4 v = lo;
                if (mu) {
                    const uint4 hi = reinterpret_cast<const uint4*>(sb)[u + 1];
                    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                    uint32_t r[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        uint32_t xx = 0, yy = 0;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if ((uint32_t)c == mw) { xx = w[t + c]; yy = w[t + c + 1]; }
                        r[t] = __funnelshift_r(xx, yy, sh);
                    }
                    v = make_uint4(r[0], r[1], r[2], r[3]);
                }
                dst[q] = v;
            }
        }
        __syncthreads();
    }
}

// Donated subtree written into the in-place children (after the move):
// whole aligned quads of the destination from the (shifted) fragment, single
// bytes at the two ends.
__global__ void k_write_frags(DevPop d, GenBufs g, int deferred) {
    if (halted(d)) return;
    if (deferred && *g.npend == 0) return;          // nothing deferred (or a stale plan)
    if (g.frag_off[d.P] > g.frag_cap) return;
    for (uint32_t i = blockIdx.x; i < d.P; i += gridDim.x) {
        const uint32_t fl = g.flags[i];
        if (!(fl & F_INPLACE) || (fl & F_CLONE)) continue;
        const InPlace q = inplace_of(d, g, i, deferred != 0);
        uint8_t* buf = q.buf;
        const uint8_t* fr = g.frag + g.frag_off[i];
        const uint32_t c = q.c, s = q.s;
        const uint32_t dq0 = (c + 15u) / 16u, dq1 = (c + s) / 16u;
        const uint32_t head_end = min(16u * dq0, c + s);
        const uint32_t tail_begin = max(16u * dq1, head_end);
        for (uint32_t x = c + threadIdx.x; x < head_end; x += blockDim.x) buf[x] = fr[x - c];
        for (uint32_t x = tail_begin + threadIdx.x; x < c + s; x += blockDim.x) buf[x] = fr[x - c];
        if (dq1 > dq0) {
            for (uint32_t q4 = dq0 + threadIdx.x; q4 < dq1; q4 += blockDim.x)
                reinterpret_cast<uint4*>(buf)[q4] = load16u(fr + (16u * q4 - c));
        }
    }
}

// Fitness-first order: the deferred in-place children are built; the flags
// of this generation's plan are then cleared of F_INPLACE by the plan the
// crossover takes next.
__global__ void k_inplace_done(GenBufs g) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *g.npend = 0;
}

// Individual i's bytes into `out` (a device buffer of at least cap bytes)
// for gp_get_tree: from its own buffer, or -- a child of the fitness-first
// order that is not built, or built in place only at the next crossover --
// from its mother's head, the donated subtree in its father's buffer and
// the mother's tail (Fig. 1).  meta = {size, 1 if the bytes are available}.
// Every CTA derives the same pieces and copies its share of the bytes.
__global__ void k_get_tree(DevPop d, GenBufs g, uint32_t i, uint32_t lazy_plan, uint8_t* __restrict__ out,
                           uint32_t* __restrict__ meta) {
    const uint32_t n = d.size[i], b = d.buf[i];
    uint32_t fl0 = 0, npend = 0;
    if (lazy_plan) { fl0 = g.flags[i]; npend = *g.npend; }
    const bool pending = npend && (fl0 & F_INPLACE) && !(fl0 & F_CLONE);
    const uint8_t* s0 = nullptr;
    const uint8_t* s1 = nullptr;
    const uint8_t* s2 = nullptr;
    uint32_t l0 = n, l1 = 0, ok = 1;
    if (b != BUF_NONE && !pending) {
        s0 = d.arena + (size_t)b * d.cap;
    } else {
        const uint32_t m = g.mother[i], f = g.father[i], bm = g.pbuf[m], bf = g.pbuf[f];
        if (bm == BUF_NONE || bf == BUF_NONE) {
            ok = 0;
        } else {
            s0 = d.arena + (size_t)bm * d.cap;
            if (!(g.flags[i] & F_CLONE)) {
                const uint32_t c = g.cpos[i], r = g.rsz[i];
                l0 = c;
                l1 = g.ssz[i];
                s1 = d.arena + (size_t)bf * d.cap + g.dpos[i];
                s2 = s0 + c + r;                 // the tail: child byte x >= c + l1 is mother byte x - l1 + r
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) { meta[0] = n; meta[1] = ok; }
    if (!ok || !out) return;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        out[x] = x < l0 ? s0[x] : x < l0 + l1 ? s1[x - l0] : s2[x - l0 - l1];
}

// ------------------------------------------------------------------ A7 incremental walk

template <int K>
__device__ __forceinline__ void load_vec(const float* slots, uint32_t Cpad, uint32_t slot, float (&v)[K],
                                         uint32_t cb = 0) {
    const int lane = lane_id();
    const float* p = slots + (size_t)slot * Cpad + cb * 32 * K + lane;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = __ldcg(p + k * 32);
}

template <int K>
__device__ __forceinline__ void store_blk(float* row, uint32_t cb, const float (&v)[K]) {
    float* p = row + cb * 32 * K + lane_id();
#pragma unroll
    for (int k = 0; k < K; ++k) p[k * 32] = v[k];
}

template <int K>
__device__ __forceinline__ void load_blk(const float* row, uint32_t cb, float (&v)[K]) {
    const float* p = row + cb * 32 * K + lane_id();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = p[k * 32];
}


// Shared-memory layout of one walk team (a CTA of nw warps working on one
// child): constant tables, the small-ancestor lists, the level descriptors
// of a batch, the running value vectors of the child and of the mother,
// the siblings' vectors of a batch, a few broadcast words, then per warp an
// interpreter stack and two staging buffers.
struct LevelDesc {
    uint32_t p, pend, ss, se;   // ancestor, its end in the child, sibling range [ss, se)
    int32_t pent, sib;          // mother cache entry of p (-1: small) and of the sibling (-1: interpret)
    uint32_t flags;             // op | left << 8 | child-cached << 9 | bad range << 10 | missing sibling << 11
    int32_t k;                  // ancestor index along the path
    uint32_t pslot, sslot;      // value slots of pent and sib in the mother's cache
    uint32_t pad0, pad1;
};
#define LD_LEFT (1u << 8)
#define LD_CACHED (1u << 9)
#define LD_BAD (1u << 10)
#define LD_NOSIB (1u << 11)

#define WALK_RING 32           // most levels a walk team keeps in flight (descriptors and sibling values)
#define WALK_SPIN (1u << 22)   // default bound on the polls of one wait inside a walk team (DevPop::wait_polls)

// levels in flight: fewer when value vectors are long
__host__ __device__ inline uint32_t walk_ring(uint32_t Cpad) { return Cpad <= 128 ? 32u : Cpad <= 256 ? 8u : 4u; }

template <int K>
struct TeamLayout {
    uint32_t kc, anc, ancg, lvl, desc, nv, ov, sv, mv, cur, sc, warp0, warp_bytes, total;
    __host__ __device__ TeamLayout(int W, uint32_t Cpad, uint32_t nw) {
        const uint32_t ring = walk_ring(Cpad);
        uint32_t o = 0;
        kc = o;   o += (256 + 6 * 32) * 4;
        anc = o;  o += WALK_MAXLVL * 4;
        ancg = o; o += WALK_MAXLVL * 4;
        lvl = o;  o += WALK_MAXLVL * 4;
        desc = o; o += WALK_RING * sizeof(LevelDesc);
        nv = o;   o += Cpad * 4;
        ov = o;   o += Cpad * 4;
        sv = o;   o += ring * Cpad * 4;
        mv = o;   o += ring * Cpad * 4;
        o = (o + 15u) & ~15u;
        cur = o;  o += 16;                                                  // evaluators' next item
        sc = o;   o += (16 + 2 * WALK_RING) * 4;
        o = (o + 15u) & ~15u;
        warp0 = o;
        warp_bytes = (uint32_t)W * 32 * K * 4 + 2 * STAGE_BYTES;
        total = o + nw * warp_bytes;
    }
};

// left/right combination keeping the operand order of the node
template <int K, int V>
__device__ __forceinline__ void combine(uint32_t op, bool path_left, float (&v)[K], const float (&sib)[K]) {
    if (path_left) apply_vec<K, V>(op, v, sib);
    else {
        float t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = sib[k];
        apply_vec<K, V>(op, t, v);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = t[k];
    }
}

// Evaluate bytes [s, e) of `src` (a small run: e - (s & ~15) <= STAGE_BYTES).
template <int K, int V>
__device__ __forceinline__ void eval_run(const uint8_t* src, uint32_t s, uint32_t e, uint8_t* stage,
                                         const Ictx<K>& c, float (&out)[K], uint32_t* status,
                                         const volatile uint32_t* stop = nullptr, bool* aborted = nullptr) {
    __syncwarp();
    stage_issue(stage, src, s, e);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    Istate<K> st;
#pragma unroll
    for (int k = 0; k < K; ++k) st.acc[k] = 0.f;
    st.sp = 0;
    st.ok = true;
    bool ab = false;
    interp_staged_lone<K, V>(stage, s, e, st, c, stop, &ab);
    if (ab) { if (aborted) *aborted = true; return; }
    if (!st.ok && lane_id() == 0) set_status(status, ST_STACK);
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = st.acc[k];
}

// Ancestors of the crossover point c in the child, for one warp: the
// deepest ancestor A that the mother caches, the small ancestors below it
// (positions anc[], balance offsets ancg[], nearest first) from a backward
// balance scan over at most T bytes before c, and the child ends of those
// levels (lvl[v] = end of the ancestor whose subtree closes at balance v)
// from a forward scan after the donated subtree.  Returns false on an
// inconsistency (recorded in the status word).
template <int K>
__device__ bool walk_ancestors(const DevPop& d, const CacheView& par, uint32_t i, const uint8_t* ok_, int32_t tdl,
                               uint32_t c,
                               uint32_t s, uint32_t nk, int32_t em, uint32_t me0, uint32_t me1, uint8_t* stB,
                               uint32_t* anc, int32_t* ancg, uint32_t* lvl, int32_t& A_out, uint32_t& nsmall_out,
                               int32_t& hneed_out) {
    const int lane = lane_id();
    const uint32_t T = d.T;
    int32_t A = -1;
    uint32_t nsmall = 0;
    if (em >= 0) A = par.e_par[em];
    else {
        int32_t e = find_last_lt(par.e_pos, me0, me1, c);
        uint32_t guard = 0;
        while (e >= 0 && par.e_end[e] <= c && guard++ < (1u << 24)) e = par.e_par[e];
        A = e;
        if (A < 0) { if (lane == 0) set_error(d, ST_STRUCT, 5, i, c, 0); return false; }
        // backward scan of (max(pos(A)+1, c-T+1) .. c-1]: G(j) = sum_{k=j}^{c-1} (arity_k - 1);
        // j is an ancestor of c iff G(j) >= G(m) for every m in (j, c], G(c) = 0
        const uint32_t pA = par.e_pos[A];
        const uint32_t lo = max(pA + 1, (c + 1 > T) ? c + 1 - T : 0u);
        if (lo < c) {
            __syncwarp();
            stage_issue(stB, ok_, lo, c);
            cp_async_commit();
            cp_async_wait<0>();
            __syncwarp();
            const uint32_t a16 = lo & ~15u;
            // lane l: positions c-1-32l-t, t = 0..31 (nearest first)
            int sum = 0, mx = -0x40000000;
            for (int t = 0; t < 32; ++t) {
                const int64_t j = (int64_t)c - 1 - 32 * lane - t;
                if (j >= (int64_t)lo) { sum += (stB[j - a16] < 4) ? 1 : -1; mx = max(mx, sum); }
            }
            // G offset from the lanes nearer to c, and the maximum G seen before this lane
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int ts = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += ts;
            }
            const int base = incl - sum;
            int pm = (mx > -0x40000000) ? base + mx : -0x40000000;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int tm = __shfl_up_sync(FULL, pm, o);
                if (lane >= o) pm = max(pm, tm);
            }
            int prevmax = __shfl_up_sync(FULL, pm, 1);
            if (lane == 0) prevmax = 0;            // G(c) = 0
            prevmax = max(prevmax, 0);
            uint32_t fmask = 0;
            int run = prevmax, gsum = base;
            for (int t = 0; t < 32; ++t) {
                const int64_t j = (int64_t)c - 1 - 32 * lane - t;
                if (j >= (int64_t)lo) {
                    gsum += (stB[j - a16] < 4) ? 1 : -1;
                    if (gsum >= run) { fmask |= 1u << t; run = gsum; }
                }
            }
            // compact in nearest-first order
            const uint32_t cnt = __popc(fmask);
            uint32_t off = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t tt = __shfl_up_sync(FULL, off, o);
                if (lane >= o) off += tt;
            }
            off -= cnt;
            const uint32_t tot = __shfl_sync(FULL, off + cnt, 31);
            if (tot > WALK_MAXLVL - 2) { if (lane == 0) set_status(d.status, ST_PATH); return false; }
            gsum = base;
            uint32_t k = off;
            for (int t = 0; t < 32; ++t) {
                const int64_t j = (int64_t)c - 1 - 32 * lane - t;
                if (j >= (int64_t)lo) {
                    gsum += (stB[j - a16] < 4) ? 1 : -1;
                    if (fmask & (1u << t)) {
                        anc[k] = (uint32_t)j;
                        // balance offset (>= 0 at an ancestor), operator byte in bits 24..
                        ancg[k] = (int32_t)((uint32_t)gsum | ((uint32_t)stB[j - a16] << 24));
                        ++k;
                    }
                }
            }
            nsmall = tot;
            __syncwarp();
        }
    }
    // ---- child ends of the small ancestors: forward scan after the donated subtree
    // balance relative to b[c] is 1 at c+s; lvl[v] = first position where it reaches v
    uint32_t maxv = 1;
    if (nsmall) maxv = (uint32_t)(ancg[nsmall - 1] & 0xFFFFFF) + 1;
    if (maxv >= WALK_MAXLVL) { if (lane == 0) set_status(d.status, ST_PATH); return false; }
    int32_t hneed = -1;
    if (nsmall) {
        const uint32_t f0 = c + s;
        const uint32_t f1 = f0 + T;
        // sentinel 0 for levels the scan does not reach: their sibling ranges then fail the
        // size check of the walk instead of reading a stale end
        for (uint32_t v = lane; v <= maxv; v += 32) lvl[v] = 0;
        __syncwarp();
        // child positions q >= c + s are bytes q - tdl of ok_
        const uint32_t lim = min(f1, (nk + 15u) & ~15u);
        if (f0 < lim) { stage_issue(stB, ok_, f0 - tdl, lim - tdl); }
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        const uint32_t a16 = ((f0 - tdl) & ~15u) + tdl;
        if (lane == 0) lvl[1] = f0;
        int sum = 0, mx = 0;
        // lane l: positions f0 + 32l + t
        for (int t = 0; t < 32; ++t) {
            const uint32_t q = f0 + 32 * lane + t;
            const int w = (q < nk && stB[q - a16] < 4) ? -1 : 1;
            sum += w;
            mx = max(mx, sum);
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { int ts = __shfl_up_sync(FULL, incl, o); if (lane >= o) incl += ts; }
        const int base = 1 + incl - sum;          // balance before the lane's first position
        int lmax = base + mx;                      // max after-balance in the lane (or base)
        lmax = max(lmax, base);
        int pm = lmax;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { int tm = __shfl_up_sync(FULL, pm, o); if (lane >= o) pm = max(pm, tm); }
        int prev = __shfl_up_sync(FULL, pm, 1);
        if (lane == 0) prev = 1;
        prev = max(prev, base);
        int bal = base;
        for (int t = 0; t < 32; ++t) {
            const uint32_t q = f0 + 32 * lane + t;
            bal += (q < nk && stB[q - a16] < 4) ? -1 : 1;
            if (bal > prev) { if ((uint32_t)bal < WALK_MAXLVL) lvl[bal] = q + 1; prev = bal; }
        }
        __syncwarp();
        // highest small ancestor that the child caches (needs a value even above the stop)
        for (uint32_t k = lane; k < nsmall; k += 32) {
            const uint32_t p = anc[k];
            const uint32_t pe = lvl[(ancg[k] & 0xFFFFFF) + 1];
            if (pe - p >= T) hneed = max(hneed, (int32_t)k);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hneed = max(hneed, __shfl_xor_sync(FULL, hneed, o));
    }
    A_out = A;
    nsmall_out = nsmall;
    hneed_out = hneed;
    return true;
}

// Disruption of one case between the child's value n and the mother's o:
// bit patterns differ (Boolean: each differing bit is a case); for finite
// pairs the squared difference, in binary64, joins the lane's sum.
template <int V>
__device__ __forceinline__ void dis_case(float n, float o, uint32_t& nd, uint32_t& nf, double& sq) {
    const uint32_t x = __float_as_uint(n) ^ __float_as_uint(o);
    if (V == VB) {
        nd += __popc(x);
    } else if (V == VI) {
        if (x) {
            ++nd;
            ++nf;
            const double df = (double)((long long)__float_as_int(n) - (long long)__float_as_int(o));
            sq = __dadd_rn(sq, __dmul_rn(df, df));
        }
    } else if (x) {
        ++nd;
        if (isfinite(n) && isfinite(o)) {
            ++nf;
            const double df = __dsub_rn((double)n, (double)o);
            sq = __dadd_rn(sq, __dmul_rn(df, df));
        }
    }
}

// Warp-collective: sum the lanes' counts and squares, lane 0 stores level
// `level` of child i (levels past the record's length are dropped).
template <int V>
__device__ __forceinline__ void dis_store(const GenBufs& g, uint32_t i, uint32_t level, uint32_t nd, uint32_t nf,
                                          double sq) {
    nd = __reduce_add_sync(FULL, nd);
    nf = __reduce_add_sync(FULL, nf);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq = __dadd_rn(sq, __shfl_xor_sync(FULL, sq, o));
    if (V == VB) { nf = nd; sq = (double)nd; }
    if (lane_id() == 0 && level < g.dis_L) {
        DisLevel r;
        r.nd = nd;
        r.nf = nf;
        r.sq = sq;
        g.dis[(size_t)i * g.dis_L + level] = r;
    }
}

// Bottom-up incremental evaluation of one child per team of nw warps
// (Sec. 6.2, Fig. 3).  Level 0 compares the donated subtree's value with
// the removed subtree's; each higher level combines the running values with
// the sibling's value (cached when its subtree is large, else interpreted)
// and compares the child's with the mother's.  The walk stops at the first
// level where the two agree on every case, bit for bit.  Ancestors below
// the threshold lie within T positions before the crossover point and are
// found by a backward balance scan; larger ones come from the mother's cache
// links.  The siblings' values do not depend on the path, so a team
// evaluates the siblings of several levels at once (one warp each, or one
// warp per case block), then combines them level by level and stops where
// the method stops; siblings computed past the stop are discarded.  New
// values of nodes that are cached in the child are recorded for the
// child's cache; above the stop only child-cached nodes that the mother
// does not cache need computing.
// Builder of the walk's level descriptors (one lane): the ancestors of the
// crossover point from the nearest up -- the small ones from the backward
// balance scan (anc, ancg, lvl), then the mother's cached ancestors through
// their parent links -- each with its sibling's range in the child and, for
// a large sibling, its cache entry.  `stopped` ends the building above the
// stop except for small ancestors that the child caches (they need values).

struct WalkBuilder {
    uint32_t bq, bqend, bk;
    int32_t bpe;
    bool btop;
};

struct WalkCtx {
    const uint8_t* ok_;        // child bytes before the crossover point (the mother's in fitness-first order)
    uint32_t nsmall, nk, s, r, T;
    int32_t A, hneed;
    const uint32_t* anc;
    const int32_t* ancg;
    const uint32_t* lvl;
};

// Build the next level into D; false (and btop set) when there is none.
// The walk's critical path on long paths runs through this builder, one
// dependent chain of cache-link loads per level: every field of a cached
// ancestor's entry is loaded at once (one round trip), then its operator
// byte and its large sibling's slot (a second one); a small ancestor's
// operator byte was kept by the backward scan (bits 24.. of ancg).
__device__ __forceinline__ bool build_level(const CacheView& par, const WalkCtx& w, WalkBuilder& b, bool stopped,
                                            LevelDesc& D) {
    if (b.btop) return false;
    uint32_t p, pend, op;
    int32_t pent, c0 = -1, c1 = -1, nextp = -1;
    uint32_t pslot = 0;
    if (b.bk < w.nsmall) {
        const int32_t gk = w.ancg[b.bk];
        p = w.anc[b.bk];
        pend = w.lvl[(gk & 0xFFFFFF) + 1];
        op = (uint32_t)gk >> 24;
        pent = -1;
    } else {
        pent = (b.bk == w.nsmall) ? w.A : b.bpe;
        if (pent < 0) { b.btop = true; return false; }                  // above the root
        p = __ldg(par.e_pos + pent);
        const uint32_t e = __ldg(par.e_end + pent);
        c0 = __ldg(par.e_c0 + pent);
        c1 = __ldg(par.e_c1 + pent);
        pslot = __ldg(par.e_slot + pent);
        nextp = __ldg(par.e_par + pent);
        pend = (uint32_t)((int64_t)e + ((int64_t)w.s - (int64_t)w.r));
        op = 0xFFFFFFFFu;
    }
    // above the stop only small ancestors that the child caches need values
    if (stopped && (pent >= 0 || (int32_t)b.bk > w.hneed)) { b.btop = true; return false; }
    const bool left = (b.bq == p + 1);
    const uint32_t ss = left ? b.bqend : p + 1;
    const uint32_t se = left ? pend : b.bq;
    int32_t sib = -1;
    uint32_t bad = 0;
    if (se <= ss || se > w.nk) bad = LD_BAD;
    else if (se - ss >= w.T) {
        sib = (pent < 0) ? -1 : (left ? c1 : c0);
        if (sib < 0) bad = LD_NOSIB;
    }
    if (op == 0xFFFFFFFFu) op = w.ok_[p];
    const uint32_t sslot = (sib >= 0) ? __ldg(par.e_slot + sib) : 0u;
    const uint32_t flg = op | (left ? LD_LEFT : 0u) | ((p == 0 || pend - p >= w.T) ? LD_CACHED : 0u) | bad;
    D.p = p; D.pend = pend; D.ss = ss; D.se = se; D.pent = pent; D.sib = sib; D.flags = flg;
    D.k = (int32_t)b.bk;
    D.pslot = pslot;
    D.sslot = sslot;
    D.pad0 = 0u; D.pad1 = 0u;
    if (bad) { b.btop = true; return true; }
    b.bq = p;
    b.bqend = pend;
    if (b.bk >= w.nsmall) b.bpe = nextp;
    ++b.bk;
    if (p == 0) b.btop = true;
    return true;
}

// The children one launch walks: entries [q_lo, q_hi) of the work order,
// taken through queue counter qctr; its warps use the interpreter overflow
// stacks from warp ovf_base on.
struct WalkRange {
    uint32_t q_lo, q_hi, qctr, ovf_base;
};

template <int K, int V, int MAXT>
__global__ void __launch_bounds__(MAXT, 512 / MAXT) k_walk(DevPop d, GenBufs g, CacheView par, uint32_t nw,
                                                           WalkRange wr) {
    if (halted(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t Cpad = d.Cpad, Cn = d.C, ncb = d.ncb, T = d.T;
    const TeamLayout<K> L((int)d.W, Cpad, nw);
    float* kc = reinterpret_cast<float*>(smem_raw + L.kc);
    uint32_t* anc = reinterpret_cast<uint32_t*>(smem_raw + L.anc);
    int32_t* ancg = reinterpret_cast<int32_t*>(smem_raw + L.ancg);
    uint32_t* lvl = reinterpret_cast<uint32_t*>(smem_raw + L.lvl);
    LevelDesc* desc = reinterpret_cast<LevelDesc*>(smem_raw + L.desc);
    float* nvs = reinterpret_cast<float*>(smem_raw + L.nv);
    float* ovs = reinterpret_cast<float*>(smem_raw + L.ov);
    float* svs = reinterpret_cast<float*>(smem_raw + L.sv);
    float* mvs = reinterpret_cast<float*>(smem_raw + L.mv);
    volatile uint32_t* sc = reinterpret_cast<volatile uint32_t*>(smem_raw + L.sc);
    const int lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5, tid = threadIdx.x;
    fill_kc(kc, d.consts);
    fill_kb(kc + 256);
    __syncthreads();
    unsigned char* wb = smem_raw + L.warp0 + warp * L.warp_bytes;
    Ictx<K> ic;
    ic.s = reinterpret_cast<float*>(wb);
    ic.W = (int)d.W;
    ic.maxd = (int)d.maxdepth;
    ic.kc = kc;
    ic.kb = kc + 256;
    ic.g = d.ovf + (size_t)(wr.ovf_base + blockIdx.x * nw + warp) * (d.maxdepth - d.W) * 32 * K;
    uint8_t* stA = wb + (size_t)d.W * 32 * K * 4;
    uint8_t* stB = stA + STAGE_BYTES;
    volatile uint32_t* dtag = sc + 16;                 // [WALK_RING] level + 1 whose descriptor is in the slot
    volatile uint32_t* vcnt = sc + 16 + WALK_RING;     // [WALK_RING] case blocks of the slot's sibling done
    unsigned long long* cur = reinterpret_cast<unsigned long long*>(smem_raw + L.cur);   // level << 32 | case block
    const uint32_t nev = nw - 1;                       // sibling evaluators (warps 1..nw-1)
    const uint32_t ring = walk_ring(Cpad);
    const uint32_t ahead = ring;                       // levels built ahead of the combination
    unsigned long long st_interp = 0, st_levels = 0, st_stopped = 0, st_pathops = 0;

    for (;;) {
        if (tid == 0) sc[0] = atomicAdd(&d.q[wr.qctr], 1u);
        __syncthreads();
        const uint32_t qi = wr.q_lo + sc[0];
        __syncthreads();
        if (qi >= wr.q_hi) break;
        const uint32_t i = g.order[qi];
        const uint32_t fl = g.flags[i];
        const uint32_t m = g.mother[i];
        // children evaluated in one pass (k_onepass_eval) are not walked
        if (g.onepass[i]) continue;
        if (tid == 0) {
            g.walkA[i] = -1; g.nins[i] = 0; g.pv_cnt[i] = 0;
            if (g.dis) g.dis_n[i] = 0;
        }
        if (fl & F_CLONE) {
            if (tid == 0) {
                d.fit[i] = g.pfit[m]; g.stop[i] = 0; g.plen[i] = 0; ++st_stopped;
                if (g.dis) {
                    DisLevel z;
                    z.nd = 0; z.nf = 0; z.sq = 0.0;
                    g.dis[(size_t)i * g.dis_L] = z;
                    g.dis_n[i] = 1;
                }
            }
            continue;
        }
        const uint32_t f = g.father[i], c = g.cpos[i], r = g.rsz[i], dd = g.dpos[i], s = g.ssz[i];
        const uint32_t nk = d.size[i];
        // child bytes: its own buffer, or (fitness-first mode, the child not built
        // yet) its mother's, where a position x >= c + s of the child is byte x - tdl
        const bool virt = g.lazy != 0;
        const uint8_t* ok_ = virt ? d.arena + (size_t)g.pbuf[m] * d.cap : d.arena + (size_t)d.buf[i] * d.cap;
        const int32_t tdl = virt ? (int32_t)s - (int32_t)r : 0;
        const uint32_t me0 = par.e_off[m], me1 = par.e_off[m + 1];
        const uint32_t fe0 = par.e_off[f], fe1 = par.e_off[f + 1];
        uint32_t npv = 0, nins_i = 0;

        // ---- level 0: donated subtree vs removed subtree
        int32_t ef = -1, em = -1;
        if (s >= T || dd == 0) {
            ef = find_exact(par.e_pos, fe0, fe1, dd);
            if (ef < 0) { if (tid == 0) set_error(d, ST_STRUCT, 3, i, dd, s); continue; }
        }
        if (r >= T || c == 0) {
            em = find_exact(par.e_pos, me0, me1, c);
            if (em < 0) { if (tid == 0) set_error(d, ST_STRUCT, 4, i, c, r); continue; }
        }
        // the donated subtree becomes the child's root (always cached) but the
        // father does not cache it: keep the value computed at level 0
        const bool root_rec = (c == 0 && s < T && dd != 0);
        uint32_t rslot = 0;
        if (root_rec) {
            if (tid == 0) sc[1] = atomicAdd(&g.misc[M_PV], 1u);
            __syncthreads();
            rslot = sc[1];
            __syncthreads();
            if (rslot >= g.pvcap) { if (tid == 0) set_status(d.status, ST_PATH); continue; }
        }
        // ---- level 0 (donated subtree vs removed subtree), ancestors, walk.
        // Neither the ancestors nor the siblings depend on the level-0 values,
        // so in a team of several warps the evaluators interpret the donated
        // and removed subtrees (up to T - 1 nodes each) while warp 0 finds the
        // ancestors and builds the first levels; warp 0 compares level 0 just
        // before it combines level 1.  A team of one does them in turn.
        if (tid < WALK_RING) { dtag[tid] = 0u; vcnt[tid] = 0u; }
        if (tid == 0) { *cur = 0ull; sc[8] = 0u; sc[6] = 0u; sc[4] = 0u; }
        __syncthreads();
        auto level0 = [&](uint32_t first, uint32_t step) {
            for (uint32_t it = first; it < 2 * ncb; it += step) {
                const uint32_t which = it & 1u, cb = it >> 1;
                load_cases<K>(d, cb, ic.xv);
                float v[K];
                if (which == 0) {
                    if (ef >= 0) load_vec<K>(par.slots, Cpad, par.e_slot[ef], v, cb);
                    else {
                        if (virt) eval_run<K, V>(d.arena + (size_t)g.pbuf[f] * d.cap, dd, dd + s, stA, ic, v, d.status);
                        else eval_run<K, V>(ok_, c, c + s, stA, ic, v, d.status);
                        if (cb == 0) st_interp += s;
                    }
                } else {
                    if (em >= 0) load_vec<K>(par.slots, Cpad, par.e_slot[em], v, cb);
                    else {
                        eval_run<K, V>(g.stash + g.stash_off[i], 0, r, stA, ic, v, d.status);
                        if (cb == 0) st_interp += r;
                    }
                }
                store_blk<K>(which == 0 ? nvs : ovs, cb, v);
            }
        };
        if (nev == 0) level0(0, 1);
        else if (warp >= 1) {
            level0(warp - 1, nev);
            __threadfence_block();
            __syncwarp();
            if (lane == 0) atomicAdd(const_cast<uint32_t*>(&sc[6]), 1u);
        }
        bool stopped = false;
        int32_t stop_level = -1;
        bool stopped_w = false;
        int32_t stop_level_w = -1;
        uint32_t levels_w = 0;
        if (warp == 0) {
            // ---- ancestors
            int32_t A = -1, hneed = -1;
            uint32_t nsmall = 0;
            const bool anc_ok = walk_ancestors<K>(d, par, i, ok_, tdl, c, s, nk, em, me0, me1, stB, anc, ancg, lvl, A,
                                                  nsmall, hneed);
            // level 0 compared once every level-0 item is in (bounded wait)
            bool l0done = false, fail = false;
            auto finish_level0 = [&]() {
                if (l0done) return;
                l0done = true;
                if (nev) {
                    uint32_t spins = 0, got = 0;
                    while ((got = __shfl_sync(FULL, lane == 0 ? sc[6] : 0u, 0)) < nev && ++spins < d.wait_polls)
                        __nanosleep(64);
                    if (got < nev) { if (lane == 0) set_status(d.status, ST_TIMEOUT); fail = true; return; }
                    __threadfence_block();
                }
                bool okc = true;
                for (uint32_t j = lane; j < Cn; j += 32)
                    if (__float_as_uint(nvs[j]) != __float_as_uint(ovs[j])) okc = false;
                stopped = __all_sync(FULL, okc);
                stop_level = stopped ? 0 : -1;
                stopped_w = stopped;
                stop_level_w = stop_level;
                if (root_rec) {
                    float* dst = g.pv_val + (size_t)rslot * Cpad;
                    for (uint32_t j = lane; j < Cpad; j += 32) dst[j] = nvs[j];
                    if (lane == 0) {
                        g.pv_rec[rslot] = make_uint4(i, npv, 0u, rslot | 0x80000000u);
                        g.pv_end[rslot] = s;
                        g.rec_entry[rslot] = 0xFFFFFFFFu;
                    }
                    ++npv;
                    ++nins_i;
                }
                if (g.dis) {                               // level 0 of the disruption record
                    uint32_t nd = 0, nf = 0;
                    double sq = 0.0;
                    for (uint32_t j = lane; j < Cn; j += 32) dis_case<V>(nvs[j], ovs[j], nd, nf, sq);
                    dis_store<V>(g, i, 0, nd, nf, sq);
                }
            };
            if (!anc_ok) { fail = true; if (lane == 0) sc[4] = 1u; }
            WalkBuilder b;                                 // builder state (lane 0)
            b.bq = c; b.bqend = c + s; b.bk = 0; b.bpe = (nsmall > 0) ? -1 : A; b.btop = false;
            const WalkCtx wc{ok_, nsmall, nk, s, r, T, A, hneed, anc, ancg, lvl};
            bool btop = false;
            uint32_t nb = 0, ncm = 0, level = 0;           // levels built, levels combined
            uint32_t rbase = 0, rleft = 0;                 // this child's reserved record slots
            uint32_t guard = 0;
            if (lane == 0) sc[3] = (uint32_t)A;
            while (!fail && guard++ < (1u << 24)) {
                // combine the next level as soon as its sibling values are in;
                // until then build one more level (the builder's chain of loads
                // overlaps the evaluators' work instead of delaying the combining)
                bool ready = false;
                if (ncm < nb) ready = nev == 0 || __shfl_sync(FULL, lane == 0 ? vcnt[ncm % ring] : 0u, 0) >= ncb;
                if (!ready) {
                    uint32_t built = 0;
                    if (lane == 0 && !b.btop && nb < ncm + ahead) {
                        LevelDesc& D = desc[nb % ring];
                        if (build_level(par, wc, b, stopped_w, D)) {
                            __threadfence_block();
                            dtag[nb % ring] = nb + 1;
                            ++nb;
                            built = 1;
                            if (D.flags & (LD_BAD | LD_NOSIB)) b.btop = true;
                        }
                    }
                    if (lane == 0) btop = b.btop;
                    __syncwarp();
                    nb = __shfl_sync(FULL, nb, 0);
                    btop = __shfl_sync(FULL, btop ? 1u : 0u, 0) != 0;
                    if (__shfl_sync(FULL, built, 0)) continue;
                    if (ncm == nb) {
                        if (btop) break;                                       // nothing left to combine
                        continue;
                    }
                }
                finish_level0();
                if (fail) break;
                const uint32_t slot = ncm % ring;
                LevelDesc D = desc[slot];
                if (stopped_w && (D.pent >= 0 || D.k > hneed)) break;
                // the level's sibling values: from the evaluators, or computed here in a team of one
                if (nev == 0) {
                    if (!(D.flags & (LD_BAD | LD_NOSIB))) {
                        for (uint32_t cb = 0; cb < ncb; ++cb) {
                            float v[K];
                            if (!stopped_w && D.pent >= 0) {
                                load_vec<K>(par.slots, Cpad, D.pslot, v, cb);
                                store_blk<K>(mvs + slot * Cpad, cb, v);
                            }
                            if (D.sib >= 0) load_vec<K>(par.slots, Cpad, D.sslot, v, cb);
                            else {
                                load_cases<K>(d, cb, ic.xv);
                                const uint32_t sh = (D.flags & LD_LEFT) ? (uint32_t)tdl : 0u;
                                eval_run<K, V>(ok_, D.ss - sh, D.se - sh, stA, ic, v, d.status);
                                if (cb == 0) st_interp += D.se - D.ss;
                            }
                            store_blk<K>(svs + slot * Cpad, cb, v);
                        }
                    }
                } else {
                    uint32_t spins = 0, ready = 0;
                    while ((ready = __shfl_sync(FULL, lane == 0 ? vcnt[slot] : 0u, 0)) < ncb && ++spins < d.wait_polls)
                        __nanosleep(64);
                    if (ready < ncb) { if (lane == 0) set_status(d.status, ST_TIMEOUT); fail = true; break; }
                    __threadfence_block();
                }
                __syncwarp();
                ++level;
                if (D.flags & (LD_BAD | LD_NOSIB)) {
                    if (lane == 0) set_error(d, ST_STRUCT, (D.flags & LD_BAD) ? 6 : 7, i, D.p, D.se - D.ss);
                    fail = true;
                    break;
                }
                const uint32_t op = D.flags & 0xFFu;
                const bool left = (D.flags & LD_LEFT) != 0;
                const float* svl = svs + slot * Cpad;
                const float* pvv = mvs + slot * Cpad;
                bool okl = true;
                uint32_t dnd = 0, dnf = 0;
                double dsq = 0.0;
                for (uint32_t j = lane; j < Cpad; j += 32) {
                    float o[1] = {ovs[j]};
                    const float sv1[1] = {svl[j]};
                    combine<1, V>(op, left, o, sv1);         // mother's value at p (exact recomputation)
                    if (!stopped_w) {
                        float n1[1] = {nvs[j]};
                        combine<1, V>(op, left, n1, sv1);
                        nvs[j] = n1[0];
                        if (D.pent >= 0) o[0] = pvv[j];
                        if (j < Cn && __float_as_uint(n1[0]) != __float_as_uint(o[0])) okl = false;
                        if (g.dis && j < Cn) dis_case<V>(n1[0], o[0], dnd, dnf, dsq);
                    }
                    ovs[j] = o[0];
                }
                const bool lvl_eq = __all_sync(FULL, okl);
                if (g.dis && !stopped_w) dis_store<V>(g, i, level, dnd, dnf, dsq);
                __syncwarp();
                if (!stopped_w) {
                    ++levels_w;
                    ++st_pathops;
                    if (lvl_eq) { stopped_w = true; stop_level_w = (int32_t)level; }
                }
                // record the child's value here when the child caches this node and the mother's
                // cache cannot supply it (disrupted, or not cached in the mother); above the
                // stop only small ancestors (pent < 0) get here
                if ((D.flags & LD_CACHED) && (!lvl_eq || D.pent < 0)) {
                    if (rleft == 0) {
                        uint32_t b0 = 0;
                        if (lane == 0) b0 = atomicAdd(&g.misc[M_PV], 8u);
                        rbase = __shfl_sync(FULL, b0, 0);
                        rleft = 8;
                    }
                    const uint32_t rs = rbase++;
                    --rleft;
                    if (rs >= g.pvcap) { if (lane == 0) set_status(d.status, ST_PATH); fail = true; break; }
                    const float* src = stopped_w ? ovs : nvs;
                    float* dst = g.pv_val + (size_t)rs * Cpad;
                    for (uint32_t j = lane; j < Cpad; j += 32) dst[j] = src[j];
                    if (lane == 0) {
                        g.pv_rec[rs] = make_uint4(i, npv, D.p, rs | (D.pent < 0 ? 0x80000000u : 0u));
                        g.rec_entry[rs] = 0xFFFFFFFFu;
                        g.pv_end[rs] = D.pend;
                    }
                    ++npv;
                    if (D.pent < 0) ++nins_i;
                }
                // release the slot to the builder
                if (lane == 0) vcnt[slot] = 0u;
                __syncwarp();
                ++ncm;
                if (D.p == 0) break;
            }
            // reserved record slots left unused are marked as holes
            for (uint32_t k = lane; k < rleft; k += 32)
                if (rbase + k < g.pvcap) {
                    g.pv_rec[rbase + k] = make_uint4(0xFFFFFFFFu, 0u, 0u, 0u);
                    g.rec_entry[rbase + k] = 0xFFFFFFFFu;
                }
            // a walk without levels (the child's root is the donated subtree, or
            // the ancestors failed) still compares level 0
            if (anc_ok && !fail) finish_level0();
            if (fail && lane == 0) sc[4] = 1u;
            __threadfence_block();
            if (lane == 0) sc[8] = 1u;                      // evaluators stop
        } else {
            // evaluators: each takes the next (level, case block) item in level order from a
            // shared cursor once the level's descriptor is built, so a long sibling holds up
            // only the warp evaluating it
            for (;;) {
                uint32_t k = 0, r = 0, fin = 0;
                if (lane == 0) {
                    uint32_t spins = 0;
                    for (;;) {
                        if (sc[8]) { fin = 1; break; }                  // the combination is over
                        const unsigned long long c = *reinterpret_cast<volatile unsigned long long*>(cur);
                        const uint32_t ck = (uint32_t)(c >> 32), cr = (uint32_t)c;
                        const uint32_t cs = ck % ring;
                        if (dtag[cs] == ck + 1) {
                            __threadfence_block();
                            const unsigned long long nx = (cr + 1 < ncb) ? c + 1 : ((unsigned long long)(ck + 1) << 32);
                            if (atomicCAS(cur, c, nx) == c) { k = ck; r = cr; break; }
                            continue;
                        }
                        if (++spins >= d.wait_polls) { set_status(d.status, ST_TIMEOUT); fin = 1; break; }
                        __nanosleep(64);
                    }
                }
                if (__shfl_sync(FULL, fin, 0)) break;
                k = __shfl_sync(FULL, k, 0);
                r = __shfl_sync(FULL, r, 0);
                const uint32_t cb = r;
                const uint32_t slot = k % ring;
                __threadfence_block();
                const LevelDesc D = desc[slot];
                if (!(D.flags & (LD_BAD | LD_NOSIB))) {
                    float v[K];
                    if (D.pent >= 0) {
                        load_vec<K>(par.slots, Cpad, D.pslot, v, cb);
                        store_blk<K>(mvs + slot * Cpad, cb, v);
                    }
                    bool ab = false;
                    if (D.sib >= 0) load_vec<K>(par.slots, Cpad, D.sslot, v, cb);
                    else {
                        load_cases<K>(d, cb, ic.xv);
                        const uint32_t sh = (D.flags & LD_LEFT) ? (uint32_t)tdl : 0u;
                        // abandoned once the combination is over (the walk stopped below this level)
                        eval_run<K, V>(ok_, D.ss - sh, D.se - sh, stA, ic, v, d.status, sc + 8, &ab);
                        if (cb == 0 && !ab) st_interp += D.se - D.ss;
                    }
                    if (ab) break;
                    store_blk<K>(svs + slot * Cpad, cb, v);
                }
                __threadfence_block();
                __syncwarp();
                if (lane == 0) atomicAdd(const_cast<uint32_t*>(&vcnt[slot]), 1u);
            }
        }
        __syncthreads();
        // the combiner's results, from warp 0 to the team
        if (tid == 0) { sc[9] = stopped_w ? 1u : 0u; sc[10] = (uint32_t)stop_level_w; sc[11] = levels_w; sc[12] = npv; sc[13] = nins_i; }
        __syncthreads();
        const bool walk_failed = sc[4] != 0;
        stopped = sc[9] != 0;
        stop_level = (int32_t)sc[10];
        const uint32_t levels = sc[11];
        const int32_t A = (int32_t)sc[3];
        npv = sc[12];
        nins_i = sc[13];
        if (walk_failed) {                   // an inconsistency was recorded; the next synchronising call reports it
            __syncthreads();
            continue;
        }
        // ---- fitness
        if (tid == 0) {
            g.stop[i] = stop_level;
            g.plen[i] = levels;
            if (g.dis) g.dis_n[i] = min(levels + 1, g.dis_L);
            g.pv_cnt[i] = npv;
            g.nins[i] = nins_i;
            g.walkA[i] = A;
            if (stopped) {
                d.fit[i] = g.pfit[m];
                ++st_stopped;
            } else {
                d.fit[i] = fitness_of(d, [&](uint32_t j) { return nvs[j]; });
            }
            st_levels += levels;
        }
        __syncthreads();                     // nvs and the shared words are reused by the next child
    }
    if (lane == 0) atomicAdd(&g.gstat[G_INTERP], st_interp);
    if (tid == 0) {
        atomicAdd(&g.gstat[G_LEVELS], st_levels);
        atomicAdd(&g.gstat[G_STOPPED], st_stopped);
        atomicAdd(&g.gstat[G_PATHOPS], st_pathops);
    }
}

// ---- one-pass evaluation of children of at most ONEPASS_MAX nodes.
//
// The walk's cost per level (finding the ancestor, its sibling, waiting for
// the sibling's value) pays off when the tree is large and the walk stops
// early; on a child of a few thousand nodes whose crossover point lies deep
// (a uniform random binary tree of n nodes has paths of order sqrt(n)
// levels) interpreting the whole child once costs less and gives the same
// values bit for bit, since every node is evaluated from the same operands
// in the same order (Sec. 6.2: incremental evaluation only skips work, it
// never changes a value).  The child's cache then needs new values only at
// the ancestors of the crossover point that the child caches (subtree of at
// least T nodes, or the root): every other cached node keeps the value of
// its mother's or father's entry.
//
// k_onepass_plan (a warp per child) finds those ancestors from the balance
// S(q) = sum over k < q of (arity_k - 1) of the child's bytes: p < c is an
// ancestor of c iff S never falls below S(p) on (p, c]; its subtree ends at
// the first q > c where S reaches S(p) - 1.  It reserves one walk record per
// cached ancestor (and one for a new root made of a small donated subtree),
// (the deepest stack of the right-to-left scan is max S + 1 <= n / 2 + 1
// entries: the one-pass warps have overflow stacks that deep of their own,
// so they run beside the walk).  k_onepass_eval (a warp per child
// and case block, CTAs of 4 warps) interprets the child a piece of
// OP_CHUNK bytes at a time and writes each recorded ancestor's values as
// the scan passes it; the
// warp that completes a child's last case block writes its fitness.  Which
// children take this path is decided at crossover (size at most
// onepass_max, not a clone); the walk skips them.  Disruption recording
// walks every child.
#define ONEPASS_MAX 4096                 // most nodes of a child evaluated in one pass
#define OP_BUCKETS 13                    // size buckets floor(log2(n)), n <= 4096
#define ONEPASS_DEPTH (ONEPASS_MAX / 2 + 4)   // overflow stack entries per one-pass warp
#define ONEPASS_WARPS 4                  // warps per CTA of the plan kernel
#define OP_STAGE (2 * STAGE_BYTES)       // staged bytes per warp of the plan kernel (a whole child)
#define OP_EVAL_WARPS 4                  // warps per CTA of k_onepass_eval
#define OP_CHUNK 1024                    // bytes of a child staged at a time by k_onepass_eval
#define OP_CTAS_PER_SM 6                 // at most this many k_onepass_eval CTAs per SM (24 warps)

// Shared memory of a k_onepass_eval CTA: the constant and Boolean-input
// tables, then per warp a staged piece of the child (OP_CHUNK bytes, at
// least four stack entries so that a malformed run's underflow stays in the
// warp's own region) followed by its stack window.  Staging the child a
// piece at a time (instead of whole) leaves room for more warps per SM.
template <int K>
struct OnePassEvalLayout {
    static constexpr size_t stage_bytes = (OP_CHUNK > 4 * 32 * K * 4) ? OP_CHUNK : 4 * 32 * K * 4;
    __host__ __device__ static size_t warp_bytes(int W) { return stage_bytes + SmemLayout<K>::stack_bytes(W); }
    __host__ __device__ static size_t total(int W) { return SmemLayout<K>::kc_bytes + OP_EVAL_WARPS * warp_bytes(W); }
};

struct OnePassSmem {
    uint8_t stage[ONEPASS_WARPS][OP_STAGE];
    int16_t S[ONEPASS_WARPS][ONEPASS_MAX + 8];     // balance before position q, then prefix minima after c
    uint16_t anc[ONEPASS_WARPS][ONEPASS_MAX / 2 + 8];   // ancestors of c (function nodes), nearest first
};

// Assemble bytes [lo, hi) of child i (lo a multiple of 16, hi - lo <=
// OP_CHUNK) in `stage` (warp-collective), as stage_child below does for
// the whole child.
__device__ __forceinline__ void stage_child_piece(const DevPop& d, const GenBufs& g, uint32_t i, uint32_t nk,
                                                  uint32_t lo, uint32_t hi, uint8_t* stage) {
    const int lane = lane_id();
    __syncwarp();
    if (g.lazy) {
        const uint32_t m = g.mother[i];
        const uint8_t* mb = d.arena + (size_t)g.pbuf[m] * d.cap;
        const bool clone = (g.flags[i] & F_CLONE) != 0;
        const uint32_t c = clone ? nk : g.cpos[i], r = clone ? 0 : g.rsz[i], s = clone ? 0 : g.ssz[i];
        const uint8_t* fr = g.frag + (clone ? 0 : g.frag_off[i]);
        const uint32_t q0 = lo / 16, q1 = (hi + 15) / 16;
        for (uint32_t q = q0 + lane; q < q1; q += 32)
            reinterpret_cast<uint4*>(stage)[q - q0] = child_quad(mb, fr, 16 * q, c, r, s, nk);
    } else {
        stage_issue(stage, d.arena + (size_t)d.buf[i] * d.cap, lo, hi);
        cp_async_commit();
        cp_async_wait<0>();
    }
    __syncwarp();
}

// Assemble child i's bytes [0, nk) in `stage` (warp-collective): from its
// three pieces in fitness-first order -- the mother's head, the donated
// subtree (gathered into the fragment pool at crossover), the mother's tail
// -- 16 destination bytes per lane at a time (the copy kernel's quads),
// else from its own buffer.
__device__ __forceinline__ void stage_child(const DevPop& d, const GenBufs& g, uint32_t i, uint32_t nk, uint8_t* stage) {
    const int lane = lane_id();
    __syncwarp();
    if (g.lazy) {
        const uint32_t m = g.mother[i];
        const uint8_t* mb = d.arena + (size_t)g.pbuf[m] * d.cap;
        const bool clone = (g.flags[i] & F_CLONE) != 0;
        const uint32_t c = clone ? nk : g.cpos[i], r = clone ? 0 : g.rsz[i], s = clone ? 0 : g.ssz[i];
        const uint8_t* fr = g.frag + (clone ? 0 : g.frag_off[i]);
        for (uint32_t q = lane; q < (nk + 15) / 16; q += 32)
            reinterpret_cast<uint4*>(stage)[q] = child_quad(mb, fr, 16 * q, c, r, s, nk);
    } else {
        stage_issue(stage, d.arena + (size_t)d.buf[i] * d.cap, 0, nk);
        cp_async_commit();
        cp_async_wait<0>();
    }
    __syncwarp();
}

__global__ void __launch_bounds__(ONEPASS_WARPS * 32) k_onepass_plan(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OnePassSmem& sm = *reinterpret_cast<OnePassSmem*>(smem_raw);
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    uint8_t* stage = sm.stage[warp];
    int16_t* S = sm.S[warp];
    uint16_t* anc = sm.anc[warp];
    const uint32_t T = d.T;
    const uint32_t gw = blockIdx.x * ONEPASS_WARPS + warp, nwp = gridDim.x * ONEPASS_WARPS;
    for (uint32_t i = gw; i < d.P; i += nwp) {
        if (!g.onepass[i]) continue;                      // decided at crossover (uniform per warp)
        const uint32_t nk = d.size[i];
        stage_child(d, g, i, nk, stage);
        const uint32_t c = g.cpos[i], s = g.ssz[i], dd = g.dpos[i], m = g.mother[i];
        // S(q) for q in [0, nk]: lane l sums its chunk [l L, l L + L)
        const uint32_t L = (nk + 31) / 32;
        const uint32_t q0 = min(nk, lane * L), q1 = min(nk, q0 + L);
        int tot = 0;
        for (uint32_t q = q0; q < q1; ++q) tot += (stage[q] < 4) ? 1 : -1;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { const int v = __shfl_up_sync(FULL, incl, o); if (lane >= o) incl += v; }
        int run = incl - tot, mx = run;
        for (uint32_t q = q0; q < q1; ++q) { S[q] = (int16_t)run; run += (stage[q] < 4) ? 1 : -1; mx = max(mx, run); }
        if (lane == 31) S[nk] = (int16_t)run;            // -1 for a complete tree
        __syncwarp();
        // ancestors of c: p < c with min over (p, c] of S >= S(p); lane l's chunk, nearest first
        uint32_t na = 0;
        if (c > 0) {
            const uint32_t e1 = min(q1, c);                 // the lane's positions p < e1
            // minimum of S over (q0, e1] (the lane's part of every later p's range), then over the later lanes
            int cm = 0x7FFF;
            for (uint32_t q = q0 + 1; q <= e1 && q0 < e1; ++q) cm = min(cm, (int)S[q]);
            int later = cm;                                   // suffix minimum over lanes > l
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) { const int v = __shfl_down_sync(FULL, later, o); if (lane + o < 32) later = min(later, v); }
            later = __shfl_down_sync(FULL, later, 1);
            if (lane == 31) later = 0x7FFF;
            // count, then list nearest first (the nearest ancestors are in the highest lanes)
            uint32_t cnt = 0;
            int R = 0x7FFF;
            for (int32_t p = (int32_t)e1 - 1; p >= (int32_t)q0; --p) {
                R = min(R, (int)S[p + 1]);
                if (min(R, later) >= (int)S[p]) ++cnt;
            }
            uint32_t after = cnt;                             // ancestors in lanes > l
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) { const uint32_t v = __shfl_down_sync(FULL, after, o); if (lane + o < 32) after += v; }
            na = __shfl_sync(FULL, after, 0);
            after -= cnt;
            uint32_t k = after;
            R = 0x7FFF;
            for (int32_t p = (int32_t)e1 - 1; p >= (int32_t)q0; --p) {
                R = min(R, (int)S[p + 1]);
                if (min(R, later) >= (int)S[p]) anc[k++] = (uint16_t)p;
            }
        }
        __syncwarp();
        // prefix minima of S after c, in place: PM(q) = min over (c, q] of S
        if (c + 1 <= nk) {
            const uint32_t span = nk - c, L2 = (span + 31) / 32;
            const uint32_t r0 = c + 1 + min(span, lane * L2), r1 = c + 1 + min(span, lane * L2 + L2);
            int lm = 0x7FFF;
            for (uint32_t q = r0; q < r1; ++q) lm = min(lm, (int)S[q]);
            int pre = lm;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) { const int v = __shfl_up_sync(FULL, pre, o); if (lane >= o) pre = min(pre, v); }
            int cur = __shfl_up_sync(FULL, pre, 1);
            if (lane == 0) cur = 0x7FFF;
            __syncwarp();
            for (uint32_t q = r0; q < r1; ++q) { cur = min(cur, (int)S[q]); S[q] = (int16_t)cur; }
        }
        __syncwarp();
        // per ancestor (nearest first): its end, whether the child caches it, whether the mother does
        const uint32_t me0 = par.e_off[m], me1 = par.e_off[m + 1];
        uint32_t ncached = 0;
        for (uint32_t base = 0; base < na; base += 32) {
            const uint32_t k = base + lane;
            bool cached = false;
            if (k < na) {
                const uint32_t p = anc[k];
                const int target = (int)S[p] - 1;            // S(p) is untouched (p < c)
                // first q in (c, nk] with PM(q) <= target (PM is non-increasing; PM(nk) = -1)
                uint32_t lo = c + 1, hi = nk;
                while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if ((int)S[mid] <= target) hi = mid; else lo = mid + 1; }
                cached = (p == 0) || (lo - p >= T);
            }
            const uint32_t bal = __ballot_sync(FULL, cached);
            ncached += __popc(bal);
        }
        const bool rootrec = (c == 0) && (s < T) && (dd != 0);   // a new root made of a small donated subtree
        const uint32_t R = ncached + (rootrec ? 1u : 0u);
        uint32_t base = 0;
        if (lane == 0 && R) base = atomicAdd(&g.misc[M_PV], R);
        base = __shfl_sync(FULL, base, 0);
        if (R && base + R > g.pvcap) {
            if (lane == 0) { set_status(d.status, ST_PATH); g.pv_cnt[i] = 0u; g.nins[i] = 0u; g.op_base[i] = 0u; }
            continue;
        }
        // the records, nearest ancestor first (positions decreasing: the walk's order)
        uint32_t nins = 0, done = 0;
        for (uint32_t b0 = 0; b0 < na; b0 += 32) {
            const uint32_t k = b0 + lane;
            bool cached = false;
            uint32_t p = 0, e = 0;
            if (k < na) {
                p = anc[k];
                const int target = (int)S[p] - 1;
                uint32_t lo = c + 1, hi = nk;
                while (lo < hi) { const uint32_t mid = (lo + hi) >> 1; if ((int)S[mid] <= target) hi = mid; else lo = mid + 1; }
                e = lo;
                cached = (p == 0) || (e - p >= T);
            }
            const uint32_t bal = __ballot_sync(FULL, cached);
            if (cached) {
                const uint32_t slot = base + done + __popc(bal & ((1u << lane) - 1u));
                const bool ins = find_exact(par.e_pos, me0, me1, p) < 0;
                g.pv_rec[slot] = make_uint4(i, slot - base, p, slot | (ins ? 0x80000000u : 0u));
                g.pv_end[slot] = e;
                g.rec_entry[slot] = 0xFFFFFFFFu;
                nins += ins ? 1u : 0u;
            }
            done += __popc(bal);
        }
        nins = __reduce_add_sync(FULL, nins);
        if (lane == 0) {
            if (rootrec) {
                const uint32_t slot = base + ncached;
                g.pv_rec[slot] = make_uint4(i, ncached, 0u, slot | 0x80000000u);
                g.pv_end[slot] = nk;
                g.rec_entry[slot] = 0xFFFFFFFFu;
                ++nins;
            }
            g.op_base[i] = base;
            const uint32_t bk = 31u - __clz(nk);                  // floor(log2 nk) <= 12
            g.op_bucket[(size_t)bk * d.P + atomicAdd(&g.op_cnt[bk], 1u)] = i;
            g.pv_cnt[i] = R;
            g.nins[i] = nins;
            g.walkA[i] = -1;
            g.stop[i] = -2;                 // evaluated in one pass, no walk
            g.plen[i] = 0;
        }
    }
}

template <int K, int V>
__global__ void __launch_bounds__(OP_EVAL_WARPS * 32, 1) k_onepass_eval(DevPop d, GenBufs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // CTAs beyond one warp per unit leave at once (most generations of large
    // trees have few children this small); one thread decides for the CTA
    __shared__ uint32_t s_units;
    if (threadIdx.x == 0) {
        uint32_t n = 0;
        for (int b = 0; b < OP_BUCKETS; ++b) n += __ldcg(&g.op_cnt[b]);
        s_units = halted(d) ? 0u : n * d.ncb;
    }
    __syncthreads();
    if ((unsigned long long)blockIdx.x * OP_EVAL_WARPS >= s_units) return;
    float* kc = reinterpret_cast<float*>(smem_raw);
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    fill_kc(kc, d.consts);
    fill_kb(kc + 256);
    __syncthreads();
    uint8_t* const stage = smem_raw + SmemLayout<K>::kc_bytes + (size_t)warp * OnePassEvalLayout<K>::warp_bytes((int)d.W);
    Ictx<K> ic;
    ic.s = reinterpret_cast<float*>(stage + OnePassEvalLayout<K>::stage_bytes);
    ic.W = (int)d.W;
    ic.kc = kc;
    ic.kb = kc + 256;
    const uint32_t gwarp = blockIdx.x * OP_EVAL_WARPS + warp;
    // a child of at most ONEPASS_MAX nodes needs at most ONEPASS_MAX / 2 + 1 stack entries
    ic.maxd = (int)d.W + ONEPASS_DEPTH;
    ic.g = g.ovf_op + (size_t)gwarp * ONEPASS_DEPTH * 32 * K;
    const uint32_t ncb = d.ncb, Cpad = d.Cpad;
    unsigned long long st_interp = 0;
    // units (child, case block) from the largest size bucket down: the longest
    // interpretations start first and the short ones fill in behind them
    int bk = OP_BUCKETS - 1;
    for (;;) {
        uint32_t i = 0, cb = 0, got = 0;
        if (lane == 0) {
            while (bk >= 0) {
                const uint32_t nu = __ldcg(&g.op_cnt[bk]) * ncb;
                if (nu) {
                    const uint32_t u = atomicAdd(&g.op_cnt[OP_BUCKETS + bk], 1u);
                    if (u < nu) { i = g.op_bucket[(size_t)bk * d.P + u / ncb]; cb = u % ncb; got = 1; break; }
                }
                --bk;
            }
        }
        if (!__shfl_sync(FULL, got, 0)) break;
        i = __shfl_sync(FULL, i, 0);
        cb = __shfl_sync(FULL, cb, 0);
        const uint32_t nk = d.size[i];
        load_cases<K>(d, cb, ic.xv);
        Istate<K> st;
#pragma unroll
        for (int k = 0; k < K; ++k) st.acc[k] = 0.f;
        st.sp = 0;
        st.ok = true;
        const uint32_t base = g.op_base[i], R = g.pv_cnt[i];
        auto pos = [&](uint32_t k) { return g.pv_rec[base + k].z; };
        auto cap = [&](uint32_t k) { store_blk<K>(g.pv_val + (size_t)(base + k) * Cpad, cb, st.acc); };
        CaptureCursor cur{0u, R ? (int32_t)pos(0) : -1};
        bool under = false;
        // the child a piece at a time, right to left (pieces end on multiples of OP_CHUNK)
        for (uint32_t hi = nk; hi > 0;) {
            const uint32_t lo = (hi - 1) & ~(uint32_t)(OP_CHUNK - 1);
            stage_child_piece(d, g, i, nk, lo, hi, stage);
            interp_capture_range<K, V>(stage, lo, hi, st, ic, R, cur, under, pos, cap);
            hi = lo;
        }
        if (under || st.sp != 1) st.ok = false;
        if (!st.ok && lane == 0) set_status(d.status, ST_STACK);
        float* row = g.small_val + (size_t)i * Cpad;
        store_blk<K>(row, cb, st.acc);
        if (cb == 0) st_interp += nk;
        // the warp that completes the child's last case block writes its fitness
        __threadfence();
        __syncwarp();
        uint32_t last = 0;
        if (lane == 0) last = (atomicAdd(&g.small_cnt[i], 1u) == ncb - 1) ? 1u : 0u;
        if (!__shfl_sync(FULL, last, 0)) continue;
        __threadfence();
        const float fv = fitness_warp(d, [&](uint32_t j) { return __ldcg(row + j); });
        if (lane == 0) d.fit[i] = fv;
    }
    if (lane == 0 && st_interp) atomicAdd(&g.gstat[G_INTERP], st_interp);
}

// ------------------------------------------------------------------ A9 child cache

// Walk records grouped per child in walk order (positions decreasing).
__global__ void __launch_bounds__(1024) k_pv_offsets(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < d.P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = (i < d.P) ? g.pv_cnt[i] : 0;
        const uint64_t o = block_excl_scan(v, ws, &carry);
        if (i < d.P) g.pv_off[i] = (uint32_t)o;
    }
    __syncthreads();
    if (threadIdx.x == 0) g.pv_off[d.P] = (uint32_t)carry;
}

__global__ void k_pv_scatter(DevPop d, GenBufs g) {
    if (halted(d)) return;
    const uint32_t n = min(g.misc[M_PV], g.pvcap);
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint4 rec = g.pv_rec[r];
        if (rec.x >= d.P) continue;                     // a reserved slot left unused
        if (rec.y >= g.pv_cnt[rec.x]) continue;         // a record of a walk that failed (not counted)
        g.pv_sorted[g.pv_off[rec.x] + rec.y] = make_uint4(rec.z, rec.w, g.pv_end[r], 0u);
    }
}

// ---- children's cache by merging the parents' entries (no structure pass)
//
// A child's cached nodes, in position order, are: the mother's cached nodes
// before the crossover point (ancestors of it re-sized by the size change,
// dropped when they fall below the threshold, plus ancestors that rise
// above it, which the walk recorded), the father's cached nodes inside the
// donated subtree (moved to the crossover point), then the mother's cached
// nodes after the removed subtree (moved by the size change).

__device__ __forceinline__ uint32_t lower_bound_pos(const uint32_t* e_pos, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (e_pos[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// deepest cached ancestor of c in the mother (entry index) or -1
__device__ __forceinline__ int32_t mother_anchor(const CacheView& par, uint32_t me0, uint32_t me1, uint32_t c,
                                                 uint32_t r, uint32_t T) {
    if (c == 0) return -1;
    int32_t e;
    if (r >= T) {
        e = find_exact(par.e_pos, me0, me1, c);
        return e >= 0 ? par.e_par[e] : -1;
    }
    e = find_last_lt(par.e_pos, me0, me1, c);
    uint32_t guard = 0;
    while (e >= 0 && par.e_end[e] <= c && guard++ < (1u << 24)) e = par.e_par[e];
    return e;
}

__device__ __forceinline__ bool drops(const CacheView& par, int32_t e, int32_t delta, uint32_t T) {
    const uint32_t pos = par.e_pos[e];
    return pos > 0 && (int64_t)par.e_end[e] + delta - (int64_t)pos < (int64_t)T;
}

// Warp-collective: first index in [lo, hi) of the sorted array a with
// a[i] >= x (hi if none), by 32-way splitting (two rounds for 1,000 entries).
__device__ __forceinline__ uint32_t warp_lower_bound(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t x) {
    const uint32_t lane = (uint32_t)lane_id();
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t last = min(lo + (lane + 1) * step, hi) - 1;     // last index of this lane's segment
        const uint32_t m = __ballot_sync(FULL, a[last] >= x);
        if (!m) return hi;
        const uint32_t f = (uint32_t)__ffs(m) - 1;                      // first segment ending at >= x
        const uint32_t nlo = lo + f * step;
        hi = min(nlo + step, hi);
        lo = nlo;
    }
    const uint32_t i = lo + lane;
    const uint32_t m = __ballot_sync(FULL, i < hi && a[i] >= x);
    return m ? lo + (uint32_t)__ffs(m) - 1 : hi;
}

// deepest cached ancestor of c in the mother (entry index) or -1; warp-collective
__device__ __forceinline__ int32_t warp_mother_anchor(const CacheView& par, uint32_t me0, uint32_t me1, uint32_t c,
                                                      uint32_t r, uint32_t T) {
    if (c == 0) return -1;
    const uint32_t jc = warp_lower_bound(par.e_pos, me0, me1, c);
    if (r >= T) return (jc < me1 && par.e_pos[jc] == c) ? par.e_par[jc] : -1;
    int32_t e = (jc > me0) ? (int32_t)(jc - 1) : -1;
    uint32_t guard = 0;
    while (e >= 0 && par.e_end[e] <= c && guard++ < (1u << 24)) e = par.e_par[e];
    return e;
}

// Entry count of each child (a warp per child: its four bound searches are
// warp-parallel, the walk over the dropped ancestors is short).
__global__ void k_merge_count(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    const uint32_t lane = (uint32_t)lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < d.P; i += nwarp) {
        const uint32_t m = g.mother[i];
        const uint32_t me0 = par.e_off[m], me1 = par.e_off[m + 1];
        if (g.lazy && !g.sel[i]) { if (lane == 0) g.mcnt[i] = 0; continue; }     // never a parent: no cache
        if (g.flags[i] & F_CLONE) { if (lane == 0) g.mcnt[i] = me1 - me0; continue; }
        const uint32_t f = g.father[i], c = g.cpos[i], r = g.rsz[i], dd = g.dpos[i], s = g.ssz[i];
        const int32_t delta = (int32_t)s - (int32_t)r;
        const uint32_t fe0 = par.e_off[f], fe1 = par.e_off[f + 1];
        const uint32_t jc = warp_lower_bound(par.e_pos, me0, me1, c);
        const uint32_t jcr = warp_lower_bound(par.e_pos, me0, me1, c + r);
        uint32_t jd = warp_lower_bound(par.e_pos, fe0, fe1, dd);
        const uint32_t jds = warp_lower_bound(par.e_pos, fe0, fe1, dd + s);
        // a father's root is cached whatever its size; inside the child it is
        // cached only when it becomes the child's root or is itself large
        if (dd == 0 && c != 0 && s < d.T && jd < jds) ++jd;
        uint32_t ndrop = 0;
        if (delta < 0) {
            int32_t e = warp_mother_anchor(par, me0, me1, c, r, d.T);
            uint32_t guard = 0;
            while (e >= 0 && drops(par, e, delta, d.T) && guard++ < (1u << 24)) { ++ndrop; e = par.e_par[e]; }
        }
        if (lane == 0) {
            g.mb[i] = make_uint4(jc, jcr, jd, jds);
            g.mcnt[i] = (jc - me0) - ndrop + g.nins[i] + (jds - jd) + (me1 - jcr);
        }
    }
}

// Exclusive scan of the counts into the children's entry offsets.
__global__ void __launch_bounds__(1024) k_merge_offsets(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < d.P; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = (i < d.P) ? g.mcnt[i] : 0;
        const uint64_t o = block_excl_scan(v, ws, &carry);
        if (i < d.P) { d.e_off[i] = (uint32_t)o; d.e_cnt[i] = (uint32_t)v; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.e_off[d.P] = (uint32_t)carry;
        *d.e_total = (uint32_t)carry;
        if (d.strict_cap && carry > d.Ecap) set_status(d.status, ST_ENTRIES);
        *g.stamp += 1;               // a new generation of live marks in the slot pool
    }
}

// A child's cache entry.  src is the mother's (or father's) value slot, which
// the child shares, or (bit 31 set) a walk record whose new value gets a
// free slot of the pool later (k_copy_values).
__device__ __forceinline__ void put_entry(const DevPop& d, GenBufs& g, uint32_t x, uint32_t pos, uint32_t end,
                                          uint32_t tree, uint32_t src) {
    d.e_pos[x] = pos;
    d.e_end[x] = end;
    d.e_tree[x] = tree;
    d.e_c0[x] = -1;
    d.e_c1[x] = -1;
    d.e_par[x] = -1;
    d.e_slot[x] = (src & 0x80000000u) ? SLOT_NEW : src;
    g.src[x] = src;
    if (src & 0x80000000u) g.rec_entry[src & 0x7FFFFFFFu] = x;
}

// walk record of child i at position pos (records are sorted by decreasing position), or -1
__device__ __forceinline__ int32_t find_record(const GenBufs& g, uint32_t i, uint32_t pos) {
    uint32_t lo = g.pv_off[i], hi = g.pv_off[i + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t pp = g.pv_sorted[mid].x;
        if (pp == pos) return (int32_t)mid;
        if (pp > pos) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// One CTA per child writes its entries (position, end, value source):
// the mother's entries before c (dropping ancestors that fall below the
// threshold, merged with the walk's inserted ancestors), the root made of a
// small donated subtree, the father's entries of the donated subtree, and
// the mother's entries after the removed subtree, shifted by delta.
#define MERGE_MAXINS 1024
__global__ void __launch_bounds__(256) k_merge_write(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    if (d.e_off[d.P] > d.Ecap) return;
    __shared__ uint32_t s_ins[MERGE_MAXINS];   // positions of inserted ancestors before c, decreasing
    __shared__ uint64_t ws[32];
    __shared__ uint64_t cins, ckept;
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;
    const int lane = lane_id();
    const uint32_t T = d.T;
    for (uint32_t i = blockIdx.x; i < d.P; i += gridDim.x) {
        if (g.lazy && !g.sel[i]) continue;                      // uniform per CTA
        const uint32_t o = d.e_off[i];
        const uint32_t m = g.mother[i];
        const uint32_t me0 = par.e_off[m], me1 = par.e_off[m + 1];
        if (g.flags[i] & F_CLONE) {
            for (uint32_t k = tid; k < me1 - me0; k += nthr) {
                const uint32_t e = me0 + k;
                put_entry(d, g, o + k, par.e_pos[e], par.e_end[e], i, par.e_slot[e]);
            }
            continue;
        }
        const uint32_t c = g.cpos[i], dd = g.dpos[i];
        const int32_t delta = (int32_t)g.ssz[i] - (int32_t)g.rsz[i];
        const uint4 mb = g.mb[i];
        const uint32_t jc = mb.x, jcr = mb.y, jd = mb.z, jds = mb.w;
        const uint32_t r0 = g.pv_off[i], r1 = g.pv_off[i + 1];
        if (tid == 0) { cins = 0; ckept = 0; }
        __syncthreads();
        // inserted ancestors before c, in record order (positions decreasing)
        uint32_t rootins = 0;
        for (uint32_t base = r0; base < r1; base += nthr) {
            const uint32_t q = base + tid;
            bool ins_lt = false;
            if (q < r1) {
                const uint4 rec = g.pv_sorted[q];
                const bool ins = (rec.y & 0x80000000u) != 0;
                ins_lt = ins && rec.x < c;
                if (ins && rec.x == c) rootins = 1;
            }
            const uint64_t rk = block_excl_scan(ins_lt ? 1u : 0u, ws, &cins);
            if (ins_lt && rk < MERGE_MAXINS) s_ins[rk] = g.pv_sorted[q].x;
        }
        rootins = __syncthreads_or(rootins) ? 1u : 0u;
        const uint32_t nins_lt = (uint32_t)cins;
        if (nins_lt > MERGE_MAXINS) {
            if (tid == 0) set_status(d.status, ST_PATH);
            __syncthreads();
            continue;
        }
        // part 1: mother entries before c, one row of nthr entries at a time
        for (uint32_t base = me0; base < jc; base += nthr) {
            const uint32_t e = base + tid;
            uint32_t pos = 0, end = 0;
            bool keep = false, anc = false;
            if (e < jc) {
                pos = par.e_pos[e];
                end = par.e_end[e];
                anc = end > c;
                keep = !(anc && drops(par, (int32_t)e, delta, T));
            }
            const uint64_t kb = block_excl_scan(keep ? 1u : 0u, ws, &ckept);
            if (keep) {
                // inserted ancestors before pos: s_ins is decreasing, so they are its tail
                uint32_t lo = 0, hi = nins_lt;         // first index with s_ins < pos
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_ins[mid] >= pos) lo = mid + 1; else hi = mid;
                }
                const uint32_t x = o + (uint32_t)kb + (nins_lt - lo);
                uint32_t src = par.e_slot[e];
                if (anc) {
                    const int32_t h = find_record(g, i, pos);
                    if (h >= 0) src = g.pv_sorted[h].y | 0x80000000u;
                }
                put_entry(d, g, x, pos, anc ? (uint32_t)((int64_t)end + delta) : end, i, src);
            }
        }
        const uint32_t kept = (uint32_t)ckept;
        // inserted ancestors before c (few): kept mother entries and inserts before each
        if (tid < 32) {
            const int32_t anchor = (delta < 0) ? mother_anchor(par, me0, me1, c, g.rsz[i], T) : -1;
            for (uint32_t k = lane; k < nins_lt; k += 32) {
                const uint32_t px = s_ins[k];
                uint32_t mlt = lower_bound_pos(par.e_pos, me0, jc, px) - me0;
                int32_t e = anchor;
                uint32_t guard = 0;
                while (e >= 0 && drops(par, e, delta, T) && guard++ < (1u << 24)) {
                    if (par.e_pos[e] < px) --mlt;
                    e = par.e_par[e];
                }
                const uint32_t ilt = nins_lt - 1 - k;          // s_ins is decreasing and distinct
                const int32_t h = find_record(g, i, px);
                if (h >= 0) {
                    const uint4 rec = g.pv_sorted[h];
                    put_entry(d, g, o + mlt + ilt, rec.x, rec.z, i, (rec.y & 0x7FFFFFFFu) | 0x80000000u);
                }
            }
            if (rootins && lane == 0) {
                const int32_t h = find_record(g, i, c);
                if (h >= 0) {
                    const uint4 rec = g.pv_sorted[h];
                    put_entry(d, g, o + kept + nins_lt, rec.x, rec.z, i, (rec.y & 0x7FFFFFFFu) | 0x80000000u);
                }
            }
        }
        const uint32_t o2 = o + kept + nins_lt + rootins;
        // part 2: father entries in the donated subtree
        for (uint32_t k = tid; k < jds - jd; k += nthr) {
            const uint32_t e = jd + k;
            put_entry(d, g, o2 + k, par.e_pos[e] - dd + c, par.e_end[e] - dd + c, i, par.e_slot[e]);
        }
        // part 3: mother entries after the removed subtree
        const uint32_t o3 = o2 + (jds - jd);
        for (uint32_t k = tid; k < me1 - jcr; k += nthr) {
            const uint32_t e = jcr + k;
            put_entry(d, g, o3 + k, (uint32_t)((int64_t)par.e_pos[e] + delta), (uint32_t)((int64_t)par.e_end[e] + delta),
                      i, par.e_slot[e]);
        }
        __syncthreads();              // shared lists are rewritten for the next child
    }
}

// ---- slot pool: the children's entries share the parents' value slots;
// slots that no child entry references are free again, and the walk's new
// values go to the first free ones (in slot order).

// Mark the slots the children's cache references with this generation's stamp.
__global__ void k_mark_live(DevPop d, GenBufs g) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const uint32_t stamp = *g.stamp;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < ne; x += gridDim.x * blockDim.x) {
        const uint32_t sl = d.e_slot[x];
        if (sl != SLOT_NEW && sl < d.Scap) d.live[sl] = stamp;
    }
}

__device__ __forceinline__ uint32_t block_reduce_add(uint32_t v, uint32_t* ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();
    if (lane == 0) ws[w] = v;
    __syncthreads();
    uint32_t t = 0;
    for (uint32_t k = 0; k < (blockDim.x >> 5); ++k) t += ws[k];
    return t;
}

// Free slots per tile of FREE_TILE slots (1024 threads, four slots each).
__global__ void __launch_bounds__(1024) k_free_count(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint32_t ws[32];
    const uint32_t stamp = *g.stamp;
    const uint32_t nt = (d.Scap + FREE_TILE - 1) / FREE_TILE;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const uint32_t s0 = t * FREE_TILE + 4 * threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) c += (s0 + k < d.Scap && d.live[s0 + k] != stamp) ? 1u : 0u;
        c = block_reduce_add(c, ws);
        if (threadIdx.x == 0) d.ftile[t] = c;
    }
}

// Exclusive prefix of the per-tile counts (one CTA); too few free slots for
// the walk's new values is a budget error.
__global__ void __launch_bounds__(1024) k_free_top(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t nt = (d.Scap + FREE_TILE - 1) / FREE_TILE;
    for (uint32_t base = 0; base < nt; base += blockDim.x) {
        const uint32_t t = base + threadIdx.x;
        const uint64_t v = (t < nt) ? d.ftile[t] : 0;
        const uint64_t o = block_excl_scan(v, ws, &carry);
        if (t < nt) d.ftile[t] = (uint32_t)o;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        d.ftile[nt] = (uint32_t)min(carry, (uint64_t)0xFFFFFFFFu);     // free slots in all
        if (carry < min(g.misc[M_PV], g.pvcap)) set_status(d.status, ST_SLOTS);
    }
}

// freeslot[r] = the r-th free slot, for the ranks the new values need.
__global__ void __launch_bounds__(1024) k_free_emit(DevPop d, GenBufs g) {
    if (halted(d)) return;
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry;
    const uint32_t stamp = *g.stamp;
    const uint32_t need = min(g.misc[M_PV], g.pvcap);
    const uint32_t nt = (d.Scap + FREE_TILE - 1) / FREE_TILE;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const uint32_t base = d.ftile[t];
        if (base >= need) continue;                       // uniform per CTA
        if (threadIdx.x == 0) carry = base;
        __syncthreads();
        const uint32_t s0 = t * FREE_TILE + 4 * threadIdx.x;
        uint32_t fr[4], c = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) { fr[k] = (s0 + k < d.Scap && d.live[s0 + k] != stamp) ? 1u : 0u; c += fr[k]; }
        uint32_t r = (uint32_t)block_excl_scan(c, ws, &carry);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (fr[k]) { if (r < need) d.freeslot[r] = s0 + k; ++r; }
        __syncthreads();
    }
}

// New values of the children's cache (walk records): each record that
// became an entry takes the free slot of its rank; one warp per record,
// lanes over cases.
__global__ void k_copy_values(DevPop d, GenBufs g, CacheView par) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const int lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nt = (d.Scap + FREE_TILE - 1) / FREE_TILE;
    const uint32_t nrec = min(g.misc[M_PV], g.pvcap);
    const uint32_t avail = min(nrec, d.ftile[nt]);
    for (uint32_t r = gw; r < nrec; r += nw) {
        const uint32_t x = g.rec_entry[r];
        if (x >= ne) continue;                           // not an entry of the children's cache
        if (r >= avail) { if (lane == 0) set_status(d.status, ST_SLOTS); continue; }
        const uint32_t sl = d.freeslot[r];
        const float* sp = g.pv_val + (size_t)r * d.Cpad;
        float* dp = d.slots + (size_t)sl * d.Cpad;
        for (uint32_t k = lane; k < d.Cpad; k += 32) dp[k] = __ldcg(sp + k);
        if (lane == 0) d.e_slot[x] = sl;
    }
    (void)par;
}

// equivalent-op count of the children (every opcode on every case)
__global__ void k_child_sizes(DevPop d, GenBufs g) {
    if (halted(d)) return;
    unsigned long long s = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x) s += d.size[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(&g.gstat[G_EQUIV], s);
}

// Features of each child known before its walk (16 per child, scaled to
// about [0, 1]): parent and exchanged-subtree sizes, size change, relative
// crossover points, whether the exchanged subtrees are cached, the parents'
// fitness, cache sizes and the spread of their root value vectors, a clone
// flag and a constant.
__global__ void k_mlp_features(DevPop d, GenBufs g, CacheView par, MlpBufs b) {
    if (halted(d)) return;
    // a warp per child: the lanes share the spread of the two root vectors
    const int lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < d.P; i += nwp) {
        const uint32_t m = g.mother[i], f = g.father[i];
        float spread[2];
        for (int q = 0; q < 2; ++q) {
            const uint32_t t = q ? f : m;
            const float* v = par.slots + (size_t)par.e_slot[par.e_off[t]] * d.Cpad;
            float lo = INFINITY, hi = -INFINITY;
            for (uint32_t cc = lane; cc < d.C; cc += 32) {
                const float a = (d.vkind == VI) ? (float)__float_as_int(v[cc]) : v[cc];
                if (isfinite(a)) { lo = fminf(lo, a); hi = fmaxf(hi, a); }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
                hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
            }
            spread[q] = (hi >= lo) ? fminf(log2f(1.f + (hi - lo)) / 8.f, 4.f) : 4.f;
        }
        if (lane != 0) continue;
        const uint32_t c = g.cpos[i], r = g.rsz[i], dd = g.dpos[i], s = g.ssz[i];
        const float sm = (float)g.psize[m], sf = (float)g.psize[f];
        float* x = b.feat + (size_t)i * MLP_IN;
        const float dl = (float)s - (float)r;
        x[0] = log2f(1.f + sm) / 21.f;
        x[1] = log2f(1.f + sf) / 21.f;
        x[2] = log2f(1.f + (float)r) / 21.f;
        x[3] = log2f(1.f + (float)s) / 21.f;
        x[4] = copysignf(log2f(1.f + fabsf(dl)), dl) / 21.f;
        x[5] = (float)c / sm;
        x[6] = (float)dd / sf;
        x[7] = (r >= d.T) ? 1.f : 0.f;
        x[8] = (s >= d.T) ? 1.f : 0.f;
        const float fm = g.pfit[m], ff = g.pfit[f];
        x[9] = isfinite(fm) ? fminf(log2f(1.f + fabsf(fm)) / 8.f, 4.f) : 4.f;
        x[10] = isfinite(ff) ? fminf(log2f(1.f + fabsf(ff)) / 8.f, 4.f) : 4.f;
        x[11] = log2f(1.f + (float)(par.e_off[m + 1] - par.e_off[m])) / 16.f;
        x[12] = spread[0];
        x[13] = spread[1];
        x[14] = (g.flags[i] & F_CLONE) ? 1.f : 0.f;
        x[15] = 1.f;
    }
}

// static packing key: the mother's size (largest first)
__global__ void k_static_key(DevPop d, GenBufs g, MlpBufs b) {
    if (halted(d)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x)
        b.target[i] = (float)g.psize[g.mother[i]];
}

// training targets: log2(1 + levels the walk evaluated)
__global__ void k_mlp_targets(DevPop d, GenBufs g, MlpBufs b) {
    if (halted(d)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x)
        b.target[i] = log2f(1.f + (float)g.plen[i]);
}

__global__ void k_order_identity(DevPop d, GenBufs g) {
    if (halted(d)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += gridDim.x * blockDim.x) g.order[i] = i;
}
