// Structure pass: the nodes that head subtrees of at least T nodes (the
// cached "skeleton"), with subtree ends, parents and large-child links.
//
// A prefix tree is read as a balance walk: b[0] = 0 and b[j+1] = b[j] + 1
// for a leaf, - 1 for a binary function.  The subtree that starts at node i
// is the contiguous run i .. end(i)-1 (Sec. 3.1: flattened trees keep each
// subtree contiguous), where end(i) is the first j > i with b[j] = b[i]+1.
// Hence node i heads a subtree of at least T nodes exactly when b never
// rises above b[i] on (i, i+T).  Positions past the end count as leaves.
//
// All steps are data parallel:
//   k_unit_flags    one warp per 1024-position block: flags, per-32-chunk
//                   balances and maxima (window maxima of width T-1 from
//                   segmented prefix/suffix maxima over T-aligned segments)
//   k_scan_*        prefix sums of flag counts and block balances
//   k_emit_entries  positions of flagged nodes, in order, with balances
//   k_entry_ends    per entry: first later position where the balance
//                   rises, via chunk and block maxima
//   k_entry_parents per entry: nearest earlier entry whose subtree ends no
//                   earlier (intervals are nested or disjoint), and the
//                   parent's left/right large-child link
#pragma once
#include "common.cuh"

#define NEG_INF_I (-0x3FFFFFFF)

struct StructBufs {
    uint32_t* u_flags;   // [U*32]
    int32_t* u_cv0;      // [U*32] balance before the chunk, relative to the block start
    int32_t* u_cmax;     // [U*32] max after-balance in the chunk, relative to the block start
    int32_t* u_total;    // [U]
    int32_t* u_max;      // [U]
    uint32_t* u_cnt;     // [U]
    uint32_t* u_epre;    // [U+1] exclusive prefix of counts (global entry index)
    int64_t* u_bpre;     // [U+1] exclusive prefix of block totals
    uint32_t* tile_c;    // scan tiles
    int64_t* tile_b;
    int32_t* e_bal;      // [Ecap] balance before the entry's node (within its tree)
    uint32_t* e_tree;    // [Ecap] (same array as DevPop::e_tree)
    uint32_t* e_cmax;    // [Ecap/32+1] max end per 32-entry chunk
    uint32_t Ucap;
};

// 32 leaf bits of positions p0..p0+31 (bit s = 1: leaf or past the end).
// p0 is a multiple of 32 and the buffer capacity a multiple of GP_B, so the
// 32-byte load stays inside the buffer whenever p0 < n.
__device__ __forceinline__ uint32_t leaf_bits(const uint8_t* ops, uint32_t n, uint32_t p0) {
    if (p0 >= n) return FULL;
    const uint4* q = reinterpret_cast<const uint4*>(ops + p0);
    uint4 a = __ldg(q), b = __ldg(q + 1);
    uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t m = __vcmpgeu4(w[i], 0x04040404u) & 0x01010101u;   // opcode >= 4 is a leaf
        bits |= ((m * 0x10204080u) >> 28) << (4 * i);
    }
    uint32_t left = n - p0;
    if (left < 32) bits |= FULL << left;
    return bits;
}

// balance after slot j (0..31) of a chunk whose before-balance is v0
__device__ __forceinline__ int after_bal(uint32_t bits, int v0, int j) {
    uint32_t m = (j >= 31) ? FULL : ((1u << (j + 1)) - 1u);
    return v0 + 2 * __popc(bits & m) - (j + 1);
}

__device__ __forceinline__ int warp_incl_sum(int v) {
    int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ int seg_prefix_max(int v, int L) {
    int lane = lane_id();
    for (int o = 1; o < L; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if ((lane & (L - 1)) >= o) v = max(v, t);
    }
    return v;
}

__device__ __forceinline__ int seg_suffix_max(int v, int L) {
    int lane = lane_id();
    for (int o = 1; o < L; o <<= 1) {
        int t = __shfl_down_sync(FULL, v, o);
        if ((lane & (L - 1)) + o < L) v = max(v, t);
    }
    return v;
}

// Block [base, base+GP_B) of a tree of n nodes; lane l owns positions
// base+32l .. base+32l+31.  Window maxima use pm: per-warp shared prefix
// maxima (within T-aligned segments) of blocks k and k+1; suffix maxima of
// block k are kept as a running value in a reverse sweep.
#define FLAG_WARPS 4
// offset j in [0, 2*GP_B) -> padded transposed slot: lanes touching offsets
// 32 apart (same slot s, consecutive lanes) hit consecutive banks
#define PMX(j) ((((j) & 31) * 65) + ((j) >> 5))
__global__ void __launch_bounds__(FLAG_WARPS * 32) k_unit_flags(DevPop d, StructBufs sb) {
    __shared__ int pm_all[FLAG_WARPS][32 * 65];
    int* pm = pm_all[threadIdx.x >> 5];
    const int lane = lane_id();
    const uint32_t nunits = d.blk_off[d.P];
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const int Ts = (int)d.T;
    const int L = Ts > 32 ? Ts / 32 : 1;          // lanes per T-segment
    for (uint32_t u = gw; u < nunits; u += nw) {
        const uint32_t tree = find_segment(d.blk_off, d.P, u);
        const uint32_t base = (u - d.blk_off[tree]) * GP_B;
        const uint8_t* ops = tree_ptr(d, tree);
        const uint32_t n = d.size[tree];
        const uint32_t b0 = leaf_bits(ops, n, base + 32 * lane);
        const uint32_t b1 = leaf_bits(ops, n, base + GP_B + 32 * lane);
        const int t0 = 2 * __popc(b0) - 32, t1 = 2 * __popc(b1) - 32;
        const int i0 = warp_incl_sum(t0), i1 = warp_incl_sum(t1);
        const int tot0 = __shfl_sync(FULL, i0, 31);
        const int v0 = i0 - t0;               // block k: balance before the lane's first position
        const int w0 = tot0 + i1 - t1;        // block k+1
        // lane maxima of before-balances, and in-segment prefix maxima into pm
        int m0 = NEG_INF_I, m1 = NEG_INF_I, cmax = NEG_INF_I;
        {
            int a = v0, c = w0;
#pragma unroll 4
            for (int s = 0; s < 32; ++s) {
                m0 = max(m0, a); m1 = max(m1, c);
                a += ((b0 >> s) & 1) ? 1 : -1;
                c += ((b1 >> s) & 1) ? 1 : -1;
                cmax = max(cmax, a);
            }
        }
        int ex0 = NEG_INF_I, ex1 = NEG_INF_I, exs = NEG_INF_I;   // across-lane parts within the segment
        if (Ts > 32) {
            const int p0 = seg_prefix_max(m0, L), p1 = seg_prefix_max(m1, L);
            ex0 = __shfl_up_sync(FULL, p0, 1);
            ex1 = __shfl_up_sync(FULL, p1, 1);
            if ((lane & (L - 1)) == 0) { ex0 = NEG_INF_I; ex1 = NEG_INF_I; }
            const int sf = seg_suffix_max(m0, L);
            exs = __shfl_down_sync(FULL, sf, 1);
            if ((lane & (L - 1)) == L - 1) exs = NEG_INF_I;
        }
        {
            int a = v0, c = w0, r0 = ex0, r1 = ex1;
#pragma unroll 2
            for (int s = 0; s < 32; ++s) {
                if (Ts <= 32 && (s & (Ts - 1)) == 0) { r0 = NEG_INF_I; r1 = NEG_INF_I; }
                r0 = max(r0, a); r1 = max(r1, c);
                pm[PMX(32 * lane + s)] = r0;
                pm[PMX(GP_B + 32 * lane + s)] = r1;
                a += ((b0 >> s) & 1) ? 1 : -1;
                c += ((b1 >> s) & 1) ? 1 : -1;
            }
        }
        __syncwarp();
        // reverse sweep: sm = max of before-balances over [s+1, end of s's T-segment]
        uint32_t flags = 0;
        {
            int v = v0 + t0;                  // balance after the lane's last position
            int sm = (Ts > 32) ? exs : NEG_INF_I;
#pragma unroll 2
            for (int s = 31; s >= 0; --s) {
                v -= ((b0 >> s) & 1) ? 1 : -1;     // before-balance of slot s
                const int j = 32 * lane + s;       // node i = base + j; window (i, i+T) = offsets [j+1, j+T-1]
                const int a = j + 1;
                const int pmv = pm[PMX(a + Ts - 2)];
                const int wmax = ((a & (Ts - 1)) == 0) ? pmv : max(sm, pmv);
                if (wmax <= v && (uint32_t)(base + j) < n) flags |= 1u << s;
                sm = max(sm, v);
                if (Ts <= 32 && (s & (Ts - 1)) == 0) sm = NEG_INF_I;
            }
        }
        if (base == 0 && lane == 0 && n > 0) flags |= 1u;   // every root is cached
        __syncwarp();
        sb.u_flags[(size_t)u * 32 + lane] = flags;
        sb.u_cv0[(size_t)u * 32 + lane] = v0;
        sb.u_cmax[(size_t)u * 32 + lane] = cmax;
        uint32_t cnt = __popc(flags);
        int bm = cmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt += __shfl_down_sync(FULL, cnt, o);
            bm = max(bm, __shfl_down_sync(FULL, bm, o));
        }
        if (lane == 0) { sb.u_cnt[u] = cnt; sb.u_total[u] = tot0; sb.u_max[u] = bm; }
    }
}

// ---- three-phase exclusive scan of (u_cnt, u_total) over all units ----
#define SCAN_TILE 1024

__device__ __forceinline__ void block_scan2(uint32_t& a, int64_t& b, uint32_t* wa, int64_t* wb) {
    // inclusive block scan of (a, b), 1024 threads
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t ta = __shfl_up_sync(FULL, a, o);
        int64_t tb = __shfl_up_sync(FULL, b, o);
        if (lane >= o) { a += ta; b += tb; }
    }
    if (lane == 31) { wa[w] = a; wb[w] = b; }
    __syncthreads();
    if (w == 0) {
        uint32_t xa = wa[lane];
        int64_t xb = wb[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t ta = __shfl_up_sync(FULL, xa, o);
            int64_t tb = __shfl_up_sync(FULL, xb, o);
            if (lane >= o) { xa += ta; xb += tb; }
        }
        wa[lane] = xa; wb[lane] = xb;
    }
    __syncthreads();
    if (w > 0) { a += wa[w - 1]; b += wb[w - 1]; }
    __syncthreads();
}

__global__ void __launch_bounds__(SCAN_TILE) k_scan_tiles(DevPop d, StructBufs sb) {
    __shared__ uint32_t wa[32];
    __shared__ int64_t wb[32];
    const uint32_t nunits = d.blk_off[d.P];
    const uint32_t ntiles = (nunits + SCAN_TILE - 1) / SCAN_TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint32_t u = tile * SCAN_TILE + threadIdx.x;
        uint32_t a = (u < nunits) ? sb.u_cnt[u] : 0;
        int64_t b = (u < nunits) ? sb.u_total[u] : 0;
        block_scan2(a, b, wa, wb);
        if (threadIdx.x == SCAN_TILE - 1) { sb.tile_c[tile] = a; sb.tile_b[tile] = b; }
    }
}

__global__ void __launch_bounds__(SCAN_TILE) k_scan_top(DevPop d, StructBufs sb) {
    __shared__ uint32_t wa[32];
    __shared__ int64_t wb[32];
    __shared__ uint32_t ca;
    __shared__ int64_t cb;
    const uint32_t nunits = d.blk_off[d.P];
    const uint32_t ntiles = (nunits + SCAN_TILE - 1) / SCAN_TILE;
    if (threadIdx.x == 0) { ca = 0; cb = 0; }
    __syncthreads();
    for (uint32_t t0 = 0; t0 < ntiles; t0 += SCAN_TILE) {
        uint32_t t = t0 + threadIdx.x;
        uint32_t a = (t < ntiles) ? sb.tile_c[t] : 0;
        int64_t b = (t < ntiles) ? sb.tile_b[t] : 0;
        uint32_t a0 = a;
        int64_t b0 = b;
        block_scan2(a, b, wa, wb);
        if (t < ntiles) { sb.tile_c[t] = a - a0 + ca; sb.tile_b[t] = b - b0 + cb; }   // exclusive
        __syncthreads();
        if (threadIdx.x == SCAN_TILE - 1) { ca += a; cb += b; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sb.u_epre[nunits] = ca;
        sb.u_bpre[nunits] = cb;
        *d.e_total = ca;
        if (d.strict_cap && ca > d.Ecap) set_status(d.status, ST_ENTRIES);
    }
}

__global__ void __launch_bounds__(SCAN_TILE) k_scan_apply(DevPop d, StructBufs sb) {
    __shared__ uint32_t wa[32];
    __shared__ int64_t wb[32];
    const uint32_t nunits = d.blk_off[d.P];
    const uint32_t ntiles = (nunits + SCAN_TILE - 1) / SCAN_TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        uint32_t u = tile * SCAN_TILE + threadIdx.x;
        uint32_t a = (u < nunits) ? sb.u_cnt[u] : 0;
        int64_t b = (u < nunits) ? sb.u_total[u] : 0;
        uint32_t a0 = a;
        int64_t b0 = b;
        block_scan2(a, b, wa, wb);
        if (u < nunits) {
            sb.u_epre[u] = sb.tile_c[tile] + a - a0;
            sb.u_bpre[u] = sb.tile_b[tile] + b - b0;
        }
    }
}

// e_off / e_cnt per tree from the unit prefix.
__global__ void k_tree_entry_offsets(DevPop d, StructBufs sb) {
    if (halted(d)) return;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= d.P; i += gridDim.x * blockDim.x) {
        uint32_t v = sb.u_epre[d.blk_off[i]];
        d.e_off[i] = v;
        if (i < d.P) d.e_cnt[i] = sb.u_epre[d.blk_off[i + 1]] - v;
    }
}

// Write each flagged node as an entry, in position order.
__global__ void __launch_bounds__(GP_WARPS * 32) k_emit_entries(DevPop d, StructBufs sb) {
    const int lane = lane_id();
    const uint32_t nunits = d.blk_off[d.P];
    if (sb.u_epre[nunits] > d.Ecap) return;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t u = gw; u < nunits; u += nw) {
        if (sb.u_cnt[u] == 0) continue;
        const uint32_t tree = find_segment(d.blk_off, d.P, u);
        const uint32_t base = (u - d.blk_off[tree]) * GP_B;
        const int64_t bbase = sb.u_bpre[u] - sb.u_bpre[d.blk_off[tree]];
        uint32_t fl = sb.u_flags[(size_t)u * 32 + lane];
        int v0 = sb.u_cv0[(size_t)u * 32 + lane];
        uint32_t c = __popc(fl);
        uint32_t incl = (uint32_t)warp_incl_sum((int)c);
        uint32_t e = sb.u_epre[u] + incl - c;
        if (fl) {
            uint32_t bits = leaf_bits(tree_ptr(d, tree), d.size[tree], base + 32 * lane);
            while (fl) {
                int s = __ffs(fl) - 1;
                fl &= fl - 1;
                int bal = (int)bbase + v0 + 2 * __popc(bits & ((1u << s) - 1u)) - s;
                d.e_pos[e] = base + 32 * lane + s;
                sb.e_bal[e] = bal;
                sb.e_tree[e] = tree;
                d.e_c0[e] = -1;
                d.e_c1[e] = -1;
                d.e_slot[e] = e;
                ++e;
            }
        }
    }
}

// First chunk index c >= from (of 32) whose maximum reaches `need`, or 32;
// eight independent loads per round.
__device__ __forceinline__ uint32_t first_chunk_at_least(const int32_t* cm, uint32_t from, int need) {
    for (uint32_t c0 = from; c0 < 32; c0 += 8) {
        int v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (c0 + j < 32) ? cm[c0 + j] : NEG_INF_I;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (v[j] >= need) return c0 + j;
    }
    return 32;
}

// end(entry) = first position q >= pos with after-balance >= bal + 1, plus one.
__global__ void k_entry_ends(DevPop d, StructBufs sb) {
    if (halted(d)) return;
    const uint32_t ne = sb.u_epre[d.blk_off[d.P]];
    if (ne > d.Ecap) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const uint32_t tree = sb.e_tree[e];
        const uint32_t pos = d.e_pos[e];
        const int target = sb.e_bal[e] + 1;
        const uint8_t* ops = tree_ptr(d, tree);
        const uint32_t n = d.size[tree];
        const uint32_t u0 = d.blk_off[tree], nb = d.blk_off[tree + 1] - u0;
        const int64_t bp0 = sb.u_bpre[u0];
        uint32_t k = pos / GP_B, c = (pos % GP_B) / 32, s = pos % 32;
        uint32_t endpos = 0xFFFFFFFFu;
        // 1: rest of the node's own chunk
        {
            int bb = (int)(sb.u_bpre[u0 + k] - bp0);
            int v0 = bb + sb.u_cv0[(size_t)(u0 + k) * 32 + c];
            uint32_t bits = leaf_bits(ops, n, k * GP_B + c * 32);
            for (uint32_t j = s; j < 32; ++j)
                if (after_bal(bits, v0, (int)j) >= target) { endpos = k * GP_B + c * 32 + j + 1; break; }
        }
        // 2/3: later chunks of this block, then later blocks
        uint32_t fk = 0xFFFFFFFFu, fc = 0;
        if (endpos == 0xFFFFFFFFu) {
            int bb = (int)(sb.u_bpre[u0 + k] - bp0);
            fc = first_chunk_at_least(sb.u_cmax + (size_t)(u0 + k) * 32, c + 1, target - bb);
            if (fc < 32) fk = k;
            if (fk == 0xFFFFFFFFu) {
                // later blocks, eight summaries per round of independent loads
                uint32_t hitk = 0xFFFFFFFFu;
                for (uint32_t k2 = k + 1; k2 < nb && hitk == 0xFFFFFFFFu; k2 += 8) {
                    int64_t bpv[8];
                    int mxv[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t kk = k2 + j;
                        bpv[j] = (kk < nb) ? sb.u_bpre[u0 + kk] : 0;
                        mxv[j] = (kk < nb) ? sb.u_max[u0 + kk] : NEG_INF_I;
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (hitk == 0xFFFFFFFFu && k2 + j < nb && (int)(bpv[j] - bp0) + mxv[j] >= target) hitk = k2 + j;
                }
                if (hitk != 0xFFFFFFFFu) {
                    int bb2 = (int)(sb.u_bpre[u0 + hitk] - bp0);
                    fc = first_chunk_at_least(sb.u_cmax + (size_t)(u0 + hitk) * 32, 0, target - bb2);
                    if (fc < 32) fk = hitk;
                }
            }
            if (fk != 0xFFFFFFFFu) {
                int bb2 = (int)(sb.u_bpre[u0 + fk] - bp0);
                int v0 = bb2 + sb.u_cv0[(size_t)(u0 + fk) * 32 + fc];
                uint32_t bits = leaf_bits(ops, n, fk * GP_B + fc * 32);
                for (uint32_t j = 0; j < 32; ++j)
                    if (after_bal(bits, v0, (int)j) >= target) { endpos = fk * GP_B + fc * 32 + j + 1; break; }
            }
        }
        // a well-formed tree closes exactly at its last node
        if (endpos == 0xFFFFFFFFu || endpos > n || (pos == 0 && endpos != n)) { set_error(d, ST_STRUCT, 1, tree, pos, endpos); endpos = n; }
        d.e_end[e] = endpos;
    }
}

__global__ void k_entry_chunkmax(DevPop d, StructBufs sb) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const uint32_t nch = (ne + 31) / 32;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t ch = gw; ch < nch; ch += nw) {
        uint32_t e = ch * 32 + lane_id();
        uint32_t v = (e < ne) ? d.e_end[e] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(FULL, v, o));
        if (lane_id() == 0) sb.e_cmax[ch] = v;
    }
}

// parent(e) = nearest earlier entry of the same tree whose subtree ends at
// or after end(e): earlier entries either contain e (ancestors, end >=
// end(e)) or end before pos(e) < end(e).  A cached node's parent node is
// cached too (subtree sizes grow toward the root), so the parent entry is
// the parent node and has at most two child entries: the left one starts
// right after it.  The links are written here as well.
//
// A warp takes 32 consecutive entries and reads the 32 before them in the
// same round of loads (for 40 trees of 1e6 nodes, T = 1,024: 92 % of the
// parents lie in the same chunk, 6 % in the one before).  Lanes still
// unresolved search the chunk maxima, 32 chunks per step.
__global__ void k_entry_parents(DevPop d, StructBufs sb) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const uint32_t lane = (uint32_t)lane_id();
    const uint32_t nch = (ne + 31) / 32;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t ch = gw; ch < nch; ch += nwarp) {
        const uint32_t e = ch * 32 + lane;
        const bool valid = e < ne;
        const uint32_t tree = valid ? sb.e_tree[e] : 0xFFFFFFFFu;
        const uint32_t ee = valid ? d.e_end[e] : 0u;
        const uint32_t pos = valid ? d.e_pos[e] : 0u;
        // the previous chunk: ch * 32 <= ne - 1, so all 32 of its entries exist
        const uint32_t qb = ch * 32 - 32;
        const uint32_t qt = ch ? sb.e_tree[qb + lane] : 0xFFFFFFFEu;
        const uint32_t qe = ch ? d.e_end[qb + lane] : 0u;
        // e is its tree's first entry (the root) when e - 1 belongs to another tree
        uint32_t tp = __shfl_up_sync(FULL, tree, 1);
        const uint32_t t31 = __shfl_sync(FULL, qt, 31);
        if (lane == 0) tp = t31;
        const bool need = valid && tp == tree;
        int32_t par = -1;
        // inside the chunk, nearest first (values by shuffle)
        for (uint32_t dl = 1; dl < 32; ++dl) {
            const uint32_t ve = __shfl_up_sync(FULL, ee, dl);
            const uint32_t vt = __shfl_up_sync(FULL, tree, dl);
            if (need && par < 0 && lane >= dl && vt == tree && ve >= ee) par = (int32_t)(e - dl);
        }
        // the previous chunk, a ballot per unresolved lane
        uint32_t pend = __ballot_sync(FULL, need && par < 0);
        uint32_t rest = 0;
        while (pend) {
            const uint32_t l = (uint32_t)__ffs(pend) - 1;
            pend &= pend - 1;
            const uint32_t le = __shfl_sync(FULL, ee, l), lt = __shfl_sync(FULL, tree, l);
            const uint32_t m = __ballot_sync(FULL, qt == lt && qe >= le);
            if (m) {
                if (lane == l) par = (int32_t)(qb + 31 - __clz(m));
            } else {
                rest |= 1u << l;
            }
        }
        // earlier chunks, for one lane at a time: 32 chunk maxima per step,
        // then the nearest qualifying entry of the nearest qualifying chunk
        while (rest) {
            const uint32_t l = (uint32_t)__ffs(rest) - 1;
            rest &= rest - 1;
            const uint32_t le = __shfl_sync(FULL, ee, l), lt = __shfl_sync(FULL, tree, l);
            const uint32_t l0 = d.e_off[lt];
            const int64_t first = (int64_t)(l0 / 32);
            int32_t found = -1;
            for (int64_t top = (int64_t)ch - 2; top >= first && found < 0; top -= 32) {
                const int64_t c2 = top - (int64_t)lane;
                uint32_t m = __ballot_sync(FULL, c2 >= first && sb.e_cmax[c2] >= le);
                while (m && found < 0) {
                    const int64_t cf = top - (int64_t)(__ffs(m) - 1);      // nearest chunk left
                    m &= m - 1;
                    const uint32_t q = (uint32_t)cf * 32 + lane;
                    const uint32_t mq = __ballot_sync(FULL, q >= l0 && q < ne && d.e_end[q] >= le);
                    if (mq) found = (int32_t)((uint32_t)cf * 32 + (31 - __clz(mq)));
                }
            }
            if (lane == l) par = found;
        }
        if (valid) {
            if (need && par < 0) set_error(d, ST_STRUCT, 2, tree, pos, e - d.e_off[tree]);
            d.e_par[e] = par;
            if (par >= 0) {
                if (pos == d.e_pos[par] + 1) d.e_c0[par] = (int32_t)e;
                else d.e_c1[par] = (int32_t)e;
            }
        }
    }
}

// Every cache entry must hold a value slot once a generation's values are
// assigned; one that does not would index the pool out of bounds later, so
// it gets slot 0 and the status records the inconsistency.
__global__ void k_check_slots(DevPop d) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x)
        if (d.e_slot[e] == SLOT_NEW) { d.e_slot[e] = 0; set_error(d, ST_STRUCT, 8, d.e_tree[e], d.e_pos[e], 0); }
}

// blk_off[i] = sum_{j<i} ceil(size_j / GP_B); one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_blk_offsets(DevPop d) {
    __shared__ uint32_t wa[32];
    __shared__ int64_t wb[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) { carry = 0; d.blk_off[0] = 0; }
    __syncthreads();
    for (uint32_t base = 0; base < d.P; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint32_t a = (i < d.P) ? (d.size[i] + GP_B - 1) / GP_B : 0;
        int64_t b = 0;
        block_scan2(a, b, wa, wb);
        if (i < d.P) d.blk_off[i + 1] = a + carry;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += a;
        __syncthreads();
    }
}
