// Full interpretation of a population (Sec. 4.2), split at the cached
// skeleton: first every small subtree hanging off a cached node (in
// parallel, one warp per subtree and case block), then the cached nodes
// bottom up, then the fitness of each root.
#pragma once
#include "interp.cuh"

// Work item of entry e: the part of its subtree not covered by large
// children -- the whole subtree when both children are small, else the
// small child (its value is parked in e's slot until the skeleton pass).
__global__ void k_build_items(DevPop d, const uint32_t* __restrict__ e_tree) {
    if (halted(d)) return;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int32_t c0 = d.e_c0[e], c1 = d.e_c1[e];
        uint32_t s = 0, len = 0;
        if (c0 < 0 && c1 < 0) { s = d.e_pos[e]; len = d.e_end[e] - s; }
        else if (c0 >= 0 && c1 < 0) { s = d.e_end[c0]; len = d.e_end[e] - s; }
        else if (c0 < 0 && c1 >= 0) { s = d.e_pos[e] + 1; len = d.e_pos[c1] - s; }
        const uint32_t buf = d.buf[e_tree[e]];
        d.it_desc[e] = make_uint4(s, len, d.e_slot[e], buf);
        const uint32_t op = d.arena[(size_t)buf * d.cap + d.e_pos[e]];
        const uint32_t oslot = (c0 >= 0 && c1 >= 0) ? d.e_slot[c1] : d.e_slot[e];
        d.sk_desc[e] = make_uint4(d.e_slot[e], oslot, op | ((c0 >= 0) ? 0x100u : 0u) | ((c1 >= 0) ? 0x200u : 0u),
                                  (uint32_t)c1);
        d.order[e] = e;
    }
}

// Persistent warps over (item, case block) units.  The next unit's index
// and descriptor are fetched, and its opcodes staged, while the current
// one is interpreted (two staging buffers per warp).
template <int K, int V>
__global__ void __launch_bounds__(GP_WARPS * 32) k_eval_items(DevPop d) {
    if (halted(d)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* kc = reinterpret_cast<float*>(smem_raw);
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    fill_kc(kc, d.consts);
    fill_kb(kc + 256);
    __syncthreads();
    unsigned char* wbase = smem_raw + SmemLayout<K>::kc_bytes + (size_t)warp * SmemLayout<K>::warp_bytes((int)d.W);
    Ictx<K> c;
    c.s = reinterpret_cast<float*>(wbase);
    c.W = (int)d.W;
    c.maxd = (int)d.maxdepth;
    c.kc = kc;
    c.kb = kc + 256;
    uint8_t* const stage0 = wbase + SmemLayout<K>::stack_bytes((int)d.W);   // two buffers of STAGE_BYTES
    const uint32_t gwarp = blockIdx.x * GP_WARPS + warp;
    c.g = d.ovf + (size_t)gwarp * (d.maxdepth - d.W) * 32 * K;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const uint32_t nunits = ne * d.ncb;
    unsigned long long ops_done = 0;     // nodes interpreted (once per item, not per case block)

    auto grab = [&](uint32_t& u, uint4& desc) {
        uint32_t v = 0;
        if (lane == 0) v = atomicAdd(&d.q[Q_ITEMS], 1u);
        u = __shfl_sync(FULL, v, 0);
        desc = make_uint4(0, 0, 0, 0);
        if (u < nunits) desc = d.it_desc[d.order[u / d.ncb]];
    };
    uint32_t un;
    uint4 dn;
    grab(un, dn);
    if (un < nunits && dn.y) stage_issue(stage0, d.arena + (size_t)dn.w * d.cap, dn.x, dn.x + dn.y);
    cp_async_commit();
    int cur = 0;
    while (un < nunits) {
        const uint32_t u = un;
        const uint4 desc = dn;
        grab(un, dn);
        if (un < nunits && dn.y) stage_issue(stage0 + (cur ^ 1) * STAGE_BYTES, d.arena + (size_t)dn.w * d.cap, dn.x, dn.x + dn.y);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        if (desc.y) {
            const uint32_t cbk = u % d.ncb;
            load_cases<K>(d, cbk, c.xv);
            Istate<K> st;
#pragma unroll
            for (int k = 0; k < K; ++k) st.acc[k] = 0.f;
            st.sp = 0;
            st.ok = true;
            interp_staged<K, V>(stage0 + cur * STAGE_BYTES, desc.x, desc.x + desc.y, st, c);
            if (!st.ok && lane == 0) set_status(d.status, ST_STACK);
            store_slot<K>(d, desc.z, cbk, st.acc);
            if (cbk == 0) ops_done += desc.y;
        }
        __syncwarp();
        cur ^= 1;
    }
    cp_async_wait<0>();
    if (lane == 0 && ops_done) { atomicAdd(&d.acc_ops[0], ops_done); atomicAdd(&d.acc_ops[2], ops_done); }
}

// Cached nodes bottom up: entries of a tree in decreasing position order,
// so both children of a node are done before it.  A node with one large
// child has that child at the next entry index (no other cached node lies
// between them), a node with two has its left child there.  Entries are
// taken in groups of SKB: descriptors (prefetched one group ahead) and
// operand vectors are loaded first -- they do not depend on the running
// value -- then combined in order; a right child inside the same group is
// taken from the group's own results.
#define SKB 16
template <int K, int V>
__global__ void __launch_bounds__(GP_WARPS * 32) k_eval_skeleton(DevPop d) {
    if (halted(d)) return;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const int lane = lane_id();
    if (d.e_off[d.P] > d.Ecap) return;
    for (uint32_t tree = gw; tree < d.P; tree += nw) {
        const uint32_t e0 = d.e_off[tree], e1 = d.e_off[tree + 1];
        unsigned long long cnt = 0;
        for (uint32_t cbk = 0; cbk < d.ncb; ++cbk) {
            float prev[K];
#pragma unroll
            for (int k = 0; k < K; ++k) prev[k] = 0.f;
            uint4 md = make_uint4(0, 0, 0, 0);
            if (e1 > e0 && lane < SKB && (uint32_t)lane < e1 - e0) md = d.sk_desc[e1 - 1 - lane];
            for (uint32_t top = e1; top > e0;) {
                const uint32_t nb = (top - e0 < SKB) ? top - e0 : SKB;
                const uint32_t ntop = top - nb;
                uint4 mdn = make_uint4(0, 0, 0, 0);
                if (ntop > e0 && lane < SKB && (uint32_t)lane < ntop - e0) mdn = d.sk_desc[ntop - 1 - lane];
                float opnd[SKB][K];
                uint32_t slots[SKB], info[SKB], c1s[SKB];
#pragma unroll
                for (int j = 0; j < SKB; ++j) {
                    slots[j] = __shfl_sync(FULL, md.x, j);
                    const uint32_t os = __shfl_sync(FULL, md.y, j);
                    info[j] = __shfl_sync(FULL, md.z, j);
                    c1s[j] = __shfl_sync(FULL, md.w, j);
                    if (j < (int)nb) load_slot<K>(d, os, cbk, opnd[j]);
                }
                float done[SKB][K];
#pragma unroll
                for (int j = 0; j < SKB; ++j) {
                    if (j < (int)nb) {
                        const bool has0 = info[j] & 0x100u, has1 = info[j] & 0x200u;
                        const uint32_t op = info[j] & 0xFFu;
                        float val[K];
                        if (!has0 && !has1) {
#pragma unroll
                            for (int k = 0; k < K; ++k) val[k] = opnd[j][k];
                        } else {
                            float o[K];
#pragma unroll
                            for (int k = 0; k < K; ++k) o[k] = opnd[j][k];
                            if (has0 && has1) {
#pragma unroll
                                for (int jj = 0; jj < j; ++jj)
                                    if (c1s[j] == top - 1 - jj) {
#pragma unroll
                                        for (int k = 0; k < K; ++k) o[k] = done[jj][k];
                                    }
                            }
                            if (has0) {                       // left = entry e+1 = prev
#pragma unroll
                                for (int k = 0; k < K; ++k) val[k] = prev[k];
                                apply_vec<K, V>(op, val, o);
                            } else {                          // right = entry e+1 = prev
#pragma unroll
                                for (int k = 0; k < K; ++k) val[k] = o[k];
                                apply_vec<K, V>(op, val, prev);
                            }
                            store_slot<K>(d, slots[j], cbk, val);
                            if (cbk == 0) ++cnt;
                        }
#pragma unroll
                        for (int k = 0; k < K; ++k) { done[j][k] = val[k]; prev[k] = val[k]; }
                    }
                }
                top = ntop;
                md = mdn;
            }
        }
        if (lane == 0 && cnt) atomicAdd(&d.acc_ops[0], cnt);
    }
}

// Fitness of every tree from its root's cached vector (a warp per tree).
__global__ void k_fitness(DevPop d) {
    if (halted(d)) return;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    if (d.e_off[d.P] > d.Ecap) return;
    for (uint32_t tree = gw; tree < d.P; tree += nw) {
        const float* v = d.slots + (size_t)d.e_slot[d.e_off[tree]] * d.Cpad;
        const float f = fitness_warp(d, [&](uint32_t j) { return __ldcg(v + j); });
        if (lane_id() == 0) {
            d.fit[tree] = f;
            atomicAdd(&d.acc_ops[1], (unsigned long long)d.size[tree]);
        }
    }
}
