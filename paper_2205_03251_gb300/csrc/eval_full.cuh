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
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int32_t c0 = d.e_c0[e], c1 = d.e_c1[e];
        uint32_t s = 0, len = 0;
        if (c0 < 0 && c1 < 0) { s = d.e_pos[e]; len = d.e_end[e] - s; }
        else if (c0 >= 0 && c1 < 0) { s = d.e_end[c0]; len = d.e_end[e] - s; }
        else if (c0 < 0 && c1 >= 0) { s = d.e_pos[e] + 1; len = d.e_pos[c1] - s; }
        d.it_start[e] = s;
        d.it_len[e] = len;
        d.order[e] = e;
    }
}

template <int K>
__global__ void __launch_bounds__(GP_WARPS * 32) k_eval_items(DevPop d, const uint32_t* __restrict__ e_tree) {
    extern __shared__ float smem[];
    float* kc = smem;                                      // 256 floats
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < GP_NCONST; i += blockDim.x) kc[i] = d.consts[i];
    __syncthreads();
    WarpStack<K> ws;
    ws.W = (int)d.W;
    ws.maxd = (int)d.maxdepth;
    ws.s = smem + 256 + (size_t)warp * d.W * 32 * K;
    const uint32_t gwarp = blockIdx.x * GP_WARPS + warp;
    ws.g = d.ovf + (size_t)gwarp * (d.maxdepth - d.W) * 32 * K;
    const uint32_t ne = d.e_off[d.P];
    if (ne > d.Ecap) return;
    const uint32_t nunits = ne * d.ncb;
    unsigned long long ops_done = 0;   // nodes interpreted (counted once per item, not per case block)
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(&d.q[Q_ITEMS], 1u);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        const uint32_t e = d.order[u / d.ncb];
        const uint32_t cbk = u % d.ncb;
        const uint32_t len = d.it_len[e];
        if (len == 0) continue;
        const uint32_t s = d.it_start[e];
        const uint8_t* ops = tree_ptr(d, e_tree[e]);
        float xv[K];
        load_cases<K>(d, cbk, xv);
        InterpState<K> st;
#pragma unroll
        for (int k = 0; k < K; ++k) st.acc[k] = 0.f;
        st.sp = 0;
        st.ok = true;
        interp_run<K>(ops, s, s + len, st, ws, xv, kc);
        if (!st.ok && lane == 0) set_status(d.status, ST_STACK);
        store_slot<K>(d, d.e_slot[e], cbk, st.acc);
        if (cbk == 0) ops_done += len;
    }
    if (lane == 0 && ops_done) { atomicAdd(&d.acc_ops[0], ops_done); atomicAdd(&d.acc_ops[2], ops_done); }
}

// Cached nodes bottom up: entries of a tree in decreasing position order,
// so both children of a node are done before it.  A node with one large
// child has that child at the next entry index (no other cached node lies
// between them), a node with two has its left child there.
template <int K>
__global__ void __launch_bounds__(GP_WARPS * 32) k_eval_skeleton(DevPop d) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    if (d.e_off[d.P] > d.Ecap) return;
    for (uint32_t tree = gw; tree < d.P; tree += nw) {
        const uint8_t* ops = tree_ptr(d, tree);
        const uint32_t e0 = d.e_off[tree], e1 = d.e_off[tree + 1];
        unsigned long long cnt = 0;
        for (uint32_t cbk = 0; cbk < d.ncb; ++cbk) {
            float prev[K];
#pragma unroll
            for (int k = 0; k < K; ++k) prev[k] = 0.f;
            for (uint32_t e = e1; e-- > e0;) {
                const int32_t c0 = d.e_c0[e], c1 = d.e_c1[e];
                const uint32_t slot = d.e_slot[e];
                float v[K];
                load_slot<K>(d, slot, cbk, v);
                if (c0 < 0 && c1 < 0) {
#pragma unroll
                    for (int k = 0; k < K; ++k) prev[k] = v[k];
                    continue;
                }
                const uint32_t op = ops[d.e_pos[e]];
                float val[K];
                if (c0 >= 0 && c1 >= 0) {
                    float r[K];
                    load_slot<K>(d, d.e_slot[c1], cbk, r);
#pragma unroll
                    for (int k = 0; k < K; ++k) val[k] = apply_op(op, prev[k], r[k]);
                } else if (c0 >= 0) {
#pragma unroll
                    for (int k = 0; k < K; ++k) val[k] = apply_op(op, prev[k], v[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < K; ++k) val[k] = apply_op(op, v[k], prev[k]);
                }
                store_slot<K>(d, slot, cbk, val);
#pragma unroll
                for (int k = 0; k < K; ++k) prev[k] = val[k];
                if (cbk == 0) ++cnt;
            }
        }
        if (lane_id() == 0 && cnt) atomicAdd(&d.acc_ops[0], cnt);
    }
}

// Fitness of every tree from its root's cached vector: sum over cases in
// case order of |value - target| in binary32.
__global__ void k_fitness(DevPop d) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    if (d.e_off[d.P] > d.Ecap) return;
    for (uint32_t tree = gw; tree < d.P; tree += nw) {
        if (lane_id() == 0) {
            const float* v = d.slots + (size_t)d.e_slot[d.e_off[tree]] * d.Cpad;
            float f = 0.0f;
            for (uint32_t c = 0; c < d.C; ++c) f = __fadd_rn(f, fabsf(__fsub_rn(__ldcg(v + c), d.t[c])));
            d.fit[tree] = f;
            atomicAdd(&d.acc_ops[1], (unsigned long long)d.size[tree]);
        }
    }
}
