// Warp interpreter: lanes are test cases, the opcode stream is warp-uniform.
//
// The paper's AVX interpreter makes one pass over a tree and applies each
// opcode to all test cases (Sec. 4.2), using an explicit stack as deep as
// the tree is high.  Here a warp scans a run of prefix-ordered nodes from
// right to left, which visits every node after both of its children (the
// reverse of prefix order is a postfix order of the mirrored tree, cf. the
// RPN scan of Sec. 3.1), so a stack machine needs no recursion: a leaf
// pushes, a function pops its right operand and combines it with the
// running value (the left operand).  Each lane holds K test cases; the top
// of the stack is in registers, the next W entries in shared memory and
// deeper entries in a per-warp global overflow area.
//
// Arithmetic is binary32 with explicit round-to-nearest intrinsics (never
// contracted into FMA); protected division returns 1 when the divisor
// equals zero.
#pragma once
#include "common.cuh"

template <int K> struct VecT;
template <> struct VecT<1> { typedef float type; };
template <> struct VecT<2> { typedef float2 type; };
template <> struct VecT<4> { typedef float4 type; };

template <int K>
__device__ __forceinline__ void vstore(float* p, const float (&v)[K]) {
    if constexpr (K == 1) { p[0] = v[0]; }
    else if constexpr (K == 2) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
    else { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
}
template <int K>
__device__ __forceinline__ void vload(const float* p, float (&v)[K]) {
    if constexpr (K == 1) { v[0] = p[0]; }
    else if constexpr (K == 2) { float2 t = *reinterpret_cast<const float2*>(p); v[0] = t.x; v[1] = t.y; }
    else { float4 t = *reinterpret_cast<const float4*>(p); v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
}

__device__ __forceinline__ float apply_op(uint32_t op, float a, float b) {
    switch (op) {
    case 0: return __fadd_rn(a, b);
    case 1: return __fsub_rn(a, b);
    case 2: return __fmul_rn(a, b);
    default: return (b == 0.0f) ? 1.0f : __fdiv_rn(a, b);
    }
}

template <int K>
struct WarpStack {
    float* s;     // shared: W entries x 32 lanes x K
    float* g;     // global overflow: (maxd - W) entries x 32 lanes x K
    int W;
    int maxd;
};

template <int K>
struct InterpState {
    float acc[K];
    int sp;
    bool ok;
};

template <int K>
__device__ __forceinline__ void interp_step(uint32_t op, InterpState<K>& st, const WarpStack<K>& ws,
                                            const float (&xv)[K], const float* __restrict__ kc, int lane) {
    if (op >= 4) {
        if (st.sp < ws.W) vstore<K>(ws.s + ((size_t)st.sp * 32 + lane) * K, st.acc);
        else if (st.sp < ws.maxd) vstore<K>(ws.g + ((size_t)(st.sp - ws.W) * 32 + lane) * K, st.acc);
        else st.ok = false;
        st.sp += (st.sp < ws.maxd) ? 1 : 0;
        if (op == 4) {
#pragma unroll
            for (int k = 0; k < K; ++k) st.acc[k] = xv[k];
        } else {
            float c = kc[op - 5];
#pragma unroll
            for (int k = 0; k < K; ++k) st.acc[k] = c;
        }
    } else {
        float r[K];
        if (st.sp <= 0) {
            st.ok = false;
#pragma unroll
            for (int k = 0; k < K; ++k) r[k] = 0.f;
        } else {
            --st.sp;
            if (st.sp < ws.W) vload<K>(ws.s + ((size_t)st.sp * 32 + lane) * K, r);
            else vload<K>(ws.g + ((size_t)(st.sp - ws.W) * 32 + lane) * K, r);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) st.acc[k] = apply_op(op, st.acc[k], r[k]);
    }
}

__device__ __forceinline__ uint32_t byte_of(const uint4& w, int j) {
    uint32_t word = (j < 4) ? w.x : (j < 8) ? w.y : (j < 12) ? w.z : w.w;
    return (word >> (8 * (j & 3))) & 0xFFu;
}

// Evaluate ops[s..e) right to left; on return st.acc holds the value of
// the subtree starting at s (the leftmost of the run).  The buffer must be
// readable in whole aligned 16-byte chunks around [s, e).
template <int K>
__device__ __forceinline__ void interp_run(const uint8_t* __restrict__ ops, uint32_t s, uint32_t e,
                                           InterpState<K>& st, const WarpStack<K>& ws,
                                           const float (&xv)[K], const float* __restrict__ kc) {
    const int lane = lane_id();
    if (e <= s) return;
    uint32_t cb = (e - 1) & ~15u;
    uint4 w = __ldg(reinterpret_cast<const uint4*>(ops + cb));
    uint32_t p = e;
    for (;;) {
        const uint32_t lo = cb > s ? cb : s;
        uint4 wn = w;
        if (lo > s) wn = __ldg(reinterpret_cast<const uint4*>(ops + cb - 16));   // next chunk, early
        if (lo == cb && p == cb + 16) {
#pragma unroll
            for (int j = 15; j >= 0; --j) interp_step<K>(byte_of(w, j), st, ws, xv, kc, lane);
        } else {
#pragma unroll
            for (int j = 15; j >= 0; --j) {
                const uint32_t pos = cb + j;
                if (pos >= lo && pos < p) interp_step<K>(byte_of(w, j), st, ws, xv, kc, lane);
            }
        }
        if (lo <= s) break;
        p = lo;
        cb -= 16;
        w = wn;
    }
}

template <int K>
__device__ __forceinline__ void load_cases(const DevPop& d, uint32_t cbk, float (&xv)[K]) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 0; k < K; ++k) xv[k] = d.x[cbk * 32 * K + k * 32 + lane];
}

// value vector of slot `slot`, case block cbk, as this lane's K cases
template <int K>
__device__ __forceinline__ void load_slot(const DevPop& d, uint32_t slot, uint32_t cbk, float (&v)[K]) {
    const int lane = lane_id();
    const float* p = d.slots + (size_t)slot * d.Cpad + cbk * 32 * K + lane;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = __ldcg(p + k * 32);
}

template <int K>
__device__ __forceinline__ void store_slot(const DevPop& d, uint32_t slot, uint32_t cbk, const float (&v)[K]) {
    const int lane = lane_id();
    float* p = d.slots + (size_t)slot * d.Cpad + cbk * 32 * K + lane;
#pragma unroll
    for (int k = 0; k < K; ++k) p[k * 32] = v[k];
}
