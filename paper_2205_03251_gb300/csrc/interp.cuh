// Warp interpreter: lanes are test cases, the opcode stream is warp-uniform.
//
// The paper's AVX interpreter makes one pass over a tree and applies each
// opcode to all test cases (Sec. 4.2), using an explicit stack as deep as
// the tree is high.  Here a warp scans a run of prefix-ordered nodes from
// right to left, which visits every node after both of its children (the
// reverse of prefix order is a postfix order of the mirrored tree, cf. the
// RPN scan of Sec. 3.1), so a stack machine needs no recursion: a leaf
// pushes the running value and loads its own, a function pops its right
// operand and combines it with the running value (its left operand).
// Each lane holds K test cases; the running value is in registers, the
// next W stack entries in shared memory, deeper ones in a per-warp global
// overflow area.  The opcodes of the run are first staged into shared
// memory with cp.async (one 16-byte copy per lane per 512 bytes), so the
// interpreter reads one 32-bit word per four nodes without global latency.
//
// Arithmetic is binary32 with explicit round-to-nearest intrinsics (never
// contracted into FMA); protected division returns 1 when the divisor
// equals zero.  The same interpreter runs the Boolean multiplexer sets
// (lanes hold 32-case words) and the integer set (lanes hold int32 bits).
#pragma once
#include "common.cuh"

#define STAGE_BYTES 2112     // >= 2*1024 - 1 nodes + 15 bytes of alignment, multiple of 16

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

__device__ __forceinline__ float pdiv(float a, float b) {
    return (b == 0.0f) ? 1.0f : __fdiv_rn(a, b);
}

__device__ __forceinline__ float apply_op(uint32_t op, float a, float b) {
    switch (op) {
    case 0: return __fadd_rn(a, b);
    case 1: return __fsub_rn(a, b);
    case 2: return __fmul_rn(a, b);
    default: return pdiv(a, b);
    }
}

// Boolean multiplexer sets: 0 AND, 1 OR, 2 NAND, 3 NOR on words of 32
// cases (the value bits travel in float registers).
__device__ __forceinline__ uint32_t bool_op(uint32_t op, uint32_t x, uint32_t y) {
    uint32_t r = (op & 1u) ? (x | y) : (x & y);
    return (op & 2u) ? ~r : r;
}

// Integer set: + - * wrap around modulo 2^32; protected division returns 1
// for a zero divisor and the wrapped quotient INT32_MIN for INT32_MIN / -1,
// else the quotient truncated toward zero.
__device__ __forceinline__ int32_t int_op(uint32_t op, int32_t x, int32_t y) {
    switch (op) {
    case 0: return (int32_t)((uint32_t)x + (uint32_t)y);
    case 1: return (int32_t)((uint32_t)x - (uint32_t)y);
    case 2: return (int32_t)((uint32_t)x * (uint32_t)y);
    default:
        if (y == 0) return 1;
        if (x == INT32_MIN && y == -1) return INT32_MIN;
        return x / y;
    }
}

template <int K, int V = VF>
__device__ __forceinline__ void apply_vec(uint32_t op, float (&a)[K], const float (&b)[K]) {
    if constexpr (V == VB) {
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = __uint_as_float(bool_op(op, __float_as_uint(a[k]), __float_as_uint(b[k])));
        return;
    }
    if constexpr (V == VI) {
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = __int_as_float(int_op(op, __float_as_int(a[k]), __float_as_int(b[k])));
        return;
    }
    if (op < 2) {
        if (op == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) a[k] = __fadd_rn(a[k], b[k]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) a[k] = __fsub_rn(a[k], b[k]);
        }
    } else if (op == 2) {
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = __fmul_rn(a[k], b[k]);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) a[k] = pdiv(a[k], b[k]);
    }
}

// Per-warp interpreter context.
template <int K>
struct Ictx {
    float* s;            // shared stack: W entries x 32 lanes x K (this lane's K at s + lane*K)
    float* g;            // global overflow: (maxd - W) entries x 32 lanes x K
    const float* kc;     // shared constant table indexed by opcode (kc[5..255])
    const float* kb;     // Boolean: shared words of inputs 0..4 (mux_pattern)
    int W, maxd;
    float xv[K];         // this lane's test-case inputs (Boolean: the index of each of its words)
};

// Boolean input b (opcode 4 + b: a0.. then d0..) is bit b of the case index.
// Word w holds cases 32w .. 32w + 31, so for b < 5 the word is the same
// pattern in every word, and for b >= 5 it is all ones or all zeros by bit
// b - 5 of w.
__device__ __forceinline__ uint32_t mux_pattern(uint32_t b) {
    uint32_t x = 0;
    for (uint32_t l = 0; l < 32; ++l) x |= ((l >> b) & 1u) << l;
    return x;
}
__device__ __forceinline__ uint32_t mux_word(uint32_t b, uint32_t pattern, uint32_t w) {
    return b < 5u ? pattern : 0u - ((w >> ((b - 5u) & 31u)) & 1u);
}

template <int K, int V>
__device__ __forceinline__ void leaf_value(uint32_t op, float (&acc)[K], const Ictx<K>& c, int lane) {
    if constexpr (V == VB) {
        const uint32_t b = op - 4u;
        const uint32_t pat = __float_as_uint(c.kb[b < 5u ? b : 0u]);
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = __uint_as_float(mux_word(b, pat, __float_as_uint(c.xv[k])));
    } else {
        const float cv = c.kc[op];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = (op == 4) ? c.xv[k] : cv;
    }
}

template <int K>
struct Istate {
    float acc[K];
    int sp;              // stack depth (entries)
    bool ok;
};

// Shared-memory accesses by 32-bit shared-window address (no generic
// 64-bit pointer arithmetic on the interpreter's hot path).  They are
// volatile, so they keep their order among themselves: a push is never
// moved past the pop of the same entry.
template <int K>
__device__ __forceinline__ void sts_vec(uint32_t a, const float (&v)[K]) {
    if constexpr (K == 1) asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v[0]));
    else if constexpr (K == 2) asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v[0]), "f"(v[1]));
    else asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]));
}
template <int K>
__device__ __forceinline__ void lds_vec(uint32_t a, float (&v)[K]) {
    if constexpr (K == 1) asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v[0]) : "r"(a));
    else if constexpr (K == 2) asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "r"(a));
    else asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "r"(a));
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// One node, any stack depth (bounds checked).  The shared window is
// accessed through the same volatile helpers as the fast path (so the two
// keep their order), the overflow area through ordinary global accesses.
template <int K, int V = VF>
__device__ __forceinline__ void step_checked(uint32_t op, Istate<K>& st, const Ictx<K>& c, int lane) {
    const uint32_t sw = (uint32_t)__cvta_generic_to_shared(c.s) + (uint32_t)lane * K * 4;
    if (op >= 4) {
        if (st.sp < c.W) sts_vec<K>(sw + (uint32_t)st.sp * 32 * K * 4, st.acc);
        else if (st.sp < c.maxd) vstore<K>(c.g + ((size_t)(st.sp - c.W) * 32 + lane) * K, st.acc);
        else st.ok = false;
        if (st.sp < c.maxd) ++st.sp;
        leaf_value<K, V>(op, st.acc, c, lane);
    } else {
        float r[K];
        if (st.sp <= 0) {
            st.ok = false;
#pragma unroll
            for (int k = 0; k < K; ++k) r[k] = 0.f;
        } else {
            --st.sp;
            if (st.sp < c.W) lds_vec<K>(sw + (uint32_t)st.sp * 32 * K * 4, r);
            else vload<K>(c.g + ((size_t)(st.sp - c.W) * 32 + lane) * K, r);
        }
        apply_vec<K, V>(op, st.acc, r);
    }
}

// The binary32 node of the fast path written with branches declared
// uniform (bra.uni): the opcode is the same in every lane of the warp (all
// lanes read it from the same shared word), so no branch needs the
// reconvergence bookkeeping of a possibly divergent one.  Same operations
// on the same operands as the C++ form below: a leaf pushes the running
// value and loads x or its constant; a function pops its right operand and
// applies + (subtraction as addition of the negated operand, which IEEE 754
// defines it to be), x, or protected division (1 for a zero divisor of
// either sign, else the round-to-nearest quotient), never contracted.
#define GP_SF_LEAF_SEL(k, xk) "selp.f32 %" #k ", %" #xk ", cv, pq;\n\t"
template <int K>
__device__ __forceinline__ void step_fast_f32(uint32_t op, float (&acc)[K], uint32_t& sa, uint32_t kca,
                                              const float (&xv)[K]) {
    if constexpr (K == 1) {
        asm volatile(
            "{\n\t.reg .pred pf, pq, pz;\n\t.reg .f32 r0, cv;\n\t.reg .u32 ca;\n\t"
            "setp.lt.u32 pf, %2, 4;\n\t"
            "@pf bra.uni SF_FN;\n\t"
            "st.shared.f32 [%1], %0;\n\t"
            "add.u32 %1, %1, 128;\n\t"
            "shl.b32 ca, %2, 2;\n\tadd.u32 ca, ca, %3;\n\t"
            "ld.shared.f32 cv, [ca];\n\t"
            "setp.eq.u32 pq, %2, 4;\n\t" GP_SF_LEAF_SEL(0, 4)
            "bra.uni SF_END;\n"
            "SF_FN:\n\t"
            "sub.u32 %1, %1, 128;\n\t"
            "ld.shared.f32 r0, [%1];\n\t"
            "setp.lt.u32 pq, %2, 2;\n\t"
            "@pq bra.uni SF_AS;\n\t"
            "setp.eq.u32 pq, %2, 2;\n\t"
            "@!pq bra.uni SF_DV;\n\t"
            "mul.rn.f32 %0, %0, r0;\n\t"
            "bra.uni SF_END;\n"
            "SF_DV:\n\t"
            "setp.eq.f32 pz, r0, 0f00000000;\n\tdiv.rn.f32 %0, %0, r0;\n\t@pz mov.f32 %0, 0f3F800000;\n\t"
            "bra.uni SF_END;\n"
            "SF_AS:\n\t"
            "setp.eq.u32 pq, %2, 1;\n\t"
            "@pq neg.f32 r0, r0;\n\t"
            "add.rn.f32 %0, %0, r0;\n"
            "SF_END:\n\t}"
            : "+f"(acc[0]), "+r"(sa)
            : "r"(op), "r"(kca), "f"(xv[0]));
    } else if constexpr (K == 2) {
        asm volatile(
            "{\n\t.reg .pred pf, pq, pz;\n\t.reg .f32 r0, r1, cv;\n\t.reg .u32 ca;\n\t"
            "setp.lt.u32 pf, %3, 4;\n\t"
            "@pf bra.uni SF_FN;\n\t"
            "st.shared.v2.f32 [%2], {%0, %1};\n\t"
            "add.u32 %2, %2, 256;\n\t"
            "shl.b32 ca, %3, 2;\n\tadd.u32 ca, ca, %4;\n\t"
            "ld.shared.f32 cv, [ca];\n\t"
            "setp.eq.u32 pq, %3, 4;\n\t" GP_SF_LEAF_SEL(0, 5) GP_SF_LEAF_SEL(1, 6)
            "bra.uni SF_END;\n"
            "SF_FN:\n\t"
            "sub.u32 %2, %2, 256;\n\t"
            "ld.shared.v2.f32 {r0, r1}, [%2];\n\t"
            "setp.lt.u32 pq, %3, 2;\n\t"
            "@pq bra.uni SF_AS;\n\t"
            "setp.eq.u32 pq, %3, 2;\n\t"
            "@!pq bra.uni SF_DV;\n\t"
            "mul.rn.f32 %0, %0, r0;\n\tmul.rn.f32 %1, %1, r1;\n\t"
            "bra.uni SF_END;\n"
            "SF_DV:\n\t"
            "setp.eq.f32 pz, r0, 0f00000000;\n\tdiv.rn.f32 %0, %0, r0;\n\t@pz mov.f32 %0, 0f3F800000;\n\t"
            "setp.eq.f32 pz, r1, 0f00000000;\n\tdiv.rn.f32 %1, %1, r1;\n\t@pz mov.f32 %1, 0f3F800000;\n\t"
            "bra.uni SF_END;\n"
            "SF_AS:\n\t"
            "setp.eq.u32 pq, %3, 1;\n\t"
            "@pq neg.f32 r0, r0;\n\t@pq neg.f32 r1, r1;\n\t"
            "add.rn.f32 %0, %0, r0;\n\tadd.rn.f32 %1, %1, r1;\n"
            "SF_END:\n\t}"
            : "+f"(acc[0]), "+f"(acc[1]), "+r"(sa)
            : "r"(op), "r"(kca), "f"(xv[0]), "f"(xv[1]));
    } else {
        static_assert(K == 4, "cases per lane: 1, 2 or 4");
        asm volatile(
            "{\n\t.reg .pred pf, pq, pz;\n\t.reg .f32 r0, r1, r2, r3, cv;\n\t.reg .u32 ca;\n\t"
            "setp.lt.u32 pf, %5, 4;\n\t"
            "@pf bra.uni SF_FN;\n\t"
            "st.shared.v4.f32 [%4], {%0, %1, %2, %3};\n\t"
            "add.u32 %4, %4, 512;\n\t"
            "shl.b32 ca, %5, 2;\n\tadd.u32 ca, ca, %6;\n\t"
            "ld.shared.f32 cv, [ca];\n\t"
            "setp.eq.u32 pq, %5, 4;\n\t" GP_SF_LEAF_SEL(0, 7) GP_SF_LEAF_SEL(1, 8) GP_SF_LEAF_SEL(2, 9)
            GP_SF_LEAF_SEL(3, 10)
            "bra.uni SF_END;\n"
            "SF_FN:\n\t"
            "sub.u32 %4, %4, 512;\n\t"
            "ld.shared.v4.f32 {r0, r1, r2, r3}, [%4];\n\t"
            "setp.lt.u32 pq, %5, 2;\n\t"
            "@pq bra.uni SF_AS;\n\t"
            "setp.eq.u32 pq, %5, 2;\n\t"
            "@!pq bra.uni SF_DV;\n\t"
            "mul.rn.f32 %0, %0, r0;\n\tmul.rn.f32 %1, %1, r1;\n\tmul.rn.f32 %2, %2, r2;\n\tmul.rn.f32 %3, %3, r3;\n\t"
            "bra.uni SF_END;\n"
            "SF_DV:\n\t"
            "setp.eq.f32 pz, r0, 0f00000000;\n\tdiv.rn.f32 %0, %0, r0;\n\t@pz mov.f32 %0, 0f3F800000;\n\t"
            "setp.eq.f32 pz, r1, 0f00000000;\n\tdiv.rn.f32 %1, %1, r1;\n\t@pz mov.f32 %1, 0f3F800000;\n\t"
            "setp.eq.f32 pz, r2, 0f00000000;\n\tdiv.rn.f32 %2, %2, r2;\n\t@pz mov.f32 %2, 0f3F800000;\n\t"
            "setp.eq.f32 pz, r3, 0f00000000;\n\tdiv.rn.f32 %3, %3, r3;\n\t@pz mov.f32 %3, 0f3F800000;\n\t"
            "bra.uni SF_END;\n"
            "SF_AS:\n\t"
            "setp.eq.u32 pq, %5, 1;\n\t"
            "@pq neg.f32 r0, r0;\n\t@pq neg.f32 r1, r1;\n\t@pq neg.f32 r2, r2;\n\t@pq neg.f32 r3, r3;\n\t"
            "add.rn.f32 %0, %0, r0;\n\tadd.rn.f32 %1, %1, r1;\n\tadd.rn.f32 %2, %2, r2;\n\tadd.rn.f32 %3, %3, r3;\n"
            "SF_END:\n\t}"
            : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+r"(sa)
            : "r"(op), "r"(kca), "f"(xv[0]), "f"(xv[1]), "f"(xv[2]), "f"(xv[3]));
    }
}
#undef GP_SF_LEAF_SEL

// One node when the whole stack access stays inside the shared window;
// sa is this lane's next free stack entry, kca the constant table and kba
// the Boolean input patterns (shared-window addresses).
template <int K, int V = VF>
__device__ __forceinline__ void step_fast(uint32_t op, float (&acc)[K], uint32_t& sa, uint32_t kca, uint32_t kba,
                                          const Ictx<K>& c) {
    if constexpr (V == VF) {
        step_fast_f32<K>(op, acc, sa, kca, c.xv);
        return;
    }
    if (op >= 4) {
        sts_vec<K>(sa, acc);
        sa += 32 * K * 4;
        if constexpr (V == VB) {
            const uint32_t b = op - 4u;
            const uint32_t pat = lds_u32(kba + (b < 5u ? b : 0u) * 4);
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = __uint_as_float(mux_word(b, pat, __float_as_uint(c.xv[k])));
        } else {
            const float cv = lds_f32(kca + op * 4);
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] = (op == 4) ? c.xv[k] : cv;
        }
    } else {
        sa -= 32 * K * 4;
        float r[K];
        lds_vec<K>(sa, r);
        apply_vec<K, V>(op, acc, r);
    }
}

// Evaluate the nodes [s, e) staged at `stage` (which holds bytes from
// s & ~15 on) right to left; afterwards st.acc is the value of the subtree
// starting at s.  Words of four nodes run without per-node checks while the
// shared window has room for four pushes.  A complete subtree never pops
// below the bottom of its own stack, so the fast path does not test for
// that per node: a word that ends below the bottom (a malformed run) marks
// the run failed and leaves the fast path, so at most four entries below the
// warp's stack are touched -- every shared-memory layout keeps that much
// room below each stack -- and so does a run that does not end with exactly
// one entry (the initial running value) on the stack.
//
// `stop` (optional, as in interp_staged_lone below): a shared word that,
// once nonzero, ends the run early with *aborted set; read every 16 words.
template <int K, int V = VF>
__device__ __forceinline__ void interp_staged(const uint8_t* stage, uint32_t s, uint32_t e,
                                              Istate<K>& st, const Ictx<K>& c,
                                              const volatile uint32_t* stop = nullptr, bool* aborted = nullptr) {
    const int lane = lane_id();
    const uint32_t a = s & ~15u;
    uint32_t p = e;
    // head: single nodes down to a multiple of 4
    while (p > s && (p & 3u)) {
        --p;
        step_checked<K, V>(stage[p - a], st, c, lane);
    }
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(stage);
    const uint32_t wa = (uint32_t)__cvta_generic_to_shared(stage) - a;      // shared address of byte 0
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(c.s) + lane * K * 4;
    const uint32_t kca = (uint32_t)__cvta_generic_to_shared(c.kc);
    const uint32_t kba = (V == VB) ? (uint32_t)__cvta_generic_to_shared(c.kb) : 0u;
    const int wfast = c.W - 4;
    // one unsigned test per word: the depth is within [0, wfast] (below the
    // bottom the difference wraps to a large value)
    const uint32_t span = (uint32_t)wfast * 32 * K * 4;
    bool under = false;
    uint32_t words = 0;
    while (p >= s + 4) {
        if (stop && (++words & 15u) == 0 && *stop) { *aborted = true; return; }
        if (st.sp >= 0 && st.sp <= wfast) {
            uint32_t sa = sbase + (uint32_t)st.sp * 32 * K * 4;
            do {
                if (stop && (++words & 15u) == 0 && *stop) { *aborted = true; return; }
                const uint32_t w = lds_u32(wa + p - 4);
                step_fast<K, V>(w >> 24, st.acc, sa, kca, kba, c);
                step_fast<K, V>((w >> 16) & 0xFFu, st.acc, sa, kca, kba, c);
                step_fast<K, V>((w >> 8) & 0xFFu, st.acc, sa, kca, kba, c);
                step_fast<K, V>(w & 0xFFu, st.acc, sa, kca, kba, c);
                p -= 4;
            } while (p >= s + 4 && sa - sbase <= span);
            under |= ((int32_t)(sa - sbase) < 0);
            st.sp = (int32_t)(sa - sbase) / (32 * K * 4);
        } else {
            const uint32_t w = wp[(p - 4 - a) >> 2];
            step_checked<K, V>(w >> 24, st, c, lane);
            step_checked<K, V>((w >> 16) & 0xFFu, st, c, lane);
            step_checked<K, V>((w >> 8) & 0xFFu, st, c, lane);
            step_checked<K, V>(w & 0xFFu, st, c, lane);
            p -= 4;
        }
    }
    while (p > s) {
        --p;
        step_checked<K, V>(stage[p - a], st, c, lane);
    }
    if (under || st.sp != 1) st.ok = false;
}

// The same run with a branch-free step for warps that run nearly alone
// (the incremental walk's sibling evaluators): the stack top is kept in a
// register (t1), every node stores the running value at the free entry and
// loads the entry below the top, and selects -- not branches -- pick a
// leaf's value or the function's result (only a division branches).  A
// lone warp takes about a fifth fewer cycles per node; with many warps per
// SM the extra instructions cost more than the branches, so the full
// evaluation keeps interp_staged.  Same operations on the same operands:
// the values are the same bits.
template <int K, int V>
__device__ __forceinline__ void apply_sel(uint32_t op, const float (&a)[K], const float (&b)[K], float (&r)[K]) {
    if constexpr (V == VB) {
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] = __uint_as_float(bool_op(op, __float_as_uint(a[k]), __float_as_uint(b[k])));
    } else if constexpr (V == VI) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t x = __float_as_uint(a[k]), y = __float_as_uint(b[k]);
            const uint32_t ad = x + ((op == 1) ? 0u - y : y);
            r[k] = __uint_as_float((op == 2) ? x * y : ad);
        }
        if (op == 3) {
#pragma unroll
            for (int k = 0; k < K; ++k) r[k] = __int_as_float(int_op(3, __float_as_int(a[k]), __float_as_int(b[k])));
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float ad = __fadd_rn(a[k], (op == 1) ? -b[k] : b[k]);
            const float mu = __fmul_rn(a[k], b[k]);
            r[k] = (op == 2) ? mu : ad;
        }
        if (op == 3) {
#pragma unroll
            for (int k = 0; k < K; ++k) r[k] = pdiv(a[k], b[k]);
        }
    }
}

// `stop` (optional): a shared word that, once nonzero, means the value is
// no longer wanted (a walk that has stopped below this sibling's level); it
// is read every 16 words and the run then ends early with *aborted set.
template <int K, int V>
__device__ __forceinline__ void interp_staged_lone(const uint8_t* stage, uint32_t s, uint32_t e, Istate<K>& st,
                                                   const Ictx<K>& c, const volatile uint32_t* stop = nullptr,
                                                   bool* aborted = nullptr) {
    const int lane = lane_id();
    const uint32_t a = s & ~15u;
    uint32_t p = e;
    while (p > s && (p & 3u)) {
        --p;
        step_checked<K, V>(stage[p - a], st, c, lane);
    }
    const uint32_t wa = (uint32_t)__cvta_generic_to_shared(stage) - a;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(c.s) + lane * K * 4;
    const uint32_t kca = (uint32_t)__cvta_generic_to_shared(c.kc);
    const uint32_t kba = (V == VB) ? (uint32_t)__cvta_generic_to_shared(c.kb) : 0u;
    const int wfast = c.W - 4;
    const uint32_t stride = 32 * K * 4;
    const uint32_t sfast = sbase + (uint32_t)wfast * stride;
    bool under = false;
    uint32_t words = 0;
    while (p >= s + 4) {
        if (stop && (++words & 15u) == 0 && *stop) { *aborted = true; return; }
        if (st.sp >= 0 && st.sp <= wfast) {
            uint32_t sa = sbase + (uint32_t)st.sp * stride;
            float t1[K];
            lds_vec<K>(sa - stride, t1);        // the top entry (below the base when the stack is empty: unused)
            do {
                if (stop && (++words & 15u) == 0 && *stop) { *aborted = true; return; }
                const uint32_t w = lds_u32(wa + p - 4);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t op = (w >> (24 - 8 * i)) & 0xFFu;
                    const bool leaf = op >= 4;
                    float lv[K];
                    if constexpr (V == VB) {
                        const uint32_t b = op - 4u;
                        const uint32_t pat = lds_u32(kba + (b < 5u ? b : 0u) * 4);
#pragma unroll
                        for (int k = 0; k < K; ++k) lv[k] = __uint_as_float(mux_word(b, pat, __float_as_uint(c.xv[k])));
                    } else {
                        const float cv = lds_f32(kca + op * 4);
#pragma unroll
                        for (int k = 0; k < K; ++k) lv[k] = (op == 4) ? c.xv[k] : cv;
                    }
                    sts_vec<K>(sa, st.acc);
                    float top2[K];
                    lds_vec<K>(sa - 2 * stride, top2);
                    float fn[K];
                    apply_sel<K, V>(op, st.acc, t1, fn);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float old = st.acc[k];
                        st.acc[k] = leaf ? lv[k] : fn[k];
                        t1[k] = leaf ? old : top2[k];
                    }
                    sa = leaf ? sa + stride : sa - stride;
                }
                under |= ((int32_t)(sa - sbase) < 0);
                p -= 4;
            } while (p >= s + 4 && (int32_t)(sa - sfast) <= 0 && (int32_t)(sa - sbase) >= 0);
            st.sp = (int32_t)(sa - sbase) / (32 * K * 4);
        } else {
            const uint32_t w = lds_u32(wa + p - 4);
            step_checked<K, V>(w >> 24, st, c, lane);
            step_checked<K, V>((w >> 16) & 0xFFu, st, c, lane);
            step_checked<K, V>((w >> 8) & 0xFFu, st, c, lane);
            step_checked<K, V>(w & 0xFFu, st, c, lane);
            p -= 4;
        }
    }
    while (p > s) {
        --p;
        step_checked<K, V>(stage[p - a], st, c, lane);
    }
    if (under || st.sp != 1) st.ok = false;
}

// interp_staged over one piece [lo, hi) of a tree (lo a multiple of 16,
// `stage` holding bytes lo .. hi - 1) that also hands out the value of
// chosen nodes: cap(k) is called (warp-uniformly) right after node pos(k)
// is evaluated, when st.acc holds the value of the subtree starting there;
// the positions pos(0) > pos(1) > ... (ncap of them) are visited in that
// order, since the scan runs right to left.  The pieces of a tree are
// taken right to left, the state (st, the cursor, `under`) carried from one
// to the next; after the last one (lo = 0) the caller checks
// `under || st.sp != 1`.  Words of four nodes that hold no chosen node take
// the unchecked fast path.
struct CaptureCursor {
    uint32_t k;          // captures done
    int32_t nextp;       // position of the next one, or -1
};

template <int K, int V, typename PosF, typename CapF>
__device__ __forceinline__ void interp_capture_range(const uint8_t* stage, uint32_t lo, uint32_t hi, Istate<K>& st,
                                                     const Ictx<K>& c, uint32_t ncap, CaptureCursor& cur,
                                                     bool& under, PosF pos, CapF cap) {
    const int lane = lane_id();
    auto after = [&](uint32_t p) {
        if ((int32_t)p == cur.nextp) {
            cap(cur.k);
            ++cur.k;
            cur.nextp = (cur.k < ncap) ? (int32_t)pos(cur.k) : -1;
        }
    };
    uint32_t p = hi;
    while (p > lo && (p & 3u)) {
        --p;
        step_checked<K, V>(stage[p - lo], st, c, lane);
        after(p);
    }
    const uint32_t wa = (uint32_t)__cvta_generic_to_shared(stage) - lo;      // shared address of byte 0
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(c.s) + lane * K * 4;
    const uint32_t kca = (uint32_t)__cvta_generic_to_shared(c.kc);
    const uint32_t kba = (V == VB) ? (uint32_t)__cvta_generic_to_shared(c.kb) : 0u;
    const int wfast = c.W - 4;
    const uint32_t span = (uint32_t)wfast * 32 * K * 4;
    while (p >= lo + 4) {
        if (cur.nextp >= (int32_t)p - 4) {
            // a chosen node in this word: node by node
            const uint32_t w = lds_u32(wa + p - 4);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                --p;
                step_checked<K, V>((w >> (24 - 8 * i)) & 0xFFu, st, c, lane);
                after(p);
            }
        } else if (st.sp >= 0 && st.sp <= wfast) {
            uint32_t sa = sbase + (uint32_t)st.sp * 32 * K * 4;
            do {
                const uint32_t w = lds_u32(wa + p - 4);
                step_fast<K, V>(w >> 24, st.acc, sa, kca, kba, c);
                step_fast<K, V>((w >> 16) & 0xFFu, st.acc, sa, kca, kba, c);
                step_fast<K, V>((w >> 8) & 0xFFu, st.acc, sa, kca, kba, c);
                step_fast<K, V>(w & 0xFFu, st.acc, sa, kca, kba, c);
                p -= 4;
            } while (p >= lo + 4 && cur.nextp < (int32_t)p - 4 && sa - sbase <= span);
            under |= ((int32_t)(sa - sbase) < 0);
            st.sp = (int32_t)(sa - sbase) / (32 * K * 4);
        } else {
            const uint32_t w = lds_u32(wa + p - 4);
            step_checked<K, V>(w >> 24, st, c, lane);
            step_checked<K, V>((w >> 16) & 0xFFu, st, c, lane);
            step_checked<K, V>((w >> 8) & 0xFFu, st, c, lane);
            step_checked<K, V>(w & 0xFFu, st, c, lane);
            p -= 4;
        }
    }
    while (p > lo) {
        --p;
        step_checked<K, V>(stage[p - lo], st, c, lane);
        after(p);
    }
}

// ---- staging with cp.async (16 bytes per lane per instruction) ----

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the copy of bytes [s & ~15, roundup16(e)) of `tree` into `stage`.
// The tree buffer's capacity is a multiple of 16, so the rounded range
// stays inside it.  Requires e - (s & ~15) <= STAGE_BYTES.
__device__ __forceinline__ void stage_issue(uint8_t* stage, const uint8_t* tree, uint32_t s, uint32_t e) {
    const int lane = lane_id();
    const uint32_t a = s & ~15u, b = (e + 15u) & ~15u;
    for (uint32_t q = a + 16u * lane; q < b; q += 512u) cp_async16(stage + (q - a), tree + q);
}

template <int K>
__device__ __forceinline__ void load_cases(const DevPop& d, uint32_t cbk, float (&xv)[K]) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t j = cbk * 32 * K + k * 32 + lane;
        xv[k] = (d.vkind == VB) ? __uint_as_float(j) : d.x[j];
    }
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

// Shared-memory layout of a CTA running the interpreter.
template <int K>
struct SmemLayout {
    // constants, then Boolean inputs, padded to four stack entries (at K = 4)
    // so that a malformed run's underflow stays inside the CTA's memory
    static constexpr size_t kc_bytes = (256 + 6 * 32) * sizeof(float) + 4 * 32 * 4 * sizeof(float);
    __host__ __device__ static size_t stack_bytes(int W) { return (size_t)W * 32 * K * sizeof(float); }
    __host__ __device__ static size_t warp_bytes(int W) { return stack_bytes(W) + 2 * STAGE_BYTES; }
    __host__ __device__ static size_t total(int W, int warps) { return kc_bytes + warps * warp_bytes(W); }
};

// kb[b] = the word of Boolean input b < 5 (the same in every word)
__device__ __forceinline__ void fill_kb(float* kb) {
    for (int i = threadIdx.x; i < 5; i += blockDim.x) kb[i] = __uint_as_float(mux_pattern((uint32_t)i));
}

// Fill the opcode-indexed constant table (kc[5 + i] = consts[i]).
__device__ __forceinline__ void fill_kc(float* kc, const float* consts) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) kc[i] = (i >= 5) ? consts[i - 5] : 0.0f;
}
