// Learned work packing: a 16 -> 64 -> 64 -> 1 MLP (ReLU) predicts how many
// levels each child's incremental walk will evaluate, from features known
// before the walk; the walk's queue is ordered longest first (Sec. 3: long
// tasks first; Sec. 4.1: one slow evaluation can hold up the population).
// Trained online on the levels the walks actually took: forward, backward
// and an Adam update in plain FP32 kernels; inference uses a BF16 copy of
// the weights with FP32 accumulation.  The order never changes a result --
// every child's walk is independent.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

#define MLP_IN 16
#define MLP_H 64
// parameter layout (floats)
#define MLP_W1 0                               // [64][16]
#define MLP_B1 (MLP_W1 + MLP_H * MLP_IN)       // [64]
#define MLP_W2 (MLP_B1 + MLP_H)                // [64][64]
#define MLP_B2 (MLP_W2 + MLP_H * MLP_H)        // [64]
#define MLP_W3 (MLP_B2 + MLP_H)                // [64]
#define MLP_B3 (MLP_W3 + MLP_H)                // [1]
#define MLP_NP (MLP_B3 + 1)                    // 5313
#define MLP_CH 32                              // samples per chunk of the gradient sums

struct MlpBufs {
    float* w;          // [MLP_NP] FP32 master weights
    float* m;          // Adam first moment
    float* v;          // Adam second moment
    __nv_bfloat16* wb; // BF16 inference copy
    float* grad;       // [MLP_NP]
    float* feat;       // [N][16]
    float* pred;       // [N] training forward output
    float* pred_pack;  // [N] BF16 inference output used for packing
    float* target;     // [N]
    float* h1;         // [N][64] post-ReLU
    float* h2;         // [N][64]
    float* dy;         // [N]
    float* dh2;        // [N][64]
    float* dh1;        // [N][64]
    float* loss;       // [1]
    float* part;       // [ceil(N / MLP_CH)][MLP_NP] per-chunk gradient sums
    uint32_t* step;    // [1] Adam step counter
    uint32_t cap;
};

// Weights staged in shared memory for warp-per-sample passes: W1 transposed
// ([16][64], so that lane j reads unit j's weights without bank conflicts),
// W2 both ways ([64][64] row-major for the backward pass, transposed for the
// forward pass), biases and the output layer.
struct MlpSmem {
    float w1t[MLP_IN * MLP_H];
    float b1[MLP_H];
    float w2[MLP_H * MLP_H];
    float w2t[MLP_H * MLP_H];
    float b2[MLP_H];
    float w3[MLP_H];
    float b3;
};

template <bool BF16>
__device__ void mlp_stage(MlpSmem& m, const MlpBufs& b) {
    for (uint32_t p = threadIdx.x; p < MLP_NP; p += blockDim.x) {
        const float w = BF16 ? __bfloat162float(b.wb[p]) : b.w[p];
        if (p < MLP_B1) m.w1t[(p % MLP_IN) * MLP_H + p / MLP_IN] = w;
        else if (p < MLP_W2) m.b1[p - MLP_B1] = w;
        else if (p < MLP_B2) {
            const uint32_t q = p - MLP_W2;
            m.w2[q] = w;
            m.w2t[(q % MLP_H) * MLP_H + q / MLP_H] = w;
        } else if (p < MLP_W3) m.b2[p - MLP_B2] = w;
        else if (p < MLP_B3) m.w3[p - MLP_W3] = w;
        else m.b3 = w;
    }
}

// One sample by one warp: lane l < 16 holds feature l (xv), and lane l
// holds hidden units l and l + 32 of both layers; returns the output (all
// lanes).
__device__ __forceinline__ float mlp_forward_lanes(const MlpSmem& m, float xv, float& h1a, float& h1b, float& h2a,
                                                   float& h2b) {
    const int lane = lane_id();
    float a0 = m.b1[lane], a1 = m.b1[lane + 32];
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) {
        const float xf = __shfl_sync(FULL, xv, f);
        a0 = fmaf(m.w1t[f * MLP_H + lane], xf, a0);
        a1 = fmaf(m.w1t[f * MLP_H + lane + 32], xf, a1);
    }
    h1a = a0 > 0.f ? a0 : 0.f;
    h1b = a1 > 0.f ? a1 : 0.f;
    float c0 = m.b2[lane], c1 = m.b2[lane + 32];
#pragma unroll 8
    for (int k = 0; k < MLP_H; ++k) {
        const float hk = __shfl_sync(FULL, k < 32 ? h1a : h1b, k & 31);
        c0 = fmaf(m.w2t[k * MLP_H + lane], hk, c0);
        c1 = fmaf(m.w2t[k * MLP_H + lane + 32], hk, c1);
    }
    h2a = c0 > 0.f ? c0 : 0.f;
    h2b = c1 > 0.f ? c1 : 0.f;
    float y = fmaf(m.w3[lane], h2a, m.w3[lane + 32] * h2b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(FULL, y, o);
    return y + m.b3;
}

// The same with the sample's 16 features at x (global memory).
__device__ __forceinline__ float mlp_forward_warp(const MlpSmem& m, const float* __restrict__ x, float& h1a,
                                                  float& h1b, float& h2a, float& h2b) {
    const int lane = lane_id();
    return mlp_forward_lanes(m, lane < MLP_IN ? x[lane] : 0.f, h1a, h1b, h2a, h2b);
}

// Training pass over the batch (FP32 master weights): forward, keeping the
// activations, then dL/dy for loss = mean (y - t)^2 and the activation
// gradients dh2 = dy * w3 * [h2 > 0], dh1 = (W2^T dh2) * [h1 > 0].
__global__ void __launch_bounds__(256) k_mlp_train_pass(MlpBufs b, uint32_t n) {
    __shared__ MlpSmem m;
    mlp_stage<false>(m, b);
    __syncthreads();
    const int lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t s = gw; s < n; s += nwarps) {
        float h1a, h1b, h2a, h2b;
        const float y = mlp_forward_warp(m, b.feat + (size_t)s * MLP_IN, h1a, h1b, h2a, h2b);
        float* H1 = b.h1 + (size_t)s * MLP_H;
        float* H2 = b.h2 + (size_t)s * MLP_H;
        H1[lane] = h1a; H1[lane + 32] = h1b;
        H2[lane] = h2a; H2[lane + 32] = h2b;
        const float dy = 2.f * (y - b.target[s]) / (float)n;
        if (lane == 0) { b.pred[s] = y; b.dy[s] = dy; }
        const float d2a = h2a > 0.f ? dy * m.w3[lane] : 0.f;
        const float d2b = h2b > 0.f ? dy * m.w3[lane + 32] : 0.f;
        float* D2 = b.dh2 + (size_t)s * MLP_H;
        D2[lane] = d2a; D2[lane + 32] = d2b;
        float e0 = 0.f, e1 = 0.f;
#pragma unroll 8
        for (int j = 0; j < MLP_H; ++j) {
            const float dj = __shfl_sync(FULL, j < 32 ? d2a : d2b, j & 31);
            e0 = fmaf(m.w2[j * MLP_H + lane], dj, e0);
            e1 = fmaf(m.w2[j * MLP_H + lane + 32], dj, e1);
        }
        float* D1 = b.dh1 + (size_t)s * MLP_H;
        D1[lane] = h1a > 0.f ? e0 : 0.f;
        D1[lane + 32] = h1b > 0.f ? e1 : 0.f;
    }
}

// Parameter gradients, in two steps: per chunk of MLP_CH samples (staged in
// shared memory) every parameter's sum over the chunk in sample order, then
// the chunks' sums added in chunk order.
struct MlpChunk {
    float feat[MLP_CH][MLP_IN];
    float h1[MLP_CH][MLP_H];
    float h2[MLP_CH][MLP_H];
    float dh1[MLP_CH][MLP_H];
    float dh2[MLP_CH][MLP_H];
    float dy[MLP_CH];
};

__global__ void __launch_bounds__(256) k_mlp_grad_chunks(MlpBufs b, uint32_t n) {
    __shared__ MlpChunk ch;
    const uint32_t nch = (n + MLP_CH - 1) / MLP_CH;
    for (uint32_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const uint32_t s0 = c * MLP_CH, ns = min((uint32_t)MLP_CH, n - s0);
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < ns * MLP_IN; k += blockDim.x) ch.feat[k / MLP_IN][k % MLP_IN] = b.feat[(size_t)s0 * MLP_IN + k];
        for (uint32_t k = threadIdx.x; k < ns * MLP_H; k += blockDim.x) {
            const size_t g = (size_t)s0 * MLP_H + k;
            ch.h1[k / MLP_H][k % MLP_H] = b.h1[g];
            ch.h2[k / MLP_H][k % MLP_H] = b.h2[g];
            ch.dh1[k / MLP_H][k % MLP_H] = b.dh1[g];
            ch.dh2[k / MLP_H][k % MLP_H] = b.dh2[g];
        }
        for (uint32_t k = threadIdx.x; k < ns; k += blockDim.x) ch.dy[k] = b.dy[s0 + k];
        __syncthreads();
        float* out = b.part + (size_t)c * MLP_NP;
        for (uint32_t p = threadIdx.x; p < MLP_NP; p += blockDim.x) {
            float gsum = 0.f;
            if (p < MLP_B1) {
                const uint32_t j = p / MLP_IN, f = p % MLP_IN;
                for (uint32_t t = 0; t < ns; ++t) gsum = fmaf(ch.dh1[t][j], ch.feat[t][f], gsum);
            } else if (p < MLP_W2) {
                const uint32_t j = p - MLP_B1;
                for (uint32_t t = 0; t < ns; ++t) gsum += ch.dh1[t][j];
            } else if (p < MLP_B2) {
                const uint32_t j = (p - MLP_W2) / MLP_H, k = (p - MLP_W2) % MLP_H;
                for (uint32_t t = 0; t < ns; ++t) gsum = fmaf(ch.dh2[t][j], ch.h1[t][k], gsum);
            } else if (p < MLP_W3) {
                const uint32_t j = p - MLP_B2;
                for (uint32_t t = 0; t < ns; ++t) gsum += ch.dh2[t][j];
            } else if (p < MLP_B3) {
                const uint32_t j = p - MLP_W3;
                for (uint32_t t = 0; t < ns; ++t) gsum = fmaf(ch.dy[t], ch.h2[t][j], gsum);
            } else {
                for (uint32_t t = 0; t < ns; ++t) gsum += ch.dy[t];
            }
            out[p] = gsum;
        }
    }
}

__global__ void k_mlp_grad_reduce(MlpBufs b, uint32_t n) {
    const uint32_t nch = (n + MLP_CH - 1) / MLP_CH;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NP; p += gridDim.x * blockDim.x) {
        float gsum = 0.f;
        for (uint32_t c = 0; c < nch; ++c) gsum += b.part[(size_t)c * MLP_NP + p];
        b.grad[p] = gsum;
    }
}

__global__ void k_mlp_loss(MlpBufs b, uint32_t n) {
    if (blockIdx.x != 0) return;
    __shared__ float red[256];
    float a = 0.f;
    for (uint32_t s = threadIdx.x; s < n; s += blockDim.x) {
        const float e = b.pred[s] - b.target[s];
        a += e * e;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *b.loss = red[0] / (float)(n ? n : 1);
}

// Adam (Kingma and Ba 2015), then refresh the BF16 inference copy.
__global__ void k_mlp_adam(MlpBufs b, float lr) {
    const uint32_t t = *b.step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NP; p += gridDim.x * blockDim.x) {
        const float g = b.grad[p];
        const float m = b1 * b.m[p] + (1.f - b1) * g;
        const float v = b2 * b.v[p] + (1.f - b2) * g * g;
        b.m[p] = m;
        b.v[p] = v;
        const float w = b.w[p] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        b.w[p] = w;
        b.wb[p] = __float2bfloat16_rn(w);
    }
}

__global__ void k_mlp_bump(MlpBufs b) { if (threadIdx.x == 0 && blockIdx.x == 0) *b.step += 1; }

// Inference with the BF16 copy of the weights (staged in shared memory as
// FP32), one sample per warp.
__global__ void __launch_bounds__(256) k_mlp_infer(MlpBufs b, uint32_t n, float* __restrict__ out) {
    __shared__ MlpSmem m;
    mlp_stage<true>(m, b);
    __syncthreads();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t s = gw; s < n; s += nwarps) {
        float h1a, h1b, h2a, h2b;
        const float y = mlp_forward_warp(m, b.feat + (size_t)s * MLP_IN, h1a, h1b, h2a, h2b);
        if (lane_id() == 0) out[s] = y;
    }
}

// Deterministic initialisation (He-uniform from a counter hash).
__global__ void k_mlp_init(MlpBufs b, uint64_t seed) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NP; p += gridDim.x * blockDim.x) {
        uint64_t z = seed + (p + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float u = (float)(z >> 40) * (1.0f / 16777216.0f) * 2.f - 1.f;
        float w = 0.f;
        if (p < MLP_B1) w = u * sqrtf(6.f / MLP_IN);
        else if (p >= MLP_W2 && p < MLP_B2) w = u * sqrtf(6.f / MLP_H);
        else if (p >= MLP_W3 && p < MLP_B3) w = u * sqrtf(6.f / MLP_H);
        b.w[p] = w;
        b.m[p] = 0.f;
        b.v[p] = 0.f;
        b.wb[p] = __float2bfloat16_rn(w);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *b.step = 0;
}

#define SORT_MAX 16384     // work orders of larger populations are the identity
#define RANK_TILE 1024     // keys compared by one CTA

// Descending order of n keys (NaN as -infinity; equal keys by index) by
// ranks: the rank of key i is the number of keys that come before it, so
// order[rank(i)] = i.  A CTA takes 256 keys and a tile of RANK_TILE keys to
// compare them with (staged in shared memory) and adds its partial counts;
// the grid spreads the n^2 comparisons over the GPU instead of running the
// log^2 n barrier stages of a one-block sort.  rank[] starts at zero.
__device__ __forceinline__ float sort_key(const float* key, uint32_t i) {
    const float k = key[i];
    return isnan(k) ? -INFINITY : k;
}

__global__ void __launch_bounds__(256) k_rank_desc(const float* __restrict__ key, uint32_t n, uint32_t* __restrict__ rank) {
    __shared__ float kt[RANK_TILE];
    const uint32_t t0 = blockIdx.y * RANK_TILE;
    const uint32_t tn = min((uint32_t)RANK_TILE, n - t0);
    for (uint32_t j = threadIdx.x; j < tn; j += blockDim.x) kt[j] = sort_key(key, t0 + j);
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ki = sort_key(key, i);
    uint32_t r = 0;
    for (uint32_t j = 0; j < tn; ++j) {
        const float kj = kt[j];
        r += (kj > ki || (kj == ki && t0 + j < i)) ? 1u : 0u;
    }
    if (r) atomicAdd(&rank[i], r);
}

__global__ void k_rank_scatter(const uint32_t* __restrict__ rank, uint32_t n, uint32_t* __restrict__ order) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) order[rank[i]] = i;
}

// The same order for n <= RANK_SMALL keys in one CTA: every thread ranks its
// keys against all n (staged in shared memory) and writes them to their
// places, one launch instead of a clear, the ranks and the scatter.
#define RANK_SMALL 1024
__global__ void __launch_bounds__(1024) k_rank_small(const float* __restrict__ key, uint32_t n,
                                                     uint32_t* __restrict__ order) {
    __shared__ float kt[RANK_SMALL];
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) kt[j] = sort_key(key, j);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float ki = kt[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < n; ++j) {
            const float kj = kt[j];
            r += (kj > ki || (kj == ki && j < i)) ? 1u : 0u;
        }
        order[r] = i;
    }
}
