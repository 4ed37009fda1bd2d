// gp_eval_small_noalloc: full evaluation of a batch of small trees with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: a plug-in whose host process has
// handed the whole device memory to its own pool allocator (a cudaMalloc
// there fails, or fragments memory the host accounts for), a real-time loop
// that must not take the implicit device synchronisation an allocation can
// bring, or an embedding whose memory is fixed at start-up.  They still own
// their inputs and outputs, so this entry point takes device pointers to
// both and keeps the only scratch it needs -- the interpreter's deep-stack
// overflow area, a work counter and a status word -- in one file-scope
// device array of fixed size, loaded with the library and held by every GPU
// that loads it until the process exits.
//
// The scratch array is shared by every call on a device and keeps the
// previous call's contents; each call clears the counter and status it needs
// before launching.  Two calls whose work overlaps on the GPU (different
// streams, or one not yet finished when the next is issued on another
// stream) race on that array and give undefined results: serialise them.
// Each call synchronises its stream before it returns, to read the status.
#include "gpfdp.h"

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "interp.cuh"

namespace {

constexpr int NA_K = 2;                       // test cases per lane (64 per case block)
constexpr int NA_W = 16;                      // stack entries kept in shared memory per warp
constexpr int NA_MAX_NODES = 1023;            // largest tree: at most 512 leaves, so the stack
constexpr int NA_MAXD = NA_W + 520;           //   never holds more than 514 entries
constexpr int NA_WARPS = 4;                   // warps per CTA
constexpr int NA_CTAS = 16;                   // persistent CTAs
constexpr size_t NA_OVF_FLOATS = (size_t)NA_CTAS * NA_WARPS * (NA_MAXD - NA_W) * 32 * NA_K;
constexpr size_t NA_SCRATCH_FLOATS = NA_OVF_FLOATS + 64;   // overflow stacks, then counters
}  // namespace

// The scratch: overflow stacks of the 64 resident warps (8.5 MB: 520 entries
// x 32 lanes x 2 cases x 4 bytes each), followed by the work counter and the
// status word.
static __device__ __align__(256) float g_noalloc_scratch[NA_SCRATCH_FLOATS];

namespace {

struct NaArgs {
    const uint8_t* ops;
    size_t ops_bytes;
    const uint64_t* off;
    uint32_t n_trees;
    const float* x;
    const float* t;
    const float* consts;
    uint32_t n_cases;
    float* values;
    float* fitness;
    float* scratch;       // device address of g_noalloc_scratch
};

__global__ void __launch_bounds__(NA_WARPS * 32) k_eval_small_noalloc(NaArgs a) {
    // one block of shared memory: four stack entries of room below the first
    // stack (the interpreter's fast path may touch them on a malformed tree)
    struct NaSmem {
        float pad[4 * 32 * NA_K];
        float kc[256];
        float sstack[NA_WARPS][NA_W * 32 * NA_K];
        uint8_t stage[NA_WARPS][STAGE_BYTES];
    };
    __shared__ __align__(16) NaSmem sm;
    float* const kc = sm.kc;
    float (*const sstack)[NA_W * 32 * NA_K] = sm.sstack;
    uint8_t (*const stage)[STAGE_BYTES] = sm.stage;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    fill_kc(kc, a.consts);
    __syncthreads();
    uint32_t* counter = reinterpret_cast<uint32_t*>(a.scratch + NA_OVF_FLOATS);
    uint32_t* status = counter + 1;
    Ictx<NA_K> c;
    c.s = sstack[warp];
    c.g = a.scratch + (size_t)(blockIdx.x * NA_WARPS + warp) * (NA_MAXD - NA_W) * 32 * NA_K;
    c.kc = kc;
    c.W = NA_W;
    c.maxd = NA_MAXD;
    const uint32_t ncb = (a.n_cases + 32 * NA_K - 1) / (32 * NA_K);
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(counter, 1u);
        i = __shfl_sync(FULL, i, 0);
        if (i >= a.n_trees) break;
        const uint64_t s64 = a.off[i], e64 = a.off[i + 1];
        const uint64_t n = e64 - s64;
        // ops_bytes is a multiple of 16, so e64 <= ops_bytes also keeps the
        // staged 16-byte chunks inside the buffer (no rounding that could wrap)
        if (e64 < s64 || n == 0 || n > NA_MAX_NODES || e64 > a.ops_bytes) {
            if (lane == 0) atomicOr(status, 1u);
            continue;
        }
        // stage the tree: aligned 16-byte chunks relative to the (16-aligned) ops base
        const uint32_t s = (uint32_t)(s64 & 15u), e = s + (uint32_t)n;
        __syncwarp();
        stage_issue(stage[warp], a.ops + (s64 & ~15ull), s, e);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        float fit = 0.0f;
        for (uint32_t cb = 0; cb < ncb; ++cb) {
#pragma unroll
            for (int k = 0; k < NA_K; ++k) {
                const uint32_t cc = cb * 32 * NA_K + k * 32 + lane;
                c.xv[k] = (cc < a.n_cases) ? a.x[cc] : 0.0f;
            }
            Istate<NA_K> st;
#pragma unroll
            for (int k = 0; k < NA_K; ++k) st.acc[k] = 0.f;
            st.sp = 0;
            st.ok = true;
            interp_staged<NA_K>(stage[warp], s, e, st, c);
            if (!__all_sync(FULL, st.ok)) { if (lane == 0) atomicOr(status, 2u); }
#pragma unroll
            for (int k = 0; k < NA_K; ++k) {
                const uint32_t cc = cb * 32 * NA_K + k * 32 + lane;
                if (cc < a.n_cases) a.values[(size_t)i * a.n_cases + cc] = st.acc[k];
            }
            __syncwarp();
            // fitness in case order: lane 0 walks this block's cases through the warp
#pragma unroll
            for (int k = 0; k < NA_K; ++k) {
                for (int l = 0; l < 32; ++l) {
                    const float v = __shfl_sync(FULL, st.acc[k], l);
                    const uint32_t cc = cb * 32 * NA_K + k * 32 + l;
                    if (lane == 0 && cc < a.n_cases) fit = __fadd_rn(fit, fabsf(__fsub_rn(v, a.t[cc])));
                }
            }
        }
        if (lane == 0) a.fitness[i] = fit;
    }
}

std::mutex g_na_mu;
// device address of the scratch per device ordinal, and the context it was
// looked up in: a context destroyed and re-created (cudaDeviceReset) loads
// the module again, so the address is looked up again in the new context
float* g_na_ptr[64] = {};
void* g_na_ctx[64] = {};

// the current context through the driver entry point (no link-time
// dependency on the driver library)
typedef int (*CtxGetCurrentFn)(void**);
void* current_context() {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
        looked = true;
    }
    void* ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

}  // namespace

extern "C" int gp_eval_small_noalloc(const uint8_t* d_ops, size_t ops_bytes, const uint64_t* d_off,
                                     uint32_t n_trees, const float* d_x, const float* d_t,
                                     const float* d_consts, uint32_t n_cases, float* d_values,
                                     float* d_fitness, void* stream, uint32_t* status_out) {
    if (status_out) *status_out = 0;
    if (!d_ops || !d_off || !d_x || !d_t || !d_consts || !d_values || !d_fitness) return GP_EINVAL;
    if (n_cases == 0 || n_cases > 4096) return GP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_ops) & 15u) || (ops_bytes & 15u)) return GP_EINVAL;
    if (n_trees == 0) return GP_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GP_ECUDA;
    float* scratch = nullptr;
    {
        // set-up, once per device (and context), with that device current: the
        // host-side name of the array is not a device address, so ask the
        // runtime for it
        std::lock_guard<std::mutex> lk(g_na_mu);
        void* ctx = current_context();
        if (!g_na_ptr[dev] || !ctx || ctx != g_na_ctx[dev]) {
            void* p = nullptr;
            // (creates the device's context if it does not exist yet)
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return GP_ECUDA;
            g_na_ptr[dev] = static_cast<float*>(p);
            g_na_ctx[dev] = current_context();
        }
        scratch = g_na_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the work counter and the status word start at zero on every call
    if (cudaMemsetAsync(scratch + NA_OVF_FLOATS, 0, 64 * sizeof(float), st) != cudaSuccess) return GP_ECUDA;
    NaArgs a{d_ops, ops_bytes, d_off, n_trees, d_x, d_t, d_consts, n_cases, d_values, d_fitness, scratch};
    k_eval_small_noalloc<<<NA_CTAS, NA_WARPS * 32, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return GP_ECUDA;
    uint32_t flags = 0;
    if (cudaMemcpyAsync(&flags, scratch + NA_OVF_FLOATS + 1, sizeof flags, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GP_ECUDA;
    if (status_out) *status_out = flags;
    if (flags & 1u) return GP_ECAPACITY;
    if (flags & 2u) return GP_EINVAL;
    return GP_OK;
}
