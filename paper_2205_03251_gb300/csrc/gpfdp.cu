// gpfdp: C-ABI of the GB300 GP population evaluator (see include/gpfdp.h).
#include "gpfdp.h"

#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "structure.cuh"
#include "interp.cuh"
#include "eval_full.cuh"
#include "generation.cuh"

static_assert(sizeof(DisLevel) == sizeof(gp_disruption_level) &&
                  offsetof(DisLevel, sq) == offsetof(gp_disruption_level, sum_sq),
              "disruption record layout");

namespace {

thread_local std::string g_create_error;

enum Phase { PH_STRUCT = 0, PH_ITEMS, PH_SKEL, PH_FIT, PH_XO, PH_WALK, PH_CACHE, PH_PACK, PH_MAT, PH_PLAN, NPH };
constexpr int NREC = 128;   // event pairs kept per phase: stats average the last NREC calls

}  // namespace

// One cache (entries sorted by position per tree, plus value slots).  Two
// exist: during a generation the parents' set is read while the children's
// set is built.
struct CacheSet {
    uint32_t *e_cnt = nullptr, *e_off = nullptr, *e_pos = nullptr, *e_end = nullptr, *e_slot = nullptr;
    uint32_t *order = nullptr, *e_tree = nullptr, *e_cmax = nullptr, *msrc = nullptr;
    int32_t *e_par = nullptr, *e_c0 = nullptr, *e_c1 = nullptr, *e_bal = nullptr;
    uint4 *it_desc = nullptr, *sk_desc = nullptr;
    uint32_t Ecap = 0;
    std::vector<void*> allocs;
};

int gen_crossover(gp_pop* pop, uint32_t generation);
int gen_incremental(gp_pop* pop);

struct gp_pop {
    gp_config cfg;
    cudaStream_t stream;
    DevPop d;
    StructBufs sb;
    GenBufs gb;
    int dev, nsm;
    int grid_items, grid_warps, grid_threads;
    size_t smem_items;
    std::string err;
    gp_stats stats;
    bool profiling;
    cudaEvent_t ev[NPH][NREC][2];
    uint32_t ev_count[NPH];
    // phase events recorded by a captured graph (external event-record nodes):
    // the stats of a replay average the generations of the last replay
    cudaEvent_t gev[NPH][NREC][2];
    uint32_t gev_n[NPH];
    bool gev_made, capturing, graph_prof, stats_graph;
    bool have_children;
    std::vector<void*> allocs;
    uint64_t total_nodes_last;
    uint32_t launches;
    uint8_t* stage;          // device staging for uploads
    uint64_t* stage_off;
    uint64_t stage_cap;
    std::vector<uint64_t> host_off;   // pageable copies kept alive until the next upload
    std::vector<uint32_t> host_buf;
    std::vector<uint32_t> host_free;
    uint64_t slot_limit;              // value vectors the cache budget allows
    float* pool;                      // value slots shared by both cache sets
    uint32_t* live;                   // [pool_cap] live stamps
    uint32_t* freeslot;               // [pool_cap]
    uint32_t* ftile;                  // [pool_cap / FREE_TILE + 1]
    uint64_t pool_cap;
    CacheSet sets[2];
    int cur;                          // set of the current population
    uint32_t* e_total_h;              // pinned host copy of the entry count
    unsigned long long* cum;          // device: equivalent, actual, crossover bytes, calls
    uint32_t cum_calls;
    int grid_walk;
    int grid_walk_max;
    uint32_t walk_nw;                 // warps per child in the incremental walk
    size_t smem_walk;
    uint32_t onepass_nodes;           // children of at most this many nodes are evaluated in one pass
    uint32_t walk_long_n;             // children walked by the large teams (first in the work order)
    uint32_t walk_long_nw;            // warps per large team (16 or 8; 0 = no large teams)
    int grid_walk_long;
    size_t smem_walk_long;
    cudaEvent_t wfork_ev, wjoin_ev;   // large-team walk fork / join
    cudaStream_t side3;               // fourth stream: the one-pass children beside the walk
    cudaEvent_t ofork_ev, ojoin_ev;   // one-pass fork / join
    cudaEvent_t xfork_ev[2], xjoin_ev[2];   // cache update: records beside counts, links beside the slot pool
    int grid_onepass;                 // CTAs of the one-pass interpreter (each with its own overflow stacks)
    size_t smem_onepass;              // its dynamic shared memory per CTA
    uint32_t pack_launches;           // kernels of the last work-order computation
    uint8_t* tree_out;                // [cap] device copy of one tree for gp_get_tree
    uint32_t* tree_meta;              // [4] its size and availability
    uint32_t* io_h;                   // [4] pinned host words: status, tree size and availability
    uint32_t* rank;                   // [P] work-order ranks
    int prio_high;                    // greatest stream priority of the device (the large teams' launch)
    MlpBufs mlp;
    float mlp_lr;
    uint32_t cases_stat;              // test cases per value vector (64 for the Boolean word)
    int last_kind;                    // 0 full evaluation, 1 generation
    uint32_t* gwords;                 // device: [0] = 0, [1] = generations replayed by the captured graph
    cudaGraphExec_t gexec;            // captured generation loop (graph mode)
    uint32_t graph_n;                 // generations per replay
    uint32_t graph_launches;          // kernel launches per replay
    cudaStream_t cap_stream;          // private capture stream when the population runs on the legacy stream
    cudaStream_t side;                // second stream: work order (at crossover), copies (beside the cache update)
    cudaStream_t side2;               // third stream: the packing MLP's training beside the cache update
    cudaEvent_t cfork_ev, cjoin_ev;   // copies fork / join
    cudaEvent_t fork_ev, join_ev;     // training fork / join
    cudaEvent_t pfork_ev, pjoin_ev;   // work-order fork (at crossover) / join (before the walk)
    // fitness-first materialisation
    bool have_next_plan;              // the last walk drew the next generation's plan
    uint32_t planned_gen;             // ... for this generation number
    bool lazy_pending;                // some individuals exist only through their parents
    bool have_next_plan_at_xo;        // the last crossover took a drawn plan (and built deferred children)
    uint32_t host_nfree;              // pageable source of the free-stack count upload
    // disruption diagnostics
    bool dis_valid;                   // the last walk recorded into gb.dis
    uint32_t nbuf;                    // tree buffers in the arena
};

namespace {

int fail(gp_pop* p, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (p) p->err = buf; else g_create_error = buf;
    return code;
}

#define CK(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(pop, GP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

template <typename T>
int dalloc(gp_pop* pop, T** ptr, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(pop, GP_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    pop->allocs.push_back(p);
    *ptr = static_cast<T*>(p);
    return GP_OK;
}

#define DA(ptr, n)                                   \
    do {                                             \
        int r_ = dalloc(pop, &(ptr), (size_t)(n));   \
        if (r_) return r_;                           \
    } while (0)

void phase_begin(gp_pop* pop, int ph, cudaStream_t st) {
    if (!pop->profiling) return;
    if (pop->capturing) {
        if (pop->gev_n[ph] < (uint32_t)NREC)
            cudaEventRecordWithFlags(pop->gev[ph][pop->gev_n[ph]][0], st, cudaEventRecordExternal);
        return;
    }
    cudaEventRecord(pop->ev[ph][pop->ev_count[ph] % NREC][0], st);
}
void phase_end(gp_pop* pop, int ph, cudaStream_t st) {
    if (!pop->profiling) return;
    if (pop->capturing) {
        if (pop->gev_n[ph] < (uint32_t)NREC)
            cudaEventRecordWithFlags(pop->gev[ph][pop->gev_n[ph]++][1], st, cudaEventRecordExternal);
        return;
    }
    pop->stats_graph = false;
    cudaEventRecord(pop->ev[ph][pop->ev_count[ph]++ % NREC][1], st);
}
void phase_begin(gp_pop* pop, int ph) { phase_begin(pop, ph, pop->stream); }
void phase_end(gp_pop* pop, int ph) { phase_end(pop, ph, pop->stream); }

int check_status(gp_pop* pop) {
    uint32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, pop->d.status, sizeof st, cudaMemcpyDeviceToHost, pop->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pop->stream);
    if (e != cudaSuccess) return fail(pop, GP_ECUDA, "device error: %s", cudaGetErrorString(e));
    if (!st) return GP_OK;
    uint32_t ei[4] = {0, 0, 0, 0};
    cudaMemcpy(ei, pop->d.errinfo, sizeof ei, cudaMemcpyDeviceToHost);
    cudaMemsetAsync(pop->d.status, 0, sizeof(uint32_t), pop->stream);
    cudaMemsetAsync(pop->d.errinfo, 0, sizeof ei, pop->stream);
    char where[128] = "";
    if (ei[0]) snprintf(where, sizeof where, " [site %u, individual %u, position %u, detail %u]", ei[0], ei[1], ei[2], ei[3]);
    if (st & ST_ENTRIES) return fail(pop, GP_ENOMEM, "cache entry capacity (%u) exceeded", pop->d.Ecap);
    if (st & ST_SLOTS) return fail(pop, GP_ENOMEM, "cache value budget (%u slots) exceeded", pop->d.Scap);
    if (st & ST_CAPACITY)
        return fail(pop, GP_ECAPACITY, "out of tree buffers (arena_buffers %u; reload the population)", pop->nbuf);
    if (st & ST_TIMEOUT) return fail(pop, GP_ETIMEOUT, "a bounded device wait gave up");
    if (st & ST_STACK) return fail(pop, GP_EINVAL, "interpreter stack bound exceeded (malformed tree?)");
    if (st & ST_PATH) return fail(pop, GP_ENOMEM, "incremental path scratch exceeded");
    return fail(pop, GP_EINVAL, "tree structure inconsistent (status 0x%x)%s", st, where);
}

// Validate one tree on the host: a complete prefix expression of exactly n
// nodes with opcodes of the function set.
bool valid_tree(const uint8_t* ops, uint64_t n, uint32_t funcset) {
    if (n == 0) return false;
    const uint32_t maxop = funcset == GP_BOOL_MUX6 ? 9u : funcset == GP_BOOL_MUX11 ? 14u : 255u;
    int64_t need = 1;
    for (uint64_t i = 0; i < n; ++i) {
        if (need <= 0) return false;
        uint8_t o = ops[i];
        if (o > maxop) return false;
        need += (o < 4) ? 1 : -1;
    }
    return need == 0;
}

// Copy tree i from the compact upload (any byte offset) into its aligned
// buffer, 16 destination bytes per thread; the source is read as aligned
// 16-byte chunks and shifted.  The upload buffer has 32 bytes of slack.
__global__ void k_scatter_trees(const uint8_t* __restrict__ src, const uint64_t* __restrict__ off, DevPop d) {
    for (uint32_t i = blockIdx.x; i < d.P; i += gridDim.x) {
        const uint8_t* s = src + off[i];
        uint8_t* dst = d.arena + (size_t)d.buf[i] * d.cap;
        const uint32_t n = (uint32_t)(off[i + 1] - off[i]);
        if (threadIdx.x == 0) d.size[i] = n;
        const uintptr_t sa = reinterpret_cast<uintptr_t>(s);
        const uint32_t m = (uint32_t)(sa & 15u);
        const uint4* A = reinterpret_cast<const uint4*>(sa - m);
        const uint32_t nq = (n + 15) / 16;
        for (uint32_t q = threadIdx.x; q < nq; q += blockDim.x) {
            const uint4 lo = A[q], hi = (m ? A[q + 1] : lo);
            const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
            const uint32_t mw = m >> 2, sh = (m & 3u) * 8u;
            uint32_t r[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                uint32_t a = 0, b = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if ((uint32_t)c == mw) { a = w[t + c]; b = w[t + c + 1]; }
                r[t] = __funnelshift_r(a, b, sh);
            }
            reinterpret_cast<uint4*>(dst)[q] = make_uint4(r[0], r[1], r[2], r[3]);
        }
    }
}

// Call f(K, V) with the population's cases per lane and value kind as
// compile-time constants (the instantiated pairs: binary32 with K = 1, 2,
// 4; Boolean and integer with K = 1, 2).
template <int N> using IC = std::integral_constant<int, N>;
template <typename F>
auto with_kind(const DevPop& d, F&& f) {
    if (d.vkind == VB) return d.K == 1 ? f(IC<1>{}, IC<VB>{}) : f(IC<2>{}, IC<VB>{});
    if (d.vkind == VI) return d.K == 1 ? f(IC<1>{}, IC<VI>{}) : f(IC<2>{}, IC<VI>{});
    return d.K == 1 ? f(IC<1>{}, IC<VF>{}) : d.K == 2 ? f(IC<2>{}, IC<VF>{}) : f(IC<4>{}, IC<VF>{});
}

template <int K, int V>
int setup_items_kernel(gp_pop* pop) {
    size_t smem = SmemLayout<K>::total((int)pop->d.W, GP_WARPS);
    int max_optin = 0;
    CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pop->dev));
    if (smem > (size_t)max_optin)
        return fail(pop, GP_EINVAL, "stack_window %u x cases_per_lane %u needs %zu bytes of shared memory per CTA (%d)",
                    pop->d.W, pop->d.K, smem, max_optin);
    CK(cudaFuncSetAttribute(k_eval_items<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_eval_items<K, V>, GP_WARPS * 32, smem));
    if (nb < 1) nb = 1;
    pop->grid_items = nb * pop->nsm;
    pop->smem_items = smem;
    // the one-pass interpreter: CTAs of OP_EVAL_WARPS warps, as many as fit
    // (at most OP_CTAS_PER_SM per SM), each warp with its own overflow stack
    const size_t smem_op = OnePassEvalLayout<K>::total((int)pop->d.W);
    if (smem_op > (size_t)max_optin)
        return fail(pop, GP_EINVAL, "stack_window %u x cases_per_lane %u needs %zu bytes of shared memory per CTA (%d)",
                    pop->d.W, pop->d.K, smem_op, max_optin);
    CK(cudaFuncSetAttribute(k_onepass_eval<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_op));
    int nbo = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nbo, k_onepass_eval<K, V>, OP_EVAL_WARPS * 32, smem_op));
    if (nbo < 1) nbo = 1;
    if (nbo > OP_CTAS_PER_SM) nbo = OP_CTAS_PER_SM;
    pop->grid_onepass = nbo * pop->nsm;
    pop->smem_onepass = smem_op;
    return GP_OK;
}

// Team size of the incremental walk (warps per child) and its launch
// shape.  Auto: a team of 4 -- one building and combining warp and three
// sibling evaluators; larger teams for every child measured slower (their
// evaluators take the issue slots the combining warp needs), smaller ones
// leave long children short of evaluators.  On request (long_walks) the
// children the work order puts first (the longest predicted walks) get
// teams of 16 warps in a second launch beside the first, so that the
// longest walk's sibling interpretations spread over 15 evaluators; the two
// launches use disjoint interpreter overflow stacks.  Off by default: on
// the 500 x 1e6 population it measured slower (the ordinary teams hold the
// shared memory the large ones need, so the longest walks start late).
template <int K, int V>
int setup_walk_kernel(gp_pop* pop, uint32_t team) {
    const uint32_t ovf = pop->d.ovf_warps;      // the walk shares the interpreter's per-warp overflow stacks
    int max_optin = 0;
    CK(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pop->dev));
    {
        size_t s8 = TeamLayout<K>((int)pop->d.W, pop->d.Cpad, 8).total;
        if (s8 > (size_t)max_optin) s8 = (size_t)max_optin;
        CK(cudaFuncSetAttribute(k_walk<K, V, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s8));
    }
    const size_t smem16 = TeamLayout<K>((int)pop->d.W, pop->d.Cpad, 16).total;
    const bool can16 = smem16 <= (size_t)max_optin;
    if (can16)
        CK(cudaFuncSetAttribute(k_walk<K, V, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16));
    auto shape = [&](uint32_t nw, int& grid, size_t& smem) -> int {
        smem = TeamLayout<K>((int)pop->d.W, pop->d.Cpad, nw).total;
        int nb = 0;
        if (nw > 8) CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk<K, V, 512>, (int)nw * 32, smem));
        else CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_walk<K, V, 256>, (int)nw * 32, smem));
        if (nb < 1) nb = 1;
        grid = nb * pop->nsm;
        return GP_OK;
    };
    uint32_t nw = team;
    if (!nw) nw = 4;
    if (TeamLayout<K>((int)pop->d.W, pop->d.Cpad, nw).total > (size_t)max_optin)
        return fail(pop, GP_EINVAL, "a walk team of %u warps with stack_window %u does not fit shared memory", nw, pop->d.W);
    int grid = 0;
    size_t smem = 0;
    int r = shape(nw, grid, smem);
    if (r) return r;
    // large teams for the first children of the work order
    const uint32_t P = pop->d.P;
    uint32_t nlong = pop->cfg.long_walks;
    if (nlong == 0xFFFFFFFFu) nlong = 0;
    if (nlong > P) nlong = P;
    uint32_t nwl = can16 ? 16u : 8u;
    if (nwl <= nw) nlong = 0;
    int gridl = 0;
    size_t smeml = 0;
    if (nlong) {
        r = shape(nwl, gridl, smeml);
        if (r) return r;
        if ((uint32_t)gridl > nlong) gridl = (int)nlong;
        if ((uint64_t)gridl * nwl > ovf / 2) gridl = (int)(ovf / 2 / nwl);
        if (gridl < 1) nlong = 0;
    }
    if (!nlong) { nwl = 0; gridl = 0; smeml = 0; }
    const uint32_t ovf_left = ovf - (uint32_t)gridl * nwl;
    if ((uint32_t)grid * nw > ovf_left) grid = (int)(ovf_left / nw);
    pop->walk_nw = nw;
    pop->grid_walk = grid;
    pop->smem_walk = smem;
    pop->walk_long_n = nlong;
    pop->walk_long_nw = nwl;
    pop->grid_walk_long = gridl;
    pop->smem_walk_long = smeml;
    return GP_OK;
}

template <int K, int V>
void launch_items(gp_pop* pop) {
    k_eval_items<K, V><<<pop->grid_items, GP_WARPS * 32, pop->smem_items, pop->stream>>>(pop->d);
}
template <int K, int V>
void launch_skeleton(gp_pop* pop) {
    k_eval_skeleton<K, V><<<pop->grid_warps, GP_WARPS * 32, 0, pop->stream>>>(pop->d);
}

// Advance the generation offset of a captured generation loop (last node of the graph).
__global__ void k_graph_advance(uint32_t* ctr, uint32_t n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += n;
}

// Add the last evaluation's counters to the running totals (device side, no sync).
__global__ void k_accumulate(unsigned long long* cum, const unsigned long long* acc, const unsigned long long* gst,
                             uint32_t C, int kind) {
    if (threadIdx.x != 0) return;
    if (kind == 0) {
        cum[0] += acc[1] * C;
        cum[1] += acc[0] * C;
    } else {
        cum[0] += gst[G_EQUIV] * C;
        cum[1] += (gst[G_INTERP] + gst[G_PATHOPS]) * C;
        cum[2] += gst[G_XOBYTES];
    }
}

// Point the kernels' view (DevPop, StructBufs) at the current cache set.
void bind_set(gp_pop* pop) {
    DevPop& d = pop->d;
    CacheSet& c = pop->sets[pop->cur];
    d.e_cnt = c.e_cnt; d.e_off = c.e_off; d.e_pos = c.e_pos; d.e_end = c.e_end; d.e_par = c.e_par;
    d.e_c0 = c.e_c0; d.e_c1 = c.e_c1; d.e_slot = c.e_slot; d.e_tree = c.e_tree; d.it_desc = c.it_desc;
    d.sk_desc = c.sk_desc; d.order = c.order; d.Ecap = c.Ecap;
    d.slots = pop->pool; d.live = pop->live; d.freeslot = pop->freeslot; d.ftile = pop->ftile;
    d.Scap = (uint32_t)pop->pool_cap;
    pop->sb.e_bal = c.e_bal; pop->sb.e_tree = c.e_tree; pop->sb.e_cmax = c.e_cmax;
    pop->gb.src = c.msrc;
}

CacheView view_of(const gp_pop* pop, const CacheSet& c) {
    CacheView v;
    v.e_off = c.e_off; v.e_pos = c.e_pos; v.e_end = c.e_end; v.e_par = c.e_par;
    v.e_c0 = c.e_c0; v.e_c1 = c.e_c1; v.e_slot = c.e_slot; v.slots = pop->pool;
    return v;
}

// Grow the shared slot pool to at least `want` slots, keeping the values
// and live marks it holds (the parents' values may still be in use).
int ensure_pool(gp_pop* pop, uint64_t want) {
    if (want <= pop->pool_cap) return GP_OK;
    if (want > pop->slot_limit)
        return fail(pop, GP_ENOMEM, "cache needs %llu value vectors, budget allows %llu",
                    (unsigned long long)want, (unsigned long long)pop->slot_limit);
    if (pop->stream) cudaStreamSynchronize(pop->stream); else cudaDeviceSynchronize();
    if (pop->gexec) { cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
    const size_t Cpad = pop->d.Cpad;
    float* np = nullptr;
    uint32_t *nl = nullptr, *nf = nullptr, *nt = nullptr;
    const size_t ntile = want / FREE_TILE + 2;
    if (cudaMalloc(&np, want * Cpad * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&nl, want * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&nf, want * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&nt, ntile * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(np); cudaFree(nl); cudaFree(nf); cudaFree(nt);
        return fail(pop, GP_ENOMEM, "allocation of a value pool of %llu slots failed", (unsigned long long)want);
    }
    cudaMemset(nl, 0, want * sizeof(uint32_t));
    if (pop->pool) {
        cudaMemcpy(np, pop->pool, pop->pool_cap * Cpad * sizeof(float), cudaMemcpyDeviceToDevice);
        cudaMemcpy(nl, pop->live, pop->pool_cap * sizeof(uint32_t), cudaMemcpyDeviceToDevice);
        cudaFree(pop->pool); cudaFree(pop->live); cudaFree(pop->freeslot); cudaFree(pop->ftile);
    }
    pop->pool = np; pop->live = nl; pop->freeslot = nf; pop->ftile = nt;
    pop->pool_cap = want;
    DevPop& d = pop->d;
    d.slots = np; d.live = nl; d.freeslot = nf; d.ftile = nt; d.Scap = (uint32_t)want;
    return GP_OK;
}

// (Re)allocate the index arrays of cache set `which` for ecap entries, and
// make the shared pool hold ecap values plus the walk's new ones.
int grow_set(gp_pop* pop, int which, uint32_t ecap) {
    CacheSet& c = pop->sets[which];
    const DevPop& d = pop->d;
    {
        int r = ensure_pool(pop, (uint64_t)ecap + pop->gb.pvcap);
        if (r) return r;
    }
    if (pop->stream) cudaStreamSynchronize(pop->stream); else cudaDeviceSynchronize();
    if (pop->gexec) { cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
    for (void* p : c.allocs) cudaFree(p);
    c.allocs.clear();
    auto al = [&](auto** ptr, size_t count) -> bool {
        void* p = nullptr;
        size_t bytes = count * sizeof(**ptr);
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) { cudaGetLastError(); return false; }
        c.allocs.push_back(p);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(p);
        return true;
    };
    bool ok = al(&c.e_cnt, d.P + 1) && al(&c.e_off, d.P + 1) && al(&c.e_pos, ecap) && al(&c.e_end, ecap) &&
              al(&c.e_par, ecap) && al(&c.e_c0, ecap) && al(&c.e_c1, ecap) && al(&c.e_slot, ecap) &&
              al(&c.it_desc, ecap) && al(&c.sk_desc, ecap) && al(&c.order, ecap) && al(&c.e_bal, ecap) &&
              al(&c.e_tree, ecap) && al(&c.e_cmax, ecap / 32 + 2) && al(&c.msrc, ecap);
    if (!ok) return fail(pop, GP_ENOMEM, "allocation of a cache of %u entries failed", ecap);
    cudaMemset(c.e_off, 0, sizeof(uint32_t) * (d.P + 1));
    c.Ecap = ecap;
    if (which == pop->cur) bind_set(pop);
    return GP_OK;
}

int grow_cache(gp_pop* pop, uint32_t ecap) { return grow_set(pop, pop->cur, ecap); }

// Structure pass of the current population into the current cache set:
// cached nodes with ends, parents and links (grows the set if needed).
int run_structure(gp_pop* pop) {
    DevPop& d = pop->d;
    const int gthreads = pop->grid_threads;
    k_blk_offsets<<<1, 1024, 0, pop->stream>>>(d);
    k_unit_flags<<<pop->nsm * 16, FLAG_WARPS * 32, 0, pop->stream>>>(d, pop->sb);
    const int scan_grid = pop->nsm * 2;
    k_scan_tiles<<<scan_grid, SCAN_TILE, 0, pop->stream>>>(d, pop->sb);
    k_scan_top<<<1, SCAN_TILE, 0, pop->stream>>>(d, pop->sb);
    k_scan_apply<<<scan_grid, SCAN_TILE, 0, pop->stream>>>(d, pop->sb);
    // entry count known: grow the cache arrays if this population needs more
    // (in graph mode the arrays are pre-sized and an overflow is reported instead)
    if (!d.strict_cap) {
        CK(cudaMemcpyAsync(pop->e_total_h, d.e_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, pop->stream));
        CK(cudaStreamSynchronize(pop->stream));
        if (*pop->e_total_h > d.Ecap) {
            uint64_t want = (uint64_t)*pop->e_total_h + *pop->e_total_h / 4 + 64;
            const uint64_t room = pop->slot_limit > pop->gb.pvcap ? pop->slot_limit - pop->gb.pvcap : 0;
            if (want > room) want = room;
            if (want < *pop->e_total_h)
                return fail(pop, GP_ENOMEM, "cache of %u entries exceeds the cache budget", *pop->e_total_h);
            int r = grow_cache(pop, (uint32_t)want);
            if (r) return r;
        }
    }
    k_tree_entry_offsets<<<(d.P + 256) / 256, 256, 0, pop->stream>>>(d, pop->sb);
    k_emit_entries<<<pop->grid_warps, GP_WARPS * 32, 0, pop->stream>>>(d, pop->sb);
    k_entry_ends<<<gthreads, 256, 0, pop->stream>>>(d, pop->sb);
    k_entry_chunkmax<<<pop->grid_warps, GP_WARPS * 32, 0, pop->stream>>>(d, pop->sb);
    k_entry_parents<<<gthreads, 256, 0, pop->stream>>>(d, pop->sb);
    return GP_OK;
}

// Structure pass + full evaluation of the current population.
int run_full(gp_pop* pop) {
    DevPop& d = pop->d;
    const int gthreads = pop->grid_threads;
    CK(cudaMemsetAsync(d.q, 0, sizeof(uint32_t) * NQ, pop->stream));
    CK(cudaMemsetAsync(d.acc_ops, 0, 4 * sizeof(unsigned long long), pop->stream));
    pop->launches = 15;
    pop->last_kind = 0;
    phase_begin(pop, PH_STRUCT);
    {
        int r = run_structure(pop);
        if (r) return r;
    }
    k_build_items<<<gthreads, 256, 0, pop->stream>>>(d, pop->sb.e_tree);
    phase_end(pop, PH_STRUCT);
    phase_begin(pop, PH_ITEMS);
    with_kind(pop->d, [&](auto k, auto v) { launch_items<decltype(k)::value, decltype(v)::value>(pop); return 0; });
    phase_end(pop, PH_ITEMS);
    phase_begin(pop, PH_SKEL);
    with_kind(pop->d, [&](auto k, auto v) { launch_skeleton<decltype(k)::value, decltype(v)::value>(pop); return 0; });
    phase_end(pop, PH_SKEL);
    phase_begin(pop, PH_FIT);
    k_fitness<<<pop->grid_warps, GP_WARPS * 32, 0, pop->stream>>>(d);
    phase_end(pop, PH_FIT);
    k_accumulate<<<1, 32, 0, pop->stream>>>(pop->cum, d.acc_ops, pop->gb.gstat, pop->cases_stat, 0);
    ++pop->cum_calls;
    CK(cudaGetLastError());
    return GP_OK;
}

}  // namespace

extern "C" {

// the autotuner's report when no candidate ran (read back by gp_last_error(NULL))
void gpfdp_set_create_error(const char* msg) { g_create_error = msg ? msg : ""; }

const char* gp_last_error(const gp_pop* pop) {
    return pop ? pop->err.c_str() : g_create_error.c_str();
}

int gp_pop_create(const gp_config* cfg_in, const float* x, const float* targets, const float* consts,
                  const uint8_t* ops, const uint64_t* offsets, void* stream, gp_pop** out) {
    gp_pop* pop = nullptr;
    if (!cfg_in || !out || !ops || !offsets || !consts) return fail(nullptr, GP_EINVAL, "null argument");
    *out = nullptr;
    gp_config cfg = *cfg_in;
    if (cfg.pop_size == 0) return fail(nullptr, GP_EINVAL, "pop_size must be > 0");
    if (cfg.funcset > GP_INT32_ARITH) return fail(nullptr, GP_EINVAL, "bad funcset");
    const bool boolean = cfg.funcset == GP_BOOL_MUX6 || cfg.funcset == GP_BOOL_MUX11;
    const uint32_t mux_k = cfg.funcset == GP_BOOL_MUX6 ? 2u : cfg.funcset == GP_BOOL_MUX11 ? 3u : 0u;
    // Boolean: n_cases counts 32-case words, 2^(k + 2^k) / 32 of them (6-mux 2, 11-mux 64)
    if (boolean) cfg.n_cases = (1u << (mux_k + (1u << mux_k))) / 32u;
    if (cfg.funcset == GP_BOOL_MUX6) cfg.cases_per_lane = 1;
    if (cfg.n_cases == 0 || cfg.n_cases > (1u << 20)) return fail(nullptr, GP_EINVAL, "n_cases out of range");
    if (!boolean && (!x || !targets)) return fail(nullptr, GP_EINVAL, "null x/targets");
    if (cfg.cache_threshold == 0) cfg.cache_threshold = 1024;
    uint32_t T = cfg.cache_threshold;
    if (T < 2 || T > GP_B || (T & (T - 1))) return fail(nullptr, GP_EINVAL, "cache_threshold must be a power of two in [2, 1024]");
    if (cfg.max_nodes == 0 || cfg.max_nodes > (1u << 30)) return fail(nullptr, GP_EINVAL, "max_nodes out of range");
    if (cfg.tournament == 0) cfg.tournament = 7;
    if (cfg.cache_budget_bytes == 0) cfg.cache_budget_bytes = 40ull << 30;
    uint32_t K = cfg.cases_per_lane;
    if (K == 0) K = (cfg.n_cases <= 32) ? 1 : 2;
    if (K != 1 && K != 2 && K != 4) return fail(nullptr, GP_EINVAL, "cases_per_lane must be 0, 1, 2 or 4");
    if (K == 4 && cfg.funcset != GP_FP32_ARITH)
        return fail(nullptr, GP_EINVAL, "cases_per_lane 4 is for the binary32 set only");
    if (cfg.walk_team != 0 && cfg.walk_team != 1 && cfg.walk_team != 2 && cfg.walk_team != 4 && cfg.walk_team != 8)
        return fail(nullptr, GP_EINVAL, "walk_team must be 0, 1, 2, 4 or 8");
    if (cfg.lazy_children > 1) return fail(nullptr, GP_EINVAL, "lazy_children must be 0 or 1");
    if (cfg.lazy_inplace > 1 || (cfg.lazy_inplace && !cfg.lazy_children))
        return fail(nullptr, GP_EINVAL, "lazy_inplace must be 0, or 1 with lazy_children");
    if (cfg.stack_window != 0 && cfg.stack_window != 16 && cfg.stack_window != 32 && cfg.stack_window != 64)
        return fail(nullptr, GP_EINVAL, "stack_window must be 0, 16, 32 or 64");
    if (cfg.arena_buffers && (!cfg.lazy_children || cfg.arena_buffers <= cfg.pop_size ||
                              cfg.arena_buffers > 2 * cfg.pop_size))
        return fail(nullptr, GP_EINVAL, "arena_buffers must be 0, or in (pop_size, 2 x pop_size] with lazy_children");
    const uint32_t P = cfg.pop_size;
    for (uint32_t i = 0; i < P; ++i) {
        if (offsets[i + 1] < offsets[i]) return fail(nullptr, GP_EINVAL, "offsets not increasing at %u", i);
        uint64_t n = offsets[i + 1] - offsets[i];
        if (n > cfg.max_nodes) return fail(nullptr, GP_ECAPACITY, "tree %u has %llu nodes > max_nodes", i, (unsigned long long)n);
        if (!valid_tree(ops + offsets[i], n, cfg.funcset)) return fail(nullptr, GP_EINVAL, "tree %u is not a complete prefix expression of valid opcodes", i);
    }

    pop = new gp_pop();
    pop->cfg = cfg;
    pop->stream = static_cast<cudaStream_t>(stream);
    pop->profiling = false;
    pop->have_children = false;
    pop->stage = nullptr;
    pop->stage_off = nullptr;
    pop->stage_cap = 0;
    pop->launches = 0;
    pop->e_total_h = nullptr;
    pop->io_h = nullptr;
    pop->last_kind = 0;
    pop->cases_stat = boolean ? 32u * cfg.n_cases : cfg.n_cases;
    memset(&pop->stats, 0, sizeof pop->stats);
    memset(pop->ev_count, 0, sizeof pop->ev_count);
    pop->gexec = nullptr;
    pop->graph_n = 0;
    pop->cap_stream = nullptr;
    pop->side = nullptr;
    pop->side2 = nullptr;
    pop->cfork_ev = pop->cjoin_ev = nullptr;
    pop->fork_ev = pop->join_ev = pop->pfork_ev = pop->pjoin_ev = nullptr;
    pop->wfork_ev = pop->wjoin_ev = nullptr;
    pop->side3 = nullptr;
    pop->ofork_ev = pop->ojoin_ev = nullptr;
    pop->xfork_ev[0] = pop->xfork_ev[1] = pop->xjoin_ev[0] = pop->xjoin_ev[1] = nullptr;
    pop->gev_made = pop->capturing = pop->graph_prof = pop->stats_graph = false;
    memset(pop->gev_n, 0, sizeof pop->gev_n);
    auto bail = [&](int code) { gp_pop_destroy(pop); return code; };
    cudaError_t ce = cudaGetDevice(&pop->dev);
    if (ce != cudaSuccess) { g_create_error = cudaGetErrorString(ce); delete pop; return GP_ECUDA; }
    cudaDeviceGetAttribute(&pop->nsm, cudaDevAttrMultiProcessorCount, pop->dev);
    {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) { cudaGetLastError(); greatest = 0; }
        pop->prio_high = greatest;
    }
    for (int i = 0; i < NPH; ++i)
        for (int j = 0; j < NREC; ++j) { cudaEventCreate(&pop->ev[i][j][0]); cudaEventCreate(&pop->ev[i][j][1]); }
    if (cudaStreamCreateWithFlags(&pop->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pop->side2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->cfork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->cjoin_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->pfork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->pjoin_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->wfork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->wjoin_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pop->side3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->ofork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->ojoin_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->xfork_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->xfork_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->xjoin_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pop->xjoin_ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "stream or event creation failed";
        return bail(GP_ECUDA);
    }

    DevPop& d = pop->d;
    memset(&d, 0, sizeof d);
    d.P = P;
    d.C = cfg.n_cases;
    d.K = K;
    d.ncb = (d.C + 32 * K - 1) / (32 * K);
    d.Cpad = d.ncb * 32 * K;
    d.T = T;
    d.cap = (uint32_t)(((uint64_t)cfg.max_nodes + GP_B - 1) / GP_B * GP_B);
    d.funcset = cfg.funcset;
    d.vkind = boolean ? (uint32_t)VB : cfg.funcset == GP_INT32_ARITH ? (uint32_t)VI : (uint32_t)VF;
    d.mux_k = mux_k;
    d.W = cfg.stack_window ? cfg.stack_window : 16u;   // interpreter stack entries kept in shared memory
    d.maxdepth = d.W + T + 2;       // subtrees below the threshold need at most T + 1 entries
    const uint64_t total_cap = (uint64_t)P * d.cap;
    // initial cache-entry capacity; grown on demand by gp_eval_full
    uint64_t ecap = (uint64_t)P + total_cap * 4 / T;
    if (ecap > (uint64_t)P + total_cap) ecap = (uint64_t)P + total_cap;
    if (ecap > (1ull << 26)) ecap = 1ull << 26;
    pop->slot_limit = cfg.cache_budget_bytes / ((uint64_t)d.Cpad * sizeof(float));
    if (pop->slot_limit > 0xFFFFFFF0ull) pop->slot_limit = 0xFFFFFFF0ull;
    const uint64_t pv_slots = (uint64_t)P * PV_PER_CHILD;
    if (pop->slot_limit < 2ull * P + pv_slots) { g_create_error = "cache budget too small for one vector per tree"; delete pop; return GP_ENOMEM; }
    if (ecap + pv_slots > pop->slot_limit) ecap = pop->slot_limit - pv_slots;
    const uint32_t nbuf = cfg.arena_buffers ? cfg.arena_buffers : 2 * P;   // parents + children (copy targets)
    pop->nbuf = nbuf;
    d.ovf_warps = 0;
    d.wait_polls = WALK_SPIN;

    // grids
    pop->grid_warps = pop->nsm * 8;
    pop->grid_threads = pop->nsm * 8;

#define DA2(ptr, n) do { int r_ = dalloc(pop, &(ptr), (size_t)(n)); if (r_) return bail(r_); } while (0)
    DA2(d.arena, (size_t)nbuf * d.cap + 4096);     // slack: scans and 16-byte copies may read past the last buffer
    DA2(d.buf, P);
    DA2(d.size, P);
    DA2(d.x, d.Cpad);
    DA2(d.t, d.C);
    DA2(d.consts, 256);
    DA2(d.fit, P);
    DA2(d.blk_off, P + 1);
    pop->gb.pvcap = P * PV_PER_CHILD;
    pop->cur = 0;
    for (int w = 1; w >= 0; --w) {
        int r = grow_set(pop, w, (uint32_t)ecap);
        if (r) { g_create_error = pop->err; return bail(r); }
    }
    DA2(d.status, 4);
    DA2(pop->cum, 4);
    cudaMemset(pop->cum, 0, 4 * sizeof(unsigned long long));
    pop->cum_calls = 0;
    DA2(d.errinfo, 4);
    cudaMemset(d.errinfo, 0, 4 * sizeof(uint32_t));
    DA2(d.e_total, 4);
    if (cudaMallocHost(&pop->e_total_h, sizeof(uint32_t)) != cudaSuccess) { g_create_error = "cudaMallocHost failed"; return bail(GP_ENOMEM); }
    if (cudaMallocHost(&pop->io_h, 4 * sizeof(uint32_t)) != cudaSuccess) { g_create_error = "cudaMallocHost failed"; return bail(GP_ENOMEM); }
    DA2(pop->tree_out, (size_t)d.cap + 16);
    DA2(pop->tree_meta, 4);
    DA2(d.q, NQ);
    DA2(d.acc_ops, 4);
    StructBufs& sb = pop->sb;
    sb.Ucap = (uint32_t)(total_cap / GP_B + P);
    DA2(sb.u_flags, (size_t)sb.Ucap * 32);
    DA2(sb.u_cv0, (size_t)sb.Ucap * 32);
    DA2(sb.u_cmax, (size_t)sb.Ucap * 32);
    DA2(sb.u_total, sb.Ucap);
    DA2(sb.u_max, sb.Ucap);
    DA2(sb.u_cnt, sb.Ucap);
    DA2(sb.u_epre, sb.Ucap + 1);
    DA2(sb.u_bpre, sb.Ucap + 1);
    DA2(sb.tile_c, sb.Ucap / SCAN_TILE + 2);
    DA2(sb.tile_b, sb.Ucap / SCAN_TILE + 2);

    // interpreter launch shape and its overflow stacks
    if (cudaFuncSetAttribute(k_onepass_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(OnePassSmem)) !=
        cudaSuccess) { cudaGetLastError(); g_create_error = "shared memory of the one-pass plan kernel"; return bail(GP_ECUDA); }
    {
        int r = with_kind(d, [&](auto k, auto v) { return setup_items_kernel<decltype(k)::value, decltype(v)::value>(pop); });
        if (r) { g_create_error = pop->err; return bail(r); }
        d.ovf_warps = (uint32_t)pop->grid_items * GP_WARPS;
        DA2(d.ovf, (size_t)d.ovf_warps * (d.maxdepth - d.W) * 32 * K);
    }
    // generation buffers
    {
        GenBufs& g = pop->gb;
        g.max_nodes = cfg.max_nodes;
        g.tsize = cfg.tournament;
        g.seed = cfg.seed;
        g.gen = 0;
        g.evaluated = false;
        g.dis = nullptr;
        g.dis_n = nullptr;
        g.dis_L = 0;
        pop->dis_valid = false;
        DA2(pop->gwords, 4);
        cudaMemset(pop->gwords, 0, 4 * sizeof(uint32_t));
        g.gen_add = pop->gwords;
        g.stamp = pop->gwords + 2;
        g.frag_cap = (uint64_t)P * d.cap;
        g.stash_cap = (uint64_t)P * (T + 16);
        g.shift_cap = (uint32_t)((uint64_t)P * d.cap / SHIFT_BS + P);
        // halo pool of the in-place moves: an eighth of a buffer per individual
        // (a generation whose moves need more copies the rest of its children)
        g.halo_cap = (uint64_t)P * d.cap / 8 + 65536;
        DA2(g.pbuf, P); DA2(g.psize, P); DA2(g.pfit, P);
        DA2(g.mother, P); DA2(g.father, P); DA2(g.cpos, P); DA2(g.rsz, P); DA2(g.dpos, P); DA2(g.ssz, P);
        DA2(g.flags, P); DA2(g.lastidx, P); DA2(g.free_buf, 2 * P); DA2(g.free_next, P); DA2(g.hasip, P);
        DA2(g.misc, NMISC);
        DA2(g.frag_off, P + 1); DA2(g.frag, g.frag_cap + 64);
        DA2(g.stash_off, P + 1); DA2(g.stash, g.stash_cap + 64);
        DA2(g.shift_off, P + 1); DA2(g.halo, g.halo_cap + 64); DA2(g.halo_off, P + 1);
        DA2(g.lastsel, P); DA2(g.npend, 1);
        cudaMemset(g.npend, 0, sizeof(uint32_t));
        DA2(g.copy_off, P + 1);
        DA2(g.stop, P); DA2(g.plen, P);
        DA2(g.pv_rec, g.pvcap); DA2(g.pv_cnt, P); DA2(g.pv_off, P + 1); DA2(g.pv_sorted, g.pvcap);
        DA2(g.pv_end, g.pvcap); DA2(g.pv_val, (size_t)g.pvcap * d.Cpad);
        DA2(g.rec_entry, g.pvcap);
        g.lazy = cfg.lazy_children;
        g.lazy_inplace = cfg.lazy_inplace;
        DA2(g.nmother, P); DA2(g.nfather, P); DA2(g.ncpos, P); DA2(g.nrsz, P); DA2(g.ndpos, P); DA2(g.nssz, P);
        DA2(g.nflags, P); DA2(g.sel, P); DA2(g.nfree, 1); DA2(g.pref, P);
        DA2(g.walkA, P); DA2(g.nins, P); DA2(g.mb, P); DA2(g.mcnt, P + 1);
        DA2(g.order, P); DA2(g.gstat, NGSTAT); DA2(pop->rank, P);
        DA2(g.small_cnt, P); DA2(g.small_val, (size_t)P * d.Cpad); DA2(g.onepass, P); DA2(g.op_base, P);
        DA2(g.op_cnt, 2 * OP_BUCKETS); DA2(g.op_bucket, (size_t)OP_BUCKETS * P);
        cudaMemset(g.onepass, 0, sizeof(uint32_t) * P);
        pop->onepass_nodes = cfg.onepass_nodes == 0 ? (uint32_t)ONEPASS_MAX
                             : cfg.onepass_nodes == 0xFFFFFFFFu ? 0u
                             : (cfg.onepass_nodes < (uint32_t)ONEPASS_MAX ? cfg.onepass_nodes : (uint32_t)ONEPASS_MAX);
        g.onepass_max = pop->onepass_nodes;
        g.ovf_op = nullptr;
        if (pop->onepass_nodes)
            DA2(g.ovf_op, (size_t)pop->grid_onepass * OP_EVAL_WARPS * ONEPASS_DEPTH * 32 * K);
        std::vector<uint32_t> fb(P, 0u);
        for (uint32_t i = 0; i < nbuf - P; ++i) fb[i] = P + i;   // buffers P..nbuf-1 start free
        const uint32_t nfree_init = nbuf - P;
        if (cudaMemcpy(g.nfree, &nfree_init, sizeof nfree_init, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(g.free_buf, fb.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(GP_ECUDA);
        cudaMemset(g.gstat, 0, sizeof(unsigned long long) * NGSTAT);
    }
    // incremental walk launch shape
    {
        const uint32_t team = cfg.walk_team;
        int r = with_kind(d, [&](auto k, auto v) {
            return setup_walk_kernel<decltype(k)::value, decltype(v)::value>(pop, team);
        });
        if (r) { g_create_error = pop->err; return bail(r); }
        pop->grid_walk_max = pop->grid_walk;
        if (cfg.walk_warps) {
            int g = (int)((cfg.walk_warps + pop->walk_nw - 1) / pop->walk_nw);
            if (g < pop->grid_walk) pop->grid_walk = g;
        }
    }
    // packing MLP
    {
        MlpBufs& b = pop->mlp;
        b.cap = P;
        DA2(b.w, MLP_NP); DA2(b.m, MLP_NP); DA2(b.v, MLP_NP); DA2(b.wb, MLP_NP); DA2(b.grad, MLP_NP);
        DA2(b.feat, (size_t)P * MLP_IN); DA2(b.pred, P); DA2(b.pred_pack, P); DA2(b.target, P); DA2(b.h1, (size_t)P * MLP_H);
        DA2(b.h2, (size_t)P * MLP_H); DA2(b.dy, P); DA2(b.dh2, (size_t)P * MLP_H); DA2(b.dh1, (size_t)P * MLP_H);
        DA2(b.loss, 1); DA2(b.step, 1);
        DA2(b.part, (size_t)((P + MLP_CH - 1) / MLP_CH) * MLP_NP);
        pop->mlp_lr = (cfg.mlp_lr_micro ? cfg.mlp_lr_micro : 1000u) * 1e-6f;
        k_mlp_init<<<(MLP_NP + 255) / 256, 256, 0, pop->stream>>>(b, cfg.seed ^ 0x3131A5A5ull);
        cudaMemsetAsync(b.loss, 0, sizeof(float), pop->stream);
    }

    // inputs
    // (integer set: the caller's int32 bits, copied as they are; Boolean: the
    // target's case words, bit l of word w for case 32w + l)
    std::vector<float> xp(d.Cpad, 0.0f), tp(d.C, 0.0f);
    if (!boolean) { memcpy(xp.data(), x, sizeof(float) * d.C); memcpy(tp.data(), targets, sizeof(float) * d.C); }
    else {
        for (uint32_t w = 0; w < d.C; ++w) {
            uint32_t word = 0;
            for (uint32_t l = 0; l < 32; ++l) {
                const uint64_t i = 32ull * w + l;
                const uint64_t a = i & ((1ull << mux_k) - 1);
                word |= (uint32_t)((i >> (mux_k + a)) & 1ull) << l;
            }
            memcpy(&tp[w], &word, 4);
        }
    }
    std::vector<uint32_t> bufs(P);
    for (uint32_t i = 0; i < P; ++i) bufs[i] = i;
    uint8_t* stage = nullptr;
    uint64_t* stage_off = nullptr;
    const uint64_t total = offsets[P] - offsets[0];
    std::vector<uint64_t> off0(P + 1);
    for (uint32_t i = 0; i <= P; ++i) off0[i] = offsets[i] - offsets[0];
#define CK2(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { fail(pop, GP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); g_create_error = pop->err; cudaFree(stage); cudaFree(stage_off); return bail(GP_ECUDA); } } while (0)
    CK2(cudaMalloc(&stage, total + 32));
    CK2(cudaMalloc(&stage_off, sizeof(uint64_t) * (P + 1)));
    CK2(cudaMemcpyAsync(stage, ops + offsets[0], total, cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemcpyAsync(stage_off, off0.data(), sizeof(uint64_t) * (P + 1), cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemcpyAsync(d.x, xp.data(), sizeof(float) * d.Cpad, cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemcpyAsync(d.t, tp.data(), sizeof(float) * d.C, cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemcpyAsync(d.consts, consts, sizeof(float) * GP_NCONST, cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemcpyAsync(d.buf, bufs.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, pop->stream));
    CK2(cudaMemsetAsync(d.status, 0, 4 * sizeof(uint32_t), pop->stream));
    CK2(cudaMemsetAsync(d.acc_ops, 0, 4 * sizeof(unsigned long long), pop->stream));
    CK2(cudaMemsetAsync(d.fit, 0, sizeof(float) * P, pop->stream));
    k_scatter_trees<<<(P < 4096 ? P : 4096), 256, 0, pop->stream>>>(stage, stage_off, d);
    CK2(cudaGetLastError());
    CK2(cudaStreamSynchronize(pop->stream));
    cudaFree(stage);
    cudaFree(stage_off);
    pop->total_nodes_last = total;
    *out = pop;
    return GP_OK;
}

void gp_pop_destroy(gp_pop* pop) {
    if (!pop) return;
    if (pop->stream) cudaStreamSynchronize(pop->stream); else cudaDeviceSynchronize();
    if (pop->side) cudaStreamSynchronize(pop->side);
    if (pop->side2) cudaStreamSynchronize(pop->side2);
    if (pop->gexec) cudaGraphExecDestroy(pop->gexec);
    if (pop->cap_stream) cudaStreamDestroy(pop->cap_stream);
    if (pop->side) cudaStreamDestroy(pop->side);
    if (pop->side2) cudaStreamDestroy(pop->side2);
    if (pop->side3) cudaStreamDestroy(pop->side3);
    if (pop->cfork_ev) cudaEventDestroy(pop->cfork_ev);
    if (pop->cjoin_ev) cudaEventDestroy(pop->cjoin_ev);
    if (pop->fork_ev) cudaEventDestroy(pop->fork_ev);
    if (pop->join_ev) cudaEventDestroy(pop->join_ev);
    if (pop->pfork_ev) cudaEventDestroy(pop->pfork_ev);
    if (pop->pjoin_ev) cudaEventDestroy(pop->pjoin_ev);
    if (pop->wfork_ev) cudaEventDestroy(pop->wfork_ev);
    if (pop->wjoin_ev) cudaEventDestroy(pop->wjoin_ev);
    for (int k = 0; k < 2; ++k) {
        if (pop->xfork_ev[k]) cudaEventDestroy(pop->xfork_ev[k]);
        if (pop->xjoin_ev[k]) cudaEventDestroy(pop->xjoin_ev[k]);
    }
    if (pop->ofork_ev) cudaEventDestroy(pop->ofork_ev);
    if (pop->ojoin_ev) cudaEventDestroy(pop->ojoin_ev);
    cudaFree(pop->gb.dis); cudaFree(pop->gb.dis_n);
    cudaFree(pop->pool); cudaFree(pop->live); cudaFree(pop->freeslot); cudaFree(pop->ftile);
    for (void* p : pop->allocs) cudaFree(p);
    for (int w = 0; w < 2; ++w) for (void* p : pop->sets[w].allocs) cudaFree(p);
    if (pop->e_total_h) cudaFreeHost(pop->e_total_h);
    if (pop->io_h) cudaFreeHost(pop->io_h);
    if (pop->stage) cudaFree(pop->stage);
    if (pop->stage_off) cudaFree(pop->stage_off);
    for (int i = 0; i < NPH; ++i)
        for (int j = 0; j < NREC; ++j) { cudaEventDestroy(pop->ev[i][j][0]); cudaEventDestroy(pop->ev[i][j][1]); }
    if (pop->gev_made)
        for (int i = 0; i < NPH; ++i)
            for (int j = 0; j < NREC; ++j) { cudaEventDestroy(pop->gev[i][j][0]); cudaEventDestroy(pop->gev[i][j][1]); }
    delete pop;
}

int gp_load_trees(gp_pop* pop, const uint8_t* ops, const uint64_t* offsets) {
    if (!pop || !ops || !offsets) return GP_EINVAL;
    const uint32_t P = pop->d.P;
    for (uint32_t i = 0; i < P; ++i) {
        if (offsets[i + 1] <= offsets[i]) return fail(pop, GP_EINVAL, "tree %u is empty or offsets decrease", i);
        if (offsets[i + 1] - offsets[i] > pop->cfg.max_nodes) return fail(pop, GP_ECAPACITY, "tree %u exceeds max_nodes", i);
    }
    const uint64_t total = offsets[P] - offsets[0];
    if (total > pop->stage_cap) {
        if (pop->stage) { cudaStreamSynchronize(pop->stream); cudaFree(pop->stage); cudaFree(pop->stage_off); }
        pop->stage = nullptr; pop->stage_off = nullptr; pop->stage_cap = 0;
        CK(cudaMalloc(&pop->stage, total + 32));
        CK(cudaMalloc(&pop->stage_off, sizeof(uint64_t) * (P + 1)));
        pop->stage_cap = total;
        pop->host_off.resize(P + 1);
        pop->host_buf.resize(P);
        for (uint32_t i = 0; i < P; ++i) pop->host_buf[i] = i;
    }
    for (uint32_t i = 0; i <= P; ++i) pop->host_off[i] = offsets[i] - offsets[0];
    CK(cudaMemcpyAsync(pop->stage, ops + offsets[0], total, cudaMemcpyHostToDevice, pop->stream));
    CK(cudaMemcpyAsync(pop->stage_off, pop->host_off.data(), sizeof(uint64_t) * (P + 1), cudaMemcpyHostToDevice, pop->stream));
    CK(cudaMemcpyAsync(pop->d.buf, pop->host_buf.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, pop->stream));
    k_scatter_trees<<<(P < 4096 ? P : 4096), 256, 0, pop->stream>>>(pop->stage, pop->stage_off, pop->d);
    CK(cudaGetLastError());
    if (pop->host_free.size() != P) {
        pop->host_free.assign(P, 0u);
        for (uint32_t i = 0; i < pop->nbuf - P; ++i) pop->host_free[i] = P + i;
    }
    CK(cudaMemcpyAsync(pop->gb.free_buf, pop->host_free.data(), sizeof(uint32_t) * P, cudaMemcpyHostToDevice, pop->stream));
    pop->host_nfree = pop->nbuf - P;
    // a reload starts over: no device failure of the previous population remains
    CK(cudaMemsetAsync(pop->d.status, 0, sizeof(uint32_t), pop->stream));
    CK(cudaMemsetAsync(pop->d.errinfo, 0, 4 * sizeof(uint32_t), pop->stream));
    CK(cudaMemcpyAsync(pop->gb.nfree, &pop->host_nfree, sizeof(uint32_t), cudaMemcpyHostToDevice, pop->stream));
    CK(cudaMemsetAsync(pop->gb.npend, 0, sizeof(uint32_t), pop->stream));
    pop->have_next_plan = false;
    pop->lazy_pending = false;
    pop->have_children = false;
    pop->gb.evaluated = false;
    return GP_OK;
}

int gp_set_graph_mode(gp_pop* pop, int on, uint64_t reserve_entries) {
    if (!pop) return GP_EINVAL;
    if (!on) {
        if (pop->gexec) { cudaStreamSynchronize(pop->stream); cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
        pop->d.strict_cap = 0;
        return GP_OK;
    }
    int rc = check_status(pop);
    if (rc) return rc;
    uint32_t cur_total = 0;
    CK(cudaMemcpy(&cur_total, pop->d.e_off + pop->d.P, sizeof cur_total, cudaMemcpyDeviceToHost));
    uint64_t want = reserve_entries ? reserve_entries : 2ull * cur_total + 64ull * pop->d.P;
    // the pool holds the entries' values plus the walk's new ones
    const uint64_t room = pop->slot_limit > pop->gb.pvcap ? pop->slot_limit - pop->gb.pvcap : 0;
    if (want > room) want = room;
    if (!reserve_entries && want < cur_total)
        return fail(pop, GP_ENOMEM, "the cache budget cannot hold the current cache");
    // an explicit reservation sets both sets to exactly that size; the
    // default only grows them
    for (int k = 0; k < 2; ++k) {
        const int w = k == 0 ? (pop->cur ^ 1) : pop->cur;
        if (pop->sets[w].Ecap < want || (reserve_entries && pop->sets[w].Ecap != want)) {
            int r = grow_set(pop, w, (uint32_t)want);
            if (r) return r;
            // the current set held the population's values: gp_eval_full must rebuild them
            if (w == pop->cur) pop->gb.evaluated = false;
        }
    }
    pop->d.strict_cap = 1;
    return GP_OK;
}

int gp_graph_capture(gp_pop* pop, uint32_t first_generation, uint32_t n_generations) {
    if (!pop) return GP_EINVAL;
    if (!pop->d.strict_cap) return fail(pop, GP_ESTATE, "gp_graph_capture needs graph mode (gp_set_graph_mode)");
    if (n_generations < 2 || (n_generations & 1u))
        return fail(pop, GP_EINVAL, "n_generations must be even and at least 2 (got %u)", n_generations);
    GenBufs& g = pop->gb;
    if (!g.evaluated || pop->have_children)
        return fail(pop, GP_ESTATE, "gp_graph_capture needs an evaluated population with no pending children");
    if (g.lazy && (!pop->have_next_plan || pop->planned_gen != first_generation))
        return fail(pop, GP_ESTATE, "fitness-first mode: capture after a generation, starting at the planned one");
    int rc = check_status(pop);
    if (rc) return rc;
    if (pop->gexec) { cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
    CK(cudaMemsetAsync(pop->gwords + 1, 0, sizeof(uint32_t), pop->stream));
    CK(cudaStreamSynchronize(pop->stream));
    // capturing runs the host side of every generation without executing it:
    // keep the host state and put it back afterwards (with an even count the
    // double-buffer roles end where they began)
    if (pop->profiling && !pop->gev_made) {
        for (int i = 0; i < NPH; ++i)
            for (int j = 0; j < NREC; ++j) { CK(cudaEventCreate(&pop->gev[i][j][0])); CK(cudaEventCreate(&pop->gev[i][j][1])); }
        pop->gev_made = true;
    }
    // the legacy default stream cannot be captured: capture on a private
    // stream (the graph is then launched on the population's own stream)
    cudaStream_t own = pop->stream;
    if (!own) {
        if (!pop->cap_stream) CK(cudaStreamCreateWithFlags(&pop->cap_stream, cudaStreamNonBlocking));
        pop->stream = pop->cap_stream;
    }
    cudaError_t be = cudaStreamBeginCapture(pop->stream, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
        pop->stream = own;
        cudaGetLastError();
        return fail(pop, GP_ECUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(be));
    }
    const DevPop d0 = pop->d;
    const GenBufs g0 = g;
    const int cur0 = pop->cur;
    const uint32_t calls0 = pop->cum_calls;
    const int kind0 = pop->last_kind;
    const bool dis0 = pop->dis_valid;
    const bool plan0 = pop->have_next_plan, pend0 = pop->lazy_pending;
    const uint32_t pgen0 = pop->planned_gen;
    pop->capturing = true;
    memset(pop->gev_n, 0, sizeof pop->gev_n);
    g.gen_add = pop->gwords + 1;
    uint32_t launches = 0;
    cudaGraph_t graph = nullptr;
    int r = GP_OK;
    for (uint32_t k = 0; k < n_generations && r == GP_OK; ++k) {
        r = gen_crossover(pop, first_generation + k);
        if (r == GP_OK) r = gen_incremental(pop);
        launches += pop->launches;
    }
    if (r == GP_OK) k_graph_advance<<<1, 32, 0, pop->stream>>>(pop->gwords + 1, n_generations);
    cudaError_t ce = cudaStreamEndCapture(pop->stream, &graph);
    pop->stream = own;
    pop->d = d0;
    g = g0;
    pop->cur = cur0;
    bind_set(pop);
    pop->capturing = false;
    pop->graph_prof = pop->profiling;
    pop->cum_calls = calls0;
    pop->have_next_plan = plan0;
    pop->lazy_pending = pend0;
    pop->planned_gen = pgen0;
    pop->last_kind = kind0;
    pop->dis_valid = dis0;
    pop->have_children = false;
    if (r != GP_OK) { if (graph) cudaGraphDestroy(graph); cudaGetLastError(); return r; }
    if (ce != cudaSuccess) { cudaGetLastError(); return fail(pop, GP_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce)); }
    ce = cudaGraphInstantiate(&pop->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { pop->gexec = nullptr; cudaGetLastError(); return fail(pop, GP_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce)); }
    // upload now, so that the first replay does not pay for it
    ce = cudaGraphUpload(pop->gexec, own ? own : 0);
    if (ce != cudaSuccess) { cudaGetLastError(); return fail(pop, GP_ECUDA, "graph upload failed: %s", cudaGetErrorString(ce)); }
    pop->graph_n = n_generations;
    pop->graph_launches = launches + 1;
    return GP_OK;
}

int gp_graph_launch(gp_pop* pop) {
    if (!pop) return GP_EINVAL;
    if (!pop->gexec) return fail(pop, GP_ESTATE, "no captured graph (gp_graph_capture)");
    if (!pop->gb.evaluated || pop->have_children)
        return fail(pop, GP_ESTATE, "gp_graph_launch needs an evaluated population with no pending children");
    CK(cudaGraphLaunch(pop->gexec, pop->stream));
    pop->cum_calls += pop->graph_n;
    if (pop->gb.lazy) {
        pop->planned_gen += pop->graph_n;
        pop->lazy_pending = true;
    }
    pop->stats_graph = pop->graph_prof && pop->profiling;
    pop->launches = pop->graph_launches;
    pop->last_kind = 1;
    pop->dis_valid = pop->gb.dis != nullptr;
    return GP_OK;
}

int gp_set_profiling(gp_pop* pop, int on) {
    if (!pop) return GP_EINVAL;
    pop->profiling = on != 0;
    memset(pop->ev_count, 0, sizeof pop->ev_count);
    CK(cudaMemsetAsync(pop->cum, 0, 4 * sizeof(unsigned long long), pop->stream));
    pop->cum_calls = 0;
    return GP_OK;
}

int gp_set_wait_limit(gp_pop* pop, uint32_t polls) {
    if (!pop) return GP_EINVAL;
    if (pop->stream) CK(cudaStreamSynchronize(pop->stream)); else CK(cudaDeviceSynchronize());
    if (pop->gexec) { cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
    pop->d.wait_polls = polls ? polls : WALK_SPIN;
    return GP_OK;
}

int gp_eval_full(gp_pop* pop) {
    if (!pop) return GP_EINVAL;
    if (pop->lazy_pending)
        return fail(pop, GP_ESTATE, "fitness-first mode keeps only the parents' trees; gp_load_trees before gp_eval_full");
    int rc = run_full(pop);
    if (rc) return rc;
    pop->have_children = false;
    pop->gb.evaluated = true;
    pop->have_next_plan = false;
    return GP_OK;
}

int gp_crossover(gp_pop* pop, uint32_t generation) {
    if (!pop) return GP_EINVAL;
    return gen_crossover(pop, generation);
}

int gp_eval_incremental(gp_pop* pop, gp_stats* stats) {
    if (!pop) return GP_EINVAL;
    int rc = gen_incremental(pop);
    if (rc) return rc;
    if (stats) return gp_get_stats(pop, stats);
    return GP_OK;
}

int gp_fitness(const gp_pop* cpop, float* host_out, uint32_t n) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || !host_out || n > pop->d.P) return GP_EINVAL;
    // the status word and the fitness values in one round trip (the values
    // are not used when the status reports an error)
    CK(cudaMemcpyAsync(pop->io_h, pop->d.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, pop->stream));
    CK(cudaMemcpyAsync(host_out, pop->d.fit, sizeof(float) * n, cudaMemcpyDeviceToHost, pop->stream));
    CK(cudaStreamSynchronize(pop->stream));
    if (pop->io_h[0]) return check_status(pop);
    return GP_OK;
}

int gp_root_values(const gp_pop* cpop, void* host_out, size_t bytes) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || !host_out) return GP_EINVAL;
    const DevPop& d = pop->d;
    const size_t need = (size_t)d.P * d.C * sizeof(float);
    if (bytes < need) return fail(pop, GP_EINVAL, "host buffer too small");
    int rc = check_status(pop);
    if (rc) return rc;
    std::vector<uint32_t> eoff(d.P + 1), slot(1);
    CK(cudaMemcpy(eoff.data(), d.e_off, sizeof(uint32_t) * (d.P + 1), cudaMemcpyDeviceToHost));
    for (uint32_t i = 0; i < d.P; ++i) {
        if (eoff[i + 1] == eoff[i]) {
            // fitness-first mode: a child that is not a parent keeps no cache
            const uint32_t fill = (d.vkind == VB) ? 0u : 0x7FC00000u;
            for (uint32_t k = 0; k < d.C; ++k) memcpy(static_cast<float*>(host_out) + (size_t)i * d.C + k, &fill, 4);
            continue;
        }
        CK(cudaMemcpy(slot.data(), d.e_slot + eoff[i], sizeof(uint32_t), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(static_cast<float*>(host_out) + (size_t)i * d.C, d.slots + (size_t)slot[0] * d.Cpad,
                      sizeof(float) * d.C, cudaMemcpyDeviceToHost));
    }
    return GP_OK;
}

int gp_get_tree(const gp_pop* cpop, uint32_t i, uint8_t* host_out, uint64_t cap, uint64_t* size) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || i >= pop->d.P || !size) return GP_EINVAL;
    // the status word, the tree's size and availability in one round trip;
    // the bytes (assembled on the device when the child is not built) in a second
    const uint32_t lazy_plan = (pop->gb.lazy && pop->have_next_plan) ? 1u : 0u;
    const int nb = (int)((pop->d.cap + 255) / 256) < 2 * pop->nsm ? (int)((pop->d.cap + 255) / 256) : 2 * pop->nsm;
    k_get_tree<<<nb, 256, 0, pop->stream>>>(pop->d, pop->gb, i, lazy_plan, host_out ? pop->tree_out : nullptr,
                                           pop->tree_meta);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pop->io_h, pop->d.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, pop->stream));
    CK(cudaMemcpyAsync(pop->io_h + 1, pop->tree_meta, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, pop->stream));
    CK(cudaStreamSynchronize(pop->stream));
    if (pop->io_h[0]) return check_status(pop);
    const uint32_t n = pop->io_h[1];
    *size = n;
    if (!host_out) return GP_OK;
    if (cap < n) return fail(pop, GP_EINVAL, "host buffer too small for tree %u (%u nodes)", i, n);
    if (!pop->io_h[2]) return fail(pop, GP_ESTATE, "tree %u is no longer available", i);
    CK(cudaMemcpyAsync(host_out, pop->tree_out, n, cudaMemcpyDeviceToHost, pop->stream));
    CK(cudaStreamSynchronize(pop->stream));
    return GP_OK;
}

int gp_cache_entries(const gp_pop* cpop, uint32_t i, uint32_t* pos, uint32_t* end, int32_t* parent,
                     uint32_t nmax, uint32_t* n) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || i >= pop->d.P || !n) return GP_EINVAL;
    int rc = check_status(pop);
    if (rc) return rc;
    uint32_t eo[2];
    CK(cudaMemcpy(eo, pop->d.e_off + i, sizeof eo, cudaMemcpyDeviceToHost));
    uint32_t cnt = eo[1] - eo[0];
    *n = cnt;
    uint32_t m = cnt < nmax ? cnt : nmax;
    if (m == 0) return GP_OK;
    if (pos) CK(cudaMemcpy(pos, pop->d.e_pos + eo[0], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
    if (end) CK(cudaMemcpy(end, pop->d.e_end + eo[0], sizeof(uint32_t) * m, cudaMemcpyDeviceToHost));
    if (parent) {
        CK(cudaMemcpy(parent, pop->d.e_par + eo[0], sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
        for (uint32_t j = 0; j < m; ++j) if (parent[j] >= 0) parent[j] -= (int32_t)eo[0];
    }
    return GP_OK;
}

int gp_cache_value(const gp_pop* cpop, uint32_t i, uint32_t j, void* host_out, size_t bytes) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || i >= pop->d.P || !host_out) return GP_EINVAL;
    if (bytes < sizeof(float) * pop->d.C) return fail(pop, GP_EINVAL, "host buffer too small");
    int rc = check_status(pop);
    if (rc) return rc;
    uint32_t eo[2];
    CK(cudaMemcpy(eo, pop->d.e_off + i, sizeof eo, cudaMemcpyDeviceToHost));
    if (j >= eo[1] - eo[0]) return fail(pop, GP_EINVAL, "entry %u out of range", j);
    uint32_t slot = 0;
    CK(cudaMemcpy(&slot, pop->d.e_slot + eo[0] + j, sizeof slot, cudaMemcpyDeviceToHost));
    // Boolean: the 32-case words in case order (as uint64: 64 cases, low half first)
    CK(cudaMemcpy(host_out, pop->d.slots + (size_t)slot * pop->d.Cpad, sizeof(float) * pop->d.C, cudaMemcpyDeviceToHost));
    return GP_OK;
}

int gp_walk_info(const gp_pop* cpop, int32_t* stop_level, uint32_t* levels, uint32_t n) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || n > pop->d.P) return GP_EINVAL;
    if (pop->last_kind != 1) return fail(pop, GP_ESTATE, "no incremental evaluation has run");
    int rc = check_status(pop);
    if (rc) return rc;
    if (stop_level) CK(cudaMemcpy(stop_level, pop->gb.stop, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    if (levels) CK(cudaMemcpy(levels, pop->gb.plen, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    return GP_OK;
}

int gp_set_disruption(gp_pop* pop, uint32_t max_levels) {
    if (!pop) return GP_EINVAL;
    if (max_levels > 65536u) return fail(pop, GP_EINVAL, "max_levels %u > 65536", max_levels);
    GenBufs& g = pop->gb;
    if (pop->stream) CK(cudaStreamSynchronize(pop->stream)); else CK(cudaDeviceSynchronize());
    if (pop->gexec) { cudaGraphExecDestroy(pop->gexec); pop->gexec = nullptr; pop->graph_n = 0; }
    cudaFree(g.dis);
    cudaFree(g.dis_n);
    g.dis = nullptr;
    g.dis_n = nullptr;
    g.dis_L = 0;
    pop->dis_valid = false;
    if (max_levels == 0) return GP_OK;
    const size_t n = (size_t)pop->d.P * max_levels;
    if (cudaMalloc(&g.dis, n * sizeof(DisLevel)) != cudaSuccess ||
        cudaMalloc(&g.dis_n, (size_t)pop->d.P * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(g.dis); cudaFree(g.dis_n);
        g.dis = nullptr; g.dis_n = nullptr;
        return fail(pop, GP_ENOMEM, "disruption records of %zu levels do not fit", n);
    }
    CK(cudaMemset(g.dis_n, 0, (size_t)pop->d.P * sizeof(uint32_t)));
    g.dis_L = max_levels;
    return GP_OK;
}

int gp_disruption(const gp_pop* cpop, gp_disruption_level* records, size_t n, uint32_t* n_levels) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop) return GP_EINVAL;
    if (pop->last_kind != 1 || !pop->dis_valid || !pop->gb.dis)
        return fail(pop, GP_ESTATE, "no incremental evaluation has recorded disruption since gp_set_disruption");
    const size_t need = (size_t)pop->d.P * pop->gb.dis_L;
    if (records && n < need) return fail(pop, GP_EINVAL, "records holds %zu < %zu entries", n, need);
    int rc = check_status(pop);
    if (rc) return rc;
    if (records) CK(cudaMemcpy(records, pop->gb.dis, need * sizeof(DisLevel), cudaMemcpyDeviceToHost));
    if (n_levels) CK(cudaMemcpy(n_levels, pop->gb.dis_n, sizeof(uint32_t) * pop->d.P, cudaMemcpyDeviceToHost));
    return GP_OK;
}

int gp_pack_info(const gp_pop* cpop, float* predicted, float* measured, float* size_key, uint32_t* order,
                 uint32_t n, float* loss) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || n > pop->d.P) return GP_EINVAL;
    if (pop->last_kind != 1) return fail(pop, GP_ESTATE, "no incremental evaluation has run");
    int rc = check_status(pop);
    if (rc) return rc;
    if (predicted) CK(cudaMemcpy(predicted, pop->mlp.pred_pack, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (measured) CK(cudaMemcpy(measured, pop->mlp.target, sizeof(float) * n, cudaMemcpyDeviceToHost));
    if (size_key) {
        std::vector<float> f((size_t)n * MLP_IN);
        CK(cudaMemcpy(f.data(), pop->mlp.feat, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < n; ++i) size_key[i] = f[(size_t)i * MLP_IN] * 21.f;
    }
    if (order) CK(cudaMemcpy(order, pop->gb.order, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
    if (loss) CK(cudaMemcpy(loss, pop->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost));
    return GP_OK;
}

int gp_mlp_eval_grad(const float* w, const float* x, const float* y, uint32_t n, float* loss, float* grad) {
    if (!w || !x || !y || !loss || !grad || n == 0) return GP_EINVAL;
    MlpBufs b{};
    std::vector<void*> mem;
    auto al = [&](auto** ptr, size_t count) -> bool {
        void* p = nullptr;
        if (cudaMalloc(&p, count * sizeof(**ptr) + 16) != cudaSuccess) { cudaGetLastError(); return false; }
        mem.push_back(p);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(p);
        return true;
    };
    int rc = GP_OK;
    if (!(al(&b.w, MLP_NP) && al(&b.grad, MLP_NP) && al(&b.feat, (size_t)n * MLP_IN) && al(&b.pred, n) &&
          al(&b.target, n) && al(&b.h1, (size_t)n * MLP_H) && al(&b.h2, (size_t)n * MLP_H) && al(&b.dy, n) &&
          al(&b.dh2, (size_t)n * MLP_H) && al(&b.dh1, (size_t)n * MLP_H) && al(&b.loss, 1) &&
          al(&b.part, (size_t)((n + MLP_CH - 1) / MLP_CH) * MLP_NP))) rc = GP_ENOMEM;
    if (rc == GP_OK) {
        cudaMemcpy(b.w, w, sizeof(float) * MLP_NP, cudaMemcpyHostToDevice);
        cudaMemcpy(b.feat, x, sizeof(float) * n * MLP_IN, cudaMemcpyHostToDevice);
        cudaMemcpy(b.target, y, sizeof(float) * n, cudaMemcpyHostToDevice);
        k_mlp_train_pass<<<(n + 7) / 8 < 1024 ? (n + 7) / 8 : 1024, 256>>>(b, n);
        k_mlp_loss<<<1, 256>>>(b, n);
        k_mlp_grad_chunks<<<(n + MLP_CH - 1) / MLP_CH, 256>>>(b, n);
        k_mlp_grad_reduce<<<(MLP_NP + 255) / 256, 256>>>(b, n);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = GP_ECUDA;
        else {
            cudaMemcpy(loss, b.loss, sizeof(float), cudaMemcpyDeviceToHost);
            cudaMemcpy(grad, b.grad, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost);
        }
    }
    for (void* p : mem) cudaFree(p);
    if (rc) g_create_error = "gp_mlp_eval_grad failed";
    return rc;
}

int gp_get_stats(const gp_pop* cpop, gp_stats* out) {
    gp_pop* pop = const_cast<gp_pop*>(cpop);
    if (!pop || !out) return GP_EINVAL;
    int rc = check_status(pop);
    if (rc) return rc;
    gp_stats s = pop->stats;
    for (int i = 0; i < NPH && i < 10; ++i) {
        s.ms[i] = 0.f;
        const bool gr = pop->stats_graph;
        uint32_t n = gr ? pop->gev_n[i] : (pop->ev_count[i] < (uint32_t)NREC ? pop->ev_count[i] : (uint32_t)NREC);
        if (!pop->profiling || n == 0) continue;
        double tot = 0.0;
        uint32_t got = 0;
        for (uint32_t j = 0; j < n; ++j) {
            float ms = 0.f;
            cudaEvent_t a = gr ? pop->gev[i][j][0] : pop->ev[i][j][0];
            cudaEvent_t b = gr ? pop->gev[i][j][1] : pop->ev[i][j][1];
            if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) { tot += ms; ++got; }
            else cudaGetLastError();          // a pair never recorded: skip it, leave no sticky error
        }
        s.ms[i] = got ? (float)(tot / got) : 0.f;     // mean over the recorded calls
    }
    uint32_t ne = 0;
    CK(cudaMemcpy(&ne, pop->d.e_off + pop->d.P, sizeof ne, cudaMemcpyDeviceToHost));
    s.cache_entries = ne;
    s.launches = pop->launches;
    {
        unsigned long long cm[4];
        CK(cudaMemcpy(cm, pop->cum, sizeof cm, cudaMemcpyDeviceToHost));
        s.cum_equivalent_ops = cm[0];
        s.cum_actual_ops = cm[1];
        s.cum_crossover_bytes = cm[2];
        s.cum_calls = pop->cum_calls;
    }
    if (pop->last_kind == 0) {
        unsigned long long acc[4];
        CK(cudaMemcpy(acc, pop->d.acc_ops, sizeof acc, cudaMemcpyDeviceToHost));
        s.actual_ops = acc[0] * pop->cases_stat;
        s.equivalent_ops = acc[1] * pop->cases_stat;
        s.interp_ops = acc[2] * pop->cases_stat;
        s.children = 0;
    } else {
        unsigned long long gs[NGSTAT];
        CK(cudaMemcpy(gs, pop->gb.gstat, sizeof gs, cudaMemcpyDeviceToHost));
        s.equivalent_ops = gs[G_EQUIV] * pop->cases_stat;
        s.interp_ops = gs[G_INTERP] * pop->cases_stat;
        s.actual_ops = (gs[G_INTERP] + gs[G_PATHOPS]) * pop->cases_stat;
        s.crossover_bytes = gs[G_XOBYTES];
        s.path_levels = gs[G_LEVELS];
        s.stopped = (uint32_t)gs[G_STOPPED];
        s.children = pop->d.P;
    }
    *out = s;
    return GP_OK;
}

}  // extern "C"

namespace {

void swap_generation(gp_pop* pop) {
    DevPop& d = pop->d;
    GenBufs& g = pop->gb;
    std::swap(d.buf, g.pbuf);
    std::swap(d.size, g.psize);
    std::swap(d.fit, g.pfit);
}

// The children of at most onepass_nodes nodes, one pass each, on a stream of
// their own (own overflow stacks; their walk records and fitness are
// disjoint from the walk's).  They need only the crossover, so they start
// as soon as it is done, beside the work order; launch_walk joins them.
bool onepass_on(const gp_pop* pop) { return !pop->gb.dis && pop->onepass_nodes; }

template <int K, int V>
int launch_onepass(gp_pop* pop, const CacheView& par) {
    const DevPop& d = pop->d;
    if (!onepass_on(pop)) return GP_OK;
    cudaStream_t os = pop->side3;
    CK(cudaEventRecord(pop->ofork_ev, pop->stream));
    CK(cudaStreamWaitEvent(os, pop->ofork_ev, 0));
    CK(cudaMemsetAsync(pop->gb.op_cnt, 0, sizeof(uint32_t) * 2 * OP_BUCKETS, os));
    CK(cudaMemsetAsync(pop->gb.small_cnt, 0, sizeof(uint32_t) * d.P, os));
    k_onepass_plan<<<pop->nsm * 3, ONEPASS_WARPS * 32, sizeof(OnePassSmem), os>>>(d, pop->gb, par);
    k_onepass_eval<K, V><<<pop->grid_onepass, OP_EVAL_WARPS * 32, pop->smem_onepass, os>>>(d, pop->gb);
    CK(cudaEventRecord(pop->ojoin_ev, os));
    return GP_OK;
}

// The walk: the first walk_long_n children of the work order by the large
// teams on the second stream, the rest by the ordinary teams beside them;
// then the one-pass children are joined.
template <int K, int V>
int launch_walk(gp_pop* pop, const CacheView& par) {
    const DevPop& d = pop->d;
    const bool op = onepass_on(pop);
    const uint32_t nl = pop->walk_long_n;
    if (nl) {
        CK(cudaEventRecord(pop->wfork_ev, pop->stream));
        CK(cudaStreamWaitEvent(pop->side2, pop->wfork_ev, 0));
        const WalkRange wl{0u, nl, (uint32_t)Q_WALK_LONG, 0u};
        // the large teams are dispatched before the ordinary ones (the highest
        // scheduling priority): they carry the longest walks
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)pop->grid_walk_long);
        lc.blockDim = dim3(pop->walk_long_nw * 32);
        lc.dynamicSmemBytes = pop->smem_walk_long;
        lc.stream = pop->side2;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributePriority;
        at[0].val.priority = pop->prio_high;
        lc.attrs = at;
        lc.numAttrs = 1;
        const GenBufs& gb = pop->gb;
        const uint32_t nwl = pop->walk_long_nw;
        if (nwl > 8) CK(cudaLaunchKernelEx(&lc, k_walk<K, V, 512>, d, gb, par, nwl, wl));
        else CK(cudaLaunchKernelEx(&lc, k_walk<K, V, 256>, d, gb, par, nwl, wl));
        CK(cudaEventRecord(pop->wjoin_ev, pop->side2));
    }
    const WalkRange wn{nl, d.P, (uint32_t)Q_WALK, (uint32_t)pop->grid_walk_long * pop->walk_long_nw};
    k_walk<K, V, 256><<<pop->grid_walk, pop->walk_nw * 32, pop->smem_walk, pop->stream>>>(d, pop->gb, par,
                                                                                         pop->walk_nw, wn);
    if (nl) CK(cudaStreamWaitEvent(pop->stream, pop->wjoin_ev, 0));
    if (op) CK(cudaStreamWaitEvent(pop->stream, pop->ojoin_ev, 0));
    return GP_OK;
}

}  // namespace

// Selection, crossover plan, fragment gather and materialisation of the
// children (copy, or in place for the last child of a mother).  The
// parents' trees stay addressable through the retained buffer indices until
// their buffers are overwritten; their cache set is kept for the walk.
// Work order of the coming walk (A10): MLP features and prediction, or the
// mother-size key, and the sort -- on the second stream, as soon as the
// plan exists, beside the crossover kernels; the walk waits for it.
int launch_pack(gp_pop* pop, const CacheView& par) {
    DevPop& d = pop->d;
    GenBufs& g = pop->gb;
    cudaStream_t ms = pop->side;
    CK(cudaEventRecord(pop->pfork_ev, pop->stream));
    CK(cudaStreamWaitEvent(ms, pop->pfork_ev, 0));
    phase_begin(pop, PH_PACK, ms);
    const int pb = (d.P + 255) / 256;
    k_mlp_features<<<(d.P + 7) / 8, 256, 0, ms>>>(d, g, par, pop->mlp);
    const int mb = (d.P + 7) / 8 < pop->nsm * 2 ? (d.P + 7) / 8 : pop->nsm * 2;   // 8 samples per CTA pass
    k_mlp_infer<<<mb, 256, 0, ms>>>(pop->mlp, d.P, pop->mlp.pred_pack);
    pop->pack_launches = 2;
    const dim3 rg((d.P + 255) / 256, (d.P + RANK_TILE - 1) / RANK_TILE);
    // the order of the keys, largest first: one CTA for small populations
    auto rank_order = [&](const float* key) -> int {
        if (d.P <= RANK_SMALL) {
            k_rank_small<<<1, 1024, 0, ms>>>(key, d.P, g.order);
            pop->pack_launches += 1;
        } else {
            CK(cudaMemsetAsync(pop->rank, 0, sizeof(uint32_t) * d.P, ms));
            k_rank_desc<<<rg, 256, 0, ms>>>(key, d.P, pop->rank);
            k_rank_scatter<<<pb, 256, 0, ms>>>(pop->rank, d.P, g.order);
            pop->pack_launches += 2;
        }
        return GP_OK;
    };
    if (pop->cfg.packing == GP_PACK_MLP && d.P <= SORT_MAX) {
        int r = rank_order(pop->mlp.pred_pack);
        if (r) return r;
    } else if (pop->cfg.packing == GP_PACK_STATIC && d.P <= SORT_MAX) {
        k_static_key<<<pb, 256, 0, ms>>>(d, g, pop->mlp);
        pop->pack_launches += 1;
        int r = rank_order(pop->mlp.target);
        if (r) return r;
    } else {
        k_order_identity<<<pb, 256, 0, ms>>>(d, g);
        pop->pack_launches += 1;
    }
    phase_end(pop, PH_PACK, ms);
    CK(cudaEventRecord(pop->pjoin_ev, ms));
    return GP_OK;
}

int gen_crossover(gp_pop* pop, uint32_t generation) {
    DevPop& d = pop->d;
    GenBufs& g = pop->gb;
    if (!g.evaluated) return fail(pop, GP_ESTATE, "gp_crossover needs an evaluated population (gp_eval_full or gp_eval_incremental first)");
    if (pop->have_children) return fail(pop, GP_ESTATE, "children of the last crossover are not evaluated yet");
    if (g.lazy && pop->have_next_plan && generation != pop->planned_gen)
        return fail(pop, GP_ESTATE, "fitness-first mode drew generation %u's plan; gp_crossover(%u) must follow",
                    pop->planned_gen, generation);
    g.gen = generation;
    pop->have_next_plan_at_xo = g.lazy && g.lazy_inplace && pop->have_next_plan;
    swap_generation(pop);
    const CacheView par = view_of(pop, pop->sets[pop->cur]);
    pop->cur ^= 1;
    bind_set(pop);
    phase_begin(pop, PH_XO);
    CK(cudaMemsetAsync(g.lastidx, 0xFF, sizeof(int32_t) * d.P, pop->stream));
    CK(cudaMemsetAsync(g.misc, 0, sizeof(uint32_t) * NMISC, pop->stream));
    CK(cudaMemsetAsync(g.gstat, 0, sizeof(unsigned long long) * NGSTAT, pop->stream));
    if (g.lazy) {
        // fitness-first: the last generation's children built in place in their
        // mothers' buffers (deferred until no sibling reads the mother); then the
        // plan (drawn after the last walk, or now for freshly evaluated parents),
        // fragments and stash; this generation's children are built later
        if (pop->have_next_plan && g.lazy_inplace) {
            k_save_halo<<<pop->nsm * 8, 256, 0, pop->stream>>>(d, g, 1);
            k_shift<<<pop->nsm * 4, 512, 0, pop->stream>>>(d, g, 1);
            k_write_frags<<<pop->nsm * 4, 256, 0, pop->stream>>>(d, g, 1);
            k_inplace_done<<<1, 32, 0, pop->stream>>>(g);
        }
        if (pop->have_next_plan) k_plan_take<<<(d.P + 255) / 256, 256, 0, pop->stream>>>(d, g);
        else k_plan<<<(d.P + 7) / 8, 256, 0, pop->stream>>>(d, g, par);
        {
            int r = launch_pack(pop, par);
            if (r) return r;
        }
        k_assign_lazy<<<1, 1024, 0, pop->stream>>>(d, g);
        k_gather<<<pop->nsm * 4, 256, 0, pop->stream>>>(d, g);
        phase_end(pop, PH_XO);
        CK(cudaGetLastError());
        pop->have_children = true;
        pop->lazy_pending = true;
        g.evaluated = false;
        pop->launches = (pop->have_next_plan_at_xo ? 4u : 0u) + 3u + pop->pack_launches;
        return GP_OK;
    }
    k_plan<<<(d.P + 7) / 8, 256, 0, pop->stream>>>(d, g, par);
    {
        int r = launch_pack(pop, par);
        if (r) return r;
    }
    k_assign<<<1, 1024, 0, pop->stream>>>(d, g);
    k_gather<<<pop->nsm * 4, 256, 0, pop->stream>>>(d, g);
    k_copy_children<<<pop->nsm * 8, 256, 0, pop->stream>>>(d, g);
    k_save_halo<<<pop->nsm * 8, 256, 0, pop->stream>>>(d, g, 0);
    k_shift<<<pop->nsm * 4, 512, 0, pop->stream>>>(d, g, 0);
    k_write_frags<<<pop->nsm * 4, 256, 0, pop->stream>>>(d, g, 0);
    phase_end(pop, PH_XO);
    CK(cudaGetLastError());
    pop->have_children = true;
    g.evaluated = false;
    pop->launches = 7 + pop->pack_launches;
    return GP_OK;
}

// Children's cache structure, the incremental walk, then the children's
// cache values.
int gen_incremental(gp_pop* pop) {
    DevPop& d = pop->d;
    GenBufs& g = pop->gb;
    if (!pop->have_children) return fail(pop, GP_ESTATE, "gp_eval_incremental needs the children of a gp_crossover");
    const CacheView par = view_of(pop, pop->sets[pop->cur ^ 1]);
    const int gt = pop->grid_threads;
    CK(cudaMemsetAsync(d.q, 0, sizeof(uint32_t) * NQ, pop->stream));
    const int pb = (d.P + 255) / 256;
    const int mb = (d.P + 7) / 8 < pop->nsm * 2 ? (d.P + 7) / 8 : pop->nsm * 2;   // 8 samples per CTA pass
    {
        int r = with_kind(d, [&](auto k, auto v) { return launch_onepass<decltype(k)::value, decltype(v)::value>(pop, par); });
        if (r) return r;
    }
    // the work order was computed on the second stream since the crossover
    CK(cudaStreamWaitEvent(pop->stream, pop->pjoin_ev, 0));
    phase_begin(pop, PH_WALK);
    {
        int r = with_kind(d, [&](auto k, auto v) { return launch_walk<decltype(k)::value, decltype(v)::value>(pop, par); });
        if (r) return r;
    }
    phase_end(pop, PH_WALK);
    if (g.lazy) {
        // the next generation's plan from these children's fitness; only the
        // children it selects as parents are built and get a cache
        phase_begin(pop, PH_PLAN);
        CK(cudaMemsetAsync(g.sel, 0, sizeof(uint32_t) * d.P, pop->stream));
        k_plan_next<<<(d.P + 7) / 8, 256, 0, pop->stream>>>(d, g, par);
        k_materialise_assign<<<1, 1024, 0, pop->stream>>>(d, g);
        phase_end(pop, PH_PLAN);
        // the copies on the second stream, beside the cache update (which
        // reads and writes caches only); joined before the generation ends
        CK(cudaEventRecord(pop->cfork_ev, pop->stream));
        CK(cudaStreamWaitEvent(pop->side, pop->cfork_ev, 0));
        phase_begin(pop, PH_MAT, pop->side);
        k_copy_children<<<pop->nsm * 8, 256, 0, pop->side>>>(d, g);
        phase_end(pop, PH_MAT, pop->side);
        CK(cudaEventRecord(pop->cjoin_ev, pop->side));
    }
    phase_begin(pop, PH_CACHE);
    // the walk records grouped per child (fourth stream) beside the children's entry counts
    CK(cudaEventRecord(pop->xfork_ev[0], pop->stream));
    CK(cudaStreamWaitEvent(pop->side3, pop->xfork_ev[0], 0));
    k_pv_offsets<<<1, 1024, 0, pop->side3>>>(d, g);
    k_pv_scatter<<<gt, 256, 0, pop->side3>>>(d, g);
    CK(cudaEventRecord(pop->xjoin_ev[0], pop->side3));
    k_merge_count<<<(d.P + 7) / 8, 256, 0, pop->stream>>>(d, g, par);
    k_merge_offsets<<<1, 1024, 0, pop->stream>>>(d, g);
    if (!d.strict_cap) {
        CK(cudaMemcpyAsync(pop->e_total_h, d.e_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, pop->stream));
        CK(cudaStreamSynchronize(pop->stream));
        if (*pop->e_total_h > d.Ecap) {
            uint64_t want = (uint64_t)*pop->e_total_h + *pop->e_total_h / 4 + 64;
            const uint64_t room = pop->slot_limit > pop->gb.pvcap ? pop->slot_limit - pop->gb.pvcap : 0;
            if (want > room) want = room;
            if (want < *pop->e_total_h) {
                if (g.lazy) cudaStreamWaitEvent(pop->stream, pop->cjoin_ev, 0);
                cudaStreamWaitEvent(pop->stream, pop->xjoin_ev[0], 0);
                return fail(pop, GP_ENOMEM, "cache of %u entries exceeds the cache budget", *pop->e_total_h);
            }
            int r = grow_cache(pop, (uint32_t)want);
            if (r) return r;
            k_merge_offsets<<<1, 1024, 0, pop->stream>>>(d, g);
        }
    }
    // online training of the packing MLP on the levels the walks took, on a
    // second stream beside the rest of the cache update (independent data;
    // joined before the generation ends)
    {
        cudaStream_t ms = pop->side2;
        CK(cudaEventRecord(pop->fork_ev, pop->stream));
        CK(cudaStreamWaitEvent(ms, pop->fork_ev, 0));
        k_mlp_targets<<<pb, 256, 0, ms>>>(d, g, pop->mlp);
        k_mlp_train_pass<<<mb, 256, 0, ms>>>(pop->mlp, d.P);
        k_mlp_loss<<<1, 256, 0, ms>>>(pop->mlp, d.P);
        k_mlp_grad_chunks<<<(d.P + MLP_CH - 1) / MLP_CH, 256, 0, ms>>>(pop->mlp, d.P);
        k_mlp_grad_reduce<<<(MLP_NP + 255) / 256, 256, 0, ms>>>(pop->mlp, d.P);
        k_mlp_adam<<<(MLP_NP + 255) / 256, 256, 0, ms>>>(pop->mlp, pop->mlp_lr);
        k_mlp_bump<<<1, 32, 0, ms>>>(pop->mlp);
        CK(cudaEventRecord(pop->join_ev, ms));
    }
    CK(cudaStreamWaitEvent(pop->stream, pop->xjoin_ev[0], 0));
    k_merge_write<<<d.P < (uint32_t)pop->nsm * 8 ? d.P : pop->nsm * 8, 256, 0, pop->stream>>>(d, g, par);
    // the entries' parent and child links (fourth stream) beside the value-slot pool
    CK(cudaEventRecord(pop->xfork_ev[1], pop->stream));
    CK(cudaStreamWaitEvent(pop->side3, pop->xfork_ev[1], 0));
    k_entry_chunkmax<<<pop->grid_warps, GP_WARPS * 32, 0, pop->side3>>>(d, pop->sb);
    k_entry_parents<<<gt, 256, 0, pop->side3>>>(d, pop->sb);
    k_child_sizes<<<(d.P + 255) / 256, 256, 0, pop->side3>>>(d, g);
    CK(cudaEventRecord(pop->xjoin_ev[1], pop->side3));
    k_mark_live<<<gt, 256, 0, pop->stream>>>(d, g);
    k_free_count<<<pop->nsm * 2, 1024, 0, pop->stream>>>(d, g);
    k_free_top<<<1, 1024, 0, pop->stream>>>(d, g);
    k_free_emit<<<pop->nsm * 2, 1024, 0, pop->stream>>>(d, g);
    k_copy_values<<<pop->nsm * 16, 256, 0, pop->stream>>>(d, g, par);
    k_check_slots<<<gt, 256, 0, pop->stream>>>(d);
    CK(cudaStreamWaitEvent(pop->stream, pop->xjoin_ev[1], 0));
    CK(cudaStreamWaitEvent(pop->stream, pop->join_ev, 0));
    if (g.lazy) CK(cudaStreamWaitEvent(pop->stream, pop->cjoin_ev, 0));
    phase_end(pop, PH_CACHE);
    k_accumulate<<<1, 32, 0, pop->stream>>>(pop->cum, d.acc_ops, g.gstat, pop->cases_stat, 1);
    ++pop->cum_calls;
    CK(cudaGetLastError());
    // walk (and the large teams), one-pass plan and evaluation, next plan and
    // copies (fitness-first order, 3), walk records (2), merge counts (2),
    // MLP training (7), merge, links (3), slot pool (6), statistics
    pop->launches += 1 + (pop->walk_long_n ? 1u : 0u) + (onepass_on(pop) ? 2u : 0u) + (g.lazy ? 3u : 0u) + 2 + 2 + 7 +
                     1 + 3 + 6 + 1;
    pop->have_children = false;
    g.evaluated = true;
    pop->last_kind = 1;
    pop->dis_valid = g.dis != nullptr;
    if (g.lazy) {
        pop->have_next_plan = true;
        pop->planned_gen = g.gen + 1;
    }
    return GP_OK;
}
