// Batched launch of many independent 2-D problems (a pattern layered on the
// method; the paper advances one mesh at a time).
//
// Every RK4 stage of all problems of a batch is two persistent kernels that
// run side by side (two branches of one CUDA graph): one over the elements
// of the variable-coefficient problems (element PCG; 81+ threads and ~75-115
// KB of shared memory per element) and one over tiles of elements of the
// constant-coefficient problems (modal route; a few KB per element).  Each
// is a grid of (SMs x resident blocks) CTAs pulling items from its own queue,
// so uneven meshes and degrees balance without per-problem launches and the
// two kinds of work share the SMs.  The stage bodies are the per-problem
// kernels' own (stage2p_body, var_stage_body), so a batched step computes
// exactly what the problem's own gdg_step computes.  A call's launches are
// captured once in a CUDA graph (per-problem dt lives in device descriptors,
// so the graph does not depend on it).  The modal tile (elements per block)
// and the PCG grid size are picked on the first step by timing the
// candidates on the batch's own data.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gdg_internal.h"
#include "gdg_stage_const.cuh"
#include "gdg_var_kernels.cuh"

namespace {

struct BatchProb {
    int kind;                 // 0 modal route (constant coefficients), 1 element PCG
    const ModalParams *mp;    // kind 0: device copy of the problem's modal parameters
    const double *lam2;       // kind 0
    VarParams vp;             // kind 1
    StepBuffers sb;
    double dt;
};

constexpr int kMaxBatchThreads = 256;

// RK4 stage coefficients and buffer roles of stage STAGE (the same table as
// the per-problem stage launches)
template <int STAGE>
struct StageRoles {
    double cA, cY;
    const double *yU, *yV, *trin;
    double *oU, *oV, *trout;
    __host__ __device__ StageRoles(const StepBuffers &B, double dt) {
        if (STAGE == 1) {
            cA = dt / 6.0; cY = 0.5 * dt; yU = B.nU; yV = B.nV; oU = B.xU; oV = B.xV; trin = B.tr0; trout = B.tr1;
        } else if (STAGE == 2) {
            cA = dt / 3.0; cY = 0.5 * dt; yU = B.xU; yV = B.xV; oU = B.yU; oV = B.yV; trin = B.tr1; trout = B.tr0;
        } else if (STAGE == 3) {
            cA = dt / 3.0; cY = dt; yU = B.yU; yV = B.yV; oU = B.xU; oV = B.xV; trin = B.tr0; trout = B.tr1;
        } else {
            cA = dt / 6.0; cY = 0.0; yU = B.xU; yV = B.xV; oU = nullptr; oV = nullptr; trin = B.tr1; trout = B.tr0;
        }
    }
};

// next work item of the block's queue, broadcast through shared memory
__device__ __forceinline__ int next_item(unsigned int *counter, int *slot) {
    if (threadIdx.x == 0) *slot = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = *slot;
    __syncthreads();
    return it;
}

// block-wide copy of a parameter struct into shared memory (whole 4-byte words)
template <typename T>
__device__ __forceinline__ void copy_to_shared(T *dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const unsigned int *s = reinterpret_cast<const unsigned int *>(src);
    unsigned int *d = reinterpret_cast<unsigned int *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// modal tiles of the constant-coefficient problems
template <int N1, int STAGE>
__global__ void __launch_bounds__(kMaxBatchThreads)
k_batch_modal(const BatchProb *__restrict__ probs, const int2 *__restrict__ items, int n_items,
              unsigned int *counter) {
    constexpr int MODE = STAGE == 1 ? M_S1 : (STAGE == 4 ? M_S4 : M_S23);
    extern __shared__ double smem[];
    __shared__ int s_item;
    __shared__ ModalParams s_mp;   // the current problem's parameters (read in every inner loop)
    int cur = -1;
    for (int it = next_item(counter, &s_item); it < n_items; it = next_item(counter, &s_item)) {
        const int2 w = items[it];
        const BatchProb &P = probs[w.x];
        if (w.x != cur) {
            copy_to_shared(&s_mp, P.mp);
            cur = w.x;
        }
        const StageRoles<STAGE> r(P.sb, P.dt);
        const StageBufs b{r.yU, r.yV, P.sb.nU, P.sb.nV, P.sb.aU, P.sb.aV, r.oU, r.oV, r.trin, r.trout, P.lam2};
        if (s_mp.alt) stage2p_body<N1, MODE, 1>(s_mp, b, r.cA, r.cY, w.y, smem);
        else stage2p_body<N1, MODE, 0>(s_mp, b, r.cA, r.cY, w.y, smem);
        __syncthreads();
    }
}

// elements of the variable-coefficient problems (one element PCG per item).
// The current problem's parameters and buffer table live in shared memory
// (kernel parameters would sit in the constant bank; in registers they would
// crowd the PCG loops).
template <int N1, int STAGE>
__device__ __forceinline__ void batch_var_item(const BatchProb *__restrict__ probs, int2 w, int &cur,
                                               VarParams &s_vp, VarBufs &s_b, double *s_c, double *smem) {
    constexpr int MODE = STAGE == 1 ? M_S1 : (STAGE == 4 ? M_S4 : M_S23);
    if (w.x != cur) {
        const BatchProb &P = probs[w.x];
        copy_to_shared(&s_vp, &P.vp);
        if (threadIdx.x == 0) {
            const StageRoles<STAGE> r(P.sb, P.dt);
            s_b = VarBufs{r.yU, r.yV, P.sb.nU, P.sb.nV, P.sb.aU, P.sb.aV, r.oU, r.oV, r.trin, r.trout};
            s_c[0] = r.cA;
            s_c[1] = r.cY;
        }
        __syncthreads();
        cur = w.x;
    }
    var_stage_body<N1, MODE>(s_vp, s_b, s_c[0], s_c[1], w.y, smem);
}

// flat grid: block b takes item b
template <int N1, int STAGE>
__global__ void __launch_bounds__(nthreads_for(N1 * N1), kVarMinBlocks)
k_batch_var(const BatchProb *__restrict__ probs, const int2 *__restrict__ items, int n_items, unsigned int *) {
    extern __shared__ double smem[];
    __shared__ VarParams s_vp;
    __shared__ VarBufs s_b;
    __shared__ double s_c[2];
    int cur = -1;
    if ((int)blockIdx.x < n_items)
        batch_var_item<N1, STAGE>(probs, items[blockIdx.x], cur, s_vp, s_b, s_c, smem);
}

// persistent grid: blocks pull items from the queue `counter`
template <int N1, int STAGE>
__global__ void __launch_bounds__(nthreads_for(N1 * N1), kVarMinBlocks)
k_batch_var_q(const BatchProb *__restrict__ probs, const int2 *__restrict__ items, int n_items,
              unsigned int *counter) {
    extern __shared__ double smem[];
    __shared__ int s_item;
    __shared__ VarParams s_vp;
    __shared__ VarBufs s_b;
    __shared__ double s_c[2];
    int cur = -1;
    for (int it = next_item(counter, &s_item); it < n_items; it = next_item(counter, &s_item)) {
        batch_var_item<N1, STAGE>(probs, items[it], cur, s_vp, s_b, s_c, smem);
        __syncthreads();
    }
}

#define GDG_BATCH_CASES(X) X(8) X(9) X(10)

// dynamic shared memory may use the opt-in maximum minus the kernel's own
// static shared memory (the work-item slot)
template <typename K>
cudaError_t raise_smem(K kernel, int lim) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)a.sharedSizeBytes);
}

template <int N1>
cudaError_t set_batch_attrs() {
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e;
    if ((e = raise_smem(k_batch_modal<N1, 1>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_modal<N1, 2>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_modal<N1, 3>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_modal<N1, 4>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_var_stage<N1, M_S1>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_var_stage<N1, M_S23>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_var_stage<N1, M_S4>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var<N1, 1>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var<N1, 2>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var<N1, 3>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var<N1, 4>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var_q<N1, 1>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var_q<N1, 2>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_var_q<N1, 3>, lim)) != cudaSuccess) return e;
    return raise_smem(k_batch_var_q<N1, 4>, lim);
}

template <int N1, bool VAR>
void launch_batch_n(int stage, int grid, int threads, size_t smem, const BatchProb *probs, const int2 *items,
                    int n_items, unsigned int *counter, cudaStream_t s) {
#define GDG_BK(st) (VAR ? (counter ? k_batch_var_q<N1, st> : k_batch_var<N1, st>) : k_batch_modal<N1, st>)
    switch (stage) {
    case 1: GDG_BK(1)<<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    case 2: GDG_BK(2)<<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    case 3: GDG_BK(3)<<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    default: GDG_BK(4)<<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    }
#undef GDG_BK
}

}  // namespace

struct gdg_batch {
    std::vector<gdg_ctx *> ctx;
    int count = 0, n1 = 0, sms = 152;
    BatchProb *d_probs = nullptr;
    ModalParams *d_mps = nullptr;
    int2 *d_var_items = nullptr, *d_mod_items = nullptr;
    int n_var = 0, n_mod = 0, mod_cap = 0, mod_tile = -1;
    unsigned int *d_counters = nullptr;   // per step: [stage 0..3][kind 0 var, 1 modal]
    size_t var_smem = 0;
    int var_threads = 0, var_grid = 0;    // PCG launch
    int mod_threads = 0, mod_grid = 0;    // modal launch (tile = mod_threads / n1)
    bool tuned = false;
    cudaStream_t cap = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = 0;
    std::vector<BatchProb> h_probs;
    std::string err;
};

namespace {

int berr(gdg_batch *b, int st, const std::string &m) {
    if (b) b->err = m;
    std::fprintf(stderr, "gdg_batch: %s\n", m.c_str());
    return st;
}

size_t modal_smem(int n1, int tile) { return (size_t)tile * (4 * n1 + 2 * n1 * (n1 + 1)) * sizeof(double); }

int upload_items(gdg_batch *b, const std::vector<int2> &items, int2 **dst, int *cap) {
    if ((int)items.size() > *cap) {
        cudaFree(*dst);
        *dst = nullptr;
        if (cudaMalloc((void **)dst, std::max<size_t>(1, items.size()) * sizeof(int2)) != cudaSuccess)
            return berr(b, GDG_ENOMEM, "items");
        *cap = (int)items.size();
    }
    if (!items.empty() &&
        cudaMemcpy(*dst, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
        return berr(b, GDG_ECUDA, "items upload");
    return GDG_OK;
}

// modal work items: tiles of `tile` elements of the constant-coefficient problems
int build_modal_items(gdg_batch *b, int tile) {
    if (tile == b->mod_tile) return GDG_OK;
    std::vector<int2> items;
    for (int i = 0; i < b->count; ++i)
        if (b->h_probs[i].kind == 0)
            for (int t = 0; t * tile < b->ctx[i]->ne; ++t) items.push_back(make_int2(i, t));
    int st = upload_items(b, items, &b->d_mod_items, &b->mod_cap);
    if (st) return st;
    b->n_mod = (int)items.size();
    b->mod_tile = tile;
    return GDG_OK;
}

template <typename K>
int resident_blocks(K kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) return 1;
    return std::max(1, n);
}

int max_resident(const gdg_batch *b, bool var, int threads, size_t smem) {
    switch (b->n1) {
#define X(n) case n: return var ? resident_blocks(k_batch_var_q<n, 2>, threads, smem) \
                                : resident_blocks(k_batch_modal<n, 2>, threads, smem);
        GDG_BATCH_CASES(X)
#undef X
    }
    return 1;
}

// The element-PCG stage as one launch per variable-coefficient problem: the
// problem's own stage kernel, its parameters as kernel arguments (no per-block
// staging), in problem order on one stream.  Same kernel body as the batched
// launches and as gdg_step.
template <int N1>
void launch_var_per_problem_n(const gdg_batch *b, int stage, cudaStream_t s) {
    constexpr int T = nthreads_for(N1 * N1);
    for (const BatchProb &P : b->h_probs) {
        if (P.kind != 1) continue;
        const size_t sm = StageSmem<N1>::bytes(P.vp.Q, P.vp.mixed, P.vp.inverse);
        switch (stage) {
#define GDG_PP(st, mode)                                                                                  \
    {                                                                                                     \
        const StageRoles<st> r(P.sb, P.dt);                                                               \
        const VarBufs vb{r.yU, r.yV, P.sb.nU, P.sb.nV, P.sb.aU, P.sb.aV, r.oU, r.oV, r.trin, r.trout};    \
        k_var_stage<N1, mode><<<P.vp.ne, T, sm, s>>>(P.vp, vb, r.cA, r.cY);                               \
    }
        case 1: GDG_PP(1, M_S1) break;
        case 2: GDG_PP(2, M_S23) break;
        case 3: GDG_PP(3, M_S23) break;
        default: GDG_PP(4, M_S4) break;
#undef GDG_PP
        }
    }
}

// kind 0: PCG elements; kind 1: modal tiles
void launch_kind(gdg_batch *b, int kind, int stage, unsigned int *counter, cudaStream_t s) {
    const bool var = kind == 0;
    const int n = var ? b->n_var : b->n_mod;
    if (!n) return;
    if (var && b->var_grid == -1) {   // one launch per problem
        switch (b->n1) {
#define X(n1_) case n1_: launch_var_per_problem_n<n1_>(b, stage, s); break;
            GDG_BATCH_CASES(X)
#undef X
        }
        return;
    }
    const int threads = var ? b->var_threads : b->mod_threads;
    const int grid = var ? (b->var_grid > 0 ? b->var_grid : n) : b->mod_grid;
    if (var && b->var_grid <= 0) counter = nullptr;   // flat grid
    const size_t smem = var ? b->var_smem : modal_smem(b->n1, b->mod_threads / b->n1);
    const int2 *items = var ? b->d_var_items : b->d_mod_items;
    switch (b->n1) {
#define X(n1_)                                                                                          \
    case n1_:                                                                                          \
        if (var) launch_batch_n<n1_, true>(stage, grid, threads, smem, b->d_probs, items, n, counter, s);  \
        else launch_batch_n<n1_, false>(stage, grid, threads, smem, b->d_probs, items, n, counter, s);     \
        break;
        GDG_BATCH_CASES(X)
#undef X
    }
}

// one RK4 step: reset the 8 queue counters, then per stage the two launches
// on two streams, joined before the next stage
void enqueue_steps(gdg_batch *b, int nsteps, cudaStream_t s) {
    for (int i = 0; i < nsteps; ++i) {
        cudaMemsetAsync(b->d_counters, 0, 8 * sizeof(unsigned int), s);
        for (int st = 1; st <= 4; ++st) {
            cudaEventRecord(b->fork, s);
            cudaStreamWaitEvent(b->side, b->fork, 0);
            launch_kind(b, 0, st, b->d_counters + 2 * (st - 1), s);
            launch_kind(b, 1, st, b->d_counters + 2 * (st - 1) + 1, b->side);
            cudaEventRecord(b->join, b->side);
            cudaStreamWaitEvent(s, b->join, 0);
        }
    }
}

float time_launch(gdg_batch *b, int kind, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaMemsetAsync(b->d_counters, 0, 8 * sizeof(unsigned int), s);
        cudaEventRecord(e0, s);
        launch_kind(b, kind, 1, b->d_counters + kind, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    return cudaGetLastError() == cudaSuccess ? ms : 1e30f;
}

// Time the candidates on the batch's own stage-1 work (stage 1 reads y_n and
// its traces and writes only buffers that the real step rewrites).
int autotune(gdg_batch *b, cudaStream_t s) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int st = GDG_OK;
    if (b->n_var) {   // PCG launch: flat grid, persistent with 1..occupancy-limit blocks per SM, or per problem
        const int maxr = max_resident(b, true, b->var_threads, b->var_smem);
        b->var_grid = 0;
        float best = time_launch(b, 0, s, e0, e1);
        int best_g = 0;
        for (int r = 1; r <= maxr; ++r) {
            b->var_grid = b->sms * r;
            const float ms = time_launch(b, 0, s, e0, e1);
            if (ms < best) { best = ms; best_g = b->var_grid; }
        }
        b->var_grid = -1;
        if (time_launch(b, 0, s, e0, e1) < best) best_g = -1;
        b->var_grid = best_g;
    }
    bool any_modal = false;
    for (const BatchProb &P : b->h_probs) any_modal |= P.kind == 0;
    if (any_modal) {  // modal tile: elements per block
        float best = 1e30f;
        int best_t = 0;
        for (int tile : {4, 7, 10, 14, 21, 28}) {
            const int threads = tile * b->n1;
            if (threads > kMaxBatchThreads) continue;
            if ((st = build_modal_items(b, tile))) break;
            b->mod_threads = threads;
            b->mod_grid = b->sms * max_resident(b, false, threads, modal_smem(b->n1, tile));
            const float ms = time_launch(b, 1, s, e0, e1);
            if (ms < best) { best = ms; best_t = tile; }
        }
        if (!st && best_t) {
            st = build_modal_items(b, best_t);
            b->mod_threads = best_t * b->n1;
            b->mod_grid = b->sms * max_resident(b, false, b->mod_threads, modal_smem(b->n1, best_t));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    b->tuned = true;
    return GDG_OK;
}

}  // namespace

extern "C" int gdg_batch_destroy(gdg_batch *b) {
    if (!b) return GDG_EINVAL;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    cudaFree(b->d_probs);
    cudaFree(b->d_mps);
    cudaFree(b->d_var_items);
    cudaFree(b->d_mod_items);
    cudaFree(b->d_counters);
    for (gdg_ctx *c : b->ctx) gdg_destroy(c);
    delete b;
    return GDG_OK;
}

extern "C" int gdg_batch_create(const gdg_problem *pbs, int count, gdg_batch **out) {
    if (!pbs || !out || count < 1) return GDG_EINVAL;
    *out = nullptr;
    gdg_batch *b = new (std::nothrow) gdg_batch();
    if (!b) return GDG_ENOMEM;
    b->count = count;
    b->n1 = pbs[0].N + 1;
    int st = GDG_OK;
    for (int i = 0; i < count && !st; ++i) {
        if (pbs[i].dim != 2 || pbs[i].N + 1 != b->n1) st = berr(b, GDG_EINVAL, "batch problems must be 2-D with one N");
        else if (b->n1 < 8 || b->n1 > 10) st = berr(b, GDG_EUNSUPPORTED, "batches support N = 7..9");
        else if (pbs[i].rows[0] || pbs[i].rows[1]) st = berr(b, GDG_EUNSUPPORTED, "batch problems are whole meshes (no bands of rows)");
    }
    if (st) { gdg_batch_destroy(b); return st; }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->ctx.assign(count, nullptr);
    b->h_probs.resize(count);
    std::vector<ModalParams> mps(count);
    std::vector<int2> var_items;
    for (int i = 0; i < count; ++i) {
        if ((st = gdg_create(&pbs[i], &b->ctx[i]))) { gdg_batch_destroy(b); return st; }
        gdg_ctx *c = b->ctx[i];
        BatchProb &P = b->h_probs[i];
        std::memset(&P, 0, sizeof(P));
        if (pbs[i].coef == GDG_COEF_CONST) {
            if (!c->mp.parity) { gdg_batch_destroy(b); return berr(nullptr, GDG_EUNSUPPORTED, "modal basis without parity"); }
            P.kind = 0;
            P.lam2 = c->d_lam2;
            P.sb = gdg_const_buffers(c);
            mps[i] = c->mp;
        } else {
            P.kind = 1;
            P.vp = c->var->vp;
            P.sb = gdg_var_buffers(c);
            b->var_smem = std::max(b->var_smem, c->var->smem_stage);
            for (int e = 0; e < c->ne; ++e) var_items.push_back(make_int2(i, e));
        }
    }
    // longest items first (higher order: more quadrature points per face), so
    // that the last blocks of a stage are short ones
    std::stable_sort(var_items.begin(), var_items.end(), [&](const int2 &a, const int2 &c) {
        return pbs[a.x].p > pbs[c.x].p;
    });
    int cap = 0;
    if (cudaMalloc((void **)&b->d_mps, count * sizeof(ModalParams)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_probs, count * sizeof(BatchProb)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_counters, 8 * sizeof(unsigned int)) != cudaSuccess ||
        upload_items(b, var_items, &b->d_var_items, &cap)) {
        gdg_batch_destroy(b);
        return GDG_ENOMEM;
    }
    b->n_var = (int)var_items.size();
    b->var_threads = nthreads_for(b->n1 * b->n1);
    for (int i = 0; i < count; ++i)
        if (b->h_probs[i].kind == 0) b->h_probs[i].mp = b->d_mps + i;
    cudaMemcpy(b->d_mps, mps.data(), count * sizeof(ModalParams), cudaMemcpyHostToDevice);
    cudaMemcpy(b->d_probs, b->h_probs.data(), count * sizeof(BatchProb), cudaMemcpyHostToDevice);
    cudaError_t ae = cudaSuccess;
    switch (b->n1) {
#define X(n) case n: ae = set_batch_attrs<n>(); break;
        GDG_BATCH_CASES(X)
#undef X
    }
    if (ae != cudaSuccess) {
        gdg_batch_destroy(b);
        return berr(nullptr, GDG_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ae));
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess) {
        gdg_batch_destroy(b);
        return GDG_ECUDA;
    }
    *out = b;
    return GDG_OK;
}

extern "C" long long gdg_batch_state_len(const gdg_batch *b, int i) {
    if (!b || i < 0 || i >= b->count) return -1;
    return b->ctx[i]->ndof;
}

extern "C" int gdg_batch_step(gdg_batch *b, double *const *u, double *const *v, const double *dt, int nsteps,
                              void *stream) {
    if (!b || !u || !v || !dt || nsteps < 0) return GDG_EINVAL;
    for (int i = 0; i < b->count; ++i)
        if (!u[i] || !v[i] || !(dt[i] > 0.0)) return GDG_EINVAL;
    if (nsteps == 0) return GDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int st;
    bool dt_changed = false;
    for (int i = 0; i < b->count; ++i)
        if (b->h_probs[i].dt != dt[i]) { b->h_probs[i].dt = dt[i]; dt_changed = true; }
    if (dt_changed &&
        cudaMemcpyAsync(b->d_probs, b->h_probs.data(), b->count * sizeof(BatchProb), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return berr(b, GDG_ECUDA, "descriptor upload");
    for (int i = 0; i < b->count; ++i) {
        gdg_ctx *c = b->ctx[i];
        st = c->pb.coef == GDG_COEF_CONST ? gdg_const_enter(c, u[i], v[i], s) : gdg_var_enter(c, u[i], v[i], s);
        if (st) return berr(b, st, "enter: " + c->err);
    }
    if (!b->tuned && (st = autotune(b, s))) return st;
    // graph of G steps, replayed
    const int G = 4;
    if (nsteps >= G) {
        if (!b->exec || b->graph_steps != G) {
            cudaGraph_t g;
            if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return berr(b, GDG_ECUDA, "capture");
            enqueue_steps(b, G, b->cap);
            if (cudaStreamEndCapture(b->cap, &g) != cudaSuccess) return berr(b, GDG_ECUDA, "capture end");
            const cudaError_t e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return berr(b, GDG_ECUDA, "instantiate");
            b->graph_steps = G;
        }
        for (int i = 0; i + G <= nsteps; i += G)
            if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return berr(b, GDG_ECUDA, "graph launch");
    }
    enqueue_steps(b, nsteps >= G ? nsteps % G : nsteps, s);
    for (int i = 0; i < b->count; ++i) {
        gdg_ctx *c = b->ctx[i];
        st = c->pb.coef == GDG_COEF_CONST ? gdg_const_leave(c, u[i], v[i], s) : gdg_var_leave(c, u[i], v[i], s);
        if (st) return berr(b, st, "leave");
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GDG_OK : berr(b, GDG_ECUDA, cudaGetErrorString(e));
}

extern "C" int gdg_batch_tuning(const gdg_batch *b, int *threads_per_block, int *blocks_per_sm, int *tile_elements) {
    if (!b) return GDG_EINVAL;
    const bool mod = b->tuned && b->n_mod > 0, var = b->tuned && b->n_var > 0;
    if (threads_per_block) *threads_per_block = mod ? b->mod_threads : 0;
    if (blocks_per_sm)
        *blocks_per_sm = var && b->sms && b->var_grid > 0 ? b->var_grid / b->sms : (var ? (b->var_grid == -1 ? -2 : -1) : 0);
    if (tile_elements) *tile_elements = mod ? b->mod_tile : 0;
    return GDG_OK;
}

extern "C" int gdg_batch_stats(gdg_batch *b, int i, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys) {
    if (!b || i < 0 || i >= b->count) return GDG_EINVAL;
    return gdg_step_stats(b->ctx[i], u_sys, v_sys);
}
