// Batched launch of many independent 2-D problems (a pattern layered on the
// method; the paper advances one mesh at a time).
//
// Every RK4 stage of all problems of a batch is one persistent kernel: a
// grid of (SMs x resident blocks) CTAs pulls work items from a queue -- first
// the elements of the variable-coefficient problems (element PCG, the
// expensive items), then tiles of elements of the constant-coefficient
// problems (modal route) -- so the long items start first and the short ones
// fill the tail.  The stage bodies are the per-problem kernels' own
// (stage2p_body, var_stage_body), so a batched step computes exactly what the
// problem's own gdg_step computes.  A call's launches are captured once in a
// CUDA graph (per-problem dt lives in device descriptors, so the graph does
// not depend on it).  The launch shape -- threads per block (which also sets
// the modal tile, threads / (N+1) elements) and resident blocks per SM -- is
// picked on the first step by timing every candidate on the batch's data.
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

template <int N1, int STAGE>
__global__ void __launch_bounds__(kMaxBatchThreads)
k_batch_stage(const BatchProb *__restrict__ probs, const int2 *__restrict__ items, int n_items,
              unsigned int *counter) {
    constexpr int MODE = STAGE == 1 ? M_S1 : (STAGE == 4 ? M_S4 : M_S23);
    extern __shared__ double smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const int2 w = items[it];
        const BatchProb &P = probs[w.x];
        const StepBuffers &B = P.sb;
        const double dt = P.dt;
        double cA, cY;
        const double *yU, *yV, *trin;
        double *oU, *oV, *trout;
        if (STAGE == 1) {
            cA = dt / 6.0; cY = 0.5 * dt; yU = B.nU; yV = B.nV; oU = B.xU; oV = B.xV; trin = B.tr0; trout = B.tr1;
        } else if (STAGE == 2) {
            cA = dt / 3.0; cY = 0.5 * dt; yU = B.xU; yV = B.xV; oU = B.yU; oV = B.yV; trin = B.tr1; trout = B.tr0;
        } else if (STAGE == 3) {
            cA = dt / 3.0; cY = dt; yU = B.yU; yV = B.yV; oU = B.xU; oV = B.xV; trin = B.tr0; trout = B.tr1;
        } else {
            cA = dt / 6.0; cY = 0.0; yU = B.xU; yV = B.xV; oU = nullptr; oV = nullptr; trin = B.tr1; trout = B.tr0;
        }
        if (P.kind == 0) {
            const StageBufs b{yU, yV, B.nU, B.nV, B.aU, B.aV, oU, oV, trin, trout, P.lam2};
            stage2p_body<N1, MODE>(*P.mp, b, cA, cY, w.y, smem);
        } else {
            const VarBufs b{yU, yV, B.nU, B.nV, B.aU, B.aV, oU, oV, trin, trout};
            var_stage_body<N1, MODE>(P.vp, b, cA, cY, w.y, smem);
        }
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
    if ((e = raise_smem(k_batch_stage<N1, 1>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_stage<N1, 2>, lim)) != cudaSuccess) return e;
    if ((e = raise_smem(k_batch_stage<N1, 3>, lim)) != cudaSuccess) return e;
    return raise_smem(k_batch_stage<N1, 4>, lim);
}

template <int N1>
void launch_batch_n(int stage, int grid, int threads, size_t smem, const BatchProb *probs, const int2 *items,
                    int n_items, unsigned int *counter, cudaStream_t s) {
    switch (stage) {
    case 1: k_batch_stage<N1, 1><<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    case 2: k_batch_stage<N1, 2><<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    case 3: k_batch_stage<N1, 3><<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    default: k_batch_stage<N1, 4><<<grid, threads, smem, s>>>(probs, items, n_items, counter); break;
    }
}

}  // namespace

struct gdg_batch {
    std::vector<gdg_ctx *> ctx;
    int count = 0, n1 = 0, sms = 152;
    BatchProb *d_probs = nullptr;
    ModalParams *d_mps = nullptr;
    int2 *d_items = nullptr;
    int n_items = 0, items_cap = 0, item_tile = -1;
    unsigned int *d_counters = nullptr;
    static constexpr int kCounters = 64;
    size_t var_smem = 0;
    int threads = 0, bpsm = 0;   // tuned launch shape (0: not tuned yet)
    cudaStream_t cap = nullptr;
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

size_t batch_smem(const gdg_batch *b, int threads) {
    const int n1 = b->n1, tile = threads / n1;
    size_t sm = (size_t)tile * (4 * n1 + 2 * n1 * (n1 + 1)) * sizeof(double);   // modal tile
    return std::max(sm, b->var_smem);
}

// work items: every element of the PCG problems, then tiles of `tile` elements
// of the modal problems
int build_items(gdg_batch *b, int tile) {
    if (tile == b->item_tile) return GDG_OK;
    std::vector<int2> items;
    for (int i = 0; i < b->count; ++i)
        if (b->h_probs[i].kind == 1)
            for (int e = 0; e < b->ctx[i]->ne; ++e) items.push_back(make_int2(i, e));
    for (int i = 0; i < b->count; ++i)
        if (b->h_probs[i].kind == 0)
            for (int t = 0; t * tile < b->ctx[i]->ne; ++t) items.push_back(make_int2(i, t));
    if ((int)items.size() > b->items_cap) {
        cudaFree(b->d_items);
        b->d_items = nullptr;
        if (cudaMalloc((void **)&b->d_items, items.size() * sizeof(int2)) != cudaSuccess)
            return berr(b, GDG_ENOMEM, "items");
        b->items_cap = (int)items.size();
    }
    if (cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
        return berr(b, GDG_ECUDA, "items upload");
    b->n_items = (int)items.size();
    b->item_tile = tile;
    return GDG_OK;
}

void launch_stage(gdg_batch *b, int stage, int counter, cudaStream_t s) {
    const int grid = b->sms * b->bpsm;
    const size_t smem = batch_smem(b, b->threads);
    switch (b->n1) {
#define X(n) case n: launch_batch_n<n>(stage, grid, b->threads, smem, b->d_probs, b->d_items, b->n_items, b->d_counters + counter, s); break;
        GDG_BATCH_CASES(X)
#undef X
    }
}

void enqueue_steps(gdg_batch *b, int nsteps, cudaStream_t s) {
    for (int i = 0; i < nsteps; ++i) {
        cudaMemsetAsync(b->d_counters, 0, 4 * sizeof(unsigned int), s);
        for (int st = 1; st <= 4; ++st) launch_stage(b, st, st - 1, s);
    }
}

// time every launch shape on the batch's own stage-1 work and keep the fastest
int autotune(gdg_batch *b, cudaStream_t s) {
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_t = 0, best_b = 0;
    const int cand_threads[] = {96, 128, 192, 256};
    for (int threads : cand_threads) {
        if (threads < ((b->n1 * b->n1 + 31) / 32) * 32) continue;
        const size_t sm = batch_smem(b, threads);
        if (sm > (size_t)lim) continue;
        int st = build_items(b, threads / b->n1);
        if (st) return st;
        const int max_b = std::max(1, std::min(8, (int)(smem_sm / (sm + 1024))));
        for (int bpsm = 1; bpsm <= max_b; ++bpsm) {
            b->threads = threads;
            b->bpsm = bpsm;
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned int), s);
                cudaEventRecord(e0, s);
                launch_stage(b, 1, 0, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (cudaGetLastError() != cudaSuccess) continue;
            if (ms < best) { best = ms; best_t = threads; best_b = bpsm; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best_t) return berr(b, GDG_ECUDA, "no launch shape ran");
    b->threads = best_t;
    b->bpsm = best_b;
    return build_items(b, best_t / b->n1);
}

}  // namespace

extern "C" int gdg_batch_destroy(gdg_batch *b) {
    if (!b) return GDG_EINVAL;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_probs);
    cudaFree(b->d_mps);
    cudaFree(b->d_items);
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
    }
    if (st) { gdg_batch_destroy(b); return st; }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->ctx.assign(count, nullptr);
    b->h_probs.resize(count);
    std::vector<ModalParams> mps(count);
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
        }
    }
    if (cudaMalloc((void **)&b->d_mps, count * sizeof(ModalParams)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_probs, count * sizeof(BatchProb)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_counters, gdg_batch::kCounters * sizeof(unsigned int)) != cudaSuccess) {
        gdg_batch_destroy(b);
        return GDG_ENOMEM;
    }
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
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
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
        if (st) return berr(b, st, "enter");
    }
    if (!b->threads && (st = autotune(b, s))) return st;
    // graph of G steps (4 launches and one counter reset each), replayed
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
    if (threads_per_block) *threads_per_block = b->threads;
    if (blocks_per_sm) *blocks_per_sm = b->bpsm;
    if (tile_elements) *tile_elements = b->threads ? b->threads / b->n1 : 0;
    return GDG_OK;
}

extern "C" int gdg_batch_stats(gdg_batch *b, int i, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys) {
    if (!b || i < 0 || i >= b->count) return GDG_EINVAL;
    return gdg_step_stats(b->ctx[i], u_sys, v_sys);
}
