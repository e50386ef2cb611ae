// Batched launch of many independent 2-D problems (a pattern layered on the
// method; the paper advances one mesh at a time).
//
// Every RK4 stage of all problems of a batch is ONE persistent launch: a grid
// of (SMs x resident blocks) CTAs of one element block each (N1^2 threads
// rounded up to a warp) walks one list of work items ordered longest first --
// the element solves of the variable-coefficient problems (element PCG in
// FP64 or mixed precision, or precomputed inverses; by decreasing degree),
// then tiles of the constant-coefficient problems' elements (modified-basis
// route, half-line body) -- block b taking turns b, b + G, ... of a few
// consecutive items.  The stage bodies are the per-problem kernels' own
// (var_stage_body, stage2h_body), so a batched step computes exactly what
// the problem's own gdg_step computes.  A call's launches are captured once
// in a CUDA graph (per-problem dt lives in device descriptors, so the graph
// does not depend on it).  The register budget of the kernel
// (gdg_batch_kernel.cuh), the resident blocks per SM and the items per turn
// are picked on the first step by timing the candidates on the batch's own
// data.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "gdg_batch_kernel.cuh"

using namespace gdg_batch_dev;

struct gdg_batch {
    std::vector<gdg_ctx *> ctx;
    int count = 0, n1 = 0, sms = 152;
    BatchProb *d_probs = nullptr;
    ModalParams *d_mps = nullptr;
    int2 *d_items = nullptr;          // element solves (longest first), then modal tiles
    int n_items = 0, n_var = 0, n_mod = 0, tile = 0;
    size_t smem = 0;                  // dynamic shared memory of the launch
    int variant = BATCH_HI;           // register budget (tuned)
    int per_sm = 0;                   // resident blocks per SM (tuned)
    int chunk = 1;                    // consecutive items per turn of a block (tuned)
    bool tuned = false;
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

const BatchOps batch_ops_hi = batch_ops_of<BATCH_HI>();

const BatchOps &ops(int variant) {
    return variant == BATCH_LO ? batch_ops_lo : variant == BATCH_MID ? batch_ops_mid : batch_ops_hi;
}

int max_resident(const gdg_batch *b, int variant) { return ops(variant).resident(b->n1, b->smem); }

void launch_stage_all(const gdg_batch *b, int stage, cudaStream_t s) {
    const int grid = b->sms * std::max(1, b->per_sm);
    ops(b->variant).launch(b->n1, stage, grid, b->smem, b->d_probs, b->count, b->d_items, b->n_items, b->chunk, s);
}

void enqueue_steps(gdg_batch *b, int nsteps, cudaStream_t s) {
    for (int i = 0; i < nsteps; ++i)
        for (int st = 1; st <= 4; ++st) launch_stage_all(b, st, s);
}

// best of two runs of stages 1, 2 and 3 of the current shape: they read y_n
// and write the stage buffers and the accumulator, which the real step's
// stage 1 rewrites, and (stage 2) the traces of y_n, which the caller
// rebuilds after tuning; stage 4, the one that writes y_n, is not run
float time_stages(gdg_batch *b, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    float t = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
        float ms = 0.f;
        cudaEventRecord(e0, s);
        for (int st = 1; st <= 3; ++st) launch_stage_all(b, st, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        t = std::min(t, ms);
    }
    return t;
}

// Time the candidates on the batch's own stages 1-3: every register budget
// x resident blocks per SM with one item per turn (each budget scanned from
// its most resident blocks down, left once a candidate is 10 % slower than
// that budget's best so far), then 2, 4 and 8 items per turn on the best.
int autotune(gdg_batch *b, cudaStream_t s) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_r = 0, best_v = BATCH_HI, best_c = 1;
    b->chunk = 1;
    for (int v = 0; v < BATCH_VARIANTS; ++v) {
        const int maxr = max_resident(b, v);
        float vbest = 1e30f;
        for (int r = maxr; r >= 1; --r) {
            b->variant = v;
            b->per_sm = r;
            const float t = time_stages(b, s, e0, e1);
            if (t < best) { best = t; best_r = r; best_v = v; }
            if (t < vbest) vbest = t;
            else if (t > 1.1f * vbest) break;
        }
    }
    if (best_r >= 1) {
        b->variant = best_v;
        b->per_sm = best_r;
        for (int c : {2, 4, 8}) {
            b->chunk = c;
            const float t = time_stages(b, s, e0, e1);
            if (t < best) { best = t; best_c = c; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return berr(b, GDG_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    if (best_r < 1) return berr(b, GDG_ENOMEM, "no launch shape fits the shared memory of the batch's element solves");
    b->variant = best_v;
    b->per_sm = best_r;
    b->chunk = best_c;
    b->tuned = true;
    return GDG_OK;
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
    b->tile = batch_tile(b->n1);   // modal elements per item (half-line body: blockDim / (2 N1))
    b->smem = batch_modal_doubles(b->n1) * sizeof(double) + sizeof(ModalParams);
    std::vector<ModalParams> mps(count);
    std::vector<int2> var_items, mod_items;
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
            for (int t = 0; t * b->tile < c->ne; ++t) mod_items.push_back(make_int2(i, t));
        } else {
            P.kind = 1;
            P.vp = c->var->vp;
            P.sb = gdg_var_buffers(c);
            b->smem = std::max(b->smem, c->var->smem_stage);
            for (int e = 0; e < c->ne; ++e) var_items.push_back(make_int2(i, e));
        }
    }
    // longest items first (higher order: more quadrature points per face, more
    // PCG work), so that the last items of a stage are short ones
    std::stable_sort(var_items.begin(), var_items.end(), [&](const int2 &a, const int2 &c) {
        return pbs[a.x].p > pbs[c.x].p;
    });
    b->n_var = (int)var_items.size();
    b->n_mod = (int)mod_items.size();
    // the modal tiles last: short items even out the blocks' ends of the stage
    // (spreading them evenly among the element solves instead measured 1-2 %
    // slower: every switch restages a problem's parameters)
    std::vector<int2> items(var_items);
    items.insert(items.end(), mod_items.begin(), mod_items.end());
    b->n_items = (int)items.size();
    if (cudaMalloc((void **)&b->d_mps, count * sizeof(ModalParams)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_probs, count * sizeof(BatchProb)) != cudaSuccess ||
        cudaMalloc((void **)&b->d_items, std::max<size_t>(1, items.size()) * sizeof(int2)) != cudaSuccess) {
        gdg_batch_destroy(b);
        return GDG_ENOMEM;
    }
    for (int i = 0; i < count; ++i)
        if (b->h_probs[i].kind == 0) b->h_probs[i].mp = b->d_mps + i;
    if (cudaMemcpy(b->d_mps, mps.data(), count * sizeof(ModalParams), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_probs, b->h_probs.data(), count * sizeof(BatchProb), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!items.empty() &&
         cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)) {
        gdg_batch_destroy(b);
        return berr(nullptr, GDG_ECUDA, "upload");
    }
    cudaError_t ae = cudaSuccess;
    for (int v = 0; v < BATCH_VARIANTS && ae == cudaSuccess; ++v) ae = ops(v).attrs(b->n1);
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
    auto enter = [&]() -> int {
        for (int i = 0; i < b->count; ++i) {
            gdg_ctx *c = b->ctx[i];
            const int e = c->pb.coef == GDG_COEF_CONST ? gdg_const_enter(c, u[i], v[i], s)
                                                       : gdg_var_enter(c, u[i], v[i], s);
            if (e) return berr(b, e, "enter: " + c->err);
        }
        return GDG_OK;
    };
    if ((st = enter())) return st;
    if (!b->tuned) {
        if (b->exec) {   // re-tuning after gdg_batch_set_tuning(.., 0): the graph holds the old shape
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
            b->graph_steps = 0;
        }
        if ((st = autotune(b, s))) return st;
        // the tuner's stage 2 overwrote the traces of y_n that the step's
        // stage 1 reads: enter again
        if ((st = enter())) return st;
    }
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

extern "C" int gdg_batch_tuning(const gdg_batch *b, int *threads_per_block, int *blocks_per_sm, int *tile_elements,
                                int *register_budget, int *registers_per_thread, int *items_per_turn) {
    if (!b) return GDG_EINVAL;
    if (threads_per_block) *threads_per_block = b->tuned ? nthreads_for(b->n1 * b->n1) : 0;
    if (blocks_per_sm) *blocks_per_sm = b->tuned ? b->per_sm : 0;
    if (tile_elements) *tile_elements = b->tuned && b->n_mod > 0 ? b->tile : 0;
    if (register_budget) *register_budget = b->tuned ? b->variant : 0;
    if (registers_per_thread) *registers_per_thread = b->tuned ? ops(b->variant).regs(b->n1) : 0;
    if (items_per_turn) *items_per_turn = b->tuned ? b->chunk : 0;
    return GDG_OK;
}

extern "C" int gdg_batch_set_tuning(gdg_batch *b, int register_budget, int blocks_per_sm, int items_per_turn) {
    if (!b || register_budget < 0 || register_budget >= BATCH_VARIANTS || blocks_per_sm < 0 || items_per_turn < 1)
        return GDG_EINVAL;
    if (blocks_per_sm == 0) {   // back to the tuner at the next step
        b->tuned = false;
        return GDG_OK;
    }
    if (blocks_per_sm > max_resident(b, register_budget))
        return berr(b, GDG_EINVAL, "more blocks per SM than registers and shared memory allow");
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);   // the graph holds the old launch shape
    b->exec = nullptr;
    b->graph_steps = 0;
    b->variant = register_budget;
    b->per_sm = blocks_per_sm;
    b->chunk = items_per_turn;
    b->tuned = true;
    return GDG_OK;
}

extern "C" int gdg_batch_stats(gdg_batch *b, int i, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys) {
    if (!b || i < 0 || i >= b->count) return GDG_EINVAL;
    return gdg_step_stats(b->ctx[i], u_sys, v_sys);
}

// the check slots of the three budgets' translation units (gdg_checks.cuh)
int gdg_checks_read_batch(GdgCheckSlot *out, int reset) {
    GdgCheckSlot acc{};
    for (int v = 0; v < BATCH_VARIANTS; ++v) {
        GdgCheckSlot s{};
        if (ops(v).checks(&s, reset)) return -1;
        if (s.count && !acc.count) acc = s;
        else acc.count += s.count;
    }
    *out = acc;
    return 0;
}
