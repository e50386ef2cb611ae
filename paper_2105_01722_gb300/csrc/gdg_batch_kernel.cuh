// Device side of the batched launch (gdg_batch.cu): one persistent kernel per
// RK4 stage over a list of work items of many independent 2-D problems.
//
// The kernel is compiled under three register budgets, one translation unit
// each so that they compile in parallel; the tuner times them on the batch's
// own data.  The element-solve bodies need about 60 registers; what a budget
// buys is resident blocks where shared memory allows them:
//   BATCH_HI  (gdg_batch.cu)      3 blocks of 96 threads per SM promised:
//                                 up to 168 registers, nothing spills;
//   BATCH_MID (gdg_batch_mid.cu)  480 threads per SM: <= 128 registers (the
//                                 FP64 PCG's 40 KB allow 5 blocks);
//   BATCH_LO  (gdg_batch_lo.cu)   960 threads per SM: <= 64 registers (the
//                                 mixed solves' 27 KB allow 8 blocks, and the
//                                 precomputed-inverse route streams its
//                                 operators and wants every warp it can get);
//                                 the modal body reads y_n and the
//                                 accumulator where it uses them (LEAN).
#pragma once

#include "gdg_checks.cuh"
#include "gdg_internal.h"
#include "gdg_stage_const.cuh"
#include "gdg_var_kernels.cuh"

namespace gdg_batch_dev {

enum { BATCH_HI = 0, BATCH_MID = 1, BATCH_LO = 2, BATCH_VARIANTS = 3 };

struct BatchProb {
    int kind;                 // 0 modal route (constant coefficients), 1 element solves
    const ModalParams *mp;    // kind 0: device copy of the problem's modal parameters
    const double *lam2;       // kind 0
    VarParams vp;             // kind 1
    StepBuffers sb;
    double dt;
};

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

// block-wide copy of a parameter struct into shared memory (whole 4-byte words)
template <typename T>
__device__ __forceinline__ void copy_to_shared(T *dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const unsigned int *s = reinterpret_cast<const unsigned int *>(src);
    unsigned int *d = reinterpret_cast<unsigned int *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// elements of the variable-coefficient problems (one element solve per item).
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

// elements of one modal work item: the half-line body (two threads per
// transverse line, bit-identical to the one-thread-per-line body and about
// 100 registers instead of 160).  The problem's ModalParams (2.8 KB) sit in
// the dynamic shared memory behind the body's tile area, which the element
// solves use for their own arrays: the block's static shared memory stays
// small, and with it the footprint that limits resident blocks.
__host__ __device__ constexpr int batch_tile(int n1) { return nthreads_for(n1 * n1) / (2 * n1); }
__host__ __device__ constexpr size_t batch_modal_doubles(int n1) {
    return (size_t)batch_tile(n1) * (4 * n1 + 2 * n1 * (n1 + 1));
}

template <int N1, int STAGE, bool LEAN>
__device__ __forceinline__ void batch_mod_item(const BatchProb *__restrict__ probs, int2 w, int &cur, double *smem) {
    constexpr int MODE = STAGE == 1 ? M_S1 : (STAGE == 4 ? M_S4 : M_S23);
    const BatchProb &P = probs[w.x];
    ModalParams *s_mp = reinterpret_cast<ModalParams *>(smem + batch_modal_doubles(N1));
    if (w.x != cur) {
        copy_to_shared(s_mp, P.mp);
        cur = w.x;
    }
    const StageRoles<STAGE> r(P.sb, P.dt);
    const StageBufs bb{r.yU, r.yV, P.sb.nU, P.sb.nV, P.sb.aU, P.sb.aV, r.oU, r.oV, r.trin, r.trout, P.lam2};
    stage2h_body<N1, MODE, LEAN>(*s_mp, bb, r.cA, r.cY, w.y, smem);
}

__host__ __device__ constexpr int batch_min_blocks(int n1, int variant) {
    return variant == BATCH_LO ? 960 / nthreads_for(n1 * n1)
           : variant == BATCH_MID ? 480 / nthreads_for(n1 * n1)
                                  : kVarMinBlocks;
}

// One persistent launch per RK stage over every problem of the batch.  The
// list of items is ordered longest first -- the element solves of the
// variable-coefficient problems (PCG or precomputed inverses, by decreasing
// degree), then the modal tiles of the constant-coefficient problems
// (batch_tile(N1) elements each) -- and cut into turns of `chunk`
// consecutive items; block b takes turns b, b + G, b + 2G, ... (G =
// gridDim.x).  No queue: the order and the static assignment make every
// stage of a block deterministic.  A block restages a problem's parameters
// in shared memory only when its next item belongs to another problem, which
// consecutive items rarely do: longer turns mean fewer restagings on the
// small problems and a coarser tail.
template <int N1, int STAGE, int VARIANT>
__global__ void __launch_bounds__(nthreads_for(N1 * N1), batch_min_blocks(N1, VARIANT))
k_batch_all(const BatchProb *__restrict__ probs, int n_probs, const int2 *__restrict__ items, int n_items,
            int chunk) {
    extern __shared__ double smem[];
    __shared__ VarParams s_vp;
    __shared__ VarBufs s_b;
    __shared__ double s_c[2];
    int cur_var = -1, cur_mod = -1;
    for (long long it0 = (long long)blockIdx.x * chunk; it0 < n_items; it0 += (long long)gridDim.x * chunk)
    for (int it = (int)it0; it < n_items && it < it0 + chunk; ++it) {
        int2 w = items[it];
        GDG_CHECK_INDEX(w.x, 0, n_probs, GDG_SITE_BATCH_PROBLEM, 0);
        const BatchProb &P = probs[w.x];
        GDG_CHECK_INDEX(w.y, 0, P.kind == 1 ? P.vp.ne : (P.mp->ne + batch_tile(N1) - 1) / batch_tile(N1),
                        GDG_SITE_BATCH_ELEMENT, 0);
        if (P.kind == 1) {
            batch_var_item<N1, STAGE>(probs, w, cur_var, s_vp, s_b, s_c, smem);
            cur_mod = -1;   // the element solve overwrote the staged ModalParams
        } else {
            batch_mod_item<N1, STAGE, VARIANT == BATCH_LO>(probs, w, cur_mod, smem);
        }
        __syncthreads();
    }
}

#define GDG_BATCH_CASES(X) X(8) X(9) X(10)

// dynamic shared memory may use the opt-in maximum minus the kernel's own
// static shared memory (the parameter slots)
template <typename K>
cudaError_t raise_smem(K kernel, int lim) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim - (int)a.sharedSizeBytes);
}

// Host side of one register budget (instantiated by one translation unit each)
template <int VARIANT>
struct BatchVariant {
    template <int N1>
    static cudaError_t attrs_n() {
        int dev = 0, lim = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaError_t e;
        if ((e = raise_smem(k_batch_all<N1, 1, VARIANT>, lim)) != cudaSuccess) return e;
        if ((e = raise_smem(k_batch_all<N1, 2, VARIANT>, lim)) != cudaSuccess) return e;
        if ((e = raise_smem(k_batch_all<N1, 3, VARIANT>, lim)) != cudaSuccess) return e;
        return raise_smem(k_batch_all<N1, 4, VARIANT>, lim);
    }
    static cudaError_t attrs(int n1) {
        switch (n1) {
#define X(n_) case n_: return attrs_n<n_>();
            GDG_BATCH_CASES(X)
#undef X
        }
        return cudaErrorInvalidValue;
    }
    // resident blocks per SM of the stage-2 kernel (the largest) at smem bytes; 0 on error
    static int resident(int n1, size_t smem) {
        int n = 0;
        switch (n1) {
#define X(n_)                                                                                                 \
    case n_:                                                                                                  \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_all<n_, 2, VARIANT>, nthreads_for(n_ * n_), \
                                                          smem) != cudaSuccess)                               \
            n = 0;                                                                                            \
        break;
            GDG_BATCH_CASES(X)
#undef X
        }
        return n;
    }
    // registers per thread of the stage-2 kernel
    static int regs(int n1) {
        cudaFuncAttributes a{};
        switch (n1) {
#define X(n_) case n_: cudaFuncGetAttributes(&a, k_batch_all<n_, 2, VARIANT>); break;
            GDG_BATCH_CASES(X)
#undef X
        }
        return a.numRegs;
    }
    template <int N1>
    static void launch_n(int stage, int grid, size_t smem, const BatchProb *probs, int n_probs, const int2 *items,
                         int n_items, int chunk, cudaStream_t s) {
        constexpr int T = nthreads_for(N1 * N1);
        switch (stage) {
        case 1: k_batch_all<N1, 1, VARIANT><<<grid, T, smem, s>>>(probs, n_probs, items, n_items, chunk); break;
        case 2: k_batch_all<N1, 2, VARIANT><<<grid, T, smem, s>>>(probs, n_probs, items, n_items, chunk); break;
        case 3: k_batch_all<N1, 3, VARIANT><<<grid, T, smem, s>>>(probs, n_probs, items, n_items, chunk); break;
        default: k_batch_all<N1, 4, VARIANT><<<grid, T, smem, s>>>(probs, n_probs, items, n_items, chunk); break;
        }
    }
    static void launch(int n1, int stage, int grid, size_t smem, const BatchProb *probs, int n_probs,
                       const int2 *items, int n_items, int chunk, cudaStream_t s) {
        switch (n1) {
#define X(n_) case n_: launch_n<n_>(stage, grid, smem, probs, n_probs, items, n_items, chunk, s); break;
            GDG_BATCH_CASES(X)
#undef X
        }
    }
};

// the host entry points of one budget (one translation unit each)
struct BatchOps {
    cudaError_t (*attrs)(int n1);
    int (*resident)(int n1, size_t smem);   // resident blocks per SM at smem bytes, 0 on error
    int (*regs)(int n1);
    void (*launch)(int n1, int stage, int grid, size_t smem, const BatchProb *probs, int n_probs,
                   const int2 *items, int n_items, int chunk, cudaStream_t s);
    int (*checks)(GdgCheckSlot *out, int reset);
};
// this translation unit's check slot (gdg_checks.cuh)
static GDG_CHECKS_READER(batch_checks_read)

template <int VARIANT>
constexpr BatchOps batch_ops_of() {
    return BatchOps{BatchVariant<VARIANT>::attrs, BatchVariant<VARIANT>::resident, BatchVariant<VARIANT>::regs,
                    BatchVariant<VARIANT>::launch, batch_checks_read};
}
extern const BatchOps batch_ops_mid;   // gdg_batch_mid.cu
extern const BatchOps batch_ops_lo;    // gdg_batch_lo.cu

}  // namespace gdg_batch_dev
