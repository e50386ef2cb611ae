// Constant-coefficient Cartesian path of libgdg: the modified-basis
// (simultaneous diagonalisation) route of Section 3.2.
//
// State inside gdg_step is the modal coefficient pair (Ubar, Vbar) with
// U = Psi Ubar, Psi = Psi_y (x) Psi_x, Psi_j^T M_j Psi_j = I,
// Psi_j^T S_j Psi_j = diag(lambda_j).  In these coordinates (Eqs.
// DG1_sparse / DG2_sparse):
//   mass matrix       -> identity
//   stiffness         -> diag(lambda_x[k] + lambda_y[l])
//   face lifts        -> rank one per line: the transverse mass matrix is the
//                        identity in the transverse modal coordinates, so
//                        Psi^T [(n.grad phi) (x) M_perp g] = gvec (x) gbar and
//                        Psi^T [phi_face (x) M_perp q] = evec (x) qbar
//                        (Section 3.2's surface terms in the new basis)
//   constrained u_t   -> dUbar/dt = Vbar + r_u / (lambda_x + lambda_y),
//                        and dUbar_00/dt = Vbar_00 for the constant mode.
// Neighbouring Cartesian elements share the transverse basis, so the fluxes
// of Section 2.2.1 are formed directly on transverse modal traces.
//
// One RK4 stage is one kernel: read the traces of the stage input (own and
// neighbours', written by the previous kernel), form fluxes, lifts and the
// diagonal solves, update the RK accumulator and the next stage input, and
// write the traces of that next input.  The grid-wide dependency between
// traces and lifts is the kernel boundary.
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gdg_checks.cuh"
#include "gdg_internal.h"
#include "gdg_stage_const.cuh"

namespace {

constexpr int MAXB2 = 256;  // largest 2-D block (epb elements x N1 threads); allows 255 registers
constexpr int TPB1 = 128;  // threads per block, 1-D kernels (one element per thread)

// ------------------------------------------------------------ 2-D stage --

template <int N1, int MODE>
__global__ void __launch_bounds__(MAXB2)
k_stage2(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    extern __shared__ double smem[];
    const int t = threadIdx.x;
    const int le = t / N1, l = t - le * N1;
    const int e = blockIdx.x * (int)(blockDim.x / N1) + le;
    const bool valid = e < mp.ne;
    double *fy = smem + le * (4 * N1);
    double *tile = smem + (blockDim.x / N1) * 4 * N1 + le * (2 * N1 * (N1 + 1));
    const int nx = mp.nx, ny = mp.ny;
    const int ex = valid ? e % nx : 0, ey = valid ? e / nx : 0;

    double gxm = 0, gxp = 0, qxm = 0, qxp = 0;
    if (valid) {
        const double *T = b.trin;
        // x faces, transverse mode l
        double vi = T[tix2<N1>(e, 0, 0, l)], di = T[tix2<N1>(e, 0, 1, l)], vo, dO;
        int en = ex - 1;
        if (en < 0 && mp.per_x) en += nx;
        bool bnd = en < 0;
        if (!bnd) { int f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2_NB + 0); vo = T[tix2<N1>(f, 1, 0, l)]; dO = T[tix2<N1>(f, 1, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 0, bnd, gxm, qxm);
        vi = T[tix2<N1>(e, 1, 0, l)]; di = T[tix2<N1>(e, 1, 1, l)];
        en = ex + 1;
        if (en >= nx && mp.per_x) en -= nx;
        bnd = en >= nx;
        if (!bnd) { int f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2_NB + 1); vo = T[tix2<N1>(f, 0, 0, l)]; dO = T[tix2<N1>(f, 0, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 1, bnd, gxp, qxp);
        // y faces, transverse mode k = l
        double g, q;
        vi = T[tix2<N1>(e, 2, 0, l)]; di = T[tix2<N1>(e, 2, 1, l)];
        en = ey - 1;
        if (en < 0 && mp.per_y) en += ny;
        bnd = en < 0;
        if (!bnd) { int f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2_NB + 2); vo = T[tix2<N1>(f, 3, 0, l)]; dO = T[tix2<N1>(f, 3, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 0, bnd, g, q);
        fy[0 * N1 + l] = g; fy[2 * N1 + l] = q;
        vi = T[tix2<N1>(e, 3, 0, l)]; di = T[tix2<N1>(e, 3, 1, l)];
        en = ey + 1;
        if (en >= ny && mp.per_y) en -= ny;
        bnd = en >= ny;
        if (!bnd) { int f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2_NB + 3); vo = T[tix2<N1>(f, 2, 0, l)]; dO = T[tix2<N1>(f, 2, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 1, bnd, g, q);
        fy[1 * N1 + l] = g; fy[3 * N1 + l] = q;
    }
    __syncthreads();

    double Ru[N1], Rv[N1];   // next stage input (or k) for row l
    if (valid) {
        const size_t row = ((size_t)e * N1 + l) * N1;
        const double *L0 = b.lam2 + l * N1;
        const double *L1 = b.lam2 + N1 * N1 + l * N1;
        const double gLy = mp.d[1].gL[l], gRy = mp.d[1].gR[l];
        const double eLy = mp.d[1].eL[l], eRy = mp.d[1].eR[l];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double Yu = b.yU[row + k], Yv = b.yV[row + k];
            const double ru = mp.d[0].gL[k] * gxm + mp.d[0].gR[k] * gxp + gLy * fy[k] + gRy * fy[N1 + k];
            const double rv = L0[k] * Yu + mp.d[0].eL[k] * qxm + mp.d[0].eR[k] * qxp +
                              eLy * fy[2 * N1 + k] + eRy * fy[3 * N1 + k];
            const double ku = Yv + L1[k] * ru;
            const double kv = rv;
            if (MODE == M_RHS) {
                b.oU[row + k] = ku;
                b.oV[row + k] = kv;
            } else if (MODE == M_S1) {
                b.aU[row + k] = cA * ku;
                b.aV[row + k] = cA * kv;
                Ru[k] = Yu + cY * ku;
                Rv[k] = Yv + cY * kv;
            } else if (MODE == M_S23) {
                b.aU[row + k] += cA * ku;
                b.aV[row + k] += cA * kv;
                Ru[k] = b.nU[row + k] + cY * ku;
                Rv[k] = b.nV[row + k] + cY * kv;
            } else {
                Ru[k] = b.nU[row + k] + b.aU[row + k] + cA * ku;
                Rv[k] = b.nV[row + k] + b.aV[row + k] + cA * kv;
            }
        }
        if (MODE != M_RHS) {
            double *dU = (MODE == M_S4) ? b.nU : b.oU;
            double *dV = (MODE == M_S4) ? b.nV : b.oV;
#pragma unroll
            for (int k = 0; k < N1; ++k) { dU[row + k] = Ru[k]; dV[row + k] = Rv[k]; }
        }
    }
    if (MODE == M_RHS) return;   // uniform across the block

    // traces of the next stage input: x faces from the row, y faces from columns
    if (valid) {
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            vL += mp.d[0].eL[k] * Rv[k];
            vR += mp.d[0].eR[k] * Rv[k];
            dL += mp.d[0].gL[k] * Ru[k];
            dR += mp.d[0].gR[k] * Ru[k];
            tile[l * (N1 + 1) + k] = Ru[k];
            tile[N1 * (N1 + 1) + l * (N1 + 1) + k] = Rv[k];
        }
        b.trout[tix2<N1>(e, 0, 0, l)] = vL;
        b.trout[tix2<N1>(e, 0, 1, l)] = dL;
        b.trout[tix2<N1>(e, 1, 0, l)] = vR;
        b.trout[tix2<N1>(e, 1, 1, l)] = dR;
    }
    __syncthreads();
    if (valid) {
        const int k = l;   // this thread's column
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const double u = tile[j * (N1 + 1) + k], v = tile[N1 * (N1 + 1) + j * (N1 + 1) + k];
            vL += mp.d[1].eL[j] * v;
            vR += mp.d[1].eR[j] * v;
            dL += mp.d[1].gL[j] * u;
            dR += mp.d[1].gR[j] * u;
        }
        b.trout[tix2<N1>(e, 2, 0, k)] = vL;
        b.trout[tix2<N1>(e, 2, 1, k)] = dL;
        b.trout[tix2<N1>(e, 3, 0, k)] = vR;
        b.trout[tix2<N1>(e, 3, 1, k)] = dR;
    }
}

template <int N1, int MODE, int ALT>
__global__ void __launch_bounds__(MAXB2)
k_stage2p(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    extern __shared__ double smem[];
    stage2p_body<N1, MODE, ALT>(mp, b, cA, cY, blockIdx.x, smem);
}

// half-line variant (two threads per line), bit-identical results
template <int N1, int MODE>
__global__ void __launch_bounds__(MAXB2)
k_stage2h(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    extern __shared__ double smem[];
    stage2h_body<N1, MODE>(mp, b, cA, cY, blockIdx.x, smem);
}

// Field-split variant of stage2p_body.  The block's first W = 32 ceil(epb N1 / 32)
// threads take the u field of every line of its epb elements (r_u, k_u, the RK
// update of u, the n.grad u traces), the next W threads the v field (r_v, k_v,
// the update of v, the v traces).  The split is warp-uniform, so each warp runs
// one path with compile-time constant operands, and every floating-point
// operation is the one stage2p_body performs, in the same order: bit-identical
// results with twice the warps of the one-line kernel per element.
template <int N1, int ALT, int FIELD>
__device__ __forceinline__ void s2f_fluxes(const ModalParams &mp, const StageBufs &b, int e, int l, double *fy,
                                           double &XA, double &XB) {
    const int nx = mp.nx, ny = mp.ny;
    const int ex = e % nx, ey = e / nx;
    const double b2 = mp.beta2, t2 = mp.tau2;
    const double *T = b.trin;
    double vi, di, vo, dO, g2m, q2m, g2p, q2p;
    int en, f;
    bool bnd;
    vi = T[tix2<N1>(e, 0, 0, l)]; di = T[tix2<N1>(e, 0, 1, l)];
    en = ex - 1;
    if (en < 0 && mp.per_x) en += nx;
    bnd = en < 0;
    if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2F_NB + 0); vo = T[tix2<N1>(f, 1, 0, l)]; dO = T[tix2<N1>(f, 1, 1, l)]; }
    else { vo = -vi; dO = -di; }
    flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
    vi = T[tix2<N1>(e, 1, 0, l)]; di = T[tix2<N1>(e, 1, 1, l)];
    en = ex + 1;
    if (en >= nx && mp.per_x) en -= nx;
    bnd = en >= nx;
    if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2F_NB + 1); vo = T[tix2<N1>(f, 0, 0, l)]; dO = T[tix2<N1>(f, 0, 1, l)]; }
    else { vo = -vi; dO = -di; }
    flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
    if (FIELD == 0) { XA = g2m + g2p; XB = g2m - g2p; }
    else { XA = q2m + q2p; XB = q2m - q2p; }
    vi = T[tix2<N1>(e, 2, 0, l)]; di = T[tix2<N1>(e, 2, 1, l)];
    en = ey - 1;
    if (en < 0 && mp.per_y) en += ny;
    bnd = en < 0;
    if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2F_NB + 2); vo = T[tix2<N1>(f, 3, 0, l)]; dO = T[tix2<N1>(f, 3, 1, l)]; }
    else { vo = -vi; dO = -di; }
    flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
    vi = T[tix2<N1>(e, 3, 0, l)]; di = T[tix2<N1>(e, 3, 1, l)];
    en = ey + 1;
    if (en >= ny && mp.per_y) en -= ny;
    bnd = en >= ny;
    if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2F_NB + 3); vo = T[tix2<N1>(f, 2, 0, l)]; dO = T[tix2<N1>(f, 2, 1, l)]; }
    else { vo = -vi; dO = -di; }
    flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
    if (FIELD == 0) { fy[l] = g2m + g2p; fy[N1 + l] = g2m - g2p; }
    else { fy[2 * N1 + l] = q2m + q2p; fy[3 * N1 + l] = q2m - q2p; }
}

// lift, diagonal solve and RK update of one field of line l, then the line's
// row traces of that field and its row of the transpose tile
template <int N1, int MODE, int FIELD>
__device__ __forceinline__ void s2f_update(const ModalParams &mp, const StageBufs &b, double cA, double cY,
                                           int e, int l, size_t row, const double *fy, double *tile, double XA,
                                           double XB, double (&R)[N1], const double (&Y)[N1],
                                           const double (&Nn)[N1], const double (&Aa)[N1]) {
    constexpr int NE = (N1 + 1) / 2;
    double *oF = FIELD == 0 ? b.oU : b.oV;
    double *aF = FIELD == 0 ? b.aU : b.aV;
    double *nF = FIELD == 0 ? b.nU : b.nV;
    const double *L = b.lam2 + l * N1;
    const double *P1 = b.lam2 + 2 * N1 * N1 + l * N1, *P2 = b.lam2 + 3 * N1 * N1 + l * N1;
    const double hy = mp.d[1].ceL[l];
    const double *F = fy + (FIELD == 0 ? 0 : 2 * N1) + (l < NE ? 0 : N1);
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        const double x = k < NE ? XA : XB;
        double kf;
        if (FIELD == 0) {
            kf = fma(P1[k], x, fma(P2[k], F[k], Y[k]));
        } else {
            kf = fma(L[k], Y[k], fma(mp.d[0].ceL[k], x, hy * F[k]));
        }
        if (MODE == M_RHS) {
            oF[row + k] = kf;
        } else if (MODE == M_S1) {
            aF[row + k] = kf;
            R[k] = fma(cY, kf, R[k]);
        } else if (MODE == M_S23) {
            aF[row + k] = fma(2.0, kf, Aa[k]);
            R[k] = fma(cY, kf, Nn[k]);
        } else {
            R[k] = fma(cA, Aa[k] + kf, Nn[k]);
        }
    }
    if (MODE == M_RHS) return;
    double *dF = MODE == M_S4 ? nF : oF;
#pragma unroll
    for (int k = 0; k < N1; ++k) dF[row + k] = R[k];
    double se = 0, so = 0;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        const double c = FIELD == 0 ? mp.d[0].gL[k] : mp.d[0].eL[k];
        if (k < NE) se = fma(c, R[k], se);
        else so = fma(c, R[k], so);
        tile[(FIELD == 0 ? 0 : N1 * (N1 + 1)) + l * (N1 + 1) + k] = R[k];
    }
    b.trout[tix2<N1>(e, 0, 1 - FIELD, l)] = se + so;
    b.trout[tix2<N1>(e, 1, 1 - FIELD, l)] = se - so;
}

// column traces (y faces) of one field from the transpose tile
template <int N1, int FIELD>
__device__ __forceinline__ void s2f_columns(const ModalParams &mp, const StageBufs &b, int e, int k,
                                            const double *tile) {
    constexpr int NE = (N1 + 1) / 2;
    const double *col = tile + (FIELD == 0 ? 0 : N1 * (N1 + 1)) + k;
    double se = 0, so = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const double c = FIELD == 0 ? mp.d[1].gL[j] : mp.d[1].eL[j];
        if (j < NE) se = fma(c, col[j * (N1 + 1)], se);
        else so = fma(c, col[j * (N1 + 1)], so);
    }
    b.trout[tix2<N1>(e, 2, 1 - FIELD, k)] = se + so;
    b.trout[tix2<N1>(e, 3, 1 - FIELD, k)] = se - so;
}

template <int N1, int MODE, int ALT>
__global__ void __launch_bounds__(2 * MAXB2)
k_stage2f(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    extern __shared__ double smem[];
    const int epb = mp.epb;
    const int W = ((epb * N1 + 31) / 32) * 32;
    const int t = threadIdx.x;
    const bool fu = t < W;   // warp-uniform: W is a multiple of 32
    const int lt = fu ? t : t - W;
    const int le = lt / N1, l = lt - le * N1;
    const int e = blockIdx.x * epb + le;
    const bool valid = le < epb && e < mp.ne;
    double *fy = smem + le * (4 * N1);
    double *tile = smem + epb * 4 * N1 + le * (2 * N1 * (N1 + 1));
    const size_t row = ((size_t)(valid ? e : 0) * N1 + l) * N1;
    // own field's stage input R (and y_n, accumulator), the other field's Y
    double R[N1], Y[N1], Nn[N1], Aa[N1];
    if (valid) {
        const double *own = fu ? b.yU : b.yV, *oth = fu ? b.yV : b.yU;
        const double *nF = fu ? b.nU : b.nV, *aF = fu ? b.aU : b.aV;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            R[k] = own[row + k];
            Y[k] = oth[row + k];
            if (MODE == M_S23 || MODE == M_S4) {
                Nn[k] = nF[row + k];
                Aa[k] = aF[row + k];
            }
        }
    }
    double XA = 0, XB = 0;
    if (valid) {
        if (fu) s2f_fluxes<N1, ALT, 0>(mp, b, e, l, fy, XA, XB);
        else s2f_fluxes<N1, ALT, 1>(mp, b, e, l, fy, XA, XB);
    }
    __syncthreads();
    if (valid) {
        if (fu) s2f_update<N1, MODE, 0>(mp, b, cA, cY, e, l, row, fy, tile, XA, XB, R, Y, Nn, Aa);
        else s2f_update<N1, MODE, 1>(mp, b, cA, cY, e, l, row, fy, tile, XA, XB, R, Y, Nn, Aa);
    }
    if (MODE == M_RHS) return;
    __syncthreads();
    if (valid) {
        if (fu) s2f_columns<N1, 0>(mp, b, e, l, tile);
        else s2f_columns<N1, 1>(mp, b, e, l, tile);
    }
}

// ------------------------------------------------ persistent 2-D step --
// All RK4 stages of nsteps steps in one cooperative launch (every CTA
// resident).  Each thread keeps its line's stage input, y_n and RK
// accumulator in registers from stage to stage; only the face traces go
// through global memory, and a grid barrier separates the stages.  Every
// floating-point operation is the one stage2p_body performs, in the same
// order, on the same values: bit-identical results to the per-stage kernels.

__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Neighbour synchronisation of the persistent step.  Blocks exchange data
// only through the face traces of their elements' face neighbours, so a
// block waits for those blocks alone, not for the whole grid.  sync[0] is
// the give-up flag; block b's flag is sync[NB_BASE + b NB_STRIDE] (its own
// 32-byte sector), all zero at launch.  After stage `round` every block
// publishes `round` (fence, then store: a release), then waits (acquire
// loads by warp 0) until every block in s_nb[0..nnb) has published it: the
// traces it is about to read are written, and the buffer its next stage
// overwrites has been read by them.  Every wait is bounded by limit_ns of
// wall time, after which the give-up flag is set; returns false when this
// block or another one gave up (the caller then leaves the kernel).
constexpr int NB_BASE = 32, NB_STRIDE = 8;
__host__ __device__ constexpr size_t sync_words(int blocks) { return NB_BASE + (size_t)NB_STRIDE * blocks; }

__device__ bool neighbour_sync(unsigned *sync, const int *s_nb, int nnb, unsigned round,
                               unsigned long long limit_ns, int *s_ok) {
    __syncthreads();   // this block's trace writes of stage `round` are done
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) {
            __threadfence();
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(sync + NB_BASE + (size_t)blockIdx.x * NB_STRIDE),
                         "r"(round) : "memory");
        }
        const unsigned long long t0 = gtimer_ns();
        int ok = 1;
        for (unsigned it = 1;; ++it) {
            bool done = true;
            for (int i = lane; i < nnb; i += 32)
                if (ld_acquire_u32(sync + NB_BASE + (size_t)s_nb[i] * NB_STRIDE) < round) done = false;
            if (__all_sync(0xffffffffu, done)) break;
            int stop = 0;
            if (lane == 0) {
                if (gtimer_ns() - t0 > limit_ns) { atomicExch(sync, 1u); stop = 1; }
                else if ((it & 63u) == 0u && *(volatile unsigned *)sync) stop = 1;
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) { ok = 0; break; }
        }
        if (lane == 0) *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// blocks holding the face neighbours of block b's elements, each once, in
// s_nb[0 .. *s_cnt) (scratch: 4 epb entries, one per element and face)
__device__ void neighbour_blocks(const ModalParams &mp, int epb, int *s_nb, int *s_cnt) {
    for (int i = threadIdx.x; i < 4 * epb; i += blockDim.x) {
        const int e = blockIdx.x * epb + (i >> 2), dir = i & 3;
        int nbb = -1;
        if (e < mp.ne) {
            const int nx = mp.nx, ny = mp.ny, ex = e % nx, ey = e / nx;
            int en = -1;
            if (dir == 0) {
                int x = ex - 1;
                if (x < 0 && mp.per_x) x += nx;
                if (x >= 0) en = ey * nx + x;
            } else if (dir == 1) {
                int x = ex + 1;
                if (x >= nx && mp.per_x) x -= nx;
                if (x < nx) en = ey * nx + x;
            } else if (dir == 2) {
                int y = ey - 1;
                if (y < 0 && mp.per_y) y += ny;
                if (y >= 0) en = y * nx + ex;
            } else {
                int y = ey + 1;
                if (y >= ny && mp.per_y) y -= ny;
                if (y < ny) en = y * nx + ex;
            }
            if (en >= 0 && en / epb != (int)blockIdx.x) nbb = en / epb;
            if (nbb >= 0) GDG_CHECK_INDEX(nbb, 0, gridDim.x, GDG_SITE_STEP2R_BLOCK, -1);
        }
        s_nb[i] = nbb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // keep each block once, in place
        int cnt = 0;
        for (int i = 0; i < 4 * epb; ++i) {
            const int nb = s_nb[i];
            bool seen = nb < 0;
            for (int j = 0; j < cnt && !seen; ++j) seen = s_nb[j] == nb;
            if (!seen) s_nb[cnt++] = nb;
        }
        *s_cnt = cnt;
    }
}

// one RK stage of stage2p_body on register state: R (stage input, becomes
// the next stage's input), Nn (y_n), Aa (accumulator), per field
template <int N1, int MODE, int ALT>
__device__ __forceinline__ void stage2r(const ModalParams &mp, const double *lam2, const double *trin,
                                        double *trout, double cA, double cY, int e, int l, bool valid,
                                        double *fy, double *tile, double (&Ru)[N1], double (&Rv)[N1],
                                        double (&Nu)[N1], double (&Nv)[N1], double (&Au)[N1], double (&Av)[N1]) {
    constexpr int NE = (N1 + 1) / 2;
    const int nx = mp.nx, ny = mp.ny;
    const int ex = valid ? e % nx : 0, ey = valid ? e / nx : 0;
    const double b2 = mp.beta2, t2 = mp.tau2;
    double GA = 0, GB = 0, QA = 0, QB = 0;
    if (valid) {
        const double *T = trin;   // written by other CTAs in the previous stage: read from L2
        double vi, di, vo, dO, g2m, q2m, g2p, q2p;
        int en, f;
        bool bnd;
        vi = __ldcg(T + tix2<N1>(e, 0, 0, l)); di = __ldcg(T + tix2<N1>(e, 0, 1, l));
        en = ex - 1;
        if (en < 0 && mp.per_x) en += nx;
        bnd = en < 0;
        if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2R_NB + 0); vo = __ldcg(T + tix2<N1>(f, 1, 0, l)); dO = __ldcg(T + tix2<N1>(f, 1, 1, l)); }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
        vi = __ldcg(T + tix2<N1>(e, 1, 0, l)); di = __ldcg(T + tix2<N1>(e, 1, 1, l));
        en = ex + 1;
        if (en >= nx && mp.per_x) en -= nx;
        bnd = en >= nx;
        if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2R_NB + 1); vo = __ldcg(T + tix2<N1>(f, 0, 0, l)); dO = __ldcg(T + tix2<N1>(f, 0, 1, l)); }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
        GA = g2m + g2p; GB = g2m - g2p; QA = q2m + q2p; QB = q2m - q2p;
        vi = __ldcg(T + tix2<N1>(e, 2, 0, l)); di = __ldcg(T + tix2<N1>(e, 2, 1, l));
        en = ey - 1;
        if (en < 0 && mp.per_y) en += ny;
        bnd = en < 0;
        if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2R_NB + 2); vo = __ldcg(T + tix2<N1>(f, 3, 0, l)); dO = __ldcg(T + tix2<N1>(f, 3, 1, l)); }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
        vi = __ldcg(T + tix2<N1>(e, 3, 0, l)); di = __ldcg(T + tix2<N1>(e, 3, 1, l));
        en = ey + 1;
        if (en >= ny && mp.per_y) en -= ny;
        bnd = en >= ny;
        if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2R_NB + 3); vo = __ldcg(T + tix2<N1>(f, 2, 0, l)); dO = __ldcg(T + tix2<N1>(f, 2, 1, l)); }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
        fy[l] = g2m + g2p; fy[N1 + l] = g2m - g2p;
        fy[2 * N1 + l] = q2m + q2p; fy[3 * N1 + l] = q2m - q2p;
    }
    __syncthreads();
    if (valid) {
        const double *L0 = lam2 + l * N1;
        const double *P1 = lam2 + 2 * N1 * N1 + l * N1, *P2 = lam2 + 3 * N1 * N1 + l * N1;
        const double cey = mp.d[1].ceL[l];
        const double *FG = fy + (l < NE ? 0 : N1);
        const double *FQ = fy + (l < NE ? 2 * N1 : 3 * N1);
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double Yu = Ru[k], Yv = Rv[k];
            const double xg = k < NE ? GA : GB, xq = k < NE ? QA : QB;
            const double ku = fma(P1[k], xg, fma(P2[k], FG[k], Yv));
            const double rv = fma(L0[k], Yu, fma(mp.d[0].ceL[k], xq, cey * FQ[k]));
            const double kv = rv;
            if (MODE == M_S1) {
                Au[k] = ku;
                Av[k] = kv;
                Ru[k] = fma(cY, ku, Yu);
                Rv[k] = fma(cY, kv, Yv);
            } else if (MODE == M_S23) {
                Au[k] = fma(2.0, ku, Au[k]);
                Av[k] = fma(2.0, kv, Av[k]);
                Ru[k] = fma(cY, ku, Nu[k]);
                Rv[k] = fma(cY, kv, Nv[k]);
            } else {
                Ru[k] = fma(cA, Au[k] + ku, Nu[k]);
                Rv[k] = fma(cA, Av[k] + kv, Nv[k]);
                Nu[k] = Ru[k];
                Nv[k] = Rv[k];
            }
        }
        double ve = 0, vo_ = 0, de = 0, do_ = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            if (k < NE) { ve = fma(mp.d[0].eL[k], Rv[k], ve); de = fma(mp.d[0].gL[k], Ru[k], de); }
            else { vo_ = fma(mp.d[0].eL[k], Rv[k], vo_); do_ = fma(mp.d[0].gL[k], Ru[k], do_); }
            tile[l * (N1 + 1) + k] = Ru[k];
            tile[N1 * (N1 + 1) + l * (N1 + 1) + k] = Rv[k];
        }
        trout[tix2<N1>(e, 0, 0, l)] = ve + vo_;
        trout[tix2<N1>(e, 0, 1, l)] = de + do_;
        trout[tix2<N1>(e, 1, 0, l)] = ve - vo_;
        trout[tix2<N1>(e, 1, 1, l)] = de - do_;
    }
    __syncthreads();
    if (valid) {
        const int k = l;
        double ve = 0, vo_ = 0, de = 0, do_ = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const double u = tile[j * (N1 + 1) + k], v = tile[N1 * (N1 + 1) + j * (N1 + 1) + k];
            if (j < NE) { ve = fma(mp.d[1].eL[j], v, ve); de = fma(mp.d[1].gL[j], u, de); }
            else { vo_ = fma(mp.d[1].eL[j], v, vo_); do_ = fma(mp.d[1].gL[j], u, do_); }
        }
        trout[tix2<N1>(e, 2, 0, k)] = ve + vo_;
        trout[tix2<N1>(e, 2, 1, k)] = de + do_;
        trout[tix2<N1>(e, 3, 0, k)] = ve - vo_;
        trout[tix2<N1>(e, 3, 1, k)] = de - do_;
    }
}

// nsteps RK4 steps of the modal state (nU, nV) in place; tr0 holds the
// traces of y_n on entry and of the result on exit (as enqueue_rk4_step).
// blockDim.x = epb * N1 (epb <= MAXB2 / N1); sync: sync_words(gridDim.x)
// words (see neighbour_sync).
// Registers are allocated per SM sub-partition (16,384 each): at <= 168 per
// thread three warps fit in one, at 169..176 only two, so the cap keeps
// 12 instead of 8 warps of the grid resident per SM.
template <int N1, int ALT>
__global__ void __maxnreg__(168)
k_step2r(const __grid_constant__ ModalParams mp, const double *lam2, double *nU, double *nV, double *tr0,
         double *tr1, double dt, int nsteps, unsigned *sync, unsigned long long limit_ns) {
    extern __shared__ double smem[];
    __shared__ int s_ok;
    __shared__ int s_nb[4 * (MAXB2 / N1)];
    const int epb = blockDim.x / N1;
    const int t = threadIdx.x;
    const int le = t / N1, l = t - le * N1;
    const int e = blockIdx.x * epb + le;
    const bool valid = le < epb && e < mp.ne;
    double *fy = smem + le * (4 * N1);
    double *tile = smem + epb * 4 * N1 + le * (2 * N1 * (N1 + 1));
    const size_t row = ((size_t)(valid ? e : 0) * N1 + l) * N1;
    __shared__ int s_cnt;
    neighbour_blocks(mp, epb, s_nb, &s_cnt);
    __syncthreads();
    const int nnb = s_cnt;
    double Ru[N1], Rv[N1], Nu[N1], Nv[N1], Au[N1], Av[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        Nu[k] = valid ? nU[row + k] : 0.0;
        Nv[k] = valid ? nV[row + k] : 0.0;
        Ru[k] = Nu[k];
        Rv[k] = Nv[k];
        Au[k] = 0.0;
        Av[k] = 0.0;
    }
    unsigned round = 0;
    for (int step = 0; step < nsteps; ++step) {
        stage2r<N1, M_S1, ALT>(mp, lam2, tr0, tr1, dt / 6.0, 0.5 * dt, e, l, valid, fy, tile, Ru, Rv, Nu, Nv, Au, Av);
        if (!neighbour_sync(sync, s_nb, nnb, ++round, limit_ns, &s_ok)) return;
        stage2r<N1, M_S23, ALT>(mp, lam2, tr1, tr0, dt / 3.0, 0.5 * dt, e, l, valid, fy, tile, Ru, Rv, Nu, Nv, Au, Av);
        if (!neighbour_sync(sync, s_nb, nnb, ++round, limit_ns, &s_ok)) return;
        stage2r<N1, M_S23, ALT>(mp, lam2, tr0, tr1, dt / 3.0, dt, e, l, valid, fy, tile, Ru, Rv, Nu, Nv, Au, Av);
        if (!neighbour_sync(sync, s_nb, nnb, ++round, limit_ns, &s_ok)) return;
        stage2r<N1, M_S4, ALT>(mp, lam2, tr1, tr0, dt / 6.0, 0.0, e, l, valid, fy, tile, Ru, Rv, Nu, Nv, Au, Av);
        if (step + 1 < nsteps && !neighbour_sync(sync, s_nb, nnb, ++round, limit_ns, &s_ok)) return;
    }
    if (valid) {
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            nU[row + k] = Nu[k];
            nV[row + k] = Nv[k];
        }
    }
}

// traces of a modal state (start of gdg_step and gdg_rhs)
template <int N1>
__global__ void __launch_bounds__(MAXB2)
k_traces2(const __grid_constant__ ModalParams mp, const double *yU, const double *yV, double *trout) {
    extern __shared__ double smem[];
    const int t = threadIdx.x;
    const int le = t / N1, l = t - le * N1;
    const int e = blockIdx.x * (int)(blockDim.x / N1) + le;
    const bool valid = e < mp.ne;
    double *tile = smem + le * (2 * N1 * (N1 + 1));
    if (valid) {
        const size_t row = ((size_t)e * N1 + l) * N1;
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double u = yU[row + k], v = yV[row + k];
            vL += mp.d[0].eL[k] * v;
            vR += mp.d[0].eR[k] * v;
            dL += mp.d[0].gL[k] * u;
            dR += mp.d[0].gR[k] * u;
            tile[l * (N1 + 1) + k] = u;
            tile[N1 * (N1 + 1) + l * (N1 + 1) + k] = v;
        }
        trout[tix2<N1>(e, 0, 0, l)] = vL;
        trout[tix2<N1>(e, 0, 1, l)] = dL;
        trout[tix2<N1>(e, 1, 0, l)] = vR;
        trout[tix2<N1>(e, 1, 1, l)] = dR;
    }
    __syncthreads();
    if (valid) {
        const int k = l;
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const double u = tile[j * (N1 + 1) + k], v = tile[N1 * (N1 + 1) + j * (N1 + 1) + k];
            vL += mp.d[1].eL[j] * v;
            vR += mp.d[1].eR[j] * v;
            dL += mp.d[1].gL[j] * u;
            dR += mp.d[1].gR[j] * u;
        }
        trout[tix2<N1>(e, 2, 0, k)] = vL;
        trout[tix2<N1>(e, 2, 1, k)] = dL;
        trout[tix2<N1>(e, 3, 0, k)] = vR;
        trout[tix2<N1>(e, 3, 1, k)] = dR;
    }
}

// Separable element transform: out = (Cy (x) Cx) diag(D) (By (x) Bx) in,
// with C and D optional (nullptr).  Matrices are n1 x n1 row-major,
// (A (x) B)[(l,k),(j,i)] = A[l][j] B[k][i].  Two fields per call (U and V
// share the matrices).
template <int N1>
__global__ void __launch_bounds__(MAXB2)
k_sep2(int ne, const double *in0, const double *in1, double *out0, double *out1,
       const double *Bx, const double *By, const double *D, const double *Cx, const double *Cy) {
    extern __shared__ double smem[];
    double *sB = smem;                 // Bx, By, Cx, Cy
    double *tiles = smem + 4 * N1 * N1;
    const int t = threadIdx.x;
    for (int i = t; i < N1 * N1; i += blockDim.x) {
        sB[i] = Bx[i];
        sB[N1 * N1 + i] = By[i];
        if (Cx) { sB[2 * N1 * N1 + i] = Cx[i]; sB[3 * N1 * N1 + i] = Cy[i]; }
    }
    const int le = t / N1, l = t - le * N1;
    const int e = blockIdx.x * (int)(blockDim.x / N1) + le;
    const bool valid = e < ne;
    double *tile = tiles + le * (2 * N1 * (N1 + 1));
    const int nf = in1 ? 2 : 1;
    __syncthreads();
    for (int f = 0; f < nf; ++f) {
        const double *in = f ? in1 : in0;
        double *out = f ? out1 : out0;
        double *T = tile + f * N1 * (N1 + 1);
        // (1) rows: T[j][k] = sum_i Bx[k][i] in[j][i]   (thread = row j)
        if (valid) {
            double x[N1];
            const size_t row = ((size_t)e * N1 + l) * N1;
#pragma unroll
            for (int i = 0; i < N1; ++i) x[i] = in[row + i];
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                double s = 0;
#pragma unroll
                for (int i = 0; i < N1; ++i) s += sB[k * N1 + i] * x[i];
                T[l * (N1 + 1) + k] = s;
            }
        }
        __syncthreads();
        // (2) columns: Z[m][k] = D[m][k] * sum_j By[m][j] T[j][k]   (thread = column k)
        double z[N1];
        if (valid) {
            const int k = l;
            double c[N1];
#pragma unroll
            for (int j = 0; j < N1; ++j) c[j] = T[j * (N1 + 1) + k];
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                double s = 0;
#pragma unroll
                for (int j = 0; j < N1; ++j) s += sB[N1 * N1 + m * N1 + j] * c[j];
                if (D) s *= D[m * N1 + k];
                z[m] = s;
            }
        }
        if (!Cx) {
            if (valid) {
                const int k = l;
#pragma unroll
                for (int m = 0; m < N1; ++m) out[((size_t)e * N1 + m) * N1 + k] = z[m];
            }
            __syncthreads();
            continue;
        }
        // (3) columns again with Cy: W[r][k] = sum_m Cy[r][m] Z[m][k]; store to T
        __syncthreads();
        if (valid) {
            const int k = l;
#pragma unroll
            for (int r = 0; r < N1; ++r) {
                double s = 0;
#pragma unroll
                for (int m = 0; m < N1; ++m) s += sB[3 * N1 * N1 + r * N1 + m] * z[m];
                T[r * (N1 + 1) + k] = s;
            }
        }
        __syncthreads();
        // (4) rows with Cx: out[r][q] = sum_k Cx[q][k] W[r][k]   (thread = row r)
        if (valid) {
            double w[N1];
#pragma unroll
            for (int k = 0; k < N1; ++k) w[k] = T[l * (N1 + 1) + k];
            const size_t row = ((size_t)e * N1 + l) * N1;
#pragma unroll
            for (int q = 0; q < N1; ++q) {
                double s = 0;
#pragma unroll
                for (int k = 0; k < N1; ++k) s += sB[2 * N1 * N1 + q * N1 + k] * w[k];
                out[row + q] = s;
            }
        }
        __syncthreads();
    }
}

// per-block partial of sum over elements of (|Vbar|^2 + c2 * lambda . Ubar^2)
// for modal (Ubar, Vbar) given in yU, yV; deterministic fixed-order tree.
template <int N1, int DIM>
__global__ void k_energy_partial(int ne, const double *yU, const double *yV, const double *lam2,
                                 double *partial) {
    __shared__ double red[1024];
    const int t = threadIdx.x;
    const int ents = DIM == 2 ? N1 * N1 : N1;
    double s = 0.0;
    const long long total = (long long)ne * ents;
    for (long long i = (long long)blockIdx.x * blockDim.x + t; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i % ents);
        const double u = yU[i], v = yV[i];
        s += v * v - lam2[m] * u * u;    // lam2[0][m] = -c2 * lambda_m
    }
    red[t] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(int n, const double *partial, double *out) {
    __shared__ double red[1024];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int i = t; i < n; i += blockDim.x) s += partial[i];
    red[t] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) out[0] = 0.5 * red[0];
}

// ------------------------------------------------------------ 1-D --------

template <int N1, int MODE>
__global__ void __launch_bounds__(TPB1)
k_stage1(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mp.ne) return;
    const int nx = mp.nx;
    const double *T = b.trin;
    double vi = T[tix1(e, 0, 0)], di = T[tix1(e, 0, 1)], vo, dO, gm, qm, gp, qp;
    int en = e - 1;
    if (en < 0 && mp.per_x) en += nx;
    if (en >= 0) {
        GDG_CHECK_INDEX(en, 0, mp.ne, GDG_SITE_STAGE1_NB + 0, 0);
        vo = T[tix1(en, 1, 0)]; dO = T[tix1(en, 1, 1)];
    } else { vo = -vi; dO = -di; }
    flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 0, en < 0, gm, qm);
    vi = T[tix1(e, 1, 0)]; di = T[tix1(e, 1, 1)];
    en = e + 1;
    if (en >= nx && mp.per_x) en -= nx;
    if (en < nx) {
        GDG_CHECK_INDEX(en, 0, mp.ne, GDG_SITE_STAGE1_NB + 1, 0);
        vo = T[tix1(en, 0, 0)]; dO = T[tix1(en, 0, 1)];
    } else { vo = -vi; dO = -di; }
    flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, 1, en >= nx, gp, qp);
    const size_t row = (size_t)e * N1;
    double Ru[N1], Rv[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        const double Yu = b.yU[row + k], Yv = b.yV[row + k];
        const double ru = mp.d[0].gL[k] * gm + mp.d[0].gR[k] * gp;
        const double rv = b.lam2[k] * Yu + mp.d[0].eL[k] * qm + mp.d[0].eR[k] * qp;
        const double ku = Yv + b.lam2[N1 + k] * ru, kv = rv;
        if (MODE == M_RHS) { b.oU[row + k] = ku; b.oV[row + k] = kv; }
        else if (MODE == M_S1) {
            b.aU[row + k] = cA * ku; b.aV[row + k] = cA * kv;
            Ru[k] = Yu + cY * ku; Rv[k] = Yv + cY * kv;
        } else if (MODE == M_S23) {
            b.aU[row + k] += cA * ku; b.aV[row + k] += cA * kv;
            Ru[k] = b.nU[row + k] + cY * ku; Rv[k] = b.nV[row + k] + cY * kv;
        } else {
            Ru[k] = b.nU[row + k] + b.aU[row + k] + cA * ku;
            Rv[k] = b.nV[row + k] + b.aV[row + k] + cA * kv;
        }
    }
    if (MODE == M_RHS) return;
    double *dU = (MODE == M_S4) ? b.nU : b.oU;
    double *dV = (MODE == M_S4) ? b.nV : b.oV;
    double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        dU[row + k] = Ru[k]; dV[row + k] = Rv[k];
        vL += mp.d[0].eL[k] * Rv[k]; vR += mp.d[0].eR[k] * Rv[k];
        dL += mp.d[0].gL[k] * Ru[k]; dR += mp.d[0].gR[k] * Ru[k];
    }
    b.trout[tix1(e, 0, 0)] = vL; b.trout[tix1(e, 0, 1)] = dL;
    b.trout[tix1(e, 1, 0)] = vR; b.trout[tix1(e, 1, 1)] = dR;
}

template <int N1>
__global__ void k_traces1(const __grid_constant__ ModalParams mp, const double *yU, const double *yV, double *trout) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= mp.ne) return;
    double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
        const double u = yU[(size_t)e * N1 + k], v = yV[(size_t)e * N1 + k];
        vL += mp.d[0].eL[k] * v; vR += mp.d[0].eR[k] * v;
        dL += mp.d[0].gL[k] * u; dR += mp.d[0].gR[k] * u;
    }
    trout[tix1(e, 0, 0)] = vL; trout[tix1(e, 0, 1)] = dL;
    trout[tix1(e, 1, 0)] = vR; trout[tix1(e, 1, 1)] = dR;
}

// out = C diag(D) B in  (1-D, two fields)
template <int N1>
__global__ void k_sep1(int ne, const double *in0, const double *in1, double *out0, double *out1,
                       const double *B, const double *D, const double *C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int nf = in1 ? 2 : 1;
    for (int f = 0; f < nf; ++f) {
        const double *in = f ? in1 : in0;
        double *out = f ? out1 : out0;
        double x[N1], z[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) x[i] = in[(size_t)e * N1 + i];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            double s = 0;
#pragma unroll
            for (int i = 0; i < N1; ++i) s += B[k * N1 + i] * x[i];
            z[k] = D ? s * D[k] : s;
        }
        if (!C) {
#pragma unroll
            for (int k = 0; k < N1; ++k) out[(size_t)e * N1 + k] = z[k];
            continue;
        }
#pragma unroll
        for (int q = 0; q < N1; ++q) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < N1; ++k) s += C[q * N1 + k] * z[k];
            out[(size_t)e * N1 + q] = s;
        }
    }
}

// ------------------------------------------------------ dispatch ---------

#define GDG_N1_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)
// element sizes of the persistent step (its register state is 6 N1 doubles per thread)
#define GDG_N1_CASES_P(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

size_t smem_stage2(int n1, int epb) { return (size_t)epb * (4 * n1 + 2 * n1 * (n1 + 1)) * sizeof(double); }
size_t smem_traces2(int n1, int epb) { return (size_t)epb * (2 * n1 * (n1 + 1)) * sizeof(double); }
size_t smem_sep2(int n1, int epb) { return (size_t)(4 * n1 * n1 + epb * 2 * n1 * (n1 + 1)) * sizeof(double); }

template <int N1>
void launch_stage2(int mode, const ModalParams &mp, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    dim3 grid((mp.ne + mp.epb - 1) / mp.epb), block(mp.epb * N1);
    size_t sm = smem_stage2(N1, mp.epb);
    if (mp.parity && mp.split == 1) {
        const dim3 gh((mp.ne + mp.epbh - 1) / mp.epbh), bh(mp.epbh * 2 * N1);
        const size_t smh = smem_stage2(N1, mp.epbh);
        switch (mode) {
        case M_RHS: k_stage2h<N1, M_RHS><<<gh, bh, smh, s>>>(mp, b, cA, cY); break;
        case M_S1: k_stage2h<N1, M_S1><<<gh, bh, smh, s>>>(mp, b, cA, cY); break;
        case M_S23: k_stage2h<N1, M_S23><<<gh, bh, smh, s>>>(mp, b, cA, cY); break;
        default: k_stage2h<N1, M_S4><<<gh, bh, smh, s>>>(mp, b, cA, cY); break;
        }
        return;
    }
    if (mp.parity && mp.split == 2) {
        const dim3 bf(2 * (((mp.epb * N1 + 31) / 32) * 32));
        switch (mode) {
#define GDG_K2F(m) (mp.alt ? k_stage2f<N1, m, 1> : k_stage2f<N1, m, 0>)
        case M_RHS: GDG_K2F(M_RHS)<<<grid, bf, sm, s>>>(mp, b, cA, cY); break;
        case M_S1: GDG_K2F(M_S1)<<<grid, bf, sm, s>>>(mp, b, cA, cY); break;
        case M_S23: GDG_K2F(M_S23)<<<grid, bf, sm, s>>>(mp, b, cA, cY); break;
        default: GDG_K2F(M_S4)<<<grid, bf, sm, s>>>(mp, b, cA, cY); break;
#undef GDG_K2F
        }
        return;
    }
    if (mp.parity) {
        switch (mode) {
#define GDG_K2P(m) (mp.alt ? k_stage2p<N1, m, 1> : k_stage2p<N1, m, 0>)
        case M_RHS: GDG_K2P(M_RHS)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        case M_S1: GDG_K2P(M_S1)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        case M_S23: GDG_K2P(M_S23)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        default: GDG_K2P(M_S4)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
#undef GDG_K2P
        }
        return;
    }
    switch (mode) {
    case M_RHS: k_stage2<N1, M_RHS><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    case M_S1: k_stage2<N1, M_S1><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    case M_S23: k_stage2<N1, M_S23><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    default: k_stage2<N1, M_S4><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    }
}

template <int N1>
void launch_stage1(int mode, const ModalParams &mp, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    dim3 grid((mp.ne + TPB1 - 1) / TPB1), block(TPB1);
    switch (mode) {
    case M_RHS: k_stage1<N1, M_RHS><<<grid, block, 0, s>>>(mp, b, cA, cY); break;
    case M_S1: k_stage1<N1, M_S1><<<grid, block, 0, s>>>(mp, b, cA, cY); break;
    case M_S23: k_stage1<N1, M_S23><<<grid, block, 0, s>>>(mp, b, cA, cY); break;
    default: k_stage1<N1, M_S4><<<grid, block, 0, s>>>(mp, b, cA, cY); break;
    }
}

void launch_stage_raw(const gdg_ctx *ctx, int mode, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    const int n1 = ctx->n1;
    if (ctx->dim == 3) {
        gdg3_stage(ctx->mp, n1, mode, b, cA, cY, s);
        return;
    }
    if (ctx->dim == 2) {
        switch (n1) {
#define X(n) case n: launch_stage2<n>(mode, ctx->mp, b, cA, cY, s); break;
            GDG_N1_CASES(X)
#undef X
        }
    } else {
        switch (n1) {
#define X(n) case n: launch_stage1<n>(mode, ctx->mp, b, cA, cY, s); break;
            GDG_N1_CASES(X)
#undef X
        }
    }
}

void launch_traces_raw(const gdg_ctx *ctx, const double *yU, const double *yV, double *tr, cudaStream_t s) {
    const int n1 = ctx->n1;
    if (ctx->dim == 3) {
        gdg3_traces(ctx->mp, n1, yU, yV, tr, s);
        return;
    }
    if (ctx->dim == 2) {
        const int epb = ctx->mp.epb;
        dim3 grid((ctx->ne + epb - 1) / epb), block(epb * n1);
        switch (n1) {
#define X(n) case n: k_traces2<n><<<grid, block, smem_traces2(n, epb), s>>>(ctx->mp, yU, yV, tr); break;
            GDG_N1_CASES(X)
#undef X
        }
    } else {
        dim3 grid((ctx->ne + TPB1 - 1) / TPB1), block(TPB1);
        switch (n1) {
#define X(n) case n: k_traces1<n><<<grid, block, 0, s>>>(ctx->mp, yU, yV, tr); break;
            GDG_N1_CASES(X)
#undef X
        }
    }
}

// table offsets inside ctx->d_mats: [dir][P, Psi, PsiT][n1*n1]
const double *mat(const gdg_ctx *ctx, int dir, int which) {
    return ctx->d_mats + ((size_t)dir * 3 + which) * ctx->n1 * ctx->n1;
}
enum { T_P = 0, T_PSI = 1, T_PSIT = 2 };

// out = (C) diag(D) (B) in, over both fields when in1 != nullptr
void launch_sep_raw(const gdg_ctx *ctx, const double *in0, const double *in1, double *out0, double *out1,
                int B, const double *D, int C, cudaStream_t s) {
    const int n1 = ctx->n1;
    if (ctx->dim == 3) {
        gdg3_sep(n1, ctx->ne, in0, in1, out0, out1, mat(ctx, 0, B), mat(ctx, 1, B), mat(ctx, 2, B), D,
                 C >= 0 ? mat(ctx, 0, C) : nullptr, C >= 0 ? mat(ctx, 1, C) : nullptr,
                 C >= 0 ? mat(ctx, 2, C) : nullptr, s);
        return;
    }
    if (ctx->dim == 2) {
        const int epb = ctx->mp.epb;
        dim3 grid((ctx->ne + epb - 1) / epb), block(epb * n1);
        const double *Bx = mat(ctx, 0, B), *By = mat(ctx, 1, B);
        const double *Cx = C >= 0 ? mat(ctx, 0, C) : nullptr, *Cy = C >= 0 ? mat(ctx, 1, C) : nullptr;
        switch (n1) {
#define X(n) case n: k_sep2<n><<<grid, block, smem_sep2(n, epb), s>>>(ctx->ne, in0, in1, out0, out1, Bx, By, D, Cx, Cy); break;
            GDG_N1_CASES(X)
#undef X
        }
    } else {
        dim3 grid((ctx->ne + TPB1 - 1) / TPB1), block(TPB1);
        const double *Bm = mat(ctx, 0, B), *Cm = C >= 0 ? mat(ctx, 0, C) : nullptr;
        switch (n1) {
#define X(n) case n: k_sep1<n><<<grid, block, 0, s>>>(ctx->ne, in0, in1, out0, out1, Bm, D, Cm); break;
            GDG_N1_CASES(X)
#undef X
        }
    }
}

void launch_stage(gdg_ctx *ctx, int mode, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    GDG_PROF(ctx, GDG_K_STAGE, s, launch_stage_raw(ctx, mode, b, cA, cY, s));
}
void launch_traces(gdg_ctx *ctx, const double *yU, const double *yV, double *tr, cudaStream_t s) {
    GDG_PROF(ctx, GDG_K_TRACES, s, launch_traces_raw(ctx, yU, yV, tr, s));
}
void launch_sep(gdg_ctx *ctx, const double *in0, const double *in1, double *out0, double *out1,
                int B, const double *D, int C, cudaStream_t s) {
    GDG_PROF(ctx, GDG_K_TRANSFORM, s, launch_sep_raw(ctx, in0, in1, out0, out1, B, D, C, s));
}

double *buf(gdg_ctx *ctx, int i) { return ctx->d_state + (size_t)i * ctx->ndof; }
enum { B_NU = 0, B_NV, B_AU, B_AV, B_XU, B_XV, B_YU, B_YV, B_KU, B_KV, B_COUNT };

// The persistent step needs every CTA of its grid resident at once.  Its
// elements per block: the per-stage kernels' choice if that grid fits,
// else the fitting one with the best (used lanes) x (element balance over
// the SMs); 0 if none fits.
template <int N1>
int persist_epb_n(const gdg_ctx *ctx) {
    const ModalParams &mp = ctx->mp;
    int coop = 0, sms = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (!coop || sms <= 0) return 0;
    auto fits = [&](int epb) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mp.alt ? k_step2r<N1, 1> : k_step2r<N1, 0>, epb * N1,
                                                          smem_stage2(N1, epb)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return (long long)nb * sms >= (mp.ne + epb - 1) / epb;
    };
    if (fits(mp.epb)) return mp.epb;
    int best = 0;
    double best_eff = -1.0;
    for (int epb = 1; epb * N1 <= MAXB2; ++epb) {
        if (!fits(epb)) continue;
        const int threads = epb * N1, warps = (threads + 31) / 32;
        const int blocks = (mp.ne + epb - 1) / epb, per_sm = (blocks + sms - 1) / sms;
        const double eff = (double)threads / (32.0 * warps) * (((double)mp.ne / sms) / ((double)per_sm * epb));
        if (eff > best_eff + 1e-9) { best_eff = eff; best = epb; }
    }
    return best;
}

int persist_epb(const gdg_ctx *ctx) {
    if (ctx->dim != 2 || !ctx->mp.parity || !ctx->d_sync) return 0;
    switch (ctx->n1) {
#define X(n) case n: return persist_epb_n<n>(ctx);
        GDG_N1_CASES_P(X)
#undef X
    }
    return 0;
}
bool persist_fits(gdg_ctx *ctx) {
    ctx->mp.epbp = persist_epb(ctx);
    return ctx->mp.epbp > 0;
}

template <int N1>
void launch_persist_n(gdg_ctx *ctx, double dt, int nsteps, cudaStream_t s) {
    const ModalParams &mp = ctx->mp;
    const dim3 grid((mp.ne + mp.epbp - 1) / mp.epbp), block(mp.epbp * N1);
    const double *lam2 = ctx->d_lam2;
    double *nU = buf(ctx, B_NU), *nV = buf(ctx, B_NV), *tr0 = ctx->d_tr, *tr1 = ctx->d_tr + ctx->tr_len;
    unsigned *sync = ctx->d_sync;
    unsigned long long lim = ctx->wait_limit_ns;
    void *args[] = {(void *)&mp, (void *)&lam2, (void *)&nU, (void *)&nV, (void *)&tr0, (void *)&tr1,
                    (void *)&dt, (void *)&nsteps, (void *)&sync, (void *)&lim};
    cudaLaunchCooperativeKernel(mp.alt ? (const void *)k_step2r<N1, 1> : (const void *)k_step2r<N1, 0>, grid, block,
                                args, smem_stage2(N1, mp.epbp), s);
}

// nsteps RK4 steps of the modal state in one persistent launch (tr0 holds
// the traces of y_n before and after); the give-up flag is read by
// persist_failed once the stream has run
void launch_persist(gdg_ctx *ctx, double dt, int nsteps, cudaStream_t s) {
    // at most 2^16 steps per launch keeps the barrier counters far from overflow
    for (int done = 0; done < nsteps;) {
        const int k = std::min(nsteps - done, 1 << 16);
        cudaMemsetAsync(ctx->d_sync, 0, sync_words((ctx->mp.ne + ctx->mp.epbp - 1) / ctx->mp.epbp) * sizeof(unsigned), s);
        switch (ctx->n1) {
#define X(n) case n: GDG_PROF(ctx, GDG_K_STAGE, s, launch_persist_n<n>(ctx, dt, k, s)); break;
            GDG_N1_CASES_P(X)
#undef X
        }
        done += k;
    }
}

// copy the give-up flag to the host and wait for the stream: true if a grid
// barrier of the last persistent launch gave up (not while s is capturing)
bool persist_failed(gdg_ctx *ctx, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) return false;
    unsigned *flag = reinterpret_cast<unsigned *>(ctx->h_red + 7);
    *flag = 0;
    cudaMemcpyAsync(flag, ctx->d_sync, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return *flag != 0;
}

int set_smem_limits() {
    // the 2-D kernels may need more than the 48 KB default of dynamic shared
    // memory; the attribute is per device, so it is set once on each device
    constexpr int kDevs = 64;
    static bool done[kDevs] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GDG_ECUDA;
    if (dev >= 0 && dev < kDevs && done[dev]) return GDG_OK;
    const int lim = 200 * 1024;
#define X(n)                                                                               \
    cudaFuncSetAttribute(k_stage2<n, M_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2<n, M_S1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);   \
    cudaFuncSetAttribute(k_stage2<n, M_S23>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2<n, M_S4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);   \
    cudaFuncSetAttribute(k_stage2p<n, M_RHS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2p<n, M_S1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2p<n, M_S23, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2p<n, M_S4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2p<n, M_RHS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2p<n, M_S1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2p<n, M_S23, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2p<n, M_S4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2h<n, M_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2h<n, M_S1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2h<n, M_S23>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2h<n, M_S4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2f<n, M_RHS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2f<n, M_S1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2f<n, M_S23, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2f<n, M_S4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2f<n, M_RHS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2f<n, M_S1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage2f<n, M_S23, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage2f<n, M_S4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_traces2<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);        \
    cudaFuncSetAttribute(k_sep2<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    GDG_N1_CASES(X)
#undef X
#define X(n)                                                                                   \
    cudaFuncSetAttribute(k_step2r<n, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);    \
    cudaFuncSetAttribute(k_step2r<n, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    GDG_N1_CASES_P(X)
#undef X
    gdg3_set_smem_limits();
    if (dev >= 0 && dev < kDevs) done[dev] = true;
    return GDG_OK;
}

// Elements per block of the 2-D kernels: maximise (used warp lanes) x
// (balance of elements over the SMs), with up to `resident` blocks per SM.
int choose_epb(int ne, int n1, int sms, int tpe) {
    int best = 1;
    double best_eff = -1.0;
    for (int epb = 1; epb * tpe <= MAXB2; ++epb) {
        const int threads = epb * tpe;
        const int warps = (threads + 31) / 32;
        const double lanes = (double)threads / (32.0 * warps);
        const size_t sm = smem_stage2(n1, epb);
        int resident = 48 / warps;                          // 48 warps per SM
        const int by_smem = (int)((200.0 * 1024) / (double)sm);
        if (by_smem < resident) resident = by_smem;
        const int by_regs = 65536 / (warps * 32 * 168);     // the stage kernels use up to ~168 registers
        if (by_regs < resident) resident = by_regs;
        if (resident < 1) continue;
        const int blocks = (ne + epb - 1) / epb;
        // elements on the busiest SM vs the average
        const int per_sm_blocks = (blocks + sms - 1) / sms;
        const double busiest = (double)per_sm_blocks * epb;
        const double balance = ((double)ne / sms) / busiest;
        // too few warps per SM to keep the FP64 pipe fed
        const double fill = std::min(1.0, (double)std::min(per_sm_blocks, resident) * warps / 8.0);
        const double eff = lanes * balance * fill;
        if (eff > best_eff + 1e-9) { best_eff = eff; best = epb; }
    }
    return best;
}

// one RK4 step on the internal modal state (y_n in B_N*, traces of y_n in tr0)
void enqueue_rk4_step(gdg_ctx *ctx, double dt, cudaStream_t s) {
    double *tr0 = ctx->d_tr, *tr1 = ctx->d_tr + ctx->tr_len;
    const double *lam2 = ctx->d_lam2;
    StageBufs b{};
    b.nU = buf(ctx, B_NU); b.nV = buf(ctx, B_NV);
    b.aU = buf(ctx, B_AU); b.aV = buf(ctx, B_AV);
    b.lam2 = lam2;
    // stage 1: Y1 = y_n -> acc = dt/6 k1, X = y_n + dt/2 k1
    b.yU = b.nU; b.yV = b.nV; b.oU = buf(ctx, B_XU); b.oV = buf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    launch_stage(ctx, M_S1, b, dt / 6.0, 0.5 * dt, s);
    // stage 2: k2 = f(X) -> acc += dt/3 k2, Y = y_n + dt/2 k2
    b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV); b.oU = buf(ctx, B_YU); b.oV = buf(ctx, B_YV); b.trin = tr1; b.trout = tr0;
    launch_stage(ctx, M_S23, b, dt / 3.0, 0.5 * dt, s);
    // stage 3: k3 = f(Y) -> acc += dt/3 k3, X = y_n + dt k3
    b.yU = buf(ctx, B_YU); b.yV = buf(ctx, B_YV); b.oU = buf(ctx, B_XU); b.oV = buf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    launch_stage(ctx, M_S23, b, dt / 3.0, dt, s);
    // stage 4: k4 = f(X) -> y_n += acc + dt/6 k4 (traces of y_{n+1} to tr0)
    b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV); b.oU = nullptr; b.oV = nullptr; b.trin = tr1; b.trout = tr0;
    launch_stage(ctx, M_S4, b, dt / 6.0, 0.0, s);
}

// ---------------------------------------------- nodal-state route ------
// GDG_ROUTE_NODAL: the state stays nodal between stages.  Every stage
// transforms its input to the modified basis (two n1 x n1 contractions per
// direction and field, launch_sep), evaluates k there with the same stage
// kernel as gdg_rhs, transforms k back, and combines on nodal vectors.  It
// computes the modal route's U', V' to rounding and does four separable
// transforms more per stage; it exists to measure the two routes against
// each other.

// RK4 combination on nodal vectors (the modal route's coefficients: the
// accumulator holds k1 + 2 k2 + 2 k3, stage 4 forms y_n + cA (acc + k4))
__global__ void k_rk_nodal(size_t n, int mode, double *nU, double *nV, const double *kU, const double *kV,
                           double *aU, double *aV, double *yU, double *yV, double cA, double cY) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double ku = kU[i], kv = kV[i];
        if (mode == M_S1) {
            aU[i] = ku; aV[i] = kv;
            yU[i] = fma(cY, ku, nU[i]); yV[i] = fma(cY, kv, nV[i]);
        } else if (mode == M_S23) {
            aU[i] = fma(2.0, ku, aU[i]); aV[i] = fma(2.0, kv, aV[i]);
            yU[i] = fma(cY, ku, nU[i]); yV[i] = fma(cY, kv, nV[i]);
        } else {
            nU[i] = fma(cA, aU[i] + ku, nU[i]); nV[i] = fma(cA, aV[i] + kv, nV[i]);
        }
    }
}

// one RK4 step of the nodal state (u, v): stage inputs in B_Y*, nodal k in
// B_N* (free on this route), the modal stage input and k in B_X* / B_K*
void enqueue_rk4_step_nodal(gdg_ctx *ctx, double *u, double *v, double dt, cudaStream_t s) {
    const size_t n = (size_t)ctx->ndof;
    const int threads = 256, blocks = (int)std::min<size_t>((n + threads - 1) / threads, 4096);
    double *yU = buf(ctx, B_YU), *yV = buf(ctx, B_YV), *kU = buf(ctx, B_NU), *kV = buf(ctx, B_NV);
    const double cY[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
    const int mode[4] = {M_S1, M_S23, M_S23, M_S4};
    for (int st = 0; st < 4; ++st) {
        const double *inU = st == 0 ? u : yU, *inV = st == 0 ? v : yV;
        launch_sep(ctx, inU, inV, buf(ctx, B_XU), buf(ctx, B_XV), T_P, nullptr, -1, s);
        launch_traces(ctx, buf(ctx, B_XU), buf(ctx, B_XV), ctx->d_tr, s);
        StageBufs b{};
        b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV);
        b.oU = buf(ctx, B_KU); b.oV = buf(ctx, B_KV);
        b.trin = ctx->d_tr; b.lam2 = ctx->d_lam2;
        launch_stage(ctx, M_RHS, b, 0.0, 0.0, s);
        launch_sep(ctx, buf(ctx, B_KU), buf(ctx, B_KV), kU, kV, T_PSI, nullptr, -1, s);
        k_rk_nodal<<<blocks, threads, 0, s>>>(n, mode[st], u, v, kU, kV, buf(ctx, B_AU), buf(ctx, B_AV), yU, yV,
                                              dt / 6.0, cY[st]);
    }
}

int step_nodal(gdg_ctx *ctx, double *u, double *v, double dt, int nsteps, cudaStream_t s) {
    int st;
    const int G = (nsteps >= 8 && !ctx->prof.on) ? 8 : 0;
    if (G) {   // a graph of G steps on (u, v), replayed
        GraphCache &gc = ctx->graph;
        if (!gc.exec || gc.dt != dt || gc.steps != G || gc.u != u || gc.v != v) {
            if (gc.exec) cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            cudaGraph_t g;
            if ((st = gdg_cuda_check(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "capture")))
                return st;
            for (int i = 0; i < G; ++i) enqueue_rk4_step_nodal(ctx, u, v, dt, ctx->cap_stream);
            if ((st = gdg_cuda_check(ctx, cudaStreamEndCapture(ctx->cap_stream, &g), "capture end"))) return st;
            st = gdg_cuda_check(ctx, cudaGraphInstantiate(&gc.exec, g, 0), "instantiate");
            cudaGraphDestroy(g);
            if (st) return st;
            gc.dt = dt;
            gc.steps = G;
            gc.u = u;
            gc.v = v;
        }
        for (int i = 0; i + G <= nsteps; i += G)
            if ((st = gdg_cuda_check(ctx, cudaGraphLaunch(gc.exec, s), "graph launch"))) return st;
    }
    const int rem = G ? nsteps % G : nsteps;
    for (int i = 0; i < rem; ++i) enqueue_rk4_step_nodal(ctx, u, v, dt, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step (nodal-state route)");
}

// ---------------------------------------------- partitioned meshes ------
// One mesh split by rows of elements over several contexts.  The stage
// kernels read a halo side's neighbour traces from a ghost row of the trace
// buffer (element rows -1 and ny); between stages the boundary rows' y-face
// traces go out through the caller's exchange function.  Buffer layout of a
// side: [ex][field 0 = v, 1 = n.grad u][transverse mode].

template <int N1>
__global__ void k_halo_pack(int nx, int ny, const double *T, double *send_lo, double *send_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * 2 * N1) return;
    const int ex = i / (2 * N1), fld = (i / N1) % 2, m = i % N1;
    if (send_lo) send_lo[i] = T[tix2<N1>(ex, 2, fld, m)];                      // first row, lower face
    if (send_hi) send_hi[i] = T[tix2<N1>((ny - 1) * nx + ex, 3, fld, m)];      // last row, upper face
}

template <int N1>
__global__ void k_halo_unpack(int nx, int ny, double *T, const double *recv_lo, const double *recv_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * 2 * N1) return;
    const int ex = i / (2 * N1), fld = (i / N1) % 2, m = i % N1;
    // the row below's upper-face traces into ghost row -1, the row above's
    // lower-face traces into ghost row ny (where the stage kernel looks)
    if (recv_lo) T[tix2<N1>(-nx + ex, 3, fld, m)] = recv_lo[i];
    if (recv_hi) T[tix2<N1>(ny * nx + ex, 2, fld, m)] = recv_hi[i];
}

bool has_halo(const gdg_ctx *ctx) { return ctx->mp.halo_lo || ctx->mp.halo_hi; }

// traces in T -> send buffers, the caller's exchange, receive buffers -> ghost rows
int halo_exchange(gdg_ctx *ctx, double *T, cudaStream_t s) {
    const int n = ctx->nx * 2 * ctx->n1, threads = 256, blocks = (n + threads - 1) / threads;
    switch (ctx->n1) {
#define X(n_) case n_: k_halo_pack<n_><<<blocks, threads, 0, s>>>(ctx->nx, ctx->ny, T, ctx->halo_send[0], ctx->halo_send[1]); break;
        GDG_N1_CASES(X)
#undef X
    }
    int st = gdg_cuda_check(ctx, cudaGetLastError(), "halo pack");
    if (st) return st;
    const int rc = ctx->halo_fn(ctx->halo_user, (void *)s);
    if (rc != 0) return gdg_set_err(ctx, GDG_EHALO, "halo exchange function returned " + std::to_string(rc));
    switch (ctx->n1) {
#define X(n_) case n_: k_halo_unpack<n_><<<blocks, threads, 0, s>>>(ctx->nx, ctx->ny, T, ctx->halo_recv[0], ctx->halo_recv[1]); break;
        GDG_N1_CASES(X)
#undef X
    }
    return gdg_cuda_check(ctx, cudaGetLastError(), "halo unpack");
}

// one RK4 step of a partitioned mesh: the stages of enqueue_rk4_step, each
// followed by the exchange of the traces it wrote (except, when `last`, the
// traces of y_{n+1}: the next gdg_step call recomputes them)
int rk4_step_halo(gdg_ctx *ctx, double dt, bool last, cudaStream_t s) {
    double *tr0 = ctx->d_tr, *tr1 = ctx->d_tr + ctx->tr_len;
    StageBufs b{};
    b.nU = buf(ctx, B_NU); b.nV = buf(ctx, B_NV);
    b.aU = buf(ctx, B_AU); b.aV = buf(ctx, B_AV);
    b.lam2 = ctx->d_lam2;
    int st;
    b.yU = b.nU; b.yV = b.nV; b.oU = buf(ctx, B_XU); b.oV = buf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    launch_stage(ctx, M_S1, b, dt / 6.0, 0.5 * dt, s);
    if ((st = halo_exchange(ctx, tr1, s))) return st;
    b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV); b.oU = buf(ctx, B_YU); b.oV = buf(ctx, B_YV); b.trin = tr1; b.trout = tr0;
    launch_stage(ctx, M_S23, b, dt / 3.0, 0.5 * dt, s);
    if ((st = halo_exchange(ctx, tr0, s))) return st;
    b.yU = buf(ctx, B_YU); b.yV = buf(ctx, B_YV); b.oU = buf(ctx, B_XU); b.oV = buf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    launch_stage(ctx, M_S23, b, dt / 3.0, dt, s);
    if ((st = halo_exchange(ctx, tr1, s))) return st;
    b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV); b.oU = nullptr; b.oV = nullptr; b.trin = tr1; b.trout = tr0;
    launch_stage(ctx, M_S4, b, dt / 6.0, 0.0, s);
    return last ? GDG_OK : halo_exchange(ctx, tr0, s);
}

}  // namespace

// ------------------------------------------------------------- API -------

extern "C" long long gdg_halo_len(const gdg_ctx *ctx) {
    if (!ctx || ctx->var || !has_halo(ctx)) return -1;
    return (long long)ctx->nx * 2 * ctx->n1;
}

extern "C" int gdg_set_halo(gdg_ctx *ctx, double *send_lo, double *send_hi, double *recv_lo, double *recv_hi,
                            gdg_halo_fn fn, void *user) {
    if (!ctx || ctx->var || !has_halo(ctx) || !fn) return GDG_EINVAL;
    if (ctx->mp.halo_lo && (!send_lo || !recv_lo))
        return gdg_set_err(ctx, GDG_EINVAL, "gdg_set_halo: the lower side needs send_lo and recv_lo");
    if (ctx->mp.halo_hi && (!send_hi || !recv_hi))
        return gdg_set_err(ctx, GDG_EINVAL, "gdg_set_halo: the upper side needs send_hi and recv_hi");
    ctx->halo_send[0] = ctx->mp.halo_lo ? send_lo : nullptr;
    ctx->halo_recv[0] = ctx->mp.halo_lo ? recv_lo : nullptr;
    ctx->halo_send[1] = ctx->mp.halo_hi ? send_hi : nullptr;
    ctx->halo_recv[1] = ctx->mp.halo_hi ? recv_hi : nullptr;
    ctx->halo_fn = fn;
    ctx->halo_user = user;
    return GDG_OK;
}

int gdg_const_setup(gdg_ctx *ctx) {
    const int n1 = ctx->n1, nn = n1 * n1;
    ModalParams &mp = ctx->mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.nx = ctx->nx;
    mp.ny = ctx->ny;
    mp.nz = ctx->nz;
    mp.ne = ctx->ne;
    mp.per_x = ctx->pb.bc[0] == GDG_BC_PERIODIC;
    mp.per_y = ctx->dim >= 2 && ctx->pb.bc[1] == GDG_BC_PERIODIC;
    // a band of rows of a larger mesh has a halo side where a neighbour band lies
    const bool band = ctx->dim == 2 && (ctx->pb.rows[0] || ctx->pb.rows[1]);
    mp.halo_lo = band && ctx->pb.rows[0] > 0;
    mp.halo_hi = band && ctx->pb.rows[1] < ctx->pb.n_elem[1];
    mp.per_z = ctx->dim == 3 && ctx->pb.bc[2] == GDG_BC_PERIODIC;
    mp.c2 = ctx->pb.c2;
    if (ctx->pb.flux == GDG_FLUX_UPWIND) {
        double xi = ctx->pb.xi > 0 ? ctx->pb.xi : std::sqrt(ctx->pb.c2);
        mp.beta = 0.5 * xi;
        mp.tau = 0.5 / xi;
    }
    mp.beta2 = 2.0 * mp.beta;
    mp.tau2 = 2.0 * mp.tau;
    mp.alt = ctx->pb.flux == GDG_FLUX_ALTERNATING;
    // Mode order: even modes (Psi[N-i][k] = Psi[i][k]) first, then odd ones,
    // each group by ascending eigenvalue; the constant mode stays first.
    // If some eigenvector has no clean parity the generic kernel is used.
    std::vector<int> perm(n1);
    {
        double big = 0.0;
        for (int i = 0; i < nn; ++i) big = std::max(big, std::fabs(ctx->Psih[i]));
        std::vector<int> even, odd;
        bool clean = true;
        for (int k = 0; k < n1; ++k) {
            double dot = 0.0;
            for (int i = 0; i < n1; ++i) dot += ctx->Psih[i * n1 + k] * ctx->Psih[(n1 - 1 - i) * n1 + k];
            const double sgn = dot >= 0.0 ? 1.0 : -1.0;
            for (int i = 0; i < n1; ++i)
                if (std::fabs(ctx->Psih[(n1 - 1 - i) * n1 + k] - sgn * ctx->Psih[i * n1 + k]) > 1e-9 * big) clean = false;
            (sgn > 0 ? even : odd).push_back(k);
        }
        mp.parity = clean && (int)even.size() == (n1 + 1) / 2 && even[0] == 0 && ctx->dim >= 2;
        if (mp.parity) {
            for (int k = 0; k < (int)even.size(); ++k) perm[k] = even[k];
            for (int k = 0; k < (int)odd.size(); ++k) perm[even.size() + k] = odd[k];
        } else {
            for (int k = 0; k < n1; ++k) perm[k] = k;
        }
    }
    std::vector<double> tables((size_t)3 * 3 * nn, 0.0);
    std::vector<double> lam[3];
    for (int d = 0; d < ctx->dim; ++d) {
        const double H = (ctx->pb.hi[d] - ctx->pb.lo[d]) / ctx->pb.n_elem[d];
        const double sq = std::sqrt(H);
        std::vector<double> Psi(nn), M(nn);
        for (int i = 0; i < n1; ++i)
            for (int k = 0; k < n1; ++k) Psi[i * n1 + k] = ctx->Psih[i * n1 + perm[k]] / sq;
        for (int i = 0; i < nn; ++i) M[i] = H * ctx->Mh[i];
        lam[d].resize(n1);
        for (int k = 0; k < n1; ++k) lam[d][k] = ctx->lamh[perm[k]] / (H * H);
        double *P = &tables[((size_t)d * 3 + T_P) * nn];
        double *Ps = &tables[((size_t)d * 3 + T_PSI) * nn];
        double *PT = &tables[((size_t)d * 3 + T_PSIT) * nn];
        for (int k = 0; k < n1; ++k)
            for (int i = 0; i < n1; ++i) {
                double s = 0;
                for (int a = 0; a < n1; ++a) s += Psi[a * n1 + k] * M[a * n1 + i];
                P[k * n1 + i] = s;             // Psi^T M
                Ps[i * n1 + k] = Psi[i * n1 + k];
                PT[k * n1 + i] = Psi[i * n1 + k];
            }
        ModalDir &md = mp.d[d];
        for (int k = 0; k < n1; ++k) {
            md.eL[k] = Psi[0 * n1 + k];
            md.eR[k] = Psi[(n1 - 1) * n1 + k];
            double gl = 0, gr = 0;
            for (int i = 0; i < n1; ++i) {
                gl += Psi[i * n1 + k] * (-ctx->dphiL[i] / H);
                gr += Psi[i * n1 + k] * (ctx->dphiR[i] / H);
            }
            md.gL[k] = gl;
            md.gR[k] = gr;
            md.lam[k] = lam[d][k];
            md.hgL[k] = 0.5 * gl;
            md.ceL[k] = 0.5 * ctx->pb.c2 * md.eL[k];
        }
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    mp.epb = ctx->dim == 2 ? choose_epb(ctx->ne, n1, sms, n1) : 1;
    mp.epbh = ctx->dim == 2 ? choose_epb(ctx->ne, n1, sms, 2 * n1) : 1;
    mp.split = 0;   // decided by timing at the first gdg_step (one-line kernel on partitioned meshes)
    const int ents = ctx->dim == 3 ? nn * n1 : (ctx->dim == 2 ? nn : n1);
    // rows: -c^2 lambda, 1/lambda (0 on the constant mode); 2-D and 3-D also
    // the u lifts folded with the diagonal solve, one row per direction:
    // P1 = hgL_x/lambda, P2 = hgL_y/lambda (, P3 = hgL_z/lambda), which the
    // parity stage kernels apply
    std::vector<double> l2((size_t)(ctx->dim == 2 ? 4 : (ctx->dim == 3 ? 5 : 2)) * ents, 0.0);
    for (int m = 0; m < ents; ++m) {
        double L = ctx->dim == 3   ? lam[0][m % n1] + lam[1][(m / n1) % n1] + lam[2][m / nn]
                   : ctx->dim == 2 ? lam[0][m % n1] + lam[1][m / n1]
                                   : lam[0][m];
        l2[m] = -ctx->pb.c2 * L;
        l2[ents + m] = m == 0 ? 0.0 : 1.0 / L;
        if (ctx->dim == 2) {
            l2[2 * ents + m] = l2[ents + m] * mp.d[0].hgL[m % n1];
            l2[3 * ents + m] = l2[ents + m] * mp.d[1].hgL[m / n1];
        } else if (ctx->dim == 3) {   // m = (mz n1 + my) n1 + mx
            l2[2 * ents + m] = l2[ents + m] * mp.d[0].hgL[m % n1];
            l2[3 * ents + m] = l2[ents + m] * mp.d[1].hgL[(m / n1) % n1];
            l2[4 * ents + m] = l2[ents + m] * mp.d[2].hgL[m / nn];
        }
    }
    ctx->tr_len = (long long)ctx->ne * (ctx->dim == 3 ? 12 * nn : (ctx->dim == 2 ? 8 * n1 : 4));
    // a partitioned mesh keeps one ghost row of element traces below and
    // above its own rows (filled from the neighbours' exchanged traces)
    const long long ghost = (mp.halo_lo || mp.halo_hi) ? (long long)ctx->nx * 8 * n1 : 0;
    ctx->tr_len += 2 * ghost;
    ctx->red_len = 1024;
    int st;
    if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_mats, tables.size() * sizeof(double)), "alloc")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_lam2, l2.size() * sizeof(double)), "alloc")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_state, (size_t)B_COUNT * ctx->ndof * sizeof(double)), "alloc")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_tr_alloc, (size_t)2 * ctx->tr_len * sizeof(double)), "alloc")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_red, (size_t)(ctx->red_len + 1) * sizeof(double)), "alloc")) ||
        (st = gdg_cuda_check(ctx, cudaMallocHost((void **)&ctx->h_red, 8 * sizeof(double)), "alloc")) ||
        (ctx->dim == 2 && (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_sync, sync_words(ctx->ne) * sizeof(unsigned)), "alloc"))))
        return st;
    if (ghost && !mp.parity)
        return gdg_set_err(ctx, GDG_EUNSUPPORTED, "partitioned meshes need the parity stage kernel (clean even/odd modes)");
    ctx->d_tr = ctx->d_tr_alloc + ghost;
    if (ghost &&
        (st = gdg_cuda_check(ctx, cudaMemset(ctx->d_tr_alloc, 0, (size_t)2 * ctx->tr_len * sizeof(double)), "clear traces")))
        return st;
    if (ghost) {   // partitioned meshes run the one-line stage kernel, stage by stage
        mp.split = 0;
        ctx->stage_tuned = true;
    }
    if ((st = gdg_cuda_check(ctx, cudaMemcpy(ctx->d_mats, tables.data(), tables.size() * sizeof(double), cudaMemcpyHostToDevice), "upload")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpy(ctx->d_lam2, l2.data(), l2.size() * sizeof(double), cudaMemcpyHostToDevice), "upload")))
        return st;
    set_smem_limits();
    return gdg_cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "stream");
}

void gdg_const_free(gdg_ctx *ctx) {
    if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
    ctx->graph.exec = nullptr;
    cudaFree(ctx->d_mats);
    cudaFree(ctx->d_lam2);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_tr_alloc);
    cudaFree(ctx->d_red);
    cudaFree(ctx->d_sync);
    ctx->d_sync = nullptr;
    if (ctx->h_red) cudaFreeHost(ctx->h_red);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    ctx->d_mats = ctx->d_lam2 = ctx->d_state = ctx->d_tr = ctx->d_tr_alloc = ctx->d_red = ctx->h_red = nullptr;
    ctx->cap_stream = nullptr;
}

int gdg_const_rhs(gdg_ctx *ctx, const double *u, const double *v, double *du, double *dv, cudaStream_t s) {
    // modal state of (u, v), its traces, k = f(Y) in modal form, back to nodal
    launch_sep(ctx, u, v, buf(ctx, B_XU), buf(ctx, B_XV), T_P, nullptr, -1, s);
    launch_traces(ctx, buf(ctx, B_XU), buf(ctx, B_XV), ctx->d_tr, s);
    if (has_halo(ctx)) {
        if (!ctx->halo_fn) return gdg_set_err(ctx, GDG_EINVAL, "gdg_rhs: halo sides need gdg_set_halo first");
        const int st = halo_exchange(ctx, ctx->d_tr, s);
        if (st) return st;
    }
    StageBufs b{};
    b.yU = buf(ctx, B_XU); b.yV = buf(ctx, B_XV);
    b.oU = buf(ctx, B_KU); b.oV = buf(ctx, B_KV);
    b.trin = ctx->d_tr; b.lam2 = ctx->d_lam2;
    launch_stage(ctx, M_RHS, b, 0.0, 0.0, s);
    launch_sep(ctx, buf(ctx, B_KU), buf(ctx, B_KV), du, dv, T_PSI, nullptr, -1, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_rhs launch");
}

int gdg_const_mass_solve(gdg_ctx *ctx, int which, const double *b, double *x, cudaStream_t s) {
    // x = Psi D Psi^T b with D = I (M^-1) or D = Lambda^+ (constrained S solve)
    const int ents = (int)(ctx->ndof / ctx->ne);
    const double *D = which == GDG_OP_M ? nullptr : ctx->d_lam2 + ents;
    launch_sep(ctx, b, nullptr, x, nullptr, T_PSIT, D, T_PSI, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_mass_solve launch");
}

// Pick the stage kernel of a 2-D parity context by timing: one line per
// thread (k_stage2p), two (k_stage2h), one per line and field (k_stage2f),
// or the persistent step (k_step2r) where its grid fits the GPU at once.
// All compute bit-identical results.  The per-stage trials write only
// buffers the step then rewrites; the persistent trials advance the modal
// state, which is then rebuilt from (u, v).
int tune_stage_kernel(gdg_ctx *ctx, double dt, cudaStream_t s, const double *u, const double *v) {
    ModalParams &mp = ctx->mp;
    ctx->stage_tuned = true;
    if (ctx->dim != 2 || !mp.parity) return GDG_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    StageBufs b{};
    b.nU = buf(ctx, B_NU); b.nV = buf(ctx, B_NV);
    b.aU = buf(ctx, B_AU); b.aV = buf(ctx, B_AV);
    b.lam2 = ctx->d_lam2;
    b.yU = b.nU; b.yV = b.nV; b.oU = buf(ctx, B_XU); b.oV = buf(ctx, B_XV);
    b.trin = ctx->d_tr; b.trout = ctx->d_tr + ctx->tr_len;
    // best of 5 repetitions of 4 launches each (stage-1 and stage-2/3 kinds
    // alternately; these write only X, the accumulator and the second trace
    // buffer, which the step's first stage overwrites); another variant must
    // beat the one-line kernel by 1 % to replace it
    float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int split = 0; split < 3; ++split) {
        mp.split = split;
        for (int rep = 0; rep < 5; ++rep) {
            float ms = 0.f;
            cudaEventRecord(e0, s);
            for (int i = 0; i < 4; ++i)
                launch_stage_raw(ctx, (i & 1) ? M_S23 : M_S1, b, (i & 1) ? dt / 3.0 : dt / 6.0, 0.5 * dt, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            best[split] = std::min(best[split], ms);
        }
    }
    if (persist_fits(ctx)) {   // one step = 4 stages per trial launch
        mp.split = 3;
        for (int rep = 0; rep < 5; ++rep) {
            float ms = 0.f;
            cudaEventRecord(e0, s);
            launch_persist(ctx, dt, 1, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            best[3] = std::min(best[3], ms);
        }
        if (persist_failed(ctx, s)) best[3] = 1e30f;
        launch_sep(ctx, u, v, buf(ctx, B_NU), buf(ctx, B_NV), T_P, nullptr, -1, s);
        launch_traces(ctx, buf(ctx, B_NU), buf(ctx, B_NV), ctx->d_tr, s);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int pick = 0;
    for (int k = 1; k < 4; ++k)
        if (best[k] < 0.99f * best[0] && best[k] < best[pick]) pick = k;
    mp.split = pick;
    return gdg_cuda_check(ctx, cudaGetLastError(), "stage kernel choice");
}

extern "C" int gdg_set_wait_limit(gdg_ctx *ctx, double seconds) {
    if (!ctx || !(seconds > 0.0) || !std::isfinite(seconds)) return GDG_EINVAL;
    const double ns = seconds * 1e9;
    ctx->wait_limit_ns = ns < 1.0 ? 1ull : (ns > 1e18 ? 1000000000000000000ull : (unsigned long long)ns);
    return GDG_OK;
}

extern "C" int gdg_set_stage_variant(gdg_ctx *ctx, int variant) {
    if (!ctx || ctx->var || ctx->dim != 2 || !ctx->mp.parity || variant < -1 || variant > 3) return GDG_EINVAL;
    if (has_halo(ctx) && variant != 0)
        return gdg_set_err(ctx, GDG_EUNSUPPORTED, "partitioned meshes run the one-line stage kernel (variant 0)");
    if (variant == 3 && !persist_fits(ctx))
        return gdg_set_err(ctx, GDG_EUNSUPPORTED, "persistent step: the grid does not fit the GPU at once");
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    ctx->stage_tuned = variant >= 0;
    ctx->mp.split = variant > 0 ? variant : 0;
    return GDG_OK;
}

extern "C" int gdg_get_stage_variant(const gdg_ctx *ctx, int *variant) {
    if (!ctx || !variant || ctx->var || ctx->dim != 2 || !ctx->mp.parity) return GDG_EINVAL;
    *variant = ctx->stage_tuned ? ctx->mp.split : -1;
    return GDG_OK;
}

int gdg_const_step(gdg_ctx *ctx, double *u, double *v, double dt, int nsteps, cudaStream_t s) {
    int st;
    if (ctx->pb.route == GDG_ROUTE_NODAL) return step_nodal(ctx, u, v, dt, nsteps, s);
    launch_sep(ctx, u, v, buf(ctx, B_NU), buf(ctx, B_NV), T_P, nullptr, -1, s);
    launch_traces(ctx, buf(ctx, B_NU), buf(ctx, B_NV), ctx->d_tr, s);
    if ((st = gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step prologue"))) return st;
    if (has_halo(ctx)) {   // partitioned mesh: stages launched one by one, exchanges between them
        if (!ctx->halo_fn) return gdg_set_err(ctx, GDG_EINVAL, "gdg_step: halo sides need gdg_set_halo first");
        if ((st = halo_exchange(ctx, ctx->d_tr, s))) return st;
        for (int i = 0; i < nsteps; ++i)
            if ((st = rk4_step_halo(ctx, dt, i + 1 == nsteps, s))) return st;
        launch_sep(ctx, buf(ctx, B_NU), buf(ctx, B_NV), u, v, T_PSI, nullptr, -1, s);
        return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step (partitioned mesh)");
    }
    if (!ctx->stage_tuned && (st = tune_stage_kernel(ctx, dt, s, u, v))) return st;
    if (ctx->dim == 2 && ctx->mp.parity && ctx->mp.split == 3) {
        if (nsteps > 0) launch_persist(ctx, dt, nsteps, s);
        launch_sep(ctx, buf(ctx, B_NU), buf(ctx, B_NV), u, v, T_PSI, nullptr, -1, s);
        if ((st = gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step (persistent)"))) return st;
        if (nsteps > 0 && persist_failed(ctx, s))
            return gdg_set_err(ctx, GDG_ETIMEOUT, "persistent step: a grid barrier gave up (wait limit)");
        return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step (persistent)");
    }
    // graph of G steps, replayed; the remainder is launched directly
    const int G = (nsteps >= 16 && !ctx->prof.on) ? 16 : 0;
    if (G) {
        GraphCache &gc = ctx->graph;
        if (!gc.exec || gc.dt != dt || gc.steps != G) {
            if (gc.exec) cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            cudaGraph_t g;
            if ((st = gdg_cuda_check(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "capture")))
                return st;
            for (int i = 0; i < G; ++i) enqueue_rk4_step(ctx, dt, ctx->cap_stream);
            if ((st = gdg_cuda_check(ctx, cudaStreamEndCapture(ctx->cap_stream, &g), "capture end"))) return st;
            st = gdg_cuda_check(ctx, cudaGraphInstantiate(&gc.exec, g, 0), "instantiate");
            cudaGraphDestroy(g);
            if (st) return st;
            gc.dt = dt;
            gc.steps = G;
        }
        for (int i = 0; i + G <= nsteps; i += G)
            if ((st = gdg_cuda_check(ctx, cudaGraphLaunch(gc.exec, s), "graph launch"))) return st;
    }
    const int rem = G ? nsteps % G : nsteps;
    for (int i = 0; i < rem; ++i) enqueue_rk4_step(ctx, dt, s);
    launch_sep(ctx, buf(ctx, B_NU), buf(ctx, B_NV), u, v, T_PSI, nullptr, -1, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step");
}

int gdg_const_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, cudaStream_t s) {
    launch_sep(ctx, u, v, buf(ctx, B_KU), buf(ctx, B_KV), T_P, nullptr, -1, s);
    const int blocks = 256;
    if (ctx->dim == 3) {
        gdg3_energy_partial(ctx->n1, ctx->ne, buf(ctx, B_KU), buf(ctx, B_KV), ctx->d_lam2, ctx->d_red, blocks, s);
    } else if (ctx->dim == 2) {
        switch (ctx->n1) {
#define X(n) case n: k_energy_partial<n, 2><<<blocks, 256, 0, s>>>(ctx->ne, buf(ctx, B_KU), buf(ctx, B_KV), ctx->d_lam2, ctx->d_red); break;
            GDG_N1_CASES(X)
#undef X
        }
    } else {
        switch (ctx->n1) {
#define X(n) case n: k_energy_partial<n, 1><<<blocks, 256, 0, s>>>(ctx->ne, buf(ctx, B_KU), buf(ctx, B_KV), ctx->d_lam2, ctx->d_red); break;
            GDG_N1_CASES(X)
#undef X
        }
    }
    k_sum_partials<<<1, 256, 0, s>>>(blocks, ctx->d_red, ctx->d_red + ctx->red_len);
    int st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(ctx->h_red, ctx->d_red + ctx->red_len, sizeof(double), cudaMemcpyDeviceToHost, s), "energy d2h")))
        return st;
    if ((st = gdg_cuda_check(ctx, cudaStreamSynchronize(s), "energy sync"))) return st;
    *E = ctx->h_red[0];
    return GDG_OK;
}

StepBuffers gdg_const_buffers(gdg_ctx *ctx) {
    StepBuffers b;
    b.nU = buf(ctx, B_NU); b.nV = buf(ctx, B_NV); b.aU = buf(ctx, B_AU); b.aV = buf(ctx, B_AV);
    b.xU = buf(ctx, B_XU); b.xV = buf(ctx, B_XV); b.yU = buf(ctx, B_YU); b.yV = buf(ctx, B_YV);
    b.tr0 = ctx->d_tr; b.tr1 = ctx->d_tr + ctx->tr_len;
    return b;
}

int gdg_const_enter(gdg_ctx *ctx, const double *u, const double *v, cudaStream_t s) {
    launch_sep(ctx, u, v, buf(ctx, B_NU), buf(ctx, B_NV), T_P, nullptr, -1, s);
    launch_traces(ctx, buf(ctx, B_NU), buf(ctx, B_NV), ctx->d_tr, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "enter");
}

int gdg_const_leave(gdg_ctx *ctx, double *u, double *v, cudaStream_t s) {
    launch_sep(ctx, buf(ctx, B_NU), buf(ctx, B_NV), u, v, T_PSI, nullptr, -1, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "leave");
}

// ------------------------------------------- allocation-free gdg_rhs ------
//
// gdg_rhs_static: the constant-coefficient gdg_rhs for callers that cannot
// allocate device memory.  It needs no context: the host builds the basis
// and the modal tables in fixed-size stack arrays, and every device-side
// intermediate (tables, the modal state, the modal derivative and the face
// traces) lives in one file-scope static device array.

namespace {

// 16 MiB of scratch per device, shared by every gdg_rhs_static call.
constexpr size_t kStaticScratchDoubles = (size_t)2 * 1024 * 1024;
static __device__ __align__(256) double g_rhs_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_rhs_scratch_addr[kMaxDevices];   // device address of g_rhs_scratch, per device

// Host-built tables of one gdg_rhs_static call, passed by value as a kernel
// parameter (6 n1^2 + 2 n1^2 doubles at n1 = 16: 16 KB, within the 32 KB
// parameter limit) and written into the static array by k_put_tables.
struct StaticTables {
    double v[8 * GDG_MAXN1 * GDG_MAXN1];
};
static_assert(sizeof(StaticTables) <= 16384, "parameter block");

__global__ void k_put_tables(const __grid_constant__ StaticTables t, int n, double *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = t.v[i];
}

// Gauss-Legendre on [0,1], fixed-size arrays (Newton on the Legendre recurrence)
void gl_fixed(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), pn = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p0 = 1.0; p1 = z; }
            pn = p1;
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p0 = 1.0; p1 = z; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = 0.5 * (1.0 - z);
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[i] = w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Reference 1-D basis data without heap allocation: M, S (Section 3.1),
// one-sided face slopes, and the modified basis Psi, lambda (Section 3.2).
bool basis_fixed(int p, int N, double *M, double *S, double *dL, double *dR, double *Psi, double *lam) {
    const int n1 = N + 1;
    double gx[GDG_MAXN1], gw[GDG_MAXN1], phi[GDG_MAXN1], dphi[GDG_MAXN1];
    gl_fixed(p + 1, gx, gw);
    for (int i = 0; i < n1 * n1; ++i) { M[i] = 0.0; S[i] = 0.0; }
    for (int k = 0; k < N; ++k)
        for (int g = 0; g <= p; ++g) {
            gdg_eval_basis(p, N, (k + gx[g]) / N, k, phi, dphi);
            const double w = gw[g] / N;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) {
                    M[a * n1 + b] += w * phi[a] * phi[b];
                    S[a * n1 + b] += w * dphi[a] * dphi[b];
                }
        }
    gdg_eval_basis(p, N, 0.0, 0, phi, dL);
    gdg_eval_basis(p, N, 1.0, N - 1, phi, dR);
    // S psi = lambda M psi: M = L L^T, Jacobi on L^-1 S L^-T
    double L[GDG_MAXN1 * GDG_MAXN1] = {0}, Li[GDG_MAXN1 * GDG_MAXN1] = {0};
    double C[GDG_MAXN1 * GDG_MAXN1], V[GDG_MAXN1 * GDG_MAXN1];
    for (int j = 0; j < n1; ++j) {
        double d = M[j * n1 + j];
        for (int k = 0; k < j; ++k) d -= L[j * n1 + k] * L[j * n1 + k];
        if (!(d > 0.0)) return false;
        L[j * n1 + j] = std::sqrt(d);
        for (int i = j + 1; i < n1; ++i) {
            double s = M[i * n1 + j];
            for (int k = 0; k < j; ++k) s -= L[i * n1 + k] * L[j * n1 + k];
            L[i * n1 + j] = s / L[j * n1 + j];
        }
    }
    for (int c = 0; c < n1; ++c)
        for (int i = 0; i < n1; ++i) {
            double s = i == c ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * n1 + k] * Li[k * n1 + c];
            Li[i * n1 + c] = s / L[i * n1 + i];
        }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n1; ++j) {
            double s = 0.0;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) s += Li[i * n1 + a] * S[a * n1 + b] * Li[j * n1 + b];
            C[i * n1 + j] = s;
        }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < i; ++j) C[i * n1 + j] = C[j * n1 + i] = 0.5 * (C[i * n1 + j] + C[j * n1 + i]);
    for (int i = 0; i < n1 * n1; ++i) V[i] = (i % (n1 + 1)) == 0 ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n1 * n1; ++i) {
            tot += C[i] * C[i];
            if (i % (n1 + 1)) off += C[i] * C[i];
        }
        if (off <= 1e-30 * tot) break;
        for (int a = 0; a < n1 - 1; ++a)
            for (int b = a + 1; b < n1; ++b) {
                const double cab = C[a * n1 + b];
                if (std::fabs(cab) < 1e-300) continue;
                const double th = (C[b * n1 + b] - C[a * n1 + a]) / (2.0 * cab);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n1; ++k) {
                    const double x = C[k * n1 + a], y = C[k * n1 + b];
                    C[k * n1 + a] = c * x - s * y;
                    C[k * n1 + b] = s * x + c * y;
                }
                for (int k = 0; k < n1; ++k) {
                    const double x = C[a * n1 + k], y = C[b * n1 + k];
                    C[a * n1 + k] = c * x - s * y;
                    C[b * n1 + k] = s * x + c * y;
                }
                for (int k = 0; k < n1; ++k) {
                    const double x = V[k * n1 + a], y = V[k * n1 + b];
                    V[k * n1 + a] = c * x - s * y;
                    V[k * n1 + b] = s * x + c * y;
                }
            }
    }
    int order[GDG_MAXN1];
    for (int i = 0; i < n1; ++i) order[i] = i;
    for (int i = 1; i < n1; ++i)
        for (int j = i; j > 0 && C[order[j] * (n1 + 1)] < C[order[j - 1] * (n1 + 1)]; --j) {
            const int tmp = order[j];
            order[j] = order[j - 1];
            order[j - 1] = tmp;
        }
    for (int k = 0; k < n1; ++k) {
        lam[k] = C[order[k] * (n1 + 1)];
        for (int i = 0; i < n1; ++i) {
            double s = 0.0;
            for (int a = 0; a < n1; ++a) s += Li[a * n1 + i] * V[a * n1 + order[k]];
            Psi[i * n1 + k] = s;
        }
    }
    // exact constant mode, then M-orthonormalise the others
    double oMo = 0.0;
    for (int i = 0; i < n1 * n1; ++i) oMo += M[i];
    lam[0] = 0.0;
    for (int i = 0; i < n1; ++i) Psi[i * n1] = 1.0 / std::sqrt(oMo);
    for (int k = 1; k < n1; ++k) {
        for (int j = 0; j <= k; ++j) {
            double c = 0.0;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) c += Psi[a * n1 + j] * M[a * n1 + b] * Psi[b * n1 + k];
            if (j < k) {
                for (int i = 0; i < n1; ++i) Psi[i * n1 + k] -= c * Psi[i * n1 + j];
            } else {
                for (int i = 0; i < n1; ++i) Psi[i * n1 + k] /= std::sqrt(c);
            }
        }
    }
    return true;
}

}  // namespace

extern "C" int gdg_rhs_static(const gdg_problem *pb, const double *u, const double *v, double *du, double *dv,
                              void *stream) {
    if (!pb || !u || !v || !du || !dv) return GDG_EINVAL;
    if (du == u || du == v || dv == u || dv == v) return GDG_EINVAL;
    if (pb->dim != 1 && pb->dim != 2) return GDG_EINVAL;
    if (pb->coef != GDG_COEF_CONST || !(pb->c2 > 0.0)) return GDG_EINVAL;
    if (pb->rows[0] || pb->rows[1]) return GDG_EUNSUPPORTED;   // whole meshes only
    if (pb->p < 1 || pb->p % 2 == 0 || pb->N < pb->p) return GDG_EINVAL;
    if (pb->N + 1 > GDG_MAXN1) return GDG_EUNSUPPORTED;
    if (pb->flux != GDG_FLUX_CENTRAL && pb->flux != GDG_FLUX_UPWIND && pb->flux != GDG_FLUX_ALTERNATING)
        return GDG_EINVAL;
    for (int d = 0; d < pb->dim; ++d) {
        if (pb->n_elem[d] < 1 || !(pb->hi[d] > pb->lo[d])) return GDG_EINVAL;
        if (pb->bc[d] != GDG_BC_DIRICHLET && pb->bc[d] != GDG_BC_PERIODIC) return GDG_EINVAL;
    }
    const int n1 = pb->N + 1, nn = n1 * n1, dim = pb->dim;
    const int nx = pb->n_elem[0], ny = dim == 2 ? pb->n_elem[1] : 1;
    const long long ne = (long long)nx * ny;
    const int ents = dim == 2 ? nn : n1;
    const long long ndof = ne * ents;
    const long long tr_len = ne * (dim == 2 ? 8 * n1 : 4);
    const long long ntab = 6LL * nn + 2LL * ents;
    // scratch: tables | modal state (2 fields) | modal derivative (2 fields) | traces
    const long long need = ntab + 4 * ndof + tr_len;
    if (need > (long long)kStaticScratchDoubles) {
        std::fprintf(stderr,
                     "gdg_rhs_static: the problem needs %lld doubles of scratch but the static buffer holds %zu "
                     "(16 MiB); use gdg_rhs with a context for larger meshes\n",
                     need, kStaticScratchDoubles);
        return GDG_EUNSUPPORTED;
    }
    // set-up, once per device (with that device current): device address of the array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GDG_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GDG_EUNSUPPORTED;
    if (!g_rhs_scratch_addr[dev]) {
        void *addr = nullptr;
        if (cudaGetSymbolAddress(&addr, g_rhs_scratch) != cudaSuccess || !addr) return GDG_ECUDA;
        g_rhs_scratch_addr[dev] = static_cast<double *>(addr);
    }
    double *base = g_rhs_scratch_addr[dev];

    // host tables in fixed-size arrays
    double Mh[GDG_MAXN1 * GDG_MAXN1], Sh[GDG_MAXN1 * GDG_MAXN1], dL[GDG_MAXN1], dR[GDG_MAXN1];
    double Psih[GDG_MAXN1 * GDG_MAXN1], lamh[GDG_MAXN1];
    if (!basis_fixed(pb->p, pb->N, Mh, Sh, dL, dR, Psih, lamh)) return GDG_EINVAL;
    static_assert(GDG_MAXN1 <= 16, "table size");
    double tab[6 * 256 + 2 * 256] = {0};
    double lam[2][GDG_MAXN1];
    ModalParams mp;
    std::memset(&mp, 0, sizeof(mp));
    mp.nx = nx;
    mp.ny = ny;
    mp.ne = (int)ne;
    mp.per_x = pb->bc[0] == GDG_BC_PERIODIC;
    mp.per_y = dim == 2 && pb->bc[1] == GDG_BC_PERIODIC;
    mp.c2 = pb->c2;
    if (pb->flux == GDG_FLUX_UPWIND) {
        const double xi = pb->xi > 0 ? pb->xi : std::sqrt(pb->c2);
        mp.beta = 0.5 * xi;
        mp.tau = 0.5 / xi;
    }
    mp.beta2 = 2.0 * mp.beta;
    mp.tau2 = 2.0 * mp.tau;
    mp.alt = pb->flux == GDG_FLUX_ALTERNATING;
    mp.parity = 0;     // generic stage kernel
    mp.epb = dim == 2 ? 16 : 1;
    for (int d = 0; d < dim; ++d) {
        const double H = (pb->hi[d] - pb->lo[d]) / pb->n_elem[d], sq = std::sqrt(H);
        double *P = tab + ((size_t)d * 3 + T_P) * nn, *Ps = tab + ((size_t)d * 3 + T_PSI) * nn;
        double *PT = tab + ((size_t)d * 3 + T_PSIT) * nn;
        for (int k = 0; k < n1; ++k) {
            lam[d][k] = lamh[k] / (H * H);
            for (int i = 0; i < n1; ++i) {
                double s = 0.0;
                for (int a = 0; a < n1; ++a) s += (Psih[a * n1 + k] / sq) * (H * Mh[a * n1 + i]);
                P[k * n1 + i] = s;
                Ps[i * n1 + k] = Psih[i * n1 + k] / sq;
                PT[k * n1 + i] = Psih[i * n1 + k] / sq;
            }
        }
        ModalDir &md = mp.d[d];
        for (int k = 0; k < n1; ++k) {
            md.eL[k] = Psih[k] / sq;
            md.eR[k] = Psih[(n1 - 1) * n1 + k] / sq;
            double gl = 0.0, gr = 0.0;
            for (int i = 0; i < n1; ++i) {
                gl += (Psih[i * n1 + k] / sq) * (-dL[i] / H);
                gr += (Psih[i * n1 + k] / sq) * (dR[i] / H);
            }
            md.gL[k] = gl;
            md.gR[k] = gr;
            md.lam[k] = lam[d][k];
            md.hgL[k] = 0.5 * gl;
            md.ceL[k] = 0.5 * pb->c2 * md.eL[k];
        }
    }
    double *l2 = tab + 6 * nn;
    for (int m = 0; m < ents; ++m) {
        const double Lm = dim == 2 ? lam[0][m % n1] + lam[1][m / n1] : lam[0][m];
        l2[m] = -pb->c2 * Lm;
        l2[ents + m] = m == 0 ? 0.0 : 1.0 / Lm;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the tables travel by value in the launch's parameter block (16 KB at
    // most): no copy from host memory, so the call never waits for the host
    StaticTables st;
    std::memcpy(st.v, tab, (size_t)ntab * sizeof(double));
    k_put_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, s>>>(st, (int)ntab, base);

    // a context on the stack holding only what the launch helpers read
    gdg_ctx c;
    c.dim = dim;
    c.nx = nx;
    c.ny = ny;
    c.N = pb->N;
    c.n1 = n1;
    c.p = pb->p;
    c.ne = (int)ne;
    c.ndof = ndof;
    c.pb = *pb;
    c.mp = mp;
    c.d_mats = base;
    c.d_lam2 = base + 6 * nn;
    double *Yu = base + ntab, *Yv = Yu + ndof, *Ku = Yv + ndof, *Kv = Ku + ndof, *tr = Kv + ndof;
    set_smem_limits();
    launch_sep(&c, u, v, Yu, Yv, T_P, nullptr, -1, s);
    launch_traces(&c, Yu, Yv, tr, s);
    StageBufs b{};
    b.yU = Yu; b.yV = Yv; b.oU = Ku; b.oV = Kv; b.trin = tr; b.lam2 = c.d_lam2;
    launch_stage(&c, M_RHS, b, 0.0, 0.0, s);
    launch_sep(&c, Ku, Kv, du, dv, T_PSI, nullptr, -1, s);
    c.d_mats = c.d_lam2 = nullptr;   // not owned
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}

// ---------------------------------------------------- index checks ------

// this translation unit's check slot (gdg_checks.cuh)
GDG_CHECKS_READER(gdg_checks_read_const)

namespace {
__global__ void k_check_selftest(long long index, long long bound) {
#if GDG_CHECKS
    long long i = index;
    GDG_CHECK_INDEX(i, 0, bound, GDG_SITE_SELFTEST, 0);
#else
    (void)index;
    (void)bound;
#endif
}
}  // namespace

extern "C" int gdg_check_selftest(long long index, long long bound, void *stream) {
    if (!GDG_CHECKS) return GDG_EUNSUPPORTED;
    k_check_selftest<<<1, 1, 0, (cudaStream_t)stream>>>(index, bound);
    return cudaGetLastError() == cudaSuccess ? GDG_OK : GDG_ECUDA;
}
