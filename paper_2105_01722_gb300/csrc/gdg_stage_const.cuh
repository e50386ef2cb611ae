// Device code of the constant-coefficient modal stage shared by the
// per-problem kernels (gdg_const.cu) and the batched kernels (gdg_batch.cu).
#pragma once

#include "gdg_internal.h"

namespace {


struct StageBufs {
    const double *yU, *yV;   // stage input (modal)
    double *nU, *nV;         // y_n
    double *aU, *aV;         // RK accumulator
    double *oU, *oV;         // next stage input, or k (M_RHS)
    const double *trin;      // traces of the stage input
    double *trout;           // traces of the next stage input
    const double *lam2;      // [2][n1^d] : -c2 * lambda, 1/lambda (0 on mode 0)
};

// trace buffer index: 2-D [e][face 0..3 = xm,xp,ym,yp][field 0 = v, 1 = n.grad u][N1]
template <int N1>
__device__ __forceinline__ size_t tix2(int e, int face, int fld, int i) {
    return (((size_t)e * 4 + face) * 2 + fld) * N1 + i;
}
// 1-D: [e][face 0..1][field]
__device__ __forceinline__ size_t tix1(int e, int face, int fld) {
    return ((size_t)e * 2 + face) * 2 + fld;
}

// Fluxes of Section 2.2.1 in normal form (alpha = 1/2):
//   v* = (vi + vo)/2 - beta (di + do),  q* = (di - do)/2 - tau (vi - vo)
// returns g = v* - vi and c2 * q*.
__device__ __forceinline__ void flux(double vi, double di, double vo, double dO, double beta,
                                     double tau, double c2, double &g, double &q) {
    g = 0.5 * (vo - vi) - beta * (di + dO);
    q = c2 * (0.5 * (di - dO) - tau * (vi - vo));
}

// Body of the parity stage kernel for element tile `etile` (blockDim.x / N1
// elements per block).  Parity version of the generic stage: the GD element is symmetric under r -> 1-r,
// so every modified-basis vector is even or odd: Psi[N-i][k] = s_k Psi[i][k].
// With the NE = (N1+1)/2 even modes stored first, eR = s eL and gR = s gL:
// both face traces of a line come from one even/odd split dot, and each
// lift is one FMA per entry.  Fluxes carry a factor 2 (g2 = 2(v* - v_in),
// q2 = 2 q*) that is folded into the lift vectors hgL = gL/2, ceL = c^2 eL/2.
template <int N1, int MODE>
__device__ __forceinline__ void stage2p_body(const ModalParams &mp, const StageBufs &b, double cA, double cY,
                                             int etile, double *smem) {
    constexpr int NE = (N1 + 1) / 2;
    const int epb = blockDim.x / N1;
    const int t = threadIdx.x;
    const int le = t / N1, l = t - le * N1;
    const int e = etile * epb + le;
    const bool valid = le < epb && e < mp.ne;
    double *fy = smem + le * (4 * N1);   // per column: GA, GB, QA, QB of the y faces
    double *tile = smem + epb * 4 * N1 + le * (2 * N1 * (N1 + 1));
    const int nx = mp.nx, ny = mp.ny;
    const int ex = valid ? e % nx : 0, ey = valid ? e / nx : 0;
    const double b2 = mp.beta2, t2 = mp.tau2;
    const size_t row = ((size_t)(valid ? e : 0) * N1 + l) * N1;

    // issue every row load of this stage before the barrier so their latency
    // overlaps the flux work (a few warps per SM only at small element counts)
    double Ru[N1], Rv[N1], Nu[N1], Nv[N1], Au[N1], Av[N1];
    if (valid) {
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            Ru[k] = b.yU[row + k];
            Rv[k] = b.yV[row + k];
            if (MODE == M_S23 || MODE == M_S4) {
                Nu[k] = b.nU[row + k];
                Nv[k] = b.nV[row + k];
                Au[k] = b.aU[row + k];
                Av[k] = b.aV[row + k];
            }
        }
    }

    double GA = 0, GB = 0, QA = 0, QB = 0;
    if (valid) {
        const double *T = b.trin;
        double vi, di, vo, dO, d1, g2m, q2m, g2p, q2p;
        int en, f;
        // x faces, transverse mode l
        vi = T[tix2<N1>(e, 0, 0, l)]; di = T[tix2<N1>(e, 0, 1, l)];
        en = ex - 1;
        if (en < 0 && mp.per_x) en += nx;
        if (en >= 0) { f = ey * nx + en; vo = T[tix2<N1>(f, 1, 0, l)]; dO = T[tix2<N1>(f, 1, 1, l)]; }
        else { vo = -vi; dO = -di; }
        d1 = vo - vi;
        g2m = fma(-b2, di + dO, d1);
        q2m = fma(t2, d1, di - dO);
        vi = T[tix2<N1>(e, 1, 0, l)]; di = T[tix2<N1>(e, 1, 1, l)];
        en = ex + 1;
        if (en >= nx && mp.per_x) en -= nx;
        if (en < nx) { f = ey * nx + en; vo = T[tix2<N1>(f, 0, 0, l)]; dO = T[tix2<N1>(f, 0, 1, l)]; }
        else { vo = -vi; dO = -di; }
        d1 = vo - vi;
        g2p = fma(-b2, di + dO, d1);
        q2p = fma(t2, d1, di - dO);
        GA = g2m + g2p; GB = g2m - g2p; QA = q2m + q2p; QB = q2m - q2p;
        // y faces, transverse mode k = l
        vi = T[tix2<N1>(e, 2, 0, l)]; di = T[tix2<N1>(e, 2, 1, l)];
        en = ey - 1;
        if (en < 0 && mp.per_y) en += ny;
        if (en >= 0) { f = en * nx + ex; vo = T[tix2<N1>(f, 3, 0, l)]; dO = T[tix2<N1>(f, 3, 1, l)]; }
        else { vo = -vi; dO = -di; }
        d1 = vo - vi;
        g2m = fma(-b2, di + dO, d1);
        q2m = fma(t2, d1, di - dO);
        vi = T[tix2<N1>(e, 3, 0, l)]; di = T[tix2<N1>(e, 3, 1, l)];
        en = ey + 1;
        if (en >= ny && mp.per_y) en -= ny;
        if (en < ny) { f = en * nx + ex; vo = T[tix2<N1>(f, 2, 0, l)]; dO = T[tix2<N1>(f, 2, 1, l)]; }
        else { vo = -vi; dO = -di; }
        d1 = vo - vi;
        g2p = fma(-b2, di + dO, d1);
        q2p = fma(t2, d1, di - dO);
        fy[l] = g2m + g2p; fy[N1 + l] = g2m - g2p;
        fy[2 * N1 + l] = q2m + q2p; fy[3 * N1 + l] = q2m - q2p;
    }
    __syncthreads();

    if (valid) {
        const double *L0 = b.lam2 + l * N1;
        const double *L1 = b.lam2 + N1 * N1 + l * N1;
        const double hgy = mp.d[1].hgL[l], cey = mp.d[1].ceL[l];
        const double *FG = fy + (l < NE ? 0 : N1);
        const double *FQ = fy + (l < NE ? 2 * N1 : 3 * N1);
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double Yu = Ru[k], Yv = Rv[k];
            const double xg = k < NE ? GA : GB, xq = k < NE ? QA : QB;
            const double ru = fma(mp.d[0].hgL[k], xg, hgy * FG[k]);
            const double rv = fma(L0[k], Yu, fma(mp.d[0].ceL[k], xq, cey * FQ[k]));
            const double ku = fma(L1[k], ru, Yv);
            const double kv = rv;
            if (MODE == M_RHS) {
                b.oU[row + k] = ku;
                b.oV[row + k] = kv;
            } else if (MODE == M_S1) {
                b.aU[row + k] = cA * ku;
                b.aV[row + k] = cA * kv;
                Ru[k] = fma(cY, ku, Yu);
                Rv[k] = fma(cY, kv, Yv);
            } else if (MODE == M_S23) {
                b.aU[row + k] = fma(cA, ku, Au[k]);
                b.aV[row + k] = fma(cA, kv, Av[k]);
                Ru[k] = fma(cY, ku, Nu[k]);
                Rv[k] = fma(cY, kv, Nv[k]);
            } else {
                Ru[k] = fma(cA, ku, Nu[k] + Au[k]);
                Rv[k] = fma(cA, kv, Nv[k] + Av[k]);
            }
        }
        if (MODE != M_RHS) {
            double *dU = (MODE == M_S4) ? b.nU : b.oU;
            double *dV = (MODE == M_S4) ? b.nV : b.oV;
#pragma unroll
            for (int k = 0; k < N1; ++k) { dU[row + k] = Ru[k]; dV[row + k] = Rv[k]; }
        }
    }
    if (MODE == M_RHS) return;

    if (valid) {
        double ve = 0, vo_ = 0, de = 0, do_ = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            if (k < NE) { ve = fma(mp.d[0].eL[k], Rv[k], ve); de = fma(mp.d[0].gL[k], Ru[k], de); }
            else { vo_ = fma(mp.d[0].eL[k], Rv[k], vo_); do_ = fma(mp.d[0].gL[k], Ru[k], do_); }
            tile[l * (N1 + 1) + k] = Ru[k];
            tile[N1 * (N1 + 1) + l * (N1 + 1) + k] = Rv[k];
        }
        b.trout[tix2<N1>(e, 0, 0, l)] = ve + vo_;
        b.trout[tix2<N1>(e, 0, 1, l)] = de + do_;
        b.trout[tix2<N1>(e, 1, 0, l)] = ve - vo_;
        b.trout[tix2<N1>(e, 1, 1, l)] = de - do_;
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
        b.trout[tix2<N1>(e, 2, 0, k)] = ve + vo_;
        b.trout[tix2<N1>(e, 2, 1, k)] = de + do_;
        b.trout[tix2<N1>(e, 3, 0, k)] = ve - vo_;
        b.trout[tix2<N1>(e, 3, 1, k)] = de - do_;
    }
}

}  // namespace
